"""FP64 reference of the bed / flying classification and of the extraction
of impact and rebound events of saltating spheres (Sec. 4.3.1, steps 1-3).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module. The GPU product path never imports it.

Step 1 (bed and flying spheres). The bottom layer is the spheres whose
centre lies less than one diameter above the bottom, z < D (the paper's
vertical axis y is z here; the bottom is z = 0). Bed spheres are those of the
bottom layer and every sphere in contact (d < 2R) with a bed sphere, directly
or through other bed spheres; the rest fly. The paper finds them by sweeping
over all spheres until the bed count stops changing; this module sweeps the
same way. Reading: the bottom-layer spheres stay bed spheres in every sweep
(the listing, read literally, would drop a bottom sphere that touches no
other bed sphere, which the text's definition does not).

Steps 2-3 (saltation and events), per sphere and step, given the time t of
the state:
- a departure (bed -> flying) starts a flight at the current centre height;
- a flying sphere whose centre rises more than h_r above the height of its
  departure is saltating (h_r = D/2 in the paper); rolling spheres do not;
- an impact (flying -> bed) of a saltating sphere opens an impact event,
  recording the time and the velocities;
- the next departure closes it: a rebound if it comes within t_cir of the
  impact (t_cir = 5 T_c in the paper), an entrainment after enduring contact
  otherwise.
The first step seen sets the states and emits nothing.

Parity: pinned. The bed sets are checked against connected components of the
contact graph computed by scipy (a library routine) and against hand-built
chains, clusters and floating spheres; the events against hand-built
trajectories whose outcome follows from the definitions.
"""
from __future__ import annotations

import numpy as np

from . import pairs as _pairs


def bed_flags(d, x, R) -> np.ndarray:
    """1 for bed spheres, 0 for flying ones (uint8, n_p)."""
    x = np.asarray(x, dtype=np.float64)
    n_p = x.shape[1]
    nb = [[] for _ in range(n_p)]
    for p, q in _pairs(d, x, 2.0 * R):
        nb[p].append(int(q))
        nb[q].append(int(p))
    seed = x[2] < 2.0 * R
    bed = seed.copy()
    n_bed, n_temp = int(bed.sum()), -1
    while n_bed != n_temp:
        n_temp = n_bed
        n_bed = 0
        for i in range(n_p):
            if seed[i] or any(bed[j] for j in nb[i]):
                bed[i] = True
                n_bed += 1
            else:
                bed[i] = False
    return bed.astype(np.uint8)


class Tracker:
    """Per-sphere states of steps 2-3 and the events emitted so far."""

    def __init__(self, n_p: int):
        self.n_p = n_p
        self.started = False
        self.prev = np.zeros(n_p, dtype=np.uint8)
        self.dep_z = np.zeros(n_p)
        self.salt = np.zeros(n_p, dtype=bool)
        self.pend = np.zeros(n_p, dtype=bool)
        self.t_imp = np.zeros(n_p)
        self.u_imp = np.zeros((n_p, 3))
        self.om_imp = np.zeros((n_p, 3))

    def step(self, t, bed, x, u, om, h_r, t_cir):
        """Advances every sphere by one observed state; returns the events it
        closes, in sphere order, as dicts."""
        x = np.asarray(x, dtype=np.float64)
        u = np.asarray(u, dtype=np.float64)
        om = np.asarray(om, dtype=np.float64)
        events = []
        if not self.started:
            self.started = True
            self.prev[:] = bed
            self.dep_z[:] = x[2]
            self.salt[:] = False
            self.pend[:] = False
            return events
        for p in range(self.n_p):
            z = x[2, p]
            was, now = self.prev[p], bed[p]
            if not was and not now:
                if z - self.dep_z[p] > h_r:
                    self.salt[p] = True
            elif not was and now:
                if self.salt[p]:
                    self.pend[p] = True
                    self.t_imp[p] = t
                    self.u_imp[p] = u[:, p]
                    self.om_imp[p] = om[:, p]
                self.salt[p] = False
            elif was and not now:
                if self.pend[p]:
                    events.append(dict(particle=p, rebound=int(t - self.t_imp[p] < t_cir),
                                       t_impact=self.t_imp[p], t_departure=t,
                                       u_impact=self.u_imp[p].copy(),
                                       omega_impact=self.om_imp[p].copy(),
                                       u_departure=u[:, p].copy(),
                                       omega_departure=om[:, p].copy()))
                    self.pend[p] = False
                self.dep_z[p] = z
                self.salt[p] = False
            self.prev[p] = now
        return events
