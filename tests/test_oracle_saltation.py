"""CPU pins of the oracle's bed / flying classification and saltation events
(Sec. 4.3.1): hand-built chains, clusters and floating spheres, connected
components from scipy, and hand-built trajectories whose events follow from
the definitions."""
import numpy as np
import pytest

import oracle as O
from oracle import saltation as S
from paper_2108_01814_gb300 import workloads as W

R = 1.0
L = (20.0, 20.0, 40.0)


def _d(periodic=(1, 1, 0)):
    return O.dem_params(R, 2.65, 1.0, 0.9, 0.39, 0.4, 0.05, (0.0, 0.0, 0.0), L, periodic)


def test_chain_cluster_and_floating_sphere():
    gap = 2 * R * (1 - 1e-3)            # touching
    chain = [[5.0, 5.0, R + k * gap] for k in range(6)]          # from the bottom up
    lone = [[12.0, 12.0, 30.0]]                                  # floating
    cluster = [[15.0, 5.0, 20.0], [15.0 + gap, 5.0, 20.0], [15.0 + gap, 5.0 + gap, 20.0]]
    bottom = [[2.0, 15.0, 1.5]]                                  # bottom layer, alone
    x = np.array(chain + lone + cluster + bottom).T.copy()
    f = S.bed_flags(_d(), x, R)
    assert list(f) == [1] * 6 + [0] + [0, 0, 0] + [1]


def test_chain_across_the_periodic_face():
    gap = 2 * R * (1 - 1e-3)
    # a bottom sphere near x = 0, a sphere above the bottom layer touching it
    # across the periodic face, a sphere on top of that one, and a far one
    dz = 1.2
    ax = np.sqrt(gap * gap - dz * dz)
    x1 = L[0] - ax + 0.4
    x = np.array([[0.4, 10.0, R], [x1, 10.0, R + dz], [x1, 10.0, R + dz + gap],
                  [10.0, 10.0, 10.0]]).T.copy()
    assert x[2, 1] >= 2 * R               # not in the bottom layer
    assert list(S.bed_flags(_d(), x, R)) == [1, 1, 1, 0]
    # without the periodic axis the bridge is broken
    assert list(S.bed_flags(_d((0, 1, 0)), x, R)) == [1, 0, 0, 0]


def test_bed_equals_components_with_a_bottom_sphere():
    sp = pytest.importorskip("scipy.sparse")
    cg = pytest.importorskip("scipy.sparse.csgraph")
    w = W.small_bed(seed=3)
    d = O.dem_params(w.R, w.rho_p, w.rho_f, w.e_n, w.e_t, w.mu, w.T_c, w.g, w.L, w.periodic)
    f = S.bed_flags(d, w.x, w.R)
    pr = O.pairs(d, w.x, 2 * w.R)
    a = sp.coo_matrix((np.ones(len(pr)), (pr[:, 0], pr[:, 1])), shape=(w.n_p, w.n_p))
    _, lab = cg.connected_components(a, directed=False)
    seeds = np.unique(lab[w.x[2] < 2 * w.R])
    ref = np.isin(lab, seeds).astype(np.uint8)
    assert np.array_equal(f, ref)
    assert 0 < f.sum() < w.n_p            # a bed and some lofted spheres


def _track(seq, h_r=0.5, t_cir=1.0):
    # seq: list of (t, bed flags, z per sphere); velocities encode the time
    n = len(seq[0][1])
    tr = S.Tracker(n)
    out = []
    for t, bed, z in seq:
        x = np.zeros((3, n))
        x[2] = z
        u = np.full((3, n), t)
        om = np.full((3, n), -t)
        out += tr.step(t, np.array(bed, dtype=np.uint8), x, u, om, h_r, t_cir)
    return out


def test_events_from_hand_built_trajectories():
    # sphere 0 saltates and rebounds; 1 rolls (rises 0.3 < h_r); 2 saltates
    # and stays in the bed longer than t_cir; 3 starts flying and saltates
    seq = [
        (0.0, [1, 1, 1, 0], [1.0, 1.0, 1.0, 5.0]),
        (1.0, [0, 0, 0, 0], [1.2, 1.1, 1.2, 5.2]),    # departures of 0, 1, 2 at these heights
        (2.0, [0, 0, 0, 0], [2.0, 1.4, 1.9, 5.6]),    # 0, 2, 3 rise more than 0.5
        (3.0, [1, 1, 1, 1], [1.0, 1.0, 1.0, 1.0]),    # impacts
        (3.5, [0, 0, 1, 1], [1.3, 1.2, 1.0, 1.0]),    # 0 departs 0.5 after impact: rebound
        (5.0, [0, 1, 1, 0], [1.3, 1.0, 1.0, 1.3]),    # 3 departs 2.0 after impact: entrained
        (9.0, [0, 0, 0, 0], [1.3, 1.2, 1.2, 1.3]),    # 2 departs 6.0 after: entrained; 1 rolled
    ]
    ev = _track(seq)
    got = [(e["particle"], e["rebound"], e["t_impact"], e["t_departure"]) for e in ev]
    assert got == [(0, 1, 3.0, 3.5), (3, 0, 3.0, 5.0), (2, 0, 3.0, 9.0)]
    e0 = ev[0]
    assert np.array_equal(e0["u_impact"], [3.0] * 3) and np.array_equal(e0["u_departure"], [3.5] * 3)
    assert np.array_equal(e0["omega_impact"], [-3.0] * 3)


def test_first_state_emits_nothing_and_ties_are_strict():
    # a rise of exactly h_r is not saltation; T_i exactly t_cir is no rebound
    seq = [
        (0.0, [1, 1], [1.0, 1.0]),
        (1.0, [0, 0], [1.0, 1.0]),
        (2.0, [0, 0], [1.5, 1.75]),    # sphere 0 rises exactly 0.5, sphere 1 more
        (3.0, [1, 1], [1.0, 1.0]),
        (4.0, [0, 0], [1.0, 1.0]),     # sphere 1 departs exactly t_cir after impact
    ]
    ev = _track(seq)
    assert [(e["particle"], e["rebound"]) for e in ev] == [(1, 0)]
    assert _track(seq[:1]) == []
