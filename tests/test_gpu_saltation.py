"""GPU parity of the bed / flying classification and of the saltation events
(Sec. 4.3.1) against the FP64 oracle, through the C ABI: flags and events
bit for bit."""
import numpy as np
import pytest

import oracle as O
from oracle import saltation as S
from paper_2108_01814_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _ctx(w, x=None, u=None, om=None):
    from paper_2108_01814_gb300 import binding as B
    c = B.Context(w.n, w.h, w.periodic, precision="fp32")
    c.create_particles(w.n_p, w.R, w.rho_p, w.rho_f)
    c.write_state(w.x if x is None else x, w.u if u is None else u, w.om if om is None else om)
    return c


def _dem(w):
    return O.dem_params(w.R, w.rho_p, w.rho_f, w.e_n, w.e_t, w.mu, w.T_c, w.g, w.L, w.periodic)


@pytest.mark.parametrize("name", ["small_bed", "bed"])
def test_bed_flags_bit_exact(name):
    w = W.small_bed(seed=3) if name == "small_bed" else W.bed()
    c = _ctx(w)
    got = c.bed_detect()
    c.close()
    ref = S.bed_flags(_dem(w), w.x, w.R)
    assert np.array_equal(got, ref)
    assert 0 < ref.sum() < w.n_p


def test_bed_flags_hand_built():
    # a chain from the bottom, a floating cluster, a lone bottom sphere, and a
    # bridge across the periodic face
    R = 1.0
    gap = 2 * R * (1 - 1e-3)
    dz = 1.2
    ax = np.sqrt(gap * gap - dz * dz)
    pts = [[5.0, 5.0, R + k * gap] for k in range(6)]
    pts += [[12.0, 12.0, 30.0], [15.0, 5.0, 20.0], [15.0 + gap, 5.0, 20.0],
            [2.0, 15.0, 1.5], [0.4, 10.0, R], [20.0 - ax + 0.4, 10.0, R + dz],
            [20.0 - ax + 0.4, 10.0, R + dz + gap]]
    x = np.array(pts).T.copy()
    z = np.zeros_like(x)
    w = W.Workload(name="hand", n=(20, 20, 40), h=1.0, periodic=(1, 1, 0), R=R, rho_p=2.65,
                   rho_f=1.0, x=x, u=z, om=z, dt=0.01, n_sub=50, e_n=0.9, e_t=0.39, mu=0.4,
                   T_c=0.1, g=(0.0, 0.0, 0.0), fluid_mean="none", fluid_std=0.1)
    c = _ctx(w)
    got = c.bed_detect()
    c.close()
    assert list(got) == [1] * 6 + [0, 0, 0, 1, 1, 1, 1]
    assert np.array_equal(got, S.bed_flags(_dem(w), x, R))


def _movers(w, k=6):
    # top bed spheres: nothing rests on them, and lifted by up to 3.7 R they
    # are clear of every other sphere
    d = _dem(w)
    bed = S.bed_flags(d, w.x, w.R)
    pr = O.pairs(d, w.x, 2 * w.R)
    above = np.zeros(w.n_p, dtype=bool)
    for p, q in pr:
        lo, hi = (p, q) if w.x[2, p] < w.x[2, q] else (q, p)
        above[lo] = True
    out = []
    for p in np.nonzero(bed & ~above)[0]:
        ok = True
        for lift in (2.5, 3.7):
            y = w.x[:, p].copy()
            y[2] += lift * w.R
            dd = w.x - y[:, None]
            for a in range(2):
                dd[a] -= w.L[a] * np.round(dd[a] / w.L[a])
            dist = np.sqrt((dd * dd).sum(0))
            dist[p] = np.inf
            ok = ok and dist.min() > 2 * w.R + 0.1
        if ok:
            out.append(int(p))
        if len(out) == k:
            break
    assert len(out) == k
    return out


def test_saltation_events_bit_exact():
    w = W.small_bed(seed=3)
    m = _movers(w)
    R = w.R
    lift = {0: {}, 1: {p: 2.5 for p in m}, 2: {**{p: 3.7 for p in m[:3]}, **{p: 2.5 for p in m[3:]}},
            3: {}, 4: {m[0]: 2.5}, 5: {m[0]: 2.5, m[1]: 2.5}, 6: {m[0]: 2.5, m[1]: 2.5, m[3]: 2.5}}
    times = [0.0, 0.1, 0.2, 0.3, 0.35, 0.6, 0.7]
    h_r, t_cir = R, 0.1
    rng = np.random.Generator(np.random.PCG64(8))
    c = _ctx(w)
    tr = S.Tracker(w.n_p)
    d = _dem(w)
    got, ref = [], []
    for k, t in enumerate(times):
        x = w.x.copy()
        for p, l in lift[k].items():
            x[2, p] += l * R
        u = rng.normal(size=x.shape)
        om = rng.normal(size=x.shape)
        c.write_state(x, u, om)
        got += list(c.track_saltation(t, h_r, t_cir))
        ref += tr.step(t, S.bed_flags(d, x, R), x, u, om, h_r, t_cir)
    c.close()
    # m0 rebounds (0.05 after its impact), m1 is entrained (0.3 after), m2 has
    # not departed again, m3 rolled
    assert [(e["particle"], e["rebound"]) for e in ref] == [(m[0], 1), (m[1], 0)]
    assert len(got) == len(ref)
    for g, r in zip(got, ref):
        for key in ("particle", "rebound", "t_impact", "t_departure"):
            assert g[key] == r[key], key
        for key in ("u_impact", "omega_impact", "u_departure", "omega_departure"):
            assert np.array_equal(g[key], r[key]), key


def test_saltation_capacity_and_reset():
    from paper_2108_01814_gb300 import binding as B
    w = W.small_bed(seed=3)
    m = _movers(w, 2)
    c = _ctx(w)
    c.track_saltation(0.0, w.R, 1.0)
    x25, x37 = w.x.copy(), w.x.copy()
    x25[2, m] += 2.5 * w.R
    x37[2, m] += 3.7 * w.R
    for t, x in ((1.0, x25), (1.5, x37), (2.0, w.x)):       # depart, saltate, impact
        c.write_state(x, w.u, w.om)
        assert len(c.track_saltation(t, w.R, 1.0)) == 0
    c.write_state(x25, w.u, w.om)
    with pytest.raises(B.PrsError) as e:
        c.track_saltation(2.5, w.R, 1.0, max_events=1)      # two events close
    assert e.value.status == -7                              # PRS_ERR_CAPACITY
    c.reset_saltation()
    assert len(c.track_saltation(3.0, w.R, 1.0)) == 0      # starts afresh
    c.close()
