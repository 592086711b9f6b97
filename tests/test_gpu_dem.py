"""GPU parity of the DEM half (cell-list contact search, contact history,
spring-dashpot forces, Newton-Euler update) against the FP64 oracle,
through the C ABI. Contact and neighbour sets must match bit for bit;
states and forces within 1e-10 (normwise relative)."""
import numpy as np
import pytest

import oracle as O
from paper_2108_01814_gb300 import workloads as W
from tests.gpu_helpers import packing, rel_err

pytestmark = pytest.mark.gpu

OPTS = dict(e_n=0.9, e_t=0.39, mu=0.4, T_c=0.05)


TOLS = {"fp64": 1e-10, "fp32": 1e-5}


def _ctx(n, h, periodic, R, x, u, om, rho_p=2.65, rho_f=1.0, precision="fp64"):
    from paper_2108_01814_gb300 import binding as B
    c = B.Context(n, h, periodic, precision=precision)
    c.create_particles(x.shape[1], R, rho_p, rho_f)
    c.write_state(x, u, om)
    return c


def _oracle_params(L, periodic, R, g=(0.0, 0.0, 0.0), rho_p=2.65, rho_f=1.0):
    return O.dem_params(R, rho_p, rho_f, OPTS["e_n"], OPTS["e_t"], OPTS["mu"], OPTS["T_c"], g,
                        L, periodic)


def _gpu_hist_to_oracle(h):
    o = O.History(len(h["cnt"]))
    for k in ("cnt", "pid", "uin", "dlt", "wact", "wuin", "wdlt"):
        getattr(o, k)[...] = h[k]
    return o


CASES = [
    # (grid n, periodic, R, n_particles, seed)
    ((24, 24, 24), (1, 1, 1), 1.0, 500, 1),
    ((20, 16, 24), (1, 1, 0), 1.0, 380, 2),
    ((16, 16, 16), (0, 0, 0), 1.5, 90, 3),
]


@pytest.mark.parametrize("case", CASES)
def test_contact_and_neighbour_sets_bit_exact(case):
    n, per, R, n_p, seed = case
    L = tuple(float(v) for v in n)
    x, u, om = packing(n_p, L, R, seed, periodic=per)
    c = _ctx(n, 1.0, per, R, x, u, om)
    d = _oracle_params(L, per, R)
    for cut in (2 * R, 2 * R + 1.0, 2 * R + 0.25):
        got = c.find_pairs(cut)
        ref = O.pairs(d, x, cut)
        assert got.shape == ref.shape and np.array_equal(got, ref), cut
    assert len(O.pairs(d, x, 2 * R)) > 20  # the packing has real contacts
    c.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES)
def test_one_substep_parity(case, precision):
    # FP32 form: FP32 spring-dashpot arithmetic on FP64 overlap, history and
    # state; contact sets still exact
    n, per, R, n_p, seed = case
    L = tuple(float(v) for v in n)
    x, u, om = packing(n_p, L, R, seed, periodic=per)
    g = (0.0, 0.0, -0.5) if not per[2] else (0.0, 0.0, 0.0)
    tol = TOLS[precision]
    c = _ctx(n, 1.0, per, R, x, u, om, precision=precision)
    dt_p = 1e-3
    c.dem_step(dt_p, 1, g=g, **OPTS)
    xg, ug, og = c.read_state()
    fg = c.read_forces()
    hg = c.read_history()
    d = _oracle_params(L, per, R, g=g)
    z = np.zeros((3, n_p))
    xo, uo, oo, Fc, Tc, ho, ov = O.dem_substep(d, dt_p, x, u, om, z, z, O.History(n_p))
    assert not ov
    # contact sets: exact
    assert np.array_equal(hg["cnt"], ho.cnt)
    assert np.array_equal(hg["pid"], ho.pid)
    assert np.array_equal(hg["wact"], ho.wact)
    # states, forces, history values
    for a, b in ((xg, xo), (ug, uo), (og, oo), (fg["F_c"], Fc), (fg["T_c"], Tc),
                 (hg["uin"], ho.uin), (hg["dlt"], ho.dlt), (hg["wdlt"], ho.wdlt)):
        assert rel_err(a, b) <= tol
    c.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES[:2])
def test_many_substeps_parity(case, precision):
    # 40 sub-steps with history carried over: new, existing and finished
    # events all occur; GPU and oracle stay together
    n, per, R, n_p, seed = case
    L = tuple(float(v) for v in n)
    x, u, om = packing(n_p, L, R, seed, periodic=per, vel=0.5)
    g = (0.0, 0.0, -0.5) if not per[2] else (0.0, 0.0, 0.0)
    tol = TOLS[precision]
    c = _ctx(n, 1.0, per, R, x, u, om, precision=precision)
    dt_p, k = 1e-3, 40
    Fh = np.zeros((3, n_p))
    c.dem_step(dt_p, k, g=g, **OPTS)
    xg, ug, og = c.read_state()
    hg = c.read_history()
    d = _oracle_params(L, per, R, g=g)
    xo, uo, oo, Fc, Tc, ho, ov = O.dem_run(d, dt_p, k, x, u, om, Fh, Fh, O.History(n_p))
    assert np.array_equal(hg["pid"], ho.pid)
    assert np.array_equal(hg["cnt"], ho.cnt)
    for a, b in ((xg, xo), (ug, uo), (og, oo), (hg["dlt"], ho.dlt)):
        assert rel_err(a, b) <= tol
    c.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_clipped_normal_force_parity(precision):
    # the variant whose normal force is clipped to be repulsive, sphere-sphere
    # and sphere-wall, 40 sub-steps against the oracle's clipped law; the
    # plain law ends elsewhere, so the option is in effect
    n, per, R, n_p, seed = CASES[1]
    L = tuple(float(v) for v in n)
    x, u, om = packing(n_p, L, R, seed, periodic=per, vel=0.5)
    g = (0.0, 0.0, -0.5)
    c = _ctx(n, 1.0, per, R, x, u, om, precision=precision)
    dt_p, k = 1e-3, 40
    c.dem_step(dt_p, k, g=g, clip_normal=True, **OPTS)
    xg, ug, og = c.read_state()
    hg = c.read_history()
    c.close()
    z = np.zeros((3, n_p))
    d = O.dem_params(R, 2.65, 1.0, OPTS["e_n"], OPTS["e_t"], OPTS["mu"], OPTS["T_c"], g, L, per,
                     clip_normal=True)
    xo, uo, oo, _, _, ho, ov = O.dem_run(d, dt_p, k, x, u, om, z, z, O.History(n_p))
    assert not ov
    assert np.array_equal(hg["pid"], ho.pid) and np.array_equal(hg["cnt"], ho.cnt)
    assert np.array_equal(hg["wact"], ho.wact)
    for a, b in ((xg, xo), (ug, uo), (og, oo), (hg["dlt"], ho.dlt)):
        assert rel_err(a, b) <= TOLS[precision]
    _, up, _, _, _, _, _ = O.dem_run(_oracle_params(L, per, R, g=g), dt_p, k, x, u, om, z, z,
                                     O.History(n_p))
    assert rel_err(up, uo) > 100 * TOLS[precision]


def test_history_resume_is_bit_identical():
    # checkpoint after 10 sub-steps, restore into a fresh context, continue:
    # same result as running straight through
    n, per, R, n_p, seed = CASES[0]
    L = tuple(float(v) for v in n)
    x, u, om = packing(n_p, L, R, seed, periodic=per, vel=0.5)
    a = _ctx(n, 1.0, per, R, x, u, om)
    a.dem_step(1e-3, 20, **OPTS)
    xa, ua, oa = a.read_state()
    b = _ctx(n, 1.0, per, R, x, u, om)
    b.dem_step(1e-3, 10, **OPTS)
    st = b.read_state()
    hist = b.read_history()
    c = _ctx(n, 1.0, per, R, *st)
    c.write_history(**hist)
    c.dem_step(1e-3, 10, **OPTS)
    xc, uc, oc = c.read_state()
    assert np.array_equal(xa, xc) and np.array_equal(ua, uc) and np.array_equal(oa, oc)
    for k in (a, b, c):
        k.close()


def test_contact_overflow_reported():
    from paper_2108_01814_gb300 import binding as B
    rng = np.random.Generator(np.random.PCG64(4))
    dirs = rng.normal(size=(3, 13))
    dirs /= np.linalg.norm(dirs, axis=0)
    x = np.concatenate([np.full((3, 1), 10.0), 10.0 + 1.5 * dirs], axis=1)
    z = np.zeros_like(x)
    c = _ctx((20, 20, 20), 1.0, (1, 1, 1), 1.0, x, z, z)
    c.dem_step(1e-4, 1, **OPTS)
    with pytest.raises(B.PrsError) as e:
        c.read_state()
    assert e.value.status == -5
    c.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_bed_substep_parity(precision):
    # the 8448-sphere channel bed (walls in z, gravity, spheres resting on
    # each other), one sub-step
    w = W.bed()
    from paper_2108_01814_gb300 import binding as B
    c = B.Context(w.n, w.h, w.periodic, precision=precision)
    c.create_particles(w.n_p, w.R, w.rho_p, w.rho_f)
    # settle the bed onto the wall a little so there are wall contacts
    x = w.x.copy()
    x[2] -= 0.3
    c.write_state(x, w.u, w.om)
    dt_p = w.dt / w.n_sub
    c.dem_step(dt_p, 1, e_n=w.e_n, e_t=w.e_t, mu=w.mu, T_c=w.T_c, g=w.g)
    xg, ug, og = c.read_state()
    hg = c.read_history()
    d = O.dem_params(w.R, w.rho_p, w.rho_f, w.e_n, w.e_t, w.mu, w.T_c, w.g, w.L, w.periodic)
    z = np.zeros((3, w.n_p))
    xo, uo, oo, Fc, Tc, ho, ov = O.dem_substep(d, dt_p, x, w.u, w.om, z, z, O.History(w.n_p))
    assert hg["wact"].sum() == ho.wact.sum() > 0
    assert (ho.cnt > 0).mean() > 0.9
    assert np.array_equal(hg["pid"], ho.pid)
    for a, b in ((xg, xo), (ug, uo), (og, oo)):
        assert rel_err(a, b) <= TOLS[precision]
    c.close()


def _near_touching_pairs(L, R, eps, seed):
    # one pair per relative gap eps: centres d = 2R (1 + eps) apart along a
    # random direction, pairs far apart from each other, some across the
    # periodic faces and at large coordinates (where FP32 positions are
    # coarsest)
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = []
    spacing = 2 * R + 4.0
    slots = [(i, j) for i in range(int(L[0] // spacing)) for j in range(int(L[1] // spacing))]
    rng.shuffle(slots)
    for k, e in enumerate(eps):
        i, j = slots[k]
        c = np.array([(i + 0.5) * spacing, (j + 0.5) * spacing, L[2] / 2])
        c[:2] += rng.uniform(-0.5, 0.5, 2)
        if k % 3 == 0:          # straddle the periodic face in x
            c[0] = L[0] - 0.3 * R
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        a, b = c - R * (1 + e) * n, c + R * (1 + e) * n
        for q in (a, b):
            q[:2] %= L[:2]
            pts.append(q)
    return np.array(pts).T.copy()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_near_touching_pairs_decided_exactly(precision):
    # pairs at relative gaps from 1e-3 down to 1e-13 and exactly 2R, on a
    # large box: the contact set after one sub-step matches the FP64 oracle's
    # decision d < 2R bit for bit (the FP32 form decides clear cases in FP32,
    # narrow ones in FP32 pair arithmetic, the narrowest in FP64)
    n, per, R = (1024, 768, 64), (1, 1, 0), 3.0
    L = np.array(n, float)
    eps = [s * 10.0 ** -k for k in range(3, 14) for s in (1, -1)] + [0.0]
    x = _near_touching_pairs(L, R, eps, seed=17)
    z = np.zeros_like(x)
    c = _ctx(n, 1.0, per, R, x, z, z, precision=precision)
    c.dem_step(1e-6, 1, **OPTS)
    hg = c.read_history()
    c.close()
    d = _oracle_params(tuple(L), per, R)
    _, _, _, _, _, ho, ov = O.dem_substep(d, 1e-6, x, z, z, z, z, O.History(x.shape[1]))
    assert not ov
    assert 10 <= len(O.pairs(d, x, 2 * R)) <= 12  # the pairs with eps < 0 (and 0 maybe)
    assert np.array_equal(hg["cnt"], ho.cnt)
    assert np.array_equal(hg["pid"], ho.pid)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_graph_replay_matches_launches(precision):
    # the sub-steps captured once as a CUDA graph and replayed by the later
    # calls, against the same calls as plain launches: identical states,
    # history and launch counts
    import torch
    from paper_2108_01814_gb300 import binding as B
    n, per, R, n_p, seed = CASES[1]
    L = tuple(float(v) for v in n)
    x, u, om = packing(n_p, L, R, seed, periodic=per, vel=0.5)
    out = []
    for graphs in (True, False):
        s = torch.cuda.Stream()
        c = B.Context(n, 1.0, per, precision=precision, stream=s)
        c.create_particles(n_p, R, 2.65, 1.0)
        c.write_state(x, u, om)
        c.set_graphs(graphs)
        l0 = c.stats().n_launches
        used = []
        for _ in range(3):
            c.dem_step(1e-3, 10, g=(0.0, 0.0, -1.0), **OPTS)
            used.append(c.stats().dem_graph)
        out.append((c.read_state(), c.read_history(), c.stats().n_launches - l0, used))
        c.close()
    (sg, hg, lg, ug), (sl, hl, ll, ul) = out
    assert ug == [1, 1, 1] and ul == [0, 0, 0]
    assert lg == ll
    for a, b in zip(sg, sl):
        assert np.array_equal(a, b)
    for k in hg:
        assert np.array_equal(hg[k], hl[k]), k
    assert hg["cnt"].sum() > 0


def test_graph_gives_way_to_launches_when_never_replayed():
    # a step that changes on every call would cost a capture per call: after
    # two graphs that no call replayed, the context uses launches; the
    # results stay those of launches throughout
    import torch
    from paper_2108_01814_gb300 import binding as B
    n, per, R, n_p, seed = CASES[0]
    L = tuple(float(v) for v in n)
    x, u, om = packing(n_p, L, R, seed, periodic=per, vel=0.5)
    out = []
    for graphs in (True, False):
        c = B.Context(n, 1.0, per, precision="fp64", stream=torch.cuda.Stream())
        c.create_particles(n_p, R, 2.65, 1.0)
        c.write_state(x, u, om)
        c.set_graphs(graphs)
        used = []
        for k in range(5):
            c.dem_step(1e-3 * (1 + 0.1 * k), 4, **OPTS)
            used.append(c.stats().dem_graph)
        out.append((c.read_state(), used))
        c.close()
    assert out[0][1] == [1, 1, 0, 0, 0] and out[1][1] == [0] * 5
    for a, b in zip(out[0][0], out[1][0]):
        assert np.array_equal(a, b)
