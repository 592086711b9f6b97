"""prs_find_pairs_noalloc, the pair search whose scratch is a fixed array
inside the library, against prs_find_pairs through the C ABI. Pair sets must
be identical; consecutive calls share the array, so each call of a run of
calls on different inputs is checked. Collected last, so it also runs after
every other GPU test has used the library."""
import ctypes as C

import numpy as np
import pytest

from paper_2108_01814_gb300 import binding as B
from tests.gpu_helpers import packing

CASES = [
    # (grid n, periodic, R, n_particles, seed)
    ((24, 24, 24), (1, 1, 1), 1.0, 500, 1),
    ((16, 16, 16), (0, 0, 0), 1.5, 90, 3),
    ((20, 16, 24), (1, 1, 0), 1.0, 380, 2),
]


def _sorted_pairs(p):
    p = np.asarray(p, dtype=np.int64).reshape(-1, 2)
    return p[np.lexsort((p[:, 1], p[:, 0]))]


def _reference(x, n, per, R, cut):
    c = B.Context(n, 1.0, per, precision="fp64")
    c.create_particles(x.shape[1], R, 2.65, 1.0)
    z = np.zeros_like(x)
    c.write_state(x, z, z)
    ref = c.find_pairs(cut)
    c.close()
    return ref


@pytest.mark.gpu
def test_noalloc_pairs_match_context_pairs_on_consecutive_calls():
    import torch
    B.load()
    pairs = torch.empty((4096, 2), dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    n_calls = 0
    for n, per, R, n_p, seed in CASES + CASES[:1]:
        L = tuple(float(v) for v in n)
        x, _, _ = packing(n_p, L, R, seed, periodic=per)
        xd = torch.from_numpy(np.ascontiguousarray(x)).to("cuda")
        for cut in (2 * R, 2 * R + 1.0):
            pairs.fill_(-1)
            B.find_pairs_noalloc(xd, L, per, cut, pairs, count)
            torch.cuda.synchronize()
            total = int(count.item())
            assert 0 < total <= pairs.shape[0]
            got = _sorted_pairs(pairs[:total].cpu().numpy())
            ref = _reference(x, n, per, R, cut)
            assert got.shape == ref.shape and np.array_equal(got, ref), (n, cut)
            n_calls += 1
    assert n_calls >= 2


@pytest.mark.gpu
def test_noalloc_reports_total_beyond_capacity():
    import torch
    n, per, R, n_p, seed = CASES[0]
    L = tuple(float(v) for v in n)
    x, _, _ = packing(n_p, L, R, seed, periodic=per)
    xd = torch.from_numpy(np.ascontiguousarray(x)).to("cuda")
    ref = _reference(x, n, per, R, 2 * R + 1.0)
    pairs = torch.full((5, 2), -1, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    B.find_pairs_noalloc(xd, L, per, 2 * R + 1.0, pairs, count)
    torch.cuda.synchronize()
    assert int(count.item()) == len(ref)
    got = pairs.cpu().numpy()
    refset = {tuple(r) for r in ref}
    assert all(tuple(r) in refset for r in got)


def test_noalloc_rejects_sizes_beyond_the_limit_without_gpu():
    lib = B.load()
    L = (C.c_double * 3)(10.0, 10.0, 10.0)
    per = (C.c_int * 3)(1, 1, 1)
    fake = C.c_void_p(256)  # never dereferenced: arguments are checked first
    st = lib.prs_find_pairs_noalloc(fake, B.NOALLOC_MAX_PARTICLES + 1, C.cast(L, C.c_void_p),
                                    C.cast(per, C.c_void_p), 1.0, fake, 10, fake, None)
    assert st == -1 and b"limit" in lib.prs_last_error_string()
    st = lib.prs_find_pairs_noalloc(fake, 10, C.cast(L, C.c_void_p), C.cast(per, C.c_void_p),
                                    0.0, fake, 10, fake, None)
    assert st == -1 and b"cutoff" in lib.prs_last_error_string()
    st = lib.prs_find_pairs_noalloc(fake, 10, None, C.cast(per, C.c_void_p), 1.0, fake, 10,
                                    fake, None)
    assert st == -1


def _oracle_pairs(x, L, per, cut):
    import oracle as O
    d = O.dem_params(1.0, 2.65, 1.0, 0.9, 0.39, 0.4, 0.1, (0.0, 0.0, 0.0), L, per)
    return O.pairs(d, x, cut)


def _noalloc(x, L, per, cut, cap=1 << 16, stream=None):
    import torch
    xd = torch.from_numpy(np.ascontiguousarray(x)).to("cuda")
    pairs = torch.full((cap, 2), -1, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    B.find_pairs_noalloc(xd, L, per, cut, pairs, count, stream=stream)
    torch.cuda.synchronize()
    total = int(count.item())
    return total, _sorted_pairs(pairs[:min(total, cap)].cpu().numpy())


@pytest.mark.gpu
@pytest.mark.parametrize("case", ["coarsened", "short_periodic_axis", "side_stream"])
def test_noalloc_pairs_match_oracle(case):
    # the FP64 oracle's brute-force pair set (Eq. A.1, A.3), directly
    import torch
    rng = np.random.Generator(np.random.PCG64(77))
    if case == "coarsened":
        # (200 / 2.5)^3 = 512,000 cells of the cutoff: more than the fixed
        # array holds, so the cells are widened
        L, per, n_p, cut = (200.0, 200.0, 200.0), (1, 1, 1), 6000, 2.5
        assert (200 / 2.5) ** 3 > B.NOALLOC_MAX_CELLS
    elif case == "short_periodic_axis":
        # a periodic axis shorter than three cutoffs: every cell along it is
        # a neighbour, each listed once
        L, per, n_p, cut = (5.0, 30.0, 30.0), (1, 1, 0), 900, 2.0
    else:
        L, per, n_p, cut = (24.0, 24.0, 24.0), (1, 1, 1), 500, 2.5
    x = rng.uniform(0.0, 1.0, (3, n_p)) * np.array(L)[:, None]
    ref = _oracle_pairs(x, L, per, cut)
    assert len(ref) > 10
    if case == "side_stream":
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            total, got = _noalloc(x, L, per, cut, stream=s.cuda_stream)
    else:
        total, got = _noalloc(x, L, per, cut)
    assert total == len(ref)
    assert np.array_equal(got, ref)


@pytest.mark.gpu
def test_noalloc_no_spheres_gives_no_pairs():
    import torch
    pairs = torch.full((4, 2), -1, dtype=torch.int32, device="cuda")
    count = torch.full((1,), 7, dtype=torch.int64, device="cuda")
    x = torch.zeros((3, 0), dtype=torch.float64, device="cuda")
    B.find_pairs_noalloc(x, (10.0, 10.0, 10.0), (1, 1, 1), 1.0, pairs, count)
    torch.cuda.synchronize()
    assert int(count.item()) == 0
    assert bool((pairs == -1).all())
