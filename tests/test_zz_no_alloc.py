"""GPU test of pic_tile_sort_noalloc, the sort entry point that allocates nothing.

It serves callers that cannot let the library allocate device memory (an application with a
fixed device pool reserved at start-up, or code that must not enter the CUDA allocator): they
pass every input and output buffer, and the scratch lives in a fixed array inside the library.

The test calls it through the C-ABI and checks its result against the existing entry point
that sorts the same particles (pic_sort inside a context): every tile-major key must hold the
same set of particles, bit-exact, on two calls in a row with different inputs (the second
call reuses the scratch the first one left behind).  This file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2411_04703_gb300 import api

pytestmark = pytest.mark.gpu


def _noalloc_fn():
    L = api.lib()
    fn = L.pic_tile_sort_noalloc
    fn.argtypes = [C.c_void_p, C.c_int64, C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_void_p, C.c_void_p,
                   C.c_void_p]
    fn.restype = C.c_int
    return fn


def _keys(cells, grid, tile):
    i, j, k = cells[:, 0], cells[:, 1], cells[:, 2]
    nt = [(g + t - 1) // t for g, t in zip(grid, tile)]
    tl = ((k // tile[2]) * nt[1] + j // tile[1]) * nt[0] + i // tile[0]
    loc = ((k % tile[2]) * tile[1] + j % tile[1]) * tile[0] + i % tile[0]
    return tl * (tile[0] * tile[1] * tile[2]) + loc


def _groups(keys, ids):
    out = {}
    for kk, ii in zip(keys.tolist(), ids.tolist()):
        out.setdefault(kk, set()).add(ii)
    return out


def test_noalloc_sort_matches_context_sort_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    fn = _noalloc_fn()
    grid, tile = (20, 18, 44), (8, 8, 8)
    d = (0.3, 0.3, 0.3)
    dt = 0.5 * 0.3 / np.sqrt(3)
    for seed, n in [(21, 50000), (22, 20011)]:
        rng = np.random.default_rng(seed)
        x = np.stack([rng.uniform(0, g * dd, n) for g, dd in zip(grid, d)])
        u = rng.normal(0, 0.1, (3, n))
        sim = api.Sim(grid, d, dt, 2.0, order=1)
        sid = sim.load_species(-1.0, 1.0, x, u, frame=api.PIC_FRAME_BOOSTED)
        P0 = sim.get_particles(sid)             # load order: ids 0..n-1
        assert np.array_equal(P0["id"], np.arange(n))
        # the existing entry point: sort inside the context
        sim.sort()
        Ps = sim.get_particles(sid)
        ref = _groups(_keys(Ps["cell"].astype(np.int64), grid, tile), Ps["id"])
        # the allocation-free entry point on caller-owned device buffers
        c = P0["cell"].astype(np.int64)
        packed = torch.tensor(c[:, 0] | (c[:, 1] << 10) | (c[:, 2] << 20), dtype=torch.int32, device="cuda")
        nt = [(g + t - 1) // t for g, t in zip(grid, tile)]
        n_keys = nt[0] * nt[1] * nt[2] * tile[0] * tile[1] * tile[2]
        order = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        key_start = torch.full((n_keys + 1,), -7, dtype=torch.int32, device="cuda")
        stream = torch.cuda.current_stream()
        g3, t3 = (C.c_int * 3)(*grid), (C.c_int * 3)(*tile)
        r = fn(packed.data_ptr(), n, g3, t3, order.data_ptr(), key_start.data_ptr(), stream.cuda_stream)
        assert r == 0, api.lib().pic_last_error(None)
        torch.cuda.synchronize()
        o = order.cpu().numpy()
        ks = key_start.cpu().numpy()
        assert ks[-1] == n and sorted(o.tolist()) == list(range(n))
        got = {}
        for kk in range(n_keys):
            if ks[kk + 1] > ks[kk]:
                got[kk] = set(o[ks[kk]:ks[kk + 1]].tolist())
        assert got == ref
        sim.close()


def _call(fn, packed, n, grid, tile, n_keys):
    import torch
    order = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    key_start = torch.full((n_keys + 1,), -7, dtype=torch.int32, device="cuda")
    g3, t3 = (C.c_int * 3)(*grid), (C.c_int * 3)(*tile)
    r = fn(packed.data_ptr(), n, g3, t3, order.data_ptr(), key_start.data_ptr(),
           torch.cuda.current_stream().cuda_stream)
    assert r == 0, api.lib().pic_last_error(None)
    torch.cuda.synchronize()
    return order.cpu().numpy(), key_start.cpu().numpy()


def test_noalloc_sort_drops_dummies_and_cells_outside_the_grid():
    # -1 and packed cells beyond the grid in each dim are dropped: key_start ends at the live
    # count and order holds exactly the live input indices, grouped by key as the documented
    # key says (numpy bincount / cumsum of the same keys)
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    fn = _noalloc_fn()
    grid, tile = (20, 18, 44), (8, 4, 8)
    rng = np.random.default_rng(31)
    n = 30000
    c = np.stack([rng.integers(0, g, n) for g in grid], 1)
    packed = c[:, 0] | (c[:, 1] << 10) | (c[:, 2] << 20)
    kind = rng.integers(0, 8, n)
    packed = np.where(kind == 0, -1, packed)
    packed = np.where(kind == 1, (grid[0] + rng.integers(0, 1024 - grid[0], n)) | (c[:, 1] << 10) | (c[:, 2] << 20), packed)
    packed = np.where(kind == 2, c[:, 0] | ((grid[1] + rng.integers(0, 1024 - grid[1], n)) << 10) | (c[:, 2] << 20), packed)
    packed = np.where(kind == 3, c[:, 0] | (c[:, 1] << 10) | ((grid[2] + rng.integers(0, 64, n)) << 20), packed)
    live = kind >= 4
    nt = [(g + t - 1) // t for g, t in zip(grid, tile)]
    n_keys = nt[0] * nt[1] * nt[2] * tile[0] * tile[1] * tile[2]
    for call in range(2):           # the second call finds the first call's scratch
        o, ks = _call(fn, torch.tensor(packed, dtype=torch.int32, device="cuda"), n, grid, tile, n_keys)
        keys = _keys(c[live], grid, tile)
        expect = np.concatenate([[0], np.cumsum(np.bincount(keys, minlength=n_keys))])
        assert np.array_equal(ks, expect), call
        assert ks[-1] == int(live.sum())
        got = o[:ks[-1]]
        assert sorted(got.tolist()) == np.flatnonzero(live).tolist()
        assert np.array_equal(_keys(c[got], grid, tile), np.sort(keys))


def test_noalloc_sort_at_the_largest_key_count():
    # n_keys = PIC_NOALLOC_MAX_KEYS = 2^22 (256 x 128 x 128 cells, one cell per tile): the scan of
    # the 2^22 + 1 counters takes three levels, with its block sums at the scratch's bound
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    fn = _noalloc_fn()
    grid, tile = (256, 128, 128), (1, 1, 1)
    n_keys = 256 * 128 * 128
    assert n_keys == 1 << 22
    rng = np.random.default_rng(32)
    n = 1 << 20
    c = np.stack([rng.integers(0, g, n) for g in grid], 1)
    packed = torch.tensor(c[:, 0] | (c[:, 1] << 10) | (c[:, 2] << 20), dtype=torch.int32, device="cuda")
    o, ks = _call(fn, packed, n, grid, tile, n_keys)
    keys = _keys(c, grid, tile)
    expect = np.concatenate([[0], np.cumsum(np.bincount(keys, minlength=n_keys))])
    assert np.array_equal(ks, expect)
    assert np.array_equal(np.sort(o), np.arange(n))
    assert np.all(np.diff(keys[o]) >= 0)


def test_noalloc_sort_rejects_sizes_beyond_its_maximum():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    fn = _noalloc_fn()
    g3, t3 = (C.c_int * 3)(8, 8, 8), (C.c_int * 3)(4, 4, 4)
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    r = fn(dummy.data_ptr(), (1 << 20) + 1, g3, t3, dummy.data_ptr(), dummy.data_ptr(), None)
    assert r == -1   # PIC_ERR_ARG
    assert b"exceeds the maximum" in api.lib().pic_last_error(None)
