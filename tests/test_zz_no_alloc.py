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
