"""Host-side fault injection on the GPU path (no fault, trap or hang of the GPU itself):

* a particle loaded with a NaN momentum: the push turns it into a dummy and raises the device
  error word; pic_sync reports PIC_ERR_DEVICE naming the cause, and the context can still be
  destroyed;
* a caller allocator that refuses the k-th request, for every k that pic_create makes: the call
  returns PIC_ERR_ALLOC, hands back no context, and returns every buffer it had obtained.
"""
import ctypes

import numpy as np
import pytest

from paper_2411_04703_gb300 import api, workloads as W

pytestmark = pytest.mark.gpu

PIC_ERR_ALLOC, PIC_ERR_DEVICE = -3, -5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def test_nan_momentum_is_reported_through_the_error_word():
    w = W.mini_vacuum(order=1)              # periodic box: every deposit index wraps
    sim, _ = api.from_workload(w, beam=False)
    n = 64
    rng = np.random.default_rng(3)
    x = np.stack([rng.uniform(2.0, w.grid[d] - 2.0, n) * w.d[d] for d in range(3)])
    u = np.zeros((3, n))
    u[2] = 1.0
    u[0, 17] = np.nan
    sim.load_species(-1.0, 1.0, x, u, np.ones(n), frame=api.PIC_FRAME_BOOSTED)
    with pytest.raises(api.PicError) as err:
        sim.step(1)
        sim.sync()
    assert err.value.code == PIC_ERR_DEVICE, err.value
    assert "non-finite momentum" in str(err.value)
    sim.close()


def test_refused_allocation_in_create_is_reported_and_released():
    import torch
    L = api.lib()
    stream = torch.cuda.Stream(0)
    bc = api.pic_boundaries()
    for d in range(2):
        bc.face[d][0] = bc.face[d][1] = 1       # PML on x and y: the layers' buffers too
    bc.pml_cells = 4
    made = None
    for refuse in range(64):
        live, calls = {}, [0]

        def _alloc(nbytes, user):
            calls[0] += 1
            if calls[0] == refuse + 1:
                return None
            try:
                p = torch.cuda.caching_allocator_alloc(int(nbytes), 0, stream)
            except Exception:
                return None
            live[p] = nbytes
            return p

        def _free(ptr, nbytes, user):
            if ptr in live:
                del live[ptr]
                torch.cuda.caching_allocator_delete(ptr)

        fa, ff = api.ALLOC_FN(_alloc), api.FREE_FN(_free)
        dev = api.pic_device()
        dev.alloc, dev.free, dev.device = fa, ff, 0
        dev.stream = ctypes.c_void_p(stream.cuda_stream)
        h = ctypes.c_void_p()
        r = L.pic_create(ctypes.byref(h), api.pic_grid(16, 16, 32), (ctypes.c_double * 3)(1.0, 1.0, 1.0), 0.4, 10.0,
                         ctypes.byref(bc), 2, ctypes.byref(dev))
        if r == 0:
            made = calls[0]
            assert L.pic_destroy(h) == 0
            assert not live
            break
        assert r == PIC_ERR_ALLOC, (refuse, r, L.pic_last_error(None))
        assert not h.value, refuse
        assert not live, (refuse, len(live))
    assert made is not None and made >= 10, made
