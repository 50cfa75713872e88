"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads without a GPU and
exports every function include/gbpic.h declares.  No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gbpic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ["pic_create", "pic_load_species", "pic_set_external_field", "pic_set_plasma", "pic_step",
                 "pic_get_fields", "pic_get_moments", "pic_destroy", "pic_last_error", "pic_create_batch",
                 "pic_load_species_batch", "pic_set_external_field_batch", "pic_set_plasma_batch",
                 "pic_get_moments_run", "pic_autotune", "pic_use_graphs", "pic_checkpoint", "pic_backward", "pic_set_pusher", "pic_resolution_factor",
                 "pic_resonant_wavenumber"]:
        assert need in names


def test_library_exports_every_declared_symbol():
    from paper_2411_04703_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads_without_gpu():
    from paper_2411_04703_gb300 import api
    L = api.lib()
    # before any failed call the context-free message is an empty string, not NULL
    assert isinstance(L.pic_last_error(None), bytes)


# ------------------------------------------------------------------ Eq. RadLambda (host-only call)

def test_resonant_wavenumber_matches_the_oracle(oracle_lib):
    import math

    import oracle
    from paper_2411_04703_gb300 import api
    for lam_u, K, gB, gR in [(0.02, 1.0, 100.0, 10.0), (2.0, 1.5, 2000.0, 2000.0 / math.sqrt(2.125)),
                             (7.3, 0.0, 300.0, 50.0), (1.0, 2.0, 5.0, 1.0)]:
        k_lab = api.resonant_wavenumber(lam_u, K, gB)
        assert k_lab == pytest.approx(2 * math.pi / oracle.resonant_wavelength(lam_u, K, gB), rel=1e-13)
        # the boosted image is the lab wave pattern moving with the beam's mean velocity, whose
        # longitudinal Lorentz factor is gamma_B / sqrt(1 + K^2/2): stretched by Eq. Belon's factor.
        # Both forms of the mean velocity agree to leading order, 1 - beta_z = 1/(2 gamma_z^2); they
        # differ by the next term, of relative size 1/gamma_z^2 at most
        gz = gB / math.sqrt(1 + 0.5 * K * K)
        k_rrf = api.resonant_wavenumber(lam_u, K, gB, gR, api.PIC_FRAME_BOOSTED)
        assert k_rrf == pytest.approx(k_lab / oracle.beam_elongation(gz, gR), rel=1.0 / gz ** 2)


def test_resonant_wavenumber_rejects_bad_arguments():
    from paper_2411_04703_gb300 import api
    for args in [(0.0, 1.0, 100.0), (1.0, -1.0, 100.0), (1.0, 1.0, 0.5), (float("nan"), 1.0, 100.0)]:
        with pytest.raises(api.PicError, match="pic_resonant_wavenumber"):
            api.resonant_wavenumber(*args)
    with pytest.raises(api.PicError, match="frame"):
        api.resonant_wavenumber(1.0, 1.0, 100.0, 10.0, 7)


# ------------------------------------------------------------------ argument validation
# pic_create checks its arguments before any CUDA call, so its error behaviour (PIC_ERR_ARG and
# the message kept for pic_last_error(NULL)) is testable without a GPU.

PIC_ERR_ARG, PIC_ERR_CUDA = -1, -2


def _create(L, api, grid=(16, 16, 16), dx=(1.0, 1.0, 1.0), dt=0.4, gamma=10.0, faces=((0, 0),) * 3, pml=0,
            moving=0, window_v=0.0, order=1, runs=None):
    h = ctypes.c_void_p()
    bc = api.pic_boundaries()
    for d in range(3):
        for f in range(2):
            bc.face[d][f] = faces[d][f]
    bc.pml_cells, bc.moving_window, bc.window_v = pml, moving, window_v
    g = api.pic_grid(*grid)
    d3 = (ctypes.c_double * 3)(*dx)
    if runs is None:
        r = L.pic_create(ctypes.byref(h), g, d3, dt, gamma, ctypes.byref(bc), order, None)
    else:
        r = L.pic_create_batch(ctypes.byref(h), runs, g, d3, dt, gamma, ctypes.byref(bc), order, None)
    return r, h


def _message(L):
    m = L.pic_last_error(None)
    return m.decode() if isinstance(m, bytes) else str(m)


def test_create_rejects_bad_arguments_before_touching_the_device():
    from paper_2411_04703_gb300 import api
    L = api.lib()
    PML, OPEN = 1, 2
    cases = [
        (dict(order=3), "shape_order"),
        (dict(dt=0.6), "Courant"),                       # 1/sqrt(3) = 0.577 for unit cells
        (dict(gamma=0.5), "gamma_boost"),
        (dict(dx=(1.0, 0.0, 1.0)), "cell sizes"),
        (dict(grid=(2048, 16, 16)), "nx and ny"),
        (dict(faces=((0, 1), (0, 0), (0, 0))), "periodic on both faces"),
        (dict(faces=((PML, PML), (0, 0), (0, 0)), pml=0), "pml_cells"),
        (dict(faces=((PML, PML), (0, 0), (0, 0)), pml=8), "thicker than half"),
        (dict(moving=1, window_v=0.5), "non-periodic z"),
        (dict(faces=((0, 0), (0, 0), (OPEN, OPEN)), moving=1, window_v=3.0), "window_v"),
        (dict(runs=0), "runs must be"),
        (dict(runs=4, faces=((0, 0), (0, 0), (OPEN, OPEN))), "z must be periodic"),
        (dict(runs=4, grid=(16, 16, 12)), "multiple of the tile size"),
    ]
    for kw, words in cases:
        r, h = _create(L, api, **kw)
        assert r == PIC_ERR_ARG, (kw, r)
        assert not h.value, kw
        assert words in _message(L), (kw, _message(L))


def test_null_handles_are_refused_and_destroy_accepts_null():
    from paper_2411_04703_gb300 import api
    L = api.lib()
    assert L.pic_destroy(None) == 0
    assert L.pic_step(None, 1) == PIC_ERR_ARG
    assert L.pic_sync(None) == PIC_ERR_ARG
    r, h = ctypes.c_double(), ctypes.c_int()
    assert L.pic_resolution_factor(None, 1.0, ctypes.byref(r), ctypes.byref(h)) == PIC_ERR_ARG


def test_valid_create_without_a_gpu_fails_loudly():
    # no CPU fallback: with valid arguments and no device, creation reports the CUDA failure
    import pytest
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2411_04703_gb300 import api
    L = api.lib()
    r, h = _create(L, api)
    assert r == PIC_ERR_CUDA and not h.value, r
    assert "cuda" in _message(L).lower()


def test_noalloc_sort_rejects_out_of_range_sizes_before_any_device_work():
    # every case fails its host-side checks, so the (placeholder, never dereferenced) buffer
    # addresses are not touched
    from paper_2411_04703_gb300 import api, build
    L = api.lib()                                      # pic_last_error(NULL) with its signature
    S = ctypes.CDLL(build.build()).pic_tile_sort_noalloc
    S.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    S.restype = ctypes.c_int
    fake = ctypes.c_void_p(256)
    g = (ctypes.c_int * 3)(64, 64, 64)
    t = (ctypes.c_int * 3)(8, 8, 8)
    cases = [
        ((None, 10, g, t, fake, fake), "null pointer"),
        ((fake, -1, g, t, fake, fake), "negative n"),
        ((fake, (1 << 20) + 1, g, t, fake, fake), "exceeds the maximum"),
        ((fake, 10, g, (ctypes.c_int * 3)(8, 128, 8), fake, fake), "out of range"),
        ((fake, 10, (ctypes.c_int * 3)(1024, 1024, 8), (ctypes.c_int * 3)(1, 1, 1), fake, fake), "keys exceed"),
        # one tile as large as the grid limits: 2^31 cells, more than an int holds
        ((fake, 10, (ctypes.c_int * 3)(1024, 1024, 2048), (ctypes.c_int * 3)(1024, 1024, 2048), fake, fake),
         "keys exceed"),
    ]
    for (cells, n, grid, tile, order, key_start), words in cases:
        r = S(cells, n, grid, tile, order, key_start, None)
        assert r == PIC_ERR_ARG, (words, r)
        assert words in _message(L), (words, _message(L))
