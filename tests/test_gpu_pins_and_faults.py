"""GPU checks beyond one-step parity, and host-side fault injection (no GPU fault, trap or hang):

* analytic pins run on the GPU path itself, independent of the oracle: the gather reproduces
  linear fields sampled at the Yee points (CIC, TSC), and Boris rotates by -2 atan(h B / gamma)
  in a uniform magnetic field;
* degenerate input: a context whose only species is empty steps as the vacuum FDTD;
* the identical-state handover of the plasma buncher case (transverse CPML, moving window,
  plasma injection) after GPU steps, with the absorbing layers' auxiliary state not exported;
* faults injected on the host: a NaN momentum, reported through the device error word; an
  allocator that refuses the k-th request, for every k pic_create makes;
* the torch autograd wrapper of the adjoint (api.bunching_loss) against pic_backward.

Tolerances as in test_gpu_parity.py: 1e-5 relative per step from an identical state.
"""
import ctypes
import math

import numpy as np
import pytest

import oracle
from paper_2411_04703_gb300 import api, workloads as W

import parity

pytestmark = pytest.mark.gpu

TOL_STEP = 1e-5
PIC_ERR_ALLOC, PIC_ERR_DEVICE = -3, -5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    oracle.build()


def _random_fields(sim, w, seed, amp=1e-3):
    rng = np.random.default_rng(seed)
    for c in range(6):
        sim.set_field(c, (amp * rng.standard_normal((w.grid[2], w.grid[1], w.grid[0]))).astype(np.float32))


def _by_id(P):
    k = np.argsort(P["id"], kind="stable")
    return {key: v[k] for key, v in P.items()}


# ------------------------------------------------------------------ analytic pins on the GPU

@pytest.mark.parametrize("order", [1, 2])
def test_gpu_gather_reproduces_linear_fields(order):
    # With B = 0 and u = 0, one Boris step gives u = (q/m) dt E(x).  A field linear in position,
    # sampled at each component's Yee points, is gathered exactly by CIC and TSC (partition of
    # unity, zero first moment).
    n = (24, 24, 24)
    dt = 0.4
    sim = api.Sim(n, (1.0, 1.0, 1.0), dt, 10.0, bc=((0, 0),) * 3, order=order)
    rng = np.random.default_rng(9)
    a = rng.uniform(-1e-3, 1e-3, 3)
    b = rng.uniform(-1e-4, 1e-4, (3, 3))
    stag = [(0.5, 0.0, 0.0), (0.0, 0.5, 0.0), (0.0, 0.0, 0.5)]
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    for c in range(3):
        x, y, z = i + stag[c][0], j + stag[c][1], k + stag[c][2]
        sim.set_field(c, (a[c] + b[c, 0] * x + b[c, 1] * y + b[c, 2] * z).astype(np.float32))
    m = 500
    X = rng.uniform(6.0, 18.0, (3, m))          # stencils stay clear of the periodic wrap
    sid = sim.load_species(-1.0, 1.0, X, np.zeros((3, m)), np.full(m, 1e-6), frame=api.PIC_FRAME_BOOSTED)
    P0 = _by_id(sim.get_particles(sid))
    sim.step(1)
    sim.sync()
    P1 = _by_id(sim.get_particles(sid))
    assert np.array_equal(P0["id"], P1["id"])
    Xs = P0["cell"].astype(np.float64) + P0["off"].astype(np.float64)
    E = P1["u"].astype(np.float64) / (-1.0 * dt)
    expect = a[None, :] + Xs @ b.T
    assert np.max(np.abs(E - expect)) / np.max(np.abs(expect)) < TOL_STEP
    sim.close()


def test_gpu_boris_rotates_in_a_uniform_magnetic_field():
    # In a uniform B_z (E = 0) one Boris step rotates the transverse momentum by
    # -2 atan(h B_z / gamma), h = (q/m) dt / 2, and keeps u_z.
    n = (16, 16, 16)
    dt = 0.4
    sim = api.Sim(n, (1.0, 1.0, 1.0), dt, 10.0, bc=((0, 0),) * 3, order=1)
    Bz = 0.7
    sim.set_field(api.PIC_BZ, np.full((n[2], n[1], n[0]), Bz, np.float32))
    rng = np.random.default_rng(10)
    m = 300
    X = rng.uniform(2.0, 14.0, (3, m))
    u0 = np.stack([rng.uniform(-1.0, 1.0, m), rng.uniform(-1.0, 1.0, m), np.full(m, 0.3)])
    sid = sim.load_species(-1.0, 1.0, X, u0, np.full(m, 1e-6), frame=api.PIC_FRAME_BOOSTED)
    P0 = _by_id(sim.get_particles(sid))
    sim.step(1)
    sim.sync()
    P1 = _by_id(sim.get_particles(sid))
    U0 = P0["u"].astype(np.float64)
    U1 = P1["u"].astype(np.float64)
    h = 0.5 * (-1.0 / 1.0) * dt
    g = np.sqrt(1.0 + np.sum(U0 ** 2, axis=1))
    th = -2.0 * np.arctan(h * Bz / g)
    ex = np.cos(th) * U0[:, 0] - np.sin(th) * U0[:, 1]
    ey = np.sin(th) * U0[:, 0] + np.cos(th) * U0[:, 1]
    scale = np.max(np.abs(U0))
    assert np.max(np.abs(U1[:, 0] - ex)) / scale < TOL_STEP
    assert np.max(np.abs(U1[:, 1] - ey)) / scale < TOL_STEP
    assert np.max(np.abs(U1[:, 2] - U0[:, 2])) < 1e-6
    sim.close()


def test_gpu_entrance_ramp_leaves_no_transverse_drift():
    # The GPU path against the closed form (no oracle): zero-weight electrons of the long
    # undulator's beam meet the undulator with u_x = 0; past a one-period linear ramp their
    # canonical drift P = u_x - K sin(k_u z_lab) vanishes for any entrance phase, past a sudden
    # entrance it is -K sin(theta) up to the leap-frog error of the jump.
    w = W.long_undulator(grid=(16, 16, 64), n_beam=4)
    K, lam = w.undulator.K, w.undulator.lambda_u
    gR, dz, dt = w.gamma_R, w.d[2], w.dt
    ku = 2 * math.pi / lam
    gB = 2000.0
    bB = math.sqrt(1 - 1 / gB ** 2)
    bR = math.sqrt(1 - 1 / gR ** 2)
    vp = (bB - bR) / (1 - bB * bR)
    for theta in (math.pi / 2, 0.3 + 2 * math.pi, 4.0):
        for ramp in (lam, 0.0):
            sim = api.Sim((16, 16, 64), w.d, dt, gR, bc=((0, 0),) * 3, order=2)
            zs = theta / ku
            sim.set_external_field(K, lam, 0.0, zs, ramp)
            x = np.zeros((3, 3))
            x[0] = [0.0, 0.3, -0.2]
            u = np.zeros((3, 3))
            u[2] = math.sqrt(gB * gB - 1)
            sid = sim.load_species(-1.0, 1.0, x, u, np.zeros(3), frame=api.PIC_FRAME_LAB, origin=(8.0, 8.0, 10.0))
            P0 = _by_id(sim.get_particles(sid))
            z0 = (P0["cell"][:, 2] + P0["off"][:, 2]).min()
            n = int(((zs + ramp) / gR - z0 * dz) / ((vp + bR) * dt)) + 20
            sim.step(n)
            A = _by_id(sim.get_particles(sid))
            sim.step(1)
            Bp = _by_id(sim.get_particles(sid))
            zc = A["cell"][:, 2].astype(np.float64) + A["off"][:, 2]
            zlab = gR * (zc * dz + bR * n * dt)
            P = 0.5 * (A["u"][:, 0].astype(np.float64) + Bp["u"][:, 0]) - K * np.sin(ku * zlab)
            if ramp > 0:
                assert np.all(np.abs(P) < 5e-3 * K), (theta, P / K)
            else:
                assert np.all(np.abs(P + K * math.sin(theta)) < 0.05 * K), (theta, P / K)
            sim.close()


# ------------------------------------------------------------------ degenerate and handover cases

def test_empty_species_steps_as_vacuum():
    # a context whose only particle species is empty (loaded with n = 0) steps as the vacuum
    # FDTD, which the oracle (no species at all) computes; the species stays empty
    w = W.mini_vacuum(order=2)
    sim, _ = api.from_workload(w, beam=False)
    sid = sim.load_species(-1.0, 1.0, None, None, None, frame=api.PIC_FRAME_LAB, origin=w.beam.origin)
    _random_fields(sim, w, seed=11)
    o = oracle.Sim(w.grid, w.d, w.dt, w.gamma_R, bc=w.bc, order=w.order)
    for c in range(6):
        o.set_field(c, sim.get_field(c).astype(np.float64))
    sim.step(3)
    sim.sync()
    o.step(3)
    assert sim.get_count(sid) == 0
    f = parity.compare_fields(sim, o)
    assert max(f.values()) < TOL_STEP, f
    sim.close()


def test_identical_state_after_gpu_steps_with_cpml_and_window():
    # The plasma buncher case after 9 GPU steps (window shift, injected planes) is handed to the
    # oracle for one more step (no window shift falls on it).  The CPML's auxiliary (psi) state is
    # not exported: the oracle restarts it at zero.  That changes E and B inside the absorbing
    # layers and, through the three sub-steps of one update (B half, E, B half), at most two
    # cells beyond them.  The particles (pushed with the exported E^n, B^n) and the currents are
    # compared everywhere, E and B three cells clear of the layers.
    w = W.mini_plasma()
    sim, ids = api.from_workload(w)
    _random_fields(sim, w, seed=7)
    sim.step(9)
    sim.sync()
    o, oid = parity.oracle_from_gpu(w, sim, ids)
    sim.step(1)
    sim.sync()
    o.step(1)
    for name in ids:
        r = parity.compare_species(w, sim, ids[name], o, oid[name])
        assert r["cell_mismatch"] == 0 and r["u_rel_err"] < TOL_STEP, (name, r)
    m = w.pml + 3
    keep = tuple(slice(m, w.grid[d] - m) if w.bc[d][0] == W.PML else slice(None) for d in (2, 1, 0))
    f = parity.compare_fields(sim, o, comps=range(6, 9))
    for c in range(6):
        f[c] = parity.rel_err(sim.get_field(c).astype(np.float64)[keep], o.field(c)[keep])
    assert max(f.values()) < TOL_STEP, f
    sim.close()


# ------------------------------------------------------------------ host-side fault injection

def test_nan_momentum_is_reported_through_the_error_word():
    # the push turns the particle into a dummy and raises the device error word; pic_sync
    # reports PIC_ERR_DEVICE naming the cause, and the context can still be destroyed
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
    # an allocator that refuses the k-th request, for every k pic_create makes: PIC_ERR_ALLOC, no
    # context, and every buffer obtained before the refusal handed back
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


# ------------------------------------------------------------------ autograd wrapper

def _k_rrf(w):
    return api.rrf_resonant_wavenumber(w)


def test_torch_autograd_wrapper_gives_the_adjoint():
    # api.bunching_loss runs the differentiated run through torch.autograd: its loss and
    # gradients are pic_backward's (checked against the oracle in test_gpu_adjoint.py), up to
    # FP32 run-to-run rounding
    torch = pytest.importorskip("torch")
    w = W.mini_adjoint()
    sim, ids = api.from_workload(w)
    sim.checkpoint(10)
    sim.step(w.steps)
    g = sim.backward(ids["beam"], _k_rrf(w))
    sim.close()
    K = torch.tensor(w.undulator.K, dtype=torch.float64, requires_grad=True)
    prof = torch.tensor(w.plasma.n_nodes, dtype=torch.float64, requires_grad=True)
    loss = api.bunching_loss(w, K, prof, checkpoint_every=10, k_bunch=_k_rrf(w))
    loss.backward()
    assert loss.item() == pytest.approx(g["loss"], rel=1e-4)
    assert K.grad.item() == pytest.approx(g["dL_dK"], rel=2e-3)
    scale = np.max(np.abs(g["dL_dprofile"]))
    assert np.max(np.abs(prof.grad.numpy() - g["dL_dprofile"])) < 2e-3 * scale
