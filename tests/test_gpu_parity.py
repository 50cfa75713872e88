"""GPU (sm_103a, through the C-ABI) against the FP64 oracle on the same seeded inputs.

Tolerances: integer cell indices and the sort are bit-exact (particles within 1e-5 cell of a
face are counted as ties and excluded, see the tie reading); fields and momenta after one step
from an identical state within 1e-5 relative (max|gpu - ref| / max|ref| per component);
FP64 diagnostics computed from an identical FP32 state within 1e-9 relative.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2411_04703_gb300 import api, workloads as W

import parity

pytestmark = pytest.mark.gpu

TOL_STEP = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    oracle.build()


def random_fields(sim, w, seed, amp=1e-3):
    rng = np.random.default_rng(seed)
    for c in range(6):
        sim.set_field(c, (amp * rng.standard_normal((w.grid[2], w.grid[1], w.grid[0]))).astype(np.float32))


def _und3d(w):
    # the planar undulator with its cosh/sinh transverse dependence (PIC_EXT_PLANAR_UNDULATOR_3D)
    w.undulator.kind = 2
    return w


@pytest.mark.parametrize("kind", [1, 2])
def test_lab_to_boosted_load_matches_oracle(kind):
    # the matched load uses A_x of the field kind (times cosh(k_u y) off axis for kind 2)
    w = W.mini_vacuum(order=1)
    w.undulator.kind = kind
    x, u, wt = W.sample_beam(w)
    sim, ids = api.from_workload(w, beam_arrays=(x, u, wt))
    o = oracle.Sim(w.grid, w.d, w.dt, w.gamma_R, bc=w.bc, order=w.order)
    o.set_external(w.undulator.K, w.undulator.lambda_u, kind=kind)
    s = o.add_species(-1.0, 1.0, capacity=x.shape[1])
    o.load(s, x, u, wt, frame=oracle.LAB, origin=w.beam.origin, match_undulator=True)
    r = parity.compare_species(w, sim, ids["beam"], o, s)
    assert r["only_gpu"] == 0 and r["only_oracle"] == 0
    assert r["cell_mismatch"] == 0
    assert r["pos_abs_err"] < 1e-6
    assert r["u_rel_err"] < 1e-6


CASES = {
    "vacuum_cic": lambda: W.mini_vacuum(order=1),
    "vacuum_tsc": lambda: W.mini_vacuum(order=2),
    "plasma_tsc_pml_window": lambda: W.mini_plasma(),
    "long_undulator_tsc_pml_ramp": lambda: W.mini_long_undulator(),
    "vacuum_tsc_undulator_3d": lambda: _und3d(W.mini_vacuum(order=2)),
    "long_undulator_3d_pml_ramp": lambda: _und3d(W.mini_long_undulator()),
    "plasma_2d_tsc_pml_window": lambda: W.mini_plasma_2d(),
    "dense_bunch_cic": lambda: W.mini_dense_bunch(order=1),
    "dense_bunch_tsc": lambda: W.mini_dense_bunch(order=2),
}


@pytest.mark.parametrize("case", list(CASES))
def test_one_step_from_identical_state(case):
    w = CASES[case]()
    sim, ids = api.from_workload(w)
    random_fields(sim, w, seed=hash(case) % 1000)
    o, oid = parity.oracle_from_gpu(w, sim, ids)
    sim.step(1)
    sim.sync()
    o.step(1)
    for name in ids:
        r = parity.compare_species(w, sim, ids[name], o, oid[name])
        assert r["only_gpu"] == 0 and r["only_oracle"] == 0, (name, r)
        assert r["cell_mismatch"] == 0, (name, r)
        assert r["u_rel_err"] < TOL_STEP, (name, r)
        assert r["pos_abs_err"] < 1e-5, (name, r)
    f = parity.compare_fields(sim, o)
    for k in ["Ex", "Ey", "Ez", "Bx", "By", "Bz"]:
        assert f[k] < TOL_STEP, (k, f)
    for k in ["Jx", "Jy", "Jz"]:
        assert f[k] < TOL_STEP, (k, f)


@pytest.mark.parametrize("tile", [(8, 4, 4), (4, 4, 4), (8, 8, 4)])
@pytest.mark.parametrize("case", ["vacuum_cic", "plasma_tsc_pml_window", "dense_bunch_tsc"])
def test_one_step_on_other_tiles_from_identical_state(case, tile):
    # tiles other than 8^3 run the particle kernel's runtime-sized region (what the tile
    # autotuner can choose): the same per-step bar against the oracle
    w = CASES[case]()
    sim, ids = api.from_workload(w, tuning={"tile": tile, "sort_every": 4, "margin": 1})
    random_fields(sim, w, seed=17)
    sim.sort()
    o, oid = parity.oracle_from_gpu(w, sim, ids)
    sim.step(1)
    sim.sync()
    o.step(1)
    for name in ids:
        r = parity.compare_species(w, sim, ids[name], o, oid[name])
        assert r["only_gpu"] == 0 and r["only_oracle"] == 0 and r["cell_mismatch"] == 0, (name, r)
        assert r["u_rel_err"] < TOL_STEP, (name, r)
    f = parity.compare_fields(sim, o)
    assert max(f.values()) < TOL_STEP, f


@pytest.mark.parametrize("case", ["vacuum_cic", "vacuum_tsc", "plasma_tsc_pml_window", "plasma_2d_tsc_pml_window"])
def test_one_step_energy_conserving_gather_from_identical_state(case):
    # the energy-conserving gather (one order lower along each component's staggered dims)
    w = CASES[case]()
    sim, ids = api.from_workload(w)
    sim.set_gather(api.PIC_GATHER_ENERGY)
    random_fields(sim, w, seed=43)
    o, oid = parity.oracle_from_gpu(w, sim, ids)
    o.set_gather(1)
    sim.step(1)
    sim.sync()
    o.step(1)
    for name in ids:
        r = parity.compare_species(w, sim, ids[name], o, oid[name])
        assert r["only_gpu"] == 0 and r["only_oracle"] == 0 and r["cell_mismatch"] == 0, (name, r)
        assert r["u_rel_err"] < TOL_STEP, (name, r)
    f = parity.compare_fields(sim, o)
    assert max(f.values()) < TOL_STEP, f
    # and it is not the momentum-conserving result (the random fields vary on the grid scale)
    sim2, ids2 = api.from_workload(w)
    random_fields(sim2, w, seed=43)
    sim2.step(1)
    sim2.sync()
    key = "beam" if "beam" in ids else "plasma_e"
    du = np.max(np.abs(sim.get_particles(ids[key])["u"] - sim2.get_particles(ids2[key])["u"]))
    assert du > 0.0


@pytest.mark.parametrize("case", ["vacuum_tsc", "plasma_tsc_pml_window"])
def test_one_step_vay_pusher_from_identical_state(case):
    w = CASES[case]()
    sim, ids = api.from_workload(w)
    sim.set_pusher(api.PIC_PUSHER_VAY)
    random_fields(sim, w, seed=31)
    o, oid = parity.oracle_from_gpu(w, sim, ids)
    o.set_pusher(1)
    sim.step(1)
    sim.sync()
    o.step(1)
    for name in ids:
        r = parity.compare_species(w, sim, ids[name], o, oid[name])
        assert r["only_gpu"] == 0 and r["only_oracle"] == 0 and r["cell_mismatch"] == 0, (name, r)
        assert r["u_rel_err"] < TOL_STEP, (name, r)
    f = parity.compare_fields(sim, o)
    assert max(f.values()) < TOL_STEP, f


def test_vay_keeps_the_lab_static_plasma_at_rest_in_the_undulator():
    # in the RRF a lab-static plasma drifts at -beta_R through E'_x = -beta_R B'_y: the force
    # vanishes.  Boris leaves a spurious transverse momentum; Vay's pusher only FP32 rounding.
    e = W.mini_ensemble()
    ux = {}
    for pusher in (api.PIC_PUSHER_BORIS, api.PIC_PUSHER_VAY):
        sim, ids = api.from_ensemble(e, beam=False)
        sim.set_pusher(pusher)
        sim.step(20)
        ux[pusher] = float(np.max(np.abs(sim.get_particles(ids["plasma_e"])["u"][:, 0])))
        sim.close()
    assert ux[api.PIC_PUSHER_BORIS] > 1e-7, ux
    assert ux[api.PIC_PUSHER_VAY] < 0.1 * ux[api.PIC_PUSHER_BORIS], ux


def test_identical_state_after_gpu_steps():
    # run the GPU alone, then hand its state to the oracle and compare one more step
    w = CASES["vacuum_cic"]()
    sim, ids = api.from_workload(w)
    random_fields(sim, w, seed=7)
    sim.step(9)
    sim.sync()
    o, oid = parity.oracle_from_gpu(w, sim, ids)
    sim.step(1)
    sim.sync()
    o.step(1)
    for name in ids:
        r = parity.compare_species(w, sim, ids[name], o, oid[name])
        assert r["cell_mismatch"] == 0 and r["u_rel_err"] < TOL_STEP, (name, r)
    f = parity.compare_fields(sim, o)
    assert max(f.values()) < TOL_STEP, f


@pytest.mark.parametrize("case", list(CASES))
def test_whole_run_tracks_oracle(case):
    # same initial state, 20 steps each: FP32 drift stays far below the ensemble tolerance
    w = CASES[case]()
    sim, ids = api.from_workload(w)
    o, oid = parity.oracle_from_gpu(w, sim, ids)
    sim.step(20)
    sim.sync()
    o.step(20)
    assert sim.get_time() == o.time()
    for name in ids:
        r = parity.compare_species(w, sim, ids[name], o, oid[name])
        assert r["only_gpu"] + r["only_oracle"] <= max(2, r["ties"]), (name, r)
        assert r["u_rel_err"] < 1e-3, (name, r)
    if "beam" in ids:
        for frame in (api.PIC_FRAME_BOOSTED, api.PIC_FRAME_LAB):
            mg = sim.get_moments(ids["beam"], frame, k_bunch=1.0)
            mo = o.moments(oid["beam"], frame=0 if frame == api.PIC_FRAME_BOOSTED else 1, k=1.0)
            for key in ["emit_nx", "emit_ny", "rel_energy_spread", "rms_z", "mean_gamma"]:
                assert mg[key] == pytest.approx(mo[key], rel=1e-3), (frame, key)


def test_long_undulator_entry_through_the_ramp_tracks_oracle():
    # The long undulator's bunch in front of the undulator at t' = 0 (its entrance two cells past
    # the bunch's 3-sigma head), through the one-period ramp until the whole bunch is inside: the
    # same initial state on both sides, then the GPU and the oracle step on their own (self fields
    # of a bunch of 1e-3 of the workload's charge, CPML on every face); the bunch's momenta and
    # diagnostics in both frames agree within the ensemble tolerance, no particle is lost, and the
    # bunch ends up oscillating in the field.
    import math
    import os
    grid = (48, 40, 96)
    w = W.long_undulator(grid=grid, n_beam=4000, steps=200, pml=4, name="long undulator entry 48x40x96")
    w.beam.sigma_r = 3.0 * w.d[0]
    w.beam.weight *= 1e-3
    w.beam.origin = (24.0, 20.0, 40.0)
    sig = grid[2] / 12.0                        # RRF bunch length (cells) before the entrance
    un, b = w.undulator, w.beam
    gR = w.gamma_R
    un.z_start = gR * (b.origin[2] + 3 * sig + 2) * w.d[2]
    bR, bB = math.sqrt(1 - 1 / gR ** 2), math.sqrt(1 - 1 / b.gamma ** 2)
    vp = (bB - bR) / (1 - bB * bR)              # RRF velocity before the entrance
    n = int(math.ceil(((un.z_start + un.ramp) / gR - (b.origin[2] - 3 * sig) * w.d[2]) / ((bR + vp) * w.dt))) + 10
    sim, ids = api.from_workload(w)
    o, oid = parity.oracle_from_gpu(w, sim, ids)
    o.set_threads(os.cpu_count() or 1)
    n0 = sim.get_count(ids["beam"])
    sim.step(n)
    sim.sync()
    o.step(n)
    assert sim.get_count(ids["beam"]) == n0 == o.count(oid["beam"])
    r = parity.compare_species(w, sim, ids["beam"], o, oid["beam"])
    assert r["only_gpu"] + r["only_oracle"] <= max(2, r["ties"]), r
    assert r["u_rel_err"] < 1e-3, r
    for frame in (api.PIC_FRAME_BOOSTED, api.PIC_FRAME_LAB):
        mg = sim.get_moments(ids["beam"], frame, k_bunch=1.0)
        mo = o.moments(oid["beam"], frame=0 if frame == api.PIC_FRAME_BOOSTED else 1, k=1.0)
        for key in ["emit_nx", "emit_ny", "rel_energy_spread", "rms_z", "mean_gamma"]:
            assert mg[key] == pytest.approx(mo[key], rel=1e-3), (frame, key)
        assert abs(mg["mean_ux"] - mo["mean_ux"]) < 1e-3 * un.K, frame
    ux = sim.get_particles(ids["beam"])["u"][:, 0]
    assert np.sqrt(np.mean(ux.astype(np.float64) ** 2)) > 0.5 * un.K   # inside the field


PML_CASES = ["plasma_tsc_pml_window", "long_undulator_tsc_pml_ramp"]


@pytest.mark.parametrize("case", PML_CASES)
def test_cpml_layers_track_oracle_over_steps(case):
    # Random fields everywhere, the absorbing layers included, and auxiliary CPML state zero on
    # both sides: after the first step the layers' psi is nonzero, so steps 2 and 3 exercise the
    # b psi recursion term.  All nodes of E and B, layers included, are compared after 3 steps at
    # the per-step tolerance (three steps of FP32 rounding stay well inside it), and after 20 steps
    # within 1e-4 (FP32 drift of the fields and particles over 20 steps).
    w = CASES[case]()
    sim, ids = api.from_workload(w)
    random_fields(sim, w, seed=101)
    o, oid = parity.oracle_from_gpu(w, sim, ids)
    sim.step(3)
    sim.sync()
    o.step(3)
    f = parity.compare_fields(sim, o)
    for k in ["Ex", "Ey", "Ez", "Bx", "By", "Bz"]:
        assert f[k] < TOL_STEP, (3, k, f)
    # the layers' own nodes: the first/last pml cells of each absorbing dim
    n = w.pml
    for c in range(6):
        g = sim.get_field(c).astype(np.float64)
        r = o.field(c)
        for dd, axis in ((0, 2), (1, 1), (2, 0)):
            if w.bc[dd][0] != W.PML:
                continue
            sl_lo = [slice(None)] * 3
            sl_hi = [slice(None)] * 3
            sl_lo[axis] = slice(0, n)
            sl_hi[axis] = slice(w.grid[dd] - n, w.grid[dd])
            for sl in (tuple(sl_lo), tuple(sl_hi)):
                den = np.max(np.abs(r))
                assert np.max(np.abs(g[sl] - r[sl])) < TOL_STEP * den, (c, dd)
                assert np.max(np.abs(r[sl])) > 1e-3 * den      # the layers hold field
    sim.step(17)
    sim.sync()
    o.step(17)
    f = parity.compare_fields(sim, o)
    for k in ["Ex", "Ey", "Ez", "Bx", "By", "Bz"]:
        assert f[k] < 1e-4, (20, k, f)


def test_moments_from_identical_state_match_fp64():
    w = W.mini_vacuum(order=2)
    sim, ids = api.from_workload(w)
    sim.step(3)
    o, oid = parity.oracle_from_gpu(w, sim, ids)
    k_lab = api.resonant_wavenumber(w.undulator.lambda_u, w.undulator.K, w.beam.gamma)
    for frame, oframe, k in [(api.PIC_FRAME_BOOSTED, 0, 0.7), (api.PIC_FRAME_LAB, 1, k_lab)]:
        mg = sim.get_moments(ids["beam"], frame, k_bunch=k)
        mo = o.moments(oid["beam"], frame=oframe, k=k)
        for key, v in mo.items():
            if key == "field_energy":
                assert mg[key] == pytest.approx(v, rel=1e-6)
            elif key == "bunching":
                assert mg[key] == pytest.approx(v, rel=1e-6, abs=1e-9)
            else:
                assert mg[key] == pytest.approx(v, rel=1e-9, abs=1e-12), (frame, key)


def test_tile_sort_is_bit_exact():
    w = W.mini_plasma()
    sim, ids = api.from_workload(w)
    sim.step(3)
    sim.sort()
    for name, sid in ids.items():
        if name == "plasma_i":
            continue   # the frozen ions are held as lattice planes, not sorted records
        P = sim.get_particles(sid)
        X = P["cell"].astype(np.float64) + P["off"].astype(np.float64)
        order, keys = oracle.tile_sort(X, w.grid, w.tile)
        # storage order after the sort is by ascending tile-major key
        gk = keys[np.argsort(order)]
        assert np.all(np.diff(gk) >= 0), name
        # per-key id sets equal those of the oracle's stable sort of the same particles
        ok = keys
        oids = P["id"][order]
        gids = P["id"]
        bounds = np.flatnonzero(np.diff(ok)) + 1
        for a, b in zip(np.r_[0, bounds], np.r_[bounds, len(ok)]):
            assert set(oids[a:b]) == set(gids[a:b])


def test_gauss_law_invariant_on_gpu():
    w = W.mini_vacuum(order=2)
    w.beam.weight *= 1e6   # strong self-fields
    sim, ids = api.from_workload(w)
    d = w.d

    def gauss():
        ex, ey, ez = (sim.get_field(c).astype(np.float64) for c in range(3))
        rho = sim.get_field(api.PIC_RHO).astype(np.float64)
        div = ((ex - np.roll(ex, 1, 2)) / d[0] + (ey - np.roll(ey, 1, 1)) / d[1] + (ez - np.roll(ez, 1, 0)) / d[2])
        return div - rho, np.max(np.abs(rho))

    G0, r0 = gauss()
    for _ in range(5):
        sim.step(4)
        G, r = gauss()
        assert np.max(np.abs(G - G0)) < 1e-4 * r0
    assert np.max(np.abs(sim.get_field(api.PIC_EX))) > 0


def test_moving_window_plasma_lattice_on_gpu():
    w = W.mini_plasma()
    w.beam = None
    sim, ids = api.from_workload(w, beam=False)
    o, oid = parity.oracle_from_gpu(w, sim, ids)
    for _ in range(6):
        sim.step(15)
        o.step(15)
        assert sim.get_time() == o.time()
        for name in ("plasma_e", "plasma_i"):
            P = sim.get_particles(ids[name])
            X, _, _, oids = o.particles(oid[name])
            assert sorted(P["id"].tolist()) == sorted(oids.tolist())
            cg = np.bincount(P["cell"][:, 2], minlength=w.grid[2])
            co = np.bincount(np.floor(X[:, 2]).astype(int), minlength=w.grid[2])
            assert np.array_equal(cg, co)
    assert sim.get_time()[1] > 0   # the window moved


def test_resolution_factor_matches_oracle():
    for w in (W.mini_vacuum(order=1), W.mini_long_undulator()):
        sim, ids = api.from_workload(w, beam=False)
        lam = api.resonant_wavenumber(w.undulator.lambda_u, w.undulator.K, w.beam.gamma)
        lam = 2 * math.pi / lam
        r, ok = sim.resolution_factor(lam)
        ro = oracle.resolution_factor(w.grid[2] * w.d[2], w.grid[2], w.gamma_R)
        assert r == pytest.approx(ro, rel=1e-8)
        assert ok == (ro < lam)
        sim.close()


@pytest.mark.parametrize("case", ["vacuum_tsc", "long_undulator_tsc_pml_ramp"])
def test_artificial_ion_ramp_tracks_oracle(case):
    # the beam compensated by artificial ions at load (fields zero), faded over 3.5 steps; each
    # side computes the ions' density and current itself: one step within 1e-5, five within 1e-4
    w = CASES[case]()
    sim, ids = api.from_workload(w)
    o, oid = parity.oracle_from_gpu(w, sim, ids)
    T = 3.5 * w.dt
    sim.set_ion_ramp(ids["beam"], T)
    o.set_ion_ramp(oid["beam"], T)
    for n, tol in ((1, TOL_STEP), (4, 1e-4)):
        sim.step(n)
        sim.sync()
        o.step(n)
        f = parity.compare_fields(sim, o)
        assert max(f.values()) < tol, (n, f)
    r = parity.compare_species(w, sim, ids["beam"], o, oid["beam"])
    assert r["u_rel_err"] < 1e-4, r


def test_artificial_ion_ramp_keeps_gauss_law_on_gpu():
    w = W.mini_vacuum(order=2)
    w.beam.weight *= 1e6   # strong self-fields
    sim, ids = api.from_workload(w)
    d = w.d
    rho0 = sim.get_field(api.PIC_RHO).astype(np.float64)
    mean = rho0.mean(axis=0, keepdims=True)      # periodic z: the column mean stays as background
    T = 6.5 * w.dt
    sim.set_ion_ramp(ids["beam"], T)
    for n in range(10):
        ex, ey, ez = (sim.get_field(c).astype(np.float64) for c in range(3))
        rho = sim.get_field(api.PIC_RHO).astype(np.float64)
        div = ((ex - np.roll(ex, 1, 2)) / d[0] + (ey - np.roll(ey, 1, 1)) / d[1] + (ez - np.roll(ez, 1, 0)) / d[2])
        f = min(1.0, n * w.dt / T)
        G = div - rho - (-(rho0 - mean) * (1.0 - f) - mean)
        assert np.max(np.abs(G)) < 1e-4 * np.max(np.abs(rho0)), n
        sim.step(1)
    assert np.max(np.abs(sim.get_field(api.PIC_EZ))) > 0


def test_adjoint_refuses_what_it_does_not_differentiate():
    # the artificial ions' current, the energy-conserving gather and the Vay pusher are not
    # reversed by the adjoint: recording is refused with them, and they are refused while recording
    w = W.mini_vacuum(order=1)
    sim, ids = api.from_workload(w)
    sim.set_ion_ramp(ids["beam"], 3.0 * w.dt)
    with pytest.raises(api.PicError, match="artificial ions"):
        sim.checkpoint(10)
    sim.set_ion_ramp(ids["beam"], 0.0)
    sim.set_gather(api.PIC_GATHER_ENERGY)
    with pytest.raises(api.PicError, match="momentum-conserving gather"):
        sim.checkpoint(10)
    sim.set_gather(api.PIC_GATHER_MOMENTUM)
    sim.checkpoint(10)
    with pytest.raises(api.PicError, match="artificial ions"):
        sim.set_ion_ramp(ids["beam"], 3.0 * w.dt)
    with pytest.raises(api.PicError, match="Boris"):
        sim.set_pusher(api.PIC_PUSHER_VAY)
    sim.checkpoint(0)
    sim.close()


def test_lab_snapshot_tracks_oracle():
    # The time-skew reconstruction at one lab time on the GPU against the oracle's: the long
    # undulator case (entrance ramp, PML, TSC), both sides loading the same seeded lab beam; the
    # snapshot time is a little past the latest particle's lab time at load, so every particle
    # records during the following steps.  Records per particle (FP32 drift over the steps) and
    # the snapshot's moments (the long-run tolerance) agree.
    w = W.mini_long_undulator()
    x, u, wt = W.sample_beam(w)
    sim, ids = api.from_workload(w, beam_arrays=(x, u, wt))
    o = oracle.Sim(w.grid, w.d, w.dt, w.gamma_R, bc=w.bc, pml=w.pml, order=w.order)
    un = w.undulator
    o.set_external(un.K, un.lambda_u, un.phase, un.z_start, un.ramp, kind=un.kind)
    sb = o.add_species(-1.0, 1.0, capacity=x.shape[1])
    o.load(sb, x, u, wt, frame=oracle.LAB, origin=w.beam.origin, match_undulator=un.match)
    X, _, _, _ = o.particles(sb)
    bR = o.beta_R
    t_lab = w.gamma_R * bR * X[:, 2] * w.d[2]
    T = float(np.max(t_lab)) + 2.0 * w.gamma_R * w.dt
    sim.lab_snapshot(ids["beam"], T)
    o.snapshot_begin(sb, T)
    for _ in range(60):
        sim.step(5)
        o.step(5)
        _, so = o.snapshot()
        if np.all(so != 0):
            break
    rg, sg = sim.lab_snapshot_read()
    ro, so = o.snapshot()
    assert np.array_equal(sg, so)
    # (the beam's transverse tails start in the absorbing layers of this small grid and leave:
    # those particles never record, on either side)
    assert np.sum(so == 1) > 0.5 * x.shape[1]
    rec = so == 1
    size = np.std(ro[rec, :3], axis=0)
    for c in range(3):
        np.testing.assert_allclose(rg[rec, c] - ro[rec, c], 0.0, atol=1e-4 * size[c])
    for c in range(3, 6):
        np.testing.assert_allclose(rg[rec, c], ro[rec, c], rtol=0, atol=1e-4 * np.max(np.abs(ro[rec, c])))
    k_lab = api.resonant_wavenumber(un.lambda_u, un.K, w.beam.gamma)
    mg = sim.lab_snapshot_moments(k_lab)
    mo = o.snapshot_moments(k_lab)
    assert mg["count"] == mo["count"] and mg["mean_t"] == mo["mean_t"] == T
    for key in ("bunching", "emit_nx", "emit_ny", "rel_energy_spread", "rms_z", "mean_gamma"):
        assert mg[key] == pytest.approx(mo[key], rel=1e-3), key
    sim.lab_snapshot(ids["beam"], float("nan"))
