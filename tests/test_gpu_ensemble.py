"""Batched ensembles on the GPU: independent runs of uneven beam size, undulator K and plasma
density stacked in one context (one launch per kernel for all runs), against the FP64 oracle
run by run and against separate single-run contexts.

Tolerances as in test_gpu_parity.py: one step from an identical state within 1e-5 relative per
component and per run (cells bit-exact away from ties; the plasma electrons' momenta by their
per-particle vector error, see compare_species; currents and the fields they drive against the
largest single-species current, see current_scale); separate contexts vs the ensemble within
1e-4 relative after 12 steps (two FP32 runs whose reductions differ in order and scale); whole-run beam diagnostics per run
within 1e-3 of the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2411_04703_gb300 import api, workloads as W

import parity

pytestmark = pytest.mark.gpu

TOL_STEP = 1e-5
TOL_MULTI = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    oracle.build()


def _random_fields(sim, seed, amp=1e-3):
    rng = np.random.default_rng(seed)
    for c in range(6):
        sim.set_field(c, (amp * rng.standard_normal((sim.grid[2], sim.grid[1], sim.grid[0]))).astype(np.float32))


def test_ensemble_one_step_per_run_matches_oracle():
    e = W.mini_ensemble()
    sim, ids = api.from_ensemble(e)
    _random_fields(sim, 3)
    nzr = e.base.grid[2]
    oracles = [parity.oracle_from_gpu_run(e, sim, ids, r) for r in range(e.runs)]
    scales = [parity.current_scale(W.ensemble_run(e, r), {n: parity.run_particles(sim, ids[n], r, nzr) for n in ids})
              for r in range(e.runs)]
    sim.step(1)
    sim.sync()
    for r, (o, oid) in enumerate(oracles):
        o.step(1)
        for name in ids:
            res = parity.compare_species_run(e, sim, ids[name], o, oid[name], r)
            assert res["n"] > 0, (r, name)
            assert res["only_gpu"] == 0 and res["only_oracle"] == 0, (r, name, res)
            assert res["cell_mismatch"] == 0, (r, name, res)
            assert res["u_vec_rel_err"] < TOL_STEP, (r, name, res)
            if name == "beam":
                # per component too; the lab-static plasma's transverse momentum is the FP32
                # residual of cancelling undulator forces, so only its vector error is meaningful
                assert res["u_rel_err"] < TOL_STEP, (r, name, res)
            assert res["pos_abs_err"] < 1e-5, (r, name, res)
        # J_z is the residual of the drifting electrons' and frozen ions' opposite currents: its
        # error (and that of E, which J drives) is measured against one species' current
        f = parity.compare_fields_run(sim, o, r, nzr, j_scale=scales[r], dt=e.base.dt)
        assert max(f.values()) < TOL_STEP, (r, f)


def test_ensemble_runs_are_independent_of_each_other():
    # the ensemble against one single-run context per run, same inputs, across a sort
    e = W.mini_ensemble()
    sim, ids = api.from_ensemble(e)
    nzr = e.base.grid[2]
    steps = 12
    sim.step(steps)
    sim.sync()
    for r in range(e.runs):
        w = W.ensemble_run(e, r)
        one, oids = api.from_workload(w)
        one.step(steps)
        one.sync()
        gs = [sim.get_field(c)[r * nzr:(r + 1) * nzr].astype(np.float64) for c in range(9)]
        ss = [one.get_field(c).astype(np.float64) for c in range(9)]
        for c in range(9):
            # two FP32 runs that differ in the order of float atomics and in the fixed-point scale
            # of the current (the ensemble's bound spans every run) drift apart by rounding over
            # 12 steps, measured against the largest component of the same field (a component
            # that is nearly zero carries only that rounding); a current or field leaking between
            # runs would be O(1)
            grp = range(3 * (c // 3), 3 * (c // 3) + 3)
            floor = max(float(np.max(np.abs(ss[q]))) for q in grp)
            assert parity.rel_err_scaled(gs[c], ss[c], floor) < TOL_MULTI, (r, c)
        for name, keys in (("beam", ("mean_z", "rms_z", "mean_gamma", "emit_nx", "field_energy")),
                           ("plasma_e", ("mean_z", "rms_z", "mean_gamma"))):
            mr = sim.get_moments_run(ids[name], r, api.PIC_FRAME_BOOSTED, k_bunch=1.0)
            m1 = one.get_moments(oids[name], api.PIC_FRAME_BOOSTED, k_bunch=1.0)
            assert mr["count"] == m1["count"], (r, name)
            for key in keys:
                assert mr[key] == pytest.approx(m1[key], rel=TOL_MULTI, abs=1e-12), (r, name, key)
        one.close()


def test_ensemble_whole_run_tracks_oracle_per_run():
    # every run loaded independently on each side from the same lab-frame arrays, 20 steps
    e = W.mini_ensemble()
    sim, ids = api.from_ensemble(e)
    sim.step(e.base.steps)
    sim.sync()
    for r in range(e.runs):
        w = W.ensemble_run(e, r)
        o = oracle.Sim(w.grid, w.d, w.dt, w.gamma_R, bc=w.bc, order=w.order)
        o.set_external(w.undulator.K, w.undulator.lambda_u)
        se = o.add_species(-1.0, 1.0)
        si = o.add_species(1.0, 1836.15267343, frozen=True)
        p = w.plasma
        o.set_plasma(se, si, p.ppc, p.xrange, p.z_nodes, p.n_nodes)
        x, u, wt = W.sample_beam(w)
        sb = o.add_species(-1.0, 1.0, capacity=x.shape[1])
        o.load(sb, x, u, wt, frame=oracle.LAB, origin=w.beam.origin, match_undulator=True)
        o.step(w.steps)
        # bunching at the run's own resonant wavenumber (its K) in each frame
        un = w.undulator
        kb = {api.PIC_FRAME_BOOSTED: api.resonant_wavenumber(un.lambda_u, un.K, w.beam.gamma, w.gamma_R,
                                                             api.PIC_FRAME_BOOSTED),
              api.PIC_FRAME_LAB: api.resonant_wavenumber(un.lambda_u, un.K, w.beam.gamma)}
        for frame, oframe in ((api.PIC_FRAME_BOOSTED, 0), (api.PIC_FRAME_LAB, 1)):
            mg = sim.get_moments_run(ids["beam"], r, frame, k_bunch=kb[frame])
            mo = o.moments(sb, frame=oframe, k=kb[frame])
            assert mg["count"] == mo["count"]
            for key in ("emit_nx", "emit_ny", "rel_energy_spread", "mean_gamma", "rms_z", "mean_z", "bunching"):
                assert mg[key] == pytest.approx(mo[key], rel=1e-3), (r, frame, key)
        assert sim.get_moments_run(ids["plasma_e"], r)["count"] == o.count(se)


def test_autotuner_picks_a_cadence_and_keeps_physics():
    # the trials are real steps: the run advances by their total and still tracks a twin context
    # that steps the same number of times with the default cadence (ensemble diagnostics per run
    # within 1e-3, the long-run tolerance)
    e = W.mini_ensemble()
    sim, ids = api.from_ensemble(e)
    twin, tids = api.from_ensemble(e)
    se = sim.autotune(8)
    assert se in (1, 2, 3, 4, 6, 8)
    n = sim.get_time()[0]
    assert n >= 2 * 6 * 32
    twin.step(n)
    sim.sync()
    twin.sync()
    for r in range(e.runs):
        for frame in (api.PIC_FRAME_BOOSTED, api.PIC_FRAME_LAB):
            ma = sim.get_moments_run(ids["beam"], r, frame, k_bunch=1.0)
            mb = twin.get_moments_run(tids["beam"], r, frame, k_bunch=1.0)
            assert ma["count"] == mb["count"]
            for key in ("mean_gamma", "rel_energy_spread", "emit_nx", "emit_ny", "rms_z", "field_energy"):
                assert ma[key] == pytest.approx(mb[key], rel=1e-3), (r, frame, key)


def test_tile_autotuner_picks_a_tile_and_cadence_and_keeps_physics():
    # the tile is tuned together with the cadence: the first candidate is the compiled 8^3
    # region, the others the runtime-sized region; the run then tracks a twin that kept the
    # default tuning for as many steps (per-run diagnostics within 1e-3)
    e = W.mini_ensemble()
    sim, ids = api.from_ensemble(e)
    twin, tids = api.from_ensemble(e)
    cands = ((8, 8, 8), (8, 8, 4), (4, 4, 4))
    # (a short cadence search keeps the run near the length of the cadence test above: the twins
    # drift apart by FP32 summation order, which grows with the steps)
    tile, se = sim.autotune_tiles(cands, max_sort_every=2)
    assert tile in cands and se in (1, 2)
    n = sim.get_time()[0]
    assert n >= 2 * len(cands) * 32
    twin.step(n)
    sim.sync()
    twin.sync()
    for r in range(e.runs):
        for frame in (api.PIC_FRAME_BOOSTED, api.PIC_FRAME_LAB):
            ma = sim.get_moments_run(ids["beam"], r, frame, k_bunch=1.0)
            mb = twin.get_moments_run(tids["beam"], r, frame, k_bunch=1.0)
            assert ma["count"] == mb["count"]
            for key in ("mean_gamma", "rel_energy_spread", "emit_nx", "emit_ny", "rms_z", "field_energy"):
                assert ma[key] == pytest.approx(mb[key], rel=1e-3), (r, frame, key)
    with pytest.raises(api.PicError, match="tile"):
        sim.autotune_tiles(((8, 8, 8), (32, 8, 8)))
