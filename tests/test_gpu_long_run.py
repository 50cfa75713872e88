"""Long-run parity of the ensemble diagnostics: the vacuum-undulator workload at full size
(32 x 32 x 64 periodic grid, 65,536 beam electrons, CIC, K = 1, gamma_R = 10), 200 steps on
the GPU (FP32 state) and in the FP64 oracle, each loading the same seeded lab-frame beam and
transforming it into the RRF on its own.

Tolerance: the bunching factor at the lab resonant wavenumber (Eq. RadLambda) and at its RRF
image, the normalised emittances and the relative energy spread agree to 1e-3 relative after
the whole run, in both frames; the particle count is exact.
"""
import numpy as np
import pytest

import oracle
from paper_2411_04703_gb300 import api, workloads as W

pytestmark = pytest.mark.gpu

TOL_DIAG = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    oracle.build()


def test_vacuum_undulator_200_steps_diagnostics_track_oracle():
    w = W.vacuum_undulator()
    x, u, wt = W.sample_beam(w)
    sim, ids = api.from_workload(w, beam_arrays=(x, u, wt))
    o = oracle.Sim(w.grid, w.d, w.dt, w.gamma_R, bc=w.bc, order=w.order)
    o.set_external(w.undulator.K, w.undulator.lambda_u)
    s = o.add_species(-1.0, 1.0, capacity=x.shape[1])
    o.load(s, x, u, wt, frame=oracle.LAB, origin=w.beam.origin, match_undulator=True)
    sim.step(w.steps)
    sim.sync()
    o.step(w.steps)
    assert sim.get_time()[0] == o.time()[0] == w.steps
    k_lab = api.resonant_wavenumber(w.undulator.lambda_u, w.undulator.K, w.beam.gamma)
    # RRF image of the lab resonant wavenumber for a structure moving with the beam (mean lab
    # velocity beta_z): its period is stretched by 1 / (gamma_R (1 - beta_z beta_R)), the beam
    # elongation of Eq. Belon, so k' = k_r gamma_R (1 - beta_z beta_R)
    mo_b = o.moments(s, frame=0, k=0.0)
    gR = w.gamma_R
    bR = np.sqrt(1 - 1 / gR ** 2)
    mo_lab0 = o.moments(s, frame=1, k=0.0)
    bz = mo_lab0["mean_uz"] / mo_lab0["mean_gamma"]
    k_rrf = k_lab * gR * (1 - bz * bR)
    for frame, oframe, k in [(api.PIC_FRAME_LAB, 1, k_lab), (api.PIC_FRAME_BOOSTED, 0, k_rrf)]:
        mg = sim.get_moments(ids["beam"], frame, k_bunch=k)
        mo = o.moments(s, frame=oframe, k=k)
        assert mg["count"] == mo["count"] == w.beam.n
        for key in ["bunching", "emit_nx", "emit_ny", "rel_energy_spread", "mean_gamma", "rms_z"]:
            assert mg[key] == pytest.approx(mo[key], rel=TOL_DIAG), (frame, key, mg[key], mo[key])
    assert mo_b["count"] == w.beam.n
    # the fields the beam radiated agree too (whole-grid energy)
    assert sim.get_moments(ids["beam"])["field_energy"] == pytest.approx(o.moments(s)["field_energy"], rel=TOL_DIAG)


def test_plasma_buncher_300_steps_diagnostics_track_oracle():
    # The plasma-buncher physics (boost 20, lab gamma 400 beam in a cold lab-static plasma with
    # frozen neutralising ions, TSC, transverse CPML, moving window with plasma injection) on the
    # oracle-sized grid 28 x 26 x 52 (5 um longitudinal cells: the window shifts ~50 times in 300
    # steps).  Both sides load the same seeded lab beam and fill the same plasma lattice; after 300
    # steps the beam's bunching (at the plasma wavenumber of the normalised units, k = 1, and at
    # twice it), emittances and energy spread agree to 1e-3 in both frames, and the plasma
    # electron count is exact.
    import os
    w = W.mini_plasma(steps=300)
    x, u, wt = W.sample_beam(w)
    sim, ids = api.from_workload(w, beam_arrays=(x, u, wt))
    o = oracle.Sim(w.grid, w.d, w.dt, w.gamma_R, bc=w.bc, pml=w.pml, order=w.order,
                   moving_window=w.moving_window, window_v=w.window_v)
    o.set_threads(os.cpu_count() or 1)
    se = o.add_species(-1.0, 1.0)
    si = o.add_species(1.0, 1836.15267343, frozen=True)
    sb = o.add_species(-1.0, 1.0, capacity=x.shape[1])
    p = w.plasma
    o.set_plasma(se, si, p.ppc, p.xrange, p.z_nodes, p.n_nodes)
    o.load(sb, x, u, wt, frame=oracle.LAB, origin=w.beam.origin)
    sim.step(w.steps)
    sim.sync()
    o.step(w.steps)
    assert sim.get_time() == o.time()
    assert sim.get_time()[1] >= 40          # the window moved through the plasma
    assert sim.get_count(ids["plasma_e"]) == o.count(se)
    for frame, oframe in ((api.PIC_FRAME_BOOSTED, 0), (api.PIC_FRAME_LAB, 1)):
        for k in (1.0, 2.0):
            mg = sim.get_moments(ids["beam"], frame, k_bunch=k)
            mo = o.moments(sb, frame=oframe, k=k)
            assert mg["count"] == mo["count"]
            for key in ("bunching", "emit_nx", "emit_ny", "rel_energy_spread"):
                assert mg[key] == pytest.approx(mo[key], rel=TOL_DIAG), (frame, k, key, mg[key], mo[key])
    sim.close()


def test_plasma_buncher_after_the_tile_autotuner_tracks_oracle():
    # The same plasma-buncher physics, with the tile size and sort cadence chosen by
    # pic_autotune_tiles on the GPU run itself: its trial steps (several hundred, each candidate
    # re-tiling the species, with window shifts and plasma injection) are real steps, and the
    # oracle takes as many from the same initial state; the beam's diagnostics in both frames agree
    # to 1e-3 and the plasma electron count is exact.
    import os
    w = W.mini_plasma(steps=300)
    x, u, wt = W.sample_beam(w)
    sim, ids = api.from_workload(w, beam_arrays=(x, u, wt))
    o = oracle.Sim(w.grid, w.d, w.dt, w.gamma_R, bc=w.bc, pml=w.pml, order=w.order,
                   moving_window=w.moving_window, window_v=w.window_v)
    o.set_threads(os.cpu_count() or 1)
    se = o.add_species(-1.0, 1.0)
    si = o.add_species(1.0, 1836.15267343, frozen=True)
    sb = o.add_species(-1.0, 1.0, capacity=x.shape[1])
    p = w.plasma
    o.set_plasma(se, si, p.ppc, p.xrange, p.z_nodes, p.n_nodes)
    o.load(sb, x, u, wt, frame=oracle.LAB, origin=w.beam.origin)
    cands = ((8, 8, 8), (4, 4, 4))
    tile, se_ = sim.autotune_tiles(cands, max_sort_every=2)
    assert tile in cands and se_ in (1, 2)
    n = sim.get_time()[0]
    sim.sync()
    o.step(n)
    assert sim.get_time() == o.time()
    assert n >= 4 * 32 and sim.get_time()[1] >= 30     # the window moved through the plasma
    assert sim.get_count(ids["plasma_e"]) == o.count(se)
    for frame, oframe in ((api.PIC_FRAME_BOOSTED, 0), (api.PIC_FRAME_LAB, 1)):
        mg = sim.get_moments(ids["beam"], frame, k_bunch=1.0)
        mo = o.moments(sb, frame=oframe, k=1.0)
        assert mg["count"] == mo["count"]
        for key in ("bunching", "emit_nx", "emit_ny", "rel_energy_spread"):
            assert mg[key] == pytest.approx(mo[key], rel=TOL_DIAG), (frame, key, mg[key], mo[key])
    sim.close()
