"""Parity at the full plasma-buncher size (128 x 128 x 512, 4,194,304 beam electrons, 61M plasma
electrons and 61M frozen ions, TSC, CPML, moving window), in the launch configuration bench.py
times.  The oracle cannot run this state whole, so the checks are those it can compute one
unit at a time, and properties that hold at any size:

* the FDTD update of the full grid (oracle run on the GPU's E^n, B^n and J^{n+1/2}),
* the momentum push of a 20,000-particle sample (oracle gather + Boris on the GPU's fields),
* charge continuity rho^{n+1} - rho^n + dt div J = 0 at every node,
* the storage order after the sort (ascending tile/cell/octant key on a sample).
Tolerances as in test_gpu_parity.py (1e-5 relative per step; continuity to FP32 rounding).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2411_04703_gb300 import api, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def state():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    oracle.build()
    w = W.plasma_buncher()
    sim, ids = api.from_workload(w)
    yield w, sim, ids
    sim.close()


def _div(J, d):
    jx, jy, jz = J
    out = (jx - np.pad(jx, ((0, 0), (0, 0), (1, 0)))[:, :, :-1]) / d[0]
    out += (jy - np.pad(jy, ((0, 0), (1, 0), (0, 0)))[:, :-1, :]) / d[1]
    out += (jz - np.pad(jz, ((1, 0), (0, 0), (0, 0)))[:-1, :, :]) / d[2]
    return out


def test_full_size_step_fields_push_and_continuity(state):
    w, sim, ids = state
    assert sim.get_time() == (0, 0, sim.get_time()[2])
    rng = np.random.default_rng(99)
    # random E, B so that the gather and the Boris rotation are exercised (PML auxiliaries
    # still start at zero, so the oracle's field update from the same state is exact)
    for c in range(6):
        sim.set_field(c, (1e-3 * rng.standard_normal((w.grid[2], w.grid[1], w.grid[0]))).astype(np.float32))
    # sampled particles before the step (state n)
    samples = {}
    for name in ("beam", "plasma_e"):
        P = sim.get_particles(ids[name])
        k = rng.choice(len(P["id"]), 10000, replace=False)
        samples[name] = {key: v[k] for key, v in P.items()}
    E0 = [sim.get_field(c).astype(np.float64) for c in range(3)]
    B0 = [sim.get_field(3 + c).astype(np.float64) for c in range(3)]
    rho0 = sim.get_field(api.PIC_RHO).astype(np.float64)
    sim.step(1)
    sim.sync()
    assert sim.get_time()[1] == 0     # no window shift in this step
    J = [sim.get_field(6 + c).astype(np.float64) for c in range(3)]
    rho1 = sim.get_field(api.PIC_RHO).astype(np.float64)
    # continuity at every node: the residual must be FP32 rounding of the species' charge
    # densities (plasma |rho| = gamma_R n_lab), far below one step's transfer of a species
    resid = (rho1 - rho0) / w.dt + _div(J, w.d)
    rho_species = w.gamma_R * max(w.plasma.n_nodes)
    assert np.max(np.abs(resid)) < 1e-5 * rho_species / w.dt
    # FDTD of the whole grid: oracle from E^n, B^n, J (PML auxiliaries start at zero)
    o = oracle.Sim(w.grid, w.d, w.dt, w.gamma_R, bc=w.bc, pml=w.pml, order=w.order,
                   moving_window=w.moving_window, window_v=w.window_v)
    for c in range(3):
        o.set_field(c, E0[c])
        o.set_field(3 + c, B0[c])
        o.set_field(6 + c, J[c])
    o.fdtd()
    for c in range(6):
        g = sim.get_field(c).astype(np.float64)
        r = o.field(c)
        den = max(np.max(np.abs(r)), 1e-30)
        assert np.max(np.abs(g - r)) / den < 1e-5, c
    # sampled push: oracle gather on the GPU fields of state n + Boris
    for c in range(3):
        o.set_field(c, E0[c])
        o.set_field(3 + c, B0[c])
    after = {name: sim.get_particles(ids[name]) for name in samples}
    for name, smp in samples.items():
        A = after[name]
        by_id = np.argsort(A["id"], kind="stable")
        ids_sorted = A["id"][by_id]
        at = np.minimum(np.searchsorted(ids_sorted, smp["id"]), len(ids_sorted) - 1)
        found = ids_sorted[at] == smp["id"]
        got, ref = [], []
        for k in range(len(smp["id"])):
            if not found[k]:
                continue
            j = by_id[at[k]]
            X = smp["cell"][k].astype(np.float64) + smp["off"][k].astype(np.float64)
            EB = o.gather_at(X)
            u1 = oracle.boris(-1.0, w.dt, EB[:3], EB[3:], smp["u"][k].astype(np.float64))
            got.append(A["u"][j].astype(np.float64))
            ref.append(u1)
        got, ref = np.array(got), np.array(ref)
        assert len(got) > 9000
        for c in range(3):
            den = max(np.max(np.abs(ref[:, c])), 1e-30)
            assert np.max(np.abs(got[:, c] - ref[:, c])) / den < 1e-5, (name, c)


def test_full_size_sort_order(state):
    w, sim, ids = state
    sim.sort()
    for name in ("plasma_e", "beam"):
        P = sim.get_particles(ids[name])
        n = len(P["id"])
        a = np.random.default_rng(5).integers(0, max(n - 200000, 1))
        X = P["cell"][a:a + 200000].astype(np.float64) + P["off"][a:a + 200000].astype(np.float64)
        order, keys = oracle.tile_sort(X, w.grid, w.tile)
        # keys of the GPU's storage order (the oracle's key definition) never decrease
        storage_keys = keys[np.argsort(order)]
        assert np.all(np.diff(storage_keys) >= 0), name
