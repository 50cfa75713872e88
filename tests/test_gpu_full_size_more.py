"""Parity at full size for the long undulator (256 x 256 x 1024, 33,554,432 beam electrons, TSC,
CPML on every face, undulator with its entrance ramp) and the batched ensemble (64 runs of
64 x 64 x 128 with their own K, plasma density and beam), in the configurations bench.py and the
workloads define.  The oracle cannot run these states whole; the checks are what it computes one
unit at a time and what holds at any size (as for the plasma buncher):

* the momentum push of sampled particles: the oracle's gather on the GPU's fields at step n,
  plus the undulator field at the particle (the run's own K), then Boris, against the GPU;
* charge continuity rho^{n+1} - rho^n + dt div J = 0 at every node;
* ensemble: the FDTD update of whole runs (oracle run on the run's own block of E, B, J).
Tolerances as in test_gpu_parity.py: 1e-5 relative per step.
"""
import numpy as np
import pytest

import oracle
from paper_2411_04703_gb300 import api, workloads as W

import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    oracle.build()


def _div(J, d):
    jx, jy, jz = J
    out = (jx - np.roll(jx, 1, 2)) / d[0]
    out += (jy - np.roll(jy, 1, 1)) / d[1]
    out += (jz - np.roll(jz, 1, 0)) / d[2]
    return out


def _div_open(J, d):
    jx, jy, jz = J
    out = (jx - np.pad(jx, ((0, 0), (0, 0), (1, 0)))[:, :, :-1]) / d[0]
    out += (jy - np.pad(jy, ((0, 0), (1, 0), (0, 0)))[:, :-1, :]) / d[1]
    out += (jz - np.pad(jz, ((1, 0), (0, 0), (0, 0)))[:-1, :, :]) / d[2]
    return out


def _sampled_push_check(w, o, before, after, tp, qm=-1.0, tol=1e-5):
    """The GPU's u^{n+1/2} of sampled particles against the oracle's gather + external + Boris."""
    A = after
    by_id = np.argsort(A["id"], kind="stable")
    ids_sorted = A["id"][by_id]
    at = np.minimum(np.searchsorted(ids_sorted, before["id"]), len(ids_sorted) - 1)
    found = ids_sorted[at] == before["id"]
    got, ref = [], []
    for k in range(len(before["id"])):
        if not found[k]:
            continue
        X = before["cell"][k].astype(np.float64) + before["off"][k].astype(np.float64)
        EB = o.gather_at(X)
        if w.undulator is not None:
            Ee, Be = o.external_at(X[2] * w.d[2], tp)
            EB = EB + np.concatenate([Ee, Be])
        got.append(A["u"][by_id[at[k]]].astype(np.float64))
        ref.append(oracle.boris(qm, w.dt, EB[:3], EB[3:], before["u"][k].astype(np.float64)))
    got, ref = np.array(got), np.array(ref)
    assert len(got) > 0.9 * len(before["id"])
    for c in range(3):
        den = max(np.max(np.abs(ref[:, c])), 1e-30)
        assert np.max(np.abs(got[:, c] - ref[:, c])) / den < tol, c
    return len(got)


def test_long_undulator_full_size_push_and_continuity():
    w = W.long_undulator(z_start=0.0)      # the bunch inside the field from the first step
    sim, ids = api.from_workload(w)
    rng = np.random.default_rng(7)
    for c in range(6):
        sim.set_field(c, (1e-3 * rng.standard_normal((w.grid[2], w.grid[1], w.grid[0]))).astype(np.float32))
    P = sim.get_particles(ids["beam"])
    k = rng.choice(len(P["id"]), 10000, replace=False)
    before = {key: v[k] for key, v in P.items()}
    del P
    E0 = [sim.get_field(c) for c in range(3)]
    B0 = [sim.get_field(3 + c) for c in range(3)]
    rho0 = sim.get_field(api.PIC_RHO).astype(np.float64)
    t0 = sim.get_time()[0] * w.dt
    sim.step(1)
    sim.sync()
    J = [sim.get_field(6 + c).astype(np.float64) for c in range(3)]
    rho1 = sim.get_field(api.PIC_RHO).astype(np.float64)
    resid = (rho1 - rho0) / w.dt + _div_open(J, w.d)
    del J, rho0
    scale = np.max(np.abs(rho1)) / w.dt
    assert np.max(np.abs(resid)) < 1e-5 * scale
    del resid, rho1
    # sampled push: the oracle gathers from the GPU's fields (no PML needed for a gather)
    un = w.undulator
    o = oracle.Sim(w.grid, w.d, w.dt, w.gamma_R, bc=w.bc, order=w.order)
    o.set_external(un.K, un.lambda_u, un.phase, un.z_start, un.ramp)
    for c in range(3):
        o.set_field(c, E0[c].astype(np.float64))
        o.set_field(3 + c, B0[c].astype(np.float64))
    del E0, B0
    after = sim.get_particles(ids["beam"])
    assert _sampled_push_check(w, o, before, after, t0) > 9000
    sim.close()


def test_ensemble_full_size_fields_push_and_continuity():
    e = W.batched_ensemble()
    sim, ids = api.from_ensemble(e)
    nzr = e.base.grid[2]
    rng = np.random.default_rng(8)
    sim.step(3)                      # past the first step, with a developed adaptive current scale
    sim.sync()
    runs = (0, 37, 63)
    E0 = [sim.get_field(c) for c in range(3)]
    B0 = [sim.get_field(3 + c) for c in range(3)]
    rho0 = sim.get_field(api.PIC_RHO).astype(np.float64)
    def split(P, r):
        kk = P["cell"][:, 2]
        m = (kk >= r * nzr) & (kk < (r + 1) * nzr)
        out = {key: v[m].copy() for key, v in P.items()}
        out["cell"][:, 2] -= r * nzr
        return out

    samples = {}
    for name in ("beam", "plasma_e"):
        P = sim.get_particles(ids[name])
        for r in runs:
            Pr = split(P, r)
            k = rng.choice(len(Pr["id"]), min(3000, len(Pr["id"])), replace=False)
            samples[(r, name)] = {key: v[k] for key, v in Pr.items()}
        del P
    t0 = sim.get_time()[0] * e.base.dt
    sim.step(1)
    sim.sync()
    J = [sim.get_field(6 + c).astype(np.float64) for c in range(3)]
    rho1 = sim.get_field(api.PIC_RHO).astype(np.float64)
    Eg = [sim.get_field(c).astype(np.float64) for c in range(3)]
    Bg = [sim.get_field(3 + c).astype(np.float64) for c in range(3)]
    after_all = {name: sim.get_particles(ids[name]) for name in ("beam", "plasma_e")}
    for r in runs:
        sl = slice(r * nzr, (r + 1) * nzr)
        w = W.ensemble_run(e, r)
        # continuity inside the run (periodic in its own rows)
        resid = (rho1[sl] - rho0[sl]) / w.dt + _div([J[c][sl] for c in range(3)], w.d)
        rho_species = w.gamma_R * max(w.plasma.n_nodes)
        assert np.max(np.abs(resid)) < 1e-5 * rho_species / w.dt, r
        # FDTD of the run's block
        o = oracle.Sim(w.grid, w.d, w.dt, w.gamma_R, bc=w.bc, order=w.order)
        for c in range(3):
            o.set_field(c, E0[c][sl].astype(np.float64))
            o.set_field(3 + c, B0[c][sl].astype(np.float64))
            o.set_field(6 + c, J[c][sl])
        o.fdtd()
        for c in range(3):
            assert parity.rel_err(Eg[c][sl], o.field(c)) < 1e-5, (r, c)
            assert parity.rel_err(Bg[c][sl], o.field(3 + c)) < 1e-5, (r, 3 + c)
        # sampled push with the run's own K (the oracle gathers from the run's block at step n)
        o2 = oracle.Sim(w.grid, w.d, w.dt, w.gamma_R, bc=w.bc, order=w.order)
        o2.set_external(w.undulator.K, w.undulator.lambda_u)
        for c in range(3):
            o2.set_field(c, E0[c][sl].astype(np.float64))
            o2.set_field(3 + c, B0[c][sl].astype(np.float64))
        for name in ("beam", "plasma_e"):
            after = split(after_all[name], r)
            # the plasma's transverse momentum is the residual of cancelling undulator forces
            # (see compare_species): its push is checked by the per-particle vector error, the
            # beam's per component
            before = samples[(r, name)]
            if name == "beam":
                _sampled_push_check(w, o2, before, after, t0)
            else:
                A = after
                by_id = np.argsort(A["id"], kind="stable")
                at = np.searchsorted(A["id"][by_id], before["id"])
                got, ref = [], []
                for kk in range(len(before["id"])):
                    X = before["cell"][kk].astype(np.float64) + before["off"][kk].astype(np.float64)
                    EB = o2.gather_at(X)
                    Ee, Be = o2.external_at(X[2] * w.d[2], t0)
                    EB = EB + np.concatenate([Ee, Be])
                    u1 = oracle.boris(-1.0, w.dt, EB[:3], EB[3:], before["u"][kk].astype(np.float64))
                    ref.append(u1)
                    got.append(A["u"][by_id[at[kk]]].astype(np.float64))
                got, ref = np.array(got), np.array(ref)
                err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
                assert np.max(err) < 1e-5, (r, float(np.max(err)))
    sim.close()
