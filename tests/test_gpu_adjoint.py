"""The hand-written adjoint (pic_checkpoint / pic_backward) on the oracle-sized reduction of the
differentiated run (16 x 16 x 32 periodic grid, 2000 beam electrons, 4-per-cell plasma with frozen
ions whose lab density is a 32-node piecewise-linear profile, undulator K = 1, first-order shape,
30 steps checkpointed every 10).

Loss: the beam's bunching factor in the boosted frame at the RRF image of the resonant
wavenumber.  Parameters: K (through the undulator field seen during the steps; the loaded beam is
held fixed) and the profile nodes (through the plasma weights).  Checked against
  * the FP64 oracle's gradient: central differences of the oracle run (h = 1e-4 relative), for K
    and every one of the 32 profile nodes, to 2e-3 relative (the adjoint is exact for the discrete
    scheme; FP32 rounding remains);
  * central differences of the GPU forward itself for K, to 3e-2 relative.  Its FP32 rounding
    (float atomics in varying order: ~1e-6 of the loss from run to run) divided by 2h limits that
    estimate, so it takes h = 1e-3 (at h = 1e-4 the noise alone is ~10 %).
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2411_04703_gb300 import api, workloads as W

pytestmark = pytest.mark.gpu

H = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    oracle.build()


def _k_rrf(w):
    return api.rrf_resonant_wavenumber(w)


def _workload(profile_scale=None):
    w = W.mini_adjoint()
    if profile_scale is not None:
        q, f = profile_scale
        dn = list(w.plasma.n_nodes)
        dn[q] *= f
        w.plasma.n_nodes = tuple(dn)
    return w


def _gpu_loss(w, K=None):
    sim, ids = api.from_workload(w)
    if K is not None:   # after the matched load: only the field seen during the steps changes
        sim.set_external_field(K, w.undulator.lambda_u)
    sim.step(w.steps)
    b = sim.get_moments(ids["beam"], api.PIC_FRAME_BOOSTED, k_bunch=_k_rrf(w))["bunching"]
    sim.close()
    return b


def _oracle_loss(w, K=None):
    o = oracle.Sim(w.grid, w.d, w.dt, w.gamma_R, bc=w.bc, order=w.order)
    # the particle loop on the host cores: its FP64 sums then run in another order, a change of
    # ~1e-16 relative, far below the differences taken here
    o.set_threads(os.cpu_count() or 1)
    o.set_external(w.undulator.K, w.undulator.lambda_u)
    se = o.add_species(-1.0, 1.0)
    si = o.add_species(1.0, 1836.15267343, frozen=True)
    p = w.plasma
    o.set_plasma(se, si, p.ppc, p.xrange, p.z_nodes, p.n_nodes)
    x, u, wt = W.sample_beam(w)
    sb = o.add_species(-1.0, 1.0, capacity=x.shape[1])
    o.load(sb, x, u, wt, frame=oracle.LAB, origin=w.beam.origin, match_undulator=True)
    if K is not None:
        o.set_external(K, w.undulator.lambda_u)
    o.step(w.steps)
    return o.moments(sb, frame=0, k=_k_rrf(w))["bunching"]


@pytest.fixture(scope="module")
def adjoint():
    w = _workload()
    sim, ids = api.from_workload(w)
    sim.checkpoint(10)
    sim.step(w.steps)
    g = sim.backward(ids["beam"], _k_rrf(w))
    # the context is back at the final state: the diagnostic there is the loss
    b = sim.get_moments(ids["beam"], api.PIC_FRAME_BOOSTED, k_bunch=_k_rrf(w))["bunching"]
    sim.close()
    return w, g, b


def test_backward_returns_the_loss_and_leaves_the_final_state(adjoint):
    w, g, b = adjoint
    assert g["loss"] == pytest.approx(b, rel=1e-6)
    assert len(g["dL_dprofile"]) == len(w.plasma.n_nodes)
    assert np.all(np.isfinite(g["dL_dprofile"])) and math.isfinite(g["dL_dK"])


def test_adjoint_matches_fp64_oracle_gradient(adjoint):
    w, g, _ = adjoint
    K0 = w.undulator.K
    assert g["loss"] == pytest.approx(_oracle_loss(w), rel=1e-4)
    dK = (_oracle_loss(w, K0 * (1 + H)) - _oracle_loss(w, K0 * (1 - H))) / (2 * H * K0)
    assert g["dL_dK"] == pytest.approx(dK, rel=2e-3), (g["dL_dK"], dK)
    scale = np.max(np.abs(g["dL_dprofile"]))
    for q in range(len(w.plasma.n_nodes)):
        n0 = w.plasma.n_nodes[q]
        d = (_oracle_loss(_workload((q, 1 + H))) - _oracle_loss(_workload((q, 1 - H)))) / (2 * H * n0)
        assert abs(g["dL_dprofile"][q] - d) < 2e-3 * max(abs(d), scale), (q, g["dL_dprofile"][q], d)


def test_adjoint_matches_gpu_central_differences(adjoint):
    w, g, _ = adjoint
    K0 = w.undulator.K
    h = 1e-3
    dK = (_gpu_loss(w, K0 * (1 + h)) - _gpu_loss(w, K0 * (1 - h))) / (2 * h * K0)
    assert g["dL_dK"] == pytest.approx(dK, rel=3e-2), (g["dL_dK"], dK)
    # (the profile's effect on the loss, ~1e-7 per node, is below the FP32 forward's rounding at
    # h = 1e-4; the oracle's FP64 differences check that part)
