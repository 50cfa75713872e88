"""Host logic of the torch autograd wrapper around pic_checkpoint / pic_backward
(api.bunching_loss), with a stand-in simulation: what the forward passes to the library and
how the backward scales the library's gradients.  The GPU run itself is checked against the
oracle in test_gpu_adjoint.py."""
import numpy as np
import pytest

from paper_2411_04703_gb300 import api, workloads as W


def test_bunching_loss_plumbs_the_adjoint(monkeypatch):
    torch = pytest.importorskip("torch")
    calls = {}

    class StandIn:
        def set_external_field(self, K, lambda_u, *rest, **kw):
            calls["K"] = K

        def checkpoint(self, k):
            calls["every"] = k

        def step(self, n):
            calls["steps"] = n

        def backward(self, sid, kb):
            calls["seed"] = (sid, kb)
            return {"loss": 0.25, "dL_dK": 3.0, "dL_dprofile": np.arange(4.0)}

        def close(self):
            calls["closed"] = True

    def from_workload(w, device=0):
        calls["nodes"] = w.plasma.n_nodes
        return StandIn(), {"beam": 7}

    monkeypatch.setattr(api, "from_workload", from_workload)
    w = W.mini_adjoint()
    w.plasma.z_nodes = w.plasma.z_nodes[:4]
    w.plasma.n_nodes = w.plasma.n_nodes[:4]
    before = w.plasma.n_nodes
    K = torch.tensor(1.1, dtype=torch.float64, requires_grad=True)
    prof = torch.tensor([1.0, 2.0, 3.0, 4.0], dtype=torch.float64, requires_grad=True)
    loss = api.bunching_loss(w, K, prof, checkpoint_every=5, k_bunch=2.0)
    (2.0 * loss).backward()
    assert loss.item() == 0.25
    assert K.grad.item() == 6.0
    assert torch.equal(prof.grad, 2.0 * torch.arange(4.0, dtype=torch.float64))
    assert calls["K"] == pytest.approx(1.1)
    assert calls["every"] == 5 and calls["steps"] == w.steps and calls["seed"] == (7, 2.0)
    assert calls["closed"]
    assert calls["nodes"] == (1.0, 2.0, 3.0, 4.0)
    assert w.plasma.n_nodes == before          # the caller's workload is not modified
    # float32 inputs get float32 gradients
    K32 = torch.tensor(1.0, dtype=torch.float32, requires_grad=True)
    p32 = torch.ones(4, dtype=torch.float32, requires_grad=True)
    api.bunching_loss(w, K32, p32, k_bunch=2.0).backward()
    assert K32.grad.dtype == torch.float32 and p32.grad.dtype == torch.float32
    assert K32.grad.item() == 3.0


def test_bunching_loss_default_wavenumber_and_profile_length(monkeypatch):
    torch = pytest.importorskip("torch")
    seen = {}

    class StandIn:
        def set_external_field(self, *a, **kw):
            pass

        def checkpoint(self, k):
            pass

        def step(self, n):
            pass

        def backward(self, sid, kb):
            seen["kb"] = kb
            return {"loss": 0.0, "dL_dK": 0.0, "dL_dprofile": np.zeros(32)}

        def close(self):
            pass

    monkeypatch.setattr(api, "from_workload", lambda w, device=0: (StandIn(), {"beam": 0}))
    w = W.mini_adjoint()
    K = torch.tensor(w.undulator.K, dtype=torch.float64, requires_grad=True)
    prof = torch.tensor(w.plasma.n_nodes, dtype=torch.float64, requires_grad=True)
    api.bunching_loss(w, K, prof)
    # the default k_bunch is the boosted-frame image of the lab resonant wavenumber, from the
    # library's Eq. RadLambda call at the workload's K, beam gamma and gamma_R
    un, g, gR = w.undulator, w.beam.gamma, w.gamma_R
    expect = api.resonant_wavenumber(un.lambda_u, un.K, g, gR, api.PIC_FRAME_BOOSTED)
    assert seen["kb"] == pytest.approx(expect, rel=1e-12)
    with pytest.raises(ValueError):
        api.bunching_loss(w, K, prof[:5])
