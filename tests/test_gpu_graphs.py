"""CUDA-graph replay of captured step sequences against launching every kernel: the same run
(periodic vacuum undulator with a beam, and a periodic plasma ensemble) stepped both ways agrees
within FP32 reduction-order noise (40 steps: two graph replays of a pair of
sort periods and eager steps around them), and the step counters match.  Both runs are FP32 with
float atomics in different orders, so they agree to rounding noise that grows over the run
(1e-4 relative after 40 steps); a stale parameter or a missed step would differ at O(1)."""
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


def _pair(make):
    a, ids = make()
    b, _ = make()
    b.use_graphs(False)
    return a, b, ids


@pytest.mark.parametrize("case", ["vacuum_cic", "ensemble_tsc"])
def test_graph_replay_matches_launching_every_kernel(case):
    if case == "vacuum_cic":
        a, b, ids = _pair(lambda: api.from_workload(W.mini_vacuum(order=1)))
    else:
        e = W.mini_ensemble()
        a, b, ids = _pair(lambda: api.from_ensemble(e))
    for n in (5, 32, 0, 3):   # eager steps to reach a period start, whole periods, a tail
        if n:
            a.step(n)
            b.step(n)
    a.sync()
    b.sync()
    assert a.get_time() == b.get_time()
    for c in range(9):
        assert parity.rel_err(a.get_field(c).astype(np.float64), b.get_field(c).astype(np.float64)) < 1e-4, c
    for name, sid in ids.items():
        pa, pb = a.get_particles(sid), b.get_particles(sid)
        oa, ob = np.argsort(pa["id"]), np.argsort(pb["id"])
        assert np.array_equal(pa["id"][oa], pb["id"][ob]), name
        ua, ub = pa["u"][oa].astype(np.float64), pb["u"][ob].astype(np.float64)
        assert np.max(np.abs(ua - ub)) <= 1e-4 * np.max(np.abs(ub)), name
