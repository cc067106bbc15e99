"""The bounded device waits of the tensor-core M2L run out cleanly.

Every mbarrier wait of the contraction gives up after a time limit, raises a
status bit and lets the CTA drain its copies and MMAs, free its tensor memory
and return (no trap, no hang).  fmm_set_wait_limit shortens only the
pipeline's waits (producer, MMA issuer, drain) so that a normal launch runs
out; the waits before a CTA exits keep the full limit.  The call must then
report FMM_ERR_TIMEOUT, and the next call with the default limit must be
correct again.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("precision", ["tf32x3", "bf16x3"])
def test_pipeline_wait_runs_out_and_recovers(torch_cuda, precision):
    torch = torch_cuda
    from paper_2305_17867_gb300 import _lib
    from paper_2305_17867_gb300.fmm import FMM

    L = _lib.load()
    rng = np.random.default_rng(71)
    src = torch.tensor(rng.random((40000, 3)), device="cuda")
    w = torch.tensor(rng.uniform(-1, 1, 40000), device="cuda")
    plan = FMM("laplace", d=3, p=10, levels=4, precision=precision)
    ref = plan.eval(src, w, check_status=True)
    torch.cuda.synchronize()
    assert L.fmm_set_wait_limit(plan._h, 1) == 0  # every pipeline wait that blocks runs out
    plan.eval(src, w)
    assert plan.last_status() == -5  # FMM_ERR_TIMEOUT
    assert L.fmm_set_wait_limit(plan._h, 0) == 0  # the default limit again
    again = plan.eval(src, w, check_status=True)
    torch.cuda.synchronize()
    assert float(torch.linalg.norm(again - ref) / torch.linalg.norm(ref)) < 1e-14


def test_wait_limit_argument_checks(torch_cuda):
    from paper_2305_17867_gb300 import _lib
    from paper_2305_17867_gb300.fmm import FMM

    L = _lib.load()
    plan = FMM("laplace", d=3, p=4, levels=2, precision="tf32x3")
    assert L.fmm_set_wait_limit(plan._h, -1) == -1
    assert L.fmm_set_wait_limit(None, 5) == -1
