"""GPU parity of the 2D biharmonic kernel G = r^2 log r (PDE Laplacian^2,
c = 4; Sec. 4.4) against the oracle's same-tree FMM, FP64 at 1e-12, and
against the direct sum of eq. (1) within the truncation error."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def rel_l2(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def gpu_bih2(torch, p, L, src, w, tgt=None, precision="fp64", m2l="dense", grad=False):
    from paper_2305_17867_gb300.fmm import FMM

    plan = FMM("biharmonic", d=2, p=p, levels=L, precision=precision, m2l=m2l)
    out = plan.eval(torch.tensor(src, device="cuda"), torch.tensor(w, device="cuda"),
                    None if tgt is None else torch.tensor(tgt, device="cuda"), grad=grad,
                    check_status=True)
    torch.cuda.synchronize()
    if grad:
        return out[0].cpu().numpy(), out[1].cpu().numpy()
    return out.cpu().numpy()


@pytest.mark.parametrize("p,L,m2l", [(8, 4, "dense"), (12, 5, "dense"), (12, 5, "fft")])
def test_fp64_matches_oracle(torch_cuda, oracle, p, L, m2l):
    rng = np.random.default_rng(81)
    src = rng.random((20000, 2))
    w = rng.uniform(-1, 1, 20000)
    tgt = rng.random((8000, 2))
    ref = oracle.fmm_uniform("biharmonic", 2, p, L, src, w, tgt)
    got = gpu_bih2(torch_cuda, p, L, src, w, tgt, m2l=m2l)
    assert rel_l2(got, ref) < FP64_TOL


def test_gradient_and_shared_points(torch_cuda, oracle):
    rng = np.random.default_rng(82)
    src = rng.random((15000, 2))
    w = rng.uniform(-1, 1, 15000)
    ref, gref = oracle.fmm_uniform("biharmonic", 2, 10, 4, src, w, src, grad=True)
    got, g = gpu_bih2(torch_cuda, 10, 4, src, w, grad=True)
    assert rel_l2(got, ref) < FP64_TOL
    assert rel_l2(g, gref) < FP64_TOL


def test_root_box_not_unit(torch_cuda, oracle):
    # a root of side 3: the log(s) parts of the box scaling are exercised
    from paper_2305_17867_gb300.fmm import FMM

    rng = np.random.default_rng(83)
    src = rng.random((6000, 2)) * 3.0 - 1.0
    w = rng.uniform(-1, 1, 6000)
    lo = np.array([-1.0, -1.0])
    ref = oracle.fmm_uniform("biharmonic", 2, 8, 4, src, w, src, lo=lo, size=3.0)
    plan = FMM("biharmonic", d=2, p=8, levels=4, root_lo=list(lo), root_size=3.0)
    got = plan.eval(torch_cuda.tensor(src, device="cuda"),
                    torch_cuda.tensor(w, device="cuda"), check_status=True).cpu().numpy()
    assert rel_l2(got, ref) < FP64_TOL


def test_converges_to_direct_sum(torch_cuda, oracle):
    rng = np.random.default_rng(84)
    src = rng.random((8000, 2))
    w = rng.uniform(-1, 1, 8000)
    tgt = rng.random((400, 2))
    ref = oracle.direct("biharmonic", 2, src, w, tgt)
    errs = [rel_l2(gpu_bih2(torch_cuda, p, 4, src, w, tgt), ref) for p in (6, 10, 14)]
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-7, errs
