"""GPU parity of the Helmholtz kernel G = e^{i kappa r}/r (PDE Laplacian +
kappa^2; Sec. 5.1's varying-order example).  The GPU evaluates the real and
the imaginary part of G as two real FMMs sharing the tree, P2M and M2M; the
oracle composes the same two parts.  FP64 results are held to the oracle's
same-tree FMM at 1e-12 (relative L2 of the complex potential); the mixed
forms to stated tolerances, and the FMM to the direct sum within its
truncation error.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = {"fp32": 5e-6, "tf32x3": 5e-6, "bf16x3": 5e-5}


def rel_l2(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def gpu_helm(torch, p, L, src, w, tgt, kap, precision="fp64", m2l="dense", grad=False):
    from paper_2305_17867_gb300.fmm import FMM

    plan = FMM("helmholtz", d=3, p=p, levels=L, lam=kap, precision=precision, m2l=m2l)
    out = plan.eval(torch.tensor(src, device="cuda"), torch.tensor(w, device="cuda"),
                    None if tgt is None else torch.tensor(tgt, device="cuda"), grad=grad,
                    check_status=True)
    torch.cuda.synchronize()
    if grad:
        return out[0].cpu().numpy(), out[1].cpu().numpy()
    return out.cpu().numpy()


def case(n_src=12000, n_tgt=5000, seed=61):
    rng = np.random.default_rng(seed)
    return rng.random((n_src, 3)), rng.uniform(-1, 1, n_src), rng.random((n_tgt, 3))


@pytest.mark.parametrize("p,L,kap,m2l", [(8, 3, 1.0, "dense"), (12, 3, 1.0, "dense"),
                                         (10, 4, 6.0, "dense"), (8, 3, 1.0, "fft"),
                                         (12, 4, 6.0, "fft")])
def test_fp64_matches_oracle(torch_cuda, oracle, p, L, kap, m2l):
    src, w, tgt = case()
    ref = oracle.fmm_uniform("helmholtz", 3, p, L, src, w, tgt, lam=kap)
    got = gpu_helm(torch_cuda, p, L, src, w, tgt, kap, m2l=m2l)
    assert got.dtype == np.complex128
    assert rel_l2(got, ref) < FP64_TOL


def test_fp64_gradient_matches_oracle(torch_cuda, oracle):
    src, w, tgt = case(9000, 4000, 62)
    ref, gref = oracle.fmm_uniform("helmholtz", 3, 8, 3, src, w, tgt, lam=2.0, grad=True)
    got, g = gpu_helm(torch_cuda, 8, 3, src, w, tgt, 2.0, grad=True)
    assert rel_l2(got, ref) < FP64_TOL
    assert rel_l2(g, gref) < FP64_TOL


@pytest.mark.parametrize("precision", ["fp32", "tf32x3", "bf16x3"])
def test_mixed_precision(torch_cuda, oracle, precision):
    src, w, _ = case(30000, 0, 63)
    ref = oracle.fmm_uniform("helmholtz", 3, 10, 4, src, w, src, lam=1.0)
    got = gpu_helm(torch_cuda, 10, 4, src, w, None, 1.0, precision=precision)
    err = rel_l2(got, ref)
    print(f"helmholtz p=10 L=4 {precision}: rel L2 vs oracle {err:.3e}")
    assert err < MIXED_TOL[precision]


def test_converges_to_direct_sum(torch_cuda, oracle):
    src, w, tgt = case(8000, 300, 64)
    ref = oracle.direct("helmholtz", 3, src, w, tgt, lam=3.0)
    errs = [rel_l2(gpu_helm(torch_cuda, p, 3, src, w, tgt, 3.0), ref) for p in (4, 8, 12)]
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-6, errs


def test_rejected_forms(torch_cuda):
    from paper_2305_17867_gb300._lib import FMMError
    from paper_2305_17867_gb300.fmm import FMM

    with pytest.raises(FMMError):
        FMM("helmholtz", d=3, p=6, levels=-5, lam=1.0)  # adaptive trees: not provided
    with pytest.raises(FMMError):
        FMM("helmholtz", d=3, p=6, levels=3, lam=0.0)   # kappa must be positive
