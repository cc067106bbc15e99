"""GPU parity of the F16X3 tensor-core M2L (fp16 hi + lo operands, three
passes, FP32 accumulation; eq. (m2l_toeplitz) grouped by offset).

fp16 carries tf32's 11-bit significand, so the split products are as exact
as TF32X3's; its 5-bit exponent is covered by exact power-of-two scalings of
every box's multipole and of the offset matrices, undone in float.  The tests
hold F16X3 to the TF32X3 bound (relative L2 5e-6 against the oracle's same-tree
FMM) and check that the scalings make the result independent of the units:

* the kernels with shared (Laplace, biharmonic) and per-level (Yukawa) offset
  tables, orders whose |j| takes one or several column blocks and stacked
  child classes (Laplace p = 10: two classes of 128 columns);
* weights scaled by 1e+6 and 1e-6, and roots of side 1e-3 and 1e+3 (the
  derivative tables scale by the side's powers): the relative error stays
  at the unscaled one;
* weights spanning eight orders of magnitude between the halves of the
  domain: the small half's targets keep their relative accuracy.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 5e-6


def rel_l2(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def gpu_eval(torch, kernel, p, L, src, w, tgt=None, lam=0.0, precision="f16x3", root_size=1.0,
             root_lo=None, grad=False):
    from paper_2305_17867_gb300.fmm import FMM

    plan = FMM(kernel, d=3, p=p, levels=L, lam=lam, precision=precision, root_size=root_size,
               root_lo=root_lo)
    out = plan.eval(torch.tensor(src, device="cuda"), torch.tensor(w, device="cuda"),
                    None if tgt is None else torch.tensor(tgt, device="cuda"), grad=grad,
                    check_status=True)
    torch.cuda.synchronize()
    if grad:
        return out[0].cpu().numpy(), out[1].cpu().numpy()
    return out.cpu().numpy()


def case(n, seed, n_sample=96):
    rng = np.random.default_rng(seed)
    src = rng.random((n, 3))
    w = rng.uniform(-1.0, 1.0, n)
    return src, w, np.sort(rng.choice(n, n_sample, replace=False))


@pytest.mark.parametrize("kernel,p,lam,L", [("laplace", 4, 0.0, 4), ("laplace", 10, 0.0, 4),
                                            ("laplace", 16, 0.0, 3), ("biharmonic", 8, 0.0, 4),
                                            ("biharmonic", 12, 0.0, 3), ("yukawa", 8, 1.5, 4),
                                            ("yukawa", 12, 1.0, 3)])
def test_matches_oracle(torch_cuda, oracle, kernel, p, lam, L):
    src, w, idx = case(24000, 500 + p)
    ref = oracle.fmm_uniform(kernel, 3, p, L, src, w, src, lam=lam, sample=idx)
    got = gpu_eval(torch_cuda, kernel, p, L, src, w, lam=lam)[idx]
    t32 = gpu_eval(torch_cuda, kernel, p, L, src, w, lam=lam, precision="tf32x3")[idx]
    err, err32 = rel_l2(got, ref), rel_l2(t32, ref)
    print(f"{kernel} p={p} L={L}: f16x3 {err:.3e}, tf32x3 {err32:.3e}")
    assert err < TOL, (err, err32)


@pytest.mark.parametrize("wscale", [1e6, 1e-6])
@pytest.mark.parametrize("kernel", ["laplace", "biharmonic"])
def test_weight_scale_is_invisible(torch_cuda, oracle, kernel, wscale):
    src, w, idx = case(16000, 71)
    ref = oracle.fmm_uniform(kernel, 3, 8, 3, src, w * wscale, src, sample=idx)
    got = gpu_eval(torch_cuda, kernel, 8, 3, src, w * wscale)[idx]
    assert rel_l2(got, ref) < TOL


@pytest.mark.parametrize("size", [1e-3, 1e3])
@pytest.mark.parametrize("kernel,lam", [("laplace", 0.0), ("biharmonic", 0.0), ("yukawa", 1.0)])
def test_root_size_is_invisible(torch_cuda, oracle, kernel, lam, size):
    src, w, idx = case(16000, 72)
    src = src * size
    lam_s = lam / size  # the same screening length in box units
    lo = np.zeros(3)
    ref = oracle.fmm_uniform(kernel, 3, 8, 3, src, w, src, lo=lo, size=size, lam=lam_s,
                             sample=idx)
    got = gpu_eval(torch_cuda, kernel, 8, 3, src, w, lam=lam_s, root_size=size,
                   root_lo=[0.0, 0.0, 0.0])[idx]
    assert rel_l2(got, ref) < TOL


def test_weights_over_eight_orders(torch_cuda, oracle):
    src, w, _ = case(20000, 73)
    big = src[:, 0] < 0.5
    w = np.where(big, w * 1e4, w * 1e-4)
    rng = np.random.default_rng(74)
    small_idx = np.sort(rng.choice(np.nonzero(~big & (src[:, 0] > 0.75))[0], 64, replace=False))
    ref = oracle.fmm_uniform("laplace", 3, 8, 4, src, w, src, sample=small_idx)
    got = gpu_eval(torch_cuda, "laplace", 8, 4, src, w)[small_idx]
    t32 = gpu_eval(torch_cuda, "laplace", 8, 4, src, w, precision="tf32x3")[small_idx]
    # the small-weight targets (a quarter box width away from the big half)
    # are dominated by the far big half; both forms hold them to the bound
    err, err32 = rel_l2(got, ref), rel_l2(t32, ref)
    print(f"small half: f16x3 {err:.3e}, tf32x3 {err32:.3e}")
    assert err < TOL


def test_gradient(torch_cuda, oracle):
    src, w, idx = case(16000, 75)
    ref, gref = oracle.fmm_uniform("laplace", 3, 8, 3, src, w, src, sample=idx, grad=True)
    got, g = gpu_eval(torch_cuda, "laplace", 8, 3, src, w, grad=True)
    assert rel_l2(got[idx], ref) < TOL
    assert rel_l2(g[idx], gref) < TOL
