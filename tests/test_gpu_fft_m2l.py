"""GPU parity of the FFT form of M2L (eq. (convolution_m2l)) against the oracle.

The convolution form computes the same local coefficients as eq.
(m2l_toeplitz) up to rounding, so it is held to the oracle's same-tree FMM.
Rounding: each transformed coefficient is a sum of at most prod(n) =
(2p+1)^{d-1}(2c-1) terms whose magnitudes, after the scaling g^{|q|} with
g = 3p/8 (Sec. 4.1.1), still span a few decades, so the relative error of a
translation is up to ~1e3 unit roundoffs.  Measured on the potentials (GB300):
FP64 9e-16 .. 5.3e-14 over every case here and the high-order cases (3D
Laplace p = 16: 1.5e-14 and 3.9e-14; biharmonic p = 16: 5.3e-14), so the FP64
form is held to the same 1e-12 as the dense FP64 form; FP32 up to 1.8e-5
(biharmonic p = 16), tolerance 1e-4.
"""
import numpy as np
import pytest

from paper_2305_17867_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FFT_TOL = {"fp64": 1e-12, "fp32": 1e-4}


def rel_l2(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def fft_fmm(torch, kernel, d, p, L, src, w, tgt=None, lam=0.0, precision="fp64", grad=False,
            m2l="fft"):
    from paper_2305_17867_gb300.fmm import FMM

    plan = FMM(kernel, d=d, p=p, levels=L, lam=lam, precision=precision, m2l=m2l)
    s = torch.tensor(src, device="cuda")
    wt = torch.tensor(w, device="cuda")
    t = None if tgt is None else torch.tensor(tgt, device="cuda")
    out = plan.eval(s, wt, t, grad=grad, check_status=True)
    torch.cuda.synchronize()
    if grad:
        return out[0].cpu().numpy(), out[1].cpu().numpy()
    return out.cpu().numpy()


@pytest.mark.parametrize("L,n", [(2, 3000), (3, 20000), (4, 30011)])
def test_fft_laplace3d_fp64(torch_cuda, oracle, L, n):
    wl = W.WORKLOADS["laplace3d_p10_L5_n1m"]
    src, w, _ = W.make_inputs(wl, n_src=n)
    ref = oracle.fmm_uniform("laplace", 3, 10, L, src, w, src)
    got = fft_fmm(torch_cuda, "laplace", 3, 10, L, src, w)
    assert rel_l2(got, ref) < FFT_TOL["fp64"]


def test_fft_laplace2d_fp64(torch_cuda, oracle):
    wl = W.WORKLOADS["laplace2d_p8_L4_n2k"]
    src, w, _ = W.make_inputs(wl)
    ref = oracle.fmm_uniform("laplace", 2, 8, 4, src, w, src)
    got = fft_fmm(torch_cuda, "laplace", 2, 8, 4, src, w)
    assert rel_l2(got, ref) < FFT_TOL["fp64"]


# biharmonic p = 2 and p = 3: c = 4 > p, every multi-index is stored and the
# m_s axis of the grid shrinks to 2p + 1
@pytest.mark.parametrize("kernel,p,lam", [("yukawa", 8, 1.0), ("yukawa", 12, 1.0),
                                          ("biharmonic", 2, 0.0), ("biharmonic", 3, 0.0),
                                          ("biharmonic", 8, 0.0), ("laplace", 1, 0.0),
                                          ("laplace", 16, 0.0)])
def test_fft_other_kernels_fp64(torch_cuda, oracle, kernel, p, lam):
    rng = np.random.default_rng(27)
    src = rng.random((9000, 3))
    w = rng.uniform(-1, 1, 9000)
    tgt = rng.random((5000, 3))
    ref = oracle.fmm_uniform(kernel, 3, p, 3, src, w, tgt, lam=lam)
    got = fft_fmm(torch_cuda, kernel, 3, p, 3, src, w, tgt, lam=lam)
    assert rel_l2(got, ref) < FFT_TOL["fp64"]


def test_fft_gradient_fp64(torch_cuda, oracle):
    rng = np.random.default_rng(28)
    src = rng.random((12000, 3))
    w = rng.uniform(-1, 1, 12000)
    tgt = rng.random((7000, 3))
    ref, gref = oracle.fmm_uniform("laplace", 3, 8, 3, src, w, tgt, grad=True)
    got, g = fft_fmm(torch_cuda, "laplace", 3, 8, 3, src, w, tgt, grad=True)
    assert rel_l2(got, ref) < FFT_TOL["fp64"]
    assert rel_l2(g, gref) < FFT_TOL["fp64"]


@pytest.mark.parametrize("kernel,p,lam", [("laplace", 10, 0.0), ("yukawa", 12, 1.0),
                                          ("biharmonic", 8, 0.0)])
def test_fft_fp32(torch_cuda, oracle, kernel, p, lam):
    rng = np.random.default_rng(29)
    src = rng.random((30011, 3))
    w = rng.uniform(-1, 1, 30011)
    ref = oracle.fmm_uniform(kernel, 3, p, 4, src, w, src, lam=lam)
    got = fft_fmm(torch_cuda, kernel, 3, p, 4, src, w, lam=lam, precision="fp32")
    assert rel_l2(got, ref) < FFT_TOL["fp32"]


def test_fft_full_size_sampled(torch_cuda, oracle):
    # the measured workload (1e6 points, p = 10, L = 5) with the FFT form in
    # FP64; a seeded sample of targets is evaluated by the oracle one by one
    wl = W.WORKLOADS["laplace3d_p10_L5_n1m"]
    src, w, _ = W.make_inputs(wl)
    got = fft_fmm(torch_cuda, "laplace", 3, 10, 5, src, w)
    idx = np.random.default_rng(97).choice(len(w), 64, replace=False)
    ref = oracle.fmm_uniform("laplace", 3, 10, 5, src, w, src, sample=idx)
    assert rel_l2(got[idx], ref) < FFT_TOL["fp64"]


def test_fft_and_dense_agree_on_gpu(torch_cuda):
    # both M2L forms on the same device inputs (no oracle): FP64 results agree
    # to the FFT rounding level
    rng = np.random.default_rng(30)
    src = rng.random((50000, 3))
    w = rng.uniform(-1, 1, 50000)
    a = fft_fmm(torch_cuda, "laplace", 3, 10, 4, src, w, m2l="fft")
    b = fft_fmm(torch_cuda, "laplace", 3, 10, 4, src, w, m2l="dense")
    assert rel_l2(a, b) < FFT_TOL["fp64"]


def test_fft_rejects_tensor_precisions(torch_cuda):
    from paper_2305_17867_gb300._lib import FMMError
    from paper_2305_17867_gb300.fmm import FMM

    for prec in ("tf32", "tf32x3", "bf16x3"):
        with pytest.raises(FMMError):
            FMM("laplace", d=3, p=8, levels=3, precision=prec, m2l="fft")


@pytest.mark.parametrize("precision,expect", [("fp64", "fft"), ("fp32", "fft"),
                                               ("tf32x3", "dense")])
def test_auto_m2l_matches_its_choice(torch_cuda, precision, expect):
    # AUTO resolves by arithmetic; its results equal the chosen form's bit for bit
    rng = np.random.default_rng(33)
    src = rng.random((20000, 3))
    w = rng.uniform(-1, 1, 20000)
    a = fft_fmm(torch_cuda, "laplace", 3, 8, 4, src, w, precision=precision, m2l="auto")
    b = fft_fmm(torch_cuda, "laplace", 3, 8, 4, src, w, precision=precision, m2l=expect)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("kernel,lam", [("laplace", 0.0), ("yukawa", 1.0)])
def test_uncompressed_taylor_with_fft(torch_cuda, oracle, kernel, lam):
    # Table `compressed`, row 2: the plain Taylor FMM (PDE d_z^(p+1): nothing is
    # compressed, the m_s axis of the grid has 2p+1 points) with the FFT form of
    # M2L, held to the oracle's uncompressed FMM
    from paper_2305_17867_gb300.fmm import FMM

    p, L = 6, 3
    rng = np.random.default_rng(37)
    src = rng.random((12000, 3))
    w = rng.uniform(-1, 1, 12000)
    plan = FMM(kernel, d=3, p=p, levels=L, lam=lam, m2l="fft", pde=([(0, 0, p + 1)], [1.0]))
    assert plan.nj == plan.nfull
    got = plan.eval(torch_cuda.tensor(src, device="cuda"), torch_cuda.tensor(w, device="cuda"),
                    check_status=True).cpu().numpy()
    ref = oracle.fmm_uniform(kernel, 3, p, L, src, w, src, lam=lam, compressed=False)
    assert rel_l2(got, ref) < FFT_TOL["fp64"]
