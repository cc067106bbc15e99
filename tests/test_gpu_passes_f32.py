"""GPU parity of the warp-per-box float passes (P2M, M2M, L2L and L2P of 3D
uniform trees in the mixed-precision modes; orders 4, 6, 8, 10, 12, 16).

Each order runs through them for the Laplace, biharmonic and Yukawa kernels
(the last one with scaled recurrence coefficients, so the decompression and
compression sweeps take powers of the box side) and is held to the oracle's
same-tree FMM on a seeded sample of targets.  Inputs are clustered, so that
leaves hold from none to a few hundred points: empty leaves (zero multipoles,
no targets), leaves of several 32-source chunks, and leaves of one point.

Tolerance: relative L2 5e-6 in TF32x3, the bound the mixed modes are held to
elsewhere (float shifts and float power tables add a few float roundoffs per
coefficient, ~1e-7, below the tf32x3 contraction's ~1e-6).  Order 5 runs the
block-per-box fallback with the same bound.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 5e-6
N_SAMPLE = 96


def rel_l2(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def clustered(n, seed):
    """60% of the points in a ball of radius 0.08 around (0.3, 0.6, 0.4), the
    rest uniform in the unit cube; weights U(-1, 1)."""
    rng = np.random.default_rng(seed)
    nc = int(0.6 * n)
    v = rng.normal(size=(nc, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    r = 0.08 * rng.random(nc) ** (1.0 / 3.0)
    ball = np.array([0.3, 0.6, 0.4]) + v * r[:, None]
    pts = np.concatenate([ball, rng.random((n - nc, 3))])
    return pts, rng.uniform(-1.0, 1.0, n), np.sort(rng.choice(n, N_SAMPLE, replace=False))


def gpu_eval(torch, kernel, p, L, src, w, lam, grad=False, precision="tf32x3"):
    from paper_2305_17867_gb300.fmm import FMM

    plan = FMM(kernel, d=3, p=p, levels=L, lam=lam, precision=precision)
    out = plan.eval(torch.tensor(src, device="cuda"), torch.tensor(w, device="cuda"), grad=grad,
                    check_status=True)
    torch.cuda.synchronize()
    if grad:
        return out[0].cpu().numpy(), out[1].cpu().numpy()
    return out.cpu().numpy()


@pytest.mark.parametrize("p", [4, 5, 6, 8, 10, 12, 16])
@pytest.mark.parametrize("kernel,lam", [("laplace", 0.0), ("biharmonic", 0.0), ("yukawa", 2.0)])
def test_float_passes_match_oracle(torch_cuda, oracle, kernel, lam, p):
    src, w, idx = clustered(24000, 300 + p)
    ref = oracle.fmm_uniform(kernel, 3, p, 4, src, w, src, lam=lam, sample=idx)
    got = gpu_eval(torch_cuda, kernel, p, 4, src, w, lam)[idx]
    err = rel_l2(got, ref)
    print(f"{kernel} p={p}: rel L2 vs oracle {err:.3e}")
    assert err < TOL, err


@pytest.mark.parametrize("p", [6, 10])
def test_float_l2p_gradient_matches_oracle(torch_cuda, oracle, p):
    src, w, idx = clustered(20000, 400 + p)
    ref, gref = oracle.fmm_uniform("laplace", 3, p, 4, src, w, src, sample=idx, grad=True)
    got, g = gpu_eval(torch_cuda, "laplace", p, 4, src, w, 0.0, grad=True)
    assert rel_l2(got[idx], ref) < TOL
    assert rel_l2(g[idx], gref) < TOL


def test_fp32_modes_use_the_same_passes(torch_cuda, oracle):
    # the FP32 forms (CUDA-core and FFT M2L) go through the same float passes
    src, w, idx = clustered(16000, 77)
    ref = oracle.fmm_uniform("laplace", 3, 8, 3, src, w, src, sample=idx)
    for prec in ("fp32", "bf16x3"):
        got = gpu_eval(torch_cuda, "laplace", 8, 3, src, w, 0.0, precision=prec)[idx]
        assert rel_l2(got, ref) < (2e-5 if prec == "fp32" else 3e-5), prec
