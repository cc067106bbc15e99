"""GPU parity of the adaptive-tree FMM (U, V, W, X lists) against the oracle.

The tree (boxes and depth) must match the oracle's exactly; potentials must
match the oracle's adaptive FMM with the same tree and p to 1e-12 (FP64), and
to the stated tolerances in the float and tensor-core forms.
"""
import numpy as np
import pytest

from paper_2305_17867_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
TC_TOL = {"tf32x3": 2e-5, "bf16x3": 1e-4, "tf32": 3e-3}


def rel_l2(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def gpu_adaptive(torch, kernel, p, src, w, tgt=None, lam=0.0, max_leaf=64, depth=10,
                 counts=False, precision="fp64"):
    from paper_2305_17867_gb300.fmm import FMM

    plan = FMM(kernel, d=3, p=p, levels=-depth, lam=lam, max_leaf=max_leaf, precision=precision)
    s = torch.tensor(src, device="cuda")
    wt = torch.tensor(w, device="cuda")
    t = None if tgt is None else torch.tensor(tgt, device="cuda")
    out = plan.eval(s, wt, t, check_status=True)
    torch.cuda.synchronize()
    if counts:
        return out.cpu().numpy(), plan.last_tree(), plan.last_m2l_count()
    return out.cpu().numpy(), plan.last_tree()


def plummer_case(n_src, n_tgt, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    src = W.plummer_points(rng, n_src)
    w = rng.normal(size=n_src)
    tgt = rng.random((n_tgt, 3))
    return src, w, tgt


def test_complete_tree_matches_uniform(torch_cuda, oracle):
    rng = np.random.default_rng(41)
    src = rng.random((12000, 3))
    w = rng.uniform(-1, 1, 12000)
    got, (nb, depth) = gpu_adaptive(torch_cuda, "laplace", 8, src, w, max_leaf=200)
    assert depth == 3 and nb == 1 + 8 + 64 + 512
    ref = oracle.fmm_uniform("laplace", 3, 8, 3, src, w, src)
    assert rel_l2(got, ref) < FP64_TOL


@pytest.mark.parametrize("kernel,p,lam,n", [("laplace", 8, 0.0, 20000), ("laplace", 12, 0.0, 6000),
                                            ("yukawa", 8, 1.0, 20000), ("yukawa", 12, 1.0, 5000),
                                            ("biharmonic", 6, 0.0, 20000)])
def test_plummer_matches_oracle(torch_cuda, oracle, kernel, p, lam, n):
    src, w, tgt = plummer_case(n, n // 5, 42)
    ref, st, _ = oracle.fmm_adaptive(kernel, 3, p, src, w, tgt, max_leaf=32, lam=lam,
                                     want_stats=True)
    assert st["W"] > 0 and st["X"] > 0
    # W and X pairs of both kinds: summed directly (boxes of at most |j|
    # points) and through M2P / P2L (the few larger boxes)
    assert 0 < st["WX_direct"] < st["W"] + st["X"]
    got, (nb, depth), nv = gpu_adaptive(torch_cuda, kernel, p, src, w, tgt, lam=lam,
                                        max_leaf=32, counts=True)
    assert (nb, depth) == (st["boxes"], st["depth"])
    assert nv == st["V"]  # interaction-list entries of the boxes holding targets
    assert rel_l2(got, ref) < FP64_TOL


def test_sources_are_targets(torch_cuda, oracle):
    src, w, _ = plummer_case(15000, 1, 43)
    ref = oracle.fmm_adaptive("laplace", 3, 8, src, w, src, max_leaf=40)
    got, _ = gpu_adaptive(torch_cuda, "laplace", 8, src, w, max_leaf=40)
    assert rel_l2(got, ref) < FP64_TOL


def test_depth_cap(torch_cuda, oracle):
    rng = np.random.default_rng(44)
    src = np.concatenate([0.3 + 1e-4 * rng.random((2000, 3)), rng.random((3000, 3))])
    w = rng.normal(size=5000)
    tgt = rng.random((2000, 3))
    ref, st, _ = oracle.fmm_adaptive("laplace", 3, 6, src, w, tgt, max_leaf=8, max_depth=5,
                                     want_stats=True)
    assert 0 < st["WX_direct"] < st["W"] + st["X"]  # the capped cluster: M2P and P2L
    got, (nb, depth) = gpu_adaptive(torch_cuda, "laplace", 6, src, w, tgt, max_leaf=8, depth=5)
    assert depth == 5 and nb == st["boxes"]
    assert rel_l2(got, ref) < FP64_TOL


def test_tiny_and_empty(torch_cuda, oracle):
    rng = np.random.default_rng(45)
    src = rng.random((50, 3))
    w = rng.normal(size=50)
    tgt = rng.random((30, 3))
    ref = oracle.direct("laplace", 3, src, w, tgt)  # one leaf: all direct
    got, (nb, depth) = gpu_adaptive(torch_cuda, "laplace", 6, src, w, tgt, max_leaf=100)
    assert (nb, depth) == (1, 0)
    assert rel_l2(got, ref) < 1e-14
    z = np.zeros((0, 3))
    got, _ = gpu_adaptive(torch_cuda, "laplace", 6, z, np.zeros(0), tgt, max_leaf=8)
    assert np.all(got == 0.0)


@pytest.mark.parametrize("precision", ["fp64", "bf16x3"])
def test_yukawa_plummer_full_size_sampled(torch_cuda, oracle, precision):
    # the adaptive Yukawa workload: 2e6 Plummer sources, 2e6 uniform targets,
    # p = 12, at most 64 points per leaf; the oracle evaluates 16 seeded
    # targets on the same tree.  In BF16x3 the sparse levels (6-8) run the
    # tensor-core M2L over gathered target lists of thousands of entries per
    # class, the dense ones (2-5) over window tiles.
    wl = W.WORKLOADS["yukawa3d_p12_adaptive_n2m"]
    src, w, tgt = W.make_inputs(wl)
    got, (nb, depth) = gpu_adaptive(torch_cuda, "yukawa", 12, src, w, tgt, lam=wl.lam,
                                    max_leaf=wl.max_leaf, precision=precision)
    idx = np.random.default_rng(96).choice(len(tgt), 16, replace=False)
    ref, st, _ = oracle.fmm_adaptive("yukawa", 3, 12, src, w, tgt, max_leaf=wl.max_leaf,
                                     lam=wl.lam, sample=idx, want_stats=True)
    assert (nb, depth) == (st["boxes"], st["depth"])
    assert rel_l2(got[idx], ref) < (FP64_TOL if precision == "fp64" else TC_TOL[precision])


# Float forms (P2M, M2L, P2L, L2P, P2P, M2P in float; M2M and L2L in
# double-word floats, the derivative tables in FP64): ~24-bit products with the
# sums' cancellation.
FP32_TOL = 2e-5


@pytest.mark.parametrize("kernel,p,lam", [("laplace", 8, 0.0), ("yukawa", 8, 1.0),
                                          ("biharmonic", 6, 0.0), ("yukawa", 12, 1.0)])
def test_adaptive_fp32_matches_oracle(torch_cuda, oracle, kernel, p, lam):
    src, w, tgt = plummer_case(20000 if p < 12 else 6000, 4000 if p < 12 else 1200, 42)
    ref = oracle.fmm_adaptive(kernel, 3, p, src, w, tgt, max_leaf=32, lam=lam)
    got, _ = gpu_adaptive(torch_cuda, kernel, p, src, w, tgt, lam=lam, max_leaf=32,
                          precision="fp32")
    err = rel_l2(got, ref)
    print(kernel, p, "adaptive fp32 rel err", err)
    assert err < FP32_TOL


def test_adaptive_fp32_sources_are_targets(torch_cuda, oracle):
    src, w, _ = plummer_case(15000, 1, 43)
    ref = oracle.fmm_adaptive("laplace", 3, 8, src, w, src, max_leaf=40)
    got, _ = gpu_adaptive(torch_cuda, "laplace", 8, src, w, max_leaf=40, precision="fp32")
    assert rel_l2(got, ref) < FP32_TOL


def test_adaptive_fp32_leaf_shapes(torch_cuda, oracle):
    # the float leaf pass spreads a leaf's targets over the lanes of a warp:
    # leaves of up to 64 targets (sources are targets, 64 per leaf), a cluster
    # below the depth cap whose leaves hold hundreds of targets (taken 64 at a
    # time), and W boxes above |j| sources next to it (M2P, the second kernel)
    rng = np.random.default_rng(46)
    src = np.concatenate([0.3 + 1e-3 * rng.random((3000, 3)), rng.random((9000, 3))])
    w = rng.normal(size=len(src))
    ref, st, _ = oracle.fmm_adaptive("laplace", 3, 6, src, w, src, max_leaf=64, max_depth=6,
                                     want_stats=True)
    assert 0 < st["WX_direct"] < st["W"] + st["X"]
    got, (nb, depth) = gpu_adaptive(torch_cuda, "laplace", 6, src, w, max_leaf=64, depth=6,
                                    precision="fp32")
    assert depth == 6 and nb == st["boxes"]
    assert rel_l2(got, ref) < FP32_TOL


# Tensor-core M2L on the adaptive tree (dense levels in window tiles, sparse
# ones over gathered target lists); tolerances (TC_TOL, top of the file) as for
# the uniform tree's mixed-precision forms.


@pytest.mark.parametrize("precision", ["tf32x3", "bf16x3", "tf32"])
@pytest.mark.parametrize("kernel,p,lam", [("laplace", 8, 0.0), ("yukawa", 12, 1.0),
                                          ("biharmonic", 6, 0.0)])
def test_adaptive_tensor_m2l(torch_cuda, oracle, kernel, p, lam, precision):
    n = 20000 if p < 12 else 6000
    src, w, tgt = plummer_case(n, n // 5, 42)
    ref, st, _ = oracle.fmm_adaptive(kernel, 3, p, src, w, tgt, max_leaf=32, lam=lam,
                                     want_stats=True)
    got, (nb, depth), nv = gpu_adaptive(torch_cuda, kernel, p, src, w, tgt, lam=lam,
                                        max_leaf=32, counts=True, precision=precision)
    assert nv == st["V"]
    err = rel_l2(got, ref)
    print(kernel, p, precision, "adaptive tensor-core rel err", err)
    assert err < TC_TOL[precision]


def test_adaptive_tensor_m2l_window_paths(torch_cuda, oracle):
    # Two Plummer clusters (scale 0.03) on the diagonal and uniform targets:
    # the deep levels' windows span both clusters.  With 80,000 sources and
    # 16,000 targets at most 32 points per leaf (Laplace p = 8, BF16x3: 128
    # K columns per window row), a CPU count of the tree and of the window
    # arena gives levels 7-8 windows larger than the arena (CUDA-core M2L),
    # levels 5-6 gathered target lists with level 5 not fitting beside level
    # 6 (a second contraction launch over the reused arena), levels 2-4 tiles.
    rng = np.random.Generator(np.random.PCG64(11))
    half = []
    for c in (0.2, 0.8):
        half.append(W.plummer_points(rng, 40000, 3, a=0.03, center=0.5) - 0.5 + c)
    src = np.clip(np.concatenate(half), 0.0, 1.0 - 1e-12)
    w = rng.normal(size=src.shape[0])
    tgt = rng.random((16000, 3))
    idx = np.sort(np.random.default_rng(12).choice(len(tgt), 64, replace=False))
    ref, st, _ = oracle.fmm_adaptive("laplace", 3, 8, src, w, tgt, max_leaf=32, sample=idx,
                                     want_stats=True)
    got, (nb, depth) = gpu_adaptive(torch_cuda, "laplace", 8, src, w, tgt, max_leaf=32,
                                    precision="bf16x3")
    assert (nb, depth) == (st["boxes"], st["depth"])
    err = rel_l2(got[idx], ref)
    print("two clusters, bf16x3 adaptive rel err", err, "depth", depth)
    assert err < TC_TOL["bf16x3"]
