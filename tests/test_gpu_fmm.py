"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

FP64 results must match the oracle's same-tree, same-p FMM to relative L2
error 1e-12 (the target the method's FP64 form is held to).
"""
import numpy as np
import pytest

from paper_2305_17867_gb300 import workloads as W

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


def gpu_fmm(torch, kernel, d, p, L, src, w, tgt=None, lam=0.0, precision="fp64", grad=False,
            root_lo=None, root_size=1.0):
    from paper_2305_17867_gb300.fmm import FMM

    plan = FMM(kernel, d=d, p=p, levels=L, lam=lam, precision=precision, root_lo=root_lo,
               root_size=root_size)
    s = torch.tensor(src, device="cuda")
    wt = torch.tensor(w, device="cuda")
    t = None if tgt is None else torch.tensor(tgt, device="cuda")
    out = plan.eval(s, wt, t, grad=grad, check_status=True)
    torch.cuda.synchronize()
    if grad:
        return out[0].cpu().numpy(), out[1].cpu().numpy()
    return out.cpu().numpy()


@pytest.mark.parametrize("L,n", [(2, 3000), (3, 20000), (4, 30011)])
def test_laplace3d_fp64_matches_oracle(torch_cuda, oracle, L, n):
    wl = W.WORKLOADS["laplace3d_p10_L5_n1m"]
    src, w, _ = W.make_inputs(wl, n_src=n)
    ref = oracle.fmm_uniform("laplace", 3, 10, L, src, w, src)
    got = gpu_fmm(torch_cuda, "laplace", 3, 10, L, src, w)
    assert rel_l2(got, ref) < FP64_TOL


def test_laplace2d_config_fp64(torch_cuda, oracle):
    wl = W.WORKLOADS["laplace2d_p8_L4_n2k"]
    src, w, _ = W.make_inputs(wl)
    ref = oracle.fmm_uniform("laplace", 2, 8, 4, src, w, src)
    got = gpu_fmm(torch_cuda, "laplace", 2, 8, 4, src, w)
    assert rel_l2(got, ref) < FP64_TOL
    direct = oracle.direct("laplace", 2, src, w, src)
    assert rel_l2(got, direct) < 1e-5


@pytest.mark.parametrize("kernel,p,lam", [("yukawa", 8, 1.0), ("yukawa", 12, 1.0),
                                          ("biharmonic", 4, 0.0), ("biharmonic", 8, 0.0)])
def test_other_kernels_fp64_matches_oracle(torch_cuda, oracle, kernel, p, lam):
    rng = np.random.default_rng(7)
    src = rng.random((9000, 3))
    w = rng.uniform(-1, 1, 9000)
    tgt = rng.random((5000, 3))
    ref = oracle.fmm_uniform(kernel, 3, p, 3, src, w, tgt, lam=lam)
    got = gpu_fmm(torch_cuda, kernel, 3, p, 3, src, w, tgt, lam=lam)
    assert rel_l2(got, ref) < FP64_TOL


def test_gradient_fp64_matches_oracle(torch_cuda, oracle):
    rng = np.random.default_rng(8)
    src = rng.random((12000, 3))
    w = rng.uniform(-1, 1, 12000)
    tgt = rng.random((7000, 3))
    ref, gref = oracle.fmm_uniform("laplace", 3, 8, 3, src, w, tgt, grad=True)
    got, g = gpu_fmm(torch_cuda, "laplace", 3, 8, 3, src, w, tgt, grad=True)
    assert rel_l2(got, ref) < FP64_TOL
    assert rel_l2(g, gref) < FP64_TOL


def test_full_size_laplace3d_sampled(torch_cuda, oracle):
    # the measured workload: 1e6 uniform points, p = 10, L = 5; the oracle
    # evaluates a seeded sample of targets one by one on the same tree.
    wl = W.WORKLOADS["laplace3d_p10_L5_n1m"]
    src, w, _ = W.make_inputs(wl)
    got = gpu_fmm(torch_cuda, "laplace", 3, 10, 5, src, w)
    idx = np.random.default_rng(99).choice(len(w), 64, replace=False)
    ref = oracle.fmm_uniform("laplace", 3, 10, 5, src, w, src, sample=idx)
    assert rel_l2(got[idx], ref) < FP64_TOL


# Mixed-precision tolerances (relative L2 against the FP64 oracle on the same
# tree).  fp32 and tf32x3 keep ~22-24 significant bits per product, so the
# result carries ~1e-7 relative error amplified by the cancellation of the
# sums; bf16x3 keeps ~16 bits (hi + lo bf16, unit roundoff ~2^-17 per
# operand); tf32 keeps 11 bits (unit roundoff 2^-11 ~ 4.9e-4 per operand).
MIXED_TOL = {"fp32": 2e-6, "tf32x3": 2e-6, "bf16x3": 5e-5, "tf32": 2e-3}


@pytest.mark.parametrize("precision", ["fp32", "tf32x3", "bf16x3", "tf32"])
@pytest.mark.parametrize("L,n", [(3, 20000), (4, 30011)])
def test_mixed_precision_error(torch_cuda, oracle, precision, L, n):
    wl = W.WORKLOADS["laplace3d_p10_L5_n1m"]
    src, w, _ = W.make_inputs(wl, n_src=n)
    ref = oracle.fmm_uniform("laplace", 3, 10, L, src, w, src)
    got = gpu_fmm(torch_cuda, "laplace", 3, 10, L, src, w, precision=precision)
    assert rel_l2(got, ref) < MIXED_TOL[precision]


@pytest.mark.parametrize("precision", ["tf32x3", "bf16x3", "tf32"])
def test_tensor_m2l_full_size_sampled(torch_cuda, oracle, precision):
    wl = W.WORKLOADS["laplace3d_p10_L5_n1m"]
    src, w, _ = W.make_inputs(wl)
    got = gpu_fmm(torch_cuda, "laplace", 3, 10, 5, src, w, precision=precision)
    idx = np.random.default_rng(98).choice(len(w), 48, replace=False)
    ref = oracle.fmm_uniform("laplace", 3, 10, 5, src, w, src, sample=idx)
    assert rel_l2(got[idx], ref) < MIXED_TOL[precision]


@pytest.mark.parametrize("precision,tol", [("tf32x3", 1e-5), ("bf16x3", 2e-4)])
@pytest.mark.parametrize("kernel,p,lam", [("yukawa", 12, 1.0), ("biharmonic", 8, 0.0)])
def test_tensor_m2l_other_kernels(torch_cuda, oracle, kernel, p, lam, precision, tol):
    # |j| = 169 (Yukawa p=12) and 130 (biharmonic p=8): two 128-row M tiles
    rng = np.random.default_rng(17)
    src = rng.random((20000, 3))
    w = rng.uniform(-1, 1, 20000)
    ref = oracle.fmm_uniform(kernel, 3, p, 4, src, w, src, lam=lam)
    got = gpu_fmm(torch_cuda, kernel, 3, p, 4, src, w, lam=lam, precision=precision)
    assert rel_l2(got, ref) < tol


# ---- edge cases -------------------------------------------------------------
def test_empty_sources_and_targets(torch_cuda):
    z = np.zeros((0, 3))
    tgt = np.random.default_rng(1).random((50, 3))
    got = gpu_fmm(torch_cuda, "laplace", 3, 4, 2, z, np.zeros(0), tgt)
    assert np.all(got == 0.0)
    got = gpu_fmm(torch_cuda, "laplace", 3, 4, 2, tgt, np.ones(50), z)
    assert got.shape == (0,)


def test_clustered_and_boundary_points(torch_cuda, oracle):
    # 600 points in one leaf (several passes of the leaf kernel), points on
    # the root box faces, and exact duplicates (skipped pairs).
    rng = np.random.default_rng(3)
    a = 0.51 + 0.01 * rng.random((600, 3))
    b = rng.random((400, 3))
    b[:20, 0] = 1.0
    b[20:40, 1] = 0.0
    src = np.concatenate([a, b, a[:10]])
    w = rng.uniform(-1, 1, len(src))
    ref = oracle.fmm_uniform("laplace", 3, 6, 3, src, w, src)
    got = gpu_fmm(torch_cuda, "laplace", 3, 6, 3, src, w)
    assert rel_l2(got, ref) < FP64_TOL


def test_auto_root_box(torch_cuda, oracle):
    rng = np.random.default_rng(4)
    src = rng.random((5000, 3)) * 3.0 - 1.0
    w = rng.uniform(-1, 1, 5000)
    lo = src.min(axis=0)
    size = float((src.max(axis=0) - lo).max())
    ref = oracle.fmm_uniform("laplace", 3, 6, 3, src, w, src, lo=lo, size=size)
    got = gpu_fmm(torch_cuda, "laplace", 3, 6, 3, src, w, root_size=0.0)
    assert rel_l2(got, ref) < FP64_TOL


def test_domain_error_flag(torch_cuda):
    from paper_2305_17867_gb300.fmm import FMM
    from paper_2305_17867_gb300._lib import FMMError

    torch = torch_cuda
    plan = FMM("laplace", d=3, p=4, levels=2)
    src = torch.rand(100, 3, device="cuda", dtype=torch.float64)
    src[0, 0] = 1.5
    with pytest.raises(FMMError) as ei:
        plan.eval(src, torch.ones(100, device="cuda", dtype=torch.float64), check_status=True)
    assert ei.value.code == -6


def test_bad_arguments_rejected(torch_cuda):
    from paper_2305_17867_gb300.fmm import FMM
    from paper_2305_17867_gb300._lib import FMMError

    with pytest.raises(FMMError):
        FMM("laplace", d=3, p=0, levels=3)
    with pytest.raises(FMMError):
        FMM("yukawa", d=2, p=4, levels=3, lam=1.0)
    with pytest.raises(FMMError):
        FMM("laplace", d=3, p=4, levels=9)


def test_autograd_against_direct_gradients(torch_cuda, oracle):
    torch = torch_cuda
    from paper_2305_17867_gb300.fmm import FMM, fmm_potential

    rng = np.random.default_rng(21)
    n = 1000
    src = rng.random((n, 3))
    tgt = rng.random((n, 3))
    w = rng.uniform(-1, 1, n)
    u = rng.normal(size=n)
    plan = FMM("laplace", d=3, p=12, levels=3)
    s = torch.tensor(src, device="cuda", requires_grad=True)
    t = torch.tensor(tgt, device="cuda", requires_grad=True)
    wt = torch.tensor(w, device="cuda", requires_grad=True)
    phi = fmm_potential(plan, s, wt, t)
    loss = (phi * torch.tensor(u, device="cuda")).sum()
    loss.backward()
    # d/dw_j = sum_i u_i G(x_i - y_j); d/dx_i = u_i grad phi(x_i);
    # d/dy_j = w_j grad psi(y_j), psi(y) = sum_i u_i G(y - x_i).
    # Same tree and order as the oracle's FMM (transposed for psi): FP64 parity.
    gw_fmm, gy_fmm = oracle.fmm_uniform("laplace", 3, 12, 3, tgt, u, src, grad=True)
    _, gx_fmm = oracle.fmm_uniform("laplace", 3, 12, 3, src, w, tgt, grad=True)
    assert rel_l2(wt.grad.cpu().numpy(), gw_fmm) < FP64_TOL
    assert rel_l2(t.grad.cpu().numpy(), u[:, None] * gx_fmm) < FP64_TOL
    assert rel_l2(s.grad.cpu().numpy(), w[:, None] * gy_fmm) < FP64_TOL
    # against the plain definition: within the p = 12 truncation error
    gw_ref, gy = oracle.direct("laplace", 3, tgt, u, src, grad=True)
    _, gx = oracle.direct("laplace", 3, src, w, tgt, grad=True)
    assert rel_l2(wt.grad.cpu().numpy(), gw_ref) < 1e-6
    assert rel_l2(t.grad.cpu().numpy(), u[:, None] * gx) < 2e-5
    assert rel_l2(s.grad.cpu().numpy(), w[:, None] * gy) < 2e-5
    # finite differences of the FMM loss itself on a few coordinates
    def loss_at(sv, wv, tv):
        ph = plan.eval(torch.tensor(sv, device="cuda"), torch.tensor(wv, device="cuda"),
                       torch.tensor(tv, device="cuda"))
        return float((ph.cpu().numpy() * u).sum())
    h = 1e-6
    for (arr, which, i, k) in [(src, "s", 3, 0), (tgt, "t", 5, 2), (w, "w", 7, None)]:
        ap, am = arr.copy(), arr.copy()
        if k is None:
            ap[i] += h
            am[i] -= h
        else:
            ap[i, k] += h
            am[i, k] -= h
        args_p = {"s": (ap, w, tgt), "t": (src, w, ap), "w": (src, ap, tgt)}[which]
        args_m = {"s": (am, w, tgt), "t": (src, w, am), "w": (src, am, tgt)}[which]
        fd = (loss_at(*args_p) - loss_at(*args_m)) / (2 * h)
        g = {"s": s.grad, "t": t.grad, "w": wt.grad}[which].cpu().numpy()
        an = g[i] if k is None else g[i, k]
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (which, fd, an)


@pytest.mark.parametrize("d,L", [(3, 5), (2, 4), (3, 3)])
def test_uniform_m2l_translation_count(torch_cuda, d, L):
    # the library's count of interaction-list entries against an independent
    # count over the box grid
    import bench
    from paper_2305_17867_gb300.fmm import FMM

    plan = FMM("laplace", d=d, p=4, levels=L)
    assert plan.last_m2l_count() == bench.m2l_count(d, L)


@pytest.mark.parametrize("kernel,p,lam", [("laplace", 8, 0.0), ("yukawa", 8, 1.0),
                                          ("biharmonic", 6, 0.0)])
@pytest.mark.parametrize("precision", ["fp32", "tf32x3"])
def test_mixed_precision_gradient(torch_cuda, oracle, kernel, p, lam, precision):
    # the float leaf kernel with the analytic gradient (packed pair arithmetic),
    # separate targets and sources = targets
    rng = np.random.default_rng(31)
    src = rng.random((20000, 3))
    w = rng.uniform(-1, 1, 20000)
    for tgt in (rng.random((9000, 3)), None):
        t = src if tgt is None else tgt
        ref, gref = oracle.fmm_uniform(kernel, 3, p, 4, src, w, t, lam=lam, grad=True)
        got, g = gpu_fmm(torch_cuda, kernel, 3, p, 4, src, w, tgt, lam=lam,
                         precision=precision, grad=True)
        assert rel_l2(got, ref) < 5e-6
        assert rel_l2(g, gref) < 5e-5


def test_backward_workload_full_size_sampled(torch_cuda, oracle):
    # 1e6 sources and 1e6 separate targets, p = 8, L = 5: potential and
    # target gradient on seeded sampled targets (FP64 against the oracle,
    # tf32x3 within the mixed-precision tolerance)
    wl = W.WORKLOADS["laplace3d_p8_L5_bwd_n1m"]
    src, w, tgt = W.make_inputs(wl)
    idx = np.random.default_rng(95).choice(len(tgt), 24, replace=False)
    ref, gref = oracle.fmm_uniform("laplace", 3, 8, 5, src, w, tgt, sample=idx, grad=True)
    got, g = gpu_fmm(torch_cuda, "laplace", 3, 8, 5, src, w, tgt, grad=True)
    assert rel_l2(got[idx], ref) < FP64_TOL
    assert rel_l2(g[idx], gref) < FP64_TOL
    got, g = gpu_fmm(torch_cuda, "laplace", 3, 8, 5, src, w, tgt, grad=True,
                     precision="tf32x3")
    assert rel_l2(got[idx], ref) < MIXED_TOL["tf32x3"]
    assert rel_l2(g[idx], gref) < 2e-5


def test_biharmonic_workload_full_size_sampled(torch_cuda, oracle):
    # 4e6 points, L = 6, p = 8: dense tensor-core M2L and the FFT form
    from paper_2305_17867_gb300.fmm import FMM

    wl = W.WORKLOADS["biharmonic3d_p8_L6_n4m"]
    src, w, _ = W.make_inputs(wl)
    idx = np.random.default_rng(94).choice(len(w), 16, replace=False)
    ref = oracle.fmm_uniform("biharmonic", 3, 8, 6, src, w, src, sample=idx)
    s = torch_cuda.tensor(src, device="cuda")
    wt = torch_cuda.tensor(w, device="cuda")
    for prec, m2l, tol in (("tf32x3", "dense", 2e-5), ("fp32", "fft", 1e-4),
                           ("fp64", "fft", 1e-12)):
        plan = FMM("biharmonic", d=3, p=8, levels=6, precision=prec, m2l=m2l)
        got = plan.eval(s, wt, check_status=True).cpu().numpy()
        assert rel_l2(got[idx], ref) < tol, (prec, m2l)


# ---- user-supplied PDEs (eq. (define_pde_op)) -------------------------------
def _plan_eval(torch, kernel, p, L, src, w, pde=None, lam=0.0, precision="fp64"):
    from paper_2305_17867_gb300.fmm import FMM

    plan = FMM(kernel, d=3, p=p, levels=L, lam=lam, precision=precision, pde=pde)
    out = plan.eval(torch.tensor(src, device="cuda"), torch.tensor(w, device="cuda"),
                    check_status=True)
    return out.cpu().numpy(), plan


def test_user_pde_equal_to_the_kernels_own(torch_cuda):
    # the same operators given explicitly (scaled, reordered) compress identically
    rng = np.random.default_rng(34)
    src = rng.random((20000, 3))
    w = rng.uniform(-1, 1, 20000)
    lap = ([(0, 0, 2), (2, 0, 0), (0, 2, 0)], [3.0, 3.0, 3.0])
    a, _ = _plan_eval(torch_cuda, "laplace", 8, 3, src, w)
    b, _ = _plan_eval(torch_cuda, "laplace", 8, 3, src, w, pde=lap)
    assert np.array_equal(a, b)
    yuk = ([(2, 0, 0), (0, 2, 0), (0, 0, 2), (0, 0, 0)], [1.0, 1.0, 1.0, -1.0])
    a, _ = _plan_eval(torch_cuda, "yukawa", 8, 3, src, w, lam=1.0)
    b, _ = _plan_eval(torch_cuda, "yukawa", 8, 3, src, w, pde=yuk, lam=1.0)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("kernel,lam", [("laplace", 0.0), ("biharmonic", 0.0),
                                        ("yukawa", 1.0)])
def test_uncompressed_taylor_fmm(torch_cuda, oracle, kernel, lam):
    # PDE d_z^(p+1): every multi-index of M(p) is stored and nothing is
    # compressed, i.e. the plain Taylor FMM (Sec. 2), held to the oracle's
    # uncompressed FMM
    p, L = 6, 3
    rng = np.random.default_rng(35)
    src = rng.random((12000, 3))
    w = rng.uniform(-1, 1, 12000)
    pde = ([(0, 0, p + 1)], [1.0])
    got, plan = _plan_eval(torch_cuda, kernel, p, L, src, w, pde=pde, lam=lam)
    assert plan.nj == plan.nfull == (p + 1) * (p + 2) * (p + 3) // 6
    ref = oracle.fmm_uniform(kernel, 3, p, L, src, w, src, lam=lam, compressed=False)
    assert rel_l2(got, ref) < FP64_TOL
    got, _ = _plan_eval(torch_cuda, kernel, p, L, src, w, pde=pde, lam=lam,
                        precision="tf32x3")
    assert rel_l2(got, ref) < 2e-5


def test_user_pde_the_kernel_does_not_satisfy_is_rejected(torch_cuda):
    # eq. (Pv): the plan checks P applied to the kernel's derivatives at a far
    # offset; a PDE the kernel does not satisfy would compress away information
    from paper_2305_17867_gb300.fmm import FMM
    from paper_2305_17867_gb300._lib import FMMError

    lap = ([(2, 0, 0), (0, 2, 0), (0, 0, 2)], [1.0, 1.0, 1.0])
    screened = ([(2, 0, 0), (0, 2, 0), (0, 0, 2), (0, 0, 0)], [1.0, 1.0, 1.0, -1.0])
    for kernel, pde, lam in (("laplace", screened, 0.0), ("biharmonic", lap, 0.0),
                             ("yukawa", lap, 1.0), ("helmholtz", screened, 1.0)):
        with pytest.raises(FMMError) as ei:
            FMM(kernel, d=3, p=8, levels=3, lam=lam, pde=pde)
        assert ei.value.code == -2, kernel
    # the kernel's own operators, and the Helmholtz operator for Helmholtz, pass
    FMM("laplace", d=3, p=8, levels=3, pde=lap)
    FMM("helmholtz", d=3, p=8, levels=3, lam=1.0,
        pde=([(2, 0, 0), (0, 2, 0), (0, 0, 2), (0, 0, 0)], [1.0, 1.0, 1.0, 1.0]))


def test_user_pde_of_higher_order(torch_cuda, oracle):
    # G = 1/(4 pi r) also satisfies d_z Laplacian (order 3): the plan keeps the
    # multi-indices with m_z < 3 and decompresses through the third-order
    # recurrence; the potentials are those of the kernel's own compression
    rng = np.random.default_rng(36)
    src = rng.random((15000, 3))
    w = rng.uniform(-1, 1, 15000)
    pde = ([(2, 0, 1), (0, 2, 1), (0, 0, 3)], [1.0, 1.0, 1.0])
    got, plan = _plan_eval(torch_cuda, "laplace", 8, 3, src, w, pde=pde)
    assert plan.c == 3 and plan.nj == 45 + 36 + 28  # slabs m_z = 0, 1, 2 of M(8)
    ref = oracle.fmm_uniform("laplace", 3, 8, 3, src, w, src)
    assert rel_l2(got, ref) < FP64_TOL


@pytest.mark.parametrize("d,L,same", [(3, 4, True), (3, 3, False), (2, 5, False)])
def test_last_stats(torch_cuda, d, L, same):
    # fmm_last_stats against independent host counts: the interaction lists of
    # a uniform tree and the near-field pairs of the point set
    import bench
    from paper_2305_17867_gb300.fmm import FMM

    rng = np.random.default_rng(40 + d + L)
    src = rng.random((20000, d))
    tgt = src if same else rng.random((7000, d))
    w = rng.uniform(-1, 1, 20000)
    plan = FMM("laplace", d=d, p=6, levels=L, precision="fp64")
    plan.set_timing(True)
    plan.eval(torch_cuda.tensor(src, device="cuda"), torch_cuda.tensor(w, device="cuda"),
              None if same else torch_cuda.tensor(tgt, device="cuda"))
    st = plan.last_stats()
    assert st["status"] == 0 and st["depth"] == L and st["launches"] > 0
    assert st["m2l_translations"] == bench.m2l_count(d, L)
    pairs = bench.near_pairs(src, tgt, L) + (len(src) if same else 0)  # coincident included
    assert st["p2p_pairs"] == pairs
    assert sum(st["phase_ms"].values()) > 0.0
    plan.set_timing(False)


@pytest.mark.parametrize("precision,same", [("fp64", True), ("tf32x3", False)])
def test_float32_entry(torch_cuda, precision, same):
    # fmm_eval_f32 widens the float32 inputs on the device and then runs the
    # evaluation of fmm_eval: its results are fmm_eval's on the widened inputs,
    # rounded to float32
    from paper_2305_17867_gb300.fmm import FMM

    torch = torch_cuda
    rng = np.random.default_rng(45)
    s32 = torch.tensor(rng.random((30000, 3)), device="cuda", dtype=torch.float32)
    w32 = torch.tensor(rng.uniform(-1, 1, 30000), device="cuda", dtype=torch.float32)
    t32 = s32 if same else torch.tensor(rng.random((9000, 3)), device="cuda",
                                        dtype=torch.float32)
    plan = FMM("laplace", d=3, p=8, levels=4, precision=precision)
    phi32, g32 = plan.eval_f32(s32, w32, None if same else t32, grad=True, check_status=True)
    phi64, g64 = plan.eval(s32.double(), w32.double(), None if same else t32.double(),
                           grad=True, check_status=True)
    torch.cuda.synchronize()
    assert phi32.dtype == torch.float32 and g32.dtype == torch.float32
    assert torch.equal(phi32, phi64.float())
    assert torch.equal(g32, g64.float())
