"""Gradients of the backward workload: 3D Laplace p = 8, uniform octree L = 5,
10^6 sources and 10^6 separate targets, loss = sum_i u_i phi(x_i), u ~ N(0, 1).

* Against the oracle.  d loss/d w_j = psi(y_j) and d loss/d y_j =
  w_j grad psi(y_j), psi(y) = sum_i u_i G(y - x_i), are the transposed FMM
  (targets as sources with weights u); d loss/d x_i = u_i grad phi(x_i).  The
  oracle's swapped-roles FMM on the same tree gives them on a seeded sample.
* Against finite differences of the FP64 loss.  For 3D Laplace the compressed
  FMM equals the plain Taylor FMM (Thm 11; the Taylor polynomial of a harmonic
  function truncated at degree p is harmonic), and the Taylor FMM operator is
  symmetric -- sum_{i,q} (x-c_t)^i/i! d^{i+q}G(c_t-c_s) (c_s-y)^q/q! is
  unchanged when source and target trade places -- so the transposed FMM is the
  exact adjoint of the forward one and the gradients are the exact derivatives
  of the FMM loss itself.  Every coordinate of a seeded subset of 1,000 sources
  and 1,000 targets is checked through directional derivatives: the loss is
  evaluated at (y + h v, w + h v_w, x + h v_x) +- and (L+ - L-) / 2h compared
  with <v, grad>.  Points closer than 100 h to a face of their leaf are left
  out of the subset: there the truncated expansion changes box, and the
  FMM potential jumps by its truncation error.
"""
import numpy as np
import pytest

from paper_2305_17867_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FD_TOL = 1e-6      # relative, the FP64 gradients against finite differences
MIXED_GRAD = 5e-5  # tf32x3 gradients against the FP64 oracle (rel. L2)
L = 5
P = 8


def rel_l2(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def workload():
    wl = W.WORKLOADS["laplace3d_p8_L5_bwd_n1m"]
    src, w, tgt = W.make_inputs(wl)
    u = W.cotangent(len(tgt), wl.seed)
    return src, w, tgt, u


def autograd_grads(torch, precision, src, w, tgt, u):
    from paper_2305_17867_gb300.fmm import FMM, fmm_potential

    plan = FMM("laplace", d=3, p=P, levels=L, precision=precision)
    s = torch.tensor(src, device="cuda", requires_grad=True)
    t = torch.tensor(tgt, device="cuda", requires_grad=True)
    wt = torch.tensor(w, device="cuda", requires_grad=True)
    phi = fmm_potential(plan, s, wt, t)
    loss = (phi * torch.tensor(u, device="cuda")).sum()
    loss.backward()
    torch.cuda.synchronize()
    return (wt.grad.cpu().numpy(), s.grad.cpu().numpy(), t.grad.cpu().numpy(),
            phi.detach().cpu().numpy())


def away_from_faces(x, h, n_leaf):
    frac = x * n_leaf - np.floor(x * n_leaf)
    return np.all((frac > 100 * h * n_leaf) & (frac < 1 - 100 * h * n_leaf), axis=1)


def test_mixed_precision_gradients_against_oracle(torch_cuda, oracle, workload):
    src, w, tgt, u = workload
    gw, gs, gt, phi = autograd_grads(torch_cuda, "tf32x3", src, w, tgt, u)
    rng = np.random.default_rng(96)
    js = np.sort(rng.choice(len(w), 24, replace=False))
    it = np.sort(rng.choice(len(tgt), 24, replace=False))
    psi, gpsi = oracle.fmm_uniform("laplace", 3, P, L, tgt, u, src, sample=js, grad=True)
    ref_phi, gphi = oracle.fmm_uniform("laplace", 3, P, L, src, w, tgt, sample=it, grad=True)
    errs = {"grad_w": rel_l2(gw[js], psi),
            "grad_src": rel_l2(gs[js], w[js, None] * gpsi),
            "grad_tgt": rel_l2(gt[it], u[it, None] * gphi),
            "phi": rel_l2(phi[it], ref_phi)}
    print("tf32x3 gradients vs oracle:", {k: f"{v:.2e}" for k, v in errs.items()})
    assert max(errs.values()) < MIXED_GRAD, errs


def test_fp64_gradients_against_finite_differences(torch_cuda, workload):
    torch = torch_cuda
    from paper_2305_17867_gb300.fmm import FMM

    src, w, tgt, u = workload
    gw, gs, gt, _ = autograd_grads(torch, "fp64", src, w, tgt, u)
    g32 = autograd_grads(torch, "tf32x3", src, w, tgt, u)
    plan = FMM("laplace", d=3, p=P, levels=L, precision="fp64")
    ud = torch.tensor(u, device="cuda")

    def loss(sv, wv, tv):
        phi = plan.eval(torch.tensor(sv, device="cuda"), torch.tensor(wv, device="cuda"),
                        torch.tensor(tv, device="cuda"), check_status=True)
        return float(torch.dot(phi, ud))

    h = 1e-8
    n_leaf = 1 << L
    rng = np.random.default_rng(4321)
    js = rng.permutation(np.nonzero(away_from_faces(src, h, n_leaf))[0])[:1000]
    it = rng.permutation(np.nonzero(away_from_faces(tgt, h, n_leaf))[0])[:1000]
    assert len(js) == 1000 and len(it) == 1000
    worst = {}
    worst32 = {}
    for kind in ("src", "w", "tgt"):
        for _ in range(3):
            sp, sm_, wp, wm, tp, tm = src.copy(), src.copy(), w.copy(), w.copy(), tgt.copy(), \
                tgt.copy()
            if kind == "src":
                v = rng.uniform(-1, 1, (1000, 3))
                sp[js] += h * v
                sm_[js] -= h * v
                an, an32 = (gs[js] * v).sum(), (g32[1][js] * v).sum()
                step = h
            elif kind == "w":
                v = rng.uniform(-1, 1, 1000)
                hw = 1e-3  # the loss is linear in w: any step is exact
                wp[js] += hw * v
                wm[js] -= hw * v
                an, an32 = (gw[js] * v).sum(), (g32[0][js] * v).sum()
                step = hw
            else:
                v = rng.uniform(-1, 1, (1000, 3))
                tp[it] += h * v
                tm[it] -= h * v
                an, an32 = (gt[it] * v).sum(), (g32[2][it] * v).sum()
                step = h
            fd = (loss(sp, wp, tp) - loss(sm_, wm, tm)) / (2 * step)
            worst[kind] = max(worst.get(kind, 0.0), abs(fd - an) / abs(fd))
            worst32[kind] = max(worst32.get(kind, 0.0), abs(fd - an32) / abs(fd))
    print("fp64 gradients vs finite differences:", {k: f"{v:.2e}" for k, v in worst.items()})
    print("tf32x3 gradients vs finite differences:",
          {k: f"{v:.2e}" for k, v in worst32.items()})
    assert max(worst.values()) < FD_TOL, worst
    assert max(worst32.values()) < MIXED_GRAD, worst32
