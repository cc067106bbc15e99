"""Pins of the CPU oracle against facts the paper and the mathematics fix.

None of these compare the oracle with itself re-typed: each check uses an
independent closed form, an identity the paper proves, a value the paper
prints, or brute force on a tiny input.
"""
import math
import os

import numpy as np
import pytest
from scipy.special import eval_legendre

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def binom(n, k):
    return math.comb(n, k) if 0 <= k <= n else 0


# --------------------------------------------------------------------------
# Sec. 3.1: |j| = N(p) - N(p-c) with N(p) = C(p+d, d); shape of j (Fig. j,
# Lemma 5, Sec. 4.4.1).
# --------------------------------------------------------------------------
@pytest.mark.parametrize("d,p,kernel", [(2, 8, "laplace"), (2, 16, "biharmonic"),
                                        (3, 10, "laplace"), (3, 12, "yukawa"),
                                        (3, 4, "biharmonic"), (3, 16, "biharmonic")])
def test_stored_count_and_shape(oracle, d, p, kernel):
    e = oracle.Expansion(d, p, kernel, lam=1.0)
    c = e.c
    assert e.nfull == binom(p + d, d)
    assert e.nj == binom(p + d, d) - binom(p - c + d, d)
    # Lemma 5 with the last axis slowest: j = {m : m_d < c}
    stored = {tuple(e.mi[i]) for i in e.j}
    expect = {tuple(m) for m in e.mi if m[-1] < c}
    assert stored == expect


def test_fig_j_laplace_2d(oracle):
    # Sec. 4.4.1 / Fig. j(a): j = {(n,0): n<=p} U {(n,1): n<=p-1}
    e = oracle.Expansion(2, 16, "laplace")
    stored = {tuple(e.mi[i]) for i in e.j}
    assert stored == {(n, 0) for n in range(17)} | {(n, 1) for n in range(16)}
    assert e.nj == 2 * 16 + 1


def test_fig_j_mixed_pde(oracle):
    # Fig. j(c) / eq. (two-slice-example): the PDE d_x d_y (+ d_x + d_y) keeps
    # exactly the two axis slices m_x = 0 or m_y = 0.
    mi1 = oracle.multi_indices(2, 2)
    a = np.zeros(len(mi1))
    a[oracle.mi_index(2, [1, 1])] = 1.0
    for with_lower in (False, True):
        if with_lower:
            a[oracle.mi_index(2, [1, 0])] = 1.0
            a[oracle.mi_index(2, [0, 1])] = 1.0
        e = oracle.Expansion(2, 12, pde=(2, a))
        stored = {tuple(e.mi[i]) for i in e.j}
        assert stored == {tuple(m) for m in e.mi if m[0] == 0 or m[1] == 0}


# --------------------------------------------------------------------------
# Sec. 4.4: derivatives of G against independent closed forms.
# --------------------------------------------------------------------------
def test_derivatives_laplace2d_complex_closed_form(oracle):
    # log r = Re log z, d_x = d/dz, d_y = i d/dz on holomorphic functions:
    # d_x^a d_y^b log r = Re[i^b (-1)^(n-1) (n-1)! z^-n], n = a + b >= 1.
    x = np.array([0.37, -0.81])
    pmax = 20
    D = oracle.derivatives("laplace", 2, pmax, x)
    z = complex(x[0], x[1])
    worst = 0.0
    for i, (a, b) in enumerate(oracle.multi_indices(2, pmax)):
        n = a + b
        if n == 0:
            ref = math.log(abs(z))
        else:
            ref = ((1j) ** b * (-1) ** (n - 1) * math.factorial(n - 1) * z ** (-n)).real
        scale = math.factorial(max(n - 1, 0)) / abs(z) ** max(n, 1)
        worst = max(worst, abs(D[i] - ref) / scale)
    assert worst < 1e-13


def test_derivatives_laplace3d_legendre(oracle):
    # d_z^n (1/r) = (-1)^n n! P_n(z/r) / r^(n+1)  (classical Legendre form)
    x = np.array([0.3, -0.45, 0.62])
    r = np.linalg.norm(x)
    pmax = 24
    D = oracle.derivatives("laplace", 3, pmax, x) * 4 * math.pi
    for n in range(pmax + 1):
        ref = (-1) ** n * math.factorial(n) * eval_legendre(n, x[2] / r) / r ** (n + 1)
        got = D[oracle.mi_index(3, [0, 0, n])]
        assert abs(got - ref) <= 1e-13 * math.factorial(n) / r ** (n + 1)


def test_derivatives_yukawa_on_axis(oracle):
    # On the z axis, d_z^n [e^{-lam z}/z] by Leibniz:
    # sum_k C(n,k) (-lam)^(n-k) e^{-lam z} (-1)^k k! / z^(k+1)
    lam, z = 1.7, 0.8
    pmax = 20
    D = oracle.derivatives("yukawa", 3, pmax, [0.0, 0.0, z], lam)
    for n in range(pmax + 1):
        ref = sum(binom(n, k) * (-lam) ** (n - k) * math.exp(-lam * z) * (-1) ** k
                  * math.factorial(k) / z ** (k + 1) for k in range(n + 1))
        got = D[oracle.mi_index(3, [0, 0, n])]
        assert abs(got - ref) <= 1e-13 * abs(ref) + 1e-300


def test_derivatives_biharmonic_on_axis(oracle):
    # G = r on the z axis: d_z r = 1, d_z^n r = 0 (n >= 2); d_x^2 r = 1/z there.
    z = 0.9
    D = oracle.derivatives("biharmonic", 3, 8, [0.0, 0.0, z])
    assert abs(D[oracle.mi_index(3, [0, 0, 0])] - z) < 1e-15
    assert abs(D[oracle.mi_index(3, [0, 0, 1])] - 1.0) < 1e-15
    for n in range(2, 9):
        assert abs(D[oracle.mi_index(3, [0, 0, n])]) < 1e-13
    assert abs(D[oracle.mi_index(3, [2, 0, 0])] - 1.0 / z) < 1e-14
    assert abs(D[oracle.mi_index(3, [0, 2, 0])] - 1.0 / z) < 1e-14


@pytest.mark.parametrize("kernel,d,lam", [("laplace", 2, 0.0), ("laplace", 3, 0.0),
                                          ("yukawa", 3, 1.3), ("biharmonic", 3, 0.0),
                                          ("biharmonic", 2, 0.0)])
def test_derivatives_finite_differences(oracle, kernel, d, lam):
    # low orders against central differences of G itself (order 0 entry)
    x = np.array([0.41, -0.27, 0.33][:d])
    D = oracle.derivatives(kernel, d, 3, x, lam)
    G = lambda y: oracle.derivatives(kernel, d, 0, y, lam)[0]

    def fd(y, mm, h):
        # finite-difference d^m G via nested central differences
        k = next((i for i in range(d) if mm[i] > 0), None)
        if k is None:
            return G(y)
        e = np.zeros(d)
        e[k] = h
        m2 = list(mm)
        m2[k] -= 1
        return (fd(y + e, m2, h) - fd(y - e, m2, h)) / (2 * h)

    for m in oracle.multi_indices(d, 2):
        h = 2e-3
        ref = (4 * fd(x, list(m), h / 2) - fd(x, list(m), h)) / 3  # Richardson, O(h^4)
        got = D[oracle.mi_index(d, m)]
        assert abs(got - ref) <= 1e-7 * max(1.0, abs(ref)), (m, got, ref)


@pytest.mark.parametrize("kernel,lam", [("laplace", 0.0), ("yukawa", 1.3), ("biharmonic", 0.0)])
def test_derivatives_satisfy_pde(oracle, kernel, lam):
    # eq. (Pv): every derivative of G satisfies the PDE away from 0.
    x = np.array([0.52, -0.31, 0.44])
    pmax = 22
    D = oracle.derivatives(kernel, 3, pmax, x, lam)
    E = np.eye(3, dtype=int)
    c = 4 if kernel == "biharmonic" else 2
    for m in oracle.multi_indices(3, pmax - c):
        if kernel == "biharmonic":
            terms = [D[oracle.mi_index(3, m + 2 * E[a] + 2 * E[b])] for a in range(3) for b in range(3)]
            res = sum(terms)
        else:
            terms = [D[oracle.mi_index(3, m + 2 * E[a])] for a in range(3)]
            res = sum(terms) - lam * lam * D[oracle.mi_index(3, m)]
            terms.append(lam * lam * D[oracle.mi_index(3, m)])
        assert abs(res) <= 1e-13 * max(abs(t) for t in terms)


# --------------------------------------------------------------------------
# Sec. 3.1, eq. (decompression): M [D G]_j reproduces the full vector.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kernel,d,p,lam", [("laplace", 2, 12, 0.0), ("laplace", 3, 10, 0.0),
                                            ("yukawa", 3, 12, 1.0), ("biharmonic", 3, 8, 0.0),
                                            ("biharmonic", 3, 16, 0.0), ("biharmonic", 2, 12, 0.0)])
def test_decompression_reproduces_derivatives(oracle, kernel, d, p, lam):
    e = oracle.Expansion(d, p, kernel, lam=lam)
    M = e.M
    assert np.array_equal(M[e.j], np.eye(e.nj))
    for x in ([0.6, -0.35, 0.5][:d], [-0.2, 0.9, -0.4][:d]):
        D = oracle.derivatives(kernel, d, p, x, lam)
        Dr = e.decompress(D[e.j])
        scale = np.abs(D).max()
        assert np.abs(Dr - D).max() <= 1e-13 * scale


def test_compress_is_adjoint_of_decompress(oracle):
    e = oracle.Expansion(3, 8, "yukawa", lam=0.7)
    rng = np.random.default_rng(0)
    s = rng.normal(size=e.nj)
    a = rng.normal(size=e.nfull)
    assert abs(e.decompress(s) @ a - s @ e.compress(a)) < 1e-11 * np.abs(a).sum() * np.abs(s).sum()


# --------------------------------------------------------------------------
# Expansions (Secs. 2, 3.2-3.5): convergence to G(x - y) at the truncation
# rate, brute force against the direct sum.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kernel,lam", [("laplace", 0.0), ("yukawa", 1.0), ("biharmonic", 0.0)])
def test_p2m_m2p_converges(oracle, kernel, lam):
    rng = np.random.default_rng(1)
    c = np.zeros(3)
    y = rng.uniform(-0.1, 0.1, size=(20, 3))
    w = rng.uniform(-1, 1, 20)
    x = np.array([0.55, -0.4, 0.35])
    ref = oracle.direct(kernel, 3, y, w, x[None, :], lam)[0]
    errs = []
    for p in (4, 8, 12):
        e = oracle.Expansion(3, p, kernel, lam=lam)
        errs.append(abs(e.m2p(c, e.p2m(c, y, w), x) - ref) / abs(ref))
    # R/|x-c| ~ 0.2: each +4 in p gains roughly 0.2^4
    assert errs[1] < errs[0] * 0.05 and errs[2] < errs[1] * 0.05 and errs[2] < 1e-9


@pytest.mark.parametrize("kernel,lam", [("laplace", 0.0), ("yukawa", 1.0), ("biharmonic", 0.0)])
def test_p2l_l2p_converges_and_gradient(oracle, kernel, lam):
    rng = np.random.default_rng(2)
    c = np.zeros(3)
    y = np.array([[0.8, 0.5, -0.6], [-0.7, 0.9, 0.4]])
    w = np.array([0.7, -1.2])
    x = c + rng.uniform(-0.1, 0.1, 3)
    ref, gref = oracle.direct(kernel, 3, y, w, x[None, :], lam, grad=True)
    errs = []
    for p in (4, 8, 12):
        e = oracle.Expansion(3, p, kernel, lam=lam)
        v, g = e.l2p(c, e.p2l(c, y, w), x, grad=True)
        errs.append(abs(v - ref[0]) / abs(ref[0]))
    assert errs[2] < 1e-10 and errs[1] < errs[0]
    assert np.abs(g - gref[0]).max() < 1e-9 * np.abs(gref[0]).max()


def test_m2l_compressed_equals_naive_uncompressed(oracle):
    # eq. (m2l_toeplitz): the compressed M2L is the uncompressed O(p^{2d}) one
    # restricted to j, and M L_j recovers every uncompressed coefficient.
    for kernel, d, p, lam in (("laplace", 3, 8, 0.0), ("yukawa", 3, 6, 1.2),
                              ("biharmonic", 3, 6, 0.0), ("laplace", 2, 10, 0.0)):
        e = oracle.Expansion(d, p, kernel, lam=lam)
        rng = np.random.default_rng(3)
        alpha = rng.normal(size=e.nfull) * 0.1 ** e.mi.sum(axis=1)
        beta = e.compress(alpha)
        h = np.array([2.0, -1.0, 3.0][:d])
        D2 = oracle.derivatives(kernel, d, 2 * p, h, lam)
        Lfull = oracle.m2l_naive(d, p, D2, alpha)
        Lc = e.m2l(h, beta)
        scale = np.abs(Lfull).max()
        assert np.abs(Lc - Lfull[e.j]).max() <= 1e-12 * scale
        assert np.abs(e.decompress(Lc) - Lfull).max() <= 1e-12 * scale


def test_l2l_compressed_equals_uncompressed_laplace(oracle):
    # For an equal-order PDE the shifted local polynomial still satisfies the
    # PDE, so the compressed L2L (Sec. 4.2) reproduces the uncompressed one.
    ec = oracle.Expansion(3, 10, "laplace")
    ef = oracle.Expansion(3, 10, "laplace", compressed=False)
    y = np.array([[1.3, -0.9, 1.1], [-1.2, 1.4, 0.8]])
    w = np.array([1.0, -0.6])
    c1 = np.zeros(3)
    h = np.array([0.125, -0.125, 0.125])
    Lc = ec.l2l(h, ec.p2l(c1, y, w))
    Lf = ef.l2l(h, ef.p2l(c1, y, w))
    assert np.abs(ec.decompress(Lc) - Lf).max() <= 1e-13 * np.abs(Lf).max()


def test_l2l_converges_to_direct_local(oracle):
    for kernel, lam in (("laplace", 0.0), ("yukawa", 1.0), ("biharmonic", 0.0)):
        y = np.array([[1.3, -0.9, 1.1]])
        w = np.array([1.0])
        c1, c2 = np.zeros(3), np.array([0.1, -0.05, 0.08])
        errs = []
        for p in (6, 12):
            e = oracle.Expansion(3, p, kernel, lam=lam)
            L2 = e.l2l(c2 - c1, e.p2l(c1, y, w))
            Lref = e.p2l(c2, y, w)
            errs.append(abs(L2[0] - Lref[0]) / abs(Lref[0]))
        assert errs[1] < 1e-6 and errs[1] < errs[0]


# --------------------------------------------------------------------------
# Thm 11 and Fig. m2m_accuracy (Sec. 5.1): compressed M2M equals the
# uncompressed one for equal-order PDEs; for Yukawa the extra error behaves
# like R^(p+1) (Thm 12, like the printed Helmholtz curves).
# --------------------------------------------------------------------------
def _golden_m2m():
    rows = []
    with open(os.path.join(GOLDEN, "m2m_accuracy_fig.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, d, p, R, eps = line.split()
            rows.append((k, int(d), int(p), float(R), float(eps)))
    return rows


def m2m_experiment(oracle, kernel, d, p, R, lam=0.0, nsrc=50, ntgt=20):
    g = np.linspace(-1.0, 1.0, nsrc)
    c1 = np.full(d, R)
    src = np.stack(np.meshgrid(*([g] * d), indexing="ij"), -1).reshape(-1, d) * R + c1
    rng = np.random.default_rng(5)
    w = rng.uniform(0.0, 1.0, src.shape[0])
    gt = np.linspace(-0.5, 0.5, ntgt)
    tgt = np.stack(np.meshgrid(*([gt] * d), indexing="ij"), -1).reshape(-1, d) + 1.0
    ec = oracle.Expansion(d, p, kernel, lam=lam)
    ef = oracle.Expansion(d, p, kernel, lam=lam, compressed=False)
    alpha = ef.p2m(c1, src, w)          # uncompressed (M = I)
    beta = ec.compress(alpha)
    h = -c1                              # c2 - c1 with c2 = 0
    rho = ef.m2m_full(h, alpha)
    psi = ec.m2m(h, beta)
    D = oracle.derivatives_batch(kernel, d, p, tgt, lam)
    full = D @ rho
    comp = D[:, ec.j] @ psi
    return np.sqrt(np.sum((comp - full) ** 2) / np.sum(full ** 2))


@pytest.mark.parametrize("kernel,d", [("laplace", 2), ("biharmonic", 2), ("laplace", 3),
                                      ("biharmonic", 3)])
def test_m2m_equal_order_matches_fig(oracle, kernel, d):
    rows = [r for r in _golden_m2m() if r[0] == kernel and r[1] == d]
    assert len(rows) == 54
    for p in (4, 10):
        for R in (2.0 ** -10, 0.25):
            printed = next(r[4] for r in rows if r[2] == p and r[3] == R)
            ours = m2m_experiment(oracle, kernel, d, p, R)
            # the paper's claim (Thm 11): roundoff only, below 1e-14
            assert ours < 1e-14 and printed < 1e-14, (p, R, ours, printed)


def test_m2m_yukawa_error_scales_like_truncation(oracle):
    # Thm 12: extra error O(R^(p+1)); Helmholtz (kappa = 1) curves printed in
    # Fig. m2m_accuracy(f) grow with slope p+1 and are ~5e-3 at p=2, R=1/4.
    e_small = m2m_experiment(oracle, "yukawa", 3, 2, 2.0 ** -6, lam=1.0, nsrc=12, ntgt=8)
    e_big = m2m_experiment(oracle, "yukawa", 3, 2, 2.0 ** -2, lam=1.0, nsrc=12, ntgt=8)
    slope = math.log(e_big / e_small) / math.log(16.0)
    assert 2.5 < slope < 3.5
    printed = next(r[4] for r in _golden_m2m() if r[0] == "helmholtz" and r[1] == 3
                   and r[2] == 2 and r[3] == 0.25)
    assert printed / 10 < e_big < printed * 10
    e12 = m2m_experiment(oracle, "yukawa", 3, 12, 2.0 ** -2, lam=1.0, nsrc=12, ntgt=8)
    assert e12 < 1e-4


# --------------------------------------------------------------------------
# Whole FMM (uniform tree): against the plain definition, eq. (1).
# --------------------------------------------------------------------------
def test_fmm_converges_to_direct_sum(oracle):
    rng = np.random.default_rng(11)
    src = rng.random((2500, 3))
    w = rng.uniform(-1, 1, 2500)
    ref = oracle.direct("laplace", 3, src, w, src)
    errs = []
    for p in (2, 6, 10):
        phi = oracle.fmm_uniform("laplace", 3, p, 3, src, w, src)
        errs.append(np.linalg.norm(phi - ref) / np.linalg.norm(ref))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-5


@pytest.mark.parametrize("kernel,d,lam,p", [("laplace", 2, 0.0, 12), ("yukawa", 3, 1.0, 8),
                                            ("biharmonic", 3, 0.0, 8)])
def test_fmm_other_kernels_vs_direct(oracle, kernel, d, lam, p):
    rng = np.random.default_rng(12)
    n = 1500
    src = rng.random((n, d))
    tgt = rng.random((700, d))
    w = rng.uniform(-1, 1, n)
    ref = oracle.direct(kernel, d, src, w, tgt, lam)
    phi = oracle.fmm_uniform(kernel, d, p, 3, src, w, tgt, lam=lam)
    err = np.linalg.norm(phi - ref) / np.linalg.norm(ref)
    assert err < 1e-4, err


@pytest.mark.parametrize("kernel", ["laplace", "biharmonic"])
def test_fmm_compressed_equals_uncompressed(oracle, kernel):
    # Secs. 4.1-4.3: no additional error for equal-order PDEs.
    rng = np.random.default_rng(13)
    src = rng.random((1500, 3))
    w = rng.uniform(-1, 1, 1500)
    a = oracle.fmm_uniform(kernel, 3, 6, 3, src, w, src)
    b = oracle.fmm_uniform(kernel, 3, 6, 3, src, w, src, compressed=False)
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-13


def test_fmm_gradient_vs_direct(oracle):
    rng = np.random.default_rng(14)
    src = rng.random((1500, 3))
    tgt = rng.random((500, 3))
    w = rng.uniform(-1, 1, 1500)
    _, gref = oracle.direct("laplace", 3, src, w, tgt, grad=True)
    _, g = oracle.fmm_uniform("laplace", 3, 10, 3, src, w, tgt, grad=True)
    assert np.linalg.norm(g - gref) / np.linalg.norm(gref) < 1e-4


def test_fmm_sampled_matches_full(oracle):
    rng = np.random.default_rng(15)
    src = rng.random((3000, 3))
    w = rng.uniform(-1, 1, 3000)
    full = oracle.fmm_uniform("laplace", 3, 6, 4, src, w, src)
    idx = rng.choice(3000, 40, replace=False)
    part = oracle.fmm_uniform("laplace", 3, 6, 4, src, w, src, sample=idx)
    assert np.array_equal(part, full[idx])


def test_fmm_self_interaction_excluded(oracle):
    # reading: x == y pairs are skipped; two coincident points see each other's
    # partner only.
    src = np.array([[0.1, 0.1, 0.1], [0.9, 0.9, 0.9]])
    w = np.array([1.0, 2.0])
    phi = oracle.fmm_uniform("laplace", 3, 4, 2, src, w, src)
    r = np.linalg.norm(src[0] - src[1])
    assert np.allclose(phi, [2.0 / (4 * np.pi * r), 1.0 / (4 * np.pi * r)], rtol=1e-12)
