"""Pins of the oracle's 2D biharmonic kernel G = r^2 log r (PDE Laplacian^2,
c = 4; Sec. 4.4, eq. (deriv_biharmonic_2d)) beyond the derivative, M2M and
decompression pins shared with the other kernels:

* every derivative satisfies the biharmonic equation away from 0 (eq. (Pv));
* on the x axis, d_x^n (x^2 log|x|) has its closed form;
* the FMM converges to the direct sum of eq. (1) as p grows.
"""
import math

import numpy as np


def test_derivatives_satisfy_pde(oracle):
    x = np.array([0.52, -0.31])
    pmax = 20
    D = oracle.derivatives("biharmonic", 2, pmax, x)
    for m in oracle.multi_indices(2, pmax - 4):
        terms = [D[oracle.mi_index(2, m + np.array(e))] for e in ((4, 0), (0, 4), (2, 2), (2, 2))]
        assert abs(sum(terms)) <= 1e-12 * max(abs(t) for t in terms), (tuple(m), terms)


def test_axis_closed_form(oracle):
    # f(x) = x^2 log x: f' = 2x log x + x, f'' = 2 log x + 3, and for n >= 3
    # f^(n) = 2 (-1)^(n-1) (n-3)! x^(2-n)
    x = 0.7
    D = oracle.derivatives("biharmonic", 2, 10, np.array([x, 0.0]))
    want = {0: x * x * math.log(x), 1: 2 * x * math.log(x) + x, 2: 2 * math.log(x) + 3}
    for n in range(3, 11):
        want[n] = 2.0 * (-1) ** (n - 1) * math.factorial(n - 3) * x ** (2 - n)
    for n, v in want.items():
        got = D[oracle.mi_index(2, [n, 0])]
        assert abs(got - v) <= 1e-13 * max(1.0, abs(v)), (n, got, v)


def test_fmm_converges_to_direct_sum(oracle):
    rng = np.random.default_rng(15)
    src = rng.random((3000, 2))
    w = rng.uniform(-1, 1, 3000)
    tgt = rng.random((500, 2))
    ref = oracle.direct("biharmonic", 2, src, w, tgt)
    errs = [float(np.linalg.norm(oracle.fmm_uniform("biharmonic", 2, p, 4, src, w, tgt) - ref) /
                  np.linalg.norm(ref)) for p in (6, 10, 14)]
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-7, errs
