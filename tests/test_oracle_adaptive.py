"""Pins of the oracle's adaptive-tree FMM (U, V, W, X lists) to facts that do
not come from the oracle itself:

* a tree that refines every box to the same depth is the uniform tree, so the
  adaptive driver must reproduce the uniform driver (W = X = empty);
* the lists of a target's leaf and of its ancestors must reach every source
  exactly once (counted with multiplicity through U, V, W and X, whether a W
  or X pair goes through an expansion or, for a box of at most |j| points,
  is summed directly);
* the result converges to the direct sum of eq. (1) as p grows.
"""
import numpy as np
import pytest

from paper_2305_17867_gb300 import workloads as W


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def plummer_case(n_src=6000, n_tgt=1200, seed=3):
    rng = np.random.Generator(np.random.PCG64(seed))
    src = W.plummer_points(rng, n_src)
    w = rng.normal(size=n_src)
    tgt = rng.random((n_tgt, 3))
    return src, w, tgt


def test_complete_tree_is_the_uniform_tree(oracle):
    rng = np.random.default_rng(11)
    src = rng.random((12000, 3))
    w = rng.uniform(-1, 1, 12000)
    # sources = targets: level-2 boxes hold ~2*188 points (> 200), level-3
    # boxes ~2*23 (< 200), so every box down to level 3 splits and none below
    phi, st, cov = oracle.fmm_adaptive("laplace", 3, 5, src, w, src, max_leaf=200,
                                       want_stats=True)
    assert st["leaves"] == 512 and st["depth"] == 3
    assert st["W"] == 0 and st["X"] == 0
    ref = oracle.fmm_uniform("laplace", 3, 5, 3, src, w, src)
    assert rel(phi, ref) < 1e-14


@pytest.mark.parametrize("same", [False, True])
def test_lists_reach_every_source_once(oracle, same):
    src, w, tgt = plummer_case(5000, 800)
    if same:
        tgt = src
    _, st, cov = oracle.fmm_adaptive("laplace", 3, 2, src, w, tgt, max_leaf=24,
                                     want_stats=True)
    assert st["W"] > 0 and st["X"] > 0 and st["depth"] >= 5
    # |j| = 9 at p = 2 against leaves of up to 24 points: some W and X pairs
    # are summed directly, the others through M2P and P2L
    assert 0 < st["WX_direct"] < st["W"] + st["X"]
    expect = len(w) - (1 if same else 0)  # the coinciding source is skipped
    assert np.all(cov == expect)


def test_two_dimensional_lists(oracle):
    rng = np.random.default_rng(12)
    src = np.concatenate([rng.random((300, 2)) * 0.05 + 0.6, rng.random((700, 2))])
    w = rng.normal(size=1000)
    tgt = rng.random((400, 2))
    phi, st, cov = oracle.fmm_adaptive("laplace", 2, 12, src, w, tgt, max_leaf=16,
                                       want_stats=True)
    assert st["W"] > 0 and st["X"] > 0
    assert np.all(cov == len(w))
    ref = oracle.direct("laplace", 2, src, w, tgt)
    assert rel(phi, ref) < 1e-5


@pytest.mark.parametrize("kernel,lam", [("laplace", 0.0), ("yukawa", 1.0)])
def test_converges_to_direct_sum(oracle, kernel, lam):
    src, w, tgt = plummer_case(4000, 600)
    ref = oracle.direct(kernel, 3, src, w, tgt, lam=lam)
    errs = [rel(oracle.fmm_adaptive(kernel, 3, p, src, w, tgt, max_leaf=32, lam=lam), ref)
            for p in (2, 4, 6)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 2e-3


def test_sampled_equals_full(oracle):
    src, w, tgt = plummer_case(3000, 500)
    full = oracle.fmm_adaptive("laplace", 3, 4, src, w, tgt, max_leaf=20)
    idx = np.array([0, 7, 123, 499, 250])
    part = oracle.fmm_adaptive("laplace", 3, 4, src, w, tgt, max_leaf=20, sample=idx)
    assert np.array_equal(part, full[idx])


def test_depth_cap_keeps_every_pair(oracle):
    # a cluster finer than the deepest level: leaves exceed max_leaf
    rng = np.random.default_rng(13)
    src = np.concatenate([0.3 + 1e-4 * rng.random((400, 3)), rng.random((600, 3))])
    w = rng.normal(size=1000)
    tgt = rng.random((300, 3))
    phi, st, cov = oracle.fmm_adaptive("laplace", 3, 4, src, w, tgt, max_leaf=8,
                                       max_depth=4, want_stats=True)
    assert st["depth"] == 4
    assert np.all(cov == len(w))
    ref = oracle.direct("laplace", 3, src, w, tgt)
    assert rel(phi, ref) < 1e-2


def test_point_outside_root_is_rejected(oracle):
    src = np.array([[0.5, 0.5, 0.5], [1.5, 0.2, 0.2]])
    with pytest.raises(ValueError):
        oracle.fmm_adaptive("laplace", 3, 2, src, np.ones(2), src, max_leaf=1)


def test_repeatable_across_thread_counts(oracle):
    """The oracle gives the same bits for the same input: the adaptive M2M adds
    the children of a parent in Morton order whatever the thread count (Sec.
    4.3; an order that followed thread timing once made two calls differ)."""
    src, w, tgt = plummer_case(3000, 500)
    old = oracle.num_threads()
    try:
        oracle.set_num_threads(8)
        a = oracle.fmm_adaptive("laplace", 3, 6, src, w, tgt, max_leaf=12)
        b = oracle.fmm_adaptive("laplace", 3, 6, src, w, tgt, max_leaf=12)
        oracle.set_num_threads(1)
        c = oracle.fmm_adaptive("laplace", 3, 6, src, w, tgt, max_leaf=12)
    finally:
        oracle.set_num_threads(old)
    assert np.array_equal(a, b)
    assert np.array_equal(a, c)
