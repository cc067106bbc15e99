"""Host logic of bench.py that the reported numbers rest on, checked on CPU.

* The M2L translation count of a uniform tree (the unit of the roofline's
  algorithmic FLOP figure) against a brute-force enumeration of the
  interaction lists: target t and source s of the same level interact when
  their parents are adjacent and they are not (Sec. 4.1, List 2).
* The parser of the committed ncu summaries that supply the roofline's
  traffic figure, and its refusal to report a figure for changed sources.
* The near-field pair count of the whole-step roofline, and the subtree
  sample of the CPU baseline.
* The leaf key (boxes lexicographic, x fastest).
"""
import itertools

import numpy as np
import pytest

import bench


def brute_force_m2l(d, L):
    """(count, largest list) by enumerating every (target, source) pair per level."""
    total, longest = 0, 0
    for l in range(2, L + 1):
        n = 1 << l
        boxes = list(itertools.product(range(n), repeat=d))
        for t in boxes:
            k = 0
            for s in boxes:
                par_adj = all(abs((a >> 1) - (b >> 1)) <= 1 for a, b in zip(t, s))
                adj = all(abs(a - b) <= 1 for a, b in zip(t, s))
                if par_adj and not adj:
                    k += 1
            total += k
            longest = max(longest, k)
    return total, longest


@pytest.mark.parametrize("d,L", [(2, 3), (2, 5), (3, 3)])
def test_m2l_count_matches_enumeration(d, L):
    total, longest = brute_force_m2l(d, L)
    assert bench.m2l_count(d, L) == total
    # an interior box's list: 6^d children of the parent's neighbours minus 3^d
    assert longest == 6 ** d - 3 ** d


def test_m2l_count_level_two_closed_form():
    # at level 2 every pair of parents is adjacent: all n^2 pairs per axis minus
    # the 3n - 2 adjacent ones, n = 4, raised to the dimension
    for d in (2, 3):
        assert bench.m2l_count(d, 2) == 16 ** d - 10 ** d
    per_level = [bench.m2l_count(3, L) - bench.m2l_count(3, L - 1) for L in range(3, 6)]
    assert per_level == sorted(per_level)


def test_traffic_figure_only_for_the_captured_sources(monkeypatch, tmp_path):
    (tmp_path / "m2l_tc_case.md").write_text(
        "Command ...\n\n`traffic: tf32x3 123456 sources abcdef0123456789 workload wl_a`\n"
        "`traffic: bf16x3 999 sources abcdef0123456789 workload wl_a`\n")
    monkeypatch.setattr(bench, "m2l_source_hash", lambda: "abcdef0123456789")
    got, src = bench.profiled_traffic("tf32x3", "wl_a", profiles=str(tmp_path))
    assert got == 123456 and "ncu" in src
    got, _ = bench.profiled_traffic("bf16x3", "wl_a", profiles=str(tmp_path))
    assert got == 999
    got, src = bench.profiled_traffic("tf32x3", "wl_b", profiles=str(tmp_path))
    assert got is None
    monkeypatch.setattr(bench, "m2l_source_hash", lambda: "0" * 16)
    got, src = bench.profiled_traffic("tf32x3", "wl_a", profiles=str(tmp_path))
    assert got is None and "changed" in src


def test_near_field_pairs_against_enumeration():
    # the near-field pair count of the whole-step roofline against a brute-force
    # count over points: same leaf or adjacent leaves, coinciding points excluded
    rng = np.random.default_rng(5)
    src = rng.random((400, 3))
    tgt = rng.random((300, 3))
    L = 2
    n = 1 << L
    cs = np.minimum(np.floor(src * n), n - 1)
    ct = np.minimum(np.floor(tgt * n), n - 1)
    brute = int((np.abs(ct[:, None, :] - cs[None, :, :]).max(axis=2) <= 1).sum())
    assert bench.near_pairs(src, tgt, L) == brute
    same = int((np.abs(cs[:, None, :] - cs[None, :, :]).max(axis=2) <= 1).sum()) - len(src)
    assert bench.near_pairs(src, src, L) == same


def test_subtree_targets_lie_in_one_box():
    rng = np.random.default_rng(6)
    tgt = rng.random((5000, 3))
    idx, box = bench.subtree_targets(tgt, 2, np.random.default_rng(1))
    inside = np.all(np.floor(tgt * 4) == box, axis=1)
    assert np.array_equal(np.sort(idx), np.nonzero(inside)[0])


def test_leaf_key_is_lexicographic_x_fastest():
    L = 2
    x = np.array([[0.1, 0.1, 0.1], [0.3, 0.1, 0.1], [0.1, 0.3, 0.1], [0.1, 0.1, 0.3],
                  [0.99, 0.99, 0.99]])
    assert bench.leaf_of(x, L).tolist() == [0, 1, 4, 16, 63]


def test_code_digest_ignores_comments_only():
    a = "int f() {  // returns one\n  return 1;\n}\n"
    b = "// a new note\nint f() {  // returns 1\n\n  return 1;   \n}\n"
    c = "int f() {\n  return 2;\n}\n"
    assert bench.code_digest([a]) == bench.code_digest([b])
    assert bench.code_digest([a]) != bench.code_digest([c])
