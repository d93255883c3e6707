"""Pins of the oracle's two tree rules that no numerical identity reaches.

* Refinement (Section 4, reading R8): a leaf is split while the largest
  tensor Legendre coefficient of total degree >= K-1 of f on its K x K nodes
  exceeds refine_tol * f_scale.  For f = exp(a x + b y) those coefficients have
  a closed form: on a leaf of centre (cx, cy) and half-side h,
  c_mn = exp(a cx + b cy) (2m+1) i_m(a h) (2n+1) i_n(b h), with i_n the
  modified spherical Bessel functions (the Legendre expansion of exp(z u) is
  sum (2n+1) i_n(z) P_n(u)).  Splitting by that formula from the root gives
  the whole adaptive tree independently of the oracle's discrete transform;
  every leaf then meets the criterion and every split parent violates it.
* Extension lists (Section 4, reading R6): an exterior leaf is owned by the
  cut leaf with the nearest centre among those whose extension square (the
  leaf's square enlarged three times about its centre) overlaps it; on a tie
  the cut leaf later in Z-order wins, and a leaf overlapped by no extension
  square has no owner.  Checked by brute force in exact integer arithmetic on
  the finest grid of each tree.
"""
import numpy as np
import pytest
from scipy.special import spherical_in

import workloads as W
from oracle import oracle as O


# ----------------------------------------------------------------- refinement

def _closed_form_tail(K, a, b, leaf):
    """max over m + n >= K-1 of |c_mn| for f = exp(a x + b y) on the leaf."""
    l, ix, iy = leaf
    h = 0.5 ** (l + 1)
    cx, cy = -0.5 + (2 * ix + 1) * h, -0.5 + (2 * iy + 1) * h
    m = np.arange(K)
    cxm = (2 * m + 1) * spherical_in(m, a * h)
    cyn = (2 * m + 1) * spherical_in(m, b * h)
    best = 0.0
    for n in range(K):
        for mm in range(K):
            if mm + n >= K - 1:
                best = max(best, abs(np.exp(a * cx + b * cy) * cxm[mm] * cyn[n]))
    return best


def _predicted_leaves(K, a, b, thr, min_level, max_level):
    """Leaves of the tree split by the closed-form tail from the root, and the
    smallest |log(tail / threshold)| met at a decision (the margin by which no
    decision is close)."""
    leaves, margin, front = [], np.inf, [(0, 0, 0)]
    while front:
        nxt = []
        for leaf in front:
            l, ix, iy = leaf
            kids = [(l + 1, 2 * ix + p, 2 * iy + q) for q in (0, 1) for p in (0, 1)]
            if l < min_level:
                nxt += kids
                continue
            c = _closed_form_tail(K, a, b, leaf)
            if l < max_level:
                margin = min(margin, abs(np.log(c / thr)))
            if l < max_level and c > thr:
                nxt += kids
            else:
                leaves.append(leaf)
        front = nxt
    return sorted(leaves), margin


R8_CASES = [(8, 7.0, 5.0, 1e-7), (8, 8.0, 3.0, 1e-7), (6, 6.0, 4.0, 1e-6)]


@pytest.mark.parametrize("K,a,b,tol", R8_CASES)
def test_refinement_matches_closed_form_legendre_tails(K, a, b, tol):
    """The oracle's adaptive tree for f = exp(a x + b y) on the whole box equals
    the tree split by the closed-form Legendre tails.  The discrete transform
    on K Gauss-Legendre nodes aliases degrees >= K into the coefficients, a
    relative change of order (a h)^2 / (4 K^2) < 1e-3 at the deciding levels;
    every decision here clears the threshold by more than 1 % (checked), so
    aliasing cannot flip one."""
    pred, margin = _predicted_leaves(K, a, b, tol, 1, 9)
    assert margin > 0.01, margin
    opts = W.TreeOptions(K=K, min_level=1, max_level=9, refine_tol=tol, f_scale=1.0)
    tree = O.build_tree(W.WholeBoxDomain(), opts, lambda xy: np.exp(a * xy[:, 0] + b * xy[:, 1]))
    assert len({l for l, _, _ in pred}) >= 3            # a genuinely adaptive tree
    assert sorted(tree.leaves) == pred
    # every leaf meets the criterion; every split parent at or below min_level violates it
    leaves = set(tree.leaves)
    for leaf in tree.leaves:
        assert _closed_form_tail(K, a, b, leaf) <= tol
        l, ix, iy = leaf
        if l - 1 >= 1:
            assert _closed_form_tail(K, a, b, (l - 1, ix >> 1, iy >> 1)) > tol
    assert all(O.ancestor(leaf, lv) not in leaves for leaf in tree.leaves for lv in range(leaf[0]))


def test_refinement_stops_for_polynomials_below_degree_k_minus_1():
    """f of total degree K-2 has no tail at all: the tree stays at min_level
    however small the tolerance; one term of degree K-1 refines it."""
    K = 8
    opts = W.TreeOptions(K=K, min_level=2, max_level=7, refine_tol=1e-14, f_scale=1.0)
    low = O.build_tree(W.WholeBoxDomain(), opts, lambda xy: xy[:, 0] ** 3 * xy[:, 1] ** 3 + xy[:, 0] ** 6)
    assert all(b[0] == 2 for b in low.leaves) and low.n_leaves == 16
    high = O.build_tree(W.WholeBoxDomain(), opts, lambda xy: xy[:, 0] ** 4 * xy[:, 1] ** 3)
    assert max(b[0] for b in high.leaves) > 2


# ----------------------------------------------------------- extension lists

def _owner_brute_force(tree):
    """Owners by the R6 rule in exact integers: boxes on the finest grid of the
    tree, centres doubled so that they are integers."""
    L = max(b[0] for b in tree.leaves)

    def box(b):
        l, ix, iy = b
        s = 1 << (L - l)
        return ix * s, iy * s, s

    cut = [i for i, c in enumerate(tree.cls) if c == O.CUT]
    owner = [-1] * tree.n_leaves
    ties = 0
    first_differs = 0
    for j, bj in enumerate(tree.leaves):
        if tree.cls[j] != O.EXTERIOR:
            continue
        x0, y0, s = box(bj)
        cxj, cyj = 2 * x0 + s, 2 * y0 + s
        best, best_i, first, n_best = None, -1, -1, 0
        for i in cut:                                   # Z-order
            u0, v0, t = box(tree.leaves[i])
            # extension square [u0 - t, u0 + 2t] x [v0 - t, v0 + 2t]; overlap of positive area
            if min(x0 + s, u0 + 2 * t) <= max(x0, u0 - t) or min(y0 + s, v0 + 2 * t) <= max(y0, v0 - t):
                continue
            if first < 0:
                first = i
            d2 = (2 * u0 + t - cxj) ** 2 + (2 * v0 + t - cyj) ** 2
            if best is None or d2 < best:
                best, best_i, n_best = d2, i, 1
            elif d2 == best:
                best_i, n_best = i, n_best + 1          # the later one in Z-order
        owner[j] = best_i
        ties += n_best > 1
        first_differs += first >= 0 and first != best_i
    return owner, ties, first_differs


OWNER_TREES = {
    "disk_l4": lambda: W.disk_sincos(level=4),
    "starfish_k8": lambda: W.starfish_gaussian(K=8, tol=1e-8, max_level=8),
    "lshape_small": lambda: W.lshape_expsin(K=8, base_level=4, max_level=7, corner_levels=4),
    "exterior_k8": lambda: W.exterior_three_stars(K=8, tol=1e-5, max_level=7),
}


@pytest.mark.parametrize("name", list(OWNER_TREES))
def test_extension_owners_brute_force(name):
    w = OWNER_TREES[name]()
    tree = O.build_tree(w.domain, w.opts, w.sources[0])
    want, _, _ = _owner_brute_force(tree)
    assert list(tree.owner) == want


def test_owner_rule_cases_are_exercised():
    """The trees above contain exterior leaves equidistant from two cut leaves
    (the tie-break decides) and leaves whose first overlapping cut leaf is not
    the nearest (the distance decides)."""
    ties = differs = 0
    for make in OWNER_TREES.values():
        w = make()
        _, t, d = _owner_brute_force(O.build_tree(w.domain, w.opts, w.sources[0]))
        ties += t
        differs += d
    assert ties > 0 and differs > 0
