"""Mutation checks of the oracle's pins: each test plants one plausible mistake
in the CPU oracle (on the CPU, by replacing one of its functions for the test)
and requires the pin that guards that part to fail.  A pin that passed with the
mistake in place would not be a pin."""
import numpy as np
import pytest

from oracle import oracle as O
import test_oracle_pins as P


def test_dropped_two_pi_in_the_potential_is_caught(monkeypatch):
    real = O.volume_potential
    monkeypatch.setattr(O, "volume_potential", lambda *a, **k: real(*a, **k) * (2 * np.pi))
    with pytest.raises(AssertionError):
        P.test_potential_of_unit_source_on_D()
    with pytest.raises(AssertionError):
        P.test_potential_of_gaussian_matches_closed_form()


def test_leaf_centre_off_by_half_a_side_is_caught(monkeypatch):
    real = O.box_center
    monkeypatch.setattr(O, "box_center", lambda b: tuple(c + 0.5 * O.box_side(b[0]) for c in real(b)))
    with pytest.raises(AssertionError):
        P.test_potential_of_unit_source_on_D()


def test_transposed_grid_order_in_the_operator_is_caught(monkeypatch):
    """The rows of the Kbar x Kbar grid taken y-fastest instead of x-fastest.
    (Reordering the columns, the support points G, would be no mistake: the
    least-squares extension A_E A_I^+ does not depend on the basis order.)"""
    real = O.universal_matrix

    def transposed(K):
        A = real(K).copy()
        nS, Kb = K * K, O.stencil_params(K)[1]
        blk = A[nS:nS + Kb * Kb].reshape(Kb, Kb, -1)
        A[nS:nS + Kb * Kb] = blk.transpose(1, 0, 2).reshape(Kb * Kb, -1)
        return A
    monkeypatch.setattr(O, "universal_matrix", transposed)
    with pytest.raises(AssertionError):
        P.test_extension_reproduces_total_degree_q_polynomials("disk_l3_k8")


def test_swapped_interpolation_axes_are_caught(monkeypatch):
    def swapped(tree, Vleaf, pts):
        K, t = tree.K, tree.t
        out = np.zeros((len(pts), Vleaf.shape[2]))
        for k, p in enumerate(pts):
            i = O.locate_leaf(tree, p)
            cx, cy = O.box_center(tree.leaves[i])
            h = 0.5 * O.box_side(tree.leaves[i][0])
            u, v = (p[0] - cx) / h, (p[1] - cy) / h
            la = np.array([np.prod([(u - t[m]) / (t[a] - t[m]) for m in range(K) if m != a]) for a in range(K)])
            lb = np.array([np.prod([(v - t[m]) / (t[a] - t[m]) for m in range(K) if m != a]) for a in range(K)])
            out[k] = np.outer(la, lb).ravel() @ Vleaf[i]      # planted: x and y weights exchanged
        return out
    monkeypatch.setattr(O, "interpolate_at", swapped)
    with pytest.raises(AssertionError):
        P.test_interpolation_exact_for_tensor_polynomials()


def test_dropped_sign_in_the_rational_weights_is_caught(monkeypatch):
    real = O.fh_weights
    monkeypatch.setattr(O, "fh_weights", lambda x, d: np.abs(real(x, d)))
    with pytest.raises(AssertionError):
        P.test_fh_reproduces_polynomials_of_degree_d()
    with pytest.raises(AssertionError):
        P.test_line_extension_exact_for_quadratic_along_rays()


def test_net_charge_without_the_leaf_jacobian_is_caught(monkeypatch):
    def half_jacobian(tree, values):
        _, w = O.gauss_legendre(tree.K)
        w2 = np.outer(w, w).ravel()
        return sum(0.5 * O.box_side(b[0]) * (values[i] @ w2) for i, b in enumerate(tree.leaves))
    monkeypatch.setattr(O, "net_charge", half_jacobian)      # planted: (side/2) in place of (side/2)^2
    with pytest.raises(AssertionError):
        P.test_net_charge_exact_for_polynomials_on_an_adaptive_tree()
    with pytest.raises(AssertionError):
        P.test_net_charge_of_a_gaussian_is_pi_s_squared()
    with pytest.raises(AssertionError):
        P.test_net_charge_is_the_growth_of_the_potential_at_infinity()


def _first_overlapping_owner(tree):
    """Planted: the first cut leaf (Z-order) whose extension square overlaps the
    exterior leaf, in place of the nearest one."""
    cut = tree.cut_leaves()
    owner = [-1] * tree.n_leaves
    for j, b in enumerate(tree.leaves):
        if tree.cls[j] != O.EXTERIOR:
            continue
        x0, x1, y0, y1 = O.box_bounds(b)
        for i in cut:
            a0, a1, b0, b1 = O.box_bounds(tree.leaves[i])
            s = a1 - a0
            if min(x1, a1 + s) > max(x0, a0 - s) and min(y1, b1 + s) > max(y0, b0 - s):
                owner[j] = i
                break
    return owner


_REAL_OWNERS = O.extension_owners


def _earlier_wins_ties(tree):
    """Planted: the nearest cut leaf, but the earlier one in Z-order on a tie."""
    real = _REAL_OWNERS(tree)
    cut = tree.cut_leaves()
    owner = list(real)
    for j, o in enumerate(real):
        if o < 0:
            continue
        cj = np.array(O.box_center(tree.leaves[j]))
        d2o = np.sum((np.array(O.box_center(tree.leaves[o])) - cj) ** 2)
        for i in cut:
            if i >= o:
                break
            a0, a1, b0, b1 = O.box_bounds(tree.leaves[i])
            s = a1 - a0
            x0, x1, y0, y1 = O.box_bounds(tree.leaves[j])
            ov = min(x1, a1 + s) > max(x0, a0 - s) and min(y1, b1 + s) > max(y0, b0 - s)
            if ov and np.sum((np.array(O.box_center(tree.leaves[i])) - cj) ** 2) == d2o:
                owner[j] = i
                break
    return owner


@pytest.mark.parametrize("planted", [_first_overlapping_owner, _earlier_wins_ties])
def test_wrong_extension_owner_rule_is_caught(monkeypatch, planted):
    import test_oracle_tree_rules as T
    monkeypatch.setattr(O, "extension_owners", planted)
    caught = 0
    for name in T.OWNER_TREES:
        try:
            T.test_extension_owners_brute_force(name)
        except AssertionError:
            caught += 1
    assert caught > 0


@pytest.mark.parametrize("mask", ["degree_K", "tensor"])
def test_wrong_refinement_tail_is_caught(monkeypatch, mask):
    """Planted: the tail taken from total degree >= K (the K-1 diagonal dropped),
    or as a tensor tail (max(m, n) >= K-1) in place of the total degree."""
    import test_oracle_tree_rules as T

    def planted(F, Vinv, K):
        C = Vinv @ F @ Vinv.T
        mm, nn = np.meshgrid(np.arange(K), np.arange(K), indexing="xy")
        sel = (mm + nn) >= K if mask == "degree_K" else np.maximum(mm, nn) >= K - 1
        return float(np.max(np.abs(C[sel])))
    monkeypatch.setattr(O, "legendre_tail_max", planted)
    with pytest.raises(AssertionError):
        T.test_refinement_matches_closed_form_legendre_tails(*T.R8_CASES[0])
