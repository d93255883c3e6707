"""Error bounds shared by the GPU parity tests, computed from the oracle's own
operators (test infrastructure: nothing here runs on the device)."""
import math

import numpy as np

from oracle import oracle as O

EPS = np.finfo(float).eps

# unit roundoff of the mixed form's extension: its grid stage (A c over the
# coarse grid) is a five-slice bf16 pass (8-bit digits), each operand rounded
# to 2^-40 of its row or vector maximum and product orders above 4 dropped
MIXED_EXT_EPS = 2.0 ** -37

# Two schedules of the mixed form (engine, pairs per tile, chain or per-level
# launches, batch or single plan) sum the same slice products in other orders,
# so a pass's FP64 output can differ in its last bit.  The next pass re-slices
# that output: where a coefficient lies within one FP64 rounding of a half
# unit of its fifth 8-bit digit, the two schedules round it to neighbouring
# slice values, 2^-39 of its vector's maximum apart.  Such coefficients travel
# through up to 15 levels of M2M/L2L and the M2L and L2T passes; 1e-10 of
# max|V| (about 55 of those units) leaves room for a few per level and stays
# ten times below the mixed form's own parity gate of 1e-9.
MIXED_SCHEDULE_TOL = 1e-10


def chebyshev_stage_norm(b, K, targets):
    """Infinity norm of the map Kbar x Kbar grid values -> truncated Chebyshev
    expansion (m + n < Kbar) evaluated at the targets (Section 4.1)."""
    from numpy.polynomial import chebyshev as C
    q, Kbar, NG = O.stencil_params(K)
    cx, cy = O.box_center(b)
    r = 1.5 * O.box_side(b[0])
    Tinv = np.linalg.inv(C.chebvander(O.chebyshev1_nodes(Kbar), Kbar - 1))
    z = (targets - np.array([cx, cy])) / r
    TX, TY = C.chebvander(z[:, 0], Kbar - 1), C.chebvander(z[:, 1], Kbar - 1)
    mm, nn = np.meshgrid(np.arange(Kbar), np.arange(Kbar), indexing="ij")
    keep = (mm + nn) < Kbar
    # target value = sum_{ax,by} W[t, ax, by] F[ax, by]
    W = np.einsum("tm,ma,tn,nb,mn->tab", TX, Tinv, TY, Tinv, keep.astype(float))
    return max(np.abs(W).reshape(len(targets), -1).sum(axis=1).max(), 1.0)


def extension_bounds(tree, dom, meta, only=None):
    """Per extended leaf: the forward-error factor of the two-stage
    extrapolation, kappa = Lambda * ||A_E|| * ||A_I^+|| (infinity norms), with
    Lambda the norm of the Chebyshev stage (grid values -> target values);
    both implementations are backward stable, so they differ by
    O(eps * kappa * max|f_I|).  Computed from the oracle's own operators;
    `only` restricts it to the given cut leaves (and the leaves they own)."""
    owned = {}
    for j, o in enumerate(tree.owner):
        if o >= 0:
            owned.setdefault(o, []).append(j)
    K = tree.K
    q, Kbar, NG = O.stencil_params(K)
    A = O.universal_matrix(K)
    kappa = {}
    for i in tree.cut_leaves():
        if only is not None and i not in only:
            continue
        off, n, masks = meta[i]
        AI = A[np.concatenate(masks)]
        AE = A[K * K:K * K + Kbar * Kbar][~masks[1]]
        nAE = np.abs(AE).sum(axis=1).max() if len(AE) else 0.0
        nP = np.abs(O.pseudo_inverse(AI)).sum(axis=1).max()
        tg = np.concatenate([O.leaf_nodes(tree.leaves[i], tree.t)] +
                            [O.leaf_nodes(tree.leaves[j], tree.t) for j in owned.get(i, [])])
        lam = chebyshev_stage_norm(tree.leaves[i], K, tg)
        k = lam * (1.0 + nAE * nP)
        kappa[i] = k
        for j in owned.get(i, []):
            kappa[j] = k
    return kappa


def extension_potential_bound(tree, kappa, fmax, eps):
    """Bound on the potential of the extension's rounding: a perturbation delta
    of the values on a leaf of side s changes V by at most
    |delta| s^2 (|log s| + 2) / (2 pi); summed over the extended leaves with
    |delta| <= 64 eps kappa max|f_I|."""
    b = 0.0
    for i, k in kappa.items():
        s = 2.0 ** -tree.leaves[i][0]
        b += 64 * eps * k * fmax * s * s * (abs(math.log(s)) + 2) / (2 * math.pi)
    return b
