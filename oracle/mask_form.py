"""The paper's vectorized formulation (Sec. III), FP64.

Test infrastructure only. Algorithm 1 (vectorized RNEA) and Algorithm 2
(vectorized CRBA) written with the ancestor mask U: every spatial quantity is
expressed in the root frame 0, and sums along the tree become products with U
(down the tree) or U^T (up the tree). The poses come from ``rbd.fk`` (the one
loop the paper keeps); everything after that is mask products. This is an
independent second formulation of ``rbd.rnea`` / ``rbd.crba``.
"""

import numpy as np

from .rbd import Layout, ancestor_mask, base_acceleration, body_inertia, fk, motion_subspace
from .spatial import crf, crm, matvec, motion_transform, motion_transform_inverse


def prepare(model, q):
    """The algorithms' "Prepare" step: ^0S_i (B, 6, k_i) and ^0I_i (B, 6, 6)."""
    lay = Layout(model)
    R, p = fk(model, q)
    S0, I0 = [], []
    for i in range(lay.n):
        to_world = motion_transform_inverse(R[:, i], p[:, i])
        from_world = motion_transform(R[:, i], p[:, i])
        S0.append(to_world @ motion_subspace(model, i))
        I0.append(np.swapaxes(from_world, -1, -2) @ body_inertia(model, i) @ from_world)
    return S0, np.stack(I0, 1)


def rnea_vectorized(model, q, qd, qdd, gravity=True):
    """Algorithm 1: V = U (S qd), A = a_g + U (S qdd + V x S qd),
    F = U^T (I A + V x* I V), Gamma_i = S_i . F_i (no external forces)."""
    lay = Layout(model)
    U = ancestor_mask(model).astype(np.float64)
    S0, I0 = prepare(model, q)
    Sqd = np.stack([matvec(S0[i], qd[:, lay.vslice(i)]) for i in range(lay.n)], 1)
    Sqdd = np.stack([matvec(S0[i], qdd[:, lay.vslice(i)]) for i in range(lay.n)], 1)
    V = np.einsum("ij,bjk->bik", U, Sqd)
    ag = base_acceleration(model, np.result_type(q, qd, qdd))
    if not gravity:
        ag = np.zeros_like(ag)
    A = ag + np.einsum("ij,bjk->bik", U, Sqdd + matvec(crm(V), Sqd))
    IV = matvec(I0, V)
    F = np.einsum("ji,bjk->bik", U, matvec(I0, A) + matvec(crf(V), IV))
    tau = np.zeros((q.shape[0], lay.nv), dtype=F.dtype)
    for i in range(lay.n):
        tau[:, lay.vslice(i)] = np.einsum("bk,bkj->bj", F[:, i], S0[i])
    return tau


def crba_vectorized(model, q):
    """Algorithm 2: C = U^T I, M_lower = U (.) (S_i^T C_i S_j),
    M = Symmetrize(M_lower) (copy the lower triangle to the upper)."""
    lay = Layout(model)
    U = ancestor_mask(model)
    S0, I0 = prepare(model, q)
    C = np.einsum("ji,bjkl->bikl", U.astype(np.float64), I0)
    M = np.zeros((q.shape[0], lay.nv, lay.nv), dtype=C.dtype)
    for i in range(lay.n):
        for j in range(lay.n):
            if U[i, j]:
                blk = np.swapaxes(S0[i], -1, -2) @ C[:, i] @ S0[j]
                M[:, lay.vslice(i), lay.vslice(j)] = blk
                if i != j:
                    M[:, lay.vslice(j), lay.vslice(i)] = np.swapaxes(blk, -1, -2)
    return M
