"""Recursive rigid-body algorithms, FP64, batched over instances.

Test infrastructure only (see the package docstring). Every loop runs over the
bodies of one model in index order (parent[i] < i) and over all instances at
once with numpy broadcasting; no step is reordered, blocked or fused.

The algorithms are the textbook recursions of Featherstone's formulation
(Sec. II): forward kinematics, RNEA (inverse dynamics, Eq. 1 with f = 0),
CRBA (the mass matrix M), and forward dynamics (Eq. 2) as a dense solve.
"""

import numpy as np

from .spatial import (crf, crm, matvec, motion_transform, motion_transform_inverse,
                      quat_to_rotation, rotation_about_axis, skew, spatial_inertia)

REVOLUTE = 0
FREE = 1


class Layout:
    """Per-body offsets into q (nq entries) and qd (nv entries)."""

    def __init__(self, model):
        self.n = int(len(model.parent))
        self.parent = [int(p) for p in model.parent]
        self.jtype = [int(t) for t in model.joint_type]
        self.iq, self.iv, self.kq, self.kv = [], [], [], []
        nq = nv = 0
        for t in self.jtype:
            kq, kv = (7, 6) if t == FREE else (1, 1)
            self.iq.append(nq)
            self.iv.append(nv)
            self.kq.append(kq)
            self.kv.append(kv)
            nq += kq
            nv += kv
        self.nq, self.nv = nq, nv

    def vslice(self, i):
        return slice(self.iv[i], self.iv[i] + self.kv[i])

    def qslice(self, i):
        return slice(self.iq[i], self.iq[i] + self.kq[i])

    def ancestors(self, i):
        """Anc(i) including i itself (the paper's convention for U), from i
        towards the root."""
        out = [i]
        while self.parent[out[-1]] >= 0:
            out.append(self.parent[out[-1]])
        return out


def ancestor_mask(model):
    """U in {0,1}^{n x n}: U[i, j] = 1 iff j in Anc(i), with i in Anc(i)
    (Sec. III, Table III). Lower triangular for a topological order."""
    lay = Layout(model)
    U = np.zeros((lay.n, lay.n), dtype=np.int64)
    for i in range(lay.n):
        for j in lay.ancestors(i):
            U[i, j] = 1
    return U


def motion_subspace(model, i):
    """S_i in body-i coordinates: [axis; 0] for a revolute joint, I_6 for the
    free-flyer (its velocity is the body-frame twist [w_b; v_b])."""
    if int(model.joint_type[i]) == FREE:
        return np.eye(6)
    S = np.zeros((6, 1))
    S[:3, 0] = model.axis[i]
    return S


def body_inertia(model, i):
    m = model.inertia[i, 0]
    c = model.inertia[i, 1:4]
    xx, yy, zz, xy, xz, yz = model.inertia[i, 4:10]
    Ic = np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]])
    return spatial_inertia(m, c, Ic)


def joint_frame(model, lay, i, q):
    """(E, r): orientation (body i -> parent coords) and origin (parent coords)
    of body i, ^lambda T_i = placement_i * joint_i(q_i)."""
    RT = model.placement[i, :9].reshape(3, 3)
    pT = model.placement[i, 9:]
    qi = q[:, lay.qslice(i)]
    if lay.jtype[i] == FREE:
        Rq = quat_to_rotation(qi[:, 3:7])
        E = RT @ Rq
        r = pT + matvec(RT, qi[:, 0:3])
    else:
        E = RT @ rotation_about_axis(model.axis[i], qi[:, 0])
        r = np.broadcast_to(pT, (q.shape[0], 3)).astype(E.dtype)
    return E, r


def joint_transforms(model, q):
    """^iX_lambda(i) for every body, (B, 6, 6) each."""
    lay = Layout(model)
    return [motion_transform(*joint_frame(model, lay, i, q)) for i in range(lay.n)]


def base_acceleration(model, dtype=np.float64):
    """a_0 = [0; -g]: gravity applied as a fictitious upward acceleration of
    the world (the reading of Table III's a_g that makes tau include g(q))."""
    a0 = np.zeros(6, dtype=dtype)
    a0[3:] = -np.asarray(model.gravity)
    return a0


# ---------------------------------------------------------------- kinematics

def fk(model, q):
    """World pose of every body: (R (B, n, 3, 3), p (B, n, 3)).
    ^0T_i = ^0T_lambda(i) * ^lambda T_i."""
    lay = Layout(model)
    B = q.shape[0]
    R = np.zeros((B, lay.n, 3, 3), dtype=q.dtype)
    p = np.zeros((B, lay.n, 3), dtype=q.dtype)
    for i in range(lay.n):
        E, r = joint_frame(model, lay, i, q)
        k = lay.parent[i]
        if k < 0:
            R[:, i], p[:, i] = E, r
        else:
            R[:, i] = R[:, k] @ E
            p[:, i] = p[:, k] + matvec(R[:, k], r)
    return R, p


def fk_flat(model, q):
    """Poses in the ABI layout: per body R row-major (9) then p (3)."""
    R, p = fk(model, q)
    B, n = p.shape[:2]
    return np.concatenate([R.reshape(B, n, 9), p], -1).reshape(B, n * 12)


def jacobian(model, q, frames):
    """Geometric Jacobian of each frame body k, (B, nf, 6, nv): the map from
    qd to [omega (world); d/dt p_k (world)]. Column block of joint j is its
    motion subspace carried to world coordinates, ^0S_j = (^jX_0)^-1 S_j,
    shifted from the world origin to the frame origin p_k; zero unless
    j in Anc(k)."""
    lay = Layout(model)
    R, p = fk(model, q)
    B = q.shape[0]
    out = np.zeros((B, len(frames), 6, lay.nv), dtype=q.dtype)
    for f, k in enumerate(frames):
        shift = np.zeros((B, 6, 6), dtype=q.dtype)
        shift[:, :3, :3] = np.eye(3)
        shift[:, 3:, 3:] = np.eye(3)
        shift[:, 3:, :3] = -skew(p[:, k])
        for j in lay.ancestors(k):
            S0 = motion_transform_inverse(R[:, j], p[:, j]) @ motion_subspace(model, j)
            out[:, f, :, lay.vslice(j)] = shift @ S0
    return out


# ------------------------------------------------------------------ dynamics

def external_body_forces(model, q, fext):
    """Algorithm 1's external forces ^0F_ext,i, given as (B, n, 6) spatial
    forces on the bodies in root-frame Pluecker coordinates [moment about the
    root origin; force], expressed in each body's frame:
    ^iF = (^iX_0)^* ^0F = [R_i^T (n - p_i x f); R_i^T f]."""
    R, p = fk(model, q)
    n_, f_ = fext[..., :3], fext[..., 3:]
    Rt = np.swapaxes(R, -1, -2)
    nb = np.einsum("bnij,bnj->bni", Rt, n_ - np.cross(p, f_))
    fb = np.einsum("bnij,bnj->bni", Rt, f_)
    return np.concatenate([nb, fb], -1)


def rnea(model, q, qd, qdd, gravity=True, fext=None):
    """Inverse dynamics tau = M qdd + c + g (Eq. 1) by the recursive
    Newton-Euler algorithm: outward velocity/acceleration sweep, body forces
    f_i = I_i a_i + v_i x* I_i v_i - F_ext,i (Algorithm 1 subtracts the
    external force; fext as in external_body_forces, None for none), inward
    force sweep, tau_i = S_i^T f_i."""
    lay = Layout(model)
    dt = np.result_type(q, qd, qdd) if fext is None else np.result_type(q, qd, qdd, fext)
    B = q.shape[0]
    X = joint_transforms(model, q)
    fb = None if fext is None else external_body_forces(model, q, fext)
    a0 = base_acceleration(model, dt) if gravity else np.zeros(6, dt)
    v, a, f = [None] * lay.n, [None] * lay.n, [None] * lay.n
    for i in range(lay.n):
        S = motion_subspace(model, i)
        vJ = matvec(S, qd[:, lay.vslice(i)])
        k = lay.parent[i]
        vp = np.zeros((B, 6), dt) if k < 0 else v[k]
        ap = np.broadcast_to(a0, (B, 6)) if k < 0 else a[k]
        v[i] = matvec(X[i], vp) + vJ
        a[i] = matvec(X[i], ap) + matvec(S, qdd[:, lay.vslice(i)]) + matvec(crm(v[i]), vJ)
        I = body_inertia(model, i)
        f[i] = matvec(I, a[i]) + matvec(crf(v[i]), matvec(I, v[i]))
        if fb is not None:
            f[i] = f[i] - fb[:, i]
    tau = np.zeros((B, lay.nv), dt)
    for i in reversed(range(lay.n)):
        S = motion_subspace(model, i)
        tau[:, lay.vslice(i)] = f[i] @ S
        k = lay.parent[i]
        if k >= 0:
            f[k] = f[k] + matvec(np.swapaxes(X[i], -1, -2), f[i])
    return tau


def crba(model, q):
    """Mass matrix M(q) by the composite-rigid-body algorithm: composite
    inertias I^c_lambda += X_i^T I^c_i X_i inward, then
    M[i, j] = S_j^T (^jX_i)^* I^c_i S_i for j in Anc(i), mirrored."""
    lay = Layout(model)
    B = q.shape[0]
    X = joint_transforms(model, q)
    Ic = [np.broadcast_to(body_inertia(model, i), (B, 6, 6)).astype(q.dtype) for i in range(lay.n)]
    for i in reversed(range(lay.n)):
        k = lay.parent[i]
        if k >= 0:
            Ic[k] = Ic[k] + np.swapaxes(X[i], -1, -2) @ Ic[i] @ X[i]
    H = np.zeros((B, lay.nv, lay.nv), q.dtype)
    for i in range(lay.n):
        Si = motion_subspace(model, i)
        F = Ic[i] @ Si
        H[:, lay.vslice(i), lay.vslice(i)] = Si.T @ F
        j = i
        while lay.parent[j] >= 0:
            F = np.swapaxes(X[j], -1, -2) @ F
            j = lay.parent[j]
            blk = motion_subspace(model, j).T @ F
            H[:, lay.vslice(j), lay.vslice(i)] = blk
            H[:, lay.vslice(i), lay.vslice(j)] = np.swapaxes(blk, -1, -2)
    return H


def ltdl(M):
    """The factorisation M = L^T D L with L unit lower triangular and D
    diagonal (positive for SPD M). Plain definition: reversing the index order
    turns it into the ordinary M' = L' D' L'^T, which a dense Cholesky of the
    reversed matrix gives (L' = C diag(C)^-1, D' = diag(C)^2)."""
    n = M.shape[-1]
    rev = np.arange(n)[::-1]
    Mr = M[..., rev[:, None], rev[None, :]]
    C = np.linalg.cholesky(Mr)
    d = np.diagonal(C, axis1=-2, axis2=-1)
    Lp = C / d[..., None, :]
    L = np.swapaxes(Lp, -1, -2)[..., rev[:, None], rev[None, :]]
    D = (d * d)[..., rev]
    return L, D


def pack_ltdl(L, D):
    """ABI layout of the factor: packed lower triangle row-major,
    entry (i, j <= i) at i(i+1)/2 + j, holding D_i on the diagonal and
    L_ij below it."""
    n = D.shape[-1]
    out = []
    for i in range(n):
        for j in range(i + 1):
            out.append(D[..., i] if i == j else L[..., i, j])
    return np.stack(out, -1)


def aba(model, q, qd, tau, fext=None):
    """Forward dynamics as Eq. 2 itself:
    qdd = M(q)^-1 (tau - c(q, qd) - g(q) + sum_i J_i^T F_ext,i), the bias
    term being RNEA(q, qd, 0) with the same external forces."""
    bias = rnea(model, q, qd, np.zeros_like(tau), fext=fext)
    M = crba(model, q)
    return np.linalg.solve(M, (tau - bias)[..., None])[..., 0]


def aba_recursive(model, q, qd, tau, gravity=True, fext=None):
    """The articulated-body algorithm (Featherstone): velocity sweep,
    articulated inertias I^A / bias forces p^A inward (p^A_i = v_i x* I_i v_i
    - F_ext,i), accelerations outward. A second formulation of ``aba`` used
    by the tests."""
    lay = Layout(model)
    dt = np.result_type(q, qd, tau)
    B = q.shape[0]
    X = joint_transforms(model, q)
    fb = None if fext is None else external_body_forces(model, q, fext)
    a0 = base_acceleration(model, dt) if gravity else np.zeros(6, dt)
    v, c, IA, pA = [None] * lay.n, [None] * lay.n, [None] * lay.n, [None] * lay.n
    for i in range(lay.n):
        S = motion_subspace(model, i)
        vJ = matvec(S, qd[:, lay.vslice(i)])
        k = lay.parent[i]
        vp = np.zeros((B, 6), dt) if k < 0 else v[k]
        v[i] = matvec(X[i], vp) + vJ
        c[i] = matvec(crm(v[i]), vJ)
        I = body_inertia(model, i)
        IA[i] = np.broadcast_to(I, (B, 6, 6)).astype(dt)
        pA[i] = matvec(crf(v[i]), matvec(I, v[i]))
        if fb is not None:
            pA[i] = pA[i] - fb[:, i]
    Us, Dinv, u = [None] * lay.n, [None] * lay.n, [None] * lay.n
    for i in reversed(range(lay.n)):
        S = motion_subspace(model, i)
        Us[i] = IA[i] @ S
        Dinv[i] = np.linalg.inv(S.T @ Us[i])
        u[i] = tau[:, lay.vslice(i)] - pA[i] @ S
        k = lay.parent[i]
        if k >= 0:
            Ia = IA[i] - Us[i] @ Dinv[i] @ np.swapaxes(Us[i], -1, -2)
            pa = pA[i] + matvec(Ia, c[i]) + matvec(Us[i] @ Dinv[i], u[i])
            Xt = np.swapaxes(X[i], -1, -2)
            IA[k] = IA[k] + Xt @ Ia @ X[i]
            pA[k] = pA[k] + matvec(Xt, pa)
    qdd = np.zeros((B, lay.nv), dt)
    a = [None] * lay.n
    for i in range(lay.n):
        S = motion_subspace(model, i)
        k = lay.parent[i]
        ap = np.broadcast_to(a0, (B, 6)) if k < 0 else a[k]
        a_ = matvec(X[i], ap) + c[i]
        qi = matvec(Dinv[i], u[i] - np.einsum("bi,bik->bk", a_, Us[i]))
        qdd[:, lay.vslice(i)] = qi
        a[i] = a_ + matvec(S, qi)
    return qdd
