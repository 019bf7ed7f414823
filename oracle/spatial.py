"""Spatial algebra in plain numpy (FP64 or complex128 for complex-step).

Featherstone's 6-D spatial vectors, ordered [angular; linear] (the cross
products x and x* of Table III). Every function broadcasts over leading
batch dimensions. Nothing here takes an absolute value or a conjugate, so all
of it is complex-analytic and complex-step differentiation goes through it.
"""

import numpy as np


def skew(v):
    """[v]x, the 3x3 matrix with [v]x u = v x u."""
    x, y, z = v[..., 0], v[..., 1], v[..., 2]
    o = np.zeros_like(x)
    return np.stack([
        np.stack([o, -z, y], -1),
        np.stack([z, o, -x], -1),
        np.stack([-y, x, o], -1),
    ], -2)


def block(a, b, c, d):
    """[[a, b], [c, d]] from four (..., 3, 3) blocks."""
    return np.concatenate([np.concatenate([a, b], -1), np.concatenate([c, d], -1)], -2)


def crm(m):
    """Motion cross product operator m x (Table III), 6x6."""
    W = skew(m[..., :3])
    V = skew(m[..., 3:])
    return block(W, np.zeros_like(W), V, W)


def crf(m):
    """Force cross product operator m x* = -(m x)^T (Table III), 6x6."""
    return -np.swapaxes(crm(m), -1, -2)


def motion_transform(E, r):
    """Plücker transform taking motion vectors from a parent frame to a child
    frame whose orientation is E (child coords -> parent coords) and whose
    origin is r (parent coords): omega' = E^T omega, v' = E^T (v - r x omega)."""
    Et = np.swapaxes(E, -1, -2)
    return block(Et, np.zeros_like(Et), -Et @ skew(r), Et)


def motion_transform_inverse(E, r):
    """Inverse of ``motion_transform(E, r)``: child -> parent coordinates."""
    return block(E, np.zeros_like(E), skew(r) @ E, E)


def spatial_inertia(m, c, Ic):
    """Spatial inertia about the body origin of a body with mass m, centre of
    mass c and rotational inertia Ic about the centre of mass."""
    C = skew(c)
    Ct = np.swapaxes(C, -1, -2)
    eye = np.broadcast_to(np.eye(3), C.shape)
    return block(Ic + m * (C @ Ct), m * C, m * Ct, m * eye)


def rotation_about_axis(axis, angle):
    """Rodrigues: rotation by ``angle`` (batch,) about the unit ``axis`` (3,)."""
    K = skew(np.asarray(axis))
    s = np.sin(angle)[..., None, None]
    c = np.cos(angle)[..., None, None]
    return np.eye(3) + s * K + (1.0 - c) * (K @ K)


def quat_to_rotation(quat):
    """Rotation matrix of a unit quaternion (x, y, z, w), batched."""
    x, y, z, w = quat[..., 0], quat[..., 1], quat[..., 2], quat[..., 3]
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], -1),
        np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], -1),
        np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], -1),
    ], -2)


def quat_multiply(a, b):
    """Hamilton product a (x) b of quaternions stored (x, y, z, w)."""
    av, aw = a[..., :3], a[..., 3:4]
    bv, bw = b[..., :3], b[..., 3:4]
    v = aw * bv + bw * av + np.cross(av, bv)
    w = aw * bw - np.sum(av * bv, -1, keepdims=True)
    return np.concatenate([v, w], -1)


def quat_exp(w):
    """Unit quaternion of the rotation vector w: [sin(|w|/2) w/|w|, cos(|w|/2)].
    |w| is taken as sqrt(w.w) without a conjugate so complex steps pass."""
    th2 = np.sum(w * w, -1, keepdims=True)
    th = np.sqrt(th2)
    with np.errstate(divide="ignore", invalid="ignore"):
        k = np.where(th2 == 0, 0.5, np.sin(th / 2) / np.where(th2 == 0, 1.0, th))
    return np.concatenate([k * w, np.cos(th / 2)], -1)


def matvec(A, x):
    return np.einsum("...ij,...j->...i", A, x)
