"""Independent physics used to pin the oracle (no recursion, no spatial
inertia): body twists from complex-step derivatives of forward kinematics,
kinetic energy from centre-of-mass velocities, potential energy from
centre-of-mass heights, and the Lagrangian equations of motion by finite
differences."""

import numpy as np

from oracle import rbd
from oracle.derivatives import retract

H = 1e-30


def twists(model, q, qd):
    """Body-frame twists [omega_b; v_b] (B, n, 6) of every body for joint
    velocity qd: d/dt of forward kinematics along the motion (complex step)."""
    R1, p1 = rbd.fk(model, retract(model, q, 1j * H * qd.astype(np.complex128)))
    Rd, pd = np.imag(R1) / H, np.imag(p1) / H
    R, p = rbd.fk(model, q)
    Rt = np.swapaxes(R, -1, -2)
    W = Rt @ Rd
    w = np.stack([W[..., 2, 1], W[..., 0, 2], W[..., 1, 0]], -1)
    v = np.einsum("bnij,bnj->bni", Rt, pd)
    return np.concatenate([w, v], -1)


def _inertia_parts(model):
    m = model.inertia[:, 0]
    c = model.inertia[:, 1:4]
    xx, yy, zz, xy, xz, yz = model.inertia[:, 4:10].T
    Ic = np.stack([np.stack([xx, xy, xz], -1), np.stack([xy, yy, yz], -1), np.stack([xz, yz, zz], -1)], -2)
    return m, c, Ic


def kinetic_bilinear(model, q, a, b):
    """B(a, b) with T = B(qd, qd) / 2: sum over bodies of
    m v_c(a) . v_c(b) + w(a)^T Ic w(b), v_c the COM velocity."""
    m, c, Ic = _inertia_parts(model)
    ta, tb = twists(model, q, a), twists(model, q, b)
    wa, wb = ta[..., :3], tb[..., :3]
    vca = ta[..., 3:] + np.cross(wa, c)
    vcb = tb[..., 3:] + np.cross(wb, c)
    return np.sum(m * np.sum(vca * vcb, -1) + np.einsum("bni,nij,bnj->bn", wa, Ic, wb), -1)


def kinetic_energy(model, q, qd):
    return 0.5 * kinetic_bilinear(model, q, qd, qd)


def potential_energy(model, q):
    """V = -sum m_i g . c_i (world COM positions)."""
    m, c, _ = _inertia_parts(model)
    R, p = rbd.fk(model, q)
    cw = p + np.einsum("bnij,nj->bni", R, c)
    return -np.sum(m * (cw @ np.asarray(model.gravity)), -1)


def momentum(model, q, qd):
    """Generalised momentum dT/dqd (T quadratic in qd)."""
    nv = qd.shape[1]
    return np.stack([kinetic_bilinear(model, q, qd, np.tile(np.eye(nv)[j], (q.shape[0], 1)))
                     for j in range(nv)], -1)


def lagrange_tau(model, q, qd, qdd, h=1e-5):
    """tau = d/dt dL/dqd - dL/dq for a fixed-base model, L = T - V, with the
    time derivative along (qd, qdd) and dL/dq by central differences."""
    nv = qd.shape[1]
    dpdt = (momentum(model, q + h * qd, qd) - momentum(model, q - h * qd, qd)) / (2 * h) \
        + momentum(model, q, qdd)
    L = lambda qq: kinetic_energy(model, qq, qd) - potential_energy(model, qq)
    dLdq = np.stack([(L(q + h * np.eye(nv)[j]) - L(q - h * np.eye(nv)[j])) / (2 * h) for j in range(nv)], -1)
    return dpdt - dLdq


def energy_rate(model, q, qd, qdd, h=1e-5):
    """d/dt (T + V) along the motion with velocity qd and acceleration qdd:
    the configuration part by central differences along q (+) h qd, the
    velocity part dT/dqd . qdd exactly (T is quadratic in qd)."""
    E = lambda qq: kinetic_energy(model, qq, qd) + potential_energy(model, qq)
    dEdq = (E(retract(model, q, h * qd)) - E(retract(model, q, -h * qd))) / (2 * h)
    return dEdq + kinetic_bilinear(model, q, qd, qdd)


def normwise(x, ref):
    """Max over instances of ||x - ref||_inf / max(||ref||_inf, 1e-12)."""
    B = ref.shape[0]
    d = np.abs(np.asarray(x) - np.asarray(ref)).reshape(B, -1).max(1)
    r = np.maximum(np.abs(np.asarray(ref)).reshape(B, -1).max(1), 1e-12)
    return float(np.max(d / r))
