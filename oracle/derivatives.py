"""Exact first derivatives of RNEA and forward dynamics, and their VJPs.

Test infrastructure only. The derivative of an analytic function f at x in
direction e is Im f(x + i h e) / h up to rounding for a tiny h (complex-step
differentiation, no subtractive cancellation); with h = 1e-30 this is the
derivative to FP64 precision. The paper differentiates its dynamics with JAX
(Sec. I, Sec. IV-A) and lists analytic RNEA derivatives as future work
(Sec. VI); the derivative itself is the plain definition the oracle uses.

Configuration derivatives are taken in the tangent space (nv directions):
q (+) d moves a revolute angle by d_i and a free-flyer root by
T' = T * Exp([dw; dv]) with dw, dv in the body frame. ``to_ambient`` maps a
tangent cotangent onto the nq-entry layout of q: a revolute entry is copied,
the root position gets R dv_bar and the root quaternion 2 Q(quat) dw_bar,
where Q(quat) w = quat (x) [w; 0]; that vector is tangent to the unit sphere
and satisfies quat_bar . dquat = dw_bar . dw for every dquat = Q dw / 2.
"""

import numpy as np

from .rbd import Layout, FREE, aba, crba, fk, rnea
from .spatial import matvec, quat_exp, quat_multiply, quat_to_rotation

H_STEP = 1e-30


def retract(model, q, d):
    """q (+) d: (B, nq) x (B, nv) -> (B, nq), complex-safe."""
    lay = Layout(model)
    out = q.astype(np.result_type(q, d)).copy()
    for i in range(lay.n):
        qs, vs = lay.qslice(i), lay.vslice(i)
        if lay.jtype[i] == FREE:
            qi = q[:, qs]
            di = d[:, vs]
            R = quat_to_rotation(qi[:, 3:7])
            out[:, qs.start:qs.start + 3] = qi[:, 0:3] + matvec(R, di[:, 3:6])
            out[:, qs.start + 3:qs.start + 7] = quat_multiply(qi[:, 3:7], quat_exp(di[:, 0:3]))
        else:
            out[:, qs] = q[:, qs] + d[:, vs]
    return out


def to_ambient(model, q, gt):
    """Tangent cotangent (B, nv) -> ambient gradient layout (B, nq)."""
    lay = Layout(model)
    out = np.zeros((q.shape[0], lay.nq), dtype=np.result_type(q, gt))
    for i in range(lay.n):
        qs, vs = lay.qslice(i), lay.vslice(i)
        g = gt[:, vs]
        if lay.jtype[i] == FREE:
            quat = q[:, qs.start + 3:qs.start + 7]
            R = quat_to_rotation(quat)
            out[:, qs.start:qs.start + 3] = matvec(R, g[:, 3:6])
            w4 = np.concatenate([g[:, 0:3], np.zeros_like(g[:, :1])], -1)
            out[:, qs.start + 3:qs.start + 7] = 2.0 * quat_multiply(quat, w4)
        else:
            out[:, qs] = g
    return out


def complex_step_jacobian(fun, B, n_in, h=H_STEP):
    """(B, n_out, n_in) Jacobian of fun: (B, n_in) complex perturbation ->
    (B, n_out), one complex evaluation per input direction."""
    cols = []
    for k in range(n_in):
        d = np.zeros((B, n_in), dtype=np.complex128)
        d[:, k] = 1j * h
        cols.append(np.imag(fun(d)) / h)
    return np.stack(cols, -1)


def rnea_derivatives(model, q, qd, qdd, gravity=True):
    """(dtau/dq [tangent], dtau/dqd, dtau/dqdd), each (B, nv, nv)."""
    lay = Layout(model)
    B = q.shape[0]
    dq = complex_step_jacobian(lambda d: rnea(model, retract(model, q, d), qd, qdd, gravity), B, lay.nv)
    dqd = complex_step_jacobian(lambda d: rnea(model, q, qd + d, qdd, gravity), B, lay.nv)
    dqdd = complex_step_jacobian(lambda d: rnea(model, q, qd, qdd + d, gravity), B, lay.nv)
    return dq, dqd, dqdd


def aba_derivatives(model, q, qd, tau):
    """(dqdd/dq [tangent], dqdd/dqd, dqdd/dtau), each (B, nv, nv), of the
    forward dynamics of Eq. 2."""
    lay = Layout(model)
    B = q.shape[0]
    dq = complex_step_jacobian(lambda d: aba(model, retract(model, q, d), qd, tau), B, lay.nv)
    dqd = complex_step_jacobian(lambda d: aba(model, q, qd + d, tau), B, lay.nv)
    dtau = complex_step_jacobian(lambda d: aba(model, q, qd, tau + d), B, lay.nv)
    return dq, dqd, dtau


def rnea_vjp(model, q, qd, qdd, gbar):
    """gbar^T d tau: (q_bar (B, nq) ambient, qd_bar (B, nv), qdd_bar (B, nv))."""
    dq, dqd, dqdd = rnea_derivatives(model, q, qd, qdd)
    vt = lambda J: np.einsum("bi,bij->bj", gbar, J)
    return to_ambient(model, q, vt(dq)), vt(dqd), vt(dqdd)


def aba_vjp(model, q, qd, tau, gbar):
    """gbar^T d qdd: (q_bar (B, nq) ambient, qd_bar (B, nv), tau_bar (B, nv))."""
    dq, dqd, dtau = aba_derivatives(model, q, qd, tau)
    vt = lambda J: np.einsum("bi,bij->bj", gbar, J)
    return to_ambient(model, q, vt(dq)), vt(dqd), vt(dtau)


def mass_matrix_rate(model, q, qd):
    """dM/dt along the motion q(t) with q(0) = q, tangent qd (complex step)."""
    d = np.zeros(q.shape[:1] + (Layout(model).nv,), dtype=np.complex128)
    d[:] = 1j * H_STEP * qd
    return np.imag(crba(model, retract(model, q, d))) / H_STEP


# ------------------------------------------------ forward mode (JVPs)
# One complex evaluation along the tangent direction: the directional
# derivative, what jax.jvp returns (Sec. IV-A uses it on the dynamics).

def rnea_jvp(model, q, qd, qdd, dq, dqd, dqdd):
    """d tau along (dq [tangent], dqd, dqdd): (B, nv)."""
    h = H_STEP
    t = rnea(model, retract(model, q, 1j * h * dq.astype(np.complex128)), qd + 1j * h * dqd,
             qdd + 1j * h * dqdd)
    return np.imag(t) / h


def aba_jvp(model, q, qd, tau, dq, dqd, dtau):
    """d qdd along (dq [tangent], dqd, dtau) of Eq. 2: (B, nv)."""
    h = H_STEP
    a = aba(model, retract(model, q, 1j * h * dq.astype(np.complex128)), qd + 1j * h * dqd, tau + 1j * h * dtau)
    return np.imag(a) / h


def fk_jvp(model, q, dq, frames):
    """Motion of each frame body along dq: [omega; d p] (B, nf, 6) in world
    coordinates, omega = vee(dR R^T)."""
    h = H_STEP
    Rc, pc = fk(model, retract(model, q, 1j * h * dq.astype(np.complex128)))
    R, p = fk(model, q)
    f = list(frames)
    W = (np.imag(Rc[:, f]) / h) @ np.swapaxes(R[:, f], -1, -2)
    w = np.stack([W[..., 2, 1], W[..., 0, 2], W[..., 1, 0]], -1)
    return np.concatenate([w, np.imag(pc[:, f]) / h], -1)
