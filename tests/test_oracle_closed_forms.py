"""Pins of the FP64 oracle against closed forms: single pendulum, planar
double pendulum (equations of motion derived symbolically from its
Lagrangian), a single free rigid body (Newton-Euler), planar forward
kinematics. Each fixes a convention the paper leaves open (the sign of the
gravity term a_g in Algorithm 1, the free-flyer coordinates)."""

import numpy as np
import pytest

from gen import RobotModel
from oracle import rbd
from oracle.derivatives import rnea_derivatives
from tests.pins import normwise


def _model(parent, jt, axis, placement, inertia, g=(0.0, 0.0, -9.81)):
    n = len(parent)
    return RobotModel("t", np.array(parent, np.int32), np.array(jt, np.int32),
                      np.array(axis, float).reshape(n, 3), np.array(placement, float).reshape(n, 12),
                      np.array(inertia, float).reshape(n, 10), np.array(g, float))


EYE = [1, 0, 0, 0, 1, 0, 0, 0, 1]


def pendulum(m=1.7, l=0.6, Ixx=0.03):
    # joint about world x at the origin; COM hangs at (0, 0, -l) for q = 0
    return _model([-1], [0], [1, 0, 0], EYE + [0, 0, 0],
                  [m, 0, 0, -l, Ixx, 0.05, 0.02, 0.004, -0.003, 0.001])


def test_pendulum_rnea_crba_aba():
    m, l, Ixx, g = 1.7, 0.6, 0.03, 9.81
    mod = pendulum(m, l, Ixx)
    rng = np.random.default_rng(0)
    q = rng.uniform(-np.pi, np.pi, (64, 1))
    qd = rng.uniform(-2, 2, (64, 1))
    qdd = rng.uniform(-5, 5, (64, 1))
    Ia = Ixx + m * l * l
    tau = Ia * qdd + m * g * l * np.sin(q)
    assert np.allclose(rbd.rnea(mod, q, qd, qdd), tau, rtol=1e-13, atol=1e-13)
    assert np.allclose(rbd.crba(mod, q)[:, 0, 0], Ia, rtol=1e-14)
    assert np.allclose(rbd.aba(mod, q, qd, tau), qdd, atol=1e-12)
    assert np.allclose(rbd.aba_recursive(mod, q, qd, tau), qdd, atol=1e-12)
    dq, dqd, dqdd = rnea_derivatives(mod, q, qd, qdd)
    assert np.allclose(dq[:, 0, 0], m * g * l * np.cos(q[:, 0]), rtol=1e-12, atol=1e-12)
    assert np.allclose(dqd, 0.0, atol=1e-13)
    assert np.allclose(dqdd[:, 0, 0], Ia, rtol=1e-14)


def test_gravity_sign_horizontal_pendulum():
    """Holding the pendulum horizontal (q = pi/2, COM at +y) takes a positive
    torque m g l about +x: tau contains +g(q) (Eq. 1)."""
    m, l = 2.0, 0.5
    mod = pendulum(m, l)
    tau = rbd.rnea(mod, np.array([[np.pi / 2]]), np.zeros((1, 1)), np.zeros((1, 1)))
    assert tau[0, 0] == pytest.approx(m * 9.81 * l, rel=1e-14)


def _double_pendulum_closed_form():
    sp = pytest.importorskip("sympy")
    t1, t2, d1, d2, a1, a2 = sp.symbols("t1 t2 d1 d2 a1 a2")
    m1, m2, l1, c1, c2, I1, I2, g = sp.symbols("m1 m2 l1 c1 c2 I1 I2 g")
    # planar coordinates (y, z) of both COMs, angles from the downward vertical
    y1, z1 = c1 * sp.sin(t1), -c1 * sp.cos(t1)
    y2 = l1 * sp.sin(t1) + c2 * sp.sin(t1 + t2)
    z2 = -l1 * sp.cos(t1) - c2 * sp.cos(t1 + t2)
    q, qd, qdd = [t1, t2], [d1, d2], [a1, a2]
    dt = lambda e: sum(sp.diff(e, q[k]) * qd[k] for k in range(2))
    T = (m1 * (dt(y1) ** 2 + dt(z1) ** 2) + I1 * d1 ** 2
         + m2 * (dt(y2) ** 2 + dt(z2) ** 2) + I2 * (d1 + d2) ** 2) / 2
    V = g * (m1 * z1 + m2 * z2)
    L = T - V
    taus = []
    for k in range(2):
        p = sp.diff(L, qd[k])
        dpdt = sum(sp.diff(p, q[j]) * qd[j] + sp.diff(p, qd[j]) * qdd[j] for j in range(2))
        taus.append(sp.simplify(dpdt - sp.diff(L, q[k])))
    return sp.lambdify((t1, t2, d1, d2, a1, a2, m1, m2, l1, c1, c2, I1, I2, g), taus, "numpy")


def test_double_pendulum_lagrangian():
    f = _double_pendulum_closed_form()
    m1, m2, l1, c1, c2, I1, I2 = 1.3, 0.9, 0.45, 0.2, 0.25, 0.02, 0.011
    mod = _model([-1, 0], [0, 0], [1, 0, 0, 1, 0, 0],
                 EYE + [0, 0, 0] + EYE + [0, 0, -l1],
                 [m1, 0, 0, -c1, I1, 0.03, 0.01, 0, 0, 0,
                  m2, 0, 0, -c2, I2, 0.02, 0.015, 0, 0, 0])
    rng = np.random.default_rng(1)
    q = rng.uniform(-np.pi, np.pi, (32, 2))
    qd = rng.uniform(-2, 2, (32, 2))
    qdd = rng.uniform(-5, 5, (32, 2))
    ref = np.stack(f(q[:, 0], q[:, 1], qd[:, 0], qd[:, 1], qdd[:, 0], qdd[:, 1],
                     m1, m2, l1, c1, c2, I1, I2, 9.81), -1)
    assert normwise(rbd.rnea(mod, q, qd, qdd), ref) < 1e-13
    # mass matrix = coefficients of qdd
    M = rbd.crba(mod, q)
    for j in range(2):
        e = np.zeros((32, 2))
        e[:, j] = 1
        colj = np.stack(f(q[:, 0], q[:, 1], 0 * q[:, 0], 0 * q[:, 0], e[:, 0], e[:, 1],
                          m1, m2, l1, c1, c2, I1, I2, 0.0), -1)
        assert normwise(M[:, :, j], colj) < 1e-13


def test_planar_forward_kinematics():
    l1 = 0.45
    mod = _model([-1, 0], [0, 0], [1, 0, 0, 1, 0, 0], EYE + [0, 0, 0] + EYE + [0, 0, -l1],
                 [1, 0, 0, 0, 0.1, 0.1, 0.1, 0, 0, 0] * 2)
    rng = np.random.default_rng(2)
    q = rng.uniform(-np.pi, np.pi, (16, 2))
    R, p = rbd.fk(mod, q)
    assert np.allclose(p[:, 1], np.stack([0 * q[:, 0], l1 * np.sin(q[:, 0]), -l1 * np.cos(q[:, 0])], -1), atol=1e-15)
    th = q[:, 0] + q[:, 1]
    Rx = np.zeros((16, 3, 3))
    Rx[:, 0, 0] = 1
    Rx[:, 1, 1], Rx[:, 1, 2] = np.cos(th), -np.sin(th)
    Rx[:, 2, 1], Rx[:, 2, 2] = np.sin(th), np.cos(th)
    assert np.allclose(R[:, 1], Rx, atol=1e-15)


def test_free_rigid_body_newton_euler():
    """One free-flying body with COM offset c: the root wrench RNEA returns is
    [Ic w' + w x Ic w + c x F; F] with F = m (v' + w' x c + w x (v + w x c))
    - m R^T g, all in body coordinates (q = [p, quat(x,y,z,w)],
    qd = [w_b; v_b], qdd = d/dt qd)."""
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    m = 3.1
    c = np.array([0.05, -0.02, 0.07])
    Icm = np.array([[0.04, 0.003, -0.002], [0.003, 0.05, 0.001], [-0.002, 0.001, 0.03]])
    mod = _model([-1], [1], [1, 0, 0], EYE + [0, 0, 0],
                 [m, *c, Icm[0, 0], Icm[1, 1], Icm[2, 2], Icm[0, 1], Icm[0, 2], Icm[1, 2]])
    rng = np.random.default_rng(3)
    B = 32
    quat = rng.standard_normal((B, 4))
    quat /= np.linalg.norm(quat, axis=1, keepdims=True)
    q = np.concatenate([rng.uniform(-1, 1, (B, 3)), quat], 1)
    qd = rng.uniform(-1, 1, (B, 6))
    qdd = rng.uniform(-5, 5, (B, 6))
    R = Rot.from_quat(quat).as_matrix()  # scalar-last (x, y, z, w)
    w, v, wd, vd = qd[:, :3], qd[:, 3:], qdd[:, :3], qdd[:, 3:]
    gb = np.einsum("bji,j->bi", R, np.array([0, 0, -9.81]))
    F = m * (vd + np.cross(wd, c) + np.cross(w, v + np.cross(w, c))) - m * gb
    n = wd @ Icm.T + np.cross(w, w @ Icm.T) + np.cross(c, F)
    assert normwise(rbd.rnea(mod, q, qd, qdd), np.concatenate([n, F], 1)) < 1e-13
    Rf, pf = rbd.fk(mod, q)
    assert np.allclose(Rf[:, 0], R, atol=1e-14) and np.allclose(pf[:, 0], q[:, :3], atol=1e-15)
