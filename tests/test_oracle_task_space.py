"""Pins of the task-space oracle: Jdot qd against finite differences of
forward kinematics alone; Lambda of a free rigid body against its spatial
inertia written out from mass, centre of mass and inertia; and the
controller against the closed-loop identity J ABA(q, qd, tau) + Jdot qd =
x_dd_des (the defining property of the operational-space controller).

The random trees are not used: their frames have at most five joints above
them, so J M^-1 J^T is singular for a 6-D task."""

import numpy as np
import pytest

import gen
from oracle import rbd, task_space
from oracle.derivatives import retract
from tests.pins import normwise
from tests.test_oracle_closed_forms import _model, EYE


def _frame_motion(model, q, frame):
    R, p = rbd.fk(model, q)
    return R[:, frame], p[:, frame]


@pytest.mark.parametrize("name", ["chain7", "humanoid"])
def test_jdot_qd_is_the_fk_second_derivative(models, name):
    """Along the curve q(t) = q (+) t qd: p_dd by a central second difference
    of the frame position, omega_dot by a central first difference of
    omega(t) = vee(Rdot R^T), Rdot itself by central differences. Revolute
    joints move at constant rate on that curve; a free root moves its origin
    along the fixed world direction R(0) v, so its body-frame linear velocity
    turns at -omega x v, an acceleration J adds to the frame's."""
    m = models[name]
    s = gen.draw_states(m, 6, 51)
    frame = m.end_frames[0]
    h = 1e-4
    at = lambda t: retract(m, s.q, t * s.qd)
    pos = lambda t: _frame_motion(m, at(t), frame)[1]
    pdd = (pos(h) - 2 * pos(0.0) + pos(-h)) / (h * h)

    def omega(t, e=1e-6):
        Rp = _frame_motion(m, at(t + e), frame)[0]
        Rm = _frame_motion(m, at(t - e), frame)[0]
        R0 = _frame_motion(m, at(t), frame)[0]
        W = ((Rp - Rm) / (2 * e)) @ np.swapaxes(R0, -1, -2)
        return np.stack([W[:, 2, 1], W[:, 0, 2], W[:, 1, 0]], -1)

    wd = (omega(h) - omega(-h)) / (2 * h)
    jd = task_space.jdot_qd(m, s.q, s.qd, frame)
    if m.has_free_root:
        qdd_curve = np.zeros_like(s.qd)
        qdd_curve[:, 3:6] = -np.cross(s.qd[:, 0:3], s.qd[:, 3:6])
        jd = jd + np.einsum("bij,bj->bi", rbd.jacobian(m, s.q, [frame])[:, 0], qdd_curve)
    assert normwise(jd, np.concatenate([wd, pdd], -1)) < 1e-5


@pytest.mark.parametrize("name", ["chain7", "humanoid"])
def test_osc_closed_loop_identity(models, name):
    m = models[name]
    s = gen.draw_states(m, 8, 52)
    frame = m.end_frames[-1]
    xdd = np.random.default_rng(53).uniform(-3, 3, (8, 6))
    tau, Lam = task_space.osc(m, s.q, s.qd, frame, xdd)
    qdd = rbd.aba(m, s.q, s.qd, tau)
    J = rbd.jacobian(m, s.q, [frame])[:, 0]
    achieved = np.einsum("bij,bj->bi", J, qdd) + task_space.jdot_qd(m, s.q, s.qd, frame)
    assert normwise(achieved, xdd) < 1e-8
    assert normwise(Lam, np.swapaxes(Lam, -1, -2)) < 1e-10
    assert np.linalg.eigvalsh(0.5 * (Lam + np.swapaxes(Lam, -1, -2))).min() > 0


def test_free_body_lambda_is_its_spatial_inertia():
    """One free body, task frame at its origin: J = diag(R, R), so
    Lambda = diag(R, R) I_o diag(R, R)^T with I_o the spatial inertia about
    the body origin, and tau = I_o (R^T xdd) + v x* I_o v - (gravity)."""
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    m, c = 2.3, np.array([0.04, -0.03, 0.06])
    Icm = np.array([[0.05, 0.002, -0.001], [0.002, 0.04, 0.003], [-0.001, 0.003, 0.06]])
    fb = _model([-1], [1], [1, 0, 0], EYE + [0, 0, 0],
                [m, *c, Icm[0, 0], Icm[1, 1], Icm[2, 2], Icm[0, 1], Icm[0, 2], Icm[1, 2]])
    rng = np.random.default_rng(54)
    quat = rng.standard_normal((5, 4))
    quat /= np.linalg.norm(quat, axis=1, keepdims=True)
    q = np.concatenate([rng.uniform(-1, 1, (5, 3)), quat], 1)
    qd = rng.uniform(-1, 1, (5, 6))
    C = np.array([[0, -c[2], c[1]], [c[2], 0, -c[0]], [-c[1], c[0], 0]])
    Io = np.block([[Icm + m * C @ C.T, m * C], [m * C.T, m * np.eye(3)]])
    R = Rot.from_quat(quat).as_matrix()
    T = np.zeros((5, 6, 6))
    T[:, :3, :3] = R
    T[:, 3:, 3:] = R
    _, Lam = task_space.osc(fb, q, qd, 0, np.zeros((5, 6)))
    assert normwise(Lam, T @ Io @ np.swapaxes(T, -1, -2)) < 1e-10
