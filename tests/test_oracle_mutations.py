"""The oracle's pins catch plausible mistakes: each test plants one mistake in
the oracle (on the CPU, by replacing one function of oracle.rbd) and checks
that at least one pin then fails. Pins used here: the pendulum closed form,
the free rigid body (Newton-Euler), the Lagrangian built from FK alone, the
paper's mask-form Algorithm 1, kinetic energy from FK twists, and columns of
M from RNEA."""

import numpy as np
import pytest

import gen
from oracle import mask_form, rbd, spatial
from tests import pins
from tests.pins import normwise
from tests.test_oracle_closed_forms import pendulum, _model, EYE


def _pin_results():
    """True for every pin that holds with the oracle as it currently is."""
    out = {}
    mod = pendulum(1.7, 0.6, 0.03)
    rng = np.random.default_rng(0)
    q = rng.uniform(-np.pi, np.pi, (8, 1))
    qd = rng.uniform(-2, 2, (8, 1))
    qdd = rng.uniform(-5, 5, (8, 1))
    out["pendulum"] = np.allclose(rbd.rnea(mod, q, qd, qdd), (0.03 + 1.7 * 0.36) * qdd + 1.7 * 9.81 * 0.6 * np.sin(q),
                                  atol=1e-10)
    # free rigid body with COM offset
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    m, c = 3.1, np.array([0.05, -0.02, 0.07])
    Icm = np.array([[0.04, 0.003, -0.002], [0.003, 0.05, 0.001], [-0.002, 0.001, 0.03]])
    fb = _model([-1], [1], [1, 0, 0], EYE + [0, 0, 0],
                [m, *c, Icm[0, 0], Icm[1, 1], Icm[2, 2], Icm[0, 1], Icm[0, 2], Icm[1, 2]])
    quat = rng.standard_normal((8, 4))
    quat /= np.linalg.norm(quat, axis=1, keepdims=True)
    qf = np.concatenate([rng.uniform(-1, 1, (8, 3)), quat], 1)
    vf, af = rng.uniform(-1, 1, (8, 6)), rng.uniform(-5, 5, (8, 6))
    R = Rot.from_quat(quat).as_matrix()
    w, v, wd, vd = vf[:, :3], vf[:, 3:], af[:, :3], af[:, 3:]
    gb = np.einsum("bji,j->bi", R, np.array([0, 0, -9.81]))
    F = m * (vd + np.cross(wd, c) + np.cross(w, v + np.cross(w, c))) - m * gb
    n = wd @ Icm.T + np.cross(w, w @ Icm.T) + np.cross(c, F)
    out["free_body"] = normwise(rbd.rnea(fb, qf, vf, af), np.concatenate([n, F], 1)) < 1e-10
    # chain: Lagrangian, mask form, kinetic energy, M columns
    ch = gen.chain7(0)
    s = gen.draw_states(ch, 4, 3)
    tau = rbd.rnea(ch, s.q, s.qd, s.qdd)
    out["lagrangian"] = normwise(tau, pins.lagrange_tau(ch, s.q, s.qd, s.qdd)) < 1e-6
    out["mask_form"] = normwise(tau, mask_form.rnea_vectorized(ch, s.q, s.qd, s.qdd)) < 1e-10
    M = rbd.crba(ch, s.q)
    T = 0.5 * np.einsum("bi,bij,bj->b", s.qd, M, s.qd)
    out["kinetic"] = np.max(np.abs(T - pins.kinetic_energy(ch, s.q, s.qd)) / np.abs(T)) < 1e-10
    cols = np.stack([rbd.rnea(ch, s.q, 0 * s.qd, np.tile(np.eye(7)[j], (4, 1)), gravity=False) for j in range(7)], -1)
    out["mass_columns"] = normwise(M, cols) < 1e-10
    return out


def test_all_pins_hold_unmutated():
    assert all(_pin_results().values())


def _crf_wrong_sign(m):
    return np.swapaxes(spatial.crm(m), -1, -2)


def _gravity_wrong_sign(model, dtype=np.float64):
    a0 = np.zeros(6, dtype=dtype)
    a0[3:] = np.asarray(model.gravity)
    return a0


def _transform_transposed(E, r):
    return spatial.motion_transform(np.swapaxes(E, -1, -2), r)


def _no_velocity_product(m):
    return np.zeros(m.shape[:-1] + (6, 6), dtype=m.dtype)


def _no_parallel_axis(m, c, Ic):
    C = spatial.skew(c)
    Ct = np.swapaxes(C, -1, -2)
    eye = np.broadcast_to(np.eye(3), C.shape)
    return spatial.block(Ic, m * C, m * Ct, m * eye)


def _quat_wxyz(quat):
    return spatial.quat_to_rotation(np.concatenate([quat[..., 1:4], quat[..., :1]], -1))


def _placement_after_joint(model, lay, i, q):
    RT = model.placement[i, :9].reshape(3, 3)
    pT = model.placement[i, 9:]
    qi = q[:, lay.qslice(i)]
    if lay.jtype[i] == rbd.FREE:
        Rq = spatial.quat_to_rotation(qi[:, 3:7])
        return RT @ Rq, pT + spatial.matvec(RT, qi[:, 0:3])
    E = spatial.rotation_about_axis(model.axis[i], qi[:, 0]) @ RT
    return E, np.broadcast_to(pT, (q.shape[0], 3)).astype(E.dtype)


MUTATIONS = {
    "crf_sign": ("crf", _crf_wrong_sign),
    "gravity_sign": ("base_acceleration", _gravity_wrong_sign),
    "transposed_transform": ("motion_transform", _transform_transposed),
    "dropped_velocity_product": ("crm", _no_velocity_product),
    "no_parallel_axis": ("spatial_inertia", _no_parallel_axis),
    "quaternion_order": ("quat_to_rotation", _quat_wxyz),
    "placement_order": ("joint_frame", _placement_after_joint),
}


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_planted_mistake_is_caught(monkeypatch, name):
    attr, fn = MUTATIONS[name]
    monkeypatch.setattr(rbd, attr, fn)
    res = _pin_results()
    failed = [k for k, ok in res.items() if not ok]
    assert failed, f"mutation {name} passed every pin"
