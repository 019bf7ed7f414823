"""Pins of the oracle's external forces (Algorithm 1's ^0F_ext, Eq. 1/2's
J^T f): the virtual-power identity against FK twists alone, a pendulum
pushed at its tip (statics by hand), and forward dynamics inverting inverse
dynamics with the same forces. Planted mistakes (sign, moment about the body
origin instead of the root origin, body instead of root coordinates) each
fail a pin."""

import numpy as np
import pytest

import gen
from oracle import rbd
from tests import pins
from tests.pins import normwise
from tests.test_oracle_closed_forms import pendulum


def _world_twists(model, q, qd):
    """Root-frame Pluecker velocities [omega; v_O] of every body, v_O the
    velocity of the body-fixed point at the root origin: from FK only."""
    tw = pins.twists(model, q, qd)
    R, p = rbd.fk(model, q)
    w = np.einsum("bnij,bnj->bni", R, tw[..., :3])
    pdot = np.einsum("bnij,bnj->bni", R, tw[..., 3:])
    return np.concatenate([w, pdot - np.cross(w, p)], -1)


def _power_pin(model, seed):
    """qd^T (tau(F = 0) - tau(F)) = sum_i F_i . V_i: the torques an
    external wrench takes off the joints do its virtual work."""
    s = gen.draw_states(model, 6, seed)
    F = np.random.default_rng(seed + 1).standard_normal((6, model.n_bodies, 6))
    t0 = rbd.rnea(model, s.q, s.qd, s.qdd)
    tF = rbd.rnea(model, s.q, s.qd, s.qdd, fext=F)
    lhs = np.einsum("bi,bi->b", s.qd, t0 - tF)
    rhs = np.einsum("bni,bni->b", F, _world_twists(model, s.q, s.qd))
    return np.max(np.abs(lhs - rhs)) / np.max(np.abs(rhs))


@pytest.mark.parametrize("name", ["chain7", "humanoid", "tree_a"])
def test_virtual_power(models, name):
    assert _power_pin(models[name], 81) < 1e-8


def _pendulum_pin():
    """Pendulum about world x, COM at (0, 0, -l): a force f at the world
    point c on the body adds the moment (c x f)_x about the joint, so
    tau = (I_x + m l^2) qdd + m g l sin q - (c x f)_x."""
    m, l, Ixx, g = 1.7, 0.6, 0.03, 9.81
    mod = pendulum(m, l, Ixx)
    rng = np.random.default_rng(82)
    q = rng.uniform(-np.pi, np.pi, (8, 1))
    qdd = rng.uniform(-5, 5, (8, 1))
    c = np.stack([rng.uniform(-0.1, 0.1, 8), 0.9 * np.sin(q[:, 0]), -0.9 * np.cos(q[:, 0])], -1)
    f = rng.standard_normal((8, 3))
    F = np.concatenate([np.cross(c, f), f], -1)[:, None, :]
    tau = rbd.rnea(mod, q, 0 * q, qdd, fext=F)
    ref = (Ixx + m * l * l) * qdd[:, 0] + m * g * l * np.sin(q[:, 0]) - np.cross(c, f)[:, 0]
    return np.max(np.abs(tau[:, 0] - ref))


def test_pendulum_pushed_at_tip():
    assert _pendulum_pin() < 1e-10


@pytest.mark.parametrize("name", ["chain7", "humanoid", "tree_a"])
def test_forward_dynamics_with_forces(models, name):
    m = models[name]
    s = gen.draw_states(m, 6, 83)
    F = np.random.default_rng(84).standard_normal((6, m.n_bodies, 6))
    qdd = rbd.aba(m, s.q, s.qd, s.tau, fext=F)
    assert normwise(rbd.rnea(m, s.q, s.qd, qdd, fext=F), s.tau) < 1e-10
    assert normwise(rbd.aba_recursive(m, s.q, s.qd, s.tau, fext=F), qdd) < 1e-9


def _sign_flipped(model, q, fext):
    return -_true(model, q, fext)


def _moment_about_body_origin(model, q, fext):
    R, _ = rbd.fk(model, q)
    Rt = np.swapaxes(R, -1, -2)
    return np.concatenate([np.einsum("bnij,bnj->bni", Rt, fext[..., :3]),
                           np.einsum("bnij,bnj->bni", Rt, fext[..., 3:])], -1)


def _root_coordinates(model, q, fext):
    R, p = rbd.fk(model, q)
    n_, f_ = fext[..., :3], fext[..., 3:]
    return np.concatenate([n_ - np.cross(p, f_), f_], -1)


_true = rbd.external_body_forces


@pytest.mark.parametrize("fn", [_sign_flipped, _moment_about_body_origin, _root_coordinates])
def test_planted_mistakes_fail_a_pin(monkeypatch, models, fn):
    monkeypatch.setattr(rbd, "external_body_forces", fn)
    failed = _power_pin(models["chain7"], 81) > 1e-8 or _pendulum_pin() > 1e-10
    assert failed
