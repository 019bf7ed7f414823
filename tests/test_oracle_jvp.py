"""Pins of the oracle's forward-mode derivatives (JVPs): central finite
differences of the real functions along the same direction, and the parts
with closed forms: d tau along qdd is M qdd-direction, d qdd along tau is
M^-1 dtau, and the motion of a frame along dq is J dq."""

import numpy as np
import pytest

import gen
from oracle import derivatives as dv
from oracle import rbd
from tests.pins import normwise


def _dirs(model, B, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((B, model.nv)) for _ in range(3))


@pytest.mark.parametrize("name", ["chain7", "humanoid", "tree_a"])
def test_rnea_aba_jvp_vs_central_differences(models, name):
    m = models[name]
    s = gen.draw_states(m, 5, 111)
    dq, dqd, dx = _dirs(m, 5, 112)
    h = 1e-6
    step = lambda e: (dv.retract(m, s.q, e * dq), s.qd + e * dqd)
    qp, qdp = step(h)
    qm, qdm = step(-h)
    fd = (rbd.rnea(m, qp, qdp, s.qdd + h * dx) - rbd.rnea(m, qm, qdm, s.qdd - h * dx)) / (2 * h)
    assert normwise(dv.rnea_jvp(m, s.q, s.qd, s.qdd, dq, dqd, dx), fd) < 1e-7
    fd = (rbd.aba(m, qp, qdp, s.tau + h * dx) - rbd.aba(m, qm, qdm, s.tau - h * dx)) / (2 * h)
    assert normwise(dv.aba_jvp(m, s.q, s.qd, s.tau, dq, dqd, dx), fd) < 1e-6


@pytest.mark.parametrize("name", ["chain7", "humanoid"])
def test_jvp_closed_form_parts(models, name):
    m = models[name]
    s = gen.draw_states(m, 5, 113)
    _, _, dx = _dirs(m, 5, 114)
    z = np.zeros_like(dx)
    M = rbd.crba(m, s.q)
    assert normwise(dv.rnea_jvp(m, s.q, s.qd, s.qdd, z, z, dx), np.einsum("bij,bj->bi", M, dx)) < 1e-12
    assert normwise(dv.aba_jvp(m, s.q, s.qd, s.tau, z, z, dx), np.linalg.solve(M, dx[..., None])[..., 0]) < 1e-10


@pytest.mark.parametrize("name", ["chain7", "humanoid", "tree_a"])
def test_fk_jvp_is_jacobian_times_direction(models, name):
    m = models[name]
    s = gen.draw_states(m, 5, 115)
    dq, _, _ = _dirs(m, 5, 116)
    frames = list(m.end_frames)[:4]
    J = rbd.jacobian(m, s.q, frames)
    assert normwise(dv.fk_jvp(m, s.q, dq, frames), np.einsum("bfij,bj->bfi", J, dq)) < 1e-12
