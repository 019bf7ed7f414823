"""Pins of the oracle's complex-step derivatives and VJPs: FP64 central
differences (step 1e-6), the identities dtau/dqdd = M, dqdd/dtau = M^-1 and
dqdd/dq = -M^-1 dtau/dq (implicit function theorem on Eq. 1/Eq. 2), and the
ambient mapping of free-flyer gradients."""

import numpy as np
import pytest

import gen
from oracle import derivatives as dv
from oracle import rbd
from tests.pins import normwise

B = 6
FD_H = 1e-6


def _central(fun, x, n, h=FD_H):
    cols = []
    for k in range(n):
        d = np.zeros((x.shape[0], n))
        d[:, k] = h
        cols.append((fun(d) - fun(-d)) / (2 * h))
    return np.stack(cols, -1)


@pytest.mark.parametrize("name", ["chain7", "humanoid", "tree_a"])
def test_rnea_derivatives_vs_central_differences(models, name):
    m = models[name]
    s = gen.draw_states(m, B, 11)
    dq, dqd, dqdd = dv.rnea_derivatives(m, s.q, s.qd, s.qdd)
    fq = _central(lambda d: rbd.rnea(m, dv.retract(m, s.q, d), s.qd, s.qdd), s.q, m.nv)
    fqd = _central(lambda d: rbd.rnea(m, s.q, s.qd + d, s.qdd), s.q, m.nv)
    assert normwise(dq, fq) < 1e-7
    assert normwise(dqd, fqd) < 1e-7
    assert normwise(dqdd, rbd.crba(m, s.q)) < 1e-12


@pytest.mark.parametrize("name", ["chain7", "humanoid", "tree_a"])
def test_aba_derivatives(models, name):
    m = models[name]
    s = gen.draw_states(m, B, 12)
    dq, dqd, dtau = dv.aba_derivatives(m, s.q, s.qd, s.tau)
    fq = _central(lambda d: rbd.aba(m, dv.retract(m, s.q, d), s.qd, s.tau), s.q, m.nv)
    fqd = _central(lambda d: rbd.aba(m, s.q, s.qd + d, s.tau), s.q, m.nv)
    assert normwise(dq, fq) < 1e-6
    assert normwise(dqd, fqd) < 1e-6
    M = rbd.crba(m, s.q)
    Minv = np.linalg.inv(M)
    assert normwise(dtau, Minv) < 1e-11
    qdd = rbd.aba(m, s.q, s.qd, s.tau)
    rq, rqd, _ = dv.rnea_derivatives(m, s.q, s.qd, qdd)
    assert normwise(dq, -Minv @ rq) < 1e-10
    assert normwise(dqd, -Minv @ rqd) < 1e-10


def test_vjp_ambient_mapping(models):
    """For any tangent direction d: q_bar . (d/de q (+) e d) = (gbar^T J) . d,
    so the ambient gradient is the tangent one pushed into q's layout."""
    m = models["humanoid"]
    s = gen.draw_states(m, B, 13)
    g = gen.draw_gbar(m.nv, B, 14)
    qbar, qdbar, qddbar = dv.rnea_vjp(m, s.q, s.qd, s.qdd, g)
    dq, dqd, dqdd = dv.rnea_derivatives(m, s.q, s.qd, s.qdd)
    d = np.random.default_rng(15).standard_normal((B, m.nv))
    dqamb = (dv.retract(m, s.q, FD_H * d) - dv.retract(m, s.q, -FD_H * d)) / (2 * FD_H)
    lhs = np.sum(qbar * dqamb, -1)
    rhs = np.einsum("bi,bij,bj->b", g, dq, d)
    assert np.max(np.abs(lhs - rhs) / np.abs(rhs)) < 1e-7
    quat = s.q[:, 3:7]
    assert np.max(np.abs(np.sum(qbar[:, 3:7] * quat, -1))) < 1e-12  # tangent to S^3
    assert normwise(qddbar, np.einsum("bi,bij->bj", g, rbd.crba(m, s.q))) < 1e-12
    assert normwise(qdbar, np.einsum("bi,bij->bj", g, dqd)) < 1e-14


def test_aba_vjp_matches_rnea_vjp_identity(models):
    """ABA VJP: tau_bar = M^-1 g, q_bar = -(dtau/dq)^T w, qd_bar =
    -(dtau/dqd)^T w with w = M^-1 g, evaluated at qdd = ABA(q, qd, tau)."""
    m = models["chain7"]
    s = gen.draw_states(m, B, 16)
    g = gen.draw_gbar(m.nv, B, 17)
    qbar, qdbar, taubar = dv.aba_vjp(m, s.q, s.qd, s.tau, g)
    M = rbd.crba(m, s.q)
    w = np.linalg.solve(M, g[..., None])[..., 0]
    qdd = rbd.aba(m, s.q, s.qd, s.tau)
    rq, rqd, _ = dv.rnea_vjp(m, s.q, s.qd, qdd, w)
    assert normwise(taubar, w) < 1e-11
    assert normwise(qbar, -rq) < 1e-10
    assert normwise(qdbar, -rqd) < 1e-10
