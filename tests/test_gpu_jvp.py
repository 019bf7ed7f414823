"""GPU forward-mode derivatives (frax_fk_jvp, frax_rnea_jvp, frax_aba_jvp) vs
the FP64 oracle's complex-step JVPs, and against the GPU's own VJPs by the
adjoint identity <gbar, J d> = <J^T gbar, d>. Tolerances: 1e-4 on values and
frame motions, 1e-3 on the dynamics' derivatives (as the VJPs)."""

import numpy as np
import pytest
import torch

import gen
import paper_2604_04310_gb300 as fx
from oracle import derivatives as dv
from oracle import rbd
from tests.gpu_util import dev, host, states
from tests.pins import normwise

pytestmark = pytest.mark.gpu

TOL = 1e-4
TOL_GRAD = 1e-3

MODELS = {
    "chain7": gen.chain7(0),
    "humanoid": gen.humanoid(0),
    "tree101": gen.random_tree(101),
    "tree_big": gen.random_tree(7, 64),
}


@pytest.fixture(scope="module")
def fxm():
    return {k: fx.Model.from_robot(m) for k, m in MODELS.items()}


def _dirs(model, B, seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((B, model.nv)).astype(np.float32).astype(np.float64) for _ in range(3)]


@pytest.mark.parametrize("name", list(MODELS))
def test_rnea_jvp(fxm, name):
    m, h = MODELS[name], fxm[name]
    B = 300
    s, d = states(m, B, 121)
    dq, dqd, dqdd = _dirs(m, B, 122)
    tau, dtau = fx.frax_rnea_jvp(h, d["q"], d["qd"], d["qdd"], dev(dq), dev(dqd), dev(dqdd), want_tau=True)
    assert normwise(host(tau), rbd.rnea(m, s.q, s.qd, s.qdd)) < TOL
    assert normwise(host(dtau), dv.rnea_jvp(m, s.q, s.qd, s.qdd, dq, dqd, dqdd)) < TOL_GRAD
    none, dtau0 = fx.frax_rnea_jvp(h, d["q"], d["qd"], d["qdd"], dev(dq), dev(dqd))
    assert none is None
    assert normwise(host(dtau0), dv.rnea_jvp(m, s.q, s.qd, s.qdd, dq, dqd, 0 * dqdd)) < TOL_GRAD


@pytest.mark.parametrize("name", list(MODELS))
def test_aba_jvp(fxm, name):
    m, h = MODELS[name], fxm[name]
    B = 300
    s, d = states(m, B, 123)
    dq, dqd, dtau = _dirs(m, B, 124)
    qdd = fx.frax_aba(h, d["q"], d["qd"], d["tau"])
    dqdd = fx.frax_aba_jvp(h, d["q"], d["qd"], d["tau"], qdd, dev(dq), dev(dqd), dev(dtau))
    assert normwise(host(dqdd), dv.aba_jvp(m, s.q, s.qd, s.tau, dq, dqd, dtau)) < TOL_GRAD
    dqdd0 = fx.frax_aba_jvp(h, d["q"], d["qd"], d["tau"], qdd, dev(dq), dev(dqd))
    assert normwise(host(dqdd0), dv.aba_jvp(m, s.q, s.qd, s.tau, dq, dqd, 0 * dtau)) < TOL_GRAD


@pytest.mark.parametrize("name", list(MODELS))
def test_fk_jvp(fxm, name):
    m, h = MODELS[name], fxm[name]
    B = 300
    s, d = states(m, B, 125)
    dq, _, _ = _dirs(m, B, 126)
    frames = list(m.end_frames)[:8]
    dp = fx.frax_fk_jvp(h, d["q"], dev(dq), frames)
    assert normwise(host(dp), dv.fk_jvp(m, s.q, dq, frames).reshape(B, -1)) < TOL
    _, J = fx.frax_jacobian(h, d["q"], frames)
    Jh = host(J).reshape(B, len(frames), 6, m.nv)
    assert normwise(host(dp), np.einsum("bfij,bj->bfi", Jh, dq).reshape(B, -1)) < TOL


@pytest.mark.parametrize("name", ["chain7", "tree101"])
def test_jvp_vjp_adjoint_identity(fxm, name):
    """Fixed-base models (tangent = ambient): <gbar, dtau(d)> equals
    <qbar, dq> + <qdbar, dqd> + <qddbar, dqdd> from the GPU's own VJP."""
    m, h = MODELS[name], fxm[name]
    B = 256
    s, d = states(m, B, 127)
    dq, dqd, dqdd = _dirs(m, B, 128)
    g = np.random.default_rng(129).standard_normal((B, m.nv))
    _, dtau = fx.frax_rnea_jvp(h, d["q"], d["qd"], d["qdd"], dev(dq), dev(dqd), dev(dqdd))
    qb, qdb, qddb = fx.frax_rnea_vjp(h, d["q"], d["qd"], d["qdd"], dev(g))
    lhs = np.einsum("bi,bi->b", g, host(dtau))
    rhs = sum(np.einsum("bi,bi->b", host(x), y) for x, y in ((qb, dq), (qdb, dqd), (qddb, dqdd)))
    scale = np.abs(g).sum(1) * np.abs(host(dtau)).max(1)
    assert np.max(np.abs(lhs - rhs) / scale) < 1e-4


@pytest.mark.parametrize("B", [1, 127, 129])
def test_jvp_batch_edges_and_ld(fxm, B):
    m, h = MODELS["humanoid"], fxm["humanoid"]
    ld = B + 11
    s, d = states(m, B, 130, ld=ld)
    dq, dqd, dx = _dirs(m, B, 131)
    _, dtau = fx.frax_rnea_jvp(h, d["q"], d["qd"], d["qdd"], dev(dq, ld), dev(dqd, ld), dev(dx, ld))
    assert dtau.stride(0) == ld
    assert normwise(host(dtau), dv.rnea_jvp(m, s.q, s.qd, s.qdd, dq, dqd, dx)) < TOL_GRAD
    dp = fx.frax_fk_jvp(h, d["q"], dev(dq, ld), [6, 29])
    assert normwise(host(dp), dv.fk_jvp(m, s.q, dq, [6, 29]).reshape(B, -1)) < TOL


def test_jvp_full_size_sampled(fxm):
    """2^18 humanoid instances per launch; 64 sampled against the oracle."""
    m, h = MODELS["humanoid"], fxm["humanoid"]
    B = 1 << 18
    s = gen.draw_states(m, B, 132).as_f32()
    dq, dqd, dx = _dirs(m, B, 133)
    q, qd, qdd, tau = dev(s.q), dev(s.qd), dev(s.qdd), dev(s.tau)
    _, dtau = fx.frax_rnea_jvp(h, q, qd, qdd, dev(dq), dev(dqd), dev(dx))
    a = fx.frax_aba(h, q, qd, tau)
    da = fx.frax_aba_jvp(h, q, qd, tau, a, dev(dq), dev(dqd), dev(dx))
    idx = np.random.default_rng(134).choice(B, 64, replace=False)
    ss = s.take(idx)
    assert normwise(host(dtau[:, idx]), dv.rnea_jvp(m, ss.q, ss.qd, ss.qdd, dq[idx], dqd[idx], dx[idx])) < TOL_GRAD
    assert normwise(host(da[:, idx]), dv.aba_jvp(m, ss.q, ss.qd, ss.tau, dq[idx], dqd[idx], dx[idx])) < TOL_GRAD


def test_jvp_empty_and_errors(fxm):
    h = fxm["chain7"]
    e = lambda k: torch.empty((k, 0), device="cuda")
    _, dt = fx.frax_rnea_jvp(h, e(7), e(7), e(7), e(7), e(7))
    assert dt.shape == (7, 0)
    s, d = states(MODELS["chain7"], 4, 135)
    with pytest.raises(fx.FraxError, match="frame body"):
        fx.frax_fk_jvp(h, d["q"], d["qd"], [9])
