"""GPU operational-space controller (frax_osc) vs the FP64 oracle.

The controller solves with Lambda^-1 = J M^-1 J^T, so its FP32 error scales
with the condition number kappa of that 6x6 matrix, which random joint
configurations push up to 1e7 on the 64-body tree. The bound per instance is
the first-order one of a linear solve: relative error <= 1e-5 + kappa u,
u = 2^-24 (an FP32 rounding), on tau and on Lambda, both relative to the
instance's largest entry."""

import numpy as np
import pytest
import torch

import gen
import paper_2604_04310_gb300 as fx
from oracle import rbd, task_space
from tests.gpu_util import dev, host, states

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24

MODELS = {
    "chain7": gen.chain7(0),
    "humanoid": gen.humanoid(0),
    "tree_big": gen.random_tree(7, 64),
}
TASKS = [("chain7", 6), ("chain7", 5), ("humanoid", 6), ("humanoid", 12), ("humanoid", 22), ("humanoid", 29), ("humanoid", 0),
         ("tree_big", 34)]


@pytest.fixture(scope="module")
def fxm():
    return {k: fx.Model.from_robot(m) for k, m in MODELS.items()}


def _xdd(B, seed):
    return np.random.default_rng(seed).uniform(-3, 3, (B, 6)).astype(np.float32).astype(np.float64)


def _per_instance(a, r):
    B = a.shape[0]
    return np.max(np.abs(a - r).reshape(B, -1), 1) / np.max(np.abs(r).reshape(B, -1), 1)


def _check(m, task, s, xdd, tau, Lam):
    rt, rL = task_space.osc(m, s.q, s.qd, task, xdd)
    bound = 1e-5 + np.linalg.cond(rL) * U32
    assert np.all(_per_instance(tau, rt) <= bound)
    assert np.all(_per_instance(Lam.reshape(-1, 6, 6), rL) <= bound)


@pytest.mark.parametrize("name,task", TASKS)
def test_osc_matches_oracle(fxm, name, task):
    m, h = MODELS[name], fxm[name]
    B = 300
    s, d = states(m, B, 61)
    xdd = _xdd(B, 62)
    tau, Lam = fx.frax_osc(h, task, d["q"], d["qd"], dev(xdd), want_lambda=True)
    _check(m, task, s, xdd, host(tau), host(Lam))
    tau2, none = fx.frax_osc(h, task, d["q"], d["qd"], dev(xdd))
    assert none is None and torch.equal(tau, tau2)


@pytest.mark.parametrize("name,task", [("chain7", 6), ("humanoid", 29)])
def test_osc_closed_loop_on_gpu(fxm, name, task):
    """The GPU's own ABA under the GPU controller's tau reaches the task
    acceleration: J qdd + Jdot qd = xdd_des (J from frax_jacobian; Jdot qd
    from the oracle)."""
    m, h = MODELS[name], fxm[name]
    B = 257
    s, d = states(m, B, 63)
    xdd = _xdd(B, 64)
    tau, _ = fx.frax_osc(h, task, d["q"], d["qd"], dev(xdd))
    qdd = fx.frax_aba(h, d["q"], d["qd"], tau)
    _, J = fx.frax_jacobian(h, d["q"], [task])
    Jh = host(J).reshape(B, 6, m.nv)
    got = np.einsum("bij,bj->bi", Jh, host(qdd)) + task_space.jdot_qd(m, s.q, s.qd, task)
    rL = task_space.osc(m, s.q, s.qd, task, xdd)[1]
    err = np.max(np.abs(got - xdd), 1) / np.max(np.abs(xdd), 1)
    assert np.all(err <= 1e-4 + np.linalg.cond(rL) * 8 * U32)


@pytest.mark.parametrize("B", [1, 127, 128, 129])
def test_osc_batch_edges_and_ld(fxm, B):
    m, h = MODELS["humanoid"], fxm["humanoid"]
    ld = B + 37
    s, d = states(m, B, 65, ld=ld)
    xdd = _xdd(B, 66)
    tau, Lam = fx.frax_osc(h, 22, d["q"], d["qd"], dev(xdd, ld), want_lambda=True)
    assert tau.stride(0) == ld
    _check(m, 22, s, xdd, host(tau), host(Lam))


def test_osc_full_size_sampled(fxm):
    """2^18 humanoid instances in one launch; 64 sampled against the oracle."""
    m, h = MODELS["humanoid"], fxm["humanoid"]
    B = 1 << 18
    s = gen.draw_states(m, B, 67).as_f32()
    xdd = _xdd(B, 68)
    tau, Lam = fx.frax_osc(h, 29, dev(s.q), dev(s.qd), dev(xdd), want_lambda=True)
    idx = np.random.default_rng(69).choice(B, 64, replace=False)
    _check(m, 29, s.take(idx), xdd[idx], host(tau[:, idx]), host(Lam[:, idx]))


def test_osc_empty_and_errors(fxm):
    h = fxm["humanoid"]
    q = torch.empty((h.nq, 0), device="cuda")
    qd = torch.empty((h.nv, 0), device="cuda")
    tau, _ = fx.frax_osc(h, 6, q, qd, torch.empty((6, 0), device="cuda"))
    assert tau.shape == (h.nv, 0)
    tree = fx.Model.from_robot(gen.random_tree(101))
    s, d = states(gen.random_tree(101), 8, 70)
    with pytest.raises(fx.FraxError, match="fewer than 6 dofs"):
        fx.frax_osc(tree, 13, d["q"], d["qd"], dev(_xdd(8, 71)))
