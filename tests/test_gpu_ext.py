"""GPU inverse and forward dynamics with external forces (frax_rnea_ext,
frax_aba_ext) vs the FP64 oracle. Forces are standard normal on every body
(root-frame Pluecker), plus a case with point forces at the humanoid's feet
only. Tolerances as the force-free kernels: 1e-4 on tau and on the chain's
qdd, 1e-3 on trees' qdd."""

import numpy as np
import pytest
import torch

import gen
import paper_2604_04310_gb300 as fx
from oracle import rbd
from tests.gpu_util import dev, host, states
from tests.pins import normwise

pytestmark = pytest.mark.gpu

TOL = 1e-4
TOL_ABA_TREE = 1e-3

MODELS = {
    "chain7": gen.chain7(0),
    "humanoid": gen.humanoid(0),
    "tree101": gen.random_tree(101),
    "tree_big": gen.random_tree(7, 64),
}


@pytest.fixture(scope="module")
def fxm():
    return {k: fx.Model.from_robot(m) for k, m in MODELS.items()}


def _forces(model, B, seed):
    F = np.random.default_rng(seed).standard_normal((B, model.n_bodies, 6))
    return F.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("name", list(MODELS))
def test_rnea_aba_with_forces(fxm, name):
    m, h = MODELS[name], fxm[name]
    B = 300
    s, d = states(m, B, 91)
    F = _forces(m, B, 92)
    Fd = dev(F.reshape(B, -1))
    tau = fx.frax_rnea_ext(h, d["q"], d["qd"], d["qdd"], Fd)
    assert normwise(host(tau), rbd.rnea(m, s.q, s.qd, s.qdd, fext=F)) < TOL
    bias = fx.frax_rnea_ext(h, d["q"], d["qd"], None, Fd)
    assert normwise(host(bias), rbd.rnea(m, s.q, s.qd, np.zeros_like(s.qd), fext=F)) < TOL
    qdd = fx.frax_aba_ext(h, d["q"], d["qd"], d["tau"], Fd)
    tol = TOL if name == "chain7" else TOL_ABA_TREE
    assert normwise(host(qdd), rbd.aba(m, s.q, s.qd, s.tau, fext=F)) < tol


@pytest.mark.parametrize("name", ["chain7", "humanoid"])
def test_zero_forces_match_force_free_kernels(fxm, name):
    m, h = MODELS[name], fxm[name]
    B = 200
    s, d = states(m, B, 93)
    Z = torch.zeros((6 * m.n_bodies, B), device="cuda")
    t0 = fx.frax_rnea(h, d["q"], d["qd"], d["qdd"])
    t1 = fx.frax_rnea_ext(h, d["q"], d["qd"], d["qdd"], Z)
    assert normwise(host(t1), host(t0)) < 1e-6
    # frax_aba_ext always runs one thread per instance; at this batch frax_aba
    # would pick the lane groups, whose sums over a body's children run in
    # another order, so the comparison pins frax_aba to the same path
    h.set_tree_path("thread")
    try:
        a0 = fx.frax_aba(h, d["q"], d["qd"], d["tau"])
    finally:
        h.set_tree_path("auto")
    a1 = fx.frax_aba_ext(h, d["q"], d["qd"], d["tau"], Z)
    assert normwise(host(a1), host(a0)) < 1e-6


def test_contact_forces_at_the_feet(fxm):
    """Point forces at the soles of the humanoid's feet (3 cm below each
    foot's origin, in the foot frame) as [c x f; f]; all other rows zero."""
    m, h = MODELS["humanoid"], fxm["humanoid"]
    B = 257
    s, d = states(m, B, 94)
    R, p = rbd.fk(m, s.q)
    F = np.zeros((B, m.n_bodies, 6))
    rng = np.random.default_rng(95)
    for foot in (6, 12):
        c = p[:, foot] + np.einsum("bij,j->bi", R[:, foot], [0.0, 0.0, -0.03])
        f = rng.uniform(-50, 50, (B, 3)) + [0, 0, 300]
        F[:, foot] = np.concatenate([np.cross(c, f), f], -1)
    F = F.astype(np.float32).astype(np.float64)
    Fd = dev(F.reshape(B, -1))
    tau = fx.frax_rnea_ext(h, d["q"], d["qd"], d["qdd"], Fd)
    assert normwise(host(tau), rbd.rnea(m, s.q, s.qd, s.qdd, fext=F)) < TOL
    qdd = fx.frax_aba_ext(h, d["q"], d["qd"], d["tau"], Fd)
    assert normwise(host(qdd), rbd.aba(m, s.q, s.qd, s.tau, fext=F)) < TOL_ABA_TREE


@pytest.mark.parametrize("B", [1, 129])
def test_batch_edges_and_ld(fxm, B):
    m, h = MODELS["humanoid"], fxm["humanoid"]
    ld = B + 19
    s, d = states(m, B, 96, ld=ld)
    F = _forces(m, B, 97)
    Fd = dev(F.reshape(B, -1), ld)
    tau = fx.frax_rnea_ext(h, d["q"], d["qd"], d["qdd"], Fd)
    qdd = fx.frax_aba_ext(h, d["q"], d["qd"], d["tau"], Fd)
    assert tau.stride(0) == ld and qdd.stride(0) == ld
    assert normwise(host(tau), rbd.rnea(m, s.q, s.qd, s.qdd, fext=F)) < TOL
    assert normwise(host(qdd), rbd.aba(m, s.q, s.qd, s.tau, fext=F)) < TOL_ABA_TREE


def test_full_size_sampled(fxm):
    """2^18 humanoid instances in one launch each; 64 sampled."""
    m, h = MODELS["humanoid"], fxm["humanoid"]
    B = 1 << 18
    s = gen.draw_states(m, B, 98).as_f32()
    F = _forces(m, B, 99)
    q, qd, qdd, tau, Fd = dev(s.q), dev(s.qd), dev(s.qdd), dev(s.tau), dev(F.reshape(B, -1))
    t = fx.frax_rnea_ext(h, q, qd, qdd, Fd)
    a = fx.frax_aba_ext(h, q, qd, tau, Fd)
    idx = np.random.default_rng(100).choice(B, 64, replace=False)
    ss = s.take(idx)
    assert normwise(host(t[:, idx]), rbd.rnea(m, ss.q, ss.qd, ss.qdd, fext=F[idx])) < TOL
    assert normwise(host(a[:, idx]), rbd.aba(m, ss.q, ss.qd, ss.tau, fext=F[idx])) < TOL_ABA_TREE


def test_empty_and_errors(fxm):
    h = fxm["chain7"]
    e = lambda k: torch.empty((k, 0), device="cuda")
    out = fx.frax_rnea_ext(h, e(7), e(7), e(7), e(42))
    assert out.shape == (7, 0)
    s, d = states(MODELS["chain7"], 4, 101)
    with pytest.raises(fx.FraxError, match="fext"):
        fx.frax_rnea_ext(h, d["q"], d["qd"], d["qdd"], torch.zeros((6, 4), device="cuda"))
