"""GPU FP32 kernels vs the FP64 oracle, element by element, through the C ABI.

Error metric (per instance, per output array): ||x_gpu - x_ref||_inf /
max(||x_ref||_inf, 1e-12), max over instances. Tolerances: 1e-4 on poses,
Jacobians, tau, M and its factor; 1e-3 on forward dynamics of the humanoid and
on every gradient. Batch sizes span several 128-thread blocks with a ragged
tail; full-size batches are checked on sampled instances."""

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
TOL_ABA_TREE = 1e-3
TOL_GRAD = 1e-3

MODELS = {
    "chain7": gen.chain7(0),
    "humanoid": gen.humanoid(0),
    "tree101": gen.random_tree(101),
    "tree117": gen.random_tree(117),
    "tree_big": gen.random_tree(7, 64),
    "tree32": gen.random_tree(9, 32),
}


@pytest.fixture(scope="module")
def fxm():
    return {k: fx.Model.from_robot(m) for k, m in MODELS.items()}


def _aba_tol(name):
    return TOL if name == "chain7" else TOL_ABA_TREE


@pytest.mark.parametrize("name", list(MODELS))
@pytest.mark.parametrize("B", [300])
def test_fk_jacobian(fxm, name, B):
    m, h = MODELS[name], fxm[name]
    s, d = states(m, B, 21)
    frames = list(m.end_frames)[:8]
    pose, J = fx.frax_jacobian(h, d["q"], frames, want_pose=True)
    assert normwise(host(pose), rbd.fk_flat(m, s.q)) < TOL
    assert normwise(host(J), rbd.jacobian(m, s.q, frames).reshape(B, -1)) < TOL
    pose2 = fx.frax_fk(h, d["q"])
    assert torch.equal(pose, pose2)


@pytest.mark.parametrize("name", list(MODELS))
def test_rnea(fxm, name):
    m, h = MODELS[name], fxm[name]
    B = 300
    s, d = states(m, B, 22)
    tau = fx.frax_rnea(h, d["q"], d["qd"], d["qdd"])
    assert normwise(host(tau), rbd.rnea(m, s.q, s.qd, s.qdd)) < TOL
    bias = fx.frax_rnea(h, d["q"], d["qd"], None)
    assert normwise(host(bias), rbd.rnea(m, s.q, s.qd, np.zeros_like(s.qd))) < TOL


@pytest.mark.parametrize("name", list(MODELS))
def test_crba_ltdl(fxm, name):
    m, h = MODELS[name], fxm[name]
    B = 300
    s, d = states(m, B, 23)
    M, LD = fx.frax_crba(h, d["q"], want_M=True, want_LD=True)
    Mref = rbd.crba(m, s.q)
    assert normwise(host(M), Mref.reshape(B, -1)) < TOL
    L, D = rbd.ltdl(Mref)
    assert normwise(host(LD), rbd.pack_ltdl(L, D)) < TOL
    M_only, none = fx.frax_crba(h, d["q"], want_M=True, want_LD=False)
    assert none is None and torch.equal(M_only, M)
    _, LD_only = fx.frax_crba(h, d["q"], want_M=False, want_LD=True)
    assert torch.equal(LD_only, LD)


@pytest.mark.parametrize("name", list(MODELS))
def test_aba(fxm, name):
    m, h = MODELS[name], fxm[name]
    B = 300
    s, d = states(m, B, 24)
    qdd = fx.frax_aba(h, d["q"], d["qd"], d["tau"])
    assert normwise(host(qdd), rbd.aba(m, s.q, s.qd, s.tau)) < _aba_tol(name)


def test_chain7_config0_every_instance(fxm):
    """The 7-revolute chain from model seed 0 with its batch of 1024 states
    drawn from seed 1000 (q U[-pi, pi], qd U[-2, 2], qdd and tau U[-5, 5]):
    FK, RNEA, CRBA and ABA on the GPU in FP32 against the FP64 oracle, every
    instance and every element compared."""
    m, h = MODELS["chain7"], fxm["chain7"]
    B = 1024
    s, d = states(m, B, 1000)
    pose = fx.frax_fk(h, d["q"])
    tau = fx.frax_rnea(h, d["q"], d["qd"], d["qdd"])
    M, LD = fx.frax_crba(h, d["q"], want_M=True, want_LD=True)
    qdd = fx.frax_aba(h, d["q"], d["qd"], d["tau"])
    qdd_sweep = fx.frax_aba_articulated(h, d["q"], d["qd"], d["tau"])
    Mref = rbd.crba(m, s.q)
    assert normwise(host(pose), rbd.fk_flat(m, s.q)) < TOL
    assert normwise(host(tau), rbd.rnea(m, s.q, s.qd, s.qdd)) < TOL
    assert normwise(host(M), Mref.reshape(B, -1)) < TOL
    assert normwise(host(LD), rbd.pack_ltdl(*rbd.ltdl(Mref))) < TOL
    qref = rbd.aba(m, s.q, s.qd, s.tau)
    assert normwise(host(qdd), qref) < TOL
    assert normwise(host(qdd_sweep), qref) < TOL


@pytest.mark.parametrize("name", list(MODELS))
def test_aba_articulated(fxm, name):
    """frax_aba_articulated always runs the O(n) articulated-body sweeps (the
    7-body chain's frax_aba solves through the mass-matrix factor instead)."""
    m, h = MODELS[name], fxm[name]
    B = 300
    s, d = states(m, B, 32)
    qdd = fx.frax_aba_articulated(h, d["q"], d["qd"], d["tau"])
    assert normwise(host(qdd), rbd.aba(m, s.q, s.qd, s.tau)) < _aba_tol(name)


@pytest.mark.parametrize("name", ["chain7", "humanoid", "tree101", "tree_big"])
def test_rnea_vjp(fxm, name):
    m, h = MODELS[name], fxm[name]
    B = 160
    s, d = states(m, B, 25)
    g = gen.draw_gbar(m.nv, B, 26).astype(np.float32).astype(np.float64)
    qb, qdb, qddb = fx.frax_rnea_vjp(h, d["q"], d["qd"], d["qdd"], dev(g))
    rq, rqd, rqdd = dv.rnea_vjp(m, s.q, s.qd, s.qdd, g)
    assert normwise(host(qb), rq) < TOL_GRAD
    assert normwise(host(qdb), rqd) < TOL_GRAD
    assert normwise(host(qddb), rqdd) < TOL_GRAD


@pytest.mark.parametrize("name", ["chain7", "humanoid", "tree101", "tree_big"])
def test_aba_vjp(fxm, name):
    m, h = MODELS[name], fxm[name]
    B = 160
    s, d = states(m, B, 27)
    g = gen.draw_gbar(m.nv, B, 28).astype(np.float32).astype(np.float64)
    qdd = fx.frax_aba(h, d["q"], d["qd"], d["tau"])
    qb, qdb, tb = fx.frax_aba_vjp(h, d["q"], d["qd"], d["tau"], qdd, dev(g))
    rq, rqd, rt = dv.aba_vjp(m, s.q, s.qd, s.tau, g)
    assert normwise(host(qb), rq) < TOL_GRAD
    assert normwise(host(qdb), rqd) < TOL_GRAD
    assert normwise(host(tb), rt) < TOL_GRAD


@pytest.mark.parametrize("name", ["chain7", "humanoid"])
def test_vjp_vs_central_differences(fxm, name):
    """GPU VJPs against FP64 central differences (step 1e-6) of the oracle's
    RNEA and forward dynamics, contracted with the same seed."""
    m, h = MODELS[name], fxm[name]
    B = 8
    s, d = states(m, B, 29)
    g = gen.draw_gbar(m.nv, B, 30).astype(np.float32).astype(np.float64)
    hstep = 1e-6

    def central(fun, n):
        cols = []
        for k in range(n):
            e = np.zeros((B, n))
            e[:, k] = hstep
            cols.append((fun(e) - fun(-e)) / (2 * hstep))
        return np.stack(cols, -1)

    Jq = central(lambda e: rbd.rnea(m, dv.retract(m, s.q, e), s.qd, s.qdd), m.nv)
    Jqd = central(lambda e: rbd.rnea(m, s.q, s.qd + e, s.qdd), m.nv)
    qb, qdb, _ = fx.frax_rnea_vjp(h, d["q"], d["qd"], d["qdd"], dev(g))
    assert normwise(host(qb), dv.to_ambient(m, s.q, np.einsum("bi,bij->bj", g, Jq))) < TOL_GRAD
    assert normwise(host(qdb), np.einsum("bi,bij->bj", g, Jqd)) < TOL_GRAD
    Aq = central(lambda e: rbd.aba(m, dv.retract(m, s.q, e), s.qd, s.tau), m.nv)
    Aqd = central(lambda e: rbd.aba(m, s.q, s.qd + e, s.tau), m.nv)
    At = central(lambda e: rbd.aba(m, s.q, s.qd, s.tau + e), m.nv)
    qdd = fx.frax_aba(h, d["q"], d["qd"], d["tau"])
    qb, qdb, tb = fx.frax_aba_vjp(h, d["q"], d["qd"], d["tau"], qdd, dev(g))
    assert normwise(host(qb), dv.to_ambient(m, s.q, np.einsum("bi,bij->bj", g, Aq))) < TOL_GRAD
    assert normwise(host(qdb), np.einsum("bi,bij->bj", g, Aqd)) < TOL_GRAD
    assert normwise(host(tb), np.einsum("bi,bij->bj", g, At)) < TOL_GRAD


@pytest.mark.parametrize("B", [1, 31, 32, 33, 127, 128, 129, 257])
def test_edge_batch_sizes_and_padding(fxm, B):
    """Ragged batches, and ld > B: the padding columns are never written."""
    m, h = MODELS["chain7"], fxm["chain7"]
    ld = B + 13
    s = gen.draw_states(m, B, 31).as_f32()
    q, qd, qdd, tau = (dev(x, ld) for x in (s.q, s.qd, s.qdd, s.tau))
    out = torch.full((m.nv, ld), 7.0, device="cuda")
    fx.frax_rnea(h, q, qd, qdd, tau=out[:, :B])
    assert normwise(host(out[:, :B]), rbd.rnea(m, s.q, s.qd, s.qdd)) < TOL
    assert torch.all(out[:, B:] == 7.0)
    qddo = fx.frax_aba(h, q, qd, tau)
    assert normwise(host(qddo), rbd.aba(m, s.q, s.qd, s.tau)) < TOL


def test_empty_batch_is_noop(fxm):
    h = fxm["chain7"]
    z = torch.empty((7, 0), device="cuda")
    assert fx.frax_rnea(h, torch.empty((7, 0), device="cuda"), z, z).shape == (7, 0)
    e = dev(np.zeros((0, 7)))  # empty arrays made the way the other tests make inputs
    assert fx.frax_crba(h, e)[0].shape == (49, 0)
    assert fx.frax_aba(h, e, e, e).shape == (7, 0)


def test_argument_errors(fxm):
    h = fxm["chain7"]
    q = torch.zeros((7, 16), device="cuda")
    with pytest.raises(fx.FraxError):
        fx.frax_rnea(h, q, torch.zeros((6, 16), device="cuda"))
    with pytest.raises(fx.FraxError):
        fx.frax_rnea(h, q.double(), q)
    with pytest.raises(fx.FraxError):
        fx.frax_jacobian(h, q, [9])


@pytest.mark.parametrize("name,B", [("chain7", 1 << 20), ("humanoid", 1 << 18)])
def test_full_size_sampled(fxm, name, B):
    """The configurations the bench times, in its launch configuration: every
    op on the full batch, a random sample of instances checked against the
    oracle."""
    m, h = MODELS[name], fxm[name]
    s, d = states(m, B, 1000 + (1 if name == "chain7" else 2))
    idx = np.sort(np.random.default_rng(5).choice(B, 96, replace=False))
    idx[-1] = B - 1
    ss = s.take(idx)
    frames = list(m.end_frames)
    pose, J = fx.frax_jacobian(h, d["q"], frames, want_pose=True)
    tau = fx.frax_rnea(h, d["q"], d["qd"], d["qdd"])
    M, LD = fx.frax_crba(h, d["q"], want_LD=True)
    qdd = fx.frax_aba(h, d["q"], d["qd"], d["tau"])
    sel = torch.from_numpy(idx).cuda()
    pick = lambda t: host(t.index_select(1, sel))
    assert normwise(pick(pose), rbd.fk_flat(m, ss.q)) < TOL
    assert normwise(pick(J), rbd.jacobian(m, ss.q, frames).reshape(len(idx), -1)) < TOL
    assert normwise(pick(tau), rbd.rnea(m, ss.q, ss.qd, ss.qdd)) < TOL
    Mref = rbd.crba(m, ss.q)
    assert normwise(pick(M), Mref.reshape(len(idx), -1)) < TOL
    assert normwise(pick(LD), rbd.pack_ltdl(*rbd.ltdl(Mref))) < TOL
    assert normwise(pick(qdd), rbd.aba(m, ss.q, ss.qd, ss.tau)) < _aba_tol(name)
    g = gen.draw_gbar(m.nv, B, 77).astype(np.float32).astype(np.float64)
    gd = dev(g)
    qb, qdb, qddb = fx.frax_rnea_vjp(h, d["q"], d["qd"], d["qdd"], gd)
    rq, rqd, rqdd = dv.rnea_vjp(m, ss.q, ss.qd, ss.qdd, g[idx])
    assert normwise(pick(qb), rq) < TOL_GRAD and normwise(pick(qdb), rqd) < TOL_GRAD
    assert normwise(pick(qddb), rqdd) < TOL_GRAD
    aq, aqd, at = fx.frax_aba_vjp(h, d["q"], d["qd"], d["tau"], qdd, gd)
    rq, rqd, rt = dv.aba_vjp(m, ss.q, ss.qd, ss.tau, g[idx])
    assert normwise(pick(aq), rq) < TOL_GRAD and normwise(pick(aqd), rqd) < TOL_GRAD
    assert normwise(pick(at), rt) < TOL_GRAD


def test_autograd_functions(fxm):
    m, h = MODELS["humanoid"], fxm["humanoid"]
    B = 64
    s, d = states(m, B, 33)
    q, qd, qdd, tau = (d[k].clone().requires_grad_(True) for k in ("q", "qd", "qdd", "tau"))
    g = torch.randn((m.nv, B), device="cuda")
    out = fx.rnea(h, q, qd, qdd)
    gq, gqd, gqdd = torch.autograd.grad(out, (q, qd, qdd), g)
    rq, rqd, rqdd = fx.frax_rnea_vjp(h, d["q"], d["qd"], d["qdd"], g)
    assert torch.equal(gq, rq) and torch.equal(gqd, rqd) and torch.equal(gqdd, rqdd)
    a = fx.aba(h, q, qd, tau)
    gq, gqd, gt = torch.autograd.grad(a, (q, qd, tau), g)
    aq, aqd, at = fx.frax_aba_vjp(h, d["q"], d["qd"], d["tau"], a.detach(), g)
    assert torch.equal(gq, aq) and torch.equal(gqd, aqd) and torch.equal(gt, at)


@pytest.mark.parametrize("name", list(MODELS))
def test_ltdl_solve_and_inverse(fxm, name):
    """Solves with the factor frax_crba returns: x = M^-1 b, M^-1 itself, and
    M^-1 (tau - c - g) equal to the articulated-body forward dynamics."""
    m, h = MODELS[name], fxm[name]
    B = 300
    s, d = states(m, B, 41)
    _, LD = fx.frax_crba(h, d["q"], want_M=False, want_LD=True)
    Mref = rbd.crba(m, s.q)
    x = fx.frax_ltdl_solve(h, LD, d["tau"])
    assert normwise(host(x), np.linalg.solve(Mref, s.tau[..., None])[..., 0]) < TOL_ABA_TREE
    Minv = fx.frax_ltdl_inverse(h, LD)
    assert normwise(host(Minv), np.linalg.inv(Mref).reshape(B, -1)) < TOL_ABA_TREE
    bias = fx.frax_rnea(h, d["q"], d["qd"], None)
    qdd_solve = fx.frax_ltdl_solve(h, LD, d["tau"] - bias)
    qdd_aba = fx.frax_aba(h, d["q"], d["qd"], d["tau"])
    assert normwise(host(qdd_solve), host(qdd_aba)) < TOL_ABA_TREE


@pytest.mark.parametrize("name", ["humanoid", "tree_big"])
def test_structural_zeros_are_written(fxm, name):
    """Outputs pre-filled with NaN: every entry of J, M and the factor is
    written, the structural zeros (non-ancestor pairs, the same for every
    instance) included: the Jacobian's by the row fill, M's and the factor's
    by the CRBA kernel's own threads, for each of its three output variants."""
    m, h = MODELS[name], fxm[name]
    B = 300
    s, d = states(m, B, 27)
    frames = list(m.end_frames)[:8]
    nan = lambda rows: torch.full((rows, B), float("nan"), device="cuda")
    J = nan(len(frames) * 6 * m.nv)
    fx.frax_jacobian(h, d["q"], frames, J=J)
    assert normwise(host(J), rbd.jacobian(m, s.q, frames).reshape(B, -1)) < TOL
    M, LD = nan(m.nv * m.nv), nan(m.nv * (m.nv + 1) // 2)
    fx.frax_crba(h, d["q"], M=M, LD=LD)
    Mref = rbd.crba(m, s.q)
    assert normwise(host(M), Mref.reshape(B, -1)) < TOL
    assert normwise(host(LD), rbd.pack_ltdl(*rbd.ltdl(Mref))) < TOL
    LD2 = nan(m.nv * (m.nv + 1) // 2)
    fx.frax_crba(h, d["q"], LD=LD2, want_M=False)
    assert torch.equal(LD2, LD)
    M2 = nan(m.nv * m.nv)
    fx.frax_crba(h, d["q"], M=M2, want_LD=False)
    assert torch.equal(M2, M)


@pytest.mark.parametrize("name,B", [("chain7", 65536), ("humanoid", 16384)])
def test_autograd_full_batch_vs_central_differences(fxm, name, B):
    """The differentiation workload: RNEA and forward dynamics through the
    autograd functions on the whole batch (velocities recomputed inside the
    adjoint kernels, nothing stored per body), 12 sampled instances checked
    against FP64 central differences (step 1e-6) of the oracle."""
    m, h = MODELS[name], fxm[name]
    s, d = states(m, B, 1003)
    q, qd, qdd, tau = (d[k].clone().requires_grad_(True) for k in ("q", "qd", "qdd", "tau"))
    g = gen.draw_gbar(m.nv, B, 1004).astype(np.float32).astype(np.float64)
    gd = dev(g)
    rq, rqd, _ = torch.autograd.grad(fx.rnea(h, q, qd, qdd), (q, qd, qdd), gd)
    aq, aqd, at = torch.autograd.grad(fx.aba(h, q, qd, tau), (q, qd, tau), gd)
    idx = np.sort(np.random.default_rng(1005).choice(B, 12, replace=False))
    ss, gs = s.take(idx), g[idx]
    sel = torch.from_numpy(idx).cuda()
    pick = lambda t: host(t.index_select(1, sel))
    hstep = 1e-6

    def vjp_fd(fun, n):
        out = np.zeros((len(idx), n))
        for k in range(n):
            e = np.zeros((len(idx), n))
            e[:, k] = hstep
            out[:, k] = np.einsum("bi,bi->b", gs, (fun(e) - fun(-e)) / (2 * hstep))
        return out

    assert normwise(pick(rq), dv.to_ambient(m, ss.q, vjp_fd(
        lambda e: rbd.rnea(m, dv.retract(m, ss.q, e), ss.qd, ss.qdd), m.nv))) < TOL_GRAD
    assert normwise(pick(rqd), vjp_fd(lambda e: rbd.rnea(m, ss.q, ss.qd + e, ss.qdd), m.nv)) < TOL_GRAD
    assert normwise(pick(aq), dv.to_ambient(m, ss.q, vjp_fd(
        lambda e: rbd.aba(m, dv.retract(m, ss.q, e), ss.qd, ss.tau), m.nv))) < TOL_GRAD
    assert normwise(pick(aqd), vjp_fd(lambda e: rbd.aba(m, ss.q, ss.qd + e, ss.tau), m.nv)) < TOL_GRAD
    assert normwise(pick(at), vjp_fd(lambda e: rbd.aba(m, ss.q, ss.qd, ss.tau + e), m.nv)) < TOL_GRAD


def test_joint_angle_sin_cos_accuracy():
    """The kernels' joint sin/cos (reduction by 2 pi, then the SFU
    approximations) through FK of one revolute body about z: R = Rot_z(q), so
    R[0][0] = cos q and R[1][0] = sin q. Absolute error below 1e-6 for angles
    up to 1000 rad (sincosf's own error is below 2e-7 here)."""
    from tests.test_oracle_closed_forms import _model, EYE
    body = _model([-1], [0], [0, 0, 1], EYE + [0, 0, 0], [1.0, 0, 0, 0, 0.1, 0.1, 0.1, 0, 0, 0])
    h = fx.Model.from_robot(body)
    q = np.concatenate([np.linspace(-50, 50, 200001), np.linspace(-1000, 1000, 20001)]).astype(np.float32)
    pose = host(fx.frax_fk(h, torch.from_numpy(q[None, :]).cuda()))
    qd = q.astype(np.float64)
    assert np.max(np.abs(pose[:, 0] - np.cos(qd))) < 1e-6
    assert np.max(np.abs(pose[:, 3] - np.sin(qd))) < 1e-6


@pytest.mark.parametrize("name", ["humanoid", "tree_big"])
def test_crba_single_outputs_match_both(fxm, name):
    """M alone, the factor alone and both at once (three kernel variants on
    trees) give the same bits."""
    m, h = MODELS[name], fxm[name]
    s, d = states(m, 200, 43)
    M, LD = fx.frax_crba(h, d["q"], want_M=True, want_LD=True)
    M1, _ = fx.frax_crba(h, d["q"], want_M=True, want_LD=False)
    _, LD1 = fx.frax_crba(h, d["q"], want_M=False, want_LD=True)
    assert torch.equal(M, M1) and torch.equal(LD, LD1)



@pytest.mark.parametrize("name", ["chain7", "humanoid", "tree101"])
def test_aba_vjp_without_taubar_matches(fxm, name):
    """taubar NULL: the chain runs its one-launch adjoint (factor solve and
    sweep fused) instead of the two launches; trees skip the taubar stores.
    Same q and qd gradients either way."""
    m, h = MODELS[name], fxm[name]
    s, d = states(m, 300, 45)
    g = dev(gen.draw_gbar(m.nv, 300, 46))
    qdd = fx.frax_aba(h, d["q"], d["qd"], d["tau"])
    qb, qdb, tb = fx.frax_aba_vjp(h, d["q"], d["qd"], d["tau"], qdd, g)
    qb0, qdb0, tb0 = fx.frax_aba_vjp(h, d["q"], d["qd"], d["tau"], qdd, g, want_taubar=False)
    assert tb0 is None and tb is not None
    for x, y in ((qb, qb0), (qdb, qdb0)):
        xh, yh = host(x), host(y)
        assert np.max(np.abs(xh - yh)) <= 1e-5 * np.max(np.abs(xh))


@pytest.mark.parametrize("B", [1, 33, 129])
def test_chain_unrolled_kernels_edge_batches(fxm, B):
    """The chain's own kernels (unrolled adjoint, JVP and external-force
    sweeps, the factor-based solves) on ragged batches with ld > B: results
    match the oracle and the padding columns of every output stay untouched."""
    m, h = MODELS["chain7"], fxm["chain7"]
    ld = B + 13
    s, d = states(m, B, 47, ld=ld)
    rng = np.random.default_rng(48)
    draw = lambda rows: rng.standard_normal((B, rows)).astype(np.float32).astype(np.float64)
    g, dq, dqd, dx = draw(7), draw(7), draw(7), draw(7)
    F = draw(6 * 7)
    pad = lambda rows: torch.full((rows, ld), 7.0, device="cuda")
    outs = {k: pad(r) for k, r in (("qb", 7), ("qdb", 7), ("qddb", 7), ("aqb", 7), ("aqdb", 7), ("tb", 7),
                                     ("dt", 7), ("da", 7), ("dp", 6), ("te", 7), ("ae", 7))}
    v = lambda k: outs[k][:, :B]
    fx.frax_rnea_vjp(h, d["q"], d["qd"], d["qdd"], dev(g, ld), qbar=v("qb"), qdbar=v("qdb"), qddbar=v("qddb"))
    qdd = fx.frax_aba(h, d["q"], d["qd"], d["tau"])
    fx.frax_aba_vjp(h, d["q"], d["qd"], d["tau"], qdd, dev(g, ld), qbar=v("aqb"), qdbar=v("aqdb"), taubar=v("tb"))
    fx.frax_rnea_jvp(h, d["q"], d["qd"], d["qdd"], dev(dq, ld), dev(dqd, ld), dev(dx, ld), dtau=v("dt"))
    fx.frax_aba_jvp(h, d["q"], d["qd"], d["tau"], qdd, dev(dq, ld), dev(dqd, ld), dev(dx, ld), dqdd=v("da"))
    fx.frax_fk_jvp(h, d["q"], dev(dq, ld), [6], dpose=v("dp"))
    fx.frax_rnea_ext(h, d["q"], d["qd"], d["qdd"], dev(F, ld), tau=v("te"))
    fx.frax_aba_ext(h, d["q"], d["qd"], d["tau"], dev(F, ld), qdd=v("ae"))
    for k, t in outs.items():
        assert torch.all(t[:, B:] == 7.0), k
    qb, qdb, qddb = dv.rnea_vjp(m, s.q, s.qd, s.qdd, g)
    assert normwise(host(v("qb")), qb) < TOL_GRAD and normwise(host(v("qdb")), qdb) < TOL_GRAD
    assert normwise(host(v("qddb")), qddb) < TOL_GRAD
    aq, aqd, at = dv.aba_vjp(m, s.q, s.qd, s.tau, g)
    assert normwise(host(v("aqb")), aq) < TOL_GRAD and normwise(host(v("aqdb")), aqd) < TOL_GRAD
    assert normwise(host(v("tb")), at) < TOL_GRAD
    assert normwise(host(v("dt")), dv.rnea_jvp(m, s.q, s.qd, s.qdd, dq, dqd, dx)) < TOL_GRAD
    assert normwise(host(v("da")), dv.aba_jvp(m, s.q, s.qd, s.tau, dq, dqd, dx)) < TOL_GRAD
    assert normwise(host(v("dp")), dv.fk_jvp(m, s.q, dq, [6]).reshape(B, -1)) < TOL
    Fb = F.reshape(B, 7, 6)
    assert normwise(host(v("te")), rbd.rnea(m, s.q, s.qd, s.qdd, fext=Fb)) < TOL
    assert normwise(host(v("ae")), rbd.aba(m, s.q, s.qd, s.tau, fext=Fb)) < TOL


LG_MODELS = ["humanoid", "tree101", "tree117", "tree32"]


@pytest.mark.parametrize("name", LG_MODELS)
@pytest.mark.parametrize("B", [1, 15, 16, 17, 300])
def test_lane_group_paths(fxm, name, B):
    """Trees of up to 32 bodies: the lane-group kernels (four lanes per
    instance) against the oracle, forced on and off, on ragged batches
    (16 instances per block)."""
    m, h = MODELS[name], fxm[name]
    s, d = states(m, B, 33)
    try:
        h.set_tree_path("lane_group")
        tau = fx.frax_rnea(h, d["q"], d["qd"], d["qdd"])
        bias = fx.frax_rnea(h, d["q"], d["qd"], None)
        qdd = fx.frax_aba(h, d["q"], d["qd"], d["tau"])
        qdd2 = fx.frax_aba_articulated(h, d["q"], d["qd"], d["tau"])
        # CRBA into NaN-filled outputs: every entry, structural zeros included, is written
        Mn = torch.full((m.nv * m.nv, B), float("nan"), device="cuda")
        LDn = torch.full((m.nv * (m.nv + 1) // 2, B), float("nan"), device="cuda")
        fx.frax_crba(h, d["q"], M=Mn, LD=LDn)
        M_only, _ = fx.frax_crba(h, d["q"], want_M=True, want_LD=False)
        # FK and Jacobians into NaN-filled outputs (the structural zeros come from the row fill)
        frames = list(m.end_frames)[:8]
        pose_n = torch.full((12 * m.n_bodies, B), float("nan"), device="cuda")
        J_n = torch.full((len(frames) * 6 * m.nv, B), float("nan"), device="cuda")
        fx.frax_jacobian(h, d["q"], frames, pose=pose_n, J=J_n)
        pose_fk = fx.frax_fk(h, d["q"])
        h.set_tree_path("thread")
        tau_t = fx.frax_rnea(h, d["q"], d["qd"], d["qdd"])
        qdd_t = fx.frax_aba(h, d["q"], d["qd"], d["tau"])
    finally:
        h.set_tree_path("auto")
    assert normwise(host(tau), rbd.rnea(m, s.q, s.qd, s.qdd)) < TOL
    assert normwise(host(bias), rbd.rnea(m, s.q, s.qd, np.zeros_like(s.qd))) < TOL
    qref = rbd.aba(m, s.q, s.qd, s.tau)
    assert normwise(host(qdd), qref) < TOL_ABA_TREE
    assert torch.equal(qdd, qdd2)
    Mref = rbd.crba(m, s.q)
    assert not torch.isnan(Mn).any() and not torch.isnan(LDn).any()
    assert normwise(host(Mn), Mref.reshape(B, -1)) < TOL
    assert normwise(host(LDn), rbd.pack_ltdl(*rbd.ltdl(Mref))) < TOL
    assert torch.equal(M_only, Mn)
    assert not torch.isnan(pose_n).any() and not torch.isnan(J_n).any()
    assert normwise(host(pose_n), rbd.fk_flat(m, s.q)) < TOL
    assert normwise(host(J_n), rbd.jacobian(m, s.q, frames).reshape(B, -1)) < TOL
    assert torch.equal(pose_fk, pose_n)
    # the two paths agree to FP32 rounding of the branch sums
    assert normwise(host(tau), host(tau_t)) < 1e-5
    assert normwise(host(qdd), host(qdd_t)) < TOL_ABA_TREE


@pytest.mark.parametrize("name", LG_MODELS)
@pytest.mark.parametrize("B", [1, 17, 64])
def test_lane_group_adjoints(fxm, name, B):
    """The RNEA and ABA adjoints on the lane-group path against the oracle's
    complex-step VJPs and against the one-thread path."""
    m, h = MODELS[name], fxm[name]
    s, d = states(m, B, 35)
    g = gen.draw_gbar(m.nv, B, 36).astype(np.float32).astype(np.float64)
    gb = dev(g)
    try:
        h.set_tree_path("lane_group")
        qdd = fx.frax_aba(h, d["q"], d["qd"], d["tau"])
        r_lg = fx.frax_rnea_vjp(h, d["q"], d["qd"], d["qdd"], gb)
        a_lg = fx.frax_aba_vjp(h, d["q"], d["qd"], d["tau"], qdd, gb)
        h.set_tree_path("thread")
        r_t = fx.frax_rnea_vjp(h, d["q"], d["qd"], d["qdd"], gb)
        a_t = fx.frax_aba_vjp(h, d["q"], d["qd"], d["tau"], qdd, gb)
    finally:
        h.set_tree_path("auto")
    for x, ref in zip(r_lg, dv.rnea_vjp(m, s.q, s.qd, s.qdd, g)):
        assert normwise(host(x), ref) < TOL_GRAD
    for x, ref in zip(a_lg, dv.aba_vjp(m, s.q, s.qd, s.tau, g)):
        assert normwise(host(x), ref) < TOL_GRAD
    for x, y in zip(r_lg + a_lg, r_t + a_t):
        assert normwise(host(x), host(y)) < TOL_GRAD


def test_lane_group_auto_dispatch_and_padding(fxm):
    """The default path picks the lane groups while the batch fits one resident
    wave of the lane-group kernel (4096 here) and one thread per instance
    beyond (2^17 + 1); ld > B padding columns are never written."""
    m, h = MODELS["humanoid"], fxm["humanoid"]
    for B in (4096, (1 << 17) + 1):
        ld = B + 5
        s = gen.draw_states(m, B, 34).as_f32()
        q, qd, tau = (dev(x, ld) for x in (s.q, s.qd, s.tau))
        out = torch.full((m.nv, ld), 7.0, device="cuda")
        fx.frax_aba(h, q, qd, tau, qdd=out[:, :B])
        idx = np.arange(0, B, 97)
        assert normwise(host(out[:, :B])[idx], rbd.aba(m, s.q[idx], s.qd[idx], s.tau[idx])) < TOL_ABA_TREE
        assert torch.all(out[:, B:] == 7.0)
    assert fx.lib().frax_model_set_tree_path(h.handle, 7) == 1  # FRAX_EINVAL
