"""Pins of the FP64 oracle against invariants, a second formulation and
brute force, on the synthetic chain, humanoid and random trees."""

import numpy as np
import pytest

import gen
from oracle import mask_form, rbd
from oracle.derivatives import mass_matrix_rate
from tests import pins
from tests.pins import normwise

B = 12


def _states(model, seed=7):
    return gen.draw_states(model, B, seed)


@pytest.mark.parametrize("name", ["chain7", "humanoid", "tree_a", "tree_b"])
def test_recursive_equals_paper_vectorized_form(models, name):
    """RNEA == Algorithm 1 and CRBA == Algorithm 2 (mask form, root frame)."""
    m = models[name]
    s = _states(m)
    assert normwise(rbd.rnea(m, s.q, s.qd, s.qdd), mask_form.rnea_vectorized(m, s.q, s.qd, s.qdd)) < 1e-12
    assert normwise(rbd.crba(m, s.q), mask_form.crba_vectorized(m, s.q)) < 1e-12


@pytest.mark.parametrize("name", ["chain7", "humanoid", "tree_a"])
def test_mass_matrix_spd_and_rnea_columns(models, name):
    m = models[name]
    s = _states(m)
    M = rbd.crba(m, s.q)
    assert normwise(M, np.swapaxes(M, -1, -2)) < 1e-14
    assert np.linalg.eigvalsh(M).min() > 0
    zero = np.zeros_like(s.qd)
    cols = np.stack([rbd.rnea(m, s.q, zero, np.tile(np.eye(m.nv)[j], (B, 1)), gravity=False)
                     for j in range(m.nv)], -1)
    assert normwise(M, cols) < 1e-12
    # Eq. 1: tau = M qdd + (c + g)
    tau = rbd.rnea(m, s.q, s.qd, s.qdd)
    bias = rbd.rnea(m, s.q, s.qd, zero)
    assert normwise(tau, np.einsum("bij,bj->bi", M, s.qdd) + bias) < 1e-12


@pytest.mark.parametrize("name", ["chain7", "humanoid", "tree_a"])
def test_kinetic_energy(models, name):
    """qd^T M qd / 2 equals the bodies' kinetic energies from FK twists."""
    m = models[name]
    s = _states(m)
    M = rbd.crba(m, s.q)
    T = 0.5 * np.einsum("bi,bij,bj->b", s.qd, M, s.qd)
    assert np.max(np.abs(T - pins.kinetic_energy(m, s.q, s.qd)) / np.abs(T)) < 1e-12


@pytest.mark.parametrize("name", ["chain7", "tree_a", "tree_b"])
def test_lagrangian_brute_force(models, name):
    """tau from RNEA equals d/dt dL/dqd - dL/dq with L = T - V built from
    forward kinematics alone (fixed-base models)."""
    m = models[name]
    s = _states(m)
    assert normwise(rbd.rnea(m, s.q, s.qd, s.qdd), pins.lagrange_tau(m, s.q, s.qd, s.qdd)) < 1e-7


@pytest.mark.parametrize("name", ["chain7", "humanoid", "tree_a"])
def test_skew_property(models, name):
    """qd^T c(q, qd) = qd^T Mdot qd / 2 (gravity off)."""
    m = models[name]
    s = _states(m)
    c = rbd.rnea(m, s.q, s.qd, np.zeros_like(s.qd), gravity=False)
    lhs = np.sum(s.qd * c, -1)
    rhs = 0.5 * np.einsum("bi,bij,bj->b", s.qd, mass_matrix_rate(m, s.q, s.qd), s.qd)
    assert np.max(np.abs(lhs - rhs) / (np.abs(lhs) + 1e-9)) < 1e-11


@pytest.mark.parametrize("name", ["chain7", "humanoid", "tree_a", "tree_b"])
def test_forward_dynamics(models, name):
    """ABA: Eq. 2 == articulated-body recursion; RNEA(q, qd, ABA(q, qd, tau))
    = tau; power balance d/dt (T + V) = qd . tau along qdd = ABA."""
    m = models[name]
    s = _states(m)
    qdd = rbd.aba(m, s.q, s.qd, s.tau)
    assert normwise(rbd.aba_recursive(m, s.q, s.qd, s.tau), qdd) < 1e-11
    assert normwise(rbd.rnea(m, s.q, s.qd, qdd), s.tau) < 1e-12
    power = np.sum(s.qd * s.tau, -1)
    rate = pins.energy_rate(m, s.q, s.qd, qdd)
    assert np.max(np.abs(rate - power) / (np.abs(power) + 1.0)) < 1e-7


@pytest.mark.parametrize("name", ["chain7", "humanoid", "tree_a", "tree_b"])
def test_ltdl(models, name):
    """M = L^T D L, L unit lower with L_ij = 0 unless dof j belongs to an
    ancestor of dof i's body (no fill-in), D > 0, and the factor solves M."""
    m = models[name]
    s = _states(m)
    M = rbd.crba(m, s.q)
    L, D = rbd.ltdl(M)
    assert normwise(np.swapaxes(L, -1, -2) @ (D[..., None] * L), M) < 1e-13
    assert np.allclose(np.diagonal(L, axis1=-2, axis2=-1), 1.0)
    assert np.all(np.triu(L, 1) == 0)
    assert np.all(D > 0)
    lay = rbd.Layout(m)
    body = np.concatenate([[i] * lay.kv[i] for i in range(lay.n)])
    U = rbd.ancestor_mask(m)
    allowed = U[body[:, None], body[None, :]].astype(bool)
    assert np.max(np.abs(L[:, ~allowed])) < 1e-13 * np.max(np.abs(L))
    b = s.tau
    y = np.linalg.solve(np.swapaxes(L, -1, -2), b[..., None])[..., 0]
    x = np.linalg.solve(L, (y / D)[..., None])[..., 0]
    assert normwise(x, np.linalg.solve(M, b[..., None])[..., 0]) < 1e-11
    packed = rbd.pack_ltdl(L, D)
    assert packed.shape == (B, m.nv * (m.nv + 1) // 2)


@pytest.mark.parametrize("name", ["chain7", "humanoid", "tree_a"])
def test_jacobian_is_fk_derivative(models, name):
    """J qd = [omega (world); d/dt p_k] from complex-step FK twists; columns
    of non-ancestor joints are zero."""
    m = models[name]
    s = _states(m)
    frames = list(m.end_frames)
    J = rbd.jacobian(m, s.q, frames)
    tw = pins.twists(m, s.q, s.qd)
    R, _ = rbd.fk(m, s.q)
    for f, k in enumerate(frames):
        ref = np.concatenate([np.einsum("bij,bj->bi", R[:, k], tw[:, k, :3]),
                              np.einsum("bij,bj->bi", R[:, k], tw[:, k, 3:])], -1)
        assert normwise(np.einsum("bij,bj->bi", J[:, f], s.qd), ref) < 1e-12
        lay = rbd.Layout(m)
        anc = set(lay.ancestors(k))
        for j in range(lay.n):
            if j not in anc:
                assert np.all(J[:, f, :, lay.vslice(j)] == 0)


def test_ancestor_mask_lower_triangular(models):
    for m in models.values():
        U = rbd.ancestor_mask(m)
        assert np.all(np.triu(U, 1) == 0) and np.all(np.diag(U) == 1)
    U = rbd.ancestor_mask(models["humanoid"])
    assert U[22, 15] == 1 and U[22, 0] == 1 and U[22, 6] == 0 and U[29, 22] == 0


@pytest.mark.parametrize("name", ["chain7", "humanoid", "tree_a", "tree_b"])
def test_fk_rotations_are_proper(models, name):
    """Every body's world rotation is orthonormal with determinant +1."""
    m = models[name]
    R, _ = rbd.fk(m, _states(m).q)
    eye = np.broadcast_to(np.eye(3), R.shape)
    assert np.max(np.abs(np.swapaxes(R, -1, -2) @ R - eye)) < 1e-13
    assert np.max(np.abs(np.linalg.det(R) - 1.0)) < 1e-13


@pytest.mark.parametrize("name", ["chain7", "humanoid", "tree_a"])
def test_jacobian_central_differences(models, name):
    """Column j of J is the frame's motion along tangent direction e_j, by
    FP64 central differences of FK alone: the origin's displacement, and the
    rotation vector log(R(q (+) h e_j) R(q (-) h e_j)^T) / 2h."""
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    from oracle.derivatives import retract
    m = models[name]
    s = gen.draw_states(m, 3, 9)
    frames = list(m.end_frames)
    J = rbd.jacobian(m, s.q, frames)
    h = 1e-6
    for j in range(m.nv):
        e = np.zeros((3, m.nv))
        e[:, j] = h
        Rp, pp = rbd.fk(m, retract(m, s.q, e))
        Rm, pm = rbd.fk(m, retract(m, s.q, -e))
        for f, k in enumerate(frames):
            dR = Rp[:, k] @ np.swapaxes(Rm[:, k], -1, -2)
            w = Rot.from_matrix(dR).as_rotvec() / (2 * h)
            v = (pp[:, k] - pm[:, k]) / (2 * h)
            fd = np.concatenate([w, v], -1)
            assert np.max(np.abs(fd - J[:, f, :, j])) < 1e-7 * max(1.0, np.max(np.abs(J[:, f])))
