"""The pins of the oracle's composite functions catch plausible mistakes.

Each case plants one mistake on the CPU (by replacing one function of the
oracle for the duration of the test) and runs the pin tests that are meant
to guard that function; at least one of them must then fail. The mistakes
are those a restatement of the algorithms could plausibly contain: CRBA with
a force or composite inertia not carried to the parent's frame, or without
the mirrored upper triangle; the L^T D L factor taken without the index
reversal or with D unsquared; the packed factor read across the diagonal;
Eq. 2 with the wrong bias; Jacobian columns left in the joint frame or not
shifted to the frame origin; the free-flyer cotangent map without its factor
2; J-dot q-dot dropped; Lambda left uninverted; the ancestor mask used
transposed in the mask form; a free-flyer retraction that moves the root in
world instead of body coordinates; JVPs that drop one direction or take the
frame's angular rate from the transposed product. The unmutated copies of CRBA, the
Jacobian and the retraction written here agree with the oracle's own to
rounding, so each case differs from the oracle by its one planted mistake."""

import numpy as np
import pytest

import gen
from oracle import derivatives as dv
from oracle import mask_form, rbd, task_space
from oracle.spatial import matvec, motion_transform_inverse, quat_exp, quat_multiply, quat_to_rotation, skew
from tests import pins as pin_helpers
from tests import test_oracle_derivatives as pins_der
from tests import test_oracle_invariants as pins_inv
from tests import test_oracle_jvp as pins_jvp
from tests import test_oracle_task_space as pins_ts
from tests.pins import normwise


@pytest.fixture(scope="module")
def models():
    return {"chain7": gen.chain7(0), "humanoid": gen.humanoid(0), "tree_a": gen.random_tree(101),
            "tree_b": gen.random_tree(117)}


# ------------------------------------------------------------------ a pin of the packed layout

def packed_factor_reproduces_m(models, name):
    """The packed factor, read back by the index rule the ABI documents
    (entry (i, j <= i) at i(i+1)/2 + j: D_i on the diagonal, L_ij below),
    rebuilds M as L^T D L."""
    m = models[name]
    s = gen.draw_states(m, 6, 21)
    M = rbd.crba(m, s.q)
    P = rbd.pack_ltdl(*rbd.ltdl(M))
    n = m.nv
    L = np.zeros_like(M)
    D = np.zeros(M.shape[:2])
    for i in range(n):
        D[:, i] = P[:, i * (i + 1) // 2 + i]
        L[:, i, i] = 1.0
        for j in range(i):
            L[:, i, j] = P[:, i * (i + 1) // 2 + j]
    assert normwise(np.swapaxes(L, -1, -2) @ (D[..., None] * L), M) < 1e-12


def test_packed_factor_pin_holds(models):
    for name in models:
        packed_factor_reproduces_m(models, name)


# ------------------------------------------------------------------ mutated copies

def _crba_copy(force_to_parent=True, composite_to_parent=True):
    """rbd.crba restated, with one step switchable off."""
    def crba(model, q):
        lay = rbd.Layout(model)
        B = q.shape[0]
        X = rbd.joint_transforms(model, q)
        Ic = [np.broadcast_to(rbd.body_inertia(model, i), (B, 6, 6)).astype(q.dtype) for i in range(lay.n)]
        for i in reversed(range(lay.n)):
            k = lay.parent[i]
            if k >= 0:
                Xt = np.swapaxes(X[i], -1, -2)
                Ic[k] = Ic[k] + (Xt @ Ic[i] @ X[i] if composite_to_parent else Ic[i])
        H = np.zeros((B, lay.nv, lay.nv), q.dtype)
        for i in range(lay.n):
            Si = rbd.motion_subspace(model, i)
            F = Ic[i] @ Si
            H[:, lay.vslice(i), lay.vslice(i)] = Si.T @ F
            j = i
            while lay.parent[j] >= 0:
                if force_to_parent:
                    F = np.swapaxes(X[j], -1, -2) @ F
                j = lay.parent[j]
                blk = rbd.motion_subspace(model, j).T @ F
                H[:, lay.vslice(j), lay.vslice(i)] = blk
                H[:, lay.vslice(i), lay.vslice(j)] = np.swapaxes(blk, -1, -2)
        return H
    return crba


def _jacobian_copy(to_world=True, shift_to_frame=True):
    """rbd.jacobian restated, with one step switchable off."""
    def jacobian(model, q, frames):
        lay = rbd.Layout(model)
        R, p = rbd.fk(model, q)
        B = q.shape[0]
        out = np.zeros((B, len(frames), 6, lay.nv), dtype=q.dtype)
        for f, k in enumerate(frames):
            shift = np.broadcast_to(np.eye(6), (B, 6, 6)).astype(q.dtype).copy()
            if shift_to_frame:
                shift[:, 3:, :3] = -skew(p[:, k])
            for j in lay.ancestors(k):
                S = rbd.motion_subspace(model, j)
                if to_world:
                    S0 = motion_transform_inverse(R[:, j], p[:, j]) @ S
                else:
                    S0 = np.broadcast_to(S, (B, 6, S.shape[1]))
                out[:, f, :, lay.vslice(j)] = shift @ S0
        return out
    return jacobian


def test_unmutated_copies_equal_the_oracle(models):
    for name, m in models.items():
        s = gen.draw_states(m, 4, 22)
        assert normwise(_crba_copy()(m, s.q), rbd.crba(m, s.q)) < 1e-14
        frames = list(m.end_frames) or [m.nv - 1]
        assert normwise(_jacobian_copy()(m, s.q, frames), rbd.jacobian(m, s.q, frames)) < 1e-14


_ltdl = rbd.ltdl
_crba = rbd.crba
_to_ambient = dv.to_ambient
_ancestor_mask = rbd.ancestor_mask


def _ltdl_no_reversal(M):
    C = np.linalg.cholesky(M)  # M = L D L^T with L lower: the wrong orientation
    d = np.diagonal(C, axis1=-2, axis2=-1)
    return C / d[..., None, :], d * d


def _ltdl_d_unsquared(M):
    L, D = _ltdl(M)
    return L, np.sqrt(D)


def _pack_across_diagonal(L, D):
    n = D.shape[-1]
    return np.stack([D[..., i] if i == j else L[..., j, i] for i in range(n) for j in range(i + 1)], -1)


def _aba_bias_without_gravity(model, q, qd, tau, fext=None):
    bias = rbd.rnea(model, q, qd, np.zeros_like(tau), gravity=False, fext=fext)
    return np.linalg.solve(_crba(model, q), (tau - bias)[..., None])[..., 0]


def _aba_bias_added(model, q, qd, tau, fext=None):
    bias = rbd.rnea(model, q, qd, np.zeros_like(tau), fext=fext)
    return np.linalg.solve(_crba(model, q), (tau + bias)[..., None])[..., 0]


def _to_ambient_without_factor_two(model, q, gt):
    out = _to_ambient(model, q, gt)
    lay = rbd.Layout(model)
    for i in range(lay.n):
        if lay.jtype[i] == rbd.FREE:
            qs = lay.qslice(i)
            out[:, qs.start + 3:qs.start + 7] *= 0.5
    return out


def _jdot_qd_dropped(model, q, qd, frame):
    return np.zeros((q.shape[0], 6))


def _osc_lambda_uninverted(model, q, qd, frame, xdd_des):
    M = rbd.crba(model, q)
    J = rbd.jacobian(model, q, [frame])[:, 0]
    bias = rbd.rnea(model, q, qd, np.zeros_like(qd))
    Lam = J @ np.linalg.solve(M, np.swapaxes(J, -1, -2))
    rhs = xdd_des - task_space.jdot_qd(model, q, qd, frame)
    return np.einsum("bji,bj->bi", J, np.einsum("bij,bj->bi", Lam, rhs)) + bias, Lam


def _mask_transposed(model):
    return _ancestor_mask(model).T


# (module, attribute, replacement, pins meant to guard it)
CRBA_PINS = [(pins_inv.test_mass_matrix_spd_and_rnea_columns, "chain7"),
             (pins_inv.test_mass_matrix_spd_and_rnea_columns, "humanoid"),
             (pins_inv.test_kinetic_energy, "humanoid"),
             (pins_inv.test_recursive_equals_paper_vectorized_form, "tree_a")]
LTDL_PINS = [(pins_inv.test_ltdl, "chain7"), (pins_inv.test_ltdl, "humanoid"),
             (packed_factor_reproduces_m, "humanoid")]
ABA_PINS = [(pins_inv.test_forward_dynamics, "chain7"), (pins_inv.test_forward_dynamics, "humanoid")]
JAC_PINS = [(pins_inv.test_jacobian_is_fk_derivative, "chain7"),
            (pins_inv.test_jacobian_is_fk_derivative, "humanoid")]
MUTATIONS = {
    "crba_force_not_carried": (rbd, "crba", _crba_copy(force_to_parent=False), CRBA_PINS),
    "crba_composite_not_carried": (rbd, "crba", _crba_copy(composite_to_parent=False), CRBA_PINS),
    "crba_not_mirrored": (rbd, "crba", lambda model, q: np.tril(_crba(model, q)), CRBA_PINS),
    "ltdl_no_index_reversal": (rbd, "ltdl", _ltdl_no_reversal, LTDL_PINS),
    "ltdl_d_unsquared": (rbd, "ltdl", _ltdl_d_unsquared, LTDL_PINS),
    "pack_across_diagonal": (rbd, "pack_ltdl", _pack_across_diagonal, LTDL_PINS),
    "aba_bias_without_gravity": (rbd, "aba", _aba_bias_without_gravity, ABA_PINS),
    "aba_bias_sign": (rbd, "aba", _aba_bias_added, ABA_PINS),
    "jacobian_joint_frame_columns": (rbd, "jacobian", _jacobian_copy(to_world=False), JAC_PINS),
    "jacobian_not_shifted": (rbd, "jacobian", _jacobian_copy(shift_to_frame=False), JAC_PINS),
    "ambient_quaternion_half": (dv, "to_ambient", _to_ambient_without_factor_two,
                                [(pins_der.test_vjp_ambient_mapping, None)]),
    "jdot_qd_dropped": (task_space, "jdot_qd", _jdot_qd_dropped,
                        [(pins_ts.test_jdot_qd_is_the_fk_second_derivative, "chain7"),
                         (pins_ts.test_osc_closed_loop_identity, "chain7")]),
    "osc_lambda_uninverted": (task_space, "osc", _osc_lambda_uninverted,
                              [(pins_ts.test_osc_closed_loop_identity, "chain7"),
                               (pins_ts.test_osc_closed_loop_identity, "humanoid")]),
    "mask_transposed": (mask_form, "ancestor_mask", _mask_transposed,
                        [(pins_inv.test_recursive_equals_paper_vectorized_form, "chain7"),
                         (pins_inv.test_recursive_equals_paper_vectorized_form, "humanoid")]),
}


def _fails(pin, models, name):
    try:
        pin(models) if name is None else pin(models, name)
    except (AssertionError, np.linalg.LinAlgError):
        return True
    return False


def test_pins_hold_unmutated(models):
    for _, _, _, pins in MUTATIONS.values():
        for pin, name in pins:
            assert not _fails(pin, models, name), (pin.__name__, name)


@pytest.mark.parametrize("case", list(MUTATIONS))
def test_planted_mistake_is_caught(monkeypatch, models, case):
    module, attr, fn, pins = MUTATIONS[case]
    monkeypatch.setattr(module, attr, fn)
    caught = [(pin.__name__, name) for pin, name in pins if _fails(pin, models, name)]
    assert caught, f"{case} passed every pin meant to guard it"


def _retract_copy(body_frame_translation=True, body_frame_rotation=True):
    """derivatives.retract restated: q (+) d moves a free root by
    T * Exp([dw; dv]); either half switchable to world coordinates."""
    def retract(model, q, d):
        lay = rbd.Layout(model)
        out = q.astype(np.result_type(q, d)).copy()
        for i in range(lay.n):
            qs, vs = lay.qslice(i), lay.vslice(i)
            if lay.jtype[i] == rbd.FREE:
                qi, di = q[:, qs], d[:, vs]
                dv_world = matvec(quat_to_rotation(qi[:, 3:7]), di[:, 3:6]) if body_frame_translation else di[:, 3:6]
                out[:, qs.start:qs.start + 3] = qi[:, 0:3] + dv_world
                turn = quat_exp(di[:, 0:3])
                out[:, qs.start + 3:qs.start + 7] = (quat_multiply(qi[:, 3:7], turn) if body_frame_rotation
                                                     else quat_multiply(turn, qi[:, 3:7]))
            else:
                out[:, qs] = q[:, qs] + d[:, vs]
        return out
    return retract


RETRACT_PINS = [(pins_inv.test_kinetic_energy, "humanoid"), (pins_inv.test_forward_dynamics, "humanoid"),
                (pins_der.test_vjp_ambient_mapping, None)]


def test_unmutated_retract_copy_equals_the_oracle(models):
    m = models["humanoid"]
    s = gen.draw_states(m, 4, 23)
    d = np.random.default_rng(24).standard_normal((4, m.nv))
    assert normwise(_retract_copy()(m, s.q, d), dv.retract(m, s.q, d)) < 1e-15


@pytest.mark.parametrize("case", ["translation_in_world", "rotation_in_world"])
def test_planted_retraction_mistake_is_caught(monkeypatch, models, case):
    """The retraction is the free-flyer convention that the pins' own curves
    (FK twists, energy along q (+) h qd) and the oracle's derivatives share,
    so the mistake is planted in all of them at once."""
    fn = _retract_copy(body_frame_translation=case != "translation_in_world",
                       body_frame_rotation=case != "rotation_in_world")
    for module in (dv, pin_helpers, task_space):
        monkeypatch.setattr(module, "retract", fn)
    caught = [(pin.__name__, name) for pin, name in RETRACT_PINS if _fails(pin, models, name)]
    assert caught, f"{case} passed every pin meant to guard it"


_rnea_jvp, _aba_jvp, _fk_jvp = dv.rnea_jvp, dv.aba_jvp, dv.fk_jvp


def _rnea_jvp_without_dqd(model, q, qd, qdd, dq, dqd, dqdd):
    return _rnea_jvp(model, q, qd, qdd, dq, np.zeros_like(dqd), dqdd)


def _aba_jvp_without_dq(model, q, qd, tau, dq, dqd, dtau):
    return _aba_jvp(model, q, qd, tau, np.zeros_like(dq), dqd, dtau)


def _fk_jvp_transposed_rate(model, q, dq, frames):
    """omega from vee(R^T dR) (the body-frame rate) instead of vee(dR R^T)."""
    h = dv.H_STEP
    Rc, pc = rbd.fk(model, dv.retract(model, q, 1j * h * dq.astype(np.complex128)))
    R, _ = rbd.fk(model, q)
    f = list(frames)
    W = np.swapaxes(R[:, f], -1, -2) @ (np.imag(Rc[:, f]) / h)
    w = np.stack([W[..., 2, 1], W[..., 0, 2], W[..., 1, 0]], -1)
    return np.concatenate([w, np.imag(pc[:, f]) / h], -1)


JVP_MUTATIONS = {
    "rnea_jvp_without_dqd": ("rnea_jvp", _rnea_jvp_without_dqd,
                             [(pins_jvp.test_rnea_aba_jvp_vs_central_differences, "chain7")]),
    "aba_jvp_without_dq": ("aba_jvp", _aba_jvp_without_dq,
                           [(pins_jvp.test_rnea_aba_jvp_vs_central_differences, "humanoid")]),
    "fk_jvp_body_frame_rate": ("fk_jvp", _fk_jvp_transposed_rate,
                               [(pins_jvp.test_fk_jvp_is_jacobian_times_direction, "chain7"),
                                (pins_jvp.test_fk_jvp_is_jacobian_times_direction, "humanoid")]),
}


def test_jvp_pins_hold_unmutated(models):
    for _, _, pins in JVP_MUTATIONS.values():
        for pin, name in pins:
            assert not _fails(pin, models, name), (pin.__name__, name)


@pytest.mark.parametrize("case", list(JVP_MUTATIONS))
def test_planted_jvp_mistake_is_caught(monkeypatch, models, case):
    attr, fn, pins = JVP_MUTATIONS[case]
    monkeypatch.setattr(dv, attr, fn)
    caught = [(pin.__name__, name) for pin, name in pins if _fails(pin, models, name)]
    assert caught, f"{case} passed every pin meant to guard it"
