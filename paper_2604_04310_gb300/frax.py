"""Python binding of the C ABI: the same names as include/frax.h, argument
marshalling only. Every computation runs in libfrax's CUDA kernels; torch
supplies device memory and the current stream.

Batched tensors are FP32 CUDA tensors in the ABI's structure-of-arrays
layout: shape (entries, B) with stride (ld, 1), ld >= B, the same ld for
every tensor of one call. Outputs are allocated with torch on the inputs'
device unless passed in.
"""

from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib

OK = 0
STATUS = {0: "FRAX_OK", 1: "FRAX_EINVAL", 2: "FRAX_ECUDA", 3: "FRAX_ENOMEM", 4: "FRAX_ETIMEOUT",
          5: "FRAX_EBUSY", 6: "FRAX_EINTERNAL"}
JOINT_REVOLUTE, JOINT_FREE = 0, 1
MAX_FRAMES = 8


class FraxError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def lib():
    return _lib.load()


def _check(status):
    if status != OK:
        raise FraxError(status, lib().frax_last_error().decode())


def frax_version() -> str:
    return lib().frax_version().decode()


def frax_last_error() -> str:
    return lib().frax_last_error().decode()


class Model:
    """Owns a frax_model_t built by frax_model_create (host-only; the model
    reaches the GPU inside every launch)."""

    def __init__(self, parent, joint_type, axis, placement, inertia, gravity=(0.0, 0.0, -9.81), name="model"):
        self.name = name
        self.parent = np.ascontiguousarray(parent, dtype=np.int32)
        self.joint_type = np.ascontiguousarray(joint_type, dtype=np.int32)
        self.axis = np.ascontiguousarray(axis, dtype=np.float64).reshape(-1)
        self.placement = np.ascontiguousarray(placement, dtype=np.float64).reshape(-1)
        self.inertia = np.ascontiguousarray(inertia, dtype=np.float64).reshape(-1)
        self.gravity = np.ascontiguousarray(gravity, dtype=np.float64).reshape(-1)
        n = int(self.parent.shape[0])
        if (self.joint_type.shape[0] != n or self.axis.shape[0] != 3 * n or self.placement.shape[0] != 12 * n
                or self.inertia.shape[0] != 10 * n or self.gravity.shape[0] != 3):
            raise FraxError(1, "frax_model_create: array sizes do not match n_bodies")
        h = ctypes.c_void_p()
        L = lib()
        _check(L.frax_model_create(
            n, self.parent.ctypes.data_as(_lib.c_i32), self.joint_type.ctypes.data_as(_lib.c_i32),
            self.axis.ctypes.data_as(_lib.c_d), self.placement.ctypes.data_as(_lib.c_d),
            self.inertia.ctypes.data_as(_lib.c_d), self.gravity.ctypes.data_as(_lib.c_d), ctypes.byref(h)))
        self.handle = h
        nq, nv, nb, kind = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(L.frax_model_dims(h, ctypes.byref(nq), ctypes.byref(nv), ctypes.byref(nb)))
        _check(L.frax_model_kind(h, ctypes.byref(kind)))
        self.nq, self.nv, self.n_bodies, self.kind = nq.value, nv.value, nb.value, kind.value

    TREE_PATHS = {"auto": 0, "thread": 1, "lane_group": 2}

    def set_tree_path(self, path: str):
        """'auto' (default), 'thread' (one thread per instance) or
        'lane_group' (four lanes per instance) for trees of up to 32 bodies."""
        _check(lib().frax_model_set_tree_path(self.handle, self.TREE_PATHS[path]))

    @classmethod
    def from_robot(cls, robot):
        """From any object with parent, joint_type, axis, placement, inertia,
        gravity arrays (e.g. the seeded generators' RobotModel)."""
        return cls(robot.parent, robot.joint_type, robot.axis, robot.placement, robot.inertia, robot.gravity,
                   name=getattr(robot, "name", "model"))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                lib().frax_model_destroy(h)
            except Exception:
                pass
            self.handle = None


def frax_model_create(parent, joint_type, axis, placement, inertia, gravity=(0.0, 0.0, -9.81)) -> Model:
    return Model(parent, joint_type, axis, placement, inertia, gravity)


# ----------------------------------------------------------------- marshalling

_raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)


def _stream(t):
    """The current CUDA stream of t's device, as the ABI's void* (an int)."""
    if _raw_stream is not None:
        return _raw_stream(t.get_device())
    return torch.cuda.current_stream(t.device).cuda_stream


def _soa(t, rows, name, ld=None, B=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or t.dtype is not torch.float32 or not t.is_cuda:
        raise FraxError(1, f"{name} must be a float32 CUDA tensor")
    shape, stride = t.shape, t.stride()
    if len(shape) != 2 or shape[0] != rows or (rows > 0 and shape[1] > 1 and stride[1] != 1):
        raise FraxError(1, f"{name} must have shape ({rows}, B) with unit stride along B")
    if ld is not None and rows > 1 and shape[1] > 0 and stride[0] != ld:
        raise FraxError(1, f"{name}: every tensor of one call must share the same leading dimension")
    if B is not None and shape[1] != B:
        raise FraxError(1, f"{name}: batch size {shape[1]} != {B}")
    return t


def _ld(t):
    return t.stride(0) if t.shape[0] > 1 and t.shape[1] > 0 else t.shape[1]


def _out(rows, like, ld, B):
    if ld == B:
        return torch.empty((rows, B), dtype=torch.float32, device=like.device)
    return torch.empty((rows, ld), dtype=torch.float32, device=like.device)[:, :B]


def _p(t):
    return t.data_ptr() if t is not None else None


def _prep(model, q, **others):
    _soa(q, model.nq, "q")
    B, ld = q.shape[1], _ld(q)
    for name, (t, rows) in others.items():
        _soa(t, rows, name, ld, B)
    return B, ld


# -------------------------------------------------------------------- the ABI

def frax_fk(model: Model, q, pose=None):
    """World pose of every body, (n_bodies*12, B): R row-major then p."""
    B, ld = _prep(model, q, pose=(pose, 12 * model.n_bodies))
    pose = _out(12 * model.n_bodies, q, ld, B) if pose is None else pose
    _check(lib().frax_fk(model.handle, B, ld, _p(q), _p(pose), _stream(q)))
    return pose


def frax_fk_scan(model: Model, q, pose=None):
    """frax_fk for serial chains by a warp-level prefix product over SE(3)."""
    B, ld = _prep(model, q, pose=(pose, 12 * model.n_bodies))
    pose = _out(12 * model.n_bodies, q, ld, B) if pose is None else pose
    _check(lib().frax_fk_scan(model.handle, B, ld, _p(q), _p(pose), _stream(q)))
    return pose


def frax_jacobian(model: Model, q, frames, pose=None, J=None, want_pose=False):
    """Frame Jacobians (n_frames*6*nv, B); returns (pose or None, J)."""
    frames = np.ascontiguousarray(frames, dtype=np.int32).reshape(-1)
    nf = int(frames.shape[0])
    B, ld = _prep(model, q, pose=(pose, 12 * model.n_bodies), J=(J, nf * 6 * model.nv))
    J = _out(nf * 6 * model.nv, q, ld, B) if J is None else J
    if pose is None and want_pose:
        pose = _out(12 * model.n_bodies, q, ld, B)
    _check(lib().frax_jacobian(model.handle, B, ld, _p(q), nf, frames.ctypes.data_as(_lib.c_i32), _p(pose),
                               _p(J), _stream(q)))
    return pose, J


def frax_rnea(model: Model, q, qd, qdd=None, tau=None):
    """tau = M qdd + c + g (Eq. 1); qdd=None gives the bias forces c + g."""
    B, ld = _prep(model, q, qd=(qd, model.nv), qdd=(qdd, model.nv), tau=(tau, model.nv))
    tau = _out(model.nv, q, ld, B) if tau is None else tau
    _check(lib().frax_rnea(model.handle, B, ld, _p(q), _p(qd), _p(qdd), _p(tau), _stream(q)))
    return tau


def frax_crba(model: Model, q, M=None, LD=None, want_M=True, want_LD=False):
    """Mass matrix (nv*nv, B) and/or packed L^T D L factor (nv(nv+1)/2, B)."""
    nv = model.nv
    B, ld = _prep(model, q, M=(M, nv * nv), LD=(LD, nv * (nv + 1) // 2))
    if M is None and want_M:
        M = _out(nv * nv, q, ld, B)
    if LD is None and want_LD:
        LD = _out(nv * (nv + 1) // 2, q, ld, B)
    _check(lib().frax_crba(model.handle, B, ld, _p(q), _p(M), _p(LD), _stream(q)))
    return M, LD


def frax_aba(model: Model, q, qd, tau, qdd=None):
    """qdd = M^-1 (tau - c - g) (Eq. 2): the articulated-body algorithm on
    trees, a solve through the mass-matrix factor on 7-body chains."""
    B, ld = _prep(model, q, qd=(qd, model.nv), tau=(tau, model.nv), qdd=(qdd, model.nv))
    qdd = _out(model.nv, q, ld, B) if qdd is None else qdd
    _check(lib().frax_aba(model.handle, B, ld, _p(q), _p(qd), _p(tau), _p(qdd), _stream(q)))
    return qdd


def frax_aba_articulated(model: Model, q, qd, tau, qdd=None):
    """qdd (Eq. 2) always by the O(n) articulated-body sweeps (for 7-body
    chains frax_aba solves through the mass-matrix factor instead)."""
    B, ld = _prep(model, q, qd=(qd, model.nv), tau=(tau, model.nv), qdd=(qdd, model.nv))
    qdd = _out(model.nv, q, ld, B) if qdd is None else qdd
    _check(lib().frax_aba_articulated(model.handle, B, ld, _p(q), _p(qd), _p(tau), _p(qdd), _stream(q)))
    return qdd


def frax_rnea_ext(model: Model, q, qd, qdd, fext, tau=None):
    """tau = M qdd + c + g - sum_i J_i^T F_ext,i; fext (6*n_bodies, B) holds
    each body's external spatial force in root-frame Pluecker coordinates
    [moment about the root origin; force]; qdd=None means zero."""
    B, ld = _prep(model, q, qd=(qd, model.nv), qdd=(qdd, model.nv), fext=(fext, 6 * model.n_bodies),
                  tau=(tau, model.nv))
    tau = _out(model.nv, q, ld, B) if tau is None else tau
    _check(lib().frax_rnea_ext(model.handle, B, ld, _p(q), _p(qd), _p(qdd), _p(fext), _p(tau), _stream(q)))
    return tau


def frax_aba_ext(model: Model, q, qd, tau, fext, qdd=None):
    """qdd = M^-1 (tau - c - g + sum_i J_i^T F_ext,i), fext as frax_rnea_ext."""
    B, ld = _prep(model, q, qd=(qd, model.nv), tau=(tau, model.nv), fext=(fext, 6 * model.n_bodies),
                  qdd=(qdd, model.nv))
    qdd = _out(model.nv, q, ld, B) if qdd is None else qdd
    _check(lib().frax_aba_ext(model.handle, B, ld, _p(q), _p(qd), _p(tau), _p(fext), _p(qdd), _stream(q)))
    return qdd


def frax_fk_jvp(model: Model, q, dq, frames, dpose=None):
    """Motion [omega; p_dot] (world) of each frame along the tangent dq:
    (n_frames*6, B)."""
    frames = np.ascontiguousarray(frames, dtype=np.int32).reshape(-1)
    nf = int(frames.shape[0])
    B, ld = _prep(model, q, dq=(dq, model.nv), dpose=(dpose, 6 * nf))
    dpose = _out(6 * nf, q, ld, B) if dpose is None else dpose
    _check(lib().frax_fk_jvp(model.handle, B, ld, _p(q), _p(dq), nf, frames.ctypes.data_as(_lib.c_i32), _p(dpose),
                             _stream(q)))
    return dpose


def frax_rnea_jvp(model: Model, q, qd, qdd, dq, dqd, dqdd=None, tau=None, dtau=None, want_tau=False):
    """(tau or None, dtau): RNEA and its derivative along the tangent
    direction (dq, dqd, dqdd); qdd/dqdd None mean zero."""
    nv = model.nv
    B, ld = _prep(model, q, qd=(qd, nv), qdd=(qdd, nv), dq=(dq, nv), dqd=(dqd, nv), dqdd=(dqdd, nv),
                  tau=(tau, nv), dtau=(dtau, nv))
    dtau = _out(nv, q, ld, B) if dtau is None else dtau
    if tau is None and want_tau:
        tau = _out(nv, q, ld, B)
    _check(lib().frax_rnea_jvp(model.handle, B, ld, _p(q), _p(qd), _p(qdd), _p(dq), _p(dqd), _p(dqdd), _p(tau),
                               _p(dtau), _stream(q)))
    return tau, dtau


def frax_aba_jvp(model: Model, q, qd, tau, qdd, dq, dqd, dtau=None, dqdd=None):
    """Derivative of qdd = ABA(q, qd, tau) along (dq, dqd, dtau), at the
    saved forward result qdd; dtau None means zero."""
    nv = model.nv
    B, ld = _prep(model, q, qd=(qd, nv), tau=(tau, nv), qdd=(qdd, nv), dq=(dq, nv), dqd=(dqd, nv),
                  dtau=(dtau, nv), dqdd=(dqdd, nv))
    dqdd = _out(nv, q, ld, B) if dqdd is None else dqdd
    _check(lib().frax_aba_jvp(model.handle, B, ld, _p(q), _p(qd), _p(tau), _p(qdd), _p(dq), _p(dqd), _p(dtau),
                              _p(dqdd), _stream(q)))
    return dqdd


def frax_rnea_vjp(model: Model, q, qd, qdd, gbar, qbar=None, qdbar=None, qddbar=None, want_qddbar=True):
    """(dtau/dq)^T gbar [ambient, nq], (dtau/dqd)^T gbar, M gbar."""
    nv = model.nv
    B, ld = _prep(model, q, qd=(qd, nv), qdd=(qdd, nv), gbar=(gbar, nv), qbar=(qbar, model.nq),
                  qdbar=(qdbar, nv), qddbar=(qddbar, nv))
    qbar = _out(model.nq, q, ld, B) if qbar is None else qbar
    qdbar = _out(nv, q, ld, B) if qdbar is None else qdbar
    if qddbar is None and want_qddbar:
        qddbar = _out(nv, q, ld, B)
    _check(lib().frax_rnea_vjp(model.handle, B, ld, _p(q), _p(qd), _p(qdd), _p(gbar), _p(qbar), _p(qdbar),
                               _p(qddbar), _stream(q)))
    return qbar, qdbar, qddbar


def frax_aba_vjp(model: Model, q, qd, tau, qdd, gbar, qbar=None, qdbar=None, taubar=None, want_taubar=True):
    """VJP of Eq. 2 at qdd = ABA(q, qd, tau): (qbar [nq], qdbar, taubar = M^-1 gbar);
    with want_taubar False and no taubar buffer, taubar is not written (None)."""
    nv = model.nv
    B, ld = _prep(model, q, qd=(qd, nv), tau=(tau, nv), qdd=(qdd, nv), gbar=(gbar, nv),
                  qbar=(qbar, model.nq), qdbar=(qdbar, nv), taubar=(taubar, nv))
    qbar = _out(model.nq, q, ld, B) if qbar is None else qbar
    qdbar = _out(nv, q, ld, B) if qdbar is None else qdbar
    if taubar is None and want_taubar:
        taubar = _out(nv, q, ld, B)
    _check(lib().frax_aba_vjp(model.handle, B, ld, _p(q), _p(qd), _p(tau), _p(qdd), _p(gbar), _p(qbar),
                              _p(qdbar), _p(taubar), _stream(q)))
    return qbar, qdbar, taubar


def frax_ltdl_solve(model: Model, LD, b, x=None):
    """x = M^-1 b from the packed factor frax_crba returns (want_LD=True)."""
    nv = model.nv
    _soa(LD, nv * (nv + 1) // 2, "LD")
    B, ld = LD.shape[1], _ld(LD)
    _soa(b, nv, "b", ld, B)
    _soa(x, nv, "x", ld, B)
    x = _out(nv, LD, ld, B) if x is None else x
    _check(lib().frax_ltdl_solve(model.handle, B, ld, _p(LD), _p(b), _p(x), _stream(LD)))
    return x


def frax_ltdl_inverse(model: Model, LD, Minv=None):
    """M^-1 (nv*nv, B) from the packed factor."""
    nv = model.nv
    _soa(LD, nv * (nv + 1) // 2, "LD")
    B, ld = LD.shape[1], _ld(LD)
    _soa(Minv, nv * nv, "Minv", ld, B)
    Minv = _out(nv * nv, LD, ld, B) if Minv is None else Minv
    _check(lib().frax_ltdl_inverse(model.handle, B, ld, _p(LD), _p(Minv), _stream(LD)))
    return Minv


def frax_osc(model: Model, task_body: int, q, qd, xdd_des, tau=None, Lam=None, want_lambda=False):
    """Operational-space control of one task body: returns (tau (nv, B),
    Lambda (36, B) row-major world-aligned, or None)."""
    B, ld = _prep(model, q, qd=(qd, model.nv), xdd_des=(xdd_des, 6), tau=(tau, model.nv), Lam=(Lam, 36))
    tau = _out(model.nv, q, ld, B) if tau is None else tau
    if Lam is None and want_lambda:
        Lam = _out(36, q, ld, B)
    _check(lib().frax_osc(model.handle, int(task_body), B, ld, _p(q), _p(qd), _p(xdd_des), _p(tau), _p(Lam),
                          _stream(q)))
    return tau, Lam


# ------------------------------------------------------- allocation-free batch

class BatchRequest(ctypes.Structure):
    """frax_batch_request_t"""
    _fields_ = [("model", ctypes.c_void_p), ("op", ctypes.c_int), ("B", ctypes.c_int64),
                ("inputs", ctypes.c_void_p * 4), ("outputs", ctypes.c_void_p * 3)]


NOALLOC_OPS = {"rnea": 0, "crba": 1, "aba": 2, "rnea_grad": 3}


def frax_serve_batch_noalloc(requests):
    """Evaluates a mixed batch in one launch without allocating: each request
    is (model, op, inputs, outputs) with CUDA float32 tensors of shape
    (rows, B), ld = B, supplied by the caller (outputs included)."""
    n = len(requests)
    arr = (BatchRequest * max(1, n))()
    stream = None
    for i, (model, op, inputs, outputs) in enumerate(requests):
        r = arr[i]
        r.model = model.handle.value
        r.op = NOALLOC_OPS[op]
        B = inputs[0].shape[1]
        r.B = B
        for k, t in enumerate(list(inputs) + list(outputs)):
            if t.dtype != torch.float32 or not t.is_cuda or t.dim() != 2 or t.shape[1] != B or (
                    B > 1 and t.stride(1) != 1) or (t.shape[0] > 1 and B > 0 and t.stride(0) != B):
                raise FraxError(1, "frax_serve_batch_noalloc: tensors must be contiguous float32 CUDA (rows, B)")
        for k, t in enumerate(inputs):
            r.inputs[k] = t.data_ptr()
        for k, t in enumerate(outputs):
            r.outputs[k] = t.data_ptr()
        stream = stream or _stream(inputs[0])
    _check(lib().frax_serve_batch_noalloc(ctypes.cast(arr, ctypes.c_void_p), n,
                                          stream if stream is not None else ctypes.c_void_p(0)))


def frax_fp32_probe(packed: bool, blocks: int, iters: int, sink) -> float:
    """Launches the FP32 peak probe (independent FMA chains; packed = the
    two-lane form) on sink's stream; returns the FP32 operations it performs."""
    if sink.dtype != torch.float32 or not sink.is_cuda or sink.numel() < blocks * 256:
        raise FraxError(1, "frax_fp32_probe: sink must be a CUDA float32 tensor of blocks * 256 elements")
    flops = ctypes.c_double()
    _check(lib().frax_fp32_probe(int(bool(packed)), int(blocks), int(iters), ctypes.c_void_p(sink.data_ptr()),
                                 ctypes.byref(flops), _stream(sink)))
    return flops.value


# ------------------------------------------------------------- autograd wrappers

class RneaFn(torch.autograd.Function):
    """tau = RNEA(q, qd, qdd) with the hand-written adjoint as backward.
    Saves only q, qd, qdd; the backward recomputes the sweeps."""

    @staticmethod
    def forward(ctx, model, q, qd, qdd):
        ctx.model = model
        ctx.save_for_backward(q, qd, qdd)
        return frax_rnea(model, q, qd, qdd)

    @staticmethod
    def backward(ctx, gtau):
        q, qd, qdd = ctx.saved_tensors
        qbar, qdbar, qddbar = frax_rnea_vjp(ctx.model, q, qd, qdd, gtau.contiguous())
        return None, qbar, qdbar, qddbar


class AbaFn(torch.autograd.Function):
    """qdd = ABA(q, qd, tau) with the hand-written adjoint as backward.
    Saves q, qd, tau and qdd only (no per-body state)."""

    @staticmethod
    def forward(ctx, model, q, qd, tau):
        qdd = frax_aba(model, q, qd, tau)
        ctx.model = model
        ctx.save_for_backward(q, qd, tau, qdd)
        return qdd

    @staticmethod
    def backward(ctx, g):
        q, qd, tau, qdd = ctx.saved_tensors
        qbar, qdbar, taubar = frax_aba_vjp(ctx.model, q, qd, tau, qdd, g.contiguous())
        return None, qbar, qdbar, taubar


def rnea(model, q, qd, qdd):
    return RneaFn.apply(model, q, qd, qdd)


def aba(model, q, qd, tau):
    return AbaFn.apply(model, q, qd, tau)
