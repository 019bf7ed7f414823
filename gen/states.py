"""Seeded random joint states and the SoA layout the CUDA path uses.

States are FP64 arrays with the instance index first: q (B, nq), qd (B, nv),
qdd (B, nv), tau (B, nv). The kernels take FP32 structure-of-arrays,
``[entries][ld]`` with the instance index fastest; ``to_soa``/``from_soa``
convert.

Draw order (``default_rng(seed)``): revolute q U[-pi, pi], qd U[-2, 2],
qdd U[-5, 5], tau U[-5, 5] (each a (B, n_revolute) block); then, for a
free-flyer root, position U[-1, 1]^3, quaternion (x, y, z, w) from 4 normals
normalised (uniform on SO(3)), root velocity U[-1, 1]^6, root acceleration
U[-5, 5]^6 and root wrench U[-5, 5]^6.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .models import FREE, RobotModel


@dataclass
class States:
    q: np.ndarray
    qd: np.ndarray
    qdd: np.ndarray
    tau: np.ndarray

    @property
    def B(self) -> int:
        return int(self.q.shape[0])

    def as_f32(self) -> "States":
        """The same states rounded to FP32 and widened back to FP64, so an
        FP64 oracle sees exactly the inputs an FP32 kernel sees."""
        r = lambda x: x.astype(np.float32).astype(np.float64)
        return States(r(self.q), r(self.qd), r(self.qdd), r(self.tau))

    def take(self, idx) -> "States":
        return States(self.q[idx], self.qd[idx], self.qdd[idx], self.tau[idx])


def draw_states(model: RobotModel, B: int, seed: int) -> States:
    rng = np.random.default_rng(seed)
    free = model.has_free_root
    nr = model.n_bodies - (1 if free else 0)
    q_r = rng.uniform(-np.pi, np.pi, (B, nr))
    qd_r = rng.uniform(-2.0, 2.0, (B, nr))
    qdd_r = rng.uniform(-5.0, 5.0, (B, nr))
    tau_r = rng.uniform(-5.0, 5.0, (B, nr))
    if not free:
        return States(q_r, qd_r, qdd_r, tau_r)
    assert model.joint_type[0] == FREE
    pos = rng.uniform(-1.0, 1.0, (B, 3))
    quat = rng.standard_normal((B, 4))
    quat /= np.linalg.norm(quat, axis=1, keepdims=True)
    v0 = rng.uniform(-1.0, 1.0, (B, 6))
    a0 = rng.uniform(-5.0, 5.0, (B, 6))
    t0 = rng.uniform(-5.0, 5.0, (B, 6))
    return States(
        np.concatenate([pos, quat, q_r], axis=1),
        np.concatenate([v0, qd_r], axis=1),
        np.concatenate([a0, qdd_r], axis=1),
        np.concatenate([t0, tau_r], axis=1),
    )


def draw_gbar(nv: int, B: int, seed: int) -> np.ndarray:
    """Adjoint seeds for vector-Jacobian products: standard normals (B, nv)."""
    return np.random.default_rng(seed).standard_normal((B, nv))


def to_soa(x: np.ndarray, ld: int | None = None, dtype=np.float32) -> np.ndarray:
    """(B, k) instance-major -> (k, ld) entry-major, zero-padded to ld."""
    B, k = x.shape
    ld = B if ld is None else ld
    out = np.zeros((k, ld), dtype=dtype)
    out[:, :B] = x.T
    return out


def from_soa(x: np.ndarray, B: int) -> np.ndarray:
    """(k, ld) entry-major -> (B, k) FP64 instance-major."""
    return np.ascontiguousarray(np.asarray(x)[:, :B].T, dtype=np.float64)
