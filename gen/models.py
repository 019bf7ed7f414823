"""Seeded random kinematic trees.

A model is described by plain arrays, the same ones the C ABI's
``frax_model_create`` takes:

* ``parent``     (n,) int32   parent body index, -1 = world; parent[i] < i
* ``joint_type`` (n,) int32   0 = revolute, 1 = free-flyer (only body 0)
* ``axis``       (n, 3)       unit joint axis in the joint frame (revolute)
* ``placement``  (n, 12)      joint frame in the parent body frame:
                              R (3x3, row-major; joint->parent) then p (3)
* ``inertia``    (n, 10)      m, COM c (3, body frame), rotational inertia
                              about the COM (xx, yy, zz, xy, xz, yz)
* ``gravity``    (3,)         world gravity, e.g. (0, 0, -9.81)

Draw order (numpy PCG64 ``default_rng(seed)``), for each body in index order:
axis (3 normals, normalised); placement rotation (quaternion from 4 normals,
normalised); placement translation U[-0.2, 0.2]^3; mass U[m_lo, m_hi];
COM U[-0.1, 0.1]^3; 3 principal moments U[1e-3, 5e-2]; principal-axis
rotation (4 normals). A free-flyer root then has its placement reset to the
identity (the draws are still taken so the stream stays aligned).
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

REVOLUTE = 0
FREE = 1


@dataclass
class RobotModel:
    name: str
    parent: np.ndarray
    joint_type: np.ndarray
    axis: np.ndarray
    placement: np.ndarray
    inertia: np.ndarray
    gravity: np.ndarray = field(default_factory=lambda: np.array([0.0, 0.0, -9.81]))
    end_frames: tuple = ()

    @property
    def n_bodies(self) -> int:
        return int(self.parent.shape[0])

    @property
    def has_free_root(self) -> bool:
        return bool(self.joint_type[0] == FREE)

    @property
    def nq(self) -> int:
        return int(sum(7 if t == FREE else 1 for t in self.joint_type))

    @property
    def nv(self) -> int:
        return int(sum(6 if t == FREE else 1 for t in self.joint_type))


def _quat_to_matrix(qx, qy, qz, qw):
    # Input generation only: turns a random unit quaternion into a rotation
    # matrix for the drawn placements and principal axes.
    return np.array([
        [1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qz * qw), 2 * (qx * qz + qy * qw)],
        [2 * (qx * qy + qz * qw), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qx * qw)],
        [2 * (qx * qz - qy * qw), 2 * (qy * qz + qx * qw), 1 - 2 * (qx * qx + qy * qy)],
    ])


def _random_rotation(rng):
    v = rng.standard_normal(4)
    v /= np.linalg.norm(v)
    return _quat_to_matrix(*v)


def _draw_links(rng, n, mass_range):
    axis = np.zeros((n, 3))
    placement = np.zeros((n, 12))
    inertia = np.zeros((n, 10))
    for i in range(n):
        a = rng.standard_normal(3)
        axis[i] = a / np.linalg.norm(a)
        R = _random_rotation(rng)
        p = rng.uniform(-0.2, 0.2, 3)
        placement[i, :9] = R.reshape(-1)
        placement[i, 9:] = p
        m = rng.uniform(*mass_range)
        c = rng.uniform(-0.1, 0.1, 3)
        eig = rng.uniform(1e-3, 5e-2, 3)
        Q = _random_rotation(rng)
        Ic = Q @ np.diag(eig) @ Q.T
        inertia[i] = [m, c[0], c[1], c[2],
                      Ic[0, 0], Ic[1, 1], Ic[2, 2], Ic[0, 1], Ic[0, 2], Ic[1, 2]]
    return axis, placement, inertia


def chain7(seed: int = 0) -> RobotModel:
    """Fixed-base serial chain of 7 revolute joints (a Panda-shaped arm)."""
    rng = np.random.default_rng(seed)
    n = 7
    axis, placement, inertia = _draw_links(rng, n, (0.5, 4.0))
    parent = np.arange(-1, n - 1, dtype=np.int32)
    jt = np.zeros(n, dtype=np.int32)
    return RobotModel("chain7", parent, jt, axis, placement, inertia, end_frames=(6,))


# Humanoid body order (depth-first): root; left leg (6); right leg (6);
# waist (3); left arm (7) and right arm (7), both hanging off the waist end.
HUMANOID_PARENT = np.array(
    [-1]
    + [0, 1, 2, 3, 4, 5]
    + [0, 7, 8, 9, 10, 11]
    + [0, 13, 14]
    + [15, 16, 17, 18, 19, 20, 21]
    + [15, 23, 24, 25, 26, 27, 28],
    dtype=np.int32,
)
HUMANOID_END_FRAMES = (6, 12, 22, 29)  # left foot, right foot, left hand, right hand


def humanoid(seed: int = 0) -> RobotModel:
    """Free-flyer root + 29 revolute joints (a G1-shaped tree), 30 bodies."""
    rng = np.random.default_rng(seed)
    n = HUMANOID_PARENT.shape[0]
    axis, placement, inertia = _draw_links(rng, n, (0.3, 8.0))
    jt = np.zeros(n, dtype=np.int32)
    jt[0] = FREE
    placement[0, :9] = np.eye(3).reshape(-1)
    placement[0, 9:] = 0.0
    return RobotModel("humanoid", HUMANOID_PARENT.copy(), jt, axis, placement, inertia,
                      end_frames=HUMANOID_END_FRAMES)


def random_tree(seed: int, n: int | None = None) -> RobotModel:
    """Fixed-base tree of n revolute bodies; parent of 1-indexed body i drawn
    U{0..i-1} with 0 the fixed base (so -1 = world after 0-indexing)."""
    rng = np.random.default_rng(seed)
    if n is None:
        n = int(rng.integers(3, 65))
    drawn = np.array([rng.integers(0, i) for i in range(1, n + 1)], dtype=np.int32)
    parent = (drawn - 1).astype(np.int32)
    axis, placement, inertia = _draw_links(rng, n, (0.5, 4.0))
    jt = np.zeros(n, dtype=np.int32)
    children = np.zeros(n, dtype=bool)
    for p in parent:
        if p >= 0:
            children[p] = True
    leaves = tuple(int(i) for i in range(n) if not children[i])
    return RobotModel(f"tree{seed}_{n}", parent, jt, axis, placement, inertia, end_frames=leaves)


def serial_chain(seed: int, n: int, free_root: bool = False) -> RobotModel:
    """Serial chain of n bodies (parent of i is i - 1): n revolute joints, or
    a free-flyer root followed by n - 1 revolute joints."""
    rng = np.random.default_rng(seed)
    axis, placement, inertia = _draw_links(rng, n, (0.3, 4.0))
    parent = np.arange(-1, n - 1, dtype=np.int32)
    jt = np.zeros(n, dtype=np.int32)
    if free_root:
        jt[0] = FREE
        placement[0, :9] = np.eye(3).reshape(-1)
        placement[0, 9:] = 0.0
    return RobotModel(f"serial{n}{'f' if free_root else ''}_{seed}", parent, jt, axis, placement, inertia,
                      end_frames=(n - 1,))


def serving_pool(n_random: int = 32):
    """The models a serving stream draws from: chain, humanoid and random trees
    (seeds 100..100+n_random-1, 3-64 bodies)."""
    return [chain7(0), humanoid(0)] + [random_tree(100 + k) for k in range(n_random)]
