"""Task-space (operational-space) dynamics, FP64. Test infrastructure only.

The paper benchmarks an operational-space controller (OSC) built from M, J,
c and g (Sec. V, Table II). Written here as its plain definition:

  x_dd = J qdd + Jdot qd                 task acceleration of frame k
  Lambda = (J M^-1 J^T)^-1                operational-space inertia (6x6)
  tau = J^T Lambda (x_dd_des - Jdot qd) + c + g

without a null-space term. J is the world-aligned frame Jacobian of
rbd.jacobian, so x_dd = [omega_dot; p_dd] of the frame origin in world
coordinates.
"""

import numpy as np

from . import rbd
from .derivatives import H_STEP, retract


def jdot_qd(model, q, qd, frame):
    """Jdot qd: d/dt (J(q) qd) along q(t) with velocity qd and zero joint
    acceleration, by a complex step of J along qd. (B, 6)."""
    d = 1j * H_STEP * qd.astype(np.complex128)
    Jc = rbd.jacobian(model, retract(model, q, d), [frame])[:, 0]
    return np.imag(np.einsum("bij,bj->bi", Jc, qd.astype(np.complex128))) / H_STEP


def osc(model, q, qd, frame, xdd_des):
    """(tau (B, nv), Lambda (B, 6, 6)) of the operational-space controller."""
    M = rbd.crba(model, q)
    J = rbd.jacobian(model, q, [frame])[:, 0]
    bias = rbd.rnea(model, q, qd, np.zeros_like(qd))
    Minv_Jt = np.linalg.solve(M, np.swapaxes(J, -1, -2))
    Lam = np.linalg.inv(J @ Minv_Jt)
    rhs = xdd_des - jdot_qd(model, q, qd, frame)
    tau = np.einsum("bji,bj->bi", J, np.einsum("bij,bj->bi", Lam, rhs)) + bias
    return tau, Lam
