"""Batched arrays whose rows lie gigabytes apart.

The ABI allows a leading dimension up to 2^30; the kernels address entry k of
an instance as k * ld * 4 bytes past its first entry. With rows 1 GB (chain)
and 256 MB (humanoid) apart, the later entries sit beyond 4 GB of their array's
start, so these calls only match the FP64 oracle if every row offset keeps its
64-bit result. Each call is checked on the one-thread and the lane-group paths
of the tree."""

import numpy as np
import pytest
import torch

import gen
import paper_2604_04310_gb300 as fx
from oracle import rbd
from tests.gpu_util import host
from tests.pins import normwise

pytestmark = pytest.mark.gpu

CASES = [("chain7", gen.chain7(0), (1 << 28) + 16, 1e-4), ("humanoid", gen.humanoid(0), (1 << 26) + 16, 1e-3)]


@pytest.mark.parametrize("name,robot,ld,tol", CASES, ids=[c[0] for c in CASES])
def test_rows_gigabytes_apart(name, robot, ld, tol):
    B = 33
    rows = [robot.nq, robot.nv, robot.nv, robot.nv, robot.nv]  # q, qd, tau, qdd, tau again
    need = sum(rows) * ld * 4
    free, _ = torch.cuda.mem_get_info()
    if free < need + (2 << 30):
        pytest.skip(f"needs {need / 2**30:.0f} GiB of free device memory")
    m = fx.Model.from_robot(robot)
    s = gen.draw_states(robot, B, 61).as_f32()

    def put(x):  # (B, k) -> a (k, B) view with row stride ld; only the first B columns are written
        t = torch.empty((x.shape[1], ld), dtype=torch.float32, device="cuda")
        t[:, :B].copy_(torch.from_numpy(np.ascontiguousarray(x.T, dtype=np.float32)))
        return t[:, :B]

    def empty(k):
        return torch.empty((k, ld), dtype=torch.float32, device="cuda")[:, :B]

    q, qd, tau = put(s.q), put(s.qd), put(s.tau)
    qdd, tau2 = empty(robot.nv), empty(robot.nv)
    ref = rbd.aba(robot, s.q, s.qd, s.tau)
    try:
        for path in ("thread", "auto"):
            m.set_tree_path(path)
            fx.frax_aba(m, q, qd, tau, qdd=qdd)
            fx.frax_rnea(m, q, qd, qdd, tau=tau2)
            torch.cuda.synchronize()
            got = host(qdd)
            assert normwise(got, ref) < tol, path
            # RNEA at the computed accelerations gives back tau (Eq. 1 and Eq. 2 are inverses)
            assert normwise(host(tau2), rbd.rnea(robot, s.q, s.qd, got)) < 1e-4, path
    finally:
        del q, qd, tau, qdd, tau2
        torch.cuda.empty_cache()
