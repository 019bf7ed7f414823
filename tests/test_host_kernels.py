"""The kernels' device functions compiled as host code (tests/host_kernels.cpp,
g++, no GPU) against the FP64 oracle: FK and Jacobians, RNEA, CRBA + LTDL,
ABA, both adjoints, the JVPs and the external-force variants, for the 7-DoF
chain (through the chain's own unrolled code, as the CUDA dispatch runs it),
the floating-base humanoid and a fixed-base random tree. The same tolerances
as the GPU parity tests."""

import os
import shutil
import subprocess

import numpy as np
import pytest

import gen
from oracle import derivatives as dv
from oracle import rbd, task_space
from tests.pins import normwise

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TOL = 1e-4
TOL_TREE = 1e-3  # tree ABA and every derivative
CUDA_INCLUDE = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")

MODELS = {"chain7": gen.chain7(0), "humanoid": gen.humanoid(0), "tree101": gen.random_tree(101),
          "tree117": gen.random_tree(117), "star": gen.random_tree(3, 12),
          # degenerate trees: one revolute body, one free body, a free body with one child
          "one": gen.serial_chain(11, 1), "free1": gen.serial_chain(12, 1, free_root=True),
          "free2": gen.serial_chain(13, 2, free_root=True)}


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.isdir(CUDA_INCLUDE):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("hk") / "host_kernels")
    r = subprocess.run(["g++", "-std=c++17", "-O1", "-x", "c++", f"-I{CUDA_INCLUDE}", f"-I{ROOT}",
                        os.path.join(ROOT, "tests", "host_kernels.cpp"), "-x", "none",
                        os.path.join(ROOT, "paper_2604_04310_gb300", "csrc", "model.cpp"), "-o", exe],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return exe


def _run(exe, tmp_path, m, s, frames, extra):
    B = s.q.shape[0]
    f32 = lambda x: gen.to_soa(x).astype(np.float32)
    with open(tmp_path / "in.bin", "wb") as f:
        np.array([m.n_bodies, B, len(frames)], np.int32).tofile(f)
        np.asarray(m.parent, np.int32).tofile(f)
        np.asarray(m.joint_type, np.int32).tofile(f)
        for a in (m.axis, m.placement, m.inertia, m.gravity):
            np.asarray(a, np.float64).tofile(f)
        np.asarray(frames, np.int32).tofile(f)
        for a in (s.q, s.qd, s.qdd, s.tau, extra["g"], extra["dq"], extra["dqd"], extra["dx"],
                  extra["F"].reshape(B, -1)):
            f32(a).tofile(f)
    r = subprocess.run([exe, str(tmp_path / "in.bin"), str(tmp_path / "out.bin")], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    out = {}
    with open(tmp_path / "out.bin", "rb") as f:
        n = int(np.fromfile(f, np.int32, 1)[0])
        for _ in range(n):
            name = f.read(32).split(b"\0")[0].decode()
            size = int(np.fromfile(f, np.int64, 1)[0])
            out[name] = np.fromfile(f, np.float32, size).reshape(-1, B).T.astype(np.float64)
    return out


@pytest.mark.parametrize("name", list(MODELS))
def test_host_compiled_kernels_match_the_oracle(harness, tmp_path, name):
    m = MODELS[name]
    B = 24
    s = gen.draw_states(m, B, 4242).as_f32()
    rng = np.random.default_rng(4243)
    draw = lambda *shape: rng.standard_normal(shape).astype(np.float32).astype(np.float64)
    extra = {"g": draw(B, m.nv), "dq": draw(B, m.nv), "dqd": draw(B, m.nv), "dx": draw(B, m.nv),
             "F": draw(B, m.n_bodies, 6)}
    frames = list(m.end_frames)[:8]
    o = _run(harness, tmp_path, m, s, frames, extra)
    tol_aba = TOL if name == "chain7" else TOL_TREE
    assert normwise(o["pose"], rbd.fk_flat(m, s.q)) < TOL
    assert normwise(o["J"], rbd.jacobian(m, s.q, frames).reshape(B, -1)) < TOL
    assert normwise(o["rnea"], rbd.rnea(m, s.q, s.qd, s.qdd)) < TOL
    Mref = rbd.crba(m, s.q)
    assert normwise(o["M"], Mref.reshape(B, -1)) < TOL
    assert normwise(o["LD"], rbd.pack_ltdl(*rbd.ltdl(Mref))) < TOL
    assert normwise(o["aba"], rbd.aba(m, s.q, s.qd, s.tau)) < tol_aba
    for got, ref in zip(("rnea_vjp_q", "rnea_vjp_qd", "rnea_vjp_qdd"), dv.rnea_vjp(m, s.q, s.qd, s.qdd, extra["g"])):
        assert normwise(o[got], ref) < TOL_TREE, got
    # the ABA adjoint is taken at the host's own forward result, as the kernels are
    for got, ref in zip(("aba_vjp_q", "aba_vjp_qd", "aba_vjp_tau"), dv.aba_vjp(m, s.q, s.qd, s.tau, extra["g"])):
        assert normwise(o[got], ref) < TOL_TREE, got
    assert normwise(o["rnea_jvp"], dv.rnea_jvp(m, s.q, s.qd, s.qdd, extra["dq"], extra["dqd"], extra["dx"])) < TOL_TREE
    assert normwise(o["aba_jvp"], dv.aba_jvp(m, s.q, s.qd, s.tau, extra["dq"], extra["dqd"], extra["dx"])) < TOL_TREE
    assert normwise(o["fk_jvp"], dv.fk_jvp(m, s.q, extra["dq"], frames).reshape(B, -1)) < TOL
    re, ae = rbd.rnea(m, s.q, s.qd, s.qdd, fext=extra["F"]), rbd.aba(m, s.q, s.qd, s.tau, fext=extra["F"])
    if m.nv < 6:
        # one or two dofs: tau - tau_ext can cancel to 1e-4 of its terms in
        # some instances, so the error is taken against the terms' scale
        rp, ap = rbd.rnea(m, s.q, s.qd, s.qdd), rbd.aba(m, s.q, s.qd, s.tau)
        scale = lambda a, b: np.maximum(np.abs(a).max(1, keepdims=True), np.abs(b).max(1, keepdims=True))
        assert np.max(np.abs(o["rnea_ext"] - re) / scale(re, rp)) < TOL
        assert np.max(np.abs(o["aba_ext"] - ae) / scale(ae, ap)) < tol_aba
    else:
        assert normwise(o["rnea_ext"], re) < TOL
        assert normwise(o["aba_ext"], ae) < tol_aba
    # operational-space control of the last frame (the chain through its unrolled code), task accelerations
    # = the first six rows of dx; the FP32 bound of a solve with Lambda^-1 (cond(Lambda) * 2^-24)
    path_dofs, j = 0, frames[-1]
    while j >= 0:
        path_dofs += 6 if m.joint_type[j] == 1 else 1
        j = int(m.parent[j])
    if path_dofs >= 6:  # fewer dofs leave Lambda^-1 singular
        rt, rL = task_space.osc(m, s.q, s.qd, frames[-1], extra["dx"][:, :6])
        bound = 1e-5 + np.linalg.cond(rL) * 2.0 ** -24
        rel = lambda a, r: np.max(np.abs(a - r).reshape(B, -1), 1) / np.max(np.abs(r).reshape(B, -1), 1)
        assert np.all(rel(o["osc"], rt) <= bound)
        assert np.all(rel(o["osc_lambda"], rL.reshape(B, -1)) <= bound)
    if m.n_bodies <= 32:  # the lane-group sweeps, lanes run one after another in each step
        assert normwise(o["rnea_lg"], rbd.rnea(m, s.q, s.qd, s.qdd)) < TOL
        assert normwise(o["bias_lg"], rbd.rnea(m, s.q, s.qd, np.zeros_like(s.qd))) < TOL
        assert normwise(o["aba_lg"], rbd.aba(m, s.q, s.qd, s.tau)) < tol_aba
        assert normwise(o["fk_lg_pose"], rbd.fk_flat(m, s.q)) < TOL
        assert normwise(o["fk_lg_J"], rbd.jacobian(m, s.q, frames).reshape(B, -1)) < TOL
        assert normwise(o["crba_lg_M"], Mref.reshape(B, -1)) < TOL
        assert normwise(o["crba_lg_LD"], rbd.pack_ltdl(*rbd.ltdl(Mref))) < TOL
        for got, ref in zip(("rnea_vjp_lg_q", "rnea_vjp_lg_qd", "rnea_vjp_lg_qdd"),
                            dv.rnea_vjp(m, s.q, s.qd, s.qdd, extra["g"])):
            assert normwise(o[got], ref) < TOL_TREE, got
        for got, ref in zip(("aba_vjp_lg_q", "aba_vjp_lg_qd", "aba_vjp_lg_tau"),
                            dv.aba_vjp(m, s.q, s.qd, s.tau, extra["g"])):
            assert normwise(o[got], ref) < TOL_TREE, got
