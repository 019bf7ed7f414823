"""Host-side pieces of bench.py: the roofline arithmetic, the algorithmic
byte counts, the CPU-baseline leg and the reference arm's JSON line."""

import json
import os
import subprocess
import sys

import gen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_bytes_per_instance_chain_and_humanoid():
    c, h = gen.chain7(0), gen.humanoid(0)
    assert bench.bytes_per_instance("rnea", c.nq, c.nv, c.n_bodies, 1) == 112
    assert bench.bytes_per_instance("fk_jac", c.nq, c.nv, c.n_bodies, 1) == 532
    assert bench.bytes_per_instance("crba_ltdl", h.nq, h.nv, h.n_bodies, 4) == 4 * (36 + 35 * 35 + 35 * 36 // 2)
    assert bench.bytes_per_instance("fk_jac", h.nq, h.nv, h.n_bodies, 4) == 4 * (36 + 360 + 840)


def test_roofline_fraction_is_the_slower_roof():
    c = gen.chain7(0)
    B = 1 << 20
    out = bench.roofline_of({"rnea": 0.1, "fk_jac": 0.1}, bench.FLOPS["chain7"], B, 80.0, 6000.0, c)
    r = out["rnea"]
    assert r["bound"] == "alu" and abs(r["roofline_frac"] - bench.FLOPS["chain7"]["rnea"] * B / 80e12 / 1e-4) < 1e-9
    f = out["fk_jac"]
    assert f["bound"] == "hbm" and abs(f["roofline_frac"] - 532 * B / 6000e9 / 1e-4) < 1e-9


def test_cpu_baseline_child_and_reference_arm():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--cpu-baseline-child", "--cpu-seconds",
                        "0.5"], capture_output=True, text=True, cwd=ROOT, timeout=300)
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["kind"] == "oracle" and d["cores"] == 1 and d["value"] > 0
    assert set(d["per_op"]) == set(bench.OPS)
    # the aggregate is the six-op rate: 6 / sum of 1 / per-op rates
    assert abs(d["value"] - 6 / sum(1 / v for v in d["per_op"].values())) < 1e-9 * d["value"]
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--cpu-baseline-child", "--cpu-robot",
                        "humanoid", "--cpu-seconds", "0.5"], capture_output=True, text=True, cwd=ROOT, timeout=300)
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert set(d["per_op"]) == set(bench.HUMANOID_OPS) and all(v > 0 for v in d["per_op"].values())
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--cpu-seconds", "0.5"], capture_output=True, text=True, cwd=ROOT,
                       timeout=300)
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] == 0


def test_cpu_baseline_all_cores_sums_processes():
    r = bench.run_cpu_baseline_all_cores(1.0)
    assert r["cores"] == (os.cpu_count() or 1) and r["value"] > 0 and r["kind"] == "oracle"
    assert "single-threaded processes" in r["sample"] and r["cpu_model"]


def test_kernels_per_call_matches_the_dispatch():
    """The gpu_launches claim counts kernels per public call: the chain's ABA
    adjoint with taubar is two launches (factor solve, adjoint sweep); a tree's
    FK+J adds the fill of its Jacobians' structural zeros; the tree CRBA
    writes its zeros itself (one launch); everything else is one launch."""
    c, h, t = gen.chain7(0), gen.humanoid(0), gen.random_tree(101)
    assert bench.kernels_per_call(c, "aba_vjp") == 2
    assert all(bench.kernels_per_call(c, op) == 1 for op in bench.OPS if op != "aba_vjp")
    assert bench.kernels_per_call(h, "fk_jac") == 2
    assert bench.kernels_per_call(h, "crba_ltdl") == 1
    assert all(bench.kernels_per_call(h, op) == 1 for op in ("rnea", "bias", "aba", "rnea_vjp", "aba_vjp"))
    # a frame whose ancestors are every body has no zero column: no fill
    chain_tree = gen.serial_chain(3, 5)
    assert bench.kernels_per_call(chain_tree, "fk_jac") == 1
    assert bench.kernels_per_call(t, "crba_ltdl") == 1



def test_concurrent_groups_keep_the_adjoint_after_the_aba():
    """Every op of a step lies in exactly one stream group, and the ABA adjoint
    (which reads the ABA's output) shares the ABA's group, after it."""
    for ops in (bench.OPS, bench.HUMANOID_OPS):
        groups = bench.concurrent_groups(ops)
        flat = [o for g in groups for o in g]
        assert sorted(flat) == sorted(ops)
        g = next(g for g in groups if "aba_vjp" in g)
        assert g.index("aba") < g.index("aba_vjp")
        assert all(len(g) == 1 for g in groups if "aba" not in g)
