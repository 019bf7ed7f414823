#!/usr/bin/env python
"""Throughput benchmark of the batched rigid-body hot path on one GB300.

One step = one pass of the whole path over one resident batch of the 7-DoF
serial chain (2^20 instances, FP32 SoA): FK + end-effector Jacobian, RNEA,
CRBA + L^T D L, ABA, RNEA VJP and ABA VJP. The metric counts one evaluation
per op per instance (6 x 2^20 per step). Per-kernel CUDA-event times feed the
roofline of the dominant kernel; a short served stream gives p50/p99; the FP64
oracle is timed on the host cores on a bounded sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl frax|reference]

Under torchrun (N > 1) every rank runs its own replica of the batch (the
instances are independent: weak scaling, no collective on the data path).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ABA/RNEA evals/sec at 1 GB300 vs roofline; served p50/p99 latency at 1e-4 rel err"
UNIT = "evals/s"
OPS = ["fk_jac", "rnea", "crba_ltdl", "aba", "rnea_vjp", "aba_vjp"]
HBM_OPS = ("fk_jac", "crba_ltdl")  # bound by their output writes; the other four by FP32 arithmetic
SM_COUNT = 152
FP32_LANES_PER_SM = 128


# ------------------------------------------------------------- flop accounting
# Algorithmic FP32 operations per instance (fma = 2 flops, add/sub/mul = 1;
# sincos, sqrt and divisions are not in the FMA-pipe count), counted exactly
# by running the device code on the host with a counting float
# (`python bench.py --count-flops` rebuilds flopcount.cu and reprints them).
# Where a kernel trades flops for registers (the adjoints recompute forward
# state by stepping back through the joints; the tree ABA recomputes
# velocities; the tree factor comes from articulated inertias) the table
# keeps the count of the direct formulation that stores instead, so the
# roofline is against the algorithm's work, not the kernel's extra work.
# Articulated inertias are counted with the zeros of their projection
# (I^A - U U^T / D annihilates e_z) skipped, as every kernel skips them. The
# chain ABA adjoint = its M^-1 solve through the mass-matrix factor (1677)
# plus the stored-state RNEA adjoint (4272); the chain's forward dynamics
# go through the same factor, RNEA bias (1683) + solve (1677) = 3360
# ("aba_factor"); the "direct_*" lines of
# --count-flops give the stored-state counts. The JVPs' counts leave out the
# 208-flop step back through a joint that the kernels make instead of storing
# (6 per chain sweep, 24 per humanoid sweep). With external forces: the
# plain kernel's count plus the force sweep's (554 chain, 2585 humanoid).
FLOPS = {
    "chain7": {"fk_jac": 748, "fk": 664, "rnea": 1683, "bias": 1683, "crba_ltdl": 1586, "crba": 1453,
               "aba": 3360, "aba_sweep": 3431, "rnea_vjp": 4272, "aba_vjp": 5949, "osc": 7730, "rnea_ext": 2237,
               "aba_ext": 3914, "fk_jvp": 593, "rnea_jvp": 4175, "aba_jvp": 5859},
    "humanoid": {"fk_jac": 4685, "fk": 3173, "rnea": 7761, "bias": 7755, "crba_ltdl": 13474, "crba": 9704,
                 "aba": 17399, "aba_sweep": 17399, "rnea_vjp": 19471, "aba_vjp": 32178, "osc": 22680, "rnea_ext": 10346,
                 "aba_ext": 19984, "fk_jvp": 2584, "rnea_jvp": 17866, "aba_jvp": 30662},
}
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# chain step's kernels, from one `ncu --set full` capture of this bench's
# workload; an entry is removed when its kernel changes. aba_vjp = the factor
# solve plus the adjoint sweep.
NCU_TRAFFIC = {
    "fk_jac": 29.39e6 + 490.03e6, "rnea": 88.11e6 + 3.83e6, "crba_ltdl": 25.22e6 + 260.06e6,
    "aba": 88.13e6 + 6.27e6, "rnea_vjp": 117.51e6 + 40.27e6, "aba_vjp": 54.56e6 + 0.35e6 + 117.51e6 + 22.37e6,
}
# operational-space control task bodies (the last end frame of each model)
OSC_TASK = {"chain7": 6, "humanoid": 29}


def jacobian_nonzeros(robot):
    """Structurally non-zero Jacobian entries of the end frames: 6 per dof
    whose body is an ancestor of (or is) the frame body."""
    anc = []
    for i, p in enumerate(robot.parent):
        anc.append((anc[int(p)] if p >= 0 else 0) | (1 << i))
    dof_body = [i for i, t in enumerate(robot.joint_type) for _ in range(6 if t == 1 else 1)]
    return sum(6 for f in robot.end_frames for b in dof_body if (anc[f] >> b) & 1)


def bytes_per_instance(op, nq, nv, nb, nframes, j_nonzero=None):
    """Minimum HBM traffic: inputs read once, outputs written once (FP32).
    For the Jacobians only the structurally non-zero entries count when
    j_nonzero is given (the dense zero-filled write is reported beside)."""
    f = 4
    return {
        "fk_jac": f * (nq + 12 * nb + (nframes * 6 * nv if j_nonzero is None else j_nonzero)),
        "rnea": f * (nq + 3 * nv), "bias": f * (nq + 2 * nv),
        "crba_ltdl": f * (nq + nv * nv + nv * (nv + 1) // 2),
        "aba": f * (nq + 3 * nv), "aba_sweep": f * (nq + 3 * nv),
        "rnea_vjp": f * (2 * nq + 5 * nv), "aba_vjp": f * (2 * nq + 5 * nv),
        "osc": f * (nq + 2 * nv + 6),
        "rnea_ext": f * (nq + 3 * nv + 6 * nb), "aba_ext": f * (nq + 3 * nv + 6 * nb),
        "fk_jvp": f * (nq + nv + 6 * nframes), "rnea_jvp": f * (nq + 6 * nv), "aba_jvp": f * (nq + 6 * nv),
    }[op]


def count_flops():
    """Builds flopcount.cu (host-only) and prints the per-op table."""
    import gen
    exe = os.path.join(ROOT, "_build", "flopcount")
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    subprocess.run(["g++", "-std=c++17", "-O1", "-x", "c++", "-I/usr/local/cuda/include", "-w",
                    "-o", exe, os.path.join(ROOT, "flopcount.cu"),
                    os.path.join(ROOT, "paper_2604_04310_gb300", "csrc", "model.cpp")], check=True)
    for m in (gen.chain7(0), gen.humanoid(0)):
        fr = list(m.end_frames)
        ints = lambda xs: " ".join(str(int(x)) for x in xs)
        flts = lambda xs: " ".join(repr(float(x)) for x in xs)
        text = " ".join([ints([m.n_bodies, *m.parent, *m.joint_type]),
                         flts([*m.axis.ravel(), *m.placement.ravel(), *m.inertia.ravel(), *m.gravity]),
                         ints([len(fr), *fr])])
        r = subprocess.run([exe], input=text, capture_output=True, text=True, check=True)
        print(m.name, r.stdout)


def fp32_peak_tflops(sm_mhz: float) -> float:
    return SM_COUNT * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


# ------------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- workloads
def make_inputs(robot, B, seed, device):
    import torch

    import gen
    s = gen.draw_states(robot, B, seed)
    g = gen.draw_gbar(robot.nv, B, seed + 7)
    host = {k: torch.from_numpy(gen.to_soa(v)) for k, v in
            (("q", s.q), ("qd", s.qd), ("qdd", s.qdd), ("tau", s.tau), ("gbar", g))}
    dev = {k: v.to(device) for k, v in host.items()}
    return host, dev


def kernels_per_call(robot, op):
    """Kernel launches one public call makes: the chain's ABA adjoint runs as
    the factor solve plus the adjoint sweep; a tree's FK+J adds the fill of its
    structural zeros (rows for non-ancestor frame bodies) when it has any (the
    tree CRBA kernel writes its own)."""
    chain7 = robot.n_bodies == 7 and all(int(p) == i - 1 for i, p in enumerate(robot.parent)) \
        and not robot.has_free_root
    if chain7:
        return 2 if op == "aba_vjp" else 1
    anc = []
    for i, p in enumerate(robot.parent):
        anc.append((anc[int(p)] if p >= 0 else 0) | (1 << i))
    bodies = range(robot.n_bodies)
    if op == "fk_jac":
        return 1 + any(not (anc[f] >> b) & 1 for f in robot.end_frames for b in bodies)
    return 1


class Step:
    """The whole hot path over one resident batch; output buffers are
    allocated once (torch), the kernels write into them."""

    def __init__(self, fx, model, robot, dev, device, ops, task=None, flat=False):
        import torch
        self.fx, self.m, self.d, self.ops = fx, model, dev, ops
        B = dev["q"].shape[1]
        nv, nb = model.nv, model.n_bodies
        self.frames = list(robot.end_frames)
        rows = {"pose": 12 * nb, "J": len(self.frames) * 6 * nv, "tau": nv, "M": nv * nv,
                "LD": nv * (nv + 1) // 2, "qdd": nv, "rq": model.nq, "rqd": nv, "rqdd": nv,
                "aq": model.nq, "aqd": nv, "at": nv}
        if flat:  # every output a [rows][B] view of one buffer (one copy brings them all back)
            self.flat_out = torch.empty(sum(rows.values()) * B, dtype=torch.float32, device=device)
            self.out, off = {}, 0
            for k, r in rows.items():
                self.out[k] = self.flat_out[off:off + r * B].view(r, B)
                off += r * B
        else:
            self.out = {k: torch.empty((r, B), dtype=torch.float32, device=device) for k, r in rows.items()}
        if "fk_jvp" in ops:
            self.out["dpose"] = torch.empty((6 * len(self.frames), B), dtype=torch.float32, device=device)
        fx_, m, d, o = fx, model, dev, self.out
        table = {
            "fk_jac": lambda: fx_.frax_jacobian(m, d["q"], self.frames, pose=o["pose"], J=o["J"]),
            "rnea": lambda: fx_.frax_rnea(m, d["q"], d["qd"], d["qdd"], tau=o["tau"]),
            "bias": lambda: fx_.frax_rnea(m, d["q"], d["qd"], None, tau=o["tau"]),
            "crba_ltdl": lambda: fx_.frax_crba(m, d["q"], M=o["M"], LD=o["LD"]),
            "aba": lambda: fx_.frax_aba(m, d["q"], d["qd"], d["tau"], qdd=o["qdd"]),
            "aba_sweep": lambda: fx_.frax_aba_articulated(m, d["q"], d["qd"], d["tau"], qdd=o["qdd"]),
            "rnea_vjp": lambda: fx_.frax_rnea_vjp(m, d["q"], d["qd"], d["qdd"], d["gbar"], qbar=o["rq"],
                                                  qdbar=o["rqd"], qddbar=o["rqdd"]),
            "aba_vjp": lambda: fx_.frax_aba_vjp(m, d["q"], d["qd"], d["tau"], o["qdd"], d["gbar"], qbar=o["aq"],
                                                qdbar=o["aqd"], taubar=o["at"]),
            "osc": lambda: fx_.frax_osc(m, task, d["q"], d["qd"], d["xdd"], tau=o["tau"]),
            "rnea_ext": lambda: fx_.frax_rnea_ext(m, d["q"], d["qd"], d["qdd"], d["fext"], tau=o["tau"]),
            "fk_jvp": lambda: fx_.frax_fk_jvp(m, d["q"], d["dq"], self.frames, dpose=o["dpose"]),
            "fk": lambda: fx_.frax_fk(m, d["q"], pose=o["pose"]),
            "fk_scan": lambda: fx_.frax_fk_scan(m, d["q"], pose=o["pose"]),
            "rnea_jvp": lambda: fx_.frax_rnea_jvp(m, d["q"], d["qd"], d["qdd"], d["dq"], d["dqd"], d["dx"],
                                                  dtau=o["at"]),
            "aba_jvp": lambda: fx_.frax_aba_jvp(m, d["q"], d["qd"], d["tau"], d["qdd"], d["dq"], d["dqd"], d["dx"],
                                                dqdd=o["aqd"]),
            "aba_ext": lambda: fx_.frax_aba_ext(m, d["q"], d["qd"], d["tau"], d["fext"], qdd=o["qdd"]),
        }
        self.launches = [(n, table[n]) for n in ops]
        self.kernels = sum(kernels_per_call(robot, n) for n in ops)
        self.B = B

    def run(self, events=None):
        for name, fn in self.launches:
            if events is not None:
                events[name][0].record()
            fn()
            if events is not None:
                events[name][1].record()
        return self.kernels

    def run_groups(self, streams, groups):
        """The same calls, group g issued in order on streams[g] (forked from and
        joined back into the current stream): the groups overlap on the GPU."""
        import torch
        cur = torch.cuda.current_stream()
        fns = dict(self.launches)
        for st in streams:
            st.wait_stream(cur)
        for st, g in zip(streams, groups):
            with torch.cuda.stream(st):
                for name in g:
                    fns[name]()
        for st in streams:
            cur.wait_stream(st)
        return self.kernels

    def run_split(self, side, side_ops):
        """The same calls, those in side_ops issued on the stream `side`
        (forked from and joined back into the current stream), the rest on
        the current stream: independent ops overlap on the GPU."""
        import torch
        cur = torch.cuda.current_stream()
        side.wait_stream(cur)
        with torch.cuda.stream(side):
            for name, fn in self.launches:
                if name in side_ops:
                    fn()
        for name, fn in self.launches:
            if name not in side_ops:
                fn()
        cur.wait_stream(side)
        return self.kernels


def time_step(step, steps, warmup, flush, world, dist, clocks=None):
    """Times `steps` passes of the step with CUDA events (per step and per
    kernel) on torch's current stream, the stream the kernels are launched
    on; L2 is flushed between steps outside the events. Returns the median
    step time (ms), the median time of each op, launches, wall seconds and
    the clock record."""
    import torch
    for _ in range(warmup):
        step.run()
    torch.cuda.synchronize()
    ev = [{n: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for n in step.ops}
          for _ in range(steps)]
    sev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.start()
        time.sleep(0.3)
    t0 = time.perf_counter()
    launches = 0
    for k in range(steps):
        flush.zero_()
        sev[k][0].record()
        launches += step.run(ev[k])
        sev[k][1].record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if world > 1:
        dist.barrier()
    clk = clocks.stop() if clocks is not None else None
    step_ms = statistics.median(a.elapsed_time(b) for a, b in sev)
    per_op_ms = {n: statistics.median(e[n][0].elapsed_time(e[n][1]) for e in ev) for n in step.ops}
    return step_ms, per_op_ms, launches, wall, clk


def time_graph(step, steps, warmup, flush, world, dist, clocks=None, side_ops=(), groups=None):
    """The same step captured once as a CUDA graph (the same calls, the same
    kernels; replaying it trims the host's launch gaps between them) and
    replayed `steps` times, L2 flushed between replays outside the events.
    With side_ops, those calls go on a second stream inside the capture (the
    graph then runs them beside the others). Returns (median step ms,
    launches, wall, clocks, None), or five Nones but the last, the reason,
    when the capture fails."""
    import torch
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(max(3, warmup)):
            step.run()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    fork = torch.cuda.Stream()
    gstreams = [torch.cuda.Stream() for _ in (groups or ())]
    try:
        with torch.cuda.graph(g):
            if groups:
                step.run_groups(gstreams, groups)
            elif side_ops:
                step.run_split(fork, set(side_ops))
            else:
                step.run()
    except Exception as e:  # noqa: BLE001 - reported in the bench line
        torch.cuda.synchronize()
        return None, None, None, None, str(e).splitlines()[0][:200]
    for _ in range(warmup):
        g.replay()
    torch.cuda.synchronize()
    sev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.start()
        time.sleep(0.3)
    t0 = time.perf_counter()
    for k in range(steps):
        flush.zero_()
        sev[k][0].record()
        g.replay()
        sev[k][1].record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if world > 1:
        dist.barrier()
    clk = clocks.stop() if clocks is not None else None
    return statistics.median(a.elapsed_time(b) for a, b in sev), steps * step.kernels, wall, clk, None


def whole_job(step_ms, evals_per_step, world, dist, device):
    """Replicas: every rank times its own batch; the job's step time is the
    slowest rank's median step (max over ranks) and the value counts every
    rank's evaluations. Returns (ms per step, evaluations per second)."""
    import torch
    t = torch.tensor([step_ms], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_per_step = float(t.item())
    return ms_per_step, world * evals_per_step / (ms_per_step / 1e3)


def roofline_of(per_op_ms, flops, B, peak, hbm_gbs, robot):
    """Per kernel: achieved FP32 rate and HBM rate from the algorithmic work,
    and the roofline fraction t_roof / t_measured with
    t_roof = max(flops / FP32 peak, bytes / HBM peak)."""
    out = {}
    for n, ms in per_op_ms.items():
        t = ms / 1e3
        by = bytes_per_instance(n, robot.nq, robot.nv, robot.n_bodies, len(robot.end_frames),
                                jacobian_nonzeros(robot))
        dense = bytes_per_instance(n, robot.nq, robot.nv, robot.n_bodies, len(robot.end_frames))
        tf = flops[n] * B / t / 1e12
        gbs = by * B / t / 1e9
        t_alu = flops[n] * B / (peak * 1e12)
        t_hbm = by * B / (hbm_gbs * 1e9)
        out[n] = {"ms": ms, "evals_per_s": B / t, "flops_per_instance": flops[n], "bytes_per_instance": by,
                  "bytes_dense_per_instance": dense,
                  "tflops": tf, "gbs": gbs, "frac_fp32_peak": tf / peak, "frac_hbm_peak": gbs / hbm_gbs,
                  "bound": "alu" if t_alu >= t_hbm else "hbm", "roofline_frac": max(t_alu, t_hbm) / t}
    return out


def measured_hbm_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


HUMANOID_OPS = ["fk_jac", "bias", "crba_ltdl", "aba", "rnea_vjp", "aba_vjp"]


def cpu_baseline_child(args):
    """Times the FP64 oracle (as it stands), single-threaded, op by op, on
    bounded samples of one robot's workload (the chain's six ops, or the
    humanoid's with bias forces in place of RNEA): each op runs on batches
    of fresh seeded states until its share of the time budget is spent
    (perf_counter around many batches, as the paper times its Python
    calls). Prints one JSON object with each op's evaluations per second
    and the six-op aggregate 6 / sum(1 / rate)."""
    import numpy as np

    import gen
    from oracle import derivatives as dv
    from oracle import rbd
    robot = gen.chain7(0) if args.cpu_robot == "chain7" else gen.humanoid(0)
    ops = OPS if args.cpu_robot == "chain7" else HUMANOID_OPS
    frames = list(robot.end_frames)
    per_op, inst = {}, {}
    budget = args.cpu_seconds / len(ops)
    for n, op in enumerate(ops):
        S = 256 if args.cpu_robot == "chain7" else 64  # the oracle's cost per call is mostly per batch
        done, el, k = 0, 0.0, 0
        while el < budget:
            s = gen.draw_states(robot, S, 99 + 1000 * n + k)
            g = gen.draw_gbar(robot.nv, S, 5 + 1000 * n + k)
            t0 = time.perf_counter()
            if op == "fk_jac":
                rbd.fk_flat(robot, s.q)
                rbd.jacobian(robot, s.q, frames)
            elif op == "rnea":
                rbd.rnea(robot, s.q, s.qd, s.qdd)
            elif op == "bias":
                rbd.rnea(robot, s.q, s.qd, np.zeros_like(s.qd))
            elif op == "crba_ltdl":
                rbd.ltdl(rbd.crba(robot, s.q))
            elif op == "aba":
                rbd.aba(robot, s.q, s.qd, s.tau)
            elif op == "rnea_vjp":
                dv.rnea_vjp(robot, s.q, s.qd, s.qdd, g)
            else:
                dv.aba_vjp(robot, s.q, s.qd, s.tau, g)
            el += time.perf_counter() - t0
            done += S
            k += 1
        per_op[op] = done / el
        inst[op] = done
    agg = len(ops) / sum(1.0 / r for r in per_op.values())
    print(json.dumps({"value": agg, "unit": UNIT, "cores": 1, "kind": "oracle", "per_op": per_op,
                      "instances_per_op": inst,
                      "sample": f"{args.cpu_robot}: each of {len(ops)} ops on fresh seeded states for "
                                f"{budget:.1f} s ({sum(inst.values())} instances in all), FP64 numpy oracle, "
                                f"1 thread; value = {len(ops)} / sum over ops of 1 / (evals/s)"}))


def _child_cmd(robot, seconds):
    return [sys.executable, os.path.abspath(__file__), "--cpu-baseline-child", "--cpu-robot", robot,
            "--cpu-seconds", str(seconds)]


_CPU_ENV = dict(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")


def run_cpu_baseline(seconds, robot="chain7"):
    env = dict(os.environ, **_CPU_ENV)
    r = subprocess.run(_child_cmd(robot, seconds), capture_output=True, text=True, env=env, cwd=ROOT)
    for line in r.stdout.splitlines()[::-1]:
        if line.startswith("{"):
            return json.loads(line)
    return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": "failed: " + r.stderr[-300:]}


def cpu_model():
    """The host CPU's model string (x86: model name; Arm: implementer/part)."""
    try:
        info = open("/proc/cpuinfo").read()
    except OSError:
        return "unknown"
    for key in ("model name", "Model name"):
        for line in info.splitlines():
            if line.startswith(key):
                return line.split(":", 1)[1].strip()
    parts = {}
    for line in info.splitlines():
        if ":" in line:
            k, v = (x.strip() for x in line.split(":", 1))
            parts.setdefault(k, v)
    if "CPU part" in parts:
        return f"Arm implementer {parts.get('CPU implementer', '?')} part {parts['CPU part']}"
    return "unknown"


def run_cpu_baseline_all_cores(seconds, robot="chain7"):
    """The same per-op oracle timing in one single-threaded process per host
    core, all at once; each op's value sums the processes' rates."""
    n = os.cpu_count() or 1
    env = dict(os.environ, **_CPU_ENV)
    procs = [subprocess.Popen(_child_cmd(robot, seconds), stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                              env=env, cwd=ROOT) for _ in range(n)]
    per_op, inst = {}, 0
    for p in procs:
        out, _ = p.communicate()
        for line in out.splitlines()[::-1]:
            if line.startswith("{"):
                d = json.loads(line)
                for k, v in d["per_op"].items():
                    per_op[k] = per_op.get(k, 0.0) + v
                inst += sum(d["instances_per_op"].values())
                break
    agg = len(per_op) / sum(1.0 / r for r in per_op.values()) if per_op else None
    return {"value": agg, "unit": UNIT, "cores": n, "kind": "oracle", "cpu_model": cpu_model(), "per_op": per_op,
            "sample": f"{n} single-threaded processes at once, {robot}, {inst} instances in all, FP64 numpy "
                      f"oracle, {seconds:.0f} s each"}


SERVE_OPS = ["rnea", "crba", "aba", "rnea_grad"]


SERVE_LOADS = (0.25, 0.5, 0.75, 0.9)


def serve_stream(fx, seconds, check_batched=True, repeats=3):
    """Served workload: requests for the 7-DoF chain, the humanoid and 32
    random trees (3-64 bodies), op uniform over rnea / crba / aba /
    rnea-gradient, instance count log-uniform in [1, 4096]. The request
    traces are replayed natively (frax_server_replay): first a burst that
    gives the saturation rate, then Poisson arrivals at 25, 50, 75 and 90 % of it,
    each point repeated (p50/p99 per repeat and their medians); latency =
    completion seen by the host - arrival. Every pool request is also timed
    alone, so each point reports how long requests waited beyond their solo
    latency, and a one-instance chain request alone gives the latency floor. The server's device error word
    and kernel launch count are reported with the results, and 64 small
    served requests are compared with the batched entry points."""
    import numpy as np

    import gen
    from paper_2604_04310_gb300.serving import Server
    robots = gen.serving_pool(32)
    models = [fx.Model.from_robot(r) for r in robots]
    srv = Server(budget_bytes=4 << 30, idle_exit_ms=20.0)
    ids = [srv.add_model(m) for m in models]
    rng = np.random.default_rng(2026)
    pool = []
    for k in range(256):
        mi = int(rng.integers(len(robots)))
        op = SERVE_OPS[int(rng.integers(4))]
        B = int(np.clip(np.floor(np.exp(rng.uniform(0.0, np.log(4097.0)))), 1, 4096))
        r = robots[mi]
        st = gen.draw_states(r, B, 50000 + k).as_f32()
        g = gen.draw_gbar(r.nv, B, 60000 + k).astype(np.float32).astype(np.float64)
        arrays = {"rnea": [st.q, st.qd, st.qdd], "crba": [st.q], "aba": [st.q, st.qd, st.tau],
                  "rnea_grad": [st.q, st.qd, st.qdd, g]}[op]
        pool.append((mi, op, B, [gen.to_soa(a) for a in arrays], st, g))
    trace_rng = np.random.default_rng(7)

    def trace(n):
        ks = trace_rng.integers(len(pool), size=n)
        return ks, [(ids[pool[k][0]], pool[k][1], pool[k][3]) for k in ks]

    # latency of every pool request alone (3 ms apart, nothing queues; the
    # smaller of two passes), and the floor: a one-instance chain RNEA
    solo_tr = [(ids[p[0]], p[1], p[3]) for p in pool]
    lat_a, _ = srv.replay(solo_tr + solo_tr, np.arange(2 * len(pool)) * 3000.0)
    solo = np.minimum(lat_a[:len(pool)], lat_a[len(pool):])
    st1 = gen.draw_states(robots[0], 1, 49999).as_f32()
    one = [gen.to_soa(a) for a in (st1.q, st1.qd, st1.qdd)]
    lat_f, _ = srv.replay([(ids[0], "rnea", one)] * 200, np.arange(200) * 200.0)
    floor = {"request": "chain7 rnea, 1 instance, alone (200 requests 200 us apart)",
             "p50_us": float(np.percentile(lat_f, 50)), "p99_us": float(np.percentile(lat_f, 99))}

    # saturation: everything arrives at once
    ks, tr = trace(3000)
    t0 = time.perf_counter()
    srv.replay(tr, np.zeros(len(tr)))
    el = time.perf_counter() - t0
    sat_req = len(tr) / el
    sat_inst = sum(pool[k][2] for k in ks) / el
    points = []
    for frac in SERVE_LOADS:
        rate = frac * sat_req
        n = int(max(200, rate * seconds))
        reps = []
        for _ in range(repeats):
            ks, tr = trace(n)
            arrival = np.cumsum(trace_rng.exponential(1e6 / rate, size=n))
            t0 = time.perf_counter()
            lat, _ = srv.replay(tr, arrival)
            el = time.perf_counter() - t0
            wait = lat - solo[ks]  # beyond the same request's solo latency
            reps.append({"p50_us": float(np.percentile(lat, 50)), "p99_us": float(np.percentile(lat, 99)),
                         "wait_beyond_solo_p50_us": float(np.percentile(wait, 50)),
                         "wait_beyond_solo_p99_us": float(np.percentile(wait, 99)),
                         "mean_us": float(lat.mean()), "max_us": float(lat.max()),
                         "evals_per_s": sum(pool[k][2] for k in ks) / el,
                         "device_status": srv.info()["device_status"]})
        points.append({"load": frac, "offered_rate_hz": rate, "requests_per_repeat": n, "repeats": reps,
                       "p50_us": statistics.median(r["p50_us"] for r in reps),
                       "p99_us": statistics.median(r["p99_us"] for r in reps),
                       "wait_beyond_solo_p50_us": statistics.median(r["wait_beyond_solo_p50_us"] for r in reps),
                       "wait_beyond_solo_p99_us": statistics.median(r["wait_beyond_solo_p99_us"] for r in reps),
                       "evals_per_s": statistics.median(r["evals_per_s"] for r in reps)})
    # served results against the library's batched entry points on the same
    # inputs (those are pinned to the FP64 oracle by the parity tests)
    diff, checked = {}, 0
    if check_batched:
        import torch
        small = [k for k in range(len(pool)) if pool[k][2] <= 256][:64]
        tr = [(ids[pool[k][0]], pool[k][1], pool[k][3]) for k in small]
        _, outs = srv.replay(tr, np.cumsum(np.full(len(tr), 50.0)), keep_outputs=True)
        for k, o in zip(small, outs):
            mi, op, B, arrays, _, _ = pool[k]
            m = models[mi]
            d = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda() for a in arrays]
            ref = {"rnea": lambda: [fx.frax_rnea(m, *d)], "crba": lambda: [fx.frax_crba(m, d[0])[0]],
                   "aba": lambda: [fx.frax_aba(m, *d)], "rnea_grad": lambda: list(fx.frax_rnea_vjp(m, *d))}[op]()
            checked += 1
            for x, rt in zip(o, ref):
                rr = rt.cpu().numpy().T.astype(np.float64)
                xx = np.asarray(x, np.float64).T
                e = np.abs(xx - rr).reshape(B, -1).max(1) / np.maximum(np.abs(rr).reshape(B, -1).max(1), 1e-12)
                diff[op] = max(diff.get(op, 0.0), float(e.max()))
    info = srv.info()
    srv.close(force=True)
    return {"workload": "requests for chain7 / humanoid / 32 random trees (3-64 bodies), ops rnea, crba, aba, "
                        "rnea-gradient uniform, 1-4096 instances log-uniform; replayed natively; latency = "
                        "host-seen completion - arrival",
            "saturation_req_per_s": sat_req, "saturation_evals_per_s": sat_inst, "points": points,
            "latency_floor": floor,
            "solo": {"what": "each of the 256 pool requests alone", "p50_us": float(np.percentile(solo, 50)),
                     "p99_us": float(np.percentile(solo, 99)),
                     "p50_by_op_us": {op: float(np.median([solo[k] for k in range(len(pool)) if pool[k][1] == op]))
                                      for op in SERVE_OPS}},
            "max_rel_diff_vs_batched": diff, "checked_requests": checked,
            "kernel_launches": info["kernel_launches"], "resident_ctas": info["resident_ctas"],
            "device_status": info["device_status"], "completed": info["completed"],
            "idle_exit_ms": 20.0}


def concurrent_groups(ops):
    """One stream per op of the step, the ABA and its adjoint (which reads
    the ABA's output) on one."""
    groups, rest = [], list(ops)
    if "aba" in rest and "aba_vjp" in rest:
        groups.append(["aba", "aba_vjp"])
        rest = [o for o in rest if o not in ("aba", "aba_vjp")]
    return groups + [[o] for o in rest]


SWEEP_B = [1, 4, 16, 64, 256, 1024, 4096, 16384, 1 << 16, 1 << 18, 1 << 20]


def batch_sweep(fx, device, flush):
    """Throughput against batch size (the shape of the paper's Fig. 2) for the
    chain's and the humanoid's six-op steps: kernel time (the step's public
    calls captured once as a CUDA graph and replayed, CUDA events, L2 flushed
    between replays), the same graph with each independent op on its own
    stream (small batches leave most SMs idle, so the ops then run side by
    side), end to end with that graph replayed between the copies, the calls issued one by one (CUDA events between them),
    the host time to issue one public call (Python binding + C ABI + launch,
    no synchronisation), and end to end through the public API (the inputs,
    one pinned [rows][B] block, copied in with one copy; the six calls; the
    outputs, views of one device buffer, copied back with one copy;
    synchronised; host clock). Medians over the repetitions."""
    import torch

    import gen
    res = {"workload": "six-op steps of the 7-DoF chain (FK+J, RNEA, CRBA+LTDL, ABA, RNEA-VJP, ABA-VJP) and the "
                       "humanoid (bias in place of RNEA) at each batch size; evals = 6 x B per step",
           "statistic": "median over repetitions", "launches": 0}
    for name, robot, ops, bmax in (("chain7", gen.chain7(0), OPS, 1 << 20),
                                   ("humanoid", gen.humanoid(0), HUMANOID_OPS, 1 << 18)):
        model = fx.Model.from_robot(robot)
        rows = []
        for B in [b for b in SWEEP_B if b <= bmax]:
            host, dev0 = make_inputs(robot, B, 4004, device)
            # inputs and outputs each one [rows][B] block: one copy in, one copy out
            keys = list(host)
            nrow = [host[k].shape[0] for k in keys]
            hin = torch.cat([host[k] for k in keys]).pin_memory()
            din = hin.to(device)
            dev, r0 = {}, 0
            for k, r in zip(keys, nrow):
                dev[k] = din[r0:r0 + r]
                r0 += r
            del dev0
            step = Step(fx, model, robot, dev, device, ops, flat=True)
            reps = 200 if B <= 4096 else (40 if B <= (1 << 16) else 12)
            g_ms, g_l, _, _, why = time_graph(step, reps, 3, flush, 1, None)
            # the same calls with every independent op on its own stream (the
            # ABA adjoint reads the ABA's output, so the two share one)
            c_ms, c_l, _, _, _ = time_graph(step, reps, 3, flush, 1, None, groups=concurrent_groups(ops))
            e_ms, _, e_l, _, _ = time_step(step, reps, 3, flush, 1, None)
            res["launches"] += (g_l or 0) + (c_l or 0) + e_l
            torch.cuda.synchronize()
            host_us = []
            for _ in range(reps):
                t0 = time.perf_counter()
                step.run()
                host_us.append((time.perf_counter() - t0) * 1e6 / len(ops))
                torch.cuda.synchronize()
            res["launches"] += reps * step.kernels
            # the outputs of the step's ops lie in one span of the flat buffer
            outk = [k for n in ops for k in OUT_OF[n]]
            spans = [(step.out[k].data_ptr() - step.flat_out.data_ptr()) // 4 for k in outk]
            lo = min(spans)
            hi = max(sp + step.out[k].numel() for sp, k in zip(spans, outk))
            dspan = step.flat_out[lo:hi]
            hout = torch.empty(hi - lo, dtype=torch.float32).pin_memory()
            e2e_us = []
            for _ in range(reps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                din.copy_(hin, non_blocking=True)
                step.run()
                hout.copy_(dspan, non_blocking=True)
                torch.cuda.synchronize()
                e2e_us.append((time.perf_counter() - t0) * 1e6)
            res["launches"] += reps * step.kernels
            # end to end again, the six calls replayed as the concurrent graph
            # between the two copies (the public calls captured once, as a
            # caller issuing the same batch shape every cycle would)
            ge2e_us = []
            gstreams = [torch.cuda.Stream() for _ in concurrent_groups(ops)]
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                step.run_groups(gstreams, concurrent_groups(ops))
            torch.cuda.current_stream().wait_stream(side)
            torch.cuda.synchronize()
            ge = torch.cuda.CUDAGraph()
            try:
                with torch.cuda.graph(ge):
                    step.run_groups(gstreams, concurrent_groups(ops))
            except Exception:  # noqa: BLE001 - the row then has no graph figure
                ge = None
                torch.cuda.synchronize()
            if ge is not None:
                for _ in range(reps):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    din.copy_(hin, non_blocking=True)
                    ge.replay()
                    hout.copy_(dspan, non_blocking=True)
                    torch.cuda.synchronize()
                    ge2e_us.append((time.perf_counter() - t0) * 1e6)
                res["launches"] += (reps + 1) * step.kernels
            ev = len(ops) * B
            e2e = statistics.median(e2e_us)
            ge2e = statistics.median(ge2e_us) if ge2e_us else None
            rows.append({"B": B, "reps": reps,
                         "kernel_us": g_ms * 1e3 if g_ms is not None else None,
                         "kernel_evals_per_s": ev / (g_ms / 1e3) if g_ms is not None else None,
                         "graph": why or "replayed",
                         "concurrent_us": c_ms * 1e3 if c_ms is not None else None,
                         "concurrent_evals_per_s": ev / (c_ms / 1e3) if c_ms is not None else None,
                         "eager_us": e_ms * 1e3, "eager_evals_per_s": ev / (e_ms / 1e3),
                         "host_us_per_call": statistics.median(host_us),
                         "e2e_us": e2e, "e2e_evals_per_s": ev / (e2e / 1e6),
                         "e2e_graph_us": ge2e, "e2e_graph_evals_per_s": ev / (ge2e / 1e6) if ge2e else None,
                         "h2d_bytes": hin.numel() * 4, "d2h_bytes": hout.numel() * 4})
            del step, dev, host, hin, din, hout, dspan, ge, gstreams
        res[name] = rows
    return res


TREE_PATH_B = [64, 512, 4096, 8192, 16384, 1 << 15, 1 << 18]


def tree_paths(fx, device, flush):
    """The humanoid's FK + Jacobians, RNEA, bias forces, CRBA + LTDL, ABA and both adjoints on both tree
    paths, one thread per instance and four lanes per instance (lane groups),
    at batch sizes from 64 to 2^18: each op captured alone as a CUDA graph and
    replayed (kernel time only, CUDA events, L2 flushed between replays),
    median."""
    import gen
    robot = gen.humanoid(0)
    model = fx.Model.from_robot(robot)
    rows, launches = [], 0
    try:
        for B in TREE_PATH_B:
            _, dev = make_inputs(robot, B, 4005, device)
            reps = 100 if B <= 4096 else 30
            for op in ("fk_jac", "rnea", "bias", "crba_ltdl", "aba", "rnea_vjp", "aba_vjp"):
                row = {"B": B, "op": op}
                for path in ("thread", "lane_group"):
                    model.set_tree_path(path)
                    step = Step(fx, model, robot, dev, device, [op])
                    ms, n, _, _, why = time_graph(step, reps, 3, flush, 1, None)
                    launches += n or 0
                    row[f"{path}_us"] = ms * 1e3 if ms is not None else None
                    row[f"{path}_evals_per_s"] = B / (ms / 1e3) if ms is not None else None
                    del step
                rows.append(row)
            del dev
    finally:
        model.set_tree_path("auto")
    return {"workload": "humanoid (root + 29 revolute), FK+J / RNEA / bias / CRBA+LTDL / ABA / RNEA-VJP / ABA-VJP at each batch size "
                        "on both tree paths",
            "rows": rows, "launches": launches}


def fp32_probe(fx, device, phys):
    """The FP32 rate a kernel of independent FMA chains attains here (scalar
    FFMA and the packed two-lane form), best of five 10 ms launches, with the
    SM clock sampled meanwhile."""
    import torch
    blocks = SM_COUNT * 8
    sink = torch.empty(blocks * 256, dtype=torch.float32, device=device)
    clocks = ClockSampler(phys)
    out = {}
    clocks.start()
    time.sleep(0.2)
    for packed in (False, True):
        fx.frax_fp32_probe(packed, blocks, 2000, sink)
        best = 0.0
        for _ in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fl = fx.frax_fp32_probe(packed, blocks, 50000, sink)
            b.record()
            torch.cuda.synchronize()
            best = max(best, fl / (a.elapsed_time(b) / 1e3) / 1e12)
        out["packed_tflops" if packed else "scalar_tflops"] = best
    out["clocks"] = clocks.stop()
    out["kernel"] = "frax_fp32_probe: 152 x 8 blocks of 256 threads, 8 independent FMA chains per thread"
    return out


# ---------------------------------------------------------------- main arms
def reference_arm(args, rank, world):
    if rank != 0:
        return
    base = run_cpu_baseline(min(30.0, args.cpu_seconds * 2))
    base["cpu_model"] = cpu_model()
    line = {"impl": "reference", "metric": METRIC, "value": base["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "7-DoF revolute chain (seed 0), 2^20 instances, FK+J/RNEA/CRBA+LTDL/ABA/"
                                   "RNEA-VJP/ABA-VJP", "global_batch": 1 << 20, "parallelism": "replicas"},
            "cpu_baseline": base,
            "e2e": {"value": base["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


OUT_OF = {"fk_jac": ("pose", "J"), "rnea": ("tau",), "bias": ("tau",), "crba_ltdl": ("M", "LD"), "aba": ("qdd",),
          "aba_sweep": ("qdd",),
          "rnea_vjp": ("rq", "rqd", "rqdd"), "aba_vjp": ("aq", "aqd", "at")}


def copy_ceiling(device, nbytes=1 << 30):
    """This box's pinned host <-> device copy rates (GB/s, best of three 1 GiB
    copies each way, CUDA events): the ceiling of a copy-bound end-to-end
    step."""
    import torch
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device=device)
    out = {}
    for name, dst, src in (("h2d_gbs", d, h), ("d2h_gbs", h, d)):
        best = 0.0
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            dst.copy_(src, non_blocking=True)
            b.record()
            torch.cuda.synchronize()
            best = max(best, nbytes / (a.elapsed_time(b) / 1e3) / 1e9)
        out[name] = best
    del h, d
    return out


def e2e_pipeline(fx, model, robot, host, dev, step, device, steps, world, dist):
    import torch
    cs = torch.cuda.current_stream(device)
    hs, ds = torch.cuda.Stream(device), torch.cuda.Stream(device)
    pin = {k: v.pin_memory() for k, v in host.items()}
    devs = [dev, {k: torch.empty_like(v) for k, v in dev.items()}]
    stps = [step, Step(fx, model, robot, devs[1], device, step.ops)]
    outs_h = [{k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in st.out.items()} for st in stps]
    h2d = sum(v.numel() * 4 for v in pin.values())
    d2h = sum(v.numel() * 4 for v in outs_h[0].values())
    in_free = [torch.cuda.Event(), torch.cuda.Event()]
    out_free = [torch.cuda.Event(), torch.cuda.Event()]
    for e in in_free + out_free:
        e.record(cs)
    n = max(4, min(steps, 20))
    launches = 0

    def one(k):
        nonlocal launches
        b = k % 2
        with torch.cuda.stream(hs):
            hs.wait_event(in_free[b])
            for key in devs[b]:
                devs[b][key].copy_(pin[key], non_blocking=True)
            ready = torch.cuda.Event()
            ready.record(hs)
        cs.wait_event(ready)
        cs.wait_event(out_free[b])
        for name, fn in stps[b].launches:
            fn()
            launches += 1
            done = torch.cuda.Event()
            done.record(cs)
            ds.wait_event(done)
            with torch.cuda.stream(ds):
                for key in OUT_OF[name]:
                    outs_h[b][key].copy_(stps[b].out[key], non_blocking=True)
        in_free[b].record(cs)
        out_free[b].record(ds)

    for k in range(2):
        one(k)
    torch.cuda.synchronize()
    launches = 0
    t0 = time.perf_counter()
    for k in range(n):
        one(k)
    torch.cuda.synchronize()
    el = (time.perf_counter() - t0) / n
    tt = torch.tensor([el], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    res = {"value": world * len(step.ops) * step.B / float(tt.item()), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": float(tt.item()) * 1e3, "steps": n, "launches": launches,
            "pipelining": "H2D, kernels and per-op D2H on three streams, double-buffered"}
    ceil = copy_ceiling(device)
    res["copy_ceiling"] = ceil
    # the step's D2H bytes at this box's D2H rate: the least time a step can take
    res["frac_of_copy_ceiling"] = (d2h / (ceil["d2h_gbs"] * 1e9)) / float(tt.item())
    return res


def frax_arm(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist

    import gen
    import paper_2604_04310_gb300 as fx

    device = torch.device("cuda", local_rank)
    torch.cuda.set_device(device)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)  # > L2 (129 MB)
    peak = fp32_peak_tflops(2070.0)
    phys = local_rank
    if "CUDA_VISIBLE_DEVICES" in os.environ and os.environ["CUDA_VISIBLE_DEVICES"]:
        phys = int(os.environ["CUDA_VISIBLE_DEVICES"].split(",")[local_rank])

    # main workload: the 7-DoF chain, 2^20 instances per GPU, the whole path
    robot = gen.chain7(0)
    B = args.batch
    model = fx.Model.from_robot(robot)
    host, dev = make_inputs(robot, B, 1001 + rank, device)
    step = Step(fx, model, robot, dev, device, OPS)
    clocks = ClockSampler(phys)
    # per op: the calls one by one with CUDA events between them; the step
    # itself: the same calls replayed as one CUDA graph
    step_ms, per_op_ms, launches, wall, clk = time_step(step, args.steps, args.warmup, flush, world, dist,
                                                        clocks if args.eager else None)
    launch_mode = "eager: one public call per op"
    graph_one_stream = None
    if not args.eager:
        # the step's calls as one CUDA graph; the memory-bound ops (FK+J, CRBA)
        # on a second stream beside the ALU-bound ones unless --one-stream
        side_ops = () if args.one_stream else HBM_OPS
        g_ms, g_launches, g_wall, g_clk, why = time_graph(step, args.steps, args.warmup, flush, world, dist, clocks,
                                                          side_ops)
        if g_ms is not None:
            step_ms, launches, wall, clk = g_ms, g_launches, g_wall, g_clk
            launch_mode = "the step's public calls captured once as a CUDA graph and replayed" + (
                "; FK+J and CRBA+LTDL (memory-bound) on a second stream beside the four ALU-bound ops"
                if side_ops else "")
            if side_ops:
                o_ms, o_l, _, _, _ = time_graph(step, args.steps, args.warmup, flush, world, dist, None)
                launches += o_l or 0
                graph_one_stream = {"ms_per_step": o_ms, "evals_per_s": len(OPS) * B / (o_ms / 1e3)} \
                    if o_ms is not None else None
        else:
            launch_mode += f" (graph capture failed: {why})"
    ms_per_step, value = whole_job(step_ms, len(OPS) * B, world, dist, device)
    hbm, hbm_src = measured_hbm_gbs()
    per_op = roofline_of(per_op_ms, FLOPS["chain7"], B, peak, hbm, robot)
    per_op["aba"]["method"] = ("forward dynamics through the mass-matrix factor (RNEA bias + CRBA + L^T D L solves), "
                               "what frax_aba runs on the 7-body chain; next_rows.chain7.aba_sweep times the O(n) "
                               "articulated-body sweeps")
    dom = max(OPS, key=lambda n: per_op_ms[n])
    d = per_op[dom]
    if d["bound"] == "alu":
        roofline = {"bound": "alu", "kernel": dom, "achieved": d["tflops"], "peak": peak, "unit": "TFLOP/s",
                    "frac": d["frac_fp32_peak"],
                    "peak_basis": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz max SM clock (recipe unit counts)"}
    else:
        roofline = {"bound": "hbm", "kernel": dom, "achieved": d["gbs"], "peak": hbm, "unit": "GB/s",
                    "frac": d["frac_hbm_peak"], "peak_basis": f"{hbm_src} HBM copy bandwidth"}
    roofline["traffic"] = NCU_TRAFFIC.get(dom)

    # end to end through the public API with pinned host buffers: every step
    # copies its inputs in (H2D stream) and every output back (D2H stream,
    # each op's outputs as soon as that op is done), double-buffered so the
    # copies of one step overlap the kernels of the next
    e2e = None
    if not args.no_e2e:
        # three repeats of the pipelined run, the median reported (single runs
        # have come out at 5.8 or, on some boxes, about 10 ms per step)
        reps = [e2e_pipeline(fx, model, robot, host, dev, step, device, args.steps, world, dist) for _ in range(3)]
        launches += sum(r.pop("launches") for r in reps)
        e2e = sorted(reps, key=lambda r: r["ms_per_step"])[1]
        e2e["repeats_ms_per_step"] = [r["ms_per_step"] for r in reps]
        e2e["statistic"] = "median of 3 repeats of the pipelined run"
        e2e["frac_of_copy_ceiling"] = (e2e["d2h_bytes_per_step"] / (e2e["copy_ceiling"]["d2h_gbs"] * 1e9)) / (
            e2e["ms_per_step"] / 1e3)
    del step, dev, host

    # second workload: the floating-base humanoid (30 bodies, nv = 35), 2^18
    humanoid = None
    if not args.no_humanoid:
        hrobot = gen.humanoid(0)
        hB = args.humanoid_batch
        hmodel = fx.Model.from_robot(hrobot)
        _, hdev = make_inputs(hrobot, hB, 2002 + rank, device)
        hops = ["fk_jac", "bias", "crba_ltdl", "aba", "rnea_vjp", "aba_vjp"]
        hstep = Step(fx, hmodel, hrobot, hdev, device, hops)
        hsteps = max(20, args.steps // 4)
        hms, hper, hl, _, _ = time_step(hstep, hsteps, max(3, args.warmup), flush, world, dist)
        launches += hl
        # the same six calls captured once as a CUDA graph, the two memory-bound
        # ones on a second stream beside the ALU-bound ones (as the chain's step)
        gms, gl, _, _, gwhy = time_graph(hstep, hsteps, max(3, args.warmup), flush, world, dist, None, HBM_OPS)
        launches += gl or 0
        humanoid = {"workload": "floating-base humanoid (root + 29 revolute, seed 0), 2^18 instances; FK + 4 "
                                "end-frame Jacobians, bias forces, CRBA + LTDL, ABA, RNEA-VJP, ABA-VJP",
                    "batch": hB, "steps": hsteps, "ms_per_step": hms, "statistic": "median over steps",
                    "launch": "eager: one public call per op, CUDA events between them",
                    "evals_per_s": world * len(hops) * hB / (hms / 1e3),
                    "graph": ({"ms_per_step": gms, "evals_per_s": world * len(hops) * hB / (gms / 1e3),
                               "launch": "the six calls captured once as a CUDA graph and replayed; FK+J and "
                                         "CRBA+LTDL on a second stream"} if gms is not None
                              else {"unavailable": gwhy}),
                    "per_op": roofline_of(hper, FLOPS["humanoid"], hB, peak, hbm, hrobot)}
        del hstep, hdev

    # further rows on the same two robots: operational-space control of the
    # last end frame, and RNEA / ABA with external forces on every body;
    # chain at 2^20, humanoid at 2^18
    nxt = None
    if not args.no_next:
        nxt = {"workload": "operational-space control tau = J^T Lambda (xdd - Jdot qd) + c + g for the last end "
                           "frame (xdd uniform in [-3, 3]); for the chain, forward dynamics by the O(n) "
                           "articulated-body sweeps (aba_sweep, frax_aba_articulated) beside frax_aba's factor "
                           "solve; RNEA and ABA with standard-normal external spatial "
                           "forces on every body; JVPs of FK (end frames), RNEA and ABA along standard-normal "
                           "directions (the ABA JVP at the input qdd as saved forward result); 7-DoF chain 2^20, "
                           "humanoid 2^18 instances"}
        for oname, orobot, oB in (("chain7", gen.chain7(0), B), ("humanoid", gen.humanoid(0), args.humanoid_batch)):
            omodel = fx.Model.from_robot(orobot)
            _, odev = make_inputs(orobot, oB, 3003 + rank, device)
            rng = np.random.default_rng(3004 + rank)
            odev["xdd"] = torch.from_numpy(rng.uniform(-3, 3, (6, oB)).astype(np.float32)).to(device)
            odev["fext"] = torch.from_numpy(rng.standard_normal((6 * orobot.n_bodies, oB), np.float32)).to(device)
            for k in ("dq", "dqd", "dx"):
                odev[k] = torch.from_numpy(rng.standard_normal((orobot.nv, oB), np.float32)).to(device)
            oops = ["osc", "rnea_ext", "aba_ext", "fk_jvp", "rnea_jvp", "aba_jvp"]
            if oname == "chain7":  # the O(n) articulated-body sweeps beside the factor solve frax_aba runs
                oops.append("aba_sweep")
            ostep = Step(fx, omodel, orobot, odev, device, oops, task=OSC_TASK[oname])
            osteps = max(20, args.steps // 4)
            oms, oper, ol, _, _ = time_step(ostep, osteps, max(3, args.warmup), flush, world, dist)
            launches += ol
            nxt[oname] = {"osc_task_body": OSC_TASK[oname], "batch": oB, "steps": osteps,
                          "per_op": roofline_of(oper, FLOPS[oname], oB, peak, hbm, orobot)}
            del ostep, odev

    # serial-chain FK: the thread-per-instance loop vs the warp-level SE(3)
    # prefix scan, on a 64-body chain at a small and a large batch
    if nxt is not None:
        srobot = gen.serial_chain(5, 64)
        smodel = fx.Model.from_robot(srobot)
        nxt["fk_scan"] = {"workload": "64-body serial chain (seed 5): frax_fk (sequential loop per thread) vs "
                                      "frax_fk_scan (prefix product over SE(3), one warp per instance)"}
        for sB in (256, 1 << 16):
            _, sdev = make_inputs(srobot, sB, 3005 + rank, device)
            sstep = Step(fx, smodel, srobot, sdev, device, ["fk", "fk_scan"])
            _, sper, sl, _, _ = time_step(sstep, 50, 5, flush, world, dist)
            launches += sl
            nxt["fk_scan"][f"B{sB}"] = {"fk_us": sper["fk"] * 1e3, "fk_scan_us": sper["fk_scan"] * 1e3}
            del sstep, sdev

    sweep = paths = None
    if not args.no_sweep:
        sweep = batch_sweep(fx, device, flush)
        launches += sweep.pop("launches")
        paths = tree_paths(fx, device, flush)
        launches += paths.pop("launches")

    # the FP32 rate a kernel of independent FMA chains attains: each ALU-bound
    # op's rate is also given as a fraction of it (scalar and packed)
    probe = fp32_probe(fx, device, phys)
    launches += 12
    tables = [per_op] + ([humanoid["per_op"]] if humanoid else []) + \
        ([nxt[k]["per_op"] for k in ("chain7", "humanoid")] if nxt else [])
    for tab in tables:
        for r in tab.values():
            r["frac_of_measured_fp32_scalar"] = r["tflops"] / probe["scalar_tflops"]
            r["frac_of_measured_fp32_packed"] = r["tflops"] / probe["packed_tflops"]
    if roofline["bound"] == "alu":
        roofline["frac_of_measured_fp32_scalar"] = roofline["achieved"] / probe["scalar_tflops"]
        roofline["frac_of_measured_fp32_packed"] = roofline["achieved"] / probe["packed_tflops"]

    serve = None
    if rank == 0 and not args.no_serve:
        serve = serve_stream(fx, args.serve_seconds)

    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = run_cpu_baseline(args.cpu_seconds)
        cpu["cpu_model"] = cpu_model()
        hcpu = run_cpu_baseline(args.cpu_seconds, "humanoid")
        cpu["humanoid"] = {k: hcpu.get(k) for k in ("value", "per_op", "sample")}
        cpu_all = run_cpu_baseline_all_cores(min(8.0, args.cpu_seconds))
        hall = run_cpu_baseline_all_cores(min(8.0, args.cpu_seconds), "humanoid")
        cpu_all["humanoid"] = {k: hall.get(k) for k in ("value", "per_op", "sample")}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "statistic": "median over steps",
                "config": {"workload": "7-DoF revolute chain (seed 0), 2^20 instances per GPU; one step = "
                                       "FK+EE Jacobian, RNEA, CRBA+LTDL, ABA, RNEA-VJP, ABA-VJP",
                           "global_batch": B * world, "parallelism": f"replicas x{world}",
                           "l2": "256 MB buffer written between steps (L2 flush)", "launch": launch_mode},
                "clocks": clk, "gpu_launches": launches, "wall_s": wall, "per_op": per_op, "roofline": roofline,
                "graph_one_stream": graph_one_stream,
                "e2e": e2e, "humanoid": humanoid, "next_rows": nxt, "batch_sweep": sweep, "tree_paths": paths,
                "fp32_peak_measured": probe, "cpu_baseline": cpu,
                "cpu_baseline_all_cores": cpu_all, "serving": serve}
        print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="frax", choices=["frax", "reference"])
    ap.add_argument("--batch", type=int, default=1 << 20)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-humanoid", action="store_true")
    ap.add_argument("--no-next", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--eager", action="store_true", help="time the step as separate calls, not a CUDA graph")
    ap.add_argument("--one-stream", action="store_true", help="capture every call of the step on one stream")
    ap.add_argument("--humanoid-batch", type=int, default=1 << 18)
    ap.add_argument("--count-flops", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--cpu-baseline-child", action="store_true")
    ap.add_argument("--cpu-robot", default="chain7", choices=["chain7", "humanoid"])
    args = ap.parse_args()
    if args.cpu_baseline_child:
        cpu_baseline_child(args)
        return
    if args.count_flops:
        count_flops()
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    frax_arm(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
