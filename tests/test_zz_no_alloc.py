"""frax_serve_batch_noalloc, the allocation-free batch entry point, against
the regular entry points (frax_rnea, frax_crba, frax_aba, frax_rnea_vjp) and
against the FP64 oracle on the same inputs, within the parity tolerances, on
two calls in a row. The entry point keeps its scratch in a fixed device array
shared by all calls; the second call uses other inputs and another request
order, so results left in that array by the first call would show up as
mismatches. A call made while its stream is being captured is refused.

Kept in a file that pytest collects last, so a run that stops at the first
failure has already run every other test."""

import numpy as np
import pytest
import torch

import gen
import paper_2604_04310_gb300 as fx
from oracle import derivatives as dv
from oracle import rbd
from tests.gpu_util import dev, host
from tests.pins import normwise

pytestmark = pytest.mark.gpu

ROBOTS = {"chain7": gen.chain7(0), "humanoid": gen.humanoid(0), "tree105": gen.random_tree(105),
          "tree64": gen.random_tree(7, 64)}


def _request(models, name, op, B, seed):
    robot, m = ROBOTS[name], models[name]
    s = gen.draw_states(robot, B, seed).as_f32()
    g = gen.draw_gbar(robot.nv, B, seed + 1)
    q, qd, qdd, tau, gb = dev(s.q), dev(s.qd), dev(s.qdd), dev(s.tau), dev(g)
    e = lambda rows: torch.empty((rows, B), dtype=torch.float32, device="cuda")
    tol = 1e-3 if op in ("aba", "rnea_grad") else 1e-4
    if B == 0:  # an empty request rides along; there is nothing to compare
        nin, rows = {"rnea": (3, [m.nv]), "crba": (1, [m.nv * m.nv]), "aba": (3, [m.nv]),
                     "rnea_grad": (4, [m.nq, m.nv, m.nv])}[op]
        return (m, op, [q, qd, qdd, gb][:nin], [e(r) for r in rows]), ([], []), tol
    gq = g.astype(np.float32).astype(np.float64)
    if op == "rnea":
        ins, outs = [q, qd, qdd], [e(m.nv)]
        ref = [fx.frax_rnea(m, q, qd, qdd)]
        oref = [rbd.rnea(robot, s.q, s.qd, s.qdd)]
    elif op == "crba":
        ins, outs = [q], [e(m.nv * m.nv)]
        ref = [fx.frax_crba(m, q)[0]]
        oref = [rbd.crba(robot, s.q).reshape(B, -1)]
    elif op == "aba":
        ins, outs = [q, qd, tau], [e(m.nv)]
        ref = [fx.frax_aba(m, q, qd, tau)]
        oref = [rbd.aba(robot, s.q, s.qd, s.tau)]
    else:
        ins, outs = [q, qd, qdd, gb], [e(m.nq), e(m.nv), e(m.nv)]
        ref = list(fx.frax_rnea_vjp(m, q, qd, qdd, gb))
        oref = list(dv.rnea_vjp(robot, s.q, s.qd, s.qdd, gq))
    return (m, op, ins, outs), (ref, oref), tol


def _check(models, mix, seed0):
    reqs, refs = [], []
    for k, (name, op, B) in enumerate(mix):
        r, ref, tol = _request(models, name, op, B, seed0 + 10 * k)
        reqs.append(r)
        refs.append((ref, tol, B))
    fx.frax_serve_batch_noalloc(reqs)
    torch.cuda.synchronize()
    for (m, op, ins, outs), ((ref, oref), tol, B) in zip(reqs, refs):
        if not B:
            continue
        for o, rf in zip(outs, ref):  # the regular GPU entry points
            assert normwise(host(o), host(rf)) < tol, (op, B)
        for o, rf in zip(outs, oref):  # the FP64 oracle
            assert normwise(host(o), rf) < tol, (op, B, "oracle")


def test_noalloc_batch_matches_regular_entry_points():
    models = {k: fx.Model.from_robot(r) for k, r in ROBOTS.items()}
    mix1 = [("chain7", "rnea", 300), ("humanoid", "aba", 500), ("tree105", "crba", 129),
            ("humanoid", "rnea_grad", 64), ("tree64", "rnea", 1), ("chain7", "crba", 0),
            ("chain7", "aba", 257), ("tree105", "rnea_grad", 33)]
    _check(models, mix1, 100)
    mix2 = [("tree64", "aba", 77), ("humanoid", "crba", 200), ("chain7", "rnea_grad", 128),
            ("tree105", "rnea", 1000), ("humanoid", "rnea", 3)]
    _check(models, mix2, 500)


def test_noalloc_batch_limits():
    m = fx.Model.from_robot(ROBOTS["chain7"])
    q = torch.zeros((7, 1), device="cuda")
    reqs = [(m, "crba", [q], [torch.zeros((49, 1), device="cuda")])] * 257
    with pytest.raises(fx.FraxError) as e:
        fx.frax_serve_batch_noalloc(reqs)
    assert "256" in str(e.value)
    fx.frax_serve_batch_noalloc([])


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")
def test_noalloc_batch_refused_while_capturing():
    """Under stream capture the call returns FRAX_EINVAL and enqueues nothing,
    so the capture stays valid and ends as an empty graph."""
    m = fx.Model.from_robot(ROBOTS["chain7"])
    q = torch.zeros((7, 4), device="cuda")
    out = torch.zeros((49, 4), device="cuda")
    reqs = [(m, "crba", [q], [out])]
    fx.frax_serve_batch_noalloc(reqs)  # the per-device set-up, before any capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        q2 = torch.zeros((7, 4), device="cuda")
        out2 = torch.zeros((49, 4), device="cuda")
    torch.cuda.synchronize()
    refused = None
    with torch.cuda.graph(g, stream=s):
        try:
            fx.frax_serve_batch_noalloc([(m, "crba", [q2], [out2])])
        except fx.FraxError as e:
            refused = e
    assert refused is not None and refused.status == 1 and "captur" in str(refused)
    torch.cuda.synchronize()
    fx.frax_serve_batch_noalloc(reqs)  # still usable after the refusal
    torch.cuda.synchronize()
