"""The bench's headline launch configuration: the step's six public calls
captured once as a CUDA graph, the two memory-bound ones on a second stream
inside the capture, and replayed. Every output of the replay must equal, bit
for bit, what the same calls write when issued one by one (which the parity
tests compare with the FP64 oracle), for the chain at the bench's full batch
and for the humanoid."""

import os
import sys

import pytest
import torch

import gen
import paper_2604_04310_gb300 as fx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
import bench  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,B", [("chain7", 1 << 20), ("humanoid", 1 << 16)])
def test_replayed_two_stream_graph_matches_eager(name, B):
    robot = gen.chain7(0) if name == "chain7" else gen.humanoid(0)
    ops = bench.OPS if name == "chain7" else bench.HUMANOID_OPS
    device = torch.device("cuda:0")
    model = fx.Model.from_robot(robot)
    _, dev = bench.make_inputs(robot, B, 1001, device)
    step = bench.Step(fx, model, robot, dev, device, ops)
    step.run()
    torch.cuda.synchronize()
    eager = {k: v.clone() for k, v in step.out.items()}
    g = torch.cuda.CUDAGraph()
    fork = torch.cuda.Stream()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # warm-up on a side stream, as the bench does before capture
        step.run_split(fork, set(bench.HBM_OPS))
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        step.run_split(fork, set(bench.HBM_OPS))
    for v in step.out.values():
        v.fill_(float("nan"))
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    written = [k for k in eager if k in {"pose", "J", "tau", "M", "LD", "qdd", "rq", "rqd", "rqdd", "aq", "aqd", "at"}]
    for k in written:
        assert torch.equal(step.out[k], eager[k]), k
