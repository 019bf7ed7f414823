"""GPU serial-chain FK by the warp-level SE(3) prefix scan (frax_fk_scan) vs
the FP64 oracle and vs the thread-per-instance frax_fk, on chains of 7, 32,
33 and 64 bodies, fixed or floating base. Tolerance 1e-4 (poses; long chains
compose up to 64 FP32 rotations either way)."""

import numpy as np
import pytest
import torch

import gen
import paper_2604_04310_gb300 as fx
from oracle import rbd
from tests.gpu_util import dev, host
from tests.pins import normwise

pytestmark = pytest.mark.gpu

CHAINS = [gen.chain7(0), gen.serial_chain(3, 32), gen.serial_chain(4, 33), gen.serial_chain(5, 64),
          gen.serial_chain(6, 64, free_root=True), gen.serial_chain(7, 1)]


@pytest.mark.parametrize("robot", CHAINS, ids=lambda r: r.name)
@pytest.mark.parametrize("B", [1, 5, 300])
def test_fk_scan_matches_oracle_and_fk(robot, B):
    m = fx.Model.from_robot(robot)
    s = gen.draw_states(robot, B, 141).as_f32()
    q = dev(s.q)
    pose = fx.frax_fk_scan(m, q)
    assert normwise(host(pose), rbd.fk_flat(robot, s.q)) < 1e-4
    assert normwise(host(pose), host(fx.frax_fk(m, q))) < 1e-4


def test_fk_scan_ld_and_errors():
    robot = gen.serial_chain(8, 40)
    m = fx.Model.from_robot(robot)
    B, ld = 77, 101
    s = gen.draw_states(robot, B, 142).as_f32()
    pose = fx.frax_fk_scan(m, dev(s.q, ld))
    assert pose.stride(0) == ld
    assert normwise(host(pose), rbd.fk_flat(robot, s.q)) < 1e-4
    tree = fx.Model.from_robot(gen.random_tree(101))
    with pytest.raises(fx.FraxError, match="serial chain"):
        fx.frax_fk_scan(tree, torch.zeros((tree.nq, 4), device="cuda"))
    assert fx.frax_fk_scan(m, torch.empty((m.nq, 0), device="cuda")).shape == (12 * 40, 0)
