"""Seeded synthetic robots and states.

This package is the one piece shared by the CUDA path's callers (tests, bench,
smoke) and the FP64 oracle. It only draws random numbers and lays them out:
it holds none of the dynamics arithmetic (no transforms, no recursions).

Robots follow the shapes of the paper's workloads (a 7-DoF serial arm like the
Franka Panda and a floating-base humanoid like the Unitree G1, Sec. I and
Sec. IV); their parameters are random because the real robots' URDFs are not
available.
"""

from .models import RobotModel, chain7, humanoid, random_tree, serial_chain, serving_pool
from .states import States, draw_states, draw_gbar, to_soa, from_soa

__all__ = [
    "RobotModel", "chain7", "humanoid", "random_tree", "serial_chain", "serving_pool",
    "States", "draw_states", "draw_gbar", "to_soa", "from_soa",
]
