"""Shared helpers for the GPU parity tests: move seeded states to the device
in the ABI's SoA layout and read results back."""

import numpy as np
import torch

import gen


def dev(x_bk: np.ndarray, ld: int | None = None) -> torch.Tensor:
    """(B, k) FP64 -> (k, B) FP32 CUDA tensor, stride (ld, 1)."""
    soa = gen.to_soa(x_bk, ld)
    t = torch.from_numpy(soa).cuda()
    return t[:, : x_bk.shape[0]]


def host(t: torch.Tensor) -> np.ndarray:
    """(k, B) CUDA tensor -> (B, k) FP64."""
    return t.detach().cpu().double().numpy().T.copy()


def states(model, B, seed, ld=None):
    """FP32-rounded states (FP64 arrays) and their device copies."""
    s = gen.draw_states(model, B, seed).as_f32()
    d = {k: dev(getattr(s, k), ld) for k in ("q", "qd", "qdd", "tau")}
    return s, d
