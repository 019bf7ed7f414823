"""The FP32 peak probe: the rate it reports is only meaningful if each launch
does the fused multiply-adds it claims. Every thread's stored sum is checked
against the same FMA chains run in numpy (each step rounded to FP32), so a
dropped or extra iteration, a lost chain or a wrong lane fails."""

import numpy as np
import pytest
import torch

import paper_2604_04310_gb300 as fx

pytestmark = pytest.mark.gpu

BLOCK, CHAINS = 256, 8
A, B = np.float32(0.999999), np.float32(1e-6)


def _fma32(x, a, b):
    """fp32 fused multiply-add: the product of two fp32 values is exact in
    fp64, so one rounding to fp32 after the fp64 sum (itself nearly always
    exact here) is the fused result."""
    return (x.astype(np.float64) * np.float64(a) + np.float64(b)).astype(np.float32)


def _expected(blocks, iters, packed):
    tid = np.arange(blocks * BLOCK)
    t = (tid & 7).astype(np.float64)
    lanes = []
    for k in range(CHAINS):
        x0 = (np.float64(np.float32(1e-3)) * t + k).astype(np.float32)
        lanes.append([x0, np.full_like(x0, np.float32(0.5 * k))] if packed else [x0])
    for _ in range(iters):
        lanes = [[_fma32(x, A, B) for x in chain] for chain in lanes]
    s = np.zeros(blocks * BLOCK, np.float32)
    for chain in lanes:
        s = s + (chain[0] + chain[1] if packed else chain[0])
    return s


@pytest.mark.parametrize("packed", [False, True])
def test_probe_does_the_work_it_counts(packed):
    blocks, iters = 6, 1500
    sink = torch.full((blocks * BLOCK,), float("nan"), device="cuda")
    flops = fx.frax_fp32_probe(packed, blocks, iters, sink)
    torch.cuda.synchronize()
    assert flops == blocks * BLOCK * iters * CHAINS * (4 if packed else 2)
    got = sink.cpu().numpy()
    want = _expected(blocks, iters, packed)
    assert np.isfinite(got).all()
    # one iteration fewer moves every thread's sum by 6e-7 of itself or more,
    # above the few fp32 ulps by which a starting value's rounding may differ
    rtol = 2.5e-7
    np.testing.assert_allclose(got, want, rtol=rtol, atol=0)
    fewer = _expected(blocks, iters - 1, packed)
    assert (np.abs(fewer - want) > rtol * np.abs(want)).all()
