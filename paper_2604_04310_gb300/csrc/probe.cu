// FP32 peak probe: a kernel that does nothing but independent FMA chains, so
// its rate is the FP32 pipe's attainable peak on this GPU at the clock it
// runs at. Scalar FFMA and the packed two-lane form (fma.rn.f32x2, written
// in inline PTX) are measured separately; the kernels here are timed against
// both.
#include <cuda_runtime.h>

#include <string>

#include "handles.h"

namespace frax {
namespace {

constexpr int kProbeBlock = 256;
constexpr int kProbeChains = 8;  // independent accumulators per thread

__device__ __forceinline__ unsigned long long pack2(float x, float y) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ void unpack2(unsigned long long v, float* x, float* y) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(*x), "=f"(*y) : "l"(v));
}
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
  unsigned long long d;
  asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// Each thread: kProbeChains chains of `iters` dependent FMAs, x <- x * a + b
// (|a| < 1 keeps them bounded); the sum is stored so nothing is dropped.
template <bool PACKED>
__global__ void __launch_bounds__(kProbeBlock) k_fp32_probe(float* sink, int iters, float a, float b) {
  const int tid = blockIdx.x * kProbeBlock + threadIdx.x;
  float s = 0.f;
  if constexpr (PACKED) {
    unsigned long long x[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) x[k] = pack2(1e-3f * (tid & 7) + k, 0.5f * k);
    const unsigned long long A = pack2(a, a), Bv = pack2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < kProbeChains; ++k) x[k] = ffma2(x[k], A, Bv);
    }
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) {
      float u, v;
      unpack2(x[k], &u, &v);
      s += u + v;
    }
  } else {
    float x[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) x[k] = 1e-3f * (tid & 7) + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < kProbeChains; ++k) x[k] = fmaf(x[k], a, b);
    }
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) s += x[k];
  }
  sink[tid] = s;
}

}  // namespace
}  // namespace frax

extern "C" frax_status frax_fp32_probe(int packed, int blocks, int iters, float* sink, double* flops,
                                       void* stream) {
  if (blocks < 1 || iters < 1 || !sink)
    return frax::set_error(FRAX_EINVAL, "frax_fp32_probe: blocks, iters >= 1 and a sink are required");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (packed)
    frax::k_fp32_probe<true><<<blocks, frax::kProbeBlock, 0, s>>>(sink, iters, 0.999999f, 1e-6f);
  else
    frax::k_fp32_probe<false><<<blocks, frax::kProbeBlock, 0, s>>>(sink, iters, 0.999999f, 1e-6f);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return frax::set_error(FRAX_ECUDA, std::string("frax_fp32_probe: launch: ") + cudaGetErrorString(e));
  if (flops)
    *flops = double(blocks) * frax::kProbeBlock * double(iters) * frax::kProbeChains * (packed ? 4.0 : 2.0);
  return frax::clear_error();
}
