// Structural zeros of the batched Jacobians. The tree's sparsity pattern is
// the same for every instance: a Jacobian column vanishes off the frame's
// ancestors. In the SoA layout each such entry is a whole row of B floats, so
// one bandwidth kernel writes them (coalesced streaming stores, one block row
// per entry) and the per-instance kernel skips them. (M's and the factor's
// zeros, M_ij and L_ij for pairs where neither body is an ancestor of the
// other, are written by the CRBA kernel's own threads after their sweeps:
// measured faster than a separate fill there, slower here.)
#include "launch.h"

namespace frax {

__global__ void __launch_bounds__(256) k_zero_rows(const __grid_constant__ ZeroRows z, float* base0, float* base1,
                                                   int64_t ld, int64_t B) {
  const int r = blockIdx.y;
  float* p = (r < z.n0 ? base0 : base1) + int64_t(z.row[r]) * ld;
  for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < B; k += int64_t(gridDim.x) * blockDim.x)
    __stcs(p + k, 0.f);
}

cudaError_t launch_zero_rows(const ZeroRows& z, float* base0, float* base1, int64_t ld, int64_t B,
                             cudaStream_t stream) {
  if (z.n == 0 || B == 0) return cudaSuccess;
  // about 8 K floats per block: enough blocks to fill the GPU for any row count
  const int64_t per_block = 256 * 32;
  const unsigned gx = unsigned((B + per_block - 1) / per_block);
  k_zero_rows<<<dim3(gx, unsigned(z.n)), 256, 0, stream>>>(z, base0, base1, ld, B);
  return cudaGetLastError();
}

}  // namespace frax
