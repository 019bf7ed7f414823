// Internal launcher interface between the C ABI (api.cu) and the kernel
// translation units (one per topology family, compiled in parallel).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/frax.h"
#include "model.h"

namespace frax {

enum Op { kOpFk = 0, kOpJac, kOpRnea, kOpCrba, kOpAba, kOpRneaVjp, kOpAbaVjp, kOpLtdlSolve, kOpLtdlInverse,
          kOpOsc, kOpRneaExt, kOpAbaExt, kOpFkJvp, kOpRneaJvp, kOpAbaJvp,
          kOpAbaSweep,  // forward dynamics by the articulated-body sweeps whatever the topology
          kOpCount };

struct FramesArg {
  int n;
  int body[8];
};

// Rows (entries of an SoA output) to be zeroed: rows [0, n0) of the first
// array, [n0, n) of the second. Sized for M and the packed factor of the
// largest model (69 x 69 + 69 x 70 / 2 entries).
constexpr int kMaxZeroRows = kMaxDofs * kMaxDofs + kMaxDofs * (kMaxDofs + 1) / 2;
struct ZeroRows {
  int32_t n0 = 0, n = 0;
  uint16_t row[kMaxZeroRows];
};

struct OpArgs {
  int64_t B = 0, ld = 0;
  const float* q = nullptr;
  const float* qd = nullptr;
  const float* qdd = nullptr;
  const float* tau = nullptr;
  const float* gbar = nullptr;
  const float* in_LD = nullptr;
  const float* in_xdd = nullptr;  // task accelerations (kOpOsc)
  const float* in_fext = nullptr;  // external forces (kOpRneaExt, kOpAbaExt)
  const float* in_dq = nullptr;    // JVP directions: dq, dqd, and dqdd or dtau
  const float* in_dqd = nullptr;
  const float* in_dx = nullptr;
  float* out0 = nullptr;  // pose / tau / M / qdd / qbar
  float* out1 = nullptr;  // J / LD / qdbar / Lambda
  float* out2 = nullptr;  // qddbar / taubar
  FramesArg frames{0, {0}};  // kOpOsc: body[0] is the task body
  const ZeroRows* zeros = nullptr;  // kOpCrba on trees: structural zeros the kernel writes
  int tree_path = 0;  // FRAX_TREE_PATH_*: trees of up to 32 bodies, the lane-group kernels or not
  cudaStream_t stream = nullptr;
};

cudaError_t launch_zero_rows(const ZeroRows& z, float* base0, float* base1, int64_t ld, int64_t B,
                             cudaStream_t stream);

// Each returns the launch status (cudaGetLastError after the launch).
cudaError_t launch_chain7(const HostModel& m, Op op, const OpArgs& a);
cudaError_t launch_tree32(const HostModel& m, Op op, const OpArgs& a);
cudaError_t launch_tree64(const HostModel& m, Op op, const OpArgs& a);
// serial chains, one warp per instance (prefix product over SE(3))
cudaError_t launch_fk_scan(const HostModel& m, const OpArgs& a);

constexpr int kBlock = 128;

}  // namespace frax
