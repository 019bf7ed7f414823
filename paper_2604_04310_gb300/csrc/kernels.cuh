// __global__ wrappers: one thread per instance, 128-thread blocks, the model
// image as a __grid_constant__ parameter (read through the constant bank).
// The chain kernels' register caps (blocks per SM in __launch_bounds__) were
// chosen by measurement: more resident warps beat the few spills they cause.
#pragma once
#include "dyn.cuh"
#include "seg.cuh"
#include "solve.cuh"
#include "osc.cuh"
#include "ext.cuh"
#include "jvp.cuh"
#include "launch.h"

namespace frax {

#define FRAX_TID()                                                     \
  const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; \
  if (b >= B) return;                                                \
  const Col col{ld, b};

template <class T>
__global__ void __launch_bounds__(kBlock, 8) k_fk(const __grid_constant__ ModelImage<T::NBMAX> M, int64_t B,
                                                int64_t ld, const float* q, float* pose,
                                                const __grid_constant__ Frames fr, float* J) {
  FRAX_TID();
  fk_one<T>(M, q, pose, fr, J, col);
}

template <class T>
__global__ void __launch_bounds__(kBlock, 8) k_rnea(const __grid_constant__ ModelImage<T::NBMAX> M, int64_t B,
                                                  int64_t ld, const float* q, const float* qd,
                                                  const float* qdd, float* tau) {
  FRAX_TID();
  rnea_one<T>(M, q, qd, qdd, tau, col);
}

template <class T>
__global__ void __launch_bounds__(kBlock, 8) k_crba(const __grid_constant__ ModelImage<T::NBMAX> M, int64_t B,
                                                  int64_t ld, const float* q, float* Mout, float* LD) {
  FRAX_TID();
  crba_one<T>(M, q, Mout, LD, col);
}

template <class T>
__global__ void __launch_bounds__(kBlock, 4) k_aba(const __grid_constant__ ModelImage<T::NBMAX> M, int64_t B,
                                                 int64_t ld, const float* q, const float* qd,
                                                 const float* tau, float* qdd) {
  FRAX_TID();
  aba_one<T>(M, q, qd, tau, qdd, col);
}

// RNEA adjoint: 8 blocks/SM (64 registers) for chains, 7 for trees (measured
// best; the tree JVP below keeps 8).
template <class T>
__global__ void __launch_bounds__(kBlock, T::kSeg ? 7 : 8) k_rnea_vjp(const __grid_constant__ ModelImage<T::NBMAX> M, int64_t B,
                                                      int64_t ld, const float* q, const float* qd,
                                                      const float* qdd, const float* gbar, float* qbar,
                                                      float* qdbar, float* qddbar) {
  FRAX_TID();
  if constexpr (T::kSeg) rnea_vjp_seg_one<T>(M, q, qd, qdd, gbar, qbar, qdbar, qddbar, col);
  else rnea_vjp_one<T>(M, q, qd, qdd, gbar, qbar, qdbar, qddbar, col);
}

template <class T>
__global__ void __launch_bounds__(kBlock, T::kSeg ? 7 : 8) k_aba_vjp(const __grid_constant__ ModelImage<T::NBMAX> M, int64_t B,
                                                     int64_t ld, const float* q, const float* qd,
                                                     const float* tau, const float* qdd, const float* gbar,
                                                     float* qbar, float* qdbar, float* taubar) {
  FRAX_TID();
  if constexpr (T::kSeg) aba_vjp_seg_one<T>(M, q, qd, tau, qdd, gbar, qbar, qdbar, taubar, col);
  else aba_vjp_one<T>(M, q, qd, tau, qdd, gbar, qbar, qdbar, taubar, col);
}

template <class T>
__global__ void __launch_bounds__(kBlock) k_ltdl_solve(const __grid_constant__ ModelImage<T::NBMAX> M, int64_t B,
                                                        int64_t ld, const float* LD, const float* rhs, float* x) {
  FRAX_TID();
  ltdl_solve_vec<T>(M, LD, rhs, x, col);
}

template <class T>
__global__ void __launch_bounds__(kBlock) k_ltdl_inverse(const __grid_constant__ ModelImage<T::NBMAX> M,
                                                          int64_t B, int64_t ld, const float* LD, float* Minv) {
  FRAX_TID();
  ltdl_inverse<T>(M, LD, Minv, col);
}

// Trees (segment-unrolled). FK+J and CRBA leave the structural zeros of J, M
// and the factor to the row fill of zeros.cu. Register caps (128-thread blocks per SM) chosen
// by measurement on the humanoid at 2^18 instances: 8 for FK, 7 for RNEA, ABA
// (which keeps 6 floats per body in thread-local memory between its sweeps)
// and both adjoints, 5 for CRBA with both outputs; more resident warps hide
// those memory latencies better than the registers they cost, down to about
// 7 blocks.
template <class T>
__global__ void __launch_bounds__(kBlock, 8) k_fk_seg(const __grid_constant__ ModelImage<T::NBMAX> M, int64_t B,
                                                       int64_t ld, const float* q, float* pose,
                                                       const __grid_constant__ Frames fr, float* J) {
  FRAX_TID();
  fk_seg<T, ModelImage<T::NBMAX>, Col, false>(M, q, pose, fr, J, col);
}
template <class T>
__global__ void __launch_bounds__(kBlock, 7) k_rnea_seg(const __grid_constant__ ModelImage<T::NBMAX> M,
                                                         int64_t B, int64_t ld, const float* q, const float* qd,
                                                         const float* qdd, float* tau) {
  FRAX_TID();
  rnea_seg<T>(M, q, qd, qdd, tau, col);
}
// CRBA on segments; OUT 1: M only, 2: the factor only, 3: both. A call for
// one output runs the kernel that carries only that sweep's state (fewer
// registers); for both, one kernel (two would repeat the sweeps: slower).
// The structural zeros (the same entries for every instance) are written by
// the same threads after their sweeps, from the row list Z: the stores fill
// the memory system while other warps compute. A warp whose 32 instances are
// all in the batch writes them as 16-byte stores, each lane four instances
// of every fourth row (when ld and both outputs allow 16-byte alignment); a
// partial warp writes one float per thread and row.
template <class T, int OUT>
__global__ void __launch_bounds__(kBlock, OUT == 1 ? 8 : (OUT == 3 ? 5 : 6)) k_crba_seg(const __grid_constant__ ModelImage<T::NBMAX> M,
                                                                       const __grid_constant__ ZeroRows Z, int64_t B,
                                                                       int64_t ld, const float* q, float* Mout,
                                                                       float* LD) {
  FRAX_TID();
  prefetch_entries(q, M.nq, col);  // measured: helps here, not in the kernels that also read qd, tau
  crba_seg<T, ModelImage<T::NBMAX>, Col, false, OUT>(M, q, Mout, LD, col);
  const int64_t b0 = b & ~int64_t(31);  // the warp's first instance (blocks are whole warps)
  const bool vec = b0 + 32 <= B &&
                   ((uint64_t(ld) | reinterpret_cast<uintptr_t>(Mout) | reinterpret_cast<uintptr_t>(LD)) & 3) == 0 &&
                   ((reinterpret_cast<uintptr_t>(Mout) | reinterpret_cast<uintptr_t>(LD)) & 15) == 0;
  if (vec) {
    const int lane = int(threadIdx.x & 31);
    const int sub = lane >> 3;  // row offset within a group of four rows
    const int64_t off = b0 + (lane & 7) * 4;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int r = sub; r < Z.n0; r += 4) __stcs(reinterpret_cast<float4*>(at_row(Mout + off, Z.row[r], ld)), z4);
    for (int r = Z.n0 + sub; r < Z.n; r += 4) __stcs(reinterpret_cast<float4*>(at_row(LD + off, Z.row[r], ld)), z4);
    return;
  }
#pragma unroll 4
  for (int r = 0; r < Z.n0; ++r) col.out(Mout, Z.row[r], 0.f);
#pragma unroll 4
  for (int r = Z.n0; r < Z.n; ++r) col.out(LD, Z.row[r], 0.f);
}
template <class T>
__global__ void __launch_bounds__(kBlock, 7) k_aba_seg(const __grid_constant__ ModelImage<T::NBMAX> M, int64_t B,
                                                        int64_t ld, const float* q, const float* qd,
                                                        const float* tau, float* qdd) {
  FRAX_TID();
  P3Local<T::NBMAX> P;
  aba_seg<T>(M, q, qd, tau, qdd, col, P);
}

template <class T>
__global__ void __launch_bounds__(kBlock, 5) k_osc_seg(const __grid_constant__ ModelImage<T::NBMAX> M, int64_t B,
                                                        int64_t ld, int task, const float* q, const float* qd,
                                                        const float* xdd, float* tau, float* Lam) {
  FRAX_TID();
  osc_seg<T>(M, task, q, qd, xdd, tau, Lam, col);
}

// External forces. Trees: RNEA and ABA take them inside their own sweeps
// (Algorithm 1's body-frame subtraction); per-body-array trees compute
// tau_ext in one more sweep.
// RNEA with external forces: 5 blocks per SM (the world pose it carries
// spills at 64 registers; humanoid 2^18: 152 us against 156 at 8 blocks).
template <class T>
__global__ void __launch_bounds__(kBlock, 5) k_rnea_ext(const __grid_constant__ ModelImage<T::NBMAX> M, int64_t B,
                                                         int64_t ld, const float* q, const float* qd,
                                                         const float* qdd, const float* fext, float* tau) {
  FRAX_TID();
  if constexpr (T::kSeg) {
    // the forces enter RNEA's own outward sweep (Algorithm 1's -F_ext,i)
    rnea_seg<T, ModelImage<T::NBMAX>, Col, false, true>(M, q, qd, qdd, tau, col, -1, SV{}, fext);
  } else {
    rnea_one<T>(M, q, qd, qdd, tau, col);
    ext_tau<T>(M, q, fext, col, SubFromGlobal<T>{tau, ColT<false>{ld, b}});
  }
}
template <class T>
__global__ void __launch_bounds__(kBlock, 8) k_aba_ext(const __grid_constant__ ModelImage<T::NBMAX> M, int64_t B,
                                                        int64_t ld, const float* q, const float* qd,
                                                        const float* tau, const float* fext, float* qdd) {
  FRAX_TID();
  if constexpr (T::kSeg) {
    // the forces enter the bias forces of ABA's own sweeps
    P3Local<T::NBMAX> P;
    aba_seg_core<T, ModelImage<T::NBMAX>, true, RhsFromGlobal<T, Col>, OutToGlobal<T, Col>, Col, P3Local<T::NBMAX>,
                 true>(M, q, qd, RhsFromGlobal<T, Col>{tau, col}, OutToGlobal<T, Col>{qdd, col}, col, P, fext);
  } else {
    LocalVec<T> w;
    ext_tau<T>(M, q, fext, col, OutToLocal<T>{&w});
    const RhsPlusLocal<T, Col> rhs{tau, col, &w};
    aba_core<T, ModelImage<T::NBMAX>, true>(M, q, qd, rhs, OutToGlobal<T, Col>{qdd, col}, col);
  }
}

// Forward-mode derivatives on segments (the 7-body chain has unrolled
// kernels of its own).
template <class T>
__global__ void __launch_bounds__(kBlock, 8) k_rnea_jvp(const __grid_constant__ ModelImage<T::NBMAX> M, int64_t B,
                                                      int64_t ld, const float* q, const float* qd,
                                                      const float* qdd, const float* dq, const float* dqd,
                                                      const float* dqdd, float* tau, float* dtau) {
  FRAX_TID();
  rnea_jvp_seg<T>(M, q, qd, qdd, dq, dqd, dqdd, JvpToGlobal<T, Col>{tau, dtau, col}, col);
}
template <class T>
__global__ void __launch_bounds__(kBlock, 8) k_aba_jvp(const __grid_constant__ ModelImage<T::NBMAX> M, int64_t B,
                                                     int64_t ld, const float* q, const float* qd,
                                                     const float* qdd, const float* dq, const float* dqd,
                                                     const float* dtau, float* dqdd) {
  FRAX_TID();
  aba_jvp_seg_one<T>(M, q, qd, qdd, dq, dqd, dtau, dqdd, col);
}
template <class T>
__global__ void __launch_bounds__(kBlock, 6) k_fk_jvp(const __grid_constant__ ModelImage<T::NBMAX> M, int64_t B,
                                                       int64_t ld, const float* q, const float* dq,
                                                       const __grid_constant__ Frames fr, float* out) {
  FRAX_TID();
  fk_jvp_seg<T>(M, q, dq, fr, out, col);
}

template <class T>
cudaError_t launch_topo(const ModelImage<T::NBMAX>& img, Op op, const OpArgs& a) {
  const dim3 grid(unsigned((a.B + kBlock - 1) / kBlock)), block(kBlock);
  Frames fr{a.frames.n, {0}};
  for (int k = 0; k < 8; ++k) fr.body[k] = a.frames.body[k];
  switch (op) {
    case kOpFk:
    case kOpJac:
      if constexpr (T::kSeg) k_fk_seg<T><<<grid, block, 0, a.stream>>>(img, a.B, a.ld, a.q, a.out0, fr, a.out1);
      else k_fk<T><<<grid, block, 0, a.stream>>>(img, a.B, a.ld, a.q, a.out0, fr, a.out1);
      break;
    case kOpRnea:
      if constexpr (T::kSeg) k_rnea_seg<T><<<grid, block, 0, a.stream>>>(img, a.B, a.ld, a.q, a.qd, a.qdd, a.out0);
      else k_rnea<T><<<grid, block, 0, a.stream>>>(img, a.B, a.ld, a.q, a.qd, a.qdd, a.out0);
      break;
    case kOpCrba:
      if constexpr (T::kSeg) {
        static const ZeroRows kNone{};
        const ZeroRows& Z = a.zeros ? *a.zeros : kNone;
        if (a.out0 && a.out1) k_crba_seg<T, 3><<<grid, block, 0, a.stream>>>(img, Z, a.B, a.ld, a.q, a.out0, a.out1);
        else if (a.out0) k_crba_seg<T, 1><<<grid, block, 0, a.stream>>>(img, Z, a.B, a.ld, a.q, a.out0, nullptr);
        else k_crba_seg<T, 2><<<grid, block, 0, a.stream>>>(img, Z, a.B, a.ld, a.q, nullptr, a.out1);
      }
      else k_crba<T><<<grid, block, 0, a.stream>>>(img, a.B, a.ld, a.q, a.out0, a.out1);
      break;
    case kOpAba:
    case kOpAbaSweep:
      if constexpr (T::kSeg) k_aba_seg<T><<<grid, block, 0, a.stream>>>(img, a.B, a.ld, a.q, a.qd, a.tau, a.out0);
      else k_aba<T><<<grid, block, 0, a.stream>>>(img, a.B, a.ld, a.q, a.qd, a.tau, a.out0);
      break;
    case kOpLtdlSolve:
      k_ltdl_solve<T><<<grid, block, 0, a.stream>>>(img, a.B, a.ld, a.in_LD, a.qd, a.out0);
      break;
    case kOpLtdlInverse:
      k_ltdl_inverse<T><<<grid, block, 0, a.stream>>>(img, a.B, a.ld, a.in_LD, a.out0);
      break;
    case kOpRneaVjp:
      k_rnea_vjp<T><<<grid, block, 0, a.stream>>>(img, a.B, a.ld, a.q, a.qd, a.qdd, a.gbar, a.out0, a.out1,
                                                  a.out2);
      break;
    case kOpAbaVjp:
      k_aba_vjp<T><<<grid, block, 0, a.stream>>>(img, a.B, a.ld, a.q, a.qd, a.tau, a.qdd, a.gbar, a.out0,
                                                 a.out1, a.out2);
      break;
    case kOpRneaExt:
      k_rnea_ext<T><<<grid, block, 0, a.stream>>>(img, a.B, a.ld, a.q, a.qd, a.qdd, a.in_fext, a.out0);
      break;
    case kOpAbaExt:
      k_aba_ext<T><<<grid, block, 0, a.stream>>>(img, a.B, a.ld, a.q, a.qd, a.tau, a.in_fext, a.out0);
      break;
    case kOpFkJvp:
      if constexpr (T::kSeg) k_fk_jvp<T><<<grid, block, 0, a.stream>>>(img, a.B, a.ld, a.q, a.in_dq, fr, a.out0);
      else return cudaErrorInvalidValue;
      break;
    case kOpRneaJvp:
      if constexpr (T::kSeg)
        k_rnea_jvp<T><<<grid, block, 0, a.stream>>>(img, a.B, a.ld, a.q, a.qd, a.qdd, a.in_dq, a.in_dqd, a.in_dx,
                                                    a.out0, a.out1);
      else
        return cudaErrorInvalidValue;
      break;
    case kOpAbaJvp:
      if constexpr (T::kSeg)
        k_aba_jvp<T><<<grid, block, 0, a.stream>>>(img, a.B, a.ld, a.q, a.qd, a.qdd, a.in_dq, a.in_dqd, a.in_dx,
                                                   a.out0);
      else
        return cudaErrorInvalidValue;
      break;
    case kOpOsc:
      if constexpr (T::kSeg)
        k_osc_seg<T><<<grid, block, 0, a.stream>>>(img, a.B, a.ld, a.frames.body[0], a.q, a.qd, a.in_xdd, a.out0,
                                                   a.out1);
      else
        return cudaErrorInvalidValue;
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace frax
