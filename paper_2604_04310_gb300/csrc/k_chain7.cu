// Serial chains of 7 revolute bodies: topology compiled in, registers only.
#include "kernels.cuh"

namespace frax {

// 7-body chains: the ABA adjoint in one launch (used when taubar is not
// wanted): the solve through the mass-matrix factor (chain_minv), then the
// unrolled RNEA adjoint.
__global__ void __launch_bounds__(kBlock) k_aba_vjp_chain7(const __grid_constant__ ModelImage<8> M, int64_t B,
                                                            int64_t ld, const float* q, const float* qd,
                                                            const float* qdd, const float* gbar, float* qbar,
                                                            float* qdbar, float* taubar) {
  FRAX_TID();
  aba_vjp_chain_one<7>(M, q, qd, qdd, gbar, qbar, qdbar, taubar, col);
}

// 7-body chains: the ABA JVP with its solve through the mass-matrix factor.
__global__ void __launch_bounds__(kBlock) k_aba_jvp_chain7(const __grid_constant__ ModelImage<8> M, int64_t B,
                                                            int64_t ld, const float* q, const float* qd,
                                                            const float* qdd, const float* dq, const float* dqd,
                                                            const float* dtau, float* dqdd) {
  const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const Col64 col{ld, b};
  aba_jvp_chain_one<7>(M, q, qd, qdd, dq, dqd, dtau, dqdd, col);
}

// 7-body chains: forward dynamics through the mass-matrix factor,
// qdd = M^-1 (tau - c - g) (the Cholesky-style solve of the Sec. VI
// footnote): c + g by RNEA into qdd, then the register factor solve reading
// it back. 3353 flops against the articulated-body algorithm's 3431, and 64
// registers instead of 128.
struct TauMinusBias {
  const float* tau;
  const float* bias;
  Col col;
  ColT<false> own;  // bias was written by this thread: read through L2
  FD float operator()(int k) const { return col.in(tau, k) - own.in(bias, k); }
};
__global__ void __launch_bounds__(kBlock) k_aba_chain7(const __grid_constant__ ModelImage<8> M, int64_t B,
                                                         int64_t ld, const float* q, const float* qd,
                                                         const float* tau, float* qdd) {
  FRAX_TID();
  rnea_one<ChainTopo<7>>(M, q, qd, nullptr, qdd, col);
  float w[7];
  chain_minv<7>(M, q, TauMinusBias{tau, qdd, col, ColT<false>{ld, b}}, w, col);
#pragma unroll
  for (int k = 0; k < 7; ++k) col.out(qdd, k, w[k]);
}

// With external forces: right-hand side tau + tau_ext - (c + g).
struct TauExtMinusBias {
  const float* tau;
  const float* bias;
  const LocalVec<ChainTopo<7>>* ext;
  Col64 col;
  ColT<false, false> own;
  FD float operator()(int k) const { return (col.in(tau, k) + (*ext)(k)) - own.in(bias, k); }
};
__global__ void __launch_bounds__(kBlock) k_aba_ext_chain7(const __grid_constant__ ModelImage<8> M, int64_t B,
                                                             int64_t ld, const float* q, const float* qd,
                                                             const float* tau, const float* fext, float* qdd) {
  const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const Col64 col{ld, b};
  using T = ChainTopo<7>;
  LocalVec<T> w;
  ext_tau_chain<7>(M, q, fext, col, OutToLocal<T>{&w});
  rnea_one<T>(M, q, qd, nullptr, qdd, col);
  float x[7];
  chain_minv<7>(M, q, TauExtMinusBias{tau, qdd, &w, col, ColT<false, false>{ld, b}}, x, col);
#pragma unroll
  for (int k = 0; k < 7; ++k) col.out(qdd, k, x[k]);
}

// The ABA adjoint in two launches when taubar is asked for (it is w itself):
// w = M^-1 gbar through the factor into taubar, then the RNEA adjoint seeded
// with it. Each kernel stays small enough for the instruction cache.
__global__ void __launch_bounds__(kBlock, 8) k_minv_chain7(const __grid_constant__ ModelImage<8> M, int64_t B,
                                                          int64_t ld, const float* q, const float* g, float* w) {
  FRAX_TID();
  float x[7];
  chain_minv<7>(M, q, RhsFromGlobal<ChainTopo<7>, Col>{g, col}, x, col);
#pragma unroll
  for (int k = 0; k < 7; ++k) col.out(w, k, x[k]);
}
__global__ void __launch_bounds__(kBlock) k_aba_vjp_tail_chain7(const __grid_constant__ ModelImage<8> M, int64_t B,
                                                                 int64_t ld, const float* q, const float* qd,
                                                                 const float* qdd, const float* w, float* qbar,
                                                                 float* qdbar) {
  FRAX_TID();
  using T = ChainTopo<7>;
  rnea_vjp_chain<7>(M, q, qd, qdd, RhsFromGlobal<T, Col>{w, col}, vjp_sink<T>(M, q, qbar, qdbar, nullptr, -1.f, col),
                    col);
}

// 7-body chains: RNEA with external forces, tau_ext unrolled.
__global__ void __launch_bounds__(kBlock) k_rnea_ext_chain7(const __grid_constant__ ModelImage<8> M, int64_t B,
                                                            int64_t ld, const float* q, const float* qd,
                                                            const float* qdd, const float* fext, float* tau) {
  FRAX_TID();
  using T = ChainTopo<7>;
  rnea_one<T>(M, q, qd, qdd, tau, col);
  ext_tau_chain<7>(M, q, fext, col, SubFromGlobal<T>{tau, ColT<false>{ld, b}});
}

// 7-body chains: the FK JVP, unrolled.
__global__ void __launch_bounds__(kBlock) k_fk_jvp_chain7(const __grid_constant__ ModelImage<8> M, int64_t B,
                                                          int64_t ld, const float* q, const float* dq,
                                                          const __grid_constant__ Frames fr, float* out) {
  FRAX_TID();
  fk_jvp_chain<7>(M, q, dq, fr, out, col);
}

// 7-body chains: the RNEA JVP, both sweeps unrolled.
__global__ void __launch_bounds__(kBlock) k_rnea_jvp_chain7(const __grid_constant__ ModelImage<8> M, int64_t B,
                                                            int64_t ld, const float* q, const float* qd,
                                                            const float* qdd, const float* dq, const float* dqd,
                                                            const float* dqdd, float* tau, float* dtau) {
  FRAX_TID();
  rnea_jvp_chain<7>(M, q, qd, qdd, dq, dqd, dqdd, JvpToGlobal<ChainTopo<7>, Col>{tau, dtau, col}, col);
}

// 7-body chains: the RNEA adjoint, both sweeps unrolled. No register cap:
// at 95 registers (5 blocks per SM) it ran faster than capped at 72 or 64.
__global__ void __launch_bounds__(kBlock) k_rnea_vjp_chain7(const __grid_constant__ ModelImage<8> M, int64_t B,
                                                              int64_t ld, const float* q, const float* qd,
                                                              const float* qdd, const float* gbar, float* qbar,
                                                              float* qdbar, float* qddbar) {
  FRAX_TID();
  using T = ChainTopo<7>;
  rnea_vjp_chain<7>(M, q, qd, qdd, RhsFromGlobal<T, Col>{gbar, col},
                    vjp_sink<T>(M, q, qbar, qdbar, qddbar, 1.f, col), col);
}

// 7-body chains: operational-space control with every sweep unrolled. Capped
// at 4 blocks per SM (128 registers, no spills): 199 us at 2^20 against 212
// uncapped (161 registers) and 211 at 5 blocks (spills).
__global__ void __launch_bounds__(kBlock, 4) k_osc_chain7(const __grid_constant__ ModelImage<8> M, int64_t B,
                                                        int64_t ld, int task, const float* q, const float* qd,
                                                        const float* xdd, float* tau, float* Lam) {
  FRAX_TID();
  osc_chain<7>(M, task, q, qd, xdd, tau, Lam, col);
}

cudaError_t launch_chain7(const HostModel& m, Op op, const OpArgs& a) {
  if (op == kOpAbaVjp && a.out2) {
    const ModelImage<8>& img8 = m.image<8>();
    const dim3 grid(unsigned((a.B + kBlock - 1) / kBlock));
    k_minv_chain7<<<grid, kBlock, 0, a.stream>>>(img8, a.B, a.ld, a.q, a.gbar, a.out2);
    k_aba_vjp_tail_chain7<<<grid, kBlock, 0, a.stream>>>(img8, a.B, a.ld, a.q, a.qd, a.qdd, a.out2, a.out0,
                                                         a.out1);
    return cudaGetLastError();
  }
  if (op == kOpRneaExt) {
    const ModelImage<8>& img8 = m.image<8>();
    const dim3 grid(unsigned((a.B + kBlock - 1) / kBlock));
    k_rnea_ext_chain7<<<grid, kBlock, 0, a.stream>>>(img8, a.B, a.ld, a.q, a.qd, a.qdd, a.in_fext, a.out0);
    return cudaGetLastError();
  }
  if (op == kOpAbaExt) {
    const ModelImage<8>& img8 = m.image<8>();
    const dim3 grid(unsigned((a.B + kBlock - 1) / kBlock));
    k_aba_ext_chain7<<<grid, kBlock, 0, a.stream>>>(img8, a.B, a.ld, a.q, a.qd, a.tau, a.in_fext, a.out0);
    return cudaGetLastError();
  }
  if (op == kOpAba) {
    const ModelImage<8>& img8 = m.image<8>();
    const dim3 grid(unsigned((a.B + kBlock - 1) / kBlock));
    k_aba_chain7<<<grid, kBlock, 0, a.stream>>>(img8, a.B, a.ld, a.q, a.qd, a.tau, a.out0);
    return cudaGetLastError();
  }
  if (op == kOpAbaJvp) {
    const ModelImage<8>& img8 = m.image<8>();
    const dim3 grid(unsigned((a.B + kBlock - 1) / kBlock));
    k_aba_jvp_chain7<<<grid, kBlock, 0, a.stream>>>(img8, a.B, a.ld, a.q, a.qd, a.qdd, a.in_dq, a.in_dqd, a.in_dx,
                                                    a.out0);
    return cudaGetLastError();
  }
  if (op == kOpAbaVjp) {
    const ModelImage<8>& img8 = m.image<8>();
    const dim3 grid(unsigned((a.B + kBlock - 1) / kBlock));
    k_aba_vjp_chain7<<<grid, kBlock, 0, a.stream>>>(img8, a.B, a.ld, a.q, a.qd, a.qdd, a.gbar, a.out0, a.out1,
                                                    a.out2);
    return cudaGetLastError();
  }
  if (op == kOpRneaVjp) {
    const ModelImage<8>& img8 = m.image<8>();
    const dim3 grid(unsigned((a.B + kBlock - 1) / kBlock));
    k_rnea_vjp_chain7<<<grid, kBlock, 0, a.stream>>>(img8, a.B, a.ld, a.q, a.qd, a.qdd, a.gbar, a.out0, a.out1,
                                                     a.out2);
    return cudaGetLastError();
  }
  if (op == kOpRneaJvp) {
    const ModelImage<8>& img8 = m.image<8>();
    const dim3 grid(unsigned((a.B + kBlock - 1) / kBlock));
    k_rnea_jvp_chain7<<<grid, kBlock, 0, a.stream>>>(img8, a.B, a.ld, a.q, a.qd, a.qdd, a.in_dq, a.in_dqd, a.in_dx,
                                                     a.out0, a.out1);
    return cudaGetLastError();
  }
  if (op == kOpFkJvp) {
    const ModelImage<8>& img8 = m.image<8>();
    Frames fr{a.frames.n, {0}};
    for (int f = 0; f < a.frames.n; ++f) fr.body[f] = a.frames.body[f];
    const dim3 grid(unsigned((a.B + kBlock - 1) / kBlock));
    k_fk_jvp_chain7<<<grid, kBlock, 0, a.stream>>>(img8, a.B, a.ld, a.q, a.in_dq, fr, a.out0);
    return cudaGetLastError();
  }
  if (op == kOpOsc) {
    const dim3 grid(unsigned((a.B + kBlock - 1) / kBlock));
    k_osc_chain7<<<grid, kBlock, 0, a.stream>>>(m.image<8>(), a.B, a.ld, a.frames.body[0], a.q, a.qd, a.in_xdd,
                                                a.out0, a.out1);
    return cudaGetLastError();
  }
  return launch_topo<ChainTopo<7>>(m.image<7>(), op, a);
}
}  // namespace frax
