// Serial chains of 7 revolute bodies: topology compiled in, registers only
// (the adjoints run the segment code on the same chain).
#include "kernels.cuh"

namespace frax {

// 7-body chains: the ABA adjoint with its solve through the mass-matrix
// factor (chain_minv), on the 8-slot image the segment code reads.
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
  FRAX_TID();
  aba_jvp_chain_one<7>(M, q, qd, qdd, dq, dqd, dtau, dqdd, col);
}

cudaError_t launch_chain7(const HostModel& m, Op op, const OpArgs& a) {
  if (op == kOpAbaJvp) {
    ModelImage<8> img8;
    m.pack(&img8);
    const dim3 grid(unsigned((a.B + kBlock - 1) / kBlock));
    k_aba_jvp_chain7<<<grid, kBlock, 0, a.stream>>>(img8, a.B, a.ld, a.q, a.qd, a.qdd, a.in_dq, a.in_dqd, a.in_dx,
                                                    a.out0);
    return cudaGetLastError();
  }
  if (op == kOpAbaVjp) {
    ModelImage<8> img8;
    m.pack(&img8);
    const dim3 grid(unsigned((a.B + kBlock - 1) / kBlock));
    k_aba_vjp_chain7<<<grid, kBlock, 0, a.stream>>>(img8, a.B, a.ld, a.q, a.qd, a.qdd, a.gbar, a.out0, a.out1,
                                                    a.out2);
    return cudaGetLastError();
  }
  if (op == kOpRneaVjp || op == kOpOsc || op == kOpRneaJvp || op == kOpFkJvp) {
    // the adjoints step the forward state back through the joints instead
    // of keeping it per body: far fewer live registers than the unrolled form
    ModelImage<8> img8;
    m.pack(&img8);
    return launch_topo<SegTopo<8, false>>(img8, op, a);
  }
  ModelImage<7> img;
  m.pack(&img);
  return launch_topo<ChainTopo<7>>(img, op, a);
}
}  // namespace frax
