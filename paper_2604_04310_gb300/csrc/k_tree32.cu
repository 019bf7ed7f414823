// General trees (segment-unrolled kernels) of up to 32 bodies (fixed base or free-flyer root), and their
// lane-group kernels for small batches.
#include "kernels.cuh"
#include "lg.cuh"

namespace frax {
namespace {

template <class K>
cudaError_t lg_smem(K kernel, int bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_lg(const HostModel& m, const ModelImage<32>& img, Op op, const OpArgs& a) {
  const LanePlan& P = m.lane_plan;
  const dim3 grid(unsigned((a.B + kLgInst - 1) / kLgInst));
  const int no = P.n_oslot, ni = P.n_islot;
  // shared memory: model image, plan, the block's staged input columns, scratch
  auto bytes = [&](int floats, int in_rows) { return kLgImgBytes + kLgPlanBytes + kLgInst * (floats + in_rows) * 4; };
  const int r3 = m.nq + 2 * m.nv, r4 = m.nq + 3 * m.nv;
  cudaError_t e;
  switch (op) {
    case kOpRnea: {
      auto k = m.free_root ? k_rnea_lg<true> : k_rnea_lg<false>;
      const int sm = bytes(lg_rnea_floats(m.nb, no, ni), r3);
      if ((e = lg_smem(k, sm)) != cudaSuccess) return e;
      k<<<grid, kLgBlock, sm, a.stream>>>(img, P, a.B, a.ld, a.q, a.qd, a.qdd, a.out0);
      break;
    }
    case kOpAba:
    case kOpAbaSweep: {
      auto k = m.free_root ? k_aba_lg<true> : k_aba_lg<false>;
      const int sm = bytes(lg_aba_floats(m.nb, no, ni), r3);
      if ((e = lg_smem(k, sm)) != cudaSuccess) return e;
      k<<<grid, kLgBlock, sm, a.stream>>>(img, P, a.B, a.ld, a.q, a.qd, a.tau, a.out0);
      break;
    }
    case kOpRneaVjp: {
      auto k = m.free_root ? k_rnea_vjp_lg<true> : k_rnea_vjp_lg<false>;
      const int sm = bytes(lg_vjp_floats(m.nb, no, ni), r4);
      if ((e = lg_smem(k, sm)) != cudaSuccess) return e;
      k<<<grid, kLgBlock, sm, a.stream>>>(img, P, a.B, a.ld, a.q, a.qd, a.qdd, a.gbar, a.out0, a.out1, a.out2);
      break;
    }
    case kOpAbaVjp: {
      auto k = m.free_root ? k_aba_vjp_lg<true> : k_aba_vjp_lg<false>;
      const int sm = bytes(lg_aba_vjp_floats(m.nb, m.nv, no, ni), r4);
      if ((e = lg_smem(k, sm)) != cudaSuccess) return e;
      k<<<grid, kLgBlock, sm, a.stream>>>(img, P, a.B, a.ld, a.q, a.qd, a.qdd, a.gbar, a.out0, a.out1, a.out2);
      break;
    }
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

bool has_lg(Op op) {
  return op == kOpRnea || op == kOpAba || op == kOpAbaSweep || op == kOpRneaVjp || op == kOpAbaVjp;
}

}  // namespace

cudaError_t launch_tree32(const HostModel& m, Op op, const OpArgs& a) {
  const ModelImage<32>& img = m.image<32>();
  if (a.lane_group && m.lane_plan.T > 0 && has_lg(op)) return launch_lg(m, img, op, a);
  return m.free_root ? launch_topo<SegTopo<32, true>>(img, op, a) : launch_topo<SegTopo<32, false>>(img, op, a);
}
}  // namespace frax
