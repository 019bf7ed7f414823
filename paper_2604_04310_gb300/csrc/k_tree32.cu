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
  const bool aba = op != kOpRnea;
  const int per_inst = aba ? lg_aba_floats(m.nb, P.n_oslot, P.n_islot) : lg_rnea_floats(m.nb, P.n_oslot, P.n_islot);
  const int bytes = kLgImgBytes + kLgPlanBytes + kLgInst * per_inst * 4;
  cudaError_t e;
  if (aba) {
    auto k = m.free_root ? k_aba_lg<true> : k_aba_lg<false>;
    if ((e = lg_smem(k, bytes)) != cudaSuccess) return e;
    k<<<grid, kLgBlock, bytes, a.stream>>>(img, P, a.B, a.ld, a.q, a.qd, a.tau, a.out0);
  } else {
    auto k = m.free_root ? k_rnea_lg<true> : k_rnea_lg<false>;
    if ((e = lg_smem(k, bytes)) != cudaSuccess) return e;
    k<<<grid, kLgBlock, bytes, a.stream>>>(img, P, a.B, a.ld, a.q, a.qd, a.qdd, a.out0);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tree32(const HostModel& m, Op op, const OpArgs& a) {
  const ModelImage<32>& img = m.image<32>();
  if (a.lane_group && m.lane_plan.T > 0 && (op == kOpRnea || op == kOpAba || op == kOpAbaSweep))
    return launch_lg(m, img, op, a);
  return m.free_root ? launch_topo<SegTopo<32, true>>(img, op, a) : launch_topo<SegTopo<32, false>>(img, op, a);
}
}  // namespace frax
