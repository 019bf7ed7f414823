// General trees (segment-unrolled kernels) of up to 32 bodies (fixed base or free-flyer root).
#include "kernels.cuh"

namespace frax {
cudaError_t launch_tree32(const HostModel& m, Op op, const OpArgs& a) {
  const ModelImage<32>& img = m.image<32>();
  return m.free_root ? launch_topo<SegTopo<32, true>>(img, op, a) : launch_topo<SegTopo<32, false>>(img, op, a);
}
}  // namespace frax
