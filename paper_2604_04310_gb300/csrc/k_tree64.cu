// General trees (segment-unrolled kernels) of up to 64 bodies (fixed base or free-flyer root).
#include "kernels.cuh"

namespace frax {
cudaError_t launch_tree64(const HostModel& m, Op op, const OpArgs& a) {
  const ModelImage<64>& img = m.image<64>();
  return m.free_root ? launch_topo<SegTopo<64, true>>(img, op, a) : launch_topo<SegTopo<64, false>>(img, op, a);
}
}  // namespace frax
