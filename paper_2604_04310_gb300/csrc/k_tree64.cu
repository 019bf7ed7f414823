// General trees (segment-unrolled kernels) of up to 64 bodies (fixed base or free-flyer root).
#include "kernels.cuh"

namespace frax {
cudaError_t launch_tree64(const HostModel& m, Op op, const OpArgs& a) {
  ModelImage<64> img;
  m.pack(&img);
  return m.free_root ? launch_topo<SegTopo<64, true>>(img, op, a) : launch_topo<SegTopo<64, false>>(img, op, a);
}
}  // namespace frax
