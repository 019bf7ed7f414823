// Serial chains of 7 revolute bodies: topology compiled in, registers only.
#include "kernels.cuh"

namespace frax {
cudaError_t launch_chain7(const HostModel& m, Op op, const OpArgs& a) {
  ModelImage<7> img;
  m.pack(&img);
  return launch_topo<ChainTopo<7>>(img, op, a);
}
}  // namespace frax
