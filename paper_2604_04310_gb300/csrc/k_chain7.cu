// Serial chains of 7 revolute bodies: topology compiled in, registers only
// (the adjoints run the segment code on the same chain).
#include "kernels.cuh"

namespace frax {
cudaError_t launch_chain7(const HostModel& m, Op op, const OpArgs& a) {
  if (op == kOpRneaVjp || op == kOpAbaVjp) {
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
