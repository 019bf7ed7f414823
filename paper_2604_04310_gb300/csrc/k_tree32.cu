// General trees (segment-unrolled kernels) of up to 32 bodies (fixed base or free-flyer root), and their
// lane-group kernels for small batches.
#include <mutex>

#include "kernels.cuh"
#include "lg.cuh"

namespace frax {
namespace {

template <class K>
cudaError_t lg_smem(K kernel, int bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// Instances one resident wave of a lane-group kernel holds on this device
// (SMs x blocks per SM x instances per block), memoised per device, kernel
// and shared-memory size. Past one wave the lane groups lose to one thread
// per instance (measured on the humanoid: each op's crossover sits at its
// wave size), so the automatic path choice compares the batch with it.
template <class K>
int64_t lg_wave(K kernel, int bytes) {
  struct Entry {
    int dev;
    const void* k;
    int bytes;
    int64_t wave;
  };
  static std::mutex mu;
  static Entry cache[32];
  static int n = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  std::lock_guard<std::mutex> lk(mu);
  for (int i = 0; i < n; ++i)
    if (cache[i].dev == dev && cache[i].k == reinterpret_cast<const void*>(kernel) && cache[i].bytes == bytes)
      return cache[i].wave;
  int sms = 0, per_sm = 0;
  if (lg_smem(kernel, bytes) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kLgBlock, bytes)) {
    cudaGetLastError();
    return 0;
  }
  const int64_t wave = int64_t(sms) * per_sm * kLgInst;
  if (n < 32) cache[n++] = Entry{dev, reinterpret_cast<const void*>(kernel), bytes, wave};
  return wave;
}

// Launches the lane-group kernel of `op`; with `decide` set, first checks
// that the batch fits one resident wave and returns cudaErrorNotSupported
// (nothing launched) if it does not.
cudaError_t launch_lg(const HostModel& m, const ModelImage<32>& img, Op op, const OpArgs& a, bool decide) {
  const LanePlan& P = m.lane_plan;
  const dim3 grid(unsigned((a.B + kLgInst - 1) / kLgInst));
  const int no = P.n_oslot, ni = P.n_islot;
  // shared memory: model image, plan, the block's staged input columns, scratch
  auto bytes = [&](int floats, int in_rows) { return kLgImgBytes + kLgPlanBytes + kLgInst * (floats + in_rows) * 4; };
  const int r3 = m.nq + 2 * m.nv, r4 = m.nq + 3 * m.nv;
  cudaError_t e;
  auto go = [&](auto k, int sm, auto&&... args) -> cudaError_t {
    if (decide && a.B > lg_wave(k, sm)) return cudaErrorNotSupported;
    if ((e = lg_smem(k, sm)) != cudaSuccess) return e;
    k<<<grid, kLgBlock, sm, a.stream>>>(img, P, args...);
    return cudaGetLastError();
  };
  switch (op) {
    case kOpRnea:
      return go(m.free_root ? k_rnea_lg<true> : k_rnea_lg<false>, bytes(lg_rnea_floats(m.nb, no, ni), r3), a.B,
                a.ld, a.q, a.qd, a.qdd, a.out0);
    case kOpAba:
    case kOpAbaSweep:
      return go(m.free_root ? k_aba_lg<true> : k_aba_lg<false>, bytes(lg_aba_floats(m.nb, no, ni), r3), a.B,
                a.ld, a.q, a.qd, a.tau, a.out0);
    case kOpRneaVjp:
      return go(m.free_root ? k_rnea_vjp_lg<true> : k_rnea_vjp_lg<false>, bytes(lg_vjp_floats(m.nb, no, ni), r4),
                a.B, a.ld, a.q, a.qd, a.qdd, a.gbar, a.out0, a.out1, a.out2);
    case kOpFk:
    case kOpJac: {
      Frames fr{a.frames.n, {0}};
      for (int k = 0; k < 8; ++k) fr.body[k] = a.frames.body[k];
      return go(m.free_root ? k_fk_lg<true> : k_fk_lg<false>, bytes(lg_fk_floats(m.nb, no), m.nq), a.B, a.ld, a.q,
                a.out0, fr, a.out1);
    }
    case kOpCrba: {
      static const ZeroRows kNone{};
      return go(m.free_root ? k_crba_lg<true> : k_crba_lg<false>, bytes(lg_crba_floats(m.nb, ni), m.nq),
                a.zeros ? *a.zeros : kNone, a.B, a.ld, a.q, a.out0, a.out1);
    }
    case kOpAbaVjp:
      return go(m.free_root ? k_aba_vjp_lg<true> : k_aba_vjp_lg<false>,
                bytes(lg_aba_vjp_floats(m.nb, m.nv, no, ni), r4), a.B, a.ld, a.q, a.qd, a.qdd, a.gbar, a.out0,
                a.out1, a.out2);
    default:
      return cudaErrorInvalidValue;
  }
}

bool has_lg(Op op) {
  return op == kOpRnea || op == kOpAba || op == kOpAbaSweep || op == kOpRneaVjp || op == kOpAbaVjp || op == kOpCrba ||
         op == kOpFk || op == kOpJac;
}

}  // namespace

cudaError_t launch_tree32(const HostModel& m, Op op, const OpArgs& a) {
  const ModelImage<32>& img = m.image<32>();
  if (a.tree_path != FRAX_TREE_PATH_THREAD && m.lane_plan.T > 0 && has_lg(op)) {
    const cudaError_t e = launch_lg(m, img, op, a, a.tree_path == FRAX_TREE_PATH_AUTO);
    if (e != cudaErrorNotSupported) return e;  // else: more than one wave, one thread per instance
  }
  return m.free_root ? launch_topo<SegTopo<32, true>>(img, op, a) : launch_topo<SegTopo<32, false>>(img, op, a);
}
}  // namespace frax
