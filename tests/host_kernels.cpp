// The kernels' per-instance device functions compiled as host code (a
// test harness, not part of the library): reads one model and a batch of
// states (SoA, FP32) from a file, evaluates every op with the same device
// functions the CUDA kernels call, and writes the outputs to a file for the
// oracle to check on the CPU. Build (no GPU needed):
//   g++ -std=c++17 -O1 -x c++ -I<cuda>/include -I<repo> tests/host_kernels.cpp \
//       paper_2604_04310_gb300/csrc/model.cpp -o host_kernels
// Usage: host_kernels <input file> <output file>
#include <math.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <string>
#include <vector>

#include <cuda_runtime.h>

// the device builtin rsqrtf has no host counterpart in the C library
static inline float rsqrtf(float x) { return 1.0f / std::sqrt(x); }

#include "paper_2604_04310_gb300/csrc/model.h"
#include "paper_2604_04310_gb300/csrc/osc.cuh"
#include "paper_2604_04310_gb300/csrc/ext.cuh"
#include "paper_2604_04310_gb300/csrc/jvp.cuh"
#include "paper_2604_04310_gb300/csrc/lg.cuh"

using namespace frax;

namespace {

struct Reader {
  FILE* f;
  template <class X>
  std::vector<X> take(size_t n) {
    std::vector<X> v(n);
    if (n && std::fread(v.data(), sizeof(X), n, f) != n) throw std::string("short input");
    return v;
  }
};

struct Out {
  std::deque<std::pair<std::string, std::vector<float>>> arrays;  // references stay valid as it grows
  std::vector<float>& add(const std::string& name, size_t rows, int B) {
    arrays.emplace_back(name, std::vector<float>(rows * size_t(B), 0.f));
    return arrays.back().second;
  }
};

// Every op for one topology T (segment code, or the chain's own unrolled code
// where the CUDA dispatch uses it).
template <class T, int NBI>
void run_all(const HostModel& hm, int B, int nf, const int* frames, const float* q, const float* qd,
             const float* qdd, const float* tau, const float* gbar, const float* dq, const float* dqd,
             const float* dx, const float* fext, Out& o, bool chain7) {
  ModelImage<NBI> img;
  hm.pack(&img);
  const int nb = hm.nb, nq = hm.nq, nv = hm.nv;
  Frames fr{nf, {0}};
  for (int f = 0; f < nf; ++f) fr.body[f] = frames[f];
  auto& pose = o.add("pose", 12 * nb, B);
  auto& J = o.add("J", size_t(nf) * 6 * nv, B);
  auto& tau_r = o.add("rnea", nv, B);
  auto& M = o.add("M", size_t(nv) * nv, B);
  auto& LD = o.add("LD", size_t(nv) * (nv + 1) / 2, B);
  auto& qdd_a = o.add("aba", nv, B);
  auto& rq = o.add("rnea_vjp_q", nq, B);
  auto& rqd = o.add("rnea_vjp_qd", nv, B);
  auto& rqdd = o.add("rnea_vjp_qdd", nv, B);
  auto& aq = o.add("aba_vjp_q", nq, B);
  auto& aqd = o.add("aba_vjp_qd", nv, B);
  auto& at = o.add("aba_vjp_tau", nv, B);
  auto& dtau = o.add("rnea_jvp", nv, B);
  auto& dqdd = o.add("aba_jvp", nv, B);
  auto& dpose = o.add("fk_jvp", size_t(6) * nf, B);
  auto& tau_e = o.add("rnea_ext", nv, B);
  auto& qdd_e = o.add("aba_ext", nv, B);
  auto& osc_t = o.add("osc", nv, B);
  auto& osc_l = o.add("osc_lambda", 36, B);
  const int task = frames[nf - 1];
  for (int b = 0; b < B; ++b) {
    const Col col{B, b};
    fk_seg<T, ModelImage<NBI>, Col, true>(img, q, pose.data(), fr, J.data(), col);
    rnea_seg<T>(img, q, qd, qdd, tau_r.data(), col);
    crba_seg<T, ModelImage<NBI>, Col, true, 3>(img, q, M.data(), LD.data(), col);
    {
      P3Local<T::NBMAX> P;
      aba_seg<T>(img, q, qd, tau, qdd_a.data(), col, P);
    }
    rnea_jvp_seg<T>(img, q, qd, qdd, dq, dqd, dx, JvpToGlobal<T, Col>{nullptr, dtau.data(), col}, col);
    if (chain7) {
      using C7 = ChainTopo<7>;
      rnea_vjp_chain<7>(img, q, qd, qdd, RhsFromGlobal<C7, Col>{gbar, col},
                        vjp_sink<C7>(img, q, rq.data(), rqd.data(), rqdd.data(), 1.f, col), col);
      aba_vjp_chain_one<7>(img, q, qd, qdd_a.data(), gbar, aq.data(), aqd.data(), at.data(), col);
      aba_jvp_chain_one<7>(img, q, qd, qdd_a.data(), dq, dqd, dx, dqdd.data(), col);
      fk_jvp_chain<7>(img, q, dq, fr, dpose.data(), col);
      rnea_one<C7>(img, q, qd, qdd, tau_e.data(), col);
      ext_tau_chain<7>(img, q, fext, col, SubFromGlobal<C7>{tau_e.data(), ColT<false>{B, b}});
    } else {
      rnea_vjp_seg_one<T>(img, q, qd, qdd, gbar, rq.data(), rqd.data(), rqdd.data(), col);
      aba_vjp_seg_one<T>(img, q, qd, tau, qdd_a.data(), gbar, aq.data(), aqd.data(), at.data(), col);
      aba_jvp_seg_one<T>(img, q, qd, qdd_a.data(), dq, dqd, dx, dqdd.data(), col);
      fk_jvp_seg<T>(img, q, dq, fr, dpose.data(), col);
      // as k_rnea_ext: the forces inside RNEA's outward sweep
      rnea_seg<T, ModelImage<NBI>, Col, false, true>(img, q, qd, qdd, tau_e.data(), col, -1, SV{}, fext);
    }
    // operational-space control of the last frame, task accelerations = the
    // first six rows of dx
    if (chain7)
      osc_chain<7>(img, task, q, qd, dx, osc_t.data(), osc_l.data(), col);
    else
      osc_seg<T>(img, task, q, qd, dx, osc_t.data(), osc_l.data(), col);
    {  // ABA with external forces, as k_aba_ext on trees: the forces in the bias forces of its sweeps
      P3Local<T::NBMAX> P;
      aba_seg_core<T, ModelImage<NBI>, true, RhsFromGlobal<T, Col>, OutToGlobal<T, Col>, Col, P3Local<T::NBMAX>,
                   true>(img, q, qd, RhsFromGlobal<T, Col>{tau, col}, OutToGlobal<T, Col>{qdd_e.data(), col}, col, P,
                         fext);
    }
  }
}

// The lane-group sweeps (lg.cuh) for trees of up to 32 bodies: the lanes of
// one instance run one after another within each step, the dataflow of the
// lockstep kernel; the plan's invariants are checked first.
std::string check_plan(const HostModel& hm) {
  const LanePlan& P = hm.lane_plan;
  const int n = hm.nb;
  std::vector<int> step(n, -1), lane(n, -1);
  if (P.T < 1 || P.T > n) return "plan: bad step count";
  for (int t = 0; t < P.T; ++t)
    for (int l = 0; l < kLgLanes; ++l) {
      const int i = P.body[t][l];
      if (i < -1 || i >= n) return "plan: bad body";
      if (i >= 0) {
        if (step[i] >= 0) return "plan: body scheduled twice";
        step[i] = t;
        lane[i] = l;
      }
    }
  for (int i = 0; i < n; ++i) {
    if (step[i] < 0) return "plan: body not scheduled";
    if (P.flag[step[i]][lane[i]] & kLgCarry) {  // the next step on the lane is a child
      const int c = step[i] + 1 < P.T ? P.body[step[i] + 1][lane[i]] : -1;
      if (c < 0 || hm.parent[c] != i) return "plan: carry without a child";
    }
    const int p = hm.parent[i];
    if (p < 0) continue;
    if (step[p] >= step[i]) return "plan: child before parent";
    const bool reg = lane[p] == lane[i] && step[p] == step[i] - 1;
    const int fl = P.flag[step[i]][lane[i]];
    if (reg == bool(fl & kLgLoad)) return "plan: outward load flag";
    if (!reg && (P.oslot[p] < 0 || !(P.flag[step[p]][lane[p]] & kLgStoreOut))) return "plan: missing outward slot";
    if (reg == bool(fl & kLgStoreIn)) return "plan: inward store flag";
    if (reg && !(P.flag[step[p]][lane[p]] & kLgCarry)) return "plan: carry flag";
    bool listed = false;
    for (int r = 0; r < P.rc_count[p]; ++r) listed = listed || P.rc_list[P.rc_first[p] + r] == i;
    if (listed == reg) return "plan: remote child list";
  }
  return "";
}

template <bool FREE>
void run_lane_groups(const HostModel& hm, int B, int nf, const int* frames, const float* q, const float* qd,
                     const float* qdd, const float* tau, const float* gbar, Out& o) {
  ModelImage<32> img;
  hm.pack(&img);
  const LanePlan& P = hm.lane_plan;
  auto& tau_r = o.add("rnea_lg", hm.nv, B);
  auto& bias = o.add("bias_lg", hm.nv, B);
  auto& qdd_a = o.add("aba_lg", hm.nv, B);
  auto& pose_lg = o.add("fk_lg_pose", 12 * hm.nb, B);
  auto& J_lg = o.add("fk_lg_J", size_t(nf) * 6 * hm.nv, B);
  std::vector<float> sf(lg_fk_floats(hm.nb, P.n_oslot), 0.f);
  Frames fr{nf, {0}};
  for (int f = 0; f < nf; ++f) fr.body[f] = frames[f];
  auto& Mlg = o.add("crba_lg_M", size_t(hm.nv) * hm.nv, B);
  auto& LDlg = o.add("crba_lg_LD", size_t(hm.nv) * (hm.nv + 1) / 2, B);
  std::vector<float> sc(lg_crba_floats(hm.nb, P.n_islot), 0.f);
  auto& rq = o.add("rnea_vjp_lg_q", hm.nq, B);
  auto& rqd = o.add("rnea_vjp_lg_qd", hm.nv, B);
  auto& rqdd = o.add("rnea_vjp_lg_qdd", hm.nv, B);
  auto& aq = o.add("aba_vjp_lg_q", hm.nq, B);
  auto& aqd = o.add("aba_vjp_lg_qd", hm.nv, B);
  auto& at = o.add("aba_vjp_lg_tau", hm.nv, B);
  std::vector<float> sr(lg_rnea_floats(hm.nb, P.n_oslot, P.n_islot), 0.f);
  std::vector<float> sa(lg_aba_floats(hm.nb, P.n_oslot, P.n_islot), 0.f);
  std::vector<float> sv(lg_vjp_floats(hm.nb, P.n_oslot, P.n_islot), 0.f);
  std::vector<float> sav(lg_aba_vjp_floats(hm.nb, hm.nv, P.n_oslot, P.n_islot), 0.f);
  using T = SegTopo<32, FREE>;
  for (int b = 0; b < B; ++b) {
    const Col col{B, b};
    for (int pass = 0; pass < 2; ++pass) {
      std::vector<RneaLg<FREE, Col>> L;
      for (int l = 0; l < kLgLanes; ++l)
        L.push_back(RneaLg<FREE, Col>{img, P, LgScratch{sr.data(), 1}, col, l, true, q, qd, pass ? nullptr : qdd,
                                      pass ? bias.data() : tau_r.data()});
      for (int t = 0; t < P.T; ++t)
        for (auto& x : L) x.out_step(t);
      for (int t = P.T - 1; t >= 0; --t)
        for (auto& x : L) x.in_step(t);
    }
    using AbaL = AbaLg<FREE, true, Col, RhsFromGlobal<T, Col>, OutToGlobal<T, Col>>;
    std::vector<AbaL> L;
    for (int l = 0; l < kLgLanes; ++l)
      L.push_back(AbaL{img, P, LgScratch{sa.data(), 1}, col, l, true, q, qd, RhsFromGlobal<T, Col>{tau, col},
                       OutToGlobal<T, Col>{qdd_a.data(), col}});
    for (int t = 0; t < P.T; ++t)
      for (auto& x : L) x.vel_step(t);
    for (int t = P.T - 1; t >= 0; --t)
      for (auto& x : L) x.inward_step(t);
    for (int t = 0; t < P.T; ++t)
      for (auto& x : L) x.acc_step(t);
    // FK and Jacobians (the structural zeros stay as the output was cleared)
    using FL = FkLg<FREE, Col>;
    std::vector<FL> Fk;
    for (int l = 0; l < kLgLanes; ++l)
      Fk.push_back(FL{img, P, LgScratch{sf.data(), 1}, col, l, true, q, pose_lg.data(), fr, J_lg.data()});
    for (int t = 0; t < P.T; ++t)
      for (auto& x : Fk) x.out_step(t);
    for (auto& x : Fk) x.jacobians();
    // CRBA + L^T D L (the structural zeros stay as the output was cleared)
    using CL = CrbaLg<FREE, Col>;
    std::vector<CL> Cg;
    for (int l = 0; l < kLgLanes; ++l)
      Cg.push_back(CL{img, P, LgScratch{sc.data(), 1}, col, l, true, q, Mlg.data(), LDlg.data()});
    for (int t = 0; t < P.T; ++t)
      for (auto& x : Cg) x.sincos_step(t);
    for (int t = P.T - 1; t >= 0; --t)
      for (auto& x : Cg) x.in_step(t);
    // the RNEA adjoint
    using VjpL = RneaVjpLg<FREE, Col, RhsFromGlobal<T, Col>, VjpToGlobal<T, Col>>;
    std::vector<VjpL> V;
    for (int l = 0; l < kLgLanes; ++l)
      V.push_back(VjpL{img, P, LgScratch{sv.data(), 1}, col, l, true, q, qd, qdd, RhsFromGlobal<T, Col>{gbar, col},
                       vjp_sink<T>(img, q, rq.data(), rqd.data(), rqdd.data(), 1.f, col)});
    for (int t = 0; t < P.T; ++t)
      for (auto& x : V) x.out_step(t);
    for (int t = P.T - 1; t >= 0; --t)
      for (auto& x : V) x.in_step(t);
    // the ABA adjoint at this instance's own forward result, as the kernel is run
    const int W0 = lg_aba_floats(hm.nb, P.n_oslot, P.n_islot);
    const LgScratch S{sav.data(), 1};
    using WL = AbaLg<FREE, false, Col, RhsFromGlobal<T, Col>, OutToLgVec<T, Col>>;
    std::vector<WL> W;
    for (int l = 0; l < kLgLanes; ++l)
      W.push_back(WL{img, P, S, col, l, true, q, qd, RhsFromGlobal<T, Col>{gbar, col},
                     OutToLgVec<T, Col>{S, W0, at.data(), col}});
    for (int t = 0; t < P.T; ++t)
      for (auto& x : W) x.vel_step(t);
    for (int t = P.T - 1; t >= 0; --t)
      for (auto& x : W) x.inward_step(t);
    for (int t = 0; t < P.T; ++t)
      for (auto& x : W) x.acc_step(t);
    using AVL = RneaVjpLg<FREE, Col, LgVec<T>, VjpToGlobal<T, Col>>;
    std::vector<AVL> A;
    for (int l = 0; l < kLgLanes; ++l)
      A.push_back(AVL{img, P, LgScratch{sav.data() + W0 + hm.nv, 1}, col, l, true, q, qd, qdd_a.data(),
                      LgVec<T>{S, W0}, vjp_sink<T>(img, q, aq.data(), aqd.data(), nullptr, -1.f, col)});
    for (int t = 0; t < P.T; ++t)
      for (auto& x : A) x.out_step(t);
    for (int t = P.T - 1; t >= 0; --t)
      for (auto& x : A) x.in_step(t);
  }
}

}  // namespace

int main(int argc, char** argv) {
  if (argc != 3) {
    std::fprintf(stderr, "usage: %s <input> <output>\n", argv[0]);
    return 2;
  }
  try {
    FILE* f = std::fopen(argv[1], "rb");
    if (!f) throw std::string("cannot open input");
    Reader r{f};
    const auto hdr = r.take<int32_t>(3);
    const int n = hdr[0], B = hdr[1], nf = hdr[2];
    const auto parent = r.take<int32_t>(n);
    const auto jt = r.take<int32_t>(n);
    const auto axis = r.take<double>(3 * n);
    const auto place = r.take<double>(12 * n);
    const auto inert = r.take<double>(10 * n);
    const auto grav = r.take<double>(3);
    const auto frames = r.take<int32_t>(nf);
    HostModel hm;
    const std::string err =
        build_model(n, parent.data(), jt.data(), axis.data(), place.data(), inert.data(), grav.data(), &hm);
    if (!err.empty()) throw err;
    const int nq = hm.nq, nv = hm.nv;
    const auto q = r.take<float>(size_t(nq) * B);
    const auto qd = r.take<float>(size_t(nv) * B);
    const auto qdd = r.take<float>(size_t(nv) * B);
    const auto tau = r.take<float>(size_t(nv) * B);
    const auto gbar = r.take<float>(size_t(nv) * B);
    const auto dq = r.take<float>(size_t(nv) * B);
    const auto dqd = r.take<float>(size_t(nv) * B);
    const auto dx = r.take<float>(size_t(nv) * B);
    const auto fext = r.take<float>(size_t(6) * n * B);
    std::fclose(f);
    Out o;
    const bool chain7 = hm.kind == kKindChain && n == 7;
    if (chain7)
      run_all<SegTopo<8, false>, 8>(hm, B, nf, frames.data(), q.data(), qd.data(), qdd.data(), tau.data(),
                                    gbar.data(), dq.data(), dqd.data(), dx.data(), fext.data(), o, true);
    else if (hm.free_root)
      run_all<SegTopo<64, true>, 64>(hm, B, nf, frames.data(), q.data(), qd.data(), qdd.data(), tau.data(),
                                     gbar.data(), dq.data(), dqd.data(), dx.data(), fext.data(), o, false);
    else
      run_all<SegTopo<64, false>, 64>(hm, B, nf, frames.data(), q.data(), qd.data(), qdd.data(), tau.data(),
                                      gbar.data(), dq.data(), dqd.data(), dx.data(), fext.data(), o, false);
    if (n <= 32) {
      const std::string perr = check_plan(hm);
      if (!perr.empty()) throw perr;
      if (hm.free_root)
        run_lane_groups<true>(hm, B, nf, frames.data(), q.data(), qd.data(), qdd.data(), tau.data(), gbar.data(), o);
      else
        run_lane_groups<false>(hm, B, nf, frames.data(), q.data(), qd.data(), qdd.data(), tau.data(), gbar.data(),
                               o);
    }
    FILE* g = std::fopen(argv[2], "wb");
    if (!g) throw std::string("cannot open output");
    const int32_t count = static_cast<int32_t>(o.arrays.size());
    std::fwrite(&count, sizeof(count), 1, g);
    for (auto& a : o.arrays) {
      char name[32] = {0};
      std::strncpy(name, a.first.c_str(), sizeof(name) - 1);
      const int64_t len = static_cast<int64_t>(a.second.size());
      std::fwrite(name, 1, sizeof(name), g);
      std::fwrite(&len, sizeof(len), 1, g);
      std::fwrite(a.second.data(), sizeof(float), a.second.size(), g);
    }
    std::fclose(g);
  } catch (const std::string& e) {
    std::fprintf(stderr, "host_kernels: %s\n", e.c_str());
    return 1;
  }
  return 0;
}
