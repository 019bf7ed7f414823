// Counts the FP32 operations of each kernel's formulation per instance by
// running the device code on the host with `float` replaced by a counting
// type (fma = 2 flops, add/sub/mul = 1; divisions, sqrt and sincos counted
// separately, outside the FMA-pipe roofline). Used by bench.py --count-flops.
//   g++ -std=c++17 -x c++ -I/usr/local/cuda/include -o flopcount flopcount.cu \
//        paper_2604_04310_gb300/csrc/model.cpp
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "paper_2604_04310_gb300/csrc/model.h"  // model image keeps real floats

struct Counts {
  long long add = 0, mul = 0, fma = 0, div = 0, sfu = 0;
};
static Counts g;

struct CF {
  float v;
  CF() = default;
  CF(float x) : v(x) {}
  CF(double x) : v(float(x)) {}
  CF(int x) : v(float(x)) {}
};
inline CF operator+(CF a, CF b) { g.add++; return CF(a.v + b.v); }
inline CF operator-(CF a, CF b) { g.add++; return CF(a.v - b.v); }
inline CF operator*(CF a, CF b) { g.mul++; return CF(a.v * b.v); }
inline CF operator/(CF a, CF b) { g.div++; return CF(a.v / b.v); }
inline CF operator-(CF a) { return CF(-a.v); }
inline CF& operator+=(CF& a, CF b) { g.add++; a.v += b.v; return a; }
inline CF& operator-=(CF& a, CF b) { g.add++; a.v -= b.v; return a; }
inline CF& operator*=(CF& a, CF b) { g.mul++; a.v *= b.v; return a; }
inline CF fmaf(CF a, CF b, CF c) { g.fma++; return CF(std::fma(a.v, b.v, c.v)); }
inline CF sqrtf(CF a) { g.sfu++; return CF(std::sqrt(a.v)); }
inline CF rsqrtf(CF a) { g.sfu++; return CF(1.f / std::sqrt(a.v)); }
inline void sincosf(CF x, CF* s, CF* c) { g.sfu++; s->v = std::sin(x.v); c->v = std::cos(x.v); }

#define float CF
#include "paper_2604_04310_gb300/csrc/osc.cuh"
#include "paper_2604_04310_gb300/csrc/ext.cuh"
#include "paper_2604_04310_gb300/csrc/jvp.cuh"
#undef float

using namespace frax;

// One JVP step back through a joint, and how many a sweep makes (bodies after
// the first of each revolute segment): the direct formulation that stores the
// forward state does not make them.
template <class Img>
void count_stepback(const Img& M) {
  SV v{mk(0.1f, 0.2f, 0.3f), mk(0.4f, 0.5f, 0.6f)}, a = v, dv = v, da = v;
  g = Counts{};
  jvp_step_back(M.body[M.nb - 1], CF(0.8f), CF(0.6f), CF(0.1f), CF(0.2f), CF(0.3f), CF(0.4f), CF(0.5f), v, a, dv, da, DhOn{});
  int n = 0;
  for (int s = (M.free_root ? 1 : 0); s < M.n_seg; ++s) n += M.seg_len[s] - 1;
  printf("  \"jvp_stepback\": {\"flops\": %lld, \"count\": %d},\n", 2 * g.fma + g.add + g.mul, n);
  g = Counts{};
}


template <class T, class Img>
void count(const Img& M, int nf, const int* frames) {
  int nq = M.nq, nv = M.nv, nb = M.nb;
  std::vector<CF> q(nq, CF(0.3f)), qd(nv, CF(0.2f)), qdd(nv, CF(0.1f)), tau(nv, CF(0.5f)), gb(nv, CF(0.7f));
  if (M.free_root) { q[3] = q[4] = q[5] = CF(0.f); q[6] = CF(1.f); }
  std::vector<CF> o1(nb * 12 + 64), o2(nf * 6 * nv + 64), o3(nv * nv + 64), o4(nv * (nv + 1) / 2 + 64), o5(nq + 8), o6(nv + 8), o7(nv + 8);
  Col col{1, 0};
  Frames fr{nf, {0}};
  for (int f = 0; f < nf; ++f) fr.body[f] = frames[f];
  auto rep = [&](const char* name) {
    printf("  \"%s\": {\"flops\": %lld, \"fma\": %lld, \"add\": %lld, \"mul\": %lld, \"div\": %lld, \"sfu\": %lld},\n",
           name, 2 * g.fma + g.add + g.mul, g.fma, g.add, g.mul, g.div, g.sfu);
    g = Counts{};
  };
  g = Counts{};
  if constexpr (T::kSeg) {
    static P3Local<T::NBMAX> P3;
    fk_seg<T>(M, q.data(), o1.data(), fr, o2.data(), col); rep("fk_jac");
    fk_seg<T>(M, q.data(), o1.data(), Frames{0, {0}}, nullptr, col); rep("fk");
    rnea_seg<T>(M, q.data(), qd.data(), qdd.data(), o6.data(), col); rep("rnea");
    rnea_seg<T>(M, q.data(), qd.data(), nullptr, o6.data(), col); rep("bias");
    crba_seg<T>(M, q.data(), o3.data(), o4.data(), col); rep("crba_ltdl");
    crba_seg<T>(M, q.data(), o3.data(), nullptr, col); rep("crba");
    aba_seg<T>(M, q.data(), qd.data(), tau.data(), o6.data(), col, P3); rep("aba");
  } else {
    fk_one<T>(M, q.data(), o1.data(), fr, o2.data(), col); rep("fk_jac");
    fk_one<T>(M, q.data(), o1.data(), Frames{0, {0}}, nullptr, col); rep("fk");
    rnea_one<T>(M, q.data(), qd.data(), qdd.data(), o6.data(), col); rep("rnea");
    rnea_one<T>(M, q.data(), qd.data(), nullptr, o6.data(), col); rep("bias");
    crba_one<T>(M, q.data(), o3.data(), o4.data(), col); rep("crba_ltdl");
    crba_one<T>(M, q.data(), o3.data(), nullptr, col); rep("crba");
    aba_one<T>(M, q.data(), qd.data(), tau.data(), o6.data(), col); rep("aba");
  }
  {
    std::vector<CF> fe(6 * nb + 8, CF(0.4f)), o8(nv + 8);
    LocalVec<T> w;
    ext_tau<T>(M, q.data(), fe.data(), col, OutToLocal<T>{&w}); rep("ext_tau");
  }
  if constexpr (T::kSeg) {
    std::vector<CF> dq(nv, CF(0.3f)), dqd(nv, CF(0.2f)), dx(nv, CF(0.1f)), o9(nv + 8), o10(6 * nf + 8);
    rnea_jvp_seg<T>(M, q.data(), qd.data(), qdd.data(), dq.data(), dqd.data(), dx.data(),
                    JvpToGlobal<T, Col>{o6.data(), o9.data(), col}, col); rep("rnea_jvp");
    aba_jvp_seg_one<T>(M, q.data(), qd.data(), qdd.data(), dq.data(), dqd.data(), dx.data(), o9.data(), col);
    rep("aba_jvp");
    fk_jvp_seg<T>(M, q.data(), dq.data(), fr, o10.data(), col); rep("fk_jvp");
    count_stepback(M);
    rnea_vjp_seg_one<T>(M, q.data(), qd.data(), qdd.data(), gb.data(), o5.data(), o6.data(), o7.data(), col); rep("rnea_vjp");
    aba_vjp_seg_one<T>(M, q.data(), qd.data(), tau.data(), qdd.data(), gb.data(), o5.data(), o6.data(), o7.data(), col); rep("aba_vjp");
    std::vector<CF> lam(36 + 8);
    osc_seg<T>(M, frames[nf - 1], q.data(), qd.data(), qdd.data(), o6.data(), nullptr, col); rep("osc");
    osc_seg<T>(M, frames[nf - 1], q.data(), qd.data(), qdd.data(), o6.data(), lam.data(), col); rep("osc_lambda");
  }
}

// The direct formulations that keep per-body state instead of recomputing it
// (dyn.cuh, one thread per instance, no segments): the algorithm's own work,
// the basis of the roofline where a kernel trades flops for registers.
template <class T, class Img>
void count_direct(const Img& M) {
  int nq = M.nq, nv = M.nv;
  std::vector<CF> q(nq, CF(0.3f)), qd(nv, CF(0.2f)), qdd(nv, CF(0.1f)), tau(nv, CF(0.5f)), gb(nv, CF(0.7f));
  if (M.free_root) { q[3] = q[4] = q[5] = CF(0.f); q[6] = CF(1.f); }
  std::vector<CF> o3(nv * nv + 64), o4(nv * (nv + 1) / 2 + 64), o5(nq + 8), o6(nv + 8), o7(nv + 8);
  Col col{1, 0};
  auto rep = [&](const char* name) {
    printf("  \"%s\": {\"flops\": %lld},\n", name, 2 * g.fma + g.add + g.mul);
    g = Counts{};
  };
  g = Counts{};
  crba_one<T>(M, q.data(), o3.data(), o4.data(), col); rep("direct_crba_ltdl");
  aba_one<T>(M, q.data(), qd.data(), tau.data(), o6.data(), col); rep("direct_aba");
  rnea_vjp_one<T>(M, q.data(), qd.data(), qdd.data(), gb.data(), o5.data(), o6.data(), o7.data(), col);
  rep("direct_rnea_vjp");
  aba_vjp_one<T>(M, q.data(), qd.data(), tau.data(), qdd.data(), gb.data(), o5.data(), o6.data(), o7.data(), col);
  rep("direct_aba_vjp");
}

// The chain's adjoints run on the segment code (SegTopo<8, false>).
template <class Img>
void count_chain_vjp(const Img& M) {
  using T = SegTopo<8, false>;
  int nq = M.nq, nv = M.nv;
  std::vector<CF> q(nq, CF(0.3f)), qd(nv, CF(0.2f)), qdd(nv, CF(0.1f)), tau(nv, CF(0.5f)), gb(nv, CF(0.7f));
  std::vector<CF> o5(nq + 8), o6(nv + 8), o7(nv + 8);
  Col col{1, 0};
  auto rep = [&](const char* name) {
    printf("  \"%s\": {\"flops\": %lld, \"fma\": %lld, \"add\": %lld, \"mul\": %lld, \"div\": %lld, \"sfu\": %lld},\n",
           name, 2 * g.fma + g.add + g.mul, g.fma, g.add, g.mul, g.div, g.sfu);
    g = Counts{};
  };
  g = Counts{};
  rnea_vjp_seg_one<T>(M, q.data(), qd.data(), qdd.data(), gb.data(), o5.data(), o6.data(), o7.data(), col); rep("rnea_vjp_seg");
  aba_vjp_chain_one<7>(M, q.data(), qd.data(), qdd.data(), gb.data(), o5.data(), o6.data(), o7.data(), col); rep("aba_vjp_chain");
  std::vector<CF> w(8);
  chain_minv<7>(M, q.data(), RhsFromGlobal<ChainTopo<7>, Col>{gb.data(), col}, w.data(), col); rep("minv_factor");
  rnea_one<ChainTopo<7>>(M, q.data(), qd.data(), nullptr, o6.data(), col);
  chain_minv<7>(M, q.data(), RhsFromGlobal<ChainTopo<7>, Col>{gb.data(), col}, w.data(), col);
  rep("aba_factor");
  std::vector<CF> dq(nv, CF(0.3f)), dqd(nv, CF(0.2f)), dx(nv, CF(0.1f)), o9(nv + 8), o10(6 + 8);
  rnea_jvp_seg<T>(M, q.data(), qd.data(), qdd.data(), dq.data(), dqd.data(), dx.data(),
                  JvpToGlobal<T, Col>{o6.data(), o9.data(), col}, col); rep("rnea_jvp");
  aba_jvp_chain_one<7>(M, q.data(), qd.data(), qdd.data(), dq.data(), dqd.data(), dx.data(), o9.data(), col);
  rep("aba_jvp");
  fk_jvp_seg<T>(M, q.data(), dq.data(), Frames{1, {6}}, o10.data(), col); rep("fk_jvp");
  count_stepback(M);
  std::vector<CF> lam(36 + 8);
  osc_seg<T>(M, 6, q.data(), qd.data(), qdd.data(), o6.data(), nullptr, col); rep("osc");
  osc_seg<T>(M, 6, q.data(), qd.data(), qdd.data(), o6.data(), lam.data(), col); rep("osc_lambda");
}

int main(int argc, char** argv) {
  // stdin: n, parent[n], joint_type[n], axis[3n], placement[12n], inertia[10n], gravity[3], nf, frames[nf]
  int n;
  if (scanf("%d", &n) != 1) return 1;
  std::vector<int32_t> parent(n), jt(n);
  std::vector<double> axis(3 * n), plc(12 * n), inr(10 * n), grav(3);
  for (auto& x : parent) scanf("%d", &x);
  for (auto& x : jt) scanf("%d", &x);
  for (auto& x : axis) scanf("%lf", &x);
  for (auto& x : plc) scanf("%lf", &x);
  for (auto& x : inr) scanf("%lf", &x);
  for (auto& x : grav) scanf("%lf", &x);
  int nf;
  scanf("%d", &nf);
  std::vector<int> frames(nf);
  for (auto& x : frames) scanf("%d", &x);
  HostModel hm;
  std::string err = build_model(n, parent.data(), jt.data(), axis.data(), plc.data(), inr.data(), grav.data(), &hm);
  if (!err.empty()) { fprintf(stderr, "%s\n", err.c_str()); return 1; }
  printf("{\n");
  if (hm.kind == kKindChain) {
    static ModelImage<7> img; hm.pack(&img); count<ChainTopo<7>>(img, nf, frames.data());
    count_direct<ChainTopo<7>>(img);
    static ModelImage<8> img8; hm.pack(&img8); count_chain_vjp(img8);
  } else if (hm.free_root) {
    static ModelImage<64> img; hm.pack(&img); count<SegTopo<64, true>>(img, nf, frames.data());
    count_direct<TreeTopo<64, true, true>>(img);
  } else {
    static ModelImage<64> img; hm.pack(&img); count<SegTopo<64, false>>(img, nf, frames.data());
    count_direct<TreeTopo<64, false, true>>(img);
  }
  printf("  \"nb\": %d, \"nv\": %d\n}\n", hm.nb, hm.nv);
  return 0;
}
