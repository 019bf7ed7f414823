// Lane-group tree sweeps: one instance spread over kLgLanes lanes of a warp
// (lanes over the tree's branches), for batches too small to fill the GPU
// with one thread per instance. Each lane walks its own root-to-leaf paths of
// the model's LanePlan (model_image.h) in lockstep with the others: outward
// sweeps run the plan's steps forwards, inward sweeps backwards, with a warp
// barrier after every step. Per-body state lives in shared memory; state
// crosses lanes only where a path starts, through the plan's slots. The
// per-body arithmetic is that of the segment kernels (seg.cuh); only the
// order of the additions at a branch body differs.
//
// Each sweep is a step function of one lane's state (RneaLg, AbaLg): the
// kernel runs for t: step(t); __syncwarp(); on the device, and a host
// harness can run the lanes of one instance one after another within each
// step, which is the same dataflow.
#pragma once
#include "seg.cuh"

namespace frax {

constexpr int kLgBlock = 64;                    // threads per block
constexpr int kLgInst = kLgBlock / kLgLanes;    // instances per block
constexpr int kLgImgBytes = (int(sizeof(ModelImage<32>)) + 15) / 16 * 16;
constexpr int kLgPlanBytes = (int(sizeof(LanePlan)) + 15) / 16 * 16;

// Per-instance scratch floats. ABA: per body cos, sin, velocity and the six
// factors of its outward step, velocity + acceleration slots, articulated
// inertia + bias slots. RNEA: per body cos, sin and net force, velocity +
// acceleration slots, force slots.
inline int lg_aba_floats(int nb, int no, int ni) { return 14 * nb + 12 * no + 27 * ni; }
inline int lg_rnea_floats(int nb, int no, int ni) { return 8 * nb + 12 * no + 6 * ni; }

// One instance's scratch, field f at base[f * stride] (instance-major in
// shared memory: stride = instances per block).
struct LgScratch {
  float* base;
  int stride;
  FD float& operator[](int f) const { return base[f * stride]; }
  FD SV get6(int f) const {
    return SV{mk((*this)[f], (*this)[f + 1], (*this)[f + 2]), mk((*this)[f + 3], (*this)[f + 4], (*this)[f + 5])};
  }
  FD void put6(int f, const SV& x) const {
    (*this)[f] = x.w.x; (*this)[f + 1] = x.w.y; (*this)[f + 2] = x.w.z;
    (*this)[f + 3] = x.v.x; (*this)[f + 4] = x.v.y; (*this)[f + 5] = x.v.z;
  }
  FD void put_ai(int f, const AI& I) const {
    for (int k = 0; k < 6; ++k) (*this)[f + k] = I.A[k];
    for (int k = 0; k < 9; ++k) (*this)[f + 6 + k] = I.B[k];
    for (int k = 0; k < 6; ++k) (*this)[f + 15 + k] = I.C[k];
  }
  FD void add_ai(int f, AI& I) const {
    for (int k = 0; k < 6; ++k) I.A[k] += (*this)[f + k];
    for (int k = 0; k < 9; ++k) I.B[k] += (*this)[f + 6 + k];
    for (int k = 0; k < 6; ++k) I.C[k] += (*this)[f + 15 + k];
  }
};

// RNEA (Eq. 1, f = 0) for one lane; qdd == nullptr gives the bias forces.
template <bool FREE, class C>
struct RneaLg {
  using T = SegTopo<32, FREE>;
  const ModelImage<32>& M;
  const LanePlan& P;
  LgScratch S;
  C col;
  int lane;
  bool valid;
  const float *q, *qd, *qdd;
  float* tau;
  SV v, a, F;  // carried from this lane's previous step
  FD int CS() const { return 0; }
  FD int SN() const { return M.nb; }
  FD int F0() const { return 2 * M.nb; }
  FD int OS() const { return 8 * M.nb; }
  FD int IS() const { return 8 * M.nb + 12 * P.n_oslot; }

  // outward: velocities, accelerations and each body's net force
  FD void out_step(int t) {
    const int i = P.body[t][lane];
    if (!valid || i < 0) return;
    const int fl = P.flag[t][lane];
    const BodyImage& bi = M.body[i];
    const RBI I = rbi_of(bi);
    const SV ag = gravity_acc(M.g);
    if (FREE && i == 0) {
      const RootPose RP = root_pose(M, q, col);
      v = load6(qd, 0, col);
      a = SV{mk(0, 0, 0), rotT(RP.E, ag.v)};
      if (qdd) a = a + load6(qdd, 0, col);
    } else {
      const int p = M.parent[i];
      if (p < 0) {
        v = szero();
        a = ag;
      } else if (fl & kLgLoad) {
        v = S.get6(OS() + 12 * P.oslot[p]);
        a = S.get6(OS() + 12 * P.oslot[p] + 6);
      }
      float sn, cs;
      joint_sincos(col.in(q, iq_of<T>(i)) + bi.th0, &sn, &cs);
      S[CS() + i] = cs;
      S[SN() + i] = sn;
      const float qdi = col.in(qd, iv_of<T>(i));
      const float qddi = qdd ? col.in(qdd, iv_of<T>(i)) : 0.f;
      with_dh(bi.dh, [&](auto dh) {
        v = mot_in(bi, cs, sn, v, dh);
        a = mot_in(bi, cs, sn, a, dh);
      });
      v.w.z += qdi;
      a.w.z += qddi;
      a = a + ez_velprod(v, qdi);
    }
    S.put6(F0() + 6 * i, crf_add(rbi_mul(I, a), v, rbi_mul(I, v)));
    if (fl & kLgStoreOut) {
      S.put6(OS() + 12 * P.oslot[i], v);
      S.put6(OS() + 12 * P.oslot[i] + 6, a);
    }
  }
  // inward: forces summed over each subtree, tau_i = S_i^T F_i
  FD void in_step(int t) {
    const int i = P.body[t][lane];
    if (!valid || i < 0) return;
    const int fl = P.flag[t][lane];
    SV Fi = S.get6(F0() + 6 * i);
    if (fl & kLgCarry) Fi = Fi + F;
    for (int r = 0; r < P.rc_count[i]; ++r) Fi = Fi + S.get6(IS() + 6 * P.islot[P.rc_list[P.rc_first[i] + r]]);
    if (FREE && i == 0) {
      store6(tau, 0, col, Fi);
      return;
    }
    col.out(tau, iv_of<T>(i), Fi.w.z);
    const BodyImage& bi = M.body[i];
    const float cs = S[CS() + i], sn = S[SN() + i];
    with_dh(bi.dh, [&](auto dh) { F = frc_out(bi, cs, sn, Fi, dh); });
    if (fl & kLgStoreIn) S.put6(IS() + 6 * P.islot[i], F);
  }
};

// ABA (Eq. 2, f = 0) for one lane: velocities outward, articulated inertias
// inward (each body's outward-step factors kept in the scratch), then
// accelerations outward.
template <bool FREE, class C>
struct AbaLg {
  using T = SegTopo<32, FREE>;
  const ModelImage<32>& M;
  const LanePlan& P;
  LgScratch S;
  C col;
  int lane;
  bool valid;
  const float *q, *qd, *tau;
  float* qdd;
  SV v, a, pa, a0;  // carried from this lane's previous step; a0: the free root's acceleration
  AI Ia;
  V3 gam;           // free root: gravity in root coordinates
  FD int CS() const { return 0; }
  FD int SN() const { return M.nb; }
  FD int V0() const { return 2 * M.nb; }
  FD int P0() const { return 8 * M.nb; }
  FD int OS() const { return 14 * M.nb; }
  FD int IS() const { return 14 * M.nb + 12 * P.n_oslot; }

  FD void vel_step(int t) {
    const int i = P.body[t][lane];
    if (!valid || i < 0) return;
    const int fl = P.flag[t][lane];
    if (FREE && i == 0) {
      const RootPose RP = root_pose(M, q, col);
      gam = rotT(RP.E, gravity_acc(M.g).v);
      v = load6(qd, 0, col);
    } else {
      const BodyImage& bi = M.body[i];
      const int p = M.parent[i];
      if (p < 0) v = szero();
      else if (fl & kLgLoad) v = S.get6(OS() + 12 * P.oslot[p]);
      float sn, cs;
      joint_sincos(col.in(q, iq_of<T>(i)) + bi.th0, &sn, &cs);
      S[CS() + i] = cs;
      S[SN() + i] = sn;
      with_dh(bi.dh, [&](auto dh) { v = mot_in(bi, cs, sn, v, dh); });
      v.w.z += col.in(qd, iv_of<T>(i));
    }
    S.put6(V0() + 6 * i, v);
    if (fl & kLgStoreOut) S.put6(OS() + 12 * P.oslot[i], v);
  }
  FD void inward_step(int t) {
    const int i = P.body[t][lane];
    if (!valid || i < 0) return;
    const int fl = P.flag[t][lane];
    const BodyImage& bi = M.body[i];
    const RBI Ib = rbi_of(bi);
    const SV vi = S.get6(V0() + 6 * i);
    AI IA = ai_of(Ib);
    SV pA = crf(vi, rbi_mul(Ib, vi));
    if (fl & kLgCarry) {
      ai_add(IA, Ia);
      pA = pA + pa;
    }
    for (int r = 0; r < P.rc_count[i]; ++r) {
      const int f = IS() + 27 * P.islot[P.rc_list[P.rc_first[i] + r]];
      S.add_ai(f, IA);
      pA = pA + S.get6(f + 21);
    }
    if (FREE && i == 0) {
      a0 = spd6_solve(IA, load6(tau, 0, col) - pA);
      return;
    }
    const float cs = S[CS() + i], sn = S[SN() + i];
    const SV cb = ez_velprod(vi, col.in(qd, iv_of<T>(i)));
    const SV U = ai_col_z(IA);
    const float dinv = rcp(U.w.z);
    const float ud = (col.in(tau, iv_of<T>(i)) - pA.w.z) * dinv;
    SV Ud = dinv * U;
    Ud.w.z = 1.f;
    S[P0() + 6 * i] = Ud.w.x;
    S[P0() + 6 * i + 1] = Ud.w.y;
    S[P0() + 6 * i + 2] = Ud.v.x;
    S[P0() + 6 * i + 3] = Ud.v.y;
    S[P0() + 6 * i + 4] = Ud.v.z;
    S[P0() + 6 * i + 5] = ud;
    Ia = IA;
    ai_rank1_sub_d(Ia, Ud, U);
    pa = pA + ai_mul(Ia, cb) + ud * U;
    with_dh(bi.dh, [&](auto dh) {
      ai_out(bi, cs, sn, Ia, dh);
      pa = frc_out(bi, cs, sn, pa, dh);
    });
    if (fl & kLgStoreIn) {
      const int f = IS() + 27 * P.islot[i];
      S.put_ai(f, Ia);
      S.put6(f + 21, pa);
    }
  }
  FD void acc_step(int t) {
    const int i = P.body[t][lane];
    if (!valid || i < 0) return;
    const int fl = P.flag[t][lane];
    if (FREE && i == 0) {
      a = a0;
      store6(qdd, 0, col, a0 - SV{mk(0, 0, 0), gam});
    } else {
      const BodyImage& bi = M.body[i];
      const int p = M.parent[i];
      if (p < 0) a = gravity_acc(M.g);
      else if (fl & kLgLoad) a = S.get6(OS() + 12 * P.oslot[p] + 6);
      const float cs = S[CS() + i], sn = S[SN() + i];
      const SV cb = ez_velprod(S.get6(V0() + 6 * i), col.in(qd, iv_of<T>(i)));
      with_dh(bi.dh, [&](auto dh) { a = mot_in(bi, cs, sn, a, dh) + cb; });
      const int f = P0() + 6 * i;
      const float x = S[f + 5] - (fmaf(S[f], a.w.x, fmaf(S[f + 1], a.w.y, a.w.z)) +
                                  fmaf(S[f + 2], a.v.x, fmaf(S[f + 3], a.v.y, S[f + 4] * a.v.z)));
      a.w.z += x;
      col.out(qdd, iv_of<T>(i), x);
    }
    if (fl & kLgStoreOut) S.put6(OS() + 12 * P.oslot[i] + 6, a);
  }
};

#ifdef __CUDACC__
// Stages the model image and the plan in shared memory (body constants are
// then read per lane without serialising on the constant cache).
__device__ __forceinline__ void lg_stage(const ModelImage<32>& Mg, const LanePlan& Pg, char* smem) {
  const float4* s1 = reinterpret_cast<const float4*>(&Mg);
  float4* d1 = reinterpret_cast<float4*>(smem);
  for (int k = threadIdx.x; k < int(sizeof(ModelImage<32>) / 16); k += kLgBlock) d1[k] = s1[k];
  const int4* s2 = reinterpret_cast<const int4*>(&Pg);
  int4* d2 = reinterpret_cast<int4*>(smem + kLgImgBytes);
  for (int k = threadIdx.x; k < int(sizeof(LanePlan) / 16); k += kLgBlock) d2[k] = s2[k];
  __syncthreads();
}

#define FRAX_LG_PROLOGUE()                                                                    \
  extern __shared__ __align__(16) char smem[];                                                \
  lg_stage(Mg, Pg, smem);                                                                     \
  const ModelImage<32>& M = *reinterpret_cast<const ModelImage<32>*>(smem);                   \
  const LanePlan& P = *reinterpret_cast<const LanePlan*>(smem + kLgImgBytes);                 \
  const int lane = threadIdx.x % kLgLanes, inst = threadIdx.x / kLgLanes;                     \
  const int64_t b = int64_t(blockIdx.x) * kLgInst + inst;                                     \
  const bool valid = b < B;                                                                   \
  const Col col{ld, valid ? b : 0};                                                           \
  const LgScratch S{reinterpret_cast<float*>(smem + kLgImgBytes + kLgPlanBytes) + inst, kLgInst};

template <bool FREE>
__global__ void __launch_bounds__(kLgBlock) k_rnea_lg(const __grid_constant__ ModelImage<32> Mg,
                                                      const __grid_constant__ LanePlan Pg, int64_t B, int64_t ld,
                                                      const float* __restrict__ q, const float* __restrict__ qd,
                                                      const float* __restrict__ qdd, float* __restrict__ tau) {
  FRAX_LG_PROLOGUE();
  RneaLg<FREE, Col> L{M, P, S, col, lane, valid, q, qd, qdd, tau};
  for (int t = 0; t < P.T; ++t) {
    L.out_step(t);
    __syncwarp();
  }
  for (int t = P.T - 1; t >= 0; --t) {
    L.in_step(t);
    __syncwarp();
  }
}

template <bool FREE>
__global__ void __launch_bounds__(kLgBlock) k_aba_lg(const __grid_constant__ ModelImage<32> Mg,
                                                     const __grid_constant__ LanePlan Pg, int64_t B, int64_t ld,
                                                     const float* __restrict__ q, const float* __restrict__ qd,
                                                     const float* __restrict__ tau, float* __restrict__ qdd) {
  FRAX_LG_PROLOGUE();
  AbaLg<FREE, Col> L{M, P, S, col, lane, valid, q, qd, tau, qdd};
  for (int t = 0; t < P.T; ++t) {
    L.vel_step(t);
    __syncwarp();
  }
  for (int t = P.T - 1; t >= 0; --t) {
    L.inward_step(t);
    __syncwarp();
  }
  for (int t = 0; t < P.T; ++t) {
    L.acc_step(t);
    __syncwarp();
  }
}
#undef FRAX_LG_PROLOGUE
#endif

}  // namespace frax
