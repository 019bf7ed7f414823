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
FD int lg_aba_floats(int nb, int no, int ni) { return 14 * nb + 12 * no + 27 * ni; }
FD int lg_rnea_floats(int nb, int no, int ni) { return 8 * nb + 12 * no + 6 * ni; }

// Column accessor of the lane-group kernels: inputs are read from the
// block's staged copy in shared memory ([row][kLgInst], this instance's
// column), outputs written to the caller's global arrays.
struct LgCol {
  int64_t ld, b;  // global output column
  int inst;       // staged input column
  FD float in(const float* __restrict__ p, int k) const { return p[k * kLgInst + inst]; }
  // this instance's entry k of a global output
  template <class F>
  FD F* at(F* p, int k) const { return at_row(p + b, k, ld); }
  FD void out(float* __restrict__ p, int k, float v) const { st_cs(at(p, k), v); }
};

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
// accelerations outward. rhs(i) / rhs.root() give the joint forces, out(i, x)
// / out.root(a) take the accelerations. Without VEL: zero velocity and no
// gravity, i.e. x = M^-1 rhs (the solve of the ABA adjoint).
template <bool FREE, bool VEL, class C, class Rhs, class Out>
struct AbaLg {
  using T = SegTopo<32, FREE>;
  const ModelImage<32>& M;
  const LanePlan& P;
  LgScratch S;
  C col;
  int lane;
  bool valid;
  const float *q, *qd;
  Rhs rhs;
  Out out;
  SV v, a, pa, a0;  // carried from this lane's previous step; a0: the free root's acceleration
  AI Ia;
  V3 gam;           // free root: gravity in root coordinates
  FD int CS() const { return 0; }
  FD int SN() const { return M.nb; }
  FD int V0() const { return 2 * M.nb; }
  FD int P0() const { return 8 * M.nb; }
  FD int OS() const { return 14 * M.nb; }
  FD int IS() const { return 14 * M.nb + 12 * P.n_oslot; }
  FD SV ag() const { return VEL ? gravity_acc(M.g) : szero(); }

  // velocities (and each joint's cos, sin)
  FD void vel_step(int t) {
    const int i = P.body[t][lane];
    if (!valid || i < 0) return;
    const int fl = P.flag[t][lane];
    if (FREE && i == 0) {
      if (VEL) {
        const RootPose RP = root_pose(M, q, col);
        gam = rotT(RP.E, ag().v);
        v = load6(qd, 0, col);
      } else {
        gam = mk(0, 0, 0);
        v = szero();
      }
    } else {
      const BodyImage& bi = M.body[i];
      const int p = M.parent[i];
      if (p < 0) v = szero();
      else if (fl & kLgLoad) v = S.get6(OS() + 12 * P.oslot[p]);
      float sn, cs;
      joint_sincos(col.in(q, iq_of<T>(i)) + bi.th0, &sn, &cs);
      S[CS() + i] = cs;
      S[SN() + i] = sn;
      if (VEL) {
        with_dh(bi.dh, [&](auto dh) { v = mot_in(bi, cs, sn, v, dh); });
        v.w.z += col.in(qd, iv_of<T>(i));
      }
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
    SV pA = VEL ? crf(vi, rbi_mul(Ib, vi)) : szero();
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
      a0 = spd6_solve(IA, rhs.root() - pA);
      return;
    }
    const float cs = S[CS() + i], sn = S[SN() + i];
    const SV U = ai_col_z(IA);
    const float dinv = rcp(U.w.z);
    const float ud = (rhs(i) - pA.w.z) * dinv;
    SV Ud = dinv * U;
    Ud.w.z = 1.f;
    S[P0() + 6 * i] = Ud.w.x;
    S[P0() + 6 * i + 1] = Ud.w.y;
    S[P0() + 6 * i + 2] = Ud.v.x;
    S[P0() + 6 * i + 3] = Ud.v.y;
    S[P0() + 6 * i + 4] = Ud.v.z;
    S[P0() + 6 * i + 5] = ud;
    Ia = IA;
    ai_rank1_sub_d_z(Ia, Ud, U);
    pa = axpy(ud, U, pA);
    if (VEL) pa = ai_mul_z_add(pa, Ia, ez_velprod(vi, col.in(qd, iv_of<T>(i))));
    with_dh(bi.dh, [&](auto dh) {
      ai_out_z(bi, cs, sn, Ia, dh);
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
      out.root(a0 - SV{mk(0, 0, 0), gam});
    } else {
      const BodyImage& bi = M.body[i];
      const int p = M.parent[i];
      if (p < 0) a = ag();
      else if (fl & kLgLoad) a = S.get6(OS() + 12 * P.oslot[p] + 6);
      const float cs = S[CS() + i], sn = S[SN() + i];
      const SV cb = VEL ? ez_velprod(S.get6(V0() + 6 * i), col.in(qd, iv_of<T>(i))) : szero();
      with_dh(bi.dh, [&](auto dh) { a = mot_in(bi, cs, sn, a, dh) + cb; });
      const int f = P0() + 6 * i;
      const float x = S[f + 5] - (fmaf(S[f], a.w.x, fmaf(S[f + 1], a.w.y, a.w.z)) +
                                  fmaf(S[f + 2], a.v.x, fmaf(S[f + 3], a.v.y, S[f + 4] * a.v.z)));
      a.w.z += x;
      out(i, x);
    }
    if (fl & kLgStoreOut) S.put6(OS() + 12 * P.oslot[i] + 6, a);
  }
};

// A per-dof vector in the scratch (the ABA adjoint's w), optionally copied
// to a global array too.
template <class T>
struct LgVec {
  LgScratch S;
  int f0;
  FD float operator()(int i) const { return S[f0 + iv_of<T>(i)]; }
  FD SV root() const { return S.get6(f0); }
};
template <class T, class C>
struct OutToLgVec {
  LgScratch S;
  int f0;
  float* also;  // global copy or nullptr
  C col;
  FD void operator()(int i, float x) const {
    S[f0 + iv_of<T>(i)] = x;
    if (also) col.out(also, iv_of<T>(i), x);
  }
  FD void root(const SV& x) const {
    S.put6(f0, x);
    if (also) store6(also, 0, col, x);
  }
};

// The RNEA adjoint (reverse mode of Eq. 1) for one lane: the forward state
// and the seed's propagation outward (each body's v, a and Fb kept in the
// scratch), then the adjoint sweep inward. gb(i) / gb.root() seed it, sink
// takes (qbar, qdbar, qddbar) per body. The arithmetic is rnea_vjp_seg's.
template <bool FREE, class C, class Seed, class Sink>
struct RneaVjpLg {
  using T = SegTopo<32, FREE>;
  const ModelImage<32>& M;
  const LanePlan& P;
  LgScratch S;
  C col;
  int lane;
  bool valid;
  const float *q, *qd, *qdd;
  Seed gb;
  Sink sink;
  SV v, a, Fb;      // outward carry
  SV Fc, abc, vbc;  // inward carry (contributions to the parent, in its frame)
  V3 gam;
  FD int CS() const { return 0; }
  FD int SN() const { return M.nb; }
  FD int V0() const { return 2 * M.nb; }
  FD int A0() const { return 8 * M.nb; }
  FD int B0() const { return 14 * M.nb; }
  FD int OS() const { return 20 * M.nb; }
  FD int IS() const { return 20 * M.nb + 18 * P.n_oslot; }

  FD void out_step(int t) {
    const int i = P.body[t][lane];
    if (!valid || i < 0) return;
    const int fl = P.flag[t][lane];
    const SV ag = gravity_acc(M.g);
    if (FREE && i == 0) {
      const RootPose RP = root_pose(M, q, col);
      gam = rotT(RP.E, ag.v);
      v = load6(qd, 0, col);
      a = SV{mk(0, 0, 0), gam} + load6(qdd, 0, col);
      Fb = gb.root();
    } else {
      const BodyImage& bi = M.body[i];
      const int p = M.parent[i];
      if (p < 0) {
        v = szero();
        a = ag;
        Fb = szero();
      } else if (fl & kLgLoad) {
        const int f = OS() + 18 * P.oslot[p];
        v = S.get6(f);
        a = S.get6(f + 6);
        Fb = S.get6(f + 12);
      }
      float sn, cs;
      joint_sincos(col.in(q, iq_of<T>(i)) + bi.th0, &sn, &cs);
      S[CS() + i] = cs;
      S[SN() + i] = sn;
      const float qdi = col.in(qd, iv_of<T>(i));
      with_dh(bi.dh, [&](auto dh) {
        v = mot_in(bi, cs, sn, v, dh);
        a = mot_in(bi, cs, sn, a, dh);
        Fb = mot_in(bi, cs, sn, Fb, dh);
      });
      v.w.z += qdi;
      a.w.z += col.in(qdd, iv_of<T>(i));
      a = a + ez_velprod(v, qdi);
      Fb.w.z += gb(i);
    }
    S.put6(V0() + 6 * i, v);
    S.put6(A0() + 6 * i, a);
    S.put6(B0() + 6 * i, Fb);
    if (fl & kLgStoreOut) {
      const int f = OS() + 18 * P.oslot[i];
      S.put6(f, v);
      S.put6(f + 6, a);
      S.put6(f + 12, Fb);
    }
  }
  FD void in_step(int t) {
    const int i = P.body[t][lane];
    if (!valid || i < 0) return;
    const int fl = P.flag[t][lane];
    SV Fs = szero(), abs_ = szero(), vbs = szero();  // children's contributions, this body's frame
    if (fl & kLgCarry) {
      Fs = Fc;
      abs_ = abc;
      vbs = vbc;
    }
    for (int r = 0; r < P.rc_count[i]; ++r) {
      const int f = IS() + 18 * P.islot[P.rc_list[P.rc_first[i] + r]];
      Fs = Fs + S.get6(f);
      abs_ = abs_ + S.get6(f + 6);
      vbs = vbs + S.get6(f + 12);
    }
    const BodyImage& bi = M.body[i];
    const RBI I = rbi_of(bi);
    const SV vi = S.get6(V0() + 6 * i), ai = S.get6(A0() + 6 * i), Fbi = S.get6(B0() + 6 * i);
    if (FREE && i == 0) {
      const SV ab = rbi_mul_add(abs_, I, Fbi);
      const SV vb = rbi_mul_sub(crf_sub(vbs, Fbi, rbi_mul(I, vi)), I, crm(vi, Fbi));
      sink.root(cross(ab.v, gam), vb, ab);
      return;
    }
    const float cs = S[CS() + i], sn = S[SN() + i];
    const float qdi = col.in(qd, iv_of<T>(i));
    SV xa = ai - ez_velprod(vi, qdi);
    xa.w.z -= col.in(qdd, iv_of<T>(i));
    const SV Iv = rbi_mul(I, vi);
    const SV F = crf_add(rbi_mul_add(Fs, I, ai), vi, Iv);
    const SV ab = rbi_mul_add(abs_, I, Fbi);
    const SV vb = rbi_mul_sub(crf_sub(vbs, Fbi, Iv), I, crm(vi, Fbi)) + qdi * ez_crf(ab);
    const SV ef = ez_crf(F), ea = ez_crm(xa), ev = ez_crm(vi);
    const float q1 = fmaf(Fbi.w.x, ef.w.x, fmaf(Fbi.w.y, ef.w.y, fmaf(Fbi.v.x, ef.v.x, Fbi.v.y * ef.v.y)));
    const float q2 = fmaf(ab.w.x, ea.w.x, fmaf(ab.w.y, ea.w.y, fmaf(ab.v.x, ea.v.x, ab.v.y * ea.v.y)));
    const float q3 = fmaf(vb.w.x, ev.w.x, fmaf(vb.w.y, ev.w.y, fmaf(vb.v.x, ev.v.x, vb.v.y * ev.v.y)));
    const float qdb =
        fmaf(-ab.w.x, ev.w.x, fmaf(-ab.w.y, ev.w.y, fmaf(-ab.v.x, ev.v.x, fmaf(-ab.v.y, ev.v.y, vb.w.z))));
    sink(i, q1 - q2 - q3, qdb, ab.w.z);
    with_dh(bi.dh, [&](auto dh) {
      Fc = frc_out(bi, cs, sn, F, dh);
      abc = frc_out(bi, cs, sn, ab, dh);
      vbc = frc_out(bi, cs, sn, vb, dh);
    });
    if (fl & kLgStoreIn) {
      const int f = IS() + 18 * P.islot[i];
      S.put6(f, Fc);
      S.put6(f + 6, abc);
      S.put6(f + 12, vbc);
    }
  }
};

// CRBA + L^T D L (Algorithm 2's M and its factor) for one lane: joint
// cos/sin outward, then inward the composite inertia (M) and the articulated
// inertia at rest (the factor) of every subtree; each body emits its rows by
// the ancestor walk of crba_seg (structural zeros written separately).
template <bool FREE, class C>
struct CrbaLg {
  using T = SegTopo<32, FREE>;
  const ModelImage<32>& M;
  const LanePlan& P;
  LgScratch S;
  C col;
  int lane;
  bool valid;
  const float* q;
  float *Mout, *LD;
  RBI Cc;  // carried contributions to the parent, in its frame
  AI Ia;
  FD int CS() const { return 0; }
  FD int SN() const { return M.nb; }
  FD int IS() const { return 2 * M.nb; }
  struct SinCos {
    LgScratch S;
    int cs, sn;
    FD float cos(int j) const { return S[cs + j]; }
    FD float sin(int j) const { return S[sn + j]; }
  };

  FD void sincos_step(int t) {
    const int i = P.body[t][lane];
    if (!valid || i < 0 || (FREE && i == 0)) return;
    float sn, cs;
    joint_sincos(col.in(q, iq_of<T>(i)) + M.body[i].th0, &sn, &cs);
    S[CS() + i] = cs;
    S[SN() + i] = sn;
  }
  FD void in_step(int t) {
    const int i = P.body[t][lane];
    if (!valid || i < 0) return;
    const int fl = P.flag[t][lane];
    const BodyImage& b = M.body[i];
    RBI Ci = rbi_of(b);
    AI IAi = ai_of(Ci);
    if (fl & kLgCarry) {
      Ci = rbi_add(Ci, Cc);
      ai_add(IAi, Ia);
    }
    for (int r = 0; r < P.rc_count[i]; ++r) {
      const int f = IS() + 31 * P.islot[P.rc_list[P.rc_first[i] + r]];
      Ci = rbi_add(Ci, RBI{S[f], mk(S[f + 1], S[f + 2], S[f + 3]), S[f + 4], S[f + 5], S[f + 6], S[f + 7],
                           S[f + 8], S[f + 9]});
      S.add_ai(f + 10, IAi);
    }
    const int nv = FREE ? M.nb + 5 : M.nb;
    auto putM = [&](int r, int c, float x) {  // r >= c
      col.out(Mout, r * nv + c, x);
      if (r != c) col.out(Mout, c * nv + r, x);
    };
    auto putL = [&](int r, int c, float x) { col.out(LD, MSink::tri(r, c), x); };
    if (FREE && i == 0) {
      if (Mout) crba_root_block(Ci, putM);
      if (LD) crba_root_factor(IAi, putL);
      return;
    }
    const int di = iv_of<T>(i);
    const SV FM{mk(Ci.xz, Ci.yz, Ci.zz), mk(-Ci.h.y, Ci.h.x, 0.f)};  // I^c_i e_z
    if (Mout) col.out(Mout, di * nv + di, FM.w.z);
    const SV U = ai_col_z(IAi);
    const float dinv = rcp(U.w.z);
    if (LD) putL(di, di, U.w.z);
    crba_emit_row<T, ModelImage<32>, C, false, 3>(M, i, FM, dinv * U, Mout, LD, SinCos{S, CS(), SN()}, col);
    ai_rank1_sub_z(IAi, U, dinv);
    const float cs = S[CS() + i], sn = S[SN() + i];
    with_dh(b.dh, [&](auto dh) {
      Cc = rbi_out(b, cs, sn, Ci, dh);
      ai_out_z(b, cs, sn, IAi, dh);
    });
    Ia = IAi;
    if (fl & kLgStoreIn) {
      const int f = IS() + 31 * P.islot[i];
      S[f] = Cc.m;
      S[f + 1] = Cc.h.x;
      S[f + 2] = Cc.h.y;
      S[f + 3] = Cc.h.z;
      S[f + 4] = Cc.xx;
      S[f + 5] = Cc.yy;
      S[f + 6] = Cc.zz;
      S[f + 7] = Cc.xy;
      S[f + 8] = Cc.xz;
      S[f + 9] = Cc.yz;
      S.put_ai(f + 10, Ia);
    }
  }
};
FD int lg_crba_floats(int nb, int ni) { return 2 * nb + 31 * ni; }

// FK and frame Jacobians for one lane: world rotations and origins outward
// (each body's pose written, its world axis and origin kept in the scratch),
// then each lane builds the Jacobians of the frames lane, lane + 4, ...:
// column j of frame k is [z_j; z_j x (p_k - p_j)] for every ancestor j (the
// structural zeros are left to the caller's fill, as for fk_seg).
template <bool FREE, class C>
struct FkLg {
  using T = SegTopo<32, FREE>;
  const ModelImage<32>& M;
  const LanePlan& P;
  LgScratch S;
  C col;
  int lane;
  bool valid;
  const float* q;
  float* pose;
  const Frames& fr;
  float* J;
  float R[9];  // carried: world rotation and origin of the previous body
  V3 p;
  FD int Z0() const { return 0; }
  FD int PO() const { return 3 * M.nb; }
  FD int R0() const { return 6 * M.nb; }
  FD int OS() const { return 6 * M.nb + 9; }

  FD void pose_out(int i) const {
    const BodyImage& b = M.body[i];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int cc = 0; cc < 3; ++cc)
        col.out(pose, 12 * i + 3 * r + cc,
                fmaf(R[3 * r], b.Q[3 * cc], fmaf(R[3 * r + 1], b.Q[3 * cc + 1], R[3 * r + 2] * b.Q[3 * cc + 2])));
    col.out(pose, 12 * i + 9, p.x);
    col.out(pose, 12 * i + 10, p.y);
    col.out(pose, 12 * i + 11, p.z);
  }
  FD void out_step(int t) {
    const int i = P.body[t][lane];
    if (!valid || i < 0) return;
    const int fl = P.flag[t][lane];
    if (FREE && i == 0) {
      const RootPose RP = root_pose(M, q, col);
#pragma unroll
      for (int u = 0; u < 9; ++u) S[R0() + u] = R[u] = RP.E[u];
      p = RP.r;
    } else {
      const BodyImage& b = M.body[i];
      const int par = M.parent[i];
      if (par < 0) {
#pragma unroll
        for (int u = 0; u < 9; ++u) R[u] = (u % 4 == 0) ? 1.f : 0.f;
        p = mk(0, 0, 0);
      } else if (fl & kLgLoad) {
        const int f = OS() + 12 * P.oslot[par];
#pragma unroll
        for (int u = 0; u < 9; ++u) R[u] = S[f + u];
        p = mk(S[f + 9], S[f + 10], S[f + 11]);
      }
      float sn, cs;
      joint_sincos(col.in(q, iq_of<T>(i)) + b.th0, &sn, &cs);
      float A[9];
      with_dh(b.dh, [&](auto dh) { mat_mul_b(R, b, A, dh); });
      p = p + rot(R, mk(b.p[0], b.p[1], b.p[2]));
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        R[3 * r] = fmaf(cs, A[3 * r], sn * A[3 * r + 1]);
        R[3 * r + 1] = fmaf(-sn, A[3 * r], cs * A[3 * r + 1]);
        R[3 * r + 2] = A[3 * r + 2];
      }
    }
    S[Z0() + 3 * i] = R[2];
    S[Z0() + 3 * i + 1] = R[5];
    S[Z0() + 3 * i + 2] = R[8];
    S[PO() + 3 * i] = p.x;
    S[PO() + 3 * i + 1] = p.y;
    S[PO() + 3 * i + 2] = p.z;
    if (pose) pose_out(i);
    if (fl & kLgStoreOut) {
      const int f = OS() + 12 * P.oslot[i];
#pragma unroll
      for (int u = 0; u < 9; ++u) S[f + u] = R[u];
      S[f + 9] = p.x;
      S[f + 10] = p.y;
      S[f + 11] = p.z;
    }
  }
  FD void jacobians() const {
    if (!valid || !J) return;
    const int nv = FREE ? M.nb + 5 : M.nb;
    auto pos = [&](int j) { return mk(S[PO() + 3 * j], S[PO() + 3 * j + 1], S[PO() + 3 * j + 2]); };
    auto jcol = [&](int base, int cj, V3 z, V3 lin) {
      col.out(J, base + 0 * nv + cj, z.x);
      col.out(J, base + 1 * nv + cj, z.y);
      col.out(J, base + 2 * nv + cj, z.z);
      col.out(J, base + 3 * nv + cj, lin.x);
      col.out(J, base + 4 * nv + cj, lin.y);
      col.out(J, base + 5 * nv + cj, lin.z);
    };
    for (int f = lane; f < fr.n; f += kLgLanes) {
      const int kf = fr.body[f];
      uint64_t rest = M.anc[kf];
      const int base = f * 6 * nv;
      const V3 pk = pos(kf);
      if (FREE) {  // the root is an ancestor of every body
        const V3 d = pk - pos(0);
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          const V3 zr = mk(S[R0() + m], S[R0() + 3 + m], S[R0() + 6 + m]);
          jcol(base, m, zr, cross(zr, d));
          jcol(base, 3 + m, mk(0, 0, 0), zr);
        }
        rest &= ~1ull;
      }
      for (; rest; rest &= rest - 1) {
        const int j = low_bit(rest);
        const V3 zj = mk(S[Z0() + 3 * j], S[Z0() + 3 * j + 1], S[Z0() + 3 * j + 2]);
        jcol(base, iv_of<T>(j), zj, cross(zj, pk - pos(j)));
      }
    }
  }
};
FD int lg_fk_floats(int nb, int no) { return 6 * nb + 9 + 12 * no; }

// Scratch floats of the adjoint sweep and of the ABA adjoint (its solve's
// sweep, w, then the adjoint sweep over a second region).
FD int lg_vjp_floats(int nb, int no, int ni) { return 20 * nb + 18 * no + 18 * ni; }
FD int lg_aba_vjp_floats(int nb, int nv, int no, int ni) {
  return lg_aba_floats(nb, no, ni) + nv + lg_vjp_floats(nb, no, ni);
}

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

// Copies rows [0, rows) of this block's kLgInst instances of a global SoA
// array into shared memory as [row][kLgInst] (consecutive threads read
// consecutive instances: coalesced), zeros past the batch's end; returns the
// next free float of the staging area.
__device__ __forceinline__ float* lg_stage_rows(const float* __restrict__ src, int rows, int64_t ld, int64_t B,
                                                float* dst) {
  const int64_t b0 = int64_t(blockIdx.x) * kLgInst;
  for (int k = threadIdx.x; k < rows * kLgInst; k += kLgBlock) {
    const int r = k / kLgInst, j = k % kLgInst;
    dst[k] = b0 + j < B ? __ldg(src + r * ld + b0 + j) : 0.f;
  }
  return dst + rows * kLgInst;
}

// Staged inputs first (fixed per kernel: `nin` arrays with their row counts),
// then the per-instance scratch.
#define FRAX_LG_PROLOGUE(NIN_FLOATS)                                                          \
  extern __shared__ __align__(16) char smem[];                                                \
  lg_stage(Mg, Pg, smem);                                                                     \
  const ModelImage<32>& M = *reinterpret_cast<const ModelImage<32>*>(smem);                   \
  const LanePlan& P = *reinterpret_cast<const LanePlan*>(smem + kLgImgBytes);                 \
  const int lane = threadIdx.x % kLgLanes, inst = threadIdx.x / kLgLanes;                     \
  const int64_t b = int64_t(blockIdx.x) * kLgInst + inst;                                     \
  const bool valid = b < B;                                                                   \
  const LgCol col{ld, valid ? b : 0, inst};                                                   \
  float* const stage = reinterpret_cast<float*>(smem + kLgImgBytes + kLgPlanBytes);           \
  const LgScratch S{stage + (NIN_FLOATS) * kLgInst + inst, kLgInst};

template <bool FREE>
__global__ void __launch_bounds__(kLgBlock) k_rnea_lg(const __grid_constant__ ModelImage<32> Mg,
                                                      const __grid_constant__ LanePlan Pg, int64_t B, int64_t ld,
                                                      const float* __restrict__ q, const float* __restrict__ qd,
                                                      const float* __restrict__ qdd, float* __restrict__ tau) {
  FRAX_LG_PROLOGUE(M.nq + 2 * M.nv);
  float* sq = stage;
  float* sqd = lg_stage_rows(q, M.nq, ld, B, sq);
  float* sqdd = lg_stage_rows(qd, M.nv, ld, B, sqd);
  if (qdd) lg_stage_rows(qdd, M.nv, ld, B, sqdd);
  __syncthreads();
  RneaLg<FREE, LgCol> L{M, P, S, col, lane, valid, sq, sqd, qdd ? sqdd : nullptr, tau};
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
  FRAX_LG_PROLOGUE(M.nq + 2 * M.nv);
  using T = SegTopo<32, FREE>;
  float* sq = stage;
  float* sqd = lg_stage_rows(q, M.nq, ld, B, sq);
  float* stau = lg_stage_rows(qd, M.nv, ld, B, sqd);
  lg_stage_rows(tau, M.nv, ld, B, stau);
  __syncthreads();
  AbaLg<FREE, true, LgCol, RhsFromGlobal<T, LgCol>, OutToGlobal<T, LgCol>> L{
      M, P, S, col, lane, valid, sq, sqd, RhsFromGlobal<T, LgCol>{stau, col}, OutToGlobal<T, LgCol>{qdd, col}};
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

template <bool FREE>
__global__ void __launch_bounds__(kLgBlock) k_rnea_vjp_lg(const __grid_constant__ ModelImage<32> Mg,
                                                          const __grid_constant__ LanePlan Pg, int64_t B, int64_t ld,
                                                          const float* __restrict__ q, const float* __restrict__ qd,
                                                          const float* __restrict__ qdd, const float* __restrict__ gbar,
                                                          float* qbar, float* qdbar, float* qddbar) {
  FRAX_LG_PROLOGUE(M.nq + 3 * M.nv);
  using T = SegTopo<32, FREE>;
  float* sq = stage;
  float* sqd = lg_stage_rows(q, M.nq, ld, B, sq);
  float* sqdd = lg_stage_rows(qd, M.nv, ld, B, sqd);
  float* sg = lg_stage_rows(qdd, M.nv, ld, B, sqdd);
  lg_stage_rows(gbar, M.nv, ld, B, sg);
  __syncthreads();
  RneaVjpLg<FREE, LgCol, RhsFromGlobal<T, LgCol>, VjpToGlobal<T, LgCol>> L{
      M, P, S, col, lane, valid, sq, sqd, sqdd, RhsFromGlobal<T, LgCol>{sg, col},
      vjp_sink<T>(M, sq, qbar, qdbar, qddbar, 1.f, col)};
  for (int t = 0; t < P.T; ++t) {
    L.out_step(t);
    __syncwarp();
  }
  for (int t = P.T - 1; t >= 0; --t) {
    L.in_step(t);
    __syncwarp();
  }
}

// The ABA adjoint at qdd = ABA(q, qd, tau): w = M^-1 gbar by the
// zero-velocity sweeps (into taubar when asked), then the RNEA adjoint
// seeded with w, negated.
template <bool FREE>
__global__ void __launch_bounds__(kLgBlock) k_aba_vjp_lg(const __grid_constant__ ModelImage<32> Mg,
                                                         const __grid_constant__ LanePlan Pg, int64_t B, int64_t ld,
                                                         const float* __restrict__ q, const float* __restrict__ qd,
                                                         const float* __restrict__ qdd, const float* __restrict__ gbar,
                                                         float* qbar, float* qdbar, float* taubar) {
  FRAX_LG_PROLOGUE(M.nq + 3 * M.nv);
  using T = SegTopo<32, FREE>;
  float* sq = stage;
  float* sqd = lg_stage_rows(q, M.nq, ld, B, sq);
  float* sqdd = lg_stage_rows(qd, M.nv, ld, B, sqd);
  float* sg = lg_stage_rows(qdd, M.nv, ld, B, sqdd);
  lg_stage_rows(gbar, M.nv, ld, B, sg);
  __syncthreads();
  const int W0 = lg_aba_floats(M.nb, P.n_oslot, P.n_islot);
  const LgScratch S2{&S[W0 + M.nv], kLgInst};
  {
    AbaLg<FREE, false, LgCol, RhsFromGlobal<T, LgCol>, OutToLgVec<T, LgCol>> L{
        M, P, S, col, lane, valid, sq, sqd, RhsFromGlobal<T, LgCol>{sg, col},
        OutToLgVec<T, LgCol>{S, W0, taubar, col}};
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
  RneaVjpLg<FREE, LgCol, LgVec<T>, VjpToGlobal<T, LgCol>> L{
      M, P, S2, col, lane, valid, sq, sqd, sqdd, LgVec<T>{S, W0}, vjp_sink<T>(M, sq, qbar, qdbar, nullptr, -1.f, col)};
  for (int t = 0; t < P.T; ++t) {
    L.out_step(t);
    __syncwarp();
  }
  for (int t = P.T - 1; t >= 0; --t) {
    L.in_step(t);
    __syncwarp();
  }
}
// CRBA + L^T D L; each lane writes its share of the structural zeros (rows
// lane, lane + 4, ... of the list Z).
template <bool FREE>
__global__ void __launch_bounds__(kLgBlock) k_crba_lg(const __grid_constant__ ModelImage<32> Mg,
                                                      const __grid_constant__ LanePlan Pg,
                                                      const __grid_constant__ ZeroRows Z, int64_t B, int64_t ld,
                                                      const float* __restrict__ q, float* Mout, float* LD) {
  FRAX_LG_PROLOGUE(M.nq);
  float* sq = stage;
  lg_stage_rows(q, M.nq, ld, B, sq);
  __syncthreads();
  CrbaLg<FREE, LgCol> L{M, P, S, col, lane, valid, sq, Mout, LD};
  for (int t = 0; t < P.T; ++t) {
    L.sincos_step(t);
    __syncwarp();
  }
  for (int t = P.T - 1; t >= 0; --t) {
    L.in_step(t);
    __syncwarp();
  }
  if (valid) {
    for (int r = lane; r < Z.n0; r += kLgLanes) col.out(Mout, Z.row[r], 0.f);
    for (int r = Z.n0 + lane; r < Z.n; r += kLgLanes) col.out(LD, Z.row[r], 0.f);
  }
}
// FK (every body's pose) and, when J is given, the frames' Jacobians.
template <bool FREE>
__global__ void __launch_bounds__(kLgBlock) k_fk_lg(const __grid_constant__ ModelImage<32> Mg,
                                                    const __grid_constant__ LanePlan Pg, int64_t B, int64_t ld,
                                                    const float* __restrict__ q, float* pose,
                                                    const __grid_constant__ Frames fr, float* J) {
  FRAX_LG_PROLOGUE(M.nq);
  float* sq = stage;
  lg_stage_rows(q, M.nq, ld, B, sq);
  __syncthreads();
  FkLg<FREE, LgCol> L{M, P, S, col, lane, valid, sq, pose, fr, J};
  for (int t = 0; t < P.T; ++t) {
    L.out_step(t);
    __syncwarp();
  }
  L.jacobians();
}
#undef FRAX_LG_PROLOGUE
#endif

}  // namespace frax
