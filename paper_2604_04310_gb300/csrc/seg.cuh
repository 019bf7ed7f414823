// Segment-unrolled tree algorithms, one thread per instance.
//
// A tree is cut into segments (model_image.h): runs of single-child bodies,
// at most kMaxSeg long. A segment's sweep is unrolled like the chain kernel,
// so its per-body state sits in registers (slot k = k-th body of the
// segment); only what crosses segment boundaries lives in small per-thread
// arrays indexed by body: the velocity/acceleration/pose of bodies that have
// child segments, the force or inertia that child segments hand back, and
// the sweep state of segments whose inward sweep has to wait for their
// children. Segments are visited depth-first (M.act), so that waiting state
// is bounded by the depth of the segment tree, and outward-only passes run
// over the segments in topological order.
#pragma once
#include "dyn.cuh"

namespace frax {

template <int NBM, bool FREE>
struct SegTopo {
  static constexpr int NBMAX = NBM;
  static constexpr int NVMAX = NBM + (FREE ? 5 : 0);
  static constexpr bool kFree = FREE;
  static constexpr bool kStatic = false;
  static constexpr bool kSeg = true;
  template <class Img>
  FD static int nb(const Img& M) { return M.nb; }
  template <class Img>
  FD static int parent(const Img& M, int i) { return M.parent[i]; }
  template <class Img>
  FD static int dparent(const Img& M, int k) { return M.dparent[k]; }
};

// v x (e_z qd): the velocity-product acceleration of a revolute joint
FD SV ez_velprod(const SV& v, float qd) { return qd * SV{mk(v.w.y, -v.w.x, 0.f), mk(v.v.y, -v.v.x, 0.f)}; }

// ====================================================================== RNEA
// With EXT, the spatial force fext (body coordinates) is added to the net
// force of body ext_body, so tau gains J_ext^T fext.
// With EXTW, fw holds every body's external spatial force in root-frame
// Pluecker coordinates ([moment about the root origin; force], 6 rows per
// body, Algorithm 1's ^0F_ext,i): the outward sweep also carries each body's
// world rotation R and origin p, and subtracts the force in body coordinates,
// [R^T (n - p x f); R^T f], from the body's net force, so tau loses
// sum_i J_i^T F_ext,i in the same sweep.
template <class T, class Img, class C, bool EXT = false, bool EXTW = false>
FD void rnea_seg(const Img& M, const float* __restrict__ q, const float* __restrict__ qd,
                 const float* __restrict__ qdd, float* __restrict__ tau, const C& col, int ext_body = -1,
                 SV fext = SV{}, const float* __restrict__ fw = nullptr) {
  constexpr int NB = T::NBMAX;
  SV bv[NB], ba[NB], Fa[NB], sf[NB];
  float sc[NB], ss[NB];
  float bR[EXTW ? NB : 1][9];  // world rotation and origin of bodies with child segments
  V3 bp[EXTW ? NB : 1];
  const SV ag = gravity_acc(M.g);
  // body-frame form of an external force given in root-frame coordinates
  auto ext_in = [&](const float* R, V3 o, int i) {
    const SV F = load6(fw, 6 * i, col);
    return SV{rotT(R, F.w - cross(o, F.v)), rotT(R, F.v)};
  };
#pragma unroll 1
  for (int t = 0; t < M.n_act; ++t) {
    const int act = M.act[t];
    const int s = act & 63, kind = act >> 6;
    const int st = M.seg_start[s], len = M.seg_len[s];
    if (T::kFree && s == 0) {  // the free-flyer root is a one-body segment
      if (kind != kActClose) {
        const RootPose P = root_pose(M, q, col);
        const SV v0 = load6(qd, 0, col);
        SV a0 = SV{mk(0, 0, 0), rotT(P.E, ag.v)};
        if (qdd) a0 = a0 + load6(qdd, 0, col);
        const RBI I = rbi_of(M.body[0]);
        SV f0 = crf_add(rbi_mul(I, a0), v0, rbi_mul(I, v0));
        if constexpr (EXT) {
          if (ext_body == 0) f0 = f0 + fext;
        }
        if constexpr (EXTW) {
          f0 = f0 - ext_in(P.E, P.r, 0);
          if (kind == kActOpen) {
#pragma unroll
            for (int u = 0; u < 9; ++u) bR[0][u] = P.E[u];
            bp[0] = P.r;
          }
        }
        if (kind == kActLeaf) {
          store6(tau, 0, col, f0);
        } else {
          bv[0] = v0;
          ba[0] = a0;
          sf[0] = f0;
          Fa[0] = szero();
        }
      } else {
        store6(tau, 0, col, sf[0] + Fa[0]);
      }
      continue;
    }
    SV f[kMaxSeg];
    float cc[kMaxSeg], sn[kMaxSeg];
    if (kind != kActClose) {
      const int p = M.seg_parent[s];
      SV v = p < 0 ? szero() : bv[p];
      SV a = p < 0 ? ag : ba[p];
      float R[EXTW ? 9 : 1];
      V3 o = mk(0, 0, 0);
      if constexpr (EXTW) {
#pragma unroll
        for (int u = 0; u < 9; ++u) R[u] = p < 0 ? ((u % 4 == 0) ? 1.f : 0.f) : bR[p][u];
        if (p >= 0) o = bp[p];
      }
#pragma unroll
      for (int k = 0; k < kMaxSeg; ++k) {
        if (k < len) {
          const int i = M.order[st + k];
          const BodyImage& b = M.body[i];
          joint_sincos(col.in(q, iq_of<T>(i)) + M.body[i].th0, &sn[k], &cc[k]);
          const float qdi = col.in(qd, iv_of<T>(i));
          const float qddi = qdd ? col.in(qdd, iv_of<T>(i)) : 0.f;
          v = mot_in(b, cc[k], sn[k], v, k > 0);
          v.w.z += qdi;
          a = mot_in(b, cc[k], sn[k], a, k > 0);
          a.w.z += qddi;
          a = a + ez_velprod(v, qdi);
          const RBI I = rbi_of(b);
          f[k] = crf_add(rbi_mul(I, a), v, rbi_mul(I, v));
          if constexpr (EXT) {
            if (i == ext_body) f[k] = f[k] + fext;
          }
          if constexpr (EXTW) {  // world pose: R <- R R_b Rot_z(q), o <- o + R p_b
            float A[9];
            mat_mul_b(R, b, A, k > 0);
            o = o + rot(R, mk(b.p[0], b.p[1], b.p[2]));
#pragma unroll
            for (int r = 0; r < 3; ++r) {
              R[3 * r] = fmaf(cc[k], A[3 * r], sn[k] * A[3 * r + 1]);
              R[3 * r + 1] = fmaf(-sn[k], A[3 * r], cc[k] * A[3 * r + 1]);
              R[3 * r + 2] = A[3 * r + 2];
            }
            f[k] = f[k] - ext_in(R, o, i);
          }
        }
      }
      if (kind == kActOpen) {
        const int last = M.order[st + len - 1];
        bv[last] = v;
        ba[last] = a;
        if constexpr (EXTW) {
#pragma unroll
          for (int u = 0; u < 9; ++u) bR[last][u] = R[u];
          bp[last] = o;
        }
        Fa[last] = szero();
#pragma unroll
        for (int k = 0; k < kMaxSeg; ++k)
          if (k < len) {
            const int i = M.order[st + k];
            sf[i] = f[k];
            sc[i] = cc[k];
            ss[i] = sn[k];
          }
        continue;
      }
    } else {
#pragma unroll
      for (int k = 0; k < kMaxSeg; ++k)
        if (k < len) {
          const int i = M.order[st + k];
          f[k] = sf[i];
          cc[k] = sc[i];
          sn[k] = ss[i];
        }
    }
    SV F = kind == kActClose ? Fa[M.order[st + len - 1]] : szero();
#pragma unroll
    for (int k = kMaxSeg - 1; k >= 0; --k) {
      if (k < len) {
        const int i = M.order[st + k];
        F = F + f[k];
        col.out(tau, iv_of<T>(i), F.w.z);
        F = frc_out(M.body[i], cc[k], sn[k], F, k > 0);
      }
    }
    const int p = M.seg_parent[s];
    if (p >= 0) Fa[p] = Fa[p] + F;
  }
}

// ======================================================================= ABA
// Between the inward and the final outward sweep every body needs U / D and
// u / D (U = I^A e_z, D = U_z, u = tau - e_z^T p^A): the outward step is then
// qdd_i = u/D - (U/D)^T a', and (U/D)_z = 1 is not stored, so 6 floats per
// body. The outward sweep recomputes the joint sin/cos and velocities rather
// than storing them.
template <int NB>
struct P3Local {  // all in thread-local memory
  float v[NB * 6];
  FD void put(int i, int f, float x) { v[i * 6 + f] = x; }
  FD float get(int i, int f) const { return v[i * 6 + f]; }
};
// (Holding the first bodies' factors in shared memory instead, with the
// occupancy that leaves, measured 22-36 % slower: the shared memory comes out
// of the L1 that serves the thread-local arrays.)

// With EXTW (and VEL), fw holds every body's external spatial force in
// root-frame Pluecker coordinates (6 rows per body, Algorithm 1's ^0F_ext,i):
// the velocity sweep also carries each body's world rotation and origin, the
// inward sweep steps them back with the velocity and subtracts the body-frame
// force from the body's bias force.
template <class T, class Img, bool VEL, class Rhs, class Out, class C, class P3, bool EXTW = false>
FD void aba_seg_core(const Img& M, const float* __restrict__ q, const float* __restrict__ qd, const Rhs& rhs_at,
                     const Out& out_at, const C& col, P3& P, const float* __restrict__ fw = nullptr) {
  constexpr int NB = T::NBMAX;
  SV bv[NB], bA[NB], pAa[NB];
  AI IAa[NB];
  float bR[EXTW ? NB : 1][9];  // world rotation and origin of segment tips with child segments
  V3 bp[EXTW ? NB : 1];
  auto ext_in = [&](const float* R, V3 o, int i) {
    const SV F = load6(fw, 6 * i, col);
    return SV{rotT(R, F.w - cross(o, F.v)), rotT(R, F.v)};
  };
  const SV ag = VEL ? gravity_acc(M.g) : szero();
  V3 gam = mk(0, 0, 0);  // root: E^T (-g)
  uint64_t opened = 0;  // segments with child segments: their tips' accelerations are kept
  // bodies whose IAa / pAa hold a child segment's contribution: the first
  // contribution is stored, later ones added (no zero fill, no read of zeros)
  uint64_t acc = 0;
#pragma unroll 1
  for (int t = 0; t < M.n_act; ++t) {
    const int act = M.act[t];
    const int s = act & 63, kind = act >> 6;
    const int st = M.seg_start[s], len = M.seg_len[s];
    if (kind == kActOpen) opened |= 1ull << s;
    if (T::kFree && s == 0) {
      const RBI I0 = rbi_of(M.body[0]);
      if (kind != kActClose) {
        const RootPose RP = root_pose(M, q, col);
        gam = rotT(RP.E, ag.v);
        bv[0] = VEL ? load6(qd, 0, col) : szero();
        if constexpr (EXTW) {
#pragma unroll
          for (int u = 0; u < 9; ++u) bR[0][u] = RP.E[u];
          bp[0] = RP.r;
        }
        if (kind == kActOpen) continue;
      }
      AI IA0 = ai_of(I0);
      SV pAc = szero();
      if (acc & 1ull) {
        ai_add(IA0, IAa[0]);
        pAc = pAa[0];
      }
      SV pA0 = VEL ? crf(bv[0], rbi_mul(I0, bv[0])) : szero();
      if constexpr (EXTW) {
        const RootPose RP = root_pose(M, q, col);
        pA0 = pA0 - ext_in(RP.E, RP.r, 0);
      }
      const SV a0 = spd6_solve(IA0, rhs_at.root() - (pA0 + pAc));
      out_at.root(a0 - SV{mk(0, 0, 0), gam});
      bA[0] = a0;
      continue;
    }
    const int last = M.order[st + len - 1];
    SV vtip = szero();
    float Rt[EXTW ? 9 : 1];  // world pose of the body the inward sweep is at
    V3 ot = mk(0, 0, 0);
    if (kind != kActClose) {
      const int p = M.seg_parent[s];
      SV vv = (!VEL || p < 0) ? szero() : bv[p];
      if constexpr (EXTW) {
#pragma unroll
        for (int u = 0; u < 9; ++u) Rt[u] = p < 0 ? ((u % 4 == 0) ? 1.f : 0.f) : bR[p][u];
        if (p >= 0) ot = bp[p];
      }
      if (VEL) {
        seg_outward(len, M.body[M.order[st]].dh, [&](int k, auto dh) {
          const int i = M.order[st + k];
          const BodyImage& b = M.body[i];
          float sn, cs;
          joint_sincos(col.in(q, iq_of<T>(i)) + b.th0, &sn, &cs);
          vv = mot_in(b, cs, sn, vv, dh);
          vv.w.z += col.in(qd, iv_of<T>(i));
          if constexpr (EXTW) {  // R <- R R_b Rot_z(q), o <- o + R p_b
            float A[9];
            mat_mul_b(Rt, b, A, dh);
            ot = ot + rot(Rt, mk(b.p[0], b.p[1], b.p[2]));
#pragma unroll
            for (int r = 0; r < 3; ++r) {
              Rt[3 * r] = fmaf(cs, A[3 * r], sn * A[3 * r + 1]);
              Rt[3 * r + 1] = fmaf(-sn, A[3 * r], cs * A[3 * r + 1]);
              Rt[3 * r + 2] = A[3 * r + 2];
            }
          }
        });
      }
      vtip = vv;
      if (kind == kActOpen) {
        bv[last] = vv;
        if constexpr (EXTW) {
#pragma unroll
          for (int u = 0; u < 9; ++u) bR[last][u] = Rt[u];
          bp[last] = ot;
        }
        continue;
      }
    } else {
      vtip = bv[last];
      if constexpr (EXTW) {
#pragma unroll
        for (int u = 0; u < 9; ++u) Rt[u] = bR[last][u];
        ot = bp[last];
      }
    }
    // inward sweep: articulated inertias and bias forces
    AI Ia;
    SV pa;
    const bool closing = kind == kActClose;
    seg_inward(len, M.body[M.order[st]].dh, [&](int k, auto dh) {
      {
        const int i = M.order[st + k];
        const BodyImage& b = M.body[i];
        const RBI Ib = rbi_of(b);
        const SV vk = vtip;  // velocity of body i, stepped back from the segment's tip
        float sk, ck;
        joint_sincos(col.in(q, iq_of<T>(i)) + b.th0, &sk, &ck);
        AI IA = ai_of(Ib);
        SV pAt = szero();
        SV cb = szero();
        if (VEL) {
          const float qdi = col.in(qd, iv_of<T>(i));
          cb = ez_velprod(vk, qdi);
          pAt = crf(vk, rbi_mul(Ib, vk));
        }
        if constexpr (EXTW) pAt = pAt - ext_in(Rt, ot, i);
        if (k == len - 1) {
          if (closing && ((acc >> last) & 1ull)) {
            ai_add(IA, IAa[last]);
            pAt = pAt + pAa[last];
          }
        } else {
          ai_add(IA, Ia);
          pAt = pAt + pa;
        }
        const SV U = ai_col_z(IA);
        const float dinv = rcp(U.w.z);
        const float ud = (rhs_at(i) - pAt.w.z) * dinv;
        SV Ud = dinv * U;
        Ud.w.z = 1.f;
        P.put(i, 0, Ud.w.x);
        P.put(i, 1, Ud.w.y);
        P.put(i, 2, Ud.v.x);
        P.put(i, 3, Ud.v.y);
        P.put(i, 4, Ud.v.z);
        P.put(i, 5, ud);
        Ia = IA;
        ai_rank1_sub_d_z(Ia, Ud, U);
        pa = axpy(ud, U, pAt);
        if (VEL) pa = ai_mul_z_add(pa, Ia, cb);
        ai_out_z(b, ck, sk, Ia, dh);
        pa = frc_out(b, ck, sk, pa, dh);
        if (VEL && k > 0) {
          SV vp = vk;
          vp.w.z -= col.in(qd, iv_of<T>(i));
          vtip = mot_out(b, ck, sk, vp, dh);
        }
        if constexpr (EXTW) {
          if (k > 0) {  // back to the parent: R <- R Rot_z(q)^T R_b^T, o <- o - R p_b
            float A[9];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
              A[3 * r] = fmaf(ck, Rt[3 * r], -sk * Rt[3 * r + 1]);
              A[3 * r + 1] = fmaf(sk, Rt[3 * r], ck * Rt[3 * r + 1]);
              A[3 * r + 2] = Rt[3 * r + 2];
            }
            mat_mul_bT(A, b, Rt, dh);
            ot = ot - rot(Rt, mk(b.p[0], b.p[1], b.p[2]));
          }
        }
      }
    });
    const int p = M.seg_parent[s];
    if (p >= 0) {
      if ((acc >> p) & 1ull) {
        ai_add(IAa[p], Ia);
        pAa[p] = pAa[p] + pa;
      } else {
        IAa[p] = Ia;
        pAa[p] = pa;
        acc |= 1ull << p;
      }
    }
  }
  // outward sweep: accelerations, segment by segment in the reverse of the
  // order in which the inward sweep finished them (a parent still comes
  // before its children): the factors written last, still in L2, are read
  // first
#pragma unroll 1
  for (int t = M.n_act - 1; t >= 0; --t) {
    const int act = M.act[t];
    const int s = act & 63;
    if ((act >> 6) == kActOpen || (T::kFree && s == 0)) continue;
    const int st = M.seg_start[s], len = M.seg_len[s];
    const int p = M.seg_parent[s];
    SV a = p < 0 ? ag : bA[p];
    SV vv = (!VEL || p < 0) ? szero() : bv[p];
    seg_outward(len, M.body[M.order[st]].dh, [&](int k, auto dh) {
      {
        const int i = M.order[st + k];
        const BodyImage& b = M.body[i];
        float sn, cs;
        joint_sincos(col.in(q, iq_of<T>(i)) + b.th0, &sn, &cs);
        SV cb = szero();
        if (VEL) {
          const float qdi = col.in(qd, iv_of<T>(i));
          vv = mot_in(b, cs, sn, vv, dh);
          vv.w.z += qdi;
          cb = ez_velprod(vv, qdi);
        }
        a = mot_in(b, cs, sn, a, dh) + cb;
        const float x = P.get(i, 5) - (fmaf(P.get(i, 0), a.w.x, fmaf(P.get(i, 1), a.w.y, a.w.z)) +
                                       fmaf(P.get(i, 2), a.v.x, fmaf(P.get(i, 3), a.v.y, P.get(i, 4) * a.v.z)));
        a.w.z += x;
        out_at(i, x);
      }
    });
    if ((opened >> s) & 1ull) bA[M.order[st + len - 1]] = a;
  }
}

template <class T, class Img, class C, class P3>
FD void aba_seg(const Img& M, const float* __restrict__ q, const float* __restrict__ qd,
                const float* __restrict__ tau, float* __restrict__ qdd, const C& col, P3& P) {
  aba_seg_core<T, Img, true>(M, q, qd, RhsFromGlobal<T, C>{tau, col}, OutToGlobal<T, C>{qdd, col}, col, P);
}

// ============================================================= CRBA + LTDL
// M from composite inertias (Algorithm 2's result) and, when asked, the
// factor M = L^T D L of the same tree from articulated-body inertias: with
// dofs eliminated from the leaves up, D_i = S_i^T I^A_i S_i and
// L_ij = S_j^T (^jX_i)^* U_i / D_i for j in Anc(i), U_i = I^A_i S_i, where
// I^A is the articulated inertia of ABA at zero velocity (the Schur
// complement of M's trailing block). A free-flyer root's own 6x6 block is
// the root's articulated inertia, factored densely. No matrix entry is
// updated in place.
// Emits body i's row of M and/or L: S_j^T F at every ancestor dof j (the
// forces carried to the root through the joint transforms) and zeros at the
// dofs of non-ancestors.
// With ZEROS false the structural zeros (non-ancestor pairs) are left to the
// caller (a separate fill of those rows, the same for every instance).
// Joint cos/sin of every body, from per-thread arrays.
struct SinCosArrays {
  const float* c;
  const float* s;
  FD float cos(int j) const { return c[j]; }
  FD float sin(int j) const { return s[j]; }
};

template <class T, class Img, class C, bool ZEROS, int OUT, class SC>
FD void crba_emit_row(const Img& M, int i, SV FM, SV FL, float* __restrict__ Mout,
                                           float* __restrict__ LD, const SC& scs, C col) {
  const int nv = T::kFree ? M.nb + 5 : M.nb;
  const int di = iv_of<T>(i);
  const bool wM = (OUT & 1) && Mout != nullptr, wL = (OUT & 2) && LD != nullptr;
  // this instance's row di of M, column di of M and row di of the factor:
  // entry c of each one multiply and one add away
  float* const rowM = wM ? col.at(Mout, di * nv) : nullptr;
  float* const colM = wM ? col.at(Mout, di) : nullptr;
  float* const rowL = wL ? col.at(LD, MSink::tri(di, 0)) : nullptr;
  auto put = [&](int c, float m, float l) {  // c < di
    if (wM) {
      st_cs(at_row(rowM, c, col.ld), m);
      st_cs(at_row(colM, c * nv, col.ld), m);
    }
    if (wL) st_cs(at_row(rowL, c, col.ld), l);
  };
  int j = i;
  while (true) {
    const int k = M.parent[j];
    if (k < 0) break;
    const BodyImage& b = M.body[j];
    const float cj = scs.cos(j), sj = scs.sin(j);
    with_dh(b.dh, [&](auto dh) {
      if (wM) FM = frc_out(b, cj, sj, FM, dh);
      if (wL) FL = frc_out(b, cj, sj, FL, dh);
    });
    j = k;
    if (T::kFree && j == 0) {
      put(0, FM.w.x, FL.w.x); put(1, FM.w.y, FL.w.y); put(2, FM.w.z, FL.w.z);
      put(3, FM.v.x, FL.v.x); put(4, FM.v.y, FL.v.y); put(5, FM.v.z, FL.v.z);
    } else {
      put(iv_of<T>(j), FM.w.z, FL.w.z);
    }
  }
  if (!ZEROS) return;
  const uint64_t anc = M.anc[i];
  for (int jj = 0; jj < i; ++jj) {
    if ((anc >> jj) & 1ull) continue;
    if (T::kFree && jj == 0) {
      for (int m = 0; m < 6; ++m) put(m, 0.f, 0.f);
    } else {
      put(iv_of<T>(jj), 0.f, 0.f);
    }
  }
}

// A free-flyer root's 6x6 block of M from its composite inertia Cc
// (put(r, c, x) for c <= r).
template <class Put>
FD void crba_root_block(const RBI& Cc, const Put& put) {
  const float blk[6][6] = {{Cc.xx, Cc.xy, Cc.xz, 0.f, -Cc.h.z, Cc.h.y},
                           {Cc.xy, Cc.yy, Cc.yz, Cc.h.z, 0.f, -Cc.h.x},
                           {Cc.xz, Cc.yz, Cc.zz, -Cc.h.y, Cc.h.x, 0.f},
                           {0.f, Cc.h.z, -Cc.h.y, Cc.m, 0.f, 0.f},
                           {-Cc.h.z, 0.f, Cc.h.x, 0.f, Cc.m, 0.f},
                           {Cc.h.y, -Cc.h.x, 0.f, 0.f, 0.f, Cc.m}};
#pragma unroll
  for (int r = 0; r < 6; ++r)
#pragma unroll
    for (int c = 0; c <= r; ++c) put(r, c, blk[r][c]);
}

// Its block of the factor: the dense L^T D L of the root's articulated
// inertia A0, last dof first.
template <class Put>
FD void crba_root_factor(const AI& A0, const Put& put) {
  const float* Af = A0.A;
  const float* Cf = A0.C;
  float H[6][6] = {{Af[0], Af[3], Af[4], A0.B[0], A0.B[1], A0.B[2]},
                   {Af[3], Af[1], Af[5], A0.B[3], A0.B[4], A0.B[5]},
                   {Af[4], Af[5], Af[2], A0.B[6], A0.B[7], A0.B[8]},
                   {A0.B[0], A0.B[3], A0.B[6], Cf[0], Cf[3], Cf[4]},
                   {A0.B[1], A0.B[4], A0.B[7], Cf[3], Cf[1], Cf[5]},
                   {A0.B[2], A0.B[5], A0.B[8], Cf[4], Cf[5], Cf[2]}};
#pragma unroll
  for (int k = 5; k >= 0; --k) {
    const float rk = rcp(H[k][k]);
#pragma unroll
    for (int i = k - 1; i >= 0; --i) {
      const float a = H[k][i] * rk;
#pragma unroll
      for (int j = i; j >= 0; --j) H[i][j] = fmaf(-a, H[k][j], H[i][j]);
      H[k][i] = a;
    }
  }
#pragma unroll
  for (int r = 0; r < 6; ++r)
#pragma unroll
    for (int c = 0; c <= r; ++c) put(r, c, H[r][c]);
}

// OUT selects at compile time what the kernel can produce (1: M, 2: the
// factor, 3: both): a kernel for one of them carries only that sweep's state.
template <class T, class Img, class C, bool ZEROS = true, int OUT = 3>
FD void crba_seg(const Img& M, const float* __restrict__ q, float* __restrict__ Mout, float* __restrict__ LD,
                 const C& col) {
  constexpr int NB = T::NBMAX;
  constexpr bool kM = (OUT & 1) != 0, kL = (OUT & 2) != 0;
  RBI ICa[kM ? NB : 1];
  AI IAa[kL ? NB : 1];
  float sc[NB], ss[NB];
  const int nb = M.nb;
  const int nv = T::kFree ? nb + 5 : nb;
  const bool wantM = kM && Mout != nullptr;
  const bool wantL = kL && LD != nullptr;
  auto putM = [&](int r, int c, float val) {  // r >= c
    col.out(Mout, r * nv + c, val);
    if (r != c) col.out(Mout, c * nv + r, val);
  };
  auto putL = [&](int r, int c, float val) { col.out(LD, MSink::tri(r, c), val); };
  const RBI rzero{0.f, mk(0, 0, 0), 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  AI azero;
#pragma unroll
  for (int k = 0; k < 6; ++k) { azero.A[k] = 0.f; azero.C[k] = 0.f; }
#pragma unroll
  for (int k = 0; k < 9; ++k) azero.B[k] = 0.f;
#pragma unroll 1
  for (int t = 0; t < M.n_act; ++t) {
    const int act = M.act[t];
    const int s = act & 63, kind = act >> 6;
    const int st = M.seg_start[s], len = M.seg_len[s];
    if (T::kFree && s == 0) {
      if (kind != kActClose) {
        if constexpr (kM) ICa[0] = rzero;
        if constexpr (kL) IAa[0] = azero;
      }
      if (kind == kActOpen) continue;
      if constexpr (kM) if (wantM) crba_root_block(rbi_add(rbi_of(M.body[0]), ICa[0]), putM);
      if constexpr (kL) if (wantL) {
        AI A0 = ai_of(rbi_of(M.body[0]));
        ai_add(A0, IAa[0]);
        crba_root_factor(A0, putL);
      }
      continue;
    }
    const int last = M.order[st + len - 1];
    if (kind != kActClose) {
#pragma unroll 1
      for (int k = 0; k < len; ++k) {
        const int i = M.order[st + k];
        joint_sincos(col.in(q, iq_of<T>(i)) + M.body[i].th0, &ss[i], &sc[i]);
      }
      if (kind == kActOpen) {
        if constexpr (kM) ICa[last] = rzero;
        if constexpr (kL) IAa[last] = azero;
        continue;
      }
    }
    RBI Cc = rbi_of(M.body[last]);
    AI IA = ai_of(Cc);
    if (kind == kActClose) {
      if constexpr (kM) Cc = rbi_add(Cc, ICa[last]);
      if constexpr (kL) ai_add(IA, IAa[last]);
    }
#pragma unroll 1
    for (int k = len - 1; k >= 0; --k) {
      {
        const int i = M.order[st + k];
        const int di = iv_of<T>(i);
        const BodyImage& b = M.body[i];
        SV FM = szero();
        if constexpr (kM) {
          FM = SV{mk(Cc.xz, Cc.yz, Cc.zz), mk(-Cc.h.y, Cc.h.x, 0.f)};  // I^c_i e_z
          if (wantM) col.out(Mout, di * nv + di, FM.w.z);
        }
        SV FL = szero();
        AI Ia;
        if constexpr (kL) if (wantL) {
          const SV U = ai_col_z(IA);
          const float dinv = rcp(U.w.z);
          putL(di, di, U.w.z);
          FL = dinv * U;
          Ia = IA;
          ai_rank1_sub_z(Ia, U, dinv);
          ai_out_z(b, sc[i], ss[i], Ia);
        }
        crba_emit_row<T, Img, C, ZEROS, OUT>(M, i, FM, FL, Mout, LD, SinCosArrays{sc, ss}, col);
        const RBI Ip = rbi_of(M.body[M.order[st + (k > 0 ? k - 1 : 0)]]);
        if constexpr (kM) {
          const RBI up = rbi_out(b, sc[i], ss[i], Cc);
          Cc = k > 0 ? rbi_add(Ip, up) : up;
        }
        if constexpr (kL) if (wantL) {
          if (k > 0) {
            IA = ai_of(Ip);
            ai_add(IA, Ia);
          } else {
            IA = Ia;
          }
        }
      }
    }
    const int p = M.seg_parent[s];
    if (p >= 0) {
      if constexpr (kM) ICa[p] = rbi_add(ICa[p], Cc);
      if constexpr (kL) if (wantL) ai_add(IAa[p], IA);
    }
  }
}

// ============================================================ FK + Jacobians
// Poses segment by segment (depth-first), each segment's frames in
// registers; the joint axes and origins of the bodies of open ancestor
// segments are kept per body so a frame's Jacobian is written as soon as its
// segment is done. Column j of frame k: [z_j; z_j x (p_k - p_j)], 0 off Anc(k).
template <class T, class Img, class C, bool ZEROS = true>
FD void fk_seg(const Img& M, const float* __restrict__ q, float* __restrict__ pose, const Frames& fr,
               float* __restrict__ J, const C& col) {
  constexpr int NB = T::NBMAX;
  float bR[NB][9];    // world rotation (internal frame) of bodies with child segments
  V3 bp[NB];
  V3 zs[NB], ps[NB];  // joint axis and origin of every body reached so far
  float R0[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
  V3 p0 = mk(0, 0, 0);
  const int nb = M.nb;
  const int nv = T::kFree ? nb + 5 : nb;
  auto pose_out = [&](int i, const float* R, V3 p) {
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
  };
  auto jcol = [&](int base, int cj, bool on, V3 z, V3 lin) {
    if (!ZEROS && !on) return;  // a structural zero, written by the caller
    col.out(J, base + 0 * nv + cj, on ? z.x : 0.f);
    col.out(J, base + 1 * nv + cj, on ? z.y : 0.f);
    col.out(J, base + 2 * nv + cj, on ? z.z : 0.f);
    col.out(J, base + 3 * nv + cj, on ? lin.x : 0.f);
    col.out(J, base + 4 * nv + cj, on ? lin.y : 0.f);
    col.out(J, base + 5 * nv + cj, on ? lin.z : 0.f);
  };
#pragma unroll 1
  for (int t = 0; t < M.n_act; ++t) {
    const int act = M.act[t];
    const int s = act & 63, kind = act >> 6;
    if (kind == kActClose) continue;
    const int st = M.seg_start[s], len = M.seg_len[s];
    float R[9];
    V3 p;
    if (T::kFree && s == 0) {
      const RootPose P = root_pose(M, q, col);
#pragma unroll
      for (int u = 0; u < 9; ++u) R[u] = R0[u] = P.E[u];
      p = p0 = P.r;
      ps[0] = p;
      if (pose) pose_out(0, R, p);
    } else {
      const int par = M.seg_parent[s];
      if (par >= 0) {
#pragma unroll
        for (int u = 0; u < 9; ++u) R[u] = bR[par][u];
        p = bp[par];
      } else {
#pragma unroll
        for (int u = 0; u < 9; ++u) R[u] = (u % 4 == 0) ? 1.f : 0.f;
        p = mk(0, 0, 0);
      }
#pragma unroll 1
      for (int k = 0; k < len; ++k) {
        const int i = M.order[st + k];
        const BodyImage& b = M.body[i];
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
        zs[i] = mk(R[2], R[5], R[8]);
        ps[i] = p;
        if (pose) pose_out(i, R, p);
      }
    }
    const int last = M.order[st + len - 1];
    if (kind == kActOpen) {
#pragma unroll
      for (int u = 0; u < 9; ++u) bR[last][u] = R[u];
      bp[last] = p;
    }
    if (!J) continue;
    // frames in this segment: every ancestor has been reached already
    for (int f = 0; f < fr.n; ++f) {
      const int kf = fr.body[f];
      if (M.seg_of[kf] != s) continue;
      const uint64_t anc = M.anc[kf];
      const int base = f * 6 * nv;
      const V3 pk = ps[kf];
      if constexpr (!ZEROS) {  // the ancestors' columns only
        uint64_t rest = anc;
        if (T::kFree) {  // the root is an ancestor of every body
          const V3 d = pk - p0;
#pragma unroll
          for (int m = 0; m < 3; ++m) {
            const V3 zr = mk(R0[m], R0[3 + m], R0[6 + m]);
            jcol(base, m, true, zr, cross(zr, d));
            jcol(base, 3 + m, true, mk(0, 0, 0), zr);
          }
          rest &= ~1ull;
        }
#pragma unroll 1
        for (; rest; rest &= rest - 1) {
          const int j = low_bit(rest);
          jcol(base, iv_of<T>(j), true, zs[j], cross(zs[j], pk - ps[j]));
        }
        continue;
      }
#pragma unroll 1
      for (int j = 0; j < nb; ++j) {
        const bool on = (anc >> j) & 1ull;
        if (T::kFree && j == 0) {
          const V3 d = pk - p0;
#pragma unroll
          for (int m = 0; m < 3; ++m) {
            const V3 zr = mk(R0[m], R0[3 + m], R0[6 + m]);
            jcol(base, m, on, zr, cross(zr, d));
            jcol(base, 3 + m, on, mk(0, 0, 0), zr);
          }
        } else {
          const V3 zj = on ? zs[j] : mk(0, 0, 0);
          const V3 pj = on ? ps[j] : mk(0, 0, 0);
          jcol(base, iv_of<T>(j), on, zj, cross(zj, pk - pj));
        }
      }
    }
  }
}

// ================================================================ RNEA VJP
// The adjoint of RNEA (see rnea_vjp_core) on segments. Outward: v, a and the
// adjoint force Fb = X Fb_parent + e gbar. Inward, inside a segment, the
// per-body forward state is not stored but stepped back from the segment's
// tip by inverting each joint transform (v_parent = X^-1 (v - e qd),
// a_parent = X^-1 (a - e qdd - v x e qd), Fb_parent = X^-1 (Fb - e gbar)),
// and the body force is recomputed; only segment tips and the accumulated
// adjoints handed to branch bodies are kept per body.
template <class T, class Img, class Seed, class Sink, class C>
FD void rnea_vjp_seg(const Img& M, const float* __restrict__ q, const float* __restrict__ qd,
                     const float* __restrict__ qdd, const Seed& gb_at, const Sink& sink, const C& col) {
  constexpr int NB = T::NBMAX;
  SV bv[NB], ba[NB], bF[NB];     // tip state of bodies with child segments
  SV aF[NB], aab[NB], avb[NB];   // adjoint contributions of child segments
  float sc[NB], ss[NB];
  const SV ag = gravity_acc(M.g);
  V3 gam = mk(0, 0, 0);
  // bodies whose aF / aab / avb hold a child segment's contribution (the
  // first one is stored, later ones added)
  uint64_t acc = 0;
#pragma unroll 1
  for (int t = 0; t < M.n_act; ++t) {
    const int act = M.act[t];
    const int s = act & 63, kind = act >> 6;
    const int st = M.seg_start[s], len = M.seg_len[s];
    if (T::kFree && s == 0) {
      const RBI I = rbi_of(M.body[0]);
      if (kind != kActClose) {
        const RootPose P = root_pose(M, q, col);
        gam = rotT(P.E, ag.v);
        bv[0] = load6(qd, 0, col);
        ba[0] = SV{mk(0, 0, 0), gam} + load6(qdd, 0, col);
        bF[0] = gb_at.root();
        if (kind == kActOpen) continue;
      }
      const SV v0 = bv[0], Fb0 = bF[0];
      const bool has = acc & 1ull;
      const SV ab = rbi_mul_add(has ? aab[0] : szero(), I, Fb0);
      const SV vb = rbi_mul_sub(crf_sub(has ? avb[0] : szero(), Fb0, rbi_mul(I, v0)), I, crm(v0, Fb0));
      sink.root(cross(ab.v, gam), vb, ab);
      continue;
    }
    const int last = M.order[st + len - 1];
    SV v, a, Fb;
    if (kind != kActClose) {
      const int p = M.seg_parent[s];
      v = p < 0 ? szero() : bv[p];
      a = p < 0 ? ag : ba[p];
      Fb = p < 0 ? szero() : bF[p];
      seg_outward(len, M.body[M.order[st]].dh, [&](int k, auto dh) {
        const int i = M.order[st + k];
        const BodyImage& b = M.body[i];
        {
          float sn, cs;
          joint_sincos(col.in(q, iq_of<T>(i)) + b.th0, &sn, &cs);
          sc[i] = cs;
          ss[i] = sn;
          const float qdi = col.in(qd, iv_of<T>(i));
          v = mot_in(b, cs, sn, v, dh);
          v.w.z += qdi;
          a = mot_in(b, cs, sn, a, dh);
          a.w.z += col.in(qdd, iv_of<T>(i));
          a = a + ez_velprod(v, qdi);
          Fb = mot_in(b, cs, sn, Fb, dh);
          Fb.w.z += gb_at(i);
        }
      });
      if (kind == kActOpen) {
        bv[last] = v;
        ba[last] = a;
        bF[last] = Fb;
        continue;
      }
    } else {
      v = bv[last];
      a = ba[last];
      Fb = bF[last];
    }
    const bool closing = kind == kActClose && ((acc >> last) & 1ull);
    SV Fc = closing ? aF[last] : szero();
    SV abc = closing ? aab[last] : szero();
    SV vbc = closing ? avb[last] : szero();
    seg_inward(len, M.body[M.order[st]].dh, [&](int k, auto dh) {
      const int i = M.order[st + k];
      const BodyImage& b = M.body[i];
      {
        const RBI I = rbi_of(b);
        const float cs = sc[i], sn = ss[i];
        const float qdi = col.in(qd, iv_of<T>(i));
        SV xa = a - ez_velprod(v, qdi);
        xa.w.z -= col.in(qdd, iv_of<T>(i));
        const SV Iv = rbi_mul(I, v);
        const SV F = crf_add(rbi_mul_add(Fc, I, a), v, Iv);
        const SV ab = rbi_mul_add(abc, I, Fb);
        const SV vb = rbi_mul_sub(crf_sub(vbc, Fb, Iv), I, crm(v, Fb)) + qdi * ez_crf(ab);
        // Fb . (e_z x* F) - ab . (e_z x xa) - vb . (e_z x v): three short FMA
        // chains (the z parts of these e_z products vanish)
        const SV ef = ez_crf(F), ea = ez_crm(xa), ev = ez_crm(v);
        const float q1 = fmaf(Fb.w.x, ef.w.x, fmaf(Fb.w.y, ef.w.y, fmaf(Fb.v.x, ef.v.x, Fb.v.y * ef.v.y)));
        const float q2 = fmaf(ab.w.x, ea.w.x, fmaf(ab.w.y, ea.w.y, fmaf(ab.v.x, ea.v.x, ab.v.y * ea.v.y)));
        const float q3 = fmaf(vb.w.x, ev.w.x, fmaf(vb.w.y, ev.w.y, fmaf(vb.v.x, ev.v.x, vb.v.y * ev.v.y)));
        const float qb = q1 - q2 - q3;
        const float qdb = fmaf(-ab.w.x, ev.w.x, fmaf(-ab.w.y, ev.w.y, fmaf(-ab.v.x, ev.v.x, fmaf(-ab.v.y, ev.v.y, vb.w.z))));
        sink(i, qb, qdb, ab.w.z);
        Fc = frc_out(b, cs, sn, F, dh);
        abc = frc_out(b, cs, sn, ab, dh);
        vbc = frc_out(b, cs, sn, vb, dh);
        if (k > 0) {
          SV vp = v;
          vp.w.z -= qdi;
          v = mot_out(b, cs, sn, vp, dh);
          a = mot_out(b, cs, sn, xa, dh);
          SV Fp = Fb;
          Fp.w.z -= gb_at(i);
          Fb = mot_out(b, cs, sn, Fp, dh);
        }
      }
    });
    const int p = M.seg_parent[s];
    if (p >= 0) {
      if ((acc >> p) & 1ull) {
        aF[p] = aF[p] + Fc;
        aab[p] = aab[p] + abc;
        avb[p] = avb[p] + vbc;
      } else {
        aF[p] = Fc;
        aab[p] = abc;
        avb[p] = vbc;
        acc |= 1ull << p;
      }
    }
  }
}

// The same adjoint for a fixed-base serial chain of N bodies with both
// sweeps unrolled: the body index, and with it every model constant's offset
// in the parameter image and each joint's frame form (k > 0), is known at
// compile time, so no index arithmetic or table lookup is left. The inward
// sweep steps the forward state back as rnea_vjp_seg does; the joint sin/cos
// pairs stay in registers.
// A seed held in a register array (entry k = dof k of a fixed-base chain).
struct RegVec {
  const float* x;
  FD float operator()(int k) const { return x[k]; }
};

template <int N, class Img, class Seed, class Sink, class C>
FD void rnea_vjp_chain(const Img& M, const float* __restrict__ q, const float* __restrict__ qd,
                       const float* __restrict__ qdd, const Seed& gb_at, const Sink& sink, const C& col) {
  float sc[N], ss[N];
  SV v = szero(), a = gravity_acc(M.g), Fb = szero();
  auto outward = [&](int k, auto dh) {
    const BodyImage& b = M.body[k];
    joint_sincos(col.in(q, k) + b.th0, &ss[k], &sc[k]);
    const float qdi = col.in(qd, k);
    v = mot_in(b, sc[k], ss[k], v, dh);
    v.w.z += qdi;
    a = mot_in(b, sc[k], ss[k], a, dh);
    a.w.z += col.in(qdd, k);
    a = a + ez_velprod(v, qdi);
    Fb = mot_in(b, sc[k], ss[k], Fb, dh);
    Fb.w.z += gb_at(k);
  };
  // (Rolling these loops after peeling body 0, which keeps the unrolled code
  // out of the instruction cache's way, measured 5-6 % slower.)
  outward(0, DhOff{});
#pragma unroll
  for (int k = 1; k < N; ++k) outward(k, DhOn{});
  SV Fc = szero(), abc = szero(), vbc = szero();
  auto inward = [&](int k, auto dh) {
    const BodyImage& b = M.body[k];
    const RBI I = rbi_of(b);
    const float cs = sc[k], sn = ss[k];
    const float qdi = col.in(qd, k);
    SV xa = a - ez_velprod(v, qdi);
    xa.w.z -= col.in(qdd, k);
    const SV Iv = rbi_mul(I, v);
    const SV F = crf_add(rbi_mul_add(Fc, I, a), v, Iv);
    const SV ab = rbi_mul_add(abc, I, Fb);
    const SV vb = rbi_mul_sub(crf_sub(vbc, Fb, Iv), I, crm(v, Fb)) + qdi * ez_crf(ab);
    const SV ef = ez_crf(F), ea = ez_crm(xa), ev = ez_crm(v);
    const float q1 = fmaf(Fb.w.x, ef.w.x, fmaf(Fb.w.y, ef.w.y, fmaf(Fb.v.x, ef.v.x, Fb.v.y * ef.v.y)));
    const float q2 = fmaf(ab.w.x, ea.w.x, fmaf(ab.w.y, ea.w.y, fmaf(ab.v.x, ea.v.x, ab.v.y * ea.v.y)));
    const float q3 = fmaf(vb.w.x, ev.w.x, fmaf(vb.w.y, ev.w.y, fmaf(vb.v.x, ev.v.x, vb.v.y * ev.v.y)));
    const float qdb = fmaf(-ab.w.x, ev.w.x, fmaf(-ab.w.y, ev.w.y, fmaf(-ab.v.x, ev.v.x, fmaf(-ab.v.y, ev.v.y, vb.w.z))));
    sink(k, q1 - q2 - q3, qdb, ab.w.z);
    if (dh) {  // not the first body: carry the adjoints to the parent, step the state back
      Fc = frc_out(b, cs, sn, F, dh);
      abc = frc_out(b, cs, sn, ab, dh);
      vbc = frc_out(b, cs, sn, vb, dh);
      SV vp = v;
      vp.w.z -= qdi;
      v = mot_out(b, cs, sn, vp, dh);
      a = mot_out(b, cs, sn, xa, dh);
      SV Fp = Fb;
      Fp.w.z -= gb_at(k);
      Fb = mot_out(b, cs, sn, Fp, dh);
    }
  };
#pragma unroll
  for (int k = N - 1; k >= 1; --k) inward(k, DhOn{});
  inward(0, DhOff{});
}

template <class T, class Img, class C>
FD void rnea_vjp_seg_one(const Img& M, const float* q, const float* qd, const float* qdd, const float* gbar,
                         float* qbar, float* qdbar, float* qddbar, const C& col) {
  rnea_vjp_seg<T>(M, q, qd, qdd, RhsFromGlobal<T, C>{gbar, col},
                  vjp_sink<T>(M, q, qbar, qdbar, qddbar, 1.f, col), col);
}

// ABA VJP on segments: w = M^-1 gbar by the articulated-body sweeps at zero
// velocity and gravity (kept per dof), then the RNEA adjoint seeded with w.
template <class T, class Img, class C>
FD void aba_vjp_seg_one(const Img& M, const float* q, const float* qd, const float* tau, const float* qdd,
                        const float* gbar, float* qbar, float* qdbar, float* taubar, const C& col) {
  (void)tau;
  LocalVec<T> w;
  P3Local<T::NBMAX> P;
  aba_seg_core<T, Img, false>(M, q, qd, RhsFromGlobal<T, C>{gbar, col}, OutToLocal<T>{&w}, col, P);
  const int nv = T::kFree ? M.nb + 5 : M.nb;
  if (taubar)
    for (int k = 0; k < nv; ++k) col.out(taubar, k, w.x[k]);
  rnea_vjp_seg<T>(M, q, qd, qdd, w, vjp_sink<T>(M, q, qbar, qdbar, nullptr, -1.f, col), col);
}

// ============================================= chain ABA VJP via the factor
// For a short serial chain the solve w = M^-1 gbar is cheaper through the
// mass matrix than through articulated inertias: composite inertias give M's
// lower triangle (registers), factored in place as M = L^T D L, then
// L^T u = gbar (back substitution), L w = D^-1 u (forward substitution).
// The rest is the unrolled chain RNEA adjoint seeded with w.
// g(k): right-hand side entry k (a global column or a thread-local vector).
template <int N, class Img, class G, class C>
FD void chain_minv(const Img& M, const float* __restrict__ q, const G& g, float* w, const C& col) {
  using T = ChainTopo<N>;
  constexpr int NT = N * (N + 1) / 2;
  float H[NT];
  float cq[N], sq[N];
  RBI Ic[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    Ic[i] = rbi_of(M.body[i]);
    joint_sincos(col.in(q, i) + M.body[i].th0, &sq[i], &cq[i]);
  }
#pragma unroll
  for (int i = N - 1; i >= 1; --i) Ic[i - 1] = rbi_add(Ic[i - 1], rbi_out(M.body[i], cq[i], sq[i], Ic[i], true));
#pragma unroll
  for (int i = 0; i < N; ++i) {
    SV F{mk(Ic[i].xz, Ic[i].yz, Ic[i].zz), mk(-Ic[i].h.y, Ic[i].h.x, 0.f)};
    H[MSink::tri(i, i)] = F.w.z;
#pragma unroll
    for (int j = i; j >= 1; --j) {
      F = frc_out(M.body[j], cq[j], sq[j], F, true);
      H[MSink::tri(i, j - 1)] = F.w.z;
    }
  }
#pragma unroll
  for (int k = N - 1; k >= 0; --k) {
    const float rk = rcp(H[MSink::tri(k, k)]);
#pragma unroll
    for (int i = k - 1; i >= 0; --i) {
      const float a = H[MSink::tri(k, i)] * rk;
#pragma unroll
      for (int j = i; j >= 0; --j) H[MSink::tri(i, j)] = fmaf(-a, H[MSink::tri(k, j)], H[MSink::tri(i, j)]);
      H[MSink::tri(k, i)] = a;
    }
  }
  float u[N];
#pragma unroll
  for (int k = N - 1; k >= 0; --k) {
    float x = g(k);
#pragma unroll
    for (int i = k + 1; i < N; ++i) x = fmaf(-H[MSink::tri(i, k)], u[i], x);
    u[k] = x;
  }
#pragma unroll
  for (int k = 0; k < N; ++k) {
    float x = u[k] * rcp(H[MSink::tri(k, k)]);
#pragma unroll
    for (int j = 0; j < k; ++j) x = fmaf(-H[MSink::tri(k, j)], w[j], x);
    w[k] = x;
  }
  (void)sizeof(T);
}

template <int N, class Img, class C>
FD void aba_vjp_chain_one(const Img& M, const float* q, const float* qd, const float* qdd, const float* gbar,
                          float* qbar, float* qdbar, float* taubar, const C& col) {
  float w[N];
  chain_minv<N>(M, q, RhsFromGlobal<ChainTopo<N>, C>{gbar, col}, w, col);
  if (taubar) {
#pragma unroll
    for (int k = 0; k < N; ++k) col.out(taubar, k, w[k]);
  }
  rnea_vjp_chain<N>(M, q, qd, qdd, RegVec{w}, vjp_sink<ChainTopo<N>>(M, q, qbar, qdbar, nullptr, -1.f, col), col);
}

}  // namespace frax
