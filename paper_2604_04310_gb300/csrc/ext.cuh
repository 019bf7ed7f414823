// External forces (Algorithm 1's ^0F_ext,i; Eq. 1 and 2's J^T f), one thread
// per instance. Forces arrive as spatial forces on the bodies in root-frame
// Pluecker coordinates, [moment about the root origin; force], so they add
// without any transform; their generalized force is
//
//   tau_ext_j = (^0S_j)^T sum_{i in subtree(j)} ^0F_ext,i,
//   ^0S_j = [z_j; p_j x z_j]  =>  tau_ext_j = z_j . (n - p_j x f)
//
// for a revolute joint with world axis z_j through the world point p_j, and
// the subtree's wrench in the root body's coordinates for a free-flyer root.
// One sweep: world axes and joint origins outward segment by segment
// (depth-first, as the segment kernels), world force sums inward. Algorithm 1
// subtracts the external force, so inverse dynamics is RNEA - tau_ext and
// forward dynamics is ABA with tau + tau_ext.
#pragma once
#include "seg.cuh"

namespace frax {

template <class T, class Img, class C, class Sink>
FD void ext_tau(const Img& M, const float* __restrict__ q, const float* __restrict__ fext, const C& col,
                const Sink& sink) {
  constexpr int NB = T::NBMAX;
  float bE[NB][9];  // world rotation of bodies with child segments
  V3 bp[NB];        // and their origins
  SV Fa[NB];        // world force sums handed back by child segments
  V3 sz[NB], sp[NB];  // axes and origins of open segments' bodies
  SV F0 = szero();
#pragma unroll 1
  for (int t = 0; t < M.n_act; ++t) {
    const int act = M.act[t];
    const int s = act & 63, kind = act >> 6;
    const int st = M.seg_start[s], len = M.seg_len[s];
    if (T::kFree && s == 0) {
      const RootPose P = root_pose(M, q, col);
      if (kind != kActClose) {
        F0 = load6(fext, 0, col);
        if (kind == kActOpen) {
#pragma unroll
          for (int k = 0; k < 9; ++k) bE[0][k] = P.E[k];
          bp[0] = P.r;
          Fa[0] = szero();
          continue;
        }
      } else {
        F0 = F0 + Fa[0];
      }
      // the subtree's wrench in root-body coordinates: [E^T (n - r x f); E^T f]
      sink.root(SV{rotT(P.E, F0.w - cross(P.r, F0.v)), rotT(P.E, F0.v)});
      continue;
    }
    V3 z[kMaxSeg], p[kMaxSeg];
    const int last = M.order[st + len - 1];
    if (kind != kActClose) {
      const int ps = M.seg_parent[s];
      float E[9];
      V3 o;
      if (ps < 0) {
#pragma unroll
        for (int k = 0; k < 9; ++k) E[k] = (k % 4 == 0) ? 1.f : 0.f;
        o = mk(0, 0, 0);
      } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) E[k] = bE[ps][k];
        o = bp[ps];
      }
#pragma unroll
      for (int k = 0; k < kMaxSeg; ++k) {
        if (k < len) {
          const int i = M.order[st + k];
          const BodyImage& b = M.body[i];
          o = o + rot(E, mk(b.p[0], b.p[1], b.p[2]));
          float ER[9];
          mat_mul_b(E, b, ER, k > 0);
          z[k] = mk(ER[2], ER[5], ER[8]);
          p[k] = o;
          if (kind == kActOpen && k == len - 1) {
            float sn, cs;
            joint_sincos(col.in(q, iq_of<T>(i)) + M.body[i].th0, &sn, &cs);
#pragma unroll
            for (int r = 0; r < 3; ++r) {
              const float x = ER[3 * r], y = ER[3 * r + 1];
              bE[i][3 * r] = fmaf(cs, x, sn * y);
              bE[i][3 * r + 1] = fmaf(-sn, x, cs * y);
              bE[i][3 * r + 2] = ER[3 * r + 2];
            }
            bp[i] = o;
          } else if (k < len - 1) {
            float sn, cs;
            joint_sincos(col.in(q, iq_of<T>(i)) + M.body[i].th0, &sn, &cs);
#pragma unroll
            for (int r = 0; r < 3; ++r) {
              const float x = ER[3 * r], y = ER[3 * r + 1];
              E[3 * r] = fmaf(cs, x, sn * y);
              E[3 * r + 1] = fmaf(-sn, x, cs * y);
              E[3 * r + 2] = ER[3 * r + 2];
            }
          }
        }
      }
      if (kind == kActOpen) {
        Fa[last] = szero();
#pragma unroll
        for (int k = 0; k < kMaxSeg; ++k)
          if (k < len) {
            const int i = M.order[st + k];
            sz[i] = z[k];
            sp[i] = p[k];
          }
        continue;
      }
    } else {
#pragma unroll
      for (int k = 0; k < kMaxSeg; ++k)
        if (k < len) {
          const int i = M.order[st + k];
          z[k] = sz[i];
          p[k] = sp[i];
        }
    }
    SV F = kind == kActClose ? Fa[last] : szero();
#pragma unroll
    for (int k = kMaxSeg - 1; k >= 0; --k) {
      if (k < len) {
        const int i = M.order[st + k];
        F = F + load6(fext, 6 * i, col);
        sink(i, dot(z[k], F.w - cross(p[k], F.v)));
      }
    }
    const int ps = M.seg_parent[s];
    if (ps >= 0) Fa[ps] = Fa[ps] + F;
  }
}

// The same for a fixed-base serial chain of N bodies, unrolled: the world
// axes and joint origins stay in registers.
template <int N, class Img, class C, class Sink>
FD void ext_tau_chain(const Img& M, const float* __restrict__ q, const float* __restrict__ fext, const C& col,
                      const Sink& sink) {
  V3 z[N], p[N];
  float E[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
  V3 o = mk(0, 0, 0);
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const BodyImage& b = M.body[k];
    o = o + rot(E, mk(b.p[0], b.p[1], b.p[2]));
    float ER[9];
    mat_mul_b(E, b, ER, k > 0);
    z[k] = mk(ER[2], ER[5], ER[8]);
    p[k] = o;
    if (k < N - 1) {
      float sn, cs;
      joint_sincos(col.in(q, k) + b.th0, &sn, &cs);
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const float x = ER[3 * r], y = ER[3 * r + 1];
        E[3 * r] = fmaf(cs, x, sn * y);
        E[3 * r + 1] = fmaf(-sn, x, cs * y);
        E[3 * r + 2] = ER[3 * r + 2];
      }
    }
  }
  SV F = szero();
#pragma unroll
  for (int k = N - 1; k >= 0; --k) {
    F = F + load6(fext, 6 * k, col);
    sink(k, dot(z[k], F.w - cross(p[k], F.v)));
  }
}

// tau -= x: the RNEA output, read back through L2 (this thread wrote it).
template <class T>
struct SubFromGlobal {
  float* p;
  ColT<false> col;
  FD void operator()(int i, float x) const { col.out(p, iv_of<T>(i), col.in(p, iv_of<T>(i)) - x); }
  FD void root(const SV& x) const { store6(p, 0, col, load6(p, 0, col) - x); }
};

// tau + tau_ext as the right-hand side of ABA.
template <class T, class C>
struct RhsPlusLocal {
  const float* p;
  C col;
  const LocalVec<T>* w;
  FD float operator()(int i) const { return col.in(p, iv_of<T>(i)) + (*w)(i); }
  FD SV root() const { return load6(p, 0, col) + w->root(); }
};

}  // namespace frax
