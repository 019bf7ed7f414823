// Per-instance rigid-body algorithms (one thread = one instance), templated on
// the topology: ChainTopo<N> compiles the parent array in (parent = i - 1),
// so every loop unrolls and per-body state lives in registers; TreeTopo reads
// parents from the model image and keeps per-body state in thread-local
// arrays. Both run the same recursions:
//   FK      ^0T_i = ^0T_parent * (R Rot_z(q_i), p)            (Sec. II)
//   RNEA    Featherstone's recursive Newton-Euler (Eq. 1, f = 0)
//   CRBA    composite inertias + ancestor walk, then the tree-sparse L^T D L
//   ABA     articulated-body algorithm (Eq. 2, f = 0)
//   VJPs    hand-derived adjoints of RNEA; ABA's via w = M^-1 gbar
// All spatial quantities are in each body's internal frame (joint axis = z).
#pragma once
#include <stdint.h>

#include <type_traits>

#include "spatial.cuh"

namespace frax {

template <int N>
struct ChainTopo {
  static constexpr int NBMAX = N;
  static constexpr bool kDhRt = false;  // every body after the first is Rot_x
  static constexpr int NVMAX = N;
  static constexpr bool kFree = false;
  static constexpr bool kStatic = true;
  static constexpr bool kSeg = false;
  template <class Img>
  FD static int nb(const Img&) { return N; }
  template <class Img>
  FD static int parent(const Img&, int i) { return i - 1; }
  template <class Img>
  FD static int dparent(const Img&, int k) { return k - 1; }
};

template <int NBM, bool FREE, bool DHRT = false>
struct TreeTopo {
  static constexpr int NBMAX = NBM;
  // the Rot_x form of a body's R is taken from b.dh at run time when set (the
  // flop counter's direct formulations); the kernels keep the general form
  static constexpr bool kDhRt = DHRT;
  static constexpr int NVMAX = NBM + (FREE ? 5 : 0);
  static constexpr bool kFree = FREE;
  static constexpr bool kStatic = false;
  static constexpr bool kSeg = false;
  template <class Img>
  FD static int nb(const Img& M) { return M.nb; }
  template <class Img>
  FD static int parent(const Img& M, int i) { return M.parent[i]; }
  template <class Img>
  FD static int dparent(const Img& M, int k) { return M.dparent[k]; }
};

template <class T>
FD int iv_of(int i) { return (T::kFree && i > 0) ? i + 5 : i; }
template <class T>
FD int iq_of(int i) { return (T::kFree && i > 0) ? i + 6 : i; }

// One instance's column in the SoA arrays: element k at p[k * ld + b].
// kNC = true loads through the read-only (non-coherent) path; false loads
// through L2 only (ld.cg), for memory a running kernel sees rewritten by
// copies (the serving slab).
// streaming store (evict-first in L2) of a value written once
FD void st_cs(float* p, float v) {
#ifdef __CUDA_ARCH__
  __stcs(p, v);
#else
  *p = v;
#endif
}

// Byte offset of entry k of a batched array, k * ld floats: the boundary
// keeps ld below 2^30, so the row stride in bytes fits 32 bits and the
// offset is one 32 x 32 -> 64-bit multiply (not a 64-bit multiply and add per
// access).
FD uint64_t row_off(int k, int64_t ld) { return uint64_t(uint32_t(k)) * uint64_t(uint32_t(ld) * 4u); }
template <class F>
FD F* at_row(F* base, int k, int64_t ld) {
  using Byte = typename std::conditional<std::is_const<F>::value, const char, char>::type;
  return reinterpret_cast<F*>(reinterpret_cast<Byte*>(base) + row_off(k, ld));
}

// kRow32 = false addresses entry k as p + k * ld + b in 64-bit arithmetic:
// the two uncapped chain kernels that solve through the register factor after
// an extra sweep (forces, JVP) are scheduled better by the compiler that way
// (128 registers, 104 and 146 us at 2^20, against 96 registers and 117 and
// 163 us with the 32-bit offsets).
template <bool kNC, bool kRow32 = true>
struct ColT {
  int64_t ld, b;
  // this instance's entry k of p
  template <class F>
  FD F* at(F* p, int k) const {
    if constexpr (kRow32) return at_row(p + b, k, ld);
    else return p + k * ld + b;
  }
  FD float in(const float* __restrict__ p, int k) const {
#ifdef __CUDA_ARCH__
    return kNC ? __ldg(at(p, k)) : __ldcg(at(p, k));
#else
    return *at(p, k);
#endif
  }
  // outputs are written once and not read again by the kernel that writes
  // them (except through ColT<false>): streaming stores (evict-first in L2)
  FD void out(float* __restrict__ p, int k, float v) const { st_cs(at(p, k), v); }
};
using Col = ColT<true>;
using Col64 = ColT<true, false>;

// Asks L2 for this instance's n entries of p (one line per warp and entry)
// ahead of a sweep that reads them one body at a time.
template <class C>
FD void prefetch_entries(const float* p, int n, const C& col) {
#ifdef __CUDA_ARCH__
  for (int k = 0; k < n; ++k) asm volatile("prefetch.global.L2 [%0];" ::"l"(col.at(p, k)));
#endif
}

// Whether body i's R takes the Rot_x form here: always after the first body
// of a chain (known once the loops are unrolled), from the image when the
// topology asks for it, else never.
template <class T, class Img>
FD bool dh_of(const Img& M, int i) {
  return T::kStatic ? i > 0 : (T::kDhRt && M.body[i].dh);
}

template <class GT>
FD SV gravity_acc(const GT* g) { return SV{mk(0, 0, 0), mk(-g[0], -g[1], -g[2])}; }

// Free-flyer root: ^0R_0 = R_T R(quat), ^0p_0 = p_T + R_T p_q.
struct RootPose {
  float E[9];
  V3 r;
};
template <class Img, class C>
FD RootPose root_pose(const Img& M, const float* q, const C& c) {
  float Rq[9];
  quat_to_R(c.in(q, 3), c.in(q, 4), c.in(q, 5), c.in(q, 6), Rq);
  RootPose P;
  mat_mul(M.body[0].R, Rq, P.E);
  V3 pq = mk(c.in(q, 0), c.in(q, 1), c.in(q, 2));
  P.r = mk(M.body[0].p[0], M.body[0].p[1], M.body[0].p[2]) + rot(M.body[0].R, pq);
  return P;
}
template <class C>
FD SV load6(const float* p, int k0, const C& c) {
  return SV{mk(c.in(p, k0), c.in(p, k0 + 1), c.in(p, k0 + 2)), mk(c.in(p, k0 + 3), c.in(p, k0 + 4), c.in(p, k0 + 5))};
}
template <class C>
FD void store6(float* p, int k0, const C& c, const SV& v) {
  c.out(p, k0, v.w.x); c.out(p, k0 + 1, v.w.y); c.out(p, k0 + 2, v.w.z);
  c.out(p, k0 + 3, v.v.x); c.out(p, k0 + 4, v.v.y); c.out(p, k0 + 5, v.v.z);
}

// ============================================================ FK + Jacobians
struct Frames {
  int n;
  int body[8];
};

template <class T, class Img, class C>
FD void fk_one(const Img& M, const float* __restrict__ q, float* __restrict__ pose, const Frames& fr,
               float* __restrict__ J, const C& col) {
  const int nb = T::nb(M);
  float Rw[T::NBMAX][9];  // world rotation of the internal frames
  V3 pw[T::NBMAX];
#pragma unroll(T::kStatic ? T::NBMAX : 1)
  for (int i = 0; i < T::NBMAX; ++i) {
    if (i >= nb) break;
    const BodyImage& b = M.body[i];
    const int k = T::parent(M, i);
    if (T::kFree && i == 0) {
      RootPose P = root_pose(M, q, col);
#pragma unroll
      for (int t = 0; t < 9; ++t) Rw[0][t] = P.E[t];
      pw[0] = P.r;
    } else {
      float s, c;
      joint_sincos(col.in(q, iq_of<T>(i)) + M.body[i].th0, &s, &c);
      float A[9];
      if (k < 0) {
#pragma unroll
        for (int t = 0; t < 9; ++t) A[t] = b.R[t];
        pw[i] = mk(b.p[0], b.p[1], b.p[2]);
      } else {
        mat_mul_b(Rw[k], b, A, dh_of<T>(M, i));
        pw[i] = pw[k] + rot(Rw[k], mk(b.p[0], b.p[1], b.p[2]));
      }
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        Rw[i][3 * r] = fmaf(c, A[3 * r], s * A[3 * r + 1]);
        Rw[i][3 * r + 1] = fmaf(-s, A[3 * r], c * A[3 * r + 1]);
        Rw[i][3 * r + 2] = A[3 * r + 2];
      }
    }
    if (pose) {
      // user body frame: R_user = R_internal Q^T
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int cc = 0; cc < 3; ++cc)
          col.out(pose, 12 * i + 3 * r + cc,
                  fmaf(Rw[i][3 * r], b.Q[3 * cc], fmaf(Rw[i][3 * r + 1], b.Q[3 * cc + 1], Rw[i][3 * r + 2] * b.Q[3 * cc + 2])));
      col.out(pose, 12 * i + 9, pw[i].x);
      col.out(pose, 12 * i + 10, pw[i].y);
      col.out(pose, 12 * i + 11, pw[i].z);
    }
  }
  if (!J) return;
  const int nv = T::kFree ? nb + 5 : nb;
  for (int f = 0; f < fr.n; ++f) {
    const int kf = fr.body[f];
    const uint64_t anc = M.anc[kf];
    const V3 pk = pw[kf];
    const int base = f * 6 * nv;
#pragma unroll(T::kStatic ? T::NBMAX : 1)
    for (int j = 0; j < T::NBMAX; ++j) {
      if (j >= nb) break;
      const bool on = (anc >> j) & 1ull;
      if (T::kFree && j == 0) {
        const V3 d = pk - pw[0];
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          V3 z = mk(Rw[0][m], Rw[0][3 + m], Rw[0][6 + m]);
          V3 lin = cross(z, d);
          // angular-velocity column m
          col.out(J, base + 0 * nv + m, on ? z.x : 0.f);
          col.out(J, base + 1 * nv + m, on ? z.y : 0.f);
          col.out(J, base + 2 * nv + m, on ? z.z : 0.f);
          col.out(J, base + 3 * nv + m, on ? lin.x : 0.f);
          col.out(J, base + 4 * nv + m, on ? lin.y : 0.f);
          col.out(J, base + 5 * nv + m, on ? lin.z : 0.f);
          // linear-velocity column 3 + m
          col.out(J, base + 0 * nv + 3 + m, 0.f);
          col.out(J, base + 1 * nv + 3 + m, 0.f);
          col.out(J, base + 2 * nv + 3 + m, 0.f);
          col.out(J, base + 3 * nv + 3 + m, on ? z.x : 0.f);
          col.out(J, base + 4 * nv + 3 + m, on ? z.y : 0.f);
          col.out(J, base + 5 * nv + 3 + m, on ? z.z : 0.f);
        }
      } else {
        const int cj = iv_of<T>(j);
        V3 z = mk(Rw[j][2], Rw[j][5], Rw[j][8]);
        V3 lin = cross(z, pk - pw[j]);
        col.out(J, base + 0 * nv + cj, on ? z.x : 0.f);
        col.out(J, base + 1 * nv + cj, on ? z.y : 0.f);
        col.out(J, base + 2 * nv + cj, on ? z.z : 0.f);
        col.out(J, base + 3 * nv + cj, on ? lin.x : 0.f);
        col.out(J, base + 4 * nv + cj, on ? lin.y : 0.f);
        col.out(J, base + 5 * nv + cj, on ? lin.z : 0.f);
      }
    }
  }
}

// ====================================================================== RNEA
template <class T, class Img, class C>
FD void rnea_one(const Img& M, const float* __restrict__ q, const float* __restrict__ qd,
                 const float* __restrict__ qdd, float* __restrict__ tau, const C& col) {
  const int nb = T::nb(M);
  SV v[T::NBMAX], a[T::NBMAX], f[T::NBMAX];
  float cq[T::NBMAX], sq[T::NBMAX];
  const SV ag = gravity_acc(M.g);
#pragma unroll(T::kStatic ? T::NBMAX : 1)
  for (int i = 0; i < T::NBMAX; ++i) {
    if (i >= nb) break;
    const BodyImage& b = M.body[i];
    const RBI I = rbi_of(b);
    if (T::kFree && i == 0) {
      RootPose P = root_pose(M, q, col);
      v[0] = load6(qd, 0, col);
      a[0] = SV{mk(0, 0, 0), rotT(P.E, ag.v)};
      if (qdd) a[0] = a[0] + load6(qdd, 0, col);
    } else {
      const int k = T::parent(M, i);
      joint_sincos(col.in(q, iq_of<T>(i)) + M.body[i].th0, &sq[i], &cq[i]);
      const float qdi = col.in(qd, iv_of<T>(i));
      const float qddi = qdd ? col.in(qdd, iv_of<T>(i)) : 0.f;
      SV vi = k < 0 ? szero() : mot_in(b, cq[i], sq[i], v[k], dh_of<T>(M, i));
      SV ai = mot_in(b, cq[i], sq[i], k < 0 ? ag : a[k], dh_of<T>(M, i));
      vi.w.z += qdi;
      ai.w.z += qddi;
      ai = ai + qdi * SV{mk(vi.w.y, -vi.w.x, 0.f), mk(vi.v.y, -vi.v.x, 0.f)};  // v x e qd
      v[i] = vi;
      a[i] = ai;
    }
    f[i] = crf_add(rbi_mul(I, a[i]), v[i], rbi_mul(I, v[i]));
  }
#pragma unroll(T::kStatic ? T::NBMAX : 1)
  for (int i = T::NBMAX - 1; i >= 0; --i) {
    if (i >= nb) continue;
    if (T::kFree && i == 0) {
      store6(tau, 0, col, f[0]);
    } else {
      col.out(tau, iv_of<T>(i), f[i].w.z);
      const int k = T::parent(M, i);
      if (k >= 0) f[k] = f[k] + frc_out(M.body[i], cq[i], sq[i], f[i], dh_of<T>(M, i));
    }
  }
}

// ============================================================= CRBA + LTDL
// Mass-matrix entry sink: full M (row-major) and/or the packed lower
// triangle that the in-place L^T D L factorisation then works on.
struct MSink {
  float* M;
  float* LD;
  int nv;
  FD static int tri(int i, int j) { return i * (i + 1) / 2 + j; }
};

template <class T, class Img, class C>
FD void crba_one(const Img& M, const float* __restrict__ q, float* __restrict__ Mout,
                 float* __restrict__ LD, const C& col) {
  const int nb = T::nb(M);
  const int nv = T::kFree ? nb + 5 : nb;
  float cq[T::NBMAX], sq[T::NBMAX];
  RBI Ic[T::NBMAX];
  // chain: keep the lower triangle in registers for the factorisation
  constexpr int NT = T::kStatic ? T::NVMAX * (T::NVMAX + 1) / 2 : 1;
  float H[NT];
#pragma unroll(T::kStatic ? T::NBMAX : 1)
  for (int i = 0; i < T::NBMAX; ++i) {
    if (i >= nb) break;
    Ic[i] = rbi_of(M.body[i]);
    if (!(T::kFree && i == 0)) joint_sincos(col.in(q, iq_of<T>(i)) + M.body[i].th0, &sq[i], &cq[i]);
  }
#pragma unroll(T::kStatic ? T::NBMAX : 1)
  for (int i = T::NBMAX - 1; i >= 1; --i) {
    if (i >= nb) continue;
    const int k = T::parent(M, i);
    if (k >= 0) Ic[k] = rbi_add(Ic[k], rbi_out(M.body[i], cq[i], sq[i], Ic[i], dh_of<T>(M, i)));
  }
  auto put = [&](int r, int c, float val) {  // r >= c
    if (Mout) {
      col.out(Mout, r * nv + c, val);
      if (r != c) col.out(Mout, c * nv + r, val);
    }
    if (LD) {
      if (T::kStatic) H[MSink::tri(r, c)] = val;
      else col.out(LD, MSink::tri(r, c), val);
    }
  };
#pragma unroll(T::kStatic ? T::NBMAX : 1)
  for (int i = 0; i < T::NBMAX; ++i) {
    if (i >= nb) break;
    if (T::kFree && i == 0) {
      // 6x6 block = the root composite inertia [[I, [h]x], [[h]x^T, m 1]]
      const RBI& Cc = Ic[0];
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
      continue;
    }
    const int di = iv_of<T>(i);
    const RBI& Cc = Ic[i];
    SV F{mk(Cc.xz, Cc.yz, Cc.zz), mk(-Cc.h.y, Cc.h.x, 0.f)};  // I^c_i e_z
    put(di, di, F.w.z);
    int j = i;
    uint64_t done = 1ull << i;
#pragma unroll(T::kStatic ? T::NBMAX : 1)
    for (int step = 0; step < T::NBMAX; ++step) {
      const int k = T::parent(M, j);
      if (k < 0) break;
      F = frc_out(M.body[j], cq[j], sq[j], F, dh_of<T>(M, j));
      j = k;
      done |= 1ull << j;
      if (T::kFree && j == 0) {
        put(di, 0, F.w.x); put(di, 1, F.w.y); put(di, 2, F.w.z);
        put(di, 3, F.v.x); put(di, 4, F.v.y); put(di, 5, F.v.z);
      } else {
        put(di, iv_of<T>(j), F.w.z);
      }
    }
    if (!T::kStatic) {
      // zeros for the non-ancestor pairs (j < i, j not in Anc(i))
      for (int jj = 0; jj < i; ++jj) {
        if ((done >> jj) & 1ull) continue;
        if (T::kFree && jj == 0) {
          for (int m = 0; m < 6; ++m) put(di, m, 0.f);
        } else {
          put(di, iv_of<T>(jj), 0.f);
        }
      }
    }
  }
  if (!LD) return;
  // In-place L^T D L (Featherstone's LTDL): for k from the last dof up, with
  // lambda the dof-level parent, H(i, j) -= H(k, i)/H(k, k) * H(k, j) along
  // the path, then H(k, i) becomes L_ki. Fill-in stays inside Anc.
  if (T::kStatic) {
#pragma unroll
    for (int k = T::NVMAX - 1; k >= 0; --k) {
      const float rk = rcp(H[MSink::tri(k, k)]);
#pragma unroll
      for (int i = k - 1; i >= 0; --i) {
        const float a = H[MSink::tri(k, i)] * rk;
#pragma unroll
        for (int j = i; j >= 0; --j) H[MSink::tri(i, j)] = fmaf(-a, H[MSink::tri(k, j)], H[MSink::tri(i, j)]);
        H[MSink::tri(k, i)] = a;
      }
    }
#pragma unroll
    for (int t = 0; t < NT; ++t) col.out(LD, t, H[t]);
  } else {
    const ColT<false> own{col.ld, col.b};  // LD is rewritten in place: read through L2
    for (int k = nv - 1; k >= 0; --k) {
      const float rk = rcp(own.in(LD, MSink::tri(k, k)));
      int i = T::dparent(M, k);
      while (i >= 0) {
        const float a = own.in(LD, MSink::tri(k, i)) * rk;
        int j = i;
        while (j >= 0) {
          col.out(LD, MSink::tri(i, j), fmaf(-a, own.in(LD, MSink::tri(k, j)), own.in(LD, MSink::tri(i, j))));
          j = T::dparent(M, j);
        }
        col.out(LD, MSink::tri(k, i), a);
        i = T::dparent(M, i);
      }
    }
  }
}

// ======================================================================= ABA
// 6x6 SPD solve x = A^-1 b for the free-flyer root (dense Cholesky).
FD SV spd6_solve(const AI& I, const SV& rhs) {
  float A[6][6];
  const float* Af = I.A;
  const float* Cf = I.C;
  const float As[3][3] = {{Af[0], Af[3], Af[4]}, {Af[3], Af[1], Af[5]}, {Af[4], Af[5], Af[2]}};
  const float Cs[3][3] = {{Cf[0], Cf[3], Cf[4]}, {Cf[3], Cf[1], Cf[5]}, {Cf[4], Cf[5], Cf[2]}};
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      A[r][c] = As[r][c];
      A[r][3 + c] = I.B[3 * r + c];
      A[3 + r][c] = I.B[3 * c + r];
      A[3 + r][3 + c] = Cs[r][c];
    }
  float L[6][6];
  float dinv[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    float d = A[j][j];
#pragma unroll
    for (int k = 0; k < j; ++k) d = fmaf(-L[j][k], L[j][k], d);
    dinv[j] = rsqrtf(d);
    const float sd = d * dinv[j];
    L[j][j] = sd;
#pragma unroll
    for (int i = j + 1; i < 6; ++i) {
      float x = A[i][j];
#pragma unroll
      for (int k = 0; k < j; ++k) x = fmaf(-L[i][k], L[j][k], x);
      L[i][j] = x * dinv[j];
    }
  }
  float y[6] = {rhs.w.x, rhs.w.y, rhs.w.z, rhs.v.x, rhs.v.y, rhs.v.z};
#pragma unroll
  for (int i = 0; i < 6; ++i) {
#pragma unroll
    for (int k = 0; k < i; ++k) y[i] = fmaf(-L[i][k], y[k], y[i]);
    y[i] *= dinv[i];
  }
#pragma unroll
  for (int i = 5; i >= 0; --i) {
#pragma unroll
    for (int k = i + 1; k < 6; ++k) y[i] = fmaf(-L[k][i], y[k], y[i]);
    y[i] *= dinv[i];
  }
  return SV{mk(y[0], y[1], y[2]), mk(y[3], y[4], y[5])};
}

// Articulated-body algorithm. With `with_velocity` false the same sweeps solve
// M x = rhs (zero velocity, no gravity): the M^-1 of the ABA adjoint.
// rhs_at(i) gives tau for revolute body i; rhs0 the root wrench.
template <class T, class Img, bool VEL, class Rhs, class Out, class C>
FD void aba_core(const Img& M, const float* __restrict__ q, const float* __restrict__ qd, const Rhs& rhs_at,
                 const Out& out_at, const C& col) {
  const int nb = T::nb(M);
  float cq[T::NBMAX], sq[T::NBMAX];
  SV v[T::NBMAX], cb[T::NBMAX], pA[T::NBMAX], U[T::NBMAX], a[T::NBMAX];
  float Dinv[T::NBMAX], u[T::NBMAX];
  AI IA[T::NBMAX];
  RootPose P;
  const SV ag = VEL ? gravity_acc(M.g) : szero();
#pragma unroll(T::kStatic ? T::NBMAX : 1)
  for (int i = 0; i < T::NBMAX; ++i) {
    if (i >= nb) break;
    const BodyImage& b = M.body[i];
    const RBI I = rbi_of(b);
    IA[i] = ai_of(I);
    if (T::kFree && i == 0) {
      P = root_pose(M, q, col);
      v[0] = VEL ? load6(qd, 0, col) : szero();
      cb[0] = szero();
    } else {
      const int k = T::parent(M, i);
      joint_sincos(col.in(q, iq_of<T>(i)) + M.body[i].th0, &sq[i], &cq[i]);
      if (VEL) {
        const float qdi = col.in(qd, iv_of<T>(i));
        SV vi = k < 0 ? szero() : mot_in(b, cq[i], sq[i], v[k], dh_of<T>(M, i));
        vi.w.z += qdi;
        v[i] = vi;
        cb[i] = qdi * SV{mk(vi.w.y, -vi.w.x, 0.f), mk(vi.v.y, -vi.v.x, 0.f)};
      } else {
        v[i] = szero();
        cb[i] = szero();
      }
    }
    pA[i] = VEL ? crf(v[i], rbi_mul(I, v[i])) : szero();
  }
#pragma unroll(T::kStatic ? T::NBMAX : 1)
  for (int i = T::NBMAX - 1; i >= 0; --i) {
    if (i >= nb) continue;
    if (T::kFree && i == 0) continue;
    const SV Ui = ai_col_z(IA[i]);
    const float di = rcp(Ui.w.z);
    const float ui = rhs_at(i) - pA[i].w.z;
    U[i] = Ui;
    Dinv[i] = di;
    u[i] = ui;
    const int k = T::parent(M, i);
    if (k >= 0) {
      AI Ia = IA[i];
      ai_rank1_sub_z(Ia, Ui, di);
      SV pa = axpy(ui * di, Ui, pA[i]);
      if (VEL) pa = ai_mul_z_add(pa, Ia, cb[i]);
      ai_out_z(M.body[i], cq[i], sq[i], Ia, dh_of<T>(M, i));
      ai_add(IA[k], Ia);
      pA[k] = pA[k] + frc_out(M.body[i], cq[i], sq[i], pa, dh_of<T>(M, i));
    }
  }
#pragma unroll(T::kStatic ? T::NBMAX : 1)
  for (int i = 0; i < T::NBMAX; ++i) {
    if (i >= nb) break;
    if (T::kFree && i == 0) {
      const SV ap = SV{mk(0, 0, 0), rotT(P.E, ag.v)};
      const SV rhs0 = rhs_at.root() - pA[0];
      a[0] = spd6_solve(IA[0], rhs0);
      out_at.root(a[0] - ap);
    } else {
      const int k = T::parent(M, i);
      SV ap = mot_in(M.body[i], cq[i], sq[i], k < 0 ? ag : a[k], dh_of<T>(M, i)) + cb[i];
      const float qddi = (u[i] - dot(U[i], ap)) * Dinv[i];
      ap.w.z += qddi;
      a[i] = ap;
      out_at(i, qddi);
    }
  }
}

template <class T, class C>
struct RhsFromGlobal {
  const float* p;
  C col;
  FD float operator()(int i) const { return col.in(p, iv_of<T>(i)); }
  FD SV root() const { return load6(p, 0, col); }
};
template <class T, class C>
struct OutToGlobal {
  float* p;
  C col;
  FD void operator()(int i, float x) const { col.out(p, iv_of<T>(i), x); }
  FD void root(const SV& x) const { store6(p, 0, col, x); }
};

template <class T, class Img, class C>
FD void aba_one(const Img& M, const float* __restrict__ q, const float* __restrict__ qd,
                const float* __restrict__ tau, float* __restrict__ qdd, const C& col) {
  aba_core<T, Img, true>(M, q, qd, RhsFromGlobal<T, C>{tau, col}, OutToGlobal<T, C>{qdd, col}, col);
}

// ================================================================ RNEA VJP
// Reverse-mode adjoint of the RNEA recursion. Forward: v, a, f as in RNEA
// and Fb_i = X_i Fb_parent + e gbar_i (the adjoint of the inward force sum).
// Inward: with F_i the accumulated force, abar_i = I Fb_i + sum X_c^T abar_c,
// vbar_i = -(Fb_i x* I v_i) - I (v_i x Fb_i) + (e qd_i) x* abar_i
//          + sum X_c^T vbar_c;
// qbar_i = Fb_i.(e x* F_i) - abar_i.(e x X_i a_par) - vbar_i.(e x X_i v_par),
// qdbar_i = e.vbar_i + abar_i.(v_i x e), qddbar_i = e.abar_i.
template <class T, class Img, class Seed, class Sink, class C>
FD void rnea_vjp_core(const Img& M, const float* __restrict__ q, const float* __restrict__ qd,
                      const float* __restrict__ qdd, const Seed& gb_at, const Sink& sink, const C& col) {
  const int nb = T::nb(M);
  float cq[T::NBMAX], sq[T::NBMAX];
  SV v[T::NBMAX], xa[T::NBMAX], F[T::NBMAX], Fb[T::NBMAX], ab[T::NBMAX], vb[T::NBMAX];
  RootPose P;
  const SV ag = gravity_acc(M.g);
  SV a_prev[T::NBMAX];
#pragma unroll(T::kStatic ? T::NBMAX : 1)
  for (int i = 0; i < T::NBMAX; ++i) {
    if (i >= nb) break;
    const BodyImage& b = M.body[i];
    const RBI I = rbi_of(b);
    SV ai;
    if (T::kFree && i == 0) {
      P = root_pose(M, q, col);
      v[0] = load6(qd, 0, col);
      xa[0] = SV{mk(0, 0, 0), rotT(P.E, ag.v)};
      ai = xa[0] + load6(qdd, 0, col);
      Fb[0] = gb_at.root();
    } else {
      const int k = T::parent(M, i);
      joint_sincos(col.in(q, iq_of<T>(i)) + M.body[i].th0, &sq[i], &cq[i]);
      const float qdi = col.in(qd, iv_of<T>(i));
      SV vi = k < 0 ? szero() : mot_in(b, cq[i], sq[i], v[k], dh_of<T>(M, i));
      xa[i] = mot_in(b, cq[i], sq[i], k < 0 ? ag : a_prev[k], dh_of<T>(M, i));
      vi.w.z += qdi;
      v[i] = vi;
      ai = xa[i];
      ai.w.z += col.in(qdd, iv_of<T>(i));
      ai = ai + qdi * SV{mk(vi.w.y, -vi.w.x, 0.f), mk(vi.v.y, -vi.v.x, 0.f)};
      SV fb = k < 0 ? szero() : mot_in(b, cq[i], sq[i], Fb[k], dh_of<T>(M, i));
      fb.w.z += gb_at(i);
      Fb[i] = fb;
    }
    a_prev[i] = ai;
    F[i] = crf_add(rbi_mul(I, ai), v[i], rbi_mul(I, v[i]));
    ab[i] = szero();
    vb[i] = szero();
  }
#pragma unroll(T::kStatic ? T::NBMAX : 1)
  for (int i = T::NBMAX - 1; i >= 0; --i) {
    if (i >= nb) continue;
    const BodyImage& b = M.body[i];
    const RBI I = rbi_of(b);
    const SV abi = ab[i] + rbi_mul(I, Fb[i]);
    SV vbi = crf_sub(vb[i], Fb[i], rbi_mul(I, v[i])) - rbi_mul(I, crm(v[i], Fb[i]));
    if (T::kFree && i == 0) {
      // root: q enters only through X_0 a_g; translation has no effect
      sink.root(cross(abi.v, xa[0].v), vbi, abi);
    } else {
      const float qdi = col.in(qd, iv_of<T>(i));
      vbi = vbi + qdi * ez_crf(abi);
      const float qddb = abi.w.z;
      const float qdb = vbi.w.z - dot(abi, ez_crm(v[i]));
      const float qb = dot(Fb[i], ez_crf(F[i])) - dot(abi, ez_crm(xa[i])) - dot(vbi, ez_crm(v[i]));
      sink(i, qb, qdb, qddb);
      const int k = T::parent(M, i);
      if (k >= 0) {
        F[k] = F[k] + frc_out(b, cq[i], sq[i], F[i], dh_of<T>(M, i));
        ab[k] = ab[k] + frc_out(b, cq[i], sq[i], abi, dh_of<T>(M, i));
        vb[k] = vb[k] + frc_out(b, cq[i], sq[i], vbi, dh_of<T>(M, i));
      }
    }
  }
}

// Writes VJP results (scaled by `sign`) to global memory; the free-flyer
// root's tangent q-gradient goes to the ambient layout: position slots get
// R * 0 (tau does not depend on the root position) and the quaternion slots
// 2 quat (x) [w_bar; 0].
template <class T, class C>
struct VjpToGlobal {
  float* qbar;
  float* qdbar;
  float* qddbar;
  float sign;
  float quat[4];
  C col;
  FD void operator()(int i, float qb, float qdb, float qddb) const {
    if (qbar) col.out(qbar, iq_of<T>(i), sign * qb);
    if (qdbar) col.out(qdbar, iv_of<T>(i), sign * qdb);
    if (qddbar) col.out(qddbar, iv_of<T>(i), sign * qddb);
  }
  FD void root(V3 wbar, const SV& vbar, const SV& abar) const {
    if (qbar) {
      const float x = quat[0], y = quat[1], z = quat[2], w = quat[3];
      // quat (x) [wbar; 0]: vector part w*wbar + qv x wbar, scalar -qv.wbar
      const V3 qv = mk(x, y, z);
      const V3 vp = w * wbar + cross(qv, wbar);
      const float sp = -dot(qv, wbar);
      col.out(qbar, 0, 0.f);
      col.out(qbar, 1, 0.f);
      col.out(qbar, 2, 0.f);
      col.out(qbar, 3, 2.f * sign * vp.x);
      col.out(qbar, 4, 2.f * sign * vp.y);
      col.out(qbar, 5, 2.f * sign * vp.z);
      col.out(qbar, 6, 2.f * sign * sp);
    }
    if (qdbar) store6(qdbar, 0, col, sign * vbar);
    if (qddbar) store6(qddbar, 0, col, sign * abar);
  }
};

template <class T, class Img, class C>
FD VjpToGlobal<T, C> vjp_sink(const Img& M, const float* q, float* qbar, float* qdbar, float* qddbar,
                              float sign, const C& col) {
  VjpToGlobal<T, C> s{qbar, qdbar, qddbar, sign, {0, 0, 0, 1}, col};
  if (T::kFree) {
    s.quat[0] = col.in(q, 3);
    s.quat[1] = col.in(q, 4);
    s.quat[2] = col.in(q, 5);
    s.quat[3] = col.in(q, 6);
  }
  return s;
}

template <class T, class Img, class C>
FD void rnea_vjp_one(const Img& M, const float* q, const float* qd, const float* qdd, const float* gbar,
                     float* qbar, float* qdbar, float* qddbar, const C& col) {
  rnea_vjp_core<T>(M, q, qd, qdd, RhsFromGlobal<T, C>{gbar, col}, vjp_sink<T>(M, q, qbar, qdbar, qddbar, 1.f, col),
                   col);
}

// ================================================================= ABA VJP
// w = M^-1 gbar by the articulated-body sweeps at zero velocity and gravity,
// kept per body; then the RNEA adjoint at (q, qd, qdd) seeded with w, negated.
template <class T>
struct LocalVec {
  float x[T::NVMAX];
  FD float operator()(int i) const { return x[iv_of<T>(i)]; }
  FD SV root() const { return SV{mk(x[0], x[1], x[2]), mk(x[3], x[4], x[5])}; }
};
template <class T>
struct OutToLocal {
  LocalVec<T>* w;
  FD void operator()(int i, float v) const { w->x[iv_of<T>(i)] = v; }
  FD void root(const SV& v) const {
    w->x[0] = v.w.x; w->x[1] = v.w.y; w->x[2] = v.w.z;
    w->x[3] = v.v.x; w->x[4] = v.v.y; w->x[5] = v.v.z;
  }
};

template <class T, class Img, class C>
FD void aba_vjp_one(const Img& M, const float* q, const float* qd, const float* tau, const float* qdd,
                    const float* gbar, float* qbar, float* qdbar, float* taubar, const C& col) {
  (void)tau;  // the derivative is evaluated at the saved qdd = ABA(q, qd, tau)
  LocalVec<T> w;
  aba_core<T, Img, false>(M, q, qd, RhsFromGlobal<T, C>{gbar, col}, OutToLocal<T>{&w}, col);
  const int nv = T::kFree ? T::nb(M) + 5 : T::nb(M);
  if (taubar) {
#pragma unroll(T::kStatic ? T::NVMAX : 1)
    for (int k = 0; k < T::NVMAX; ++k) {
      if (k >= nv) break;
      col.out(taubar, k, w.x[k]);
    }
  }
  rnea_vjp_core<T>(M, q, qd, qdd, w, vjp_sink<T>(M, q, qbar, qdbar, nullptr, -1.f, col), col);
}

}  // namespace frax
