// Device spatial algebra, FP32, one instance per thread: 3-vectors, 6-D
// spatial vectors [angular; linear], compact rigid-body inertias and
// articulated (general symmetric 6x6) inertias, and the joint transforms in
// the internal frames of model_image.h (joint axis = local z).
#pragma once
#include <cuda_runtime.h>

#include "model_image.h"

namespace frax {

#define FD __host__ __device__ __forceinline__

// index of the lowest set bit of a non-zero mask
FD int low_bit(uint64_t m) {
#ifdef __CUDA_ARCH__
  return __ffsll(static_cast<long long>(m)) - 1;
#else
  return __builtin_ctzll(m);
#endif
}

// sin and cos of a joint angle: reduced to [-pi, pi] by 2 pi split in two
// parts (Cody and Waite's additive reduction), then the SFU approximations
// (absolute error below 5e-7 on [-pi, pi]). Host builds call sincosf.
FD void joint_sincos(float x, float* s, float* c) {
#ifdef __CUDA_ARCH__
  const float k = rintf(x * 0.15915494309189535f);           // x / (2 pi)
  const float r = fmaf(-k, 6.28318548202514648f, x);         // minus k hi
  __sincosf(fmaf(k, 1.7484555314695172e-07f, r), s, c);     // minus k lo
#else
  sincosf(x, s, c);
#endif
}

// 1 / x by the SFU reciprocal (at most 2 ulp from the rounded quotient, for
// the pivots and articulated inertias here, all well inside the normal range)
FD float rcp(float x) {
#ifdef __CUDA_ARCH__
  return __fdividef(1.f, x);
#else
  return 1.f / x;
#endif
}

struct V3 {
  float x, y, z;
};
struct SV {
  V3 w, v;  // motion: [omega; v]   force: [n; f]
};

FD V3 mk(float x, float y, float z) { return V3{x, y, z}; }
FD V3 operator+(V3 a, V3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
FD V3 operator-(V3 a, V3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
FD V3 operator-(V3 a) { return mk(-a.x, -a.y, -a.z); }
FD V3 operator*(float s, V3 a) { return mk(s * a.x, s * a.y, s * a.z); }
FD float dot(V3 a, V3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
FD V3 cross(V3 a, V3 b) {
  return mk(fmaf(a.y, b.z, -a.z * b.y), fmaf(a.z, b.x, -a.x * b.z), fmaf(a.x, b.y, -a.y * b.x));
}
// c + a x b and c - a x b, each component two FMAs on the accumulator
FD V3 cross_add(V3 c, V3 a, V3 b) {
  return mk(fmaf(a.y, b.z, fmaf(-a.z, b.y, c.x)), fmaf(a.z, b.x, fmaf(-a.x, b.z, c.y)),
            fmaf(a.x, b.y, fmaf(-a.y, b.x, c.z)));
}
FD V3 cross_sub(V3 c, V3 a, V3 b) {
  return mk(fmaf(-a.y, b.z, fmaf(a.z, b.y, c.x)), fmaf(-a.z, b.x, fmaf(a.x, b.z, c.y)),
            fmaf(-a.x, b.y, fmaf(a.y, b.x, c.z)));
}
FD SV operator+(const SV& a, const SV& b) { return SV{a.w + b.w, a.v + b.v}; }
FD SV operator-(const SV& a, const SV& b) { return SV{a.w - b.w, a.v - b.v}; }
FD SV operator*(float s, const SV& a) { return SV{s * a.w, s * a.v}; }
FD float dot(const SV& a, const SV& b) { return dot(a.w, b.w) + dot(a.v, b.v); }
FD SV szero() { return SV{mk(0, 0, 0), mk(0, 0, 0)}; }
// s x + y with every component one FMA (no contraction left to the compiler)
FD SV axpy(float s, const SV& x, const SV& y) {
  return SV{mk(fmaf(s, x.w.x, y.w.x), fmaf(s, x.w.y, y.w.y), fmaf(s, x.w.z, y.w.z)),
            mk(fmaf(s, x.v.x, y.v.x), fmaf(s, x.v.y, y.v.y), fmaf(s, x.v.z, y.v.z))};
}

// motion x motion (Table III's x); sums of cross products as FMA chains
FD SV crm(const SV& a, const SV& b) { return SV{cross(a.w, b.w), cross_add(cross(a.w, b.v), a.v, b.w)}; }
// motion x* force (Table III's x*)
FD SV crf(const SV& a, const SV& f) { return SV{cross_add(cross(a.w, f.w), a.v, f.v), cross(a.w, f.v)}; }
// acc + a x* f and acc - a x* f, accumulated in place
FD SV crf_add(const SV& acc, const SV& a, const SV& f) {
  return SV{cross_add(cross_add(acc.w, a.w, f.w), a.v, f.v), cross_add(acc.v, a.w, f.v)};
}
FD SV crf_sub(const SV& acc, const SV& a, const SV& f) {
  return SV{cross_sub(cross_sub(acc.w, a.w, f.w), a.v, f.v), cross_sub(acc.v, a.w, f.v)};
}

// --- rotations --------------------------------------------------------------
template <class RT>
FD V3 rot(const RT* R, V3 a) {  // R a, R row-major
  return mk(fmaf(R[0], a.x, fmaf(R[1], a.y, R[2] * a.z)), fmaf(R[3], a.x, fmaf(R[4], a.y, R[5] * a.z)),
            fmaf(R[6], a.x, fmaf(R[7], a.y, R[8] * a.z)));
}
template <class RT>
FD V3 rotT(const RT* R, V3 a) {  // R^T a
  return mk(fmaf(R[0], a.x, fmaf(R[3], a.y, R[6] * a.z)), fmaf(R[1], a.x, fmaf(R[4], a.y, R[7] * a.z)),
            fmaf(R[2], a.x, fmaf(R[5], a.y, R[8] * a.z)));
}
// Rot_z(q) a and Rot_z(q)^T a with (c, s) = (cos q, sin q)
FD V3 rotz(float c, float s, V3 a) { return mk(fmaf(c, a.x, -s * a.y), fmaf(s, a.x, c * a.y), a.z); }
FD V3 rotzT(float c, float s, V3 a) { return mk(fmaf(c, a.x, s * a.y), fmaf(-s, a.x, c * a.y), a.z); }

// rotation matrix of a unit quaternion (x, y, z, w), row-major
FD void quat_to_R(float x, float y, float z, float w, float* R) {
  float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z, wx = w * x,
        wy = w * y, wz = w * z;
  R[0] = 1.f - 2.f * (yy + zz); R[1] = 2.f * (xy - wz);       R[2] = 2.f * (xz + wy);
  R[3] = 2.f * (xy + wz);       R[4] = 1.f - 2.f * (xx + zz); R[5] = 2.f * (yz - wx);
  R[6] = 2.f * (xz - wy);       R[7] = 2.f * (yz + wx);       R[8] = 1.f - 2.f * (xx + yy);
}
// C = A B (3x3 row-major)
template <class AT, class BT>
FD void mat_mul(const AT* A, const BT* B, float* C) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      C[3 * r + c] = fmaf(A[3 * r], B[c], fmaf(A[3 * r + 1], B[3 + c], A[3 * r + 2] * B[6 + c]));
}

// --- a body's constant rotation R -------------------------------------------
// Compile-time forms of the dh flag below. A loop over bodies whose forms are
// only known at run time writes its body as a generic lambda and runs it
// through with_dh: one specialised copy per form behind one uniform branch,
// instead of a branch in every transform.
struct DhOn {
  FD constexpr operator bool() const { return true; }
};
struct DhOff {
  FD constexpr operator bool() const { return false; }
};
template <class F>
FD void with_dh(bool dh, const F& f) {
  if (dh) f(DhOn{});
  else f(DhOff{});
}
// f(k, dh) over the len bodies of a segment, outward (k = 0, 1, ...) or
// inward: the first body (k = 0) with the frame form its flag dh0 gives,
// every later one sparse (a segment body after the first is its parent's
// only child), so the rolled loop holds one copy of its body and no branch.
template <class F>
FD void seg_outward(int len, bool dh0, const F& f) {
  with_dh(dh0, [&](auto dh) { f(0, dh); });
#pragma unroll 1
  for (int k = 1; k < len; ++k) f(k, DhOn{});
}
template <class F>
FD void seg_inward(int len, bool dh0, const F& f) {
#pragma unroll 1
  for (int k = len - 1; k >= 1; --k) f(k, DhOn{});
  with_dh(dh0, [&](auto dh) { f(0, dh); });
}
// With dh (the caller knows R = Rot_x(alpha), see BodyImage) the sparse form,
// else the general one; callers pass a value the compiler can fold (a loop
// index after unrolling), so each call site keeps one form.
FD V3 rot_b(const BodyImage& b, V3 a, bool dh = false) {  // R a
  if (dh) return mk(a.x, fmaf(b.ca, a.y, -b.sa * a.z), fmaf(b.sa, a.y, b.ca * a.z));
  return rot(b.R, a);
}
FD V3 rotT_b(const BodyImage& b, V3 a, bool dh = false) {  // R^T a
  if (dh) return mk(a.x, fmaf(b.ca, a.y, b.sa * a.z), fmaf(-b.sa, a.y, b.ca * a.z));
  return rotT(b.R, a);
}
// C = E R (E row-major)
FD void mat_mul_b(const float* E, const BodyImage& b, float* C, bool dh = false) {
  if (dh) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float y = E[3 * r + 1], z = E[3 * r + 2];
      C[3 * r] = E[3 * r];
      C[3 * r + 1] = fmaf(b.ca, y, b.sa * z);
      C[3 * r + 2] = fmaf(-b.sa, y, b.ca * z);
    }
    return;
  }
  mat_mul(E, b.R, C);
}

// C = E R^T (E row-major): the inverse of mat_mul_b's step
FD void mat_mul_bT(const float* E, const BodyImage& b, float* C, bool dh = false) {
  if (dh) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float y = E[3 * r + 1], z = E[3 * r + 2];
      C[3 * r] = E[3 * r];
      C[3 * r + 1] = fmaf(b.ca, y, -b.sa * z);
      C[3 * r + 2] = fmaf(b.sa, y, b.ca * z);
    }
    return;
  }
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      C[3 * r + c] = fmaf(E[3 * r], b.R[3 * c], fmaf(E[3 * r + 1], b.R[3 * c + 1], E[3 * r + 2] * b.R[3 * c + 2]));
}

// --- joint transforms (internal frames) -------------------------------------
// A revolute body i sits at ^parent'T_i' = (R Rot_z(q + th0), p) with R, p
// constant; (c, s) below are cos and sin of q + th0.
// Motion vectors: parent' -> child' coordinates.
FD SV mot_in(const BodyImage& b, float c, float s, const SV& m, bool dh = false) {
  V3 p = mk(b.p[0], b.p[1], b.p[2]);
  return SV{rotzT(c, s, rotT_b(b, m.w, dh)), rotzT(c, s, rotT_b(b, cross_sub(m.v, p, m.w), dh))};
}
// Force vectors: child' -> parent' coordinates (the transpose of mot_in).
FD SV frc_out(const BodyImage& b, float c, float s, const SV& f, bool dh = false) {
  V3 p = mk(b.p[0], b.p[1], b.p[2]);
  V3 fl = rot_b(b, rotz(c, s, f.v), dh);
  return SV{cross_add(rot_b(b, rotz(c, s, f.w), dh), p, fl), fl};
}
// Motion vectors child' -> parent' (inverse of mot_in); used by adjoints.
FD SV mot_out(const BodyImage& b, float c, float s, const SV& m, bool dh = false) {
  V3 p = mk(b.p[0], b.p[1], b.p[2]);
  V3 w = rot_b(b, rotz(c, s, m.w), dh);
  return SV{w, cross_add(rot_b(b, rotz(c, s, m.v), dh), p, w)};
}

// e x m and e x* f for e = [z; 0] (the revolute motion subspace)
FD SV ez_crm(const SV& m) { return SV{mk(-m.w.y, m.w.x, 0.f), mk(-m.v.y, m.v.x, 0.f)}; }
FD SV ez_crf(const SV& f) { return SV{mk(-f.w.y, f.w.x, 0.f), mk(-f.v.y, f.v.x, 0.f)}; }

// --- compact rigid-body inertia (m, h = m c, I about the origin) -------------
struct RBI {
  float m;
  V3 h;
  float xx, yy, zz, xy, xz, yz;
};
FD RBI rbi_of(const BodyImage& b) {
  return RBI{b.m, mk(b.h[0], b.h[1], b.h[2]), b.I[0], b.I[1], b.I[2], b.I[3], b.I[4], b.I[5]};
}
FD V3 symv(float xx, float yy, float zz, float xy, float xz, float yz, V3 a) {
  return mk(fmaf(xx, a.x, fmaf(xy, a.y, xz * a.z)), fmaf(xy, a.x, fmaf(yy, a.y, yz * a.z)),
            fmaf(xz, a.x, fmaf(yz, a.y, zz * a.z)));
}
// [I_o w + h x v_lin; m v_lin - h x w], each component one FMA chain
FD SV rbi_mul(const RBI& I, const SV& v) {
  const V3 hv = cross(I.h, v.v);
  const V3 n = mk(fmaf(I.xx, v.w.x, fmaf(I.xy, v.w.y, fmaf(I.xz, v.w.z, hv.x))),
                  fmaf(I.xy, v.w.x, fmaf(I.yy, v.w.y, fmaf(I.yz, v.w.z, hv.y))),
                  fmaf(I.xz, v.w.x, fmaf(I.yz, v.w.y, fmaf(I.zz, v.w.z, hv.z))));
  const V3 f = mk(fmaf(I.m, v.v.x, fmaf(I.h.z, v.w.y, -I.h.y * v.w.z)),
                  fmaf(I.m, v.v.y, fmaf(I.h.x, v.w.z, -I.h.z * v.w.x)),
                  fmaf(I.m, v.v.z, fmaf(I.h.y, v.w.x, -I.h.x * v.w.y)));
  return SV{n, f};
}
// acc + I v and acc - I v, accumulated in place
FD SV rbi_mul_add(const SV& acc, const RBI& I, const SV& v) {
  const V3 n0 = cross_add(acc.w, I.h, v.v);
  const V3 n = mk(fmaf(I.xx, v.w.x, fmaf(I.xy, v.w.y, fmaf(I.xz, v.w.z, n0.x))),
                  fmaf(I.xy, v.w.x, fmaf(I.yy, v.w.y, fmaf(I.yz, v.w.z, n0.y))),
                  fmaf(I.xz, v.w.x, fmaf(I.yz, v.w.y, fmaf(I.zz, v.w.z, n0.z))));
  const V3 f0 = cross_sub(acc.v, I.h, v.w);
  return SV{n, mk(fmaf(I.m, v.v.x, f0.x), fmaf(I.m, v.v.y, f0.y), fmaf(I.m, v.v.z, f0.z))};
}
FD SV rbi_mul_sub(const SV& acc, const RBI& I, const SV& v) {
  const V3 n0 = cross_sub(acc.w, I.h, v.v);
  const V3 n = mk(fmaf(-I.xx, v.w.x, fmaf(-I.xy, v.w.y, fmaf(-I.xz, v.w.z, n0.x))),
                  fmaf(-I.xy, v.w.x, fmaf(-I.yy, v.w.y, fmaf(-I.yz, v.w.z, n0.y))),
                  fmaf(-I.xz, v.w.x, fmaf(-I.yz, v.w.y, fmaf(-I.zz, v.w.z, n0.z))));
  const V3 f0 = cross_add(acc.v, I.h, v.w);
  return SV{n, mk(fmaf(-I.m, v.v.x, f0.x), fmaf(-I.m, v.v.y, f0.y), fmaf(-I.m, v.v.z, f0.z))};
}
FD RBI rbi_add(const RBI& a, const RBI& b) {
  return RBI{a.m + b.m, a.h + b.h, a.xx + b.xx, a.yy + b.yy, a.zz + b.zz,
             a.xy + b.xy, a.xz + b.xz, a.yz + b.yz};
}

// symmetric S (6 entries) -> Rot_z S Rot_z^T
FD void sym_rotz(float c, float s, float* S) {
  float xx = S[0], yy = S[1], xy = S[3], xz = S[4], yz = S[5];
  float cc = c * c, ss = s * s, cs = c * s;
  S[0] = fmaf(cc, xx, fmaf(-2.f * cs, xy, ss * yy));
  S[1] = fmaf(ss, xx, fmaf(2.f * cs, xy, cc * yy));
  S[3] = fmaf(cs, xx - yy, (cc - ss) * xy);
  S[4] = fmaf(c, xz, -s * yz);
  S[5] = fmaf(s, xz, c * yz);
}
// symmetric S (xx yy zz xy xz yz) -> R S R^T, R row-major
template <class RT>
FD void sym_rot(const RT* R, float* S) {
  float T[9];  // T = S R^T
  float Sf[9] = {S[0], S[3], S[4], S[3], S[1], S[5], S[4], S[5], S[2]};
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      T[3 * i + j] = fmaf(Sf[3 * i], R[3 * j], fmaf(Sf[3 * i + 1], R[3 * j + 1], Sf[3 * i + 2] * R[3 * j + 2]));
  auto o = [&](int i, int j) {
    return fmaf(R[3 * i], T[j], fmaf(R[3 * i + 1], T[3 + j], R[3 * i + 2] * T[6 + j]));
  };
  S[0] = o(0, 0); S[1] = o(1, 1); S[2] = o(2, 2); S[3] = o(0, 1); S[4] = o(0, 2); S[5] = o(1, 2);
}
// general M (row-major 9) -> R M R^T
template <class RT>
FD void gen_rot(const RT* R, float* M) {
  float T[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      T[3 * i + j] = fmaf(M[3 * i], R[3 * j], fmaf(M[3 * i + 1], R[3 * j + 1], M[3 * i + 2] * R[3 * j + 2]));
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      M[3 * i + j] = fmaf(R[3 * i], T[j], fmaf(R[3 * i + 1], T[3 + j], R[3 * i + 2] * T[6 + j]));
}
// general M -> Rot_z M Rot_z^T
FD void gen_rotz(float c, float s, float* M) {
  // rows: A = Rot_z M
  float a0 = fmaf(c, M[0], -s * M[3]), a1 = fmaf(c, M[1], -s * M[4]), a2 = fmaf(c, M[2], -s * M[5]);
  float b0 = fmaf(s, M[0], c * M[3]), b1 = fmaf(s, M[1], c * M[4]), b2 = fmaf(s, M[2], c * M[5]);
  float d0 = M[6], d1 = M[7], d2 = M[8];
  // columns: A Rot_z^T
  M[0] = fmaf(c, a0, -s * a1); M[1] = fmaf(s, a0, c * a1); M[2] = a2;
  M[3] = fmaf(c, b0, -s * b1); M[4] = fmaf(s, b0, c * b1); M[5] = b2;
  M[6] = fmaf(c, d0, -s * d1); M[7] = fmaf(s, d0, c * d1); M[8] = d2;
}

// symmetric S -> Rot_x S Rot_x^T
FD void sym_rotx(float c, float s, float* S) {
  float yy = S[1], zz = S[2], xy = S[3], xz = S[4], yz = S[5];
  float cc = c * c, ss = s * s, cs = c * s;
  S[1] = fmaf(cc, yy, fmaf(-2.f * cs, yz, ss * zz));
  S[2] = fmaf(ss, yy, fmaf(2.f * cs, yz, cc * zz));
  S[5] = fmaf(cs, yy - zz, (cc - ss) * yz);
  S[3] = fmaf(c, xy, -s * xz);
  S[4] = fmaf(s, xy, c * xz);
}
// general M -> Rot_x M Rot_x^T
FD void gen_rotx(float c, float s, float* M) {
  // rows: A = Rot_x M
  float a0 = M[0], a1 = M[1], a2 = M[2];
  float b0 = fmaf(c, M[3], -s * M[6]), b1 = fmaf(c, M[4], -s * M[7]), b2 = fmaf(c, M[5], -s * M[8]);
  float d0 = fmaf(s, M[3], c * M[6]), d1 = fmaf(s, M[4], c * M[7]), d2 = fmaf(s, M[5], c * M[8]);
  // columns: A Rot_x^T
  M[0] = a0; M[1] = fmaf(c, a1, -s * a2); M[2] = fmaf(s, a1, c * a2);
  M[3] = b0; M[4] = fmaf(c, b1, -s * b2); M[5] = fmaf(s, b1, c * b2);
  M[6] = d0; M[7] = fmaf(c, d1, -s * d2); M[8] = fmaf(s, d1, c * d2);
}
// S -> R S R^T and R^T S R, M -> R M R^T and R^T M R with a body's R
FD void sym_rot_b(const BodyImage& b, float* S, bool dh = false) {
  if (dh) sym_rotx(b.ca, b.sa, S);
  else sym_rot(b.R, S);
}
FD void sym_rotT_b(const BodyImage& b, float* S, bool dh = false) {
  if (dh) {
    sym_rotx(b.ca, -b.sa, S);
  } else {
    const float Rt[9] = {b.R[0], b.R[3], b.R[6], b.R[1], b.R[4], b.R[7], b.R[2], b.R[5], b.R[8]};
    sym_rot(Rt, S);
  }
}
FD void gen_rot_b(const BodyImage& b, float* M, bool dh = false) {
  if (dh) gen_rotx(b.ca, b.sa, M);
  else gen_rot(b.R, M);
}
FD void gen_rotT_b(const BodyImage& b, float* M, bool dh = false) {
  if (dh) {
    gen_rotx(b.ca, -b.sa, M);
  } else {
    const float Rt[9] = {b.R[0], b.R[3], b.R[6], b.R[1], b.R[4], b.R[7], b.R[2], b.R[5], b.R[8]};
    gen_rot(Rt, M);
  }
}

// Composite inertia of body i (child' coords) carried to parent' coords:
// X^T I X for ^child X_parent = the revolute joint transform.
FD RBI rbi_out(const BodyImage& b, float c, float s, const RBI& I, bool dh = false) {
  float S[6] = {I.xx, I.yy, I.zz, I.xy, I.xz, I.yz};
  sym_rotz(c, s, S);
  sym_rot_b(b, S, dh);
  V3 hr = rot_b(b, rotz(c, s, I.h), dh);
  V3 p = mk(b.p[0], b.p[1], b.p[2]);
  V3 hn = hr + I.m * p;
  float sh = dot(p, hn + hr);
  // I' = I_r + (p.(h'+h_r)) 1 - (p h'^T + h_r p^T)
  RBI o;
  o.m = I.m;
  o.h = hn;
  o.xx = S[0] + sh - (p.x * hn.x + hr.x * p.x);
  o.yy = S[1] + sh - (p.y * hn.y + hr.y * p.y);
  o.zz = S[2] + sh - (p.z * hn.z + hr.z * p.z);
  o.xy = S[3] - (p.x * hn.y + hr.x * p.y);
  o.xz = S[4] - (p.x * hn.z + hr.x * p.z);
  o.yz = S[5] - (p.y * hn.z + hr.y * p.z);
  return o;
}

// --- articulated inertia: symmetric 6x6 [[A, B], [B^T, C]] -------------------
struct AI {
  float A[6];  // xx yy zz xy xz yz
  float B[9];  // row-major
  float C[6];  // xx yy zz xy xz yz
};
FD AI ai_of(const RBI& I) {
  AI o;
  o.A[0] = I.xx; o.A[1] = I.yy; o.A[2] = I.zz; o.A[3] = I.xy; o.A[4] = I.xz; o.A[5] = I.yz;
  // B = [h]x
  o.B[0] = 0.f;    o.B[1] = -I.h.z; o.B[2] = I.h.y;
  o.B[3] = I.h.z;  o.B[4] = 0.f;    o.B[5] = -I.h.x;
  o.B[6] = -I.h.y; o.B[7] = I.h.x;  o.B[8] = 0.f;
  o.C[0] = I.m; o.C[1] = I.m; o.C[2] = I.m; o.C[3] = 0.f; o.C[4] = 0.f; o.C[5] = 0.f;
  return o;
}
FD SV ai_mul(const AI& I, const SV& v) {
  V3 n = symv(I.A[0], I.A[1], I.A[2], I.A[3], I.A[4], I.A[5], v.w) + rot(I.B, v.v);
  V3 f = rotT(I.B, v.w) + symv(I.C[0], I.C[1], I.C[2], I.C[3], I.C[4], I.C[5], v.v);
  return SV{n, f};
}
FD void ai_add(AI& a, const AI& b) {
#pragma unroll
  for (int k = 0; k < 6; ++k) { a.A[k] += b.A[k]; a.C[k] += b.C[k]; }
#pragma unroll
  for (int k = 0; k < 9; ++k) a.B[k] += b.B[k];
}
// column z of the angular part: I e_z = [A[:,2]; B[2,:]^T]
FD SV ai_col_z(const AI& I) { return SV{mk(I.A[4], I.A[5], I.A[2]), mk(I.B[6], I.B[7], I.B[8])}; }
// Shift of a symmetric force-space tensor to a frame whose origin sits at
// -p: C' = C, B' = B + P C, A' = A - (Y P + (Y P)^T), P = [p]x, Y = B + P C / 2.
FD void ai_shift(const V3& p, AI& I) {
  float Cf[9] = {I.C[0], I.C[3], I.C[4], I.C[3], I.C[1], I.C[5], I.C[4], I.C[5], I.C[2]};
  float W[9];  // P C: column j = p x C[:, j]
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    V3 col = cross(p, mk(Cf[j], Cf[3 + j], Cf[6 + j]));
    W[j] = col.x; W[3 + j] = col.y; W[6 + j] = col.z;
  }
  float Y[9], Z[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) { Y[k] = fmaf(0.5f, W[k], I.B[k]); I.B[k] += W[k]; }
  // Z = Y P: row i = Y[i,:] x p
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    V3 r = cross(mk(Y[3 * i], Y[3 * i + 1], Y[3 * i + 2]), p);
    Z[3 * i] = r.x; Z[3 * i + 1] = r.y; Z[3 * i + 2] = r.z;
  }
  I.A[0] -= 2.f * Z[0]; I.A[1] -= 2.f * Z[4]; I.A[2] -= 2.f * Z[8];
  I.A[3] -= Z[1] + Z[3]; I.A[4] -= Z[2] + Z[6]; I.A[5] -= Z[5] + Z[7];
}
// X^T I X for the revolute joint transform (child' -> parent'): rotate all
// blocks by E = R Rot_z(q), then shift by the joint origin p.
FD void ai_out(const BodyImage& b, float c, float s, AI& I, bool dh = false) {
  sym_rotz(c, s, I.A); sym_rot_b(b, I.A, dh);
  sym_rotz(c, s, I.C); sym_rot_b(b, I.C, dh);
  gen_rotz(c, s, I.B); gen_rot_b(b, I.B, dh);
  ai_shift(mk(b.p[0], b.p[1], b.p[2]), I);
}
// The inverse congruence, parent' -> child': shift by -p, then rotate all
// blocks by E^T.
FD void ai_in(const BodyImage& b, float c, float s, AI& I, bool dh = false) {
  ai_shift(mk(-b.p[0], -b.p[1], -b.p[2]), I);
  sym_rotT_b(b, I.A, dh); sym_rotz(c, -s, I.A);
  sym_rotT_b(b, I.C, dh); sym_rotz(c, -s, I.C);
  gen_rotT_b(b, I.B, dh); gen_rotz(c, -s, I.B);
}

// --- the projected articulated inertia Ia = I^A - U U^T / D ------------------
// With U = I^A e_z and D = U_z, Ia e_z = U - U = 0: the z row and column of A
// and the z row of B vanish, leaving 15 free entries. The _z forms below set
// those entries to zero and skip their arithmetic in the projection, in the
// product with a velocity product v x e_z qd (whose z components vanish too)
// and in the congruence to the parent's coordinates.

// I -= d u^T with d = U / D (so d_z = 1), leaving the zeros exact
FD void ai_rank1_sub_d_z(AI& I, const SV& d, const SV& u) {
  const float a[6] = {u.w.x, u.w.y, u.w.z, u.v.x, u.v.y, u.v.z};
  const float e[6] = {d.w.x, d.w.y, d.w.z, d.v.x, d.v.y, d.v.z};
  I.A[0] = fmaf(-e[0], a[0], I.A[0]);
  I.A[1] = fmaf(-e[1], a[1], I.A[1]);
  I.A[3] = fmaf(-e[0], a[1], I.A[3]);
  I.A[2] = 0.f; I.A[4] = 0.f; I.A[5] = 0.f;
  const int si[6] = {0, 1, 2, 0, 0, 1}, sj[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
  for (int t = 0; t < 6; ++t) I.C[t] = fmaf(-e[3 + si[t]], a[3 + sj[t]], I.C[t]);
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) I.B[3 * r + c] = fmaf(-e[r], a[3 + c], I.B[3 * r + c]);
  I.B[6] = 0.f; I.B[7] = 0.f; I.B[8] = 0.f;
}
// I -= k u u^T with k = 1 / u_z, leaving the zeros exact
FD void ai_rank1_sub_z(AI& I, const SV& u, float k) {
  SV d = k * u;
  d.w.z = 1.f;
  ai_rank1_sub_d_z(I, d, u);
}
// acc + Ia m for m with m.w.z = m.v.z = 0 (a velocity product v x e_z qd)
FD SV ai_mul_z_add(const SV& acc, const AI& I, const SV& m) {
  const float wx = m.w.x, wy = m.w.y, vx = m.v.x, vy = m.v.y;
  const V3 n = mk(fmaf(I.A[0], wx, fmaf(I.A[3], wy, fmaf(I.B[0], vx, fmaf(I.B[1], vy, acc.w.x)))),
                  fmaf(I.A[3], wx, fmaf(I.A[1], wy, fmaf(I.B[3], vx, fmaf(I.B[4], vy, acc.w.y)))), acc.w.z);
  const V3 f = mk(fmaf(I.B[0], wx, fmaf(I.B[3], wy, fmaf(I.C[0], vx, fmaf(I.C[3], vy, acc.v.x)))),
                  fmaf(I.B[1], wx, fmaf(I.B[4], wy, fmaf(I.C[3], vx, fmaf(I.C[1], vy, acc.v.y)))),
                  fmaf(I.B[2], wx, fmaf(I.B[5], wy, fmaf(I.C[4], vx, fmaf(I.C[5], vy, acc.v.z)))));
  return SV{n, f};
}
// ai_out (below) for Ia: the rotation by Rot_z(q) keeps the zeros, a Rot_x
// rotation (dh) fills them from the non-zero entries alone
FD void ai_out_z(const BodyImage& b, float c, float s, AI& I, bool dh = false) {
  {  // A: only xx, yy, xy are non-zero
    const float xx = I.A[0], yy = I.A[1], xy = I.A[3];
    const float cc = c * c, ss = s * s, cs = c * s;
    I.A[0] = fmaf(cc, xx, fmaf(-2.f * cs, xy, ss * yy));
    I.A[1] = fmaf(ss, xx, fmaf(2.f * cs, xy, cc * yy));
    I.A[3] = fmaf(cs, xx - yy, (cc - ss) * xy);
  }
  sym_rotz(c, s, I.C);
  {  // B: row z is zero
    const float a0 = fmaf(c, I.B[0], -s * I.B[3]), a1 = fmaf(c, I.B[1], -s * I.B[4]);
    const float a2 = fmaf(c, I.B[2], -s * I.B[5]);
    const float b0 = fmaf(s, I.B[0], c * I.B[3]), b1 = fmaf(s, I.B[1], c * I.B[4]);
    const float b2 = fmaf(s, I.B[2], c * I.B[5]);
    I.B[0] = fmaf(c, a0, -s * a1); I.B[1] = fmaf(s, a0, c * a1); I.B[2] = a2;
    I.B[3] = fmaf(c, b0, -s * b1); I.B[4] = fmaf(s, b0, c * b1); I.B[5] = b2;
  }
  if (dh) {
    const float ca = b.ca, sa = b.sa;
    {  // A: Rot_x with zz = xz = yz = 0
      const float yy = I.A[1], xy = I.A[3];
      I.A[1] = (ca * ca) * yy;
      I.A[2] = (sa * sa) * yy;
      I.A[5] = (ca * sa) * yy;
      I.A[3] = ca * xy;
      I.A[4] = sa * xy;
    }
    sym_rotx(ca, sa, I.C);
    {  // B: Rot_x B Rot_x^T with row z zero
      const float m0 = I.B[0], m1 = I.B[1], m2 = I.B[2], m3 = I.B[3], m4 = I.B[4], m5 = I.B[5];
      const float t1 = fmaf(ca, m4, -sa * m5), t2 = fmaf(sa, m4, ca * m5);
      I.B[0] = m0; I.B[1] = fmaf(ca, m1, -sa * m2); I.B[2] = fmaf(sa, m1, ca * m2);
      I.B[3] = ca * m3; I.B[4] = ca * t1; I.B[5] = ca * t2;
      I.B[6] = sa * m3; I.B[7] = sa * t1; I.B[8] = sa * t2;
    }
  } else {
    sym_rot(b.R, I.A);
    sym_rot(b.R, I.C);
    gen_rot(b.R, I.B);
  }
  ai_shift(mk(b.p[0], b.p[1], b.p[2]), I);
}

}  // namespace frax
