// Operational-space control of one task frame, one thread per instance:
//
//   tau = J^T Lambda (xdd_des - Jdot qd) + c + g,   Lambda = (J M^-1 J^T)^-1
//
// the inverse-dynamics controller the paper times (Sec. V, Table II), with
// J the world-aligned Jacobian of the task body's origin. Nothing of M is
// formed. The inverse operational-space inertia in task-body coordinates,
// Omega = Lambda^-1 (the map from a spatial force applied at the task body to
// its spatial acceleration, at rest), follows from the articulated-body
// inertias along the path Anc(k) from the root to the task body k
// (Featherstone's recursion for the apparent inverse inertia):
//
//   Omega_i = P_i (X_i Omega_p X_i^T) P_i^T + S_i D_i^-1 S_i^T,
//   P_i = 1 - S_i U_i^T / D_i,   U_i = I^A_i S_i,   D_i = S_i^T U_i,
//
// starting from Omega = 0 above a fixed base, or from (I^A_0)^-1 for a
// free-flyer root. Sweeps: (1) articulated inertias over the whole tree,
// keeping U_i, 1/D_i of the path bodies; (2) outward along the path: Omega,
// the velocity-product acceleration Jdot qd and the task body's world
// rotation; (3) a 6x6 solve for the task wrench f = Lambda r in body
// coordinates; (4) RNEA at q, qd, qdd = 0 with f added to the task body's
// force, which yields c + g + J^T f in one inward pass.
//
// A motion-space tensor such as Omega transforms as X Omega X^T. With its
// angular and linear halves swapped it transforms like a force-space
// tensor under the inverse transform, so it is stored as an AI whose A
// block is the linear-linear part, C the angular-angular part and B[r][c]
// the (linear r, angular c) part, and moved outward with ai_in.
#pragma once
#include "seg.cuh"

namespace frax {

// Dense [[A, B], [B^T, C]] of a symmetric 6x6 tensor.
FD void ai_dense(const AI& I, float A[6][6]) {
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
}

// Inverse of a symmetric positive definite 6x6 matrix by Cholesky
// (A = G G^T, A^-1 = G^-T G^-1), dense, in place.
FD void spd6_invert(float A[6][6]) {
  float G[6][6], dinv[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    float d = A[j][j];
#pragma unroll
    for (int k = 0; k < j; ++k) d = fmaf(-G[j][k], G[j][k], d);
    dinv[j] = rsqrtf(d);
#pragma unroll
    for (int i = j + 1; i < 6; ++i) {
      float x = A[i][j];
#pragma unroll
      for (int k = 0; k < j; ++k) x = fmaf(-G[i][k], G[j][k], x);
      G[i][j] = x * dinv[j];
    }
  }
  // H = G^-1 (lower triangular)
  float H[6][6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    H[j][j] = dinv[j];
#pragma unroll
    for (int i = j + 1; i < 6; ++i) {
      float x = 0.f;
#pragma unroll
      for (int k = j; k < i; ++k) x = fmaf(-G[i][k], H[k][j], x);
      H[i][j] = x * dinv[i];
    }
  }
  // A^-1 = H^T H
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      float x = 0.f;
#pragma unroll
      for (int k = i; k < 6; ++k) x = fmaf(H[k][i], H[k][j], x);
      A[i][j] = x;
      A[j][i] = x;
    }
}

// Per path body: U (6 floats) and 1/D, in thread-local memory by body.
template <int NB>
struct PathLocal {
  float v[NB * 7];
  FD float& at(int i, int f) { return v[i * 7 + f]; }
};

// Sweep 1: articulated-body inertias at zero velocity over the whole tree
// (the same inward recursion as the factor of crba_seg). Keeps U_i, 1/D_i of
// the bodies in `path`; returns a free-flyer root's articulated inertia.
template <class T, class Img, class C, class PL>
FD AI osc_inertias(const Img& M, const float* __restrict__ q, uint64_t path, PL& P, const C& col) {
  constexpr int NB = T::NBMAX;
  AI IAa[NB];
  AI azero;
#pragma unroll
  for (int k = 0; k < 6; ++k) { azero.A[k] = 0.f; azero.C[k] = 0.f; }
#pragma unroll
  for (int k = 0; k < 9; ++k) azero.B[k] = 0.f;
  AI IA0 = azero;
#pragma unroll 1
  for (int t = 0; t < M.n_act; ++t) {
    const int act = M.act[t];
    const int s = act & 63, kind = act >> 6;
    const int st = M.seg_start[s], len = M.seg_len[s];
    if (T::kFree && s == 0) {
      if (kind != kActClose) IAa[0] = azero;
      if (kind == kActOpen) continue;
      IA0 = ai_of(rbi_of(M.body[0]));
      ai_add(IA0, IAa[0]);
      continue;
    }
    const int last = M.order[st + len - 1];
    if (kind == kActOpen) {
      IAa[last] = azero;
      continue;
    }
    AI IA = ai_of(rbi_of(M.body[last]));
    if (kind == kActClose) ai_add(IA, IAa[last]);
#pragma unroll 1
    for (int k = len - 1; k >= 0; --k) {
      const int i = M.order[st + k];
      const BodyImage& b = M.body[i];
      float sn, cs;
      joint_sincos(col.in(q, iq_of<T>(i)) + b.th0, &sn, &cs);
      const SV U = ai_col_z(IA);
      const float dinv = rcp(U.w.z);
      if ((path >> i) & 1ull) {
        P.at(i, 0) = U.w.x; P.at(i, 1) = U.w.y; P.at(i, 2) = U.w.z;
        P.at(i, 3) = U.v.x; P.at(i, 4) = U.v.y; P.at(i, 5) = U.v.z;
        P.at(i, 6) = dinv;
      }
      ai_rank1_sub_z(IA, U, dinv);
      with_dh(b.dh, [&](auto dh) { ai_out_z(b, cs, sn, IA, dh); });
      if (k > 0) {
        AI Ip = ai_of(rbi_of(M.body[M.order[st + k - 1]]));
        ai_add(Ip, IA);
        IA = Ip;
      }
    }
    const int p = M.seg_parent[s];
    if (p >= 0) ai_add(IAa[p], IA);
  }
  return IA0;
}

struct OscPath {
  AI Om;     // Omega of the task body, halves swapped (see above)
  SV v, a;   // task body velocity and its acceleration at qdd = 0, no gravity
  float E[9];  // world rotation of the task body's (internal) frame
};

// One step of sweep 2 through revolute body b (cos, sin of its joint), with
// u = U / D of its articulated inertia: Omega, v, the velocity-product
// acceleration and the world rotation of the path so far.
template <class DH>
FD void osc_path_step(const BodyImage& b, float cs, float sn, float qdj, const SV& U, float dinv, OscPath& o,
                      DH dh) {
  ai_in(b, cs, sn, o.Om, dh);
  const SV u = dinv * U;
  const SV y = ai_mul(o.Om, SV{u.v, u.w});  // W u as [linear; angular]
  const float uWu = dot(u.w, y.v) + dot(u.v, y.w);
  o.Om.B[2] -= y.w.x;
  o.Om.B[5] -= y.w.y;
  o.Om.B[8] -= y.w.z;
  o.Om.C[4] -= y.v.x;
  o.Om.C[5] -= y.v.y;
  o.Om.C[2] += fmaf(-2.f, y.v.z, uWu + dinv);
  o.v = mot_in(b, cs, sn, o.v, dh);
  o.v.w.z += qdj;
  o.a = mot_in(b, cs, sn, o.a, dh) + ez_velprod(o.v, qdj);
  float ER[9];
  mat_mul_b(o.E, b, ER, dh);
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float x = ER[3 * r], z = ER[3 * r + 1];
    o.E[3 * r] = fmaf(cs, x, sn * z);
    o.E[3 * r + 1] = fmaf(-sn, x, cs * z);
    o.E[3 * r + 2] = ER[3 * r + 2];
  }
}

// Sweep 2: outward along the path to the task body.
template <class T, class Img, class C, class PL>
FD OscPath osc_path(const Img& M, const float* __restrict__ q, const float* __restrict__ qd, uint64_t path,
                    const AI& IA0, PL& P, const C& col) {
  OscPath o;
#pragma unroll
  for (int k = 0; k < 6; ++k) { o.Om.A[k] = 0.f; o.Om.C[k] = 0.f; }
#pragma unroll
  for (int k = 0; k < 9; ++k) { o.Om.B[k] = 0.f; o.E[k] = (k % 4 == 0) ? 1.f : 0.f; }
  o.v = szero();
  o.a = szero();
  uint64_t rest = path;
  if (T::kFree) {  // the root is on every path
    float A[6][6];
    ai_dense(IA0, A);
    spd6_invert(A);
    // swap halves: A block <- linear-linear, C <- angular-angular
    o.Om.A[0] = A[3][3]; o.Om.A[1] = A[4][4]; o.Om.A[2] = A[5][5];
    o.Om.A[3] = A[3][4]; o.Om.A[4] = A[3][5]; o.Om.A[5] = A[4][5];
    o.Om.C[0] = A[0][0]; o.Om.C[1] = A[1][1]; o.Om.C[2] = A[2][2];
    o.Om.C[3] = A[0][1]; o.Om.C[4] = A[0][2]; o.Om.C[5] = A[1][2];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) o.Om.B[3 * r + c] = A[3 + r][c];
    o.v = load6(qd, 0, col);
    const RootPose RP = root_pose(M, q, col);
#pragma unroll
    for (int k = 0; k < 9; ++k) o.E[k] = RP.E[k];
    rest &= ~1ull;
  }
#pragma unroll 1
  for (; rest; rest &= rest - 1) {
    const int j = low_bit(rest);
    const BodyImage& b = M.body[j];
    float sn, cs;
    joint_sincos(col.in(q, iq_of<T>(j)) + b.th0, &sn, &cs);
    const SV U{mk(P.at(j, 0), P.at(j, 1), P.at(j, 2)), mk(P.at(j, 3), P.at(j, 4), P.at(j, 5))};
    with_dh(b.dh, [&](auto dh) { osc_path_step(b, cs, sn, col.in(qd, iv_of<T>(j)), U, P.at(j, 6), o, dh); });
  }
  return o;
}

// Sweep 3: the task wrench f = Lambda r in task-body coordinates, with
// r = E^T xdd - Jdot qd, and (optionally) Lambda written world-aligned.
template <class C>
FD SV osc_task_wrench(const OscPath& o, const float* __restrict__ xdd, float* __restrict__ Lam, const C& col) {
  // r = E^T xdd - Jdot qd in body coordinates; Jdot qd = [a_w; a_v + w x v]
  const SV xw = load6(xdd, 0, col);
  const V3 rw = rotT(o.E, xw.w) - o.a.w;
  const V3 rv = rotT(o.E, xw.v) - (o.a.v + cross(o.v.w, o.v.v));
  // f = Omega^-1 r; in the swapped halves the solution is [f_lin; f_ang]
  const SV fs = spd6_solve(o.Om, SV{rv, rw});
  if (Lam) {
    float A[6][6];
    ai_dense(o.Om, A);
    spd6_invert(A);  // Lambda in body coordinates, halves swapped
    // world-aligned: each 3x3 block (unswapped) becomes E X E^T
#pragma unroll
    for (int bi = 0; bi < 2; ++bi)
#pragma unroll
      for (int bj = 0; bj < 2; ++bj) {
        const int si = 3 * (1 - bi), sj = 3 * (1 - bj);  // swapped offsets
        float X[9], T1[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int c = 0; c < 3; ++c) X[3 * r + c] = A[si + r][sj + c];
#pragma unroll
        for (int r = 0; r < 3; ++r)  // T1 = E X
#pragma unroll
          for (int c = 0; c < 3; ++c)
            T1[3 * r + c] = fmaf(o.E[3 * r], X[c], fmaf(o.E[3 * r + 1], X[3 + c], o.E[3 * r + 2] * X[6 + c]));
#pragma unroll
        for (int r = 0; r < 3; ++r)  // T1 E^T
#pragma unroll
          for (int c = 0; c < 3; ++c)
            col.out(Lam, (3 * bi + r) * 6 + 3 * bj + c,
                    fmaf(T1[3 * r], o.E[3 * c], fmaf(T1[3 * r + 1], o.E[3 * c + 1], T1[3 * r + 2] * o.E[3 * c + 2])));
      }
  }
  return SV{fs.v, fs.w};
}

// Whole controller for one instance. xdd: task acceleration [omega_dot;
// p_ddot] of the task body's origin in world coordinates (6 rows); tau: nv
// rows; Lam (optional): 36 rows, Lambda row-major in world-aligned
// coordinates.
template <class T, class Img, class C>
FD void osc_seg(const Img& M, int task, const float* __restrict__ q, const float* __restrict__ qd,
                const float* __restrict__ xdd, float* __restrict__ tau, float* __restrict__ Lam, const C& col) {
  const uint64_t path = M.anc[task];
  PathLocal<T::NBMAX> P;
  const AI IA0 = osc_inertias<T>(M, q, path, P, col);
  const OscPath o = osc_path<T>(M, q, qd, path, IA0, P, col);
  const SV f = osc_task_wrench(o, xdd, Lam, col);
  rnea_seg<T, Img, C, true>(M, q, qd, nullptr, tau, col, task, f);
}

// The same controller on a fixed-base serial chain of N revolute bodies with
// every sweep unrolled: body indices, and with them each model constant's
// offset in the parameter image and each joint's frame form (Rot_x after
// the first body), are known at compile time, and the per-body state (joint
// cos/sin, U, 1/D, the RNEA sweep) lives in registers. The path to the task
// body is bodies 0 .. task.
template <int N, class Img, class C>
FD void osc_chain(const Img& M, int task, const float* __restrict__ q, const float* __restrict__ qd,
                  const float* __restrict__ xdd, float* __restrict__ tau, float* __restrict__ Lam, const C& col) {
  using T = ChainTopo<N>;
  float cs[N], sn[N];
#pragma unroll
  for (int k = 0; k < N; ++k) joint_sincos(col.in(q, k) + M.body[k].th0, &sn[k], &cs[k]);
  // sweep 1: articulated inertias at zero velocity, tip to base
  SV U[N];
  float dinv[N];
  AI IA;
#pragma unroll
  for (int k = N - 1; k >= 0; --k) {
    const BodyImage& b = M.body[k];
    AI Ik = ai_of(rbi_of(b));
    if (k < N - 1) ai_add(Ik, IA);
    IA = Ik;
    U[k] = ai_col_z(IA);
    dinv[k] = rcp(U[k].w.z);
    ai_rank1_sub_z(IA, U[k], dinv[k]);
    ai_out_z(b, cs[k], sn[k], IA, k > 0);
  }
  // sweep 2: outward along bodies 0 .. task
  OscPath o;
#pragma unroll
  for (int k = 0; k < 6; ++k) { o.Om.A[k] = 0.f; o.Om.C[k] = 0.f; }
#pragma unroll
  for (int k = 0; k < 9; ++k) { o.Om.B[k] = 0.f; o.E[k] = (k % 4 == 0) ? 1.f : 0.f; }
  o.v = szero();
  o.a = szero();
#pragma unroll
  for (int k = 0; k < N; ++k) {
    if (k > task) break;
    if (k > 0) osc_path_step(M.body[k], cs[k], sn[k], col.in(qd, k), U[k], dinv[k], o, DhOn{});
    else osc_path_step(M.body[k], cs[k], sn[k], col.in(qd, k), U[k], dinv[k], o, DhOff{});
  }
  // sweep 3: the task wrench
  const SV fext = osc_task_wrench(o, xdd, Lam, col);
  // sweep 4: RNEA at qdd = 0 with f added to the task body's force
  SV v = szero(), a = gravity_acc(M.g), F[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const BodyImage& b = M.body[k];
    const float qdk = col.in(qd, k);
    v = mot_in(b, cs[k], sn[k], v, k > 0);
    v.w.z += qdk;
    a = mot_in(b, cs[k], sn[k], a, k > 0) + ez_velprod(v, qdk);
    const RBI I = rbi_of(b);
    F[k] = crf_add(rbi_mul(I, a), v, rbi_mul(I, v));
    if (k == task) F[k] = F[k] + fext;
  }
  SV Fs = szero();
#pragma unroll
  for (int k = N - 1; k >= 0; --k) {
    Fs = Fs + F[k];
    col.out(tau, k, Fs.w.z);
    if (k > 0) Fs = frc_out(M.body[k], cs[k], sn[k], Fs, true);
  }
  (void)sizeof(T);
}

}  // namespace frax
