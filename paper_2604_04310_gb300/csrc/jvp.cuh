// Forward-mode derivatives (JVPs), one thread per instance: the directional
// derivatives jax.jvp gives on the dynamics (Sec. IV-A), written as tangent
// recursions beside the value recursions.
//
// With X_i(q_i) the motion transform parent' -> child' of a revolute joint,
// dX_i/dq_i = -(e_z x) X_i, so along a direction (dq, dqd, dqdd):
//   dv_i = X dv_p - dq_i e_z x (X v_p) + e_z dqd_i
//   da_i = X da_p - dq_i e_z x (X a_p) + e_z dqdd_i + dv_i x e_z qd_i + v_i x e_z dqd_i
//   df_i = I da_i + dv_i x* I v_i + v_i x* I dv_i
//   dF_p += X_i^T (dF_i + dq_i e_z x* F_i),   dtau_i = e_z . dF_i
// (a free-flyer root: dv_0 = dqd_0, da_0 = dqdd_0 + [0; -dtheta x E^T(-g)]).
// As in the adjoints, the inward sweep steps v, a, dv, da back through each
// joint instead of storing them per body.
#pragma once
#include "seg.cuh"

namespace frax {

// One step back through joint b: from the child's v, a, dv, da to the
// parent's, all recomputed rather than stored (X v_p = v - e_z qd, ...).
template <class DH>
FD void jvp_step_back(const BodyImage& b, float cs, float sn, float qdi, float qddi, float dqi, float dqdi,
                      float dqddi, SV& v, SV& a, SV& dv, SV& da, DH dh) {
  SV Xv = v;
  Xv.w.z -= qdi;
  SV Xa = a - ez_velprod(v, qdi);
  Xa.w.z -= qddi;
  SV Xdv = dv + dqi * ez_crm(Xv);
  Xdv.w.z -= dqdi;
  SV Xda = da - ez_velprod(dv, qdi) - ez_velprod(v, dqdi) + dqi * ez_crm(Xa);
  Xda.w.z -= dqddi;
  v = mot_out(b, cs, sn, Xv, dh);
  a = mot_out(b, cs, sn, Xa, dh);
  dv = mot_out(b, cs, sn, Xdv, dh);
  da = mot_out(b, cs, sn, Xda, dh);
}

template <class T, class Img, class C, class Sink>
FD void rnea_jvp_seg(const Img& M, const float* __restrict__ q, const float* __restrict__ qd,
                     const float* __restrict__ qdd, const float* __restrict__ dq, const float* __restrict__ dqd,
                     const float* __restrict__ dqdd, const Sink& sink, const C& col) {
  constexpr int NB = T::NBMAX;
  SV bv[NB], ba[NB], bdv[NB], bda[NB];  // tip state of bodies with child segments
  SV aF[NB], adF[NB];                    // forces handed back by child segments
  float sc[NB], ss[NB];
  const SV ag = gravity_acc(M.g);
  auto in0 = [&](const float* p, int k) { return p ? col.in(p, k) : 0.f; };
#pragma unroll 1
  for (int t = 0; t < M.n_act; ++t) {
    const int act = M.act[t];
    const int s = act & 63, kind = act >> 6;
    const int st = M.seg_start[s], len = M.seg_len[s];
    if (T::kFree && s == 0) {
      const RBI I = rbi_of(M.body[0]);
      if (kind != kActClose) {
        const RootPose P = root_pose(M, q, col);
        const V3 gam = rotT(P.E, ag.v);
        bv[0] = load6(qd, 0, col);
        bdv[0] = load6(dqd, 0, col);
        ba[0] = SV{mk(0, 0, 0), gam};
        if (qdd) ba[0] = ba[0] + load6(qdd, 0, col);
        bda[0] = SV{mk(0, 0, 0), -cross(mk(col.in(dq, 0), col.in(dq, 1), col.in(dq, 2)), gam)};
        if (dqdd) bda[0] = bda[0] + load6(dqdd, 0, col);
        aF[0] = adF[0] = szero();
        if (kind == kActOpen) continue;
      }
      const SV v = bv[0], dv = bdv[0];
      const SV Iv = rbi_mul(I, v);
      const SV F = crf_add(rbi_mul_add(aF[0], I, ba[0]), v, Iv);
      const SV dF = crf_add(crf_add(rbi_mul_add(adF[0], I, bda[0]), dv, Iv), v, rbi_mul(I, dv));
      sink.root(F, dF);
      continue;
    }
    const int last = M.order[st + len - 1];
    SV v, a, dv, da;
    if (kind != kActClose) {
      const int p = M.seg_parent[s];
      v = p < 0 ? szero() : bv[p];
      a = p < 0 ? ag : ba[p];
      dv = p < 0 ? szero() : bdv[p];
      da = p < 0 ? szero() : bda[p];
      seg_outward(len, M.body[M.order[st]].dh, [&](int k, auto dh) {
        const int i = M.order[st + k];
        const BodyImage& b = M.body[i];
        {
          float sn, cs;
          joint_sincos(col.in(q, iq_of<T>(i)) + b.th0, &sn, &cs);
          sc[i] = cs;
          ss[i] = sn;
          const int iv = iv_of<T>(i);
          const float qdi = col.in(qd, iv), dqi = col.in(dq, iv), dqdi = col.in(dqd, iv);
          const SV Xv = mot_in(b, cs, sn, v, dh);
          const SV Xa = mot_in(b, cs, sn, a, dh);
          dv = mot_in(b, cs, sn, dv, dh) - dqi * ez_crm(Xv);
          dv.w.z += dqdi;
          v = Xv;
          v.w.z += qdi;
          da = mot_in(b, cs, sn, da, dh) - dqi * ez_crm(Xa) + ez_velprod(dv, qdi) + ez_velprod(v, dqdi);
          da.w.z += in0(dqdd, iv);
          a = Xa + ez_velprod(v, qdi);
          a.w.z += in0(qdd, iv);
        }
      });
      if (kind == kActOpen) {
        bv[last] = v;
        ba[last] = a;
        bdv[last] = dv;
        bda[last] = da;
        aF[last] = adF[last] = szero();
        continue;
      }
    } else {
      v = bv[last];
      a = ba[last];
      dv = bdv[last];
      da = bda[last];
    }
    const bool closing = kind == kActClose;
    SV Fc = closing ? aF[last] : szero();
    SV dFc = closing ? adF[last] : szero();
    seg_inward(len, M.body[M.order[st]].dh, [&](int k, auto dh) {
      const int i = M.order[st + k];
      const BodyImage& b = M.body[i];
      {
        const RBI I = rbi_of(b);
        const float cs = sc[i], sn = ss[i];
        const int iv = iv_of<T>(i);
        const float qdi = col.in(qd, iv), dqi = col.in(dq, iv), dqdi = col.in(dqd, iv);
        const SV Iv = rbi_mul(I, v);
        const SV F = crf_add(rbi_mul_add(Fc, I, a), v, Iv);
        const SV dF = crf_add(crf_add(rbi_mul_add(dFc, I, da), dv, Iv), v, rbi_mul(I, dv));
        sink(i, F.w.z, dF.w.z);
        Fc = frc_out(b, cs, sn, F, dh);
        dFc = frc_out(b, cs, sn, dF + dqi * ez_crf(F), dh);
        if (k > 0) jvp_step_back(b, cs, sn, qdi, in0(qdd, iv), dqi, dqdi, in0(dqdd, iv), v, a, dv, da, dh);
      }
    });
    const int p = M.seg_parent[s];
    if (p >= 0) {
      aF[p] = aF[p] + Fc;
      adF[p] = adF[p] + dFc;
    }
  }
}

// The same tangent recursion for a fixed-base serial chain of N bodies with
// both sweeps unrolled (compile-time body index and frame form, k > 0), as
// rnea_vjp_chain does for the adjoint.
template <int N, class Img, class C, class Sink>
FD void rnea_jvp_chain(const Img& M, const float* __restrict__ q, const float* __restrict__ qd,
                       const float* __restrict__ qdd, const float* __restrict__ dq, const float* __restrict__ dqd,
                       const float* __restrict__ dqdd, const Sink& sink, const C& col) {
  float sc[N], ss[N];
  auto in0 = [&](const float* p, int k) { return p ? col.in(p, k) : 0.f; };
  SV v = szero(), a = gravity_acc(M.g), dv = szero(), da = szero();
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const BodyImage& b = M.body[k];
    const bool dh = k > 0;
    joint_sincos(col.in(q, k) + b.th0, &ss[k], &sc[k]);
    const float cs = sc[k], sn = ss[k];
    const float qdi = col.in(qd, k), dqi = col.in(dq, k), dqdi = col.in(dqd, k);
    const SV Xv = mot_in(b, cs, sn, v, dh);
    const SV Xa = mot_in(b, cs, sn, a, dh);
    dv = mot_in(b, cs, sn, dv, dh) - dqi * ez_crm(Xv);
    dv.w.z += dqdi;
    v = Xv;
    v.w.z += qdi;
    da = mot_in(b, cs, sn, da, dh) - dqi * ez_crm(Xa) + ez_velprod(dv, qdi) + ez_velprod(v, dqdi);
    da.w.z += in0(dqdd, k);
    a = Xa + ez_velprod(v, qdi);
    a.w.z += in0(qdd, k);
  }
  SV Fc = szero(), dFc = szero();
#pragma unroll
  for (int k = N - 1; k >= 0; --k) {
    const BodyImage& b = M.body[k];
    const bool dh = k > 0;
    const RBI I = rbi_of(b);
    const float cs = sc[k], sn = ss[k];
    const float qdi = col.in(qd, k), dqi = col.in(dq, k), dqdi = col.in(dqd, k);
    const SV Iv = rbi_mul(I, v);
    const SV F = crf_add(rbi_mul_add(Fc, I, a), v, Iv);
    const SV dF = crf_add(crf_add(rbi_mul_add(dFc, I, da), dv, Iv), v, rbi_mul(I, dv));
    sink(k, F.w.z, dF.w.z);
    if (k > 0) {
      Fc = frc_out(b, cs, sn, F, dh);
      dFc = frc_out(b, cs, sn, dF + dqi * ez_crf(F), dh);
      jvp_step_back(b, cs, sn, qdi, in0(qdd, k), dqi, dqdi, in0(dqdd, k), v, a, dv, da, dh);
    }
  }
}

// tau (optional) and dtau to global memory
template <class T, class C>
struct JvpToGlobal {
  float* tau;
  float* dtau;
  C col;
  FD void operator()(int i, float t, float dt) const {
    if (tau) col.out(tau, iv_of<T>(i), t);
    col.out(dtau, iv_of<T>(i), dt);
  }
  FD void root(const SV& t, const SV& dt) const {
    if (tau) store6(tau, 0, col, t);
    store6(dtau, 0, col, dt);
  }
};

// r = dtau - (the RNEA JVP along (dq, dqd, 0)) into a thread-local vector
template <class T, class C>
struct JvpResidual {
  LocalVec<T>* r;
  const float* dtau;
  C col;
  FD float d(int k) const { return dtau ? col.in(dtau, k) : 0.f; }
  FD void operator()(int i, float, float dt) const { r->x[iv_of<T>(i)] = d(iv_of<T>(i)) - dt; }
  FD void root(const SV&, const SV& dt) const {
    r->x[0] = d(0) - dt.w.x; r->x[1] = d(1) - dt.w.y; r->x[2] = d(2) - dt.w.z;
    r->x[3] = d(3) - dt.v.x; r->x[4] = d(4) - dt.v.y; r->x[5] = d(5) - dt.v.z;
  }
};

// ABA JVP: differentiating RNEA(q, qd, qdd) = tau along the direction gives
// M dqdd = dtau - (dRNEA along (dq, dqd, 0)) at the forward result qdd.
template <class T, class Img, class C>
FD void aba_jvp_seg_one(const Img& M, const float* q, const float* qd, const float* qdd, const float* dq,
                        const float* dqd, const float* dtau, float* dqdd, const C& col) {
  LocalVec<T> r;
  rnea_jvp_seg<T>(M, q, qd, qdd, dq, dqd, nullptr, JvpResidual<T, C>{&r, dtau, col}, col);
  P3Local<T::NBMAX> P;
  aba_seg_core<T, Img, false>(M, q, qd, r, OutToGlobal<T, C>{dqdd, col}, col, P);
}

// chains: the solve through the register mass-matrix factor
template <int N, class Img, class C>
FD void aba_jvp_chain_one(const Img& M, const float* q, const float* qd, const float* qdd, const float* dq,
                          const float* dqd, const float* dtau, float* dqdd, const C& col) {
  using T = ChainTopo<N>;
  LocalVec<T> r;
  rnea_jvp_chain<N>(M, q, qd, qdd, dq, dqd, nullptr, JvpResidual<T, C>{&r, dtau, col}, col);
  float w[N];
  chain_minv<N>(M, q, r, w, col);
#pragma unroll
  for (int k = 0; k < N; ++k) col.out(dqdd, k, w[k]);
}

// FK JVP: the motion [omega; p_dot] (world) of each requested frame along dq,
// i.e. J dq without forming J: body twists outward with dq as the joint
// rates, rotated to world at the frame bodies. Segments in topological order.
template <class T, class Img, class C>
FD void fk_jvp_seg(const Img& M, const float* __restrict__ q, const float* __restrict__ dq, const Frames& fr,
                   float* __restrict__ out, const C& col) {
  constexpr int NB = T::NBMAX;
  SV bv[NB];
  float bE[NB][9];
  // bodies that are frames, and segments whose tips have child segments (only
  // those tips' state is kept)
  uint64_t frames = 0, opened = 0;
  for (int f = 0; f < fr.n; ++f) frames |= 1ull << fr.body[f];
  for (int s = 0; s < M.n_seg; ++s)
    if (M.seg_parent[s] >= 0) opened |= 1ull << M.seg_of[M.seg_parent[s]];
  auto emit = [&](int i, const float* E, const SV& v) {
    if (!((frames >> i) & 1ull)) return;
    for (int f = 0; f < fr.n; ++f)
      if (fr.body[f] == i) store6(out, 6 * f, col, SV{rot(E, v.w), rot(E, v.v)});
  };
  int s0 = 0;
  if (T::kFree) {
    const RootPose P = root_pose(M, q, col);
    bv[0] = load6(dq, 0, col);
#pragma unroll
    for (int k = 0; k < 9; ++k) bE[0][k] = P.E[k];
    emit(0, bE[0], bv[0]);
    s0 = 1;
  }
#pragma unroll 1
  for (int s = s0; s < M.n_seg; ++s) {
    const int st = M.seg_start[s], len = M.seg_len[s];
    const int p = M.seg_parent[s];
    SV v = p < 0 ? szero() : bv[p];
    float E[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) E[k] = p < 0 ? ((k % 4 == 0) ? 1.f : 0.f) : bE[p][k];
    seg_outward(len, M.body[M.order[st]].dh, [&](int k, auto dh) {
      const int i = M.order[st + k];
      const BodyImage& b = M.body[i];
      float sn, cs;
      joint_sincos(col.in(q, iq_of<T>(i)) + b.th0, &sn, &cs);
      float ER[9];
      v = mot_in(b, cs, sn, v, dh);
      mat_mul_b(E, b, ER, dh);
      v.w.z += col.in(dq, iv_of<T>(i));
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const float x = ER[3 * r], y = ER[3 * r + 1];
        E[3 * r] = fmaf(cs, x, sn * y);
        E[3 * r + 1] = fmaf(-sn, x, cs * y);
        E[3 * r + 2] = ER[3 * r + 2];
      }
      emit(i, E, v);
    });
    if ((opened >> s) & 1ull) {
      const int last = M.order[st + len - 1];
      bv[last] = v;
#pragma unroll
      for (int k = 0; k < 9; ++k) bE[last][k] = E[k];
    }
  }
}

// The FK JVP of a fixed-base serial chain of N bodies, unrolled.
template <int N, class Img, class C>
FD void fk_jvp_chain(const Img& M, const float* __restrict__ q, const float* __restrict__ dq, const Frames& fr,
                     float* __restrict__ out, const C& col) {
  SV v = szero();
  float E[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const BodyImage& b = M.body[k];
    float sn, cs;
    joint_sincos(col.in(q, k) + b.th0, &sn, &cs);
    float ER[9];
    v = mot_in(b, cs, sn, v, k > 0);
    mat_mul_b(E, b, ER, k > 0);
    v.w.z += col.in(dq, k);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float x = ER[3 * r], y = ER[3 * r + 1];
      E[3 * r] = fmaf(cs, x, sn * y);
      E[3 * r + 1] = fmaf(-sn, x, cs * y);
      E[3 * r + 2] = ER[3 * r + 2];
    }
    for (int f = 0; f < fr.n; ++f)
      if (fr.body[f] == k) store6(out, 6 * f, col, SV{rot(E, v.w), rot(E, v.v)});
  }
}

}  // namespace frax
