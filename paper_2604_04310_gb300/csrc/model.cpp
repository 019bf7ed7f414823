// Model validation, derived tree structure and FP32 image packing (host only).
#include "model.h"

#include <memory>
#include <type_traits>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

namespace frax {
namespace {

struct M3 {
  double a[9];
  double operator()(int r, int c) const { return a[3 * r + c]; }
  double& operator()(int r, int c) { return a[3 * r + c]; }
};

M3 mul(const M3& A, const M3& B) {
  M3 C{};
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += A(r, k) * B(k, c);
      C(r, c) = s;
    }
  return C;
}

M3 transpose(const M3& A) {
  M3 T{};
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) T(r, c) = A(c, r);
  return T;
}

M3 identity() {
  M3 I{};
  I(0, 0) = I(1, 1) = I(2, 2) = 1;
  return I;
}

// A rotation Q with Q e_z = a (a unit): the internal frame of a revolute body.
M3 frame_with_z(const double a[3]) {
  double h[3] = {1, 0, 0};
  if (std::fabs(a[0]) > 0.9) { h[0] = 0; h[1] = 1; }
  double d = h[0] * a[0] + h[1] * a[1] + h[2] * a[2];
  double x[3] = {h[0] - d * a[0], h[1] - d * a[1], h[2] - d * a[2]};
  double nx = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  for (double& v : x) v /= nx;
  double y[3] = {a[1] * x[2] - a[2] * x[1], a[2] * x[0] - a[0] * x[2], a[0] * x[1] - a[1] * x[0]};
  M3 Q{};
  for (int r = 0; r < 3; ++r) {
    Q(r, 0) = x[r];
    Q(r, 1) = y[r];
    Q(r, 2) = a[r];
  }
  return Q;
}

M3 rot_z(double t) {
  M3 R = identity();
  R(0, 0) = std::cos(t); R(0, 1) = -std::sin(t);
  R(1, 0) = std::sin(t); R(1, 1) = std::cos(t);
  return R;
}

M3 rot_x(double t) {
  M3 R = identity();
  R(1, 1) = std::cos(t); R(1, 2) = -std::sin(t);
  R(2, 1) = std::sin(t); R(2, 2) = std::cos(t);
  return R;
}

bool finite_all(const double* p, int n) {
  for (int k = 0; k < n; ++k)
    if (!std::isfinite(p[k])) return false;
  return true;
}

std::string fmt(const char* f, int i) {
  char buf[256];
  std::snprintf(buf, sizeof(buf), f, i);
  return buf;
}

// The lane-group schedule of LanePlan: heavy paths (each body continues
// into its child with the deepest subtree), list-scheduled onto kLgLanes
// lanes in order of the step at which each path can start (one step after
// its head's parent), longest path first on ties; then the flags and slots
// that carry state across lanes.
void build_lane_plan(HostModel* mp) {
  HostModel& m = *mp;
  LanePlan& P = m.lane_plan;
  P = LanePlan{};
  const int n = m.nb;
  std::vector<std::vector<int>> kids(n);
  for (int i = 0; i < n; ++i)
    if (m.parent[i] >= 0) kids[m.parent[i]].push_back(i);
  std::vector<int> height(n, 1), heavy(n, -1);  // bodies on the longest path down; its first child
  for (int i = n - 1; i >= 0; --i)  // children come after their parents
    for (int c : kids[i]) {
      if (heavy[i] < 0 || height[c] > height[heavy[i]]) heavy[i] = c;
      height[i] = std::max(height[i], 1 + height[c]);
    }
  std::vector<int> step(n, -1), lane(n, -1);
  std::vector<int> lane_free(kLgLanes, 0);
  // pending path heads with the step they can start at
  std::vector<std::pair<int, int>> pend;
  for (int i = 0; i < n; ++i)
    if (m.parent[i] < 0) pend.push_back({0, i});
  int T = 0;
  while (!pend.empty()) {
    size_t best = 0;
    for (size_t k = 1; k < pend.size(); ++k) {
      const auto& a = pend[k];
      const auto& b = pend[best];
      if (a.first < b.first || (a.first == b.first && height[a.second] > height[b.second])) best = k;
    }
    const int ready = pend[best].first, head = pend[best].second;
    pend.erase(pend.begin() + static_cast<long>(best));
    int l = 0;
    for (int k = 1; k < kLgLanes; ++k)
      if (std::max(lane_free[k], ready) < std::max(lane_free[l], ready)) l = k;
    int t = std::max(lane_free[l], ready);
    for (int i = head; i >= 0; i = heavy[i], ++t) {
      step[i] = t;
      lane[i] = l;
      for (int c : kids[i])
        if (c != heavy[i]) pend.push_back({t + 1, c});
    }
    lane_free[l] = t;
    T = std::max(T, t);
  }
  if (T > kMaxBodies) return;  // cannot happen: at most one body per step and lane
  P.T = T;
  for (int t = 0; t < kMaxBodies; ++t)
    for (int l = 0; l < kLgLanes; ++l) {
      P.body[t][l] = -1;
      P.flag[t][l] = 0;
    }
  for (int i = 0; i < kMaxBodies; ++i) P.oslot[i] = P.islot[i] = -1, P.rc_first[i] = P.rc_count[i] = 0;
  for (int i = 0; i < n; ++i) P.body[step[i]][lane[i]] = static_cast<int8_t>(i);
  auto at = [&](int t, int l) { return (t >= 0 && t < T) ? static_cast<int>(P.body[t][l]) : -1; };
  // outward: a parent processed at the previous step on the same lane hands
  // its state over in registers; any other parent stores it in a slot
  for (int i = 0; i < n; ++i) {
    const int p = m.parent[i];
    if (p < 0 || at(step[i] - 1, lane[i]) == p) continue;
    P.flag[step[i]][lane[i]] |= kLgLoad;
    if (P.oslot[p] < 0) {
      P.oslot[p] = static_cast<int8_t>(P.n_oslot++);
      P.flag[step[p]][lane[p]] |= kLgStoreOut;
    }
  }
  // inward (the table read backwards): the lane's carry is a child's when
  // the next step on the lane is that child; other children are remote
  int nrc = 0;
  for (int i = 0; i < n; ++i) {
    const int cnext = at(step[i] + 1, lane[i]);
    if (cnext >= 0 && m.parent[cnext] == i) P.flag[step[i]][lane[i]] |= kLgCarry;
    P.rc_first[i] = static_cast<int8_t>(nrc);
    for (int c : kids[i]) {
      if (c == cnext) continue;
      P.rc_list[nrc++] = static_cast<int8_t>(c);
      P.islot[c] = static_cast<int8_t>(P.n_islot++);
      P.flag[step[c]][lane[c]] |= kLgStoreIn;
    }
    P.rc_count[i] = static_cast<int8_t>(nrc - P.rc_first[i]);
  }
}

}  // namespace

std::string build_model(int n, const int32_t* parent, const int32_t* joint_type, const double* axis,
                        const double* placement, const double* inertia, const double* gravity,
                        HostModel* out) {
  if (n < 1 || n > kMaxBodies) return fmt("n_bodies must be in [1, 64], got %d", n);
  if (!parent || !joint_type || !axis || !placement || !inertia || !gravity || !out)
    return "null argument to frax_model_create";
  if (!finite_all(gravity, 3)) return "gravity is not finite";
  HostModel m;
  m.nb = n;
  m.parent.assign(parent, parent + n);
  for (int i = 0; i < n; ++i) {
    if (parent[i] < -1 || parent[i] >= i)
      return fmt("body %d: parent must be in [-1, i-1] (topological order)", i);
    if (joint_type[i] != 0 && joint_type[i] != 1) return fmt("body %d: unknown joint type", i);
    if (joint_type[i] == 1 && (i != 0 || parent[i] != -1))
      return fmt("body %d: a free-flyer joint is only allowed at body 0 with parent -1", i);
    if (!finite_all(axis + 3 * i, 3) || !finite_all(placement + 12 * i, 12) ||
        !finite_all(inertia + 10 * i, 10))
      return fmt("body %d: non-finite parameter", i);
  }
  m.free_root = joint_type[0] == 1;
  int nq = 0, nv = 0;
  for (int i = 0; i < n; ++i) {
    m.iq.push_back(nq);
    m.iv.push_back(nv);
    bool fr = joint_type[i] == 1;
    nq += fr ? 7 : 1;
    nv += fr ? 6 : 1;
  }
  m.nq = nq;
  m.nv = nv;
  m.dof_parent.assign(nv, -1);
  m.anc.assign(n, 0);
  m.depth.assign(n, 0);
  for (int i = 0; i < n; ++i) {
    int k = parent[i];
    m.anc[i] = (k >= 0 ? m.anc[k] : 0) | (uint64_t(1) << i);
    m.depth[i] = k >= 0 ? m.depth[k] + 1 : 0;
    if (joint_type[i] == 1) {
      for (int d = 0; d < 6; ++d) m.dof_parent[m.iv[i] + d] = d - 1;
    } else {
      int last_parent_dof = k < 0 ? -1 : m.iv[k] + (joint_type[k] == 1 ? 5 : 0);
      m.dof_parent[m.iv[i]] = last_parent_dof;
    }
  }
  for (int k = 0; k < 3; ++k) m.gravity[k] = gravity[k];

  std::vector<M3> Q(n);
  for (int i = 0; i < n; ++i) {
    if (joint_type[i] == 1) {
      Q[i] = identity();
      continue;
    }
    const double* a = axis + 3 * i;
    double na = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    if (std::fabs(na - 1.0) > 1e-6) return fmt("body %d: joint axis is not a unit vector", i);
    double au[3] = {a[0] / na, a[1] / na, a[2] / na};
    Q[i] = frame_with_z(au);
  }
  // Denavit-Hartenberg turn of the internal frames: a revolute body k whose
  // only child c is revolute turns its frame about z by phi_k so that its x
  // lies on the common normal of the two axes. With the child's axis in k's
  // frame u = Rot_z(g1) Rot_x(b) e_z = (sin b sin g1, -sin b cos g1, cos b),
  // phi_k = g1; c's constant rotation becomes Rot_x(b) Rot_z(th0).
  std::vector<int> nchild(n, 0), only_child(n, -1);
  for (int i = 0; i < n; ++i)
    if (parent[i] >= 0) {
      nchild[parent[i]]++;
      only_child[parent[i]] = i;
    }
  std::vector<int> dh_child(n, -1);
  for (int k = 0; k < n; ++k) {
    const int c = only_child[k];
    if (nchild[k] != 1 || joint_type[k] == 1 || joint_type[c] == 1) continue;
    dh_child[k] = c;
    M3 RTc{};
    for (int t = 0; t < 9; ++t) RTc.a[t] = placement[12 * c + t];
    const M3 Rc = mul(mul(transpose(Q[k]), RTc), Q[c]);
    const double ux = Rc(0, 2), uy = Rc(1, 2);
    const double phi = std::hypot(ux, uy) > 1e-12 ? std::atan2(ux, -uy) : 0.0;
    Q[k] = mul(Q[k], rot_z(phi));
  }
  std::vector<char> is_dh(n, 0);
  for (int k = 0; k < n; ++k)
    if (dh_child[k] >= 0) is_dh[dh_child[k]] = 1;

  m.bodies.resize(n);
  for (int i = 0; i < n; ++i) {
    M3 RT{};
    for (int k = 0; k < 9; ++k) RT.a[k] = placement[12 * i + k];
    M3 RtR = mul(transpose(RT), RT);
    double err = 0, det = 0;
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) err = std::fmax(err, std::fabs(RtR(r, c) - (r == c ? 1.0 : 0.0)));
    det = RT(0, 0) * (RT(1, 1) * RT(2, 2) - RT(1, 2) * RT(2, 1)) -
          RT(0, 1) * (RT(1, 0) * RT(2, 2) - RT(1, 2) * RT(2, 0)) +
          RT(0, 2) * (RT(1, 0) * RT(2, 1) - RT(1, 1) * RT(2, 0));
    if (err > 1e-6 || det < 0) return fmt("body %d: placement rotation is not a proper rotation", i);
    const double* pT = placement + 12 * i + 9;
    const double* in = inertia + 10 * i;
    double mass = in[0];
    if (!(mass > 0)) return fmt("body %d: mass must be positive", i);
    M3 Ic{};
    Ic(0, 0) = in[4]; Ic(1, 1) = in[5]; Ic(2, 2) = in[6];
    Ic(0, 1) = Ic(1, 0) = in[7];
    Ic(0, 2) = Ic(2, 0) = in[8];
    Ic(1, 2) = Ic(2, 1) = in[9];
    // positive definiteness by leading principal minors
    double d1 = Ic(0, 0), d2 = Ic(0, 0) * Ic(1, 1) - Ic(0, 1) * Ic(1, 0);
    double d3 = Ic(0, 0) * (Ic(1, 1) * Ic(2, 2) - Ic(1, 2) * Ic(2, 1)) -
                Ic(0, 1) * (Ic(1, 0) * Ic(2, 2) - Ic(1, 2) * Ic(2, 0)) +
                Ic(0, 2) * (Ic(1, 0) * Ic(2, 1) - Ic(1, 1) * Ic(2, 0));
    if (!(d1 > 0 && d2 > 0 && d3 > 0))
      return fmt("body %d: rotational inertia is not positive definite", i);

    BodyImage& b = m.bodies[i];
    int k = parent[i];
    M3 Qp = k >= 0 ? Q[k] : identity();
    M3 Rint = joint_type[i] == 1 ? RT : mul(mul(transpose(Qp), RT), Q[i]);  // before any dh rewrite
    double pint[3];
    for (int r = 0; r < 3; ++r) {
      pint[r] = joint_type[i] == 1 ? pT[r]
                                   : Qp(0, r) * pT[0] + Qp(1, r) * pT[1] + Qp(2, r) * pT[2];
    }
    b.dh = 0;
    b.ca = 1.f;
    b.sa = 0.f;
    b.th0 = 0.f;
    if (is_dh[i]) {
      // Rint = Rot_x(alpha) Rot_z(th0) =
      //   [[ct, -st, 0], [ca st, ca ct, -sa], [sa st, sa ct, ca]]
      const double alpha = std::atan2(-Rint(1, 2), Rint(2, 2));
      const double th0 = std::atan2(-Rint(0, 1), Rint(0, 0));
      const M3 Rdh = mul(rot_x(alpha), rot_z(th0));
      double res = 0;
      for (int t = 0; t < 9; ++t) res = std::fmax(res, std::fabs(Rdh.a[t] - Rint.a[t]));
      // the turn above makes the child's axis (0, -sin a, cos a), so this
      // form is exact; chain kernels rely on it for every body after the first
      if (!(res < 1e-9)) return fmt("body %d: internal Denavit-Hartenberg frame failed", i);
      b.dh = 1;
      b.ca = static_cast<float>(std::cos(alpha));
      b.sa = static_cast<float>(std::sin(alpha));
      b.th0 = static_cast<float>(th0);
      Rint = rot_x(alpha);
    }
    for (int t = 0; t < 9; ++t) b.R[t] = static_cast<float>(Rint.a[t]);
    for (int t = 0; t < 3; ++t) b.p[t] = static_cast<float>(pint[t]);
    for (int t = 0; t < 9; ++t) b.Q[t] = static_cast<float>(Q[i].a[t]);
    // inertia in internal coordinates, about the body origin
    const double* c = in + 1;
    double ci[3];
    for (int r = 0; r < 3; ++r) ci[r] = Q[i](0, r) * c[0] + Q[i](1, r) * c[1] + Q[i](2, r) * c[2];
    M3 Ici = mul(mul(transpose(Q[i]), Ic), Q[i]);
    double c2 = ci[0] * ci[0] + ci[1] * ci[1] + ci[2] * ci[2];
    M3 Io{};
    for (int r = 0; r < 3; ++r)
      for (int s = 0; s < 3; ++s) Io(r, s) = Ici(r, s) + mass * ((r == s ? c2 : 0.0) - ci[r] * ci[s]);
    b.m = static_cast<float>(mass);
    for (int t = 0; t < 3; ++t) b.h[t] = static_cast<float>(mass * ci[t]);
    b.I[0] = static_cast<float>(Io(0, 0));
    b.I[1] = static_cast<float>(Io(1, 1));
    b.I[2] = static_cast<float>(Io(2, 2));
    b.I[3] = static_cast<float>(Io(0, 1));
    b.I[4] = static_cast<float>(Io(0, 2));
    b.I[5] = static_cast<float>(Io(1, 2));
  }
  // segments (see model_image.h), numbered in topological order
  {
    std::vector<int> nchild(n, 0), seg_of(n, -1);
    for (int i = 0; i < n; ++i)
      if (parent[i] >= 0) nchild[parent[i]]++;
    std::vector<std::vector<int>> segs;
    for (int i = 0; i < n; ++i) {
      const int k = parent[i];
      bool extend = k >= 0 && nchild[k] == 1 && !(m.free_root && k == 0) && !(m.free_root && i == 0);
      if (extend) {
        auto& sg = segs[seg_of[k]];
        extend = sg.back() == k && static_cast<int>(sg.size()) < kMaxSeg;
      }
      if (extend) {
        segs[seg_of[k]].push_back(i);
        seg_of[i] = seg_of[k];
      } else {
        seg_of[i] = static_cast<int>(segs.size());
        segs.push_back({i});
      }
    }
    const int ns = static_cast<int>(segs.size());
    m.seg_of.assign(n, 0);
    m.pos_of.assign(n, 0);
    for (int s2 = 0; s2 < ns; ++s2)
      for (int k = 0; k < static_cast<int>(segs[s2].size()); ++k) {
        m.seg_of[segs[s2][k]] = s2;
        m.pos_of[segs[s2][k]] = k;
      }
    std::vector<std::vector<int>> kids(ns);
    for (int s2 = 0; s2 < ns; ++s2) {
      const int p = parent[segs[s2][0]];
      m.seg_start.push_back(static_cast<int>(m.order.size()));
      m.seg_len.push_back(static_cast<int>(segs[s2].size()));
      m.seg_parent.push_back(p);
      for (int b : segs[s2]) m.order.push_back(b);
      if (p >= 0) kids[seg_of[p]].push_back(s2);
    }
    // depth-first schedule; explicit stack of (segment, next child)
    std::vector<std::pair<int, int>> stack;
    for (int s2 = 0; s2 < ns; ++s2) {
      if (m.seg_parent[s2] >= 0) continue;
      stack.push_back({s2, 0});
      while (!stack.empty()) {
        auto& top = stack.back();
        const int cur = top.first;
        if (kids[cur].empty()) {
          m.act.push_back((kActLeaf << 6) | cur);
          stack.pop_back();
          continue;
        }
        if (top.second == 0) m.act.push_back((kActOpen << 6) | cur);
        if (top.second < static_cast<int>(kids[cur].size())) {
          const int c = kids[cur][top.second++];
          stack.push_back({c, 0});
        } else {
          m.act.push_back((kActClose << 6) | cur);
          stack.pop_back();
        }
      }
    }
  }
  bool chain = !m.free_root;
  for (int i = 0; i < n; ++i) chain = chain && parent[i] == i - 1;
  m.kind = (chain && n == 7) ? kKindChain : kKindTree;
  // structural zeros: dofs whose bodies are not in an ancestor relation
  m.dof_body.assign(m.nv, 0);
  for (int i = 0; i < n; ++i)
    for (int d = 0; d < (joint_type[i] == 1 ? 6 : 1); ++d) m.dof_body[m.iv[i] + d] = i;
  auto related = [&](int a, int b) {
    const int ba = m.dof_body[a], bb = m.dof_body[b];
    return ((m.anc[ba] >> bb) & 1ull) || ((m.anc[bb] >> ba) & 1ull);
  };
  for (int r = 0; r < m.nv; ++r)
    for (int c = 0; c < m.nv; ++c) {
      if (!related(r, c)) m.zero_M.push_back(static_cast<uint16_t>(r * m.nv + c));
      if (c < r && !related(r, c)) m.zero_LD.push_back(static_cast<uint16_t>(r * (r + 1) / 2 + c));
    }
  // kernels that unroll a segment take the Rot_x form for every body after
  // the segment's first: each such body is the only child of a revolute body
  for (int i = 0; i < n; ++i)
    if (m.pos_of[i] > 0 && !m.bodies[i].dh) return fmt("body %d: segment body without a Rot_x frame", i);
  build_lane_plan(&m);
  auto packed = [&](auto* tag) {
    using Img = std::remove_pointer_t<decltype(tag)>;
    auto p = std::make_shared<Img>();
    m.pack(p.get());
    return std::shared_ptr<const Img>(std::move(p));
  };
  m.img64 = packed(static_cast<ModelImage<64>*>(nullptr));
  if (m.kind == kKindChain) {
    m.img7 = packed(static_cast<ModelImage<7>*>(nullptr));
    m.img8 = packed(static_cast<ModelImage<8>*>(nullptr));
  } else if (n <= 32) {
    m.img32 = packed(static_cast<ModelImage<32>*>(nullptr));
  }
  *out = std::move(m);
  return "";
}

}  // namespace frax
