// C ABI: argument validation, model handles, kernel dispatch.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "fault.h"
#include "handles.h"
#include "launch.h"

namespace {
thread_local std::string g_last_error;
}

namespace frax {
frax_status set_error(frax_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}
frax_status clear_error() {
  g_last_error.clear();
  return FRAX_OK;
}

namespace {
std::atomic<int> g_fault_point{kFaultNone};
std::atomic<int> g_fault_countdown{0};
bool fault_injection_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("FRAX_FAULT_INJECTION");
    return v && std::strcmp(v, "1") == 0;
  }();
  return on;
}
}  // namespace

bool fault_hit(int point) {
  if (g_fault_point.load(std::memory_order_relaxed) != point) return false;
  if (g_fault_countdown.fetch_sub(1) > 0) return false;
  int expected = point;
  return g_fault_point.compare_exchange_strong(expected, kFaultNone);
}
}  // namespace frax

namespace {

frax_status fail(frax_status s, const std::string& msg) { return frax::set_error(s, msg); }
frax_status ok() { return frax::clear_error(); }

frax_status check_batch(frax_model_t model, int64_t B, int64_t ld, const char* fn) {
  if (!model) return fail(FRAX_EINVAL, std::string(fn) + ": model is NULL");
  if (B < 0) return fail(FRAX_EINVAL, std::string(fn) + ": B must be >= 0");
  if (B > 0 && ld < B) return fail(FRAX_EINVAL, std::string(fn) + ": ld must be >= B");
  // the kernels address entry k as k * ld * 4 bytes in 32 x 32-bit products
  if (ld >= (int64_t(1) << 30)) return fail(FRAX_EINVAL, std::string(fn) + ": ld must be below 2^30");
  if (B > (int64_t(1) << 40)) return fail(FRAX_EINVAL, std::string(fn) + ": B too large");
  return FRAX_OK;
}

frax_status need(const void* p, const char* fn, const char* name) {
  if (!p) return fail(FRAX_EINVAL, std::string(fn) + ": " + name + " is NULL");
  return FRAX_OK;
}

frax_status dispatch(frax_model_t model, frax::Op op, const frax::OpArgs& args, const char* fn) {
  const frax::HostModel& m = model->m;
  frax::OpArgs a = args;
  a.tree_path = model->tree_path;
  cudaError_t e;
  if (m.kind == frax::kKindChain)
    e = frax::launch_chain7(m, op, a);
  else if (m.nb <= 32)
    e = frax::launch_tree32(m, op, a);
  else
    e = frax::launch_tree64(m, op, a);
  if (e != cudaSuccess)
    return fail(FRAX_ECUDA, std::string(fn) + ": kernel launch failed: " + cudaGetErrorString(e));
  return ok();
}

// Structural zeros of a tree's outputs: the Jacobian's by one row fill after
// the per-instance kernel (which skips them), M's and the factor's by the
// CRBA kernel itself from the same row list. ZeroRows is large (14 KB): one
// per thread, reused.
frax_status fill_zeros(frax::ZeroRows& z, float* base0, float* base1, const frax::OpArgs& a, const char* fn) {
  const cudaError_t e = frax::launch_zero_rows(z, base0, base1, a.ld, a.B, a.stream);
  if (e != cudaSuccess) return fail(FRAX_ECUDA, std::string(fn) + ": zero fill launch failed: " + cudaGetErrorString(e));
  return ok();
}
thread_local frax::ZeroRows g_zero_rows;

#define FRAX_TRY(expr)                    \
  do {                                    \
    frax_status s_ = (expr);              \
    if (s_ != FRAX_OK) return s_;         \
  } while (0)

}  // namespace

extern "C" {

const char* frax_last_error(void) { return g_last_error.c_str(); }

frax_status frax_debug_inject_fault(int point, int after) {
  if (!frax::fault_injection_enabled())
    return fail(FRAX_EINVAL, "frax_debug_inject_fault: disabled (start the process with FRAX_FAULT_INJECTION=1)");
  if (point < frax::kFaultNone || point >= frax::kFaultCount || after < 0)
    return fail(FRAX_EINVAL, "frax_debug_inject_fault: bad point or count");
  frax::g_fault_countdown.store(after);
  frax::g_fault_point.store(point);
  return ok();
}
const char* frax_version(void) { return "frax-gb300 0.1 (sm_103a)"; }

frax_status frax_model_create(int n_bodies, const int32_t* parent, const int32_t* joint_type,
                              const double* axis, const double* placement, const double* inertia,
                              const double* gravity, frax_model_t* out) {
  if (!out) return fail(FRAX_EINVAL, "frax_model_create: out is NULL");
  *out = nullptr;
  frax_model_s* h = new (std::nothrow) frax_model_s;
  if (!h) return fail(FRAX_ENOMEM, "frax_model_create: out of host memory");
  std::string err =
      frax::build_model(n_bodies, parent, joint_type, axis, placement, inertia, gravity, &h->m);
  if (!err.empty()) {
    delete h;
    return fail(FRAX_EINVAL, "frax_model_create: " + err);
  }
  if (h->m.kind != frax::kKindChain) {
    for (int want = 1; want <= 3; ++want) {
      frax::ZeroRows* z = new (std::nothrow) frax::ZeroRows;
      if (!z) {
        delete h;
        return fail(FRAX_ENOMEM, "frax_model_create: out of host memory");
      }
      z->n0 = z->n = 0;
      if (want & 1)
        for (uint16_t r : h->m.zero_M) z->row[z->n++] = r;
      z->n0 = z->n;
      if (want & 2)
        for (uint16_t r : h->m.zero_LD) z->row[z->n++] = r;
      h->crba_zeros[want].reset(z);
    }
  }
  *out = h;
  return ok();
}

frax_status frax_model_destroy(frax_model_t model) {
  delete model;
  return ok();
}

frax_status frax_model_dims(frax_model_t model, int* nq, int* nv, int* n_bodies) {
  if (!model) return fail(FRAX_EINVAL, "frax_model_dims: model is NULL");
  if (nq) *nq = model->m.nq;
  if (nv) *nv = model->m.nv;
  if (n_bodies) *n_bodies = model->m.nb;
  return ok();
}

frax_status frax_model_set_tree_path(frax_model_t model, int path) {
  if (!model) return fail(FRAX_EINVAL, "frax_model_set_tree_path: model is NULL");
  if (path < FRAX_TREE_PATH_AUTO || path > FRAX_TREE_PATH_LANE_GROUP)
    return fail(FRAX_EINVAL, "frax_model_set_tree_path: unknown path");
  model->tree_path = path;
  return ok();
}

frax_status frax_model_kind(frax_model_t model, int* kind) {
  if (!model || !kind) return fail(FRAX_EINVAL, "frax_model_kind: NULL argument");
  *kind = model->m.kind;
  return ok();
}

frax_status frax_fk(frax_model_t model, int64_t B, int64_t ld, const float* q, float* pose, void* stream) {
  FRAX_TRY(check_batch(model, B, ld, "frax_fk"));
  if (B == 0) return ok();
  FRAX_TRY(need(q, "frax_fk", "q"));
  FRAX_TRY(need(pose, "frax_fk", "pose"));
  frax::OpArgs a;
  a.B = B; a.ld = ld; a.q = q; a.out0 = pose; a.stream = static_cast<cudaStream_t>(stream);
  return dispatch(model, frax::kOpFk, a, "frax_fk");
}

frax_status frax_jacobian(frax_model_t model, int64_t B, int64_t ld, const float* q, int n_frames,
                          const int32_t* frame_body, float* pose, float* J, void* stream) {
  FRAX_TRY(check_batch(model, B, ld, "frax_jacobian"));
  if (n_frames < 1 || n_frames > FRAX_MAX_FRAMES)
    return fail(FRAX_EINVAL, "frax_jacobian: n_frames must be in [1, 8]");
  FRAX_TRY(need(frame_body, "frax_jacobian", "frame_body"));
  frax::OpArgs a;
  a.frames.n = n_frames;
  for (int f = 0; f < n_frames; ++f) {
    if (frame_body[f] < 0 || frame_body[f] >= model->m.nb)
      return fail(FRAX_EINVAL, "frax_jacobian: frame body index out of range");
    a.frames.body[f] = frame_body[f];
  }
  if (B == 0) return ok();
  FRAX_TRY(need(q, "frax_jacobian", "q"));
  FRAX_TRY(need(J, "frax_jacobian", "J"));
  a.B = B; a.ld = ld; a.q = q; a.out0 = pose; a.out1 = J; a.stream = static_cast<cudaStream_t>(stream);
  FRAX_TRY(dispatch(model, frax::kOpJac, a, "frax_jacobian"));
  const frax::HostModel& m = model->m;
  if (m.kind == frax::kKindChain) return ok();
  frax::ZeroRows& z = g_zero_rows;
  z.n0 = z.n = 0;
  for (int f = 0; f < n_frames; ++f)
    for (int c = 0; c < m.nv; ++c)
      if (!((m.anc[frame_body[f]] >> m.dof_body[c]) & 1ull))
        for (int r = 0; r < 6; ++r) z.row[z.n++] = static_cast<uint16_t>((f * 6 + r) * m.nv + c);
  z.n0 = z.n;
  return fill_zeros(z, J, nullptr, a, "frax_jacobian");
}

frax_status frax_rnea(frax_model_t model, int64_t B, int64_t ld, const float* q, const float* qd,
                      const float* qdd, float* tau, void* stream) {
  FRAX_TRY(check_batch(model, B, ld, "frax_rnea"));
  if (B == 0) return ok();
  FRAX_TRY(need(q, "frax_rnea", "q"));
  FRAX_TRY(need(qd, "frax_rnea", "qd"));
  FRAX_TRY(need(tau, "frax_rnea", "tau"));
  frax::OpArgs a;
  a.B = B; a.ld = ld; a.q = q; a.qd = qd; a.qdd = qdd; a.out0 = tau;
  a.stream = static_cast<cudaStream_t>(stream);
  return dispatch(model, frax::kOpRnea, a, "frax_rnea");
}

frax_status frax_crba(frax_model_t model, int64_t B, int64_t ld, const float* q, float* M, float* LD,
                      void* stream) {
  FRAX_TRY(check_batch(model, B, ld, "frax_crba"));
  if (B == 0) return ok();
  FRAX_TRY(need(q, "frax_crba", "q"));
  if (!M && !LD) return fail(FRAX_EINVAL, "frax_crba: M and LD are both NULL");
  frax::OpArgs a;
  a.B = B; a.ld = ld; a.q = q; a.out0 = M; a.out1 = LD; a.stream = static_cast<cudaStream_t>(stream);
  const frax::HostModel& m = model->m;
  if (m.kind != frax::kKindChain)  // the tree kernel writes the structural zeros too
    a.zeros = model->crba_zeros[(M ? 1 : 0) | (LD ? 2 : 0)].get();
  return dispatch(model, frax::kOpCrba, a, "frax_crba");
}

frax_status frax_aba(frax_model_t model, int64_t B, int64_t ld, const float* q, const float* qd,
                     const float* tau, float* qdd, void* stream) {
  FRAX_TRY(check_batch(model, B, ld, "frax_aba"));
  if (B == 0) return ok();
  FRAX_TRY(need(q, "frax_aba", "q"));
  FRAX_TRY(need(qd, "frax_aba", "qd"));
  FRAX_TRY(need(tau, "frax_aba", "tau"));
  FRAX_TRY(need(qdd, "frax_aba", "qdd"));
  frax::OpArgs a;
  a.B = B; a.ld = ld; a.q = q; a.qd = qd; a.tau = tau; a.out0 = qdd;
  a.stream = static_cast<cudaStream_t>(stream);
  return dispatch(model, frax::kOpAba, a, "frax_aba");
}

frax_status frax_aba_articulated(frax_model_t model, int64_t B, int64_t ld, const float* q, const float* qd,
                                 const float* tau, float* qdd, void* stream) {
  FRAX_TRY(check_batch(model, B, ld, "frax_aba_articulated"));
  if (B == 0) return ok();
  FRAX_TRY(need(q, "frax_aba_articulated", "q"));
  FRAX_TRY(need(qd, "frax_aba_articulated", "qd"));
  FRAX_TRY(need(tau, "frax_aba_articulated", "tau"));
  FRAX_TRY(need(qdd, "frax_aba_articulated", "qdd"));
  frax::OpArgs a;
  a.B = B; a.ld = ld; a.q = q; a.qd = qd; a.tau = tau; a.out0 = qdd;
  a.stream = static_cast<cudaStream_t>(stream);
  return dispatch(model, frax::kOpAbaSweep, a, "frax_aba_articulated");
}

frax_status frax_rnea_vjp(frax_model_t model, int64_t B, int64_t ld, const float* q, const float* qd,
                          const float* qdd, const float* gbar, float* qbar, float* qdbar, float* qddbar,
                          void* stream) {
  FRAX_TRY(check_batch(model, B, ld, "frax_rnea_vjp"));
  if (B == 0) return ok();
  FRAX_TRY(need(q, "frax_rnea_vjp", "q"));
  FRAX_TRY(need(qd, "frax_rnea_vjp", "qd"));
  FRAX_TRY(need(qdd, "frax_rnea_vjp", "qdd"));
  FRAX_TRY(need(gbar, "frax_rnea_vjp", "gbar"));
  if (!qbar && !qdbar && !qddbar) return fail(FRAX_EINVAL, "frax_rnea_vjp: all outputs are NULL");
  frax::OpArgs a;
  a.B = B; a.ld = ld; a.q = q; a.qd = qd; a.qdd = qdd; a.gbar = gbar;
  a.out0 = qbar; a.out1 = qdbar; a.out2 = qddbar; a.stream = static_cast<cudaStream_t>(stream);
  return dispatch(model, frax::kOpRneaVjp, a, "frax_rnea_vjp");
}

frax_status frax_aba_vjp(frax_model_t model, int64_t B, int64_t ld, const float* q, const float* qd,
                         const float* tau, const float* qdd, const float* gbar, float* qbar, float* qdbar,
                         float* taubar, void* stream) {
  FRAX_TRY(check_batch(model, B, ld, "frax_aba_vjp"));
  if (B == 0) return ok();
  FRAX_TRY(need(q, "frax_aba_vjp", "q"));
  FRAX_TRY(need(qd, "frax_aba_vjp", "qd"));
  FRAX_TRY(need(qdd, "frax_aba_vjp", "qdd"));
  FRAX_TRY(need(gbar, "frax_aba_vjp", "gbar"));
  if (!qbar && !qdbar && !taubar) return fail(FRAX_EINVAL, "frax_aba_vjp: all outputs are NULL");
  frax::OpArgs a;
  a.B = B; a.ld = ld; a.q = q; a.qd = qd; a.tau = tau; a.qdd = qdd; a.gbar = gbar;
  a.out0 = qbar; a.out1 = qdbar; a.out2 = taubar; a.stream = static_cast<cudaStream_t>(stream);
  return dispatch(model, frax::kOpAbaVjp, a, "frax_aba_vjp");
}

frax_status frax_ltdl_solve(frax_model_t model, int64_t B, int64_t ld, const float* LD, const float* b, float* x,
                            void* stream) {
  FRAX_TRY(check_batch(model, B, ld, "frax_ltdl_solve"));
  if (B == 0) return ok();
  FRAX_TRY(need(LD, "frax_ltdl_solve", "LD"));
  FRAX_TRY(need(b, "frax_ltdl_solve", "b"));
  FRAX_TRY(need(x, "frax_ltdl_solve", "x"));
  frax::OpArgs a;
  a.B = B; a.ld = ld; a.in_LD = LD; a.qd = b; a.out0 = x; a.stream = static_cast<cudaStream_t>(stream);
  return dispatch(model, frax::kOpLtdlSolve, a, "frax_ltdl_solve");
}

frax_status frax_ltdl_inverse(frax_model_t model, int64_t B, int64_t ld, const float* LD, float* Minv,
                              void* stream) {
  FRAX_TRY(check_batch(model, B, ld, "frax_ltdl_inverse"));
  if (B == 0) return ok();
  FRAX_TRY(need(LD, "frax_ltdl_inverse", "LD"));
  FRAX_TRY(need(Minv, "frax_ltdl_inverse", "Minv"));
  frax::OpArgs a;
  a.B = B; a.ld = ld; a.in_LD = LD; a.out0 = Minv; a.stream = static_cast<cudaStream_t>(stream);
  return dispatch(model, frax::kOpLtdlInverse, a, "frax_ltdl_inverse");
}

frax_status frax_rnea_ext(frax_model_t model, int64_t B, int64_t ld, const float* q, const float* qd,
                          const float* qdd, const float* fext, float* tau, void* stream) {
  FRAX_TRY(check_batch(model, B, ld, "frax_rnea_ext"));
  if (B == 0) return ok();
  FRAX_TRY(need(q, "frax_rnea_ext", "q"));
  FRAX_TRY(need(qd, "frax_rnea_ext", "qd"));
  FRAX_TRY(need(fext, "frax_rnea_ext", "fext"));
  FRAX_TRY(need(tau, "frax_rnea_ext", "tau"));
  frax::OpArgs a;
  a.B = B; a.ld = ld; a.q = q; a.qd = qd; a.qdd = qdd; a.in_fext = fext; a.out0 = tau;
  a.stream = static_cast<cudaStream_t>(stream);
  return dispatch(model, frax::kOpRneaExt, a, "frax_rnea_ext");
}

frax_status frax_aba_ext(frax_model_t model, int64_t B, int64_t ld, const float* q, const float* qd,
                         const float* tau, const float* fext, float* qdd, void* stream) {
  FRAX_TRY(check_batch(model, B, ld, "frax_aba_ext"));
  if (B == 0) return ok();
  FRAX_TRY(need(q, "frax_aba_ext", "q"));
  FRAX_TRY(need(qd, "frax_aba_ext", "qd"));
  FRAX_TRY(need(tau, "frax_aba_ext", "tau"));
  FRAX_TRY(need(fext, "frax_aba_ext", "fext"));
  FRAX_TRY(need(qdd, "frax_aba_ext", "qdd"));
  frax::OpArgs a;
  a.B = B; a.ld = ld; a.q = q; a.qd = qd; a.tau = tau; a.in_fext = fext; a.out0 = qdd;
  a.stream = static_cast<cudaStream_t>(stream);
  return dispatch(model, frax::kOpAbaExt, a, "frax_aba_ext");
}

frax_status frax_fk_scan(frax_model_t model, int64_t B, int64_t ld, const float* q, float* pose, void* stream) {
  FRAX_TRY(check_batch(model, B, ld, "frax_fk_scan"));
  const frax::HostModel& m = model->m;
  for (int i = 1; i < m.nb; ++i)
    if (m.parent[i] != i - 1) return fail(FRAX_EINVAL, "frax_fk_scan: the model is not a serial chain");
  if (B > (int64_t(1) << 32)) return fail(FRAX_EINVAL, "frax_fk_scan: B too large");
  if (B == 0) return ok();
  FRAX_TRY(need(q, "frax_fk_scan", "q"));
  FRAX_TRY(need(pose, "frax_fk_scan", "pose"));
  frax::OpArgs a;
  a.B = B; a.ld = ld; a.q = q; a.out0 = pose; a.stream = static_cast<cudaStream_t>(stream);
  const cudaError_t e = frax::launch_fk_scan(m, a);
  if (e != cudaSuccess)
    return fail(FRAX_ECUDA, std::string("frax_fk_scan: kernel launch failed: ") + cudaGetErrorString(e));
  return ok();
}

frax_status frax_fk_jvp(frax_model_t model, int64_t B, int64_t ld, const float* q, const float* dq, int n_frames,
                        const int32_t* frame_body, float* dpose, void* stream) {
  FRAX_TRY(check_batch(model, B, ld, "frax_fk_jvp"));
  if (n_frames < 1 || n_frames > FRAX_MAX_FRAMES)
    return fail(FRAX_EINVAL, "frax_fk_jvp: n_frames must be in [1, 8]");
  FRAX_TRY(need(frame_body, "frax_fk_jvp", "frame_body"));
  frax::OpArgs a;
  a.frames.n = n_frames;
  for (int f = 0; f < n_frames; ++f) {
    if (frame_body[f] < 0 || frame_body[f] >= model->m.nb)
      return fail(FRAX_EINVAL, "frax_fk_jvp: frame body index out of range");
    a.frames.body[f] = frame_body[f];
  }
  if (B == 0) return ok();
  FRAX_TRY(need(q, "frax_fk_jvp", "q"));
  FRAX_TRY(need(dq, "frax_fk_jvp", "dq"));
  FRAX_TRY(need(dpose, "frax_fk_jvp", "dpose"));
  a.B = B; a.ld = ld; a.q = q; a.in_dq = dq; a.out0 = dpose; a.stream = static_cast<cudaStream_t>(stream);
  return dispatch(model, frax::kOpFkJvp, a, "frax_fk_jvp");
}

frax_status frax_rnea_jvp(frax_model_t model, int64_t B, int64_t ld, const float* q, const float* qd,
                          const float* qdd, const float* dq, const float* dqd, const float* dqdd, float* tau,
                          float* dtau, void* stream) {
  FRAX_TRY(check_batch(model, B, ld, "frax_rnea_jvp"));
  if (B == 0) return ok();
  FRAX_TRY(need(q, "frax_rnea_jvp", "q"));
  FRAX_TRY(need(qd, "frax_rnea_jvp", "qd"));
  FRAX_TRY(need(dq, "frax_rnea_jvp", "dq"));
  FRAX_TRY(need(dqd, "frax_rnea_jvp", "dqd"));
  FRAX_TRY(need(dtau, "frax_rnea_jvp", "dtau"));
  frax::OpArgs a;
  a.B = B; a.ld = ld; a.q = q; a.qd = qd; a.qdd = qdd; a.in_dq = dq; a.in_dqd = dqd; a.in_dx = dqdd;
  a.out0 = tau; a.out1 = dtau; a.stream = static_cast<cudaStream_t>(stream);
  return dispatch(model, frax::kOpRneaJvp, a, "frax_rnea_jvp");
}

frax_status frax_aba_jvp(frax_model_t model, int64_t B, int64_t ld, const float* q, const float* qd,
                         const float* tau, const float* qdd, const float* dq, const float* dqd, const float* dtau,
                         float* dqdd, void* stream) {
  (void)tau;  // evaluated at the saved forward result qdd = ABA(q, qd, tau)
  FRAX_TRY(check_batch(model, B, ld, "frax_aba_jvp"));
  if (B == 0) return ok();
  FRAX_TRY(need(q, "frax_aba_jvp", "q"));
  FRAX_TRY(need(qd, "frax_aba_jvp", "qd"));
  FRAX_TRY(need(qdd, "frax_aba_jvp", "qdd"));
  FRAX_TRY(need(dq, "frax_aba_jvp", "dq"));
  FRAX_TRY(need(dqd, "frax_aba_jvp", "dqd"));
  FRAX_TRY(need(dqdd, "frax_aba_jvp", "dqdd"));
  frax::OpArgs a;
  a.B = B; a.ld = ld; a.q = q; a.qd = qd; a.qdd = qdd; a.in_dq = dq; a.in_dqd = dqd; a.in_dx = dtau;
  a.out0 = dqdd; a.stream = static_cast<cudaStream_t>(stream);
  return dispatch(model, frax::kOpAbaJvp, a, "frax_aba_jvp");
}

frax_status frax_osc(frax_model_t model, int task_body, int64_t B, int64_t ld, const float* q, const float* qd,
                     const float* xdd_des, float* tau, float* Lambda, void* stream) {
  FRAX_TRY(check_batch(model, B, ld, "frax_osc"));
  const frax::HostModel& m = model->m;
  if (task_body < 0 || task_body >= m.nb)
    return fail(FRAX_EINVAL, "frax_osc: task_body out of range");
  int path_dofs = m.free_root ? 5 : 0;
  for (uint64_t x = m.anc[task_body]; x; x &= x - 1) ++path_dofs;
  if (path_dofs < 6)
    return fail(FRAX_EINVAL, "frax_osc: fewer than 6 dofs move the task body; its 6-D task inertia is singular");
  if (B == 0) return ok();
  FRAX_TRY(need(q, "frax_osc", "q"));
  FRAX_TRY(need(qd, "frax_osc", "qd"));
  FRAX_TRY(need(xdd_des, "frax_osc", "xdd_des"));
  FRAX_TRY(need(tau, "frax_osc", "tau"));
  frax::OpArgs a;
  a.B = B; a.ld = ld; a.q = q; a.qd = qd; a.in_xdd = xdd_des; a.out0 = tau; a.out1 = Lambda;
  a.frames.n = 1; a.frames.body[0] = task_body;
  a.stream = static_cast<cudaStream_t>(stream);
  return dispatch(model, frax::kOpOsc, a, "frax_osc");
}

}  // extern "C"
