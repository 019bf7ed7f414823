/*
 * frax.h — C ABI of the GB300 batched rigid-body kinematics/dynamics library.
 *
 * The operations are those the paper states its problem with (Sec. II):
 * forward kinematics FK(q) -> ^0T_i, frame Jacobians, inverse dynamics
 * (Eq. 1, tau = M qdd + c + g, no external force), the joint-space mass
 * matrix M (Algorithm 2's result) with its tree-sparse factorisation
 * M = L^T D L (the Cholesky-style solve of the Sec. VI footnote), and forward
 * dynamics (Eq. 2, qdd = M^-1 (tau - c - g)) by the articulated-body
 * algorithm, plus vector-Jacobian products of Eq. 1 and Eq. 2 (the analytic
 * derivatives Sec. VI lists as future work).
 *
 * Conventions
 *  - Spatial vectors are [angular; linear]. Body frames sit after their joint:
 *    ^parent T_i = placement_i * joint_i(q_i).
 *  - Gravity g (world) enters as the base acceleration a_0 = [0; -g], so tau
 *    includes the gravity term g(q) of Eq. 1.
 *  - A free-flyer joint (body 0 only) has 7 q entries [p (3), quat (x,y,z,w)]
 *    and 6 velocity entries, the body-frame twist [w_b; v_b]; qdd is its time
 *    derivative. Revolute joints have one entry each.
 *  - Batched arrays are FP32, structure-of-arrays, entry-major: element
 *    (entry k, instance b) lives at ptr[k * ld + b], B <= ld < 2^30 (a
 *    larger ld is an argument error). All batched pointers are DEVICE
 *    pointers, caller-owned, 4-byte aligned.
 *  - Calls are asynchronous on `stream` (a cudaStream_t passed as void*,
 *    NULL = legacy default stream) and never synchronise. Argument errors are
 *    reported before anything is launched. B == 0 is a no-op returning
 *    FRAX_OK. Outputs are undefined after an error.
 *  - The library never allocates device memory in these calls; the model
 *    travels to the GPU inside each launch's parameter block.
 *  - Thread safety: a model handle may be used from several threads at once;
 *    frax_last_error() is thread-local.
 */
#ifndef FRAX_H
#define FRAX_H

#include <stdint.h>

#if defined(__GNUC__)
#define FRAX_API __attribute__((visibility("default")))
#else
#define FRAX_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct frax_model_s* frax_model_t;

typedef enum {
  FRAX_OK = 0,
  FRAX_EINVAL = 1,    /* bad argument; frax_last_error() says which        */
  FRAX_ECUDA = 2,     /* a CUDA runtime call failed                         */
  FRAX_ENOMEM = 3,    /* host or device allocation failed / budget exceeded */
  FRAX_ETIMEOUT = 4,  /* a bounded device or host wait ran out              */
  FRAX_EBUSY = 5,     /* resource still has work in flight                  */
  FRAX_EINTERNAL = 6
} frax_status;

enum { FRAX_JOINT_REVOLUTE = 0, FRAX_JOINT_FREE = 1 };
enum { FRAX_MAX_BODIES = 64, FRAX_MAX_FRAMES = 8 };

/*
 * frax_model_create — build a model from a parent array (topological:
 * parent[i] < i, -1 = world; the ancestor structure U of Sec. III), joint
 * types, joint axes, joint placements and body inertias (Table III's S and I).
 * Host-only: validates, derives the tree structure, and packs an FP32 image
 * from the FP64 inputs. No CUDA call is made.
 *   n_bodies    1..FRAX_MAX_BODIES
 *   parent      [n] int32, parent[i] in [-1, i-1]
 *   joint_type  [n] int32, FRAX_JOINT_REVOLUTE, or FRAX_JOINT_FREE for body 0
 *               (whose parent must be -1)
 *   axis        [n*3] unit joint axis in the joint frame (ignored for FREE)
 *   placement   [n*12] joint frame in the parent body frame: R (row-major,
 *               joint->parent, orthonormal) then p
 *   inertia     [n*10] mass m > 0, COM c (3, body frame), rotational inertia
 *               about the COM (xx, yy, zz, xy, xz, yz), positive definite
 *   gravity     [3] world gravity, e.g. {0, 0, -9.81}
 *   out         receives the handle (owned by the caller; frax_model_destroy)
 * Errors: FRAX_EINVAL with a message naming the offending body.
 */
FRAX_API frax_status frax_model_create(int n_bodies, const int32_t* parent, const int32_t* joint_type,
                              const double* axis, const double* placement, const double* inertia,
                              const double* gravity, frax_model_t* out);
FRAX_API frax_status frax_model_destroy(frax_model_t model);
/* nq, nv, n_bodies of the model (any pointer may be NULL). */
FRAX_API frax_status frax_model_dims(frax_model_t model, int* nq, int* nv, int* n_bodies);
/* Kernel family the model dispatches to: 0 = 7-body serial chain (thread
 * per instance, topology compiled in), 1 = general tree (thread per
 * instance, segment sweeps). */
FRAX_API frax_status frax_model_kind(frax_model_t model, int* kind);
/* How the kernels of a general tree of up to 32 bodies spread one instance
 * over threads (the 7-body chain and larger trees always run one thread per
 * instance). FRAX_TREE_PATH_THREAD: one thread per instance, the segment
 * sweeps. FRAX_TREE_PATH_LANE_GROUP: four lanes of a warp per instance, each
 * walking its own branches of the tree (Sec. III-A's parallelism within one
 * instance), for the ops that have such kernels (frax_fk, frax_jacobian,
 * frax_rnea, frax_crba, frax_aba, frax_aba_articulated, frax_rnea_vjp,
 * frax_aba_vjp); other ops run one thread per instance.
 * FRAX_TREE_PATH_AUTO (the default): the lane groups while the batch fits
 * one resident wave of the op's lane-group kernel on the current device (a
 * few thousand instances, fewer for ops with more state per instance), where
 * one thread per instance would leave most of the GPU idle; one thread per
 * instance above. Results agree within FP32 rounding (sums at a branch body
 * are added in another order). FRAX_EINVAL for another value. Not
 * thread-safe against concurrent calls on the same model. */
enum { FRAX_TREE_PATH_AUTO = 0, FRAX_TREE_PATH_THREAD = 1, FRAX_TREE_PATH_LANE_GROUP = 2 };
FRAX_API frax_status frax_model_set_tree_path(frax_model_t model, int path);

/*
 * frax_fk — forward kinematics (Sec. II): ^0T_i(q) of every body.
 *   q     [nq][ld] in
 *   pose  [n_bodies*12][ld] out: per body R (row-major 9) then p (3), world
 */
FRAX_API frax_status frax_fk(frax_model_t model, int64_t B, int64_t ld, const float* q, float* pose,
                    void* stream);

/*
 * frax_fk_scan — frax_fk for serial chains (parent[i] = i - 1) as a parallel
 * prefix product over SE(3), one warp per instance (the associative scan
 * that replaces the FK loop for serial chains, Sec. III-A): depth 7 instead
 * of n_bodies sequential compositions. For small batches of long chains;
 * frax_fk does less work per instance and is faster for large batches.
 * FRAX_EINVAL for a model that is not a serial chain. Same layout as frax_fk.
 */
FRAX_API frax_status frax_fk_scan(frax_model_t model, int64_t B, int64_t ld, const float* q, float* pose,
                                  void* stream);

/*
 * frax_jacobian — geometric Jacobians of body frames (Sec. IV, "Jacobians"),
 * fused with forward kinematics. J maps qd to [omega (world); d/dt p_k
 * (world)] of frame body k's origin; columns of non-ancestor joints are 0.
 *   n_frames    1..FRAX_MAX_FRAMES; frame_body [n_frames] HOST int32 bodies
 *   pose        [n_bodies*12][ld] out, or NULL
 *   J           [n_frames*6*nv][ld] out, entry (f, r, c) at (f*6 + r)*nv + c
 */
FRAX_API frax_status frax_jacobian(frax_model_t model, int64_t B, int64_t ld, const float* q, int n_frames,
                          const int32_t* frame_body, float* pose, float* J, void* stream);

/*
 * frax_rnea — inverse dynamics, Eq. 1 with f = 0 (Algorithm 1's result):
 * tau = M(q) qdd + c(q, qd) + g(q), by the recursive Newton-Euler algorithm.
 *   q [nq][ld], qd [nv][ld], qdd [nv][ld] in (qdd == NULL gives the bias
 *   forces c + g); tau [nv][ld] out.
 */
FRAX_API frax_status frax_rnea(frax_model_t model, int64_t B, int64_t ld, const float* q, const float* qd,
                      const float* qdd, float* tau, void* stream);

/*
 * frax_crba — the mass matrix M(q) (Algorithm 2's result) by the
 * composite-rigid-body algorithm, and optionally its factorisation
 * M = L^T D L (L unit lower triangular, zero fill-in in the ancestor
 * pattern), the Cholesky-style factor of the Sec. VI footnote.
 *   q  [nq][ld] in
 *   M  [nv*nv][ld] out, row-major, full (symmetric); may be NULL if LD given
 *   LD [nv*(nv+1)/2][ld] out or NULL: packed lower triangle row-major,
 *      entry (i, j<=i) at i*(i+1)/2 + j; D_i on the diagonal, L_ij below.
 */
FRAX_API frax_status frax_crba(frax_model_t model, int64_t B, int64_t ld, const float* q, float* M,
                      float* LD, void* stream);

/*
 * frax_aba — forward dynamics, Eq. 2 with f = 0: qdd = M^-1 (tau - c - g),
 * by the articulated-body algorithm (O(n); named future work in Sec. VI);
 * for 7-body chains through the mass-matrix factor instead (the Cholesky-
 * style solve of the Sec. VI footnote), cheaper at that size.
 *   q [nq][ld], qd [nv][ld], tau [nv][ld] in; qdd [nv][ld] out.
 */
FRAX_API frax_status frax_aba(frax_model_t model, int64_t B, int64_t ld, const float* q, const float* qd,
                     const float* tau, float* qdd, void* stream);

/*
 * frax_aba_articulated — the same forward dynamics (Eq. 2 with f = 0),
 * always by the O(n) articulated-body algorithm: a velocity sweep outward,
 * articulated inertias and bias forces inward, accelerations outward. For
 * trees this is what frax_aba runs; for 7-body chains (where frax_aba solves
 * through the mass-matrix factor) it runs the unrolled articulated-body
 * sweeps. Arguments, layout and errors as frax_aba.
 */
FRAX_API frax_status frax_aba_articulated(frax_model_t model, int64_t B, int64_t ld, const float* q,
                                          const float* qd, const float* tau, float* qdd, void* stream);

/*
 * frax_rnea_vjp — reverse-mode derivative of Eq. 1 (analytic RNEA
 * derivatives, Sec. VI future work). Given gbar (adjoint of tau):
 *   qbar   = (dtau/dq)^T gbar     [nq][ld] (ambient layout: a free-flyer
 *            root gets R v_bar in its position slots and 2 Q(quat) w_bar in
 *            its quaternion slots, tangent to the unit sphere)
 *   qdbar  = (dtau/dqd)^T gbar    [nv][ld]
 *   qddbar = M gbar               [nv][ld]  (may be NULL)
 * Spatial velocities are recomputed inside the call, never stored.
 */
FRAX_API frax_status frax_rnea_vjp(frax_model_t model, int64_t B, int64_t ld, const float* q,
                          const float* qd, const float* qdd, const float* gbar, float* qbar,
                          float* qdbar, float* qddbar, void* stream);

/*
 * frax_aba_vjp — reverse-mode derivative of Eq. 2 at qdd = ABA(q, qd, tau)
 * (qdd is passed in, as saved by the forward call). With w = M^-1 gbar:
 *   taubar = w, qbar = -(dtau/dq)^T w (ambient layout), qdbar = -(dtau/dqd)^T w.
 * Any output may be NULL (not all three): it is not written. For a 7-body
 * serial chain a NULL taubar runs the one-launch form, a non-NULL one the
 * factor solve into taubar followed by the adjoint sweep (two launches).
 */
FRAX_API frax_status frax_aba_vjp(frax_model_t model, int64_t B, int64_t ld, const float* q,
                         const float* qd, const float* tau, const float* qdd, const float* gbar,
                         float* qbar, float* qdbar, float* taubar, void* stream);

/*
 * Forward-mode derivatives (JVPs): the directional derivatives jax.jvp
 * returns on FK and on Eq. 1 and 2 (Sec. IV-A), as tangent recursions run
 * beside the value recursions. Directions are tangent vectors (nv rows): a
 * revolute entry is the angle's rate, a free-flyer root's six entries
 * [dw; dv] perturb its pose as T * Exp([dw; dv]) (body frame).
 *
 * frax_fk_jvp — the motion of each frame body along dq, [omega; p_dot] in
 *   world coordinates (J dq without forming J).
 *   q [nq][ld], dq [nv][ld] in; n_frames 1..8, frame_body HOST int32;
 *   dpose [n_frames*6][ld] out.
 * frax_rnea_jvp — tau = RNEA(q, qd, qdd) and its derivative along
 *   (dq, dqd, dqdd). qdd or dqdd NULL: zero. tau may be NULL.
 * frax_aba_jvp — the derivative of qdd = ABA(q, qd, tau) along
 *   (dq, dqd, dtau), evaluated at the saved forward result qdd (tau itself
 *   is not read): M dqdd = dtau - dRNEA(q, qd, qdd)[dq, dqd, 0]. dtau NULL:
 *   zero. dqdd [nv][ld] out.
 */
FRAX_API frax_status frax_fk_jvp(frax_model_t model, int64_t B, int64_t ld, const float* q, const float* dq,
                                 int n_frames, const int32_t* frame_body, float* dpose, void* stream);
FRAX_API frax_status frax_rnea_jvp(frax_model_t model, int64_t B, int64_t ld, const float* q, const float* qd,
                                   const float* qdd, const float* dq, const float* dqd, const float* dqdd,
                                   float* tau, float* dtau, void* stream);
FRAX_API frax_status frax_aba_jvp(frax_model_t model, int64_t B, int64_t ld, const float* q, const float* qd,
                                  const float* tau, const float* qdd, const float* dq, const float* dqd,
                                  const float* dtau, float* dqdd, void* stream);

/*
 * frax_ltdl_solve — x = M^-1 b from the packed factor M = L^T D L that
 * frax_crba writes (the Cholesky-based solve the paper's Sec. VI footnote
 * recommends over inverting M): L^T y = b, then L x = D^-1 y, walking only
 * the dof-parent chains (L is zero outside the ancestor pattern).
 *   LD [nv*(nv+1)/2][ld], b [nv][ld] in; x [nv][ld] out (must not alias b).
 */
FRAX_API frax_status frax_ltdl_solve(frax_model_t model, int64_t B, int64_t ld, const float* LD, const float* b,
                                     float* x, void* stream);

/*
 * frax_ltdl_inverse — M^-1 (dense, symmetric, row-major nv x nv) from the
 * same factor, one sparse solve per unit vector (the direct inversion of the
 * mass matrix listed as future work in Sec. VI).
 *   LD [nv*(nv+1)/2][ld] in; Minv [nv*nv][ld] out.
 */
FRAX_API frax_status frax_ltdl_inverse(frax_model_t model, int64_t B, int64_t ld, const float* LD, float* Minv,
                                       void* stream);

/*
 * frax_rnea_ext / frax_aba_ext — inverse and forward dynamics with external
 * forces on the bodies (Eq. 1 and 2 with J^T f; Algorithm 1's ^0F_ext):
 *   tau = M qdd + c + g - sum_i J_i^T F_ext,i
 *   qdd = M^-1 (tau - c - g + sum_i J_i^T F_ext,i)
 * fext [6*n_bodies][ld] in: entry (i, r) at 6*i + r, the spatial force that
 * the environment applies to body i in root-frame Pluecker coordinates,
 * [moment about the root (world) origin; force], as Algorithm 1 takes it and
 * subtracts it. A point force f at world point c on body i is [c x f; f];
 * rows of bodies without forces must be zero. Eq. 1's f is the force the
 * robot applies, -F_ext.
 *   frax_rnea_ext: q, qd, qdd (NULL: zero), fext in; tau [nv][ld] out.
 *   frax_aba_ext:  q, qd, tau, fext in; qdd [nv][ld] out.
 */
FRAX_API frax_status frax_rnea_ext(frax_model_t model, int64_t B, int64_t ld, const float* q, const float* qd,
                                   const float* qdd, const float* fext, float* tau, void* stream);
FRAX_API frax_status frax_aba_ext(frax_model_t model, int64_t B, int64_t ld, const float* q, const float* qd,
                                  const float* tau, const float* fext, float* qdd, void* stream);

/*
 * frax_osc — operational-space control of one task body (the inverse-dynamics
 * controller of Sec. V, Table II, built from M, J, c and g):
 *   tau = J^T Lambda (xdd_des - Jdot qd) + c + g,   Lambda = (J M^-1 J^T)^-1
 * with J the world-aligned Jacobian of the task body's origin (the rows of
 * frax_jacobian), without a null-space term. One fused kernel: Lambda^-1
 * from the articulated-body inertias along the path to the task body, a 6x6
 * solve, and one RNEA pass that adds J^T f; M is never formed.
 *   task_body  0..n_bodies-1; at least 6 dofs must move it, else FRAX_EINVAL
 *              (the 6-D task inertia would be singular)
 *   q [nq][ld], qd [nv][ld], xdd_des [6][ld] ([omega_dot; p_ddot] of the
 *   task body's origin, world coordinates) in; tau [nv][ld] out;
 *   Lambda [36][ld] out, row-major world-aligned, or NULL to skip it.
 * Near a kinematic singularity Lambda grows without bound; no per-instance
 * check is made.
 */
FRAX_API frax_status frax_osc(frax_model_t model, int task_body, int64_t B, int64_t ld, const float* q,
                              const float* qd, const float* xdd_des, float* tau, float* Lambda, void* stream);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of dynamics queries for many robots. The
 * paper has no serving layer; this is the batched evaluation of Sec. III-B
 * ("thousands of parallel instances") turned into a request loop.
 *
 * A server owns one device slab of `budget_bytes` (the HBM budget every
 * request's inputs and outputs are carved from), a ring of request
 * descriptors in device memory, completion flags in mapped host memory, and
 * a persistent kernel (one or two CTAs per SM) that claims 128-instance
 * tiles of any published request as soon as it appears, so requests that
 * arrive while others run share the GPU. Every device wait is bounded: the
 * kernel exits after `idle_exit_ms` without work and is relaunched by the
 * next submit / wait call. Host buffers are SoA [rows][B] (ld = B); inputs
 * are copied before submit returns.
 *
 * ops and their arrays (rows):
 *   FRAX_OP_RNEA       in q[nq], qd[nv], qdd[nv]          out tau[nv]
 *   FRAX_OP_CRBA       in q[nq]                           out M[nv*nv]
 *   FRAX_OP_ABA        in q[nq], qd[nv], tau[nv]          out qdd[nv]
 *   FRAX_OP_RNEA_GRAD  in q[nq], qd[nv], qdd[nv], gbar[nv] out qbar[nq], qdbar[nv], qddbar[nv]
 * ---------------------------------------------------------------------- */
typedef struct frax_server_s* frax_server_t;
enum { FRAX_OP_RNEA = 0, FRAX_OP_CRBA = 1, FRAX_OP_ABA = 2, FRAX_OP_RNEA_GRAD = 3 };
enum { FRAX_SERVER_RING = 1024, FRAX_SERVER_MAX_MODELS = 64 };

typedef struct {
  int64_t budget_bytes, bytes_in_use;
  int64_t submitted, completed, in_flight;
  int64_t kernel_launches;   /* persistent-kernel (re)launches so far     */
  int32_t device_status;     /* 0, or the first error the kernel recorded */
  int32_t resident_ctas;
} frax_server_info_t;

/* Allocates the slab, ring and flags on the current CUDA device (the only
 * allocations the server makes). FRAX_ENOMEM if the slab does not fit. */
FRAX_API frax_status frax_server_create(int64_t budget_bytes, double idle_exit_ms, frax_server_t* out);
/* Copies the model's image to the device model table; returns its id. */
FRAX_API frax_status frax_server_add_model(frax_server_t srv, frax_model_t model, int* model_id);
/* Admits a request if slab space and a ring slot are free: FRAX_EBUSY if not
 * now (retry after collecting), FRAX_ENOMEM if it can never fit. */
FRAX_API frax_status frax_server_submit(frax_server_t srv, int model_id, int op, int64_t B,
                                        const float* const* inputs, int64_t* request);
/* done = 1 once every tile of the request has finished. */
FRAX_API frax_status frax_server_poll(frax_server_t srv, int64_t request, int* done);
/* Waits (host side, bounded) until some in-flight request completes;
 * FRAX_ETIMEOUT if none does within timeout_ms. */
FRAX_API frax_status frax_server_wait_any(frax_server_t srv, double timeout_ms, int64_t* request);
/* Copies a completed request's outputs to host arrays, frees its slab space
 * and ring slot, and reports its latency (submit -> completion seen). */
FRAX_API frax_status frax_server_collect(frax_server_t srv, int64_t request, float* const* outputs,
                                         double* latency_us);
FRAX_API frax_status frax_server_info(frax_server_t srv, frax_server_info_t* info);
/* Stops the kernel (bounded wait) and frees everything. FRAX_EBUSY if
 * requests are still in flight and `force` is 0; FRAX_ETIMEOUT if the
 * kernel did not stop within timeout_ms (resources are then leaked, not
 * freed under a running kernel). */
FRAX_API frax_status frax_server_destroy(frax_server_t srv, int force, double timeout_ms);
/* Replays a request trace: request k (model_id[k], op[k], B[k], host inputs
 * inputs[4k .. 4k+3]) is submitted at arrival_us[k] after the call starts
 * (later if the budget or ring is full); a second host thread collects
 * completions, copies outputs to outputs[3k .. 3k+2] (outputs may be NULL)
 * and writes latency_us[k] = completion seen - arrival. Used to measure
 * latency under a given arrival process without a scripting layer in the
 * loop. FRAX_ETIMEOUT if the whole trace is not done within timeout_ms. */
FRAX_API frax_status frax_server_replay(frax_server_t srv, int n, const int* model_id, const int* op,
                                        const int64_t* B, const float* const* inputs, const double* arrival_us,
                                        float* const* outputs, double* latency_us, double timeout_ms);

/* ------------------------------------------------------------------------
 * frax_serve_batch_noalloc — one launch that evaluates a mixed batch of
 * requests (different robots and ops, each with its own instance count) and
 * allocates no memory at all. The paper has no counterpart; this exists for
 * callers that may not allocate device memory: real-time control loops
 * (cudaMalloc can block for an unbounded time and synchronise the device),
 * and code running inside a framework that has already reserved nearly all
 * of HBM for its own pool. It is the serving kernel's tile loop without the
 * server: the caller passes device input and output buffers per request
 * (SoA [rows][B], ld = B; arrays as listed for the FRAX_OP_* ops above).
 *
 * Scratch: a fixed device array inside the library (about 165 KB: up to
 * FRAX_NOALLOC_MAX_REQUESTS descriptors and FRAX_NOALLOC_MAX_MODELS model
 * images) that every GPU loading the library keeps until the process exits.
 * Larger batches are rejected with FRAX_EINVAL. All calls on a device share
 * it; each call rewrites what it uses and clears the tile counter first, so
 * calls ordered on one stream are correct, but calls whose kernels overlap
 * (unordered streams) race on it. The first call on each device looks up the
 * array's address (cudaGetSymbolAddress) and caches it: make that first call
 * before any stream capture. The kernel runs asynchronously on `stream`, but
 * the descriptors and model images are copied from a pageable host buffer,
 * so the call may block the host until the stream's earlier work is done: a
 * control loop that must never block should order its calls accordingly.
 * While `stream` is being captured the call returns FRAX_EINVAL and enqueues
 * nothing (a captured copy would read the staging buffer at replay time).
 * ---------------------------------------------------------------------- */
enum { FRAX_NOALLOC_MAX_REQUESTS = 256, FRAX_NOALLOC_MAX_MODELS = 16 };
typedef struct {
  frax_model_t model;
  int op;             /* FRAX_OP_RNEA, _CRBA, _ABA or _RNEA_GRAD */
  int64_t B;          /* instances, 0 <= B < 2^30 (0 allowed)    */
  const float* in[4]; /* device inputs, unused entries NULL      */
  float* out[3];      /* device outputs, unused entries NULL     */
} frax_batch_request_t;
FRAX_API frax_status frax_serve_batch_noalloc(const frax_batch_request_t* reqs, int n_reqs, void* stream);

/* ------------------------------------------------------------------------
 * frax_debug_inject_fault — test support for the server's error paths (no
 * counterpart in the paper). Arms one host-side injection point: the
 * (after+1)-th time the library reaches it, the host allocation or CUDA call
 * there is skipped and treated as failed, once; the public call then returns
 * the error it documents (FRAX_ENOMEM or FRAX_ECUDA) and releases what it
 * had taken. Nothing is injected on the GPU. Points: FRAX_FAULT_SERVER_ALLOC
 * (frax_server_create's host struct), FRAX_FAULT_SLAB_HOST (its pinned host
 * mirror of the slab), FRAX_FAULT_SUBMIT_INPUT (frax_server_submit's input
 * copy), FRAX_FAULT_SUBMIT_PUBLISH (its descriptor copy),
 * FRAX_FAULT_COLLECT_COPY (frax_server_collect's output copy);
 * FRAX_FAULT_NONE disarms. Returns FRAX_EINVAL unless the process was
 * started with FRAX_FAULT_INJECTION=1 in its environment.
 * ---------------------------------------------------------------------- */
enum { FRAX_FAULT_NONE = 0, FRAX_FAULT_SERVER_ALLOC = 1, FRAX_FAULT_SLAB_HOST = 2, FRAX_FAULT_SUBMIT_INPUT = 3,
       FRAX_FAULT_SUBMIT_PUBLISH = 4, FRAX_FAULT_COLLECT_COPY = 5 };
FRAX_API frax_status frax_debug_inject_fault(int point, int after);

/* ------------------------------------------------------------------------
 * frax_fp32_probe — measurement support (no counterpart in the paper):
 * launches `blocks` blocks of 256 threads that each run 8 independent chains
 * of `iters` dependent FP32 fused multiply-adds, scalar (packed = 0) or in
 * the two-lane packed form (packed = 1), and store one float per thread
 * into `sink` (device, at least blocks * 256 floats). *flops (may be NULL)
 * receives the FP32 operations the launch performs (an FMA counts 2), so
 * flops / (launch time) is the FP32 rate this GPU attains. Asynchronous on
 * `stream`; FRAX_EINVAL on bad sizes.
 * ---------------------------------------------------------------------- */
FRAX_API frax_status frax_fp32_probe(int packed, int blocks, int iters, float* sink, double* flops, void* stream);

/* Thread-local description of the last error on this thread ("" if none). */
FRAX_API const char* frax_last_error(void);

/* Library version string. */
FRAX_API const char* frax_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FRAX_H */
