// Serving: a persistent kernel that continuously batches dynamics requests
// for many robots. Requests are carved from one HBM slab (admission by
// budget), described in a device ring, and split into 128-instance tiles.
// Each resident CTA claims the next published tile with a CAS on one global
// counter, finds its request, runs the op for its 128 instances (the same
// per-instance device code as the batched kernels) and, as the last tile of
// a request finishes, raises the request's completion flag in mapped host
// memory. Every device wait is bounded: a CTA that sees no work for
// idle_exit_ms returns; the host relaunches the kernel when work is pending
// and it is not running.
#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fault.h"
#include "handles.h"
#include "seg.cuh"

namespace frax {
namespace {

constexpr int kRing = FRAX_SERVER_RING;
constexpr int kMaxModels = FRAX_SERVER_MAX_MODELS;
constexpr int kTile = 128;
constexpr int64_t kAlign = 256;

enum ServeKind { kServeChain7 = 0, kServeTree = 1, kServeTreeFree = 2 };
enum DeviceError { kDevOk = 0, kDevBadOp = 1, kDevLookup = 2 };

struct ReqDesc {
  long long tile_begin, tile_end;  // global tile range of the request
  long long B;
  long long seq;                   // request number
  int model_id, op, kind, slot;
  unsigned long long in_off[4], out_off[3];
};

struct ServeCtl {
  unsigned long long next_tile;        // tiles claimed so far (monotonic)
  unsigned long long tiles_published;  // tiles whose request is visible
  long long oldest;                    // no claimable tile belongs to a request older than this
  unsigned long long last_claim_ns;    // globaltimer of the latest claim by any CTA
  unsigned int stop;                   // set by the host to end the kernel
  unsigned int pad;
  unsigned int done[kRing];            // finished tiles of the request in each slot
};

// What every submit publishes in one copy: the new tile count and the oldest
// request still in flight (adjacent fields of ServeCtl). Both only grow, so
// the kernel may read them separately.
struct PubStage {
  unsigned long long tiles_published;
  long long oldest;
};
static_assert(offsetof(ServeCtl, oldest) == offsetof(ServeCtl, tiles_published) + 8, "PubStage layout");

struct ServeArgs {
  const ReqDesc* ring;
  ServeCtl* ctl;
  const ModelImage<64>* models;
  char* slab;
  unsigned long long* flags;  // mapped host memory: seq + 1 once done
  int* status;                // mapped host memory: first device error
  unsigned long long idle_ns;
  long long first_req;        // oldest request possibly owning unclaimed tiles
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <class U>
__device__ __forceinline__ U ld_volatile(const U* p) {
  return *reinterpret_cast<const volatile U*>(p);
}

// Chains of 7 run the unrolled chain code for the forward ops; every other
// case runs the segment code (the same device functions as the batched
// kernels, so a request's result does not depend on how it was served).
template <class T>
__device__ void serve_tile(const ModelImage<64>& M, const ReqDesc& d, char* slab, long long b) {
  const ColT<false> col{d.B, b};
  auto in = [&](int k) { return reinterpret_cast<const float*>(slab + d.in_off[k]); };
  auto out = [&](int k) { return reinterpret_cast<float*>(slab + d.out_off[k]); };
  if constexpr (T::kSeg) {
    switch (d.op) {
      case FRAX_OP_RNEA: rnea_seg<T>(M, in(0), in(1), in(2), out(0), col); break;
      case FRAX_OP_CRBA: crba_seg<T>(M, in(0), out(0), static_cast<float*>(nullptr), col); break;
      case FRAX_OP_ABA: {
        P3Local<T::NBMAX> P;
        aba_seg<T>(M, in(0), in(1), in(2), out(0), col, P);
        break;
      }
      case FRAX_OP_RNEA_GRAD: rnea_vjp_seg_one<T>(M, in(0), in(1), in(2), in(3), out(0), out(1), out(2), col); break;
      default: break;
    }
  } else {
    switch (d.op) {
      case FRAX_OP_RNEA: rnea_one<T>(M, in(0), in(1), in(2), out(0), col); break;
      case FRAX_OP_CRBA: crba_one<T>(M, in(0), out(0), static_cast<float*>(nullptr), col); break;
      case FRAX_OP_ABA: aba_one<T>(M, in(0), in(1), in(2), out(0), col); break;
      case FRAX_OP_RNEA_GRAD: serve_tile<SegTopo<64, false>>(M, d, slab, b); break;
      default: break;
    }
  }
}

__global__ void __launch_bounds__(kTile) k_serve(const ServeArgs a) {
  __shared__ ModelImage<64> model;
  __shared__ ReqDesc desc;
  __shared__ long long s_tile;
  long long hint = a.first_req;  // per-CTA request cursor (thread 0 only)
  while (true) {
    if (threadIdx.x == 0) {
      long long got = -1;
      const unsigned long long t0 = global_ns();
      while (true) {
        const unsigned long long pub = ld_volatile(&a.ctl->tiles_published);
        const unsigned long long cur = ld_volatile(&a.ctl->next_tile);
        if (cur < pub) {
          if (atomicCAS(&a.ctl->next_tile, cur, cur + 1) == cur) {
            got = static_cast<long long>(cur);
            atomicMax(&a.ctl->last_claim_ns, global_ns());
            break;
          }
          continue;
        }
        if (ld_volatile(&a.ctl->stop)) break;
        // Bounded idle wait, left together: a CTA leaves only once no CTA
        // has claimed a tile for idle_ns (and it has waited that long
        // itself), so under light load the pool does not shrink CTA by CTA.
        const unsigned long long now = global_ns();
        const unsigned long long last = max(t0, ld_volatile(&a.ctl->last_claim_ns));
        if (now > last && now - last > a.idle_ns) break;
        __nanosleep(500);
      }
      if (got >= 0) {
        // Find the request that owns tile `got`. Tile ranges grow with the
        // request number; the owner is still in flight, and it is neither
        // older than this CTA's last request (tiles are claimed in order) nor
        // than the oldest request in flight when the host last published.
        // Between that request and the newest one there are at most kRing
        // requests, none of whose ring slots has been reused, so one pass of
        // kRing + 1 entries finds the owner. A miss (a descriptor not yet
        // visible) is retried, bounded by idle_ns.
        const unsigned long long tl0 = global_ns();
        long long r = hint;
        bool found = false;
        while (true) {
          r = max(hint, ld_volatile(&a.ctl->oldest));
          for (int it = 0; it <= kRing; ++it, ++r) {
            const ReqDesc* rd = &a.ring[r % kRing];
            const long long seq = __ldcg(&rd->seq);
            if (seq == r && got >= __ldcg(&rd->tile_begin) && got < __ldcg(&rd->tile_end)) {
              found = true;
              break;
            }
          }
          if (found || global_ns() - tl0 > a.idle_ns) break;
          __nanosleep(1000);
        }
        if (!found) {
          atomicCAS(a.status, kDevOk, kDevLookup);
          __threadfence_system();
          got = -1;
        } else {
          hint = r;
          const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&a.ring[r % kRing]);
          unsigned long long* dst = reinterpret_cast<unsigned long long*>(&desc);
          for (int k = 0; k < int(sizeof(ReqDesc) / 8); ++k) dst[k] = __ldcg(src + k);
        }
      }
      s_tile = got;
    }
    __syncthreads();
    const long long t = s_tile;
    if (t < 0) return;
    // stage the request's model image in shared memory
    {
      const float4* src = reinterpret_cast<const float4*>(&a.models[desc.model_id]);
      float4* dst = reinterpret_cast<float4*>(&model);
      for (int k = threadIdx.x; k < int(sizeof(ModelImage<64>) / 16); k += kTile) dst[k] = __ldcg(src + k);
    }
    __syncthreads();
    const long long b = (t - desc.tile_begin) * kTile + threadIdx.x;
    if (b < desc.B) {
      if (desc.op < FRAX_OP_RNEA || desc.op > FRAX_OP_RNEA_GRAD) {
        if (threadIdx.x == 0) atomicCAS(a.status, kDevOk, kDevBadOp);
      } else if (desc.kind == kServeChain7) {
        serve_tile<ChainTopo<7>>(model, desc, a.slab, b);
      } else if (desc.kind == kServeTreeFree) {
        serve_tile<SegTopo<64, true>>(model, desc, a.slab, b);
      } else {
        serve_tile<SegTopo<64, false>>(model, desc, a.slab, b);
      }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned int ntiles = static_cast<unsigned int>(desc.tile_end - desc.tile_begin);
      const unsigned int prev = atomicAdd(&a.ctl->done[desc.slot], 1u);
      if (prev + 1 == ntiles) {
        a.ctl->done[desc.slot] = 0;
        __threadfence_system();
        *reinterpret_cast<volatile unsigned long long*>(&a.flags[desc.slot]) =
            static_cast<unsigned long long>(desc.seq) + 1ull;
        __threadfence_system();
      }
    }
    __syncthreads();
  }
}

int op_arrays(int op, int nq, int nv, int* in_rows, int* out_rows, int* nin, int* nout) {
  switch (op) {
    case FRAX_OP_RNEA:
      *nin = 3; in_rows[0] = nq; in_rows[1] = nv; in_rows[2] = nv;
      *nout = 1; out_rows[0] = nv;
      return 0;
    case FRAX_OP_CRBA:
      *nin = 1; in_rows[0] = nq;
      *nout = 1; out_rows[0] = nv * nv;
      return 0;
    case FRAX_OP_ABA:
      *nin = 3; in_rows[0] = nq; in_rows[1] = nv; in_rows[2] = nv;
      *nout = 1; out_rows[0] = nv;
      return 0;
    case FRAX_OP_RNEA_GRAD:
      *nin = 4; in_rows[0] = nq; in_rows[1] = nv; in_rows[2] = nv; in_rows[3] = nv;
      *nout = 3; out_rows[0] = nq; out_rows[1] = nv; out_rows[2] = nv;
      return 0;
    default:
      return -1;
  }
}

int64_t round_up(int64_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

}  // namespace
}  // namespace frax

using namespace frax;

struct frax_server_s {
  struct Req {
    int64_t seq = 0;
    int slot = 0, op = 0, model = 0, nin = 0, nout = 0;
    int64_t B = 0, off = 0, bytes = 0, ntiles = 0;
    int out_rows[3] = {0, 0, 0};
    int64_t out_off[3] = {0, 0, 0};
    std::chrono::steady_clock::time_point t0;
    bool done = false;
    bool collecting = false;
    int64_t in_bytes = 0, out_begin = 0, out_bytes = 0;
    double latency_us = 0;
  };
  std::mutex mu;         // the request table, slab allocator and counters
  std::mutex submit_mu;  // one submitter at a time (taken before mu)
  int device = 0;
  cudaStream_t kstream = nullptr, cstream = nullptr, dstream = nullptr;
  char* slab = nullptr;
  char* slab_h = nullptr;  // pinned host mirror of the slab: staging for copies
  int64_t budget = 0, in_use = 0;
  ReqDesc* ring = nullptr;
  ServeCtl* ctl = nullptr;
  ModelImage<64>* models = nullptr;
  unsigned long long* flags_h = nullptr;
  unsigned long long* flags_d = nullptr;
  int* status_h = nullptr;
  int* status_d = nullptr;
  ReqDesc* desc_stage = nullptr;          // pinned
  PubStage* pub_stage = nullptr;            // pinned, one per slot
  ModelImage<64>* model_stage = nullptr;    // pinned
  int n_models = 0;
  int model_kind[kMaxModels] = {};
  int model_nq[kMaxModels] = {};
  int model_nv[kMaxModels] = {};
  std::map<int64_t, int64_t> free_list;  // offset -> size
  std::map<int64_t, Req> inflight;
  int64_t slot_owner[kRing];
  bool slot_done[kRing];           // the slot's request has been seen complete
  int64_t scan_lo = 0;             // no request older than this is in flight and unseen
  std::deque<int64_t> done_fifo;   // requests seen complete, in the order seen
  std::chrono::steady_clock::time_point last_query{};  // wait_any's last kernel-state query
  int64_t next_seq = 0, tiles_total = 0;
  int64_t submitted = 0, completed = 0, launches = 0;
  int ctas = 0;
  double idle_ms = 50.0;
  bool kernel_ever = false;
};

namespace {

frax_status cuda_fail(const char* what, cudaError_t e) {
  return set_error(FRAX_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define SRV_CUDA(call)                                       \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(#call, e_);      \
  } while (0)

bool kernel_running(frax_server_s* s) {
  cudaError_t e = cudaStreamQuery(s->kstream);
  if (e == cudaErrorNotReady) return true;
  if (e != cudaSuccess) cudaGetLastError();
  return false;
}

// Relaunches the persistent kernel if work is pending and it is not running.
frax_status ensure_running(frax_server_s* s) {
  if (s->inflight.empty() || kernel_running(s)) return FRAX_OK;
  int64_t first = s->next_seq;
  for (auto& kv : s->inflight)
    if (!kv.second.done) first = std::min(first, kv.first);
  ServeArgs a;
  a.ring = s->ring;
  a.ctl = s->ctl;
  a.models = s->models;
  a.slab = s->slab;
  a.flags = s->flags_d;
  a.status = s->status_d;
  a.idle_ns = static_cast<unsigned long long>(s->idle_ms * 1e6);
  a.first_req = first;
  k_serve<<<s->ctas, kTile, 0, s->kstream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail("k_serve launch", e);
  s->launches++;
  s->kernel_ever = true;
  return FRAX_OK;
}

bool slab_alloc(frax_server_s* s, int64_t bytes, int64_t* off) {
  for (auto it = s->free_list.begin(); it != s->free_list.end(); ++it) {
    if (it->second >= bytes) {
      *off = it->first;
      int64_t rest = it->second - bytes;
      int64_t start = it->first + bytes;
      s->free_list.erase(it);
      if (rest > 0) s->free_list[start] = rest;
      s->in_use += bytes;
      return true;
    }
  }
  return false;
}

void slab_free(frax_server_s* s, int64_t off, int64_t bytes) {
  s->in_use -= bytes;
  auto it = s->free_list.emplace(off, bytes).first;
  auto nx = std::next(it);
  if (nx != s->free_list.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    s->free_list.erase(nx);
  }
  if (it != s->free_list.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      s->free_list.erase(it);
    }
  }
}

void release_all(frax_server_s* s) {
  if (s->slab) cudaFree(s->slab);
  if (s->slab_h) cudaFreeHost(s->slab_h);
  if (s->dstream) cudaStreamDestroy(s->dstream);
  if (s->ring) cudaFree(s->ring);
  if (s->ctl) cudaFree(s->ctl);
  if (s->models) cudaFree(s->models);
  if (s->flags_h) cudaFreeHost(s->flags_h);
  if (s->status_h) cudaFreeHost(s->status_h);
  if (s->desc_stage) cudaFreeHost(s->desc_stage);
  if (s->pub_stage) cudaFreeHost(s->pub_stage);
  if (s->model_stage) cudaFreeHost(s->model_stage);
  if (s->kstream) cudaStreamDestroy(s->kstream);
  if (s->cstream) cudaStreamDestroy(s->cstream);
}

// Marks requests whose completion flag is up; returns how many were new.
// Reads the completion flags of the requests in flight and not yet seen
// complete. Those lie in the sequence window [scan_lo, next_seq), at most
// kRing entries, read from flat per-slot arrays (no walk of the request map);
// each newly completed request is appended to done_fifo. Returns how many
// completed since the last scan.
int scan_flags(frax_server_s* s) {
  int n = 0;
  const auto now = std::chrono::steady_clock::now();
  for (int64_t q = s->scan_lo; q < s->next_seq; ++q) {
    const int slot = static_cast<int>(q % kRing);
    if (s->slot_owner[slot] != q || s->slot_done[slot]) continue;
    const volatile unsigned long long* f = s->flags_h + slot;
    if (*f != static_cast<unsigned long long>(q) + 1ull) continue;
    s->slot_done[slot] = true;
    auto it = s->inflight.find(q);
    if (it != s->inflight.end()) {
      it->second.done = true;
      it->second.latency_us = std::chrono::duration<double, std::micro>(now - it->second.t0).count();
    }
    s->done_fifo.push_back(q);
    s->completed++;
    ++n;
  }
  while (s->scan_lo < s->next_seq) {
    const int slot = static_cast<int>(s->scan_lo % kRing);
    if (s->slot_owner[slot] == s->scan_lo && !s->slot_done[slot]) break;
    ++s->scan_lo;
  }
  return n;
}

// The oldest request seen complete and neither collected nor being
// collected; entries at the front of done_fifo that were collected are
// dropped on the way.
bool first_uncollected(frax_server_s* s, int64_t* request) {
  while (!s->done_fifo.empty()) {
    auto it = s->inflight.find(s->done_fifo.front());
    if (it == s->inflight.end()) {
      s->done_fifo.pop_front();
      continue;
    }
    if (!it->second.collecting) {
      *request = it->first;
      return true;
    }
    break;
  }
  for (int64_t q : s->done_fifo) {  // the front one is being collected
    auto it = s->inflight.find(q);
    if (it != s->inflight.end() && !it->second.collecting) {
      *request = q;
      return true;
    }
  }
  return false;
}

}  // namespace

extern "C" {

frax_status frax_server_create(int64_t budget_bytes, double idle_exit_ms, frax_server_t* out) {
  if (!out) return set_error(FRAX_EINVAL, "frax_server_create: out is NULL");
  *out = nullptr;
  if (budget_bytes < kAlign) return set_error(FRAX_EINVAL, "frax_server_create: budget_bytes too small");
  if (!(idle_exit_ms > 0) || idle_exit_ms > 60000)
    return set_error(FRAX_EINVAL, "frax_server_create: idle_exit_ms must be in (0, 60000]");
  frax_server_s* s = fault_hit(kFaultServerAlloc) ? nullptr : new (std::nothrow) frax_server_s;
  if (!s) return set_error(FRAX_ENOMEM, "frax_server_create: out of host memory");
  s->budget = round_up(budget_bytes);
  s->idle_ms = idle_exit_ms;
  for (auto& o : s->slot_owner) o = -1;
  for (auto& d : s->slot_done) d = false;
  auto bail = [&](frax_status st) {
    release_all(s);
    delete s;
    return st;
  };
  cudaError_t e;
  if ((e = cudaGetDevice(&s->device)) != cudaSuccess) return bail(cuda_fail("cudaGetDevice", e));
  if ((e = cudaMalloc(&s->slab, s->budget)) != cudaSuccess) {
    cudaGetLastError();
    return bail(set_error(FRAX_ENOMEM, "frax_server_create: slab of budget_bytes does not fit on the device"));
  }
  if (fault_hit(kFaultSlabHost) || (e = cudaHostAlloc(&s->slab_h, s->budget, cudaHostAllocDefault)) != cudaSuccess) {
    cudaGetLastError();
    return bail(set_error(FRAX_ENOMEM, "frax_server_create: pinned host staging of budget_bytes failed"));
  }
  if ((e = cudaMalloc(&s->ring, sizeof(ReqDesc) * kRing)) != cudaSuccess) return bail(cuda_fail("cudaMalloc ring", e));
  if ((e = cudaMalloc(&s->ctl, sizeof(ServeCtl))) != cudaSuccess) return bail(cuda_fail("cudaMalloc ctl", e));
  if ((e = cudaMalloc(&s->models, sizeof(ModelImage<64>) * kMaxModels)) != cudaSuccess)
    return bail(cuda_fail("cudaMalloc models", e));
  if ((e = cudaMemset(s->ring, 0xff, sizeof(ReqDesc) * kRing)) != cudaSuccess) return bail(cuda_fail("memset", e));
  if ((e = cudaMemset(s->ctl, 0, sizeof(ServeCtl))) != cudaSuccess) return bail(cuda_fail("memset", e));
  if ((e = cudaHostAlloc(&s->flags_h, sizeof(unsigned long long) * kRing, cudaHostAllocMapped)) != cudaSuccess)
    return bail(cuda_fail("cudaHostAlloc flags", e));
  if ((e = cudaHostAlloc(&s->status_h, sizeof(int), cudaHostAllocMapped)) != cudaSuccess)
    return bail(cuda_fail("cudaHostAlloc status", e));
  if ((e = cudaHostAlloc(&s->desc_stage, sizeof(ReqDesc) * kRing, cudaHostAllocDefault)) != cudaSuccess)
    return bail(cuda_fail("cudaHostAlloc", e));
  if ((e = cudaHostAlloc(&s->pub_stage, sizeof(PubStage) * kRing, cudaHostAllocDefault)) != cudaSuccess)
    return bail(cuda_fail("cudaHostAlloc", e));
  if ((e = cudaHostAlloc(&s->model_stage, sizeof(ModelImage<64>), cudaHostAllocDefault)) != cudaSuccess)
    return bail(cuda_fail("cudaHostAlloc", e));
  std::memset(s->flags_h, 0, sizeof(unsigned long long) * kRing);
  *s->status_h = 0;
  if ((e = cudaHostGetDevicePointer(&s->flags_d, s->flags_h, 0)) != cudaSuccess) return bail(cuda_fail("map", e));
  if ((e = cudaHostGetDevicePointer(&s->status_d, s->status_h, 0)) != cudaSuccess) return bail(cuda_fail("map", e));
  if ((e = cudaStreamCreateWithFlags(&s->kstream, cudaStreamNonBlocking)) != cudaSuccess)
    return bail(cuda_fail("stream", e));
  if ((e = cudaStreamCreateWithFlags(&s->cstream, cudaStreamNonBlocking)) != cudaSuccess)
    return bail(cuda_fail("stream", e));
  if ((e = cudaStreamCreateWithFlags(&s->dstream, cudaStreamNonBlocking)) != cudaSuccess)
    return bail(cuda_fail("stream", e));
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_serve, kTile, 0);
  s->ctas = std::max(1, sms) * std::max(1, std::min(per_sm, 2));
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return bail(cuda_fail("sync", e));
  s->free_list[0] = s->budget;
  *out = s;
  return clear_error();
}

frax_status frax_server_add_model(frax_server_t s, frax_model_t model, int* model_id) {
  if (!s || !model || !model_id) return set_error(FRAX_EINVAL, "frax_server_add_model: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->n_models >= kMaxModels) return set_error(FRAX_ENOMEM, "frax_server_add_model: model table full");
  const HostModel& m = model->m;
  m.pack(s->model_stage);
  const int id = s->n_models;
  SRV_CUDA(cudaMemcpyAsync(s->models + id, s->model_stage, sizeof(ModelImage<64>), cudaMemcpyHostToDevice,
                           s->cstream));
  SRV_CUDA(cudaStreamSynchronize(s->cstream));
  s->model_kind[id] = m.kind == kKindChain ? kServeChain7 : (m.free_root ? kServeTreeFree : kServeTree);
  s->model_nq[id] = m.nq;
  s->model_nv[id] = m.nv;
  s->n_models++;
  *model_id = id;
  return clear_error();
}

frax_status frax_server_submit(frax_server_t s, int model_id, int op, int64_t B, const float* const* inputs,
                               int64_t* request) {
  if (!s || !request) return set_error(FRAX_EINVAL, "frax_server_submit: NULL argument");
  const auto t_arrive = std::chrono::steady_clock::now();
  // Submitters run one at a time (requests are published in sequence
  // order); the server lock is held only to reserve and to register, so the
  // collecting thread keeps seeing completions while the inputs are copied.
  std::lock_guard<std::mutex> sub(s->submit_mu);
  int in_rows[4], out_rows[3], nin, nout;
  int64_t in_bytes[4], out_bytes[3], total = 0, off = 0, seq = 0, tile0 = 0, oldest = 0;
  int kind = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (model_id < 0 || model_id >= s->n_models) return set_error(FRAX_EINVAL, "frax_server_submit: bad model_id");
    if (B < 1 || B > (int64_t(1) << 24)) return set_error(FRAX_EINVAL, "frax_server_submit: B must be in [1, 2^24]");
    if (op_arrays(op, s->model_nq[model_id], s->model_nv[model_id], in_rows, out_rows, &nin, &nout) != 0)
      return set_error(FRAX_EINVAL, "frax_server_submit: unknown op");
    if (!inputs) return set_error(FRAX_EINVAL, "frax_server_submit: inputs is NULL");
    for (int k = 0; k < nin; ++k)
      if (!inputs[k]) return set_error(FRAX_EINVAL, "frax_server_submit: an input array is NULL");
    for (int k = 0; k < nin; ++k) total += (in_bytes[k] = round_up(int64_t(in_rows[k]) * B * 4));
    for (int k = 0; k < nout; ++k) total += (out_bytes[k] = round_up(int64_t(out_rows[k]) * B * 4));
    if (total > s->budget) return set_error(FRAX_ENOMEM, "frax_server_submit: request exceeds the whole HBM budget");
    seq = s->next_seq;
    if (s->slot_owner[seq % kRing] >= 0) return set_error(FRAX_EBUSY, "frax_server_submit: request ring full");
    if (!slab_alloc(s, total, &off)) return set_error(FRAX_EBUSY, "frax_server_submit: HBM budget in use");
    tile0 = s->tiles_total;
    kind = s->model_kind[model_id];
    // the oldest request not yet collected (this one if none): a lower bound
    // on the owner of any tile the kernel can still claim (requests collected
    // before the count is published only make it more conservative)
    oldest = s->inflight.empty() ? seq : std::min(seq, s->inflight.begin()->first);
  }
  // The slab range and the ring slot are this request's: no other submitter
  // runs, and the slot stays free until the request is registered below.
  const int slot = static_cast<int>(seq % kRing);
  const int64_t ntiles = (B + kTile - 1) / kTile;
  ReqDesc& d = s->desc_stage[slot];
  d.tile_begin = tile0;
  d.tile_end = tile0 + ntiles;
  d.B = B;
  d.seq = seq;
  d.model_id = model_id;
  d.op = op;
  d.kind = kind;
  d.slot = slot;
  int64_t cur = off;
  for (int k = 0; k < 4; ++k) d.in_off[k] = 0;
  for (int k = 0; k < 3; ++k) d.out_off[k] = 0;
  for (int k = 0; k < nin; ++k) {  // the caller's buffers are free once this returns
    d.in_off[k] = cur;
    std::memcpy(s->slab_h + cur, inputs[k], size_t(in_rows[k]) * B * 4);
    cur += in_bytes[k];
  }
  frax_server_s::Req r;
  r.in_bytes = cur - off;
  r.out_begin = cur;
  r.out_bytes = off + total - cur;
  for (int k = 0; k < nout; ++k) {
    d.out_off[k] = cur;
    r.out_off[k] = cur;
    r.out_rows[k] = out_rows[k];
    cur += out_bytes[k];
  }
  // inputs, then the descriptor, then the published-tile count, in stream
  // order on one copy stream: the kernel can only see the count after both
  cudaError_t e = fault_hit(kFaultSubmitInputCopy)
                      ? cudaErrorUnknown
                      : cudaMemcpyAsync(s->slab + off, s->slab_h + off, r.in_bytes, cudaMemcpyHostToDevice,
                                        s->cstream);
  const char* what = "frax_server_submit: input copy";
  if (e == cudaSuccess) {
    what = "frax_server_submit: publish";
    s->pub_stage[slot].tiles_published = static_cast<unsigned long long>(tile0 + ntiles);
    s->pub_stage[slot].oldest = oldest;
    e = fault_hit(kFaultSubmitPublish)
            ? cudaErrorUnknown
            : cudaMemcpyAsync(s->ring + slot, &d, sizeof(ReqDesc), cudaMemcpyHostToDevice, s->cstream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&s->ctl->tiles_published, &s->pub_stage[slot], sizeof(PubStage), cudaMemcpyHostToDevice,
                          s->cstream);
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (e != cudaSuccess) {
    slab_free(s, off, total);
    return cuda_fail(what, e);
  }
  r.seq = seq;
  r.slot = slot;
  r.op = op;
  r.model = model_id;
  r.nin = nin;
  r.nout = nout;
  r.B = B;
  r.off = off;
  r.bytes = total;
  r.ntiles = ntiles;
  r.t0 = t_arrive;
  s->inflight[seq] = r;
  s->slot_owner[slot] = seq;
  s->slot_done[slot] = false;
  s->tiles_total += ntiles;
  s->next_seq++;
  s->submitted++;
  *request = seq;
  frax_status st = ensure_running(s);
  if (st != FRAX_OK) return st;
  return clear_error();
}

frax_status frax_server_poll(frax_server_t s, int64_t request, int* done) {
  if (!s || !done) return set_error(FRAX_EINVAL, "frax_server_poll: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->inflight.find(request);
  if (it == s->inflight.end()) return set_error(FRAX_EINVAL, "frax_server_poll: unknown request");
  scan_flags(s);
  if (*s->status_h) return set_error(FRAX_EINTERNAL, "frax_server_poll: device error " + std::to_string(*s->status_h));
  *done = it->second.done ? 1 : 0;
  if (!*done) {
    frax_status st = ensure_running(s);
    if (st != FRAX_OK) return st;
  }
  return clear_error();
}

frax_status frax_server_wait_any(frax_server_t s, double timeout_ms, int64_t* request) {
  if (!s || !request) return set_error(FRAX_EINVAL, "frax_server_wait_any: NULL argument");
  const auto t_end = std::chrono::steady_clock::now() + std::chrono::microseconds(int64_t(timeout_ms * 1e3));
  while (true) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (first_uncollected(s, request)) return clear_error();  // seen complete earlier
      if (s->inflight.empty()) return set_error(FRAX_EINVAL, "frax_server_wait_any: nothing in flight");
      if (scan_flags(s) > 0 && first_uncollected(s, request)) return clear_error();
      if (*s->status_h)
        return set_error(FRAX_EINTERNAL, "frax_server_wait_any: device error " + std::to_string(*s->status_h));
      // The kernel leaves only after idle_exit_ms without a claim and every
      // submit checks it, so while waiting its state is queried at most once
      // every 20 us (each query takes the driver's lock).
      const auto now = std::chrono::steady_clock::now();
      if (now - s->last_query > std::chrono::microseconds(20)) {
        s->last_query = now;
        frax_status st = ensure_running(s);
        if (st != FRAX_OK) return st;
      }
    }
    if (std::chrono::steady_clock::now() > t_end)
      return set_error(FRAX_ETIMEOUT, "frax_server_wait_any: no request completed within the timeout");
    std::this_thread::yield();
  }
}

frax_status frax_server_collect(frax_server_t s, int64_t request, float* const* outputs, double* latency_us) {
  if (!s) return set_error(FRAX_EINVAL, "frax_server_collect: NULL server");
  frax_server_s::Req r;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->inflight.find(request);
    if (it == s->inflight.end()) return set_error(FRAX_EINVAL, "frax_server_collect: unknown request");
    scan_flags(s);
    if (!it->second.done) return set_error(FRAX_EBUSY, "frax_server_collect: request not complete");
    if (it->second.collecting) return set_error(FRAX_EBUSY, "frax_server_collect: already being collected");
    it->second.collecting = true;
    r = it->second;
  }
  // the request's slab range stays reserved until it is freed below
  frax_status st = FRAX_OK;
  if (outputs && r.out_bytes > 0) {
    cudaError_t e = cudaMemcpyAsync(s->slab_h + r.out_begin, s->slab + r.out_begin, r.out_bytes,
                                    cudaMemcpyDeviceToHost, s->dstream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->dstream);
    if (e == cudaSuccess && fault_hit(kFaultCollectCopy)) e = cudaErrorUnknown;
    if (e != cudaSuccess) st = cuda_fail("frax_server_collect: output copy", e);
    for (int k = 0; k < r.nout && st == FRAX_OK; ++k)
      if (outputs[k]) std::memcpy(outputs[k], s->slab_h + r.out_off[k], size_t(r.out_rows[k]) * r.B * 4);
  }
  if (latency_us) *latency_us = r.latency_us;
  std::lock_guard<std::mutex> lk(s->mu);
  slab_free(s, r.off, r.bytes);
  s->slot_owner[r.slot] = -1;
  s->inflight.erase(request);
  return st == FRAX_OK ? clear_error() : st;
}

frax_status frax_server_info(frax_server_t s, frax_server_info_t* info) {
  if (!s || !info) return set_error(FRAX_EINVAL, "frax_server_info: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  scan_flags(s);
  info->budget_bytes = s->budget;
  info->bytes_in_use = s->in_use;
  info->submitted = s->submitted;
  info->completed = s->completed;
  info->in_flight = static_cast<int64_t>(s->inflight.size());
  info->kernel_launches = s->launches;
  info->device_status = *s->status_h;
  info->resident_ctas = s->ctas;
  return clear_error();
}

frax_status frax_server_destroy(frax_server_t s, int force, double timeout_ms) {
  if (!s) return clear_error();
  {
    std::lock_guard<std::mutex> sub(s->submit_mu);  // a submit under way finishes first
    std::lock_guard<std::mutex> lk(s->mu);
    scan_flags(s);
    bool pending = false;
    for (auto& kv : s->inflight) pending = pending || !kv.second.done;
    if (pending && !force) return set_error(FRAX_EBUSY, "frax_server_destroy: requests still in flight");
    static const unsigned int one = 1;
    cudaMemcpyAsync(&s->ctl->stop, &one, sizeof(one), cudaMemcpyHostToDevice, s->cstream);
    cudaStreamSynchronize(s->cstream);
  }
  const auto t_end = std::chrono::steady_clock::now() + std::chrono::microseconds(int64_t(timeout_ms * 1e3));
  while (kernel_running(s)) {
    if (std::chrono::steady_clock::now() > t_end)
      return set_error(FRAX_ETIMEOUT, "frax_server_destroy: kernel did not stop in time; resources kept");
    std::this_thread::sleep_for(std::chrono::microseconds(200));
  }
  release_all(s);
  delete s;
  return clear_error();
}

frax_status frax_server_replay(frax_server_t s, int n, const int* model_id, const int* op, const int64_t* B,
                               const float* const* inputs, const double* arrival_us, float* const* outputs,
                               double* latency_us, double timeout_ms) {
  if (!s || n < 0 || (n > 0 && (!model_id || !op || !B || !inputs || !arrival_us || !latency_us)))
    return set_error(FRAX_EINVAL, "frax_server_replay: bad argument");
  using clk = std::chrono::steady_clock;
  const auto t0 = clk::now();
  const auto t_end = t0 + std::chrono::microseconds(int64_t(timeout_ms * 1e3));
  std::mutex mu;
  std::unordered_map<int64_t, int> index;  // request id -> trace position
  std::atomic<int> collected{0};
  std::atomic<int> failure{0};
  std::string fail_msg;
  auto fail = [&](int st, const char* msg) {  // the first failure wins
    std::lock_guard<std::mutex> lk(mu);
    int expect = 0;
    if (failure.compare_exchange_strong(expect, st)) fail_msg = msg ? msg : "";
  };
  auto at = [&](int k) { return t0 + std::chrono::nanoseconds(int64_t(arrival_us[k] * 1e3)); };
  std::thread collector([&]() {
    while (collected.load() < n && failure.load() == 0) {
      if (clk::now() > t_end) {
        fail(FRAX_ETIMEOUT, nullptr);
        break;
      }
      int64_t r;
      frax_status st = frax_server_wait_any(s, 1.0, &r);
      if (st == FRAX_ETIMEOUT || st == FRAX_EINVAL) {  // nothing done / nothing in flight yet
        std::this_thread::yield();
        continue;
      }
      if (st != FRAX_OK) {
        fail(st, frax_last_error());
        break;
      }
      const auto seen = clk::now();
      int k = -1;
      {
        std::lock_guard<std::mutex> lk(mu);
        auto it = index.find(r);
        if (it != index.end()) k = it->second;
      }
      if (k < 0) {  // submitted, not yet recorded by the submitting thread
        std::this_thread::yield();
        continue;
      }
      latency_us[k] = std::chrono::duration<double, std::micro>(seen - at(k)).count();
      st = frax_server_collect(s, r, outputs ? outputs + 3 * size_t(k) : nullptr, nullptr);
      if (st != FRAX_OK) {
        fail(st, frax_last_error());
        break;
      }
      collected++;
    }
  });
  for (int k = 0; k < n && failure.load() == 0; ++k) {
    while (clk::now() < at(k)) std::this_thread::yield();
    while (true) {
      int64_t r;
      frax_status st = frax_server_submit(s, model_id[k], op[k], B[k], inputs + 4 * size_t(k), &r);
      if (st == FRAX_OK) {
        std::lock_guard<std::mutex> lk(mu);
        index[r] = k;
        break;
      }
      if (st != FRAX_EBUSY) {
        fail(st, frax_last_error());
        break;
      }
      if (clk::now() > t_end) {
        fail(FRAX_ETIMEOUT, nullptr);
        break;
      }
      std::this_thread::yield();
    }
  }
  collector.join();
  if (failure.load() != 0)
    return set_error(static_cast<frax_status>(failure.load()),
                     "frax_server_replay: " + (fail_msg.empty() ? std::string("timed out") : fail_msg));
  return clear_error();
}

}  // extern "C"
