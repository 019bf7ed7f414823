// frax_serve_batch_noalloc: a one-shot variant of the serving kernel for
// callers that must not allocate device memory.
//
// Who cannot allocate: real-time control loops (the paper's kilohertz
// controllers) may not call cudaMalloc, whose latency is unbounded and which
// can synchronise the device; code embedded in a framework that has already
// reserved nearly all of HBM for its own pool; and callers whose memory is
// budgeted up front. The server (server.cu) allocates its slab, ring and
// counters at creation; this entry point instead keeps its scratch -- the
// request descriptors, the model images and the tile counter -- in one
// file-scope device array of fixed size, and the caller passes every input
// and output buffer.
//
// The array is shared by all calls on a device and keeps the last call's
// contents; every call rewrites the descriptors and models it uses and
// clears the tile counter before its kernel starts. Calls whose kernels
// overlap on the GPU (different streams, no ordering between them) race on
// the array and give wrong results; order them on one stream.
//
// Set-up: the first call on each device looks up the array's device address
// with cudaGetSymbolAddress (with that device current) and caches it; make
// that first call before any stream capture.
//
// Staging: descriptors and model images are copied from one static, pageable
// host buffer. A copy from pageable memory returns only once the buffer has
// been consumed, which is what lets the next call rewrite it at once, and it
// may wait for the stream's earlier work first: the call can block the host.
// A captured copy would instead read that buffer when the graph is replayed,
// by then holding another call's requests, so the call refuses to run while
// `stream` is capturing.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "dyn.cuh"
#include "handles.h"

namespace frax {
namespace {

constexpr int kNoallocMaxRequests = FRAX_NOALLOC_MAX_REQUESTS;
constexpr int kNoallocMaxModels = FRAX_NOALLOC_MAX_MODELS;
constexpr int kNoallocTile = 128;
constexpr int kNoallocMaxDevices = 64;

struct NoallocReq {
  long long B;
  long long tile_begin, tile_end;
  int model, op, kind, pad;
  const float* in[4];
  float* out[3];
};

struct alignas(256) NoallocScratch {
  unsigned long long next_tile;  // must start at 0: cleared by every call
  unsigned long long total_tiles;
  int n_reqs, pad[59];
  NoallocReq reqs[kNoallocMaxRequests];
  ModelImage<64> models[kNoallocMaxModels];
};

// The scratch: fixed size, no allocation. Its host-side name is only a
// handle for cudaGetSymbolAddress, never a device address.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoallocScratch)];

enum NoallocKind { kNaChain7 = 0, kNaTree = 1, kNaTreeFree = 2 };

template <class T>
__device__ void noalloc_tile(const ModelImage<64>& M, const NoallocReq& r, long long b) {
  const Col col{r.B, b};
  switch (r.op) {
    case FRAX_OP_RNEA: rnea_one<T>(M, r.in[0], r.in[1], r.in[2], r.out[0], col); break;
    case FRAX_OP_CRBA: crba_one<T>(M, r.in[0], r.out[0], static_cast<float*>(nullptr), col); break;
    case FRAX_OP_ABA: aba_one<T>(M, r.in[0], r.in[1], r.in[2], r.out[0], col); break;
    case FRAX_OP_RNEA_GRAD: rnea_vjp_one<T>(M, r.in[0], r.in[1], r.in[2], r.in[3], r.out[0], r.out[1], r.out[2], col); break;
    default: break;
  }
}

// Every CTA claims 128-instance tiles from the scratch counter until all are
// taken; all work is known at launch, so nothing waits.
__global__ void __launch_bounds__(kNoallocTile) k_serve_batch_noalloc(NoallocScratch* S) {
  __shared__ ModelImage<64> model;
  __shared__ NoallocReq req;
  __shared__ long long s_tile;
  __shared__ int s_model;
  if (threadIdx.x == 0) s_model = -1;
  while (true) {
    if (threadIdx.x == 0) {
      const unsigned long long t = atomicAdd(&S->next_tile, 1ull);
      long long got = -1;
      if (t < S->total_tiles) {
        int lo = 0, hi = S->n_reqs - 1;  // tile ranges grow with the request index
        while (lo < hi) {
          const int mid = (lo + hi + 1) / 2;
          if (static_cast<long long>(t) >= S->reqs[mid].tile_begin) lo = mid;
          else hi = mid - 1;
        }
        req = S->reqs[lo];
        got = static_cast<long long>(t);
      }
      s_tile = got;
    }
    __syncthreads();
    const long long t = s_tile;
    if (t < 0) return;
    if (req.model != s_model) {
      const float4* src = reinterpret_cast<const float4*>(&S->models[req.model]);
      float4* dst = reinterpret_cast<float4*>(&model);
      for (int k = threadIdx.x; k < int(sizeof(ModelImage<64>) / 16); k += kNoallocTile) dst[k] = src[k];
      __syncthreads();
      if (threadIdx.x == 0) s_model = req.model;
    }
    __syncthreads();
    const long long b = (t - req.tile_begin) * kNoallocTile + threadIdx.x;
    if (b < req.B) {
      if (req.kind == kNaChain7) noalloc_tile<ChainTopo<7>>(model, req, b);
      else if (req.kind == kNaTreeFree) noalloc_tile<TreeTopo<64, true>>(model, req, b);
      else noalloc_tile<TreeTopo<64, false>>(model, req, b);
    }
    __syncthreads();
  }
}

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoallocMaxDevices] = {};
NoallocScratch g_noalloc_stage;  // host staging (static: no host allocation per call)

}  // namespace
}  // namespace frax

using namespace frax;

extern "C" frax_status frax_serve_batch_noalloc(const frax_batch_request_t* reqs, int n_reqs, void* stream) {
  if (n_reqs == 0) return clear_error();
  if (!reqs || n_reqs < 0) return set_error(FRAX_EINVAL, "frax_serve_batch_noalloc: bad request list");
  {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const cudaError_t ce = cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cap);
    if (ce == cudaErrorStreamCaptureImplicit) {  // the legacy stream while another stream captures
      cudaGetLastError();
      return set_error(FRAX_EINVAL, "frax_serve_batch_noalloc: a stream capture is in progress");
    }
    if (ce != cudaSuccess)
      return set_error(FRAX_ECUDA, std::string("frax_serve_batch_noalloc: cudaStreamIsCapturing: ") +
                                       cudaGetErrorString(ce));
    if (cap != cudaStreamCaptureStatusNone)
      return set_error(FRAX_EINVAL,
                       "frax_serve_batch_noalloc: stream is capturing; the staged copies would replay another "
                       "call's requests");
  }
  if (n_reqs > kNoallocMaxRequests)
    return set_error(FRAX_EINVAL, "frax_serve_batch_noalloc: more than FRAX_NOALLOC_MAX_REQUESTS (256) requests");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  NoallocScratch& st = g_noalloc_stage;
  const frax_model_s* seen[kNoallocMaxModels];
  int n_models = 0;
  long long tiles = 0;
  for (int i = 0; i < n_reqs; ++i) {
    const frax_batch_request_t& q = reqs[i];
    if (!q.model) return set_error(FRAX_EINVAL, "frax_serve_batch_noalloc: a request has no model");
    if (q.B < 0 || q.B >= (int64_t(1) << 30))
      return set_error(FRAX_EINVAL, "frax_serve_batch_noalloc: B must be in [0, 2^30)");
    int nin, nout;
    switch (q.op) {
      case FRAX_OP_RNEA: nin = 3; nout = 1; break;
      case FRAX_OP_CRBA: nin = 1; nout = 1; break;
      case FRAX_OP_ABA: nin = 3; nout = 1; break;
      case FRAX_OP_RNEA_GRAD: nin = 4; nout = 3; break;
      default: return set_error(FRAX_EINVAL, "frax_serve_batch_noalloc: unknown op");
    }
    for (int k = 0; k < nin; ++k)
      if (q.B > 0 && !q.in[k]) return set_error(FRAX_EINVAL, "frax_serve_batch_noalloc: an input is NULL");
    for (int k = 0; k < nout; ++k)
      if (q.B > 0 && !q.out[k]) return set_error(FRAX_EINVAL, "frax_serve_batch_noalloc: an output is NULL");
    int m = -1;
    for (int j = 0; j < n_models; ++j)
      if (seen[j] == q.model) m = j;
    if (m < 0) {
      if (n_models == kNoallocMaxModels)
        return set_error(FRAX_EINVAL, "frax_serve_batch_noalloc: more than FRAX_NOALLOC_MAX_MODELS (16) models");
      m = n_models++;
      seen[m] = q.model;
      q.model->m.pack(&st.models[m]);
    }
    NoallocReq& r = st.reqs[i];
    const HostModel& hm = q.model->m;
    r.B = q.B;
    r.tile_begin = tiles;
    tiles += (q.B + kNoallocTile - 1) / kNoallocTile;
    r.tile_end = tiles;
    r.model = m;
    r.op = q.op;
    r.kind = hm.kind == kKindChain ? kNaChain7 : (hm.free_root ? kNaTreeFree : kNaTree);
    r.pad = 0;
    for (int k = 0; k < 4; ++k) r.in[k] = q.in[k];
    for (int k = 0; k < 3; ++k) r.out[k] = q.out[k];
  }
  if (tiles == 0) return clear_error();
  st.next_tile = 0;
  st.total_tiles = static_cast<unsigned long long>(tiles);
  st.n_reqs = n_reqs;

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(FRAX_ECUDA, std::string("frax_serve_batch_noalloc: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kNoallocMaxDevices)
    return set_error(FRAX_EINVAL, "frax_serve_batch_noalloc: device index beyond 63");
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return set_error(FRAX_ECUDA, std::string("frax_serve_batch_noalloc: cudaGetSymbolAddress: ") +
                                       cudaGetErrorString(e));
    g_noalloc_ptr[dev] = p;
  }
  NoallocScratch* S = static_cast<NoallocScratch*>(g_noalloc_ptr[dev]);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // Header (counter cleared), the used descriptors and the used model images.
  const size_t head = offsetof(NoallocScratch, reqs);
  e = cudaMemcpyAsync(S, &st, head, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&S->reqs[0], &st.reqs[0], sizeof(NoallocReq) * n_reqs, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&S->models[0], &st.models[0], sizeof(ModelImage<64>) * n_models, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess)
    return set_error(FRAX_ECUDA, std::string("frax_serve_batch_noalloc: copy: ") + cudaGetErrorString(e));
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long want = std::max(1, sms) * 2LL;
  const unsigned grid = static_cast<unsigned>(tiles < want ? tiles : want);
  k_serve_batch_noalloc<<<grid, kNoallocTile, 0, s>>>(S);
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return set_error(FRAX_ECUDA, std::string("frax_serve_batch_noalloc: launch: ") + cudaGetErrorString(e));
  return clear_error();
}
