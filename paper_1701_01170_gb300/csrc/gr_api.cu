// gr_api.cu — graph handles, workspaces, status words and CSR validation.
//
// The CSR layout follows the paper's memory-access design (Sec. 5.4): row
// offsets R and column indices C, with per-edge data (weights) as a separate
// structure-of-arrays.  Validation runs on the device and reports through a
// status word; it never traps.
#include <climits>
#include <cstdlib>
#include <mutex>
#include <cstring>
#include <new>
#include <vector>

#include "gr_internal.cuh"

#define GR_CUDA_TRY(expr)                    \
  do {                                       \
    cudaError_t _e = (expr);                 \
    if (_e != cudaSuccess) {                 \
      (void)cudaGetLastError();              \
      return _e == cudaErrorMemoryAllocation \
                 ? GR_ERR_OOM                \
                 : GR_ERR_CUDA;              \
    }                                        \
  } while (0)

extern "C" const char* gr_status_str(gr_status s) {
  switch (s) {
    case GR_OK: return "GR_OK";
    case GR_ERR_INVALID_ARG: return "GR_ERR_INVALID_ARG";
    case GR_ERR_OOM: return "GR_ERR_OOM";
    case GR_ERR_CUDA: return "GR_ERR_CUDA";
    case GR_ERR_CAPACITY: return "GR_ERR_CAPACITY";
    case GR_ERR_OVERFLOW: return "GR_ERR_OVERFLOW";
    case GR_ERR_TIMEOUT: return "GR_ERR_TIMEOUT";
    case GR_ERR_INVALID_GRAPH: return "GR_ERR_INVALID_GRAPH";
    case GR_ERR_UNSUPPORTED: return "GR_ERR_UNSUPPORTED";
    default: return "GR_ERR_UNKNOWN";
  }
}

extern "C" int32_t gr_version(void) { return (1 << 16) | 0; }

// ---------------------------------------------------------------------------
// validation

struct ValidateOut {
  int bad;                   // first violation code (0 = valid)
  int max_degree;
  int nonisolated;
  int pad;
  unsigned long long weight_sum;
  unsigned long long fp[4];  // symmetry fingerprints: forward / backward, two hashes
};

// Violation codes (diagnostic only; the API reports GR_ERR_INVALID_GRAPH).
enum { V_R0 = 1, V_RN, V_MONO, V_COL, V_WEIGHT, V_UNSORTED, V_ASYM };

__global__ void gr_validate_rows(int32_t n, int64_t m, const int32_t* __restrict__ R,
                                 ValidateOut* out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int local_max = 0, local_nz = 0;
  if (i == 0) {
    if (R[0] != 0) atomicCAS(&out->bad, 0, V_R0);
    if ((int64_t)R[n] != m) atomicCAS(&out->bad, 0, V_RN);
  }
  for (; i < n; i += stride) {
    int a = R[i], b = R[i + 1];
    if (b < a) atomicCAS(&out->bad, 0, V_MONO);
    int d = b - a;
    local_max = max(local_max, d);
    local_nz += d > 0;
  }
  for (int o = 16; o > 0; o >>= 1) {
    local_max = max(local_max, __shfl_xor_sync(GR_FULL_MASK, local_max, o));
    local_nz += __shfl_xor_sync(GR_FULL_MASK, local_nz, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&out->max_degree, local_max);
    atomicAdd(&out->nonisolated, local_nz);
  }
}

// Column range, weights, sortedness and (optionally) symmetry, one warp per
// row with the lanes striding its edges (coalesced).  Symmetry is checked as
// multiset equality {(u, v, w)} == {(v, u, w)}: every edge adds a mixed hash
// of (u, v, w) to one pair of 64-bit sums and of (v, u, w) to another; the
// host compares the sums.  With strictly sorted rows (checked exactly) the
// multisets are sets, and an asymmetric graph passes only through a
// simultaneous collision of two independent 64-bit hash sums.
__device__ __forceinline__ unsigned long long gr_mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void gr_validate_edges(int32_t n, const int32_t* __restrict__ R,
                                  const int32_t* __restrict__ C, const uint32_t* __restrict__ W,
                                  int symmetric, ValidateOut* out) {
  int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long wsum = 0, f[4] = {0, 0, 0, 0};
  for (int64_t u = warp; u < n; u += nwarps) {
    int a = R[u], b = R[u + 1];
    if (b < a) continue;  // reported by gr_validate_rows
    for (int e = a + lane; e < b; e += 32) {
      int v = C[e];
      if (v < 0 || v >= n) { atomicCAS(&out->bad, 0, V_COL); continue; }
      unsigned w = 0;
      if (W) {
        w = W[e];
        if (w == 0) atomicCAS(&out->bad, 0, V_WEIGHT);
        wsum += w;
      }
      if (!symmetric) continue;
      if (e > a && C[e - 1] >= v) atomicCAS(&out->bad, 0, V_UNSORTED);
      const unsigned long long fw = ((unsigned long long)u << 32) | (unsigned)v;
      const unsigned long long bw = ((unsigned long long)v << 32) | (unsigned long long)u;
      const unsigned long long salt = (unsigned long long)w * 0xD6E8FEB86659FD93ull;
      f[0] += gr_mix64(fw ^ salt);
      f[1] += gr_mix64(bw ^ salt);
      f[2] += gr_mix64(gr_mix64(fw) + salt);
      f[3] += gr_mix64(gr_mix64(bw) + salt);
    }
  }
  wsum = gr_warp_sum_u64(wsum);
  if (lane == 0 && wsum) atomicAdd(&out->weight_sum, wsum);
  if (symmetric) {
    for (int k = 0; k < 4; ++k) {
      unsigned long long x = gr_warp_sum_u64(f[k]);
      if (lane == 0 && x) atomicAdd(&out->fp[k], x);
    }
  }
}

// Bit v of word w is set when vertex v = 32 w + bit has no edges.
__global__ void gr_zero_degree_bitmap(int32_t n, const int32_t* __restrict__ R, uint32_t* bm,
                                      int64_t nwords) {
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwords;
       w += (int64_t)gridDim.x * blockDim.x) {
    uint32_t x = 0u;
    for (int b = 0; b < 32; ++b) {
      const int64_t v = w * 32 + b;
      if (v < n && R[v + 1] == R[v]) x |= 1u << b;
    }
    bm[w] = x;
  }
}

// ---------------------------------------------------------------------------
// workspaces

static size_t bitmap_words(int32_t n) { return ((size_t)n + 31) / 32 + 1; }

static int64_t chunk_capacity(const gr_graph* g, int big) {
  // every split row has degree >= big and needs ceil(deg / GR_CHUNK_EDGES)
  // entries: at most m / GR_CHUNK_EDGES + m / big + 1 in one frontier.
  if (big < 1) big = 1;
  return g->m / GR_CHUNK_EDGES + g->m / big + 2;
}

static size_t ws_bytes(const gr_graph* g, int32_t ops) {
  size_t n = (size_t)g->n + 1, bw = bitmap_words(g->n);
  size_t b = sizeof(GrCtl) + 2 * sizeof(int);
  b += 6 * n * sizeof(int32_t);                                  // queues, unvisited lists
  b += 2 * (size_t)chunk_capacity(g, 32) * sizeof(int2);         // chunks (smallest big)
  b += 4 * bw * sizeof(uint32_t);                                // visited + 3 frontiers
  b += n * sizeof(int32_t) + bw * sizeof(uint32_t);              // filter scratch
  b += (GR_MAX_SCAN_BLOCKS + 2) * sizeof(long long);             // scan scratch
  b += n * sizeof(int32_t) + 8 * sizeof(long long);              // pull tags, counters
  b += GR_PULL_DEFER_INTS * sizeof(int32_t);                     // deferred pull rows
  b += n * sizeof(long long);                                    // advance offsets
  if (ops & GR_OP_SSSP) b += n * sizeof(uint64_t) + (5 + GR_RING_K) * n * sizeof(int32_t);
  return b;
}

// Pinned host words for gr_sync_status, handed out from blocks that live until
// the process exits, so that creating or destroying a workspace never calls
// cudaMallocHost / cudaFreeHost (the latter waits for the whole device).
namespace {
std::mutex g_slot_mu;
std::vector<int*> g_slot_free;
constexpr int kSlotBlock = 1024;
}  // namespace

static int* status_slot_take() {
  std::lock_guard<std::mutex> lock(g_slot_mu);
  if (g_slot_free.empty()) {
    int* block = nullptr;
    if (cudaMallocHost((void**)&block, kSlotBlock * sizeof(int)) != cudaSuccess) {
      (void)cudaGetLastError();
      return nullptr;
    }
    for (int i = kSlotBlock - 1; i >= 0; --i) g_slot_free.push_back(block + i);
  }
  int* p = g_slot_free.back();
  g_slot_free.pop_back();
  return p;
}

static void status_slot_give(int* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lock(g_slot_mu);
  g_slot_free.push_back(p);
}

// Releases a workspace: device buffers with cudaFree, or, for a stream-ordered
// workspace, with cudaFreeAsync on `s` (after the work already queued there).
static void ws_free(gr_workspace* ws, cudaStream_t s = nullptr) {
  if (!ws) return;
  auto release = [&](void* p) {
    if (!p) return;
    if (ws->stream_ordered) cudaFreeAsync(p, s);
    else cudaFree(p);
  };
  void* ptrs[] = {ws->ctl, ws->status, ws->q[0], ws->q[1], ws->qm[0], ws->qm[1],
                  ws->ulist[0], ws->ulist[1],
                  ws->chunks[0], ws->chunks[1],
                  ws->visited, ws->front[0], ws->front[1], ws->front[2], ws->key,
                  ws->far[0], ws->far[1], ws->stamp_near, ws->stamp_far, ws->first_idx,
                  ws->claim, ws->block_sums, ws->tags, ws->pdef, ws->item_off, ws->dev_len};
  for (void* p : ptrs) release(p);
  for (int j = 0; j < GR_RING_K; ++j) release(ws->ring[j]);
  release(ws->stamp_ring);
  status_slot_give(ws->h_status);
  gr_bc_free(ws->bc);
  gr_cc_free(ws->cc);
  gr_tc_free(ws->tc);
  delete ws;
}

__global__ void gr_fill_i32(int32_t* p, int64_t len, int32_t v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

// stream_ordered: allocate with cudaMallocAsync and initialise on `s`, without
// waiting for the device (the workspace is then ready in the order of `s`).
static gr_status ws_create(const gr_graph* g, int32_t ops, gr_workspace** out,
                           bool stream_ordered = false, cudaStream_t s = nullptr) {
  gr_workspace* ws = new (std::nothrow) gr_workspace();
  if (!ws) return GR_ERR_OOM;
  ws->g = g;
  ws->ops = ops;
  ws->stream_ordered = stream_ordered;
  size_t n = (size_t)g->n + 1, bw = bitmap_words(g->n);
  ws->chunk_cap = chunk_capacity(g, 32);
#define ALLOC(ptr, bytes)                                                      \
  do {                                                                         \
    const cudaError_t e_ = stream_ordered ? cudaMallocAsync((void**)&(ptr), (bytes), s) \
                                          : cudaMalloc((void**)&(ptr), (bytes));        \
    if (e_ != cudaSuccess) {                                                   \
      (void)cudaGetLastError();                                                \
      ws_free(ws, s);                                                          \
      return GR_ERR_OOM;                                                       \
    }                                                                          \
  } while (0)
  ALLOC(ws->ctl, sizeof(GrCtl));
  ALLOC(ws->status, sizeof(int));
  ALLOC(ws->q[0], n * sizeof(int32_t));
  ALLOC(ws->q[1], n * sizeof(int32_t));
  ALLOC(ws->qm[0], n * sizeof(int32_t));
  ALLOC(ws->qm[1], n * sizeof(int32_t));
  ALLOC(ws->ulist[0], n * sizeof(int32_t));
  ALLOC(ws->ulist[1], n * sizeof(int32_t));
  ALLOC(ws->chunks[0], ws->chunk_cap * sizeof(int2));
  ALLOC(ws->chunks[1], ws->chunk_cap * sizeof(int2));
  ALLOC(ws->visited, bw * sizeof(uint32_t));
  for (int i = 0; i < 3; ++i) ALLOC(ws->front[i], bw * sizeof(uint32_t));
  ALLOC(ws->first_idx, n * sizeof(int32_t));
  ALLOC(ws->claim, bw * sizeof(uint32_t));
  ALLOC(ws->block_sums, (GR_MAX_SCAN_BLOCKS + 2) * sizeof(long long));
  ALLOC(ws->tags, n * sizeof(int32_t));
  ALLOC(ws->pdef, GR_PULL_DEFER_INTS * sizeof(int32_t));
  ALLOC(ws->item_off, n * sizeof(long long));
  ALLOC(ws->dev_len, 8 * sizeof(long long));
  if (ops & GR_OP_SSSP) {
    ALLOC(ws->key, n * sizeof(uint64_t));
    ALLOC(ws->far[0], n * sizeof(int32_t));
    ALLOC(ws->far[1], n * sizeof(int32_t));
    ALLOC(ws->stamp_near, n * sizeof(int32_t));
    ALLOC(ws->stamp_far, n * sizeof(int32_t));
    for (int j = 0; j < GR_RING_K; ++j) ALLOC(ws->ring[j], n * sizeof(int32_t));
    ALLOC(ws->stamp_ring, n * sizeof(uint32_t));
  }
#undef ALLOC
  ws->h_status = status_slot_take();
  if (!ws->h_status) {
    ws_free(ws, s);
    return GR_ERR_OOM;
  }
  bool ok = cudaMemsetAsync(ws->ctl, 0, sizeof(GrCtl), s) == cudaSuccess &&
            cudaMemsetAsync(ws->status, 0, sizeof(int), s) == cudaSuccess &&
            cudaMemsetAsync(ws->claim, 0, bw * sizeof(uint32_t), s) == cudaSuccess;
  if (ok) {
    gr_fill_i32<<<256, 256, 0, s>>>(ws->first_idx, (int64_t)n, INT32_MAX);
    ok = cudaGetLastError() == cudaSuccess &&
         (stream_ordered || cudaDeviceSynchronize() == cudaSuccess);
  }
  if (!ok) {
    (void)cudaGetLastError();
    ws_free(ws, s);
    return GR_ERR_CUDA;
  }
  *out = ws;
  return GR_OK;
}

extern "C" gr_status gr_workspace_create(const gr_graph* g, int32_t ops, gr_workspace** out) {
  if (!g || !out || (ops & ~(GR_OP_BFS | GR_OP_SSSP))) return GR_ERR_INVALID_ARG;
  if ((ops & GR_OP_SSSP) && !g->W && g->m > 0) return GR_ERR_UNSUPPORTED;
  *out = nullptr;
  return ws_create(g, ops, out);
}

extern "C" gr_status gr_workspace_destroy(gr_workspace* ws) {
  if (!ws) return GR_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  ws_free(ws);
  return GR_OK;
}

extern "C" gr_status gr_workspace_create_async(const gr_graph* g, int32_t ops, void* stream,
                                               gr_workspace** out) {
  if (!g || !out || (ops & ~(GR_OP_BFS | GR_OP_SSSP))) return GR_ERR_INVALID_ARG;
  if ((ops & GR_OP_SSSP) && !g->W && g->m > 0) return GR_ERR_UNSUPPORTED;
  *out = nullptr;
  return ws_create(g, ops, out, true, (cudaStream_t)stream);
}

extern "C" gr_status gr_workspace_destroy_async(gr_workspace* ws, void* stream) {
  if (!ws) return GR_ERR_INVALID_ARG;
  if (!ws->stream_ordered) return gr_workspace_destroy(ws);
  ws_free(ws, (cudaStream_t)stream);
  return GR_OK;
}

gr_workspace* gr_resolve_ws(const gr_graph* g, gr_workspace* ws) {
  return ws ? ws : g->ws_default;
}

cudaError_t gr_reset_ctl(gr_workspace* ws, cudaStream_t s) {
  return cudaMemsetAsync(ws->ctl, 0, sizeof(GrCtl), s);
}

// Resident CTAs per SM of a persistent kernel.  The occupancy query costs
// microseconds of host time, which a caller timing a whole query pays in
// GPU idle time, so results are cached per (device, kernel, threads, shared
// memory) and the dynamic shared-memory attribute is set once per entry.
namespace {
struct OccEntry {
  int device;
  const void* kernel;
  int threads;
  size_t smem;
  int per_sm;
};
std::mutex g_occ_mutex;
OccEntry g_occ[64];
int g_occ_n = 0;
}  // namespace

int gr_launch_blocks(const void* kernel, int threads, size_t smem, int num_sms, int requested) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lock(g_occ_mutex);
    for (int i = 0; i < g_occ_n; ++i)
      if (g_occ[i].device == dev && g_occ[i].kernel == kernel && g_occ[i].threads == threads &&
          g_occ[i].smem == smem)
        per_sm = g_occ[i].per_sm;
    if (per_sm == 0) {
      if ((smem > 48 * 1024 &&
           cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
               cudaSuccess) ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) !=
              cudaSuccess ||
          per_sm < 1) {
        (void)cudaGetLastError();
        return 0;
      }
      if (g_occ_n < 64) g_occ[g_occ_n++] = OccEntry{dev, kernel, threads, smem, per_sm};
    }
  }
  if (requested > 0 && requested < per_sm) per_sm = requested;
  return per_sm * num_sms;
}

extern "C" gr_status gr_sync_status(const gr_graph* g, gr_workspace* ws, void* stream) {
  if (!g) return GR_ERR_INVALID_ARG;
  ws = gr_resolve_ws(g, ws);
  cudaStream_t s = (cudaStream_t)stream;
  GR_CUDA_TRY(cudaMemcpyAsync(ws->h_status, ws->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  GR_CUDA_TRY(cudaStreamSynchronize(s));
  int st = *ws->h_status;
  if (st != 0) {
    GR_CUDA_TRY(cudaMemsetAsync(ws->status, 0, sizeof(int), s));
    GR_CUDA_TRY(cudaMemsetAsync(ws->ctl, 0, sizeof(GrCtl), s));
    GR_CUDA_TRY(cudaStreamSynchronize(s));
  }
  return st;
}

extern "C" gr_status gr_last_run_stats(const gr_graph* g, gr_workspace* ws, gr_run_stats* out,
                                       void* stream) {
  if (!g || !out) return GR_ERR_INVALID_ARG;
  ws = gr_resolve_ws(g, ws);
  cudaStream_t s = (cudaStream_t)stream;
  GrCtl h;
  GR_CUDA_TRY(cudaMemcpyAsync(&h, ws->ctl, sizeof(GrCtl), cudaMemcpyDeviceToHost, s));
  GR_CUDA_TRY(cudaStreamSynchronize(s));
  out->levels = h.levels;
  out->reserved = 0;
  out->edges = (int64_t)h.edges;
  out->vertices = (int64_t)h.verts;
  out->updates = (int64_t)h.updates;
  return GR_OK;
}

// ---------------------------------------------------------------------------
// graphs

extern "C" gr_status gr_graph_create_csr(int32_t n, int64_t m, const int32_t* row_offsets,
                                         const int32_t* cols, const uint32_t* weights,
                                         uint32_t flags, void* stream, gr_graph** out) {
  if (!out || n < 0 || m < 0 || m >= INT32_MAX || !row_offsets || (m > 0 && !cols) ||
      (flags & ~(GR_COPY | GR_SYMMETRIC)))
    return GR_ERR_INVALID_ARG;
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  int device = 0, num_sms = 0;
  GR_CUDA_TRY(cudaGetDevice(&device));
  GR_CUDA_TRY(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device));
  gr_graph* g = new (std::nothrow) gr_graph();
  if (!g) return GR_ERR_OOM;
  g->n = n;
  g->m = m;
  g->flags = flags;
  g->device = device;
  g->num_sms = num_sms;
  auto fail = [&](gr_status st) {
    for (void* p : g->owned)
      if (p) cudaFree(p);
    if (g->zero_deg) cudaFree(g->zero_deg);
    delete g;
    return st;
  };
  if (flags & GR_COPY) {
    size_t rb = ((size_t)n + 1) * sizeof(int32_t), cb = (size_t)m * sizeof(int32_t);
    if (cudaMalloc(&g->owned[0], rb) != cudaSuccess ||
        (m && cudaMalloc(&g->owned[1], cb) != cudaSuccess) ||
        (weights && m && cudaMalloc(&g->owned[2], (size_t)m * sizeof(uint32_t)) != cudaSuccess)) {
      (void)cudaGetLastError();
      return fail(GR_ERR_OOM);
    }
    if (cudaMemcpyAsync(g->owned[0], row_offsets, rb, cudaMemcpyDeviceToDevice, s) ||
        (m && cudaMemcpyAsync(g->owned[1], cols, cb, cudaMemcpyDeviceToDevice, s)) ||
        (weights && m &&
         cudaMemcpyAsync(g->owned[2], weights, (size_t)m * 4, cudaMemcpyDeviceToDevice, s))) {
      (void)cudaGetLastError();
      return fail(GR_ERR_CUDA);
    }
    g->R = (const int32_t*)g->owned[0];
    g->C = (const int32_t*)g->owned[1];
    g->W = weights ? (const uint32_t*)g->owned[2] : nullptr;
  } else {
    g->R = row_offsets;
    g->C = cols;
    g->W = weights;
  }
  if (weights && m == 0 && !g->W) g->W = weights;

  ValidateOut* d_out = nullptr;
  ValidateOut h_out;
  if (cudaMalloc(&d_out, sizeof(ValidateOut)) != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(GR_ERR_OOM);
  }
  bool ok = cudaMemsetAsync(d_out, 0, sizeof(ValidateOut), s) == cudaSuccess;
  if (ok) {
    int blocks = g->num_sms * 4;
    gr_validate_rows<<<blocks, 256, 0, s>>>(n, m, g->R, d_out);
    ok = cudaStreamSynchronize(s) == cudaSuccess &&
         cudaMemcpy(&h_out, d_out, sizeof(ValidateOut), cudaMemcpyDeviceToHost) == cudaSuccess;
    // column/symmetry checks only once the row offsets are known to be sane
    if (ok && h_out.bad == 0 && m > 0) {
      gr_validate_edges<<<blocks, 256, 0, s>>>(n, g->R, g->C, g->W,
                                                (flags & GR_SYMMETRIC) ? 1 : 0, d_out);
      ok = cudaStreamSynchronize(s) == cudaSuccess &&
           cudaMemcpy(&h_out, d_out, sizeof(ValidateOut), cudaMemcpyDeviceToHost) ==
               cudaSuccess;
    }
  }
  cudaFree(d_out);
  if (!ok) {
    (void)cudaGetLastError();
    return fail(GR_ERR_CUDA);
  }
  if (h_out.bad == 0 && (flags & GR_SYMMETRIC) &&
      (h_out.fp[0] != h_out.fp[1] || h_out.fp[2] != h_out.fp[3]))
    h_out.bad = V_ASYM;
  if (h_out.bad != 0) return fail(GR_ERR_INVALID_GRAPH);
  g->max_degree = h_out.max_degree;
  g->nonisolated = h_out.nonisolated;
  g->weight_sum = h_out.weight_sum;
  if ((flags & GR_SYMMETRIC) && g->nonisolated < n) {
    const int64_t nw = (int64_t)bitmap_words(n);
    if (cudaMalloc((void**)&g->zero_deg, nw * sizeof(uint32_t)) != cudaSuccess) {
      (void)cudaGetLastError();
      return fail(GR_ERR_OOM);
    }
    gr_zero_degree_bitmap<<<g->num_sms * 4, 256, 0, s>>>(n, g->R, g->zero_deg, nw);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
      (void)cudaGetLastError();
      return fail(GR_ERR_CUDA);
    }
  }
  // an edgeless graph needs no weight array to be a valid SSSP input
  const bool weighted = weights != nullptr || m == 0;
  gr_status st = ws_create(g, weighted ? (GR_OP_BFS | GR_OP_SSSP) : GR_OP_BFS, &g->ws_default);
  if (st != GR_OK) return fail(st);
  *out = g;
  return GR_OK;
}

extern "C" gr_status gr_graph_destroy(gr_graph* g) {
  if (!g) return GR_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  ws_free(g->ws_default);
  gr_ms_free(g->ms);
  if (g->zero_deg) cudaFree(g->zero_deg);
  for (void* p : g->owned)
    if (p) cudaFree(p);
  delete g;
  return GR_OK;
}

extern "C" gr_status gr_graph_info(const gr_graph* g, int32_t* n, int64_t* m, uint32_t* flags,
                                   int32_t* max_degree) {
  if (!g) return GR_ERR_INVALID_ARG;
  if (n) *n = g->n;
  if (m) *m = g->m;
  if (flags) *flags = g->flags;
  if (max_degree) *max_degree = g->max_degree;
  return GR_OK;
}

extern "C" gr_status gr_graph_footprint(const gr_graph* g, int32_t op, size_t* bytes_per_query) {
  if (!g || !bytes_per_query || (op != GR_OP_BFS && op != GR_OP_SSSP)) return GR_ERR_INVALID_ARG;
  *bytes_per_query = ws_bytes(g, op);
  return GR_OK;
}
