// gr_bfs.cu — direction-optimising BFS as one persistent, cooperative kernel.
//
// The paper's BFS (Sec. 6.1) is a bulk-synchronous loop of advance + filter
// steps on a vertex frontier, with a per-iteration host round trip to test
// for an empty frontier (Sec. 5.3).  Here the whole loop runs on the device:
// every CTA of a co-resident grid executes every level, and a bounded grid
// barrier separates levels, so no level costs a launch or a device-to-host
// copy.  Each level is either
//   * push (Sec. 5.1): advance fused with the visit functor and the filter
//     (LB_CULL-style fusion, Sec. 5.3) — the frontier arrives in three
//     size classes (Sec. 5.1.2): rows of degree >= big_degree pre-split into
//     256-edge chunks dealt out over every warp of the grid, medium rows 4
//     per warp batch, short rows 32 per warp batch, each batch expanded
//     warp-centrically (the warp scans its rows' degrees and walks the
//     concatenated edges in 32-wide strips); a visited bitmap with atomicOr
//     claims each vertex once, so the output frontier needs no separate
//     dedup pass; or
//   * pull (Sec. 5.1.4, Alg. 2 Reverse_Advance): every unvisited vertex scans
//     its row for a member of the current frontier bitmap and stops at the
//     first hit; the first pull level reads the complement of the visited
//     bitmap (4 words of 32 candidates per warp batch), later consecutive
//     pull levels the compacted unvisited list the previous one wrote.  A
//     pull level records its output as a bitmap only.
// The direction follows the paper's Eq. 5-6 (push -> pull when
// m_f > m_u * do_a, pull -> push when m_f < m_u * do_b) with m_f and m_u
// counted exactly: every discovered vertex adds its degree to m_f.
#include <climits>
#include <mutex>

#include "gr_bfs_body.cuh"

namespace {

constexpr int NT = GR_PERSIST_THREADS;

#ifndef GR_BFS_MIN_BLOCKS
#define GR_BFS_MIN_BLOCKS 2  // resident CTAs per SM the register budget is sized for
#endif
// Two instantiations: queries that may pull (direction-optimising or forced
// pull, symmetric graphs) and push-only queries, whose kernel carries no pull
// code at all (with the pull levels' code in the same loop, the push levels
// of a push-only R-MAT s22 BFS ran 2-3 % slower).
template <bool PULL>
__global__ void __launch_bounds__(NT, GR_BFS_MIN_BLOCKS) bfs_persistent(BfsArgs a) {
  GridScope sc{a.ctl, a.status, a.spin, (int64_t)blockIdx.x * NT + threadIdx.x,
               (int64_t)gridDim.x * NT, 0u};
  __shared__ GrArena ar;
  gr_bfs_body<PULL>(a, sc, ar);
}

const void* bfs_kernel(const BfsArgs& a) {
  return a.use_do || a.force_pull ? (const void*)bfs_persistent<true>
                                  : (const void*)bfs_persistent<false>;
}

#ifndef GR_BFS_CARVEOUT
#define GR_BFS_CARVEOUT -1  // preferred shared-memory share of L1 in percent; -1: driver default
#endif
// Sets the kernel's preferred L1 / shared-memory split once per process.
void bfs_carveout_once() {
#if GR_BFS_CARVEOUT >= 0
  static std::once_flag once;
  std::call_once(once, [] {
    for (const void* k : {(const void*)bfs_persistent<true>, (const void*)bfs_persistent<false>})
      (void)cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 GR_BFS_CARVEOUT);
    (void)cudaGetLastError();
  });
#endif
}

}  // namespace

extern "C" void gr_bfs_opts_default(gr_bfs_opts* o) {
  if (!o) return;
  o->direction = GR_DIR_AUTO;
  o->do_a = 0.05f;
  o->do_b = 0.05f;
  o->big_degree = GR_DEFAULT_BFS_BIG;
  o->blocks_per_sm = 0;
  o->spin_limit = GR_DEFAULT_SPIN_LIMIT;
  o->ws = nullptr;
  o->level_stats = nullptr;
  o->max_levels = 0;
  o->max_blocks = 0;
  o->bulk_edges = 0;
}

extern "C" gr_status gr_bfs(const gr_graph* g, int32_t src, int32_t* depth, int32_t* pred,
                            const gr_bfs_opts* opts, void* stream) {
  if (!g || !depth || g->n <= 0 || src < 0 || src >= g->n) return GR_ERR_INVALID_ARG;
  gr_bfs_opts o;
  gr_bfs_opts_default(&o);
  if (opts) o = *opts;
  if (o.direction < GR_DIR_AUTO || o.direction > GR_DIR_PULL || o.max_levels < 0 ||
      (o.max_levels > 0 && !o.level_stats) || o.max_blocks < 0)
    return GR_ERR_INVALID_ARG;
  const bool symmetric = (g->flags & GR_SYMMETRIC) != 0;
  if (o.direction == GR_DIR_PULL && !symmetric) return GR_ERR_UNSUPPORTED;
  gr_workspace* ws = gr_resolve_ws(g, o.ws);
  if (!ws || ws->g != g) return GR_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;

  BfsArgs a = {};
  a.n = g->n;
  a.m = g->m;
  a.R = g->R;
  a.C = g->C;
  a.depth = depth;
  a.pred = pred;
  a.visited = ws->visited;
  for (int i = 0; i < 3; ++i) a.front[i] = ws->front[i];
  a.q[0] = ws->q[0];
  a.q[1] = ws->q[1];
  a.qm[0] = ws->qm[0];
  a.qm[1] = ws->qm[1];
  a.ulist[0] = ws->ulist[0];
  a.ulist[1] = ws->ulist[1];
  a.ch[0] = ws->chunks[0];
  a.ch[1] = ws->chunks[1];
  a.chunk_cap = ws->chunk_cap;
  a.ctl = ws->ctl;
  a.status = ws->status;
  a.src = src;
  a.nwords = (int32_t)(((int64_t)g->n + 31) / 32);
  a.use_do = symmetric && o.direction != GR_DIR_PUSH;
  a.force_pull = o.direction == GR_DIR_PULL;
  a.big = o.big_degree > 0 ? (o.big_degree < 32 ? 32 : o.big_degree) : GR_DEFAULT_BFS_BIG;
  a.track_deg = a.use_do || g->max_degree >= GR_MEDIUM_DEGREE;
  a.do_a = o.do_a;
  a.do_b = o.do_b;
  a.spin = o.spin_limit ? o.spin_limit : GR_DEFAULT_SPIN_LIMIT;
  a.level_stats = o.level_stats;
  a.max_levels = o.max_levels;
  a.bulk_edges = o.bulk_edges < 0 ? 0 : (o.bulk_edges > 0 ? o.bulk_edges
                                                          : gr_default_bulk_edges(g->n));
  a.preset = symmetric ? g->zero_deg : nullptr;
  a.pdef = ws->pdef;

  bfs_carveout_once();
  const void* kernel = bfs_kernel(a);
  int blocks = gr_launch_blocks(kernel, NT, 0, g->num_sms, o.blocks_per_sm);
  if (blocks <= 0) return GR_ERR_CUDA;
  if (o.max_blocks > 0 && blocks > o.max_blocks) blocks = o.max_blocks;
  if (gr_reset_ctl(ws, s) != cudaSuccess) return GR_ERR_CUDA;
  void* args[] = {&a};
  if (cudaLaunchCooperativeKernel(kernel, dim3(blocks), dim3(NT), args, 0, s) != cudaSuccess) {
    (void)cudaGetLastError();
    return GR_ERR_CUDA;
  }
  return GR_OK;
}

// ---------------------------------------------------------------------------
// gr_bfs_static: the BFS above, with its scratch in a fixed static area.
//
// Who needs this: code that must not call cudaMalloc when it runs a query —
// a callback of a custom device allocator or memory pool (allocating there
// would re-enter the allocator), a latency-critical thread that cannot take
// the device-wide synchronisation cudaMalloc may imply, or a host runtime
// that owns all device memory and forbids allocations by libraries.  For
// them the scratch (frontier queues, edge-chunk lists, bitmaps, the control
// block and the status word) lives in one file-scope __device__ array that
// the CUDA module reserves on every GPU that loads this library and keeps
// until the process exits.  The caller still provides the CSR and the
// output arrays.
//
// In host code the array's name only denotes a host-side shadow symbol, so
// the device address is fetched with cudaGetSymbolAddress, once per device,
// by the first call on that device (with that device current).  That first
// call may load the module, so it must not happen during stream capture.
// All calls share the one array: each call clears the control block and the
// status word before its launch, and two calls whose kernels overlap on the
// GPU would race on the same scratch, so calls must be serialised (for
// example by issuing them on one stream).
namespace {

constexpr int64_t kStaticMaxVertices = GR_STATIC_MAX_VERTICES;
constexpr int64_t kStaticMaxEdges = GR_STATIC_MAX_EDGES;
// rows of at least 256 edges (the BFS default) are split into chunks; there is
// no medium-row class here, so a 32-row batch holds at most 32 x 255 edges
constexpr int kStaticBig = GR_DEFAULT_BFS_BIG;
// chunks of one frontier: at most m / chunk + m / kStaticBig + 1 entries
constexpr int64_t kStaticChunkCap =
    kStaticMaxEdges / GR_CHUNK_EDGES + kStaticMaxEdges / kStaticBig + 2;
constexpr int64_t kStaticWords = (kStaticMaxVertices + 31) / 32 + 1;

constexpr size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffCtl = 0;
constexpr size_t kOffStatus = round256(sizeof(GrCtl));
constexpr size_t kOffQ0 = kOffStatus + 256;  // [0, kOffQ0) is cleared on every call
constexpr size_t kQueueBytes = round256((size_t)(kStaticMaxVertices + 1) * sizeof(int32_t));
constexpr size_t kOffQ1 = kOffQ0 + kQueueBytes;
constexpr size_t kChunkBytes = round256((size_t)kStaticChunkCap * sizeof(int2));
constexpr size_t kOffCh0 = kOffQ1 + kQueueBytes;
constexpr size_t kOffCh1 = kOffCh0 + kChunkBytes;
constexpr size_t kBitmapBytes = round256((size_t)kStaticWords * sizeof(uint32_t));
constexpr size_t kOffVisited = kOffCh1 + kChunkBytes;
constexpr size_t kOffFront = kOffVisited + kBitmapBytes;
constexpr size_t kOffPdef = kOffFront + 3 * kBitmapBytes;
constexpr size_t kStaticBytes =
    kOffPdef + round256(GR_PULL_DEFER_INTS * sizeof(int32_t));  // about 13.1 MB

static __device__ __align__(256) unsigned char g_bfs_static_scratch[kStaticBytes];

struct StaticDevice {
  bool ready;
  unsigned char* base;  // device address of g_bfs_static_scratch
  int blocks[2];        // co-resident grid sizes of bfs_persistent<false>, <true>
};
constexpr int kMaxDevices = 64;
StaticDevice g_static_dev[kMaxDevices];
std::mutex g_static_mu;

gr_status static_setup(int device, StaticDevice** out) {
  std::lock_guard<std::mutex> lock(g_static_mu);
  StaticDevice& d = g_static_dev[device];
  if (!d.ready) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_bfs_static_scratch) != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return GR_ERR_CUDA;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
      (void)cudaGetLastError();
      return GR_ERR_CUDA;
    }
    const int b0 = gr_launch_blocks((const void*)bfs_persistent<false>, NT, 0, sms, 0);
    const int b1 = gr_launch_blocks((const void*)bfs_persistent<true>, NT, 0, sms, 0);
    if (b0 <= 0 || b1 <= 0) return GR_ERR_CUDA;
    d.base = (unsigned char*)p;
    d.blocks[0] = b0;
    d.blocks[1] = b1;
    d.ready = true;
  }
  *out = &d;
  return GR_OK;
}

}  // namespace

extern "C" gr_status gr_bfs_static(int32_t n, int64_t m, const int32_t* row_offsets,
                                   const int32_t* cols, uint32_t flags, int32_t src,
                                   int32_t* depth, int32_t* pred, int32_t* status,
                                   void* stream) {
  if (n <= 0 || m < 0 || !row_offsets || (m > 0 && !cols) || !depth || src < 0 || src >= n ||
      (flags & ~GR_SYMMETRIC))
    return GR_ERR_INVALID_ARG;
  if ((int64_t)n > kStaticMaxVertices || m > kStaticMaxEdges) return GR_ERR_CAPACITY;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices) {
    (void)cudaGetLastError();
    return GR_ERR_CUDA;
  }
  StaticDevice* d = nullptr;
  gr_status st = static_setup(device, &d);
  if (st != GR_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* base = d->base;

  BfsArgs a = {};
  a.n = n;
  a.m = m;
  a.R = row_offsets;
  a.C = cols;
  a.depth = depth;
  a.pred = pred;
  a.visited = (uint32_t*)(base + kOffVisited);
  for (int i = 0; i < 3; ++i) a.front[i] = (uint32_t*)(base + kOffFront + i * kBitmapBytes);
  a.q[0] = (int32_t*)(base + kOffQ0);
  a.q[1] = (int32_t*)(base + kOffQ1);
  a.ch[0] = (int2*)(base + kOffCh0);
  a.ch[1] = (int2*)(base + kOffCh1);
  a.chunk_cap = kStaticChunkCap;
  a.ctl = (GrCtl*)(base + kOffCtl);
  a.status = (int*)(base + kOffStatus);
  a.src = src;
  a.nwords = (int32_t)(((int64_t)n + 31) / 32);
  a.use_do = (flags & GR_SYMMETRIC) ? 1 : 0;
  a.force_pull = 0;
  a.big = kStaticBig;
  a.track_deg = 1;  // the maximum degree is unknown without a validation pass
  a.do_a = 0.05f;
  a.do_b = 0.05f;
  a.spin = GR_DEFAULT_SPIN_LIMIT;
  a.level_stats = nullptr;
  a.max_levels = 0;
  a.bulk_edges = gr_default_bulk_edges(n);
  a.pdef = (int32_t*)(base + kOffPdef);

  // the control block and the status word must start at zero; the rest of
  // the scratch is initialised by the kernel itself
  if (cudaMemsetAsync(base, 0, kOffQ0, s) != cudaSuccess) {
    (void)cudaGetLastError();
    return GR_ERR_CUDA;
  }
  void* args[] = {&a};
  if (cudaLaunchCooperativeKernel(bfs_kernel(a), dim3(d->blocks[a.use_do ? 1 : 0]), dim3(NT),
                                  args, 0, s) != cudaSuccess) {
    (void)cudaGetLastError();
    return GR_ERR_CUDA;
  }
  if (status && cudaMemcpyAsync(status, base + kOffStatus, sizeof(int32_t),
                                cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
    (void)cudaGetLastError();
    return GR_ERR_CUDA;
  }
  return GR_OK;
}
