// gr_bfs.cu — direction-optimising BFS as one persistent, cooperative kernel.
//
// The paper's BFS (Sec. 6.1) is a bulk-synchronous loop of advance + filter
// steps on a vertex frontier, with a per-iteration host round trip to test
// for an empty frontier (Sec. 5.3).  Here the whole loop runs on the device:
// every CTA of a co-resident grid executes every level, and a bounded grid
// barrier separates levels, so no level costs a launch or a device-to-host
// copy.  Each level is either
//   * push (Sec. 5.1): advance fused with the visit functor and the filter
//     (LB_CULL-style fusion, Sec. 5.3) — the frontier queue is expanded
//     warp-centrically (the warp scans its 32 rows' degrees and walks the
//     concatenated edges 32 at a time), rows of degree >= big_degree arrive
//     pre-split into 1024-edge chunks shared by the whole grid; a visited
//     bitmap with atomicOr claims each vertex once, so the output frontier
//     needs no separate dedup pass; or
//   * pull (Sec. 5.1.4, Alg. 2 Reverse_Advance): every unvisited vertex scans
//     its row for a member of the current frontier bitmap and stops at the
//     first hit; the unvisited set is the complement of the visited bitmap,
//     read one 32-vertex word per warp.
// The direction follows the paper's Eq. 5-6 (push -> pull when
// m_f > m_u * do_a, pull -> push when m_f < m_u * do_b) with m_f and m_u
// counted exactly: every discovered vertex adds its degree to m_f.
#include <climits>
#include <mutex>

#include "gr_internal.cuh"

namespace {

struct BfsArgs {
  int32_t n;
  int64_t m;
  const int32_t* __restrict__ R;
  const int32_t* __restrict__ C;
  int32_t* depth;
  int32_t* pred;
  uint32_t* visited;
  uint32_t* front[3];
  int32_t* q[2];
  int2* ch[2];
  int64_t chunk_cap;
  GrCtl* ctl;
  int* status;
  int32_t src;
  int32_t nwords;
  int use_do;       // maintain frontier bitmaps, allow pull levels
  int force_pull;   // pull on every level (testing / ablation)
  int track_deg;    // load the degree of every discovered vertex
  float do_a, do_b;
  int big;
  unsigned spin;
  int32_t* level_stats;
  int32_t max_levels;
};

constexpr int NT = GR_PERSIST_THREADS;

__global__ void __launch_bounds__(NT) bfs_persistent(BfsArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t gtid = (int64_t)blockIdx.x * NT + threadIdx.x;
  const int64_t gthreads = (int64_t)gridDim.x * NT;
  const int64_t gwarp = gtid >> 5, nwarps = gthreads >> 5;
  GrCtl* ctl = a.ctl;

  // ---- Set_Problem_Data: depth -1 / pred -1, the source at depth 0 ------
  for (int64_t v = gtid; v < a.n; v += gthreads) {
    a.depth[v] = v == a.src ? 0 : -1;
    if (a.pred) a.pred[v] = -1;
  }
  const int32_t sw = a.src >> 5;
  const uint32_t sbit = 1u << (a.src & 31);
  for (int64_t w = gtid; w < a.nwords; w += gthreads) {
    uint32_t x = w == sw ? sbit : 0u;
    a.visited[w] = x;
    if (a.use_do) {
      a.front[0][w] = x;
      a.front[1][w] = 0u;
      a.front[2][w] = 0u;
    }
  }
  if (gtid == 0) {
    int beg = a.R[a.src], deg = a.R[a.src + 1] - beg;
    if (a.track_deg && deg >= a.big)
      gr_register_chunks(a.ch[0], a.chunk_cap, &ctl->nchunk[0], &ctl->nbig[0], a.src, beg, deg,
                         a.status);
    else {
      a.q[0][0] = a.src;
      ctl->qlen[0] = 1;
    }
    ctl->mf[0] = (unsigned long long)deg;
  }
  if (!gr_grid_sync(ctl, a.status, a.spin)) return;

  const unsigned long long deadline = gr_globaltimer() + GR_TIME_LIMIT_NS;
  unsigned long long seen_edges = 0;  // sum of degrees of every visited vertex
  GrCounters cnt;
  int pull = 0;
  int L = 0;
  for (;; ++L) {
    const int s0 = L % 3, s1 = (L + 1) % 3, s2 = (L + 2) % 3;
    const int nq = min(__ldcg(&ctl->qlen[s0]), a.n);
    const int nch = (int)min((int64_t)__ldcg(&ctl->nchunk[s0]), a.chunk_cap);
    if (nq + nch == 0 || L > a.n) break;
    const int nf = nq + __ldcg(&ctl->nbig[s0]);
    const unsigned long long mf = __ldcg(&ctl->mf[s0]);
    seen_edges += mf;
    const unsigned long long mu = (unsigned long long)a.m > seen_edges
                                      ? (unsigned long long)a.m - seen_edges
                                      : 0ull;
    if (a.force_pull) {
      pull = 1;
    } else if (a.use_do) {  // Eq. 5 / Eq. 6 with exact m_f, m_u
      if (!pull && (double)mf > (double)mu * a.do_a) pull = 1;
      else if (pull && (double)mf < (double)mu * a.do_b) pull = 0;
    }
    if (gtid == 0) {
      gr_check_deadline(ctl, a.status, deadline);
      if (a.level_stats && L < a.max_levels) {
        a.level_stats[3 * L] = nf;
        a.level_stats[3 * L + 1] = pull;
        a.level_stats[3 * L + 2] = (int)min(mf, (unsigned long long)INT_MAX);
      }
      ctl->qlen[s2] = 0;
      ctl->nchunk[s2] = 0;
      ctl->nbig[s2] = 0;
      ctl->mf[s2] = 0ull;
    }
    if (a.use_do)
      for (int64_t w = gtid; w < a.nwords; w += gthreads) a.front[s2][w] = 0u;

    int32_t* qn = a.q[(L + 1) & 1];
    int2* chn = a.ch[(L + 1) & 1];
    uint32_t* fnext = a.front[s1];
    unsigned long long my_mf = 0;
    const int next_depth = L + 1;

    if (!pull) {
      // ---- push: advance + visit + cull fused ----------------------------
      const int32_t* q = a.q[L & 1];
      const int2* ch = a.ch[L & 1];
      auto visit = [&](bool active, int32_t u, uint32_t, int, int32_t v) {
        bool won = false;
        if (active) {
          ++cnt.edges;
          const uint32_t bit = 1u << (v & 31);
          uint32_t* wp = a.visited + (v >> 5);
          if (!(*wp & bit)) won = !(atomicOr(wp, bit) & bit);
        }
        int vbeg = 0, vdeg = 0;
        if (won) {
          ++cnt.updates;
          a.depth[v] = next_depth;
          if (a.pred) a.pred[v] = u;
          if (a.use_do) atomicOr(fnext + (v >> 5), 1u << (v & 31));
          if (a.track_deg) {
            vbeg = __ldg(a.R + v);
            vdeg = __ldg(a.R + v + 1) - vbeg;
            my_mf += (unsigned long long)vdeg;
          }
        }
        const bool big = won && vdeg >= a.big;
        gr_warp_append(qn, &ctl->qlen[s1], a.n, won && !big, v, lane);
        if (big)
          gr_register_chunks(chn, a.chunk_cap, &ctl->nchunk[s1], &ctl->nbig[s1], v, vbeg, vdeg,
                             a.status);
      };
      for (int64_t base = gwarp * 32; base < nq; base += nwarps * 32) {
        const int64_t i = base + lane;
        const bool valid = i < nq;
        int32_t u = 0;
        int beg = 0, deg = 0;
        if (valid) {
          ++cnt.verts;
          u = __ldcg(q + i);
          beg = __ldg(a.R + u);
          deg = __ldg(a.R + u + 1) - beg;
        }
        gr_warp_expand(a.R, a.C, valid, u, beg, deg, 0u, lane, visit);
      }
      for (int64_t c = gwarp; c < nch; c += nwarps) {
        const int2 cu = __ldcg(ch + c);
        const int e1 = min(cu.y + GR_CHUNK_EDGES, __ldg(a.R + cu.x + 1));
        if (lane == 0) ++cnt.verts;
        gr_warp_chunk(a.C, cu.x, cu.y, e1, 0u, lane, visit);
      }
    } else {
      // ---- pull: unvisited vertices look for a parent in the frontier ----
      const uint32_t* fcur = a.front[s0];
      for (int64_t w = gwarp; w < a.nwords; w += nwarps) {
        const uint32_t word = a.visited[w];
        if (word == 0xffffffffu) continue;
        const int64_t v64 = w * 32 + lane;
        const int32_t v = (int32_t)v64;
        const bool cand = v64 < a.n && !((word >> lane) & 1u);
        int32_t found = -1;
        int beg = 0, deg = 0;
        if (cand) {
          ++cnt.verts;
          beg = __ldg(a.R + v);
          deg = __ldg(a.R + v + 1) - beg;
          for (int e = beg; e < beg + deg; ++e) {
            ++cnt.edges;
            const int32_t u = __ldg(a.C + e);
            if ((fcur[u >> 5] >> (u & 31)) & 1u) {
              found = u;
              break;
            }
          }
        }
        const unsigned hit = __ballot_sync(GR_FULL_MASK, found >= 0);
        if (hit == 0u) continue;
        if (lane == 0) {
          a.visited[w] = word | hit;
          fnext[w] = hit;
        }
        if (found >= 0) {
          ++cnt.updates;
          a.depth[v] = next_depth;
          if (a.pred) a.pred[v] = found;
          my_mf += (unsigned long long)deg;
        }
        const bool big = found >= 0 && deg >= a.big;
        gr_warp_append(qn, &ctl->qlen[s1], a.n, found >= 0 && !big, v, lane);
        if (big)
          gr_register_chunks(chn, a.chunk_cap, &ctl->nchunk[s1], &ctl->nbig[s1], v, beg, deg,
                             a.status);
      }
    }
    my_mf = gr_warp_sum_u64(my_mf);
    if (lane == 0 && my_mf) atomicAdd(&ctl->mf[s1], my_mf);
    if (!gr_grid_sync(ctl, a.status, a.spin)) return;
  }
  cnt.flush(ctl);
  if (gtid == 0) ctl->levels = L;
}

}  // namespace

extern "C" void gr_bfs_opts_default(gr_bfs_opts* o) {
  if (!o) return;
  o->direction = GR_DIR_AUTO;
  o->do_a = 0.05f;
  o->do_b = 0.05f;
  o->big_degree = GR_DEFAULT_BIG_DEGREE;
  o->blocks_per_sm = 0;
  o->spin_limit = GR_DEFAULT_SPIN_LIMIT;
  o->ws = nullptr;
  o->level_stats = nullptr;
  o->max_levels = 0;
}

extern "C" gr_status gr_bfs(const gr_graph* g, int32_t src, int32_t* depth, int32_t* pred,
                            const gr_bfs_opts* opts, void* stream) {
  if (!g || !depth || g->n <= 0 || src < 0 || src >= g->n) return GR_ERR_INVALID_ARG;
  gr_bfs_opts o;
  gr_bfs_opts_default(&o);
  if (opts) o = *opts;
  if (o.direction < GR_DIR_AUTO || o.direction > GR_DIR_PULL || o.max_levels < 0 ||
      (o.max_levels > 0 && !o.level_stats))
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
  a.ch[0] = ws->chunks[0];
  a.ch[1] = ws->chunks[1];
  a.chunk_cap = ws->chunk_cap;
  a.ctl = ws->ctl;
  a.status = ws->status;
  a.src = src;
  a.nwords = (int32_t)(((int64_t)g->n + 31) / 32);
  a.use_do = symmetric && o.direction != GR_DIR_PUSH;
  a.force_pull = o.direction == GR_DIR_PULL;
  a.big = o.big_degree > 0 ? (o.big_degree < 32 ? 32 : o.big_degree) : GR_DEFAULT_BIG_DEGREE;
  a.track_deg = a.use_do || g->max_degree >= a.big;
  a.do_a = o.do_a;
  a.do_b = o.do_b;
  a.spin = o.spin_limit ? o.spin_limit : GR_DEFAULT_SPIN_LIMIT;
  a.level_stats = o.level_stats;
  a.max_levels = o.max_levels;

  const int blocks = gr_launch_blocks((const void*)bfs_persistent, NT, 0, g->num_sms,
                                      o.blocks_per_sm);
  if (blocks <= 0) return GR_ERR_CUDA;
  if (gr_reset_ctl(ws, s) != cudaSuccess) return GR_ERR_CUDA;
  void* args[] = {&a};
  if (cudaLaunchCooperativeKernel((const void*)bfs_persistent, dim3(blocks), dim3(NT), args, 0,
                                  s) != cudaSuccess) {
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
constexpr int kStaticBig = GR_DEFAULT_BIG_DEGREE;
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
constexpr size_t kStaticBytes = kOffFront + 3 * kBitmapBytes;  // about 9.6 MB

static __device__ __align__(256) unsigned char g_bfs_static_scratch[kStaticBytes];

struct StaticDevice {
  bool ready;
  unsigned char* base;  // device address of g_bfs_static_scratch
  int blocks;           // co-resident grid size for bfs_persistent
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
    const int blocks = gr_launch_blocks((const void*)bfs_persistent, NT, 0, sms, 0);
    if (blocks <= 0) return GR_ERR_CUDA;
    d.base = (unsigned char*)p;
    d.blocks = blocks;
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

  // the control block and the status word must start at zero; the rest of
  // the scratch is initialised by the kernel itself
  if (cudaMemsetAsync(base, 0, kOffQ0, s) != cudaSuccess) {
    (void)cudaGetLastError();
    return GR_ERR_CUDA;
  }
  void* args[] = {&a};
  if (cudaLaunchCooperativeKernel((const void*)bfs_persistent, dim3(d->blocks), dim3(NT), args,
                                  0, s) != cudaSuccess) {
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
