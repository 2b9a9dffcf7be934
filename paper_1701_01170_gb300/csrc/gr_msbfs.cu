// gr_msbfs.cu — bit-parallel multi-source BFS (gr_bfs_multi).
//
// The paper lists multi-source / concurrent BFS as future work (Sec. 8,
// "several active frontiers"); this is the batched form of its BFS: up to
// 256 sources traverse together, each vertex carrying W 64-bit words whose
// bit i says "reached by source i".  Per level the frontier word f[u] holds
// the bits that arrived at u in the previous level, and
//   next[v] = OR over neighbours u of f[u],   new[v] = next[v] & ~visit[v].
// A level is either
//   * push (few active vertices): the advance of Sec. 4.1 over the active
//     list with atomicOr into next[v], then a finalise pass; or
//   * pull (many active vertices, symmetric graphs only): every vertex that
//     still misses some source ORs its neighbours' frontier words.  A warp
//     takes 32 consecutive rows, walks their concatenated edges in 32-wide
//     strips (the warp-centric load balancing of the single-source kernel)
//     and combines each row's lanes with a segmented OR scan in registers —
//     no atomics.  Rows of degree >= big are cut into GR_CHUNK_EDGES-edge
//     chunks that all warps share and reduce with one atomicOr per chunk.
// visit[] after every level is kept (snapshot per level, up to 2 GB); a last
// pass turns the snapshots into the k x n depth matrix, writing each source's
// row with coalesced 128-byte stores.  A deeper traversal writes the depths
// found so far, then writes later depths directly as bits appear, keeping
// two snapshots in ping-pong.
#include <algorithm>
#include <climits>
#include <cstdint>
#include <mutex>
#include <new>
#include <vector>

#include "gr_internal.cuh"

typedef unsigned long long u64;

struct GrMsState {
  int32_t n;
  int big;
  u64* fcur;        // frontier words, n * 4
  u64* fnext;
  u64* acc;         // push accumulator / chunk accumulator, n * 4 (zero between levels)
  u64* snap;        // snapshots: snap_bytes, levels of n * W words each
  size_t snap_bytes;
  int32_t* active[2];
  int2* chunks;     // static (row, first edge) chunks of rows with degree >= big
  int nchunks;
  int32_t* d_srcs;  // up to 256 sources of the current pass
  int32_t* d_uniq;
  unsigned long long* ctl;  // [0] active count, [1] degree sum of the active vertices
  unsigned long long* h_ctl;
};

namespace {

constexpr int MS_T = 256;
constexpr int MS_MAXW = 4;
constexpr int MS_BIG = 1024;
constexpr size_t MS_SNAP_BUDGET = (size_t)2 << 30;  // bytes of per-level snapshots at most

struct MsArgs {
  int32_t n;
  const int32_t* __restrict__ R;
  const int32_t* __restrict__ C;
  const u64* fcur;
  u64* fnext;
  u64* acc;
  const u64* snap_cur;
  u64* snap_next;
  const int32_t* active;
  int nactive;
  int32_t* active_next;
  unsigned long long* ctl;
  const int2* chunks;
  int nchunks;
  int big;
  u64 mask[MS_MAXW];
  int32_t* depth;      // deep mode: depths written as bits appear (else NULL)
  int64_t row_stride;
  int32_t level_next;  // depth of the bits found in this level
};

template <int W>
__device__ __forceinline__ bool all_set(const u64 (&x)[W], const u64 (&m)[MS_MAXW]) {
  bool f = true;
#pragma unroll
  for (int w = 0; w < W; ++w) f = f && (x[w] == m[w]);
  return f;
}

template <int W>
__device__ __forceinline__ void load_words(const u64* p, u64 (&x)[W]) {
  if (W == 1) {
    x[0] = p[0];
  } else {
#pragma unroll
    for (int w = 0; w < W; w += 2) {
      ulonglong2 t = *reinterpret_cast<const ulonglong2*>(p + w);
      x[w] = t.x;
      x[w + 1] = t.y;
    }
  }
}

template <int W>
__device__ __forceinline__ void store_words(u64* p, const u64 (&x)[W]) {
  if (W == 1) {
    p[0] = x[0];
  } else {
#pragma unroll
    for (int w = 0; w < W; w += 2)
      *reinterpret_cast<ulonglong2*>(p + w) = make_ulonglong2(x[w], x[w + 1]);
  }
}

// Record the new bits of vertex v: snapshot, next frontier, active list.
// Called by all 32 lanes.
template <int W>
__device__ __forceinline__ void ms_commit(const MsArgs& a, bool valid, int32_t v,
                                          const u64 (&vis)[W], const u64 (&nw)[W], int deg,
                                          int lane, unsigned long long& degsum) {
  bool any = false;
  if (valid) {
    u64 nv[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
      nv[w] = vis[w] | nw[w];
      any = any || nw[w] != 0ull;
    }
    store_words<W>(a.snap_next + (size_t)v * W, nv);
    store_words<W>(a.fnext + (size_t)v * W, nw);
    if (any) degsum += (unsigned long long)deg;
    if (any && a.depth) {  // deep mode: one depth per new source bit
#pragma unroll
      for (int w = 0; w < W; ++w) {
        u64 x = nw[w];
        while (x) {
          const int b = __ffsll((long long)x) - 1;
          x &= x - 1ull;
          a.depth[(int64_t)(w * 64 + b) * a.row_stride + v] = a.level_next;
        }
      }
    }
  }
  unsigned mask = __ballot_sync(GR_FULL_MASK, any);
  if (mask) {
    int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(&a.ctl[0], (unsigned long long)__popc(mask));
    base = __shfl_sync(GR_FULL_MASK, base, leader);
    if (any) a.active_next[base + __popc(mask & ((1u << lane) - 1u))] = v;
  }
}

__device__ __forceinline__ void flush_degsum(unsigned long long* ctl, unsigned long long d) {
  d = gr_warp_sum_u64(d);
  if ((threadIdx.x & 31) == 0 && d) atomicAdd(&ctl[1], d);
}

// ---- push ---------------------------------------------------------------

template <int W>
__device__ __forceinline__ void push_edge(const MsArgs& a, int32_t u, int32_t v) {
  u64 x[W], vis[W];
  load_words<W>(a.fcur + (size_t)u * W, x);
  load_words<W>(a.snap_cur + (size_t)v * W, vis);
#pragma unroll
  for (int w = 0; w < W; ++w) {
    u64 y = x[w] & ~vis[w];
    if (y) gr_red_or_u64(&a.acc[(size_t)v * W + w], y);
  }
}

template <int W>
__global__ void __launch_bounds__(MS_T) ms_push(MsArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = ((int64_t)blockIdx.x * MS_T + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * MS_T) >> 5;
  for (int64_t base = gwarp * 32; base < a.nactive; base += nwarps * 32) {
    const int64_t i = base + lane;
    bool valid = i < a.nactive;
    int32_t u = 0;
    int beg = 0, deg = 0;
    if (valid) {
      u = a.active[i];
      beg = __ldg(a.R + u);
      deg = __ldg(a.R + u + 1) - beg;
      if (deg >= a.big) deg = 0;  // long rows go through the chunk list
    }
    gr_warp_expand(a.R, a.C, valid, u, beg, deg, 0u, lane,
                   [&](bool active, int32_t su, uint32_t, int, int32_t v) {
                     if (active) push_edge<W>(a, su, v);
                   });
  }
  for (int64_t c = gwarp; c < a.nchunks; c += nwarps) {
    const int2 ch = a.chunks[c];
    u64 x[W];
    load_words<W>(a.fcur + (size_t)ch.x * W, x);
    bool any = false;
#pragma unroll
    for (int w = 0; w < W; ++w) any = any || x[w] != 0ull;
    if (!any) continue;
    const int e1 = min(ch.y + GR_CHUNK_EDGES, __ldg(a.R + ch.x + 1));
    for (int e = ch.y + lane; e < e1; e += 32) push_edge<W>(a, ch.x, __ldg(a.C + e));
  }
}

template <int W>
__global__ void __launch_bounds__(MS_T) ms_finalize(MsArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * MS_T;
  unsigned long long degsum = 0;
  for (int64_t base = (int64_t)blockIdx.x * MS_T + (threadIdx.x & ~31); base < a.n;
       base += stride) {
    const int64_t v64 = base + lane;
    const bool valid = v64 < a.n;
    const int32_t v = (int32_t)v64;
    u64 vis[W], nx[W], nw[W];
    int deg = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) vis[w] = nx[w] = nw[w] = 0ull;
    if (valid) {
      load_words<W>(a.snap_cur + (size_t)v * W, vis);
      load_words<W>(a.acc + (size_t)v * W, nx);
      bool touched = false;
#pragma unroll
      for (int w = 0; w < W; ++w) {
        nw[w] = nx[w] & ~vis[w];
        touched = touched || nx[w] != 0ull;
      }
      if (touched) {
        u64 z[W];
#pragma unroll
        for (int w = 0; w < W; ++w) z[w] = 0ull;
        store_words<W>(a.acc + (size_t)v * W, z);
        deg = __ldg(a.R + v + 1) - __ldg(a.R + v);
      }
    }
    ms_commit<W>(a, valid, v, vis, nw, deg, lane, degsum);
  }
  flush_degsum(a.ctl, degsum);
}

// ---- pull ---------------------------------------------------------------

// Long rows: one warp per edge chunk ORs its neighbours' frontier words
// and merges the result into acc[row] with one atomicOr per word.
template <int W>
__global__ void __launch_bounds__(MS_T) ms_pull_chunks(MsArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = ((int64_t)blockIdx.x * MS_T + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * MS_T) >> 5;
  for (int64_t c = gwarp; c < a.nchunks; c += nwarps) {
    const int2 ch = a.chunks[c];
    u64 vis[W];
    load_words<W>(a.snap_cur + (size_t)ch.x * W, vis);
    if (all_set<W>(vis, a.mask)) continue;
    const int e1 = min(ch.y + GR_CHUNK_EDGES, __ldg(a.R + ch.x + 1));
    u64 acc[W];
#pragma unroll
    for (int w = 0; w < W; ++w) acc[w] = 0ull;
    for (int e = ch.y + lane; e < e1; e += 32) {
      u64 x[W];
      load_words<W>(a.fcur + (size_t)__ldg(a.C + e) * W, x);
#pragma unroll
      for (int w = 0; w < W; ++w) acc[w] |= x[w];
    }
#pragma unroll
    for (int w = 0; w < W; ++w) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[w] |= __shfl_xor_sync(GR_FULL_MASK, acc[w], o);
      const u64 y = acc[w] & ~vis[w];
      if (lane == 0 && y) gr_red_or_u64(&a.acc[(size_t)ch.x * W + w], y);
    }
  }
}

template <int W>
__global__ void __launch_bounds__(MS_T) ms_pull(MsArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = ((int64_t)blockIdx.x * MS_T + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * MS_T) >> 5;
  unsigned long long degsum = 0;
  for (int64_t v0 = gwarp * 32; v0 < a.n; v0 += nwarps * 32) {
    const int64_t v64 = v0 + lane;
    const bool valid = v64 < a.n;
    const int32_t v = (int32_t)v64;
    u64 vis[W];
#pragma unroll
    for (int w = 0; w < W; ++w) vis[w] = a.mask[w];
    int beg = 0, rowdeg = 0;
    if (valid) {
      load_words<W>(a.snap_cur + (size_t)v * W, vis);
      beg = __ldg(a.R + v);
      rowdeg = __ldg(a.R + v + 1) - beg;
    }
    const bool full = all_set<W>(vis, a.mask);
    const bool longrow = rowdeg >= a.big;
    const int deg = (valid && !full && !longrow) ? rowdeg : 0;
    int total;
    const int off = gr_warp_excl_scan(deg, lane, &total);
    u64 acc[W];
#pragma unroll
    for (int w = 0; w < W; ++w) acc[w] = 0ull;
    for (int base = 0; base < total; base += 32) {
      const int pos = base + lane;
      int lo = 0;
#pragma unroll
      for (int step = 16; step >= 1; step >>= 1) {
        const int cand = lo + step;
        if (__shfl_sync(GR_FULL_MASK, off, cand) <= pos) lo = cand;
      }
      const int sbeg = __shfl_sync(GR_FULL_MASK, beg, lo);
      const int soff = __shfl_sync(GR_FULL_MASK, off, lo);
      const bool active = pos < total;
      u64 x[W];
#pragma unroll
      for (int w = 0; w < W; ++w) x[w] = 0ull;
      if (active) load_words<W>(a.fcur + (size_t)__ldg(a.C + sbeg + (pos - soff)) * W, x);
      // segmented inclusive OR over lanes of the same row (rows are contiguous)
      const int row = active ? lo : 32 + lane;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int rs = __shfl_up_sync(GR_FULL_MASK, row, d);
#pragma unroll
        for (int w = 0; w < W; ++w) {
          const u64 y = __shfl_up_sync(GR_FULL_MASK, x[w], d);
          if (lane >= d && rs == row) x[w] |= y;
        }
      }
      // the owner lane of each row takes its segment's total from the
      // segment's last lane in this strip
      const int first = off - base, last = off + deg - 1 - base;
      const bool inter = deg > 0 && last >= 0 && first < 32;
      const int src = inter ? min(last, 31) : 0;
#pragma unroll
      for (int w = 0; w < W; ++w) {
        const u64 t = __shfl_sync(GR_FULL_MASK, x[w], src);
        if (inter) acc[w] |= t;
      }
    }
    if (valid && !full && longrow) {
      load_words<W>(a.acc + (size_t)v * W, acc);
      u64 z[W];
#pragma unroll
      for (int w = 0; w < W; ++w) z[w] = 0ull;
      store_words<W>(a.acc + (size_t)v * W, z);
    }
    u64 nw[W];
#pragma unroll
    for (int w = 0; w < W; ++w) nw[w] = acc[w] & ~vis[w];
    ms_commit<W>(a, valid, v, vis, nw, rowdeg, lane, degsum);
  }
  flush_degsum(a.ctl, degsum);
}

// ---- depth matrix ---------------------------------------------------------

// depth[i * n + v] = the first level whose snapshot holds bit i at v, or -1.
// Warp-lane j handles vertex v0 + j; the warps of a CTA split the sources, so
// each store instruction writes 32 consecutive ints of one source's row.
template <int W>
__global__ void __launch_bounds__(MS_T) ms_depth(int32_t n, const u64* snap, int levels, int k,
                                                 int32_t* depth, int64_t row_stride) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const size_t lvl_stride = (size_t)n * W;
  for (int64_t v0 = (int64_t)blockIdx.x * 32; v0 < n; v0 += (int64_t)gridDim.x * 32) {
    const int64_t v = v0 + lane;
    const bool valid = v < n;
    for (int i = wid; i < k; i += MS_T / 32) {
      int d = -1;
      if (valid) {
        const int w = i >> 6;
        const u64 bit = 1ull << (i & 63);
        const u64* p = snap + (size_t)v * W + w;
        if (p[(size_t)(levels - 1) * lvl_stride] & bit) {  // reached at all?
          int lo = 0, hi = levels - 1;                       // first level with the bit
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (p[(size_t)mid * lvl_stride] & bit) hi = mid;
            else lo = mid + 1;
          }
          d = lo;
        }
        depth[(int64_t)i * row_stride + v] = d;
      }
    }
  }
}

__global__ void ms_set_sources(const int32_t* srcs, int k, u64* snap0, u64* fcur, int W) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  const int32_t v = srcs[i];
  const u64 bit = 1ull << (i & 63);
  atomicOr(&snap0[(size_t)v * W + (i >> 6)], bit);
  atomicOr(&fcur[(size_t)v * W + (i >> 6)], bit);
}

__global__ void ms_collect_chunks(int32_t n, const int32_t* R, int big, int2* chunks, int* count,
                                  int cap) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int beg = R[v], deg = R[v + 1] - beg;
    if (deg < big) continue;
    const int nch = (deg + GR_CHUNK_EDGES - 1) / GR_CHUNK_EDGES;
    const int pos = atomicAdd(count, nch);
    for (int c = 0; c < nch && pos + c < cap; ++c)
      chunks[pos + c] = make_int2((int)v, beg + c * GR_CHUNK_EDGES);
  }
}

}  // namespace

void gr_ms_free(GrMsState* ms) {
  if (!ms) return;
  void* ptrs[] = {ms->fcur, ms->fnext, ms->acc, ms->snap, ms->active[0], ms->active[1],
                  ms->chunks, ms->d_srcs, ms->d_uniq, ms->ctl};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (ms->h_ctl) cudaFreeHost(ms->h_ctl);
  delete ms;
}

static gr_status ms_alloc(const gr_graph* g, GrMsState** out) {
  GrMsState* ms = new (std::nothrow) GrMsState();
  if (!ms) return GR_ERR_OOM;
  ms->n = g->n;
  ms->big = MS_BIG;
  const size_t words = ((size_t)g->n + 1) * MS_MAXW;
  const int64_t chunk_cap = g->m / GR_CHUNK_EDGES + g->m / MS_BIG + 2;
  // room for 16 levels at the widest word count, within the snapshot budget,
  // and never less than the two levels of deep mode
  ms->snap_bytes = std::max<size_t>(2 * words * 8, std::min<size_t>(16 * words * 8, MS_SNAP_BUDGET));
  bool ok = cudaMalloc(&ms->fcur, words * 8) == cudaSuccess &&
            cudaMalloc(&ms->fnext, words * 8) == cudaSuccess &&
            cudaMalloc(&ms->acc, words * 8) == cudaSuccess &&
            cudaMalloc(&ms->snap, ms->snap_bytes) == cudaSuccess &&
            cudaMalloc(&ms->active[0], ((size_t)g->n + 1) * 4) == cudaSuccess &&
            cudaMalloc(&ms->active[1], ((size_t)g->n + 1) * 4) == cudaSuccess &&
            cudaMalloc(&ms->chunks, (size_t)chunk_cap * sizeof(int2)) == cudaSuccess &&
            cudaMalloc(&ms->d_srcs, 256 * 4) == cudaSuccess &&
            cudaMalloc(&ms->d_uniq, 256 * 4) == cudaSuccess &&
            cudaMalloc(&ms->ctl, 4 * sizeof(unsigned long long)) == cudaSuccess &&
            cudaMallocHost(&ms->h_ctl, 4 * sizeof(unsigned long long)) == cudaSuccess;
  if (ok) {
    int* cnt = (int*)ms->ctl;
    ok = cudaMemset(ms->acc, 0, words * 8) == cudaSuccess &&
         cudaMemset(cnt, 0, sizeof(int)) == cudaSuccess;
    if (ok && g->m > 0) {
      ms_collect_chunks<<<g->num_sms * 4, 256>>>(g->n, g->R, MS_BIG, ms->chunks, cnt,
                                                 (int)chunk_cap);
      int h = 0;
      ok = cudaGetLastError() == cudaSuccess &&
           cudaMemcpy(&h, cnt, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess;
      ms->nchunks = (int)std::min<int64_t>(h, chunk_cap);
    }
  }
  if (!ok) {
    (void)cudaGetLastError();
    gr_ms_free(ms);
    return GR_ERR_OOM;
  }
  *out = ms;
  return GR_OK;
}

// Grow the snapshot buffer to at least `bytes` (synchronous), within
// MS_SNAP_BUDGET; returns false if that is not possible.
static bool ms_grow_snap(GrMsState* ms, size_t bytes, cudaStream_t s) {
  if (bytes <= ms->snap_bytes) return true;
  size_t cap = ms->snap_bytes;
  while (cap < bytes) cap *= 2;
  if (cap > MS_SNAP_BUDGET) cap = std::max(bytes, MS_SNAP_BUDGET);
  if (cap > MS_SNAP_BUDGET) return false;
  u64* p = nullptr;
  if (cudaMalloc(&p, cap) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  if (cudaMemcpyAsync(p, ms->snap, ms->snap_bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    (void)cudaGetLastError();
    cudaFree(p);
    return false;
  }
  cudaFree(ms->snap);
  ms->snap = p;
  ms->snap_bytes = cap;
  return true;
}

template <int W>
static gr_status ms_run(const gr_graph* g, GrMsState* ms, const int32_t* srcs, int k,
                        int32_t* depth, int64_t row_stride, int direction, float push_ratio,
                        int snapshot_levels, cudaStream_t s) {
  const int32_t n = g->n;
  // per-level snapshot stride uses W words per vertex
  const size_t lvl = (size_t)n * W;
  std::vector<int32_t> uniq(srcs, srcs + k);
  std::sort(uniq.begin(), uniq.end());
  uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
  if (cudaMemcpyAsync(ms->d_srcs, srcs, k * 4, cudaMemcpyHostToDevice, s) ||
      cudaMemcpyAsync(ms->active[0], uniq.data(), uniq.size() * 4, cudaMemcpyHostToDevice, s) ||
      cudaMemsetAsync(ms->snap, 0, lvl * 8, s) || cudaMemsetAsync(ms->fcur, 0, lvl * 8, s))
    return GR_ERR_CUDA;
  ms_set_sources<<<(k + 255) / 256, 256, 0, s>>>(ms->d_srcs, k, ms->snap, ms->fcur, W);

  MsArgs a = {};
  a.n = n;
  a.R = g->R;
  a.C = g->C;
  a.acc = ms->acc;
  a.ctl = ms->ctl;
  a.chunks = ms->chunks;
  a.nchunks = ms->nchunks;
  a.big = ms->big;
  for (int w = 0; w < MS_MAXW; ++w) {
    const int bits = k - 64 * w;
    a.mask[w] = bits >= 64 ? ~0ull : (bits <= 0 ? 0ull : ((1ull << bits) - 1ull));
  }
  const bool can_pull = (g->flags & GR_SYMMETRIC) && direction != GR_DIR_PUSH;
  const int blocks = g->num_sms * 8;
  int nactive = (int)uniq.size();
  unsigned long long degsum = 0;
  u64* fcur = ms->fcur;
  u64* fnext = ms->fnext;
  int level = 0;
  // Snapshot mode keeps one visit snapshot per level and writes the depth
  // matrix at the end in one coalesced pass; when the traversal outgrows the
  // snapshot budget (or snapshot_levels) the depths found so far are written
  // and later ones go straight to the matrix (deep mode), with two snapshot
  // slots in ping-pong.
  const int limit = snapshot_levels > 0 ? std::max(2, snapshot_levels) : INT_MAX;
  bool deep = false;
  int cur_slot = 0, next_slot = 1;
  while (nactive > 0) {
    if (!deep) {
      if (level + 2 <= limit && ms_grow_snap(ms, (size_t)(level + 2) * lvl * 8, s)) {
        cur_slot = level;
        next_slot = level + 1;
      } else {
        // levels 0..level are complete: write their depths, then go deep
        ms_depth<W><<<std::min<int64_t>(((int64_t)n + 31) / 32, (int64_t)g->num_sms * 16), MS_T, 0,
                       s>>>(n, ms->snap, level + 1, k, depth, row_stride);
        if (cudaGetLastError() != cudaSuccess) return GR_ERR_CUDA;
        deep = true;
        cur_slot = level;
        next_slot = level == 0 ? 1 : 0;
      }
    }
    a.fcur = fcur;
    a.fnext = fnext;
    a.snap_cur = ms->snap + (size_t)cur_slot * lvl;
    a.snap_next = ms->snap + (size_t)next_slot * lvl;
    a.depth = deep ? depth : nullptr;
    a.row_stride = row_stride;
    a.level_next = level + 1;
    a.active = ms->active[level & 1];
    a.nactive = nactive;
    a.active_next = ms->active[(level + 1) & 1];
    if (cudaMemsetAsync(ms->ctl, 0, 2 * sizeof(unsigned long long), s)) return GR_ERR_CUDA;
    const bool pull = can_pull && level > 0 &&
                      (direction == GR_DIR_PULL ||
                       (double)degsum > (double)g->m * (double)push_ratio);
    if (pull) {
      if (a.nchunks > 0) ms_pull_chunks<W><<<blocks, MS_T, 0, s>>>(a);
      ms_pull<W><<<blocks, MS_T, 0, s>>>(a);
    } else {
      ms_push<W><<<blocks, MS_T, 0, s>>>(a);
      ms_finalize<W><<<blocks, MS_T, 0, s>>>(a);
    }
    if (cudaGetLastError() != cudaSuccess) return GR_ERR_CUDA;
    if (cudaMemcpyAsync(ms->h_ctl, ms->ctl, 2 * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, s) ||
        cudaStreamSynchronize(s))
      return GR_ERR_CUDA;
    nactive = (int)ms->h_ctl[0];
    degsum = ms->h_ctl[1];
    std::swap(fcur, fnext);
    if (deep) std::swap(cur_slot, next_slot);
    ++level;
  }
  if (!deep) {
    // levels 0..level are valid snapshots (the last one adds nothing)
    ms_depth<W><<<std::min<int64_t>(((int64_t)n + 31) / 32, (int64_t)g->num_sms * 16), MS_T, 0,
                   s>>>(n, ms->snap, level + 1, k, depth, row_stride);
    if (cudaGetLastError() != cudaSuccess) return GR_ERR_CUDA;
  }
  return GR_OK;
}

extern "C" void gr_msbfs_opts_default(gr_msbfs_opts* o) {
  if (!o) return;
  o->direction = GR_DIR_AUTO;
  o->push_ratio = 0.02f;
  o->snapshot_levels = 0;
}

extern "C" gr_status gr_bfs_multi(const gr_graph* g, const int32_t* srcs, int32_t k,
                                  int32_t* depth, const gr_msbfs_opts* opts, void* stream) {
  if (!g || !srcs || k < 0 || (k > 0 && !depth) || g->n <= 0) return GR_ERR_INVALID_ARG;
  for (int i = 0; i < k; ++i)
    if (srcs[i] < 0 || srcs[i] >= g->n) return GR_ERR_INVALID_ARG;
  gr_msbfs_opts o;
  gr_msbfs_opts_default(&o);
  if (opts) o = *opts;
  if (o.direction < GR_DIR_AUTO || o.direction > GR_DIR_PULL || o.snapshot_levels < 0)
    return GR_ERR_INVALID_ARG;
  if (k == 0) return GR_OK;
  // The multi-source scratch belongs to the graph, so calls on one graph run
  // one at a time: a call holds its graph's lock (one of 64, picked by the
  // handle's address) until its last kernel has finished with that scratch.
  static std::mutex graph_locks[64];
  std::lock_guard<std::mutex> hold(graph_locks[((uintptr_t)g >> 4) % 64]);
  gr_graph* gm = const_cast<gr_graph*>(g);
  if (!gm->ms) {
    gr_status st = ms_alloc(g, &gm->ms);
    if (st != GR_OK) return st;
  }
  cudaStream_t s = (cudaStream_t)stream;
  gr_status st = GR_OK;
  for (int base = 0; base < k && st == GR_OK; base += 256) {
    const int kk = std::min(256, k - base);
    int32_t* out = depth + (int64_t)base * g->n;
    if (kk <= 64)
      st = ms_run<1>(g, gm->ms, srcs + base, kk, out, g->n, o.direction, o.push_ratio,
                     o.snapshot_levels, s);
    else if (kk <= 128)
      st = ms_run<2>(g, gm->ms, srcs + base, kk, out, g->n, o.direction, o.push_ratio,
                     o.snapshot_levels, s);
    else
      st = ms_run<4>(g, gm->ms, srcs + base, kk, out, g->n, o.direction, o.push_ratio,
                     o.snapshot_levels, s);
  }
  // kernels already queued still use the scratch (the depth pass reads the
  // snapshots): let them finish before the lock goes, on errors too
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    (void)cudaGetLastError();
    return GR_ERR_CUDA;
  }
  return st;
}
