// gr_ops.cu — the standalone advance and filter operators (gr_advance, gr_filter).
//
// Advance (Sec. 4.1, Fig. "advance"): a prefix-sum of the input degrees gives
// every input item its output offset; the load balancer then hands every
// warp 32 consecutive OUTPUT positions (load balance over the output
// frontier, Sec. 5.1.3), and each lane finds the input item owning its
// position by a sorted search in the scanned offsets.
//
// Filter (Sec. 4.2, Fig. "filter"): exact modes are a global scan and
// scatter (stable compaction); CULL is the inexact "uniquification" of
// Sec. 5.2.1 done with a claim bitmap.
#include <climits>

#include "gr_internal.cuh"

namespace {

constexpr int T = GR_OPS_THREADS;
constexpr int ITEMS = GR_SCAN_ITEMS;
constexpr int TILE = GR_SCAN_TILE;

__device__ __forceinline__ int64_t eff_len(const int64_t* len_dev, int64_t len_host) {
  if (!len_dev) return len_host;
  int64_t l = *len_dev;
  return l < 0 ? 0 : (l < len_host ? l : len_host);
}

// Exclusive block scan of a 64-bit value over NT threads; *total gets the block sum.
template <int NT>
__device__ __forceinline__ long long block_excl_scan(long long x, long long* total) {
  __shared__ long long warp_tot[NT / 32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(GR_FULL_MASK, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    long long t = lane < NT / 32 ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(GR_FULL_MASK, t, o);
      if (lane >= o) t += y;
    }
    if (lane < NT / 32) warp_tot[lane] = t;
  }
  __syncthreads();
  long long base = wid ? warp_tot[wid - 1] : 0;
  *total = warp_tot[NT / 32 - 1];
  __syncthreads();
  return base + incl - x;
}

// 64-bit warp-aggregated append into a user buffer with a 64-bit counter.
__device__ __forceinline__ void warp_append64(int32_t* out, unsigned long long* len, int64_t cap,
                                              bool take, int32_t v, int lane, int* status) {
  unsigned mask = __ballot_sync(GR_FULL_MASK, take);
  if (mask == 0) return;
  int leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(len, (unsigned long long)__popc(mask));
  base = __shfl_sync(GR_FULL_MASK, base, leader);
  if (take) {
    long long pos = (long long)base + __popc(mask & ((1u << lane) - 1u));
    if (pos < cap) out[pos] = v;
    else gr_set_status(status, GR_ERR_CAPACITY);
  }
}

// Single-CTA exclusive scan of `count` block sums in place (two interleaved
// arrays when `pairs`), total(s) to tot[0] (and tot[1]).
__global__ void scan_block_sums(long long* sums, int64_t count, int pairs, long long* tot) {
  __shared__ long long carry[2];
  int64_t per = (count + blockDim.x - 1) / blockDim.x;
  int64_t b0 = threadIdx.x * per, b1 = min(b0 + per, count);
  for (int k = 0; k < (pairs ? 2 : 1); ++k) {
    long long* a = sums + k * (GR_MAX_SCAN_BLOCKS / 2);
    long long s = 0;
    for (int64_t i = b0; i < b1; ++i) s += a[i];
    long long total;
    long long off = block_excl_scan<1024>(s, &total);
    for (int64_t i = b0; i < b1; ++i) {
      long long x = a[i];
      a[i] = off;
      off += x;
    }
    if (threadIdx.x == 0) carry[k] = total;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    tot[0] = carry[0];
    if (pairs) tot[1] = carry[1];
  }
}

// ---------------------------------------------------------------------------
// advance: degree scan

__global__ void adv_degree_tiles(const int32_t* __restrict__ R, const int32_t* __restrict__ in,
                                 int64_t len_host, const int64_t* len_dev, int32_t n,
                                 long long* item_off, long long* block_sums, int* status) {
  int64_t len = eff_len(len_dev, len_host);
  int64_t base = (int64_t)blockIdx.x * TILE + (int64_t)threadIdx.x * ITEMS;
  long long d[ITEMS];
  long long s = 0;
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    int64_t i = base + k;
    d[k] = 0;
    if (i < len) {
      int u = in[i];
      if (u >= 0 && u < n) d[k] = R[u + 1] - R[u];
      else gr_set_status(status, GR_ERR_INVALID_ARG);
    }
    s += d[k];
  }
  long long total;
  long long off = block_excl_scan<T>(s, &total);
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    int64_t i = base + k;
    if (i < len) item_off[i] = off;
    off += d[k];
  }
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

__device__ __forceinline__ long long item_offset(const long long* item_off,
                                                 const long long* block_sums, int64_t i) {
  return block_sums[i / TILE] + item_off[i];
}

// Largest i in [lo, hi] with offset(i) <= p (offsets are non-decreasing).
__device__ __forceinline__ int64_t search_item(const long long* item_off,
                                               const long long* block_sums, int64_t lo,
                                               int64_t hi, long long p) {
  while (lo < hi) {
    int64_t mid = lo + ((hi - lo + 1) >> 1);
    if (item_offset(item_off, block_sums, mid) <= p) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

enum { FN_NONE_ORDERED = 0, FN_NONE_EDGES = 1, FN_BFS = 2, FN_BFS_IDEM = 3, FN_RELAX = 4 };

struct ExpandArgs {
  int32_t n;
  const int32_t* R;
  const int32_t* C;
  const uint32_t* W;
  const int32_t* in;
  int64_t len_host;
  const int64_t* len_dev;
  const long long* item_off;
  const long long* block_sums;
  const long long* total;
  int32_t* out;
  int64_t cap;
  unsigned long long* out_len;
  int* status;
  // functor state
  int32_t* depth;
  int32_t* pred;
  int32_t level;
  unsigned long long* key;
  // first item of each output tile (adv_tile_map), for tiles t < tile_cap
  const int32_t* tile_item;
  int64_t tile_cap;
};

// Output-balanced expansion over output tiles: a CTA owns GR_ADV_TILE
// consecutive output positions at a time.  The tile's first input item comes
// from the tile map (the item holding the tile's first position, written by
// adv_tile_map in one pass over the items), its last from the next tile's
// entry; the items in between — their offsets, vertex ids and row starts —
// are staged in shared memory, and every output position then finds its item
// with a search in shared memory.  A warp's 32 outputs are consecutive
// positions, so the column loads and the output stores are coalesced.  Tiles
// beyond the map's capacity find their items with binary searches over the
// scanned offsets, and a tile that spans more items than the stage holds (a
// run of empty rows) searches global memory per position.
#define GR_ADV_PER_THREAD 8
#define GR_ADV_TILE (T * GR_ADV_PER_THREAD)

// tile_item[t] = the item holding output position t * GR_ADV_TILE (the
// largest item whose offset is at most that position), for every tile t <
// tile_cap that starts below the total.  Only items that own positions write.
__global__ void adv_tile_map(const long long* item_off, const long long* block_sums,
                             int64_t len_host, const int64_t* len_dev, const long long* total,
                             int32_t* tile_item, int64_t tile_cap) {
  const int64_t len = eff_len(len_dev, len_host);
  const long long tot = *total;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x) {
    const long long o = item_offset(item_off, block_sums, i);
    const long long o1 = i + 1 < len ? item_offset(item_off, block_sums, i + 1) : tot;
    for (long long t = (o + GR_ADV_TILE - 1) / GR_ADV_TILE;
         t < tile_cap && t * GR_ADV_TILE < o1; ++t)
      tile_item[t] = (int32_t)i;
  }
}
template <int FN>
__global__ void adv_expand(ExpandArgs a) {
  __shared__ long long s_off[GR_ADV_TILE + 1];
  __shared__ int s_beg[GR_ADV_TILE + 1];
  __shared__ int s_u[GR_ADV_TILE + 1];
  __shared__ long long s_i0, s_ni;
  int64_t len = eff_len(a.len_dev, a.len_host);
  long long total = *a.total;
  int lane = threadIdx.x & 31;
  long long limit = total;
  if (FN == FN_NONE_ORDERED || FN == FN_NONE_EDGES) limit = total < a.cap ? total : a.cap;
  for (long long t0 = (long long)blockIdx.x * GR_ADV_TILE; t0 < limit;
       t0 += (long long)gridDim.x * GR_ADV_TILE) {
    const long long tend = min(t0 + (long long)GR_ADV_TILE, limit);
    if (threadIdx.x == 0) {
      const long long t = t0 / GR_ADV_TILE;
      const int64_t i0 = t < a.tile_cap ? (int64_t)a.tile_item[t]
                                        : search_item(a.item_off, a.block_sums, 0, len - 1, t0);
      // the item holding the next tile's first position bounds this tile's
      // last item (staged one too many at most, which no position selects)
      int64_t i1;
      if (tend >= total) i1 = len - 1;
      else if (t + 1 < a.tile_cap) i1 = (int64_t)a.tile_item[t + 1];
      else i1 = search_item(a.item_off, a.block_sums, i0, len - 1, tend - 1);
      s_i0 = i0;
      s_ni = i1 - i0 + 1;
    }
    __syncthreads();
    const int64_t i0 = s_i0, ni = s_ni;
    const bool staged = ni <= GR_ADV_TILE + 1;
    if (staged) {
      for (int j = threadIdx.x; j < ni; j += T) {
        const int64_t i = i0 + j;
        const int32_t u = a.in[i];
        s_off[j] = item_offset(a.item_off, a.block_sums, i);
        s_u[j] = u;
        s_beg[j] = u >= 0 && u < a.n ? a.R[u] : 0;  // invalid items have no outputs
      }
    }
    __syncthreads();
    for (int k = 0; k < GR_ADV_PER_THREAD; ++k) {
    const long long p = t0 + (long long)k * T + threadIdx.x;
    bool active = p < tend;
    int32_t v = 0, u = 0;
    int e = 0;
    if (active) {
      if (staged) {
        int lo = 0, hi = (int)ni - 1;  // largest j with s_off[j] <= p
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (s_off[mid] <= p) lo = mid;
          else hi = mid - 1;
        }
        u = s_u[lo];
        e = s_beg[lo] + (int)(p - s_off[lo]);
      } else {
        const int64_t i = search_item(a.item_off, a.block_sums, i0, i0 + ni - 1, p);
        u = a.in[i];
        e = a.R[u] + (int)(p - item_offset(a.item_off, a.block_sums, i));
      }
      v = __ldg(a.C + e);
    }
    if (FN == FN_NONE_ORDERED) {
      if (active) a.out[p] = v;
    } else if (FN == FN_NONE_EDGES) {
      if (active) a.out[p] = e;
    } else if (FN == FN_BFS || FN == FN_BFS_IDEM) {
      bool won = false;
      if (active && a.depth[v] == -1) {
        if (FN == FN_BFS) {
          won = atomicCAS(&a.depth[v], -1, a.level + 1) == -1;
        } else {
          a.depth[v] = a.level + 1;
          won = true;
        }
        if (won && a.pred) a.pred[v] = u;
      }
      warp_append64(a.out, a.out_len, a.cap, won, v, lane, a.status);
    } else {  // FN_RELAX
      bool improved = false;
      if (active) {
        unsigned long long ku = a.key[u];
        unsigned du = (unsigned)(ku >> 32);
        if (du != GR_INF_DIST) {
          unsigned long long nd = (unsigned long long)du + a.W[e];
          if (nd >= (unsigned long long)GR_INF_DIST) {
            // an unrepresentable candidate matters only for an unreached target
            if ((a.key[v] >> 32) == GR_INF_DIST) gr_set_status(a.status, GR_ERR_OVERFLOW);
          } else {
            unsigned long long cand = (nd << 32) | (unsigned)u;
            if (cand < a.key[v]) {
              unsigned long long old = atomicMin(&a.key[v], cand);
              improved = (old >> 32) > nd;
            }
          }
        }
      }
      warp_append64(a.out, a.out_len, a.cap, improved, v, lane, a.status);
    }
    }
    __syncthreads();  // the next tile overwrites the stage
  }
}

__global__ void write_len_and_check(const long long* total, unsigned long long* out_len,
                                    int64_t cap, int* status) {
  long long t = *total;
  *out_len = (unsigned long long)t;
  if (t > cap) gr_set_status(status, GR_ERR_CAPACITY);
}

// ---------------------------------------------------------------------------
// ordered compaction (filters and the pull advance)

enum { CL_UNIQUE = 0, CL_UNVISITED = 1, CL_NEAR_FAR = 2, CL_PULL = 3 };

struct CompactArgs {
  int32_t n;
  const int32_t* R;
  const int32_t* C;
  const int32_t* in;
  int64_t len_host;
  const int64_t* len_dev;
  long long* block_sums;   // two interleaved halves for two-output modes
  const long long* totals; // device scan totals
  int32_t* out;
  int64_t cap;
  unsigned long long* out_len;
  int32_t* far;
  int64_t far_cap;
  unsigned long long* far_len;
  int* status;
  int32_t* first_idx;
  int32_t* depth;
  int32_t* pred;
  int32_t level;
  const unsigned long long* key;
  uint32_t threshold;
  int32_t* tags;
};

// Class of item i: 0 dropped, 1 to out, 2 to far.  In the count pass
// (SCATTER == false) CL_PULL does the neighbour scan and records the found
// parent in tags[i]; the scatter pass reads it back.
template <int CL, bool SCATTER>
__device__ __forceinline__ int classify(const CompactArgs& a, int64_t i) {
  if (CL == CL_UNVISITED) return a.depth[i] == -1 ? 1 : 0;
  int32_t v = a.in[i];
  if (v < 0 || v >= a.n) return 0;
  if (CL == CL_UNIQUE) {
    if (a.first_idx[v] != (int32_t)i) return 0;
    if (SCATTER) a.first_idx[v] = INT32_MAX;  // leave the scratch clean
    return 1;
  }
  if (CL == CL_NEAR_FAR) return (unsigned)(a.key[v] >> 32) < a.threshold ? 1 : 2;
  // CL_PULL
  if (SCATTER) return a.tags[i] >= 0 ? 1 : 0;
  int32_t found = -1;
  if (a.depth[v] == -1) {
    for (int e = a.R[v]; e < a.R[v + 1]; ++e) {
      int32_t u = __ldg(a.C + e);
      if (a.depth[u] == a.level) { found = u; break; }
    }
  }
  a.tags[i] = found;
  return found >= 0 ? 1 : 0;
}

template <int CL>
__global__ void compact_count(CompactArgs a) {
  int64_t len = CL == CL_UNVISITED ? a.n : eff_len(a.len_dev, a.len_host);
  int64_t base = (int64_t)blockIdx.x * TILE + (int64_t)threadIdx.x * ITEMS;
  long long c1 = 0, c2 = 0;
  for (int k = 0; k < ITEMS; ++k) {
    int64_t i = base + k;
    if (i >= len) break;
    int c = classify<CL, false>(a, i);
    c1 += c == 1;
    c2 += c == 2;
  }
  long long t1, t2;
  block_excl_scan<T>(c1, &t1);
  if (CL == CL_NEAR_FAR) block_excl_scan<T>(c2, &t2);
  if (threadIdx.x == 0) {
    a.block_sums[blockIdx.x] = t1;
    if (CL == CL_NEAR_FAR) a.block_sums[GR_MAX_SCAN_BLOCKS / 2 + blockIdx.x] = t2;
  }
}

template <int CL>
__global__ void compact_scatter(CompactArgs a) {
  int64_t len = CL == CL_UNVISITED ? a.n : eff_len(a.len_dev, a.len_host);
  int64_t base = (int64_t)blockIdx.x * TILE + (int64_t)threadIdx.x * ITEMS;
  unsigned char cls[ITEMS];
  long long c1 = 0, c2 = 0;
  for (int k = 0; k < ITEMS; ++k) {
    int64_t i = base + k;
    cls[k] = 0;
    if (i < len) cls[k] = (unsigned char)classify<CL, true>(a, i);
    c1 += cls[k] == 1;
    c2 += cls[k] == 2;
  }
  long long t1, t2 = 0;
  long long o1 = block_excl_scan<T>(c1, &t1) + a.block_sums[blockIdx.x];
  long long o2 = 0;
  if (CL == CL_NEAR_FAR)
    o2 = block_excl_scan<T>(c2, &t2) + a.block_sums[GR_MAX_SCAN_BLOCKS / 2 + blockIdx.x];
  for (int k = 0; k < ITEMS; ++k) {
    int64_t i = base + k;
    if (cls[k] == 1) {
      int32_t v = CL == CL_UNVISITED ? (int32_t)i : a.in[i];
      if (o1 < a.cap) a.out[o1] = v;
      if (CL == CL_PULL) {
        a.depth[v] = a.level + 1;
        if (a.pred) a.pred[v] = a.tags[i];
      }
      ++o1;
    } else if (cls[k] == 2) {
      if (o2 < a.far_cap) a.far[o2] = a.in[i];
      ++o2;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    long long tot1 = a.totals[0];
    *a.out_len = (unsigned long long)tot1;
    if (tot1 > a.cap) gr_set_status(a.status, GR_ERR_CAPACITY);
    if (CL == CL_NEAR_FAR) {
      long long tot2 = a.totals[1];
      *a.far_len = (unsigned long long)tot2;
      if (tot2 > a.far_cap) gr_set_status(a.status, GR_ERR_CAPACITY);
    }
  }
}

// Single-pass ordered compaction (decoupled look-back).  A CTA takes the
// next tile in launch order from a counter, classifies its items, publishes
// the tile's counts, then derives its output offsets from its predecessors:
// warp 0 reads their flag words 32 at a time and adds counts until it meets a
// published prefix.  A predecessor holds an earlier tile, so it is already
// running and publishes its counts before it looks back itself; the wait for
// it is still bounded (GR_ERR_TIMEOUT in the status word after `spin` polls).
// Flag word per tile: bits 63..62 state (0 none, 1 counts, 2 prefix), bits
// 61..31 the first output's count, bits 30..0 the second output's.
#define GR_LB_COUNTS 1ull
#define GR_LB_PREFIX 2ull
__device__ __forceinline__ unsigned long long lb_pack(unsigned long long st, long long c1,
                                                      long long c2) {
  return (st << 62) | ((unsigned long long)c1 << 31) | (unsigned long long)c2;
}
__device__ __forceinline__ unsigned long long lb_load(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void lb_store(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

template <int CL>
__global__ void compact_onepass(CompactArgs a, unsigned long long* flags, int* tile_ctr,
                                int64_t tiles, unsigned spin) {
  __shared__ int s_tile;
  __shared__ long long s_ex1, s_ex2;
  if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1);
  __syncthreads();
  const int64_t tile = s_tile;
  const int64_t len = CL == CL_UNVISITED ? a.n : eff_len(a.len_dev, a.len_host);
  const int64_t base = tile * TILE + (int64_t)threadIdx.x * ITEMS;
  unsigned char cls[ITEMS];
  long long c1 = 0, c2 = 0;
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    const int64_t i = base + k;
    cls[k] = i < len ? (unsigned char)classify<CL, true>(a, i) : (unsigned char)0;
    c1 += cls[k] == 1;
    c2 += cls[k] == 2;
  }
  long long t1, t2 = 0;
  long long o1 = block_excl_scan<T>(c1, &t1);
  long long o2 = 0;
  if (CL == CL_NEAR_FAR) o2 = block_excl_scan<T>(c2, &t2);
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    long long ex1 = 0, ex2 = 0;
    if (tile > 0) {
      if (lane == 0) lb_store(flags + tile, lb_pack(GR_LB_COUNTS, t1, t2));
      bool failed = false;
      unsigned polls = 0;
      for (int64_t p = tile - 1;; p -= 32) {
        const int64_t idx = p - lane;
        unsigned long long w = idx >= 0 ? lb_load(flags + idx) : lb_pack(GR_LB_PREFIX, 0, 0);
        while (!__all_sync(GR_FULL_MASK, (w >> 62) != 0ull)) {
          if (++polls > spin) {
            failed = true;
            break;
          }
          __nanosleep(32);
          if ((w >> 62) == 0ull) w = lb_load(flags + idx);
        }
        if (failed) break;
        const unsigned pm = __ballot_sync(GR_FULL_MASK, (w >> 62) == GR_LB_PREFIX);
        const int stop = pm ? __ffs(pm) - 1 : 31;  // the nearest prefix ends the walk
        long long v1 = lane <= stop ? (long long)((w >> 31) & 0x7fffffffull) : 0;
        long long v2 = lane <= stop ? (long long)(w & 0x7fffffffull) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          v1 += __shfl_xor_sync(GR_FULL_MASK, v1, o);
          v2 += __shfl_xor_sync(GR_FULL_MASK, v2, o);
        }
        ex1 += v1;
        ex2 += v2;
        if (pm) break;
      }
      if (failed && lane == 0) gr_set_status(a.status, GR_ERR_TIMEOUT);
    }
    if (lane == 0) {
      lb_store(flags + tile, lb_pack(GR_LB_PREFIX, ex1 + t1, ex2 + t2));
      s_ex1 = ex1;
      s_ex2 = ex2;
    }
  }
  __syncthreads();
  o1 += s_ex1;
  o2 += s_ex2;
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    const int64_t i = base + k;
    if (cls[k] == 1) {
      const int32_t v = CL == CL_UNVISITED ? (int32_t)i : a.in[i];
      if (o1 < a.cap) a.out[o1] = v;
      ++o1;
    } else if (cls[k] == 2) {
      if (o2 < a.far_cap) a.far[o2] = a.in[i];
      ++o2;
    }
  }
  if (tile == tiles - 1 && threadIdx.x == 0) {
    const long long tot1 = s_ex1 + t1;
    *a.out_len = (unsigned long long)tot1;
    if (tot1 > a.cap) gr_set_status(a.status, GR_ERR_CAPACITY);
    if (CL == CL_NEAR_FAR) {
      const long long tot2 = s_ex2 + t2;
      *a.far_len = (unsigned long long)tot2;
      if (tot2 > a.far_cap) gr_set_status(a.status, GR_ERR_CAPACITY);
    }
  }
}

__global__ void unique_mark_first(const int32_t* in, int64_t len_host, const int64_t* len_dev,
                                  int32_t n, int32_t* first_idx) {
  int64_t len = eff_len(len_dev, len_host);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = in[i];
    // the index only ever decreases: skip the reduction when an earlier
    // occurrence already holds a smaller one (a stale cached value only
    // costs an unnecessary reduction)
    if (v >= 0 && v < n && first_idx[v] > (int32_t)i) atomicMin(&first_idx[v], (int32_t)i);
  }
}

// CULL: claim each id once in a bitmap; emit the claimants (order unspecified).
// A CTA takes GR_CULL_ROUND items a round, stages its claimants in shared
// memory (one shared atomic per warp and pass) and reserves their output
// range with one global atomic per round, so the output counter sees tens of
// thousands of atomics instead of one per warp with a claimant.  Claimants
// past the capacity are released at once (their bits cleared), so that the
// claim bitmap is clean again after the call either way.
#define GR_CULL_PER_THREAD 8
#define GR_CULL_ROUND (T * GR_CULL_PER_THREAD)
__global__ void cull_claim(const int32_t* in, int64_t len_host, const int64_t* len_dev, int32_t n,
                           uint32_t* claim, int32_t* out, int64_t cap,
                           unsigned long long* out_len, int* status) {
  __shared__ int32_t s_buf[GR_CULL_ROUND];
  __shared__ int s_cnt;
  __shared__ unsigned long long s_base;
  const int64_t len = eff_len(len_dev, len_host);
  const int lane = threadIdx.x & 31;
  for (int64_t r0 = (int64_t)blockIdx.x * GR_CULL_ROUND; r0 < len;
       r0 += (int64_t)gridDim.x * GR_CULL_ROUND) {
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    int32_t v[GR_CULL_PER_THREAD];
#pragma unroll
    for (int k = 0; k < GR_CULL_PER_THREAD; ++k) {
      const int64_t i = r0 + (int64_t)k * T + threadIdx.x;
      v[k] = i < len ? in[i] : -1;
    }
#pragma unroll
    for (int k = 0; k < GR_CULL_PER_THREAD; ++k) {
      bool take = false;
      if (v[k] >= 0 && v[k] < n) {
        const uint32_t bit = 1u << (v[k] & 31);
        if (!(claim[v[k] >> 5] & bit)) take = !(atomicOr(&claim[v[k] >> 5], bit) & bit);
      }
      const unsigned mask = __ballot_sync(GR_FULL_MASK, take);
      if (mask) {
        int base = 0;
        if (lane == __ffs(mask) - 1) base = atomicAdd(&s_cnt, __popc(mask));
        base = __shfl_sync(GR_FULL_MASK, base, __ffs(mask) - 1);
        if (take) s_buf[base + __popc(mask & ((1u << lane) - 1u))] = v[k];
      }
    }
    __syncthreads();
    const int cnt = s_cnt;
    if (threadIdx.x == 0) {
      s_base = cnt ? atomicAdd(out_len, (unsigned long long)cnt) : 0ull;
      if (cnt && s_base + cnt > (unsigned long long)cap) gr_set_status(status, GR_ERR_CAPACITY);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < cnt; j += T) {
      const unsigned long long pos = s_base + j;
      const int32_t x = s_buf[j];
      if (pos < (unsigned long long)cap) out[pos] = x;
      else atomicAnd(&claim[x >> 5], ~(1u << (x & 31)));
    }
    __syncthreads();  // the next round reuses the stage
  }
}

__global__ void cull_release(const int32_t* out, const unsigned long long* out_len, int64_t cap,
                             uint32_t* claim) {
  long long len = (long long)*out_len;
  if (len > cap) len = cap;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (long long)gridDim.x * blockDim.x) {
    int32_t v = out[i];
    atomicAnd(&claim[v >> 5], ~(1u << (v & 31)));
  }
}

int64_t tiles_for(int64_t len) { return (len + TILE - 1) / TILE; }

// look-back polls before a tile gives up on a predecessor (each poll sleeps
// about 32 ns, so about a second)
constexpr unsigned kLookbackPolls = 1u << 25;

template <int CL>
gr_status launch_onepass(const CompactArgs& a, gr_workspace* ws, int64_t tiles, cudaStream_t s) {
  unsigned long long* flags = (unsigned long long*)ws->block_sums;
  int* ctr = (int*)(ws->dev_len + 6);
  if (cudaMemsetAsync(flags, 0, (size_t)tiles * sizeof(unsigned long long), s) != cudaSuccess ||
      cudaMemsetAsync(ctr, 0, sizeof(int), s) != cudaSuccess)
    return GR_ERR_CUDA;
  compact_onepass<CL><<<(unsigned)tiles, T, 0, s>>>(a, flags, ctr, tiles, kLookbackPolls);
  return cudaGetLastError() == cudaSuccess ? GR_OK : GR_ERR_CUDA;
}

}  // namespace

#define GR_LAUNCH_CHECK()                                      \
  do {                                                         \
    if (cudaGetLastError() != cudaSuccess) return GR_ERR_CUDA; \
  } while (0)

extern "C" gr_status gr_advance(const gr_graph* g, const int32_t* in, int64_t in_len,
                                const int64_t* in_len_dev, int32_t mode, int32_t functor,
                                const void* state, int32_t* out, int64_t out_cap,
                                int64_t* out_len, void* stream) {
  if (!g || in_len < 0 || (in_len > 0 && !in) || out_cap < 0 || !out_len ||
      (out_cap > 0 && !out) || (mode & ~(GR_V2E | GR_PULL | GR_UNORDERED | GR_IDEMPOTENT)) ||
      functor < GR_FN_NONE || functor > GR_FN_SSSP_RELAX)
    return GR_ERR_INVALID_ARG;
  if (in_len >= INT32_MAX) return GR_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  gr_workspace* ws = g->ws_default;
  unsigned long long* olen = (unsigned long long*)out_len;
  int blocks_persist = g->num_sms * 8;

  if (mode & GR_PULL) {
    if (functor != GR_FN_BFS_VISIT || !state || (mode & GR_V2E)) return GR_ERR_INVALID_ARG;
    if (!(g->flags & GR_SYMMETRIC)) return GR_ERR_UNSUPPORTED;
    if (in_len > g->n) return GR_ERR_INVALID_ARG;
    const gr_bfs_state* st = (const gr_bfs_state*)state;
    if (!st->depth) return GR_ERR_INVALID_ARG;
    if (in_len == 0) {
      if (cudaMemsetAsync(out_len, 0, sizeof(int64_t), s) != cudaSuccess) return GR_ERR_CUDA;
      return GR_OK;
    }
    CompactArgs a = {};
    a.n = g->n; a.R = g->R; a.C = g->C; a.in = in; a.len_host = in_len; a.len_dev = in_len_dev;
    a.block_sums = ws->block_sums; a.totals = ws->dev_len; a.out = out; a.cap = out_cap;
    a.out_len = olen; a.status = ws->status; a.depth = st->depth; a.pred = st->pred;
    a.level = st->level; a.tags = ws->tags;
    int64_t tiles = tiles_for(in_len);
    compact_count<CL_PULL><<<(unsigned)tiles, T, 0, s>>>(a);
    scan_block_sums<<<1, 1024, 0, s>>>(ws->block_sums, tiles, 0, ws->dev_len);
    compact_scatter<CL_PULL><<<(unsigned)tiles, T, 0, s>>>(a);
    GR_LAUNCH_CHECK();
    return GR_OK;
  }

  int fn;
  if (functor == GR_FN_NONE) fn = (mode & GR_V2E) ? FN_NONE_EDGES : FN_NONE_ORDERED;
  else if (functor == GR_FN_BFS_VISIT) fn = (mode & GR_IDEMPOTENT) ? FN_BFS_IDEM : FN_BFS;
  else fn = FN_RELAX;
  if (fn >= FN_BFS && ((mode & GR_V2E) || !state)) return GR_ERR_INVALID_ARG;
  if (fn == FN_RELAX && !g->W && g->m > 0) return GR_ERR_UNSUPPORTED;
  if ((fn == FN_BFS || fn == FN_BFS_IDEM) && !((const gr_bfs_state*)state)->depth)
    return GR_ERR_INVALID_ARG;
  if (fn == FN_RELAX && !((const gr_sssp_state*)state)->key) return GR_ERR_INVALID_ARG;

  if (in_len == 0) {
    if (cudaMemsetAsync(out_len, 0, sizeof(int64_t), s) != cudaSuccess) return GR_ERR_CUDA;
    return GR_OK;
  }
  // per-item output offsets: the workspace holds n + 1 of them; longer
  // inputs (frontiers with repeated vertices) use a stream-ordered temporary.
  long long* item_off = ws->item_off;
  bool tmp_alloc = in_len > (int64_t)g->n + 1;
  if (tmp_alloc &&
      cudaMallocAsync((void**)&item_off, (size_t)in_len * sizeof(long long), s) != cudaSuccess) {
    (void)cudaGetLastError();
    return GR_ERR_OOM;
  }
  int64_t tiles = tiles_for(in_len);
  adv_degree_tiles<<<(unsigned)tiles, T, 0, s>>>(g->R, in, in_len, in_len_dev, g->n, item_off,
                                                 ws->block_sums, ws->status);
  scan_block_sums<<<1, 1024, 0, s>>>(ws->block_sums, tiles, 0, ws->dev_len);
  ExpandArgs a = {};
  a.n = g->n;
  a.R = g->R; a.C = g->C; a.W = g->W; a.in = in; a.len_host = in_len; a.len_dev = in_len_dev;
  a.item_off = item_off; a.block_sums = ws->block_sums; a.total = ws->dev_len; a.out = out;
  a.cap = out_cap; a.out_len = olen; a.status = ws->status;
  // the tile map lives in the pull scratch (n + 1 entries: every tile of an
  // expansion of up to (n + 1) * GR_ADV_TILE outputs)
  a.tile_item = ws->tags;
  a.tile_cap = (int64_t)g->n + 1;
  {
    const int64_t mb = (in_len + T - 1) / T;
    adv_tile_map<<<(unsigned)(mb < 4096 ? mb : 4096), T, 0, s>>>(
        item_off, ws->block_sums, in_len, in_len_dev, ws->dev_len, ws->tags, a.tile_cap);
  }
  if (fn == FN_BFS || fn == FN_BFS_IDEM) {
    const gr_bfs_state* st = (const gr_bfs_state*)state;
    a.depth = st->depth; a.pred = st->pred; a.level = st->level;
  } else if (fn == FN_RELAX) {
    a.key = (unsigned long long*)((const gr_sssp_state*)state)->key;
  }
  if (fn == FN_NONE_ORDERED || fn == FN_NONE_EDGES) {
    write_len_and_check<<<1, 1, 0, s>>>(ws->dev_len, olen, out_cap, ws->status);
  } else if (cudaMemsetAsync(out_len, 0, sizeof(int64_t), s) != cudaSuccess) {
    return GR_ERR_CUDA;
  }
  switch (fn) {
    case FN_NONE_ORDERED: adv_expand<FN_NONE_ORDERED><<<blocks_persist, T, 0, s>>>(a); break;
    case FN_NONE_EDGES: adv_expand<FN_NONE_EDGES><<<blocks_persist, T, 0, s>>>(a); break;
    case FN_BFS: adv_expand<FN_BFS><<<blocks_persist, T, 0, s>>>(a); break;
    case FN_BFS_IDEM: adv_expand<FN_BFS_IDEM><<<blocks_persist, T, 0, s>>>(a); break;
    default: adv_expand<FN_RELAX><<<blocks_persist, T, 0, s>>>(a); break;
  }
  // the temporary offsets are released on every path once the launches are queued
  const bool launched = cudaGetLastError() == cudaSuccess;
  if (tmp_alloc && cudaFreeAsync(item_off, s) != cudaSuccess) return GR_ERR_CUDA;
  return launched ? GR_OK : GR_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// multisplit: a stable K-way partition by distance bucket (the near/far split
// of Sec. 5.1.5 with more than two buckets)

struct MsplitArgs {
  int32_t n;
  const int32_t* in;
  int64_t len_host;
  const int64_t* len_dev;
  const unsigned long long* key;
  uint32_t base, delta;
  int K;
  long long* counts;  // K x tiles, bucket-major (scanned in place between the passes)
  int64_t tiles;
  signed char* bucket;  // tiles * TILE bytes: each item's bucket, -1 for none
  int32_t* out;
  int64_t cap;
  int* status;
};

// Bucket of item v: -1 when v is not in [0, n), else min(K - 1, (d - base) / delta)
// for d = dist(v) >= base, and 0 below base.
__device__ __forceinline__ int msplit_bucket(const MsplitArgs& a, int32_t v) {
  if (v < 0 || v >= a.n) return -1;
  const unsigned d = (unsigned)(a.key[v] >> 32);
  const unsigned long long b = d < a.base ? 0ull : (unsigned long long)(d - a.base) / a.delta;
  return b >= (unsigned long long)(a.K - 1) ? a.K - 1 : (int)b;
}

// Per-thread bucket counts of ITEMS consecutive items, summed per warp
// (shuffles) and per CTA (one shared atomic per warp and bucket).  The bucket
// of every item is kept as a byte (ITEMS = 16 bytes a thread, one vector
// store), so that the scatter pass reads bytes in order instead of gathering
// the distances a second time.
__global__ void msplit_count(MsplitArgs a) {
  static_assert(ITEMS == 16, "one 16-byte vector of bucket bytes per thread");
  __shared__ int s_cnt[GR_RING_K];
  if (threadIdx.x < GR_RING_K) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t len = eff_len(a.len_dev, a.len_host);
  const int64_t base = (int64_t)blockIdx.x * TILE + (int64_t)threadIdx.x * ITEMS;
  int c[GR_RING_K];
#pragma unroll
  for (int j = 0; j < GR_RING_K; ++j) c[j] = 0;
  union {
    signed char b[ITEMS];
    uint4 v;
  } bk;
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    bk.b[k] = base + k < len ? (signed char)msplit_bucket(a, a.in[base + k]) : (signed char)-1;
#pragma unroll
    for (int j = 0; j < GR_RING_K; ++j) c[j] += bk.b[k] == j;
  }
  if (base < len) reinterpret_cast<uint4*>(a.bucket)[base / ITEMS] = bk.v;
#pragma unroll
  for (int j = 0; j < GR_RING_K; ++j) {
    int x = c[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(GR_FULL_MASK, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(&s_cnt[j], x);
  }
  __syncthreads();
  if (threadIdx.x < a.K) a.counts[(int64_t)threadIdx.x * a.tiles + blockIdx.x] = s_cnt[threadIdx.x];
}

// Each thread owns ITEMS consecutive items of the tile.  An item's place is
// its bucket's start in this tile (the scanned counts) + the counts of that
// bucket in the earlier warps of the CTA + in the earlier lanes of its warp
// (warp scans of the per-thread counts) + the earlier items of the thread.
__global__ void msplit_scatter(MsplitArgs a) {
  constexpr int NW = T / 32;
  __shared__ int s_wt[NW][GR_RING_K];  // per-warp bucket totals, then their exclusive scan
  const int64_t len = eff_len(a.len_dev, a.len_host);
  const int64_t base = (int64_t)blockIdx.x * TILE + (int64_t)threadIdx.x * ITEMS;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  union {
    signed char b[ITEMS];
    uint4 v;
  } bk;
  bk.v = base < len ? reinterpret_cast<const uint4*>(a.bucket)[base / ITEMS]
                    : make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);
  int pos[GR_RING_K];
#pragma unroll
  for (int j = 0; j < GR_RING_K; ++j) {
    int c = 0;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) c += bk.b[k] == j;
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(GR_FULL_MASK, incl, o);
      if (lane >= o) incl += y;
    }
    pos[j] = incl - c;
    if (lane == 31) s_wt[w][j] = incl;
  }
  __syncthreads();
  if (threadIdx.x < GR_RING_K) {
    int run = 0;
#pragma unroll
    for (int x = 0; x < NW; ++x) {
      const int t = s_wt[x][threadIdx.x];
      s_wt[x][threadIdx.x] = run;
      run += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < GR_RING_K; ++j)
    if (j < a.K) pos[j] += (int)a.counts[(int64_t)j * a.tiles + blockIdx.x] + s_wt[w][j];
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    const int b = bk.b[k];
    if (b < 0) continue;
    int at = 0;
#pragma unroll
    for (int j = 0; j < GR_RING_K; ++j)
      if (j == b) at = pos[j]++;
    if (at < a.cap) a.out[at] = a.in[base + k];
    else gr_set_status(a.status, GR_ERR_CAPACITY);
  }
}

// bucket_len[j] from the scanned counts; the total goes to out_len.
__global__ void msplit_lens(const long long* counts, int64_t tiles, int K, const long long* total,
                            int64_t* bucket_len, unsigned long long* out_len, int64_t cap,
                            int* status) {
  const int j = threadIdx.x;
  if (j < K) {
    const long long next = j + 1 < K ? counts[(int64_t)(j + 1) * tiles] : *total;
    bucket_len[j] = next - counts[(int64_t)j * tiles];
  }
  if (j == 0) {
    *out_len = (unsigned long long)*total;
    if (*total > cap) gr_set_status(status, GR_ERR_CAPACITY);
  }
}

extern "C" gr_status gr_filter(const gr_graph* g, const int32_t* in, int64_t in_len,
                               const int64_t* in_len_dev, int32_t mode, const void* state,
                               int32_t* out, int64_t out_cap, int64_t* out_len, int32_t* far,
                               int64_t far_cap, int64_t* far_len, void* stream) {
  if (!g || in_len < 0 || in_len >= INT32_MAX || out_cap < 0 || !out_len ||
      (out_cap > 0 && !out) || mode < GR_FILTER_EXACT_UNIQUE || mode > GR_FILTER_MULTISPLIT)
    return GR_ERR_INVALID_ARG;
  if (mode != GR_FILTER_UNVISITED && in_len > 0 && !in) return GR_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  gr_workspace* ws = g->ws_default;
  unsigned long long* olen = (unsigned long long*)out_len;
  CompactArgs a = {};
  a.n = g->n; a.R = g->R; a.C = g->C; a.in = in; a.len_host = in_len; a.len_dev = in_len_dev;
  a.block_sums = ws->block_sums; a.totals = ws->dev_len; a.out = out; a.cap = out_cap;
  a.out_len = olen; a.status = ws->status; a.first_idx = ws->first_idx;

  if (mode == GR_FILTER_UNVISITED) {
    const gr_bfs_state* st = (const gr_bfs_state*)state;
    if (!st || !st->depth) return GR_ERR_INVALID_ARG;
    a.depth = st->depth;
    if (g->n == 0) return cudaMemsetAsync(out_len, 0, 8, s) == cudaSuccess ? GR_OK : GR_ERR_CUDA;
    return launch_onepass<CL_UNVISITED>(a, ws, tiles_for(g->n), s);
  }
  if (mode == GR_FILTER_NEAR_FAR) {
    const gr_sssp_state* st = (const gr_sssp_state*)state;
    if (!st || !st->key || !far_len || (far_cap > 0 && !far) || far_cap < 0)
      return GR_ERR_INVALID_ARG;
    if (in_len == 0) {
      if (cudaMemsetAsync(out_len, 0, 8, s) || cudaMemsetAsync(far_len, 0, 8, s))
        return GR_ERR_CUDA;
      return GR_OK;
    }
    a.key = (const unsigned long long*)st->key;
    a.threshold = st->threshold;
    a.far = far; a.far_cap = far_cap; a.far_len = (unsigned long long*)far_len;
    return launch_onepass<CL_NEAR_FAR>(a, ws, tiles_for(in_len), s);
  }
  if (mode == GR_FILTER_MULTISPLIT) {
    const gr_multisplit_state* st = (const gr_multisplit_state*)state;
    if (!st || !st->key || !st->bucket_len || st->buckets < 2 || st->buckets > GR_RING_K ||
        st->delta == 0)
      return GR_ERR_INVALID_ARG;
    if (in_len == 0) {
      if (cudaMemsetAsync(out_len, 0, 8, s) ||
          cudaMemsetAsync(st->bucket_len, 0, (size_t)st->buckets * 8, s))
        return GR_ERR_CUDA;
      return GR_OK;
    }
    MsplitArgs m = {};
    m.n = g->n; m.in = in; m.len_host = in_len; m.len_dev = in_len_dev;
    m.key = (const unsigned long long*)st->key; m.base = st->base; m.delta = st->delta;
    m.K = st->buckets; m.tiles = tiles_for(in_len); m.out = out; m.cap = out_cap;
    m.status = ws->status;
    // one temporary: the items' bucket bytes (a whole number of tiles), then
    // the K x tiles counts
    const size_t bbytes = (size_t)m.tiles * TILE;
    const size_t cbytes = (size_t)m.K * (size_t)m.tiles * sizeof(long long);
    unsigned char* tmp = nullptr;
    if (cudaMallocAsync((void**)&tmp, bbytes + cbytes, s) != cudaSuccess) {
      (void)cudaGetLastError();
      return GR_ERR_OOM;
    }
    m.bucket = (signed char*)tmp;
    m.counts = (long long*)(tmp + bbytes);
    msplit_count<<<(unsigned)m.tiles, T, 0, s>>>(m);
    scan_block_sums<<<1, 1024, 0, s>>>(m.counts, (int64_t)m.K * m.tiles, 0, ws->dev_len);
    msplit_scatter<<<(unsigned)m.tiles, T, 0, s>>>(m);
    msplit_lens<<<1, 32, 0, s>>>(m.counts, m.tiles, m.K, ws->dev_len, st->bucket_len, olen,
                                 out_cap, ws->status);
    const bool launched = cudaGetLastError() == cudaSuccess;
    if (cudaFreeAsync(tmp, s) != cudaSuccess || !launched) {
      (void)cudaGetLastError();
      return GR_ERR_CUDA;
    }
    return GR_OK;
  }
  if (in_len == 0)
    return cudaMemsetAsync(out_len, 0, 8, s) == cudaSuccess ? GR_OK : GR_ERR_CUDA;
  if (mode == GR_FILTER_EXACT_UNIQUE) {
    unique_mark_first<<<g->num_sms * 8, T, 0, s>>>(in, in_len, in_len_dev, g->n, ws->first_idx);
    GR_LAUNCH_CHECK();
    return launch_onepass<CL_UNIQUE>(a, ws, tiles_for(in_len), s);
  }
  // GR_FILTER_CULL
  if (cudaMemsetAsync(out_len, 0, 8, s) != cudaSuccess) return GR_ERR_CUDA;
  cull_claim<<<g->num_sms * 8, T, 0, s>>>(in, in_len, in_len_dev, g->n, ws->claim, out, out_cap,
                                          olen, ws->status);
  cull_release<<<g->num_sms * 8, T, 0, s>>>(out, olen, out_cap, ws->claim);
  GR_LAUNCH_CHECK();
  return GR_OK;
}
