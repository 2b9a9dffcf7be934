// gr_internal.cuh — internal structures and device primitives of the library.
//
// Everything here is private to the CUDA library; the public boundary is
// include/gr.h.  Device-side waits are bounded: a wait that runs out of polls
// records GR_ERR_TIMEOUT in the workspace status word and returns, so no
// kernel of this library can hang the GPU.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gr.h"

#define GR_FULL_MASK 0xffffffffu

// Build-time switches (defaults are the measured best on GB300):
// GR_CLAIM_AGGREGATE  1: warp-aggregated bitmap claims (one atomic per word)
//                     0: one atomicOr per lane (measured 3x faster on R-MAT
//                        push levels and on grids: match/reduce cost more
//                        than the atomics they save)
// GR_STREAM_COLUMNS   1: column/weight streams loaded with evict-first hints
//                        (measured 13% faster SSSP: the streams no longer
//                        evict the L2-resident keys)
//                     0: plain read-only loads
#ifndef GR_CLAIM_AGGREGATE
#define GR_CLAIM_AGGREGATE 0
#endif
#ifndef GR_STREAM_COLUMNS
#define GR_STREAM_COLUMNS 1
#endif
#if GR_STREAM_COLUMNS
#define GR_LDSTREAM(p) __ldcs(p)
#else
#define GR_LDSTREAM(p) __ldg(p)
#endif

// Library defaults (tunable per call through gr_bfs_opts / gr_sssp_opts).
// Rows of at least the split threshold are expanded as edge chunks.  A warp
// batch of medium rows then holds at most GR_MEDIUM_BATCH * threshold edges,
// which should stay within about 16 rounds of the body's strips: BFS
// expands 4 strips (128 edges) per round, SSSP bulk steps 8 (256 edges).
#define GR_DEFAULT_BFS_BIG 256
#define GR_DEFAULT_SSSP_BIG 1024
#define GR_DEFAULT_BIG_DEGREE GR_DEFAULT_SSSP_BIG
#ifndef GR_CHUNK_EDGES
#define GR_CHUNK_EDGES 256           // edges per chunk of a split row
#endif
#define GR_DEFAULT_SPIN_LIMIT (1u << 24)
#define GR_TIME_LIMIT_NS (60ull * 1000000000ull)  // persistent kernels give up after 60 s
#define GR_PERSIST_THREADS 512
#define GR_OPS_THREADS 256
#define GR_SCAN_ITEMS 16             // items per thread in the operator scans
#define GR_SCAN_TILE (GR_OPS_THREADS * GR_SCAN_ITEMS)
#define GR_MAX_SCAN_BLOCKS ((int64_t)1 << 19)  // covers in_len < 2^31

// Buckets of the SSSP multi-level priority queue: the current one and the
// GR_RING_K - 1 after it have lists of their own (a ring), farther ones share
// the far pile.
#ifndef GR_RING_K
#define GR_RING_K 8
#endif

// Device control block of a workspace.  The barrier and the per-level
// counters are cleared by the host (cudaMemsetAsync) before every persistent
// launch; the status word lives separately and persists until read.
struct GrCtl {
  unsigned bar_count;              // grid barrier: arrivals since launch (monotonic)
  unsigned bar_pad;
  int abort;
  int levels;                      // BFS levels / SSSP steps executed
  int qlen[3];                     // frontier queue length, slot = step % 3
  int nchunk[3];                   // edge chunks of split rows, slot = step % 3
  int nbig[3];                     // number of split rows, slot = step % 3
  int farlen[3];                   // SSSP far pile length, slot = epoch % 3
  int work[3];                     // dynamic work counter (queue batches / pull words)
  int workc[3];                    // dynamic work counter (edge chunks)
  int ulen[3];                     // BFS unvisited-list length, slot = level % 3
  int workb[3];                    // dynamic work counter (bitmap words: SSSP collect, BFS rebuild)
  int qbuilt[3];                   // BFS: queue rows rebuilt from a pull level's bitmap
  int qmlen[3];                    // medium-row queue length, slot = step % 3
  int workm[3];                    // dynamic work counter (medium-row batches)
  int ndef[3];                     // BFS pull: rows deferred to the whole grid, slot = level % 3
  unsigned farmin[3];              // SSSP smallest distance pushed to a far pile
  int rlen[GR_RING_K];             // SSSP multi-level queue: entries of each ring slot
  int ovf_pending;                 // SSSP: some relaxation sum did not fit in 32 bits
  unsigned long long mf[3];        // sum of degrees of the next frontier
  unsigned long long edges;        // column entries read (statistics)
  unsigned long long verts;        // rows opened: frontier rows, chunks, pull candidates
  unsigned long long updates;      // BFS discoveries / SSSP successful relaxations
};

// Per-thread work counters of a persistent kernel, flushed once at exit:
// warp sums, then a shared-memory sum per CTA, then one global atomic per
// CTA and counter.  Every thread of the CTA must call flush().
struct GrCounters {
  unsigned long long edges = 0, verts = 0, updates = 0;
  __device__ __forceinline__ void flush(GrCtl* ctl) {
    __shared__ unsigned long long s_sum[3];
    unsigned long long e = edges, v = verts, u = updates;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e += __shfl_xor_sync(0xffffffffu, e, o);
      v += __shfl_xor_sync(0xffffffffu, v, o);
      u += __shfl_xor_sync(0xffffffffu, u, o);
    }
    if (threadIdx.x < 3) s_sum[threadIdx.x] = 0ull;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
      if (e) atomicAdd(&s_sum[0], e);
      if (v) atomicAdd(&s_sum[1], v);
      if (u) atomicAdd(&s_sum[2], u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (s_sum[0]) atomicAdd(&ctl->edges, s_sum[0]);
      if (s_sum[1]) atomicAdd(&ctl->verts, s_sum[1]);
      if (s_sum[2]) atomicAdd(&ctl->updates, s_sum[2]);
    }
  }
};

struct GrMsState;                  // multi-source BFS scratch (gr_msbfs.cu)
void gr_ms_free(GrMsState* ms);
struct GrBcScratch;                // betweenness-centrality scratch of a workspace (gr_bc.cu)
void gr_bc_free(GrBcScratch* b);
struct GrCcScratch;                // connected-components scratch of a workspace (gr_cc.cu)
void gr_cc_free(GrCcScratch* c);
struct GrTcScratch;                // intersection / triangle scratch of a workspace (gr_tc.cu)
void gr_tc_free(GrTcScratch* t);

struct gr_graph {
  int32_t n;
  int64_t m;
  uint32_t flags;
  const int32_t* R;
  const int32_t* C;
  const uint32_t* W;
  void* owned[3];
  int32_t max_degree;
  int32_t nonisolated;
  unsigned long long weight_sum;
  int device;
  int num_sms;
  gr_workspace* ws_default;
  GrMsState* ms;                   // allocated by the first gr_bfs_multi call
  uint32_t* zero_deg;              // symmetric graphs with isolated vertices: n-bit bitmap of
                                   // the vertices without edges (no BFS can reach them)
};

struct gr_workspace {
  const gr_graph* g;
  int32_t ops;
  GrCtl* ctl;
  int* status;
  int* h_status;        // pinned host mirror used by gr_sync_status
  int32_t* q[2];        // frontier queues (ping-pong), n entries each
  int32_t* qm[2];       // medium-row frontier queues (ping-pong), n entries each
  int32_t* ulist[2];    // BFS unvisited lists (ping-pong), n entries each
  int2* chunks[2];      // (row, first edge) chunks of split rows (ping-pong)
  int64_t chunk_cap;
  uint32_t* visited;    // n bits
  uint32_t* front[3];   // frontier bitmaps, n bits each (rotating)
  uint64_t* key;        // SSSP packed (dist << 32 | pred)
  int32_t* far[2];      // SSSP far piles (ping-pong), n entries each
  int32_t* stamp_near;  // SSSP near-queue membership stamps
  int32_t* stamp_far;   // SSSP far-pile membership stamps
  int32_t* ring[GR_RING_K];  // SSSP multi-level queue: bucket lists, n entries each
  uint32_t* stamp_ring; // SSSP: last bucket each vertex was added to
  int32_t* first_idx;   // filter scratch: n entries, INT32_MAX when clean
  uint32_t* claim;      // filter scratch: n bits, 0 when clean
  long long* block_sums;// operator scan scratch, GR_MAX_SCAN_BLOCKS + 2 entries
  int32_t* tags;        // pull scratch: n entries
  int32_t* pdef;        // BFS pull: deferred long rows, GR_PULL_DEFER_INTS entries
  long long* item_off;  // advance scratch: n + 1 per-item output offsets
  long long* dev_len;   // operator scratch: a few device counters
  GrBcScratch* bc;      // allocated by the first gr_bc call on this workspace
  GrCcScratch* cc;      // allocated by the first gr_cc call on this workspace
  GrTcScratch* tc;      // allocated by the first intersection / triangle call
  bool stream_ordered;  // buffers from cudaMallocAsync, released with cudaFreeAsync
};

// ---------------------------------------------------------------------------
// small device helpers

__device__ __forceinline__ void gr_set_status(int* status, int code) {
  atomicCAS(status, 0, code);
}

__device__ __forceinline__ unsigned gr_ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void gr_st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned gr_atom_add_acq_rel(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;"
               : "=r"(old)
               : "l"(p), "r"(v)
               : "memory");
  return old;
}

// Reductions without a return value (PTX red): the issuing warp never
// waits for them, unlike an atomic whose result register is tracked.
#ifndef GR_USE_RED
#define GR_USE_RED 1  // 0: plain atomics instead (measured 7 % slower SSSP on R-MAT s22)
#endif
__device__ __forceinline__ void gr_red_min_u64(unsigned long long* p, unsigned long long v) {
#if GR_USE_RED
  asm volatile("red.relaxed.gpu.global.min.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
#else
  atomicMin(p, v);
#endif
}
__device__ __forceinline__ void gr_red_or_u64(unsigned long long* p, unsigned long long v) {
#if GR_USE_RED
  asm volatile("red.relaxed.gpu.global.or.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
#else
  atomicOr(p, v);
#endif
}
__device__ __forceinline__ void gr_red_or_u32(uint32_t* p, uint32_t v) {
#if GR_USE_RED
  asm volatile("red.relaxed.gpu.global.or.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
#else
  atomicOr(p, v);
#endif
}

__device__ __forceinline__ int gr_ld_volatile(const int* p) {
  return *(const volatile int*)p;
}

__device__ __forceinline__ unsigned long long gr_globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Called by one thread per step of a persistent kernel: past the deadline it
// records GR_ERR_TIMEOUT and raises the abort flag, which makes every CTA
// leave at its next grid barrier.  Keeps a runaway loop from holding the GPU.
__device__ __forceinline__ void gr_check_deadline(GrCtl* ctl, int* status,
                                                  unsigned long long deadline) {
  if (gr_globaltimer() > deadline) {
    gr_set_status(status, GR_ERR_TIMEOUT);
    atomicExch(&ctl->abort, 1);
  }
}

// Grid-wide barrier for a cooperative (co-resident) launch.  Arrival is a
// fire-and-forget release increment of one monotonic counter (cleared by the
// host before every launch); block b's k-th barrier completes when the
// counter reaches k * gridDim.x.  Waits are bounded by spin_limit polls; on
// timeout (or when another block aborted) the function records
// GR_ERR_TIMEOUT, raises the abort flag and returns false, and every caller
// must then leave the kernel.  `phase` is the calling block's barrier count.
__device__ __forceinline__ bool gr_grid_sync(GrCtl* ctl, int* status, unsigned spin_limit,
                                             unsigned& phase) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    if (gr_ld_volatile(&ctl->abort)) {
      ok = 0;
    } else {
      phase += 1u;
      const unsigned target = phase * gridDim.x;
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&ctl->bar_count) : "memory");
      unsigned polls = 0;
      while ((int)(gr_ld_acquire(&ctl->bar_count) - target) < 0) {
        if (++polls > spin_limit || gr_ld_volatile(&ctl->abort)) {
          ok = 0;
          break;
        }
        __nanosleep(20);
      }
      __threadfence();
    }
    if (!ok) {
      gr_set_status(status, GR_ERR_TIMEOUT);
      atomicExch(&ctl->abort, 1);
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Warp-uniform dynamic work grab: lane 0 takes `amount` items from *counter
// and the start index is broadcast to the warp.
__device__ __forceinline__ int gr_warp_grab(int* counter, int amount, int lane) {
  int b = 0;
  if (lane == 0) b = atomicAdd(counter, amount);
  return __shfl_sync(GR_FULL_MASK, b, 0);
}

// Next batch start of the "static first, dynamic after" work loops: the
// first round covers [0, static_span) by warp index; when that already
// covered `total` items the loop ends without touching the counter.
__device__ __forceinline__ int gr_next_batch(int cur, int total, int static_span, int* counter,
                                             int amount, int lane) {
  (void)cur;
  if (total <= static_span) return total;
  return static_span + gr_warp_grab(counter, amount, lane);
}

#ifndef GR_PULL_WORDS
#define GR_PULL_WORDS 4  // bitmap words (32 candidates each) per pull batch and warp
#endif
// Rows are expanded in three classes (the paper's TWC classes, Sec. 5.1.2):
// rows shorter than GR_MEDIUM_DEGREE in batches of 32 per warp, medium rows
// in batches of GR_MEDIUM_BATCH per warp, rows of at least the split
// threshold as GR_CHUNK_EDGES-edge chunks shared by the grid.  A batch then
// holds at most 32 * 31 or GR_MEDIUM_BATCH * (split threshold) edges.
#define GR_MEDIUM_DEGREE 32
#define GR_MEDIUM_BATCH 4
#ifndef GR_PULL_SERIAL
#define GR_PULL_SERIAL 64  // neighbours a pull candidate scans alone before the warp helps
#endif
// A pull candidate whose row shows no frontier neighbour in its first
// GR_PULL_SERIAL + GR_PULL_WARP_EDGES entries, with at least GR_PULL_DEFER_MIN
// more to go, is handed to the whole grid: the rest of its row is cut into
// GR_PULL_CHUNK-edge chunks that all warps share at the top of the next level
// (at most GR_PULL_DEFER_CAP such rows per level; beyond that the warp scans
// on alone).  Each entry of the deferred list is 8 int32: vertex, first edge,
// end edge, chunks done, unused, degree, unused, unused.
#ifndef GR_PULL_WARP_EDGES
#define GR_PULL_WARP_EDGES 1024
#endif
#ifndef GR_PULL_DEFER_MIN
#define GR_PULL_DEFER_MIN 1024
#endif
#define GR_PULL_CHUNK 256
#define GR_PULL_DEFERRED (-2)  // find_parent: the row went to the deferred list
#define GR_PULL_DEFER_CAP 1024
#define GR_PULL_DEFER_INTS (8 * GR_PULL_DEFER_CAP)
#define GR_DIRECT_CLAIM_FRONTIER 32768  // below this frontier size (and twice as many
                                        // frontier edges) BFS claims without a pre-read

// Thread scopes for the query bodies (gr_bfs_body / gr_sssp_body).
// GridScope: every thread of a cooperative (co-resident) launch; the step
// barrier is the bounded grid barrier above.
struct GridScope {
  GrCtl* ctl;
  int* status;
  unsigned spin;
  int64_t tid, nthreads;
  unsigned phase;
  __device__ __forceinline__ bool sync() { return gr_grid_sync(ctl, status, spin, phase); }
};

// ClusterScope: the threads of one thread-block cluster (possibly a single
// CTA).  The step barrier is the hardware cluster barrier with release /
// acquire semantics; all CTAs of a cluster are co-scheduled, so it cannot
// wait for a CTA that never runs.  A raised abort flag ends the job.
struct ClusterScope {
  GrCtl* ctl;
  int64_t tid, nthreads;
  __device__ __forceinline__ bool sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;"
                 ::: "memory");
    return __ldcg(&ctl->abort) == 0;
  }
};

// Exclusive warp scan of an int; *total gets the warp sum.
__device__ __forceinline__ int gr_warp_excl_scan(int x, int lane, int* total) {
  int incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(GR_FULL_MASK, incl, o);
    if (lane >= o) incl += y;
  }
  *total = __shfl_sync(GR_FULL_MASK, incl, 31);
  return incl - x;
}

__device__ __forceinline__ unsigned long long gr_warp_sum_u64(unsigned long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(GR_FULL_MASK, x, o);
  return x;
}

// Warp-aggregated append of v to q (one atomic per warp).  Must be called by
// all 32 lanes.  Writes only below cap; *len still counts every item and
// capacity overflow is the caller's to detect (len > cap).
__device__ __forceinline__ void gr_warp_append(int32_t* q, int* len, int64_t cap, bool take,
                                               int32_t v, int lane) {
  unsigned mask = __ballot_sync(GR_FULL_MASK, take);
  if (mask == 0) return;
  int leader = __ffs(mask) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(len, __popc(mask));
  base = __shfl_sync(GR_FULL_MASK, base, leader);
  if (take) {
    int pos = base + __popc(mask & ((1u << lane) - 1u));
    if (pos < cap) q[pos] = v;
  }
}

// Warp-aggregated claim of vertex v in a bitmap.  Lanes whose vertices share
// a 32-bit word (common: a hub's neighbours have dense, nearby ids) issue ONE
// atomicOr with their combined bits instead of up to 32 atomics to one
// address; among lanes claiming the same vertex only the lowest may win.
// Returns true for the lane that newly set its bit.  All 32 lanes call.
__device__ __forceinline__ bool gr_warp_claim(uint32_t* bm, bool active, int32_t v, int lane) {
#if !GR_CLAIM_AGGREGATE
  if (!active) return false;
  const uint32_t b1 = 1u << (v & 31);
  return !(atomicOr(bm + (v >> 5), b1) & b1);
#endif
  const unsigned wkey = active ? (unsigned)v >> 5 : (0x80000000u | (unsigned)lane);
  const unsigned vkey = active ? (unsigned)v : (0x80000000u | (unsigned)lane);
  const unsigned peers = __match_any_sync(GR_FULL_MASK, wkey);
  const unsigned same = __match_any_sync(GR_FULL_MASK, vkey);
  const uint32_t bit = active ? 1u << (v & 31) : 0u;
  const uint32_t bits = __reduce_or_sync(peers, bit);
  const int leader = __ffs(peers) - 1;
  uint32_t old = 0u;
  if (active && lane == leader) old = atomicOr(bm + (v >> 5), bits);
  old = __shfl_sync(GR_FULL_MASK, old, leader);
  return active && !(old & bit) && (__ffs(same) - 1) == lane;
}

// Warp-aggregated setting of bit v in a bitmap (no result needed): one
// atomicOr per distinct word.  All 32 lanes call.
__device__ __forceinline__ void gr_warp_set_bit(uint32_t* bm, bool set, int32_t v, int lane) {
#if !GR_CLAIM_AGGREGATE
  if (set) gr_red_or_u32(bm + (v >> 5), 1u << (v & 31));
  return;
#endif
  const unsigned wkey = set ? (unsigned)v >> 5 : (0x80000000u | (unsigned)lane);
  const unsigned peers = __match_any_sync(GR_FULL_MASK, wkey);
  const uint32_t bits = __reduce_or_sync(peers, set ? 1u << (v & 31) : 0u);
  if (set && lane == __ffs(peers) - 1) atomicOr(bm + (v >> 5), bits);
}

// Per-CTA staging of frontier appends in shared memory.  Warps append with
// one shared-memory atomic per 32 candidates; at the end of the step the CTA
// moves its entries to the global queue with ONE global atomicAdd, instead
// of one per warp and strip (appends from every warp of the grid to a single
// counter serialise in L2).  Entries beyond the shared capacity go straight
// to global memory.
#define GR_STAGE_CAP 2048
struct GrStage {
  int* buf;  // shared, cap entries
  int* cnt;  // shared
  int* base; // shared
  int cap;
  // one thread; a __syncthreads must follow before the first append
  __device__ __forceinline__ void reset() { *cnt = 0; }
  // all 32 lanes
  __device__ __forceinline__ void append(int32_t* gq, int* glen, int64_t gcap, bool take,
                                         int32_t v, int lane) {
    const unsigned mask = __ballot_sync(GR_FULL_MASK, take);
    if (mask == 0) return;
    const int leader = __ffs(mask) - 1;
    int b = 0;
    if (lane == leader) b = atomicAdd(cnt, __popc(mask));
    b = __shfl_sync(GR_FULL_MASK, b, leader);
    const int pos = b + __popc(mask & ((1u << lane) - 1u));
    const bool over = take && pos >= cap;
    if (take && !over) buf[pos] = v;
    gr_warp_append(gq, glen, gcap, over, v, lane);
  }
  // every thread of the CTA
  __device__ __forceinline__ void flush(int32_t* gq, int* glen, int64_t gcap) {
    __syncthreads();
    reserve(glen);
    __syncthreads();
    copy_out(gq, gcap);
  }
  // The two halves of flush, for a CTA that flushes several stages at once:
  // after a __syncthreads, thread 0 reserves every stage's block (the
  // global atomics are then in flight together); after another
  // __syncthreads every thread copies.
  __device__ __forceinline__ void reserve(int* glen) {
    if (threadIdx.x != 0) return;
    const int c = min(*cnt, cap);
    *base = c > 0 ? atomicAdd(glen, c) : 0;
  }
  __device__ __forceinline__ void copy_out(int32_t* gq, int64_t gcap) {
    const int c = min(*cnt, cap);
    const int b = *base;
    for (int i = threadIdx.x; i < c; i += blockDim.x)
      if (b + i < gcap) gq[b + i] = buf[i];
  }
};

// Larger staging buffers for a kernel that runs one CTA per SM (SSSP): its
// steps append up to a few thousand vertices per CTA, more than the static
// arena holds.  Lives in dynamic shared memory.
#define GR_BIG_NEAR_CAP 16384
#define GR_BIG_MID_CAP 8192
#define GR_BIG_FAR_CAP 8192
struct GrStageBufs {
  int near[GR_BIG_NEAR_CAP];
  int mid[GR_BIG_MID_CAP];
  int far[GR_BIG_FAR_CAP];
};

// Warp-centric expansion of the rows of up to 32 sources (one per lane):
// the warp scans the lanes' degrees and walks the concatenated edge ranges
// 32 edges at a time; each lane finds the source of its edge with a 5-step
// binary search over the scanned offsets held in registers (shuffles).
// edge(active, src_lane_value, payload, e, v) is called by all 32 lanes.
template <class Edge>
__device__ __forceinline__ void gr_warp_expand(const int32_t* __restrict__ R,
                                               const int32_t* __restrict__ C, bool valid,
                                               int32_t u, int beg, int deg, uint32_t payload,
                                               int lane, Edge&& edge) {
  if (!valid) deg = 0;
  int total;
  int off = gr_warp_excl_scan(deg, lane, &total);
  for (int base = 0; base < total; base += 32) {
    int pos = base + lane;
    int lo = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
      int cand = lo + step;
      int oc = __shfl_sync(GR_FULL_MASK, off, cand);
      if (oc <= pos) lo = cand;
    }
    int sbeg = __shfl_sync(GR_FULL_MASK, beg, lo);
    int soff = __shfl_sync(GR_FULL_MASK, off, lo);
    int su = __shfl_sync(GR_FULL_MASK, u, lo);
    uint32_t sp = __shfl_sync(GR_FULL_MASK, payload, lo);
    bool active = pos < total;
    int e = sbeg + (pos - soff);
    int v = active ? __ldg(C + e) : 0;
    edge(active, su, sp, e, v);
  }
}

// As gr_warp_expand, but U strips (32 * U edges) per round, in three passes
// so that the memory accesses of the U strips overlap: first every lane
// locates its U edges and loads their columns (streaming loads, so the
// column stream does not evict the per-vertex state that lives in L2), then
// `pre(active, e, v)`
// issues the per-edge loads the functor needs (its results are returned),
// and only then `edge(active, src, payload, e, v, pre_value)` runs for each
// strip.  All lanes call both functors.  The _mid form runs two more stages
// in between, each for all U strips before the next: `mid1` and `mid2`, with
// the arguments of `edge` and the pre value by reference.  Atomics whose results a
// later stage needs, and loads that depend on those results, are then in
// flight for all strips together; issued from `edge` they would wait strip
// by strip (the compiler keeps them in program order).
template <int U, class Pre, class Mid1, class Mid2, class Edge>
__device__ __forceinline__ void gr_warp_expand_mid_u(const int32_t* __restrict__ R,
                                                     const int32_t* __restrict__ C, bool valid,
                                                     int32_t u, int beg, int deg,
                                                     uint32_t payload, int lane, Pre&& pre,
                                                     Mid1&& mid1, Mid2&& mid2, Edge&& edge) {
  if (!valid) deg = 0;
  int total;
  const int off = gr_warp_excl_scan(deg, lane, &total);
  for (int base = 0; base < total; base += 32 * U) {
    int su[U], e[U], v[U];
    uint32_t sp[U];
    bool act[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int pos = base + k * 32 + lane;
      int lo = 0;
#pragma unroll
      for (int step = 16; step >= 1; step >>= 1) {
        const int cand = lo + step;
        if (__shfl_sync(GR_FULL_MASK, off, cand) <= pos) lo = cand;
      }
      const int sbeg = __shfl_sync(GR_FULL_MASK, beg, lo);
      const int soff = __shfl_sync(GR_FULL_MASK, off, lo);
      su[k] = __shfl_sync(GR_FULL_MASK, u, lo);
      sp[k] = __shfl_sync(GR_FULL_MASK, payload, lo);
      act[k] = pos < total;
      e[k] = sbeg + (pos - soff);
    }
#pragma unroll
    for (int k = 0; k < U; ++k) v[k] = act[k] ? GR_LDSTREAM(C + e[k]) : 0;
    decltype(pre(true, 0, 0)) pv[U];
#pragma unroll
    for (int k = 0; k < U; ++k) pv[k] = pre(act[k], e[k], v[k]);
#pragma unroll
    for (int k = 0; k < U; ++k) mid1(act[k], su[k], sp[k], e[k], v[k], pv[k]);
#pragma unroll
    for (int k = 0; k < U; ++k) mid2(act[k], su[k], sp[k], e[k], v[k], pv[k]);
#pragma unroll
    for (int k = 0; k < U; ++k) edge(act[k], su[k], sp[k], e[k], v[k], pv[k]);
  }
}

struct GrNoMid {
  template <class P>
  __device__ __forceinline__ void operator()(bool, int32_t, uint32_t, int, int32_t, P&) const {}
};

template <int U, class Pre, class Edge>
__device__ __forceinline__ void gr_warp_expand_u(const int32_t* __restrict__ R,
                                                 const int32_t* __restrict__ C, bool valid,
                                                 int32_t u, int beg, int deg, uint32_t payload,
                                                 int lane, Pre&& pre, Edge&& edge) {
  gr_warp_expand_mid_u<U>(R, C, valid, u, beg, deg, payload, lane, pre, GrNoMid{}, GrNoMid{},
                          edge);
}

// Chunk counterpart of gr_warp_expand_mid_u / gr_warp_expand_u: edges
// [e0, e1) of row u.
template <int U, class Pre, class Mid1, class Mid2, class Edge>
__device__ __forceinline__ void gr_warp_chunk_mid_u(const int32_t* __restrict__ C, int32_t u,
                                                    int e0, int e1, uint32_t payload, int lane,
                                                    Pre&& pre, Mid1&& mid1, Mid2&& mid2,
                                                    Edge&& edge) {
  for (int base = e0; base < e1; base += 32 * U) {
    int e[U], v[U];
    bool act[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      e[k] = base + k * 32 + lane;
      act[k] = e[k] < e1;
      v[k] = act[k] ? GR_LDSTREAM(C + e[k]) : 0;
    }
    decltype(pre(true, 0, 0)) pv[U];
#pragma unroll
    for (int k = 0; k < U; ++k) pv[k] = pre(act[k], e[k], v[k]);
#pragma unroll
    for (int k = 0; k < U; ++k) mid1(act[k], u, payload, e[k], v[k], pv[k]);
#pragma unroll
    for (int k = 0; k < U; ++k) mid2(act[k], u, payload, e[k], v[k], pv[k]);
#pragma unroll
    for (int k = 0; k < U; ++k) edge(act[k], u, payload, e[k], v[k], pv[k]);
  }
}

template <int U, class Pre, class Edge>
__device__ __forceinline__ void gr_warp_chunk_u(const int32_t* __restrict__ C, int32_t u, int e0,
                                                int e1, uint32_t payload, int lane, Pre&& pre,
                                                Edge&& edge) {
  gr_warp_chunk_mid_u<U>(C, u, e0, e1, payload, lane, pre, GrNoMid{}, GrNoMid{}, edge);
}

// Static-first / dynamic loop over a row list, `per` rows per warp batch,
// each batch expanded with gr_warp_expand_mid_u<U>; payload(u) gives the
// value passed to the edge functor with every edge of row u.
template <int U, class Payload, class Pre, class Mid1, class Mid2, class Edge>
__device__ __forceinline__ void gr_rows_loop_mid(const int32_t* list, int len, int per,
                                                 int* counter, int swarp, int nwarps, int lane,
                                                 const int32_t* __restrict__ R,
                                                 const int32_t* __restrict__ C, GrCounters& cnt,
                                                 Payload&& payload, Pre&& pre, Mid1&& mid1,
                                                 Mid2&& mid2, Edge&& edge) {
  for (int base = swarp * per; base < len;
       base = gr_next_batch(base, len, nwarps * per, counter, per, lane)) {
    const int i = base + lane;
    const bool valid = lane < per && i < len;
    int32_t u = 0;
    int beg = 0, deg = 0;
    uint32_t pl = 0;
    if (valid) {
      ++cnt.verts;
      u = __ldcg(list + i);
      beg = __ldg(R + u);
      deg = __ldg(R + u + 1) - beg;
      pl = payload(u);
    }
    gr_warp_expand_mid_u<U>(R, C, valid, u, beg, deg, pl, lane, pre, mid1, mid2, edge);
  }
}

template <int U, class Payload, class Pre, class Edge>
__device__ __forceinline__ void gr_rows_loop(const int32_t* list, int len, int per, int* counter,
                                             int swarp, int nwarps, int lane,
                                             const int32_t* __restrict__ R,
                                             const int32_t* __restrict__ C, GrCounters& cnt,
                                             Payload&& payload, Pre&& pre, Edge&& edge) {
  gr_rows_loop_mid<U>(list, len, per, counter, swarp, nwarps, lane, R, C, cnt, payload, pre,
                      GrNoMid{}, GrNoMid{}, edge);
}

// Loop over the edge chunks of split rows.  Chunks hold at most
// GR_CHUNK_EDGES edges each, so they are dealt out statically (warp w takes
// chunks w, w + nwarps, ...; no counter), and each warp prefetches two chunks
// ahead: the entry of chunk c + 2 * nwarps and the row end and payload of
// chunk c + nwarps are in flight while chunk c is expanded; with edge values
// W (4-byte entries indexed like the columns) the columns and values of
// chunk c + nwarps are also prefetched into L2, so that its expansion starts
// from L2 instead of DRAM (1 % on R-MAT s22 SSSP; for column-only loops the
// prefetch measured slower).
__device__ __forceinline__ void gr_prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
template <int U, class Payload, class Pre, class Mid1, class Mid2, class Edge>
__device__ __forceinline__ void gr_chunks_loop_mid(const int2* ch, int nch, int swarp,
                                                   int nwarps, int lane,
                                                   const int32_t* __restrict__ R,
                                                   const int32_t* __restrict__ C,
                                                   GrCounters& cnt, Payload&& payload,
                                                   Pre&& pre, Mid1&& mid1, Mid2&& mid2,
                                                   Edge&& edge,
                                                   const uint32_t* __restrict__ W = nullptr) {
  static_assert(GR_CHUNK_EDGES <= 256, "nine 128-byte lines cover a chunk");
  int c = swarp;
  if (c >= nch) return;
  int2 cur = __ldcg(ch + c);
  int2 nxt = c + nwarps < nch ? __ldcg(ch + c + nwarps) : make_int2(0, 0);
  int cur_end = min(cur.y + GR_CHUNK_EDGES, __ldg(R + cur.x + 1));
  uint32_t cur_pl = payload(cur.x);
  for (; c < nch; c += nwarps) {
    const int cn = c + nwarps, cnn = c + 2 * nwarps;
    const int2 nn = cnn < nch ? __ldcg(ch + cnn) : make_int2(0, 0);
    int nxt_end = 0;
    uint32_t nxt_pl = 0;
    if (cn < nch) {
      nxt_end = min(nxt.y + GR_CHUNK_EDGES, __ldg(R + nxt.x + 1));
      nxt_pl = payload(nxt.x);
      // lanes 0-8: the chunk's column lines, lanes 16-24: its W lines
      const int pe = nxt.y + (lane & 15) * 32;
      if (W && (lane & 15) < 9 && pe < nxt_end)
        gr_prefetch_l2(lane < 16 ? (const void*)(C + pe) : (const void*)(W + pe));
    }
    if (lane == 0) ++cnt.verts;
    gr_warp_chunk_mid_u<U>(C, cur.x, cur.y, cur_end, cur_pl, lane, pre, mid1, mid2, edge);
    cur = nxt;
    cur_end = nxt_end;
    cur_pl = nxt_pl;
    nxt = nn;
  }
}

template <int U, class Payload, class Pre, class Edge>
__device__ __forceinline__ void gr_chunks_loop(const int2* ch, int nch, int swarp, int nwarps,
                                               int lane, const int32_t* __restrict__ R,
                                               const int32_t* __restrict__ C, GrCounters& cnt,
                                               Payload&& payload, Pre&& pre, Edge&& edge,
                                               const uint32_t* __restrict__ W = nullptr) {
  gr_chunks_loop_mid<U>(ch, nch, swarp, nwarps, lane, R, C, cnt, payload, pre, GrNoMid{},
                        GrNoMid{}, edge, W);
}

// Default SSSP bucket width: 256 * mean weight / mean degree (at least 1).
// Wide buckets trade a few repeated relaxations for far fewer grid-wide
// steps, which is what bounds both low-diameter and mesh-like graphs here.
inline uint32_t gr_default_delta(const gr_graph* g) {
  if (g->m == 0 || g->nonisolated == 0) return 1;
  double wmean = (double)g->weight_sum / (double)g->m;
  double dmean = (double)g->m / (double)g->nonisolated;
  double d = 256.0 * wmean / dmean;
  if (d < 1.0) d = 1.0;
  if (d > 1e9) d = 1e9;
  return (uint32_t)d;
}

// Walk one edge chunk [e0, e1) of row u with the whole warp.
template <class Edge>
__device__ __forceinline__ void gr_warp_chunk(const int32_t* __restrict__ C, int32_t u, int e0,
                                              int e1, uint32_t payload, int lane, Edge&& edge) {
  for (int e = e0 + lane; e - lane < e1; e += 32) {
    bool active = e < e1;
    int v = active ? __ldg(C + e) : 0;
    edge(active, u, payload, e, v);
  }
}

// Register the edge chunks of a split row (degree >= the split threshold):
// ceil(deg / GR_CHUNK_EDGES) entries (row, first edge) go to the chunk list of
// the next step, so that the whole grid shares one long row (the paper's
// "lists larger than a block" class, Sec. 5.1.2, balanced over edges as in
// Sec. 5.1.3).  Called by single lanes; no warp collectives inside.
__device__ __forceinline__ void gr_register_chunks(int2* chunks, int64_t cap, int* nchunk,
                                                   int* nbig, int32_t v, int beg, int deg,
                                                   int* status) {
  int nch = (deg + GR_CHUNK_EDGES - 1) / GR_CHUNK_EDGES;
  int pos = atomicAdd(nchunk, nch);
  atomicAdd(nbig, 1);
  for (int k = 0; k < nch; ++k) {
    if (pos + k < cap) chunks[pos + k] = make_int2(v, beg + k * GR_CHUNK_EDGES);
    else gr_set_status(status, GR_ERR_CAPACITY);
  }
}

// The source row's chunks at initialisation, written by every thread of the
// scope (tid / nthreads), one chunk each: the chunk list is empty then, so
// the row takes slots [0, nch) and thread 0 sets the counters (zero before).
// Registered by one thread, the 637 chunks of the R-MAT s22 hub row took
// 20 us before the first barrier.
__device__ __forceinline__ void gr_register_source_chunks(int2* chunks, int64_t cap, int* nchunk,
                                                          int* nbig, int32_t v, int beg, int deg,
                                                          int* status, int64_t tid,
                                                          int64_t nthreads) {
  const int nch = (deg + GR_CHUNK_EDGES - 1) / GR_CHUNK_EDGES;
  for (int64_t k = tid; k < nch; k += nthreads)
    if (k < cap) chunks[k] = make_int2(v, beg + (int)k * GR_CHUNK_EDGES);
  if (tid == 0) {
    *nchunk = nch;
    *nbig = 1;
    if (nch > cap) gr_set_status(status, GR_ERR_CAPACITY);
  }
}

// Per-CTA staging of split rows (rows of degree >= the split threshold
// discovered in a step): the CTA reserves all their edge chunks with one
// global atomicAdd at the end of the step instead of one per row.  Rows
// beyond the shared capacity are registered directly.
#define GR_BIG_STAGE_CAP 1024
struct GrBigStage {
  int* v;    // shared, GR_BIG_STAGE_CAP entries each
  int* beg;
  int* deg;
  int* off;  // shared, GR_BIG_STAGE_CAP: chunk offset of each row within the CTA
  int* cnt;  // shared
  int* tot;  // shared [0] chunks of this CTA, [1] global base
  __device__ __forceinline__ void reset() { *cnt = 0; }
  // single lane
  __device__ __forceinline__ void add(int2* chunks, int64_t cap, int* nchunk, int* nbig,
                                      int32_t row, int b, int d, int* status) {
    const int pos = atomicAdd(cnt, 1);
    if (pos < GR_BIG_STAGE_CAP) {
      v[pos] = row;
      beg[pos] = b;
      deg[pos] = d;
    } else {
      gr_register_chunks(chunks, cap, nchunk, nbig, row, b, d, status);
    }
  }
  // every thread of the CTA: chunk ranges are reserved with shared-memory
  // atomics, then one global atomicAdd places the CTA's block of chunks
  __device__ __forceinline__ void flush(int2* chunks, int64_t cap, int* nchunk, int* nbig,
                                        int* status) {
    __syncthreads();
    prepare();
    reserve(nchunk, nbig);
    __syncthreads();
    copy_out(chunks, cap, status);
  }
  // Split form for a combined flush: prepare() (every thread, after a
  // __syncthreads; ends with one) lays the CTA's chunks out, reserve() (thread
  // 0) places them, copy_out() (every thread, after a __syncthreads) writes.
  __device__ __forceinline__ void prepare() {
    const int c = min(*cnt, GR_BIG_STAGE_CAP);
    if (c == 0) return;  // uniform: every thread read the same count
    if (threadIdx.x == 0) tot[0] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < c; i += blockDim.x)
      off[i] = atomicAdd(&tot[0], (deg[i] + GR_CHUNK_EDGES - 1) / GR_CHUNK_EDGES);
    __syncthreads();
  }
  __device__ __forceinline__ void reserve(int* nchunk, int* nbig) {
    const int c = min(*cnt, GR_BIG_STAGE_CAP);
    if (threadIdx.x != 0 || c == 0) return;
    tot[1] = atomicAdd(nchunk, tot[0]);
    atomicAdd(nbig, c);
  }
  __device__ __forceinline__ void copy_out(int2* chunks, int64_t cap, int* status) {
    const int c = min(*cnt, GR_BIG_STAGE_CAP);
    if (c == 0) return;
    const int gbase = tot[1];
    for (int i = threadIdx.x >> 5; i < c; i += blockDim.x >> 5) {  // a warp per row
      const int nch = (deg[i] + GR_CHUNK_EDGES - 1) / GR_CHUNK_EDGES;
      const int o = gbase + off[i];
      for (int k = threadIdx.x & 31; k < nch; k += 32) {
        if (o + k < cap) chunks[o + k] = make_int2(v[i], beg[i] + k * GR_CHUNK_EDGES);
        else gr_set_status(status, GR_ERR_CAPACITY);
      }
    }
  }
};

// Shared-memory arena for the staging buffers of a query body; a kernel
// declares one and passes it to whichever body it runs (the batched kernel
// holds both bodies but needs only one arena).
struct GrArena {
  int buf0[GR_STAGE_CAP];  // BFS next frontier / SSSP near frontier
  int bufm[GR_STAGE_CAP];  // medium rows of the next frontier
  int buf1[GR_STAGE_CAP];  // BFS unvisited list / SSSP far pile
  int bv[GR_BIG_STAGE_CAP], bb[GR_BIG_STAGE_CAP], bd[GR_BIG_STAGE_CAP], bo[GR_BIG_STAGE_CAP];
};

// Position of the r-th (0-based) set bit of w; w must have more than r set
// bits.  Five halving steps on population counts.
__device__ __forceinline__ int gr_nth_set_bit(uint32_t w, int r) {
  int pos = 0;
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const int c = __popc(w & ((1u << s) - 1u));
    if (c <= r) {
      r -= c;
      w >>= s;
      pos += s;
    }
  }
  return pos;
}

// Warp-wide minimum of an unsigned.
__device__ __forceinline__ unsigned gr_warp_min_u32(unsigned x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = min(x, __shfl_xor_sync(GR_FULL_MASK, x, o));
  return x;
}

// Host helpers shared by the translation units.
int gr_launch_blocks(const void* kernel, int threads, size_t smem, int num_sms, int requested);
cudaError_t gr_reset_ctl(gr_workspace* ws, cudaStream_t s);
gr_workspace* gr_resolve_ws(const gr_graph* g, gr_workspace* ws);
