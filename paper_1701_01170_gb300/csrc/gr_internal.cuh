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

// Library defaults (tunable per call through gr_bfs_opts / gr_sssp_opts).
#define GR_DEFAULT_BIG_DEGREE 1024   // rows >= this are split into edge chunks
#define GR_CHUNK_EDGES 1024          // edges per chunk of a split row
#define GR_DEFAULT_SPIN_LIMIT (1u << 24)
#define GR_TIME_LIMIT_NS (60ull * 1000000000ull)  // persistent kernels give up after 60 s
#define GR_PERSIST_THREADS 512
#define GR_OPS_THREADS 256
#define GR_SCAN_ITEMS 16             // items per thread in the operator scans
#define GR_SCAN_TILE (GR_OPS_THREADS * GR_SCAN_ITEMS)
#define GR_MAX_SCAN_BLOCKS ((int64_t)1 << 19)  // covers in_len < 2^31

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
  unsigned farmin[3];              // SSSP smallest distance pushed to a far pile
  int ovf_pending;                 // SSSP: some relaxation sum did not fit in 32 bits
  unsigned long long mf[3];        // sum of degrees of the next frontier
  unsigned long long edges;        // column entries read (statistics)
  unsigned long long verts;        // rows opened: frontier rows, chunks, pull candidates
  unsigned long long updates;      // BFS discoveries / SSSP successful relaxations
};

// Per-thread work counters of a persistent kernel, flushed once at exit.
struct GrCounters {
  unsigned long long edges = 0, verts = 0, updates = 0;
  __device__ __forceinline__ void flush(GrCtl* ctl) {
    unsigned long long e = edges, v = verts, u = updates;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e += __shfl_xor_sync(0xffffffffu, e, o);
      v += __shfl_xor_sync(0xffffffffu, v, o);
      u += __shfl_xor_sync(0xffffffffu, u, o);
    }
    if ((threadIdx.x & 31) == 0) {
      if (e) atomicAdd(&ctl->edges, e);
      if (v) atomicAdd(&ctl->verts, v);
      if (u) atomicAdd(&ctl->updates, u);
    }
  }
};

struct GrMsState;                  // multi-source BFS scratch (gr_msbfs.cu)
void gr_ms_free(GrMsState* ms);

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
};

struct gr_workspace {
  const gr_graph* g;
  int32_t ops;
  GrCtl* ctl;
  int* status;
  int* h_status;        // pinned host mirror used by gr_sync_status
  int32_t* q[2];        // frontier queues (ping-pong), n entries each
  int2* chunks[2];      // (row, first edge) chunks of split rows (ping-pong)
  int64_t chunk_cap;
  uint32_t* visited;    // n bits
  uint32_t* front[3];   // frontier bitmaps, n bits each (rotating)
  uint64_t* key;        // SSSP packed (dist << 32 | pred)
  int32_t* far[2];      // SSSP far piles (ping-pong), n entries each
  int32_t* stamp_near;  // SSSP near-queue membership stamps
  int32_t* stamp_far;   // SSSP far-pile membership stamps
  int32_t* first_idx;   // filter scratch: n entries, INT32_MAX when clean
  uint32_t* claim;      // filter scratch: n bits, 0 when clean
  long long* block_sums;// operator scan scratch, GR_MAX_SCAN_BLOCKS + 2 entries
  int32_t* tags;        // pull scratch: n entries
  long long* item_off;  // advance scratch: n + 1 per-item output offsets
  long long* dev_len;   // operator scratch: a few device counters
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

#define GR_PULL_WORDS 16

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
