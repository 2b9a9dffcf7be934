// gr_sssp.cu — SSSP as one persistent, cooperative kernel with a two-level
// (near/far) priority queue.
//
// The paper's SSSP (Sec. 3 example, Alg. 1, Sec. 6.2) iterates advance with
// the Update_Label / Set_Pred functors (atomicMin on the label), a filter
// that removes redundant frontier entries (Remove_Redundant), and a priority
// queue that splits the output into a "near" pile, processed until empty,
// and a "far" pile, revisited when the near threshold is raised
// (Sec. 5.1.5, delta-stepping).  This kernel runs those steps on the device:
//   * a RELAX step expands the near frontier (warp-centric rows plus grid-
//     shared chunks of long rows, as in BFS) and relaxes every edge with one
//     64-bit atomicMin on key[v] = (dist << 32) | pred, so label and
//     predecessor change together and the final pred is the smallest-id
//     tight predecessor; a vertex whose distance dropped joins the next near
//     frontier if dist < T, else the far pile, each at most once per step /
//     epoch (stamp arrays play the role of Alg. 1's output_queue_ids);
//   * when the near frontier is empty, a SPLIT step raises T by delta (or
//     jumps to the bucket of the smallest far distance) and moves far
//     entries with dist < T to the near frontier, dropping stale ones;
//   * the loop ends when both piles are empty, then keys are unpacked into
//     the caller's dist / pred arrays.
#include <climits>

#include "gr_sssp_body.cuh"

namespace {

// CTA width, one CTA per SM.  Graphs with long rows (scale-free) run 20
// warps: the register file then allows 96 registers a thread, which this
// kernel fits without spilling, and the extra warps keep more label gathers
// in flight (on R-MAT s22 an SSSP took 3.4 % less time than with 16 warps
// at 126 registers, and 6 % less than with 24 warps at 80 registers, which
// spill).  Graphs whose rows are all short (meshes) run 16 warps: their
// thousands of small steps are bound by barriers, which wider CTAs slow
// (3 % on a 4096^2 grid).
constexpr int NT_WIDE = 640;
constexpr int NT_NARROW = 512;

#ifndef GR_SSSP_MIN_BLOCKS
#define GR_SSSP_MIN_BLOCKS 1
#endif
#ifndef GR_SSSP_BIG_STAGE
#define GR_SSSP_BIG_STAGE 1  // staging buffers in dynamic shared memory (else the static arena)
#endif
template <int NT>
__global__ void __launch_bounds__(NT, GR_SSSP_MIN_BLOCKS) sssp_persistent(SsspArgs a) {
  GridScope sc{a.ctl, a.status, a.spin, (int64_t)blockIdx.x * NT + threadIdx.x,
               (int64_t)gridDim.x * NT, 0u};
  __shared__ GrArena ar;
  extern __shared__ GrStageBufs big[];  // one CTA per SM: room for large staging buffers
  gr_sssp_body<NT == NT_NARROW>(a, sc, ar, GR_SSSP_BIG_STAGE ? big : nullptr);
}

}  // namespace

extern "C" void gr_sssp_opts_default(gr_sssp_opts* o) {
  if (!o) return;
  o->delta = 0;
  o->big_degree = GR_DEFAULT_SSSP_BIG;
  o->blocks_per_sm = 0;
  o->spin_limit = GR_DEFAULT_SPIN_LIMIT;
  o->ws = nullptr;
  o->level_stats = nullptr;
  o->max_levels = 0;
  o->bulk_rows = 0;
  o->max_blocks = 0;
  o->levels = 0;
}

// Bucket width from the graph: 256 * mean weight / mean degree, at least 1
// (wide buckets: a few repeated relaxations for far fewer grid-wide steps).
static uint32_t default_delta(const gr_graph* g) { return gr_default_delta(g); }

extern "C" gr_status gr_sssp(const gr_graph* g, int32_t src, uint32_t* dist, int32_t* pred,
                             const gr_sssp_opts* opts, void* stream) {
  if (!g || !dist || g->n <= 0 || src < 0 || src >= g->n) return GR_ERR_INVALID_ARG;
  if (!g->W && g->m > 0) return GR_ERR_UNSUPPORTED;
  gr_sssp_opts o;
  gr_sssp_opts_default(&o);
  if (opts) o = *opts;
  if (o.max_levels < 0 || (o.max_levels > 0 && !o.level_stats) || o.max_blocks < 0 ||
      (o.levels != 0 && o.levels != 2 && o.levels != GR_RING_K))
    return GR_ERR_INVALID_ARG;
  gr_workspace* ws = gr_resolve_ws(g, o.ws);
  if (!ws || ws->g != g || !ws->key) return GR_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;

  SsspArgs a = {};
  a.n = g->n;
  a.R = g->R;
  a.C = g->C;
  a.W = g->W;
  a.key = (unsigned long long*)ws->key;
  a.dist = dist;
  a.pred = pred;
  a.q[0] = ws->q[0];
  a.q[1] = ws->q[1];
  a.qm[0] = ws->qm[0];
  a.qm[1] = ws->qm[1];
  a.ch[0] = ws->chunks[0];
  a.ch[1] = ws->chunks[1];
  a.chunk_cap = ws->chunk_cap;
  a.far[0] = ws->far[0];
  a.far[1] = ws->far[1];
  a.stamp_near = ws->stamp_near;
  a.stamp_far = ws->stamp_far;
  a.touched = o.bulk_rows < 0 ? nullptr : ws->visited;  // the BFS bitmap is free here
  a.bulk_rows = o.bulk_rows > 0 ? o.bulk_rows
                 : g->max_degree >= GR_SKEWED_DEGREE ? GR_SKEWED_BULK_ROWS
                                                     : gr_default_bulk_rows(g->n);
  a.ctl = ws->ctl;
  a.status = ws->status;
  a.src = src;
  a.delta = o.delta ? o.delta : default_delta(g);
  a.big = o.big_degree > 0 ? (o.big_degree < 32 ? 32 : o.big_degree) : GR_DEFAULT_SSSP_BIG;
  a.track_deg = g->max_degree >= GR_MEDIUM_DEGREE;
  a.spin = o.spin_limit ? o.spin_limit : GR_DEFAULT_SPIN_LIMIT;
  a.level_stats = o.level_stats;
  a.max_levels = o.max_levels;
  if (o.levels != 2) {
    for (int j = 0; j < GR_RING_K; ++j) a.ring[j] = ws->ring[j];
    a.stamp_ring = ws->stamp_ring;
  }

  const bool wide = g->max_degree >= GR_MEDIUM_DEGREE;
  const void* kernel = wide ? (const void*)sssp_persistent<NT_WIDE>
                            : (const void*)sssp_persistent<NT_NARROW>;
  const int nt = wide ? NT_WIDE : NT_NARROW;
  const size_t smem = sizeof(GrStageBufs);  // the dynamic shared-memory limit is raised once
  int blocks = gr_launch_blocks(kernel, nt, smem, g->num_sms, o.blocks_per_sm);
  if (blocks <= 0) return GR_ERR_CUDA;
  if (o.max_blocks > 0 && blocks > o.max_blocks) blocks = o.max_blocks;
  if (gr_reset_ctl(ws, s) != cudaSuccess) return GR_ERR_CUDA;
  void* args[] = {&a};
  if (cudaLaunchCooperativeKernel(kernel, dim3(blocks), dim3(nt), args, smem, s) != cudaSuccess) {
    (void)cudaGetLastError();
    return GR_ERR_CUDA;
  }
  return GR_OK;
}
