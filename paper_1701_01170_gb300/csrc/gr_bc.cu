// gr_bc.cu — betweenness centrality of one source as one persistent,
// cooperative kernel (Sec. 6.3: Brandes' two passes on the frontier operators).
//
// Forward pass: the advance of BFS (Sec. 6.1) level by level.  Every edge
// (u, v) whose target has no depth yet claims it with a compare-and-swap on
// depth[v] (the winner appends v to the next level); every edge whose target
// sits on the next level (claimed now, by this thread or another) adds
// sigma[u] to sigma[v] with a 64-bit atomic, so that sigma[v] ends as the
// number of shortest src -> v paths.  Integer additions commute, so the path
// counts are exact whatever the order; an addition that would pass INT64_MAX
// records GR_ERR_OVERFLOW.  The levels are stored one after another in a BFS
// order array (level L = order[lvl[L], lvl[L+1])), and rows of at least the
// split degree are also listed as GR_CHUNK_EDGES-edge chunks per level.
//
// Backward pass: from the deepest level up, each vertex u of level L sums
// sigma[u] / sigma[v] * (1 + delta[v]) over its edges to level L + 1 — the
// dependency accumulation of the same section, taken as a reduction over u's
// row.  A warp takes 32 short rows at a time and sums per row in shared
// memory; long rows are shared by the grid as chunks whose partial sums are
// added to delta[u] with one double atomic each.  A grid barrier separates
// levels, so delta[v] is final before level L reads it.
//
// Finally bc[v] += delta[v] for every v != src (ordered source/target pairs).
#include <climits>
#include <mutex>
#include <new>

#include "gr_internal.cuh"

struct GrBcScratch {
  int32_t n;
  int32_t* depth;
  unsigned long long* sigma;
  double* delta;
  int32_t* order;   // vertices in BFS order, n entries
  int32_t* lvl;     // level starts in order[], n + 2 entries
  int32_t* clvl;    // level starts in chunks[], n + 2 entries
  int2* chunks;     // (row, first edge) chunks of the long rows of every level
  int64_t chunk_cap;
};

void gr_bc_free(GrBcScratch* b) {
  if (!b) return;
  void* ptrs[] = {b->depth, b->sigma, b->delta, b->order, b->lvl, b->clvl, b->chunks};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete b;
}

namespace {

constexpr int NT = GR_PERSIST_THREADS;
constexpr int WPC = NT / 32;
#ifndef GR_BC_STRIPS
#define GR_BC_STRIPS 2  // strips per warp round (64 registers at 2 CTAs per SM)
#endif

struct BcArgs {
  int32_t n;
  const int32_t* __restrict__ R;
  const int32_t* __restrict__ C;
  int32_t* depth;
  unsigned long long* sigma;
  double* delta;
  double* bc;
  int32_t* order;
  int32_t* lvl;
  int32_t* clvl;
  int2* chunks;
  int64_t chunk_cap;
  GrCtl* ctl;
  int* status;
  int32_t src;
  int big;
  unsigned spin;
};

constexpr unsigned long long kSigmaMax = 0x7fffffffffffffffull;

__global__ void __launch_bounds__(NT, 2) bc_persistent(BcArgs a) {
  GridScope sc{a.ctl, a.status, a.spin, (int64_t)blockIdx.x * NT + threadIdx.x,
               (int64_t)gridDim.x * NT, 0u};
  __shared__ GrArena ar;
  __shared__ double s_acc[WPC][32];
  const int lane = threadIdx.x & 31;
  const int64_t gtid = sc.tid, gthreads = sc.nthreads;
  const int64_t gwarp = gtid >> 5, nwarps = gthreads >> 5;
  const int swarp = (int)((gwarp % WPC) * (nwarps / WPC) + gwarp / WPC);
  GrCtl* ctl = a.ctl;

  // ---- initialisation: no depths, no paths, no dependencies; src at level 0
  for (int64_t v = gtid; v < a.n; v += gthreads) {
    a.depth[v] = v == a.src ? 0 : -1;
    a.sigma[v] = v == a.src ? 1ull : 0ull;
    a.delta[v] = 0.0;
  }
  if (gtid == 0) {
    a.order[0] = a.src;
    a.lvl[0] = 0;
    a.lvl[1] = 1;
    a.clvl[0] = 0;
    const int beg = a.R[a.src], deg = a.R[a.src + 1] - beg;
    if (deg >= a.big)
      gr_register_chunks(a.chunks, a.chunk_cap, &ctl->nchunk[0], &ctl->nbig[0], a.src, beg, deg,
                         a.status);
  }
  if (!sc.sync()) return;
  const unsigned long long deadline = gr_globaltimer() + GR_TIME_LIMIT_NS;

  __shared__ int s_cnt, s_nch;
  __shared__ int s_qcnt, s_qbase, s_bcnt, s_btot[2];
  GrStage stage{ar.buf0, &s_qcnt, &s_qbase, GR_STAGE_CAP};
  GrBigStage bstage{ar.bv, ar.bb, ar.bd, ar.bo, &s_bcnt, s_btot};
  GrCounters cnt;
  double* acc = s_acc[threadIdx.x >> 5];

  // ---- forward pass ------------------------------------------------------
  int lb = 0, le = 1;         // level L = order[lb, le)
  int cb = 0;                 // its chunks start at chunks[cb]
  int L = 0;
  for (;; ++L) {
    const int s0 = L % 3, s1 = (L + 1) % 3, s2 = (L + 2) % 3;
    if (threadIdx.x == 0) {
      s_nch = __ldcg(&ctl->nchunk[s0]);
      stage.reset();
      bstage.reset();
    }
    if (gtid == 0) {
      if ((L & 63) == 0) gr_check_deadline(ctl, a.status, deadline);
      ctl->qlen[s2] = 0;
      ctl->nchunk[s2] = 0;
      ctl->nbig[s2] = 0;
      ctl->work[s2] = 0;
    }
    __syncthreads();
    const int nch = (int)min((int64_t)s_nch, a.chunk_cap - cb);
    const int nq = le - lb;
    int32_t* onext = a.order + le;
    int2* cnext = a.chunks + cb + nch;
    const int64_t ocap = a.n - le;
    const int64_t ccap = a.chunk_cap - cb - nch;
    const int next_depth = L + 1;
    // claim the target if it has no depth, then add sigma[u] when it is on the
    // next level; all lanes call
    auto visit = [&](bool active, int32_t u, unsigned long long su, int32_t v, int32_t dv) {
      bool won = false;
      if (active) {
        ++cnt.edges;
        if (dv == -1) {
          const int old = atomicCAS(&a.depth[v], -1, next_depth);
          won = old == -1;
          dv = won ? next_depth : old;
        }
        if (dv == next_depth) {
          const unsigned long long old = atomicAdd(&a.sigma[v], su);
          if (su > kSigmaMax - min(old, kSigmaMax)) gr_set_status(a.status, GR_ERR_OVERFLOW);
        }
      }
      int vb = 0, vd = 0;
      if (won) {
        ++cnt.updates;
        vb = __ldg(a.R + v);
        vd = __ldg(a.R + v + 1) - vb;
      }
      stage.append(onext, &ctl->qlen[s1], ocap, won, v, lane);
      if (won && vd >= a.big)
        bstage.add(cnext, ccap, &ctl->nchunk[s1], &ctl->nbig[s1], v, vb, vd, a.status);
    };
    // short rows, 32 per warp batch (rows of the split degree or more are left
    // to their chunks)
    for (int base = swarp * 32; base < nq;
         base = gr_next_batch(base, nq, (int)nwarps * 32, &ctl->work[s0], 32, lane)) {
      const int i = base + lane;
      int32_t u = 0;
      int beg = 0, deg = 0;
      unsigned long long su = 0;
      if (i < nq) {
        ++cnt.verts;
        u = __ldcg(a.order + lb + i);
        beg = __ldg(a.R + u);
        deg = __ldg(a.R + u + 1) - beg;
        if (deg >= a.big) deg = 0;
        su = __ldcg(a.sigma + u);
      }
      gr_warp_expand_u<GR_BC_STRIPS>(
          a.R, a.C, deg > 0, u, beg, deg, (uint32_t)lane, lane,
          [&](bool act, int, int32_t v) -> int32_t { return act ? __ldcg(a.depth + v) : 0; },
          [&](bool act, int32_t uu, uint32_t row_lane, int, int32_t v, int32_t dv) {
            const unsigned long long s = __shfl_sync(GR_FULL_MASK, su, (int)row_lane);
            visit(act, uu, s, v, dv);
          });
    }
    // chunks of long rows, dealt out statically
    for (int c = swarp; c < nch; c += (int)nwarps) {
      const int2 ch = __ldcg(a.chunks + cb + c);
      const int e1 = min(ch.y + GR_CHUNK_EDGES, __ldg(a.R + ch.x + 1));
      const unsigned long long su = __ldcg(a.sigma + ch.x);
      if (lane == 0) ++cnt.verts;
      gr_warp_chunk_u<GR_BC_STRIPS>(
          a.C, ch.x, ch.y, e1, 0u, lane,
          [&](bool act, int, int32_t v) -> int32_t { return act ? __ldcg(a.depth + v) : 0; },
          [&](bool act, int32_t uu, uint32_t, int, int32_t v, int32_t dv) {
            visit(act, uu, su, v, dv);
          });
    }
    __syncthreads();
    bstage.prepare();
    stage.reserve(&ctl->qlen[s1]);
    bstage.reserve(&ctl->nchunk[s1], &ctl->nbig[s1]);
    __syncthreads();
    stage.copy_out(onext, ocap);
    bstage.copy_out(cnext, ccap, a.status);
    if (!sc.sync()) return;
    if (threadIdx.x == 0) {
      s_cnt = __ldcg(&ctl->qlen[s1]);
      s_nch = __ldcg(&ctl->nchunk[s1]);
    }
    __syncthreads();
    const int cnt_next = (int)min((int64_t)s_cnt, ocap);
    cb += nch;
    lb = le;
    le += cnt_next;
    if (gtid == 0) {
      a.clvl[L + 1] = cb;
      a.lvl[L + 2] = le;
    }
    if (cnt_next == 0) break;
  }
  // the last forward level (L + 1) is empty; levels 0..L hold vertices
  if (gtid == 0) a.clvl[L + 2] = cb + (int)min((int64_t)s_nch, a.chunk_cap - cb);
  if (!sc.sync()) return;
  const int nlevels = L + 1;

  // ---- backward pass -----------------------------------------------------
  for (int lev = nlevels - 2; lev >= 0; --lev) {
    const int s0 = lev % 3;
    if (gtid == 0) {
      ctl->work[(lev + 2) % 3] = 0;  // the slot the next (shallower) level uses after this one
    }
    const int ob = __ldcg(a.lvl + lev), oe = __ldcg(a.lvl + lev + 1);
    const int c0 = __ldcg(a.clvl + lev), c1 = __ldcg(a.clvl + lev + 1);
    const int nq = oe - ob, nch = c1 - c0;
    const int child = lev + 1;
    auto term = [&](bool act, double su, int32_t v, int32_t dv) -> double {
      if (!act || dv != child) return 0.0;
      ++cnt.edges;
      const double sv = (double)__ldcg(a.sigma + v);
      return su / sv * (1.0 + __ldcg(a.delta + v));
    };
    for (int base = swarp * 32; base < nq;
         base = gr_next_batch(base, nq, (int)nwarps * 32, &ctl->work[s0], 32, lane)) {
      const int i = base + lane;
      int32_t u = 0;
      int beg = 0, deg = 0;
      double su = 0.0;
      bool mine = false;
      if (i < nq) {
        u = __ldcg(a.order + ob + i);
        beg = __ldg(a.R + u);
        deg = __ldg(a.R + u + 1) - beg;
        mine = deg < a.big;          // long rows are summed by their chunks
        if (!mine) deg = 0;
        su = (double)__ldcg(a.sigma + u);
      }
      acc[lane] = 0.0;
      __syncwarp();
      gr_warp_expand_u<GR_BC_STRIPS>(
          a.R, a.C, deg > 0, u, beg, deg, (uint32_t)lane, lane,
          [&](bool act, int, int32_t v) -> int32_t { return act ? __ldcg(a.depth + v) : 0; },
          [&](bool act, int32_t, uint32_t row_lane, int, int32_t v, int32_t dv) {
            const double s = __shfl_sync(GR_FULL_MASK, su, (int)row_lane);
            const double t = term(act, s, v, dv);
            if (t != 0.0) atomicAdd(&acc[row_lane], t);
          });
      __syncwarp();
      if (mine) a.delta[u] = acc[lane];
      __syncwarp();
    }
    for (int c = swarp; c < nch; c += (int)nwarps) {
      const int2 ch = __ldcg(a.chunks + c0 + c);
      const int e1 = min(ch.y + GR_CHUNK_EDGES, __ldg(a.R + ch.x + 1));
      const double su = (double)__ldcg(a.sigma + ch.x);
      double part = 0.0;
      gr_warp_chunk_u<GR_BC_STRIPS>(
          a.C, ch.x, ch.y, e1, 0u, lane,
          [&](bool act, int, int32_t v) -> int32_t { return act ? __ldcg(a.depth + v) : 0; },
          [&](bool act, int32_t, uint32_t, int, int32_t v, int32_t dv) {
            part += term(act, su, v, dv);
          });
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(GR_FULL_MASK, part, o);
      if (lane == 0 && part != 0.0) atomicAdd(&a.delta[ch.x], part);
    }
    if (!sc.sync()) return;
  }

  // ---- accumulate: bc[v] += delta[v] for v != src ---------------------------
  if (a.bc)
    for (int64_t v = gtid; v < a.n; v += gthreads)
      if (v != a.src) a.bc[v] += a.delta[v];
  cnt.flush(ctl);
  if (gtid == 0) ctl->levels = nlevels;
}

std::mutex g_bc_mu;  // lazy allocation of a workspace's BC scratch

gr_status bc_scratch(const gr_graph* g, gr_workspace* ws, GrBcScratch** out) {
  std::lock_guard<std::mutex> lock(g_bc_mu);
  if (ws->bc) {
    *out = ws->bc;
    return GR_OK;
  }
  GrBcScratch* b = new (std::nothrow) GrBcScratch();
  if (!b) return GR_ERR_OOM;
  const size_t n = (size_t)g->n + 2;
  b->n = g->n;
  b->chunk_cap = g->m / GR_CHUNK_EDGES + g->m / 32 + 2;
  bool ok = cudaMalloc((void**)&b->depth, n * sizeof(int32_t)) == cudaSuccess &&
            cudaMalloc((void**)&b->sigma, n * sizeof(unsigned long long)) == cudaSuccess &&
            cudaMalloc((void**)&b->delta, n * sizeof(double)) == cudaSuccess &&
            cudaMalloc((void**)&b->order, n * sizeof(int32_t)) == cudaSuccess &&
            cudaMalloc((void**)&b->lvl, (n + 2) * sizeof(int32_t)) == cudaSuccess &&
            cudaMalloc((void**)&b->clvl, (n + 2) * sizeof(int32_t)) == cudaSuccess &&
            cudaMalloc((void**)&b->chunks, (size_t)b->chunk_cap * sizeof(int2)) == cudaSuccess;
  if (!ok) {
    (void)cudaGetLastError();
    gr_bc_free(b);
    return GR_ERR_OOM;
  }
  ws->bc = b;
  *out = b;
  return GR_OK;
}

}  // namespace

extern "C" void gr_bc_opts_default(gr_bc_opts* o) {
  if (!o) return;
  o->big_degree = GR_DEFAULT_BFS_BIG;
  o->blocks_per_sm = 0;
  o->spin_limit = GR_DEFAULT_SPIN_LIMIT;
  o->ws = nullptr;
}

extern "C" gr_status gr_bc(const gr_graph* g, int32_t src, int32_t* depth, int64_t* sigma,
                           double* delta, double* bc, const gr_bc_opts* opts, void* stream) {
  if (!g || g->n <= 0 || src < 0 || src >= g->n) return GR_ERR_INVALID_ARG;
  gr_bc_opts o;
  gr_bc_opts_default(&o);
  if (opts) o = *opts;
  gr_workspace* ws = gr_resolve_ws(g, o.ws);
  if (!ws || ws->g != g) return GR_ERR_INVALID_ARG;
  GrBcScratch* s = nullptr;
  gr_status st = bc_scratch(g, ws, &s);
  if (st != GR_OK) return st;
  cudaStream_t cs = (cudaStream_t)stream;

  BcArgs a = {};
  a.n = g->n;
  a.R = g->R;
  a.C = g->C;
  a.depth = depth ? depth : s->depth;
  a.sigma = sigma ? (unsigned long long*)sigma : s->sigma;
  a.delta = delta ? delta : s->delta;
  a.bc = bc;
  a.order = s->order;
  a.lvl = s->lvl;
  a.clvl = s->clvl;
  a.chunks = s->chunks;
  a.chunk_cap = s->chunk_cap;
  a.ctl = ws->ctl;
  a.status = ws->status;
  a.src = src;
  a.big = o.big_degree > 0 ? (o.big_degree < 32 ? 32 : o.big_degree) : GR_DEFAULT_BFS_BIG;
  a.spin = o.spin_limit ? o.spin_limit : GR_DEFAULT_SPIN_LIMIT;

  int blocks = gr_launch_blocks((const void*)bc_persistent, NT, 0, g->num_sms, o.blocks_per_sm);
  if (blocks <= 0) return GR_ERR_CUDA;
  if (gr_reset_ctl(ws, cs) != cudaSuccess) return GR_ERR_CUDA;
  void* args[] = {&a};
  if (cudaLaunchCooperativeKernel((const void*)bc_persistent, dim3(blocks), dim3(NT), args, 0,
                                  cs) != cudaSuccess) {
    (void)cudaGetLastError();
    return GR_ERR_CUDA;
  }
  return GR_OK;
}
