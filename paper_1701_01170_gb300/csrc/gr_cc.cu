// gr_cc.cu — connected-component labelling as one persistent, cooperative
// kernel (Sec. 6.4: hooking with a filter on an edge frontier, then pointer
// jumping, repeated until no edge joins two labels).
//
// Labels start as comp[v] = v and only ever decrease, always to the id of a
// vertex of the same component:
//   * hook: for every edge (u, v) of the frontier whose end points carry
//     different labels cu != cv, comp[max(cu, cv)] takes min(cu, cv) through
//     an atomic minimum; the filter keeps exactly those edges for the next
//     iteration and drops edges whose end points already agree;
//   * pointer jumping: every vertex follows comp[] to the vertex that points
//     to itself and takes its label (comp[x] <= x along the way, so the walk
//     ends).
// The first iteration reads the CSR itself (each undirected edge once, as
// (u, v) with u < v; rows of at least the split degree as grid-shared
// chunks), later ones the surviving (u, v) pairs.  When no edge survives,
// every component carries one label, and since the smallest vertex id of a
// component can never be lowered (no smaller id is reachable from it), that
// label is the component's smallest vertex id — a canonical answer.
//
// Survivors are written through warp-private blocks of GR_CC_BLOCK slots
// (one global atomic per block instead of one per warp and strip); a block's
// unused tail is filled with (-1, -1) entries, which the next iteration skips.
#include <climits>
#include <mutex>
#include <new>

#include "gr_internal.cuh"

#define GR_CC_BLOCK 256
#define GR_CC_JUMP 32   // label steps a vertex follows per pointer-jumping round

struct GrCcScratch {
  int2* edges[2];    // surviving edges (ping-pong)
  int64_t edge_cap;
  int2* chunks;      // chunks of the long rows (first iteration)
  int64_t chunk_cap;
};

void gr_cc_free(GrCcScratch* c) {
  if (!c) return;
  void* ptrs[] = {c->edges[0], c->edges[1], c->chunks};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete c;
}

namespace {

constexpr int NT = GR_PERSIST_THREADS;
constexpr int WPC = NT / 32;
#ifndef GR_CC_STRIPS
#define GR_CC_STRIPS 4
#endif

struct CcArgs {
  int32_t n;
  const int32_t* __restrict__ R;
  const int32_t* __restrict__ C;
  int32_t* comp;
  int32_t* ncomp;      // device, or NULL
  int2* edges[2];
  int64_t edge_cap;
  int2* chunks;
  int64_t chunk_cap;
  GrCtl* ctl;
  int* status;
  int big;
  unsigned spin;
};

// Warp-private output blocks: a warp appends the pairs its lanes keep into a
// block of GR_CC_BLOCK slots reserved with one atomic, takes a new block when
// the current one cannot hold the next strip, and pads the unused tail of a
// block with (-1, -1).  All 32 lanes call every member.
struct WarpBlockOut {
  int2* out;
  int64_t cap;
  int* counter;   // slots reserved so far (global)
  int* status;
  int base = -1;  // first slot of the current block (-1: none yet)
  int used = 0;
  __device__ __forceinline__ void pad(int lane) {
    if (base < 0) return;
    for (int k = used + lane; k < GR_CC_BLOCK; k += 32)
      if ((int64_t)base + k < cap) out[base + k] = make_int2(-1, -1);
  }
  __device__ __forceinline__ void append(bool take, int2 e, int lane) {
    const unsigned mask = __ballot_sync(GR_FULL_MASK, take);
    if (!mask) return;
    const int cntk = __popc(mask);
    if (base < 0 || used + cntk > GR_CC_BLOCK) {
      pad(lane);
      int b = 0;
      if (lane == 0) b = atomicAdd(counter, GR_CC_BLOCK);
      base = __shfl_sync(GR_FULL_MASK, b, 0);
      used = 0;
    }
    if (take) {
      const int64_t pos = (int64_t)base + used + __popc(mask & ((1u << lane) - 1u));
      if (pos < cap) out[pos] = e;
      else gr_set_status(status, GR_ERR_CAPACITY);
    }
    used += cntk;
  }
};

__global__ void __launch_bounds__(NT, 2) cc_persistent(CcArgs a) {
  GridScope sc{a.ctl, a.status, a.spin, (int64_t)blockIdx.x * NT + threadIdx.x,
               (int64_t)gridDim.x * NT, 0u};
  __shared__ GrArena ar;
  const int lane = threadIdx.x & 31;
  const int64_t gtid = sc.tid, gthreads = sc.nthreads;
  const int64_t gwarp = gtid >> 5, nwarps = gthreads >> 5;
  const int swarp = (int)((gwarp % WPC) * (nwarps / WPC) + gwarp / WPC);
  GrCtl* ctl = a.ctl;
  GrCounters cnt;

  for (int64_t v = gtid; v < a.n; v += gthreads) a.comp[v] = (int32_t)v;
  if (!sc.sync()) return;
  const unsigned long long deadline = gr_globaltimer() + GR_TIME_LIMIT_NS;

  // hook one edge; returns whether the filter keeps it
  auto hook = [&](bool active, int32_t u, int32_t v) -> bool {
    if (!active) return false;
    ++cnt.edges;
    const int32_t cu = __ldcg(a.comp + u), cv = __ldcg(a.comp + v);
    if (cu == cv) return false;
    ++cnt.updates;
    atomicMin(&a.comp[max(cu, cv)], min(cu, cv));
    return true;
  };
  // Pointer jumping, in rounds: every vertex follows its labels for up to
  // GR_CC_JUMP steps and keeps the label it reached; a round in which some
  // vertex stopped short of a vertex that labels itself is followed by
  // another (roots do not change while jumping, so the rounds end).  The
  // decision is taken from a flag in one of three rotating slots, set during
  // the round and read by every CTA after the round's barrier.
  __shared__ int s_more;
  unsigned jr = 0;  // jumping rounds so far (selects the flag slot)
  auto jump = [&]() -> bool {
    for (;; ++jr) {
      int* flag = &ctl->workb[jr % 3];
      if (gtid == 0) ctl->workb[(jr + 1) % 3] = 0;
      if (threadIdx.x == 0) s_more = 0;
      __syncthreads();
      int more = 0;
      for (int64_t v = gtid; v < a.n; v += gthreads) {
        const int32_t c0 = __ldcg(a.comp + v);
        int32_t c = c0;
        int steps = 0;
        for (; steps < GR_CC_JUMP; ++steps) {
          const int32_t cc = __ldcg(a.comp + c);
          if (cc == c) break;
          c = cc;
        }
        if (c != c0) a.comp[v] = c;
        more |= steps == GR_CC_JUMP;
      }
      if (__any_sync(GR_FULL_MASK, more) && lane == 0) s_more = 1;
      __syncthreads();
      if (threadIdx.x == 0 && s_more) atomicOr(flag, 1);
      if (!sc.sync()) return false;
      const bool again = __ldcg(flag) != 0;
      if (!again) {
        ++jr;
        return true;
      }
    }
  };

  // ---- iteration 0: the CSR edges (u, v) with u < v -----------------------
  __shared__ int s_bcnt, s_btot[2];
  GrBigStage bstage{ar.bv, ar.bb, ar.bd, ar.bo, &s_bcnt, s_btot};
  WarpBlockOut wout{a.edges[0], a.edge_cap, &ctl->qlen[0], a.status};
  if (threadIdx.x == 0) bstage.reset();
  __syncthreads();
  {
    auto pre = [&](bool, int, int32_t) -> int { return 0; };
    auto edge = [&](bool act, int32_t u, uint32_t, int, int32_t v, int) {
      const bool keep = hook(act && v > u, u, v);
      wout.append(keep, make_int2(u, v), lane);
    };
    const int nbatch = (int)(((int64_t)a.n + 31) / 32);
    for (int b = swarp; b < nbatch; b = gr_next_batch(b, nbatch, (int)nwarps, &ctl->work[0], 1, lane)) {
      const int64_t u64 = (int64_t)b * 32 + lane;
      const bool ok = u64 < a.n;
      const int32_t u = ok ? (int32_t)u64 : 0;
      int beg = 0, deg = 0;
      if (ok) {
        ++cnt.verts;
        beg = __ldg(a.R + u);
        deg = __ldg(a.R + u + 1) - beg;
      }
      if (ok && deg >= a.big) {
        bstage.add(a.chunks, a.chunk_cap, &ctl->nchunk[0], &ctl->nbig[0], u, beg, deg, a.status);
        deg = 0;
      }
      gr_warp_expand_u<GR_CC_STRIPS>(a.R, a.C, deg > 0, u, beg, deg, 0u, lane, pre, edge);
    }
    bstage.flush(a.chunks, a.chunk_cap, &ctl->nchunk[0], &ctl->nbig[0], a.status);
    if (!sc.sync()) return;
    const int nch = (int)min((int64_t)__ldcg(&ctl->nchunk[0]), a.chunk_cap);
    auto no_payload = [](int32_t) -> uint32_t { return 0u; };
    gr_chunks_loop<GR_CC_STRIPS>(a.chunks, nch, swarp, (int)nwarps, lane, a.R, a.C, cnt,
                                 no_payload, pre, edge);
    wout.pad(lane);
  }
  if (!sc.sync()) return;
  if (!jump()) return;

  // ---- later iterations: the surviving edges --------------------------------
  int it = 1;
  for (;; ++it) {
    const int s0 = (it - 1) % 3, s1 = it % 3, s2 = (it + 1) % 3;
    const int64_t len = min((int64_t)__ldcg(&ctl->qlen[s0]), a.edge_cap);
    if (len == 0 || it > a.n + 1) break;
    if (gtid == 0) {
      if ((it & 63) == 0) gr_check_deadline(ctl, a.status, deadline);
      ctl->qlen[s2] = 0;
    }
    const int2* in = a.edges[(it - 1) & 1];
    WarpBlockOut out{a.edges[it & 1], a.edge_cap, &ctl->qlen[s1], a.status};
    for (int64_t base = gwarp * 32 * GR_CC_STRIPS; base < len;
         base += nwarps * 32 * GR_CC_STRIPS) {
      int2 e[GR_CC_STRIPS];
#pragma unroll
      for (int k = 0; k < GR_CC_STRIPS; ++k) {
        const int64_t i = base + k * 32 + lane;
        e[k] = i < len ? __ldcs(in + i) : make_int2(-1, -1);
      }
#pragma unroll
      for (int k = 0; k < GR_CC_STRIPS; ++k) {
        const bool keep = hook(e[k].x >= 0, e[k].x, e[k].y);
        out.append(keep, e[k], lane);
      }
    }
    out.pad(lane);
    if (!sc.sync()) return;
    if (!jump()) return;
  }

  // ---- the number of components: vertices that label themselves ------------
  if (a.ncomp) {
    __shared__ int s_roots;
    if (threadIdx.x == 0) s_roots = 0;
    __syncthreads();
    int mine = 0;
    for (int64_t v = gtid; v < a.n; v += gthreads) mine += __ldcg(a.comp + v) == (int32_t)v;
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(GR_FULL_MASK, mine, o);
    if (lane == 0 && mine) atomicAdd(&s_roots, mine);
    __syncthreads();
    if (threadIdx.x == 0 && s_roots) atomicAdd(a.ncomp, s_roots);
  }
  cnt.flush(ctl);
  if (gtid == 0) ctl->levels = it;
}

std::mutex g_cc_mu;  // lazy allocation of a workspace's CC scratch

gr_status cc_scratch(const gr_graph* g, gr_workspace* ws, int blocks, GrCcScratch** out) {
  std::lock_guard<std::mutex> lock(g_cc_mu);
  const int64_t nwarps = (int64_t)blocks * WPC;
  // every edge once (u < v), plus one partly used block per warp
  const int64_t need = g->m / 2 + 1 + (nwarps + 1) * GR_CC_BLOCK;
  if (ws->cc && ws->cc->edge_cap >= need) {
    *out = ws->cc;
    return GR_OK;
  }
  gr_cc_free(ws->cc);
  ws->cc = nullptr;
  GrCcScratch* c = new (std::nothrow) GrCcScratch();
  if (!c) return GR_ERR_OOM;
  c->edge_cap = need;
  c->chunk_cap = g->m / GR_CHUNK_EDGES + g->m / 32 + 2;
  bool ok = cudaMalloc((void**)&c->edges[0], (size_t)need * sizeof(int2)) == cudaSuccess &&
            cudaMalloc((void**)&c->edges[1], (size_t)need * sizeof(int2)) == cudaSuccess &&
            cudaMalloc((void**)&c->chunks, (size_t)c->chunk_cap * sizeof(int2)) == cudaSuccess;
  if (!ok) {
    (void)cudaGetLastError();
    gr_cc_free(c);
    return GR_ERR_OOM;
  }
  ws->cc = c;
  *out = c;
  return GR_OK;
}

}  // namespace

extern "C" void gr_cc_opts_default(gr_cc_opts* o) {
  if (!o) return;
  o->big_degree = 1024;
  o->blocks_per_sm = 0;
  o->spin_limit = GR_DEFAULT_SPIN_LIMIT;
  o->ws = nullptr;
}

extern "C" gr_status gr_cc(const gr_graph* g, int32_t* comp, int32_t* num_components,
                           const gr_cc_opts* opts, void* stream) {
  if (!g || !comp || g->n <= 0) return GR_ERR_INVALID_ARG;
  if (!(g->flags & GR_SYMMETRIC)) return GR_ERR_UNSUPPORTED;
  gr_cc_opts o;
  gr_cc_opts_default(&o);
  if (opts) o = *opts;
  gr_workspace* ws = gr_resolve_ws(g, o.ws);
  if (!ws || ws->g != g) return GR_ERR_INVALID_ARG;
  int blocks = gr_launch_blocks((const void*)cc_persistent, NT, 0, g->num_sms, o.blocks_per_sm);
  if (blocks <= 0) return GR_ERR_CUDA;
  GrCcScratch* s = nullptr;
  gr_status st = cc_scratch(g, ws, blocks, &s);
  if (st != GR_OK) return st;
  cudaStream_t cs = (cudaStream_t)stream;

  CcArgs a = {};
  a.n = g->n;
  a.R = g->R;
  a.C = g->C;
  a.comp = comp;
  a.ncomp = num_components;
  a.edges[0] = s->edges[0];
  a.edges[1] = s->edges[1];
  a.edge_cap = s->edge_cap;
  a.chunks = s->chunks;
  a.chunk_cap = s->chunk_cap;
  a.ctl = ws->ctl;
  a.status = ws->status;
  a.big = o.big_degree > 0 ? (o.big_degree < 32 ? 32 : o.big_degree) : 1024;
  a.spin = o.spin_limit ? o.spin_limit : GR_DEFAULT_SPIN_LIMIT;

  if (gr_reset_ctl(ws, cs) != cudaSuccess) return GR_ERR_CUDA;
  if (num_components && cudaMemsetAsync(num_components, 0, sizeof(int32_t), cs) != cudaSuccess) {
    (void)cudaGetLastError();
    return GR_ERR_CUDA;
  }
  void* args[] = {&a};
  if (cudaLaunchCooperativeKernel((const void*)cc_persistent, dim3(blocks), dim3(NT), args, 0,
                                  cs) != cudaSuccess) {
    (void)cudaGetLastError();
    return GR_ERR_CUDA;
  }
  return GR_OK;
}
