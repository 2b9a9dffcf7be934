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

#include "gr_internal.cuh"

namespace {

struct SsspArgs {
  int32_t n;
  const int32_t* __restrict__ R;
  const int32_t* __restrict__ C;
  const uint32_t* __restrict__ W;
  unsigned long long* key;
  uint32_t* dist;
  int32_t* pred;
  int32_t* q[2];
  int2* ch[2];
  int64_t chunk_cap;
  int32_t* far[2];
  int32_t* stamp_near;
  int32_t* stamp_far;
  GrCtl* ctl;
  int* status;
  int32_t src;
  uint32_t delta;
  int big;
  int track_deg;
  unsigned spin;
};

constexpr int NT = GR_PERSIST_THREADS;
constexpr unsigned long long KEY_INF = ~0ull;

__global__ void __launch_bounds__(NT) sssp_persistent(SsspArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t gtid = (int64_t)blockIdx.x * NT + threadIdx.x;
  const int64_t gthreads = (int64_t)gridDim.x * NT;
  const int64_t gwarp = gtid >> 5, nwarps = gthreads >> 5;
  GrCtl* ctl = a.ctl;

  // ---- Set_Problem_Data (Alg. 1): labels infinite, preds -1, root 0 -----
  for (int64_t v = gtid; v < a.n; v += gthreads) {
    a.key[v] = v == a.src ? 0xffffffffull : KEY_INF;
    a.stamp_near[v] = v == a.src ? 0 : -1;
    a.stamp_far[v] = -1;
  }
  if (gtid == 0) {
    const int beg = a.R[a.src], deg = a.R[a.src + 1] - beg;
    if (a.track_deg && deg >= a.big)
      gr_register_chunks(a.ch[0], a.chunk_cap, &ctl->nchunk[0], &ctl->nbig[0], a.src, beg, deg,
                         a.status);
    else {
      a.q[0][0] = a.src;
      ctl->qlen[0] = 1;
    }
    for (int k = 0; k < 3; ++k) ctl->farmin[k] = UINT_MAX;
  }
  if (!gr_grid_sync(ctl, a.status, a.spin)) return;

  const unsigned long long deadline = gr_globaltimer() + GR_TIME_LIMIT_NS;
  unsigned long long T = a.delta;  // near iff dist < T
  int fe = 0;                      // far-pile epoch
  int it = 0;                      // near step
  GrCounters cnt;
  bool ovf_seen = false;
  for (;; ++it) {
    const int s0 = it % 3, s1 = (it + 1) % 3, s2 = (it + 2) % 3;
    const int nq = min(__ldcg(&ctl->qlen[s0]), a.n);
    const int nch = (int)min((int64_t)__ldcg(&ctl->nchunk[s0]), a.chunk_cap);
    const int fs = fe % 3;
    const int flen = min(__ldcg(&ctl->farlen[fs]), a.n);
    if (nq + nch == 0 && flen == 0) break;
    if (gtid == 0) {
      gr_check_deadline(ctl, a.status, deadline);
      ctl->qlen[s2] = 0;
      ctl->nchunk[s2] = 0;
      ctl->nbig[s2] = 0;
    }
    int32_t* qn = a.q[(it + 1) & 1];
    int2* chn = a.ch[(it + 1) & 1];
    const int next_stamp = it + 1;

    // join the next near frontier (once per step) — all lanes call this
    auto to_near = [&](bool take, int32_t v) {
      if (take) take = atomicExch(&a.stamp_near[v], next_stamp) != next_stamp;
      int vbeg = 0, vdeg = 0;
      if (take && a.track_deg) {
        vbeg = __ldg(a.R + v);
        vdeg = __ldg(a.R + v + 1) - vbeg;
      }
      const bool big = take && vdeg >= a.big;
      gr_warp_append(qn, &ctl->qlen[s1], a.n, take && !big, v, lane);
      if (big)
        gr_register_chunks(chn, a.chunk_cap, &ctl->nchunk[s1], &ctl->nbig[s1], v, vbeg, vdeg,
                           a.status);
    };
    // join far pile `epoch` (once per epoch) — all lanes call this
    auto to_far = [&](bool take, int32_t v, unsigned d, int epoch) {
      if (take) take = atomicExch(&a.stamp_far[v], epoch) != epoch;
      gr_warp_append(a.far[epoch & 1], &ctl->farlen[epoch % 3], a.n, take, v, lane);
      const unsigned mn = gr_warp_min_u32(take ? d : UINT_MAX);
      if (lane == 0 && mn != UINT_MAX) atomicMin(&ctl->farmin[epoch % 3], mn);
    };

    if (nq + nch > 0) {
      // ---- RELAX: advance + Update_Label / Set_Pred + Remove_Redundant ----
      const int32_t* q = a.q[it & 1];
      const int2* ch = a.ch[it & 1];
      auto relax = [&](bool active, int32_t u, uint32_t du, int e, int32_t v) {
        bool imp = false;
        unsigned long long nd = 0;
        if (active) {
          ++cnt.edges;
          nd = (unsigned long long)du + __ldg(a.W + e);
          if (nd >= (unsigned long long)GR_INF_DIST) {
            // not representable: drop the candidate; whether a true distance
            // overflows is decided after convergence
            if (!ovf_seen) {
              ovf_seen = true;
              atomicExch(&ctl->ovf_pending, 1);
            }
          } else {
            const unsigned long long cand = (nd << 32) | (unsigned)u;
            if (cand < a.key[v]) imp = (atomicMin(&a.key[v], cand) >> 32) > nd;
            cnt.updates += imp;
          }
        }
        to_near(imp && nd < T, v);
        to_far(imp && nd >= T, v, (unsigned)nd, fe);
      };
      for (int64_t base = gwarp * 32; base < nq; base += nwarps * 32) {
        const int64_t i = base + lane;
        const bool valid = i < nq;
        int32_t u = 0;
        int beg = 0, deg = 0;
        uint32_t du = 0;
        if (valid) {
          ++cnt.verts;
          u = __ldcg(q + i);
          beg = __ldg(a.R + u);
          deg = __ldg(a.R + u + 1) - beg;
          du = (uint32_t)(a.key[u] >> 32);
        }
        gr_warp_expand(a.R, a.C, valid, u, beg, deg, du, lane, relax);
      }
      for (int64_t c = gwarp; c < nch; c += nwarps) {
        const int2 cu = __ldcg(ch + c);
        const int e1 = min(cu.y + GR_CHUNK_EDGES, __ldg(a.R + cu.x + 1));
        const uint32_t du = (uint32_t)(a.key[cu.x] >> 32);
        if (lane == 0) ++cnt.verts;
        gr_warp_chunk(a.C, cu.x, cu.y, e1, du, lane, relax);
      }
    } else {
      // ---- SPLIT: raise the threshold, move far entries below it to near --
      const unsigned fm = __ldcg(&ctl->farmin[fs]);
      unsigned long long Tn = T + a.delta;
      if (fm != UINT_MAX) {
        const unsigned long long jump = ((unsigned long long)fm / a.delta + 1ull) * a.delta;
        if (jump > Tn) Tn = jump;
      }
      if (gtid == 0) {
        ctl->farlen[(fe + 2) % 3] = 0;
        ctl->farmin[(fe + 2) % 3] = UINT_MAX;
      }
      const int32_t* fp = a.far[fe & 1];
      for (int64_t base = gwarp * 32; base < flen; base += nwarps * 32) {
        const int64_t i = base + lane;
        int32_t v = 0;
        unsigned long long d = 0;
        const bool valid = i < flen;
        if (valid) {
          ++cnt.verts;
          v = __ldcg(fp + i);
          d = a.key[v] >> 32;
        }
        to_near(valid && d >= T && d < Tn, v);
        to_far(valid && d >= Tn, v, (unsigned)d, fe + 1);
      }
      T = Tn;
      ++fe;
    }
    if (!gr_grid_sync(ctl, a.status, a.spin)) return;
  }
  // ---- overflow check: with every unrepresentable candidate dropped, a
  // vertex keeps an infinite label while a reached neighbour exists only if
  // its true distance is >= UINT32_MAX.
  if (__ldcg(&ctl->ovf_pending)) {
    for (int64_t u = gtid; u < a.n; u += gthreads) {
      if ((a.key[u] >> 32) == GR_INF_DIST) continue;
      for (int e = __ldg(a.R + u); e < __ldg(a.R + u + 1); ++e)
        if (a.key[__ldg(a.C + e)] == KEY_INF) {
          gr_set_status(a.status, GR_ERR_OVERFLOW);
          break;
        }
    }
  }
  // ---- unpack labels and predecessors -----------------------------------
  for (int64_t v = gtid; v < a.n; v += gthreads) {
    const unsigned long long k = a.key[v];
    a.dist[v] = (uint32_t)(k >> 32);
    if (a.pred) a.pred[v] = (int32_t)(uint32_t)(k & 0xffffffffull);
  }
  cnt.flush(ctl);
  if (gtid == 0) ctl->levels = it;
}

}  // namespace

extern "C" void gr_sssp_opts_default(gr_sssp_opts* o) {
  if (!o) return;
  o->delta = 0;
  o->big_degree = GR_DEFAULT_BIG_DEGREE;
  o->blocks_per_sm = 0;
  o->spin_limit = GR_DEFAULT_SPIN_LIMIT;
  o->ws = nullptr;
}

// Bucket width from the graph: about one warp's worth of average edges
// (warp size * mean weight / mean degree), at least 1.
static uint32_t default_delta(const gr_graph* g) {
  if (g->m == 0 || g->nonisolated == 0) return 1;
  double wmean = (double)g->weight_sum / (double)g->m;
  double dmean = (double)g->m / (double)g->nonisolated;
  double d = 32.0 * wmean / dmean;
  if (d < 1.0) d = 1.0;
  if (d > 1e9) d = 1e9;
  return (uint32_t)d;
}

extern "C" gr_status gr_sssp(const gr_graph* g, int32_t src, uint32_t* dist, int32_t* pred,
                             const gr_sssp_opts* opts, void* stream) {
  if (!g || !dist || g->n <= 0 || src < 0 || src >= g->n) return GR_ERR_INVALID_ARG;
  if (!g->W && g->m > 0) return GR_ERR_UNSUPPORTED;
  gr_sssp_opts o;
  gr_sssp_opts_default(&o);
  if (opts) o = *opts;
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
  a.ch[0] = ws->chunks[0];
  a.ch[1] = ws->chunks[1];
  a.chunk_cap = ws->chunk_cap;
  a.far[0] = ws->far[0];
  a.far[1] = ws->far[1];
  a.stamp_near = ws->stamp_near;
  a.stamp_far = ws->stamp_far;
  a.ctl = ws->ctl;
  a.status = ws->status;
  a.src = src;
  a.delta = o.delta ? o.delta : default_delta(g);
  a.big = o.big_degree > 0 ? (o.big_degree < 32 ? 32 : o.big_degree) : GR_DEFAULT_BIG_DEGREE;
  a.track_deg = g->max_degree >= a.big;
  a.spin = o.spin_limit ? o.spin_limit : GR_DEFAULT_SPIN_LIMIT;

  const int blocks = gr_launch_blocks((const void*)sssp_persistent, NT, 0, g->num_sms,
                                      o.blocks_per_sm);
  if (blocks <= 0) return GR_ERR_CUDA;
  if (gr_reset_ctl(ws, s) != cudaSuccess) return GR_ERR_CUDA;
  void* args[] = {&a};
  if (cudaLaunchCooperativeKernel((const void*)sssp_persistent, dim3(blocks), dim3(NT), args, 0,
                                  s) != cudaSuccess) {
    (void)cudaGetLastError();
    return GR_ERR_CUDA;
  }
  return GR_OK;
}
