// gr_sssp_body.cuh — one SSSP query (init, near/far steps, overflow check,
// unpack) as a device function templated on the scope of threads that run
// it; shared by the cooperative single-query kernel (gr_sssp.cu) and the
// batched many-graph kernel (gr_batch.cu).  See gr_sssp.cu for the method.
#pragma once

#include <climits>

#include "gr_internal.cuh"

#ifndef GR_RELAX_STRIPS
#define GR_RELAX_STRIPS 4  // 32-edge strips a warp relaxes per round
#endif
#ifndef GR_BULK_STRIPS
#define GR_BULK_STRIPS 8   // 32-edge strips a warp relaxes per round in bulk steps
#endif

#ifndef GR_COLLECT_WORDS
#define GR_COLLECT_WORDS 4  // non-empty bitmap words a warp collects per round
#endif
// Bulk steps (fire-and-forget atomics and a label-change bitmap, then one
// pass over the bitmap builds the next piles) pay one extra barrier and a
// pass over n bits, so by default they start at n / GR_BULK_DIVISOR near rows
// (a chunk counting as 8), and at GR_BULK_MIN_ROWS at least.
#define GR_BULK_DIVISOR 64
#define GR_BULK_MIN_ROWS 4096
__host__ __device__ inline int32_t gr_default_bulk_rows(int64_t n) {
  const int64_t r = n / GR_BULK_DIVISOR;
  return (int32_t)(r > GR_BULK_MIN_ROWS ? r : GR_BULK_MIN_ROWS);
}
// On a graph with rows of GR_SKEWED_DEGREE or more edges (scale-free degree
// distributions) the default is far lower, GR_SKEWED_BULK_ROWS: a step of a
// few rows can hold a hub's hundred thousand edges, which the per-edge path
// relaxes with returning atomics one strip after another, and the pass over
// n bits is cheap beside it.  R-MAT s22 (hub and 20 random sources): mean
// SSSP 2.04 ms at 64 rows against 2.16 ms at n / 64, and 2.10 / 2.13 ms at
// 1024 / 8192 rows; the 4096^2 grid keeps n / 64 (84 ms per query against
// 126-144 ms at 16-4096 rows).
#define GR_SKEWED_DEGREE 1024
#define GR_SKEWED_BULK_ROWS 64

struct SsspArgs {
  int32_t n;
  const int32_t* __restrict__ R;
  const int32_t* __restrict__ C;
  const uint32_t* __restrict__ W;
  unsigned long long* key;
  uint32_t* dist;
  int32_t* pred;
  int32_t* q[2];
  int32_t* qm[2];     // medium-row queues (NULL: medium rows go to q)
  int2* ch[2];
  int64_t chunk_cap;
  int32_t* far[2];
  int32_t* stamp_near;
  int32_t* stamp_far;
  uint32_t* touched;  // n-bit label-change bitmap of bulk steps (NULL: no bulk steps)
  int32_t bulk_rows;  // near rows (a chunk counts as 8) from which a step runs in bulk
  GrCtl* ctl;
  int* status;
  int32_t src;
  uint32_t delta;
  int big;
  int track_deg;
  unsigned spin;
  int32_t* level_stats;
  int32_t max_levels;
  // Multi-level priority queue (NULL: the two-level near/far queue): ring[j]
  // holds the vertices of bucket b = dist / delta with b % GR_RING_K == j for
  // the GR_RING_K - 1 buckets after the current one; stamp_ring[v] is the last
  // bucket v was added to.  Needs the large staging buffers.
  int32_t* ring[GR_RING_K];
  uint32_t* stamp_ring;
};

constexpr unsigned long long GR_KEY_INF = ~0ull;

// STAGED selects the staged per-edge RELAX (atomics and dependent loads of all
// strips of a round in flight together): 11 % faster on the 4096^2 grid,
// whose small steps all take that path, but 3 % slower on R-MAT s22 through
// the register allocation of its bulk steps, so only the mesh instantiation
// uses it.
template <bool STAGED, class S>
__device__ __forceinline__ void gr_sssp_body(const SsspArgs& a, S& sc, GrArena& ar,
                                             GrStageBufs* big = nullptr) {
  const int lane = threadIdx.x & 31;
  const int64_t gtid = sc.tid;
  const int64_t gthreads = sc.nthreads;
  const int64_t gwarp = gtid >> 5, nwarps = gthreads >> 5;
  // Static-first batches are dealt out across CTAs: batch k of a step goes to
  // CTA k mod (number of CTAs), so a small step spreads over every SM instead
  // of filling the first CTAs (and their staging buffers) alone.
  const int wpc = (int)(blockDim.x >> 5);
  const int swarp = (int)((gwarp % wpc) * (nwarps / wpc) + gwarp / wpc);
  GrCtl* ctl = a.ctl;
  const unsigned long long t_entry = gr_globaltimer();  // time base of level_stats

  // ---- Set_Problem_Data (Alg. 1): labels infinite, preds -1, root 0 -----
  for (int64_t v = gtid; v < a.n; v += gthreads) {
    a.key[v] = v == a.src ? 0xffffffffull : GR_KEY_INF;
    a.stamp_near[v] = v == a.src ? 0 : -1;
    a.stamp_far[v] = -1;
    if (a.stamp_ring) a.stamp_ring[v] = UINT_MAX;
  }
  const int nwords = (int)(((int64_t)a.n + 31) >> 5);
  if (a.touched)
    for (int64_t w = gtid; w < nwords; w += gthreads) a.touched[w] = 0u;
  {
    const int beg = __ldg(a.R + a.src), deg = __ldg(a.R + a.src + 1) - beg;
    if (a.track_deg && deg >= a.big) {
      gr_register_source_chunks(a.ch[0], a.chunk_cap, &ctl->nchunk[0], &ctl->nbig[0], a.src,
                                beg, deg, a.status, gtid, gthreads);
    } else if (gtid == 0) {
      a.q[0][0] = a.src;
      ctl->qlen[0] = 1;
    }
    if (gtid == 0)
      for (int k = 0; k < 3; ++k) ctl->farmin[k] = UINT_MAX;
  }
  if (!sc.sync()) return;

  const unsigned long long deadline = gr_globaltimer() + GR_TIME_LIMIT_NS;
  unsigned long long T = a.delta;  // near iff dist < T
  int fe = 0;                      // far-pile epoch
  // multi-level queue: the current bucket is T / delta - 1; ring_left counts the
  // ring slots known to hold entries, reset_slot is the slot drained by the
  // last SPLIT step (its length is cleared at the start of the next step)
  int ring_left = 0;
  int reset_slot = -1;
  int it = 0;                      // near step
  GrCounters cnt;
  bool ovf_seen = false;
  // step counters are read once per CTA and broadcast through shared memory
  __shared__ int s_nq, s_nqm, s_nch, s_nbig, s_flen;
  __shared__ unsigned s_fm;
  __shared__ int s_ncnt, s_nbase, s_fcnt, s_fbase;
  __shared__ unsigned s_farmin;
  GrStage near_stage{big ? big->near : ar.buf0, &s_ncnt, &s_nbase,
                     big ? GR_BIG_NEAR_CAP : GR_STAGE_CAP};
  __shared__ int s_mcnt, s_mbase;
  GrStage mid_stage{big ? big->mid : ar.bufm, &s_mcnt, &s_mbase,
                    big ? GR_BIG_MID_CAP : GR_STAGE_CAP};
  GrStage far_stage{big ? big->far : ar.buf1, &s_fcnt, &s_fbase,
                    big ? GR_BIG_FAR_CAP : GR_STAGE_CAP};
  __shared__ int s_bcnt, s_btot[2];
  GrBigStage bstage{ar.bv, ar.bb, ar.bd, ar.bo, &s_bcnt, s_btot};
  for (;; ++it) {
    const int s0 = it % 3, s1 = (it + 1) % 3, s2 = (it + 2) % 3;
    const int fs = fe % 3;
    if (threadIdx.x == 0) {
      s_nq = __ldcg(&ctl->qlen[s0]);
      s_nqm = __ldcg(&ctl->qmlen[s0]);
      s_nch = __ldcg(&ctl->nchunk[s0]);
      s_nbig = __ldcg(&ctl->nbig[s0]);
      s_flen = __ldcg(&ctl->farlen[fs]);
      s_fm = __ldcg(&ctl->farmin[fs]);
      near_stage.reset();
      mid_stage.reset();
      far_stage.reset();
      bstage.reset();
      s_farmin = UINT_MAX;
    }
    __syncthreads();
    const int nq = min(s_nq, a.n);
    const int nqm = min(s_nqm, a.n);
    const int nch = (int)min((int64_t)s_nch, a.chunk_cap);
    const int nrows = nq + nqm + nch;  // zero: a SPLIT step
    const int flen = min(s_flen, a.n);
    const unsigned fm_step = s_fm;
    if (nrows == 0 && flen == 0 && ring_left == 0) break;
    if (reset_slot >= 0) {
      if (gtid == 0) ctl->rlen[reset_slot] = 0;
      reset_slot = -1;
    }
    if (gtid == 0) {
      if ((it & 63) == 0) gr_check_deadline(ctl, a.status, deadline);
      if (a.level_stats && it < a.max_levels) {
        a.level_stats[4 * it] = nq + nqm + s_nbig;
        a.level_stats[4 * it + 1] = nrows == 0;
        a.level_stats[4 * it + 2] = flen;
        // start of this step in ns after the kernel started
        a.level_stats[4 * it + 3] =
            (int)min(gr_globaltimer() - t_entry, (unsigned long long)INT_MAX);
      }
      ctl->qlen[s2] = 0;
      ctl->qmlen[s2] = 0;
      ctl->workm[s2] = 0;
      ctl->nchunk[s2] = 0;
      ctl->nbig[s2] = 0;
      ctl->work[s2] = 0;
      ctl->workc[s2] = 0;
      ctl->workb[s2] = 0;
    }
    int32_t* qn = a.q[(it + 1) & 1];
    int32_t* qmn = a.qm[0] ? a.qm[(it + 1) & 1] : nullptr;
    int2* chn = a.ch[(it + 1) & 1];
    const int next_stamp = it + 1;

    // append to the next near frontier — all lanes call this
    // (vbeg, vdeg: the row of v when the caller has loaded it already)
    auto near_append_row = [&](bool take, int32_t v, int vbeg, int vdeg) {
      const bool big = take && vdeg >= a.big;
      const bool mid = take && !big && qmn && vdeg >= GR_MEDIUM_DEGREE;
      near_stage.append(qn, &ctl->qlen[s1], a.n, take && !big && !mid, v, lane);
      mid_stage.append(qmn, &ctl->qmlen[s1], a.n, mid, v, lane);
      if (big)
        bstage.add(chn, a.chunk_cap, &ctl->nchunk[s1], &ctl->nbig[s1], v, vbeg, vdeg, a.status);
    };
    auto near_append = [&](bool take, int32_t v) {
      int vbeg = 0, vdeg = 0;
      if (take && a.track_deg) {
        vbeg = __ldg(a.R + v);
        vdeg = __ldg(a.R + v + 1) - vbeg;
      }
      near_append_row(take, v, vbeg, vdeg);
    };
    // join the next near frontier (once per step) — all lanes call this
    auto to_near = [&](bool take, int32_t v) {
      if (take) take = atomicExch(&a.stamp_near[v], next_stamp) != next_stamp;
      near_append(take, v);
    };
    // join far pile `epoch` (once per epoch) — all lanes call this
    // (a step only ever writes one far pile: epoch fe when relaxing, fe + 1
    // when splitting)
    const int fe_out = nrows > 0 ? fe : fe + 1;
    auto to_far = [&](bool take, int32_t v, unsigned d, int epoch) {
      if (take) take = atomicExch(&a.stamp_far[v], epoch) != epoch;
      far_stage.append(a.far[epoch & 1], &ctl->farlen[epoch % 3], a.n, take, v, lane);
      const unsigned mn = gr_warp_min_u32(take ? d : UINT_MAX);
      if (lane == 0 && mn != UINT_MAX) atomicMin(&s_farmin, mn);
    };

    const bool bulk = a.touched && nq + 4ll * nqm + 8ll * nch >= a.bulk_rows;
    if (bulk) {
      // ---- bulk RELAX: Update_Label / Set_Pred as fire-and-forget 64-bit
      // atomicMin, plus one bit per changed label; no return values and no
      // per-edge queue work.  Labels are read from L2 so that a bit is set
      // only for a label that this step really lowers.
      const int32_t* q = a.q[it & 1];
      const int2* ch = a.ch[it & 1];
      struct PreB {
        uint32_t w;
        unsigned long long cur;
      };
      auto pre = [&](bool active, int e, int32_t v) -> PreB {
        PreB p{0u, 0ull};
        if (active) {
          p.w = GR_LDSTREAM(a.W + e);
          p.cur = __ldcg(a.key + v);
        }
        return p;
      };
      auto relax = [&](bool active, int32_t u, uint32_t du, int, int32_t v, const PreB& p) {
        bool hit = false;
        if (active) {
          ++cnt.edges;
          const unsigned long long nd = (unsigned long long)du + p.w;
          if (nd >= (unsigned long long)GR_INF_DIST) {
            if (!ovf_seen) {
              ovf_seen = true;
              atomicExch(&ctl->ovf_pending, 1);
            }
          } else {
            const unsigned long long cand = (nd << 32) | (unsigned)u;
            if (cand < p.cur) {
              gr_red_min_u64(&a.key[v], cand);
              hit = true;
            }
          }
        }
        if (hit) gr_red_or_u32(a.touched + (v >> 5), 1u << (v & 31));
      };
      // largest work first: chunks, medium rows, then short rows
      auto label = [&](int32_t u) -> uint32_t { return (uint32_t)(__ldcg(a.key + u) >> 32); };
      gr_chunks_loop<GR_BULK_STRIPS>(ch, nch, swarp, (int)nwarps, lane, a.R, a.C,
                                     cnt, label, pre, relax, a.W);
      if (a.qm[0])
        gr_rows_loop<GR_BULK_STRIPS>(a.qm[it & 1], nqm, GR_MEDIUM_BATCH, &ctl->workm[s0], swarp,
                                     (int)nwarps, lane, a.R, a.C, cnt, label, pre, relax);
      gr_rows_loop<GR_BULK_STRIPS>(q, nq, 32, &ctl->work[s0], swarp, (int)nwarps, lane, a.R, a.C,
                                   cnt, label, pre, relax);
      if (!sc.sync()) return;
      // ---- collect: every vertex whose label dropped in this step joins
      // the near frontier (dist < T) or, once per epoch, the far pile.  A
      // warp owns 32 bitmap words at a time and clears them.
      for (int wb = swarp * 32; wb < nwords;
           wb = gr_next_batch(wb, nwords, (int)nwarps * 32, &ctl->workb[s0], 32, lane)) {
        const int w = wb + lane;
        uint32_t word = w < nwords ? __ldcg(a.touched + w) : 0u;
        if (word) a.touched[w] = 0u;
        unsigned nz = __ballot_sync(GR_FULL_MASK, word != 0u);
        // four non-empty words per round: their labels, then the rows of the
        // near ones, are loaded together
        constexpr int KW = GR_COLLECT_WORDS;
        while (nz) {
          bool mine[KW];
          int32_t v[KW];
          unsigned d[KW];
#pragma unroll
          for (int k = 0; k < KW; ++k) {
            const int j = nz ? __ffs(nz) - 1 : -1;
            if (nz) nz &= nz - 1u;
            const uint32_t bits = __shfl_sync(GR_FULL_MASK, word, j < 0 ? 0 : j);
            mine[k] = j >= 0 && ((bits >> lane) & 1u);
            v[k] = (wb + (j < 0 ? 0 : j)) * 32 + lane;
          }
#pragma unroll
          for (int k = 0; k < KW; ++k) {
            d[k] = 0;
            if (mine[k]) {
              ++cnt.updates;
              d[k] = (unsigned)(__ldcg(a.key + v[k]) >> 32);
            }
          }
          int vb[KW], vd[KW];
#pragma unroll
          for (int k = 0; k < KW; ++k) {
            vb[k] = 0;
            vd[k] = 0;
            if (mine[k] && d[k] < T && a.track_deg) {
              vb[k] = __ldg(a.R + v[k]);
              vd[k] = __ldg(a.R + v[k] + 1) - vb[k];
            }
          }
#pragma unroll
          for (int k = 0; k < KW; ++k) {
            near_append_row(mine[k] && d[k] < T, v[k], vb[k], vd[k]);
            bool far = mine[k] && d[k] >= T;
            if (far) {
              far = a.stamp_far[v[k]] != fe;  // this thread owns v in this pass
              if (far) a.stamp_far[v[k]] = fe;
            }
            far_stage.append(a.far[fe & 1], &ctl->farlen[fe % 3], a.n, far, v[k], lane);
            const unsigned mn = gr_warp_min_u32(far ? d[k] : UINT_MAX);
            if (lane == 0 && mn != UINT_MAX) atomicMin(&s_farmin, mn);
          }
        }
      }
    } else if (nrows > 0) {
      // ---- RELAX: advance + Update_Label / Set_Pred + Remove_Redundant ----
      const int32_t* q = a.q[it & 1];
      const int2* ch = a.ch[it & 1];
      if (STAGED) {
        // Stages, each for all strips of a round before the next (every result
        // is examined one stage after its atomic or load was issued, so the
        // strips' round trips overlap):
        //  pre: weight and current key of each edge's target;
        //  tryk: Update_Label / Set_Pred as one 64-bit atomicMin on the key for
        //    candidates below the current key, and the target's row bounds
        //    (used if it joins the near frontier);
        //  stamp: for targets whose label this edge lowered below T, the
        //    near-frontier stamp exchange (joins once per step);
        //  relax: the appends.
        struct Pre {
          uint32_t w;
          uint32_t stamp;           // previous near stamp (when exchanged)
          unsigned long long key;   // current key, then the atomicMin's return value
          int32_t vbeg, vdeg;
          int32_t tried;            // an atomicMin was issued
        };
        auto pre = [&](bool active, int e, int32_t v) -> Pre {
          Pre p{0u, 0u, 0ull, 0, 0, 0};
          if (active) {
            p.w = GR_LDSTREAM(a.W + e);
            p.key = a.key[v];
          }
          return p;
        };
        auto tryk = [&](bool active, int32_t u, uint32_t du, int, int32_t v, Pre& p) {
          if (!active) return;
          ++cnt.edges;
          const unsigned long long nd = (unsigned long long)du + p.w;
          if (nd >= (unsigned long long)GR_INF_DIST) {
            // not representable: drop the candidate; whether a true distance
            // overflows is decided after convergence
            if (!ovf_seen) {
              ovf_seen = true;
              atomicExch(&ctl->ovf_pending, 1);
            }
            return;
          }
          const unsigned long long cand = (nd << 32) | (unsigned)u;
          if (cand < p.key) {
            p.tried = 1;
            p.key = atomicMin(&a.key[v], cand);
            if (nd < T && a.track_deg) {
              p.vbeg = __ldg(a.R + v);
              p.vdeg = __ldg(a.R + v + 1) - p.vbeg;
            }
          }
        };
        auto improved = [&](uint32_t du, const Pre& p) {
          return p.tried && (p.key >> 32) > (unsigned long long)du + p.w;
        };
        auto stamp = [&](bool, int32_t, uint32_t du, int, int32_t v, Pre& p) {
          if (improved(du, p) && (unsigned long long)du + p.w < T)
            p.stamp = (uint32_t)atomicExch(&a.stamp_near[v], next_stamp);
        };
        auto relax = [&](bool, int32_t, uint32_t du, int, int32_t v, const Pre& p) {
          const bool imp = improved(du, p);
          const unsigned long long nd = (unsigned long long)du + p.w;
          cnt.updates += imp;
          near_append_row(imp && nd < T && p.stamp != (uint32_t)next_stamp, v, p.vbeg, p.vdeg);
          to_far(imp && nd >= T, v, (unsigned)nd, fe);
        };
        // largest work first: chunks, medium rows, then short rows 32 at a time
        // (first batch by warp index, further batches from a counter that idle
        // warps never touch)
        auto label = [&](int32_t u) -> uint32_t { return (uint32_t)(a.key[u] >> 32); };
        gr_chunks_loop_mid<GR_RELAX_STRIPS>(ch, nch, swarp, (int)nwarps, lane, a.R, a.C, cnt,
                                            label, pre, tryk, stamp, relax, a.W);
        if (a.qm[0])
          gr_rows_loop_mid<GR_RELAX_STRIPS>(a.qm[it & 1], nqm, GR_MEDIUM_BATCH, &ctl->workm[s0],
                                            swarp, (int)nwarps, lane, a.R, a.C, cnt, label, pre,
                                            tryk, stamp, relax);
        gr_rows_loop_mid<GR_RELAX_STRIPS>(q, nq, 32, &ctl->work[s0], swarp, (int)nwarps, lane,
                                          a.R, a.C, cnt, label, pre, tryk, stamp, relax);
      } else {
        // pass 2: weight and current key of each edge's target
        struct Pre {
          uint32_t w;
          unsigned long long cur;
        };
        auto pre = [&](bool active, int e, int32_t v) -> Pre {
          Pre p{0u, 0ull};
          if (active) {
            p.w = GR_LDSTREAM(a.W + e);
            p.cur = a.key[v];
          }
          return p;
        };
        // pass 3: Update_Label / Set_Pred as one 64-bit atomicMin on the key
        auto relax = [&](bool active, int32_t u, uint32_t du, int, int32_t v, const Pre& p) {
          bool imp = false;
          unsigned long long nd = 0;
          if (active) {
            ++cnt.edges;
            nd = (unsigned long long)du + p.w;
            if (nd >= (unsigned long long)GR_INF_DIST) {
              // not representable: drop the candidate; whether a true distance
              // overflows is decided after convergence
              if (!ovf_seen) {
                ovf_seen = true;
                atomicExch(&ctl->ovf_pending, 1);
              }
            } else {
              const unsigned long long cand = (nd << 32) | (unsigned)u;
              if (cand < p.cur) imp = (atomicMin(&a.key[v], cand) >> 32) > nd;
              cnt.updates += imp;
            }
          }
          to_near(imp && nd < T, v);
          to_far(imp && nd >= T, v, (unsigned)nd, fe);
        };
        // largest work first: chunks, medium rows, then short rows 32 at a time
        // (first batch by warp index, further batches from a counter that idle
        // warps never touch)
        auto label = [&](int32_t u) -> uint32_t { return (uint32_t)(a.key[u] >> 32); };
        gr_chunks_loop<GR_RELAX_STRIPS>(ch, nch, swarp, (int)nwarps, lane, a.R, a.C,
                                        cnt, label, pre, relax, a.W);
        if (a.qm[0])
          gr_rows_loop<GR_RELAX_STRIPS>(a.qm[it & 1], nqm, GR_MEDIUM_BATCH, &ctl->workm[s0], swarp,
                                        (int)nwarps, lane, a.R, a.C, cnt, label, pre, relax);
        gr_rows_loop<GR_RELAX_STRIPS>(q, nq, 32, &ctl->work[s0], swarp, (int)nwarps, lane, a.R, a.C,
                                      cnt, label, pre, relax);
      }
    } else if (a.ring[0] && big) {
      // ---- SPLIT with the multi-level queue (a multisplit of the far pile) --
      // Phase 1: every entry of the far pile (vertices that left the current
      // bucket since the last SPLIT) goes, by its bucket b = dist / delta, to
      // ring slot b % K when b lies in the window (cb, cb + K) — once per
      // bucket, by stamp — or to the next far pile; entries whose distance
      // fell back into an earlier bucket were expanded then and are dropped.
      // Phase 2: the smallest bucket of the window with entries becomes the
      // current one and its slot is drained into the near frontier (stale
      // entries dropped); with an empty window the threshold jumps to the far
      // pile's smallest distance and the next step splits again.
      constexpr int K = GR_RING_K;
      const unsigned long long cb = T / a.delta - 1;
      if (gtid == 0) {
        ctl->farlen[(fe + 2) % 3] = 0;
        ctl->farmin[(fe + 2) % 3] = UINT_MAX;
      }
      __shared__ int s_rcnt[K], s_rbase[K], s_rcur[K];
      __shared__ int s_rn;
      // staging of this CTA's ring entries: vertex ids in the near buffer and
      // their slots as bytes in the middle buffer (both idle in this phase)
      constexpr int RCAP = GR_BIG_NEAR_CAP;
      static_assert(GR_BIG_MID_CAP * 4 >= RCAP, "slot bytes must fit the middle buffer");
      int* rv = big->near;
      unsigned char* rs = (unsigned char*)big->mid;
      if (threadIdx.x < K) {
        s_rcnt[threadIdx.x] = 0;
        s_rcur[threadIdx.x] = 0;
      }
      if (threadIdx.x == 0) s_rn = 0;
      __syncthreads();
      const int32_t* fp = a.far[fe & 1];
      for (int base = swarp * 32; base < flen;
           base = gr_next_batch(base, flen, (int)nwarps * 32, &ctl->work[s0], 32, lane)) {
        const int i = base + lane;
        int32_t v = 0;
        unsigned long long b = 0;
        const bool valid = i < flen;
        if (valid) {
          ++cnt.verts;
          v = __ldcg(fp + i);
          b = (__ldcg(a.key + v) >> 32) / a.delta;
        }
        bool to_ring = valid && b > cb && b < cb + K;
        if (to_ring) to_ring = atomicExch(&a.stamp_ring[v], (uint32_t)b) != (uint32_t)b;
        const unsigned rm = __ballot_sync(GR_FULL_MASK, to_ring);
        if (rm) {
          int pos = 0;
          if (lane == __ffs(rm) - 1) pos = atomicAdd(&s_rn, __popc(rm));
          pos = __shfl_sync(GR_FULL_MASK, pos, __ffs(rm) - 1) + __popc(rm & ((1u << lane) - 1u));
          const int j = (int)(b % K);
          const bool staged = to_ring && pos < RCAP;
          if (staged) {
            rv[pos] = v;
            rs[pos] = (unsigned char)j;
            atomicAdd(&s_rcnt[j], 1);
          }
          // staging full: straight to the ring, one global atomic per warp and slot
          const bool direct = to_ring && !staged;
          if (__any_sync(GR_FULL_MASK, direct)) {
#pragma unroll
            for (int jj = 0; jj < K; ++jj) {
              const unsigned dm = __ballot_sync(GR_FULL_MASK, direct && j == jj);
              if (!dm) continue;
              int g = 0;
              if (lane == __ffs(dm) - 1) g = atomicAdd(&ctl->rlen[jj], __popc(dm));
              g = __shfl_sync(GR_FULL_MASK, g, __ffs(dm) - 1) + __popc(dm & ((1u << lane) - 1u));
              if (direct && j == jj && g < a.n) a.ring[jj][g] = v;
            }
          }
        }
        const unsigned long long d = valid ? (__ldcg(a.key + v) >> 32) : 0ull;
        to_far(valid && b >= cb + K, v, (unsigned)d, fe + 1);
      }
      // flush the staged ring entries (one global atomic per CTA and slot) and
      // the next far pile
      __syncthreads();
      if (threadIdx.x < K && s_rcnt[threadIdx.x])
        s_rbase[threadIdx.x] = atomicAdd(&ctl->rlen[threadIdx.x], s_rcnt[threadIdx.x]);
      far_stage.reserve(&ctl->farlen[(fe + 1) % 3]);
      if (threadIdx.x == 0 && s_farmin != UINT_MAX)
        atomicMin(&ctl->farmin[(fe + 1) % 3], s_farmin);
      __syncthreads();
      const int rn = min(s_rn, RCAP);
      for (int k = threadIdx.x; k < rn; k += blockDim.x) {
        const int j = rs[k];
        const int g = s_rbase[j] + atomicAdd(&s_rcur[j], 1);
        if (g < a.n) a.ring[j][g] = rv[k];
      }
      far_stage.copy_out(a.far[(fe + 1) & 1], a.n);
      __syncthreads();  // every thread has read the stage count before it is cleared
      if (threadIdx.x == 0) {
        far_stage.reset();
        s_farmin = UINT_MAX;
      }
      if (!sc.sync()) return;
      // phase 2: pick the next bucket from the (now stable) slot lengths
      __shared__ int s_rl[K];
      __shared__ int s_fl2;
      __shared__ unsigned s_fm2;
      if (threadIdx.x < K) s_rl[threadIdx.x] = __ldcg(&ctl->rlen[threadIdx.x]);
      if (threadIdx.x == 0) {
        s_fl2 = __ldcg(&ctl->farlen[(fe + 1) % 3]);
        s_fm2 = __ldcg(&ctl->farmin[(fe + 1) % 3]);
      }
      __syncthreads();
      int nk = 0;  // the next bucket is cb + nk (0: none in the window)
      for (int k = 1; k < K && !nk; ++k)
        if (s_rl[(cb + k) % K] > 0) nk = k;
      ring_left = 0;
      for (int k = 1; k < K; ++k) ring_left += k != nk && s_rl[(cb + k) % K] > 0;
      if (nk) {
        const unsigned long long nb = cb + nk;
        const int j = (int)(nb % K);
        const int rl = min(s_rl[j], a.n);
        for (int base = swarp * 32; base < rl;
             base = gr_next_batch(base, rl, (int)nwarps * 32, &ctl->workb[s0], 32, lane)) {
          const int i = base + lane;
          int32_t v = 0;
          bool take = false;
          if (i < rl) {
            v = __ldcg(a.ring[j] + i);
            take = (__ldcg(a.key + v) >> 32) / a.delta == nb;
          }
          near_append(take, v);
        }
        T = (nb + 1) * a.delta;
        reset_slot = j;
      } else if (s_fl2 > 0 && s_fm2 != UINT_MAX) {
        // nothing in the window: the next SPLIT starts the window at the far
        // pile's smallest distance
        const unsigned long long fb = (unsigned long long)s_fm2 / a.delta;
        T = fb * a.delta;  // current bucket fb - 1: the window (fb - 1, fb - 1 + K)
        if (T == 0) T = a.delta;
      }
      ++fe;
    } else {
      // ---- SPLIT: raise the threshold, move far entries below it to near --
      const unsigned fm = fm_step;
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
      // warps take 32 far entries at a time
      for (int base = swarp * 32; base < flen;
           base = gr_next_batch(base, flen, (int)nwarps * 32, &ctl->work[s0], 32, lane)) {
        const int i = base + lane;
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
    // combined flush of the step's staged appends: one barrier, then all
    // global reservations in flight together, then the copies
    __syncthreads();
    bstage.prepare();
    near_stage.reserve(&ctl->qlen[s1]);
    mid_stage.reserve(&ctl->qmlen[s1]);
    far_stage.reserve(&ctl->farlen[fe_out % 3]);
    bstage.reserve(&ctl->nchunk[s1], &ctl->nbig[s1]);
    if (threadIdx.x == 0 && s_farmin != UINT_MAX) atomicMin(&ctl->farmin[fe_out % 3], s_farmin);
    __syncthreads();
    near_stage.copy_out(qn, a.n);
    mid_stage.copy_out(qmn, a.n);
    far_stage.copy_out(a.far[fe_out & 1], a.n);
    bstage.copy_out(chn, a.chunk_cap, a.status);
    if (!sc.sync()) return;
  }
  // one more row: the step loop's end (no near rows, no split)
  if (gtid == 0 && a.level_stats && it < a.max_levels) {
    a.level_stats[4 * it] = 0;
    a.level_stats[4 * it + 1] = 0;
    a.level_stats[4 * it + 2] = 0;
    a.level_stats[4 * it + 3] =
        (int)min(gr_globaltimer() - t_entry, (unsigned long long)INT_MAX);
  }
  // ---- overflow check: with every unrepresentable candidate dropped, a
  // vertex keeps an infinite label while a reached neighbour exists only if
  // its true distance is >= UINT32_MAX.
  if (__ldcg(&ctl->ovf_pending)) {
    for (int64_t u = gtid; u < a.n; u += gthreads) {
      if ((a.key[u] >> 32) == GR_INF_DIST) continue;
      for (int e = __ldg(a.R + u); e < __ldg(a.R + u + 1); ++e)
        if (a.key[__ldg(a.C + e)] == GR_KEY_INF) {
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

