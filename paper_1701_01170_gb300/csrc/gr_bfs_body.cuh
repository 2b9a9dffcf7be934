// gr_bfs_body.cuh — one BFS query (init + level loop) as a device function
// templated on the scope of threads that run it; shared by the cooperative
// single-query kernel (gr_bfs.cu) and the batched many-graph kernel
// (gr_batch.cu).  See gr_bfs.cu for the algorithm.
#pragma once

#include <climits>

#include "gr_internal.cuh"

#ifndef GR_VISIT_STRIPS
#define GR_VISIT_STRIPS 4  // 32-edge strips a warp expands per round
#endif
#ifndef GR_BULK_PUSH_STRIPS
#define GR_BULK_PUSH_STRIPS 4  // strips per round in the mark pass of a bulk push level
#endif
#ifndef GR_COLLECT_ROUNDS
#define GR_COLLECT_ROUNDS 4    // new vertices per lane in flight in the collect pass
#endif
// Push levels whose frontier has at least max(GR_BULK_PUSH_PER_VERTEX * n,
// GR_BULK_PUSH_MIN) edges run in bulk (see gr_bfs_body).  Below that,
// claiming as the edges arrive is faster than marking plus a collect pass
// over the whole bitmap: on R-MAT s22 (hub and 20 random sources) the
// direction-optimising mean is 0.190 ms at 2n against 0.206 ms at n / 8,
// 0.196 ms at n and 0.190 ms at 8n; push-only 0.615 ms at 2n against 0.630,
// 0.620 and 0.670 ms.
#define GR_BULK_PUSH_PER_VERTEX 2
#define GR_BULK_PUSH_MIN (1 << 16)
__host__ __device__ inline int64_t gr_default_bulk_edges(int64_t n) {
  const int64_t e = n * GR_BULK_PUSH_PER_VERTEX;
  return e > GR_BULK_PUSH_MIN ? e : GR_BULK_PUSH_MIN;
}

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
  int32_t* qm[2];     // medium-row queues (NULL: medium rows go to q)
  int32_t* ulist[2];  // unvisited lists of pull levels (NULL: rescan the bitmap every level)
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
  int64_t bulk_edges;  // push levels with a frontier of at least this many edges run in bulk
                       // (0: never); needs the frontier bitmaps front[]
  const uint32_t* preset;  // n-bit bitmap of vertices that start as visited (isolated vertices
                           // of a symmetric graph, which no edge reaches) or NULL
  int32_t* pdef;  // GR_PULL_DEFER_INTS entries: long pull rows shared by the grid (NULL: each
                  // row is scanned by the warp that owns its vertex)
};

// The whole BFS (init + level loop) for one query, executed by the threads
// of a scope S: S::tid / S::nthreads index the participating threads, and
// S::sync() is the step barrier (a bounded grid barrier for the cooperative
// single-query kernel, the hardware cluster barrier for batched jobs).
// PULL = false compiles a push-only BFS: no pull levels and none of their
// code (a.use_do and a.force_pull must then be 0).
template <bool PULL, class S>
__device__ __forceinline__ void gr_bfs_body(const BfsArgs& a, S& sc, GrArena& ar) {
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
  // ---- Set_Problem_Data: depth -1 / pred -1, the source at depth 0 ------
  for (int64_t v = gtid; v < a.n; v += gthreads) {
    a.depth[v] = v == a.src ? 0 : -1;
    if (a.pred) a.pred[v] = -1;
  }
  const int32_t sw = a.src >> 5;
  const uint32_t sbit = 1u << (a.src & 31);
  // frontier bitmaps: the next frontier of pull levels and bulk push levels
  const bool bitmaps = a.use_do || a.bulk_edges > 0;
  for (int64_t w = gtid; w < a.nwords; w += gthreads) {
    const uint32_t x = w == sw ? sbit : 0u;
    // isolated vertices start as visited, so that pull levels do not probe
    // them (on R-MAT s22 they are 43 % of the vertices); their depth stays -1
    a.visited[w] = a.preset ? (__ldg(a.preset + w) | x) : x;
    if (bitmaps) {
      a.front[0][w] = x;
      a.front[1][w] = 0u;
      a.front[2][w] = 0u;
    }
  }
  {
    const int beg = __ldg(a.R + a.src), deg = __ldg(a.R + a.src + 1) - beg;
    if (a.track_deg && deg >= a.big) {
      gr_register_source_chunks(a.ch[0], a.chunk_cap, &ctl->nchunk[0], &ctl->nbig[0], a.src,
                                beg, deg, a.status, gtid, gthreads);
    } else if (gtid == 0) {
      a.q[0][0] = a.src;
      ctl->qlen[0] = 1;
    }
    if (gtid == 0) ctl->mf[0] = (unsigned long long)deg;
  }
  if (!sc.sync()) return;

  const unsigned long long deadline = gr_globaltimer() + GR_TIME_LIMIT_NS;
  unsigned long long seen_edges = 0;  // sum of degrees of every visited vertex
  GrCounters cnt;
  // step counters are read once per CTA and broadcast through shared memory
  // (one L2 request per CTA instead of one per warp)
  __shared__ int s_nq, s_nqm, s_nch, s_nbig;
  __shared__ unsigned long long s_mf;
  __shared__ int s_qcnt, s_qbase, s_ucnt, s_ubase, s_nu;
  GrStage stage{ar.buf0, &s_qcnt, &s_qbase, GR_STAGE_CAP};
  __shared__ int s_mcnt, s_mbase;
  GrStage mstage{ar.bufm, &s_mcnt, &s_mbase, GR_STAGE_CAP};
  GrStage ustage{ar.buf1, &s_ucnt, &s_ubase, GR_STAGE_CAP};
  __shared__ int s_bcnt, s_btot[2];
  GrBigStage bstage{ar.bv, ar.bb, ar.bd, ar.bo, &s_bcnt, s_btot};
  __shared__ unsigned long long s_mfsum;
  __shared__ int s_found;
  __shared__ int s_ndef;  // rows the previous level deferred to the grid
  int list_ready = 0;  // the previous level was a pull level that wrote an unvisited list
  int pull = 0;
  int prev_pull = 0;   // the previous level was a pull level: its frontier exists as a bitmap only
  int L = 0;
  for (;; ++L) {
    const int s0 = L % 3, s1 = (L + 1) % 3, s2 = (L + 2) % 3;
    if (threadIdx.x == 0) {
      s_nq = __ldcg(&ctl->qlen[s0]);
      s_nqm = __ldcg(&ctl->qmlen[s0]);
      s_nch = __ldcg(&ctl->nchunk[s0]);
      s_nbig = __ldcg(&ctl->nbig[s0]);
      s_mf = __ldcg(&ctl->mf[s0]);
      s_nu = __ldcg(&ctl->ulen[s0]);
      s_ndef = PULL && a.pdef && L > 0 ? __ldcg(&ctl->ndef[s2]) : 0;
      stage.reset();
      mstage.reset();
      ustage.reset();
      bstage.reset();
      s_mfsum = 0ull;
      s_found = 0;
    }
    __syncthreads();
    // ---- rows the previous (pull) level deferred to the whole grid --------
    // Each listed row (vertex, first edge, end edge, chunks done, degree) is
    // cut into GR_PULL_CHUNK-edge chunks dealt out to the warps in turn.  The
    // first frontier neighbour a chunk finds claims the vertex (CAS on its
    // depth) for the previous level, whose frontier bitmap front[s2] is still
    // intact and whose counters (slot s0) the level below reads only after
    // the barrier; a chunk that starts after the claim skips its scan.  The
    // warp that completes a row's last chunk keeps the vertex on the
    // unvisited list if nothing matched.  The list's length was written
    // before the last barrier and is read with the level's other counters,
    // so every warp takes the same branch.
    if (PULL && s_ndef > 0) {
      {
        const int nd = min(s_ndef, GR_PULL_DEFER_CAP);
        const uint32_t* fprev = a.front[s2];
        uint32_t* fcur = a.front[s0];
        int32_t* ulist = a.ulist[0] ? a.ulist[L & 1] : nullptr;
        int64_t base = 0;
        for (int d = 0; d < nd; ++d) {
          int32_t* ent = a.pdef + 8 * d;
          const int32_t v = __ldcg(ent), beg = __ldcg(ent + 1), end = __ldcg(ent + 2);
          const int nchd = (end - beg + GR_PULL_CHUNK - 1) / GR_PULL_CHUNK;
          // this warp's chunks of the row: global chunk indices = swarp (mod nwarps)
          int64_t c = base + ((swarp - base) % nwarps + nwarps) % nwarps;
          for (; c < base + nchd; c += nwarps) {
            int32_t claimed = 0;
            if (lane == 0) claimed = __ldcg(a.depth + v) >= 0;
            if (!__shfl_sync(GR_FULL_MASK, claimed, 0)) {
              const int cb = beg + (int)(c - base) * GR_PULL_CHUNK;
              const int ce = min(cb + GR_PULL_CHUNK, end);
              constexpr int J = GR_PULL_CHUNK / 32;
              int32_t u[J];
#pragma unroll
              for (int j = 0; j < J; ++j) {
                const int e = cb + j * 32 + lane;
                u[j] = e < ce ? __ldg(a.C + e) : -1;
                if (u[j] >= 0) ++cnt.edges;
              }
              int32_t hu = -1;
#pragma unroll
              for (int j = J - 1; j >= 0; --j)
                if (u[j] >= 0 && ((fprev[u[j] >> 5] >> (u[j] & 31)) & 1u)) hu = u[j];
              const unsigned hm = __ballot_sync(GR_FULL_MASK, hu >= 0);
              if (hm) {
                const int32_t par = __shfl_sync(GR_FULL_MASK, hu, __ffs(hm) - 1);
                if (lane == 0 && atomicCAS(a.depth + v, -1, L) == -1) {
                  ++cnt.updates;
                  if (a.pred) a.pred[v] = par;
                  atomicOr(a.visited + (v >> 5), 1u << (v & 31));
                  atomicOr(fcur + (v >> 5), 1u << (v & 31));
                  atomicAdd(&ctl->qlen[s0], 1);
                  atomicAdd(&ctl->mf[s0], (unsigned long long)__ldcg(ent + 5));
                }
              }
            }
            if (lane == 0) {
              __threadfence();
              if (atomicAdd(ent + 3, 1) + 1 == nchd && ulist && __ldcg(a.depth + v) < 0) {
                const int pos = atomicAdd(&ctl->ulen[s0], 1);
                if (pos < a.n) ulist[pos] = v;
              }
            }
          }
          base += nchd;
        }
        if (!sc.sync()) return;
      }
      // the counters of this level, now with the deferred rows' outcomes
      if (threadIdx.x == 0) {
        s_nq = __ldcg(&ctl->qlen[s0]);
        s_mf = __ldcg(&ctl->mf[s0]);
        s_nu = __ldcg(&ctl->ulen[s0]);
      }
      __syncthreads();
    }
    // after a pull level qlen counts the discovered vertices without
    // listing them (the level's frontier is its bitmap)
    int nq = min(s_nq, a.n);
    int nqm = min(s_nqm, a.n);
    int nch = (int)min((int64_t)s_nch, a.chunk_cap);
    if (nq + nqm + nch == 0 || L > a.n) break;
    const int nf = nq + nqm + s_nbig;
    const unsigned long long mf = s_mf;
    seen_edges += mf;
    const unsigned long long mu = (unsigned long long)a.m > seen_edges
                                      ? (unsigned long long)a.m - seen_edges
                                      : 0ull;
    if (!PULL) {
      // push only
    } else if (a.force_pull) {
      pull = 1;
    } else if (a.use_do) {  // Eq. 5 / Eq. 6 with exact m_f, m_u
      if (!pull && (double)mf > (double)mu * a.do_a) pull = 1;
      else if (pull && (double)mf < (double)mu * a.do_b) pull = 0;
    }
    if (gtid == 0) {
      if ((L & 63) == 0) gr_check_deadline(ctl, a.status, deadline);
      if (a.level_stats && L < a.max_levels) {
        a.level_stats[4 * L] = nf;
        a.level_stats[4 * L + 1] = pull;
        a.level_stats[4 * L + 2] = (int)min(mf, (unsigned long long)INT_MAX);
        // start of this level in ns after the kernel started
        a.level_stats[4 * L + 3] =
            (int)min(gr_globaltimer() - t_entry, (unsigned long long)INT_MAX);
      }
      ctl->qlen[s2] = 0;
      ctl->qmlen[s2] = 0;
      ctl->workm[s2] = 0;
      ctl->nchunk[s2] = 0;
      ctl->nbig[s2] = 0;
      ctl->mf[s2] = 0ull;
      ctl->work[s2] = 0;
      ctl->workc[s2] = 0;
      ctl->workb[s2] = 0;
      ctl->qbuilt[s2] = 0;
      ctl->ulen[s2] = 0;
      ctl->ndef[s1] = 0;  // (slot s2 holds the deferred rows of the previous level)
    }
    if (bitmaps)
      for (int64_t w = gtid; w < a.nwords; w += gthreads) a.front[s2][w] = 0u;

    if (!pull && prev_pull) {
      // A push level after a pull level: list the frontier from its bitmap
      // (front[s0]); split rows go to the chunk list as usual.  One pass over
      // n bits and one barrier, only on pull -> push switches.
      const uint32_t* fb = a.front[s0];
      int32_t* qc = a.q[L & 1];
      int32_t* qmc = a.qm[0] ? a.qm[L & 1] : nullptr;
      int2* chc = a.ch[L & 1];
      for (int wb = swarp * 32; wb < a.nwords;
           wb = gr_next_batch(wb, a.nwords, (int)nwarps * 32, &ctl->workb[s0], 32, lane)) {
        const int w = wb + lane;
        const uint32_t word = w < a.nwords ? __ldcg(fb + w) : 0u;
        unsigned nz = __ballot_sync(GR_FULL_MASK, word != 0u);
        while (nz) {
          const int j = __ffs(nz) - 1;
          nz &= nz - 1u;
          const uint32_t bits = __shfl_sync(GR_FULL_MASK, word, j);
          const bool mine = (bits >> lane) & 1u;
          const int32_t v = (wb + j) * 32 + lane;
          int vb = 0, vd = 0;
          if (mine) {
            vb = __ldg(a.R + v);
            vd = __ldg(a.R + v + 1) - vb;
          }
          const bool big = mine && vd >= a.big;
          const bool mid = mine && !big && qmc && vd >= GR_MEDIUM_DEGREE;
          stage.append(qc, &ctl->qbuilt[s0], a.n, mine && !big && !mid, v, lane);
          mstage.append(qmc, &ctl->qmlen[s0], a.n, mid, v, lane);
          if (big)
            bstage.add(chc, a.chunk_cap, &ctl->nchunk[s0], &ctl->nbig[s0], v, vb, vd, a.status);
        }
      }
      stage.flush(qc, &ctl->qbuilt[s0], a.n);
      mstage.flush(qmc, &ctl->qmlen[s0], a.n);
      bstage.flush(chc, a.chunk_cap, &ctl->nchunk[s0], &ctl->nbig[s0], a.status);
      if (!sc.sync()) return;
      if (threadIdx.x == 0) {
        s_nq = __ldcg(&ctl->qbuilt[s0]);
        s_nqm = __ldcg(&ctl->qmlen[s0]);
        s_nch = __ldcg(&ctl->nchunk[s0]);
        stage.reset();
        mstage.reset();
        bstage.reset();
      }
      __syncthreads();
      nq = min(s_nq, a.n);
      nqm = min(s_nqm, a.n);
      nch = (int)min((int64_t)s_nch, a.chunk_cap);
    }

    int32_t* qn = a.q[(L + 1) & 1];
    int32_t* qmn = a.qm[0] ? a.qm[(L + 1) & 1] : nullptr;
    int2* chn = a.ch[(L + 1) & 1];
    uint32_t* fnext = a.front[s1];
    unsigned long long my_mf = 0;
    const int next_depth = L + 1;
    const bool list_pull = pull && list_ready;

    const bool bulk_push = !pull && a.bulk_edges > 0 && mf >= (unsigned long long)a.bulk_edges;
    if (bulk_push) {
      // ---- bulk push: advance + visit + cull as two passes ----------------
      // Mark: for every edge (u, v), v's word of the visited bitmap (vertices
      // of earlier levels; read-only during this pass, so it may be served
      // from L1) is loaded with the column; only a target it does not hold
      // reads its next-frontier word from L2, and if that bit is clear too,
      // sets it with a reduction that returns nothing and records u as v's
      // parent (several frontier vertices may store; each is a valid parent
      // one level up).  No per-edge atomic returns a value and no discovery
      // is classified inside the edge loop.
      const int32_t* q = a.q[L & 1];
      const int2* ch = a.ch[L & 1];
      // Both words of a target are read in the pre stage, before any mark of
      // the round: the next-frontier word only for targets the visited
      // bitmap lacks (skipping that load and marking blindly measured slower,
      // 0.80 vs 0.68 ms on R-MAT s22 push-only, as duplicate red.or traffic
      // to the same words outweighs the load).  Read in the mark stage
      // instead, each load had to wait for the previous edge's red.or to the
      // same bitmap, one L2 round trip per edge of the round.  Two edges of
      // one lane's round to the same vertex may then both mark it: the
      // reduction is idempotent and either predecessor is a valid parent.
      struct VisNext {
        uint32_t vis, next;
      };
      auto pre = [&](bool active, int, int32_t v) -> VisNext {
        const uint32_t b1 = 1u << (v & 31);
        const uint32_t vis = active ? a.visited[v >> 5] : b1;
        const uint32_t next = (vis & b1) ? b1 : __ldcg(fnext + (v >> 5));
        return VisNext{vis, next};
      };
      auto mark = [&](bool active, int32_t u, uint32_t, int, int32_t v, const VisNext& w) {
        if (!active) return;
        ++cnt.edges;
        const uint32_t b1 = 1u << (v & 31);
        if (!(w.vis & b1) && !(w.next & b1)) {
          gr_red_or_u32(fnext + (v >> 5), b1);
          if (a.pred) a.pred[v] = u;
        }
      };
      auto no_payload = [](int32_t) -> uint32_t { return 0u; };
      gr_chunks_loop<GR_BULK_PUSH_STRIPS>(ch, nch, swarp, (int)nwarps, lane, a.R, a.C, cnt,
                                          no_payload, pre, mark);
      if (a.qm[0])
        gr_rows_loop<GR_BULK_PUSH_STRIPS>(a.qm[L & 1], nqm, GR_MEDIUM_BATCH, &ctl->workm[s0],
                                          swarp, (int)nwarps, lane, a.R, a.C, cnt, no_payload,
                                          pre, mark);
      gr_rows_loop<GR_BULK_PUSH_STRIPS>(q, nq, 32, &ctl->work[s0], swarp, (int)nwarps, lane, a.R,
                                        a.C, cnt, no_payload, pre, mark);
      if (!sc.sync()) return;
      // Collect: one pass over the next-frontier bitmap.  Its set bits are
      // exactly this level's discoveries (a bit is only set for a vertex that
      // was unvisited when the level began).  Lane l of warp s takes the
      // words s + (l + 32 k) * nwarps, so the words of one warp lie far apart
      // and a dense run of discoveries (a hub's neighbourhood has clustered
      // ids) spreads over every CTA and its staging buffers.  The lane merges
      // its word into the visited bitmap; the set bits of the warp's 32 words
      // are then dealt out evenly over the lanes (a prefix count of the words'
      // bits, then each lane finds its bit), GR_COLLECT_ROUNDS vertices per
      // lane with their row loads in flight together.  Each new vertex gets
      // its depth and joins a row class of the next level.
      for (int64_t wk = swarp; wk < a.nwords; wk += 32 * nwarps) {
        const int64_t w = wk + (int64_t)lane * nwarps;
        uint32_t word = w < a.nwords ? __ldcg(fnext + w) : 0u;
        if (word) a.visited[w] = __ldcg(a.visited + w) | word;
        int total;
        const int excl = gr_warp_excl_scan(__popc(word), lane, &total);
        for (int base = 0; base < total; base += 32 * GR_COLLECT_ROUNDS) {
          int32_t v[GR_COLLECT_ROUNDS];
          bool mine[GR_COLLECT_ROUNDS];
#pragma unroll
          for (int k = 0; k < GR_COLLECT_ROUNDS; ++k) {
            const int p = base + k * 32 + lane;
            int lo = 0;  // the lane whose word holds the p-th bit of the batch
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
              const int cand = lo + step;
              if (__shfl_sync(GR_FULL_MASK, excl, cand) <= p) lo = cand;
            }
            const uint32_t ow = __shfl_sync(GR_FULL_MASK, word, lo);
            const int r = p - __shfl_sync(GR_FULL_MASK, excl, lo);
            mine[k] = p < total;
            v[k] = mine[k] ? (int32_t)((wk + (int64_t)lo * nwarps) * 32 + gr_nth_set_bit(ow, r)) : 0;
          }
          int vb[GR_COLLECT_ROUNDS], vd[GR_COLLECT_ROUNDS];
#pragma unroll
          for (int k = 0; k < GR_COLLECT_ROUNDS; ++k) {
            vb[k] = mine[k] ? __ldg(a.R + v[k]) : 0;
            vd[k] = mine[k] ? __ldg(a.R + v[k] + 1) : 0;
          }
#pragma unroll
          for (int k = 0; k < GR_COLLECT_ROUNDS; ++k) {
            vd[k] -= vb[k];
            if (mine[k]) {
              ++cnt.updates;
              a.depth[v[k]] = next_depth;
              my_mf += (unsigned long long)vd[k];
            }
            const bool big = mine[k] && vd[k] >= a.big;
            const bool mid = mine[k] && !big && qmn && vd[k] >= GR_MEDIUM_DEGREE;
            stage.append(qn, &ctl->qlen[s1], a.n, mine[k] && !big && !mid, v[k], lane);
            mstage.append(qmn, &ctl->qmlen[s1], a.n, mid, v[k], lane);
            if (big)
              bstage.add(chn, a.chunk_cap, &ctl->nchunk[s1], &ctl->nbig[s1], v[k], vb[k], vd[k],
                         a.status);
          }
        }
      }
    } else if (!pull) {
      // ---- push: advance + visit + cull fused ----------------------------
      const int32_t* q = a.q[L & 1];
      const int2* ch = a.ch[L & 1];
      // a large frontier mostly meets visited vertices: test with a plain load
      // before claiming; a small one (mesh-like graphs) claims directly and
      // saves a dependent round trip per level
      // (a few rows with many edges count as large: their targets repeat)
      const bool direct_claim =
          nf < GR_DIRECT_CLAIM_FRONTIER && (!a.track_deg || mf < 2ull * GR_DIRECT_CLAIM_FRONTIER);
      // Stages of the multi-strip expansion, each for all strips of a round
      // before the next: the visited word of each target (pre), the claims
      // (atomics with return values, all in flight together), the row bounds
      // of the targets won, then the writes and appends (visit).
      struct Claim {
        uint32_t word;
        int32_t won;
        int32_t vbeg, vdeg;
      };
      auto pre = [&](bool active, int, int32_t v) -> Claim {
        return Claim{(active && !direct_claim) ? a.visited[v >> 5] : 0u, 0, 0, 0};
      };
      auto claim = [&](bool active, int32_t, uint32_t, int, int32_t v, Claim& c) {
        const bool try_claim = active && (direct_claim || !(c.word & (1u << (v & 31))));
        c.won = gr_warp_claim(a.visited, try_claim, v, lane);
      };
      auto bounds = [&](bool, int32_t, uint32_t, int, int32_t v, Claim& c) {
        if (c.won && a.track_deg) {
          c.vbeg = __ldg(a.R + v);
          c.vdeg = __ldg(a.R + v + 1) - c.vbeg;
        }
      };
      auto visit = [&](bool active, int32_t u, uint32_t, int, int32_t v, const Claim& c) {
        if (active) ++cnt.edges;
        const bool won = c.won;
        if (a.use_do) gr_warp_set_bit(fnext, won, v, lane);
        const int vbeg = c.vbeg, vdeg = c.vdeg;
        if (won) {
          ++cnt.updates;
          a.depth[v] = next_depth;
          if (a.pred) a.pred[v] = u;
          my_mf += (unsigned long long)vdeg;
        }
        const bool big = won && vdeg >= a.big;
        const bool mid = won && !big && qmn && vdeg >= GR_MEDIUM_DEGREE;
        stage.append(qn, &ctl->qlen[s1], a.n, won && !big && !mid, v, lane);
        mstage.append(qmn, &ctl->qmlen[s1], a.n, mid, v, lane);
        if (big)
          bstage.add(chn, a.chunk_cap, &ctl->nchunk[s1], &ctl->nbig[s1], v, vbeg, vdeg,
                     a.status);
      };
      // largest work first: edge chunks of split rows, then medium rows,
      // then short rows 32 at a time (first batch by warp index, further
      // batches from a counter that idle warps never touch)
      auto no_payload = [](int32_t) -> uint32_t { return 0u; };
      gr_chunks_loop_mid<GR_VISIT_STRIPS>(ch, nch, swarp, (int)nwarps, lane, a.R, a.C, cnt,
                                          no_payload, pre, claim, bounds, visit);
      if (a.qm[0])
        gr_rows_loop_mid<GR_VISIT_STRIPS>(a.qm[L & 1], nqm, GR_MEDIUM_BATCH, &ctl->workm[s0],
                                          swarp, (int)nwarps, lane, a.R, a.C, cnt, no_payload,
                                          pre, claim, bounds, visit);
      gr_rows_loop_mid<GR_VISIT_STRIPS>(q, nq, 32, &ctl->work[s0], swarp, (int)nwarps, lane,
                                        a.R, a.C, cnt, no_payload, pre, claim, bounds, visit);
    } else {
      // ---- pull: unvisited vertices look for a parent in the frontier ----
      // (Alg. 2 Reverse_Advance: the step yields the next active frontier and
      // the next unvisited frontier)
      const uint32_t* fcur = a.front[s0];
      int32_t* unext = a.ulist[0] ? a.ulist[(L + 1) & 1] : nullptr;
      // First frontier neighbour in row order of each lane's candidate, or -1.
      // Each lane scans its first GR_PULL_SERIAL neighbours alone (rows are
      // sorted, so hubs come first and most candidates stop early); longer
      // rows that still need more are then scanned by the whole warp, 32
      // neighbours a round (four loads a lane in flight measured slower: most
      // such rows stop in the first rounds); a row still unresolved after
      // GR_PULL_WARP_EDGES more, with GR_PULL_DEFER_MIN or more left, goes to
      // the deferred list (GR_PULL_DEFERRED), which every warp of the grid
      // finishes at the top of the next level.  v and vdeg are the candidate
      // and its full degree.  All 32 lanes call.
      auto find_parent = [&](bool cand, int beg, int deg, int32_t v, int vdeg) -> int32_t {
        int32_t found = -1;
        const int p = cand ? min(deg, GR_PULL_SERIAL) : 0;
        // four neighbours per round: their column and bitmap loads overlap
        for (int e = beg; e < beg + p && found < 0; e += 4) {
          int32_t u[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            u[j] = e + j < beg + p ? __ldg(a.C + e + j) : -1;
            if (u[j] >= 0) ++cnt.edges;
          }
          bool in[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) in[j] = u[j] >= 0 && ((fcur[u[j] >> 5] >> (u[j] & 31)) & 1u);
#pragma unroll
          for (int j = 3; j >= 0; --j)
            if (in[j]) found = u[j];  // the first frontier neighbour in row order
        }
        unsigned pending = __ballot_sync(GR_FULL_MASK, cand && found < 0 && deg > GR_PULL_SERIAL);
        while (pending) {
          const int l = __ffs(pending) - 1;
          pending &= pending - 1u;
          const int lb = __shfl_sync(GR_FULL_MASK, beg, l);
          const int le = lb + __shfl_sync(GR_FULL_MASK, deg, l);
          const int32_t vl = __shfl_sync(GR_FULL_MASK, v, l);
          const int dl = __shfl_sync(GR_FULL_MASK, vdeg, l);
          int32_t f = -1;
          bool may_defer = a.pdef != nullptr;
          for (int e0 = lb + GR_PULL_SERIAL; e0 < le; e0 += 32) {
            if (may_defer && e0 - lb >= GR_PULL_SERIAL + GR_PULL_WARP_EDGES &&
                le - e0 >= GR_PULL_DEFER_MIN) {  // warp-uniform
              int slot = 0;
              if (lane == 0) slot = atomicAdd(&ctl->ndef[s0], 1);
              slot = __shfl_sync(GR_FULL_MASK, slot, 0);
              if (slot < GR_PULL_DEFER_CAP) {
                if (lane == 0) {
                  int32_t* ent = a.pdef + 8 * slot;
                  ent[0] = vl;
                  ent[1] = e0;
                  ent[2] = le;
                  ent[3] = 0;  // chunks done
                  ent[5] = dl;
                }
                f = GR_PULL_DEFERRED;
                break;
              }
              may_defer = false;  // the list is full: this warp scans on
            }
            const int e = e0 + lane;
            const bool ok = e < le;
            const int32_t u = ok ? __ldg(a.C + e) : 0;
            if (ok) ++cnt.edges;
            const unsigned hm = __ballot_sync(GR_FULL_MASK, ok && ((fcur[u >> 5] >> (u & 31)) & 1u));
            if (hm) {
              f = __shfl_sync(GR_FULL_MASK, u, __ffs(hm) - 1);
              break;
            }
          }
          if (lane == l) found = f;
        }
        return found;
      };
      // record one candidate's outcome; all 32 lanes
      // (the next frontier is the bitmap fnext; discoveries are only counted,
      // and listed by the next level if it is a push level)
      auto commit = [&](bool valid, int32_t v, int32_t found, int beg, int deg) {
        (void)beg;
        if (found >= 0) {
          ++cnt.updates;
          a.depth[v] = next_depth;
          if (a.pred) a.pred[v] = found;
          my_mf += (unsigned long long)deg;
        }
        const unsigned fm = __ballot_sync(GR_FULL_MASK, found >= 0);
        if (lane == 0 && fm) atomicAdd(&s_found, __popc(fm));
        // a vertex that can still be discovered stays on the unvisited list
        // (a deferred one is listed, if still unmatched, by its last chunk at
        // the top of the next level)
        if (unext) ustage.append(unext, &ctl->ulen[s1], a.n, valid && found == -1 && deg > 0, v, lane);
      };
      // A lane holds GR_PULL_WORDS candidates at once: their row bounds and
      // first neighbours are loaded together (independent loads in flight),
      // then each candidate whose first neighbour is not in the frontier
      // continues with find_parent from its second neighbour.
      constexpr int K = GR_PULL_WORDS;
      auto probe = [&](const bool (&cand)[K], const int32_t (&v)[K], int (&beg)[K], int (&deg)[K],
                       int32_t (&f0)[K]) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
          beg[k] = 0;
          deg[k] = 0;
          if (cand[k]) {
            ++cnt.verts;
            beg[k] = __ldg(a.R + v[k]);
            deg[k] = __ldg(a.R + v[k] + 1) - beg[k];
          }
        }
        int32_t u0[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
          u0[k] = cand[k] && deg[k] > 0 ? __ldg(a.C + beg[k]) : -1;
          if (u0[k] >= 0) ++cnt.edges;
        }
#pragma unroll
        for (int k = 0; k < K; ++k)
          f0[k] = u0[k] >= 0 && ((fcur[u0[k] >> 5] >> (u0[k] & 31)) & 1u) ? u0[k] : -1;
      };
      if (list_pull) {
        // the previous level was a pull level: walk its unvisited list,
        // K * 32 entries per warp and batch
        const int32_t* cl = a.ulist[L & 1];
        const int nc = min(s_nu, a.n);
        for (int base = swarp * 32 * K; base < nc;
             base = gr_next_batch(base, nc, (int)nwarps * 32 * K, &ctl->work[s0], 32 * K, lane)) {
          bool cand[K];
          int32_t v[K], f0[K];
          int beg[K], deg[K];
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const int i = base + k * 32 + lane;
            cand[k] = i < nc;
            v[k] = cand[k] ? __ldcg(cl + i) : 0;
          }
          probe(cand, v, beg, deg, f0);
#pragma unroll
          for (int k = 0; k < K; ++k) {
            int32_t found = f0[k];
            const int32_t rest = find_parent(cand[k] && found < 0 && deg[k] > 1, beg[k] + 1, deg[k] - 1,
                                             v[k], deg[k]);
            if (found < 0) found = rest;
            // list entries are distinct vertices: set their bits, one atomic per word
            gr_warp_set_bit(a.visited, found >= 0, v[k], lane);
            gr_warp_set_bit(fnext, found >= 0, v[k], lane);
            commit(cand[k], v[k], found, beg[k], deg[k]);
          }
        }
      } else {
        // first pull level: the unvisited set is the complement of the visited
        // bitmap; warps take K words (32 vertices each) at a time
        for (int wb = swarp * K; wb < a.nwords;
             wb = gr_next_batch(wb, a.nwords, (int)nwarps * K, &ctl->work[s0], K, lane)) {
          const uint32_t wl = lane < K && wb + lane < a.nwords ? a.visited[wb + lane] : 0xffffffffu;
          uint32_t word[K];
          bool cand[K];
          int32_t v[K], f0[K];
          int beg[K], deg[K];
#pragma unroll
          for (int k = 0; k < K; ++k) {
            word[k] = __shfl_sync(GR_FULL_MASK, wl, k);
            const int64_t v64 = (int64_t)(wb + k) * 32 + lane;
            v[k] = (int32_t)v64;
            cand[k] = v64 < a.n && !((word[k] >> lane) & 1u);
          }
          probe(cand, v, beg, deg, f0);
#pragma unroll
          for (int k = 0; k < K; ++k) {
            if (word[k] == 0xffffffffu) continue;  // warp-uniform
            int32_t found = f0[k];
            const int32_t rest = find_parent(cand[k] && found < 0 && deg[k] > 1, beg[k] + 1, deg[k] - 1,
                                             v[k], deg[k]);
            if (found < 0) found = rest;
            // the warp owns this word: visited and next-frontier bits by ballot
            // (a deferred vertex of the word gets its bits after the level's
            // barrier)
            const unsigned hit = __ballot_sync(GR_FULL_MASK, found >= 0);
            if (hit != 0u && lane == 0) {
              a.visited[wb + k] = word[k] | hit;
              fnext[wb + k] = hit;
            }
            commit(cand[k], v[k], found, beg[k], deg[k]);
          }
        }
      }
    }
    // combined flush of the level's staged appends: one barrier, then all
    // global reservations in flight together, then the copies
    my_mf = gr_warp_sum_u64(my_mf);
    if (lane == 0 && my_mf) atomicAdd(&s_mfsum, my_mf);
    const bool ulist_out = pull && a.ulist[0] != nullptr;
    __syncthreads();
    bstage.prepare();
    stage.reserve(&ctl->qlen[s1]);
    mstage.reserve(&ctl->qmlen[s1]);
    if (ulist_out) ustage.reserve(&ctl->ulen[s1]);
    bstage.reserve(&ctl->nchunk[s1], &ctl->nbig[s1]);
    if (threadIdx.x == 0 && s_mfsum) atomicAdd(&ctl->mf[s1], s_mfsum);
    if (threadIdx.x == 0 && s_found) atomicAdd(&ctl->qlen[s1], s_found);
    __syncthreads();
    stage.copy_out(qn, a.n);
    mstage.copy_out(qmn, a.n);
    if (ulist_out) ustage.copy_out(a.ulist[(L + 1) & 1], a.n);
    bstage.copy_out(chn, a.chunk_cap, a.status);
    list_ready = pull && a.ulist[0] != nullptr;
    prev_pull = pull;
    if (!sc.sync()) return;
  }
  // one more row: the loop's end (frontier 0)
  if (gtid == 0 && a.level_stats && L < a.max_levels) {
    a.level_stats[4 * L] = 0;
    a.level_stats[4 * L + 1] = 0;
    a.level_stats[4 * L + 2] = 0;
    a.level_stats[4 * L + 3] =
        (int)min(gr_globaltimer() - t_entry, (unsigned long long)INT_MAX);
  }
  cnt.flush(ctl);
  if (gtid == 0) ctl->levels = L;
}

