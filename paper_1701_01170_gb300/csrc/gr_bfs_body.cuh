// gr_bfs_body.cuh — one BFS query (init + level loop) as a device function
// templated on the scope of threads that run it; shared by the cooperative
// single-query kernel (gr_bfs.cu) and the batched many-graph kernel
// (gr_batch.cu).  See gr_bfs.cu for the algorithm.
#pragma once

#include <climits>

#include "gr_internal.cuh"

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
};

// The whole BFS (init + level loop) for one query, executed by the threads
// of a scope S: S::tid / S::nthreads index the participating threads, and
// S::sync() is the step barrier (a bounded grid barrier for the cooperative
// single-query kernel, the hardware cluster barrier for batched jobs).
template <class S>
__device__ __forceinline__ void gr_bfs_body(const BfsArgs& a, S& sc) {
  const int lane = threadIdx.x & 31;
  const int64_t gtid = sc.tid;
  const int64_t gthreads = sc.nthreads;
  const int64_t gwarp = gtid >> 5, nwarps = gthreads >> 5;
  GrCtl* ctl = a.ctl;
  // ---- Set_Problem_Data: depth -1 / pred -1, the source at depth 0 ------
  for (int64_t v = gtid; v < a.n; v += gthreads) {
    a.depth[v] = v == a.src ? 0 : -1;
    if (a.pred) a.pred[v] = -1;
  }
  const int32_t sw = a.src >> 5;
  const uint32_t sbit = 1u << (a.src & 31);
  for (int64_t w = gtid; w < a.nwords; w += gthreads) {
    uint32_t x = w == sw ? sbit : 0u;
    a.visited[w] = x;
    if (a.use_do) {
      a.front[0][w] = x;
      a.front[1][w] = 0u;
      a.front[2][w] = 0u;
    }
  }
  if (gtid == 0) {
    int beg = a.R[a.src], deg = a.R[a.src + 1] - beg;
    if (a.track_deg && deg >= a.big)
      gr_register_chunks(a.ch[0], a.chunk_cap, &ctl->nchunk[0], &ctl->nbig[0], a.src, beg, deg,
                         a.status);
    else {
      a.q[0][0] = a.src;
      ctl->qlen[0] = 1;
    }
    ctl->mf[0] = (unsigned long long)deg;
  }
  if (!sc.sync()) return;

  const unsigned long long deadline = gr_globaltimer() + GR_TIME_LIMIT_NS;
  unsigned long long seen_edges = 0;  // sum of degrees of every visited vertex
  GrCounters cnt;
  // step counters are read once per CTA and broadcast through shared memory
  // (one L2 request per CTA instead of one per warp)
  __shared__ int s_nq, s_nch, s_nbig;
  __shared__ unsigned long long s_mf;
  int pull = 0;
  int L = 0;
  for (;; ++L) {
    const int s0 = L % 3, s1 = (L + 1) % 3, s2 = (L + 2) % 3;
    if (threadIdx.x == 0) {
      s_nq = __ldcg(&ctl->qlen[s0]);
      s_nch = __ldcg(&ctl->nchunk[s0]);
      s_nbig = __ldcg(&ctl->nbig[s0]);
      s_mf = __ldcg(&ctl->mf[s0]);
    }
    __syncthreads();
    const int nq = min(s_nq, a.n);
    const int nch = (int)min((int64_t)s_nch, a.chunk_cap);
    if (nq + nch == 0 || L > a.n) break;
    const int nf = nq + s_nbig;
    const unsigned long long mf = s_mf;
    seen_edges += mf;
    const unsigned long long mu = (unsigned long long)a.m > seen_edges
                                      ? (unsigned long long)a.m - seen_edges
                                      : 0ull;
    if (a.force_pull) {
      pull = 1;
    } else if (a.use_do) {  // Eq. 5 / Eq. 6 with exact m_f, m_u
      if (!pull && (double)mf > (double)mu * a.do_a) pull = 1;
      else if (pull && (double)mf < (double)mu * a.do_b) pull = 0;
    }
    if (gtid == 0) {
      gr_check_deadline(ctl, a.status, deadline);
      if (a.level_stats && L < a.max_levels) {
        a.level_stats[3 * L] = nf;
        a.level_stats[3 * L + 1] = pull;
        a.level_stats[3 * L + 2] = (int)min(mf, (unsigned long long)INT_MAX);
      }
      ctl->qlen[s2] = 0;
      ctl->nchunk[s2] = 0;
      ctl->nbig[s2] = 0;
      ctl->mf[s2] = 0ull;
      ctl->work[s2] = 0;
      ctl->workc[s2] = 0;
    }
    if (a.use_do)
      for (int64_t w = gtid; w < a.nwords; w += gthreads) a.front[s2][w] = 0u;

    int32_t* qn = a.q[(L + 1) & 1];
    int2* chn = a.ch[(L + 1) & 1];
    uint32_t* fnext = a.front[s1];
    unsigned long long my_mf = 0;
    const int next_depth = L + 1;

    if (!pull) {
      // ---- push: advance + visit + cull fused ----------------------------
      const int32_t* q = a.q[L & 1];
      const int2* ch = a.ch[L & 1];
      auto visit = [&](bool active, int32_t u, uint32_t, int, int32_t v) {
        bool won = false;
        if (active) {
          ++cnt.edges;
          const uint32_t bit = 1u << (v & 31);
          uint32_t* wp = a.visited + (v >> 5);
          if (!(*wp & bit)) won = !(atomicOr(wp, bit) & bit);
        }
        int vbeg = 0, vdeg = 0;
        if (won) {
          ++cnt.updates;
          a.depth[v] = next_depth;
          if (a.pred) a.pred[v] = u;
          if (a.use_do) atomicOr(fnext + (v >> 5), 1u << (v & 31));
          if (a.track_deg) {
            vbeg = __ldg(a.R + v);
            vdeg = __ldg(a.R + v + 1) - vbeg;
            my_mf += (unsigned long long)vdeg;
          }
        }
        const bool big = won && vdeg >= a.big;
        gr_warp_append(qn, &ctl->qlen[s1], a.n, won && !big, v, lane);
        if (big)
          gr_register_chunks(chn, a.chunk_cap, &ctl->nchunk[s1], &ctl->nbig[s1], v, vbeg, vdeg,
                             a.status);
      };
      // warps take 32 frontier rows at a time: the first batch by warp index,
      // further batches from a counter (idle warps never touch it)
      for (int base = (int)gwarp * 32; base < nq;
           base = (int)nwarps * 32 + gr_warp_grab(&ctl->work[s0], 32, lane)) {
        const int i = base + lane;
        const bool valid = i < nq;
        int32_t u = 0;
        int beg = 0, deg = 0;
        if (valid) {
          ++cnt.verts;
          u = __ldcg(q + i);
          beg = __ldg(a.R + u);
          deg = __ldg(a.R + u + 1) - beg;
        }
        gr_warp_expand(a.R, a.C, valid, u, beg, deg, 0u, lane, visit);
      }
      // then one 1024-edge chunk of a long row at a time
      for (int c = (int)gwarp; c < nch; c = (int)nwarps + gr_warp_grab(&ctl->workc[s0], 1, lane)) {
        const int2 cu = __ldcg(ch + c);
        const int e1 = min(cu.y + GR_CHUNK_EDGES, __ldg(a.R + cu.x + 1));
        if (lane == 0) ++cnt.verts;
        gr_warp_chunk(a.C, cu.x, cu.y, e1, 0u, lane, visit);
      }
    } else {
      // ---- pull: unvisited vertices look for a parent in the frontier ----
      const uint32_t* fcur = a.front[s0];
      // warps take GR_PULL_WORDS visited words (32 vertices each) at a time
      for (int wb = (int)gwarp * GR_PULL_WORDS; wb < a.nwords;
           wb = (int)nwarps * GR_PULL_WORDS + gr_warp_grab(&ctl->work[s0], GR_PULL_WORDS, lane)) {
        const int we = min(wb + GR_PULL_WORDS, a.nwords);
      for (int64_t w = wb; w < we; ++w) {
        const uint32_t word = a.visited[w];
        if (word == 0xffffffffu) continue;
        const int64_t v64 = w * 32 + lane;
        const int32_t v = (int32_t)v64;
        const bool cand = v64 < a.n && !((word >> lane) & 1u);
        int32_t found = -1;
        int beg = 0, deg = 0;
        if (cand) {
          ++cnt.verts;
          beg = __ldg(a.R + v);
          deg = __ldg(a.R + v + 1) - beg;
          for (int e = beg; e < beg + deg; ++e) {
            ++cnt.edges;
            const int32_t u = __ldg(a.C + e);
            if ((fcur[u >> 5] >> (u & 31)) & 1u) {
              found = u;
              break;
            }
          }
        }
        const unsigned hit = __ballot_sync(GR_FULL_MASK, found >= 0);
        if (hit == 0u) continue;
        if (lane == 0) {
          a.visited[w] = word | hit;
          fnext[w] = hit;
        }
        if (found >= 0) {
          ++cnt.updates;
          a.depth[v] = next_depth;
          if (a.pred) a.pred[v] = found;
          my_mf += (unsigned long long)deg;
        }
        const bool big = found >= 0 && deg >= a.big;
        gr_warp_append(qn, &ctl->qlen[s1], a.n, found >= 0 && !big, v, lane);
        if (big)
          gr_register_chunks(chn, a.chunk_cap, &ctl->nchunk[s1], &ctl->nbig[s1], v, beg, deg,
                             a.status);
      }
      }
    }
    my_mf = gr_warp_sum_u64(my_mf);
    if (lane == 0 && my_mf) atomicAdd(&ctl->mf[s1], my_mf);
    if (!sc.sync()) return;
  }
  cnt.flush(ctl);
  if (gtid == 0) ctl->levels = L;
}

