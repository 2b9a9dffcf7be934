/*
 * oracle.c — plain, slow, obviously correct CPU reference for the frontier
 * traversal hot path (advance, filter, BFS, SSSP).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this code.  It shares no source,
 * header, helper or constant with the CUDA library, and it never calls it.
 *
 * Conventions (the paper's problem statements, Alg. 1 Set_Problem_Data and
 * Sec. 6.1 BFS): unreachable vertices have depth -1, dist UINT32_MAX and
 * pred -1; the source has depth 0, dist 0 and pred -1.
 *
 * Every function is single-threaded; concurrent calls on distinct outputs are
 * safe (no global state).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_INF32 0xFFFFFFFFu
#define ORC_INF64 0xFFFFFFFFFFFFFFFFull

/* ------------------------------------------------------------------------ */
/* BFS (Sec. 6.1): depth[v] = fewest edges on a directed path src -> v.     */
/* Textbook FIFO queue BFS; pred = the vertex that first discovered v.       */
/* Returns the number of reached vertices, or -1 on bad arguments.          */
/* ------------------------------------------------------------------------ */
int64_t orc_bfs(int32_t n, const int32_t* R, const int32_t* C, int32_t src,
                int32_t* depth, int32_t* pred) {
  if (n < 0 || src < 0 || src >= n) return -1;
  for (int32_t v = 0; v < n; ++v) { depth[v] = -1; if (pred) pred[v] = -1; }
  int32_t* queue = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  if (!queue) return -1;
  int64_t head = 0, tail = 0;
  depth[src] = 0;
  queue[tail++] = src;
  while (head < tail) {
    int32_t u = queue[head++];
    for (int64_t e = R[u]; e < R[u + 1]; ++e) {
      int32_t v = C[e];
      if (depth[v] == -1) {
        depth[v] = depth[u] + 1;
        if (pred) pred[v] = u;
        queue[tail++] = v;
      }
    }
  }
  free(queue);
  return tail;
}

/*
 * Canonical BFS parent: for every reached v != src, the smallest vertex id u
 * with an edge (u, v) and depth[u] == depth[v] - 1.  Definition written out
 * over the edge list (works for directed graphs without a transpose).
 */
void orc_bfs_min_parent(int32_t n, const int32_t* R, const int32_t* C, const int32_t* depth,
                        int32_t* pred) {
  for (int32_t v = 0; v < n; ++v) pred[v] = -1;
  for (int32_t u = 0; u < n; ++u) {
    if (depth[u] < 0) continue;
    for (int64_t e = R[u]; e < R[u + 1]; ++e) {
      int32_t v = C[e];
      if (depth[v] == depth[u] + 1 && (pred[v] == -1 || u < pred[v])) pred[v] = u;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* SSSP (Sec. 3 example, Alg. 1): dist[v] = min over src->v paths of the sum */
/* of non-negative weights.  Binary-heap Dijkstra with lazy deletion and     */
/* 64-bit keys; relax on strict <; pred set on strict improvement.          */
/* Returns 0, 1 if some finite distance does not fit below UINT32_MAX,      */
/* or -1 on bad arguments / allocation failure.                             */
/* ------------------------------------------------------------------------ */
typedef struct { uint64_t key; int32_t v; } orc_heap_item;

static void heap_push(orc_heap_item* h, int64_t* len, uint64_t key, int32_t v) {
  int64_t i = (*len)++;
  h[i].key = key; h[i].v = v;
  while (i > 0) {
    int64_t p = (i - 1) / 2;
    if (h[p].key <= h[i].key) break;
    orc_heap_item t = h[p]; h[p] = h[i]; h[i] = t;
    i = p;
  }
}

static orc_heap_item heap_pop(orc_heap_item* h, int64_t* len) {
  orc_heap_item top = h[0];
  h[0] = h[--(*len)];
  int64_t i = 0;
  for (;;) {
    int64_t l = 2 * i + 1, r = l + 1, s = i;
    if (l < *len && h[l].key < h[s].key) s = l;
    if (r < *len && h[r].key < h[s].key) s = r;
    if (s == i) break;
    orc_heap_item t = h[s]; h[s] = h[i]; h[i] = t;
    i = s;
  }
  return top;
}

int32_t orc_dijkstra(int32_t n, const int32_t* R, const int32_t* C, const uint32_t* W,
                     int32_t src, uint32_t* dist, int32_t* pred) {
  if (n < 0 || src < 0 || src >= n) return -1;
  uint64_t* d = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));
  int64_t m = R[n];
  orc_heap_item* h = (orc_heap_item*)malloc((size_t)(m + 1) * sizeof(orc_heap_item));
  if (!d || !h) { free(d); free(h); return -1; }
  for (int32_t v = 0; v < n; ++v) { d[v] = ORC_INF64; if (pred) pred[v] = -1; }
  int64_t len = 0;
  d[src] = 0;
  heap_push(h, &len, 0, src);
  while (len > 0) {
    orc_heap_item it = heap_pop(h, &len);
    int32_t u = it.v;
    if (it.key != d[u]) continue; /* stale entry */
    for (int64_t e = R[u]; e < R[u + 1]; ++e) {
      int32_t v = C[e];
      uint64_t nd = d[u] + (uint64_t)W[e];
      if (nd < d[v]) {
        d[v] = nd;
        if (pred) pred[v] = u;
        heap_push(h, &len, nd, v);
      }
    }
  }
  int32_t over = 0;
  for (int32_t v = 0; v < n; ++v) {
    if (d[v] == ORC_INF64) dist[v] = ORC_INF32;
    else if (d[v] >= (uint64_t)ORC_INF32) { dist[v] = ORC_INF32; over = 1; }
    else dist[v] = (uint32_t)d[v];
  }
  free(d); free(h);
  return over;
}

/*
 * Canonical SSSP parent: for every reached v != src, the smallest u with an
 * edge (u, v, w) and dist[u] + w == dist[v] (a "tight" edge).  With weights
 * >= 1 every tight parent has a strictly smaller distance, so this is a tree.
 */
void orc_sssp_min_parent(int32_t n, const int32_t* R, const int32_t* C, const uint32_t* W,
                         const uint32_t* dist, int32_t src, int32_t* pred) {
  for (int32_t v = 0; v < n; ++v) pred[v] = -1;
  for (int32_t u = 0; u < n; ++u) {
    if (dist[u] == ORC_INF32) continue;
    for (int64_t e = R[u]; e < R[u + 1]; ++e) {
      int32_t v = C[e];
      if (v == src) continue;
      if ((uint64_t)dist[u] + W[e] == (uint64_t)dist[v] && (pred[v] == -1 || u < pred[v]))
        pred[v] = u;
    }
  }
}

/*
 * Bellman-Ford (n-1 rounds over every edge) — brute-force cross-check for
 * Dijkstra and BFS on small graphs.  W == NULL means unit weights.
 * dist64 uses UINT64_MAX for unreachable.
 */
void orc_bellman_ford(int32_t n, const int32_t* R, const int32_t* C, const uint32_t* W,
                      int32_t src, uint64_t* dist64) {
  for (int32_t v = 0; v < n; ++v) dist64[v] = ORC_INF64;
  dist64[src] = 0;
  for (int32_t round = 0; round + 1 < n; ++round) {
    int changed = 0;
    for (int32_t u = 0; u < n; ++u) {
      if (dist64[u] == ORC_INF64) continue;
      for (int64_t e = R[u]; e < R[u + 1]; ++e) {
        uint64_t nd = dist64[u] + (W ? (uint64_t)W[e] : 1u);
        if (nd < dist64[C[e]]) { dist64[C[e]] = nd; changed = 1; }
      }
    }
    if (!changed) break;
  }
}

/*
 * Floyd-Warshall all-pairs shortest paths into D (n x n, row = source);
 * W == NULL means unit weights; UINT64_MAX for no path.
 */
void orc_floyd_warshall(int32_t n, const int32_t* R, const int32_t* C, const uint32_t* W,
                        uint64_t* D) {
  for (int64_t i = 0; i < (int64_t)n * n; ++i) D[i] = ORC_INF64;
  for (int32_t u = 0; u < n; ++u) {
    D[(int64_t)u * n + u] = 0;
    for (int64_t e = R[u]; e < R[u + 1]; ++e) {
      uint64_t w = W ? (uint64_t)W[e] : 1u;
      uint64_t* slot = &D[(int64_t)u * n + C[e]];
      if (C[e] != u && w < *slot) *slot = w;
    }
  }
  for (int32_t k = 0; k < n; ++k)
    for (int32_t i = 0; i < n; ++i) {
      uint64_t dik = D[(int64_t)i * n + k];
      if (dik == ORC_INF64) continue;
      for (int32_t j = 0; j < n; ++j) {
        uint64_t dkj = D[(int64_t)k * n + j];
        if (dkj == ORC_INF64) continue;
        if (dik + dkj < D[(int64_t)i * n + j]) D[(int64_t)i * n + j] = dik + dkj;
      }
    }
}

/* ------------------------------------------------------------------------ */
/* Advance (Sec. 4.1).  The output frontier is the concatenation, in input   */
/* order, of each input vertex's neighbour list: vertex ids (V->V) or edge  */
/* ids (V->E).  This is the placement the degree prefix-sum defines.        */
/* Returns the output length (the full length even if it exceeds cap; only  */
/* the first cap items are written).                                        */
/* ------------------------------------------------------------------------ */
int64_t orc_advance(const int32_t* R, const int32_t* C, const int32_t* in, int64_t in_len,
                    int32_t edge_ids, int32_t* out, int64_t cap) {
  int64_t k = 0;
  for (int64_t i = 0; i < in_len; ++i) {
    int32_t u = in[i];
    for (int64_t e = R[u]; e < R[u + 1]; ++e, ++k)
      if (k < cap) out[k] = edge_ids ? (int32_t)e : C[e];
  }
  return k;
}

/*
 * Push advance with the BFS visit functor (Sec. 6.1), sequential semantics:
 * walk the input in order; every neighbour v with depth[v] == -1 gets
 * depth = level + 1, pred = u, and is appended to out once.
 */
int64_t orc_advance_bfs(const int32_t* R, const int32_t* C, const int32_t* in, int64_t in_len,
                        int32_t level, int32_t* depth, int32_t* pred, int32_t* out) {
  int64_t k = 0;
  for (int64_t i = 0; i < in_len; ++i) {
    int32_t u = in[i];
    for (int64_t e = R[u]; e < R[u + 1]; ++e) {
      int32_t v = C[e];
      if (depth[v] == -1) {
        depth[v] = level + 1;
        if (pred) pred[v] = u;
        out[k++] = v;
      }
    }
  }
  return k;
}

/*
 * Pull step (Sec. 5.1.4, Alg. 2 Reverse_Advance): every candidate v that is
 * still unvisited becomes active iff some neighbour u has depth[u] == level;
 * it then gets depth = level + 1 and pred = the first such u in row order.
 * Active vertices go to `active`, the rest of the unvisited candidates to
 * `unvisited` (both in input order).  Membership is judged on the depths as
 * they were before the step.  Returns the active count; *n_unvisited gets
 * the other count.
 */
int64_t orc_pull(const int32_t* R, const int32_t* C, const int32_t* cand, int64_t len,
                 int32_t level, int32_t* depth, int32_t* pred, int32_t* active,
                 int32_t* unvisited, int64_t* n_unvisited) {
  int64_t na = 0, nu = 0;
  int32_t* found = (int32_t*)malloc((size_t)(len > 0 ? len : 1) * sizeof(int32_t));
  if (!found) return -1;
  for (int64_t i = 0; i < len; ++i) {
    int32_t v = cand[i];
    found[i] = -2; /* not a candidate (already visited) */
    if (depth[v] != -1) continue;
    found[i] = -1;
    for (int64_t e = R[v]; e < R[v + 1]; ++e)
      if (depth[C[e]] == level) { found[i] = C[e]; break; }
  }
  for (int64_t i = 0; i < len; ++i) {
    int32_t v = cand[i];
    if (found[i] >= 0) {
      depth[v] = level + 1;
      if (pred) pred[v] = found[i];
      if (active) active[na] = v;
      na++;
    } else if (found[i] == -1) {
      if (unvisited) unvisited[nu] = v;
      nu++;
    }
  }
  free(found);
  if (n_unvisited) *n_unvisited = nu;
  return na;
}

/*
 * Push advance with the SSSP relax functor (Alg. 1 Update_Label/Set_Pred),
 * Jacobi semantics: every relaxation reads dist[u] as it was before the step.
 * For each edge (u, v, w) from the input, candidate = dist[u] + w; v's new
 * distance is the minimum of its old one and all candidates (ties keep the
 * smaller u as pred).  Improved vertices are listed once each, ascending.
 * Returns the number improved, or -1 on overflow (a candidate >= UINT32_MAX).
 */
int64_t orc_advance_relax(int32_t n, const int32_t* R, const int32_t* C, const uint32_t* W,
                          const int32_t* in, int64_t in_len, uint32_t* dist, int32_t* pred,
                          int32_t* out) {
  uint32_t* d0 = (uint32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(uint32_t));
  uint64_t* best = (uint64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(uint64_t));
  int32_t* bp = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  if (!d0 || !best || !bp) { free(d0); free(best); free(bp); return -2; }
  memcpy(d0, dist, (size_t)n * sizeof(uint32_t));
  for (int32_t v = 0; v < n; ++v) { best[v] = d0[v]; bp[v] = pred ? pred[v] : -1; }
  int overflow = 0;
  for (int64_t i = 0; i < in_len; ++i) {
    int32_t u = in[i];
    if (d0[u] == ORC_INF32) continue;
    for (int64_t e = R[u]; e < R[u + 1]; ++e) {
      int32_t v = C[e];
      uint64_t cand = (uint64_t)d0[u] + W[e];
      if (cand >= (uint64_t)ORC_INF32) { overflow = 1; continue; }
      if (cand < best[v] || (cand == best[v] && cand < d0[v] && u < bp[v])) {
        best[v] = cand;
        bp[v] = u;
      }
    }
  }
  int64_t k = 0;
  for (int32_t v = 0; v < n; ++v) {
    if (best[v] < d0[v]) {
      dist[v] = (uint32_t)best[v];
      if (pred) pred[v] = bp[v];
      out[k++] = v;
    }
  }
  free(d0); free(best); free(bp);
  return overflow ? -1 : k;
}

/* ------------------------------------------------------------------------ */
/* Filter (Sec. 4.2): compaction of the items that pass a validity test.    */
/* ------------------------------------------------------------------------ */

/* Exact filter: first occurrence of every item in [0, n), in input order. */
int64_t orc_filter_unique(int32_t n, const int32_t* in, int64_t len, int32_t* out) {
  uint8_t* seen = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
  if (!seen) return -1;
  int64_t k = 0;
  for (int64_t i = 0; i < len; ++i) {
    int32_t v = in[i];
    if (v < 0 || v >= n || seen[v]) continue;
    seen[v] = 1;
    out[k++] = v;
  }
  free(seen);
  return k;
}

/* Unvisited frontier (Alg. 2 GenerateUnvisitedFrontier): v ascending with depth[v] == -1. */
int64_t orc_filter_unvisited(int32_t n, const int32_t* depth, int32_t* out) {
  int64_t k = 0;
  for (int32_t v = 0; v < n; ++v)
    if (depth[v] == -1) out[k++] = v;
  return k;
}

/*
 * Near/far split (Sec. 5.1.5, two-level priority queue): stable partition of
 * the items in [0, n) by dist[v] < threshold (near) versus >= (far).
 */
int64_t orc_filter_near_far(int32_t n, const int32_t* in, int64_t len, const uint32_t* dist,
                            uint32_t threshold, int32_t* near, int32_t* far, int64_t* far_len) {
  int64_t a = 0, b = 0;
  for (int64_t i = 0; i < len; ++i) {
    int32_t v = in[i];
    if (v < 0 || v >= n) continue;
    if (dist[v] < threshold) near[a++] = v;
    else far[b++] = v;
  }
  *far_len = b;
  return a;
}

/* ------------------------------------------------------------------------ */
/* Certificates: complete checks of a BFS / SSSP answer that need no oracle  */
/* run (textbook shortest-path optimality conditions).  Return 0 when the    */
/* answer is valid, else a positive code naming the first violated rule.    */
/* ------------------------------------------------------------------------ */
int32_t orc_bfs_certificate(int32_t n, const int32_t* R, const int32_t* C, int32_t src,
                            const int32_t* depth, const int32_t* pred) {
  if (src < 0 || src >= n) return 1;
  if (depth[src] != 0) return 2;
  if (pred && pred[src] != -1) return 3;
  for (int32_t v = 0; v < n; ++v) {
    if (depth[v] < -1) return 4;
    if (pred && ((depth[v] == -1) != (pred[v] == -1)) && v != src) return 5;
    if (v != src && depth[v] == 0) return 6;
  }
  for (int32_t u = 0; u < n; ++u) {
    if (depth[u] < 0) continue;
    for (int64_t e = R[u]; e < R[u + 1]; ++e) {
      int32_t v = C[e];
      if (depth[v] == -1) return 7;            /* edge leaves the reached set */
      if (depth[v] > depth[u] + 1) return 8;   /* edge skips a level */
    }
  }
  if (pred) {
    for (int32_t v = 0; v < n; ++v) {
      if (v == src || depth[v] <= 0) continue;
      int32_t p = pred[v];
      if (p < 0 || p >= n) return 9;
      if (depth[p] != depth[v] - 1) return 10;
    }
    /* (pred[v], v) must be an edge: one sweep over the reached rows marks
       every v whose pred's row lists it (O(m), also on a hub whose row
       holds most of the graph) */
    int8_t* ok = (int8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!ok) return 12;
    for (int32_t u = 0; u < n; ++u) {
      if (depth[u] < 0) continue;
      for (int64_t e = R[u]; e < R[u + 1]; ++e)
        if (pred[C[e]] == u) ok[C[e]] = 1;
    }
    for (int32_t v = 0; v < n; ++v)
      if (v != src && depth[v] > 0 && !ok[v]) { free(ok); return 11; }
    free(ok);
  } else {
    /* without preds, every reached v != src still needs a parent one level up */
    int32_t* has = (int32_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    if (!has) return 12;
    for (int32_t u = 0; u < n; ++u) {
      if (depth[u] < 0) continue;
      for (int64_t e = R[u]; e < R[u + 1]; ++e)
        if (depth[C[e]] == depth[u] + 1) has[C[e]] = 1;
    }
    for (int32_t v = 0; v < n; ++v)
      if (v != src && depth[v] > 0 && !has[v]) { free(has); return 13; }
    free(has);
  }
  return 0;
}

int32_t orc_sssp_certificate(int32_t n, const int32_t* R, const int32_t* C, const uint32_t* W,
                             int32_t src, const uint32_t* dist, const int32_t* pred) {
  if (src < 0 || src >= n) return 1;
  if (dist[src] != 0) return 2;
  if (pred && pred[src] != -1) return 3;
  for (int32_t u = 0; u < n; ++u) {
    if (dist[u] == ORC_INF32) continue;
    for (int64_t e = R[u]; e < R[u + 1]; ++e) {
      int32_t v = C[e];
      if ((uint64_t)dist[v] > (uint64_t)dist[u] + W[e]) return 4; /* relaxable edge */
    }
  }
  if (!pred) return 0;
  for (int32_t v = 0; v < n; ++v) {
    if (v == src) continue;
    if (dist[v] == ORC_INF32) { if (pred[v] != -1) return 5; continue; }
    int32_t p = pred[v];
    if (p < 0 || p >= n) return 6;
    if (dist[p] == ORC_INF32) return 7;
  }
  {
    /* some edge (pred[v], v) must be tight: one O(m) sweep marks them */
    int8_t* ok = (int8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!ok) return 9;
    for (int32_t u = 0; u < n; ++u) {
      if (dist[u] == ORC_INF32) continue;
      for (int64_t e = R[u]; e < R[u + 1]; ++e) {
        int32_t v = C[e];
        if (v != src && pred[v] == u && (uint64_t)dist[u] + W[e] == (uint64_t)dist[v]) ok[v] = 1;
      }
    }
    for (int32_t v = 0; v < n; ++v)
      if (v != src && dist[v] != ORC_INF32 && !ok[v]) { free(ok); return 8; }
    free(ok);
  }
  /* following pred from any reached vertex must reach src without a cycle */
  int8_t* state = (int8_t*)calloc((size_t)(n > 0 ? n : 1), 1); /* 0 new, 1 on path, 2 ok */
  int32_t* path = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  if (!state || !path) { free(state); free(path); return 9; }
  state[src] = 2;
  for (int32_t v = 0; v < n; ++v) {
    if (dist[v] == ORC_INF32 || state[v] == 2) continue;
    int32_t len = 0, x = v;
    while (state[x] == 0) { state[x] = 1; path[len++] = x; x = pred[x]; }
    if (state[x] == 1) { free(state); free(path); return 10; }
    for (int32_t i = 0; i < len; ++i) state[path[i]] = 2;
  }
  free(state); free(path);
  return 0;
}

/* Multi-source BFS reference: k independent queue BFS runs, depth is k x n. */
int32_t orc_bfs_multi(int32_t n, const int32_t* R, const int32_t* C, const int32_t* srcs,
                      int32_t k, int32_t* depth) {
  for (int32_t i = 0; i < k; ++i)
    if (orc_bfs(n, R, C, srcs[i], depth + (int64_t)i * n, NULL) < 0) return -1;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Betweenness centrality, one source (Sec. 6.3: Brandes' formulation, a     */
/* forward BFS pass that accumulates path counts and a backward pass over    */
/* the BFS levels that accumulates dependencies).                           */
/*   depth: BFS depth from src (-1 unreachable);                             */
/*   sigma[v]: number of shortest src -> v paths (sigma[src] = 1, 0 if       */
/*     unreachable), the sum of sigma[u] over edges (u, v) with              */
/*     depth[v] = depth[u] + 1;                                              */
/*   delta[u]: dependency of src on u, the sum over edges (u, v) with        */
/*     depth[v] = depth[u] + 1 of sigma[u] / sigma[v] * (1 + delta[v]),      */
/*     taken in reverse BFS order so that every delta[v] on the right is     */
/*     final (0 for unreachable vertices; delta[src] is computed the same    */
/*     way).                                                                */
/* Returns 0, 1 if some path count exceeds INT64_MAX (the counts are then    */
/* meaningless), or -1 on bad arguments / allocation failure.               */
/* ------------------------------------------------------------------------ */
int32_t orc_bc_source(int32_t n, const int32_t* R, const int32_t* C, int32_t src,
                      int32_t* depth, int64_t* sigma, double* delta) {
  if (n <= 0 || src < 0 || src >= n) return -1;
  int32_t* order = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  if (!order) return -1;
  for (int32_t v = 0; v < n; ++v) { depth[v] = -1; sigma[v] = 0; delta[v] = 0.0; }
  int32_t ovf = 0;
  int64_t head = 0, tail = 0;
  depth[src] = 0;
  sigma[src] = 1;
  order[tail++] = src;
  while (head < tail) {                      /* forward pass: FIFO BFS order */
    int32_t u = order[head++];
    for (int64_t e = R[u]; e < R[u + 1]; ++e) {
      int32_t v = C[e];
      if (depth[v] == -1) { depth[v] = depth[u] + 1; order[tail++] = v; }
      if (depth[v] == depth[u] + 1 && __builtin_add_overflow(sigma[v], sigma[u], &sigma[v]))
        ovf = 1;
    }
  }
  for (int64_t i = tail - 1; i >= 0; --i) {  /* backward pass: reverse BFS order */
    int32_t u = order[i];
    double d = 0.0;
    for (int64_t e = R[u]; e < R[u + 1]; ++e) {
      int32_t v = C[e];
      if (depth[v] == depth[u] + 1)
        d += ((double)sigma[u] / (double)sigma[v]) * (1.0 + delta[v]);
    }
    delta[u] = d;
  }
  free(order);
  return ovf;
}

/* BC over a set of sources: bc[v] = sum over the k sources s != v of the     */
/* dependency of s on v (ordered source/target pairs, Brandes' definition).  */
/* Returns 0, 1 on path-count overflow, -1 on bad arguments.                 */
int32_t orc_bc(int32_t n, const int32_t* R, const int32_t* C, const int32_t* srcs, int32_t k,
               double* bc) {
  if (n <= 0) return -1;
  int32_t* depth = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  int64_t* sigma = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  double* delta = (double*)malloc((size_t)n * sizeof(double));
  if (!depth || !sigma || !delta) { free(depth); free(sigma); free(delta); return -1; }
  for (int32_t v = 0; v < n; ++v) bc[v] = 0.0;
  int32_t rc = 0;
  for (int32_t i = 0; i < k && rc >= 0; ++i) {
    int32_t r = orc_bc_source(n, R, C, srcs[i], depth, sigma, delta);
    if (r < 0) { rc = -1; break; }
    if (r > 0) rc = 1;
    for (int32_t v = 0; v < n; ++v)
      if (v != srcs[i]) bc[v] += delta[v];
  }
  free(depth); free(sigma); free(delta);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Connected components (Sec. 6.4) of an undirected (symmetric) graph:       */
/* label[v] = the smallest vertex id of v's component.  Vertices are taken   */
/* in increasing id order; each unlabelled one starts a BFS that labels its  */
/* whole component with its own id, which is therefore the component's      */
/* smallest.  Returns the number of components, or -1 on allocation failure. */
/* ------------------------------------------------------------------------ */
int64_t orc_cc(int32_t n, const int32_t* R, const int32_t* C, int32_t* label) {
  int32_t* queue = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  if (!queue) return -1;
  for (int32_t v = 0; v < n; ++v) label[v] = -1;
  int64_t comps = 0;
  for (int32_t s = 0; s < n; ++s) {
    if (label[s] != -1) continue;
    ++comps;
    int64_t head = 0, tail = 0;
    label[s] = s;
    queue[tail++] = s;
    while (head < tail) {
      int32_t u = queue[head++];
      for (int64_t e = R[u]; e < R[u + 1]; ++e)
        if (label[C[e]] == -1) { label[C[e]] = s; queue[tail++] = C[e]; }
    }
  }
  free(queue);
  return comps;
}

/* ------------------------------------------------------------------------ */
/* Segmented intersection (Sec. 4.3): for every pair i, the ids present in   */
/* both neighbour lists N(a[i]) and N(b[i]) (rows sorted ascending without   */
/* duplicates), by a two-pointer merge.  counts[i] = size of pair i's        */
/* intersection; if out != NULL the intersections are written in pair order, */
/* each ascending, up to out_cap items.  Returns the total count.            */
/* ------------------------------------------------------------------------ */
int64_t orc_segmented_intersect(const int32_t* R, const int32_t* C, const int32_t* a,
                                const int32_t* b, int64_t len, int64_t* counts, int32_t* out,
                                int64_t out_cap) {
  int64_t total = 0;
  for (int64_t i = 0; i < len; ++i) {
    int64_t x = R[a[i]], xe = R[a[i] + 1], y = R[b[i]], ye = R[b[i] + 1], c = 0;
    while (x < xe && y < ye) {
      if (C[x] < C[y]) ++x;
      else if (C[y] < C[x]) ++y;
      else {
        if (out && total + c < out_cap) out[total + c] = C[x];
        ++c; ++x; ++y;
      }
    }
    counts[i] = c;
    total += c;
  }
  return total;
}

/* ------------------------------------------------------------------------ */
/* Triangle counting (Sec. 6.6), by the definition: every triangle           */
/* {u, v, w} of an undirected graph (u < v < w, all three edges present) is  */
/* counted once; per_vertex[x] = the number of triangles that contain x      */
/* (NULL allowed).  Neighbour lists of u are marked in a flag array; for     */
/* each v > u adjacent to u and each w > v adjacent to v, a marked w closes  */
/* a triangle.  Returns the number of triangles (-1 on allocation failure).  */
/* ------------------------------------------------------------------------ */
int64_t orc_triangles(int32_t n, const int32_t* R, const int32_t* C, int64_t* per_vertex) {
  uint8_t* mark = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
  if (!mark) return -1;
  if (per_vertex) for (int32_t v = 0; v < n; ++v) per_vertex[v] = 0;
  int64_t total = 0;
  for (int32_t u = 0; u < n; ++u) {
    for (int64_t e = R[u]; e < R[u + 1]; ++e) mark[C[e]] = 1;
    for (int64_t e = R[u]; e < R[u + 1]; ++e) {
      int32_t v = C[e];
      if (v <= u) continue;
      for (int64_t f = R[v]; f < R[v + 1]; ++f) {
        int32_t w = C[f];
        if (w <= v || !mark[w]) continue;
        ++total;
        if (per_vertex) { ++per_vertex[u]; ++per_vertex[v]; ++per_vertex[w]; }
      }
    }
    for (int64_t e = R[u]; e < R[u + 1]; ++e) mark[C[e]] = 0;
  }
  free(mark);
  return total;
}

/* ------------------------------------------------------------------------ */
/* Multisplit (the multi-level priority queue of Sec. 5.1.5 generalised to   */
/* K buckets): item v in [0, n) goes to bucket                               */
/*   b(v) = 0 if dist[v] < base, else min(K - 1, (dist[v] - base) / delta);  */
/* out = the items of bucket 0 in input order, then bucket 1, ..., and       */
/* bucket_len[j] = the number of items in bucket j.  Items outside [0, n)   */
/* are dropped.  Returns the number of items written.                        */
/* ------------------------------------------------------------------------ */
int64_t orc_multisplit(int32_t n, const int32_t* in, int64_t len, const uint32_t* dist,
                       uint32_t base, uint32_t delta, int32_t K, int32_t* out,
                       int64_t* bucket_len) {
  int64_t w = 0;
  for (int32_t j = 0; j < K; ++j) {
    bucket_len[j] = 0;
    for (int64_t i = 0; i < len; ++i) {
      int32_t v = in[i];
      if (v < 0 || v >= n) continue;
      uint32_t d = dist[v];
      uint64_t b = d < base ? 0 : (uint64_t)(d - base) / delta;
      if (b > (uint64_t)(K - 1)) b = (uint64_t)(K - 1);
      if ((int32_t)b != j) continue;
      out[w++] = v;
      ++bucket_len[j];
    }
  }
  return w;
}
