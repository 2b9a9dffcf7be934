/*
 * graphgen.c — seeded synthetic graph generators (R-MAT, 2-D grid), CSR
 * builder, edge weights and source sampling.
 *
 * This module holds no traversal arithmetic.  It only produces inputs, and
 * both the CPU oracle tests and the CUDA path consume what it writes.
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), used counter-style so the
 * result does not depend on the number of threads.
 *
 * Graph recipe (the paper's dataset rules, Sec. 7 "Datasets"):
 *   - R-MAT with edge factor ef and initiator (a, b, c, d): ef * 2^s draws,
 *     each draw descends s quadrant levels; no noise, no vertex permutation.
 *   - every graph is made undirected: both directions are stored,
 *     self-loops and duplicate edges are removed, rows are sorted ascending.
 *   - weights are uniform integers in [lo, hi], drawn once per undirected
 *     edge from a hash of (seed, min(u,v), max(u,v)), so w(u,v) == w(v,u).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static inline uint64_t gg_mix(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Next output of a SplitMix64 stream with state *s. */
static inline uint64_t gg_next(uint64_t* s) {
  uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Uniform integer in [0, range) from the high 32 bits of a 64-bit word. */
static inline uint32_t gg_below(uint64_t r, uint32_t range) {
  return (uint32_t)(((r >> 32) * (uint64_t)range) >> 32);
}

/* Hash of an undirected edge {u, v} under a seed. */
static inline uint64_t gg_edge_hash(uint64_t seed, int32_t u, int32_t v) {
  uint32_t lo = (uint32_t)(u < v ? u : v), hi = (uint32_t)(u < v ? v : u);
  return gg_mix(gg_mix(seed) ^ (((uint64_t)lo << 32) | hi));
}

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* Sort a small int32 array ascending: insertion sort below 32, else qsort. */
static void sort_row(int32_t* a, int64_t len) {
  if (len < 32) {
    for (int64_t i = 1; i < len; ++i) {
      int32_t x = a[i];
      int64_t j = i - 1;
      while (j >= 0 && a[j] > x) { a[j + 1] = a[j]; --j; }
      a[j + 1] = x;
    }
  } else {
    qsort(a, (size_t)len, sizeof(int32_t), cmp_i32);
  }
}

/*
 * Build a symmetric, self-loop-free, duplicate-free CSR with sorted rows from
 * an undirected edge list (src[i], dst[i]).  Writes R (n+1) and returns a
 * malloc'ed column array through *C_out (caller frees with gg_free).
 * Returns m (directed entries) or -1 on allocation failure.
 */
static int64_t build_csr(int32_t n, int64_t ne, const int32_t* src, const int32_t* dst,
                         int64_t* R, int32_t** C_out) {
  int64_t* deg = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!deg) return -1;
  for (int64_t i = 0; i < ne; ++i) {
    if (src[i] == dst[i]) continue;
    deg[src[i]]++;
    deg[dst[i]]++;
  }
  int64_t* off = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
  if (!off) { free(deg); return -1; }
  off[0] = 0;
  for (int32_t v = 0; v < n; ++v) off[v + 1] = off[v] + deg[v];
  int64_t tot = off[n];
  int32_t* tmp = (int32_t*)malloc((size_t)(tot > 0 ? tot : 1) * sizeof(int32_t));
  if (!tmp) { free(deg); free(off); return -1; }
  memcpy(deg, off, (size_t)n * sizeof(int64_t)); /* reuse as cursor */
  for (int64_t i = 0; i < ne; ++i) {
    int32_t u = src[i], v = dst[i];
    if (u == v) continue;
    tmp[deg[u]++] = v;
    tmp[deg[v]++] = u;
  }
  /* sort each row and drop duplicates in place; record unique counts */
#pragma omp parallel for schedule(dynamic, 1024)
  for (int32_t v = 0; v < n; ++v) {
    int32_t* row = tmp + off[v];
    int64_t len = off[v + 1] - off[v];
    sort_row(row, len);
    int64_t k = 0;
    for (int64_t j = 0; j < len; ++j)
      if (k == 0 || row[j] != row[k - 1]) row[k++] = row[j];
    deg[v] = k;
  }
  R[0] = 0;
  for (int32_t v = 0; v < n; ++v) R[v + 1] = R[v] + deg[v];
  int64_t m = R[n];
  int32_t* C = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
  if (!C) { free(deg); free(off); free(tmp); return -1; }
#pragma omp parallel for schedule(dynamic, 1024)
  for (int32_t v = 0; v < n; ++v)
    memcpy(C + R[v], tmp + off[v], (size_t)(R[v + 1] - R[v]) * sizeof(int32_t));
  free(deg); free(off); free(tmp);
  *C_out = C;
  return m;
}

/*
 * R-MAT (Chakrabarti, Zhan, Faloutsos 2004) with n = 2^scale vertices and
 * ef * n draws.  Draw i uses the SplitMix64 stream seeded with
 * mix(mix(seed) ^ i); each of the `scale` levels takes one 64-bit output and
 * compares its high 32 bits against floor(a*2^32), floor((a+b)*2^32),
 * floor((a+b+c)*2^32) to pick quadrant (0,0), (0,1), (1,0) or (1,1), where
 * the first coordinate is the row (source) bit.
 * Returns m, or -1 on failure; *C_out must be released with gg_free.
 */
int64_t gg_rmat(int32_t scale, int32_t ef, uint64_t seed, double a, double b, double c,
                int64_t* R, int32_t** C_out) {
  if (scale < 1 || scale > 30 || ef < 1) return -1;
  int32_t n = (int32_t)1 << scale;
  int64_t ne = (int64_t)ef * n;
  int32_t* src = (int32_t*)malloc((size_t)ne * sizeof(int32_t));
  int32_t* dst = (int32_t*)malloc((size_t)ne * sizeof(int32_t));
  if (!src || !dst) { free(src); free(dst); return -1; }
  const uint64_t two32 = (uint64_t)1 << 32;
  uint64_t tA = (uint64_t)(a * (double)two32);
  uint64_t tAB = (uint64_t)((a + b) * (double)two32);
  uint64_t tABC = (uint64_t)((a + b + c) * (double)two32);
  uint64_t key = gg_mix(seed);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < ne; ++i) {
    uint64_t s = gg_mix(key ^ (uint64_t)i);
    uint32_t u = 0, v = 0;
    for (int32_t l = 0; l < scale; ++l) {
      uint64_t r = gg_next(&s) >> 32;
      uint32_t rb, cb;
      if (r < tA) { rb = 0; cb = 0; }
      else if (r < tAB) { rb = 0; cb = 1; }
      else if (r < tABC) { rb = 1; cb = 0; }
      else { rb = 1; cb = 1; }
      u = (u << 1) | rb;
      v = (v << 1) | cb;
    }
    src[i] = (int32_t)u;
    dst[i] = (int32_t)v;
  }
  int64_t m = build_csr(n, ne, src, dst, R, C_out);
  free(src); free(dst);
  return m;
}

/*
 * W x W 4-neighbour grid, vertex id r*W + c.  Each undirected edge is deleted
 * with probability p_del (Bernoulli on the edge hash under `seed`), both
 * directions together.  Rows come out sorted (up, left, right, down).
 * Returns m, or -1 on failure.
 */
int64_t gg_grid(int32_t W, double p_del, uint64_t seed, int64_t* R, int32_t** C_out) {
  if (W < 1 || (int64_t)W * W > 0x7fffffffLL) return -1;
  int64_t n = (int64_t)W * W;
  uint64_t thr = (uint64_t)(p_del * 4294967296.0);
  /* keep flags for the right edge (bit 0) and down edge (bit 1) of each vertex */
  uint8_t* keep = (uint8_t*)malloc((size_t)n);
  if (!keep) return -1;
#pragma omp parallel for schedule(static)
  for (int64_t v = 0; v < n; ++v) {
    int32_t r = (int32_t)(v / W), c = (int32_t)(v % W);
    uint8_t k = 0;
    if (c + 1 < W && (gg_edge_hash(seed, (int32_t)v, (int32_t)(v + 1)) >> 32) >= thr) k |= 1;
    if (r + 1 < W && (gg_edge_hash(seed, (int32_t)v, (int32_t)(v + W)) >> 32) >= thr) k |= 2;
    keep[v] = k;
  }
  R[0] = 0;
  for (int64_t v = 0; v < n; ++v) {
    int32_t r = (int32_t)(v / W), c = (int32_t)(v % W);
    int64_t d = 0;
    if (r > 0 && (keep[v - W] & 2)) d++;
    if (c > 0 && (keep[v - 1] & 1)) d++;
    if (keep[v] & 1) d++;
    if (keep[v] & 2) d++;
    R[v + 1] = R[v] + d;
  }
  int64_t m = R[n];
  int32_t* C = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
  if (!C) { free(keep); return -1; }
#pragma omp parallel for schedule(static)
  for (int64_t v = 0; v < n; ++v) {
    int32_t r = (int32_t)(v / W), c = (int32_t)(v % W);
    int64_t p = R[v];
    if (r > 0 && (keep[v - W] & 2)) C[p++] = (int32_t)(v - W);
    if (c > 0 && (keep[v - 1] & 1)) C[p++] = (int32_t)(v - 1);
    if (keep[v] & 1) C[p++] = (int32_t)(v + 1);
    if (keep[v] & 2) C[p++] = (int32_t)(v + W);
  }
  free(keep);
  *C_out = C;
  return m;
}

/* Build a CSR from an arbitrary undirected edge list (see build_csr). */
int64_t gg_from_edges(int32_t n, int64_t ne, const int32_t* src, const int32_t* dst,
                      int64_t* R, int32_t** C_out) {
  for (int64_t i = 0; i < ne; ++i)
    if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n) return -1;
  return build_csr(n, ne, src, dst, R, C_out);
}

/* Symmetric weights in [lo, hi] for every directed CSR entry. */
void gg_weights(int32_t n, const int64_t* R, const int32_t* C, uint32_t lo, uint32_t hi,
                uint64_t seed, uint32_t* W) {
  uint32_t range = hi - lo + 1u;
#pragma omp parallel for schedule(dynamic, 4096)
  for (int32_t u = 0; u < n; ++u)
    for (int64_t e = R[u]; e < R[u + 1]; ++e)
      W[e] = lo + (range == 0 ? (uint32_t)(gg_edge_hash(seed, u, C[e]) >> 32)
                              : gg_below(gg_edge_hash(seed, u, C[e]), range));
}

/*
 * k distinct sources drawn uniformly over vertices with degree >= 1 by
 * rejection from the SplitMix64 stream seeded with `seed`.  Returns the
 * number written (less than k only if fewer candidates exist).
 */
int32_t gg_sources(int32_t n, const int64_t* R, int32_t k, uint64_t seed, int32_t* out) {
  int64_t cand = 0;
  for (int32_t v = 0; v < n; ++v) cand += (R[v + 1] > R[v]);
  if (k > cand) k = (int32_t)cand;
  uint8_t* taken = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
  if (!taken) return -1;
  uint64_t s = gg_mix(seed);
  int32_t got = 0;
  while (got < k) {
    int32_t v = (int32_t)gg_below(gg_next(&s), (uint32_t)n);
    if (R[v + 1] == R[v] || taken[v]) continue;
    taken[v] = 1;
    out[got++] = v;
  }
  free(taken);
  return got;
}

void gg_free(void* p) { free(p); }
