/*
 * synth.c -- seeded synthetic inputs shaped like the paper's workloads.
 *
 * Holds none of the PageRank arithmetic: it only draws edge lists and update
 * batches.  It serves both the CPU oracle and the CUDA library (the one module
 * the two sides share).  Every draw comes from a counter-based generator, so
 * the same edges can also be produced on the GPU (synth_cuda.cu implements the
 * identical definitions for graphs too large to generate on the host):
 *
 *   mix64(z)   = the SplitMix64 output function (Steele, Lea, Flood 2014)
 *   draw(s, k, i) = mix64(mix64(s ^ (k << 56)) + i * 0x9E3779B97F4A7C15)
 *
 * Generators:
 *   sy_rmat      R-MAT (Chakrabarti, Zhan, Faloutsos 2004) with quadrant
 *                probabilities in parts per 10^4, ids relabelled by a seeded
 *                bijection of [0, 2^scale) so hubs do not cluster at id 0.
 *                Repeats and self-loops are left in; graph builders collapse
 *                them (set semantics) and add one self-loop per vertex.
 *   sy_batch     80/20-style random batch (Sec. 5.2.2 of the paper): uniform
 *                vertex-pair insertions (u != v), deletions drawn uniformly
 *                from a caller-given candidate edge list.
 *   sy_temporal  a temporal edge stream with repeats and a heavy-tailed
 *                degree distribution (copying / preferential attachment),
 *                standing in for the SNAP temporal graphs of Table 1.
 */
#include <stdint.h>
#include <stdlib.h>

/* Built with -fopenmp; the draws are counter-based, so the output does not
 * depend on the number of threads. */

static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

uint64_t sy_draw(uint64_t seed, uint64_t stream, uint64_t ctr) {
  return mix64(mix64(seed ^ (stream << 56)) + ctr * 0x9E3779B97F4A7C15ULL);
}

/* floor(u32 * range / 2^32) */
static uint32_t scale32(uint32_t u, uint32_t range) { return (uint32_t)(((uint64_t)u * range) >> 32); }
/* floor(u64 * range / 2^64) */
static uint64_t scale64(uint64_t u, uint64_t range) { return (uint64_t)(((unsigned __int128)u * range) >> 64); }

/* seeded bijection of [0, 2^s), 1 <= s <= 31 */
uint32_t sy_perm_pow2(uint32_t x, int s, uint64_t seed) {
  uint64_t mask = (1ULL << s) - 1;
  uint64_t k1 = (sy_draw(seed, 7, 0) | 1) & mask, k2 = sy_draw(seed, 7, 1) & mask;
  uint64_t k3 = (sy_draw(seed, 7, 2) | 1) & mask;
  int sh = (s + 1) / 2;
  uint64_t y = x;
  y = (y * k1) & mask;
  y ^= y >> sh;
  y = (y + k2) & mask;
  y = (y * k3) & mask;
  y ^= y >> sh;
  return (uint32_t)y;
}

/* seeded bijection of [0, n) by cycle-walking the power-of-two bijection */
uint32_t sy_perm(uint32_t x, uint32_t n, uint64_t seed) {
  int s = 1;
  while ((1ULL << s) < n) s++;
  uint32_t y = sy_perm_pow2(x, s, seed);
  while (y >= n) y = sy_perm_pow2(y, s, seed);
  return y;
}

void sy_rmat(int scale, int64_t m, uint64_t seed, int32_t a, int32_t b, int32_t c,
             int32_t *src, int32_t *dst) {
  uint64_t t1 = ((uint64_t)a << 32) / 10000;
  uint64_t t2 = ((uint64_t)(a + b) << 32) / 10000;
  uint64_t t3 = ((uint64_t)(a + b + c) << 32) / 10000;
  /* every edge depends only on its own counter: the threads of an OpenMP
   * build draw the same list */
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; e++) {
    uint32_t u = 0, v = 0;
    uint64_t w = 0;
    for (int l = 0; l < scale; l++) {
      if ((l & 1) == 0) w = sy_draw(seed, 1, (uint64_t)e * 16 + (uint64_t)(l >> 1));
      uint64_t r = (l & 1) ? (w >> 32) : (w & 0xffffffffULL);
      uint32_t rb, cb;
      if (r < t1) { rb = 0; cb = 0; }
      else if (r < t2) { rb = 0; cb = 1; }
      else if (r < t3) { rb = 1; cb = 0; }
      else { rb = 1; cb = 1; }
      u = (u << 1) | rb;
      v = (v << 1) | cb;
    }
    src[e] = (int32_t)sy_perm_pow2(u, scale, seed);
    dst[e] = (int32_t)sy_perm_pow2(v, scale, seed);
  }
}

void sy_batch(int32_t n, const int32_t *cand_src, const int32_t *cand_dst, int64_t n_cand,
              int64_t n_del, int64_t n_ins, uint64_t seed,
              int32_t *del_src, int32_t *del_dst, int32_t *ins_src, int32_t *ins_dst) {
  for (int64_t i = 0; i < n_del && n_cand > 0; i++) {
    uint64_t j = scale64(sy_draw(seed, 3, (uint64_t)i), (uint64_t)n_cand);
    del_src[i] = cand_src[j];
    del_dst[i] = cand_dst[j];
  }
  for (int64_t i = 0; i < n_ins; i++) {
    uint64_t w = sy_draw(seed, 2, (uint64_t)i);
    uint32_t u = scale32((uint32_t)(w >> 32), (uint32_t)n);
    uint32_t v = scale32((uint32_t)(w & 0xffffffffULL), (uint32_t)n);
    if (v == u) v = (u + 1) % (uint32_t)n;
    ins_src[i] = (int32_t)u;
    ins_dst[i] = (int32_t)v;
  }
}

/*
 * Temporal stream of m directed edges over n vertices.  Vertices become
 * active over time (vertex ids below n0 + (n-n0)(t+1)/m at step t, with
 * n0 = max(1, n/64) active from the start).  Each step
 * either repeats an earlier edge (probability p_rep / 2^32), or draws a new
 * pair whose source is uniform over active vertices with probability
 * q_src / 2^32 and otherwise copies the source of a uniformly chosen earlier
 * edge (preferential by out-degree); the target likewise by in-degree.  Ids
 * are relabelled by a seeded bijection of [0, n).
 */
void sy_temporal(int32_t n, int64_t m, uint64_t seed, uint32_t p_rep, uint32_t q_src, uint32_t q_dst,
                 int32_t *src, int32_t *dst) {
  for (int64_t t = 0; t < m; t++) {
    uint64_t w0 = sy_draw(seed, 4, 3 * (uint64_t)t);
    uint64_t w1 = sy_draw(seed, 4, 3 * (uint64_t)t + 1);
    uint64_t w2 = sy_draw(seed, 4, 3 * (uint64_t)t + 2);
    uint32_t n0 = n / 64 > 0 ? (uint32_t)(n / 64) : 1u;
    uint32_t active = n0 + (uint32_t)(((uint64_t)((uint32_t)n - n0) * (uint64_t)(t + 1)) / (uint64_t)m);
    if (t > 0 && (uint32_t)(w0 >> 32) < p_rep) {
      uint64_t j = scale64(w0 << 32 | (w1 & 0xffffffffULL), (uint64_t)t);
      src[t] = src[j];
      dst[t] = dst[j];
      continue;
    }
    uint32_t u, v;
    if (t == 0 || (uint32_t)(w1 >> 32) < q_src) u = scale32((uint32_t)w1, active);
    else u = (uint32_t)src[scale64(w1 << 32 | (w0 & 0xffffffffULL), (uint64_t)t)];
    if (t == 0 || (uint32_t)(w2 >> 32) < q_dst) v = scale32((uint32_t)w2, active);
    else v = (uint32_t)dst[scale64(w2 << 32 | (w0 >> 32), (uint64_t)t)];
    src[t] = (int32_t)u;
    dst[t] = (int32_t)v;
  }
  for (int64_t t = 0; t < m; t++) {
    src[t] = (int32_t)sy_perm((uint32_t)src[t], (uint32_t)n, seed);
    dst[t] = (int32_t)sy_perm((uint32_t)dst[t], (uint32_t)n, seed);
  }
}
