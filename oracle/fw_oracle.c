/*
 * CPU oracle for all-pairs shortest paths by Floyd-Warshall.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it; the library never does.  It shares
 * no code, header or constant with the CUDA sources.
 *
 * Paper: Costanzo et al., "Comparison of HPC Architectures for Computing
 * All-Pairs Shortest Paths.  Intel Xeon Phi KNL vs NVIDIA Pascal" (arXiv 2105.07298).
 *
 * Conventions (readings of points the paper leaves open):
 *   - D is a dense n x n row-major matrix; D[i*n+j] is the length of the
 *     directed edge i -> j, +inf where there is none, 0 on the diagonal
 *     (§2.2 "FW Algorithm": a missing path has infinite distance; IEEE +inf
 *     is used so that inf + x = inf and every comparison is exact).
 *   - Algorithm 1 prints the test "D[i][j] >= D[i][k] + D[k][j]".  Taken with
 *     ">=", the step k = j (D[j][j] = 0) would set P[i][j] = j for every
 *     reachable pair and path reconstruction would never end.  The oracle uses
 *     the strict test "<"; the distances are the same under either test.
 *   - P[i][j] = -1 means "no intermediate vertex": the direct edge, i == j, or
 *     unreachable.  Otherwise P[i][j] = k, the intermediate vertex of the last
 *     strict improvement, and path(i,j) = path(i,k) ++ path(k,j).
 *
 * Parity pins (tests/test_oracle_pins.py): brute force (Dijkstra, Bellman-Ford,
 * simple-path enumeration), closed forms (chain, grid, complete, star, tree,
 * disconnected), invariants (zero diagonal, triangle inequality, D <= W,
 * reconstructed path weight = D), Johnson reweighting, blocked = classic at
 * TB = 1 and TB >= n, and finite differences for the gradient.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define EXPORT __attribute__((visibility("default")))

/* -------------------------------------------------------------------------
 * Classic Floyd-Warshall: Algorithm 1 (§2.2 "FW Algorithm"), strict "<".
 * D is updated in place (input = edge weights, output = distances).  P (may be
 * NULL) is fully written.  The i loop of one k step is split over threads:
 * row k and column k do not change during step k (D[k][k] = 0), so the rows
 * are independent and the result equals the sequential loop bit for bit.
 * k_end < n runs only the first k_end outer iterations (used to time a bounded
 * prefix of a large run; each outer iteration is n^2 relaxations).
 * ------------------------------------------------------------------------- */
#define DEFINE_FW(NAME, REAL)                                                        \
  EXPORT void NAME(REAL *D, int64_t n, int32_t *P, int64_t k_end) {                 \
    if (P)                                                                           \
      for (int64_t e = 0; e < n * n; ++e) P[e] = -1;                                 \
    if (k_end < 0 || k_end > n) k_end = n;                                           \
    for (int64_t k = 0; k < k_end; ++k) {                                            \
      _Pragma("omp parallel for schedule(static)")                                   \
      for (int64_t i = 0; i < n; ++i) {                                              \
        const REAL dik = D[i * n + k];                                               \
        for (int64_t j = 0; j < n; ++j) {                                            \
          const REAL cand = dik + D[k * n + j];                                      \
          if (cand < D[i * n + j]) {                                                 \
            D[i * n + j] = cand;                                                     \
            if (P) P[i * n + j] = (int32_t)k;                                        \
          }                                                                          \
        }                                                                            \
      }                                                                              \
    }                                                                                \
  }

DEFINE_FW(oracle_fw_f64, double)
DEFINE_FW(oracle_fw_f32, float)

/* -------------------------------------------------------------------------
 * Blocked Floyd-Warshall (§2.2 "Blocked FW Algorithm", Fig. 1).
 * D is split into TB x TB blocks; R = ceil(n / TB) rounds; round r runs
 *   phase 1: block (r,r) against itself,
 *   phase 2: blocks (r,J), J != r, against (r,r) and themselves,
 *   phase 3: blocks (I,r), I != r, against (r,r) and themselves,
 *   phase 4: blocks (I,J), I,J != r, against (I,r) and (r,J).
 * Inside every block the k loop runs over the vertices of block r in
 * ascending order with the same strict test as Algorithm 1.  When TB does not
 * divide n the last block row/column is simply shorter (the paper assumes
 * divisibility; a short block is the same as padding with isolated vertices).
 * ------------------------------------------------------------------------- */
#define DEFINE_BLOCK_UPDATE(NAME, REAL)                                              \
  static void NAME(REAL *D, int32_t *P, int64_t n, int64_t i0, int64_t i1,          \
                   int64_t j0, int64_t j1, int64_t k0, int64_t k1) {                 \
    for (int64_t k = k0; k < k1; ++k)                                                \
      for (int64_t i = i0; i < i1; ++i) {                                            \
        const REAL dik = D[i * n + k];                                               \
        for (int64_t j = j0; j < j1; ++j) {                                          \
          const REAL cand = dik + D[k * n + j];                                      \
          if (cand < D[i * n + j]) {                                                 \
            D[i * n + j] = cand;                                                     \
            if (P) P[i * n + j] = (int32_t)k;                                        \
          }                                                                          \
        }                                                                            \
      }                                                                              \
  }

DEFINE_BLOCK_UPDATE(block_update_f64, double)
DEFINE_BLOCK_UPDATE(block_update_f32, float)

#define DEFINE_BFW(NAME, REAL, UPD)                                                  \
  EXPORT int NAME(REAL *D, int64_t n, int64_t TB, int32_t *P) {                     \
    if (TB < 1) return 1;                                                            \
    if (P)                                                                           \
      for (int64_t e = 0; e < n * n; ++e) P[e] = -1;                                 \
    const int64_t R = (n + TB - 1) / TB;                                             \
    for (int64_t r = 0; r < R; ++r) {                                                \
      const int64_t k0 = r * TB, k1 = (k0 + TB < n) ? k0 + TB : n;                   \
      /* phase 1 */                                                                  \
      UPD(D, P, n, k0, k1, k0, k1, k0, k1);                                          \
      /* phase 2: row of blocks r */                                                 \
      _Pragma("omp parallel for schedule(dynamic)")                                  \
      for (int64_t J = 0; J < R; ++J) {                                              \
        if (J == r) continue;                                                        \
        const int64_t j0 = J * TB, j1 = (j0 + TB < n) ? j0 + TB : n;                 \
        UPD(D, P, n, k0, k1, j0, j1, k0, k1);                                        \
      }                                                                              \
      /* phase 3: column of blocks r */                                              \
      _Pragma("omp parallel for schedule(dynamic)")                                  \
      for (int64_t I = 0; I < R; ++I) {                                              \
        if (I == r) continue;                                                        \
        const int64_t i0 = I * TB, i1 = (i0 + TB < n) ? i0 + TB : n;                 \
        UPD(D, P, n, i0, i1, k0, k1, k0, k1);                                        \
      }                                                                              \
      /* phase 4: all remaining blocks */                                            \
      _Pragma("omp parallel for schedule(dynamic) collapse(2)")                      \
      for (int64_t I = 0; I < R; ++I)                                                \
        for (int64_t J = 0; J < R; ++J) {                                            \
          if (I == r || J == r) continue;                                            \
          const int64_t i0 = I * TB, i1 = (i0 + TB < n) ? i0 + TB : n;               \
          const int64_t j0 = J * TB, j1 = (j0 + TB < n) ? j0 + TB : n;               \
          UPD(D, P, n, i0, i1, j0, j1, k0, k1);                                      \
        }                                                                            \
    }                                                                                \
    return 0;                                                                        \
  }

DEFINE_BFW(oracle_bfw_f64, double, block_update_f64)
DEFINE_BFW(oracle_bfw_f32, float, block_update_f32)

/* -------------------------------------------------------------------------
 * Single-source brute force on the same weight matrix, independent of FW.
 * ------------------------------------------------------------------------- */

/* Dijkstra with an O(n^2) linear scan (non-negative weights).  dist has n
 * entries; unreachable vertices stay +inf. */
EXPORT void oracle_dijkstra_f64(const double *W, int64_t n, int64_t src, double *dist) {
  unsigned char *done = (unsigned char *)calloc((size_t)n, 1);
  for (int64_t v = 0; v < n; ++v) dist[v] = INFINITY;
  dist[src] = 0.0;
  for (int64_t it = 0; it < n; ++it) {
    int64_t u = -1;
    double best = INFINITY;
    for (int64_t v = 0; v < n; ++v)
      if (!done[v] && dist[v] < best) { best = dist[v]; u = v; }
    if (u < 0) break;
    done[u] = 1;
    for (int64_t v = 0; v < n; ++v) {
      const double w = W[u * n + v];
      if (v != u && w < INFINITY && best + w < dist[v]) dist[v] = best + w;
    }
  }
  free(done);
}

/* Dijkstra from several sources at once (threads over sources).  Rows of
 * out (n_src x n) follow srcs. W is float32 or float64 by is_f32. */
EXPORT void oracle_dijkstra_rows(const void *W, int is_f32, int64_t n, const int64_t *srcs,
                                 int64_t n_src, double *out) {
  _Pragma("omp parallel for schedule(dynamic)")
  for (int64_t s = 0; s < n_src; ++s) {
    double *dist = out + s * n;
    unsigned char *done = (unsigned char *)calloc((size_t)n, 1);
    for (int64_t v = 0; v < n; ++v) dist[v] = INFINITY;
    dist[srcs[s]] = 0.0;
    for (int64_t it = 0; it < n; ++it) {
      int64_t u = -1;
      double best = INFINITY;
      for (int64_t v = 0; v < n; ++v)
        if (!done[v] && dist[v] < best) { best = dist[v]; u = v; }
      if (u < 0) break;
      done[u] = 1;
      for (int64_t v = 0; v < n; ++v) {
        const double w = is_f32 ? (double)((const float *)W)[u * n + v]
                                : ((const double *)W)[u * n + v];
        if (v != u && w < INFINITY && best + w < dist[v]) dist[v] = best + w;
      }
    }
    free(done);
  }
}

/* Bellman-Ford from src (any sign of weights).  Returns 1 if a negative cycle
 * is reachable from src, else 0. */
EXPORT int oracle_bellman_ford_f64(const double *W, int64_t n, int64_t src, double *dist) {
  for (int64_t v = 0; v < n; ++v) dist[v] = INFINITY;
  dist[src] = 0.0;
  for (int64_t pass = 0; pass < n; ++pass) {
    int changed = 0;
    for (int64_t u = 0; u < n; ++u) {
      if (dist[u] == INFINITY) continue;
      for (int64_t v = 0; v < n; ++v) {
        const double w = W[u * n + v];
        if (u == v || w == INFINITY) continue;
        if (dist[u] + w < dist[v]) { dist[v] = dist[u] + w; changed = 1; }
      }
    }
    if (!changed) return 0;
    if (pass == n - 1) return 1;
  }
  return 0;
}

/* -------------------------------------------------------------------------
 * Path reconstruction from P: path(i,j) = [i, j] if P[i][j] = -1, else
 * path(i,k) ++ path(k,j) without repeating k.  Writes the vertex sequence
 * (i first, j last) into out and returns its length, or -1 if it exceeds
 * max_len (which a correct P never does for max_len >= n) or P does not
 * encode a path (a split index outside 0..ld-1, or a split that never ends).
 * ------------------------------------------------------------------------- */
static int64_t walk(const int32_t *P, int64_t ld, int64_t i, int64_t j, int64_t *out,
                    int64_t len, int64_t max_len, int64_t depth) {
  /* appends the vertices after i up to and including j; a valid P splits a
   * path of at most max_len vertices at most max_len levels deep, so deeper
   * recursion or an index outside 0..ld-1 means P encodes no path */
  if (depth > max_len) return -1;
  const int32_t k = P[i * ld + j];
  if (k < 0) {
    if (len >= max_len) return -1;
    out[len] = j;
    return len + 1;
  }
  if (k >= ld) return -1;
  len = walk(P, ld, i, k, out, len, max_len, depth + 1);
  if (len < 0) return -1;
  return walk(P, ld, k, j, out, len, max_len, depth + 1);
}

EXPORT int64_t oracle_reconstruct_path(const int32_t *P, int64_t ld, int64_t i, int64_t j,
                                       int64_t *out, int64_t max_len) {
  if (max_len < 1) return -1;
  out[0] = i;
  if (i == j) return 1;
  return walk(P, ld, i, j, out, 1, max_len, 0);
}

/* -------------------------------------------------------------------------
 * Gradient of the distances with respect to the edge weights (not in the
 * paper; an extension that keeps its arithmetic).  D[i][j] is the sum of the
 * weights on the shortest path that P encodes, so dD[i][j]/dW[u][v] is 1 when
 * the edge (u,v) lies on that path and 0 otherwise.  Hence
 *     gW[u][v] = sum over (i,j) with (u,v) on path(i,j) of gD[i][j].
 * gD, gW are n x n (gW fully written; diagonal, non-edges and unused edges get
 * 0).  Unreachable pairs (D = inf) contribute nothing.  Accumulates in fp64.
 * ------------------------------------------------------------------------- */
EXPORT int oracle_fw_backward_f64(const double *gD, const int32_t *P, const double *D,
                                  int64_t n, double *gW) {
  int64_t *buf = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int rc = 0;
  for (int64_t e = 0; e < n * n; ++e) gW[e] = 0.0;
  for (int64_t i = 0; i < n && !rc; ++i)
    for (int64_t j = 0; j < n; ++j) {
      if (i == j || !(D[i * n + j] < INFINITY)) continue;
      const int64_t len = oracle_reconstruct_path(P, n, i, j, buf, n + 1);
      if (len < 2) { rc = 1; break; }
      for (int64_t t = 0; t + 1 < len; ++t) gW[buf[t] * n + buf[t + 1]] += gD[i * n + j];
    }
  free(buf);
  return rc;
}

/* -------------------------------------------------------------------------
 * Bellman equations of sampled distance rows, for sizes where no whole-matrix
 * oracle fits in memory.  With positive weights and D[i][i] = 0, a row d is
 * the exact shortest-distance row of source i iff for every j != i
 *     d[j] = min over k != j of (d[k] + W[k][j])
 * (d[j] cannot be improved by any edge, and is attained through a
 * predecessor; by induction on d every finite d[j] is then the length of a
 * real path).  This accumulates the right-hand side over a chunk of weight
 * rows k0 .. k0+kc-1:
 *     best[t][j] = min(best[t][j], min over k in the chunk, k != j, of
 *                       Drows[t][k] + Wchunk[k - k0][j])      (in double)
 * Drows is s x n, Wchunk kc x n, best s x n (float32 inputs).
 * ------------------------------------------------------------------------- */
EXPORT void oracle_minplus_rows_f32(const float *Drows, int64_t s, int64_t n, const float *Wchunk, int64_t k0,
                                    int64_t kc, double *best) {
  _Pragma("omp parallel for schedule(static)")
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t t = 0; t < s; ++t) {
      double b = best[t * n + j];
      for (int64_t kk = 0; kk < kc; ++kk) {
        const int64_t k = k0 + kk;
        if (k == j) continue;
        const double c = (double)Drows[t * n + k] + (double)Wchunk[kk * n + j];
        if (c < b) b = c;
      }
      best[t * n + j] = b;
    }
  }
}

EXPORT int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
