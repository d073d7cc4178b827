/*
 * HistRetinex CPU oracle (FP64, single-threaded, plain loops).
 *
 * TEST INFRASTRUCTURE ONLY.  This file defines what the per-image HistRetinex pipeline
 * computes so that the CUDA path can be checked against it.  Only the test suite, the
 * package smoke check and the benchmark's CPU-baseline leg may build, load or call it;
 * the product path never does.  It shares no code, header, table or constant with the
 * CUDA library.
 *
 * Paper: Zhao et al., "HistRetinex: Optimizing Retinex model in Histogram Domain for
 * Efficient Low-Light Image Enhancement" (arXiv 2510.21100).
 *
 * Pipeline (each stage cites the passage it follows):
 *   1. S = value channel of HSV, V = max(r, g, b)                      Sec. II preamble
 *   2. H_C(S): count histogram of V, K bins                             Eq. 3
 *      H_C(grad S): count histogram of the gradient image of V         Sec. III.B, Alg. 1
 *   3. Two-level optimisation: Eq. 11 weights, Eq. 13 (R), Eq. 12 (L),
 *      Eq. 14/15 renormalisation, repeated as in Algorithm 1           Sec. III.B
 *   4. Gamma on the illumination location histogram, new location
 *      matrix, index_1 and the enhanced histogram                       Eq. 17-20
 *   5. Histogram matching of V to that histogram, as a K-entry LUT      Sec. III.C (last paragraph)
 *   6. New V applied with hue and saturation kept                       Sec. II preamble, Sec. IV.A
 *
 * Readings of points the paper leaves open:
 *   - location histogram H_B(X)_k = k/(K-1); the "/N" printed in Eq. 7 and Eq. 8 is dropped
 *     (with it every product would round to level 0; Eq. 18 has no /N);
 *   - index(i,j): i is the reflectance bin, j the illumination bin (Eq. 10);
 *   - Eq. 12/13 are used as the stationary point of Eq. 10: the weight K_ij multiplies
 *     (the printed "/(N K_ij)" is not the minimiser of Eq. 10);
 *   - with K_ij = R_i L_j / P_k, P_k the class total of Eq. 11, the sums of Eq. 12/13
 *     factor as (R_i/N) sum_j L_j^2 q_idx and (L_j/N) sum_i R'_i R_i q_idx, q_k = S_k/P_k
 *     (q_k = 0 for an empty class);
 *   - L^(0) = H_C(S); the L update uses the new, not yet renormalised R (Algorithm 1 order);
 *   - gradient = 3x3 Sobel magnitude of integer V, replicate border, rounded half up and
 *     clipped to K-1;
 *   - matching LUT[s] = smallest z with CT(z) * N >= CS(s) * CT(K-1);
 *   - colour: out_c = round_half_up(c * V'/V), and (V', V', V') where V = 0;
 *   - binned data (K bins over M > K data levels, "l levels" of Sec. II): value v in bin
 *     v >> log2(M/K); bin k located at its centre value, normalised, (k w + (w-1)/2) / (M-1)
 *     (w = M/K); class maps as FP64 argmins over those locations; the gradient level clipped to
 *     M-1 and binned likewise; the new value keeps the pixel's place in its bin.
 *
 * Canonical FP64 evaluation: every sum runs in ascending index order (cells of the K x K
 * matrices in row-major order, row = reflectance bin), one IEEE operation per written
 * operation, fma() where written; a term with a zero factor is skipped.  All terms are
 * non-negative, so skipping zero terms does not change any sum.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_INVALID_ARG 1
#define ORC_ERR_RANGE 5

typedef struct {
  int K;            /* number of levels (bins) */
  double alpha;     /* weight of the illumination prior (Eq. 9) */
  double beta;      /* weight of the reflectance prior (Eq. 9) */
  double gamma;     /* gamma of Eq. 17 */
  double eps;       /* stopping threshold of Algorithm 1 */
  int max_iter;     /* T of Algorithm 1 */
  int fixed_iters;  /* nonzero: always run max_iter iterations */
  int variants;     /* ORC_VAR_* bits: the printed forms instead of the default readings */
  int levels;       /* M, the data's levels (a power of two >= K); 0 or K: one bin per level */
} orc_params;

/* Printed forms of three points the default readings settle otherwise (each selectable alone):
 *   ORC_VAR_PRINTED_UPDATE   Eq. 12 and Eq. 13 exactly as printed, the weight K_ij dividing;
 *   ORC_VAR_NEAREST_MATCH    histogram matching to the target level whose cumulative share is
 *                            nearest to the source level's (Sec. III.C names matching only);
 *   ORC_VAR_FORWARD_GRADIENT the gradient image as forward differences of V (Sec. III.B speaks
 *                            of "the gradient image" without naming an operator). */
#define ORC_VAR_PRINTED_UPDATE 1
#define ORC_VAR_NEAREST_MATCH 2
#define ORC_VAR_FORWARD_GRADIENT 4

/* ---------- Stage 1-2: value channel, Eq. 3 histogram, gradient histogram ---------- */

static unsigned px(const unsigned char* base, size_t pitch, int elem_bytes, int x, int y, int c) {
  const unsigned char* row = base + (size_t)y * pitch;
  if (elem_bytes == 1) return row[3 * (size_t)x + c];
  const unsigned char* p = row + 2 * (3 * (size_t)x + c);
  return (unsigned)p[0] | ((unsigned)p[1] << 8); /* little-endian uint16 */
}

/* V = max(r, g, b): the value channel of HSV (Sec. II preamble). */
static unsigned value_at(const unsigned char* base, size_t pitch, int eb, int x, int y) {
  unsigned r = px(base, pitch, eb, x, y, 0), g = px(base, pitch, eb, x, y, 1), b = px(base, pitch, eb, x, y, 2);
  unsigned v = r > g ? r : g;
  return v > b ? v : b;
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* floor(sqrt(m)) for m < 2^63, by bisection on integers. */
static uint64_t isqrt_u64(uint64_t m) {
  uint64_t lo = 0, hi = 3037000500ull; /* > sqrt(2^63) */
  while (lo < hi) {
    uint64_t mid = lo + (hi - lo + 1) / 2;
    if (mid * mid <= m) lo = mid; else hi = mid - 1;
  }
  return lo;
}

/* Gradient level of pixel (x,y): 3x3 Sobel on V with replicate border (forward = 0), or the
 * forward differences gx = V(x+1,y) - V(x,y), gy = V(x,y+1) - V(x,y) with replicate border
 * (forward = 1); magnitude sqrt(gx^2 + gy^2) rounded half up, clipped to K-1. */
static unsigned gradient_level(const unsigned* V, int W, int H, int x, int y, int K, int forward) {
#define VV(xx, yy) ((int64_t)V[(size_t)clampi((yy), 0, H - 1) * W + clampi((xx), 0, W - 1)])
  int64_t gx, gy;
  if (forward) {
    gx = VV(x + 1, y) - VV(x, y);
    gy = VV(x, y + 1) - VV(x, y);
  } else {
    gx = (VV(x + 1, y - 1) + 2 * VV(x + 1, y) + VV(x + 1, y + 1)) -
         (VV(x - 1, y - 1) + 2 * VV(x - 1, y) + VV(x - 1, y + 1));
    gy = (VV(x - 1, y + 1) + 2 * VV(x, y + 1) + VV(x + 1, y + 1)) -
         (VV(x - 1, y - 1) + 2 * VV(x, y - 1) + VV(x + 1, y - 1));
  }
#undef VV
  uint64_t m2 = (uint64_t)(gx * gx) + (uint64_t)(gy * gy);
  uint64_t n = isqrt_u64(m2);
  /* sqrt(m2) >= n + 1/2  <=>  m2 > n^2 + n  (integers) */
  uint64_t g = n + (m2 > n * n + n ? 1u : 0u);
  return g > (uint64_t)(K - 1) ? (unsigned)(K - 1) : (unsigned)g;
}

/* Value channel of the whole image; returns ORC_ERR_RANGE if any V >= K. */
int orc_value_channel(const void* in, int W, int H, size_t pitch, int elem_bytes, int K, unsigned* V) {
  if (!in || !V || W < 1 || H < 1 || (elem_bytes != 1 && elem_bytes != 2) || pitch < (size_t)3 * W * elem_bytes)
    return ORC_ERR_INVALID_ARG;
  int bad = 0;
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      unsigned v = value_at((const unsigned char*)in, pitch, elem_bytes, x, y);
      if (v >= (unsigned)K) bad = 1;
      V[(size_t)y * W + x] = v;
    }
  return bad ? ORC_ERR_RANGE : ORC_OK;
}

/* log2 of the bin width w = M / K (M, K powers of two, M >= K), or -1 if they do not qualify. */
static int bin_shift(int K, int M) {
  if (K < 2 || M < K || (K & (K - 1)) || (M & (M - 1))) return -1;
  int s = 0;
  while ((K << s) < M) ++s;
  return s;
}

/* H_C(S) (Eq. 3) and H_C(grad S) (gradient histogram, Alg. 1 initialisation) over K bins of the
 * data's M levels ("l levels", Sec. II preamble): a value v falls into bin v >> log2(M / K); the
 * gradient level (clipped to the data's range, M - 1) is binned the same way.  M = K: one bin per
 * level.  forward selects the forward-difference gradient (ORC_VAR_FORWARD_GRADIENT). */
int orc_histograms_b(const void* in, int W, int H, size_t pitch, int elem_bytes, int K, int M, int forward,
                     uint64_t* S, uint64_t* G) {
  const int sh = bin_shift(K, M);
  if (sh < 0 || !S || !G) return ORC_ERR_INVALID_ARG;
  unsigned* V = (unsigned*)malloc(sizeof(unsigned) * (size_t)W * (size_t)H);
  if (!V) return ORC_ERR_INVALID_ARG;
  int st = orc_value_channel(in, W, H, pitch, elem_bytes, M, V);
  if (st != ORC_OK) { free(V); return st; }
  memset(S, 0, sizeof(uint64_t) * (size_t)K);
  memset(G, 0, sizeof(uint64_t) * (size_t)K);
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      S[V[(size_t)y * W + x] >> sh] += 1;
      G[gradient_level(V, W, H, x, y, M, forward) >> sh] += 1;
    }
  free(V);
  return ORC_OK;
}

int orc_histograms_v(const void* in, int W, int H, size_t pitch, int elem_bytes, int K, int forward, uint64_t* S,
                     uint64_t* G) {
  return orc_histograms_b(in, W, H, pitch, elem_bytes, K, K, forward, S, G);
}

int orc_histograms(const void* in, int W, int H, size_t pitch, int elem_bytes, int K, uint64_t* S, uint64_t* G) {
  return orc_histograms_v(in, W, H, pitch, elem_bytes, K, 0, S, G);
}

/* Location of bin k (H_B, Sec. III.A) when K bins cover M data levels: the bin's centre value
 * normalised to [0, 1], (k w + (w - 1) / 2) / (M - 1) with w = M / K; for M = K this is k / (K - 1). */
double orc_bin_location(int k, int K, int M) {
  const int64_t w = M / K;
  return (double)(2 * (int64_t)k * w + w - 1) / (2.0 * (double)(M - 1));
}

/* The first k minimising |p - location(k)|: the locations ascend, so the minimum lies next to the
 * first location >= p; the few neighbours around it are compared in ascending order. */
static uint32_t nearest_bin(double p, int K, int M) {
  int lo = 0, hi = K;
  while (lo < hi) {
    const int mid = (lo + hi) / 2;
    if (orc_bin_location(mid, K, M) >= p) hi = mid; else lo = mid + 1;
  }
  const int a = lo - 2 < 0 ? 0 : lo - 2, b = lo + 1 > K - 1 ? K - 1 : lo + 1;
  int best = a;
  double bd = fabs(p - orc_bin_location(a, K, M));
  for (int k = a + 1; k <= b; ++k) {
    const double d = fabs(p - orc_bin_location(k, K, M));
    if (d < bd) { bd = d; best = k; }
  }
  return (uint32_t)best;
}

/* Class map of binned data: index(i,j) = argmin_k |H_B(R)_i H_B(L)_j - H_B(S)_k| (definition under
 * Eq. 10) with the bin locations above, first minimum; cmap[i * K + j]. */
int orc_class_table(int K, int M, uint32_t* cmap) {
  if (bin_shift(K, M) < 0 || !cmap) return ORC_ERR_INVALID_ARG;
  for (int i = 0; i < K; ++i) {
    const double li = orc_bin_location(i, K, M);
    for (int j = 0; j < K; ++j) cmap[(size_t)i * K + j] = nearest_bin(li * orc_bin_location(j, K, M), K, M);
  }
  return ORC_OK;
}

/* ---------- Stage 3: class map and the two-level optimisation ---------- */

/* index(i,j) = argmin_k |H_B(L,R)_ij - H_B(S)_k| with H_B(X)_k = k/(K-1)
 * (Eq. 10 and the definition below it).  The product of locations is
 * ij/(K-1)^2, so the nearest level is round(ij/(K-1)); K-1 is odd for K a power
 * of two, so there are no ties and the closed form below is exact. */
uint32_t orc_class_index(int K, int i, int j) {
  uint64_t km1 = (uint64_t)(K - 1);
  return (uint32_t)((2ull * (uint64_t)i * (uint64_t)j + km1) / (2ull * km1));
}

/* One iteration of Algorithm 1.
 * In:  S, G (counts), R, L (current histograms, R = H_C(R)^(t), L = H_C(L)^(t)).
 * Out: P (Eq. 11 class totals of the count matrix, times N), q (S_k / P_k),
 *      Ru, Lu (Eq. 13 and Eq. 12 results before renormalisation),
 *      Rn, Ln (Eq. 15 and Eq. 14 results).
 * Any output pointer except Rn, Ln may be NULL.  printed != 0 takes Eq. 13 and Eq. 12 as printed
 * (ORC_VAR_PRINTED_UPDATE): the weight K_ij divides the data term instead of multiplying it. */
/* The class of cell (i, j): the closed form, or the table of binned data. */
static uint32_t cell_class(const uint32_t* cmap, int K, int i, int j) {
  return cmap ? cmap[(size_t)i * K + j] : orc_class_index(K, i, j);
}

static int iterate_impl(const uint64_t* S, const uint64_t* G, int K, double alpha, double beta, int printed,
                        const uint32_t* cmap, const double* R, const double* L, double* P_out, double* q_out,
                        double* Ru_out, double* Lu_out, double* Rn, double* Ln) {
  if (K < 2 || !S || !G || !R || !L || !Rn || !Ln) return ORC_ERR_INVALID_ARG;
  uint64_t Nu = 0;
  for (int k = 0; k < K; ++k) Nu += S[k];
  const double N = (double)Nu;
  const double NN = N * N;
  double* P = (double*)calloc((size_t)K, sizeof(double));
  double* q = (double*)calloc((size_t)K, sizeof(double));
  double* L2 = (double*)calloc((size_t)K, sizeof(double));
  double* Ru = (double*)calloc((size_t)K, sizeof(double));
  double* RR = (double*)calloc((size_t)K, sizeof(double));
  double* Lu = (double*)calloc((size_t)K, sizeof(double));
  if (!P || !q || !L2 || !Ru || !RR || !Lu) { free(P); free(q); free(L2); free(Ru); free(RR); free(Lu); return ORC_ERR_INVALID_ARG; }

  /* Eq. 11: P_k = sum over the cells of class k of H_C(R)_i H_C(L)_j (row-major). */
  for (int i = 0; i < K; ++i) {
    if (R[i] == 0.0) continue;
    for (int j = 0; j < K; ++j) {
      if (L[j] == 0.0) continue;
      uint32_t k = cell_class(cmap, K, i, j);
      P[k] = fma(R[i], L[j], P[k]);
    }
  }
  for (int k = 0; k < K; ++k) q[k] = P[k] > 0.0 ? (double)S[k] / P[k] : 0.0;

  /* Eq. 13: reflectance update with K_ij = R_i L_j / P_idx(i,j). */
  double sL2 = 0.0;
  for (int j = 0; j < K; ++j) sL2 = fma(L[j], L[j], sL2);
  const double dR = sL2 / NN + beta;
  for (int j = 0; j < K; ++j) L2[j] = L[j] * L[j];
  if (printed) {
    /* Eq. 13 and Eq. 12 as printed:
     *   H_C(R)_i = (sum_j H_C(L)_j H_C(S)_idx(i,j) / (N K_ij) + beta H_C(grad S)_i) / (sum_j H_C(L)_j^2 / N^2 + beta)
     *   H_C(L)_j = (sum_i H_C(R)_i H_C(S)_idx(i,j) / (N K_ij) + alpha H_C(S)_j) / (sum_i H_C(R)_i^2 / N^2 + alpha)
     * with K_ij = H_C(L,R)_ij / (class total of H_C(L,R)) by Eq. 11 (H_C(L,R)_ij = R_i L_j / N, Eq. 6)
     * from the previous iterate, the new R in the L update (Algorithm 1 order); a cell whose
     * weight is zero contributes nothing (the printed quotient is undefined there). */
    for (int i = 0; i < K; ++i) {
      double A = 0.0;
      for (int j = 0; j < K; ++j) {
        const uint32_t k = cell_class(cmap, K, i, j);
        const double Kij = P[k] > 0.0 ? ((R[i] * L[j]) / N) / (P[k] / N) : 0.0;
        if (Kij == 0.0) continue;
        A += (L[j] * (double)S[k]) / (N * Kij);
      }
      Ru[i] = (A + beta * (double)G[i]) / dR;
    }
    double sR2p = 0.0;
    for (int i = 0; i < K; ++i) sR2p = fma(Ru[i], Ru[i], sR2p);
    const double dLp = sR2p / NN + alpha;
    for (int j = 0; j < K; ++j) {
      double B = 0.0;
      for (int i = 0; i < K; ++i) {
        const uint32_t k = cell_class(cmap, K, i, j);
        const double Kij = P[k] > 0.0 ? ((R[i] * L[j]) / N) / (P[k] / N) : 0.0;
        if (Kij == 0.0) continue;
        B += (Ru[i] * (double)S[k]) / (N * Kij);
      }
      Lu[j] = (B + alpha * (double)S[j]) / dLp;
    }
  }
  for (int i = 0; i < K && !printed; ++i) {
    double A = 0.0;
    for (int j = 0; j < K; ++j) {
      double qk = q[cell_class(cmap, K, i, j)];
      if (L2[j] == 0.0 || qk == 0.0) continue;
      A = fma(L2[j], qk, A);
    }
    Ru[i] = fma(R[i] / N, A, beta * (double)G[i]) / dR;
  }

  /* Eq. 12: illumination update with the new R and the same weights K_ij. */
  double sR2 = 0.0;
  for (int i = 0; i < K; ++i) sR2 = fma(Ru[i], Ru[i], sR2);
  const double dL = sR2 / NN + alpha;
  for (int i = 0; i < K; ++i) RR[i] = Ru[i] * R[i];
  for (int j = 0; j < K && !printed; ++j) {
    double B = 0.0;
    for (int i = 0; i < K; ++i) {
      double qk = q[cell_class(cmap, K, i, j)];
      if (RR[i] == 0.0 || qk == 0.0) continue;
      B = fma(RR[i], qk, B);
    }
    Lu[j] = fma(L[j] / N, B, alpha * (double)S[j]) / dL;
  }

  /* Eq. 15 and Eq. 14: renormalise both histograms to total mass N. */
  double sR = 0.0, sL = 0.0;
  for (int i = 0; i < K; ++i) sR += Ru[i];
  for (int j = 0; j < K; ++j) sL += Lu[j];
  for (int i = 0; i < K; ++i) Rn[i] = (N * Ru[i]) / sR;
  for (int j = 0; j < K; ++j) Ln[j] = (N * Lu[j]) / sL;

  if (P_out) memcpy(P_out, P, sizeof(double) * (size_t)K);
  if (q_out) memcpy(q_out, q, sizeof(double) * (size_t)K);
  if (Ru_out) memcpy(Ru_out, Ru, sizeof(double) * (size_t)K);
  if (Lu_out) memcpy(Lu_out, Lu, sizeof(double) * (size_t)K);
  free(P); free(q); free(L2); free(Ru); free(RR); free(Lu);
  return ORC_OK;
}

int orc_iterate_v(const uint64_t* S, const uint64_t* G, int K, double alpha, double beta, int printed,
                  const double* R, const double* L, double* P_out, double* q_out,
                  double* Ru_out, double* Lu_out, double* Rn, double* Ln) {
  return iterate_impl(S, G, K, alpha, beta, printed, NULL, R, L, P_out, q_out, Ru_out, Lu_out, Rn, Ln);
}

/* One iteration on binned data (M levels, K bins): the class map is the table of orc_class_table. */
int orc_iterate_b(const uint64_t* S, const uint64_t* G, int K, int M, double alpha, double beta, int printed,
                  const double* R, const double* L, double* P_out, double* q_out,
                  double* Ru_out, double* Lu_out, double* Rn, double* Ln) {
  if (bin_shift(K, M) < 0) return ORC_ERR_INVALID_ARG;
  uint32_t* cmap = NULL;
  if (M != K) {
    cmap = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)K * (size_t)K);
    if (!cmap) return ORC_ERR_INVALID_ARG;
    orc_class_table(K, M, cmap);
  }
  const int st = iterate_impl(S, G, K, alpha, beta, printed, cmap, R, L, P_out, q_out, Ru_out, Lu_out, Rn, Ln);
  free(cmap);
  return st;
}

int orc_iterate(const uint64_t* S, const uint64_t* G, int K, double alpha, double beta,
                const double* R, const double* L, double* P_out, double* q_out,
                double* Ru_out, double* Lu_out, double* Rn, double* Ln) {
  return orc_iterate_v(S, G, K, alpha, beta, 0, R, L, P_out, q_out, Ru_out, Lu_out, Rn, Ln);
}

/* Algorithm 1: R^(0) = H_C(grad S), L^(0) = H_C(S); repeat the iteration until both
 * squared changes are <= eps, or max_iter iterations have run. */
int orc_solve(const uint64_t* S, const uint64_t* G, const orc_params* p, double* R, double* L, int* iters) {
  if (!p || p->K < 2 || p->max_iter < 1 || !(p->alpha > 0.0) || !(p->beta > 0.0)) return ORC_ERR_INVALID_ARG;
  const int K = p->K;
  uint64_t NS = 0, NG = 0;
  for (int k = 0; k < K; ++k) { NS += S[k]; NG += G[k]; }
  if (NS == 0 || NS != NG) return ORC_ERR_INVALID_ARG;
  double* Rn = (double*)malloc(sizeof(double) * (size_t)K);
  double* Ln = (double*)malloc(sizeof(double) * (size_t)K);
  if (!Rn || !Ln) { free(Rn); free(Ln); return ORC_ERR_INVALID_ARG; }
  /* binned data (p->levels = M > K): the class map of the bin locations, built once */
  const int M = p->levels > 0 ? p->levels : K;
  uint32_t* cmap = NULL;
  if (bin_shift(K, M) < 0) { free(Rn); free(Ln); return ORC_ERR_INVALID_ARG; }
  if (M != K) {
    cmap = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)K * (size_t)K);
    if (!cmap) { free(Rn); free(Ln); return ORC_ERR_INVALID_ARG; }
    orc_class_table(K, M, cmap);
  }
  for (int k = 0; k < K; ++k) { R[k] = (double)G[k]; L[k] = (double)S[k]; }
  int t = 0;
  while (t < p->max_iter) {
    iterate_impl(S, G, K, p->alpha, p->beta, (p->variants & ORC_VAR_PRINTED_UPDATE) != 0, cmap, R, L, NULL, NULL,
                 NULL, NULL, Rn, Ln);
    double dr = 0.0, dl = 0.0;
    for (int i = 0; i < K; ++i) { double d = Rn[i] - R[i]; dr = fma(d, d, dr); }
    for (int j = 0; j < K; ++j) { double d = Ln[j] - L[j]; dl = fma(d, d, dl); }
    memcpy(R, Rn, sizeof(double) * (size_t)K);
    memcpy(L, Ln, sizeof(double) * (size_t)K);
    ++t;
    if (!p->fixed_iters && dr <= p->eps && dl <= p->eps) break;
  }
  if (iters) *iters = t;
  free(Rn); free(Ln); free(cmap);
  return ORC_OK;
}

/* ---------- Stage 4: histogram reprocessing (Eq. 17-20) ---------- */

/* index_1(i,j) = argmin_k |Hbar_B(L)_j H_B(R)_i - H_B(S)_k| (Eq. 19), first minimum,
 * with Hbar_B(L)_j = (j/(K-1))^(1/gamma) (Eq. 17) and the location matrix of Eq. 18.
 * The distance |p - k/(K-1)| is unimodal in k (k/(K-1) and the subtraction are both
 * monotone under rounding), so the search only visits the neighbours of floor(p (K-1)). */
static uint32_t index1_of(int K, double p) {
  const double km1 = (double)(K - 1);
  long k0 = (long)floor(p * km1);
  long lo = k0 - 1 < 0 ? 0 : k0 - 1;
  long hi = k0 + 2 > K - 1 ? K - 1 : k0 + 2;
  if (lo > K - 1) lo = K - 1;
  if (hi < lo) hi = lo;
  long best = lo;
  double bd = fabs(p - (double)lo / km1);
  for (long k = lo + 1; k <= hi; ++k) {
    double d = fabs(p - (double)k / km1);
    if (d < bd) { bd = d; best = k; }
  }
  return (uint32_t)best;
}

int orc_index1_table(int K, double gamma, uint32_t* idx1) {
  if (K < 2 || !(gamma > 0.0) || !idx1) return ORC_ERR_INVALID_ARG;
  const double km1 = (double)(K - 1);
  const double inv_g = 1.0 / gamma;
  for (int i = 0; i < K; ++i) {
    const double hr = (double)i / km1;                /* H_B(R)_i */
    for (int j = 0; j < K; ++j) {
      const double hl = pow((double)j / km1, inv_g);  /* Hbar_B(L)_j, Eq. 17 */
      idx1[(size_t)i * K + j] = index1_of(K, hl * hr);/* Eq. 18-19 */
    }
  }
  return ORC_OK;
}

/* index_1 of binned data (M levels, K bins): the same argmin over the bin locations,
 * idx1[i * K + j] = first k minimising |location(j)^(1/gamma) location(i) - location(k)|. */
int orc_index1_table_b(int K, int M, double gamma, uint32_t* idx1) {
  if (bin_shift(K, M) < 0 || !(gamma > 0.0) || !idx1) return ORC_ERR_INVALID_ARG;
  const double inv_g = 1.0 / gamma;
  for (int i = 0; i < K; ++i) {
    const double hr = orc_bin_location(i, K, M);                  /* H_B(R)_i */
    for (int j = 0; j < K; ++j) {
      const double hl = pow(orc_bin_location(j, K, M), inv_g);    /* Hbar_B(L)_j, Eq. 17 */
      idx1[(size_t)i * K + j] = nearest_bin(hl * hr, K, M);       /* Eq. 18-19 */
    }
  }
  return ORC_OK;
}

/* Eq. 20: H_C(S~)_k = sum over the cells with index_1 = k of the count matrix
 * H_C(R,L)_ij = R_i L_j / N (row-major sums, divided by N at the end). */
int orc_target_b(const double* R, const double* L, int K, int M, double gamma, uint64_t N, double* T) {
  if (K < 2 || !R || !L || !T || N == 0 || bin_shift(K, M) < 0) return ORC_ERR_INVALID_ARG;
  uint32_t* idx1 = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)K * (size_t)K);
  if (!idx1) return ORC_ERR_INVALID_ARG;
  int st = M == K ? orc_index1_table(K, gamma, idx1) : orc_index1_table_b(K, M, gamma, idx1);
  if (st != ORC_OK) { free(idx1); return st; }
  memset(T, 0, sizeof(double) * (size_t)K);
  for (int i = 0; i < K; ++i) {
    if (R[i] == 0.0) continue;
    for (int j = 0; j < K; ++j) {
      if (L[j] == 0.0) continue;
      uint32_t k = idx1[(size_t)i * K + j];
      T[k] = fma(R[i], L[j], T[k]);
    }
  }
  /* the count matrix carries a 1/N (Eq. 6): divide each class sum once */
  const double Nd = (double)N;
  for (int k = 0; k < K; ++k) T[k] = T[k] / Nd;
  free(idx1);
  return ORC_OK;
}

int orc_target(const double* R, const double* L, int K, double gamma, uint64_t N, double* T) {
  return orc_target_b(R, L, K, K, gamma, N, T);
}

/* ---------- Stage 5: histogram matching (Sec. III.C, last paragraph) ---------- */

/* LUT[s] = smallest z with CT(z) * N >= CS(s) * TT, where CS is the integer cumulative
 * count of S, CT the cumulative sum of the target (ascending), TT = CT(K-1); K-1 if none.
 * Where CS(s) = N the condition is CT(z) >= TT, which in exact arithmetic holds from the last
 * occupied target level z_top on; that level is used directly, because a running FP64 sum
 * can absorb trailing bins far below its ulp and reach TT earlier.
 * nearest != 0 (ORC_VAR_NEAREST_MATCH): LUT[s] = the first z minimising |CT(z) * N - CS(s) * TT|,
 * the target level whose cumulative share is nearest to the source level's (z_top where
 * CS(s) = N, as above). */
int orc_lut_v(const uint64_t* S, const double* T, int K, int nearest, uint16_t* lut) {
  if (K < 2 || K > 65536 || !S || !T || !lut) return ORC_ERR_INVALID_ARG;
  double* CT = (double*)malloc(sizeof(double) * (size_t)K);
  if (!CT) return ORC_ERR_INVALID_ARG;
  double c = 0.0;
  for (int z = 0; z < K; ++z) { c += T[z]; CT[z] = c; }
  const double TT = CT[K - 1];
  uint64_t N = 0;
  for (int k = 0; k < K; ++k) N += S[k];
  const double Nd = (double)N;
  int z_top = K - 1;
  while (z_top > 0 && !(T[z_top] > 0.0)) --z_top;
  uint64_t cs = 0;
  for (int s = 0; s < K; ++s) {
    cs += S[s];
    if (cs == N) { lut[s] = (uint16_t)z_top; continue; }
    const double rhs = (double)cs * TT;
    int z = 0;
    if (nearest) {
      double best = fabs(CT[0] * Nd - rhs);
      for (int zz = 1; zz < K; ++zz) {
        const double d = fabs(CT[zz] * Nd - rhs);
        if (d < best) { best = d; z = zz; }
      }
    } else {
      while (z < K - 1 && !(CT[z] * Nd >= rhs)) ++z;
    }
    lut[s] = (uint16_t)z;
  }
  free(CT);
  return ORC_OK;
}

int orc_lut(const uint64_t* S, const double* T, int K, uint16_t* lut) { return orc_lut_v(S, T, K, 0, lut); }

/* ---------- Stage 6: apply with hue and saturation kept ---------- */

/* V' = LUT[V]; each channel c becomes round_half_up(c * V' / V) = floor((2 c V' + V) / (2 V)),
 * which keeps the HSV hue and saturation of the pixel; a black pixel (V = 0) becomes grey V'. */
/* Binned data (M levels, K bins): the LUT maps bins, and the new value keeps the pixel's place in
 * its bin, V' = LUT[s] w + (V - s w) with s = V >> log2(w), w = M / K. */
int orc_apply_b(const void* in, void* out, int W, int H, size_t in_pitch, size_t out_pitch, int elem_bytes, int K,
                int M, const uint16_t* lut) {
  const int sh = bin_shift(K, M);
  if (!in || !out || !lut || W < 1 || H < 1 || (elem_bytes != 1 && elem_bytes != 2) || sh < 0)
    return ORC_ERR_INVALID_ARG;
  int bad = 0;
  for (int y = 0; y < H; ++y) {
    for (int x = 0; x < W; ++x) {
      const unsigned char* ib = (const unsigned char*)in;
      unsigned c[3];
      for (int ch = 0; ch < 3; ++ch) c[ch] = px(ib, in_pitch, elem_bytes, x, y, ch);
      unsigned V = c[0] > c[1] ? c[0] : c[1];
      V = V > c[2] ? V : c[2];
      if (V >= (unsigned)M) { bad = 1; V = (unsigned)M - 1; }
      const unsigned sbin = V >> sh;
      uint64_t Vp = ((uint64_t)lut[sbin] << sh) | (uint64_t)(V - (sbin << sh));
      unsigned o[3];
      for (int ch = 0; ch < 3; ++ch)
        o[ch] = V == 0 ? (unsigned)Vp : (unsigned)((2ull * c[ch] * Vp + V) / (2ull * V));
      unsigned char* ob = (unsigned char*)out + (size_t)y * out_pitch;
      for (int ch = 0; ch < 3; ++ch) {
        if (elem_bytes == 1) ob[3 * (size_t)x + ch] = (unsigned char)o[ch];
        else { ob[2 * (3 * (size_t)x + ch)] = (unsigned char)(o[ch] & 0xff); ob[2 * (3 * (size_t)x + ch) + 1] = (unsigned char)(o[ch] >> 8); }
      }
    }
  }
  return bad ? ORC_ERR_RANGE : ORC_OK;
}

int orc_apply(const void* in, void* out, int W, int H, size_t in_pitch, size_t out_pitch, int elem_bytes, int K,
              const uint16_t* lut) {
  return orc_apply_b(in, out, W, H, in_pitch, out_pitch, elem_bytes, K, K, lut);
}

/* ---------- Whole pipeline ---------- */

int orc_enhance(const void* in, void* out, int W, int H, size_t in_pitch, size_t out_pitch, int elem_bytes,
                const orc_params* p, uint64_t* S, uint64_t* G, double* R, double* L, double* T,
                uint16_t* lut, int* iters) {
  if (!p) return ORC_ERR_INVALID_ARG;
  const int K = p->K, M = p->levels > 0 ? p->levels : p->K;
  int st = orc_histograms_b(in, W, H, in_pitch, elem_bytes, K, M, (p->variants & ORC_VAR_FORWARD_GRADIENT) != 0, S, G);
  if (st != ORC_OK) return st;
  st = orc_solve(S, G, p, R, L, iters);
  if (st != ORC_OK) return st;
  st = orc_target_b(R, L, K, M, p->gamma, (uint64_t)W * (uint64_t)H, T);
  if (st != ORC_OK) return st;
  st = orc_lut_v(S, T, K, (p->variants & ORC_VAR_NEAREST_MATCH) != 0, lut);
  if (st != ORC_OK) return st;
  return orc_apply_b(in, out, W, H, in_pitch, out_pitch, elem_bytes, K, M, lut);
}
