// Histogram-domain solve of HistRetinex on sm_103a: Algorithm 1 (Eq. 11-15), the enhanced
// histogram (Eq. 17-20) and the histogram-matching LUT (Sec. III.C, last paragraph).
//
// One CTA per image.  The K x K histogram count/location matrices of Eq. 6-7 are never
// materialised: they are rank one (R_i L_j / N) and the class of cell (i, j) is
// index(i, j) = round(i j / (K-1)) (i = reflectance bin, j = illumination bin).  With the
// weights of Eq. 11, K_ij = R_i L_j / P_k (P_k = class total), the sums of Eq. 13 and Eq. 12
// factor into
//     R'_i = ((R_i / N) sum_j L_j^2 q_idx(i,j) + beta G_i) / (sum_j L_j^2 / N^2 + beta)
//     L'_j = ((L_j / N) sum_i R'_i R_i q_idx(i,j) + alpha S_j) / (sum_i R'_i^2 / N^2 + alpha)
// with q_k = S_k / P_k.  Only cells whose reflectance and illumination bins are both occupied
// contribute (zero terms), so every sum runs over the compacted supports supp G x supp S.
//
// Arithmetic is FP64.  GB300 issues one 32-lane FP64 instruction per 64 cycles per SM
// sub-partition, so the work is cut into fixed-length pieces (kPiece cells, one lane each):
// every FP64 instruction carries 32 useful lanes and no dependency chain is longer than
// kPiece plus a short combine.  The summation order differs from a left-to-right loop; sums
// of non-negative terms then agree to a few ulps per term.
#include "hr_internal.cuh"

namespace hr {
namespace {

constexpr int NT = kSolveThreads;
constexpr int NW = NT / 32;

__device__ __forceinline__ int iceil_div(int a, int b) { return (a + b - 1) / b; }

// index(i, j) = floor((2 i j + K - 1) / (2 (K - 1))): nearest level to i j / (K - 1).
// n < 2^25 for K <= 4096, so a float quotient is within one of the true one.
__device__ __forceinline__ int class_index(int i, int j, int km1, float inv_d) {
  const int n = 2 * i * j + km1, d = 2 * km1;
  int q = __float2int_rz(__int2float_rn(n) * inv_d);
  const int r = n - q * d;
  q += (r < 0) ? -1 : (r >= d ? 1 : 0);
  return q;
}

// First illumination bin j with index(i, j) >= k.
__device__ __forceinline__ int jstart_index(int i, int k, int K) {
  if (k <= 0) return 0;
  if (i == 0) return K;
  const long long t = (long long)(2 * k - 1) * (K - 1);
  const long long v = (t + 2LL * i - 1) / (2LL * i);
  return v > K ? K : (int)v;
}

struct JsIndex {
  int K;
  __device__ int operator()(int i, int k) const { return jstart_index(i, k, K); }
};
struct JsTable {  // per-context table for index_1 (Eq. 19)
  const uint16_t* tab;
  int K;
  __device__ int operator()(int i, int k) const { return k >= K ? K : (int)tab[(size_t)i * (K + 1) + k]; }
};

// Deterministic block sum (fixed shuffle tree per warp, then over warps).
__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double r = l < NW ? red[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if (l == 0) red[NW] = r;
  }
  __syncthreads();
  return red[NW];
}

// Exclusive block scan of one unsigned per thread; *total gets the sum.
__device__ unsigned block_exscan(unsigned v, unsigned* red, unsigned* total) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  unsigned x = v;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned y = __shfl_up_sync(0xffffffffu, x, o);
    if (l >= o) x += y;
  }
  __syncthreads();
  if (l == 31) red[w] = x;
  __syncthreads();
  if (w == 0) {
    unsigned s = l < NW ? red[l] : 0u;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned y = __shfl_up_sync(0xffffffffu, s, o);
      if (l >= o) s += y;
    }
    if (l < NW) red[l] = s;
  }
  __syncthreads();
  const unsigned before = (w > 0 ? red[w - 1] : 0u) + x - v;
  *total = red[NW - 1];
  __syncthreads();
  return before;
}

// Exclusive scan of arr[0..n) in place (n <= K), returns the total.
__device__ unsigned block_exscan_array(unsigned* arr, int n, unsigned* red) {
  const int per = iceil_div(n, NT);
  const int b0 = threadIdx.x * per, b1 = min(n, b0 + per);
  unsigned s = 0;
  for (int i = b0; i < b1; ++i) s += arr[i];
  unsigned total;
  unsigned off = block_exscan(s, red, &total);
  for (int i = b0; i < b1; ++i) { unsigned v = arr[i]; arr[i] = off; off += v; }
  __syncthreads();
  return total;
}

// Builds the class-major cell list for the classes cls_level(c), c in [0, ncls): for each class
// the cells (a, b) with jstart(i, k) <= LJ[b] < jstart(i, k+1), rows a ascending, then b ascending,
// and cuts each class into pieces of at most kPiece cells.  Returns the number of pieces.
template <class JS, class CL>
__device__ int build_class_lists(int nR, int ncls, const uint16_t* RI, const uint16_t* posL, JS js, CL cls_level,
                                 unsigned* csize, unsigned* cstart, unsigned* pfirst, unsigned* pcount,
                                 unsigned* list, uint2* piece, unsigned* ured) {
  for (int c = threadIdx.x; c < ncls; c += NT) {
    const int k = cls_level(c);
    unsigned sz = 0;
    for (int a = 0; a < nR; ++a) {
      const int i = RI[a];
      sz += (unsigned)(posL[js(i, k + 1)] - posL[js(i, k)]);
    }
    csize[c] = sz;
    cstart[c] = sz;
    pcount[c] = (sz + kPiece - 1) / kPiece;
    pfirst[c] = pcount[c];
  }
  __syncthreads();
  block_exscan_array(cstart, ncls, ured);
  const unsigned npieces = block_exscan_array(pfirst, ncls, ured);
  for (int c = threadIdx.x; c < ncls; c += NT) {
    const int k = cls_level(c);
    unsigned pos = cstart[c];
    for (int a = 0; a < nR; ++a) {
      const int i = RI[a];
      const int lo = posL[js(i, k)], hi = posL[js(i, k + 1)];
      for (int b = lo; b < hi; ++b) list[pos++] = ((unsigned)a << 16) | (unsigned)b;
    }
    const unsigned sz = csize[c], p0 = pfirst[c], np = pcount[c];
    for (unsigned p = 0; p < np; ++p) {
      const unsigned len = min((unsigned)kPiece, sz - p * kPiece);
      piece[p0 + p] = make_uint2(cstart[c] + p * kPiece, len | ((unsigned)c << 16));
    }
  }
  __syncthreads();
  return (int)npieces;
}

// Sums the pieces p0 .. p0+np-1 of every class c in [0, ncls) and hands the total to emit(c, total).
// Classes with few pieces are summed by one lane each; larger ones by a whole warp (strided lane
// sums, then a fixed shuffle tree), so no FP64 chain is longer than about np/32 + 5.
template <class EMIT>
__device__ void combine_classes(const double* part, const unsigned* pfirst, const unsigned* pcount, int ncls,
                                EMIT emit) {
  constexpr unsigned kSmall = 4;
  for (int c = threadIdx.x; c < ncls; c += NT) {
    const unsigned p0 = pfirst[c], np = pcount[c];
    if (np > kSmall) continue;
    double s = 0.0;
    for (unsigned p = 0; p < np; ++p) s += part[p0 + p];
    emit(c, s);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int c = w; c < ncls; c += NW) {
    const unsigned p0 = pfirst[c], np = pcount[c];
    if (np <= kSmall) continue;
    double s = 0.0;
    for (unsigned p = l; p < np; p += 32) s += part[p0 + p];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (l == 0) emit(c, s);
  }
}

__global__ void __launch_bounds__(NT, 1) solve_kernel(SolveArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int K = A.K;
  const int tid = threadIdx.x;
  uint8_t* slot = A.slots + (size_t)blockIdx.x * A.slot_bytes;
  const SlotLayout& lay = A.lay;
  const unsigned* S = reinterpret_cast<const unsigned*>(slot + lay.S);
  const unsigned* G = reinterpret_cast<const unsigned*>(slot + lay.G);
  double* Rout = reinterpret_cast<double*>(slot + lay.R);
  double* Lout = reinterpret_cast<double*>(slot + lay.L);
  double* Tout = reinterpret_cast<double*>(slot + lay.T);
  uint16_t* lut = reinterpret_cast<uint16_t*>(slot + lay.lut);
  int* misc = reinterpret_cast<int*>(slot + lay.misc);
  unsigned* cls = reinterpret_cast<unsigned*>(slot + lay.cls);
  unsigned* list = reinterpret_cast<unsigned*>(slot + lay.list);
  uint2* piece = reinterpret_cast<uint2*>(slot + lay.piece);
  double* part = reinterpret_cast<double*>(slot + lay.part);

  // shared memory: index arrays, reduction scratch, then (optionally) the solver vectors
  uint16_t* RI = reinterpret_cast<uint16_t*>(smem);
  uint16_t* LJ = RI + K;
  uint16_t* posL = LJ + K;  // posL[j] = number of occupied S levels below j, j in [0, K]
  size_t off = ((size_t)(3 * K + 1) * sizeof(uint16_t) + 15) & ~(size_t)15;
  double* red = reinterpret_cast<double*>(smem + off);
  off += (NW + 2) * sizeof(double);
  unsigned* ured = reinterpret_cast<unsigned*>(smem + off);
  off += ((NW + 2) * sizeof(unsigned) + 15) & ~(size_t)15;
  double* vec = A.vec_in_smem ? reinterpret_cast<double*>(smem + off) : reinterpret_cast<double*>(slot + lay.vec);
  double* Rc = vec;           // R on supp G (compacted)
  double* Lc = vec + K;       // L on supp S (compacted)
  double* L2c = vec + 2 * K;  // L^2
  double* RRc = vec + 3 * K;  // R' R
  double* Ru = vec + 4 * K;   // Eq. 13 result before Eq. 15
  double* Lu = vec + 5 * K;   // Eq. 12 result before Eq. 14
  double* q = vec + 6 * K;    // S_k / P_k, level-indexed
  double* Sd = vec + 7 * K;   // S as double, level-indexed

  // ---- supports and N --------------------------------------------------------------------
  const int per = iceil_div(K, NT);
  const int k0 = tid * per, k1 = min(K, k0 + per);
  unsigned cr = 0, cl = 0, nsum = 0;
  for (int k = k0; k < k1; ++k) { cr += G[k] > 0u; cl += S[k] > 0u; nsum += S[k]; }
  unsigned nR, nL, Nu;
  unsigned offR = block_exscan(cr, ured, &nR);
  unsigned offL = block_exscan(cl, ured, &nL);
  block_exscan(nsum, ured, &Nu);
  for (int k = k0; k < k1; ++k) {
    if (G[k] > 0u) RI[offR++] = (uint16_t)k;
    posL[k] = (uint16_t)offL;
    if (S[k] > 0u) LJ[offL++] = (uint16_t)k;
    Sd[k] = (double)S[k];
    q[k] = 0.0;
  }
  if (tid == 0) posL[K] = (uint16_t)nL;
  __syncthreads();
  const double N = (double)Nu;
  const double NN = N * N;
  const int km1 = K - 1;
  const float inv_d = 1.0f / (float)(2 * km1);

  // ---- class-major cell list for the classes of Eq. 11 that matter (S_k > 0) --------------
  unsigned* csize = cls;
  unsigned* cstart = cls + K;
  unsigned* pfirst = cls + 2 * K;
  unsigned* pcount = cls + 3 * K;
  const int nP = build_class_lists(nR, nL, RI, posL, JsIndex{K}, [&](int c) { return (int)LJ[c]; }, csize, cstart,
                                   pfirst, pcount, list, piece, ured);

  for (int a = tid; a < (int)nR; a += NT) Rc[a] = (double)G[RI[a]];   // R^(0) = H_C(grad S)
  for (int b = tid; b < (int)nL; b += NT) Lc[b] = (double)S[LJ[b]];   // L^(0) = H_C(S)
  __syncthreads();

  const int nCa = iceil_div((int)nL, kPiece), nPA = (int)nR * nCa;
  const int nCb = iceil_div((int)nR, kPiece), nPB = (int)nL * nCb;
  int it = 0;
  for (; it < A.max_iter;) {
    // Eq. 11: class totals P_k over the class-major pieces, then q_k = S_k / P_k
    for (int p = tid; p < nP; p += NT) {
      const uint2 pc = piece[p];
      const unsigned len = pc.y & 0xffffu;
      double acc = 0.0;
      for (unsigned c = 0; c < len; ++c) {
        const unsigned cell = list[pc.x + c];
        acc = fma(Rc[cell >> 16], Lc[cell & 0xffffu], acc);
      }
      part[p] = acc;
    }
    __syncthreads();
    combine_classes(part, pfirst, pcount, (int)nL, [&](int c, double P) {
      const int k = LJ[c];
      q[k] = P > 0.0 ? Sd[k] / P : 0.0;
    });
    double sl2 = 0.0;
    for (int b = tid; b < (int)nL; b += NT) { const double l = Lc[b]; L2c[b] = l * l; sl2 = fma(l, l, sl2); }
    const double dR = block_sum(sl2, red) / NN + A.beta;   // (includes a __syncthreads)

    // Eq. 13: reflectance update, pieces over (row a, chunk of illumination bins)
    for (int p = tid; p < nPA; p += NT) {
      const int a = p / nCa, ch = p - a * nCa;
      const int i = RI[a];
      const int b0 = ch * kPiece, b1 = min((int)nL, b0 + kPiece);
      double acc = 0.0;
      for (int b = b0; b < b1; ++b) acc = fma(L2c[b], q[class_index(i, LJ[b], km1, inv_d)], acc);
      part[p] = acc;
    }
    __syncthreads();
    double sr2 = 0.0, sr = 0.0;
    for (int a = tid; a < (int)nR; a += NT) {
      double s = 0.0;
      for (int ch = 0; ch < nCa; ++ch) s += part[a * nCa + ch];
      const double r = Rc[a];
      const double ru = fma(r / N, s, A.beta * (double)G[RI[a]]) / dR;
      Ru[a] = ru;
      RRc[a] = ru * r;
      sr2 = fma(ru, ru, sr2);
      sr += ru;
    }
    const double dL = block_sum(sr2, red) / NN + A.alpha;
    const double sR = block_sum(sr, red);

    // Eq. 12: illumination update with the new R, pieces over (column b, chunk of reflectance bins)
    for (int p = tid; p < nPB; p += NT) {
      const int b = p / nCb, ch = p - b * nCb;
      const int j = LJ[b];
      const int a0 = ch * kPiece, a1 = min((int)nR, a0 + kPiece);
      double acc = 0.0;
      for (int a = a0; a < a1; ++a) acc = fma(RRc[a], q[class_index(RI[a], j, km1, inv_d)], acc);
      part[p] = acc;
    }
    __syncthreads();
    double sl = 0.0;
    for (int b = tid; b < (int)nL; b += NT) {
      double s = 0.0;
      for (int ch = 0; ch < nCb; ++ch) s += part[b * nCb + ch];
      const double l = Lc[b];
      const double lu = fma(l / N, s, A.alpha * Sd[LJ[b]]) / dL;
      Lu[b] = lu;
      sl += lu;
    }
    const double sL = block_sum(sl, red);

    // Eq. 15 and Eq. 14: renormalise to mass N; squared changes for the stopping rule
    double dr = 0.0, dl = 0.0;
    for (int a = tid; a < (int)nR; a += NT) {
      const double rn = (N * Ru[a]) / sR;
      const double d = rn - Rc[a];
      dr = fma(d, d, dr);
      Rc[a] = rn;
    }
    for (int b = tid; b < (int)nL; b += NT) {
      const double ln = (N * Lu[b]) / sL;
      const double d = ln - Lc[b];
      dl = fma(d, d, dl);
      Lc[b] = ln;
    }
    ++it;
    if (!A.fixed_iters) {
      const double DR = block_sum(dr, red);
      const double DL = block_sum(dl, red);
      if (DR <= A.eps && DL <= A.eps) break;
    } else {
      __syncthreads();
    }
  }

  // ---- Eq. 17-20: enhanced histogram through the index_1 class map ------------------------
  const int nPT = build_class_lists(nR, K, RI, posL, JsTable{A.jstart1, K}, [](int c) { return c; }, csize, cstart,
                                    pfirst, pcount, list, piece, ured);
  for (int p = tid; p < nPT; p += NT) {
    const uint2 pc = piece[p];
    const unsigned len = pc.y & 0xffffu;
    double acc = 0.0;
    for (unsigned c = 0; c < len; ++c) {
      const unsigned cell = list[pc.x + c];
      acc = fma(Rc[cell >> 16], Lc[cell & 0xffffu], acc);
    }
    part[p] = acc;
  }
  __syncthreads();
  double* T = L2c;  // reuse: level-indexed target (K entries)
  combine_classes(part, pfirst, pcount, K, [&](int c, double s) { T[c] = s / N; });  // count matrix carries 1/N (Eq. 6)
  __syncthreads();

  // ---- histogram matching LUT ---------------------------------------------------------------
  // CT = inclusive prefix sum of T (Hillis-Steele in place over K entries, per-thread chunks)
  {
    double* CT = RRc;  // reuse, K entries
    const int b0 = k0, b1 = k1;
    double s = 0.0;
    for (int k = b0; k < b1; ++k) { s += T[k]; CT[k] = s; }
    // scan of the per-thread chunk totals (NT values) in shared memory via red-like buffer in part
    double* tot = part;
    tot[tid] = s;
    __syncthreads();
    for (int o = 1; o < NT; o <<= 1) {
      double v = tid >= o ? tot[tid - o] : 0.0;
      __syncthreads();
      if (tid >= o) tot[tid] += v;
      __syncthreads();
    }
    const double before = tid > 0 ? tot[tid - 1] : 0.0;
    for (int k = b0; k < b1; ++k) CT[k] += before;
    __syncthreads();
    const double TT = CT[K - 1];
    // rhs(s) = CS(s) * TT with CS the exact integer cumulative count of S; lhs(z) = CT(z) * N.
    // Non-negative doubles order like their bit patterns; a running max makes lhs monotone so the
    // first z with lhs(z) >= rhs(s) is found by binary search.
    unsigned long long* lhs = reinterpret_cast<unsigned long long*>(Ru);  // K entries
    unsigned long long m = 0;
    for (int k = b0; k < b1; ++k) {
      const unsigned long long v = (unsigned long long)__double_as_longlong(CT[k] * N);
      m = v > m ? v : m;
      lhs[k] = m;
    }
    unsigned long long* tmax = reinterpret_cast<unsigned long long*>(part);
    __syncthreads();
    tmax[tid] = m;
    __syncthreads();
    for (int o = 1; o < NT; o <<= 1) {
      unsigned long long v = tid >= o ? tmax[tid - o] : 0ull;
      __syncthreads();
      if (tid >= o && v > tmax[tid]) tmax[tid] = v;
      __syncthreads();
    }
    const unsigned long long pm = tid > 0 ? tmax[tid - 1] : 0ull;
    for (int k = b0; k < b1; ++k) lhs[k] = lhs[k] > pm ? lhs[k] : pm;
    // z_top: last occupied target level.  Where CS(s) = N the matching condition reads
    // CT(z) >= TT, which in exact arithmetic first holds at z_top; that level is used directly.
    int top_local = -1;
    for (int k = b0; k < b1; ++k)
      if (T[k] > 0.0) top_local = k;
    unsigned* ztop = ured + NW + 1;
    if (tid == 0) *ztop = 0u;
    __syncthreads();
    if (top_local >= 0) atomicMax(ztop, (unsigned)top_local);
    unsigned cs_local = 0;
    for (int k = b0; k < b1; ++k) cs_local += S[k];
    unsigned cs_total;
    unsigned cs = block_exscan(cs_local, ured, &cs_total);  // (synchronises: ztop is final)
    const int z_top = (int)*ztop;
    for (int k = b0; k < b1; ++k) {
      cs += S[k];
      if (cs == Nu) { lut[k] = (uint16_t)z_top; continue; }
      const unsigned long long rhs = (unsigned long long)__double_as_longlong((double)cs * TT);
      int lo = 0, hi = K - 1;  // lhs[K-1] >= rhs unless no z qualifies; then K-1
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (lhs[mid] >= rhs) hi = mid; else lo = mid + 1;
      }
      lut[k] = (uint16_t)lo;
    }
  }
  __syncthreads();

  // ---- results (level-indexed) ----------------------------------------------------------------
  for (int k = tid; k < K; k += NT) { Rout[k] = 0.0; Lout[k] = 0.0; Tout[k] = T[k]; }
  __syncthreads();
  for (int a = tid; a < (int)nR; a += NT) Rout[RI[a]] = Rc[a];
  for (int b = tid; b < (int)nL; b += NT) Lout[LJ[b]] = Lc[b];
  if (tid == 0) { misc[0] = it; misc[1] = (int)nR; misc[2] = (int)nL; misc[3] = nP; }
}

}  // namespace

size_t solve_smem_bytes(int K, int vec_in_smem) {
  size_t off = ((size_t)(3 * K + 1) * sizeof(uint16_t) + 15) & ~(size_t)15;
  off += (NW + 2) * sizeof(double);
  off += ((NW + 2) * sizeof(unsigned) + 15) & ~(size_t)15;
  if (vec_in_smem) off += (size_t)kSolveVecs * K * sizeof(double);
  return off;
}

cudaError_t launch_solve(const SolveArgs& a, int n, cudaStream_t st) {
  const size_t smem = solve_smem_bytes(a.K, a.vec_in_smem);
  cudaError_t e = cudaFuncSetAttribute(solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  solve_kernel<<<n, NT, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace hr
