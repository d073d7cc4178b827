// Histogram-domain solve of HistRetinex on sm_103a: Algorithm 1 (Eq. 11-15), the enhanced
// histogram (Eq. 17-20) and the histogram-matching LUT (Sec. III.C, last paragraph).
//
// The K x K histogram count/location matrices of Eq. 6-7 are never materialised: they are
// rank one (R_i L_j / N) and the class of cell (i, j) is index(i, j) = round(i j / (K-1))
// (i = reflectance bin, j = illumination bin).  With the weights of Eq. 11,
// K_ij = R_i L_j / P_k (P_k = class total), the sums of Eq. 13 and Eq. 12 factor into
//     R'_i = ((R_i / N) sum_j L_j^2 q_idx(i,j) + beta G_i) / (sum_j L_j^2 / N^2 + beta)
//     L'_j = ((L_j / N) sum_i R'_i R_i q_idx(i,j) + alpha S_j) / (sum_i R'_i^2 / N^2 + alpha)
// with q_k = S_k / P_k.  Cells whose reflectance or illumination bin is empty contribute zero,
// so every sum runs over the compacted supports supp G x supp S.
//
// Arithmetic is FP64.  GB300 issues one 32-lane FP64 instruction per 64 cycles per SM
// sub-partition (an FP64 dependency chain costs 64 cycles a step), so the kernel keeps chains
// short and lanes full: class totals over fixed-length pieces of a class-major cell list,
// row and column sums over lane groups with shuffle trees, divisions as a hardware reciprocal
// estimate refined by two Newton steps.  One image runs on a cluster of C CTAs (C = 16 for a
// single image, C = 1 for batches): each CTA owns a slice of the classes, rows and columns,
// pushes its results into every CTA's shared memory (distributed shared memory) and meets the
// others at three cluster barriers per iteration.  The summation order differs from a
// left-to-right loop; sums of non-negative terms then agree to a few ulps per term.
#include <cooperative_groups.h>
#include <algorithm>
#include <atomic>
#include <type_traits>

#include "hr_internal.cuh"

namespace cg = cooperative_groups;

namespace hr {
namespace {

constexpr int NT = kSolveThreads;
constexpr int NW = NT / 32;
constexpr int kMaxCluster = 16;
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int iceil_div(int a, int b) { return (a + b - 1) / b; }

// x / d as x * (1/d): reciprocal estimate refined by two Newton steps (error about one ulp).
__device__ __forceinline__ double rcp64(double d) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
  double e = fma(-d, r, 1.0);
  r = fma(r, e, r);
  e = fma(-d, r, 1.0);
  return fma(r, e, r);
}

// a b + c and 1/d in the solver's arithmetic: FP64 (plain form), FP32 (reduced-precision form) or
// double-float.
__device__ __forceinline__ double fmaF(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmaF(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double rcpF(double d) { return rcp64(d); }
__device__ __forceinline__ float rcpF(float d) { return __frcp_rn(d); }

// Double-float arithmetic: a value is hi + lo, two FP32 numbers with |lo| <= ulp(hi) / 2,
// carried through error-free transformations (Dekker and Knuth: the exact rounding error of a
// sum from Knuth's two-sum, that of a product from one fused multiply-add).  Every operation
// keeps about 2^-47 relative accuracy on FP32's exponent range (all values of the solve lie
// between 1e-30 and 1e20 for images below 2^31 pixels).  GB300 runs FP32 at 64 times its FP64
// rate, so a dozen FP32 operations per step still outrun one FP64 operation.
struct df64 {
  float hi, lo;
  df64() = default;
  __device__ df64(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __device__ explicit df64(unsigned x) {
    hi = __uint2float_rz(x);                              // at most x, 24 significant bits
    lo = __uint2float_rn(x - (unsigned)hi);               // the rest is below 2^8: exact
  }
  __device__ df64(float h, float l) : hi(h), lo(l) {}
  __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ df64 df_norm(float s, float e) {  // |s| >= |e| (or s = 0)
  const float h = __fadd_rn(s, e);
  return df64(h, __fsub_rn(e, __fsub_rn(h, s)));
}
__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_norm(s, e);
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { a = a + b; return a; }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_norm(p, e);
}
__device__ __forceinline__ df64 fmaF(df64 a, df64 b, df64 c) {  // a b + c
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float s = __fadd_rn(p, c.hi);
  const float bb = __fsub_rn(s, p);
  float t = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bb)), __fsub_rn(c.hi, bb));
  t = __fadd_rn(t, __fadd_rn(e, c.lo));
  return df_norm(s, t);
}
__device__ __forceinline__ bool operator>(df64 a, df64 b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ bool operator<=(df64 a, df64 b) { return !(a > b); }
using ::__shfl_xor_sync;  // the built-in overloads stay visible beside the double-float one
__device__ __forceinline__ df64 __shfl_xor_sync(unsigned mask, df64 v, int o) {
  return df64(::__shfl_xor_sync(mask, v.hi, o), ::__shfl_xor_sync(mask, v.lo, o));
}
// 1/d: the correctly rounded FP32 reciprocal x, then one Newton step in double-float,
// x + x (1 - d x), whose residual is formed exactly enough by fused multiply-adds.
__device__ __forceinline__ df64 rcpF(df64 d) {
  const float x = __frcp_rn(d.hi);
  float r = __fmaf_rn(-d.hi, x, 1.0f);   // exact: 1 - d.hi x
  r = __fmaf_rn(-d.lo, x, r);
  return df_norm(x, __fmul_rn(x, r));
}

// index(i, j) = floor((2 i j + K - 1) / (2 (K - 1))): nearest level to i j / (K - 1).  The divisor
// d = 2 (K - 1) is fixed, so the quotient is a high multiply by M = ceil(2^(32+l) / d), l = floor(log2 d),
// and a shift (Granlund and Montgomery, division by invariant integers using multiplication): with
// e = M d - 2^(32+l) < d, n M / 2^(32+l) = n / d + n e / (d 2^(32+l)) stays below the next integer
// while n e < 2^(32+l), and n < 2 K^2, e < 2 K bound n e by 4 K^3, far below 2^(32+l) >= 2^31 d.
struct ClassDiv {
  unsigned m;
  int l;
  __device__ explicit ClassDiv(int km1) {
    const unsigned d = 2u * (unsigned)km1;
    l = 31 - __clz(d);
    m = (unsigned)(((1ull << (32 + l)) + d - 1) / d);  // < 2^32: d is not a power of two
  }
};
__device__ __forceinline__ int class_index(int i, int j, int km1, const ClassDiv& cd) {
  return (int)(__umulhi((unsigned)(2 * i * j + km1), cd.m) >> cd.l);
}

// First illumination bin j with index(i, j) >= k: ceil((2k-1)(K-1) / (2i)), at most K.
__device__ __forceinline__ int jstart_index(int i, int k, int K) {
  if (k <= 0) return 0;
  if (i == 0) return K;
  const int t = (2 * k - 1) * (K - 1), d = 2 * i;
  if (t > d * K) return K;
  int q = __float2int_rz(__fdividef(__int2float_rn(t), __int2float_rn(d)));  // within 1 of the quotient here
  int r = t - q * d;
  while (r < 0) { --q; r += d; }
  while (r >= d) { ++q; r -= d; }
  q += (r > 0);
  return q < K ? q : K;
}

// The same boundary for row a (level i = RI[a]) with the division exact through a per-row
// reciprocal: mg[a] = ceil(2^64 / (2 i)), so floor(t / (2 i)) = high 64 bits of t mg[a] for every
// t < 2^32 (the reciprocal's excess below 1 moves t mg[a] / 2^64 by under t / 2^64, less than the
// distance 1 / (2 i) from t / (2 i) to the next integer).  mg == nullptr: the float quotient.
struct JsIndex {
  int K;
  const uint16_t* RI;
  const unsigned long long* mg;
  const uint16_t* js0;  // binned data: the boundary table [K][K+1] of the class map (else nullptr)
  __device__ int operator()(int a, int k) const {
    const int i = RI[a];
    if (js0) return js0[(size_t)i * (K + 1) + k];
    if (!mg) return jstart_index(i, k, K);
    if (k <= 0) return 0;
    if (i == 0) return K;
    const unsigned t = (unsigned)((2 * k - 1) * (K - 1)), d = 2u * (unsigned)i;
    if (t > d * (unsigned)K) return K;
    unsigned q = (unsigned)__umul64hi((unsigned long long)t, mg[a]);
    q += (t - q * d) != 0u;  // ceil
    return q < (unsigned)K ? (int)q : K;
  }
};
// Exclusive block scan of one 64-bit value per thread; *total gets the sum.  r64 holds NW values.
__device__ unsigned long long block_exscan64(unsigned long long v, unsigned long long* r64,
                                             unsigned long long* total) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  unsigned long long x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(FULL, x, o);
    if (l >= o) x += y;
  }
  __syncthreads();
  if (l == 31) r64[w] = x;
  __syncthreads();
  if (w == 0) {
    unsigned long long s = l < NW ? r64[l] : 0ull;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(FULL, s, o);
      if (l >= o) s += y;
    }
    if (l < NW) r64[l] = s;
  }
  __syncthreads();
  const unsigned long long before = (w > 0 ? r64[w - 1] : 0ull) + x - v;
  *total = r64[NW - 1];
  __syncthreads();
  return before;
}

// Exclusive block scan of one unsigned per thread; *total gets the sum.
__device__ unsigned block_exscan(unsigned v, unsigned* red, unsigned* total) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  unsigned x = v;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned y = __shfl_up_sync(FULL, x, o);
    if (l >= o) x += y;
  }
  __syncthreads();
  if (l == 31) red[w] = x;
  __syncthreads();
  if (w == 0) {
    unsigned s = l < NW ? red[l] : 0u;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned y = __shfl_up_sync(FULL, s, o);
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

// Exclusive scan of arr[0..n) in place, returns the total.
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

// Number of i in [0, n) with f(i) true, over the block.
template <class F>
__device__ unsigned block_count(int n, F f, unsigned* red) {
  unsigned c = 0;
  for (int i = threadIdx.x; i < n; i += NT) c += f(i) ? 1u : 0u;
  unsigned total;
  block_exscan(c, red, &total);
  return total;
}

// Sum over the lanes of one warp (lane-strided, then a fixed shuffle tree); used from lane 0.
template <class Fn>
__device__ __forceinline__ auto warp_sum(int n, Fn f) -> decltype(f(0)) {
  const int l = threadIdx.x & 31;
  decltype(f(0)) s = 0;
  for (int i = l; i < n; i += 32) s += f(i);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
  return s;
}

// Copies arr[lo..hi) of this CTA into the same entries of every other CTA of the cluster; the
// (C-1) x n remote stores are spread over the whole block, one or two per thread.
template <typename T>
__device__ __forceinline__ void push_slice(const cg::cluster_group& cl, T* arr, int lo, int hi, int C, int rank) {
  const int n = hi - lo;
  if (C == 1 || n <= 0) return;
  for (int t = threadIdx.x; t < n * (C - 1); t += NT) {
    const int r0 = t / n, idx = lo + (t - r0 * n);
    const int r = r0 >= rank ? r0 + 1 : r0;
    cl.map_shared_rank(arr, r)[idx] = arr[idx];
  }
}

// Pull forms of the exchanges: after the cluster barrier that published the owners' entries, each
// CTA reads the entries it does not own straight from the owner's shared memory (one remote load
// per entry, all in flight together), instead of every owner storing into every peer before the
// barrier (remote stores before a barrier cost far more than remote loads after it on GB300).
// arr[map[c]] for c in [0, n), owned by owner[c].
template <typename T>
__device__ __forceinline__ void pull_mapped(const cg::cluster_group& cl, T* arr, const uint16_t* map, int n,
                                            const uint8_t* owner, int C, int rank) {
  if (C == 1) return;
  for (int c = threadIdx.x; c < n; c += NT) {
    const int r = owner[c];
    if (r != rank) {
      const int idx = map[c];
      arr[idx] = cl.map_shared_rank(arr, r)[idx];
    }
  }
}
// arr[0, n) split evenly: rank r owns [floor(n r / C), floor(n (r + 1) / C)).
template <typename T>
__device__ __forceinline__ void pull_even(const cg::cluster_group& cl, T* arr, int n, int C, int rank) {
  if (C == 1) return;
  for (int a = threadIdx.x; a < n; a += NT) {
    const int r = ((a + 1) * C - 1) / n;
    if (r != rank) arr[a] = cl.map_shared_rank(arr, r)[a];
  }
}

// Split cluster barrier: arrive (no ordering of this thread's memory accesses) and wait.  Every thread
// of every CTA alternates the two; a CTA whose shared memory others read arrives once they are done.
__device__ __forceinline__ void cluster_arrive_relaxed() { asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.aligned;" ::: "memory"); }

__device__ __forceinline__ long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Class-major cell lists.  For class c (level cls_level(c)), row a contributes the support
// columns b with jstart(i, k) <= LJ[b] < jstart(i, k+1).  Every CTA computes the sizes of all
// ncls classes (csz), their cell starts (cst) and piece starts (pst); each CTA then writes the
// cells and pieces of its own classes [cA, cB), a contiguous range balanced by cell count.
struct ClassPlan {
  int cA, cB;          // own classes
  unsigned pA, pB;     // own pieces
  unsigned cells;      // total cells over all classes
  unsigned cell0;      // first own cell (global class-major index)
  unsigned* listp;     // own cells, indexed by (cell - cell0)
  uint2* piecep;       // own pieces, indexed by (piece - pA)
  void* partp;         // own piece sums (solver arithmetic type), indexed by (piece - pbase)
  unsigned pbase;      // pA for shared-memory buffers, 0 for the global workspace
  bool glob;           // the lists are in the global workspace
};

// Own cell list, pieces and piece sums: shared-memory buffers when they fit, else the global
// workspace (same indexing either way).
struct OwnBufs {
  unsigned* s_list; uint2* s_piece; void* s_part;   // shared memory
  unsigned* g_list; uint2* g_piece; void* g_part;   // global workspace
};

template <class JS, class CL>
__device__ ClassPlan plan_classes(const cg::cluster_group& cl, int nR, int ncls, const uint16_t* RI,
                                  const uint16_t* posL, JS js, CL cls_level, unsigned* csz, unsigned* cst,
                                  unsigned* pst, const OwnBufs& ob, unsigned* ured, int rank, int C) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  // class sizes, split over the cluster (warp per class, lanes over rows), then gathered
  const int sA = (int)((long long)ncls * rank / C), sB = (int)((long long)ncls * (rank + 1) / C);
  for (int c = sA + w; c < sB; c += NW) {
    const int k = cls_level(c);
    unsigned s = 0;
#pragma unroll 4
    for (int a = l; a < nR; a += 32) {
      s += (unsigned)(posL[js(a, k + 1)] - posL[js(a, k)]);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if (l == 0) csz[c] = s;
  }
  __syncthreads();
  push_slice(cl, csz, sA, sB, C, rank);
  cl.sync();
  for (int c = threadIdx.x; c < ncls; c += NT) { cst[c] = csz[c]; pst[c] = (csz[c] + kPiece - 1) / kPiece; }
  __syncthreads();
  ClassPlan P;
  P.cells = block_exscan_array(cst, ncls, ured);
  const unsigned npieces = block_exscan_array(pst, ncls, ured);
  const unsigned lo = (unsigned)(((unsigned long long)P.cells * rank) / C);
  const unsigned hi = (unsigned)(((unsigned long long)P.cells * (rank + 1)) / C);
  P.cA = rank == 0 ? 0 : (int)block_count(ncls, [&](int c) { return cst[c] < lo; }, ured);
  P.cB = rank == C - 1 ? ncls : (int)block_count(ncls, [&](int c) { return cst[c] < hi; }, ured);
  if (P.cB < P.cA) P.cB = P.cA;
  P.pA = P.cA < ncls ? pst[P.cA] : npieces;
  P.pB = P.cB < ncls ? pst[P.cB] : npieces;
  P.cell0 = P.cA < ncls ? cst[P.cA] : P.cells;
  const unsigned cell1 = P.cB < ncls ? cst[P.cB] : P.cells;
  if (ob.s_list && cell1 - P.cell0 <= (unsigned)kListCap && P.pB - P.pA <= (unsigned)kPieceCap) {
    P.listp = ob.s_list; P.piecep = ob.s_piece; P.partp = ob.s_part;
  } else {
    P.listp = ob.g_list; P.piecep = ob.g_piece; P.partp = ob.g_part;  // whole-image indexing
    P.cell0 = 0;
  }
  P.pbase = (P.listp == ob.s_list) ? P.pA : 0u;
  P.glob = P.listp != ob.s_list;
  const unsigned pbase = P.pbase;
  for (int c = P.cA + w; c < P.cB; c += NW) {  // own cells: warp per class, lanes over rows
    if (csz[c] == 0) continue;
    const int k = cls_level(c);
    unsigned base = cst[c];
    for (int a0 = 0; a0 < nR; a0 += 32) {
      const int a = a0 + l;
      int lo_b = 0, cnt = 0;
      if (a < nR) {
        lo_b = posL[js(a, k)];
        cnt = posL[js(a, k + 1)] - lo_b;
      }
      unsigned x = (unsigned)cnt;
      for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(FULL, x, o);
        if (l >= o) x += y;
      }
      const unsigned at = base + x - (unsigned)cnt - P.cell0;
      for (int t = 0; t < cnt; ++t) P.listp[at + t] = ((unsigned)a << 16) | (unsigned)(lo_b + t);
      base += __shfl_sync(FULL, x, 31);
    }
    const unsigned np = (csz[c] + kPiece - 1) / kPiece;
    for (unsigned p = l; p < np; p += 32) {
      const unsigned len = min((unsigned)kPiece, csz[c] - p * kPiece);
      P.piecep[pst[c] + p - pbase] = make_uint2(cst[c] + p * kPiece - P.cell0, len | ((unsigned)c << 16));
    }
  }
  __syncthreads();
  return P;
}

// Sums the own pieces into the piece sums, then each own class's pieces; emit(c, total).
// Small classes are summed by one lane, larger ones by a warp (strided sums + shuffle tree).
template <typename F, class EMIT>
__device__ void class_totals(const ClassPlan& P, const unsigned* csz, const unsigned* pst, const F* Rc, const F* Lc,
                             EMIT emit) {
  F* part = static_cast<F*>(P.partp);
  const unsigned pbase = P.pbase;
  // Lists in the global workspace (large K) are read at the latency of global memory: the FP32
  // form keeps kU pieces per thread in flight (descriptors, then all their cells, then the sums).
  constexpr int kU = std::is_same<F, float>::value ? 4 : 1;
  if (kU > 1 && P.glob) {
    for (unsigned p0 = P.pA + threadIdx.x; p0 < P.pB; p0 += kU * NT) {
      uint2 pc[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const unsigned p = p0 + u * NT;
        pc[u] = p < P.pB ? P.piecep[p - pbase] : make_uint2(0u, 0u);
      }
      unsigned cl[kU][kPiece];
#pragma unroll
      for (int u = 0; u < kU; ++u)
#pragma unroll
        for (unsigned c = 0; c < (unsigned)kPiece; ++c) cl[u][c] = c < (pc[u].y & 0xffffu) ? P.listp[pc[u].x + c] : 0u;
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const unsigned len = pc[u].y & 0xffffu;
        F acc = 0;
#pragma unroll
        for (unsigned c = 0; c < (unsigned)kPiece; ++c)
          if (c < len) acc = fmaF(Rc[cl[u][c] >> 16], Lc[cl[u][c] & 0xffffu], acc);
        const unsigned p = p0 + u * NT;
        if (p < P.pB) part[p - pbase] = acc;
      }
    }
  } else {
    for (unsigned p = P.pA + threadIdx.x; p < P.pB; p += NT) {
      const uint2 pc = P.piecep[p - pbase];
      const unsigned len = pc.y & 0xffffu;
      const unsigned* cells = P.listp + pc.x;
      F acc = 0;
#pragma unroll
      for (unsigned c = 0; c < (unsigned)kPiece; ++c) {  // (all gathers of a piece in flight together)
        if (c < len) {
          const unsigned cell = cells[c];
          acc = fmaF(Rc[cell >> 16], Lc[cell & 0xffffu], acc);
        }
      }
      part[p - pbase] = acc;
    }
  }
  __syncthreads();
  constexpr unsigned kSmall = 4;
  for (int c = P.cA + threadIdx.x; c < P.cB; c += NT) {
    const unsigned np = (csz[c] + kPiece - 1) / kPiece;
    if (np > kSmall) continue;
    const F* ps = part + (pst[c] - pbase);
    F s = 0;
    for (unsigned p = 0; p < np; ++p) s += ps[p];
    emit(c, s);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int c = P.cA + w; c < P.cB; c += NW) {
    const unsigned np = (csz[c] + kPiece - 1) / kPiece;
    if (np <= kSmall) continue;
    const F* ps = part + (pst[c] - pbase);
    F s = 0;
    for (unsigned p = l; p < np; p += 32) s += ps[p];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if (l == 0) emit(c, s);
  }
}

// ---- Run sums (the FP32 form for large K, one CTA per image) -------------------------------------
// The cells of class k in row i are the support columns with levels in [js(i, k), js(i, k+1)) (a run),
// and row i meets the classes from index(i, jmin) to index(i, jmax) (jmin, jmax: the first and last
// support column).  A row sum over cells of (class weight) x (column weight) is then a sum over the
// row's runs of (class weight) x (the run's column-weight sum), a difference of two prefix sums of the
// column weights, indexed by level (zero weight at the levels outside the support, so an empty run
// adds exactly zero).  The class map is symmetric in i and j, so column sums are the same over row
// runs, and class totals scatter each row's run sums by class.  Prefix sums are double-float pairs: a
// difference loses nothing to cancellation (its error is a few units of the difference's last place
// plus 2^-48 of the prefix).  Runs are about a third of the cells at K = 4096, and no cell list is built.

__device__ __forceinline__ df64 shfl_up_df(df64 v, int o) {
  return df64(__shfl_up_sync(FULL, v.hi, o), __shfl_up_sync(FULL, v.lo, o));
}

// pre[p] = x(0) + ... + x(p - 1) for p in [0, n] as double-float (hi, lo) pairs; red holds NW values.
template <class X>
__device__ void prefix_df(int n, X x, float2* pre, df64* red) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int per = (n + NT - 1) / NT;
  const int b0 = min(n, (int)threadIdx.x * per), b1 = min(n, b0 + per);
  df64 s(0.f, 0.f);
  for (int b = b0; b < b1; ++b) s += df64(x(b), 0.f);
  df64 inc = s;
  for (int o = 1; o < 32; o <<= 1) {
    const df64 y = shfl_up_df(inc, o);
    if (l >= o) inc = inc + y;
  }
  df64 ex = shfl_up_df(inc, 1);
  if (l == 0) ex = df64(0.f, 0.f);
  __syncthreads();  // (the previous use of red is over)
  if (l == 31) red[w] = inc;
  __syncthreads();
  if (w == 0) {
    df64 t = l < NW ? red[l] : df64(0.f, 0.f);
    for (int o = 1; o < 32; o <<= 1) {
      const df64 y = shfl_up_df(t, o);
      if (l >= o) t = t + y;
    }
    if (l < NW) red[l] = t;
  }
  __syncthreads();
  df64 run = w > 0 ? red[w - 1] + ex : ex;
  for (int b = b0; b < b1; ++b) {
    pre[b] = make_float2(run.hi, run.lo);
    run += df64(x(b), 0.f);
  }
  if ((b0 < b1 && b1 == n) || (n == 0 && threadIdx.x == 0)) pre[n] = make_float2(run.hi, run.lo);
  __syncthreads();
}

// pre[p1] - pre[p0] (p1 >= p0) as a float.
__device__ __forceinline__ float run_sum(const float2* pre, int p0, int p1) {
  const float2 u = pre[p1], v = pre[p0];
  return __fadd_rn(__fsub_rn(u.x, v.x), __fsub_rn(u.y, v.y));
}

// The runs of classes [kA, kB] of line i (row i of the class map, or column i: the map is symmetric),
// by a whole warp: lane l takes the l-th of 32 contiguous blocks of the classes (of odd length, so
// per-class arrays read or updated by the lanes together fall in distinct banks) and calls f(k, s) for
// each of its classes k, s = pre[js(i, k + 1)] - pre[js(i, k)] (pre indexed by level).  The boundary
// js(i, k) = ceil(t / d), t = (2k - 1)(K - 1), d = 2i, is kept with its excess e = q d - t in [0, d)
// and advanced one class at a time (t grows by 2 (K - 1)) by integer steps: one division per lane and
// one per line, none per run, and a lane's loads for successive classes depend only on those steps.
// Line 0 holds one class, 0, over everything.
template <class Fn>
__device__ __forceinline__ void line_runs(int i, int kA, int kB, int K, const float2* pre, Fn f) {
  const int lane = threadIdx.x & 31;
  if (i == 0) {
    if (lane == 0 && kA == 0) f(0, run_sum(pre, 0, K));
    return;
  }
  // (an odd block length: the lanes' accesses to per-class arrays, per entries apart, fall in
  // distinct shared-memory banks)
  const int per = ((kB - kA + 32) >> 5) | 1;
  const int kS = kA + lane * per, kE = min(kB, kS + per - 1);
  if (kS > kE) return;
  const int km1 = K - 1, d = 2 * i;
  // quotients from a float estimate made exact by remainder corrections: dt < 2^13 and |t| < 2^26
  // (t / d < 2^17): the estimates are within 0.02 and within two of the exact values
  const float rd = __frcp_rn((float)d);
  const int dt = 2 * km1;
  int dq = __float2int_rz(__fmul_rn((float)dt, rd));
  dq += (dt - dq * d >= d) - (dt - dq * d < 0);
  const int dr = dt - dq * d;
  const int t = (2 * kS - 1) * km1;
  int q = __float2int_ru(__fmul_rn((float)t, rd));  // ceil(t / d), then e = q d - t in [0, d)
  int e = q * d - t;
  if (e < 0) { ++q; e += d; }
  if (e < 0) { ++q; e += d; }
  if (e >= d) { --q; e -= d; }
  if (e >= d) { --q; e -= d; }
  float2 u = pre[min(max(q, 0), K)];
#pragma unroll 4
  for (int k = kS; k <= kE; ++k) {
    const int x = dr - e;
    if (x > 0) { q += dq + 1; e = d - x; } else { q += dq; e = -x; }
    const float2 un = pre[min(q, K)];
    f(k, __fadd_rn(__fsub_rn(un.x, u.x), __fsub_rn(un.y, u.y)));  // (an empty run adds exactly 0)
    u = un;
  }
}

// Classes of index_1 met by row i, from its first (jmin) and last (jmax) support column: k0 + 1 =
// #{k < K : js1(i, k) <= jmin}, likewise k1 for jmax, capped at i (index_1 never exceeds i: a_j <= 1).
// js1 grows with k and js1(i, 0) = 0, so each count is found by a 32-ary search: the lanes probe 32
// boundaries stride apart, a ballot counts those within the column, the search continues from the
// last of them with a stride 32 times smaller (three rounds at K = 4096, one for K <= 32), both
// counts side by side.  The whole warp calls it.
__device__ __forceinline__ void index1_span(const uint16_t* jr, int K, int i, int jmin, int jmax, int& k0, int& k1) {
  const int lane = threadIdx.x & 31;
  int s0 = 0, s1 = 0, stride = 1;
  while (stride * 32 < K) stride *= 32;
  for (;;) {
    const int ka = s0 + lane * stride, kb = s1 + lane * stride;
    const int m0 = __popc(__ballot_sync(FULL, ka < K && (int)jr[ka] <= jmin));  // >= 1: the probe at s0
    const int m1 = __popc(__ballot_sync(FULL, kb < K && (int)jr[kb] <= jmax));
    if (stride == 1) {
      k0 = s0 + m0 - 1;
      k1 = min(s1 + m1 - 1, i);
      return;
    }
    s0 += (m0 - 1) * stride;
    s1 += (m1 - 1) * stride;
    stride /= 32;
  }
}

template <typename F>
__global__ void __launch_bounds__(NT, 1) solve_kernel(SolveArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ F conv[2][NW];
  __shared__ df64 dred[NW];  // (prefix sums of the run form)
  const cg::cluster_group cl = cg::this_cluster();
  pdl_wait();     // the histogram pass before it on the stream has finished
  pdl_trigger();  // the apply pass may be scheduled (it waits for this kernel)
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int K = A.K;
  const F alpha = (F)A.alpha, beta = (F)A.beta, eps = (F)A.eps;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int image = A.order ? A.order[blockIdx.x / C] : (int)(blockIdx.x / C);
  uint8_t* slot = A.slots + (size_t)image * A.slot_bytes;
  const SlotLayout& lay = A.lay;
  const unsigned* S = reinterpret_cast<const unsigned*>(slot + lay.S);
  const unsigned* G = reinterpret_cast<const unsigned*>(slot + lay.G);
  double* Rout = reinterpret_cast<double*>(slot + lay.R);
  double* Lout = reinterpret_cast<double*>(slot + lay.L);
  double* Tout = reinterpret_cast<double*>(slot + lay.T);
  uint16_t* lut = reinterpret_cast<uint16_t*>(slot + lay.lut);
  int* misc = reinterpret_cast<int*>(slot + lay.misc);
  long long* prof = reinterpret_cast<long long*>(slot + lay.misc + 16);
  const bool stamping = A.profile && rank == 0 && tid == 0;
  int nstamp = 0;
  auto stamp = [&]() { if (stamping && nstamp < kProfSlots) prof[nstamp++] = global_ns(); };
  if (stamping)
    for (int i = 0; i < kProfSlots; ++i) prof[i] = 0;
  stamp();

  // ---- shared memory ------------------------------------------------------------------------
  uint16_t* RI = reinterpret_cast<uint16_t*>(smem);   // occupied reflectance (gradient) levels
  uint16_t* LJ = RI + K;                                // occupied illumination (value) levels
  uint16_t* posL = LJ + K;                              // posL[j] = #occupied value levels below j
  size_t off = ((size_t)(3 * K + 1) * sizeof(uint16_t) + 15) & ~(size_t)15;
  unsigned* csz = reinterpret_cast<unsigned*>(smem + off); off += (size_t)K * 4;
  unsigned* cst = reinterpret_cast<unsigned*>(smem + off); off += (size_t)K * 4;
  unsigned* pst = reinterpret_cast<unsigned*>(smem + off); off += (size_t)K * 4;
  F* scal = reinterpret_cast<F*>(smem + off); off += 8 * sizeof(double);  // per-iteration scalars
  unsigned* ured = reinterpret_cast<unsigned*>(smem + off); off += ((NW + 2) * sizeof(unsigned) + 15) & ~(size_t)15;
  double* scr = reinterpret_cast<double*>(smem + off); off += NT * sizeof(double);   // LUT scans
  uint8_t* cowner = reinterpret_cast<uint8_t*>(smem + off); off += ((size_t)K + 15) & ~(size_t)15;  // class -> CTA
  OwnBufs ob;
  ob.s_part = nullptr; ob.s_piece = nullptr; ob.s_list = nullptr;
  if (A.list_in_smem) {  // (large K: the lists exceed any shared-memory share, so none is reserved)
    ob.s_part = smem + off; off += (size_t)kPieceCap * sizeof(F);
    ob.s_piece = reinterpret_cast<uint2*>(smem + off); off += (size_t)kPieceCap * sizeof(uint2);
    ob.s_list = reinterpret_cast<unsigned*>(smem + off); off += (size_t)kListCap * sizeof(unsigned);
  }
  ob.g_list = reinterpret_cast<unsigned*>(slot + lay.list);
  ob.g_piece = reinterpret_cast<uint2*>(slot + lay.piece);
  ob.g_part = slot + lay.part;
  F* vec = A.vec_in_smem ? reinterpret_cast<F*>(smem + off) : reinterpret_cast<F*>(slot + lay.vec);
  F* Rc = vec;           // H_C(R) on supp G (compacted)
  F* Lc = vec + K;       // H_C(L) on supp S (compacted)
  F* L2c = vec + 2 * K;  // L^2 (compacted); column sums of Eq. 12; the enhanced histogram at the end
  F* RRc = vec + 3 * K;  // R' R (compacted)
  F* Ru = vec + 4 * K;   // Eq. 13 before Eq. 15
  F* Lu = vec + 5 * K;   // Eq. 12 before Eq. 14
  F* q = vec + 6 * K;    // S_k / P_k (level-indexed)
  F* Sd = vec + 7 * K;   // S as F (level-indexed)
  // The run form (FP32, one CTA, the closed-form class map, K > 1024: the cell lists would not fit
  // shared memory) replaces the class plan and its lists; its double-float prefix sums and the
  // level -> row-position table posR take the plan's arrays csz, cst, pst (10 (K + 1) <= 12 K bytes).
  const bool runs = std::is_same<F, float>::value && C == 1 && !A.cmap && !A.printed && K > 1024;
  float2* pre = reinterpret_cast<float2*>(csz);
  uint16_t* posR = reinterpret_cast<uint16_t*>(reinterpret_cast<unsigned char*>(csz) + (size_t)(K + 1) * sizeof(float2));

  // ---- supports and N (every CTA) -------------------------------------------------------------
  const int per = iceil_div(K, NT);
  const int k0 = tid * per, k1 = min(K, k0 + per);
  unsigned cr = 0, cl_ = 0, nsum = 0;
  for (int k = k0; k < k1; ++k) { cr += G[k] > 0u; cl_ += S[k] > 0u; nsum += S[k]; }
  // the three counts in one 64-bit scan: support sizes in bits 0-15 and 16-31 (at most K <= 4096
  // each), pixels in bits 32-63
  unsigned long long tot64;
  const unsigned long long ex64 =
      block_exscan64(cr | ((unsigned long long)cl_ << 16) | ((unsigned long long)nsum << 32),
                     reinterpret_cast<unsigned long long*>(scr), &tot64);
  unsigned offR = (unsigned)(ex64 & 0xffffu), offL = (unsigned)((ex64 >> 16) & 0xffffu);
  const unsigned nRu = (unsigned)(tot64 & 0xffffu), nLu = (unsigned)((tot64 >> 16) & 0xffffu);
  const unsigned Nu = (unsigned)(tot64 >> 32);
  for (int k = k0; k < k1; ++k) {
    if (runs) posR[k] = (uint16_t)offR;
    if (G[k] > 0u) RI[offR++] = (uint16_t)k;
    posL[k] = (uint16_t)offL;
    if (S[k] > 0u) LJ[offL++] = (uint16_t)k;
    Sd[k] = (F)S[k];
    q[k] = 0.0;
  }
  if (tid == 0) posL[K] = (uint16_t)nLu;
  if (tid == 0 && runs) posR[K] = (uint16_t)nRu;
  __syncthreads();
  const int nR = (int)nRu, nL = (int)nLu;
  const F N = (F)Nu;
  const F invN = rcpF(N);
  const F invNN = rcpF(N * N);
  const int km1 = K - 1;
  const ClassDiv cdiv(km1);

  // ---- Eq. 11 classes that matter (S_k > 0): plan and own cell lists -------------------------
  cl.sync();  // every CTA of the cluster has started before any distributed shared memory access
  stamp();
  // per-row reciprocals of the Eq. 11 boundary division, in the LUT scan buffer (free until then),
  // for up to 512 rows (more rows: the FP32 quotient; a table in the workspace measured slower)
  unsigned long long* mg = nullptr;
  if (nR <= NT) mg = reinterpret_cast<unsigned long long*>(scr);
  if (mg) {
    for (int a = tid; a < nR; a += NT) mg[a] = RI[a] ? ~0ull / (2ull * RI[a]) + 1ull : 0ull;
    __syncthreads();
  }
  ClassPlan PP{};
  if (!runs)
    PP = plan_classes(cl, nR, nL, RI, posL, JsIndex{K, RI, mg, A.jstart0}, [&](int c) { return (int)LJ[c]; }, csz, cst,
                      pst, ob, ured, rank, C);
  stamp();
  // owner CTA of every class of the plan: rank r holds the classes whose first cell lies in
  // [cells r / C, cells (r + 1) / C) (rank 0 also those below, the last rank those above)
  if (!runs) {
    __shared__ unsigned rank_lo[kMaxCluster];
    if (tid < C) rank_lo[tid] = (unsigned)(((unsigned long long)PP.cells * tid) / C);
    __syncthreads();
    for (int c = tid; c < nL; c += NT) {
      int r = C - 1;
      while (r > 0 && cst[c] < rank_lo[r]) --r;
      cowner[c] = (uint8_t)r;
    }
  }
  // own rows and columns of the updates (contiguous slices)
  const int aA = (int)((long long)nR * rank / C), aB = (int)((long long)nR * (rank + 1) / C);
  const int bA = (int)((long long)nL * rank / C), bB = (int)((long long)nL * (rank + 1) / C);
  // Lanes per row in the Eq. 13 sums (GA) and per column in the Eq. 12 sums (GB).  A warp-wide FP64
  // instruction holds its SM sub-partition's FP64 pipe for about 64 cycles however many lanes are
  // active, while one lane's sum is a chain of dependent steps, so for a cluster CTA the choice
  // minimises the larger of the busiest sub-partition's FP64 cycles, ceil(warps / 4) x (terms per
  // lane + shuffle-tree levels) x 64, and a lane's chain.  A CTA alone (large batches: one image per
  // CTA, many rows each) uses 4.  (One image's arithmetic depends on C only through these group
  // sizes, the class split and the target's partial sums.)  Unrolling the Eq. 12/13 sums pays for
  // the double-float form (FP32 pipes) and costs the FP64 form more than it gains (measured on
  // GB300: 3.7 us per 7680x4320 image).
  constexpr int kSumUnroll = std::is_same<F, double>::value ? 1 : 4;
  auto group = [&](int own, int terms) {
    if (C == 1) return 4;
    int best = 32, cost = 1 << 30;
    for (int g = 4, lg = 2; g <= 32; g <<= 1, ++lg) {
      const int warps = (own * g + 31) / 32, t = (terms + g - 1) / g;
      const int pipe = ((warps + 3) / 4) * (t + lg) * 64;  // cycles of the busiest FP64 pipe
      const int chain = t * 110 + lg * 100;               // one lane's dependent steps
      const int c = pipe > chain ? pipe : chain;
      if (c < cost) { cost = c; best = g; }
    }
    return best;
  };
  const int GA = group(aB - aA, nL);
  const int GB = group(bB - bA, nR);

  for (int a = tid; a < nR; a += NT) Rc[a] = (F)G[RI[a]];   // R^(0) = H_C(grad S)
  for (int b = tid; b < nL; b += NT) Lc[b] = (F)S[LJ[b]];   // L^(0) = H_C(S)
  __syncthreads();

  // R = scR * R0 and L = scL * L0: the renormalisation of Eq. 15 / Eq. 14 is carried as two scales
  // into the next iteration (computed while its class totals run) instead of a separate pass.
  F* R0 = Rc;
  F* L0 = Lc;
  F* R1 = Ru;
  F* L1 = Lu;
  F scR = 1.0, scL = 1.0;  // R^(0) = H_C(grad S) and L^(0) = H_C(S) already have mass N
  int it = 0;
  while (it < A.max_iter) {
    // Eq. 11: class totals P_k of the own classes; q_k = S_k / P_k to every CTA.
    if (warp == NW - 1) {  // meanwhile: the L scale and 1 / denominator of Eq. 13 (every CTA alike)
      F s1 = 0.0, s2 = 0.0;
      for (int b = lane; b < nL; b += 32) { const F x = L0[b]; s1 += x; s2 = fmaF(x, x, s2); }
      for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(FULL, s1, o);
        s2 += __shfl_xor_sync(FULL, s2, o);
      }
      if (lane == 0) {
        const F sl = it == 0 ? 1.0 : N * rcpF(s1);
        scal[3] = sl;
        scal[0] = rcpF(fmaF(s2 * (sl * sl), invNN, beta));
      }  // (the second reciprocal needs the first: a chain)
    }
    // row weights of the Eq. 13 sums: L^2 (stationary point of Eq. 10), 1 (Eq. 13 as printed)
    if (!runs)
      for (int b = tid; b < nL; b += NT) { const F x = L0[b]; L2c[b] = A.printed ? (F)1.0 : x * x; }
    if (it == 1) stamp();
    if constexpr (std::is_same<F, float>::value) {
      if (runs) {
        // class totals from run sums, row by row: each warp adds R_i x (run sum of L) of its rows (every
        // NW-th), in order, into its partial totals, for CW = K / 4 classes at a time (the partials take the
        // four vectors free at this point, 4 warps x CW in each); the partials are summed in warp order
        for (int c = tid; c < nL; c += NT) RRc[c] = 0.f;  // (classes above every cell's class stay 0)
        prefix_df(K, [&](int j) { return posL[j + 1] > posL[j] ? L0[posL[j]] : 0.f; }, pre, dred);  // by level
        const int jmin = LJ[0], jmax = LJ[nL - 1];
        const int CW = K / 4;
        auto bufs = [&](int w) {  // (free until the new q is formed)
          const int b = w >> 2;
          return (b == 0 ? R1 : b == 1 ? L1 : b == 2 ? L2c : q) + (w & 3) * CW;
        };
        float* part = bufs(warp);
        const int kall = class_index(RI[nR - 1], jmax, km1, cdiv);  // the largest class of any cell
        for (int c0 = 0; c0 <= kall; c0 += CW) {
          for (int k = lane; k < CW; k += 32) part[k] = 0.f;
          __syncwarp();
          for (int a = warp; a < nR; a += NW) {  // (rows strided over the warps: their lengths grow with a)
            const int i = RI[a];
            const int kA = max(class_index(i, jmin, km1, cdiv), c0);
            const int kB = min(class_index(i, jmax, km1, cdiv), c0 + CW - 1);
            if (kA > kB) continue;
            const float r = R0[a];
            line_runs(i, kA, kB, K, pre, [&](int k, float sm) { part[k - c0] = fmaf(r, sm, part[k - c0]); });
            __syncwarp();  // (the next row's classes may fall to other lanes)
          }
          __syncthreads();
          for (int k = c0 + tid; k < min(c0 + CW, K); k += NT) {
            if (Sd[k] > 0.f) {
              float P = 0.f;
#pragma unroll
              for (int w = 0; w < NW; ++w) P += bufs(w)[k - c0];
              RRc[posL[k]] = P;
            }
          }
          __syncthreads();
        }
        for (int k = tid; k < K; k += NT) q[k] = 0.f;  // (the partials used it; classes with S_k = 0 keep q = 0)
      }
    }
    if (!runs) class_totals<F>(PP, csz, pst, R0, L0, [&](int c, F Pu) { RRc[c] = Pu; });  // (R'R is free until Eq. 13)
    __syncthreads();
    const int qc0 = runs ? 0 : PP.cA, qc1 = runs ? nL : PP.cB;
    for (int c = qc0 + tid; c < qc1; c += NT) {  // q of all own classes together (scal[3] is set)
      const int k = LJ[c];
      const F P = RRc[c] * (scR * scal[3]);
      // q_k = S_k / P_k; as printed the weight K_ij = R_i L_j / P_k divides, so q_k = S_k P_k
      q[k] = A.printed ? Sd[k] * P : (P > 0.0 ? Sd[k] * rcpF(P) : (F)0.0);
    }
    __syncthreads();
    if (it == 1) stamp();
    cl.sync();
    pull_mapped(cl, q, LJ, nL, cowner, C, rank);
    __syncthreads();
    scL = scal[3];
    if (it <= 1) stamp();

    // Eq. 13 for the own rows: lane groups of GA over the illumination bins.
    {
      const F rdR = scal[0], sl2 = A.printed ? (F)1.0 : scL * scL;
      if constexpr (std::is_same<F, float>::value) {
        if (runs) {  // a warp per row over its runs, column weights L^2 through their prefix sums
          prefix_df(K, [&](int j) { const float x = posL[j + 1] > posL[j] ? L0[posL[j]] : 0.f; return x * x; }, pre, dred);
          const int jmin = LJ[0], jmax = LJ[nL - 1];
          for (int a = warp; a < nR; a += NW) {
            const int i = RI[a];
            float acc = 0.f;
            line_runs(i, class_index(i, jmin, km1, cdiv), class_index(i, jmax, km1, cdiv), K, pre,
                      [&](int k, float sm) { acc = fmaf(q[k], sm, acc); });
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
            if (lane == 0) {
              const F r = scR * R0[a];
              const F ru = fmaF(r * invN, acc * sl2, beta * (F)G[i]) * rdR;
              R1[a] = ru;
              RRc[a] = ru * r;
            }
          }
        }
      }
      const int gi = lane / GA, gl = lane % GA, rpw = 32 / GA;
      for (int a0 = aA + warp * rpw; a0 < (runs ? aA : aB); a0 += NW * rpw) {
        const int a = a0 + gi;
        F acc = 0.0;
        if (a < aB) {
          const int i = RI[a];
          if (A.cmap) {  // binned data: the class map's table
            const uint16_t* crow = A.cmap + (size_t)i * K;
            for (int b = gl; b < nL; b += GA) acc = fmaF(L2c[b], q[crow[LJ[b]]], acc);
          } else {
#pragma unroll kSumUnroll
            for (int b = gl; b < nL; b += GA) acc = fmaF(L2c[b], q[class_index(i, LJ[b], km1, cdiv)], acc);
          }
        }
        for (int o = GA >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
        if (gl == 0 && a < aB) {
          // R'_i = ((R_i / N) sum_j L_j^2 q + beta G_i) / den; as printed ((1 / (N R_i)) sum_j S_k P_k + ...)
          const F r = scR * R0[a];
          const F rr = A.printed ? rcpF(r) : r;
          const F ru = fmaF(A.printed ? invN * rr : r * invN, acc * sl2, beta * (F)G[RI[a]]) * rdR;
          R1[a] = ru;
          RRc[a] = ru * rr;  // column weight of Eq. 12: R'_i R_i, as printed R'_i / R_i
        }
      }
    }
    __syncthreads();
    if (it == 1) stamp();
    cl.sync();
    pull_even(cl, R1, nR, C, rank);
    pull_even(cl, RRc, nR, C, rank);
    __syncthreads();
    if (it <= 1) stamp();

    // Eq. 12 for the own columns: lane groups of GB over the reflectance bins.
    if (warp == NW - 1) {  // meanwhile: 1 / denominator of Eq. 12 and the next R scale N / sum R'
      F s1 = 0.0, s2 = 0.0;
      for (int a = lane; a < nR; a += 32) { const F x = R1[a]; s1 += x; s2 = fmaF(x, x, s2); }
      for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(FULL, s1, o);
        s2 += __shfl_xor_sync(FULL, s2, o);
      }
      // the two reciprocals side by side in lanes 0 and 1 (one instruction stream)
      const F den = lane == 0 ? fmaF(s2, invNN, alpha) : s1;
      const F rd = rcpF(den);
      if (lane == 0) scal[1] = rd;
      if (lane == 1) scal[2] = N * rd;
    }
    {
      F* Bs = L2c;  // column sums (L^2 is not needed again in this iteration)
      if constexpr (std::is_same<F, float>::value) {
        if (runs) {  // a warp per column over its runs through the rows, row weights R' R by prefix sums
          prefix_df(K, [&](int i) { return posR[i + 1] > posR[i] ? RRc[posR[i]] : 0.f; }, pre, dred);  // by level
          const int imin = RI[0], imax = RI[nR - 1];
          for (int b = warp; b < nL; b += NW) {
            const int j = LJ[b];
            float acc = 0.f;
            line_runs(j, class_index(imin, j, km1, cdiv), class_index(imax, j, km1, cdiv), K, pre,
                      [&](int k, float sm) { acc = fmaf(q[k], sm, acc); });
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
            if (lane == 0) Bs[b] = acc;
          }
        }
      }
      const int gi = lane / GB, gl = lane % GB, cpw = 32 / GB;
      for (int b0 = bA + warp * cpw; b0 < (runs ? bA : bB); b0 += NW * cpw) {
        const int b = b0 + gi;
        F acc = 0.0;
        if (b < bB) {
          const int j = LJ[b];
          if (A.cmap) {
            for (int a = gl; a < nR; a += GB) acc = fmaF(RRc[a], q[A.cmap[(size_t)RI[a] * K + j]], acc);
          } else {
#pragma unroll kSumUnroll
            for (int a = gl; a < nR; a += GB) acc = fmaF(RRc[a], q[class_index(RI[a], j, km1, cdiv)], acc);
          }
        }
        for (int o = GB >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
        if (gl == 0 && b < bB) Bs[b] = acc;
      }
      __syncthreads();
      if (it == 1) stamp();
      const F rdL = scal[1];
      for (int b = bA + tid; b < bB; b += NT) {
        const F l = scL * L0[b];  // L'_j = ((L_j / N) B_j + alpha S_j) / den; as printed (B_j / (N L_j) + ...)
        L1[b] = fmaF(A.printed ? invN * rcpF(l) : l * invN, Bs[b], alpha * Sd[LJ[b]]) * rdL;
      }
    }
    __syncthreads();
    if (it == 1) stamp();
    cl.sync();
    pull_even(cl, L1, nL, C, rank);
    __syncthreads();
    if (it <= 1) stamp();

    const F scR1 = scal[2];
    ++it;
    bool done = false;
    if (!A.fixed_iters) {
      // squared changes of the renormalised histograms (identical data and order in every CTA)
      if (warp == 0) {
        const F s1 = warp_sum(nL, [&](int b) { return L1[b]; });
        if (lane == 0) scal[4] = N * rcpF(s1);
      }
      __syncthreads();
      const F scL1 = scal[4];
      F dr = 0.0, dl = 0.0;
      for (int a = tid; a < nR; a += NT) { const F d = scR1 * R1[a] - scR * R0[a]; dr = fmaF(d, d, dr); }
      for (int b = tid; b < nL; b += NT) { const F d = scL1 * L1[b] - scL * L0[b]; dl = fmaF(d, d, dl); }
      for (int o = 16; o > 0; o >>= 1) {
        dr += __shfl_xor_sync(FULL, dr, o);
        dl += __shfl_xor_sync(FULL, dl, o);
      }
      if (lane == 0) { conv[0][warp] = dr; conv[1][warp] = dl; }
      __syncthreads();
      F DR = 0.0, DL = 0.0;
      for (int w2 = 0; w2 < NW; ++w2) { DR += conv[0][w2]; DL += conv[1][w2]; }
      done = DR <= eps && DL <= eps;
    }
    F* t = R0; R0 = R1; R1 = t;
    t = L0; L0 = L1; L1 = t;
    scR = scR1;
    __syncthreads();
    stamp();
    if (done) break;
  }
  // Renormalised results of Algorithm 1 (Eq. 15 and Eq. 14 applied to the last iterate): R = scR R0
  // and L = sl L0 with sl = N / sum L0.  The target below is bilinear in R and L, so its row pass
  // runs on R0 and L0 while the last warp forms sl, and T takes the product of the scales at the end.
  if (warp == NW - 1) {
    const F s1 = warp_sum(nL, [&](int b) { return L0[b]; });
    if (lane == 0) scal[4] = N * rcpF(s1);
  }
  Rc = R0;
  Lc = L0;

  // ---- Eq. 17-20: enhanced histogram through the index_1 class map -----------------------------
  F* T = L2c;      // level-indexed enhanced histogram (rank 0)
  F sl = (F)0.0;   // the final L scale
  bool target_done = false;
  if constexpr (std::is_same<F, float>::value) {
    if (runs) {
      // run form: T_k = (1/N) sum_i R_i (run sum of L), the run sums from prefix sums of L, each
      // warp adding R_i x run sum of its own rows, in order, into partial targets for CW = K / 4
      // classes at a time (in the four vectors free until the LUT), summed in warp order; the
      // rows' class spans go where S as a float was (not needed again)
      uint16_t* rs0 = reinterpret_cast<uint16_t*>(Sd);
      uint16_t* rs1 = rs0 + K;
      prefix_df(K, [&](int j) { return posL[j + 1] > posL[j] ? Lc[posL[j]] : 0.f; }, pre, dred);  // by level
      sl = scal[4];
      const int jmin = LJ[0], jmax = LJ[nL - 1];
      for (int a = warp; a < nR; a += NW) {
        const int i = RI[a];
        int k0, k1;
        index1_span(A.jstart1 + (size_t)i * (K + 1), K, i, jmin, jmax, k0, k1);
        if (lane == 0) { rs0[a] = (uint16_t)k0; rs1[a] = (uint16_t)k1; }
      }
      __syncthreads();
      const int CW = K / 4;
      auto bufs = [&](int w) {
        const int b = w >> 2;
        return (b == 0 ? R1 : b == 1 ? L1 : b == 2 ? q : RRc) + (w & 3) * CW;
      };
      float* part = bufs(warp);
      const int kall = RI[nR - 1];  // (index_1 never exceeds i)
      int c0 = 0;
      for (; c0 <= kall; c0 += CW) {
        for (int k = lane; k < CW; k += 32) part[k] = 0.f;
        __syncwarp();
        for (int a = warp; a < nR; a += NW) {  // (rows strided over the warps: their lengths grow with a)
          const int kA = max((int)rs0[a], c0), kB = min((int)rs1[a], c0 + CW - 1);
          if (kA > kB) continue;
          const uint16_t* jr = A.jstart1 + (size_t)RI[a] * (K + 1);  // js1(i, k), k <= K (entry K holds K)
          const float r = Rc[a];
          // lane l: the l-th of 32 contiguous blocks of the classes, so its table loads for successive
          // classes are independent of each other (measured faster here than lanes over consecutive
          // classes, whose shared-memory updates avoid bank conflicts but whose loads wait in turn)
          const int per = ((kB - kA + 32) >> 5) | 1;  // (odd: the partials' banks differ)
          const int kS = kA + lane * per, kE = min(kB, kS + per - 1);
          if (kS <= kE) {
            float2 u = pre[jr[kS]];
#pragma unroll 4
            for (int k = kS; k <= kE; ++k) {
              const float2 un = pre[jr[k + 1]];
              part[k - c0] = fmaf(r, __fadd_rn(__fsub_rn(un.x, u.x), __fsub_rn(un.y, u.y)), part[k - c0]);
              u = un;
            }
          }
          __syncwarp();  // (the next row's classes may fall to other lanes)
        }
        __syncthreads();
        for (int k = c0 + tid; k < min(c0 + CW, K); k += NT) {
          float sum = 0.f;
#pragma unroll
          for (int w = 0; w < NW; ++w) sum += bufs(w)[k - c0];
          T[k] = sum;
        }
        __syncthreads();
      }
      const F tscale = invN * (scR * sl);  // the count matrix carries 1/N (Eq. 6); R and L their scales
      for (int k = tid; k < K; k += NT) T[k] = k < c0 ? T[k] * tscale : (F)0.0;
      __syncthreads();
      target_done = true;
    }
  }
  if (!target_done) {
  // The cells of class k in row i (Eq. 19) are the support columns of [js1(i, k), js1(i, k+1)),
  // so T_k = (1/N) sum_i R_i (sum of L over that run).  Row i meets the classes [k0, k1] of its
  // first and last support column (index_1 grows with j, and is at most i).  Row pass (own rows):
  // R_i times every run sum; partial pass: every CTA's T over its own rows; rank 0 then adds the
  // CTAs' partial vectors in rank order.
  unsigned* rk0 = csz;   // per own row: first class (the class-plan arrays are free by now)
  unsigned* rk1 = cst;   // per own row: last class
  // Where the row pass puts its sums, in the shared memory the cell lists used (free now) when
  // they fit, else in the workspace (the cell-list area): a few own rows (cluster CTAs) each get a
  // segment; many (a CTA alone) add into per-warp partial targets instead (a warp's rows in order,
  // then the warps in order), which spares the pass over all rows per class.
  const size_t room = (size_t)kPieceCap * (sizeof(F) + sizeof(uint2)) + (size_t)kListCap * sizeof(unsigned);
  // (decided from the largest own-row count, so every CTA of a cluster takes the same form: the
  // workspace forms, row segments and per-CTA partial blocks, share one area of the slot)
  const bool few_rows = (nR + C - 1) / C <= 32;
  F* seg_s = nullptr;
  F* wacc = nullptr;
  if (ob.s_part) {  // (s_part, s_piece and s_list are contiguous)
    if (few_rows && (size_t)(aB - aA) * K * sizeof(F) <= room) seg_s = static_cast<F*>(ob.s_part);
    if (!few_rows && (size_t)NW * K * sizeof(F) <= room) wacc = static_cast<F*>(ob.s_part);
  }
  if (!few_rows && !wacc && (size_t)C * NW * K * sizeof(F) <= (size_t)K * (K + 1) * 4)
    wacc = reinterpret_cast<F*>(slot + lay.list) + (size_t)rank * NW * K;  // (large K: a block per CTA)
  if (wacc) {
    for (int e = tid; e < NW * K; e += NT) wacc[e] = (F)0.0;
    __syncthreads();
  }
  F* seg_g = reinterpret_cast<F*>(slot + lay.list);
  auto seg_of = [&](int a) { return seg_s ? seg_s + (size_t)(a - aA) * K : seg_g + (size_t)RI[a] * (RI[a] + 1) / 2; };
  {
    const int jmin = LJ[0], jmax = LJ[nL - 1];
    for (int a = aA + warp; a < aB; a += NW) {  // own rows, a warp each
      const int i = RI[a];
      const uint16_t* jr = A.jstart1 + (size_t)i * (K + 1);  // js1(i, k), k <= K (entry K holds K)
      int k0, k1;
      index1_span(jr, K, i, jmin, jmax, k0, k1);
      if (lane == 0) { rk0[a] = (unsigned)k0; rk1[a] = (unsigned)k1; }
      const F r = Rc[a];
      F* out = wacc ? wacc + (size_t)warp * K : seg_of(a);
      // g lanes per class: a row with few classes has long runs, which g lanes sum in strides
      int g = 32;
      while (g > 1 && g * (k1 - k0 + 1) > 32) g >>= 1;
      const int gi = lane / g, gl = lane % g, cpw = 32 / g;
      for (int kk = k0; kk <= k1; kk += cpw) {
        const int k = kk + gi;
        F sum = 0.0;
        if (k <= k1) {
          const int p0 = posL[jr[k]], p1 = posL[jr[k + 1]];
          for (int b = p0 + gl; b < p1; b += g) sum += Lc[b];
        }
        for (int o = g >> 1; o > 0; o >>= 1) sum += __shfl_xor_sync(FULL, sum, o);
        if (gl == 0 && k <= k1) {
          if (wacc) out[k] += r * sum;
          else out[k] = r * sum;
        }
      }
      __syncwarp();  // (the next row's additions may come from other lanes)
    }
  }
  __syncthreads();
  F* Tp = L2c;  // this CTA's partial target (own rows)
  for (int k = tid; k < K; k += NT) {
    F sum = 0.0;
    if (wacc) {
      for (int w = 0; w < NW; ++w) sum += wacc[w * K + k];
    } else {  // a few rows, a branch per row: whole warps skip the rows that miss their classes
      for (int a = aA; a < aB; ++a)
        if ((int)rk0[a] <= k && k <= (int)rk1[a]) sum += seg_of(a)[k];
    }
    Tp[k] = sum;
  }
  cl.sync();
  stamp();
  if (rank != 0) {  // the partial is read by rank 0: stay until it has been
    cluster_arrive_relaxed();
    cluster_wait();
    return;
  }
  sl = scal[4];
  const F tscale = invN * (scR * sl);  // the count matrix carries 1/N (Eq. 6); R and L their scales
  for (int k = tid; k < K; k += NT) {
    F v[kMaxCluster];
#pragma unroll
    for (int r = 1; r < kMaxCluster; ++r) v[r] = r < C ? cl.map_shared_rank(Tp, r)[k] : (F)0.0;
    F sum = Tp[k];
#pragma unroll
    for (int r = 1; r < kMaxCluster; ++r) sum += v[r];
    T[k] = sum * tscale;
  }
  __syncthreads();
  }
  cluster_arrive_relaxed();  // the other CTAs may leave (this CTA waits for that phase at its end)
  stamp();

  // ---- histogram matching LUT (rank 0) -----------------------------------------------------------
  {
    double* CT = reinterpret_cast<double*>(RRc);                      // inclusive prefix sums of T (FP64)
    unsigned long long* lhs = reinterpret_cast<unsigned long long*>(q);  // CT(z) N, made monotone (FP64 bits)
    const int b0 = k0, b1 = k1;
    double s = 0.0;
    for (int k = b0; k < b1; ++k) { s += (double)T[k]; CT[k] = s; }
    double x = s;  // inclusive scan of the per-thread chunk sums: within the warp, then over warps
    for (int o = 1; o < 32; o <<= 1) {
      const double y = __shfl_up_sync(FULL, x, o);
      if (lane >= o) x += y;
    }
    double ex = __shfl_up_sync(FULL, x, 1);
    if (lane == 0) ex = 0.0;
    if (lane == 31) scr[warp] = x;
    __syncthreads();
    if (warp == 0) {
      double wv = lane < NW ? scr[lane] : 0.0;
      for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(FULL, wv, o);
        if (lane >= o) wv += y;
      }
      if (lane < NW) scr[NW + lane] = wv;
    }
    __syncthreads();
    const double before = ex + (warp > 0 ? scr[NW + warp - 1] : 0.0);
    for (int k = b0; k < b1; ++k) CT[k] += before;
    __syncthreads();
    stamp();
    const double TT = CT[K - 1];
    // non-negative doubles order like their bit patterns; a running max makes lhs monotone so the
    // first z with lhs(z) >= rhs(s) is found by binary search
    unsigned long long m = 0;
    for (int k = b0; k < b1; ++k) {
      const unsigned long long v = (unsigned long long)__double_as_longlong(CT[k] * (double)Nu);
      m = v > m ? v : m;
      lhs[k] = m;
    }
    unsigned long long xm = m;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(FULL, xm, o);
      if (lane >= o && y > xm) xm = y;
    }
    unsigned long long exm = __shfl_up_sync(FULL, xm, 1);
    if (lane == 0) exm = 0ull;
    unsigned long long* wmax = reinterpret_cast<unsigned long long*>(scr);
    __syncthreads();
    if (lane == 31) wmax[warp] = xm;
    __syncthreads();
    if (warp == 0) {
      unsigned long long wv = lane < NW ? wmax[lane] : 0ull;
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(FULL, wv, o);
        if (lane >= o && y > wv) wv = y;
      }
      if (lane < NW) wmax[NW + lane] = wv;
    }
    __syncthreads();
    unsigned long long pm = warp > 0 ? wmax[NW + warp - 1] : 0ull;
    if (exm > pm) pm = exm;
    for (int k = b0; k < b1; ++k) lhs[k] = lhs[k] > pm ? lhs[k] : pm;
    stamp();
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
    unsigned cs = block_exscan(cs_local, ured, &cs_total);  // (synchronises: ztop and lhs are final)
    const int z_top = (int)*ztop;
    stamp();
    for (int k = b0; k < b1; ++k) {
      cs += S[k];
      if (cs == Nu) { lut[k] = (uint16_t)z_top; continue; }
      const unsigned long long rhs = (unsigned long long)__double_as_longlong((double)cs * TT);
      int lo = 0, hi = K - 1;  // first z with lhs(z) >= rhs; K-1 if none
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (lhs[mid] >= rhs) hi = mid; else lo = mid + 1;
      }
      if (A.nearest) {
        // the first z minimising |CT(z) N - CS(s) TT|: lhs is monotone, so the minimum lies at lo or
        // at the first z of the plateau just below it (the first of equal distances is the earlier)
        const double r = __longlong_as_double((long long)rhs);
        const double d1 = fabs(__longlong_as_double((long long)lhs[lo]) - r);
        unsigned long long below = 0ull;
        bool take_below = false;
        if (lhs[lo] < rhs) {            // none reaches rhs: the nearest is the top plateau
          below = lhs[lo];
          take_below = true;
        } else if (lo > 0) {
          below = lhs[lo - 1];
          take_below = r - __longlong_as_double((long long)below) <= d1;
        }
        if (take_below) {
          int a = 0, b = lo;  // first z with lhs(z) >= below
          while (a < b) {
            const int mid = (a + b) >> 1;
            if (lhs[mid] >= below) b = mid; else a = mid + 1;
          }
          lo = a;
        }
      }
      lut[k] = (uint16_t)lo;
    }
  }
  __syncthreads();
  stamp();

  // ---- results (level-indexed) -------------------------------------------------------------------
  for (int k = tid; k < K; k += NT) { Rout[k] = 0.0; Lout[k] = 0.0; Tout[k] = (double)T[k]; }
  __syncthreads();
  for (int a = tid; a < nR; a += NT) Rout[RI[a]] = (double)(scR * Rc[a]);
  for (int b = tid; b < nL; b += NT) Lout[LJ[b]] = (double)(sl * Lc[b]);
  if (tid == 0) { misc[0] = it; misc[1] = nR; misc[2] = nL; misc[3] = (int)PP.cells; }
  stamp();
  cluster_wait();  // (every CTA has passed the set-up, where all of them read H_C(S) and H_C(grad S))
  if (A.zero_hist) {  // H_C(S) and H_C(grad S) (adjacent) cleared for the next call's histogram pass
    unsigned* SG = reinterpret_cast<unsigned*>(slot + lay.S);
    for (int k = tid; k < 2 * K; k += NT) SG[k] = 0u;
  }
}

}  // namespace

size_t solve_smem_bytes(int K, int vec_in_smem, int list_in_smem, size_t fsize) {
  size_t off = ((size_t)(3 * K + 1) * sizeof(uint16_t) + 15) & ~(size_t)15;
  off += (size_t)3 * K * 4;
  off += 8 * sizeof(double);
  off += ((NW + 2) * sizeof(unsigned) + 15) & ~(size_t)15;
  off += NT * sizeof(double);
  off += ((size_t)K + 15) & ~(size_t)15;
  if (list_in_smem) off += (size_t)kPieceCap * (fsize + sizeof(uint2)) + (size_t)kListCap * sizeof(unsigned);
  if (vec_in_smem) off += (size_t)kSolveVecs * K * fsize;
  return off;
}

// Shared memory one CTA may use (sm_103a: 227 KB).
constexpr size_t kSmemMax = 227 * 1024;

// Largest cluster (16, 8, 4, 2 or 1 CTAs) of solve_kernel<F> that can be resident for one image.
template <typename F>
int solve_cluster_size(size_t smem) {
  for (int C = kMaxCluster; C > 1; C >>= 1) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, solve_kernel<F>, &cfg) == cudaSuccess && nclusters > 0) return C;
    cudaGetLastError();
  }
  return 1;
}

template <typename F>
cudaError_t launch_solve_t(const SolveArgs& a0, int n, int cluster, cudaStream_t st, bool pdl) {
  // own cell lists in shared memory up to K = 1024 (beyond it they never fit a share); the
  // solver vectors there whenever the layout fits (for K = 4096: FP32 only)
  SolveArgs a = a0;
  a.list_in_smem = a.K <= 1024 ? 1 : 0;
  a.vec_in_smem = solve_smem_bytes(a.K, 1, a.list_in_smem, sizeof(F)) <= kSmemMax ? 1 : 0;
  const size_t smem = solve_smem_bytes(a.K, a.vec_in_smem, a.list_in_smem, sizeof(F));
  // the kernel's dynamic shared-memory limit: the most any K takes, the same value on every call, so
  // calls of contexts on several host threads cannot lower it under each other's launches
  size_t smem_max = 0;
  for (int k = 8; k <= 4096; k <<= 1) {
    const int list = k <= 1024 ? 1 : 0, vec = solve_smem_bytes(k, 1, list, sizeof(F)) <= kSmemMax ? 1 : 0;
    smem_max = std::max(smem_max, solve_smem_bytes(k, vec, list, sizeof(F)));
  }
  cudaError_t e = cudaFuncSetAttribute(solve_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(solve_kernel<F>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  // the requested cluster per image (vectors must be in shared memory), capped at what can be
  // resident; that cap is found once per K (it depends on K and F alone) and kept in an atomic
  // entry per log2 K, 0 until found, so contexts used from several host threads read whole values
  static std::atomic<int> cluster_cap[13];
  int C = 1;
  if (a.vec_in_smem && cluster > 1) {
    int lk = 0;
    while ((1 << lk) < a.K) ++lk;
    int cap = cluster_cap[lk].load(std::memory_order_relaxed);
    if (cap == 0) {
      cap = solve_cluster_size<F>(smem);
      cluster_cap[lk].store(cap, std::memory_order_relaxed);
    }
    C = cluster < cap ? cluster : cap;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n * C));
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, solve_kernel<F>, a);
}

cudaError_t launch_solve(const SolveArgs& a, int n, int cluster, cudaStream_t st, bool pdl) {
  if (a.arith == kArithF32) return launch_solve_t<float>(a, n, cluster, st, pdl);
  if (a.arith == kArithDF64) return launch_solve_t<df64>(a, n, cluster, st, pdl);
  return launch_solve_t<double>(a, n, cluster, st, pdl);
}

}  // namespace hr
