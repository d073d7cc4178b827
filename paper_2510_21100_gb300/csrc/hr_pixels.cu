// Pixel passes of HistRetinex on sm_103a:
//   hist  -- V = max(r,g,b) (Sec. II preamble), its K-bin count histogram H_C(S) (Eq. 3) and the
//            histogram of its 3x3 Sobel gradient magnitude H_C(grad S) (Algorithm 1 initialisation);
//   apply -- V' = LUT[V] and every channel scaled by V'/V, rounded half up, so hue and saturation
//            are kept (Sec. II preamble; Sec. III.C last paragraph: histogram matching).
// Both kernels walk a flat list of kTileW x kTileH tiles spanning every image of the launch, so
// one launch serves a single image or a batch of mixed sizes.
#include <algorithm>

#include "hr_internal.cuh"

namespace hr {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kVW = kTileW + 2;   // V tile row length with the two halo columns
constexpr int kVH = kTileH + 2;

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Image of global tile t: largest i with tile_start[i] <= t.
__device__ __forceinline__ int image_of_tile(const int* tile_start, int n, int t) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(tile_start + mid) <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename ET>
__device__ __forceinline__ unsigned load_value(const ImageDesc& im, int x, int y) {
  const ET* row = reinterpret_cast<const ET*>(im.in + (long long)y * im.in_pitch);
  unsigned r = row[3 * x], g = row[3 * x + 1], b = row[3 * x + 2];
  unsigned v = r > g ? r : g;
  return v > b ? v : b;
}

// Nearest integer to sqrt(m2), halves rounded up, for m2 < 2^31.
__device__ __forceinline__ unsigned round_sqrt(unsigned m2) {
  unsigned n = (unsigned)sqrtf((float)m2);
  while (n * n > m2) --n;
  while ((n + 1) * (n + 1) <= m2) ++n;
  return n + (m2 > n * n + n ? 1u : 0u);
}

template <typename ET>
__global__ void __launch_bounds__(kThreads) hist_kernel(const ImgTab tab, int total, int K,
                                                        uint8_t* slots, size_t slot_bytes, SlotLayout lay,
                                                        unsigned* status, int forward, int shift, int M) {
  pdl_wait();     // the previous kernel on the stream has finished
  pdl_trigger();  // the next one may be scheduled (it waits for this one)
  const int n = tab.n;
  const int* __restrict__ tile_start = tab.tiles;  // (n > 1 only)
  extern __shared__ __align__(16) unsigned char smem[];
  // per-warp sub-histograms when K is small (less same-address contention), else one copy
  const int copies = K <= 256 ? kWarps : 1;
  unsigned* hs = reinterpret_cast<unsigned*>(smem);
  unsigned* hg = hs + copies * K;
  unsigned short* vt = reinterpret_cast<unsigned short*>(hg + copies * K);
  const int tid = threadIdx.x, warp = tid >> 5;
  unsigned* my_hs = hs + (copies > 1 ? warp : 0) * K;
  unsigned* my_hg = hg + (copies > 1 ? warp : 0) * K;
  for (int k = tid; k < 2 * copies * K; k += kThreads) hs[k] = 0u;

  const int chunk = (total + gridDim.x - 1) / gridDim.x;
  const int t0 = blockIdx.x * chunk, t1 = min(total, t0 + chunk);
  int cur = -1;
  bool range_bad = false;
  __syncthreads();
  for (int t = t0; t < t1; ++t) {
    const int img = image_of_tile(tile_start, n, t);
    if (img != cur) {
      if (cur >= 0) {  // flush the previous image's histograms
        __syncthreads();
        unsigned* S = reinterpret_cast<unsigned*>(slots + (size_t)cur * slot_bytes + lay.S);
        unsigned* G = reinterpret_cast<unsigned*>(slots + (size_t)cur * slot_bytes + lay.G);
        for (int k = tid; k < K; k += kThreads) {
          unsigned s = 0, g = 0;
          for (int c = 0; c < copies; ++c) { s += hs[c * K + k]; g += hg[c * K + k]; hs[c * K + k] = 0u; hg[c * K + k] = 0u; }
          if (s) atomicAdd(S + k, s);
          if (g) atomicAdd(G + k, g);
        }
        __syncthreads();
      }
      cur = img;
    }
    const ImageDesc im = tab.desc(img);
    const int lt = t - tab.tile0(img);
    const int tiles_x = (im.W + kTileW - 1) / kTileW;
    const int x0 = (lt % tiles_x) * kTileW, y0 = (lt / tiles_x) * kTileH;
    // V tile with a one-pixel halo; coordinates outside the image replicate the border
    for (int e = tid; e < kVH * kVW; e += kThreads) {
      const int r = e / kVW, c = e - r * kVW;
      const int y = clampi(y0 - 1 + r, 0, im.H - 1), x = clampi(x0 - 1 + c, 0, im.W - 1);
      unsigned v = load_value<ET>(im, x, y);
      if (v >= (unsigned)M) { range_bad = true; v = M - 1; }  // (M = K unless the data is binned)
      vt[r * kVW + c] = (unsigned short)v;
    }
    __syncthreads();
    for (int e = tid; e < kTileH * kTileW; e += kThreads) {
      const int r = e / kTileW, c = e - r * kTileW;
      if (y0 + r >= im.H || x0 + c >= im.W) continue;
      const unsigned short* p = vt + (r + 1) * kVW + (c + 1);
      const int a00 = p[-kVW - 1], a01 = p[-kVW], a02 = p[-kVW + 1];
      const int a10 = p[-1], a11 = p[0], a12 = p[1];
      const int a20 = p[kVW - 1], a21 = p[kVW], a22 = p[kVW + 1];
      // 3x3 Sobel, or forward differences (the halo replicates the border, so both are zero at
      // the last column and row)
      const int gx = forward ? a12 - a11 : (a02 + 2 * a12 + a22) - (a00 + 2 * a10 + a20);
      const int gy = forward ? a21 - a11 : (a20 + 2 * a21 + a22) - (a00 + 2 * a01 + a02);
      unsigned g = round_sqrt((unsigned)(gx * gx + gy * gy));
      g = g < (unsigned)(M - 1) ? g : (unsigned)(M - 1);
      // binned data: value v and gradient level g (clipped to the data's range) fall into bins >> shift
      atomicAdd(my_hs + (a11 >> shift), 1u);
      atomicAdd(my_hg + (g >> shift), 1u);
    }
    __syncthreads();
  }
  if (cur >= 0) {
    __syncthreads();
    unsigned* S = reinterpret_cast<unsigned*>(slots + (size_t)cur * slot_bytes + lay.S);
    unsigned* G = reinterpret_cast<unsigned*>(slots + (size_t)cur * slot_bytes + lay.G);
    for (int k = tid; k < K; k += kThreads) {
      unsigned s = 0, g = 0;
      for (int c = 0; c < copies; ++c) { s += hs[c * K + k]; g += hg[c * K + k]; }
      if (s) atomicAdd(S + k, s);
      if (g) atomicAdd(G + k, g);
    }
  }
  if (range_bad) atomicOr(status, kStRange);
}

template <typename ET>
__global__ void __launch_bounds__(kThreads) apply_kernel(const ImgTab tab, int total, int K,
                                                         const uint8_t* slots, size_t slot_bytes, SlotLayout lay,
                                                         unsigned* status, int shift, int M) {
  pdl_wait();     // the previous kernel on the stream has finished
  pdl_trigger();  // the next one may be scheduled (it waits for this one)
  const int n = tab.n;
  const int* __restrict__ tile_start = tab.tiles;  // (n > 1 only)
  extern __shared__ __align__(16) unsigned char smem[];
  // per value V (8-bit data: M <= 256 entries) or per bin (16-bit data: K entries)
  const int nt = sizeof(ET) == 1 ? M : K;
  unsigned short* lut = reinterpret_cast<unsigned short*>(smem);
  float* rup = reinterpret_cast<float*>(smem + ((nt * 2 + 15) & ~15));  // V'/V rounded up (8-bit data)
  const int tid = threadIdx.x;
  const int chunk = (total + gridDim.x - 1) / gridDim.x;
  const int t0 = blockIdx.x * chunk, t1 = min(total, t0 + chunk);
  int cur = -1;
  bool range_bad = false;
  for (int t = t0; t < t1; ++t) {
    const int img = image_of_tile(tile_start, n, t);
    if (img != cur) {
      __syncthreads();
      const unsigned short* gl = reinterpret_cast<const unsigned short*>(slots + (size_t)img * slot_bytes + lay.lut);
      for (int k = tid; k < nt; k += kThreads) {
        // V' of value k: binned data keeps the value's place in its bin, LUT[s] w + (k - s w)
        const int sb = sizeof(ET) == 1 ? k >> shift : k;
        const unsigned short vp =
            sizeof(ET) == 1 ? (unsigned short)(((unsigned)gl[sb] << shift) | (unsigned)(k - (sb << shift))) : gl[k];
        lut[k] = vp;
        if (sizeof(ET) == 1) rup[k] = k > 0 ? __fdiv_ru((float)vp, (float)k) : 0.0f;
      }
      __syncthreads();
      cur = img;
    }
    const ImageDesc im = tab.desc(img);
    const int lt = t - tab.tile0(img);
    const int tiles_x = (im.W + kTileW - 1) / kTileW;
    const int x0 = (lt % tiles_x) * kTileW, y0 = (lt / tiles_x) * kTileH;
    for (int e = tid; e < kTileH * kTileW; e += kThreads) {
      const int r = e / kTileW, c = e - r * kTileW;
      const int x = x0 + c, y = y0 + r;
      if (y >= im.H || x >= im.W) continue;
      const ET* src = reinterpret_cast<const ET*>(im.in + (long long)y * im.in_pitch) + 3 * x;
      unsigned ch[3] = {src[0], src[1], src[2]};
      unsigned V = ch[0] > ch[1] ? ch[0] : ch[1];
      V = V > ch[2] ? V : ch[2];
      if (V >= (unsigned)M) { range_bad = true; V = M - 1; }
      const unsigned vp = sizeof(ET) == 1 ? lut[V] : ((unsigned)lut[V >> shift] << shift) | (V & ((1u << shift) - 1u));
      ET* dst = reinterpret_cast<ET*>(im.out + (long long)y * im.out_pitch) + 3 * x;
      if (V == 0) {
        dst[0] = (ET)vp; dst[1] = (ET)vp; dst[2] = (ET)vp;
      } else if (sizeof(ET) == 1) {
        // floor(c V'/V + 1/2) from an upward-rounded product: exact for c <= V < 256 (the
        // fraction of c V'/V + 1/2 is a multiple of 1/(2V) >= 1/510, the error is < 2^-13)
        const float rv = rup[V];
        for (int q = 0; q < 3; ++q) dst[q] = (ET)(unsigned)__fmaf_ru((float)ch[q], rv, 0.5f);
      } else {
        for (int q = 0; q < 3; ++q) dst[q] = (ET)((2u * ch[q] * vp + V) / (2u * V));
      }
    }
  }
  if (range_bad) atomicOr(status, kStRange);
}

// ------------------------------------------------------------------------------------------------
// 8-bit fast paths (rows 16-byte aligned).
//
// Histogram pass, large images and batches: the rolling strip kernel below.  Lane l of a warp owns
// the 16 pixels [x0 + 16 l, x0 + 16 l + 16) of a strip's rows, so the warp reads 1536 contiguous
// bytes per row.  Smaller launches: the staged-tile kernel further down.
//
// Apply pass: 16 pixels (48 bytes, three 16-byte vectors) per thread each way.
// ------------------------------------------------------------------------------------------------
// The strip kernel runs one CTA of 8 warps per SM, its registers capped at 128 so that three
// quarters of the register file stay free for apply-pass CTAs of other calls (partitioned calls on
// several streams overlap one image's histogram pass with another's apply pass on the same SMs:
// 60.5 against 68.6 us per 7680x4320 image with 16 warps per SM; alone the two shapes take 41 us).
#ifndef HR_HIST_WARPS
#define HR_HIST_WARPS 8
#endif
constexpr int kHW = HR_HIST_WARPS;  // warps per CTA of the fast histogram pass
constexpr int kHT = kHW * 32;
#ifndef HR_STRIP_MIN_FACTOR
#define HR_STRIP_MIN_FACTOR 2  // strips per warp from which one image takes the strip kernel
#endif
constexpr int kHBins = 256;     // per-warp histogram stride (the 8-bit pass has K <= 256)

// 16-byte copy of which only the first `nb` (0..16) bytes are read; the rest is zero-filled.
__device__ __forceinline__ void cp_async16z(void* smem_dst, const void* gsrc, int nb) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gsrc), "r"(nb) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// V of two pixels as 16-bit pairs from the 12 bytes of four pixels: a = R0 G0 B0 R1,
// b = G1 B1 R2 G2, c = B2 R3 G3 B3.  Every operand of one 3-way max carries the same filler
// byte above each channel byte, so the halfword maximum is the channel maximum.
__device__ __forceinline__ void vpairs(unsigned a, unsigned b, unsigned c, unsigned& e, unsigned& o) {
  e = __vimax3_u16x2(__byte_perm(a, b, 0x3630), __byte_perm(a, b, 0x3731), __byte_perm(a, c, 0x3432)) & 0x00ff00ffu;
  o = __vimax3_u16x2(__byte_perm(a, c, 0x4543), __byte_perm(b, c, 0x4640), __byte_perm(b, c, 0x4741)) & 0x00ff00ffu;
}

// ------------------------------------------------------------------------------------------------
// Rolling strip histogram pass (8-bit, rows 16-byte aligned).  The strips of kStripW pixels are cut
// into strip rows, column by column and image after image; warp w of the grid takes the w-th of
// equal contiguous ranges of that sequence, so a warp walks long runs down one strip column,
// building each V row once (plus two halo rows per run), and all warps finish together.  The warp
// copies every row it needs -- the strip's 1536 bytes and the 16-byte chunks on either side, which
// hold the neighbour pixels -- into its ring of kSRing row slots with asynchronous copies, kSRing
// rows ahead of use.  Building a row counts its V levels into H_C(S) and converts V to half-
// precision pairs.  The Sobel sums (integers of magnitude at most 4 * 255 = 1020, exact in half
// precision) run on pairs of pixels, and each pixel's squared magnitude (at most 2 * 1020^2 < 2^24)
// is formed exactly in FP32 by two fused multiply-adds with half-precision inputs.
// ------------------------------------------------------------------------------------------------
constexpr int kSRing = 4;                            // row slots per warp (a power of two)
constexpr int kSSlot = 16 + 3 * kStripW + 16;        // left chunk, the strip's row, right chunk
// A warp's two histogram copies (even and odd lanes), each H_C(S) then H_C(grad S), the second
// copy 16 words further on, so the two copies' counts of one level fall in different banks (24%
// fewer shared-memory wavefronts of the counts at 7680x4320).
constexpr int kHCopyWords = 2 * kHBins + 16;
constexpr size_t kRollSmem = (size_t)kHW * (2 * kHCopyWords * 4 + kSRing * kSSlot);
constexpr unsigned kHalfMagic = 0x64006400u;         // half 1024 in each half: 1024 + v for v < 1024
constexpr unsigned kHalfMinus1024 = 0xE400E400u;     // half -1024 in each half
constexpr unsigned kHalfTwo = 0x40004000u;           // half 2 in each half

__device__ __forceinline__ unsigned hadd2(unsigned a, unsigned b) {
  unsigned d;
  asm("add.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}
__device__ __forceinline__ unsigned hsub2(unsigned a, unsigned b) {
  unsigned d;
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}
__device__ __forceinline__ unsigned hfma2(unsigned a, unsigned b, unsigned c) {
  unsigned d;
  asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
// Shared-memory count without a compiler memory barrier: the histograms are read only after the
// warp and block barriers at a warp's image change and at the kernel's end.
__device__ __forceinline__ void red_sh(unsigned addr) { asm volatile("red.shared.add.u32 [%0], 1;\n" ::"r"(addr)); }
// The same count when `on` holds, as one predicated instruction (no branch around it).
__device__ __forceinline__ void red_sh_if(unsigned addr, bool on) {
  asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %1, 0;\n@p red.shared.add.u32 [%0], 1;\n}\n" ::"r"(addr),
               "r"((unsigned)on));
}
// Takes one count back (adds 2^32 - 1).
__device__ __forceinline__ void unred_sh(unsigned addr) {
  asm volatile("red.shared.add.u32 [%0], 0xffffffff;\n" ::"r"(addr));
}
__device__ __forceinline__ void cp_async16s(unsigned dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16zs(unsigned dst, const void* src, int nb) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(nb) : "memory");
}

// Gradient level of a squared magnitude m2 held exactly in FP32: the nearest integer to sqrt(m2)
// clipped to K - 1, as 0x4B000000 + level in the result's bits.  Clipping m2 at K^2 - K first gives
// the same level and keeps m2 below 2^23; sqrt.approx (flush-to-zero: no m2 here is subnormal) is
// within 2^-22 relative of sqrt(m2) there, well inside the distance 1/(4 sqrt(m2) + 2) from sqrt(m2)
// to the nearest half integer, so the round-to-nearest add of 2^23 yields the exact level.
__device__ __forceinline__ unsigned grad_bits_f(float m2, float mclipf) {
  const float f = fminf(m2, mclipf);
  float s;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(f));
  return __float_as_uint(__fadd_rn(s, 8388608.0f));
}

// Squared magnitudes of the two pixels of half-precision pairs (gx, gy), exact in FP32.
__device__ __forceinline__ void m2_pair(unsigned gx, unsigned gy, float& mlo, float& mhi) {
  asm("{\n.reg .f16 xl, xh, yl, yh;\n.reg .f32 t, u;\n"
      "mov.b32 {xl, xh}, %2;\nmov.b32 {yl, yh}, %3;\n"
      "fma.rn.f32.f16 t, yl, yl, %4;\nfma.rn.f32.f16 %0, xl, xl, t;\n"
      "fma.rn.f32.f16 u, yh, yh, %4;\nfma.rn.f32.f16 %1, xh, xh, u;\n}\n"
      : "=f"(mlo), "=f"(mhi)
      : "r"(gx), "r"(gy), "f"(0.0f));
}

// V row of one lane as half-precision pairs.
struct HRow {
  unsigned e[4], o[4];  // pixels (4w, 4w + 2) and (4w + 1, 4w + 3), w = 0..3
  unsigned l, r;        // high half of l: the pixel left of the 16; low half of r: the one right
};

// A lane's constants for one run of rows down one strip column.
struct SegLane {
  const uint8_t* in;
  long long pitch;
  int H;
  int goff;         // byte offset in a row of the lane's first 16-byte chunk (3 x0 + 16 lane)
  int xoff;         // byte offset in a row of the lane's extra chunk (lane 0: left, lane 1: right)
  int xbytes;       // bytes the extra chunk reads (0: none)
  unsigned sxo;     // slot offset of the extra chunk
  unsigned soff;    // slot offset of the lane's first copied chunk: 16 (lane + 1)
  unsigned roff;    // slot offset of the lane's 48 bytes (pixels x0 + 16 lane ..): 16 + 48 lane
  unsigned nbo;     // slot offset of the neighbour word: 12 (lane 0) or 16 + 1536 (the others)
  unsigned sel0, sel1, sel2;  // byte selectors of the neighbour pixel's three channels
  int cnt;          // pixels of the lane inside the image: W - (x0 + 16 lane)
  int rowbytes;     // 3 W
  int eo[3], eb[3]; // edge runs: the row offset and the bytes inside the row of the lane's chunks c, c + 32,
                    // c + 64 (offset 0 where none is inside; the rest of each chunk is zero-filled)
  bool lane0, lane31, left_nb, right_nb, use_nb;
};

// Copies row y (clamped: replicate border) into the slot at shared address `slot`: lane l copies
// the strip's 16-byte chunks l, l + 32 and l + 64 (so each copy instruction of the warp covers 512
// contiguous bytes) to slot offsets 16 + 16 c, lane 0 the left chunk to offset 0 and lane 1 the
// right chunk to offset 16 + 1536; lanes read their own 48 bytes after the wait and a __syncwarp.
// One commit group per call, empty when `live` is false.  Edge runs read only the bytes inside the row (the
// rest of each chunk is zero-filled).
template <bool kEdge>
__device__ __forceinline__ void roll_issue(const SegLane& s, unsigned slot, int y, bool live) {
  if (live) {
    const uint8_t* row = s.in + (long long)clampi(y, 0, s.H - 1) * s.pitch;
    const uint8_t* src = row + s.goff;
    const unsigned dst = slot + s.soff;
    if (!kEdge) {
      cp_async16s(dst, src);
      cp_async16s(dst + 512, src + 512);
      cp_async16s(dst + 1024, src + 1024);
    } else {
#pragma unroll
      for (int i = 0; i < 3; ++i) cp_async16zs(dst + 512 * i, row + s.eo[i], s.eb[i]);
    }
    if (s.xbytes > 0) cp_async16zs(slot + s.sxo, row + s.xoff, s.xbytes);
  }
  cp_async_commit();
}

// Builds one V row from a slot; counts its levels into H_C(S) when `count` is set.
template <bool kEdge, bool kClamp>
__device__ __forceinline__ void roll_build(HRow& v, const SegLane& s, const unsigned char* slotp, bool count,
                                           unsigned hs_sh, unsigned kk, bool& bad) {
  unsigned u[8];  // u[2w] = pixels (4w, 4w + 2), u[2w + 1] = pixels (4w + 1, 4w + 3): V as 16-bit pairs
  if (kEdge && s.cnt > 0 && s.cnt < 16) {
    // the lane holding the image's last pixel: the first pixel beyond it (zero-filled) takes a copy of
    // it (the replicated border of the Sobel operator), and the count that copy adds is taken back
    unsigned char* lp = const_cast<unsigned char*>(slotp) + s.roff + 3 * (s.cnt - 1);
    const unsigned c0 = lp[0], c1 = lp[1], c2 = lp[2];
    lp[3] = (unsigned char)c0;
    lp[4] = (unsigned char)c1;
    lp[5] = (unsigned char)c2;
    if (count) {
      unsigned vl = max(max(c0, c1), c2);
      if (kClamp) vl = min(vl, kk & 0xffffu);
      unred_sh(hs_sh + (vl << 2));
    }
  }
  {
    const uint4* q = reinterpret_cast<const uint4*>(slotp + s.roff);
    const uint4 a = q[0], b = q[1], c = q[2];
    vpairs(a.x, a.y, a.z, u[0], u[1]);
    vpairs(a.w, b.x, b.y, u[2], u[3]);
    vpairs(b.z, b.w, c.x, u[4], u[5]);
    vpairs(c.y, c.z, c.w, u[6], u[7]);
  }
  if (kClamp) {  // K < 256: levels above K - 1 are a range error, clamped so counting stays in bounds
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      const unsigned c = __vimin3_u16x2(u[w], kk, kk);
      bad |= c != u[w];
      u[w] = c;
    }
  }
  if (count) {  // (edge runs count the zero-filled pixels beyond the image too: level 0, taken back per run)
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      red_sh(hs_sh + ((u[2 * w] & 0xffffu) << 2));
      red_sh(hs_sh + (u[2 * w] >> 14));  // 0x00VV00WW >> 14 = VV << 2
      red_sh(hs_sh + ((u[2 * w + 1] & 0xffffu) << 2));
      red_sh(hs_sh + (u[2 * w + 1] >> 14));
    }
  }
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    v.e[w] = hadd2(u[2 * w] | kHalfMagic, kHalfMinus1024);
    v.o[w] = hadd2(u[2 * w + 1] | kHalfMagic, kHalfMinus1024);
  }
  // neighbour columns: from the adjacent lanes, at the strip's ends from the neighbour chunks, at
  // the image's ends the replicated edge pixel
  unsigned nbv;
  {
    const unsigned nbw = *reinterpret_cast<const unsigned*>(slotp + s.nbo);
    nbv = __vimax3_u16x2(__byte_perm(nbw, 0u, s.sel0), __byte_perm(nbw, 0u, s.sel1), __byte_perm(nbw, 0u, s.sel2));
    if (kClamp) {
      bad |= s.use_nb && nbv > (kk & 0xffffu);
      nbv = min(nbv, kk & 0xffffu);
    }
    nbv = hadd2(nbv | kHalfMagic, kHalfMinus1024);  // low half: the neighbour's V
  }
  const unsigned up = __shfl_up_sync(0xffffffffu, v.o[3], 1);
  const unsigned dn = __shfl_down_sync(0xffffffffu, v.e[0], 1);
  v.l = s.lane0 ? __byte_perm(s.left_nb ? nbv : v.e[0], 0u, 0x1010) : up;
  if (kEdge) {
    v.r = s.cnt == 16 ? __byte_perm(v.o[3], 0u, 0x3232) : ((s.lane31 && s.right_nb) ? nbv : dn);
  } else {
    v.r = s.lane31 ? (s.right_nb ? nbv : __byte_perm(v.o[3], 0u, 0x3232)) : dn;
  }
}

// Sobel gradient of the output row M between rows T and B, counted into H_C(grad S).
template <bool kEdge>
__device__ __forceinline__ void roll_sobel(const HRow& T, const HRow& M, const HRow& B, int cnt, float mclipf,
                                           unsigned hg_adj) {
  auto cs = [](unsigned t, unsigned m, unsigned b) { return hadd2(hfma2(m, kHalfTwo, t), b); };
  auto dd = [](unsigned t, unsigned b) { return hsub2(b, t); };
  unsigned csOp = cs(T.l, M.l, B.l), ddOp = dd(T.l, B.l);  // high half: the pixel left of the 16
  unsigned csEc = cs(T.e[0], M.e[0], B.e[0]), ddEc = dd(T.e[0], B.e[0]);
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    const unsigned csOc = cs(T.o[w], M.o[w], B.o[w]), ddOc = dd(T.o[w], B.o[w]);
    const unsigned csEn = w < 3 ? cs(T.e[w + 1], M.e[w + 1], B.e[w + 1]) : cs(T.r, M.r, B.r);
    const unsigned ddEn = w < 3 ? dd(T.e[w + 1], B.e[w + 1]) : dd(T.r, B.r);
    // odd pixels left of the even pair (4w - 1, 4w + 1); even pixels right of the odd pair (4w + 2, 4w + 4)
    const unsigned csOL = __byte_perm(csOp, csOc, 0x5432), ddOL = __byte_perm(ddOp, ddOc, 0x5432);
    const unsigned csER = __byte_perm(csEc, csEn, 0x5432), ddER = __byte_perm(ddEc, ddEn, 0x5432);
    const unsigned gxE = hsub2(csOc, csOL), gyE = hadd2(hfma2(ddEc, kHalfTwo, ddOL), ddOc);
    const unsigned gxO = hsub2(csER, csEc), gyO = hadd2(hfma2(ddOc, kHalfTwo, ddEc), ddER);
    float m0, m2, m1, m3;
    m2_pair(gxE, gyE, m0, m2);
    m2_pair(gxO, gyO, m1, m3);
    const unsigned b0 = grad_bits_f(m0, mclipf), b1 = grad_bits_f(m1, mclipf);
    const unsigned b2 = grad_bits_f(m2, mclipf), b3 = grad_bits_f(m3, mclipf);
    if (!kEdge) {
      red_sh(hg_adj + (b0 << 2));
      red_sh(hg_adj + (b1 << 2));
      red_sh(hg_adj + (b2 << 2));
      red_sh(hg_adj + (b3 << 2));
    } else {
      red_sh_if(hg_adj + (b0 << 2), 4 * w < cnt);
      red_sh_if(hg_adj + (b1 << 2), 4 * w + 1 < cnt);
      red_sh_if(hg_adj + (b2 << 2), 4 * w + 2 < cnt);
      red_sh_if(hg_adj + (b3 << 2), 4 * w + 3 < cnt);
    }
    csOp = csOc; ddOp = ddOc; csEc = csEn; ddEc = ddEn;
  }
}

// Output rows [ya, yb) (yb <= H) of one strip column for one lane; rows ya - 1 .. yb pass through
// the warp's ring, row r in slot (r - ya + 1) mod kSRing.  Returns whether a level above K - 1 was
// seen.
template <bool kEdge, bool kClamp>
__device__ __forceinline__ bool roll_run(const SegLane& s, int ya, int yb, const unsigned char* wring,
                                         unsigned wring_sh, unsigned hs_sh, unsigned hg_adj, float mclipf,
                                         unsigned kk) {
  bool bad = false;
  __syncwarp();  // (the previous run's reads of the ring are done)
#pragma unroll
  for (int k = 0; k < kSRing; ++k) roll_issue<kEdge>(s, wring_sh + k * kSSlot, ya - 1 + k, ya - 1 + k <= yb);
  HRow R0, R1, R2;
  cp_async_wait<kSRing - 1>();
  __syncwarp();
  roll_build<kEdge, kClamp>(R0, s, wring, false, hs_sh, kk, bad);
  __syncwarp();
  roll_issue<kEdge>(s, wring_sh, ya - 1 + kSRing, ya - 1 + kSRing <= yb);
  cp_async_wait<kSRing - 1>();
  __syncwarp();
  roll_build<kEdge, kClamp>(R1, s, wring + kSSlot, true, hs_sh, kk, bad);
  __syncwarp();
  roll_issue<kEdge>(s, wring_sh + kSSlot, ya + kSRing, ya + kSRing <= yb);
  int y = ya;
  auto step = [&](const HRow& T, const HRow& M, HRow& B) {
    const unsigned k = (unsigned)(y - ya + 2) & (kSRing - 1);  // slot of row y + 1
    cp_async_wait<kSRing - 1>();
    __syncwarp();
    roll_build<kEdge, kClamp>(B, s, wring + k * kSSlot, y + 1 < yb, hs_sh, kk, bad);
    __syncwarp();
    roll_issue<kEdge>(s, wring_sh + k * kSSlot, y + 1 + kSRing, y + 1 + kSRing <= yb);
    roll_sobel<kEdge>(T, M, B, s.cnt, mclipf, hg_adj);
  };
  for (;;) {
    if (y >= yb) break;
    step(R0, R1, R2);
    ++y;
    if (y >= yb) break;
    step(R1, R2, R0);
    ++y;
    if (y >= yb) break;
    step(R2, R0, R1);
    ++y;
  }
  cp_async_wait<0>();  // (the empty groups past the run's end)
  return bad;
}

// Runs of strip columns whose lanes do not all lie inside the image, kept out of line so the
// interior path has the register file to itself.
template <bool kClamp>
__device__ __noinline__ bool roll_run_edge(const SegLane s, int ya, int yb, const unsigned char* wring,
                                           unsigned wring_sh, unsigned hs_sh, unsigned hg_adj, float mclipf,
                                           unsigned kk) {
  return roll_run<true, kClamp>(s, ya, yb, wring, wring_sh, hs_sh, hg_adj, mclipf, kk);
}

template <bool kClamp>
__global__ void __launch_bounds__(kHT, 2) hist_u8s_kernel(const ImgTab tab, int total, int all_edge, int K,
                                                         uint8_t* slots, size_t slot_bytes, SlotLayout lay,
                                                         unsigned* status) {
  pdl_wait();     // the previous kernel on the stream has finished
  pdl_trigger();  // the next one may be scheduled (it waits for this one)
  const int n = tab.n;
  const int* __restrict__ unit_start = tab.units;  // (n > 1 only)
  extern __shared__ __align__(16) unsigned char hsmem[];
  // per warp two copies (even and odd lanes) of H_C(S), H_C(grad S), then the warps' rings
  auto hist = reinterpret_cast<unsigned (*)[2][kHCopyWords]>(hsmem);
  unsigned char* ring = hsmem + (size_t)kHW * 2 * kHCopyWords * 4;
  __shared__ int warp_img[kHW];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned* hw = &hist[warp][0][0];
  for (int k = lane; k < 2 * kHCopyWords; k += 32) hw[k] = 0u;
  __syncwarp();
  const unsigned hs_sh = (unsigned)__cvta_generic_to_shared(&hist[warp][lane & 1][0]);
  const unsigned hg_adj = (unsigned)__cvta_generic_to_shared(&hist[warp][lane & 1][kHBins]) - 0x2C000000u;  // - (0x4B000000 << 2)
  const float mclipf = (float)(K * K - K);
  const unsigned kk = 0x00010001u * (unsigned)(K - 1);
  const unsigned char* wring = ring + (size_t)warp * kSRing * kSSlot;
  const unsigned wring_sh = (unsigned)__cvta_generic_to_shared(wring);
  // this warp's range of strip rows (kBandH per unit, units column-major within each image)
  const long long Q = (long long)kBandH * total, NW = (long long)gridDim.x * kHW;
  const long long gw = (long long)blockIdx.x * kHW + warp;
  long long q = gw * Q / NW;
  const long long q1 = (gw + 1) * Q / NW;
  int cur = -1, img_u0 = 0, img_u1 = 0, nb = 1;
  ImageDesc im{};
  bool bad = false;
  // zero-filled pixels beyond the right edge that this warp's edge runs counted at level 0 of the
  // current image (warp-uniform)
  unsigned phantom = 0;
  auto flush_warp = [&](int im_idx) {
    __syncwarp();
    if (lane == 0) hist[warp][0][0] -= phantom;
    phantom = 0;
    __syncwarp();
    unsigned* S = reinterpret_cast<unsigned*>(slots + (size_t)im_idx * slot_bytes + lay.S);
    unsigned* G = reinterpret_cast<unsigned*>(slots + (size_t)im_idx * slot_bytes + lay.G);
    for (int k = lane; k < K; k += 32) {
      const unsigned sv = hist[warp][0][k] + hist[warp][1][k], gv = hist[warp][0][kHBins + k] + hist[warp][1][kHBins + k];
      hist[warp][0][k] = hist[warp][1][k] = hist[warp][0][kHBins + k] = hist[warp][1][kHBins + k] = 0u;
      if (sv) atomicAdd(S + k, sv);
      if (gv) atomicAdd(G + k, gv);
    }
    __syncwarp();
  };
  SegLane s;
  s.soff = 16u * (unsigned)(lane + 1);
  s.roff = 16u + 48u * (unsigned)lane;
  s.nbo = lane == 0 ? 12u : (unsigned)(16 + 3 * kStripW);
  s.sel0 = lane == 0 ? 0x4441u : 0x4440u;
  s.sel1 = lane == 0 ? 0x4442u : 0x4441u;
  s.sel2 = lane == 0 ? 0x4443u : 0x4442u;
  s.sxo = lane == 0 ? 0u : (unsigned)(16 + 3 * kStripW);
  s.lane0 = lane == 0;
  s.lane31 = lane == 31;
  while (q < q1) {
    const int u = (int)(q / kBandH);
    if (cur < 0 || u >= img_u1) {  // a warp's strip rows only grow
      const int img = n == 1 ? 0 : image_of_tile(unit_start, n, u);
      if (cur >= 0 && img != cur) flush_warp(cur);
      cur = img;
      im = tab.desc(img);
      img_u0 = tab.unit0(img);
      img_u1 = n == 1 ? total : tab.unit0(img + 1);
      nb = (im.H + kBandH - 1) / kBandH;
    }
    const int sx = (u - img_u0) / nb;
    const long long qc0 = (long long)kBandH * (img_u0 + (long long)sx * nb);  // the column's first strip row
    const long long qe = min(q1, qc0 + (long long)kBandH * nb);
    const int ya = (int)(q - qc0), yb = min((int)(qe - qc0), im.H);
    q = qe;
    if (ya >= yb) continue;
    const int x0 = sx * kStripW;
    s.in = im.in;
    s.pitch = im.in_pitch;
    s.H = im.H;
    s.goff = 3 * x0 + 16 * lane;
    s.rowbytes = 3 * im.W;
    s.cnt = im.W - (x0 + 16 * lane);
    const int rb = 3 * (im.W - x0 - kStripW);  // bytes right of the strip in a row
    s.left_nb = x0 > 0;
    s.right_nb = rb > 0;
    s.xoff = lane == 0 ? 3 * x0 - 16 : 3 * (x0 + kStripW);
    s.xbytes = lane == 0 ? (s.left_nb ? 16 : 0) : (lane == 1 ? min(max(rb, 0), 16) : 0);
    s.use_nb = (s.lane0 && s.left_nb) || (s.lane31 && s.right_nb);
    if (all_edge || x0 + kStripW > im.W) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        s.eb[i] = min(max(s.rowbytes - (s.goff + 512 * i), 0), 16);
        s.eo[i] = s.eb[i] > 0 ? s.goff + 512 * i : 0;
      }
      // every counted row adds kStripW - w pixels of level 0 beyond the image (w = W - x0 pixels
      // inside), less the one that replicates the border (counted, and taken back, at its own level)
      const int w = im.W - x0;
      if (w < kStripW) phantom += (unsigned)(yb - ya) * (unsigned)(kStripW - w - ((w & 15) ? 1 : 0));
      bad |= roll_run_edge<kClamp>(s, ya, yb, wring, wring_sh, hs_sh, hg_adj, mclipf, kk);
    } else
      bad |= roll_run<false, kClamp>(s, ya, yb, wring, wring_sh, hs_sh, hg_adj, mclipf, kk);
  }
  // the warps' last images: sum the warps that share an image, one global add per level
  __syncwarp();
  if (lane == 0) {
    hist[warp][0][0] -= phantom;
    warp_img[warp] = cur;
  }
  __syncthreads();
  for (int idx = tid; idx < 2 * kHBins; idx += kHT) {
    const int which = idx / kHBins, k = idx % kHBins;
    if (k >= K) continue;
    for (int w = 0; w < kHW; ++w) {
      const int im_idx = warp_img[w];
      bool first = im_idx >= 0;
      for (int v = 0; v < w && first; ++v) first = warp_img[v] != im_idx;
      if (!first) continue;
      unsigned sum = 0;
      for (int v = w; v < kHW; ++v)
        if (warp_img[v] == im_idx) sum += hist[v][0][which * kHBins + k] + hist[v][1][which * kHBins + k];
      unsigned* dst = reinterpret_cast<unsigned*>(slots + (size_t)im_idx * slot_bytes + (which ? lay.G : lay.S));
      if (sum) atomicAdd(dst + k, sum);
    }
  }
  if (bad) atomicOr(status, kStRange);
}

// Staged-tile histogram pass for small images and batches: a CTA per 128 x 32 tile, its rows
// staged into shared memory by asynchronous 16-byte copies (double buffered: the next tile's
// copies run while the current tile is processed); V is built four pixels per thread with byte
// permutes and the separable Sobel operator evaluated on eight pixels per thread.  With eight
// warps on each tile it has the parallelism small launches need; the strip kernel above reads
// large images faster.
constexpr int kRawRow = 416;              // staged bytes per tile row: [3 x0 - 16, 3 x0 + 400)
constexpr int kRawChunks = kRawRow / 16;
constexpr int kVTS = 136;                 // V tile row stride; column c holds x = x0 - 4 + c
constexpr int kVGroups = kVTS / 4;        // 4-pixel groups per V tile row

// Issues the copies of tile (x0, y0) of `im`: rows y0-1 .. y0+32 (clamped), bytes
// [3 x0 - 16, 3 x0 + 400) of each row; bytes outside the row are zero-filled and never read.
__device__ __forceinline__ void stage_tile(const ImageDesc& im, int x0, int y0, unsigned char* raw) {
  const long long rowbytes = 3LL * im.W;
  const long long start = 3LL * x0 - 16;
  for (int e = threadIdx.x; e < kVH * kRawChunks; e += kThreads) {
    const int r = e / kRawChunks, ch = e - r * kRawChunks;
    const int y = clampi(y0 - 1 + r, 0, im.H - 1);
    const unsigned char* row = im.in + (long long)y * im.in_pitch;
    const long long b0 = start + 16LL * ch;
    int nb = 0;
    if (b0 >= 0 && b0 < rowbytes) nb = (int)(rowbytes - b0 < 16 ? rowbytes - b0 : 16);
    cp_async16z(raw + r * kRawRow + ch * 16, nb > 0 ? (const void*)(row + b0) : (const void*)row, nb);
  }
  cp_async_commit();
}

// Nearest integer to sqrt(m2) (halves up), clipped to K-1, branch free, for 0 <= m2 < 2^23.
// float(m2) and floor() use the 2^23 magic number (no conversion unit); the hardware square
// root estimate s is within 0.25 of sqrt(m2), so g0 = floor(s + 1/4) is the answer or one
// below it, and the exact test (2 g0 + 1)^2 <= 4 m2 decides.
__device__ __forceinline__ unsigned grad_level(int m2, int K) {
  const float f = __int_as_float(0x4B000000 | m2) - 8388608.0f;
  float s;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(s) : "f"(f));
  const int g0 = __float_as_int(__fadd_rd(s + 0.25f, 8388608.0f)) & 0x7FFFFF;
  const int t = 2 * g0 + 1;
  const int g = g0 + (t * t <= 4 * m2 ? 1 : 0);
  return (unsigned)min(g, K - 1);
}

__device__ __forceinline__ unsigned byte_of(const unsigned (&w)[4], int k) { return (w[k >> 2] >> (8 * (k & 3))) & 0xffu; }

__global__ void __launch_bounds__(kThreads) hist_u8v_kernel(const ImgTab tab, int total, int K,
                                                            uint8_t* slots, size_t slot_bytes, SlotLayout lay,
                                                            unsigned* status) {
  pdl_wait();     // the previous kernel on the stream has finished
  pdl_trigger();  // the next one may be scheduled (it waits for this one)
  const int n = tab.n;
  const int* __restrict__ tile_start = tab.tiles;  // (n > 1 only)
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned* hs = reinterpret_cast<unsigned*>(smem);        // per-warp H_C(S) copies
  unsigned* hg = hs + kWarps * K;                          // per-warp H_C(grad S) copies
  unsigned char* vt = reinterpret_cast<unsigned char*>(hg + kWarps * K);
  unsigned char* raw = vt + kVH * kVTS;                    // two staging buffers
  const int tid = threadIdx.x, warp = tid >> 5;
  unsigned* my_hs = hs + warp * K;
  unsigned* my_hg = hg + warp * K;
  for (int k = tid; k < 2 * kWarps * K; k += kThreads) hs[k] = 0u;
  const unsigned kmask = K >= 256 ? 0u : 0x01010101u * (unsigned)(K - 1);

  const int chunk = (total + gridDim.x - 1) / gridDim.x;
  const int t0 = blockIdx.x * chunk, t1 = min(total, t0 + chunk);
  int cur = -1;
  bool range_bad = false;
  auto tile_xy = [&](int t, int& img, int& x0, int& y0) {
    img = image_of_tile(tile_start, n, t);
    const ImageDesc im = tab.desc(img);
    const int lt = t - tab.tile0(img);
    const int tiles_x = (im.W + kTileW - 1) / kTileW;
    x0 = (lt % tiles_x) * kTileW;
    y0 = (lt / tiles_x) * kTileH;
  };
  auto flush = [&](int im_idx) {
    __syncthreads();
    unsigned* S = reinterpret_cast<unsigned*>(slots + (size_t)im_idx * slot_bytes + lay.S);
    unsigned* G = reinterpret_cast<unsigned*>(slots + (size_t)im_idx * slot_bytes + lay.G);
    for (int k = tid; k < K; k += kThreads) {
      unsigned sv = 0, gv = 0;
      for (int c = 0; c < kWarps; ++c) {
        sv += hs[c * K + k]; gv += hg[c * K + k];
        hs[c * K + k] = 0u; hg[c * K + k] = 0u;
      }
      if (sv) atomicAdd(S + k, sv);
      if (gv) atomicAdd(G + k, gv);
    }
    __syncthreads();
  };
  __syncthreads();
  if (t0 < t1) {
    int img, x0, y0;
    tile_xy(t0, img, x0, y0);
    stage_tile(tab.desc(img), x0, y0, raw);
  }
  for (int t = t0; t < t1; ++t) {
    int img, x0, y0;
    tile_xy(t, img, x0, y0);
    unsigned char* rb = raw + ((t - t0) & 1) * (kVH * kRawRow);
    if (t + 1 < t1) {
      int img2, x2, y2;
      tile_xy(t + 1, img2, x2, y2);
      stage_tile(tab.desc(img2), x2, y2, raw + ((t + 1 - t0) & 1) * (kVH * kRawRow));
    } else {
      cp_async_commit();
    }
    cp_async_wait<1>();
    __syncthreads();
    if (img != cur) {
      if (cur >= 0) flush(cur);
      cur = img;
    }
    const ImageDesc im = tab.desc(img);
    // V = max(r, g, b), four pixels per thread: staged bytes 12u+4 .. 12u+15 hold columns 4u .. 4u+3
    for (int e = tid; e < kVH * kVGroups; e += kThreads) {
      const int r = e / kVGroups, u = e - r * kVGroups;
      const unsigned* src = reinterpret_cast<const unsigned*>(rb + r * kRawRow + 12 * u + 4);
      const unsigned w0 = src[0], w1 = src[1], w2 = src[2];  // bytes up to 12*33+15 < kRawRow
      const unsigned R = __byte_perm(__byte_perm(w0, w1, 0x0630), w2, 0x5210);
      const unsigned Gc = __byte_perm(__byte_perm(w0, w1, 0x0741), w2, 0x6210);
      const unsigned B = __byte_perm(__byte_perm(w0, w1, 0x0052), w2, 0x7410);
      unsigned v4 = __vmaxu4(__vmaxu4(R, Gc), B);
      if (kmask) {
        // only columns inside the image count for the range check
        const int xa = x0 - 4 + 4 * u;
        unsigned live = 0;
        for (int q = 0; q < 4; ++q)
          if (xa + q >= 0 && xa + q < im.W) live |= 0xffu << (8 * q);
        if (__vcmpgtu4(v4, kmask) & live) range_bad = true;
        v4 = __vminu4(v4, kmask);
      }
      *reinterpret_cast<unsigned*>(vt + r * kVTS + 4 * u) = v4;
    }
    __syncthreads();
    // replicate the border into the halo columns that fall outside the image
    if (tid < kVH) {
      unsigned char* row = vt + tid * kVTS;
      if (x0 == 0) row[3] = row[4];
      if (x0 + kTileW >= im.W) row[im.W - x0 + 4] = row[im.W - x0 + 3];
    }
    __syncthreads();
    // separable Sobel on eight pixels per thread: columns 8v+3 .. 8v+12 of three V rows
    for (int e = tid; e < kTileH * (kTileW / 8); e += kThreads) {
      const int r = e >> 4, v = e & 15;
      const int xs = x0 + 8 * v;
      if (y0 + r >= im.H || xs >= im.W) continue;
      const int npx = min(8, im.W - xs);
      const unsigned char* base = vt + r * kVTS + 8 * v;
      unsigned tw[4], mw[4], bw[4];
      {
        const uint2 a = *reinterpret_cast<const uint2*>(base), b = *reinterpret_cast<const uint2*>(base + 8);
        tw[0] = a.x; tw[1] = a.y; tw[2] = b.x; tw[3] = b.y;
        const uint2 c = *reinterpret_cast<const uint2*>(base + kVTS), d = *reinterpret_cast<const uint2*>(base + kVTS + 8);
        mw[0] = c.x; mw[1] = c.y; mw[2] = d.x; mw[3] = d.y;
        const uint2 f = *reinterpret_cast<const uint2*>(base + 2 * kVTS),
                    g = *reinterpret_cast<const uint2*>(base + 2 * kVTS + 8);
        bw[0] = f.x; bw[1] = f.y; bw[2] = g.x; bw[3] = g.y;
      }
      int cs[10], dd[10];
#pragma unroll
      for (int k = 0; k < 10; ++k) {
        const int tv = (int)byte_of(tw, k + 3), mv = (int)byte_of(mw, k + 3), bv = (int)byte_of(bw, k + 3);
        cs[k] = tv + 2 * mv + bv;
        dd[k] = bv - tv;
      }
#pragma unroll
      for (int p = 0; p < 8; ++p) {
        if (p < npx) {
          const int gx = cs[p + 2] - cs[p];
          const int gy = dd[p] + 2 * dd[p + 1] + dd[p + 2];
          const unsigned g = grad_level(gx * gx + gy * gy, K);
          atomicAdd(my_hs + byte_of(mw, p + 4), 1u);
          atomicAdd(my_hg + g, 1u);
        }
      }
    }
  }
  if (cur >= 0) flush(cur);
  if (range_bad) atomicOr(status, kStRange);
}

// kAll: K = 256, every 8-bit value is a level (no clamp, no range check).
template <bool kAll>
__global__ void __launch_bounds__(kThreads, 8) apply_u8v_kernel(const ImgTab tab, int total, int K,
                                                             const uint8_t* slots, size_t slot_bytes, SlotLayout lay,
                                                             unsigned* status) {
  pdl_wait();     // the previous kernel on the stream has finished
  pdl_trigger();  // the next one may be scheduled (it waits for this one)
  const int n = tab.n;
  const int* __restrict__ tile_start = tab.tiles;  // (n > 1 only)
  // per level V: out_c = (c F_V + B_V) >> 24 with F_V = ceil(V' 2^24 / V), B_V = 2^23, which is
  // floor(c V'/V + 1/2) exactly for c <= V < 256 (the sum is below V' 2^24 + V + 2^23 < 2^32 and
  // overshoots by at most c / 2^24 < 1/(2V)); V = 0 gives F = 0, B = V' << 24.  The result sits in
  // the top byte, so four of them go into an output word with three byte permutes.
  __shared__ uint2 fb[256];
  const int tid = threadIdx.x;
  const int chunk = (total + gridDim.x - 1) / gridDim.x;
  const int t0 = blockIdx.x * chunk, t1 = min(total, t0 + chunk);
  const unsigned vmax = (unsigned)(K - 1);
  bool range_bad = false;
  // a CTA's tiles are consecutive: the image and the tile's column and row advance incrementally
  int img = -1, img_t1 = 0, tiles_x = 1, tx = 0, ty = 0;
  ImageDesc im{};
  for (int t = t0; t < t1; ++t) {
    if (t >= img_t1) {
      img = img < 0 ? image_of_tile(tile_start, n, t) : img + 1;
      __syncthreads();
      const unsigned short* gl = reinterpret_cast<const unsigned short*>(slots + (size_t)img * slot_bytes + lay.lut);
      for (int k = tid; k < 256; k += kThreads) {
        const unsigned vp = k < K ? gl[k] : 0u;
        fb[k] = k == 0 ? make_uint2(0u, vp << 24) : make_uint2(((vp << 24) + (unsigned)k - 1u) / (unsigned)k, 1u << 23);
      }
      __syncthreads();
      im = tab.desc(img);
      img_t1 = n == 1 ? total : tab.tile0(img + 1);
      tiles_x = (im.W + kTileW - 1) / kTileW;
      const int lt = t - tab.tile0(img);
      ty = lt / tiles_x;
      tx = lt - ty * tiles_x;
    }
    const int x = tx * kTileW + 16 * (tid & 7);
    const int y = ty * kTileH + (tid >> 3);
    if (++tx == tiles_x) {
      tx = 0;
      ++ty;
    }
    if (y >= im.H || x >= im.W) continue;
    const unsigned char* src = im.in + (long long)y * im.in_pitch + 3LL * x;
    unsigned char* dst = im.out + (long long)y * im.out_pitch + 3LL * x;
    if (x + 16 <= im.W) {
      const uint4* s4 = reinterpret_cast<const uint4*>(src);
      const uint4 a = s4[0], b = s4[1], c = s4[2];
      const unsigned w[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
      unsigned o[12];
#pragma unroll
      for (int g = 0; g < 4; ++g) {  // four pixels: output words 3g .. 3g + 2
        unsigned t[12];              // output byte 12 g + b in the top byte of t[b]
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          unsigned ch[3];
#pragma unroll
          for (int q = 0; q < 3; ++q) ch[q] = __byte_perm(w[3 * g + ((3 * p + q) >> 2)], 0u, 0x4440 + ((3 * p + q) & 3));
          unsigned V = __vimax3_u32(ch[0], ch[1], ch[2]);
          if (!kAll) {
            range_bad |= V > vmax;
            V = min(V, vmax);
          }
          const uint2 f = fb[V];
#pragma unroll
          for (int q = 0; q < 3; ++q) t[3 * p + q] = ch[q] * f.x + f.y;
        }
#pragma unroll
        for (int q = 0; q < 3; ++q)
          o[3 * g + q] = __byte_perm(__byte_perm(t[4 * q], t[4 * q + 1], 0x0073),
                                     __byte_perm(t[4 * q + 2], t[4 * q + 3], 0x0073), 0x5410);
      }
      uint4* d4 = reinterpret_cast<uint4*>(dst);
      d4[0] = make_uint4(o[0], o[1], o[2], o[3]);
      d4[1] = make_uint4(o[4], o[5], o[6], o[7]);
      d4[2] = make_uint4(o[8], o[9], o[10], o[11]);
    } else {
      for (int p = 0; p < im.W - x; ++p) {
        const unsigned ch[3] = {src[3 * p], src[3 * p + 1], src[3 * p + 2]};
        unsigned V = max(max(ch[0], ch[1]), ch[2]);
        range_bad |= V > vmax;
        V = min(V, vmax);
        const uint2 f = fb[V];
        for (int q = 0; q < 3; ++q) dst[3 * p + q] = (unsigned char)((ch[q] * f.x + f.y) >> 24);
      }
    }
  }
  if (range_bad) atomicOr(status, kStRange);
}

// Self-test of the three gradient-level forms above (a test hook, not part of the method): the level
// of every squared Sobel magnitude m2 in [m2_first, m2_first + n), by form 0 (strip kernel), 1
// (staged-tile kernel) or 2 (generic kernel), written to out[m2 - m2_first].
__global__ void grad_level_probe_kernel(int form, int K, int m2_first, int n, uint16_t* out) {
  const int mclip = K * K - K;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int m2 = m2_first + t;
    unsigned g;
    if (form == 0) {
      g = grad_bits_f((float)m2, (float)mclip) - 0x4B000000u;  // m2 < 2^24: exact in FP32
    } else if (form == 1) {
      g = grad_level(m2, K);
    } else {
      g = round_sqrt((unsigned)m2);
      g = g < (unsigned)(K - 1) ? g : (unsigned)(K - 1);
    }
    out[t] = (uint16_t)g;
  }
}

}  // namespace

cudaError_t launch_grad_level_probe(int form, int K, int m2_first, int n, uint16_t* out, cudaStream_t st) {
  const int blocks = (int)std::min<long long>(4096, ((long long)n + 255) / 256);
  return launch_kernel(grad_level_probe_kernel, dim3(blocks), dim3(256), 0, st, false, form, K, m2_first, n, out);
}

cudaError_t launch_hist(const ImgTab& tab, int total_tiles, int total_units, int interior_units, int elem_bytes,
                        int K, uint8_t* slots,
                        size_t slot_bytes, SlotLayout lay, unsigned* status, int sms, int ctas_per_sm,
                        cudaStream_t st, bool fast, bool pdl, bool forward, int M) {
  const int copies = K <= 256 ? kWarps : 1;
  if (M <= 0) M = K;
  int shift = 0;
  while ((K << shift) < M) ++shift;
  if (forward || M != K) fast = false;  // forward differences and binned data run on the generic kernel
  const size_t smem = (size_t)2 * copies * K * sizeof(unsigned) + (size_t)kVH * kVW * sizeof(unsigned short);
  // strips when the launch has at least HR_STRIP_MIN_FACTOR of them per warp of a full grid (one
  // large image or a large batch), staged tiles otherwise
  if (elem_bytes == 1 && fast && K <= kHBins && total_units >= HR_STRIP_MIN_FACTOR * sms * kHW) {
    // one CTA per SM for a single image (the rest of each SM's registers for other calls' apply
    // passes), two for a batch, which runs alone (512 mixed images: 1.92 against 2.19 ms per call)
    const dim3 grid(tab.n > 1 ? 2 * sms : sms);
    const int all_edge = 8LL * interior_units < 7LL * total_units ? 1 : 0;  // more than 1/8 edge strips
    if (K < kHBins) {
      cudaFuncSetAttribute(hist_u8s_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRollSmem);
      return launch_kernel(hist_u8s_kernel<true>, grid, dim3(kHT), kRollSmem, st, pdl, tab, total_units, all_edge, K,
                           slots, slot_bytes, lay, status);
    }
    cudaFuncSetAttribute(hist_u8s_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRollSmem);
    return launch_kernel(hist_u8s_kernel<false>, grid, dim3(kHT), kRollSmem, st, pdl, tab, total_units, all_edge, K,
                         slots, slot_bytes, lay, status);
  }
  int grid = sms * ctas_per_sm;
  if (grid > total_tiles) grid = total_tiles;
  if (grid < 1) grid = 1;
  // Each kernel's dynamic shared-memory limit is set to the most any call of it takes (K = 256 for the
  // 8-bit kernels, K = 4096 for the generic one), the same value on every call, so calls of contexts
  // on several host threads cannot lower it under each other's launches; a launch still takes only
  // its own size.
  if (elem_bytes == 1 && fast) {
    const size_t smem_v = (size_t)2 * kWarps * K * sizeof(unsigned) + (size_t)kVH * kVTS + (size_t)2 * kVH * kRawRow;
    const size_t smem_v_max = (size_t)2 * kWarps * kHBins * sizeof(unsigned) + (size_t)kVH * kVTS + (size_t)2 * kVH * kRawRow;
    cudaFuncSetAttribute(hist_u8v_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_v_max);
    return launch_kernel(hist_u8v_kernel, dim3(grid), dim3(kThreads), smem_v, st, pdl, tab, total_tiles, K, slots,
                         slot_bytes, lay, status);
  }
  // (K <= 256: kWarps copies of K bins; above: one copy of up to 4096)
  const size_t smem_max = std::max((size_t)2 * kWarps * kHBins, (size_t)2 * 4096) * sizeof(unsigned) +
                          (size_t)kVH * kVW * sizeof(unsigned short);
  if (elem_bytes == 1) {
    cudaFuncSetAttribute(hist_kernel<uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    return launch_kernel(hist_kernel<uint8_t>, dim3(grid), dim3(kThreads), smem, st, pdl, tab, total_tiles, K, slots,
                         slot_bytes, lay, status, (int)forward, shift, M);
  }
  cudaFuncSetAttribute(hist_kernel<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
  return launch_kernel(hist_kernel<uint16_t>, dim3(grid), dim3(kThreads), smem, st, pdl, tab, total_tiles, K, slots,
                       slot_bytes, lay, status, (int)forward, shift, M);
}

cudaError_t launch_apply(const ImgTab& tab, int total_tiles, int elem_bytes, int K, uint8_t* slots, size_t slot_bytes,
                         SlotLayout lay, unsigned* status, int sms, int ctas_per_sm, cudaStream_t st, bool fast,
                         bool pdl, int M) {
  if (M <= 0) M = K;
  int shift = 0;
  while ((K << shift) < M) ++shift;
  if (M != K) fast = false;  // binned data: the generic kernel
  const int nt = elem_bytes == 1 ? M : K;
  const size_t smem = (size_t)((nt * 2 + 15) & ~15) + (size_t)nt * sizeof(float);
  const int grid = max(1, min(sms * ctas_per_sm, total_tiles));
  if (elem_bytes == 1 && fast) {
    if (K == 256)
      return launch_kernel(apply_u8v_kernel<true>, dim3(grid), dim3(kThreads), 0, st, pdl, tab, total_tiles, K, slots,
                           slot_bytes, lay, status);
    return launch_kernel(apply_u8v_kernel<false>, dim3(grid), dim3(kThreads), 0, st, pdl, tab, total_tiles, K, slots,
                         slot_bytes, lay, status);
  }
  if (elem_bytes == 1)
    return launch_kernel(apply_kernel<uint8_t>, dim3(grid), dim3(kThreads), smem, st, pdl, tab, total_tiles, K, slots,
                         slot_bytes, lay, status, shift, M);
  return launch_kernel(apply_kernel<uint16_t>, dim3(grid), dim3(kThreads), smem, st, pdl, tab, total_tiles, K, slots,
                       slot_bytes, lay, status, shift, M);
}

}  // namespace hr
