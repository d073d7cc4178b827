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
// Histogram pass: one warp walks one strip of kStripW x kBandH pixels.  Lane l owns the 16
// pixels [x0 + 16 l, x0 + 16 l + 16) of the strip's rows, so the warp reads 1536 contiguous bytes
// per row and the warps of a CTA, dealt consecutive strips, read whole image rows together (DRAM
// pages are read through; narrow tiles spread over many rows reached barely half the bandwidth).
// Each lane copies its 48 bytes of the ten rows y0 - 1 .. y0 + 8 (clamped to the image: replicate
// border) into its own shared-memory ring kRing rows ahead of use with asynchronous copies.
// V = max(r, g, b) is kept as packed 16-bit pairs, even and odd pixels apart, so one 32-bit add
// forms a Sobel partial sum of two pixels; the columns left and right of a lane's 16 pixels come
// from the neighbouring lanes by shuffles, or at the strip edge from one 4-byte copy.  The squared
// magnitude of each pair is unpacked with a sign extension and a high multiply.  Counts go to
// per-warp shared histograms by shared-memory reductions; each CTA deals its contiguous range of
// strips out to its warps through a shared counter.
//
// Apply pass: 16 pixels (48 bytes, three 16-byte vectors) per thread each way.
// ------------------------------------------------------------------------------------------------
#ifndef HR_HIST_WARPS
#define HR_HIST_WARPS 16
#endif
constexpr int kHW = HR_HIST_WARPS;  // warps per CTA of the fast histogram pass
constexpr int kHT = kHW * 32;
#ifndef HR_STRIP_MIN_FACTOR
#define HR_STRIP_MIN_FACTOR 2  // strips per warp from which one image takes the strip kernel
#endif
constexpr int kHBins = 256;     // per-warp histogram stride (the 8-bit pass has K <= 256)
constexpr int kRing = 3;        // rows in flight per warp (3 measured faster than 4 with 4-row bands)
constexpr int kSlot = 32 * 48;  // bytes of one ring slot of a warp: 48 per lane

// Shared memory of the fast histogram pass: per warp its two histograms, then per warp a ring
// of kRing row slots (the strip's 1536 bytes of a row: 48 bytes per lane) and of kRing neighbour
// words per lane.
constexpr size_t kHistSmem = (size_t)kHW * (4 * kHBins * 4 + kRing * kSlot + kRing * 32 * 4);

// One row of V around a lane's 16 pixels.
struct VRow {
  unsigned e[4], o[4];  // V of pixels (4w, 4w+2) and (4w+1, 4w+3) as 16-bit pairs, w = 0..3
  unsigned l, r;        // high half of l: V of the pixel left of the 16; low half of r: the one right
};

// Per-lane geometry of the current strip and the lane's view of the warp's ring.
struct LaneTile {
  const uint8_t* in;
  long long pitch;
  int W, H;
  int x0, xc, cnt;      // strip origin column, first column of the lane, W - xc
  int lx;
  unsigned char* ring;  // the lane's 48 bytes in slot 0 (slot s at + s * kSlot)
  unsigned char* slot0; // the warp's slot 0
  unsigned* nbr;        // the lane's neighbour word in slot 0 (slot s at + s * 32)
};

__device__ __forceinline__ const uint8_t* row_ptr(const LaneTile& g, int y) {
  return g.in + (long long)clampi(y, 0, g.H - 1) * g.pitch;
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
// 16-byte copy of which only the first `nb` (0..16) bytes are read; the rest is zero-filled.
__device__ __forceinline__ void cp_async16z(void* smem_dst, const void* gsrc, int nb) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gsrc), "r"(nb) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Starts the copies of row y into ring slot `slot` (one commit group per call; empty when
// `live` is false): the strip's 1536 bytes of the row as 96 chunks of 16 bytes, chunk c by lane
// c mod 32, so each copy instruction of the warp covers 512 contiguous bytes (the bytes past the
// image's last pixel are zero-filled), and the 4-byte neighbour words of lanes 0 and 31.  Lanes
// read chunks other lanes copied: a __syncwarp after the wait_group orders copies and reads, one
// before the next copies into a slot orders the reads before them.
__device__ __forceinline__ void issue_row(const LaneTile& g, int slot, int y, bool live) {
  if (live) {
    const uint8_t* row = row_ptr(g, y);
    unsigned char* dst = g.slot0 + slot * kSlot;
    const int b0 = 3 * g.x0, rowbytes = 3 * g.W;
    if (b0 + kSlot <= rowbytes) {
#pragma unroll
      for (int i = 0; i < 3; ++i) cp_async16(dst + 16 * (g.lx + 32 * i), row + b0 + 16 * (g.lx + 32 * i));
    } else {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const int off = 16 * (g.lx + 32 * i);
        const int b = min(max(rowbytes - (b0 + off), 0), 16);
        cp_async16z(dst + off, b > 0 ? (const void*)(row + b0 + off) : (const void*)row, b);
      }
    }
    if (g.lx == 0 && g.x0 > 0) cp_async4(g.nbr + slot * 32, row + 3 * g.x0 - 4);
    else if (g.lx == 31 && g.x0 + kStripW + 2 <= g.W) cp_async4(g.nbr + slot * 32, row + 3 * (g.x0 + kStripW));
  }
  cp_async_commit();
}

// V of two pixels as 16-bit pairs from the 12 bytes of four pixels: a = R0 G0 B0 R1,
// b = G1 B1 R2 G2, c = B2 R3 G3 B3.  Every operand of one 3-way max carries the same filler
// byte above each channel byte, so the halfword maximum is the channel maximum.
__device__ __forceinline__ void vpairs(unsigned a, unsigned b, unsigned c, unsigned& e, unsigned& o) {
  e = __vimax3_u16x2(__byte_perm(a, b, 0x3630), __byte_perm(a, b, 0x3731), __byte_perm(a, c, 0x3432)) & 0x00ff00ffu;
  o = __vimax3_u16x2(__byte_perm(a, c, 0x4543), __byte_perm(b, c, 0x4640), __byte_perm(b, c, 0x4741)) & 0x00ff00ffu;
}

__device__ __forceinline__ unsigned max3b(unsigned w, int s0) {  // max of bytes s0, s0+1, s0+2 of w
  return max(max((w >> (8 * s0)) & 0xffu, (w >> (8 * s0 + 8)) & 0xffu), (w >> (8 * s0 + 16)) & 0xffu);
}

// V row of one lane from ring slot `slot` (row y); all lanes of the warp call it together.
// Positions right of the image's last pixel hold zeros, except the first one, which holds the
// replica of the last pixel (replicate border).
template <bool kEdge, bool kClamp>
__device__ __forceinline__ VRow build_row(const LaneTile& g, int slot, int y, unsigned kk, bool& bad) {
  VRow v;
  const unsigned char* qb = g.ring + slot * kSlot;
  {
    const uint4* q = reinterpret_cast<const uint4*>(qb);
    const uint4 a = q[0], b = q[1], c = q[2];
    vpairs(a.x, a.y, a.z, v.e[0], v.o[0]);
    vpairs(a.w, b.x, b.y, v.e[1], v.o[1]);
    vpairs(b.z, b.w, c.x, v.e[2], v.o[2]);
    vpairs(c.y, c.z, c.w, v.e[3], v.o[3]);
  }
  if (kEdge && g.cnt <= 0) {  // lane right of the image: nothing was copied, nothing is counted
#pragma unroll
    for (int w = 0; w < 4; ++w) v.e[w] = v.o[w] = 0u;
  }
  if (kClamp) {  // K < 256: levels above K - 1 are a range error, clamped so counting stays in bounds
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const unsigned ce = __vimin3_u16x2(v.e[w], kk, kk), co = __vimin3_u16x2(v.o[w], kk, kk);
      bad |= (ce != v.e[w]) | (co != v.o[w]);
      v.e[w] = ce;
      v.o[w] = co;
    }
  }
  // neighbour columns: from the adjacent lanes of the lane row, else from the neighbour word
  v.l = __shfl_up_sync(0xffffffffu, v.o[3], 1);
  v.r = __shfl_down_sync(0xffffffffu, v.e[0], 1);
  if (g.lx == 0) {
    unsigned lv = v.e[0] & 0xffffu;  // x0 == 0: replicate pixel 0
    if (g.x0 > 0) lv = max3b(g.nbr[slot * 32], 1);
    if (kClamp) { bad |= lv > (kk & 0xffffu); lv = min(lv, kk & 0xffffu); }
    v.l = lv << 16;
  }
  if (g.xc + 16 >= g.W) {  // the lane holds the image's last pixel: replicate it to its right
    if (!kEdge || g.cnt >= 16) {
      v.r = v.o[3] >> 16;
    } else if (g.cnt > 0) {
      const unsigned char* lp = qb + 3 * (g.cnt - 1);
      unsigned vlast = max(max((unsigned)lp[0], (unsigned)lp[1]), (unsigned)lp[2]);
      if (kClamp) vlast = min(vlast, kk & 0xffffu);
      v.r = vlast;
#pragma unroll
      for (int w = 0; w < 4; ++w) {  // pixel cnt (zero-filled) becomes the replica
        if (4 * w == g.cnt) v.e[w] = (v.e[w] & 0xffff0000u) | vlast;
        if (4 * w + 2 == g.cnt) v.e[w] = (v.e[w] & 0x0000ffffu) | (vlast << 16);
        if (4 * w + 1 == g.cnt) v.o[w] = (v.o[w] & 0xffff0000u) | vlast;
        if (4 * w + 3 == g.cnt) v.o[w] = (v.o[w] & 0x0000ffffu) | (vlast << 16);
      }
    }
  } else if (g.lx == 31) {
    unsigned rv;
    if (g.x0 + kStripW + 2 <= g.W) {
      rv = max3b(g.nbr[slot * 32], 0);
    } else {  // the right neighbour is the image's last pixel
      const uint8_t* p = row_ptr(g, y) + 3 * (g.x0 + kStripW);
      rv = max(max((unsigned)p[0], (unsigned)p[1]), (unsigned)p[2]);
    }
    if (kClamp) { bad |= rv > (kk & 0xffffu); rv = min(rv, kk & 0xffffu); }
    v.r = rv;
  }
  return v;
}

__device__ __forceinline__ void red_shared(unsigned addr) {
  asm volatile("red.shared.add.u32 [%0], 1;\n" ::"r"(addr) : "memory");
}

// Counts one pixel: V level v into H_C(S); its gradient level, the nearest integer to sqrt(m2)
// clipped to K - 1, into H_C(grad S).  Clipping m2 at K^2 - K first gives the same level, keeps
// m2 below 2^23 so float(m2) is the magic-number conversion, and sqrt.approx is within 2^-19
// relative of sqrt(m2) there, well inside the distance 1/(4 sqrt(m2) + 2) from sqrt(m2) to the
// nearest half integer, so the round-to-nearest add of 2^23 yields the exact level
// (0x4B000000 + level in the float's bits; hg_adj absorbs the 0x4B000000).
__device__ __forceinline__ unsigned strip_grad_bits(int m2, int mclip) {
  const int m2c = min(m2, mclip);
  const float f = __fsub_rn(__int_as_float(0x4B000000 | m2c), 8388608.0f);
  float s;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(s) : "f"(f));
  return __float_as_uint(__fadd_rn(s, 8388608.0f));
}
__device__ __forceinline__ void count_px(int m2, unsigned v, int mclip, unsigned hs_sh, unsigned hg_adj, bool on) {
  const unsigned gb = strip_grad_bits(m2, mclip);
  if (on) {
    red_shared(hg_adj + (gb << 2));
    red_shared(hs_sh + (v << 2));
  }
}

// Two pixels from packed Sobel components: each 32-bit word is HI * 65536 + LO with LO, HI the
// signed components of the low and high pixel (exact: the packed adds never carry out of a
// half by more than the borrow this form absorbs).
__device__ __forceinline__ void count_pair(int gx, int gy, unsigned vpair, int p0, int lim, int mclip,
                                           unsigned hs_sh, unsigned hg_adj) {
  const int ax = (int)(short)gx, ay = (int)(short)gy;
  const int m2a = ax * ax + ay * ay;
  const int dx = gx - ax, dy = gy - ay;
  const int m2b = __mulhi(dx, dx) + __mulhi(dy, dy);
  count_px(m2a, vpair & 0xffffu, mclip, hs_sh, hg_adj, p0 < lim);
  count_px(m2b, vpair >> 16, mclip, hs_sh, hg_adj, p0 + 2 < lim);
}

// Separable Sobel (gx: right minus left column of [1 2 1]^T-weighted sums; gy: bottom minus top
// row of [1 2 1]-weighted sums) and counting for the output row M between rows T and B.
__device__ __forceinline__ void count_row(const VRow& T, const VRow& M, const VRow& B, int lim, int mclip,
                                          unsigned hs_sh, unsigned hg_adj) {
  // column sums cs = T + 2 M + B and differences dd = B - T + 256 per half (in [1, 511]), formed
  // word by word as the window over the four pairs moves right
  auto cs = [](unsigned t, unsigned m, unsigned b) { return t + b + 2u * m; };
  auto dd = [](unsigned t, unsigned b) { return b - t + 0x01000100u; };
  unsigned csOp = cs(T.l, M.l, B.l), ddOp = dd(T.l, B.l);  // odd pair left of pair 0 (high half: x - 1)
  unsigned csEc = cs(T.e[0], M.e[0], B.e[0]), ddEc = dd(T.e[0], B.e[0]);
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    const unsigned csOc = cs(T.o[w], M.o[w], B.o[w]), ddOc = dd(T.o[w], B.o[w]);
    const unsigned csEn = w < 3 ? cs(T.e[w + 1], M.e[w + 1], B.e[w + 1]) : cs(T.r, M.r, B.r);
    const unsigned ddEn = w < 3 ? dd(T.e[w + 1], B.e[w + 1]) : dd(T.r, B.r);
    // odd pixels left of the even pair (4w-1, 4w+1); even pixels right of the odd pair (4w+2, 4w+4)
    const unsigned csOL = __byte_perm(csOp, csOc, 0x5432), ddOL = __byte_perm(ddOp, ddOc, 0x5432);
    const unsigned csER = __byte_perm(csEc, csEn, 0x5432), ddER = __byte_perm(ddEc, ddEn, 0x5432);
    const int gxE = (int)(csOc - csOL);
    const int gyE = (int)(ddOL + 2u * ddEc + ddOc - 0x04000400u);
    const int gxO = (int)(csER - csEc);
    const int gyO = (int)(ddEc + 2u * ddOc + ddER - 0x04000400u);
    count_pair(gxE, gyE, M.e[w], 4 * w, lim, mclip, hs_sh, hg_adj);
    count_pair(gxO, gyO, M.o[w], 4 * w + 1, lim, mclip, hs_sh, hg_adj);
    csOp = csOc; ddOp = ddOc; csEc = csEn; ddEc = ddEn;
  }
}

// One strip for one lane; returns whether a level above K - 1 was seen.  Rows yb .. yb + kBandH + 1
// go through the warp's ring, kRing rows ahead of use.
template <bool kEdge, bool kClamp>
__device__ __forceinline__ bool hist_tile(const LaneTile& g, int yb, int mclip, unsigned kk, unsigned hs_sh,
                                          unsigned hg_adj) {
  constexpr int kRows = kBandH + 2;
  bool bad = false;
  __syncwarp();  // (the previous tile's reads of the ring are done)
#pragma unroll
  for (int r = 0; r < kRing; ++r) issue_row(g, r, yb + r, true);
  cp_async_wait<kRing - 1>();
  __syncwarp();
  VRow v0 = build_row<kEdge, kClamp>(g, 0, yb, kk, bad);
  __syncwarp();
  issue_row(g, 0, yb + kRing, kRing < kRows);
  cp_async_wait<kRing - 1>();
  __syncwarp();
  VRow v1 = build_row<kEdge, kClamp>(g, 1, yb + 1, kk, bad);
  __syncwarp();
  issue_row(g, 1, yb + kRing + 1, kRing + 1 < kRows);
  const int full = kEdge ? min(g.cnt, 16) : 16;
#pragma unroll
  for (int j = 0; j < kBandH; ++j) {
    cp_async_wait<kRing - 1>();
    __syncwarp();
    const VRow v2 = build_row<kEdge, kClamp>(g, (j + 2) % kRing, yb + j + 2, kk, bad);
    __syncwarp();
    issue_row(g, (j + 2) % kRing, yb + j + 2 + kRing, j + 2 + kRing < kRows);
    const int lim = kEdge ? (yb + j + 1 < g.H ? full : 0) : 16;
    count_row(v0, v1, v2, lim, mclip, hs_sh, hg_adj);
    v0 = v1;
    v1 = v2;
  }
  return bad;
}

// Tiles that cross the image's right or bottom edge, kept out of line so the interior path has
// the register file to itself.
template <bool kClamp>
__device__ __noinline__ bool hist_tile_edge(const LaneTile g, int yb, int mclip, unsigned kk, unsigned hs_sh,
                                            unsigned hg_adj) {
  return hist_tile<true, kClamp>(g, yb, mclip, kk, hs_sh, hg_adj);
}

template <bool kClamp>
__global__ void __launch_bounds__(kHT, 1) hist_u8r_kernel(const ImgTab tab, int total, int all_edge, int K,
                                                         uint8_t* slots, size_t slot_bytes, SlotLayout lay,
                                                         unsigned* status) {
  pdl_wait();     // the previous kernel on the stream has finished
  pdl_trigger();  // the next one may be scheduled (it waits for this one)
  const int n = tab.n;
  const int* __restrict__ unit_start = tab.units;  // (n > 1 only)
  extern __shared__ __align__(16) unsigned char hsmem[];
  // per warp two copies (even and odd lanes, which see the most alike levels) of H_C(S), H_C(grad S)
  auto hist = reinterpret_cast<unsigned (*)[2][2][kHBins]>(hsmem);
  unsigned char* ring = hsmem + (size_t)kHW * 4 * kHBins * 4;
  unsigned* nbr = reinterpret_cast<unsigned*>(ring + (size_t)kHW * kRing * kSlot);
  __shared__ int next_tile;
  __shared__ int warp_img[kHW];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned* hw = &hist[warp][0][0][0];
  for (int k = lane; k < 4 * kHBins; k += 32) hw[k] = 0u;
  const int chunk = (total + gridDim.x - 1) / gridDim.x;
  const int t0 = blockIdx.x * chunk, t1 = min(total, t0 + chunk);
  if (tid == 0) next_tile = t0;
  __syncthreads();

  const unsigned hs_sh = (unsigned)__cvta_generic_to_shared(hist[warp][lane & 1][0]);
  const unsigned hg_adj = (unsigned)__cvta_generic_to_shared(hist[warp][lane & 1][1]) - 0x2C000000u;  // - (0x4B000000 << 2)
  const int mclip = K * K - K;
  const unsigned kk = 0x00010001u * (unsigned)(K - 1);
  LaneTile g;
  g.lx = lane;
  g.slot0 = ring + (size_t)warp * kRing * kSlot;
  g.ring = g.slot0 + 48 * lane;
  g.nbr = nbr + warp * kRing * 32 + lane;
  int cur = -1;
  bool bad = false;
  auto flush_warp = [&](int im_idx) {
    __syncwarp();
    unsigned* S = reinterpret_cast<unsigned*>(slots + (size_t)im_idx * slot_bytes + lay.S);
    unsigned* G = reinterpret_cast<unsigned*>(slots + (size_t)im_idx * slot_bytes + lay.G);
    for (int k = lane; k < K; k += 32) {
      const unsigned sv = hist[warp][0][0][k] + hist[warp][1][0][k], gv = hist[warp][0][1][k] + hist[warp][1][1][k];
      hist[warp][0][0][k] = hist[warp][1][0][k] = hist[warp][0][1][k] = hist[warp][1][1][k] = 0u;
      if (sv) atomicAdd(S + k, sv);
      if (gv) atomicAdd(G + k, gv);
    }
    __syncwarp();
  };
  // Units of one image: first its interior strips (row-major), then the edge strips (the right
  // column, then the bottom band), so a warp runs one code path for long stretches: alternating
  // paths thrash the instruction cache.  When edge strips are many (batches of small images),
  // all strips take the edge path (all_edge).  A warp's units only grow, so the image is looked
  // up again only when a unit passes the current image's end.
  int img_start = 0, img_end = 0, nx = 0, nxi = 0, nyi = 0, n_int = 0, n_right = 0;
  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(&next_tile, 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= t1) break;
    if (cur < 0 || t >= img_end) {
      const int img = image_of_tile(unit_start, n, t);
      if (cur >= 0 && img != cur) flush_warp(cur);
      cur = img;
      const ImageDesc im = tab.desc(img);
      g.in = im.in;
      g.pitch = im.in_pitch;
      g.W = im.W;
      g.H = im.H;
      img_start = tab.unit0(img);
      img_end = n == 1 ? total : tab.unit0(img + 1);
      nx = (g.W + kStripW - 1) / kStripW;
      nxi = g.W / kStripW;
      nyi = g.H / kBandH;
      n_int = nxi * nyi;
      n_right = (nx - nxi) * nyi;
    }
    const int lt = t - img_start;
    int sx, sy;
    if (lt < n_int) {
      sy = lt / nxi;
      sx = lt - sy * nxi;
    } else if (lt - n_int < n_right) {
      sx = nxi;
      sy = lt - n_int;
    } else {
      sx = lt - n_int - n_right;
      sy = nyi;
    }
    g.x0 = sx * kStripW;
    const int y0 = sy * kBandH;
    g.xc = g.x0 + 16 * g.lx;
    g.cnt = g.W - g.xc;
    const int yb = y0 - 1;
    if (all_edge || lt >= n_int) bad |= hist_tile_edge<kClamp>(g, yb, mclip, kk, hs_sh, hg_adj);
    else bad |= hist_tile<false, kClamp>(g, yb, mclip, kk, hs_sh, hg_adj);
  }
  // the warps' last images: sum the warps that share an image, one global add per level
  if (lane == 0) warp_img[warp] = cur;
  __syncthreads();
  {
    for (int idx = tid; idx < 2 * kHBins; idx += kHT) {
      const int which = idx / kHBins, k = idx % kHBins;
      if (k >= K) continue;
      for (int w = 0; w < kHW; ++w) {
        const int im_idx = warp_img[w];
        bool first = im_idx >= 0;
        for (int u = 0; u < w && first; ++u) first = warp_img[u] != im_idx;
        if (!first) continue;
        unsigned s = 0;
        for (int u = w; u < kHW; ++u)
          if (warp_img[u] == im_idx) s += hist[u][0][which][k] + hist[u][1][which][k];
        unsigned* dst = reinterpret_cast<unsigned*>(slots + (size_t)im_idx * slot_bytes + (which ? lay.G : lay.S));
        if (s) atomicAdd(dst + k, s);
      }
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

__global__ void __launch_bounds__(kThreads) apply_u8v_kernel(const ImgTab tab, int total, int K,
                                                             const uint8_t* slots, size_t slot_bytes, SlotLayout lay,
                                                             unsigned* status) {
  pdl_wait();     // the previous kernel on the stream has finished
  pdl_trigger();  // the next one may be scheduled (it waits for this one)
  const int n = tab.n;
  const int* __restrict__ tile_start = tab.tiles;  // (n > 1 only)
  // per level V: out_c = (c F_V + B_V) >> 18 with F_V = ceil(V' 2^18 / V), B_V = 2^17, which is
  // floor(c V'/V + 1/2) exactly for c <= V < 256 (the product is at most V' 2^18 + V < 2^32 and
  // overshoots by at most c / 2^18 < 1/(2V)); V = 0 gives F = 0, B = V' << 18.
  __shared__ uint2 fb[256];
  const int tid = threadIdx.x;
  const int chunk = (total + gridDim.x - 1) / gridDim.x;
  const int t0 = blockIdx.x * chunk, t1 = min(total, t0 + chunk);
  const unsigned vmax = (unsigned)(K - 1);
  int cur = -1;
  bool range_bad = false;
  for (int t = t0; t < t1; ++t) {
    const int img = image_of_tile(tile_start, n, t);
    if (img != cur) {
      __syncthreads();
      const unsigned short* gl = reinterpret_cast<const unsigned short*>(slots + (size_t)img * slot_bytes + lay.lut);
      for (int k = tid; k < 256; k += kThreads) {
        const unsigned vp = k < K ? gl[k] : 0u;
        fb[k] = k == 0 ? make_uint2(0u, vp << 18) : make_uint2(((vp << 18) + (unsigned)k - 1u) / (unsigned)k, 1u << 17);
      }
      __syncthreads();
      cur = img;
    }
    const ImageDesc im = tab.desc(img);
    const int lt = t - tab.tile0(img);
    const int tiles_x = (im.W + kTileW - 1) / kTileW;
    const int x = (lt % tiles_x) * kTileW + 16 * (tid & 7);
    const int y = (lt / tiles_x) * kTileH + (tid >> 3);
    if (y >= im.H || x >= im.W) continue;
    const unsigned char* src = im.in + (long long)y * im.in_pitch + 3LL * x;
    unsigned char* dst = im.out + (long long)y * im.out_pitch + 3LL * x;
    if (x + 16 <= im.W) {
      const uint4* s4 = reinterpret_cast<const uint4*>(src);
      const uint4 a = s4[0], b = s4[1], c = s4[2];
      const unsigned w[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
      unsigned o[12];
#pragma unroll
      for (int q = 0; q < 12; ++q) o[q] = 0u;
#pragma unroll
      for (int p = 0; p < 16; ++p) {
        unsigned ch[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) ch[q] = __byte_perm(w[(3 * p + q) >> 2], 0u, 0x4440 + ((3 * p + q) & 3));
        unsigned V = max(max(ch[0], ch[1]), ch[2]);
        range_bad |= V > vmax;
        V = min(V, vmax);
        const uint2 f = fb[V];
#pragma unroll
        for (int q = 0; q < 3; ++q) o[(3 * p + q) >> 2] |= ((ch[q] * f.x + f.y) >> 18) << (8 * ((3 * p + q) & 3));
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
        for (int q = 0; q < 3; ++q) dst[3 * p + q] = (unsigned char)((ch[q] * f.x + f.y) >> 18);
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
      g = strip_grad_bits(m2, mclip) - 0x4B000000u;
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
    const dim3 grid(sms);
    const int all_edge = 8LL * interior_units < 7LL * total_units ? 1 : 0;  // more than 1/8 edge strips
    if (K < kHBins) {
      cudaFuncSetAttribute(hist_u8r_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kHistSmem);
      return launch_kernel(hist_u8r_kernel<true>, grid, dim3(kHT), kHistSmem, st, pdl, tab, total_units, all_edge, K, slots,
                           slot_bytes, lay, status);
    }
    cudaFuncSetAttribute(hist_u8r_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kHistSmem);
    return launch_kernel(hist_u8r_kernel<false>, grid, dim3(kHT), kHistSmem, st, pdl, tab, total_units, all_edge, K, slots,
                         slot_bytes, lay, status);
  }
  int grid = sms * ctas_per_sm;
  if (grid > total_tiles) grid = total_tiles;
  if (grid < 1) grid = 1;
  if (elem_bytes == 1 && fast) {
    const size_t smem_v = (size_t)2 * kWarps * K * sizeof(unsigned) + (size_t)kVH * kVTS + (size_t)2 * kVH * kRawRow;
    cudaFuncSetAttribute(hist_u8v_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_v);
    return launch_kernel(hist_u8v_kernel, dim3(grid), dim3(kThreads), smem_v, st, pdl, tab, total_tiles, K, slots,
                         slot_bytes, lay, status);
  }
  if (elem_bytes == 1) {
    cudaFuncSetAttribute(hist_kernel<uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return launch_kernel(hist_kernel<uint8_t>, dim3(grid), dim3(kThreads), smem, st, pdl, tab, total_tiles, K, slots,
                         slot_bytes, lay, status, (int)forward, shift, M);
  }
  cudaFuncSetAttribute(hist_kernel<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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
  if (elem_bytes == 1 && fast)
    return launch_kernel(apply_u8v_kernel, dim3(grid), dim3(kThreads), 0, st, pdl, tab, total_tiles, K, slots,
                         slot_bytes, lay, status);
  if (elem_bytes == 1)
    return launch_kernel(apply_kernel<uint8_t>, dim3(grid), dim3(kThreads), smem, st, pdl, tab, total_tiles, K, slots,
                         slot_bytes, lay, status, shift, M);
  return launch_kernel(apply_kernel<uint16_t>, dim3(grid), dim3(kThreads), smem, st, pdl, tab, total_tiles, K, slots,
                       slot_bytes, lay, status, shift, M);
}

}  // namespace hr
