// Pixel passes of HistRetinex on sm_103a:
//   hist  -- V = max(r,g,b) (Sec. II preamble), its K-bin count histogram H_C(S) (Eq. 3) and the
//            histogram of its 3x3 Sobel gradient magnitude H_C(grad S) (Algorithm 1 initialisation);
//   apply -- V' = LUT[V] and every channel scaled by V'/V, rounded half up, so hue and saturation
//            are kept (Sec. II preamble; Sec. III.C last paragraph: histogram matching).
// Both kernels walk a flat list of kTileW x kTileH tiles spanning every image of the launch, so
// one launch serves a single image or a batch of mixed sizes.
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
__global__ void __launch_bounds__(kThreads) hist_kernel(const ImageDesc* __restrict__ imgs, int n,
                                                        const int* __restrict__ tile_start, int total, int K,
                                                        uint8_t* slots, size_t slot_bytes, SlotLayout lay,
                                                        unsigned* status) {
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
    const ImageDesc im = imgs[img];
    const int lt = t - __ldg(tile_start + img);
    const int tiles_x = (im.W + kTileW - 1) / kTileW;
    const int x0 = (lt % tiles_x) * kTileW, y0 = (lt / tiles_x) * kTileH;
    // V tile with a one-pixel halo; coordinates outside the image replicate the border
    for (int e = tid; e < kVH * kVW; e += kThreads) {
      const int r = e / kVW, c = e - r * kVW;
      const int y = clampi(y0 - 1 + r, 0, im.H - 1), x = clampi(x0 - 1 + c, 0, im.W - 1);
      unsigned v = load_value<ET>(im, x, y);
      if (v >= (unsigned)K) { range_bad = true; v = K - 1; }
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
      const int gx = (a02 + 2 * a12 + a22) - (a00 + 2 * a10 + a20);
      const int gy = (a20 + 2 * a21 + a22) - (a00 + 2 * a01 + a02);
      unsigned g = round_sqrt((unsigned)(gx * gx + gy * gy));
      g = g < (unsigned)(K - 1) ? g : (unsigned)(K - 1);
      atomicAdd(my_hs + a11, 1u);
      atomicAdd(my_hg + g, 1u);
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
__global__ void __launch_bounds__(kThreads) apply_kernel(const ImageDesc* __restrict__ imgs, int n,
                                                         const int* __restrict__ tile_start, int total, int K,
                                                         const uint8_t* slots, size_t slot_bytes, SlotLayout lay,
                                                         unsigned* status) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned short* lut = reinterpret_cast<unsigned short*>(smem);
  float* rup = reinterpret_cast<float*>(smem + ((K * 2 + 15) & ~15));  // V'/V rounded up (8-bit data)
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
      for (int k = tid; k < K; k += kThreads) {
        const unsigned short vp = gl[k];
        lut[k] = vp;
        if (sizeof(ET) == 1) rup[k] = k > 0 ? __fdiv_ru((float)vp, (float)k) : 0.0f;
      }
      __syncthreads();
      cur = img;
    }
    const ImageDesc im = imgs[img];
    const int lt = t - __ldg(tile_start + img);
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
      if (V >= (unsigned)K) { range_bad = true; V = K - 1; }
      const unsigned vp = lut[V];
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
// 8-bit fast paths (rows 16-byte aligned).  The histogram pass stages each tile's rows into
// shared memory with asynchronous 16-byte copies (double buffered: the next tile's copies run
// while the current tile is processed), builds V four pixels per thread with byte permutes and
// evaluates the separable Sobel operator on eight pixels per thread.  The apply pass moves 16
// pixels (48 bytes, three 16-byte vectors) per thread each way.
// ------------------------------------------------------------------------------------------------
constexpr int kRawRow = 416;              // staged bytes per tile row: [3 x0 - 16, 3 x0 + 400)
constexpr int kRawChunks = kRawRow / 16;
constexpr int kVTS = 136;                 // V tile row stride; column c holds x = x0 - 4 + c
constexpr int kVGroups = kVTS / 4;        // 4-pixel groups per V tile row

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gsrc), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

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
    cp_async16(raw + r * kRawRow + ch * 16, nb > 0 ? (const void*)(row + b0) : (const void*)row, nb);
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

__global__ void __launch_bounds__(kThreads) hist_u8v_kernel(const ImageDesc* __restrict__ imgs, int n,
                                                            const int* __restrict__ tile_start, int total, int K,
                                                            uint8_t* slots, size_t slot_bytes, SlotLayout lay,
                                                            unsigned* status) {
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
    const ImageDesc& im = imgs[img];
    const int lt = t - __ldg(tile_start + img);
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
    stage_tile(imgs[img], x0, y0, raw);
  }
  for (int t = t0; t < t1; ++t) {
    int img, x0, y0;
    tile_xy(t, img, x0, y0);
    unsigned char* rb = raw + ((t - t0) & 1) * (kVH * kRawRow);
    if (t + 1 < t1) {
      int img2, x2, y2;
      tile_xy(t + 1, img2, x2, y2);
      stage_tile(imgs[img2], x2, y2, raw + ((t + 1 - t0) & 1) * (kVH * kRawRow));
    } else {
      cp_async_commit();
    }
    cp_async_wait1();
    __syncthreads();
    if (img != cur) {
      if (cur >= 0) flush(cur);
      cur = img;
    }
    const ImageDesc im = imgs[img];
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

__global__ void __launch_bounds__(kThreads) apply_u8v_kernel(const ImageDesc* __restrict__ imgs, int n,
                                                             const int* __restrict__ tile_start, int total, int K,
                                                             const uint8_t* slots, size_t slot_bytes, SlotLayout lay,
                                                             unsigned* status) {
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
    const ImageDesc im = imgs[img];
    const int lt = t - __ldg(tile_start + img);
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

}  // namespace

cudaError_t launch_hist(const ImageDesc* d_imgs, int n, const int* d_tile_start, int total_tiles, int elem_bytes,
                        int K, uint8_t* slots, size_t slot_bytes, SlotLayout lay, unsigned* status, int grid,
                        cudaStream_t st, bool fast) {
  const int copies = K <= 256 ? kWarps : 1;
  const size_t smem = (size_t)2 * copies * K * sizeof(unsigned) + (size_t)kVH * kVW * sizeof(unsigned short);
  if (grid > total_tiles) grid = total_tiles;
  if (grid < 1) grid = 1;
  if (elem_bytes == 1 && fast) {
    const size_t smem_v = (size_t)2 * kWarps * K * sizeof(unsigned) + (size_t)kVH * kVTS + (size_t)2 * kVH * kRawRow;
    cudaFuncSetAttribute(hist_u8v_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_v);
    hist_u8v_kernel<<<grid, kThreads, smem_v, st>>>(d_imgs, n, d_tile_start, total_tiles, K, slots, slot_bytes, lay,
                                                    status);
  } else if (elem_bytes == 1) {
    cudaFuncSetAttribute(hist_kernel<uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    hist_kernel<uint8_t><<<grid, kThreads, smem, st>>>(d_imgs, n, d_tile_start, total_tiles, K, slots, slot_bytes,
                                                       lay, status);
  } else {
    cudaFuncSetAttribute(hist_kernel<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    hist_kernel<uint16_t><<<grid, kThreads, smem, st>>>(d_imgs, n, d_tile_start, total_tiles, K, slots, slot_bytes,
                                                        lay, status);
  }
  return cudaGetLastError();
}

cudaError_t launch_apply(const ImageDesc* d_imgs, int n, const int* d_tile_start, int total_tiles, int elem_bytes,
                         int K, uint8_t* slots, size_t slot_bytes, SlotLayout lay, unsigned* status, int grid,
                         cudaStream_t st, bool fast) {
  const size_t smem = (size_t)((K * 2 + 15) & ~15) + (size_t)K * sizeof(float);
  if (grid > total_tiles) grid = total_tiles;
  if (grid < 1) grid = 1;
  if (elem_bytes == 1 && fast)
    apply_u8v_kernel<<<grid, kThreads, 0, st>>>(d_imgs, n, d_tile_start, total_tiles, K, slots, slot_bytes, lay,
                                                status);
  else if (elem_bytes == 1)
    apply_kernel<uint8_t><<<grid, kThreads, smem, st>>>(d_imgs, n, d_tile_start, total_tiles, K, slots, slot_bytes,
                                                        lay, status);
  else
    apply_kernel<uint16_t><<<grid, kThreads, smem, st>>>(d_imgs, n, d_tile_start, total_tiles, K, slots,
                                                         slot_bytes, lay, status);
  return cudaGetLastError();
}

}  // namespace hr
