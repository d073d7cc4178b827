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

}  // namespace

cudaError_t launch_hist(const ImageDesc* d_imgs, int n, const int* d_tile_start, int total_tiles, int elem_bytes,
                        int K, uint8_t* slots, size_t slot_bytes, SlotLayout lay, unsigned* status, int grid,
                        cudaStream_t st) {
  const int copies = K <= 256 ? kWarps : 1;
  const size_t smem = (size_t)2 * copies * K * sizeof(unsigned) + (size_t)kVH * kVW * sizeof(unsigned short);
  if (grid > total_tiles) grid = total_tiles;
  if (grid < 1) grid = 1;
  if (elem_bytes == 1) {
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
                         cudaStream_t st) {
  const size_t smem = (size_t)((K * 2 + 15) & ~15) + (size_t)K * sizeof(float);
  if (grid > total_tiles) grid = total_tiles;
  if (grid < 1) grid = 1;
  if (elem_bytes == 1)
    apply_kernel<uint8_t><<<grid, kThreads, smem, st>>>(d_imgs, n, d_tile_start, total_tiles, K, slots, slot_bytes,
                                                        lay, status);
  else
    apply_kernel<uint16_t><<<grid, kThreads, smem, st>>>(d_imgs, n, d_tile_start, total_tiles, K, slots,
                                                         slot_bytes, lay, status);
  return cudaGetLastError();
}

}  // namespace hr
