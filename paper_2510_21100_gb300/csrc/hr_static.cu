// Context-free, allocation-free single-image entry point (histretinex_enhance_noalloc).
//
// Some callers cannot allocate device memory: code running while a framework captures a CUDA
// graph, real-time loops that must not block in the allocator, and plug-ins whose host process
// owns every device allocation.  For them this entry point runs the same single-image pipeline
// as histretinex_enhance (histogram pass, cluster solve, apply) for K <= 256 with its whole
// workspace in one file-scope __device__ array, so it calls no cudaMalloc, cudaFree or any
// other allocating routine.  The array is kStaticBytes (1 MiB) and stays resident on every
// device that loads the library until the process exits.
//
// Every call is self-contained on its stream: it looks up the array's device address, clears the
// histograms and the status word, and rebuilds the Eq. 19 boundary table for its own (K, gamma)
// with a small kernel whose inputs travel in the kernel parameters.  Nothing a call reads is left
// over from an earlier call.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/histretinex.h"
#include "hr_internal.cuh"

namespace {

constexpr int kStaticMaxK = 256;
constexpr size_t kStaticBytes = size_t(1) << 20;

// Workspace of every call, on every device: one image slot, the Eq. 19 boundary table and the
// status word.  Shared by all calls; it keeps the previous call's contents, so each call clears
// or rewrites what it reads.
__device__ __align__(256) unsigned char g_scratch[kStaticBytes];

// The gamma-processed illumination locations of Eq. 17, (j / (K - 1))^(1 / gamma) for j < K,
// computed on the host (the same libm pow as the context path's table) and passed by value.
struct IllumLocations {
  double v[kStaticMaxK];
};

// index_1(i, j) of Eq. 19 in the same IEEE operations as the host table of the context path: the
// level nearest to the location-matrix entry hl * i / (K - 1), the first one on a tie.
__device__ __forceinline__ int index1_dev(int K, double hl, double hr) {
  const double km1 = (double)(K - 1);
  const double p = __dmul_rn(hl, hr);
  const long long c = llround(__dmul_rn(p, km1));
  const long long lo = c - 1 < 0 ? 0 : c - 1, hi = c + 1 > K - 1 ? K - 1 : c + 1;
  long long best = lo;
  double bd = fabs(__dsub_rn(p, __ddiv_rn((double)lo, km1)));
  for (long long k = lo + 1; k <= hi; ++k) {
    const double d = fabs(__dsub_rn(p, __ddiv_rn((double)k, km1)));
    if (d < bd) { bd = d; best = k; }
  }
  return (int)best;
}

// Boundary table t[i][k] = first illumination bin j with index_1(i, j) >= k (K where none), row i
// by block i: index_1 grows with j, so thread j writes the levels (index_1(i, j-1), index_1(i, j)].
__global__ void jstart1_kernel(int K, IllumLocations hl, uint16_t* t) {
  const int i = blockIdx.x;
  const double hr = __ddiv_rn((double)i, (double)(K - 1));
  uint16_t* row = t + (size_t)i * (K + 1);
  for (int j = threadIdx.x; j < K; j += blockDim.x) {
    const int c = index1_dev(K, hl.v[j], hr);
    const int cprev = j == 0 ? -1 : index1_dev(K, hl.v[j - 1], hr);
    for (int k = cprev + 1; k <= c; ++k) row[k] = (uint16_t)j;
    if (j == K - 1)
      for (int k = c + 1; k <= K; ++k) row[k] = (uint16_t)K;
  }
}

// Host cache of the locations for the last (K, gamma): host memory only, copied into the kernel
// parameters of every call.
std::mutex g_mutex;
int g_hl_K = 0;
double g_hl_gamma = 0.0;
IllumLocations g_hl;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" hr_status histretinex_enhance_noalloc(const hr_params* p, const void* d_in, void* d_out, int width,
                                                 int height, size_t in_pitch, size_t out_pitch, int elem_bytes,
                                                 void* stream) {
  hr_status s = hr::check_params(p);
  if (s != HR_OK) return s;
  if (p->K > kStaticMaxK) return HR_ERR_UNSUPPORTED;  // the static workspace is sized for K <= 256
  if (p->levels != 0 && p->levels != p->K) return HR_ERR_UNSUPPORTED;  // no binned data here
  if (!d_in || !d_out || width < 1 || height < 1 || (elem_bytes != 1 && elem_bytes != 2)) return HR_ERR_INVALID_ARG;
  const size_t row = (size_t)3 * width * elem_bytes;
  if (in_pitch < row || out_pitch < row) return HR_ERR_INVALID_ARG;
  if ((long long)width * height >= (1LL << 31)) return HR_ERR_UNSUPPORTED;
  const int K = p->K;
  const hr::SlotLayout lay = hr::make_layout(K);
  const size_t off_table = align256(lay.bytes);
  const size_t off_status = align256(off_table + sizeof(uint16_t) * (size_t)K * (K + 1));
  if (off_status + 256 > kStaticBytes) return HR_ERR_UNSUPPORTED;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HR_ERR_CUDA;
  // The device address of the workspace on the current device, looked up on every call (no
  // allocation), so that a reset of the device's context cannot leave a stale address behind.
  void* addr = nullptr;
  if (cudaGetSymbolAddress(&addr, g_scratch) != cudaSuccess || addr == nullptr) {
    cudaGetLastError();
    return HR_ERR_CUDA;
  }
  unsigned char* base = static_cast<unsigned char*>(addr);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  IllumLocations hl;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (g_hl_K != K || g_hl_gamma != p->gamma) {
      const double km1 = (double)(K - 1), ig = 1.0 / p->gamma;
      for (int j = 0; j < K; ++j) g_hl.v[j] = std::pow((double)j / km1, ig);
      g_hl_K = K;
      g_hl_gamma = p->gamma;
    }
    hl = g_hl;
  }
  hr::ImgTab tab{};  // the image travels in the kernel parameters
  tab.n = 1;
  tab.one = hr::ImageDesc{static_cast<const uint8_t*>(d_in), static_cast<uint8_t*>(d_out), width, height,
                          (long long)in_pitch, (long long)out_pitch};
  const int tiles = hr::tiles_of(width, height), units = hr::strips_of(width, height);
  // what must start at zero: the two histograms and the status word; then this call's Eq. 19 table
  cudaError_t e = cudaMemsetAsync(base + lay.S, 0, (size_t)2 * K * sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + off_status, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return HR_ERR_CUDA;
  auto* table = reinterpret_cast<uint16_t*>(base + off_table);
  if (hr::launch_kernel(jstart1_kernel, dim3(K), dim3(256), 0, st, false, K, hl, table) != cudaSuccess)
    return HR_ERR_CUDA;

  const bool fast_in = elem_bytes == 1 && ((uintptr_t)d_in % 16 == 0) && (in_pitch % 16 == 0);
  const bool fast_out = fast_in && ((uintptr_t)d_out % 16 == 0) && (out_pitch % 16 == 0);
  auto* d_status = reinterpret_cast<unsigned*>(base + off_status);
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return HR_ERR_CUDA;
  e = hr::launch_hist(tab, tiles, units, hr::interior_strips_of(width, height), elem_bytes, K, base, lay.bytes, lay,
                      d_status, sms, 8, st, fast_in, true, (p->flags & HR_FLAG_FORWARD_GRADIENT) != 0);
  if (e != cudaSuccess) return HR_ERR_CUDA;
  hr::SolveArgs a{};
  a.K = K;
  a.alpha = p->alpha;
  a.beta = p->beta;
  a.eps = p->eps;
  a.max_iter = p->max_iter;
  a.fixed_iters = (p->flags & HR_FLAG_FIXED_ITERS) ? 1 : 0;
  a.jstart1 = table;
  a.slots = base;
  a.slot_bytes = lay.bytes;
  a.lay = lay;
  a.status = d_status;
  a.profile = 0;
  a.printed = (p->flags & HR_FLAG_PRINTED_UPDATE) ? 1 : 0;
  a.nearest = (p->flags & HR_FLAG_NEAREST_MATCH) ? 1 : 0;
  a.arith = p->precision == HR_PREC_FP32 ? hr::kArithF32 : (p->precision == HR_PREC_DF64 ? hr::kArithDF64 : hr::kArithF64);
  e = hr::launch_solve(a, 1, 16, st, false);
  if (e != cudaSuccess) return HR_ERR_CUDA;
  e = hr::launch_apply(tab, tiles, elem_bytes, K, base, lay.bytes, lay, d_status, sms, 16, st, fast_out, true);
  return e == cudaSuccess ? HR_OK : HR_ERR_CUDA;
}
