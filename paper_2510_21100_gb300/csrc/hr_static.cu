// Context-free, allocation-free single-image entry point (histretinex_enhance_noalloc).
//
// Some callers cannot allocate device memory: code running while a framework captures a CUDA
// graph, real-time loops that must not block in the allocator, and plug-ins whose host process
// owns every device allocation.  For them this entry point runs the same single-image pipeline
// as histretinex_enhance (histogram pass, cluster solve, apply) for K <= 256 with its whole
// workspace in one file-scope __device__ array, so it calls no cudaMalloc, cudaFree or any
// other allocating routine.  The array is kStaticBytes (1 MiB) and stays resident on every
// device that loads the library until the process exits.
#include <cstring>
#include <mutex>

#include "../../include/histretinex.h"
#include "hr_internal.cuh"

namespace {

constexpr int kStaticMaxK = 256;
constexpr size_t kStaticBytes = size_t(1) << 20;
constexpr int kMaxDevices = 64;

// Workspace of every call, on every device: one image slot, the Eq. 19 boundary table and the
// status word.  Shared by all calls; it keeps the
// previous call's contents, so each call clears what must start at zero.
__device__ __align__(256) unsigned char g_scratch[kStaticBytes];

struct DeviceState {
  bool ready = false;
  unsigned char* base = nullptr;  // device address of g_scratch on this device
  int table_K = 0;                // (K, gamma) of the Eq. 19 table currently in the workspace
  double table_gamma = 0.0;
};
DeviceState g_state[kMaxDevices];
std::mutex g_mutex;

// Host staging for the uploads (static, so nothing is allocated per call).
uint16_t g_table_host[kStaticMaxK * (kStaticMaxK + 1)];

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" hr_status histretinex_enhance_noalloc(const hr_params* p, const void* d_in, void* d_out, int width,
                                                 int height, size_t in_pitch, size_t out_pitch, int elem_bytes,
                                                 void* stream) {
  hr_status s = hr::check_params(p);
  if (s != HR_OK) return s;
  if (p->K > kStaticMaxK) return HR_ERR_UNSUPPORTED;  // the static workspace is sized for K <= 256
  if (p->precision != HR_PREC_FP64 && p->precision != HR_PREC_FP32 && p->precision != HR_PREC_DF64)
    return HR_ERR_INVALID_ARG;
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
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HR_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceState& ds = g_state[dev];
  if (!ds.ready) {
    // once per device, with that device current: the device address of the workspace
    void* addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_scratch) != cudaSuccess || addr == nullptr) {
      cudaGetLastError();
      return HR_ERR_CUDA;
    }
    ds.base = static_cast<unsigned char*>(addr);
    ds.ready = true;
  }
  unsigned char* base = ds.base;
  if (ds.table_K != K || ds.table_gamma != p->gamma) {
    hr::build_jstart1(K, p->gamma, g_table_host);
    if (cudaMemcpyAsync(base + off_table, g_table_host, sizeof(uint16_t) * (size_t)K * (K + 1),
                        cudaMemcpyHostToDevice, st) != cudaSuccess)
      return HR_ERR_CUDA;
    ds.table_K = K;
    ds.table_gamma = p->gamma;
  }
  hr::ImgTab tab{};  // the image travels in the kernel parameters
  tab.n = 1;
  tab.one = hr::ImageDesc{static_cast<const uint8_t*>(d_in), static_cast<uint8_t*>(d_out), width, height,
                          (long long)in_pitch, (long long)out_pitch};
  const int tiles = hr::tiles_of(width, height), units = hr::strips_of(width, height);
  // what must start at zero: the two histograms and the status word
  cudaError_t e = cudaMemsetAsync(base + lay.S, 0, (size_t)2 * K * sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + off_status, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return HR_ERR_CUDA;

  const bool fast_in = elem_bytes == 1 && ((uintptr_t)d_in % 16 == 0) && (in_pitch % 16 == 0);
  const bool fast_out = fast_in && ((uintptr_t)d_out % 16 == 0) && (out_pitch % 16 == 0);
  auto* d_status = reinterpret_cast<unsigned*>(base + off_status);
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return HR_ERR_CUDA;
  e = hr::launch_hist(tab, tiles, units, hr::interior_strips_of(width, height), elem_bytes, K, base, lay.bytes, lay, d_status, sms, 8, st, fast_in, true);
  if (e != cudaSuccess) return HR_ERR_CUDA;
  hr::SolveArgs a{};
  a.K = K;
  a.alpha = p->alpha;
  a.beta = p->beta;
  a.eps = p->eps;
  a.max_iter = p->max_iter;
  a.fixed_iters = (p->flags & HR_FLAG_FIXED_ITERS) ? 1 : 0;
  a.jstart1 = reinterpret_cast<const uint16_t*>(base + off_table);
  a.slots = base;
  a.slot_bytes = lay.bytes;
  a.lay = lay;
  a.status = d_status;
  a.profile = 0;
  a.arith = p->precision == HR_PREC_FP32 ? hr::kArithF32 : (p->precision == HR_PREC_DF64 ? hr::kArithDF64 : hr::kArithF64);
  e = hr::launch_solve(a, 1, 16, st, false);
  if (e != cudaSuccess) return HR_ERR_CUDA;
  e = hr::launch_apply(tab, tiles, elem_bytes, K, base, lay.bytes, lay, d_status, sms, 16, st, fast_out, true);
  return e == cudaSuccess ? HR_OK : HR_ERR_CUDA;
}
