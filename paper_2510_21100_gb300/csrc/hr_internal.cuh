// Internal declarations of the HistRetinex CUDA library (sm_103a).
#pragma once
#include <cstddef>
#include <cstdint>
#include <functional>
#include <cuda_runtime.h>

#include "../../include/histretinex.h"

namespace hr {

// Device status bits, OR-ed into the context's status word by the kernels.
enum : unsigned { kStRange = 1u, kStTimeout = 2u, kStUnsupported = 4u };

// Length of one accumulation piece of the solver (cells summed by one lane before the
// per-target combine).  Short pieces keep the FP64 dependency chains short.
constexpr int kPiece = 8;

// Phase timestamps (ns) the solve kernel records when asked (a measurement hook).
constexpr int kProfSlots = 48;

// Shared-memory capacities of the solver's own cell list, pieces and piece sums; a CTA whose
// share is larger keeps them in its global workspace instead.
constexpr int kListCap = 20480;
constexpr int kPieceCap = 3072;

// One image of a launch: device pointers and geometry.
struct ImageDesc {
  const uint8_t* in;
  uint8_t* out;
  int W, H;
  long long in_pitch, out_pitch;
};

// The images of a launch.  One image travels inline in the kernel parameters, so a single-image
// call uploads nothing before its kernels; several are read from device tables.
struct ImgTab {
  const ImageDesc* imgs;   // n descriptors (n > 1)
  const int* tiles;        // n + 1 tile starts (n > 1)
  const int* units;        // n + 1 strip starts (n > 1)
  int n;
  ImageDesc one;           // the image (n == 1)
#ifdef __CUDACC__
  __device__ __forceinline__ ImageDesc desc(int i) const { return n == 1 ? one : imgs[i]; }
  __device__ __forceinline__ int tile0(int i) const { return n == 1 ? 0 : __ldg(tiles + i); }
  __device__ __forceinline__ int unit0(int i) const { return n == 1 ? 0 : __ldg(units + i); }
#endif
};

#ifdef __CUDACC__
// Programmatic dependent launch, device side: wait until the previous kernel on the stream has
// finished and its writes are visible (returns at once for a plain launch), and let the next
// kernel be scheduled (it waits in turn for this one to finish).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Kernel launch with the programmatic-stream-serialisation attribute when pdl is set.
template <typename... KArgs, typename... Args>
cudaError_t launch_kernel(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool pdl,
                          Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<Args&&>(args)...);
}
#endif

// Byte offsets of the per-image workspace ("slot").  Every slot has the same layout for a
// given K; slots are `slot_bytes` apart.
struct SlotLayout {
  size_t S, G;          // uint32[K] each: H_C(S), H_C(grad S)
  size_t R, L, T;       // double[K] each: results of Algorithm 1 and Eq. 20 (level-indexed)
  size_t lut;           // uint16[K]
  size_t misc;          // int[4]: iterations, nR, nL, cells; then long long[kProfSlots] phase times
  size_t vec;           // solver vectors when they do not fit in shared memory
  size_t cls;           // uint32[4*K]: spare
  size_t list;          // uint32[K*(K+1)]: class-major cell lists, (a << 16) | b; then the
                        // Eq. 19 row segments (at most K (K+1) / 2 solver values)
  size_t piece;         // uint2[max_pieces]: (cell start, len | class << 16)
  size_t part;          // double[max_parts]: piece partial sums
  size_t bytes;         // total slot size (multiple of 256)
  size_t max_pieces, max_parts;
};

SlotLayout make_layout(int K);

// Parameter validation of hr_params (HR_OK or HR_ERR_INVALID_ARG).
hr_status check_params(const hr_params* p);
// Eq. 19 class boundaries: t[i * (K + 1) + k] = first illumination bin j with index_1(i, j) >= k.
// M: the data's levels (K bins of M / K levels each, bins located at their centre values).
void build_jstart1(int K, double gamma, uint16_t* t, int M = 0);
// Binned data: the class map of Eq. 10 over the bin locations, cmap[i * K + j], and its boundaries
// js0[i * (K + 1) + k] = first j with cmap[i][j] >= k.
void build_class_tables(int K, int M, uint16_t* cmap, uint16_t* js0);

// Number of solver vectors (double[K]) and their shared-memory footprint.
constexpr int kSolveVecs = 8;       // Rc, Lc, L2c, RRc, Ru, Lu, q, spare
constexpr int kSolveThreads = 512;

// Arithmetic of the solve's sums.
enum : int { kArithF64 = 0, kArithF32 = 1, kArithDF64 = 2 };

struct SolveArgs {
  int K;
  double alpha, beta, eps;
  int max_iter;
  int fixed_iters;
  const uint16_t* jstart1;   // [K][K+1]: first illumination bin j with index_1(i, j) >= k
  uint8_t* slots;            // base of slot 0
  const int* order;          // CTA group g solves image order[g] (nullptr: image g)
  size_t slot_bytes;
  SlotLayout lay;
  unsigned* status;
  int vec_in_smem;           // 1: solver vectors in dynamic shared memory (set by launch_solve)
  int list_in_smem;          // 1: own cell lists may use shared memory (set by launch_solve)
  int profile;               // 1: record phase timestamps into the slot's misc area
  int arith;                 // kArithF64 (plain form), kArithF32 (reduced precision), kArithDF64
  int zero_hist;             // 1: clear H_C(S) and H_C(grad S) after use, ready for the next call
  int printed;               // 1: Eq. 12 / Eq. 13 as printed (the weight K_ij divides)
  int nearest;               // 1: matching to the nearest cumulative share
  const uint16_t* cmap;      // binned data: class map of Eq. 10 [K][K] (nullptr: the closed form)
  const uint16_t* jstart0;   // binned data: its boundaries [K][K+1], first j with class >= k
};

// Launchers (return cudaError_t of the launch).  pdl: programmatic dependent launch (the kernel
// may be scheduled before the previous kernel on the stream has finished; it waits for it on the
// device before touching any data).
// The histogram pass walks the tile list or, for enough 8-bit images with aligned rows, the
// strip list (kStripW x kBandH units); both lists are given, with their totals and the number of
// interior strips (strips that cross no right or bottom image edge).  Tile kernels
// run sms x ctas_per_sm CTAs, the strip kernel one CTA per SM.
// forward: the gradient image by forward differences (generic kernel) instead of the Sobel operator.
// M > K: binned data (value v in bin v >> log2(M / K); generic kernel).
cudaError_t launch_hist(const ImgTab& tab, int total_tiles, int total_units, int interior_units, int elem_bytes,
                        int K, uint8_t* slots,
                        size_t slot_bytes, SlotLayout lay, unsigned* status, int sms, int ctas_per_sm,
                        cudaStream_t st, bool fast, bool pdl, bool forward = false, int M = 0);
cudaError_t launch_solve(const SolveArgs& a, int n, int cluster, cudaStream_t st, bool pdl);
cudaError_t launch_apply(const ImgTab& tab, int total_tiles, int elem_bytes, int K, uint8_t* slots, size_t slot_bytes,
                         SlotLayout lay, unsigned* status, int sms, int ctas_per_sm, cudaStream_t st, bool fast,
                         bool pdl, int M = 0);
// Gradient levels of squared magnitudes [m2_first, m2_first + n) by one of the histogram kernels'
// three device forms (0: strip kernel, 1: staged-tile kernel, 2: generic kernel), into out[n].
cudaError_t launch_grad_level_probe(int form, int K, int m2_first, int n, uint16_t* out, cudaStream_t st);
size_t solve_smem_bytes(int K, int vec_in_smem, int list_in_smem, size_t fsize);

// SM partitions for overlapping single-image calls (green contexts): `parts` partitions of 16 SMs
// for solves, each with `sper` solve streams, and one of the remaining SMs for the pixel passes;
// `ring` pixel streams, one per workspace slot.  partitions_run forks one call from the caller's
// stream st: hist on the slot's pixel stream, solve on the next solve stream (partitions in turn),
// apply back on the pixel stream, then st waits for it.  Each StageFn enqueues its stage on the stream it is given (the partition's context is
// current while it runs).
using StageFn = std::function<cudaError_t(cudaStream_t)>;
struct Partitions;
hr_status partitions_create(int device, int parts, int sper, int ring, Partitions** out);
void partitions_destroy(Partitions* P);
int partitions_pixel_sms(const Partitions* P);
cudaError_t partitions_run(Partitions* P, int slot, cudaStream_t st, const StageFn& hist, const StageFn& solve,
                           const StageFn& apply);

// Measured ablation: the Eq. 11 class totals of n images (R, L: n x K FP32, level-indexed) into
// P (n x K FP32) by the FP32 gather on the CUDA cores (method 0) or the BF16 one-hot GEMM on the
// tensor cores (method 1); *kernel_ms gets the kernels' device time.
hr_status ablation_class_totals(int K, int n, const float* d_R, const float* d_L, float* d_P, int method,
                                unsigned* d_status, int sms, cudaStream_t st, float* kernel_ms);

// Geometry of the pixel passes: tiles of kTileW x kTileH pixels.
constexpr int kTileW = 128;
constexpr int kTileH = 32;
inline int tiles_of(int W, int H) { return ((W + kTileW - 1) / kTileW) * ((H + kTileH - 1) / kTileH); }
// Units of the 8-bit strip histogram pass: strips kStripW pixels wide and kBandH rows high, counted
// column by column within an image; the kernel deals their rows out to its warps in equal runs.
constexpr int kStripW = 512;
constexpr int kBandH = 4;
inline int strips_of(int W, int H) { return ((W + kStripW - 1) / kStripW) * ((H + kBandH - 1) / kBandH); }
inline int interior_strips_of(int W, int H) { return (W / kStripW) * (H / kBandH); }

}  // namespace hr
