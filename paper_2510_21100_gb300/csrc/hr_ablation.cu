// Measured ablation of the reduced-precision form (not part of the paper's method): the Eq. 11
// class totals of a batch of images as a dense contraction on the tcgen05 tensor cores.
//
// For a batch, P[k][n] = sum over the cells c = (i, j) of class k of R_n[i] L_n[j] (Eq. 6, Eq. 11).
// With the K^2 cells sorted by class (the class map index(i, j) = round(i j / (K - 1)) does not
// depend on the image), this is a GEMM of the one-hot class matrix Z (K x K^2, Z[k][c] = 1 where
// cell c has class k) with the cell products X (K^2 x n, X[c][n] = R_n[i] L_n[j]):  P = Z X.  A tile
// of 128 classes only meets the cells of those classes, a contiguous range of the sorted cells,
// so each tile runs over its own range (split over CTAs, partial tiles summed afterwards).  Z is
// exact in BF16; X is rounded to BF16; the tensor cores accumulate in FP32 in tensor memory.  Every
// cell is multiplied by 128 rows of Z, of which one is non-zero: the contraction does 128 times the
// useful multiply-adds, which the tensor cores' rate is set against.  The FP32 gather beside it
// sums the same products on the CUDA cores, class by class.  The split form (method 2) writes each
// product as the sum of two BF16 numbers, hi + lo, and runs the contraction over both, which keeps
// about 16 significant bits of every product.
//
// The tensor-core kernel: one CTA per (class tile, image tile, split), 256 threads.  Each 64-cell
// chunk is staged in shared memory in the no-swizzle K-major layout of 8-row x 16-byte core
// matrices (A: the one-hot rows, generated from the cells' classes; B: the images' BF16 products,
// copied from global memory), in two stages; one thread issues four tcgen05.mma of K = 16 per
// chunk into a 128 x 128 FP32 accumulator in tensor memory and commits them to the stage's
// mbarrier, which the next fill of that stage waits on.  Waits are bounded: a wait that gives up
// sets the status word, waits once more (bounded) for the MMAs in flight and frees the tensor
// memory before the kernel returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "hr_internal.cuh"

namespace hr {
namespace {

constexpr int kAbM = 128;       // classes per tile (MMA M)
constexpr int kAbN = 128;       // images per tile (MMA N)
constexpr int kAbChunk = 64;    // cells per staged chunk: four MMAs of K = 16
constexpr int kAbThreads = 256;
constexpr int kAbTileBytes = kAbM * kAbChunk * 2;   // 16 KB per operand and stage
constexpr long long kWaitLimit = 1LL << 24;           // try_wait rounds before a wait gives up

struct AbTile {
  int mt, nt;   // class tile (classes [128 mt, 128 mt + 128)), image tile (images [128 nt, ...))
  int c0, c1;   // chunk range [c0, c1) of the sorted cells
};

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Matrix descriptor of a K-major operand without swizzle: 8-row x 16-byte core matrices, lbo bytes
// apart along K, sbo bytes apart along M (or N); descriptor version 1 (bits 46-47), no base offset.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5), BF16 A and B (bits 7-9, 10-12),
// both K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kAbN >> 3) << 17) |
                            ((uint32_t)(kAbM >> 4) << 24);

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < kWaitLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__global__ void __launch_bounds__(kAbThreads, 1)
onehot_gemm_kernel(const uint16_t* __restrict__ cls_of, const uint16_t* __restrict__ Bt, const AbTile* __restrict__ tiles,
                   int ncells_pad, int passes, size_t pass_stride, float* __restrict__ part, unsigned* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ uint16_t scls[2][kAbChunk];
  __shared__ int bad;
  const AbTile t = tiles[blockIdx.x];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* sA[2] = {sm, sm + 2 * kAbTileBytes};
  unsigned char* sB[2] = {sm + kAbTileBytes, sm + 3 * kAbTileBytes};
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                 "r"(kAbN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&mbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&mbar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    bad = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const int k0 = t.mt * kAbM;
  uint32_t parity[2] = {0u, 0u};
  int last = -1;  // stage of the last commit
  const int nchunk = t.c1 - t.c0;
  for (int u = 0; u < passes * nchunk; ++u) {  // pass 1 (split form): the low parts of the products
    const int c = t.c0 + u % nchunk;
    const uint16_t* Bp = Bt + (size_t)(u / nchunk) * pass_stride;
    const int s = u & 1;
    if (u >= 2) {  // the MMAs that read this stage two chunks ago are done
      if (!mbar_wait(saddr(&mbar[s]), parity[s])) atomicExch(&bad, 1);
      parity[s] ^= 1u;
    }
    __syncthreads();
    if (bad) break;
    const int cell0 = c * kAbChunk;
    if (tid < kAbChunk) scls[s][tid] = cls_of[cell0 + tid];
    __syncthreads();
    // 128 rows x 8 groups of 8 cells; group (r, g) is row r % 8 of core matrix (r / 8, g)
    for (int p = tid; p < kAbM * (kAbChunk / 8); p += kAbThreads) {
      const int r = p >> 3, g = p & 7;
      const uint32_t off = (uint32_t)(((r >> 3) * (kAbChunk / 8) + g) * 128 + (r & 7) * 16);
      uint32_t w[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t lo = scls[s][g * 8 + 2 * q] == (uint16_t)(k0 + r) ? 0x3F80u : 0u;  // BF16 1.0
        const uint32_t hi = scls[s][g * 8 + 2 * q + 1] == (uint16_t)(k0 + r) ? 0x3F80u : 0u;
        w[q] = lo | (hi << 16);
      }
      *reinterpret_cast<uint4*>(sA[s] + off) = make_uint4(w[0], w[1], w[2], w[3]);
      *reinterpret_cast<uint4*>(sB[s] + off) =
          *reinterpret_cast<const uint4*>(Bp + (size_t)(t.nt * kAbN + r) * ncells_pad + cell0 + g * 8);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the stores, visible to the tensor cores
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int kk = 0; kk < kAbChunk / 16; ++kk) {
        // K = 16 BF16 elements = two core matrices along K (256 bytes) per MMA
        const uint64_t da = smem_desc(saddr(sA[s]) + kk * 256, 128, (kAbChunk / 8) * 128);
        const uint64_t db = smem_desc(saddr(sB[s]) + kk * 256, 128, (kAbChunk / 8) * 128);
        const uint32_t acc = (u > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da), "l"(db), "r"(kIdesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(&mbar[s]))
                   : "memory");
    }
    last = s;
  }
  // the last commit covers every MMA this CTA issued
  if (last >= 0) {
    if (!mbar_wait(saddr(&mbar[last]), parity[last])) {
      atomicExch(&bad, 1);
      mbar_wait(saddr(&mbar[last]), parity[last]);  // once more (bounded) for the MMAs in flight
    }
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!bad && last >= 0 && warp < 4) {
    // accumulator row m = class k0 + m in tensor-memory lane m; column n = image 128 nt + n
    float* dst = part + (size_t)blockIdx.x * kAbM * kAbN;
    const int m = warp * 32 + lane;
#pragma unroll 1
    for (int col = 0; col < kAbN; col += 16) {
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)col)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int q = 0; q < 16; ++q) dst[(size_t)(col + q) * kAbM + m] = __uint_as_float(v[q]);  // [image][class]
    }
  }
  if (last < 0 && warp < 4) {  // an empty range contributes zeros
    float* dst = part + (size_t)blockIdx.x * kAbM * kAbN;
    for (int e = tid; e < kAbM * kAbN; e += 128) dst[e] = 0.0f;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kAbN) : "memory");
  }
  if (tid == 0 && bad) atomicOr(status, kStTimeout);
}

// Bt[n][c] = BF16(R_n[i_c] L_n[j_c]) for the sorted cells c (zero past the last cell and image).
// With lo != nullptr also lo[n][c] = BF16(x - hi): the split form hi + lo carries about 16 bits.
__global__ void cell_products_kernel(const float* __restrict__ R, const float* __restrict__ L,
                                     const uint32_t* __restrict__ cells, int ncells, int ncells_pad, int n, int K,
                                     uint16_t* __restrict__ Bt, uint16_t* __restrict__ lo) {
  const int img = blockIdx.y;
  for (int c8 = blockIdx.x * blockDim.x + threadIdx.x; c8 < ncells_pad / 8; c8 += gridDim.x * blockDim.x) {
    uint32_t w[4], wl[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t h[2], l2[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int c = c8 * 8 + 2 * q + e;
        float x = 0.0f;
        if (img < n && c < ncells) {
          const uint32_t ij = cells[c];
          x = R[(size_t)img * K + (ij >> 16)] * L[(size_t)img * K + (ij & 0xFFFFu)];
        }
        const __nv_bfloat16 hb = __float2bfloat16_rn(x);
        h[e] = __bfloat16_as_ushort(hb);
        l2[e] = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(hb)));
      }
      w[q] = h[0] | (h[1] << 16);
      wl[q] = l2[0] | (l2[1] << 16);
    }
    *reinterpret_cast<uint4*>(Bt + (size_t)img * ncells_pad + (size_t)c8 * 8) = make_uint4(w[0], w[1], w[2], w[3]);
    if (lo) *reinterpret_cast<uint4*>(lo + (size_t)img * ncells_pad + (size_t)c8 * 8) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
  }
}

// P[n][k] = sum of the split partials of the tiles holding (class k, image n).
__global__ void sum_partials_kernel(const float* __restrict__ part, const int* __restrict__ first, int splits_max,
                                    const int* __restrict__ count, int n, int K, int ntile_n, float* __restrict__ P) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x, img = blockIdx.y;
  if (k >= K || img >= n) return;
  const int mt = k / kAbM, nt = img / kAbN, pair = mt * ntile_n + nt;
  float s = 0.0f;
  for (int q = 0; q < count[pair]; ++q)
    s += part[(size_t)(first[pair] + q) * kAbM * kAbN + (size_t)(img % kAbN) * kAbM + (k % kAbM)];
  P[(size_t)img * K + k] = s;
}

// The FP32 gather on the CUDA cores: one CTA per image, a warp per class, lanes over the class's
// sorted cells, a shuffle tree at the end.
__global__ void __launch_bounds__(256) class_totals_fp32_kernel(const float* __restrict__ R, const float* __restrict__ L,
                                                                const uint32_t* __restrict__ cells,
                                                                const int* __restrict__ cstart, int K,
                                                                float* __restrict__ P) {
  extern __shared__ float rl[];
  const int img = blockIdx.x;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    rl[k] = R[(size_t)img * K + k];
    rl[K + k] = L[(size_t)img * K + k];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int k = warp; k < K; k += nw) {
    float s = 0.0f;
    for (int c = cstart[k] + lane; c < cstart[k + 1]; c += 32) {
      const uint32_t ij = cells[c];
      s = fmaf(rl[ij >> 16], rl[K + (ij & 0xFFFFu)], s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) P[(size_t)img * K + k] = s;
  }
}

}  // namespace

// Host side of the ablation: sorted cells, tiles and splits, then the kernels (one call; device
// buffers are allocated and freed inside: the hook measures the kernels, not the allocations).
hr_status ablation_class_totals(int K, int n, const float* d_R, const float* d_L, float* d_P, int method,
                                unsigned* d_status, int sms, cudaStream_t st, float* kernel_ms) {
  const int ncells = K * K;
  const int ncells_pad = (ncells + kAbChunk - 1) / kAbChunk * kAbChunk;
  // cells sorted by class (rows ascending within a class), the class of each sorted cell
  std::vector<int> csize(K + 1, 0), cstart(K + 1, 0);
  auto cls = [&](int i, int j) { return (int)((2LL * i * j + (K - 1)) / (2LL * (K - 1))); };
  for (int i = 0; i < K; ++i)
    for (int j = 0; j < K; ++j) ++csize[cls(i, j)];
  for (int k = 0; k < K; ++k) cstart[k + 1] = cstart[k] + csize[k];
  std::vector<uint32_t> cells(ncells);
  std::vector<uint16_t> cls_of(ncells_pad, (uint16_t)0xFFFFu);
  {
    std::vector<int> at(cstart.begin(), cstart.end() - 1);
    for (int i = 0; i < K; ++i)
      for (int j = 0; j < K; ++j) {
        const int k = cls(i, j), c = at[k]++;
        cells[c] = ((uint32_t)i << 16) | (uint32_t)j;
        cls_of[c] = (uint16_t)k;
      }
  }
  uint32_t* d_cells = nullptr;
  int* d_cstart = nullptr;
  cudaError_t e = cudaMalloc(&d_cells, sizeof(uint32_t) * ncells);
  if (e == cudaSuccess) e = cudaMalloc(&d_cstart, sizeof(int) * (K + 1));
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_cells, cells.data(), sizeof(uint32_t) * ncells, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_cstart, cstart.data(), sizeof(int) * (K + 1), cudaMemcpyHostToDevice, st);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  uint16_t *d_cls = nullptr, *d_Bt = nullptr;
  float* d_part = nullptr;
  AbTile* d_tiles = nullptr;
  int *d_first = nullptr, *d_count = nullptr;
  if (e == cudaSuccess && method == 0) {
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess)
      e = launch_kernel(class_totals_fp32_kernel, dim3(n), dim3(256), (size_t)2 * K * sizeof(float), st, false, d_R, d_L,
                        (const uint32_t*)d_cells, (const int*)d_cstart, K, d_P);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  } else if (e == cudaSuccess) {
    const int ntile_m = K / kAbM, ntile_n = (n + kAbN - 1) / kAbN, n_pad = ntile_n * kAbN;
    // chunk range of each class tile, split over about `sms` CTAs in proportion to the chunks
    std::vector<int> cr0(ntile_m), cr1(ntile_m);
    long long total = 0;
    for (int m = 0; m < ntile_m; ++m) {
      cr0[m] = cstart[m * kAbM] / kAbChunk;
      cr1[m] = (cstart[(m + 1) * kAbM] + kAbChunk - 1) / kAbChunk;
      total += cr1[m] - cr0[m];
    }
    std::vector<AbTile> tiles;
    std::vector<int> first(ntile_m * ntile_n), count(ntile_m * ntile_n);
    const int per_n = std::max(1, sms / ntile_n);
    for (int m = 0; m < ntile_m; ++m) {
      const int len = cr1[m] - cr0[m];
      const int splits = std::max(1, std::min(len, (int)((long long)per_n * len / std::max(1LL, total))));
      for (int nt = 0; nt < ntile_n; ++nt) {
        first[m * ntile_n + nt] = (int)tiles.size();
        count[m * ntile_n + nt] = splits;
        for (int q = 0; q < splits; ++q)
          tiles.push_back(AbTile{m, nt, cr0[m] + (int)((long long)len * q / splits),
                                 cr0[m] + (int)((long long)len * (q + 1) / splits)});
      }
    }
    e = cudaMalloc(&d_cls, sizeof(uint16_t) * ncells_pad);
    const int passes = method == 2 ? 2 : 1;
    const size_t pass_stride = (size_t)n_pad * ncells_pad;
    if (e == cudaSuccess) e = cudaMalloc(&d_Bt, sizeof(uint16_t) * pass_stride * passes);
    if (e == cudaSuccess) e = cudaMalloc(&d_part, sizeof(float) * (size_t)tiles.size() * kAbM * kAbN);
    if (e == cudaSuccess) e = cudaMalloc(&d_tiles, sizeof(AbTile) * tiles.size());
    if (e == cudaSuccess) e = cudaMalloc(&d_first, sizeof(int) * first.size());
    if (e == cudaSuccess) e = cudaMalloc(&d_count, sizeof(int) * count.size());
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_cls, cls_of.data(), sizeof(uint16_t) * ncells_pad, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(AbTile) * tiles.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_first, first.data(), sizeof(int) * first.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_count, count.data(), sizeof(int) * count.size(), cudaMemcpyHostToDevice, st);
    const size_t smem = 4 * (size_t)kAbTileBytes;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(onehot_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess)
      e = launch_kernel(cell_products_kernel, dim3(std::max(1, std::min(64, ncells_pad / 8 / 256)), n_pad), dim3(256), 0, st,
                        false, d_R, d_L, (const uint32_t*)d_cells, ncells, ncells_pad, n, K, d_Bt,
                        passes == 2 ? d_Bt + pass_stride : (uint16_t*)nullptr);
    if (e == cudaSuccess)
      e = launch_kernel(onehot_gemm_kernel, dim3((unsigned)tiles.size()), dim3(kAbThreads), smem, st, false,
                        (const uint16_t*)d_cls, (const uint16_t*)d_Bt, (const AbTile*)d_tiles, ncells_pad, passes,
                        pass_stride, d_part, d_status);
    if (e == cudaSuccess)
      e = launch_kernel(sum_partials_kernel, dim3((K + 127) / 128, n), dim3(128), 0, st, false, (const float*)d_part,
                        (const int*)d_first, 0, (const int*)d_count, n, K, ntile_n, d_P);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  }
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess && kernel_ms) e = cudaEventElapsedTime(kernel_ms, e0, e1);
  cudaFree(d_cells); cudaFree(d_cstart); cudaFree(d_cls); cudaFree(d_Bt); cudaFree(d_part); cudaFree(d_tiles);
  cudaFree(d_first); cudaFree(d_count);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? HR_ERR_OOM : HR_ERR_CUDA;
  }
  return HR_OK;
}

}  // namespace hr
