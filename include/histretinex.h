/*
 * histretinex.h -- C ABI of the GB300 (sm_103a) HistRetinex library.
 *
 * HistRetinex (Zhao et al., arXiv 2510.21100) enhances a low-light RGB image in the
 * histogram domain.  One call runs the whole per-image pipeline on the GPU:
 *
 *   1. V = max(r, g, b), the HSV value channel the paper enhances (Sec. II preamble);
 *      its K-bin count histogram H_C(S) (Eq. 3) and the histogram H_C(grad S) of its
 *      gradient image (Algorithm 1 initialisation; 3x3 Sobel magnitude, replicate border,
 *      rounded half up, clipped to K-1);
 *   2. the two-level optimisation of Sec. III.B: class map of the histogram location
 *      matrix (Eq. 7 and the definition under Eq. 10), weights of the histogram count
 *      matrix (Eq. 6, Eq. 11), reflectance update (Eq. 13), illumination update (Eq. 12),
 *      renormalisation (Eq. 14, Eq. 15), iterated as Algorithm 1;
 *   3. histogram reprocessing (Sec. III.C): gamma on the illumination location
 *      histogram (Eq. 17), new location matrix (Eq. 18), index_1 (Eq. 19) and the
 *      enhanced histogram (Eq. 20);
 *   4. histogram matching of V to that histogram as a K-entry LUT (Sec. III.C, last
 *      paragraph): LUT[s] = smallest z with CT(z) * N >= CS(s) * CT(K-1);
 *   5. the per-pixel apply: V' = LUT[V], each channel c -> round_half_up(c * V' / V),
 *      which keeps hue and saturation (Sec. II preamble; Sec. IV.A on methods that
 *      stretch all three channels); a black pixel becomes grey (V', V', V').
 *
 * Data layout: images are interleaved RGB, row-major, 3 channels per pixel, each
 * channel one byte (elem_bytes = 1, uint8) or a little-endian uint16 (elem_bytes = 2,
 * values < K, e.g. 12-bit data with K = 4096).  Rows are `pitch` bytes apart
 * (pitch >= 3 * width * elem_bytes).  Input and output may be the same buffer.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 * Device-side calls are asynchronous on that stream; argument errors are returned
 * synchronously; errors found by the kernels (a level >= K) are recorded in a device
 * status word and returned by histretinex_sync_status().  The kernels wait only at
 * hardware barriers (CTA and cluster barriers, copy completion), never in a spin loop;
 * HR_ERR_TIMEOUT is kept for a bounded device-side wait and is not raised today.
 *
 * Ownership: the caller owns every image buffer; the context owns its device
 * workspace and per-K tables and frees them in histretinex_destroy().  A context is
 * bound to one device and must not be used from two host threads at once.
 */
#ifndef HISTRETINEX_H
#define HISTRETINEX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HR_OK = 0,
  HR_ERR_INVALID_ARG = 1,  /* a bad pointer, size, pitch or parameter */
  HR_ERR_UNSUPPORTED = 2,  /* a valid request the library does not handle (see each call) */
  HR_ERR_OOM = 3,          /* device or host allocation failed */
  HR_ERR_CUDA = 4,         /* a CUDA runtime call failed */
  HR_ERR_RANGE = 5,        /* an image held a level >= K */
  HR_ERR_TIMEOUT = 6       /* a bounded device-side wait gave up (reserved: no kernel spins) */
} hr_status;

typedef enum {
  HR_PREC_FP64 = 0,        /* the plain form: the K-dimensional solve in FP64 */
  HR_PREC_FP32 = 1,        /* reduced precision: solve sums in FP32 (histograms, CDFs exact; LUT compare in FP64) */
  HR_PREC_DF64 = 4         /* the solve in double-float pairs of FP32 numbers (about 2^-47 relative per
                              operation, within the plain form's tolerance of the FP64 result), for
                              throughput where the FP64 rate is low; LUT compare in FP64 */
} hr_precision;

enum {
  HR_FLAG_FIXED_ITERS = 1u,  /* always run max_iter iterations of Algorithm 1 (ignore eps) */
  HR_FLAG_DEBUG_OUT = 2u,    /* keep per-image intermediates for histretinex_get_debug() */
  HR_FLAG_STAGE_TIMING = 4u, /* record CUDA events around each pipeline stage (histretinex_stage_times) */
  /* Printed forms of three points the default readings settle otherwise (each may be set alone): */
  HR_FLAG_PRINTED_UPDATE = 8u,    /* Eq. 12 and Eq. 13 as printed: the weight K_ij of Eq. 11 divides the
                                     data term, sum_i H_C(R)_i H_C(S)_idx(i,j) / (N K_ij), instead of
                                     multiplying it (the default is the stationary point of Eq. 10);
                                     FP64 only (other precisions: HR_ERR_UNSUPPORTED at create) */
  HR_FLAG_NEAREST_MATCH = 16u,    /* histogram matching (Sec. III.C) to the target level whose cumulative
                                     share is nearest to the source level's: LUT[s] = first z minimising
                                     |CT(z) N - CS(s) CT(K-1)| (default: the first z that reaches it) */
  HR_FLAG_FORWARD_GRADIENT = 32u  /* the gradient image (Sec. III.B, Algorithm 1) by forward differences
                                     gx = V(x+1,y) - V(x,y), gy = V(x,y+1) - V(x,y), replicate border
                                     (default: the 3x3 Sobel operator); runs the generic histogram kernel */
};

/* Method parameters.  alpha, beta: weights of the illumination and reflectance priors
 * (Eq. 9); gamma: Eq. 17; eps, max_iter: stopping threshold and iteration cap T of
 * Algorithm 1 (stop when both squared changes are <= eps, or after max_iter).
 * K must be a power of two in [8, 4096]; elem_bytes = 1 needs K <= 256.
 * levels: 0 (one bin per level: the data's levels are 0 .. K-1), or M, a power of two in
 * [K, 4096], the data's levels binned into the K bins ("l levels", Sec. II preamble, with fewer
 * bins than levels, e.g. K = 256 on 12-bit data, M = 4096): value v falls into bin
 * v >> log2(M / K); bin k is located at its centre value, (k w + (w - 1)/2) / (M - 1) with
 * w = M / K (the location histogram of Sec. III.A; for M = K this is k / (K - 1)); the class maps
 * of Eq. 10 and Eq. 19 are the argmins over those locations; the gradient level is clipped to M - 1
 * and binned likewise; the LUT maps bins, and a pixel's new value keeps its place in its bin,
 * V' = LUT[s] w + (V - s w).  Values >= M are a range error.  8-bit data needs M <= 256.  The
 * binned form runs the generic pixel kernels. */
typedef struct {
  int K;
  double alpha;
  double beta;
  double gamma;
  double eps;
  int max_iter;
  int precision;   /* hr_precision */
  unsigned flags;  /* HR_FLAG_* */
  int levels;      /* 0, or M: data levels binned into the K bins */
} hr_params;

typedef struct hr_ctx hr_ctx;

/* Launch shapes (not part of the paper's method).  hist_ctas_per_sm, apply_ctas_per_sm: the
 * persistent grids of the two pixel passes are SMs x this many CTAs (1..32; defaults 8 and 16; the
 * 8-bit strip histogram kernel for large images and batches with 16-byte aligned rows runs one CTA
 * per SM instead);
 * solve_cluster: CTAs per thread-block cluster of an image's solve (1, 2, 4, 8 or 16; default 16,
 * lowered automatically when that cluster cannot be resident; a batch of n images uses at most
 * SMs / n, rounded down to a power of two, so that it runs in one wave); use_graph: 1 to
 * capture enhance_batch's launches into a CUDA graph that is replayed while the batch's geometry
 * (image count, sizes, element size, alignment) is unchanged (default 1).  Stage timing is not
 * recorded for graph replays.  pdl: which kernels are programmatic dependent launches (bit 0 the
 * histogram pass, bit 1 the solve, bit 2 the apply pass; 0..7): such a kernel is scheduled while
 * the kernel before it on the stream finishes and waits on the device for that kernel's results
 * (default 5, the two pixel passes; 0: plain stream order).  A dependent solve measured slower on
 * GB300 (its cluster is placed while the histogram pass drains).  groups: a graph-replayed batch
 * of at least 64 images runs as 1 or 2 groups (default 2: images [0, n/2) and [n/2, n) on two
 * streams, the second group's histogram pass after the first's, so one group's solve overlaps the
 * other's pixel passes).  partitions: 0, or the number (1..4) of 16-SM partitions the GPU's SMs are
 * split into for the solves of single-image calls, the remaining SMs forming one partition for their
 * pixel passes (green contexts; default 2).  A call then runs its histogram and apply passes in the
 * pixel partition and its solve in a solve partition, on the context's own streams, forked from and
 * joined back into the caller's stream; calls on different caller streams overlap (one image's
 * solve beside other images' pixel passes).  partition_cluster: CTAs per cluster of those solves
 * (1, 2, 4, 8 or 16; default 16); each solve partition runs 16 / partition_cluster of them at once
 * (smaller clusters take longer per image but use the SMs better: for a stream of 7680x4320 images
 * on many caller streams, partitions = 1 with partition_cluster = 4 gives the highest throughput).  A partitioned call's results are
 * bit-identical to the same call unpartitioned with solve_cluster = partition_cluster.
 * Single-image calls use a ring of workspace slots, each call the next (16 slots for workspaces of
 * up to 16 MB, else 4).  Calls under stream capture or with stage timing, and devices whose SMs
 * cannot be split so, run unpartitioned. */
typedef struct {
  int hist_ctas_per_sm;
  int apply_ctas_per_sm;
  int solve_cluster;
  int use_graph;
  int pdl;
  int groups;
  int partitions;
  int partition_cluster;
} hr_tuning;

/* Fills *p with the defaults: K = 256, alpha = beta = 1e-3, gamma = 2.2 (Sec. III.C),
 * eps = 0, max_iter = 10 (Sec. IV.C), FP64, fixed iterations, levels = 0. */
void histretinex_default_params(hr_params* p);

/* Creates a context on `device` for parameters *p (copied).  Builds the per-K tables
 * (the Eq. 19 class map as per-row class boundaries).  Returns HR_ERR_INVALID_ARG for
 * invalid parameters, HR_ERR_UNSUPPORTED for HR_FLAG_PRINTED_UPDATE with a precision other
 * than FP64, HR_ERR_CUDA / HR_ERR_OOM on device failures. */
hr_status histretinex_create(hr_ctx** out, const hr_params* p, int device);

/* Enhances one image already in device memory (Sec. III, the whole pipeline above).
 * d_in, d_out: device pointers to W x H interleaved RGB images (may alias);
 * in_pitch, out_pitch: row strides in bytes; elem_bytes: 1 or 2.
 * Asynchronous on `stream`: the call reads its input after the stream's earlier work and its
 * output is complete when the stream reaches the work queued after it.  Calls on different
 * streams may overlap on the device: each takes the next of the context's single-image
 * workspace slots and its device work waits for that slot's previous call, so such calls need no
 * ordering by the caller (with SM partitions, hr_tuning.partitions > 0, one call's solve then runs
 * beside other calls' pixel passes).  Under stream capture a call uses the context's first batch
 * slot instead and orders nothing across streams: calls captured on different streams must be
 * ordered by the caller.  A context must not be used from two host threads at once.  Images with
 * W*H >= 2^31 return HR_ERR_UNSUPPORTED. */
hr_status histretinex_enhance(hr_ctx* ctx, const void* d_in, void* d_out, int width, int height,
                              size_t in_pitch, size_t out_pitch, int elem_bytes, void* stream);

/* Enhances n images (each as in histretinex_enhance) with one launch per pipeline stage:
 * persistent kernels walk per-image work queues, so images of mixed sizes share the GPU; the
 * launches are captured into a CUDA graph and replayed while the batch geometry is unchanged.
 * The arrays are HOST arrays of length n (d_in[i], d_out[i] are device pointers).
 * Every image is solved by a cluster of C CTAs, C the largest power of two up to the tuned
 * solve_cluster with n C <= SMs (one CTA each for large batches).  An image's result (pixels,
 * LUT and FP64 histograms) depends only on the image and C: it is bit-identical whatever else is
 * in the batch for batches of the same C, and a batch of one matches histretinex_enhance.
 * Between different C the FP64 histograms agree to rounding (they are summed in another order)
 * and the pixels and LUT agree. */
hr_status histretinex_enhance_batch(hr_ctx* ctx, int n, const void* const* d_in, void* const* d_out,
                                    const int* width, const int* height, const size_t* in_pitch,
                                    const size_t* out_pitch, int elem_bytes, void* stream);

/* End-to-end form: copies a HOST image to the device, enhances it, copies the result back
 * into a HOST buffer and waits for the stream.  Pinned host memory gives full copy speed. */
hr_status histretinex_enhance_host(hr_ctx* ctx, const void* h_in, void* h_out, int width, int height,
                                   size_t in_pitch, size_t out_pitch, int elem_bytes, void* stream);

/* End-to-end form for a sequence of n HOST images (arrays of n pointers, sizes and pitches; the
 * images may differ in size): each image goes through the plain single-image pipeline of
 * histretinex_enhance, while the host-to-device copy of the next image and the device-to-host
 * copy of the previous one run on the context's own copy streams (two device buffer pairs, in
 * turn).  Work already queued on `stream` comes first; the call returns when every result is in
 * host memory.  Pinned host memory gives full copy speed.  Not part of the paper's method:
 * throughput support for host-resident images.  Errors as histretinex_enhance_host. */
hr_status histretinex_enhance_host_many(hr_ctx* ctx, int n, const void* const* h_in, void* const* h_out,
                                        const int* width, const int* height, const size_t* in_pitch,
                                        const size_t* out_pitch, int elem_bytes, void* stream);

/* Allocation-free single-image enhancement, without a context.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory at the point of the
 * call -- code running while a framework captures a CUDA graph, real-time loops that must not
 * block in an allocator, plug-ins whose host application owns all device memory.  It runs the
 * same pipeline as histretinex_enhance (parameters *p as for histretinex_create, images as for
 * histretinex_enhance) for K <= 256, with its whole workspace in one 1 MiB array that the library
 * declares in device memory; that array stays resident on every device that loads the library
 * until the process exits.  It calls no cudaMalloc, cudaFree or other allocating routine.
 * K > 256 and binned data (levels other than 0 or K) return HR_ERR_UNSUPPORTED.  Each call looks up the array's address on the current
 * device (cudaGetSymbolAddress, which allocates nothing; the first call on a device may load the
 * library's device code, so make it before any stream capture), then queues on `stream` two
 * memsets (the histograms it accumulates and its status word) and four kernels (its own table of
 * the class boundaries for its K and gamma, built from values passed by value, then the three
 * pipeline stages): nothing it reads is left over from an earlier call.  Every call uses the same
 * array, so calls whose work overlaps on the GPU (other streams, other threads) race on it and
 * must be serialised by the caller.  Levels >= K are clamped but not reported.  Asynchronous on
 * `stream`. */
hr_status histretinex_enhance_noalloc(const hr_params* p, const void* d_in, void* d_out, int width, int height,
                                      size_t in_pitch, size_t out_pitch, int elem_bytes, void* stream);

/* Intermediates of image `image` of the last enhance / enhance_batch call (index 0 for
 * enhance).  Needs HR_FLAG_DEBUG_OUT.  All outputs are HOST arrays of K entries (any may
 * be NULL): S = H_C(S), G = H_C(grad S), R = H_C(R), L = H_C(L) after Algorithm 1,
 * T = the enhanced histogram of Eq. 20, lut = the matching LUT; *iters = iterations run.
 * Synchronises the device. */
hr_status histretinex_get_debug(hr_ctx* ctx, int image, uint64_t* S, uint64_t* G, double* R, double* L,
                                double* T, uint16_t* lut, int* iters);

/* Waits for `stream` and returns the device status of the calls issued so far (HR_OK,
 * HR_ERR_RANGE or HR_ERR_TIMEOUT), then clears it. */
hr_status histretinex_sync_status(hr_ctx* ctx, void* stream);

/* Frees the context and everything it owns.  NULL is accepted. */
hr_status histretinex_destroy(hr_ctx* ctx);

/* Static description of a status code. */
const char* histretinex_status_string(hr_status s);

/* Device workspace bytes the context keeps per image of a batch (for memory budgeting). */
size_t histretinex_workspace_bytes(const hr_ctx* ctx);

/* Allocates now the workspace and descriptor buffers of batches of up to n_images images, so that
 * later calls with at most that many images allocate nothing (growing them frees the old buffers,
 * which waits for all work on the device).  Not part of the paper's method: serving support.
 * HR_ERR_INVALID_ARG for n_images < 1, HR_ERR_OOM when the allocation fails. */
hr_status histretinex_reserve(hr_ctx* ctx, int n_images);

/* Sets / reads the context's launch shapes (see hr_tuning).  Invalid fields give
 * HR_ERR_INVALID_ARG and leave the tuning unchanged. */
hr_status histretinex_set_tuning(hr_ctx* ctx, const hr_tuning* t);
hr_status histretinex_get_tuning(const hr_ctx* ctx, hr_tuning* t);

/* Stage timing (needs HR_FLAG_STAGE_TIMING): every enhance / enhance_batch call records CUDA
 * events on its own stream before and after each of its three stages.  This call waits for
 * them and writes the summed device times in milliseconds since the last reset to ms[0]
 * (histogram pass), ms[1] (solve: Algorithm 1, Eq. 20, LUT) and ms[2] (apply pass), and the
 * number of calls covered to *calls; reset != 0 clears the sums afterwards.  Not part of the
 * paper's method: a measurement hook. */
hr_status histretinex_stage_times(hr_ctx* ctx, double* ms, int* calls, int reset);

/* Solve-phase timestamps of image `image` of the last call (needs HR_FLAG_DEBUG_OUT): up to
 * *count device times in nanoseconds (%globaltimer) taken by the first CTA of the image's solve
 * at its phase boundaries (set-up, each iteration's three barriers, target, LUT), written to ns;
 * *count is set to the number written.  Synchronises the device.  A measurement hook. */
hr_status histretinex_profile_solve(hr_ctx* ctx, int image, long long* ns, int* count);

/* Self-test hook, not part of the paper's method: the gradient level of step 1 -- the nearest
 * integer to sqrt(m2), halves rounded up, clipped to K - 1 -- of every squared Sobel magnitude m2
 * in [m2_first, m2_first + n), computed by the device code of one of the histogram kernels:
 * form 0 that of the strip kernel (8-bit images: K <= 256; any m2 >= 0), form 1 that of the
 * staged-tile kernel (8-bit images: K <= 256; m2 < 2^23), form 2 that of the generic kernel
 * (K <= 4096; m2 < 2^31).  d_out: device array of n uint16 entries, d_out[t] = level of
 * m2_first + t.  Asynchronous on `stream`.  HR_ERR_INVALID_ARG for an unknown form, K not a power
 * of two in [8, 4096] (or above 256 for forms 0 and 1), m2_first < 0, n < 1, a null d_out or a
 * range beyond the form's; HR_ERR_CUDA if the launch fails. */
hr_status histretinex_gradient_levels(int form, int K, int m2_first, int n, uint16_t* d_out, void* stream);

/* Measured ablation of the reduced-precision form (the K x K products batched across images as a
 * dense contraction on the tensor cores), not part of the paper's
 * method and not on the enhancement path: the Eq. 11 class totals P_n[k] = sum over the cells
 * (i, j) of class k (index(i, j) = round(i j / (K - 1)), definition under Eq. 10) of R_n[i] L_n[j]
 * (the count matrix of Eq. 6 without its 1/N) for n images at once.  method 0: an FP32 gather on the
 * CUDA cores (a warp per class, FP32 fused multiply-adds); method 1: the class-sorted one-hot GEMM
 * P = Z X on the tcgen05 tensor cores, Z the K x K^2 0/1 class matrix (exact in BF16), X the cell
 * products rounded to BF16, FP32 accumulation in tensor memory; method 2: the same contraction over
 * each product split into two BF16 numbers, hi + lo (two passes, about 16 bits kept).  d_R, d_L: device arrays of n x K
 * FP32 values (image-major, level-indexed); d_P: device output, n x K FP32.  K must be 128 or 256,
 * 1 <= n <= 4096.  The call allocates its own device buffers, waits for its kernels, and writes their
 * device time in ms to *kernel_ms (may be NULL).  HR_ERR_TIMEOUT if a bounded wait of the tensor-core
 * kernel gave up (its results are then not valid). */
hr_status histretinex_ablation_class_totals(int K, int n, const float* d_R, const float* d_L, float* d_P, int method,
                                           float* kernel_ms, void* stream);

/* The SM partitioning single-image calls run with (see hr_tuning.partitions): *solve_parts = the
 * number of 16-SM solve partitions in use (0: unpartitioned, before the first call or where the
 * split is unavailable), *pixel_sms = the SMs of the pixel partition (all SMs when unpartitioned).
 * Not part of the paper's method. */
hr_status histretinex_partition_info(const hr_ctx* ctx, int* solve_parts, int* pixel_sms);

/* Number of kernels this library launched on the context since creation (for
 * launch accounting by callers and benchmarks). */
uint64_t histretinex_kernel_launches(const hr_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* HISTRETINEX_H */
