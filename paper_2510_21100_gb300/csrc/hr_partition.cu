// SM partitions for overlapping single-image calls (not part of the paper's method).
//
// One image's pipeline is three dependent stages: the histogram pass and the apply pass stream
// the image through HBM on every SM, the solve between them is latency-bound work on one 16-CTA
// cluster, during which the other SMs of the GPU idle.  Calls on different streams can fill that
// gap only if the solve's cluster and the other calls' pixel passes get SMs at the same time, and
// persistent pixel kernels that hold every SM keep a cluster from being placed until they end.
// So the SMs are split once, with green contexts, into `parts` partitions of 16 SMs for solves and
// one partition of the rest for pixel passes.  Each solve partition has `sper` solve streams, so
// it runs sper solves of 16 / sper CTAs at once (smaller clusters use SMs better: at 7680x4320
// one FP64 solve takes 149 us on 16 CTAs and 205 us on 4).  A call forks from the caller's stream
// into a pixel stream of its workspace slot (histogram pass), the next solve stream, partitions
// taken in turn (solve), and back (apply), then joins the caller's stream: calls on different
// caller streams overlap, each image's arithmetic is unchanged (same kernels, same cluster size
// as an unpartitioned call), and the caller's stream sees the call's results complete, as without
// partitions.
//
// The driver's green-context entry points are fetched through the runtime, so the library keeps
// no link-time dependency on the driver library.
#include <cuda.h>

#include <cstring>
#include <new>

#include "hr_internal.cuh"

namespace hr {

namespace {

struct Driver {
  CUresult (*DeviceGet)(CUdevice*, int) = nullptr;
  CUresult (*DeviceGetDevResource)(CUdevice, CUdevResource*, CUdevResourceType) = nullptr;
  CUresult (*DevSmResourceSplitByCount)(CUdevResource*, unsigned*, const CUdevResource*, CUdevResource*, unsigned,
                                        unsigned) = nullptr;
  CUresult (*DevResourceGenerateDesc)(CUdevResourceDesc*, CUdevResource*, unsigned) = nullptr;
  CUresult (*GreenCtxCreate)(CUgreenCtx*, CUdevResourceDesc, CUdevice, unsigned) = nullptr;
  CUresult (*GreenCtxDestroy)(CUgreenCtx) = nullptr;
  CUresult (*GreenCtxStreamCreate)(CUstream*, CUgreenCtx, unsigned, int) = nullptr;
  CUresult (*CtxFromGreenCtx)(CUcontext*, CUgreenCtx) = nullptr;
  CUresult (*CtxPushCurrent)(CUcontext) = nullptr;
  CUresult (*CtxPopCurrent)(CUcontext*) = nullptr;
  CUresult (*StreamDestroy)(CUstream) = nullptr;
};

template <typename Fn>
bool entry(const char* name, Fn& fn) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &p, CUDART_VERSION, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !p) {
    cudaGetLastError();
    return false;
  }
  fn = reinterpret_cast<Fn>(p);
  return true;
}

bool load_driver(Driver& d) {
  return entry("cuDeviceGet", d.DeviceGet) && entry("cuDeviceGetDevResource", d.DeviceGetDevResource) &&
         entry("cuDevSmResourceSplitByCount", d.DevSmResourceSplitByCount) &&
         entry("cuDevResourceGenerateDesc", d.DevResourceGenerateDesc) && entry("cuGreenCtxCreate", d.GreenCtxCreate) &&
         entry("cuGreenCtxDestroy", d.GreenCtxDestroy) && entry("cuGreenCtxStreamCreate", d.GreenCtxStreamCreate) &&
         entry("cuCtxFromGreenCtx", d.CtxFromGreenCtx) && entry("cuCtxPushCurrent", d.CtxPushCurrent) &&
         entry("cuCtxPopCurrent", d.CtxPopCurrent) && entry("cuStreamDestroy", d.StreamDestroy);
}

constexpr int kMaxParts = 4;
constexpr int kMaxSper = 16;   // solve streams per partition (16 one-CTA solves)
constexpr int kSolveSms = 16;  // SMs per solve partition

}  // namespace

struct Partitions {
  Driver drv;
  int parts = 0, sper = 0, ring = 0, next = 0, pixel_sms = 0;
  CUgreenCtx green[kMaxParts + 1] = {};  // [0, parts): solve partitions; [parts]: pixel partition
  CUcontext ctx[kMaxParts + 1] = {};
  CUstream solve_st[kMaxParts][kMaxSper] = {};
  CUstream* pixel_st = nullptr;          // one per workspace slot
  cudaEvent_t ev_in = nullptr;           // (primary context) the caller's stream reached the call
  cudaEvent_t ev_hist = nullptr;         // (pixel partition) the histogram pass is done
  cudaEvent_t ev_solve[kMaxParts][kMaxSper] = {};  // (solve partition p, stream k) the solve is done
  cudaEvent_t ev_out = nullptr;          // (pixel partition) the apply pass is done
};

namespace {

// Runs f with partition context c current (kernels, events and attributes then belong to it).
template <typename F>
cudaError_t in_ctx(Partitions* P, CUcontext c, F f) {
  if (P->drv.CtxPushCurrent(c) != CUDA_SUCCESS) return cudaErrorInvalidResourceHandle;
  const cudaError_t e = f();
  CUcontext old;
  P->drv.CtxPopCurrent(&old);
  return e;
}

}  // namespace

void partitions_destroy(Partitions* P) {
  if (!P) return;
  for (int i = 0; i <= P->parts; ++i) {
    if (!P->ctx[i]) continue;
    in_ctx(P, P->ctx[i], [&]() {
      cudaDeviceSynchronize();
      if (i < P->parts) {
        for (int k = 0; k < P->sper; ++k) {
          if (P->ev_solve[i][k]) cudaEventDestroy(P->ev_solve[i][k]);
          if (P->solve_st[i][k]) P->drv.StreamDestroy(P->solve_st[i][k]);
        }
      } else {
        if (P->ev_hist) cudaEventDestroy(P->ev_hist);
        if (P->ev_out) cudaEventDestroy(P->ev_out);
        for (int r = 0; P->pixel_st && r < P->ring; ++r)
          if (P->pixel_st[r]) P->drv.StreamDestroy(P->pixel_st[r]);
      }
      return cudaSuccess;
    });
  }
  for (int i = 0; i <= P->parts; ++i)
    if (P->green[i]) P->drv.GreenCtxDestroy(P->green[i]);
  if (P->ev_in) cudaEventDestroy(P->ev_in);
  delete[] P->pixel_st;
  delete P;
}

hr_status partitions_create(int device, int parts, int sper, int ring, Partitions** out) {
  *out = nullptr;
  if (parts < 1 || parts > kMaxParts || sper < 1 || sper > kMaxSper || ring < 1) return HR_ERR_INVALID_ARG;
  Partitions* P = new (std::nothrow) Partitions();
  if (!P) return HR_ERR_OOM;
  P->parts = parts;
  P->sper = sper;
  P->ring = ring;
  P->pixel_st = new (std::nothrow) CUstream[ring]();
  if (!P->pixel_st || !load_driver(P->drv)) { partitions_destroy(P); return HR_ERR_UNSUPPORTED; }
  const Driver& d = P->drv;
  CUdevice dev;
  CUdevResource all, grp[kMaxParts], rem;
  unsigned nb = (unsigned)parts;
  if (d.DeviceGet(&dev, device) != CUDA_SUCCESS || d.DeviceGetDevResource(dev, &all, CU_DEV_RESOURCE_TYPE_SM) != CUDA_SUCCESS ||
      d.DevSmResourceSplitByCount(grp, &nb, &all, &rem, CU_DEV_SM_RESOURCE_SPLIT_MAX_POTENTIAL_CLUSTER_SIZE,
                                  kSolveSms) != CUDA_SUCCESS ||
      nb != (unsigned)parts || rem.sm.smCount < (unsigned)kSolveSms) {
    partitions_destroy(P);
    return HR_ERR_UNSUPPORTED;
  }
  for (int i = 0; i < parts; ++i)
    if (grp[i].sm.smCount < (unsigned)kSolveSms) { partitions_destroy(P); return HR_ERR_UNSUPPORTED; }
  P->pixel_sms = (int)rem.sm.smCount;
  for (int i = 0; i <= parts; ++i) {
    CUdevResourceDesc desc;
    CUdevResource* res = i < parts ? &grp[i] : &rem;
    if (d.DevResourceGenerateDesc(&desc, res, 1) != CUDA_SUCCESS ||
        d.GreenCtxCreate(&P->green[i], desc, dev, CU_GREEN_CTX_DEFAULT_STREAM) != CUDA_SUCCESS ||
        d.CtxFromGreenCtx(&P->ctx[i], P->green[i]) != CUDA_SUCCESS) {
      partitions_destroy(P);
      return HR_ERR_UNSUPPORTED;
    }
  }
  cudaError_t e = cudaEventCreateWithFlags(&P->ev_in, cudaEventDisableTiming);
  for (int i = 0; i < parts && e == cudaSuccess; ++i) {
    e = in_ctx(P, P->ctx[i], [&]() {
      for (int k = 0; k < sper; ++k) {
        if (d.GreenCtxStreamCreate(&P->solve_st[i][k], P->green[i], CU_STREAM_NON_BLOCKING, 0) != CUDA_SUCCESS)
          return cudaErrorInvalidResourceHandle;
        const cudaError_t x = cudaEventCreateWithFlags(&P->ev_solve[i][k], cudaEventDisableTiming);
        if (x != cudaSuccess) return x;
      }
      return cudaSuccess;
    });
  }
  if (e == cudaSuccess) {
    e = in_ctx(P, P->ctx[parts], [&]() {
      for (int r = 0; r < ring; ++r)
        if (d.GreenCtxStreamCreate(&P->pixel_st[r], P->green[parts], CU_STREAM_NON_BLOCKING, 0) != CUDA_SUCCESS)
          return cudaErrorInvalidResourceHandle;
      cudaError_t e2 = cudaEventCreateWithFlags(&P->ev_hist, cudaEventDisableTiming);
      if (e2 == cudaSuccess) e2 = cudaEventCreateWithFlags(&P->ev_out, cudaEventDisableTiming);
      return e2;
    });
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    partitions_destroy(P);
    return e == cudaErrorMemoryAllocation ? HR_ERR_OOM : HR_ERR_UNSUPPORTED;
  }
  *out = P;
  return HR_OK;
}

int partitions_pixel_sms(const Partitions* P) { return P ? P->pixel_sms : 0; }

cudaError_t partitions_run(Partitions* P, int slot, cudaStream_t st, const StageFn& hist, const StageFn& solve,
                           const StageFn& apply) {
  const int j = P->next % P->parts, k = P->next / P->parts;  // partitions in turn, then their streams
  P->next = (P->next + 1) % (P->parts * P->sper);
  CUcontext pix = P->ctx[P->parts];
  cudaStream_t ps = reinterpret_cast<cudaStream_t>(P->pixel_st[slot % P->ring]);
  cudaStream_t ss = reinterpret_cast<cudaStream_t>(P->solve_st[j][k]);
  // (each event is waited on right after it is recorded, so one event per hand-over suffices)
  cudaError_t e = cudaEventRecord(P->ev_in, st);  // everything before the call on the caller's stream
  if (e == cudaSuccess) e = in_ctx(P, pix, [&]() {
    cudaError_t x = cudaStreamWaitEvent(ps, P->ev_in, 0);
    if (x == cudaSuccess) x = hist(ps);
    if (x == cudaSuccess) x = cudaEventRecord(P->ev_hist, ps);
    return x;
  });
  if (e == cudaSuccess) e = in_ctx(P, P->ctx[j], [&]() {
    cudaError_t x = cudaStreamWaitEvent(ss, P->ev_hist, 0);
    if (x == cudaSuccess) x = solve(ss);
    if (x == cudaSuccess) x = cudaEventRecord(P->ev_solve[j][k], ss);
    return x;
  });
  if (e == cudaSuccess) e = in_ctx(P, pix, [&]() {
    cudaError_t x = cudaStreamWaitEvent(ps, P->ev_solve[j][k], 0);
    if (x == cudaSuccess) x = apply(ps);
    if (x == cudaSuccess) x = cudaEventRecord(P->ev_out, ps);
    return x;
  });
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, P->ev_out, 0);  // the caller's stream waits for the results
  return e;
}

}  // namespace hr
