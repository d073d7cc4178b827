// C ABI of the HistRetinex CUDA library: context, workspace, per-K tables, launches.
#include <cmath>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/histretinex.h"
#include "hr_internal.cuh"

using hr::ImageDesc;
using hr::SlotLayout;
using hr::ImgTab;

struct hr_ctx {
  int device = 0;
  hr_params p{};
  SlotLayout lay{};
  int sm_count = 0;
  uint8_t* d_slots = nullptr;
  int n_slots = 0;
  uint16_t* d_jstart1 = nullptr;   // [K][K+1], index_1 class boundaries (Eq. 19)
  uint16_t* d_cmap = nullptr;      // binned data: class map of Eq. 10 [K][K] and its boundaries [K][K+1]
  uint16_t* d_jstart0 = nullptr;
  int M = 0;                       // the data's levels (K unless binned)
  unsigned* d_status = nullptr;
  ImageDesc* d_imgs = nullptr;
  int* d_tile_start = nullptr;
  int cap_imgs = 0;
  ImageDesc* h_imgs = nullptr;     // pinned staging for the descriptors
  int* h_tile_start = nullptr;
  cudaEvent_t desc_done = nullptr; // the last descriptor upload has been consumed
  std::vector<ImageDesc> last_imgs;
  void* d_io_in = nullptr;         // device copies for the host-buffer entry point
  void* d_io_out = nullptr;
  size_t io_bytes = 0;
  // host-image sequences: two device buffer pairs, a copy stream each way, per-buffer events
  void* d_pp_in[2] = {nullptr, nullptr};
  void* d_pp_out[2] = {nullptr, nullptr};
  size_t pp_bytes = 0;
  cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
  cudaEvent_t ev_in_ready[2] = {}, ev_in_free[2] = {}, ev_done[2] = {}, ev_out_free[2] = {};
  uint64_t launches = 0;
  int last_n = 0;
  // stage timing: a ring of event quadruples, folded into the sums when reused or queried
  static constexpr int kRing = 256;
  cudaEvent_t ev[kRing][4] = {};
  bool ev_used[kRing] = {};
  int ev_next = 0;
  double stage_ms[3] = {0, 0, 0};
  int stage_calls = 0;
  hr_tuning tune{8, 16, 16, 1, 5, 2, 2, 16};
  // leading slots whose H_C(S) and H_C(grad S) are known to be zero (the solve clears them after
  // use unless the intermediates are kept for histretinex_get_debug)
  int hist_clean = 0;
  // captured batch pipeline and the geometry it was captured for
  cudaGraphExec_t graph = nullptr;
  int g_n = 0, g_total = 0, g_eb = 0, g_fast_in = 0, g_fast_out = 0, g_zero = 0, g_groups = 0, g_launches = 0;
  hr_tuning g_tune{0, 0, 0, 0, 0, 0, 0, 0};
  int last_groups = 0;  // groups of the uploaded tables
  // single-image calls on SM partitions: a ring of workspace slots, each known clean or not
  static constexpr int kRingMax = 16;
  hr::Partitions* part = nullptr;
  int part_parts = 0;               // partitions the current Partitions object was made with
  int part_sper = 0;                // and its solve streams per partition
  bool part_unavailable = false;    // the split failed on this device: run unpartitioned
  uint8_t* d_ring = nullptr;
  int ring_n = 0;                   // slots of the ring: 16 for workspaces up to 16 MB, else 4
  bool ring_clean[kRingMax] = {};
  cudaEvent_t ring_free[kRingMax] = {};  // recorded on the caller's stream after the slot's last call
  bool ring_pending[kRingMax] = {};
  int ring_next = 0;
  const uint8_t* last_base = nullptr;  // slot 0 of the last call's images (debug reads)
};

namespace hr {

bool pow2(int k) { return k > 0 && (k & (k - 1)) == 0; }

hr_status check_params(const hr_params* p) {
  if (!p) return HR_ERR_INVALID_ARG;
  if (!pow2(p->K) || p->K < 8 || p->K > 4096) return HR_ERR_INVALID_ARG;
  if (!(p->alpha > 0.0) || !(p->beta > 0.0) || !(p->gamma > 0.0) || !(p->eps >= 0.0)) return HR_ERR_INVALID_ARG;
  if (!std::isfinite(p->alpha) || !std::isfinite(p->beta) || !std::isfinite(p->gamma)) return HR_ERR_INVALID_ARG;
  if (p->max_iter < 1) return HR_ERR_INVALID_ARG;
  if (p->precision != HR_PREC_FP64 && p->precision != HR_PREC_FP32 && p->precision != HR_PREC_DF64)
    return HR_ERR_INVALID_ARG;
  // the printed update's values (S_k P_k, up to about N^3 / K, and reflectance bins that shrink
  // towards zero) leave FP32's exponent range, which the FP32 and double-float forms share
  if ((p->flags & HR_FLAG_PRINTED_UPDATE) && p->precision != HR_PREC_FP64) return HR_ERR_UNSUPPORTED;
  if (p->levels != 0 && (!pow2(p->levels) || p->levels < p->K || p->levels > 4096)) return HR_ERR_INVALID_ARG;
  return HR_OK;
}

// Location of bin k of K bins over M data levels: the bin's centre value normalised to [0, 1],
// (k w + (w - 1) / 2) / (M - 1), w = M / K (for M = K: k / (K - 1)).
static double bin_location(int k, int K, int M) {
  const long long w = M / K;
  return (double)(2 * (long long)k * w + w - 1) / (2.0 * (double)(M - 1));
}

// The first bin whose location is nearest to p (locations ascend: the minimum lies next to the
// first location >= p).
static int nearest_bin(double p, int K, int M) {
  int lo = 0, hi = K;
  while (lo < hi) {
    const int mid = (lo + hi) / 2;
    if (bin_location(mid, K, M) >= p) hi = mid; else lo = mid + 1;
  }
  const int a = lo - 2 < 0 ? 0 : lo - 2, b = lo + 1 > K - 1 ? K - 1 : lo + 1;
  int best = a;
  double bd = std::fabs(p - bin_location(a, K, M));
  for (int k = a + 1; k <= b; ++k) {
    const double d = std::fabs(p - bin_location(k, K, M));
    if (d < bd) { bd = d; best = k; }
  }
  return best;
}

void build_class_tables(int K, int M, uint16_t* cmap, uint16_t* js0) {
  for (int i = 0; i < K; ++i) {
    const double li = bin_location(i, K, M);
    uint16_t* row = js0 + (size_t)i * (K + 1);
    int k = 0;
    for (int j = 0; j < K; ++j) {
      const int c = nearest_bin(li * bin_location(j, K, M), K, M);
      cmap[(size_t)i * K + j] = (uint16_t)c;
      while (k <= c) row[k++] = (uint16_t)j;
    }
    while (k <= K) row[k++] = (uint16_t)K;
  }
}

// index_1(i, j) (Eq. 17-19): the level whose location k/(K-1) is nearest to the gamma-processed
// location matrix entry (j/(K-1))^(1/gamma) * i/(K-1); the first such level on a tie.  The
// distance is unimodal in k, so the minimum lies next to the rounded position.
static int index1(int K, double hl, double hr) {
  const double km1 = (double)(K - 1);
  const double p = hl * hr;
  long c = std::lround(p * km1);
  long lo = c - 1 < 0 ? 0 : c - 1, hi = c + 1 > K - 1 ? K - 1 : c + 1;
  long best = lo;
  double bd = std::fabs(p - (double)lo / km1);
  for (long k = lo + 1; k <= hi; ++k) {
    const double d = std::fabs(p - (double)k / km1);
    if (d < bd) { bd = d; best = k; }
  }
  return (int)best;
}

// jstart1[i][k] = first illumination bin j with index_1(i, j) >= k (index_1 grows with j).
void build_jstart1(int K, double gamma, uint16_t* t, int M) {
  const bool binned = M > K;
  const double km1 = (double)(K - 1);
  const double ig = 1.0 / gamma;
  auto hl = [&](int j) { return std::pow(binned ? bin_location(j, K, M) : (double)j / km1, ig); };
  for (int i = 0; i < K; ++i) {
    const double hr = binned ? bin_location(i, K, M) : (double)i / km1;
    uint16_t* row = t + (size_t)i * (K + 1);
    int k = 0;
    for (int j = 0; j < K; ++j) {
      const int c = binned ? nearest_bin(hl(j) * hr, K, M) : index1(K, hl(j), hr);
      while (k <= c) row[k++] = (uint16_t)j;
    }
    while (k <= K) row[k++] = (uint16_t)K;
  }
}


static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

SlotLayout make_layout(int K) {
  SlotLayout L{};
  size_t o = 0;
  L.S = o; o += (size_t)K * 4;
  L.G = o; o += (size_t)K * 4;
  o = align256(o);
  L.R = o; o += (size_t)K * 8;
  L.L = o; o += (size_t)K * 8;
  L.T = o; o += (size_t)K * 8;
  L.lut = o; o += (size_t)K * 2;
  o = align256(o);
  L.misc = o; o += 16 + (size_t)kProfSlots * 8;
  o = align256(o);
  L.vec = o; o += (K > 1024) ? (size_t)kSolveVecs * K * 8 : 0;
  o = align256(o);
  L.cls = o; o += (size_t)4 * K * 4;
  o = align256(o);
  L.list = o; o += (size_t)K * (K + 1) * 4;  // class-major cell lists; later the Eq. 19 row segments
  o = align256(o);
  L.max_pieces = (size_t)K * K / kPiece + K;
  L.piece = o; o += L.max_pieces * 8;
  o = align256(o);
  size_t mp = L.max_pieces;
  const size_t dense = (size_t)K * ((K + kPiece - 1) / kPiece);
  if (dense > mp) mp = dense;
  if (mp < (size_t)kSolveThreads) mp = kSolveThreads;
  L.max_parts = mp;
  L.part = o; o += mp * 8;
  L.bytes = align256(o);
  return L;
}

}  // namespace hr

namespace {

hr_status cuda_fail(cudaError_t e) {
  // a failed runtime call also leaves its error as the thread's last error; a non-sticky one (an
  // allocation failure) is cleared so that it is not reported again by a later, unrelated check
  if (e != cudaSuccess) cudaGetLastError();
  if (e == cudaErrorMemoryAllocation) return HR_ERR_OOM;
  return e == cudaSuccess ? HR_OK : HR_ERR_CUDA;
}

#define HR_CUDA(x)                                 \
  do {                                             \
    cudaError_t e_ = (x);                          \
    if (e_ != cudaSuccess) return cuda_fail(e_);   \
  } while (0)

void drop_graph(hr_ctx* c) {  // a captured pipeline holds workspace and descriptor pointers
  if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
}

hr_status ensure_slots(hr_ctx* c, int n) {
  if (n <= c->n_slots) return HR_OK;
  drop_graph(c);
  if (c->d_slots) { cudaFree(c->d_slots); c->d_slots = nullptr; c->n_slots = 0; }
  c->hist_clean = 0;
  HR_CUDA(cudaMalloc(&c->d_slots, c->lay.bytes * (size_t)n));
  c->n_slots = n;
  return HR_OK;
}

hr_status ensure_desc(hr_ctx* c, int n) {
  if (n <= c->cap_imgs) return HR_OK;
  drop_graph(c);
  if (c->desc_done) HR_CUDA(cudaEventSynchronize(c->desc_done));
  cudaFree(c->d_imgs); cudaFree(c->d_tile_start); cudaFreeHost(c->h_imgs); cudaFreeHost(c->h_tile_start);
  c->d_imgs = nullptr; c->d_tile_start = nullptr; c->h_imgs = nullptr; c->h_tile_start = nullptr; c->cap_imgs = 0;
  c->last_imgs.clear();
  HR_CUDA(cudaMalloc(&c->d_imgs, sizeof(ImageDesc) * (size_t)n));
  // per group of images (at most two): tile starts, strip starts, then the solve's image order
  HR_CUDA(cudaMalloc(&c->d_tile_start, sizeof(int) * 3 * (size_t)(n + 2)));
  HR_CUDA(cudaMallocHost(&c->h_imgs, sizeof(ImageDesc) * (size_t)n));
  HR_CUDA(cudaMallocHost(&c->h_tile_start, sizeof(int) * 3 * (size_t)(n + 2)));
  c->cap_imgs = n;
  return HR_OK;
}

bool same_desc(const std::vector<ImageDesc>& a, const ImageDesc* b, int n) {
  if ((int)a.size() != n) return false;
  for (int i = 0; i < n; ++i)
    if (a[i].in != b[i].in || a[i].out != b[i].out || a[i].W != b[i].W || a[i].H != b[i].H ||
        a[i].in_pitch != b[i].in_pitch || a[i].out_pitch != b[i].out_pitch)
      return false;
  return true;
}

// Adds the stage times of ring entry i to the sums (waits for its last event).
hr_status fold_timing(hr_ctx* c, int i) {
  if (!c->ev_used[i]) return HR_OK;
  HR_CUDA(cudaEventSynchronize(c->ev[i][3]));
  for (int s = 0; s < 3; ++s) {
    float ms = 0.f;
    HR_CUDA(cudaEventElapsedTime(&ms, c->ev[i][s], c->ev[i][s + 1]));
    c->stage_ms[s] += ms;
  }
  c->stage_calls += 1;
  c->ev_used[i] = false;
  return HR_OK;
}

// The images one enqueue_stages call runs: their table, work totals, first slot and solve order.
struct Group {
  ImgTab tab;
  int total, units, interior;
  uint8_t* slots;
  const int* order;  // (nullptr for one image)
};

// Arguments of the solve kernel for the images of group g.
hr::SolveArgs solve_args(const hr_ctx* c, const Group& g) {
  const bool debug = (c->p.flags & HR_FLAG_DEBUG_OUT) != 0;
  hr::SolveArgs a{};
  a.K = c->p.K;
  a.alpha = c->p.alpha;
  a.beta = c->p.beta;
  a.eps = c->p.eps;
  a.max_iter = c->p.max_iter;
  a.fixed_iters = (c->p.flags & HR_FLAG_FIXED_ITERS) ? 1 : 0;
  a.jstart1 = c->d_jstart1;
  a.slots = g.slots;
  a.order = g.order;
  a.slot_bytes = c->lay.bytes;
  a.lay = c->lay;
  a.status = c->d_status;
  a.profile = debug ? 1 : 0;
  a.zero_hist = debug ? 0 : 1;
  a.printed = (c->p.flags & HR_FLAG_PRINTED_UPDATE) ? 1 : 0;
  a.nearest = (c->p.flags & HR_FLAG_NEAREST_MATCH) ? 1 : 0;
  a.cmap = c->d_cmap;
  a.jstart0 = c->d_jstart0;
  a.arith = c->p.precision == HR_PREC_FP32 ? hr::kArithF32 : (c->p.precision == HR_PREC_DF64 ? hr::kArithDF64 : hr::kArithF64);
  return a;
}

// CTAs per image of the solve: the tuned cluster for one image; for a batch as many as keep all
// images in one wave (the largest power of two with n C <= SMs, at most the tuned cluster), so a
// batch of a few images runs as fast as its images would alone and a large one on one CTA each.
int solve_ctas(const hr_ctx* c, int n, bool batched) {
  int C = c->tune.solve_cluster;
  if (batched) {
    const int per = c->sm_count / n;
    int p2 = 1;
    while (2 * p2 <= per) p2 *= 2;
    C = p2 < C ? p2 : C;
  }
  return C;
}

// The pipeline's device work for one group on one stream: zero the histograms (unless the previous
// solves left them zero), histogram pass, solve, apply.  ev (optional): four events recorded around
// the three stages; after_hist (optional): recorded after the histogram pass.
cudaError_t enqueue_stages(hr_ctx* c, const Group& g, int elem_bytes, bool fast_in, bool fast_out, bool batched,
                           bool zero, cudaStream_t st, cudaEvent_t* ev, int* launches,
                           cudaEvent_t after_hist = nullptr) {
  const int K = c->p.K, n = g.tab.n;
  const int pdl = c->tune.pdl;  // bit 0: histogram pass, bit 1: solve, bit 2: apply pass
  cudaError_t e;
  // zero H_C(S) and H_C(grad S) of every slot used (S and G are adjacent at the slot start)
  if (zero) {
    e = cudaMemset2DAsync(g.slots + c->lay.S, c->lay.bytes, 0, (size_t)2 * K * sizeof(unsigned), (size_t)n, st);
    if (e != cudaSuccess) return e;
  }
  if (ev && (e = cudaEventRecord(ev[0], st)) != cudaSuccess) return e;
  e = hr::launch_hist(g.tab, g.total, g.units, g.interior, elem_bytes, K, g.slots, c->lay.bytes, c->lay, c->d_status,
                      c->sm_count, c->tune.hist_ctas_per_sm, st, fast_in, (pdl & 1) != 0,
                      (c->p.flags & HR_FLAG_FORWARD_GRADIENT) != 0, c->M);
  if (e != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[1], st)) != cudaSuccess) return e;
  if (after_hist && (e = cudaEventRecord(after_hist, st)) != cudaSuccess) return e;
  const hr::SolveArgs a = solve_args(c, g);
  *launches += 3;
  e = hr::launch_solve(a, n, solve_ctas(c, n, batched), st, (pdl & 2) != 0);
  if (e != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[2], st)) != cudaSuccess) return e;
  e = hr::launch_apply(g.tab, g.total, elem_bytes, K, g.slots, c->lay.bytes, c->lay, c->d_status, c->sm_count,
                       c->tune.apply_ctas_per_sm, st, fast_out, (pdl & 4) != 0, c->M);
  if (e != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev[3], st)) != cudaSuccess) return e;
  return cudaSuccess;
}

// Slots [0, n) after a call that enqueued its stages (ok) or failed to: the solve clears the
// histograms it used unless debug intermediates are kept.
void note_hist_state(hr_ctx* c, int n, bool ok) {
  if (!ok || (c->p.flags & HR_FLAG_DEBUG_OUT)) c->hist_clean = 0;
  else if (n > c->hist_clean) c->hist_clean = n;
}

// Single-image calls take the slots of a ring in turn.  A call first makes its stream wait until
// the slot's previous call (on whatever stream) is done, and marks the slot's release on its own
// stream after its last kernel, so calls on different streams may overlap on the device.
hr_status ring_alloc(hr_ctx* c) {
  if (c->d_ring) return HR_OK;
  const int n = c->lay.bytes <= ((size_t)16 << 20) ? hr_ctx::kRingMax : 4;
  HR_CUDA(cudaMalloc(&c->d_ring, c->lay.bytes * (size_t)n));
  for (int i = 0; i < n; ++i) {
    c->ring_clean[i] = false;
    c->ring_pending[i] = false;
    if (!c->ring_free[i]) HR_CUDA(cudaEventCreateWithFlags(&c->ring_free[i], cudaEventDisableTiming));
  }
  c->ring_n = n;
  c->ring_next = 0;
  return HR_OK;
}

hr_status ring_acquire(hr_ctx* c, cudaStream_t st, int* r) {
  const hr_status s = ring_alloc(c);
  if (s != HR_OK) return s;
  *r = c->ring_next;
  c->ring_next = (*r + 1) % c->ring_n;
  if (c->ring_pending[*r]) HR_CUDA(cudaStreamWaitEvent(st, c->ring_free[*r], 0));
  return HR_OK;
}

hr_status ring_release(hr_ctx* c, cudaStream_t st, int r) {
  HR_CUDA(cudaEventRecord(c->ring_free[r], st));
  c->ring_pending[r] = true;
  return HR_OK;
}

bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) { cudaGetLastError(); return true; }
  return cap != cudaStreamCaptureStatusNone;
}

// One image on the caller's stream in a ring slot (unpartitioned).
hr_status run_ring(hr_ctx* c, const ImageDesc& d, int elem_bytes, bool fast_in, bool fast_out, cudaStream_t st,
                   cudaEvent_t* ev) {
  int r = 0;
  hr_status s = ring_acquire(c, st, &r);
  if (s != HR_OK) return s;
  const bool debug = (c->p.flags & HR_FLAG_DEBUG_OUT) != 0;
  Group g{};
  g.tab.n = 1;
  g.tab.one = d;
  g.total = hr::tiles_of(d.W, d.H);
  g.units = hr::strips_of(d.W, d.H);
  g.interior = hr::interior_strips_of(d.W, d.H);
  g.slots = c->d_ring + (size_t)r * c->lay.bytes;
  g.order = nullptr;
  int nl = 0;
  const cudaError_t e = enqueue_stages(c, g, elem_bytes, fast_in, fast_out, false, debug || !c->ring_clean[r], st, ev, &nl);
  c->ring_clean[r] = e == cudaSuccess && !debug;
  if (e != cudaSuccess) return cuda_fail(e);
  s = ring_release(c, st, r);
  if (s != HR_OK) return s;
  c->launches += (uint64_t)nl;
  c->last_n = 1;
  c->last_base = g.slots;
  return HR_OK;
}

// One image on the SM partitions (sets *done); returns with *done false where the call runs
// unpartitioned instead: under stream capture, or when the device's SMs cannot be split.
hr_status run_partitioned(hr_ctx* c, const ImageDesc& d, int elem_bytes, bool fast_in, bool fast_out,
                          cudaStream_t st, bool* done) {
  *done = false;
  if (c->part_unavailable) return HR_OK;
  // solves of partition_cluster CTAs, 16 / partition_cluster of them at once in each 16-SM partition
  const int sper = 16 / c->tune.partition_cluster;
  if (c->part && (c->part_parts != c->tune.partitions || c->part_sper != sper)) {
    hr::partitions_destroy(c->part);  // (synchronises the partitions' streams)
    c->part = nullptr;
  }
  if (!c->part) {
    hr_status ps = ring_alloc(c);
    if (ps != HR_OK) return ps;
    ps = hr::partitions_create(c->device, c->tune.partitions, sper, c->ring_n, &c->part);
    if (ps == HR_ERR_UNSUPPORTED) { c->part_unavailable = true; return HR_OK; }
    if (ps != HR_OK) return ps;
    c->part_parts = c->tune.partitions;
    c->part_sper = sper;
  }
  int r = 0;
  hr_status rs = ring_acquire(c, st, &r);
  if (rs != HR_OK) return rs;
  const int K = c->p.K;
  const bool debug = (c->p.flags & HR_FLAG_DEBUG_OUT) != 0;
  const bool zero = debug || !c->ring_clean[r];
  const int sms = hr::partitions_pixel_sms(c->part);
  Group g{};
  g.tab.n = 1;
  g.tab.one = d;
  g.total = hr::tiles_of(d.W, d.H);
  g.units = hr::strips_of(d.W, d.H);
  g.interior = hr::interior_strips_of(d.W, d.H);
  g.slots = c->d_ring + (size_t)r * c->lay.bytes;
  g.order = nullptr;
  const hr::SolveArgs a = solve_args(c, g);
  const bool forward = (c->p.flags & HR_FLAG_FORWARD_GRADIENT) != 0;
  // (no programmatic dependent launches: each pixel pass follows an event wait on its stream)
  auto hist = [&](cudaStream_t s) {
    if (zero) {
      const cudaError_t e = cudaMemsetAsync(g.slots + c->lay.S, 0, (size_t)2 * K * sizeof(unsigned), s);
      if (e != cudaSuccess) return e;
    }
    return hr::launch_hist(g.tab, g.total, g.units, g.interior, elem_bytes, K, g.slots, c->lay.bytes, c->lay,
                           c->d_status, sms, c->tune.hist_ctas_per_sm, s, fast_in, false, forward, c->M);
  };
  auto solve = [&](cudaStream_t s) { return hr::launch_solve(a, 1, c->tune.partition_cluster, s, false); };
  auto apply = [&](cudaStream_t s) {
    return hr::launch_apply(g.tab, g.total, elem_bytes, K, g.slots, c->lay.bytes, c->lay, c->d_status, sms,
                            c->tune.apply_ctas_per_sm, s, fast_out, false, c->M);
  };
  const cudaError_t e = hr::partitions_run(c->part, r, st, hist, solve, apply);
  c->ring_clean[r] = e == cudaSuccess && !debug;
  if (e != cudaSuccess) return cuda_fail(e);
  rs = ring_release(c, st, r);
  if (rs != HR_OK) return rs;
  *done = true;
  c->launches += 3;
  c->last_n = 1;
  c->last_base = g.slots;
  return HR_OK;
}

hr_status run_pipeline(hr_ctx* c, int n, const ImageDesc* imgs, int elem_bytes, cudaStream_t st, bool batched) {
  const int K = c->p.K;
  if (elem_bytes != 1 && elem_bytes != 2) return HR_ERR_INVALID_ARG;
  if (elem_bytes == 1 && (K > 256 || c->M > 256)) return HR_ERR_INVALID_ARG;
  long long total = 0, units = 0;
  for (int i = 0; i < n; ++i) {
    const ImageDesc& d = imgs[i];
    if (!d.in || !d.out || d.W < 1 || d.H < 1) return HR_ERR_INVALID_ARG;
    if ((long long)d.in_pitch < 3LL * d.W * elem_bytes || (long long)d.out_pitch < 3LL * d.W * elem_bytes)
      return HR_ERR_INVALID_ARG;
    if ((long long)d.W * d.H >= (1LL << 31)) return HR_ERR_UNSUPPORTED;
    total += hr::tiles_of(d.W, d.H);
    units += hr::strips_of(d.W, d.H);
  }
  if (total >= (1LL << 31) || units >= (1LL << 31)) return HR_ERR_UNSUPPORTED;
  // 8-bit fast paths need every row 16-byte aligned (input for the histogram pass, both for apply)
  bool fast_in = elem_bytes == 1 && K <= 256, fast_out = fast_in;
  for (int i = 0; i < n; ++i) {
    const ImageDesc& d = imgs[i];
    const bool ain = ((uintptr_t)d.in % 16 == 0) && (d.in_pitch % 16 == 0);
    const bool aout = ((uintptr_t)d.out % 16 == 0) && (d.out_pitch % 16 == 0);
    fast_in = fast_in && ain;
    fast_out = fast_out && ain && aout;
  }
  const bool debug = (c->p.flags & HR_FLAG_DEBUG_OUT) != 0;
  const bool timing = (c->p.flags & HR_FLAG_STAGE_TIMING) != 0;
  // single images: the ring of slots (on the SM partitions unless timing or disabled), except under
  // stream capture, where a call keeps to batch slot 0 and orders nothing across streams
  const bool ring = n == 1 && !batched && !capturing(st);
  if (ring && !timing && c->tune.partitions > 0) {
    bool partitioned = false;
    hr_status ps = run_partitioned(c, imgs[0], elem_bytes, fast_in, fast_out, st, &partitioned);
    if (partitioned || ps != HR_OK) return ps;
  }
  hr_status s = ensure_slots(c, n);
  if (s != HR_OK) return s;
  const bool graph = batched && c->tune.use_graph && n > 1 && !timing;
  // A large graph-replayed batch may run as two groups (images [0, n/2) and [n/2, n)) on two
  // streams, the second group's histogram pass after the first's, so that one group's solve
  // overlaps the other's pixel passes.
  const int G = (graph && c->tune.groups == 2 && n >= 64) ? 2 : 1;
  int g0[2] = {0, G == 2 ? n / 2 : n}, gn[2] = {G == 2 ? n / 2 : n, G == 2 ? n - n / 2 : 0};
  Group grp[2] = {};
  for (int g = 0; g < G; ++g) {
    Group& q = grp[g];
    q.tab.n = gn[g];
    q.slots = c->d_slots + (size_t)g0[g] * c->lay.bytes;
    for (int i = g0[g]; i < g0[g] + gn[g]; ++i) {
      q.total += hr::tiles_of(imgs[i].W, imgs[i].H);
      q.units += hr::strips_of(imgs[i].W, imgs[i].H);
      q.interior += hr::interior_strips_of(imgs[i].W, imgs[i].H);
    }
    if (gn[g] == 1) q.tab.one = imgs[g0[g]];  // travels in the kernel parameters: nothing to upload
  }
  if (n > 1) {
    s = ensure_desc(c, n);
    if (s != HR_OK) return s;
    if (!same_desc(c->last_imgs, imgs, n) || c->last_groups != G) {
      HR_CUDA(cudaEventSynchronize(c->desc_done));  // the previous upload has left the staging buffer
      for (int i = 0; i < n; ++i) c->h_imgs[i] = imgs[i];
      for (int g = 0; g < G; ++g) {
        const int m = gn[g], off = 3 * (g0[g] + g);
        int* tiles = c->h_tile_start + off;
        int* strips = tiles + m + 1;
        int* order = tiles + 2 * (m + 1);
        int t = 0, u = 0;
        for (int i = 0; i < m; ++i) {
          tiles[i] = t;
          strips[i] = u;
          t += hr::tiles_of(imgs[g0[g] + i].W, imgs[g0[g] + i].H);
          u += hr::strips_of(imgs[g0[g] + i].W, imgs[g0[g] + i].H);
        }
        tiles[m] = t;
        strips[m] = u;
        // the solve's CTAs take the group's images largest first (longest solves first: the last
        // wave holds the shortest ones)
        for (int i = 0; i < m; ++i) order[i] = i;
        std::stable_sort(order, order + m, [&](int x, int y) {
          const ImageDesc &dx = imgs[g0[g] + x], &dy = imgs[g0[g] + y];
          return (long long)dx.W * dx.H > (long long)dy.W * dy.H;
        });
      }
      HR_CUDA(cudaMemcpyAsync(c->d_imgs, c->h_imgs, sizeof(ImageDesc) * (size_t)n, cudaMemcpyHostToDevice, st));
      HR_CUDA(cudaMemcpyAsync(c->d_tile_start, c->h_tile_start, sizeof(int) * 3 * (size_t)(n + G),
                              cudaMemcpyHostToDevice, st));
      HR_CUDA(cudaEventRecord(c->desc_done, st));
      c->last_imgs.assign(imgs, imgs + n);
      c->last_groups = G;
    }
    for (int g = 0; g < G; ++g) {  // each group's tables: tile starts, strip starts, solve order
      if (gn[g] == 1) continue;
      const int off = 3 * (g0[g] + g);
      grp[g].tab.imgs = c->d_imgs + g0[g];
      grp[g].tab.tiles = c->d_tile_start + off;
      grp[g].tab.units = grp[g].tab.tiles + gn[g] + 1;
      grp[g].order = grp[g].tab.tiles + 2 * (gn[g] + 1);
    }
  }
  if (graph) {
    // a replayed graph cannot see whether the histograms are zero: without debug intermediates it
    // relies on the solves clearing them (cleared here first if need be), with them it zeroes
    if (!debug && c->hist_clean < n) {
      cudaError_t e = cudaMemset2DAsync(c->d_slots + c->lay.S, c->lay.bytes, 0, (size_t)2 * c->p.K * sizeof(unsigned),
                                        (size_t)n, st);
      if (e != cudaSuccess) { note_hist_state(c, n, false); return cuda_fail(e); }
      c->hist_clean = n;
    }
    const bool same = c->graph && c->g_n == n && c->g_total == (int)total && c->g_eb == elem_bytes &&
                      c->g_fast_in == (int)fast_in && c->g_fast_out == (int)fast_out && c->g_zero == (int)debug &&
                      c->g_groups == G && std::memcmp(&c->g_tune, &c->tune, sizeof(hr_tuning)) == 0;
    if (!same) {
      drop_graph(c);
      cudaStream_t cap = nullptr, cap2 = nullptr;
      cudaEvent_t fork = nullptr, hist_done = nullptr, join = nullptr;
      HR_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
      cudaError_t e = cudaSuccess;
      if (G == 2) {
        e = cudaStreamCreateWithFlags(&cap2, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&hist_done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
      }
      cudaGraph_t gr = nullptr;
      int nl = 0;  // kernels per replay
      if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        if (G == 2) {
          e = cudaEventRecord(fork, cap);
          if (e == cudaSuccess) e = cudaStreamWaitEvent(cap2, fork, 0);
        }
        if (e == cudaSuccess)
          e = enqueue_stages(c, grp[0], elem_bytes, fast_in, fast_out, batched, debug, cap, nullptr, &nl, hist_done);
        if (G == 2) {
          if (e == cudaSuccess) e = cudaStreamWaitEvent(cap2, hist_done, 0);
          if (e == cudaSuccess)
            e = enqueue_stages(c, grp[1], elem_bytes, fast_in, fast_out, batched, debug, cap2, nullptr, &nl);
          if (e == cudaSuccess) e = cudaEventRecord(join, cap2);
          if (e == cudaSuccess) e = cudaStreamWaitEvent(cap, join, 0);
        }
        cudaError_t e2 = cudaStreamEndCapture(cap, &gr);
        if (e == cudaSuccess) e = e2;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph, gr, 0);
      if (gr) cudaGraphDestroy(gr);
      if (join) cudaEventDestroy(join);
      if (hist_done) cudaEventDestroy(hist_done);
      if (fork) cudaEventDestroy(fork);
      if (cap2) cudaStreamDestroy(cap2);
      cudaStreamDestroy(cap);
      if (e != cudaSuccess) { c->graph = nullptr; return cuda_fail(e); }
      c->g_n = n; c->g_total = (int)total; c->g_eb = elem_bytes; c->g_groups = G; c->g_launches = nl;
      c->g_fast_in = (int)fast_in; c->g_fast_out = (int)fast_out; c->g_zero = (int)debug; c->g_tune = c->tune;
    }
    const cudaError_t e = cudaGraphLaunch(c->graph, st);
    note_hist_state(c, n, e == cudaSuccess);
    if (e != cudaSuccess) return cuda_fail(e);
    c->launches += (uint64_t)c->g_launches;
    c->last_n = n;
    c->last_base = c->d_slots;
    return HR_OK;
  }
  cudaEvent_t* ev = nullptr;
  if (timing) {
    const int i = c->ev_next;
    c->ev_next = (i + 1) % hr_ctx::kRing;
    hr_status fs = fold_timing(c, i);
    if (fs != HR_OK) return fs;
    if (!c->ev[i][0])
      for (int q = 0; q < 4; ++q) HR_CUDA(cudaEventCreate(&c->ev[i][q]));
    ev = c->ev[i];
    c->ev_used[i] = true;
  }
  if (ring) return run_ring(c, imgs[0], elem_bytes, fast_in, fast_out, st, ev);
  const bool zero = debug || c->hist_clean < n;
  int nl = 0;
  const cudaError_t e = enqueue_stages(c, grp[0], elem_bytes, fast_in, fast_out, batched, zero, st, ev, &nl);
  note_hist_state(c, n, e == cudaSuccess);
  if (e != cudaSuccess) return cuda_fail(e);
  c->launches += (uint64_t)nl;
  c->last_n = n;
  c->last_base = c->d_slots;
  return HR_OK;
}

// Host-device copy of `height` rows: one flat copy when both sides are contiguous (flat copies in
// the two directions overlap on GB300; pitched ones measured no overlap), else a pitched copy.
cudaError_t copy_rows(void* dst, size_t dpitch, const void* src, size_t spitch, size_t row, size_t height,
                      cudaMemcpyKind kind, cudaStream_t st) {
  if (dpitch == row && spitch == row) return cudaMemcpyAsync(dst, src, row * height, kind, st);
  return cudaMemcpy2DAsync(dst, dpitch, src, spitch, row, height, kind, st);
}

}  // namespace

extern "C" {

void histretinex_default_params(hr_params* p) {
  if (!p) return;
  p->K = 256;
  p->alpha = 1e-3;
  p->beta = 1e-3;
  p->gamma = 2.2;
  p->eps = 0.0;
  p->max_iter = 10;
  p->precision = HR_PREC_FP64;
  p->flags = HR_FLAG_FIXED_ITERS;
  p->levels = 0;
}

hr_status histretinex_create(hr_ctx** out, const hr_params* p, int device) {
  if (!out) return HR_ERR_INVALID_ARG;
  *out = nullptr;
  hr_status s = hr::check_params(p);
  if (s != HR_OK) return s;
  int ndev = 0;
  HR_CUDA(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return HR_ERR_INVALID_ARG;
  HR_CUDA(cudaSetDevice(device));
  hr_ctx* c = new (std::nothrow) hr_ctx();
  if (!c) return HR_ERR_OOM;
  c->device = device;
  c->p = *p;
  c->lay = hr::make_layout(p->K);
  c->M = p->levels > 0 ? p->levels : p->K;
  cudaError_t e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  std::vector<uint16_t> js((size_t)p->K * (p->K + 1));
  hr::build_jstart1(p->K, p->gamma, js.data(), c->M);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_jstart1, js.size() * sizeof(uint16_t));
  if (e == cudaSuccess) e = cudaMemcpy(c->d_jstart1, js.data(), js.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && c->M != p->K) {  // binned data: the class map of Eq. 10 as tables
    std::vector<uint16_t> cm((size_t)p->K * p->K), j0((size_t)p->K * (p->K + 1));
    hr::build_class_tables(p->K, c->M, cm.data(), j0.data());
    e = cudaMalloc(&c->d_cmap, cm.size() * sizeof(uint16_t));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_jstart0, j0.size() * sizeof(uint16_t));
    if (e == cudaSuccess) e = cudaMemcpy(c->d_cmap, cm.data(), cm.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_jstart0, j0.data(), j0.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMalloc(&c->d_status, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->desc_done, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    histretinex_destroy(c);
    return cuda_fail(e);
  }
  *out = c;
  return HR_OK;
}

hr_status histretinex_enhance(hr_ctx* c, const void* d_in, void* d_out, int width, int height, size_t in_pitch,
                              size_t out_pitch, int elem_bytes, void* stream) {
  if (!c) return HR_ERR_INVALID_ARG;
  ImageDesc d{static_cast<const uint8_t*>(d_in), static_cast<uint8_t*>(d_out), width, height, (long long)in_pitch,
              (long long)out_pitch};
  HR_CUDA(cudaSetDevice(c->device));
  return run_pipeline(c, 1, &d, elem_bytes, static_cast<cudaStream_t>(stream), false);
}

hr_status histretinex_enhance_batch(hr_ctx* c, int n, const void* const* d_in, void* const* d_out, const int* width,
                                    const int* height, const size_t* in_pitch, const size_t* out_pitch,
                                    int elem_bytes, void* stream) {
  if (!c || n < 1 || !d_in || !d_out || !width || !height || !in_pitch || !out_pitch) return HR_ERR_INVALID_ARG;
  std::vector<ImageDesc> v((size_t)n);
  for (int i = 0; i < n; ++i)
    v[i] = ImageDesc{static_cast<const uint8_t*>(d_in[i]), static_cast<uint8_t*>(d_out[i]), width[i], height[i],
                     (long long)in_pitch[i], (long long)out_pitch[i]};
  HR_CUDA(cudaSetDevice(c->device));
  return run_pipeline(c, n, v.data(), elem_bytes, static_cast<cudaStream_t>(stream), true);
}

hr_status histretinex_enhance_host(hr_ctx* c, const void* h_in, void* h_out, int width, int height, size_t in_pitch,
                                   size_t out_pitch, int elem_bytes, void* stream) {
  if (!c || !h_in || !h_out || width < 1 || height < 1 || (elem_bytes != 1 && elem_bytes != 2))
    return HR_ERR_INVALID_ARG;
  const size_t row = (size_t)3 * width * elem_bytes;
  if (in_pitch < row || out_pitch < row) return HR_ERR_INVALID_ARG;
  const size_t dpitch = (row + 15) / 16 * 16;  // 16-byte aligned device rows: the fast pixel paths
  const size_t bytes = dpitch * (size_t)height;
  HR_CUDA(cudaSetDevice(c->device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (bytes > c->io_bytes) {
    HR_CUDA(cudaStreamSynchronize(st));
    cudaFree(c->d_io_in); cudaFree(c->d_io_out);
    c->d_io_in = c->d_io_out = nullptr; c->io_bytes = 0;
    HR_CUDA(cudaMalloc(&c->d_io_in, bytes));
    HR_CUDA(cudaMalloc(&c->d_io_out, bytes));
    c->io_bytes = bytes;
  }
  HR_CUDA(copy_rows(c->d_io_in, dpitch, h_in, in_pitch, row, (size_t)height, cudaMemcpyHostToDevice, st));
  ImageDesc d{static_cast<const uint8_t*>(c->d_io_in), static_cast<uint8_t*>(c->d_io_out), width, height,
              (long long)dpitch, (long long)dpitch};
  hr_status s = run_pipeline(c, 1, &d, elem_bytes, st, false);
  if (s != HR_OK) return s;
  HR_CUDA(copy_rows(h_out, out_pitch, c->d_io_out, dpitch, row, (size_t)height, cudaMemcpyDeviceToHost, st));
  return histretinex_sync_status(c, stream);
}

hr_status histretinex_enhance_host_many(hr_ctx* c, int n, const void* const* h_in, void* const* h_out,
                                        const int* width, const int* height, const size_t* in_pitch,
                                        const size_t* out_pitch, int elem_bytes, void* stream) {
  if (!c || n < 1 || !h_in || !h_out || !width || !height || !in_pitch || !out_pitch ||
      (elem_bytes != 1 && elem_bytes != 2))
    return HR_ERR_INVALID_ARG;
  size_t need = 0;
  for (int i = 0; i < n; ++i) {
    if (!h_in[i] || !h_out[i] || width[i] < 1 || height[i] < 1) return HR_ERR_INVALID_ARG;
    const size_t row = (size_t)3 * width[i] * elem_bytes;
    if (in_pitch[i] < row || out_pitch[i] < row) return HR_ERR_INVALID_ARG;
    need = std::max(need, (row + 15) / 16 * 16 * (size_t)height[i]);
  }
  HR_CUDA(cudaSetDevice(c->device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!c->s_h2d) {
    HR_CUDA(cudaStreamCreateWithFlags(&c->s_h2d, cudaStreamNonBlocking));
    HR_CUDA(cudaStreamCreateWithFlags(&c->s_d2h, cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b) {
      HR_CUDA(cudaEventCreateWithFlags(&c->ev_in_ready[b], cudaEventDisableTiming));
      HR_CUDA(cudaEventCreateWithFlags(&c->ev_in_free[b], cudaEventDisableTiming));
      HR_CUDA(cudaEventCreateWithFlags(&c->ev_done[b], cudaEventDisableTiming));
      HR_CUDA(cudaEventCreateWithFlags(&c->ev_out_free[b], cudaEventDisableTiming));
    }
  }
  if (need > c->pp_bytes) {
    HR_CUDA(cudaDeviceSynchronize());
    for (int b = 0; b < 2; ++b) {
      cudaFree(c->d_pp_in[b]); cudaFree(c->d_pp_out[b]);
      c->d_pp_in[b] = c->d_pp_out[b] = nullptr;
    }
    c->pp_bytes = 0;
    for (int b = 0; b < 2; ++b) {
      HR_CUDA(cudaMalloc(&c->d_pp_in[b], need));
      HR_CUDA(cudaMalloc(&c->d_pp_out[b], need));
    }
    c->pp_bytes = need;
  }
  // everything before this call on the caller's stream comes first
  HR_CUDA(cudaEventRecord(c->ev_done[0], st));
  HR_CUDA(cudaStreamWaitEvent(c->s_h2d, c->ev_done[0], 0));
  HR_CUDA(cudaStreamWaitEvent(c->s_d2h, c->ev_done[0], 0));
  for (int i = 0; i < n; ++i) {
    const int b = i & 1;
    const size_t row = (size_t)3 * width[i] * elem_bytes, dpitch = (row + 15) / 16 * 16;
    // H2D of image i once the pipeline of image i - 2 has left buffer b
    if (i >= 2) HR_CUDA(cudaStreamWaitEvent(c->s_h2d, c->ev_in_free[b], 0));
    HR_CUDA(copy_rows(c->d_pp_in[b], dpitch, h_in[i], in_pitch[i], row, (size_t)height[i], cudaMemcpyHostToDevice,
                      c->s_h2d));
    HR_CUDA(cudaEventRecord(c->ev_in_ready[b], c->s_h2d));
    // the plain pipeline on the caller's stream, once the input is in and the D2H of image i - 2
    // has left output buffer b
    HR_CUDA(cudaStreamWaitEvent(st, c->ev_in_ready[b], 0));
    if (i >= 2) HR_CUDA(cudaStreamWaitEvent(st, c->ev_out_free[b], 0));
    ImageDesc d{static_cast<const uint8_t*>(c->d_pp_in[b]), static_cast<uint8_t*>(c->d_pp_out[b]), width[i],
                height[i], (long long)dpitch, (long long)dpitch};
    hr_status s = run_pipeline(c, 1, &d, elem_bytes, st, false);
    if (s != HR_OK) { cudaStreamSynchronize(c->s_h2d); cudaStreamSynchronize(c->s_d2h); return s; }
    HR_CUDA(cudaEventRecord(c->ev_in_free[b], st));
    HR_CUDA(cudaEventRecord(c->ev_done[b], st));
    // D2H of image i
    HR_CUDA(cudaStreamWaitEvent(c->s_d2h, c->ev_done[b], 0));
    HR_CUDA(copy_rows(h_out[i], out_pitch[i], c->d_pp_out[b], dpitch, row, (size_t)height[i],
                      cudaMemcpyDeviceToHost, c->s_d2h));
    HR_CUDA(cudaEventRecord(c->ev_out_free[b], c->s_d2h));
  }
  HR_CUDA(cudaStreamSynchronize(c->s_h2d));
  HR_CUDA(cudaStreamSynchronize(c->s_d2h));
  return histretinex_sync_status(c, stream);
}

hr_status histretinex_get_debug(hr_ctx* c, int image, uint64_t* S, uint64_t* G, double* R, double* L, double* T,
                                uint16_t* lut, int* iters) {
  if (!c || image < 0 || image >= c->last_n) return HR_ERR_INVALID_ARG;
  if (!(c->p.flags & HR_FLAG_DEBUG_OUT)) return HR_ERR_INVALID_ARG;
  HR_CUDA(cudaSetDevice(c->device));
  HR_CUDA(cudaDeviceSynchronize());
  const int K = c->p.K;
  const uint8_t* slot = c->last_base + (size_t)image * c->lay.bytes;
  std::vector<unsigned> tmp((size_t)K);
  if (S) {
    HR_CUDA(cudaMemcpy(tmp.data(), slot + c->lay.S, (size_t)K * 4, cudaMemcpyDeviceToHost));
    for (int k = 0; k < K; ++k) S[k] = tmp[k];
  }
  if (G) {
    HR_CUDA(cudaMemcpy(tmp.data(), slot + c->lay.G, (size_t)K * 4, cudaMemcpyDeviceToHost));
    for (int k = 0; k < K; ++k) G[k] = tmp[k];
  }
  if (R) HR_CUDA(cudaMemcpy(R, slot + c->lay.R, (size_t)K * 8, cudaMemcpyDeviceToHost));
  if (L) HR_CUDA(cudaMemcpy(L, slot + c->lay.L, (size_t)K * 8, cudaMemcpyDeviceToHost));
  if (T) HR_CUDA(cudaMemcpy(T, slot + c->lay.T, (size_t)K * 8, cudaMemcpyDeviceToHost));
  if (lut) HR_CUDA(cudaMemcpy(lut, slot + c->lay.lut, (size_t)K * 2, cudaMemcpyDeviceToHost));
  if (iters) {
    int m[4];
    HR_CUDA(cudaMemcpy(m, slot + c->lay.misc, sizeof(m), cudaMemcpyDeviceToHost));
    *iters = m[0];
  }
  return HR_OK;
}

hr_status histretinex_profile_solve(hr_ctx* c, int image, long long* ns, int* count) {
  if (!c || !ns || !count || image < 0 || image >= c->last_n) return HR_ERR_INVALID_ARG;
  if (!(c->p.flags & HR_FLAG_DEBUG_OUT)) return HR_ERR_INVALID_ARG;
  HR_CUDA(cudaSetDevice(c->device));
  HR_CUDA(cudaDeviceSynchronize());
  long long buf[hr::kProfSlots];
  HR_CUDA(cudaMemcpy(buf, c->last_base + (size_t)image * c->lay.bytes + c->lay.misc + 16, sizeof(buf),
                     cudaMemcpyDeviceToHost));
  int n = 0;
  while (n < hr::kProfSlots && buf[n] != 0) ++n;
  const int m = n < *count ? n : *count;
  for (int i = 0; i < m; ++i) ns[i] = buf[i];
  *count = m;
  return HR_OK;
}

hr_status histretinex_sync_status(hr_ctx* c, void* stream) {
  if (!c) return HR_ERR_INVALID_ARG;
  HR_CUDA(cudaSetDevice(c->device));
  HR_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  unsigned st = 0;
  HR_CUDA(cudaMemcpy(&st, c->d_status, sizeof(st), cudaMemcpyDeviceToHost));
  HR_CUDA(cudaMemset(c->d_status, 0, sizeof(unsigned)));
  if (st & hr::kStTimeout) return HR_ERR_TIMEOUT;
  if (st & hr::kStRange) return HR_ERR_RANGE;
  if (st & hr::kStUnsupported) return HR_ERR_UNSUPPORTED;
  return HR_OK;
}

hr_status histretinex_destroy(hr_ctx* c) {
  if (!c) return HR_OK;
  cudaSetDevice(c->device);
  if (c->desc_done) cudaEventSynchronize(c->desc_done);
  hr::partitions_destroy(c->part);
  cudaFree(c->d_ring);
  for (int i = 0; i < hr_ctx::kRingMax; ++i)
    if (c->ring_free[i]) cudaEventDestroy(c->ring_free[i]);
  cudaFree(c->d_slots);
  cudaFree(c->d_jstart1);
  cudaFree(c->d_cmap);
  cudaFree(c->d_jstart0);
  cudaFree(c->d_status);
  cudaFree(c->d_imgs);
  cudaFree(c->d_tile_start);
  cudaFreeHost(c->h_imgs);
  cudaFreeHost(c->h_tile_start);
  cudaFree(c->d_io_in);
  cudaFree(c->d_io_out);
  for (int b = 0; b < 2; ++b) {
    cudaFree(c->d_pp_in[b]);
    cudaFree(c->d_pp_out[b]);
    if (c->ev_in_ready[b]) cudaEventDestroy(c->ev_in_ready[b]);
    if (c->ev_in_free[b]) cudaEventDestroy(c->ev_in_free[b]);
    if (c->ev_done[b]) cudaEventDestroy(c->ev_done[b]);
    if (c->ev_out_free[b]) cudaEventDestroy(c->ev_out_free[b]);
  }
  if (c->s_h2d) cudaStreamDestroy(c->s_h2d);
  if (c->s_d2h) cudaStreamDestroy(c->s_d2h);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->desc_done) cudaEventDestroy(c->desc_done);
  for (int i = 0; i < hr_ctx::kRing; ++i)
    for (int q = 0; q < 4; ++q)
      if (c->ev[i][q]) cudaEventDestroy(c->ev[i][q]);
  delete c;
  return HR_OK;
}

const char* histretinex_status_string(hr_status s) {
  switch (s) {
    case HR_OK: return "ok";
    case HR_ERR_INVALID_ARG: return "invalid argument";
    case HR_ERR_UNSUPPORTED: return "unsupported request";
    case HR_ERR_OOM: return "out of memory";
    case HR_ERR_CUDA: return "CUDA runtime error";
    case HR_ERR_RANGE: return "image level >= K";
    case HR_ERR_TIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

size_t histretinex_workspace_bytes(const hr_ctx* c) { return c ? c->lay.bytes : 0; }

hr_status histretinex_reserve(hr_ctx* c, int n_images) {
  if (!c || n_images < 1) return HR_ERR_INVALID_ARG;
  HR_CUDA(cudaSetDevice(c->device));
  hr_status s = ensure_slots(c, n_images);
  if (s != HR_OK) return s;
  return ensure_desc(c, n_images);
}

hr_status histretinex_set_tuning(hr_ctx* c, const hr_tuning* t) {
  if (!c || !t) return HR_ERR_INVALID_ARG;
  if (t->hist_ctas_per_sm < 1 || t->hist_ctas_per_sm > 32 || t->apply_ctas_per_sm < 1 || t->apply_ctas_per_sm > 32)
    return HR_ERR_INVALID_ARG;
  if (t->solve_cluster < 1 || t->solve_cluster > 16 || (t->solve_cluster & (t->solve_cluster - 1)))
    return HR_ERR_INVALID_ARG;
  if (t->use_graph != 0 && t->use_graph != 1) return HR_ERR_INVALID_ARG;
  if (t->pdl < 0 || t->pdl > 7) return HR_ERR_INVALID_ARG;
  if (t->groups != 1 && t->groups != 2) return HR_ERR_INVALID_ARG;
  if (t->partitions < 0 || t->partitions > 4) return HR_ERR_INVALID_ARG;
  if (t->partition_cluster < 1 || t->partition_cluster > 16 || (t->partition_cluster & (t->partition_cluster - 1)))
    return HR_ERR_INVALID_ARG;
  c->tune = *t;
  return HR_OK;
}

hr_status histretinex_get_tuning(const hr_ctx* c, hr_tuning* t) {
  if (!c || !t) return HR_ERR_INVALID_ARG;
  *t = c->tune;
  return HR_OK;
}

hr_status histretinex_stage_times(hr_ctx* c, double* ms, int* calls, int reset) {
  if (!c) return HR_ERR_INVALID_ARG;
  HR_CUDA(cudaSetDevice(c->device));
  for (int i = 0; i < hr_ctx::kRing; ++i) {
    hr_status s = fold_timing(c, i);
    if (s != HR_OK) return s;
  }
  if (ms)
    for (int s = 0; s < 3; ++s) ms[s] = c->stage_ms[s];
  if (calls) *calls = c->stage_calls;
  if (reset) {
    c->stage_ms[0] = c->stage_ms[1] = c->stage_ms[2] = 0.0;
    c->stage_calls = 0;
  }
  return HR_OK;
}

uint64_t histretinex_kernel_launches(const hr_ctx* c) { return c ? c->launches : 0; }

hr_status histretinex_ablation_class_totals(int K, int n, const float* d_R, const float* d_L, float* d_P, int method,
                                           float* kernel_ms, void* stream) {
  if ((K != 128 && K != 256) || n < 1 || n > 4096 || !d_R || !d_L || !d_P || method < 0 || method > 2)
    return HR_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  HR_CUDA(cudaGetDevice(&dev));
  HR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  unsigned* d_status = nullptr;
  HR_CUDA(cudaMalloc(&d_status, sizeof(unsigned)));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(d_status, 0, sizeof(unsigned), st);
  hr_status s = e == cudaSuccess ? hr::ablation_class_totals(K, n, d_R, d_L, d_P, method, d_status, sms, st, kernel_ms)
                                 : cuda_fail(e);
  unsigned h = 0;
  if (s == HR_OK) {
    e = cudaMemcpy(&h, d_status, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) s = cuda_fail(e);
  }
  cudaFree(d_status);
  if (s == HR_OK && (h & hr::kStTimeout)) s = HR_ERR_TIMEOUT;
  return s;
}

hr_status histretinex_partition_info(const hr_ctx* c, int* solve_parts, int* pixel_sms) {
  if (!c || !solve_parts || !pixel_sms) return HR_ERR_INVALID_ARG;
  const bool on = c->part && c->tune.partitions == c->part_parts;  // (a changed count applies at the next call)
  *solve_parts = on ? c->part_parts : 0;
  *pixel_sms = on ? hr::partitions_pixel_sms(c->part) : c->sm_count;
  return HR_OK;
}

hr_status histretinex_gradient_levels(int form, int K, int m2_first, int n, uint16_t* d_out, void* stream) {
  if (form < 0 || form > 2 || !hr::pow2(K) || K < 8 || K > 4096 || m2_first < 0 || n < 1 || !d_out)
    return HR_ERR_INVALID_ARG;
  if (form < 2 && K > 256) return HR_ERR_INVALID_ARG;
  const long long last = (long long)m2_first + n - 1;
  if (last >= (form == 1 ? (1LL << 23) : (1LL << 31) - 1)) return HR_ERR_INVALID_ARG;
  HR_CUDA(hr::launch_grad_level_probe(form, K, m2_first, n, d_out, static_cast<cudaStream_t>(stream)));
  return HR_OK;
}

}  // extern "C"
