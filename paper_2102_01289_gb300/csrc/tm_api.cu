// tm_api.cu -- the C ABI declared in include/tm.h: parameter validation,
// context and workspace management, and the launch sequences of the forward
// path. Every entry point validates on the host before issuing GPU work.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <utility>
#include <vector>

#include <cstdint>

#include "tm.h"
#include "tm_backward.cuh"
#include "tm_host.h"
#include "tm_kernels.cuh"

using namespace tmk;

namespace {
// Job descriptors reach the device as kernel parameters of a one-block copy
// kernel, not through a host-to-device copy: such a copy waits on the copy
// engine behind any large upload in flight on another stream (the next image
// of tm_forward_host_async), which would stall the forward it starts.
constexpr int kPutJobs = 32;  // 32 jobs of under 700 bytes fit the 32 KB parameter space
template <int N>
struct JobPack {
  Job j[N];
};

template <int N>
__global__ void k_put_jobs(const __grid_constant__ JobPack<N> p, Job *dst, int n) {
  const unsigned *src = reinterpret_cast<const unsigned *>(p.j);
  unsigned *d = reinterpret_cast<unsigned *>(dst);
  const int words = n * (int)(sizeof(Job) / 4);
  for (int i = threadIdx.x; i < words; i += blockDim.x) d[i] = src[i];
}
static_assert(sizeof(Job) % 4 == 0, "jobs are copied as words");

}  // namespace

namespace tmk {
// Writes jobs h[0..n) to d on stream s; returns the launches made.
int put_jobs(const Job *h, int n, Job *d, cudaStream_t s) {
  if (n == 1) {
    JobPack<1> p;
    p.j[0] = h[0];
    k_put_jobs<1><<<1, 128, 0, s>>>(p, d, 1);
    return 1;
  }
  int launches = 0;
  for (int i = 0; i < n; i += kPutJobs) {
    JobPack<kPutJobs> p;
    const int m = std::min(kPutJobs, n - i);
    std::memcpy(p.j, h + i, sizeof(Job) * (size_t)m);
    k_put_jobs<kPutJobs><<<1, 256, 0, s>>>(p, d + i, m);
    ++launches;
  }
  return launches;
}
}  // namespace tmk

struct tm_ctx {
  tm_params p;
  std::string err;
  int debug = 0;
  int hist_path = 0;
  int sweep_tiles = 0;  // TM_OPT_SWEEP_TILES (0: one wave of the sweep's CTAs per image share)
  int sweep_width = 0;  // TM_OPT_SWEEP_WIDTH (0: automatic)
  int64_t launches = 0;
  int num_sms = 0;
  size_t smem_optin = 0;
  // device workspace (grown on demand; growing drops the cached graph)
  void *ws = nullptr;
  size_t ws_bytes = 0;
  Stats *stats = nullptr;  // one per image of the largest batch so far
  int stats_n = 0;
  // job descriptors: written to a device buffer at the start of each call by
  // put_jobs (the sweep queue is written on the device); stream-ordered like
  // the workspace. The cached batch graph has its own device buffers, written
  // by its own nodes at every replay.
  Job *djobs = nullptr;    // device copy of the job array (calls outside the graph)
  int4 *ditems = nullptr;  // sweep queue: the pop counter
  size_t djobs_bytes = 0, ditems_bytes = 0;
  Job *gdjobs = nullptr;   // device buffers written by the cached graph
  int4 *gditems = nullptr;
  size_t gdjobs_bytes = 0, gditems_bytes = 0;
  // backward workspace
  void *bws = nullptr;
  size_t bws_bytes = 0;
  // staging for tm_forward_host
  void *stage = nullptr;
  size_t stage_bytes = 0;
  // tm_forward_host_async: call k uploads into input slot k%2 on copy_stream,
  // runs the forward into output slot k%2 on fwd_stream and downloads that
  // slot on the caller's stream. hslot_free/oslot_free are recorded after the
  // last read of a slot (the forward, the download), *_full after its write.
  void *hslot[2] = {nullptr, nullptr}, *oslot[2] = {nullptr, nullptr};
  size_t hslot_bytes = 0, oslot_bytes = 0;
  cudaEvent_t hslot_free[2] = {nullptr, nullptr}, hslot_full[2] = {nullptr, nullptr};
  cudaEvent_t oslot_free[2] = {nullptr, nullptr}, oslot_full[2] = {nullptr, nullptr};
  cudaStream_t copy_stream = nullptr, fwd_stream = nullptr;
  int hslot_next = 0;
  // The forwards on fwd_stream share the workspace with the calls made on the
  // caller's streams: a call waits for fwd_done (the last forward on
  // fwd_stream) if one is pending, and the next forward on fwd_stream waits
  // for ext_done (recorded after the last such call).
  cudaEvent_t fwd_done = nullptr, ext_done = nullptr;
  bool fwd_pending = false, ext_pending = false;
  // layout of the last single-image forward (for debug exports)
  int last_W = 0, last_H = 0, last_q = 0, last_path = 0;
  uint8_t *bins = nullptr;
  int32_t *q = nullptr;
  DebugPlanes dbg{};
  // CUDA graphs of the last fused forwards (batches, or the images of a batch
  // taking the fused path, and single images), each replayed while its images
  // are unchanged; the least recently used is replaced. They share the
  // workspace and gdjobs / gditems, which each replay rewrites first. And the
  // graph of the last batch's images taking the materialised path, with that
  // pass's own workspace and descriptors.
  struct FusedGraph {
    cudaGraphExec_t exec = nullptr;
    std::vector<tm_image> in, out;
    int64_t launches = 0;
    std::vector<Job> jobs;
    uint64_t used = 0;
  };
  std::vector<FusedGraph> graphs;
  uint64_t calls = 0;  // forward calls so far (FusedGraph::used counts in them)
  // single-image (input, output) pairs seen lately without a graph, with the
  // call that saw them: a pair gets its graph when it comes back
  std::vector<std::pair<std::vector<tm_image>, uint64_t>> graph_seen;
  cudaGraphExec_t mgraph = nullptr;
  std::vector<tm_image> mgraph_in, mgraph_out;
  int64_t mgraph_launches = 0;
  void *mws = nullptr;
  size_t mws_bytes = 0;
  Job *mdjobs = nullptr;
  size_t mdjobs_bytes = 0;
  cudaStream_t graph_stream = nullptr;
  // The fused forward runs the sweep on sweep_stream (high priority) beside
  // the integral images on int_stream (low priority): the integral images
  // only need q, the sweep only the bins, and the integral tiles fill the
  // SMs that the sweep's last segments leave idle. ov_fork / ov_sweep /
  // ov_int order the two streams after the prep stage and before the lookup.
  cudaStream_t sweep_stream = nullptr, int_stream = nullptr;
  cudaEvent_t ov_fork = nullptr, ov_sweep = nullptr, ov_int = nullptr;
  // streaming range reuse (TM_OPT_REUSE_RANGE): two range states; a forward
  // bins with rr_stats[rr_cur] and leaves its own range in the other
  int reuse_range = 0;
  Stats *rr_stats = nullptr;
  int rr_cur = 0, rr_valid = 0, rr_W = 0, rr_H = 0, rr_q = 0;
  const Stats *last_stats = nullptr;  // range state of the last single-image forward
  // TM_OPT_BACKWARD_REUSE: the job descriptors of the last fused forward that
  // left its intermediates (bins, q, integral images, count planes) in the
  // workspace and the images it ran on
  int bwd_reuse = 0;
  bool fwd_valid = false;
  std::vector<Job> fwd_jobs;
  std::vector<tm_image> fwd_in;
  // automatic histogram path: the measured choice per (width, height, in dtype, out dtype),
  // and per batch of images that fit the sweep (their sizes and dtype pairs)
  std::map<std::tuple<int, int, int, int>, int> path_choice;
  std::map<std::vector<std::tuple<int, int, int, int>>, int> batch_choice;
  // stage timing: events recorded on the call's stream after each stage
  int stage_timing = 0;
  // per call, its stage marks: the event, the stage it ends (or kNoStage),
  // and the index of the mark it is timed from (-1: the one before)
  struct Mark {
    cudaEvent_t e;
    int stage, from;
  };
  std::vector<std::vector<Mark>> marks;
  std::vector<cudaEvent_t> event_pool;
  double stage_ms[16] = {};
};

namespace {

std::mutex g_create_mu;
std::string g_create_err;

tm_status fail(tm_ctx *c, tm_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  else {
    std::lock_guard<std::mutex> g(g_create_mu);
    g_create_err = buf;
  }
  return s;
}

tm_status cuda_fail(tm_ctx *c, cudaError_t e, const char *what) {
  return fail(c, TM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}
}  // namespace

namespace tmk {
tm_status fail_noctx(tm_status s, const char *msg) { return fail(nullptr, s, "%s", msg); }
}  // namespace tmk

namespace {

#define TM_CUDA(c, call)                                   \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail((c), e_, #call); \
  } while (0)

bool finite_pos(float v) { return std::isfinite(v) && v > 0.f; }

tm_status validate_params(const tm_params *p, std::string &why) {
  char b[256];
  if (!p) { why = "params is NULL"; return TM_EINVAL; }
  if (p->n_bins < 1 || p->n_bins > TM_MAX_BINS) {
    snprintf(b, sizeof b, "n_bins %d outside 1..%d", p->n_bins, TM_MAX_BINS); why = b; return TM_EINVAL;
  }
  if (p->n_fields < 1 || p->n_fields > TM_MAX_FIELDS) {
    snprintf(b, sizeof b, "n_fields %d outside 1..%d", p->n_fields, TM_MAX_FIELDS); why = b; return TM_EINVAL;
  }
  for (int f = 0; f < p->n_fields; ++f) {
    if (p->rx[f] < 0 || p->ry[f] < 0 || p->rx[f] > TM_MAX_RADIUS || p->ry[f] > TM_MAX_RADIUS) {
      snprintf(b, sizeof b, "field %d radius (%d, %d) outside 0..%d", f, p->rx[f], p->ry[f], TM_MAX_RADIUS);
      why = b; return TM_EINVAL;
    }
    if (!finite_pos(p->eps[f])) { snprintf(b, sizeof b, "field %d eps must be finite and > 0", f); why = b; return TM_EINVAL; }
    if (!std::isfinite(p->alpha[f]) || p->alpha[f] < 0.f) {
      snprintf(b, sizeof b, "field %d alpha must be finite and >= 0", f); why = b; return TM_EINVAL;
    }
  }
  if (!std::isfinite(p->ld_min) || !std::isfinite(p->ld_max) || p->ld_max < p->ld_min) {
    why = "need finite ld_min <= ld_max"; return TM_EINVAL;
  }
  if (!std::isfinite(p->sat) || p->sat < 0.f) { why = "sat must be finite and >= 0"; return TM_EINVAL; }
  if (p->flags & ~(TM_FLAG_CDF_INCLUSIVE | TM_FLAG_AREA_LITERAL | TM_FLAG_VAR_LINEAR | TM_FLAG_SRGB_U8)) {
    snprintf(b, sizeof b, "flags 0x%x has undefined bits", (unsigned)p->flags); why = b; return TM_EINVAL;
  }
  return TM_OK;
}

enum Stage { ST_RANGE, ST_PREP, ST_INTEGRAL, ST_HIST, ST_LOOKUP, ST_SWEEP, ST_BATCH,
             ST_BWD_PIXEL, ST_BWD_ADJOINT, ST_BWD_INPUT, ST_BATCH_MAT, ST_COUNT };
const char *const kStageNames[ST_COUNT] = {"range", "prep", "integral_image", "integral_histogram",
                                          "lookup", "fused_sweep", "batch", "bwd_pixel",
                                          "bwd_adjoint", "bwd_input", "batch_materialised"};

// Record a stage boundary on stream s (stage < 0 opens a new call).
// Record a stage boundary on stream s (stage -1 opens a new call; kNoStage
// marks a point that ends no stage). The stage is timed from mark `from` of
// the call (-1: the mark before). Returns this mark's index in the call (-1
// without stage timing).
constexpr int kNoStage = -2;
int mark(tm_ctx *c, cudaStream_t s, int stage, int from = -1) {
  if (!c->stage_timing) return -1;
  cudaEvent_t e;
  if (!c->event_pool.empty()) {
    e = c->event_pool.back();
    c->event_pool.pop_back();
  } else if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  if (stage == -1) c->marks.emplace_back();
  if (c->marks.empty()) c->marks.emplace_back();
  cudaEventRecord(e, s);
  c->marks.back().push_back({e, stage, from});
  return (int)c->marks.back().size() - 1;
}

size_t elem_size(int dt) { return dt == TM_F32 ? 4 : dt == TM_F16 ? 2 : 1; }

tm_status validate_image(tm_ctx *c, const tm_image *im, const char *name, bool is_input) {
  if (!im) return fail(c, TM_EINVAL, "%s descriptor is NULL", name);
  if (!im->data) return fail(c, TM_EINVAL, "%s.data is NULL", name);
  if (im->width < 1 || im->height < 1)
    return fail(c, TM_EINVAL, "%s size %dx%d must be positive", name, im->width, im->height);
  if ((long long)im->width * im->height > (1LL << 31) - 1)
    return fail(c, TM_EINVAL, "%s has more than 2^31-1 pixels", name);
  if (im->pitch < 3LL * im->width)
    return fail(c, TM_EINVAL, "%s.pitch %lld < 3*width", name, (long long)im->pitch);
  if (im->dtype != TM_F32 && im->dtype != TM_F16 && im->dtype != TM_U8)
    return fail(c, TM_EINVAL, "%s.dtype %d unknown", name, im->dtype);
  if (is_input && im->dtype == TM_U8)
    return fail(c, TM_EUNSUPPORTED, "%s: uint8 input is not supported (use F32 or F16)", name);
  if (((uintptr_t)im->data) % elem_size(im->dtype))
    return fail(c, TM_EINVAL, "%s.data is not aligned to its element size", name);
  return TM_OK;
}

size_t image_bytes(const tm_image *im) {
  return ((size_t)(im->height - 1) * im->pitch + 3 * (size_t)im->width) * elem_size(im->dtype);
}

bool overlap(const tm_image *a, const tm_image *b) {
  uintptr_t a0 = (uintptr_t)a->data, a1 = a0 + image_bytes(a);
  uintptr_t b0 = (uintptr_t)b->data, b1 = b0 + image_bytes(b);
  return a0 < b1 && b0 < a1;
}

// Q for the quantised log: the largest Q <= 24 with every window sum of q^2
// below 2^63 (|q| <= 2^(Q-1), windows of at most n_max pixels).
int choose_qbits(const tm_params &p, int W, int H) {
  unsigned long long n_max = 1;
  for (int f = 0; f < p.n_fields; ++f) {
    // the unclipped window under TM_FLAG_AREA_LITERAL (zero padding)
    const bool lit = (p.flags & TM_FLAG_AREA_LITERAL) != 0;
    unsigned long long wx = lit ? 2ULL * p.rx[f] + 1 : std::min<long long>(2LL * p.rx[f] + 1, W);
    unsigned long long wy = lit ? 2ULL * p.ry[f] + 1 : std::min<long long>(2LL * p.ry[f] + 1, H);
    n_max = std::max(n_max, wx * wy);
  }
  int Q = 24;
  while (Q > 2 && ((unsigned __int128)n_max << (2 * Q - 2)) >= ((unsigned __int128)1 << 63)) --Q;
  return Q;
}

DevParams dev_params(const tm_params &p, int qbits) {
  DevParams d{};
  d.n_bins = p.n_bins;
  d.n_fields = p.n_fields;
  for (int f = 0; f < TM_MAX_FIELDS; ++f) {
    d.rx[f] = p.rx[f];
    d.ry[f] = p.ry[f];
    d.eps[f] = p.eps[f];
    d.alpha[f] = p.alpha[f];
  }
  d.ld_min = p.ld_min;
  d.ld_max = p.ld_max;
  d.sat = p.sat;
  d.qbits = qbits;
  d.flags = p.flags;
  bool small = true;  // every unclipped window below 2^18 pixels
  for (int f = 0; f < p.n_fields; ++f) small = small && (2LL * p.rx[f] + 1) * (2LL * p.ry[f] + 1) < (1LL << 18);
  d.small_win = small ? 1 : 0;
  return d;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

tm_status ensure_device_info(tm_ctx *c) {
  if (c->num_sms) return TM_OK;
  int dev = 0, v = 0;
  TM_CUDA(c, cudaGetDevice(&dev));
  TM_CUDA(c, cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
  c->num_sms = v;
  TM_CUDA(c, cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  c->smem_optin = (size_t)v;
  return TM_OK;
}

// The side streams and events of the overlapped sweep (created once).
tm_status ensure_side_streams(tm_ctx *c) {
  if (c->sweep_stream) return TM_OK;
  int least = 0, greatest = 0;
  TM_CUDA(c, cudaDeviceGetStreamPriorityRange(&least, &greatest));
  TM_CUDA(c, cudaStreamCreateWithPriority(&c->sweep_stream, cudaStreamNonBlocking, greatest));
  TM_CUDA(c, cudaStreamCreateWithPriority(&c->int_stream, cudaStreamNonBlocking, least));
  for (cudaEvent_t *e : {&c->ov_fork, &c->ov_sweep, &c->ov_int})
    TM_CUDA(c, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  return TM_OK;
}

// Fused-forward graphs kept at once (two alternating images, each also
// through the host entry points' two staging slots, fit).
constexpr size_t kFusedGraphs = 6;

void drop_graph(tm_ctx *c) {
  for (auto &g : c->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
  if (c->mgraph) cudaGraphExecDestroy(c->mgraph);
  c->mgraph = nullptr;
  c->mgraph_in.clear();
  c->mgraph_out.clear();
}

tm_status ensure_stats(tm_ctx *c, int n) {
  if (c->stats_n >= n) return TM_OK;
  drop_graph(c);
  if (c->stats) {
    TM_CUDA(c, cudaDeviceSynchronize());
    cudaFree(c->stats);
    c->stats = nullptr;
    c->stats_n = 0;
  }
  std::vector<Stats> h((size_t)n);
  for (auto &st : h) {
    memset(&st, 0, sizeof st);
    st.min_bits = 0x7f800000u;
  }
  TM_CUDA(c, cudaMalloc(&c->stats, sizeof(Stats) * (size_t)n));
  TM_CUDA(c, cudaMemcpy(c->stats, h.data(), sizeof(Stats) * (size_t)n, cudaMemcpyHostToDevice));
  c->stats_n = n;
  return TM_OK;
}

// Range states of a single-image forward under TM_OPT_REUSE_RANGE: the image
// is binned over *cur, which holds the previous image's range, unless there
// is no usable previous image (first call, other size or Q): then *own is set
// and the range pass fills *cur first. The bin pass leaves the image's own
// range in *next, the state the following call bins over.
tm_status reuse_states(tm_ctx *c, int W, int H, int qbits, Stats **cur, Stats **next, bool *own) {
  if (!c->rr_stats) {
    Stats h[2];
    memset(h, 0, sizeof h);
    h[0].min_bits = h[1].min_bits = 0x7f800000u;
    TM_CUDA(c, cudaMalloc(&c->rr_stats, sizeof h));
    TM_CUDA(c, cudaMemcpy(c->rr_stats, h, sizeof h, cudaMemcpyHostToDevice));
  }
  *own = !(c->rr_valid && c->rr_W == W && c->rr_H == H && c->rr_q == qbits);
  *cur = c->rr_stats + c->rr_cur;
  *next = c->rr_stats + (c->rr_cur ^ 1);
  c->rr_cur ^= 1;
  c->rr_valid = 1;
  c->rr_W = W;
  c->rr_H = H;
  c->rr_q = qbits;
  return TM_OK;
}

tm_status grow_device(tm_ctx *c, void **p, size_t *have, size_t bytes) {
  if (*have >= bytes) return TM_OK;
  drop_graph(c);
  if (*p) {
    TM_CUDA(c, cudaDeviceSynchronize());
    cudaFree(*p);
    *p = nullptr;
    *have = 0;
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, TM_ENOMEM, "device allocation of %zu bytes: %s", bytes, cudaGetErrorString(e));
  }
  *have = bytes;
  return TM_OK;
}

Image to_image(const tm_image *im) {
  Image r;
  r.p = im->data;
  r.W = im->width;
  r.H = im->height;
  r.pitch = im->pitch;
  r.dtype = im->dtype;
  return r;
}

tm_status check_launch(tm_ctx *c, const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, what);
  return TM_OK;
}

bool same_images(const std::vector<tm_image> &a, const tm_image *b, int n) {
  if ((int)a.size() != n) return false;
  for (int i = 0; i < n; ++i)
    if (a[i].data != b[i].data || a[i].width != b[i].width || a[i].height != b[i].height ||
        a[i].pitch != b[i].pitch || a[i].dtype != b[i].dtype)
      return false;
  return true;
}

// Per-image sizes of the forward workspace.
struct JobLayout {
  size_t bins, q, s12, segtot, cnt, grp, claim, mom, dcnt, dvar, dw, dlf, dl, total;
};

// Workspace of one image. cnt_bytes: the sweep's count planes (0 on the
// materialised path); grp: per row and 32-column group, the bin range; mom:
// the window moments kept for the backward.
JobLayout job_layout(const tm_params &p, int W, int H, int nseg, size_t cnt_bytes, bool debug, bool mom = false,
                     int bands = 0) {
  // nseg: row segments of the integral images (integral_layout)
  JobLayout L{};
  const size_t N = (size_t)W * H;
  const size_t plane = (size_t)(W + 1) * (H + 1);
  const int s = p.n_fields;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
  L.bins = take(N);
  L.q = take(4 * N);
  L.s12 = take(16 * plane);  // the integral images of q and q^2, interleaved
  L.segtot = take(8 * integral_scratch_elems(W, H, nseg));
  L.cnt = take(cnt_bytes);
  L.grp = take(2 * (size_t)((W + 31) / 32) * H);
  L.claim = take(4 * (size_t)bands);  // the sweep's band claims
  if (mom) L.mom = take(8 * N * s);
  if (debug) {
    L.dcnt = take(4 * N * s);
    L.dvar = take(4 * N * s);
    L.dw = take(4 * N * s);
    L.dlf = take(4 * N * s);
    L.dl = take(4 * N);
  }
  L.total = off;
  return L;
}

// The materialised path for one image: range, bins, integral images,
// bin-major cumulative integral histogram, lookup. Used when the fused sweep
// does not fit the fields, or on request (TM_OPT_HIST_PATH = 2).
tm_status forward_materialised(tm_ctx *c, const tm_image *in, const tm_image *out, cudaStream_t s) {
  c->fwd_valid = false;  // its workspace layout holds no count planes
  const int W = in->width, H = in->height;
  const int qbits = choose_qbits(c->p, W, H);
  DevParams P = dev_params(c->p, qbits);
  int nseg, seg_rows;
  integral_layout(W, H, SIZE_MAX, nseg, seg_rows);
  JobLayout L = job_layout(c->p, W, H, nseg, 0, c->debug != 0);
  const size_t plane = (size_t)(W + 1) * (H + 1);
  size_t off_cpl = align256(L.total), off_hscr = 0, total = off_cpl;
  if (c->p.n_bins > 1) {
    total = off_cpl + align256(4 * plane * (size_t)(c->p.n_bins - 1));
    off_hscr = total;
    total += align256(hist_scratch_bytes(W, H, c->p.n_bins - 1));
  }
  tm_status st;
  if ((st = ensure_stats(c, 1))) return st;
  if ((st = grow_device(c, &c->ws, &c->ws_bytes, total))) return st;
  if ((st = grow_device(c, (void **)&c->djobs, &c->djobs_bytes, sizeof(Job)))) return st;
  char *ws = static_cast<char *>(c->ws);
  Job J{};
  J.in = to_image(in);
  J.out = to_image(out);
  J.st = c->stats;
  bool run_range = true;
  if (c->reuse_range) {
    bool own = true;
    if ((st = reuse_states(c, W, H, qbits, &J.st, &J.st_next, &own))) return st;
    run_range = own;
  }
  J.bins = reinterpret_cast<uint8_t *>(ws + L.bins);
  J.q = reinterpret_cast<int32_t *>(ws + L.q);
  J.s1 = reinterpret_cast<long long *>(ws + L.s12);
  J.s2 = J.s1 + 1;
  J.s_pair = 1;
  J.segtot = reinterpret_cast<long long *>(ws + L.segtot);
  J.qbits = qbits;
  J.nseg = nseg;
  J.seg_rows = seg_rows;
  if (c->debug) {
    J.dbg.cnt = reinterpret_cast<unsigned *>(ws + L.dcnt);
    J.dbg.sigma2 = reinterpret_cast<float *>(ws + L.dvar);
    J.dbg.weight = reinterpret_cast<float *>(ws + L.dw);
    J.dbg.lf = reinterpret_cast<float *>(ws + L.dlf);
    J.dbg.l = reinterpret_cast<float *>(ws + L.dl);
  }
  const int rb = range_blocks(W, H, c->num_sms, 1.0), pb = prep_blocks(W, H, c->num_sms, 1.0);
  J.b0[kStRange] = J.b0[kStPrep] = J.b0[kStRows] = J.b0[kStCols] = J.b0[kStLook] = 0;
  int64_t n = put_jobs(&J, 1, c->djobs, s);
  mark(c, s, -1);
  if (run_range) launch_range(c->djobs, 1, rb, c->p.n_bins, J.in.dtype, s);
  mark(c, s, ST_RANGE);
  launch_prep(c->djobs, 1, pb, c->p.n_bins, c->p.flags, c->p.n_fields, J.in.dtype, s);
  mark(c, s, ST_PREP);
  n += (run_range ? 2 : 1) +
       launch_integral_jobs(c->djobs, 1, integral_tile_blocks(W, nseg), integral_col_blocks(W), s);
  mark(c, s, ST_INTEGRAL);
  uint32_t *cpl = nullptr;
  if (c->p.n_bins > 1) {
    cpl = reinterpret_cast<uint32_t *>(ws + off_cpl);
    n += launch_integral_histogram(J.bins, W, H, c->p.n_bins, true, cpl, ws + off_hscr, s);
  }
  mark(c, s, ST_HIST);
  n += launch_lookup_materialised(J.in, J.out, P, J.bins, cpl, reinterpret_cast<int64_t *>(J.s1), J.dbg, s);
  mark(c, s, ST_LOOKUP);
  if ((st = check_launch(c, "forward launch"))) return st;
  c->launches = n;
  c->last_W = W;
  c->last_H = H;
  c->last_q = qbits;
  c->last_path = 2;
  c->bins = J.bins;
  c->q = J.q;
  c->dbg = J.dbg;
  c->last_stats = J.st;
  return TM_OK;
}

// The fused path over a batch of images: one launch per stage for the whole
// batch, the sweep as a persistent kernel over a queue of (image, strip, row
// band) tiles. `graph`: capture the batch into a CUDA graph of the context's
// cache and replay it while the batch is unchanged. Returns TM_EUNSUPPORTED
// if some image cannot be swept.
tm_status finish_fused(tm_ctx *c, int nimg, const tm_image *in, const std::vector<Job> &jobs, int64_t n,
                       bool run_range, std::vector<Job> *jobs_out);

tm_status forward_fused(tm_ctx *c, int nimg, const tm_image *in, const tm_image *out, cudaStream_t s,
                        bool graph, bool do_lookup = true, std::vector<Job> *jobs_out = nullptr) {
  tm_status st;
  if (graph)
    for (auto &G : c->graphs) {
      if (!same_images(G.in, in, nimg) || !same_images(G.out, out, nimg)) continue;
      c->fwd_valid = false;
      TM_CUDA(c, cudaGraphLaunch(G.exec, s));
      G.used = c->calls;
      return finish_fused(c, nimg, in, G.jobs, G.launches, true, jobs_out);
    }
  c->fwd_valid = false;  // the workspace is rewritten below
  const bool debug = c->debug != 0 && nimg == 1 && !graph;
  // under TM_OPT_BACKWARD_REUSE the lookup also keeps the window moments
  const bool keep_mom = c->bwd_reuse != 0 && do_lookup;
  double total_px = 0;
  for (int i = 0; i < nimg; ++i) total_px += (double)in[i].width * in[i].height;
  std::vector<Job> jobs((size_t)nimg);
  std::vector<JobLayout> lays((size_t)nimg);
  std::vector<size_t> offs((size_t)nimg);
  // strips of 512 own columns (one CTA per SM, with all of its shared memory)
  // where every image fits them, else 256 (two CTAs per SM)
  const DevParams P0 = dev_params(c->p, 0);
  int width = c->sweep_width == 256 ? 256 : 512;
  size_t smem_limit = 0, smem = 0;
  for (int pass = 0; pass < 2; ++pass) {
    smem_limit = width == 512 ? c->smem_optin - 2048 : std::min(c->smem_optin - 2048, (size_t)110 * 1024);
    smem = 0;
    bool ok = true;
    for (int i = 0; i < nimg && ok; ++i) {
      Job &J = jobs[(size_t)i];
      memset(&J, 0, sizeof J);
      ok = plan_sweep(P0, in[i].width, in[i].height, 1, smem_limit, width, J.plan);
      smem = std::max(smem, J.plan.smem);
    }
    if (ok) break;
    if (width == 256) return TM_EUNSUPPORTED;
    width = 256;
  }
  const int cps = std::max(1, sweep_ctas_per_sm(c->p.n_fields, smem, width));
  const int wave = c->num_sms * cps;
  size_t ws_total = 0;
  int b_range = 0, b_prep = 0, b_rows = 0, b_cols = 0, b_look = 0;
  std::vector<std::pair<double, int>> order;  // (work of one tile, image)
  for (int i = 0; i < nimg; ++i) {
    const int W = in[i].width, H = in[i].height;
    const double share = nimg == 1 ? 1.0 : std::max(1.0 / c->num_sms, W * (double)H / total_px);
    Job &J = jobs[(size_t)i];
    J.qbits = choose_qbits(c->p, W, H);
    // one wave of segments, shared among a batch's images by pixel count (the
    // segments' band claims even out the CTAs' work; two waves of them were
    // slower on 16 x 1 MP: 1.33 against 1.28 ms)
    const int target = c->sweep_tiles > 0 ? c->sweep_tiles : std::max(1, (int)std::lround(wave * share));
    plan_sweep(P0, W, H, target, smem_limit, width, J.plan);
    integral_layout(W, H, SIZE_MAX, J.nseg, J.seg_rows);
    const size_t cnt_bytes = sweep_count_bytes(P0, J.plan, J.cnt_off);
    J.cnt_wide = J.plan.cnt_wide;
    lays[(size_t)i] = job_layout(c->p, W, H, J.nseg, cnt_bytes, debug, keep_mom, J.plan.tiles_x * J.plan.tiles_y);
    offs[(size_t)i] = ws_total;
    ws_total += lays[(size_t)i].total;
    J.b0[kStRange] = b_range;
    b_range += range_blocks(W, H, c->num_sms, share);
    J.b0[kStPrep] = b_prep;
    b_prep += prep_blocks(W, H, c->num_sms, share);
    J.b0[kStRows] = b_rows;
    b_rows += integral_tile_blocks(W, J.nseg);
    J.b0[kStCols] = b_cols;
    b_cols += integral_col_blocks(W);
    J.b0[kStLook] = b_look;
    b_look += lookup_blocks(W, H);
    J.nitemA = J.plan.tiles_x * ((J.plan.tiles_y + J.plan.K - 1) / J.plan.K);
    J.nitemB = J.plan.tiles_x * J.plan.tiles_y - J.nitemA;
    const double seg = (double)J.plan.K * J.plan.TY;  // rows of a segment
    const double rows = std::min(seg + 2.0 * J.plan.Ry + 1, H + 1.0);
    const double cols = std::min(J.plan.TX + 2.0 * J.plan.Rx + 2, W + 1.0);
    order.push_back({rows * (cols * 0.05 + 100.0) + 6.0 * J.plan.TX * seg, i});
  }
  // the queue holds each image's tiles together, the images with the
  // costliest tiles first
  std::stable_sort(order.begin(), order.end(),
                   [](const std::pair<double, int> &a, const std::pair<double, int> &b) { return a.first > b.first; });
  int nitems = 0;
  for (const auto &o : order) {  // first phase: every job's group starts
    jobs[(size_t)o.second].itemA0 = nitems;
    nitems += jobs[(size_t)o.second].nitemA;
  }
  for (const auto &o : order) {  // second phase: the groups' other bands
    jobs[(size_t)o.second].itemB0 = nitems;
    nitems += jobs[(size_t)o.second].nitemB;
  }
  if ((st = ensure_stats(c, nimg))) return st;
  if ((st = grow_device(c, &c->ws, &c->ws_bytes, ws_total))) return st;
  if (graph && c->graphs.size() >= kFusedGraphs) {  // room for the graph captured below
    auto lru = std::min_element(c->graphs.begin(), c->graphs.end(),
                                [](const tm_ctx::FusedGraph &a, const tm_ctx::FusedGraph &b) { return a.used < b.used; });
    cudaGraphExecDestroy(lru->exec);
    c->graphs.erase(lru);
  }
  Job **djobs = graph ? &c->gdjobs : &c->djobs;
  int4 **ditems = graph ? &c->gditems : &c->ditems;
  if ((st = grow_device(c, (void **)djobs, graph ? &c->gdjobs_bytes : &c->djobs_bytes, sizeof(Job) * nimg)))
    return st;
  if ((st = grow_device(c, (void **)ditems, graph ? &c->gditems_bytes : &c->ditems_bytes, sizeof(int4))))
    return st;
  char *ws = static_cast<char *>(c->ws);
  for (int i = 0; i < nimg; ++i) {
    Job &J = jobs[(size_t)i];
    const JobLayout &L = lays[(size_t)i];
    char *b = ws + offs[(size_t)i];
    J.in = to_image(&in[i]);
    J.out = to_image(&out[i]);
    J.st = c->stats + i;
    J.st_next = nullptr;
    J.bins = reinterpret_cast<uint8_t *>(b + L.bins);
    J.q = reinterpret_cast<int32_t *>(b + L.q);
    J.s1 = reinterpret_cast<long long *>(b + L.s12);
    J.s2 = J.s1 + 1;
    J.s_pair = 1;
    J.segtot = reinterpret_cast<long long *>(b + L.segtot);
    J.cnt = reinterpret_cast<unsigned char *>(b + L.cnt);
    J.grp = reinterpret_cast<uint16_t *>(b + L.grp);
    J.claim = reinterpret_cast<int *>(b + L.claim);
    J.mom = keep_mom ? reinterpret_cast<float2 *>(b + L.mom) : nullptr;
    if (debug) {
      J.dbg.cnt = reinterpret_cast<unsigned *>(b + L.dcnt);
      J.dbg.sigma2 = reinterpret_cast<float *>(b + L.dvar);
      J.dbg.weight = reinterpret_cast<float *>(b + L.dw);
      J.dbg.lf = reinterpret_cast<float *>(b + L.dlf);
      J.dbg.l = reinterpret_cast<float *>(b + L.dl);
    }
  }
  bool run_range = true;
  if (c->reuse_range && nimg == 1 && !graph && do_lookup) {
    bool own = true;
    if ((st = reuse_states(c, in[0].width, in[0].height, jobs[0].qbits, &jobs[0].st, &jobs[0].st_next, &own)))
      return st;
    run_range = own;
  }
  const DevParams P = dev_params(c->p, jobs[0].qbits);  // qbits is per job
  Job *dj = *djobs;
  int *queue = reinterpret_cast<int *>(*ditems);
  const int ctas = std::min(nitems, wave);
  // a batch is captured on the context's own stream (capture is not allowed on
  // the legacy default stream) and the graph is then launched on the caller's
  const cudaStream_t caller = s;
  if ((st = ensure_side_streams(c))) return st;  // before any capture begins
  if (graph) {
    if (!c->graph_stream) TM_CUDA(c, cudaStreamCreateWithFlags(&c->graph_stream, cudaStreamNonBlocking));
    s = c->graph_stream;
    TM_CUDA(c, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  }
  int64_t n = put_jobs(jobs.data(), nimg, dj, s);
  if (!graph) mark(c, s, -1);
  const int in_dt = input_dtype(jobs.data(), nimg);
  if (run_range) launch_range(dj, nimg, b_range, c->p.n_bins, in_dt, s);
  if (!graph) mark(c, s, ST_RANGE);
  launch_prep(dj, nimg, b_prep, c->p.n_bins, c->p.flags, c->p.n_fields, in_dt, s);
  const int m_prep = graph ? -1 : mark(c, s, ST_PREP);
  // the sweep (high priority, launched first, so its CTAs take the SMs) and
  // the integral images (low priority) side by side, each timed from the end
  // of the prep stage, joined before the lookup
  TM_CUDA(c, cudaEventRecord(c->ov_fork, s));
  TM_CUDA(c, cudaStreamWaitEvent(c->sweep_stream, c->ov_fork, 0));
  TM_CUDA(c, cudaStreamWaitEvent(c->int_stream, c->ov_fork, 0));
  const int ls = launch_sweep(P, dj, nimg, nitems, queue, smem, ctas, width, c->sweep_stream);
  if (!graph) mark(c, c->sweep_stream, ST_SWEEP, m_prep);
  n += 1 + launch_integral_jobs(dj, nimg, b_rows, b_cols, c->int_stream);
  if (!graph) mark(c, c->int_stream, ST_INTEGRAL, m_prep);
  n += run_range ? 2 : 1;
  TM_CUDA(c, cudaEventRecord(c->ov_sweep, c->sweep_stream));
  TM_CUDA(c, cudaEventRecord(c->ov_int, c->int_stream));
  TM_CUDA(c, cudaStreamWaitEvent(s, c->ov_sweep, 0));
  TM_CUDA(c, cudaStreamWaitEvent(s, c->ov_int, 0));
  if (!graph) mark(c, s, kNoStage);  // the join: the lookup is timed from here
  if (do_lookup) {
    // the lookup variant: without debug planes, with or without the moments,
    // and for one dtype of every input and output when they share it
    bool wide = true;
    int dt = jobs[0].in.dtype;
    for (const Job &J : jobs) {
      wide = wide && J.cnt_wide == (1 << c->p.n_fields) - 1;
      if (J.in.dtype != dt || J.out.dtype != dt) dt = -1;
    }
    n += launch_lookup_counts(P, dj, nimg, b_look, !debug && wide, keep_mom, dt, s);
    if (!graph) mark(c, s, ST_LOOKUP);
  }
  if (graph) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (e != cudaSuccess || ls < 0) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return fail(c, TM_ECUDA, "batch capture failed: %s", cudaGetErrorString(e));
    }
    tm_ctx::FusedGraph G;
    e = cudaGraphInstantiate(&G.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
    G.in.assign(in, in + nimg);
    G.out.assign(out, out + nimg);
    G.launches = n;
    G.jobs = jobs;
    G.used = c->calls;
    c->graphs.push_back(std::move(G));
    TM_CUDA(c, cudaGraphLaunch(c->graphs.back().exec, caller));
  } else if (ls < 0) {
    return check_launch(c, "sweep shared-memory attribute");
  }
  if ((st = check_launch(c, "forward launch"))) return st;
  return finish_fused(c, nimg, in, jobs, n, run_range, jobs_out);
}

// Bookkeeping after a fused forward over `jobs` (n launches), launched or
// replayed: the intermediates the backward may reuse and, for one image, the
// layout the debug exports read.
tm_status finish_fused(tm_ctx *c, int nimg, const tm_image *in, const std::vector<Job> &jobs, int64_t n,
                       bool run_range, std::vector<Job> *jobs_out) {
  c->launches = n;
  if (jobs_out) *jobs_out = jobs;
  if (run_range) {  // each image binned over its own range, as a recomputation would
    c->fwd_jobs = jobs;
    c->fwd_in.assign(in, in + nimg);
    c->fwd_valid = true;
  }
  if (nimg == 1) {
    c->last_W = in[0].width;
    c->last_H = in[0].height;
    c->last_q = jobs[0].qbits;
    c->last_path = 1;
    c->bins = jobs[0].bins;
    c->q = jobs[0].q;
    c->dbg = jobs[0].dbg;
    c->last_stats = jobs[0].st;
  }
  return TM_OK;
}

// The materialised path over a batch of images (those whose fields do not fit
// the sweep, or for which it measured faster): the range, bin, quantised-log
// and integral-image stages run once for the whole batch; then each image's
// cumulative integral histogram and lookup, on one shared set of planes (the
// launches are stream-ordered). The stats of image i are c->stats[stats0 + i].
// `graph`: capture into the context's materialised-batch graph and replay it
// while the images are unchanged.
tm_status forward_materialised_batch(tm_ctx *c, int nimg, const tm_image *in, const tm_image *out, cudaStream_t s,
                                     bool graph, int stats0) {
  tm_status st;
  if (graph && c->mgraph && same_images(c->mgraph_in, in, nimg) && same_images(c->mgraph_out, out, nimg)) {
    TM_CUDA(c, cudaGraphLaunch(c->mgraph, s));
    c->launches = c->mgraph_launches;
    return TM_OK;
  }
  double total_px = 0;
  for (int i = 0; i < nimg; ++i) total_px += (double)in[i].width * in[i].height;
  std::vector<Job> jobs((size_t)nimg);
  std::vector<size_t> offs((size_t)nimg);
  std::vector<JobLayout> lays((size_t)nimg);
  size_t ws_total = 0, planes_bytes = 0, scratch_bytes = 0;
  int b_range = 0, b_prep = 0, b_rows = 0, b_cols = 0;
  const int nplanes = c->p.n_bins - 1;
  for (int i = 0; i < nimg; ++i) {
    const int W = in[i].width, H = in[i].height;
    const double share = nimg == 1 ? 1.0 : std::max(1.0 / c->num_sms, W * (double)H / total_px);
    Job &J = jobs[(size_t)i];
    memset(&J, 0, sizeof J);
    J.qbits = choose_qbits(c->p, W, H);
    integral_layout(W, H, SIZE_MAX, J.nseg, J.seg_rows);
    lays[(size_t)i] = job_layout(c->p, W, H, J.nseg, 0, false);
    offs[(size_t)i] = ws_total;
    ws_total += lays[(size_t)i].total;
    if (nplanes > 0) {
      planes_bytes = std::max(planes_bytes, align256(4 * (size_t)(W + 1) * (H + 1) * nplanes));
      scratch_bytes = std::max(scratch_bytes, align256(hist_scratch_bytes(W, H, nplanes)));
    }
    J.b0[kStRange] = b_range;
    b_range += range_blocks(W, H, c->num_sms, share);
    J.b0[kStPrep] = b_prep;
    b_prep += prep_blocks(W, H, c->num_sms, share);
    J.b0[kStRows] = b_rows;
    b_rows += integral_tile_blocks(W, J.nseg);
    J.b0[kStCols] = b_cols;
    b_cols += integral_col_blocks(W);
  }
  if ((st = ensure_stats(c, stats0 + nimg))) return st;
  if ((st = grow_device(c, &c->mws, &c->mws_bytes, ws_total + planes_bytes + scratch_bytes))) return st;
  if ((st = grow_device(c, (void **)&c->mdjobs, &c->mdjobs_bytes, sizeof(Job) * nimg))) return st;
  if (graph && c->mgraph) {
    cudaGraphExecDestroy(c->mgraph);  // re-captured below
    c->mgraph = nullptr;
  }
  char *ws = static_cast<char *>(c->mws);
  uint32_t *planes = nplanes > 0 ? reinterpret_cast<uint32_t *>(ws + ws_total) : nullptr;
  void *scratch = ws + ws_total + planes_bytes;
  for (int i = 0; i < nimg; ++i) {
    Job &J = jobs[(size_t)i];
    const JobLayout &L = lays[(size_t)i];
    char *b = ws + offs[(size_t)i];
    J.in = to_image(&in[i]);
    J.out = to_image(&out[i]);
    J.st = c->stats + stats0 + i;
    J.bins = reinterpret_cast<uint8_t *>(b + L.bins);
    J.q = reinterpret_cast<int32_t *>(b + L.q);
    J.s1 = reinterpret_cast<long long *>(b + L.s12);
    J.s2 = J.s1 + 1;
    J.s_pair = 1;
    J.segtot = reinterpret_cast<long long *>(b + L.segtot);
  }
  const cudaStream_t caller = s;
  if (graph) {
    if (!c->graph_stream) TM_CUDA(c, cudaStreamCreateWithFlags(&c->graph_stream, cudaStreamNonBlocking));
    s = c->graph_stream;
    TM_CUDA(c, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  }
  int64_t n = put_jobs(jobs.data(), nimg, c->mdjobs, s);
  const int in_dt = input_dtype(jobs.data(), nimg);
  launch_range(c->mdjobs, nimg, b_range, c->p.n_bins, in_dt, s);
  launch_prep(c->mdjobs, nimg, b_prep, c->p.n_bins, c->p.flags, c->p.n_fields, in_dt, s);
  n += 2 + launch_integral_jobs(c->mdjobs, nimg, b_rows, b_cols, s);
  for (int i = 0; i < nimg; ++i) {
    const Job &J = jobs[(size_t)i];
    if (planes) n += launch_integral_histogram(J.bins, J.in.W, J.in.H, c->p.n_bins, true, planes, scratch, s);
    n += launch_lookup_materialised(J.in, J.out, dev_params(c->p, J.qbits), J.bins, planes,
                                    reinterpret_cast<int64_t *>(J.s1), DebugPlanes{}, s);
  }
  if (graph) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return fail(c, TM_ECUDA, "materialised batch capture failed: %s", cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&c->mgraph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      c->mgraph = nullptr;
      return cuda_fail(c, e, "cudaGraphInstantiate");
    }
    c->mgraph_in.assign(in, in + nimg);
    c->mgraph_out.assign(out, out + nimg);
    c->mgraph_launches = n;
    TM_CUDA(c, cudaGraphLaunch(c->mgraph, caller));
  }
  if ((st = check_launch(c, "materialised batch launch"))) return st;
  c->launches = n;
  return TM_OK;
}

// Automatic histogram path: run each path twice on this image and time the
// second run with events (synchronising the stream); 1 = fused, 2 = materialised.
tm_status choose_path(tm_ctx *c, const tm_image *in, const tm_image *out, cudaStream_t s, int *choice) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  TM_CUDA(c, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    cudaGetLastError();
    return fail(c, TM_ECUDA, "cudaEventCreate");
  }
  float ms[3] = {0.f, 0.f, 0.f};
  tm_status st = TM_OK;
  bool fused_ok = true;
  for (int path = 1; path <= 2 && !st; ++path) {
    for (int rep = 0; rep < 2 && !st; ++rep) {
      cudaEventRecord(e0, s);
      st = path == 1 ? forward_fused(c, 1, in, out, s, false) : forward_materialised(c, in, out, s);
      if (path == 1 && st == TM_EUNSUPPORTED) {
        fused_ok = false;
        st = TM_OK;
        break;
      }
      cudaEventRecord(e1, s);
    }
    if (!st && (path == 2 || fused_ok)) {
      cudaError_t e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[path], e0, e1);
      if (e != cudaSuccess) st = cuda_fail(c, e, "timing the histogram paths");
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  *choice = fused_ok && ms[1] <= ms[2] ? 1 : 2;
  return TM_OK;
}

// Whether a single-image forward on (in, out) runs from a CUDA graph: yes
// when one is cached; else it is captured when the pair came in one of the
// recent calls and a graph slot is free, or the least recently used graph
// has not run for kGraphStale calls. A pair seen for the first time runs its
// launches directly, so a stream of ever-new buffers never pays for a
// capture, and pairs cycling through more slots than there are do not
// replace one another's graphs on every call.
constexpr uint64_t kGraphStale = 64;
constexpr size_t kGraphSeen = 16;

bool single_graph_ok(tm_ctx *c, const tm_image *in, const tm_image *out) {
  const std::vector<tm_image> pair{*in, *out};
  for (const auto &G : c->graphs)
    if (same_images(G.in, in, 1) && same_images(G.out, out, 1)) return true;
  auto seen = std::find_if(c->graph_seen.begin(), c->graph_seen.end(), [&](const auto &e) {
    return same_images(e.first, pair.data(), 2);
  });
  if (seen != c->graph_seen.end()) {
    seen->second = c->calls;
    bool room = c->graphs.size() < kFusedGraphs;
    for (const auto &G : c->graphs) room = room || G.used + kGraphStale < c->calls;
    if (!room) return false;
    c->graph_seen.erase(seen);
    return true;
  }
  if (c->graph_seen.size() >= kGraphSeen)
    c->graph_seen.erase(std::min_element(c->graph_seen.begin(), c->graph_seen.end(),
                                         [](const auto &a, const auto &b) { return a.second < b.second; }));
  c->graph_seen.emplace_back(pair, c->calls);
  return false;
}

// The forward launch sequence on one image (device buffers already checked).
tm_status forward_device(tm_ctx *c, const tm_image *in, const tm_image *out, cudaStream_t s) {
  tm_status st = ensure_device_info(c);
  if (st) return st;
  ++c->calls;
  int path = c->hist_path;
  if (c->p.n_bins < 2) path = 2;  // no thresholds: nothing to sweep
  if (path == 0) {
    const auto key = std::make_tuple((int)in->width, (int)in->height, (int)in->dtype, (int)out->dtype);
    auto it = c->path_choice.find(key);
    if (it == c->path_choice.end()) {
      if ((st = choose_path(c, in, out, s, &path))) return st;
      it = c->path_choice.emplace(key, path).first;
    }
    path = it->second;
  }
  if (path == 1) {
    // a cached CUDA graph per image pair unless a per-call feature is on
    const bool graph = !c->stage_timing && !c->debug && !c->reuse_range && single_graph_ok(c, in, out);
    st = forward_fused(c, 1, in, out, s, graph);
    if (st != TM_EUNSUPPORTED) return st;
    if (c->hist_path == 1)
      return fail(c, TM_EUNSUPPORTED, "fused sweep does not fit these fields (use the materialised path)");
  }
  return forward_materialised(c, in, out, s);
}

// The backward's device workspace: a header of the per-image accumulators,
// the parameter sums and the descriptor arrays of the largest group, then per
// image of a group its u / v planes, direct luminance gradient, fixed-point
// pair planes and their scratch.
size_t backward_image_bytes(const tm_params &p, int W, int H, int nseg) {
  const size_t N = (size_t)W * H, plane = (size_t)(W + 1) * (H + 1);
  const int nf = p.n_fields;
  return 2 * align256(4 * N * nf) + align256(4 * N) + align256(16 * plane * nf) +
         align256(8 * fix_integral_scratch_elems(W, H, nf, nseg));
}

// Header: accumulators, parameter sums, then the descriptors (BwdJob[n],
// FixJob[n]).
size_t backward_header_bytes(int n) {
  return align256(sizeof(BwdAcc) * n) + align256(sizeof(double) * kBwdParams) +
         align256((sizeof(BwdJob) + sizeof(FixJob)) * n);
}

// Images of a backward group: the workspace of one group stays below this
// (or holds one image), and a group has at most kBwdGroupMax images (its
// descriptors travel as kernel parameters); the groups run one after
// another on the stream.
constexpr size_t kBwdGroupBytes = size_t(4) << 30;

// Groups [g[k], g[k + 1]) of the images and each image's row segments of the
// fixed-point integrals.
void backward_groups(const tm_params &p, int n, const tm_image *in, std::vector<int> &g, std::vector<int> &nseg,
                     std::vector<int> &seg_rows) {
  g.assign(1, 0);
  size_t used = 0;
  for (int i = 0; i < n; ++i) {
    int ns, sr;
    fix_layout(in[i].width, in[i].height, 1, ns, sr);
    const size_t b = backward_image_bytes(p, in[i].width, in[i].height, ns);
    if (i > g.back() && (used + b > kBwdGroupBytes || i - g.back() >= kBwdGroupMax)) {
      g.push_back(i);
      used = 0;
    }
    used += b;
  }
  g.push_back(n);
  nseg.assign((size_t)n, 0);
  seg_rows.assign((size_t)n, 0);
  for (size_t k = 0; k + 1 < g.size(); ++k)
    for (int i = g[k]; i < g[k + 1]; ++i)
      fix_layout(in[i].width, in[i].height, (long long)p.n_fields * (g[k + 1] - g[k]), nseg[(size_t)i],
                 seg_rows[(size_t)i]);
}

// tm_backward / tm_backward_batch: validate, recompute the forward of every
// image in one batched pass (or take the last forward's intermediates), then
// run the adjoint over groups of images, each group in one launch per stage
// (the parameter gradients accumulate over all images).
tm_status backward_images(tm_ctx *c, int n, const tm_image *in, const tm_image *grad_out,
                          const tm_image *grad_in, float *grad_params, cudaStream_t s) {
  tm_status st;
  for (int i = 0; i < n; ++i) {
    char nm[40];
    snprintf(nm, sizeof nm, "in[%d]", i);
    if ((st = validate_image(c, &in[i], nm, true))) return st;
    snprintf(nm, sizeof nm, "grad_out[%d]", i);
    if ((st = validate_image(c, &grad_out[i], nm, false))) return st;
    if (grad_out[i].dtype != TM_F32) return fail(c, TM_EUNSUPPORTED, "grad_out[%d] must be float32", i);
    if (grad_out[i].width != in[i].width || grad_out[i].height != in[i].height)
      return fail(c, TM_EINVAL, "grad_out[%d] size differs from in[%d]", i, i);
    if (grad_in) {
      snprintf(nm, sizeof nm, "grad_in[%d]", i);
      if ((st = validate_image(c, &grad_in[i], nm, false))) return st;
      if (grad_in[i].dtype != TM_F32) return fail(c, TM_EUNSUPPORTED, "grad_in[%d] must be float32", i);
      if (grad_in[i].width != in[i].width || grad_in[i].height != in[i].height)
        return fail(c, TM_EINVAL, "grad_in[%d] size differs from in[%d]", i, i);
      if (overlap(&grad_in[i], &in[i]) || overlap(&grad_in[i], &grad_out[i]))
        return fail(c, TM_EINVAL, "grad_in[%d] overlaps in[%d] or grad_out[%d]", i, i, i);
    }
  }
  if (c->p.n_bins < 2 || c->hist_path == 2)
    return fail(c, TM_EUNSUPPORTED, "the backward runs on the fused path (n_bins >= 2)");
  if (c->p.flags & TM_FLAG_VAR_LINEAR)
    return fail(c, TM_EUNSUPPORTED, "the backward covers the log-domain variance (not TM_FLAG_VAR_LINEAR)");
  if ((st = ensure_device_info(c))) return st;
  std::vector<int> grp, nseg, seg_rows;
  backward_groups(c->p, n, in, grp, nseg, seg_rows);
  int gmax = 0;
  size_t need = 0;
  for (size_t k = 0; k + 1 < grp.size(); ++k) {
    size_t b = 0;
    for (int i = grp[k]; i < grp[k + 1]; ++i)
      b += backward_image_bytes(c->p, in[i].width, in[i].height, nseg[(size_t)i]);
    need = std::max(need, b);
    gmax = std::max(gmax, grp[k + 1] - grp[k]);
  }
  const size_t head = backward_header_bytes(gmax);
  need += head;
  std::vector<Job> jobs;
  int64_t launches = 0;
  if (c->bwd_reuse && c->fwd_valid && (int)c->fwd_in.size() == n && same_images(c->fwd_in, in, n)) {
    jobs = c->fwd_jobs;  // the last forward's intermediates of these images are in the workspace
  } else {
    st = forward_fused(c, n, in, in, s, false, false, &jobs);
    if (st == TM_EUNSUPPORTED) return fail(c, st, "fused sweep does not fit these fields");
    if (st) return st;
    launches = c->launches;
  }
  if ((st = grow_device(c, &c->bws, &c->bws_bytes, need))) return st;
  char *b = static_cast<char *>(c->bws);
  BwdAcc *accs = reinterpret_cast<BwdAcc *>(b);
  double *gsum = reinterpret_cast<double *>(b + align256(sizeof(BwdAcc) * gmax));
  char *desc = reinterpret_cast<char *>(gsum) + align256(sizeof(double) * kBwdParams);
  const int nf = c->p.n_fields;
  mark(c, s, -1);
  for (size_t k = 0; k + 1 < grp.size(); ++k) {
    const int i0 = grp[k], m = grp[k + 1] - i0;
    // the group's descriptors as one host block: BwdJob[m] then FixJob[m]
    std::vector<uint4> hdesc((sizeof(BwdJob) + sizeof(FixJob)) * (size_t)m / sizeof(uint4));  // 16-byte aligned
    unsigned char *hd = reinterpret_cast<unsigned char *>(hdesc.data());
    BwdJob *bj = reinterpret_cast<BwdJob *>(hd);
    FixJob *fj = reinterpret_cast<FixJob *>(hd + sizeof(BwdJob) * (size_t)m);
    BwdJob *dbj = reinterpret_cast<BwdJob *>(desc);
    FixJob *dfj = reinterpret_cast<FixJob *>(desc + sizeof(BwdJob) * (size_t)m);
    char *o = b + head;
    int pix = 0, inb = 0, tiles = 0, cols = 0;
    bool plain = true;  // float32 inputs and uint32 count planes throughout the group
    for (int r = 0; r < m; ++r) {
      const int i = i0 + r;
      const Job &J = jobs[(size_t)i];
      const int W = J.in.W, H = J.in.H;
      plain = plain && J.in.dtype == kF32 && J.cnt_wide == (1 << nf) - 1;
      const size_t N = (size_t)W * H, plane = (size_t)(W + 1) * (H + 1);
      BwdJob &B = bj[(size_t)r];
      B = BwdJob{};
      B.in = J.in;
      B.grad_out = to_image(&grad_out[i]);
      if (grad_in) B.grad_in = to_image(&grad_in[i]);
      B.st = J.st;
      B.q = J.q;
      B.s12 = reinterpret_cast<const longlong2 *>(J.s1);
      B.mom = J.mom;
      B.cnt = J.cnt;
      for (int f = 0; f < kMaxFields; ++f) B.cnt_off[f] = J.cnt_off[f];
      B.cnt_wide = J.cnt_wide;
      B.qbits = J.qbits;
      B.U = reinterpret_cast<float *>(o);
      B.V = reinterpret_cast<float *>(o + align256(4 * N * nf));
      B.gi_direct = reinterpret_cast<float *>(o + 2 * align256(4 * N * nf));
      char *iuv = o + 2 * align256(4 * N * nf) + align256(4 * N);
      B.IUV = reinterpret_cast<const longlong2 *>(iuv);
      B.acc = accs + r;
      B.b0 = pix;
      B.b0_in = inb;
      pix += bwd_pixel_blocks(W, H);
      inb += bwd_input_blocks(W, H);
      FixJob &F = fj[(size_t)r];
      F = FixJob{};
      F.u = B.U;
      F.v = B.V;
      F.amax = B.acc->amax;
      F.dst = reinterpret_cast<unsigned long long *>(iuv);
      F.scratch = reinterpret_cast<long long *>(iuv + align256(16 * plane * nf));
      F.scratch_stride = (long long)fix_integral_scratch_elems(W, H, 1, nseg[(size_t)i]);
      F.W = W;
      F.H = H;
      F.nseg = nseg[(size_t)i];
      F.seg_rows = seg_rows[(size_t)i];
      F.np = nf;
      F.b0_tile = tiles;
      F.b0_col = cols;
      tiles += fix_tile_blocks(W, F.nseg, nf);
      cols += fix_col_blocks(W, nf);
      for (int f = 0; f < nf; ++f) F.nmax[f] = window_max(dev_params(c->p, J.qbits), f, W, H);
      o += backward_image_bytes(c->p, W, H, nseg[(size_t)i]);
    }
    if (launch_backward_setup(hd, hdesc.size() * sizeof(uint4), desc, accs, m, gsum, k == 0, s) < 0)
      return fail(c, TM_EINVAL, "backward group descriptors exceed %d bytes", kBwdDescBytes);
    const DevParams P = dev_params(c->p, jobs[(size_t)i0].qbits);
    launches += 1 + launch_backward_pixel(P, dbj, m, pix, jobs[(size_t)i0].mom != nullptr, plain, gsum, s);
    mark(c, s, ST_BWD_PIXEL);
    launches += launch_fix_integrals(dfj, m, tiles, cols, s);
    mark(c, s, ST_BWD_ADJOINT);
    launches += launch_backward_input(P, dbj, m, inb, plain, gsum, k + 2 == grp.size() ? grad_params : nullptr, s);
    mark(c, s, ST_BWD_INPUT);
  }
  if ((st = check_launch(c, "backward launch"))) return st;
  c->launches = launches;
  return TM_OK;
}

}  // namespace

// Calls on a caller's stream share the workspace with the forwards that
// tm_forward_host_async runs on the context's forward stream: enter_caller
// orders stream s after the last of those forwards, leave_caller (given the
// call's status) marks the end of a successful call for the next one.
tm_status enter_caller(tm_ctx *c, cudaStream_t s) {
  if (c->fwd_pending) {
    TM_CUDA(c, cudaStreamWaitEvent(s, c->fwd_done, 0));
    c->fwd_pending = false;
  }
  return TM_OK;
}

tm_status leave_caller(tm_ctx *c, cudaStream_t s, tm_status st) {
  if (st || !c->fwd_stream) return st;
  TM_CUDA(c, cudaEventRecord(c->ext_done, s));
  c->ext_pending = true;
  return TM_OK;
}

// Whether the fused sweep fits image `in` under the context's fields.
bool sweep_fits(tm_ctx *c, const tm_image *in) {
  SweepPlan plan;
  return plan_sweep(dev_params(c->p, 0), in->width, in->height, 1,
                    std::min(c->smem_optin - 2048, (size_t)110 * 1024), 256, plan);
}

// Automatic path of a batch's images that fit the sweep: run the batched
// fused pass and the batched materialised pass twice each on them (without
// graphs) and time the second runs with events (synchronising the stream);
// 1 = fused, 2 = materialised. Both passes give bit-identical outputs (the
// counts are exact and the lookups share their arithmetic).
tm_status choose_batch_path(tm_ctx *c, int n, const tm_image *in, const tm_image *out, cudaStream_t s, int stats0,
                            int *choice) {
  cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
  for (auto &ev : e) TM_CUDA(c, cudaEventCreate(&ev));
  tm_status st = TM_OK;
  for (int rep = 0; rep < 2 && !st; ++rep) {
    cudaEventRecord(e[0], s);
    st = forward_fused(c, n, in, out, s, false);
    cudaEventRecord(e[1], s);
    if (!st) st = forward_materialised_batch(c, n, in, out, s, false, stats0);
    cudaEventRecord(e[2], s);
  }
  float ms_f = 0.f, ms_m = 0.f;
  if (!st) {
    cudaError_t r = cudaEventSynchronize(e[2]);
    if (r == cudaSuccess) r = cudaEventElapsedTime(&ms_f, e[0], e[1]);
    if (r == cudaSuccess) r = cudaEventElapsedTime(&ms_m, e[1], e[2]);
    if (r != cudaSuccess) st = cuda_fail(c, r, "timing the batch histogram paths");
  }
  for (auto &ev : e)
    if (ev) cudaEventDestroy(ev);
  if (st) return st;
  *choice = ms_f <= ms_m ? 1 : 2;
  return TM_OK;
}

// tm_forward_batch on validated arguments, n >= 1. Images whose fields do not
// fit the sweep take the materialised path; with TM_OPT_HIST_PATH = 0 the
// others take the path measured faster for this batch (cached per context by
// the images' sizes and dtype pairs). The images of each path run as one
// batched pass captured in a graph of its own.
tm_status forward_batch(tm_ctx *c, int n, const tm_image *in, const tm_image *out, cudaStream_t st) {
  tm_status s = ensure_device_info(c);
  if (s) return s;
  std::vector<tm_image> fin, fout, min_, mout;
  for (int i = 0; i < n; ++i) {
    bool fused = c->p.n_bins > 1 && c->hist_path != 2;
    if (fused && !sweep_fits(c, &in[i])) {
      if (c->hist_path == 1)
        return fail(c, TM_EUNSUPPORTED, "fused sweep does not fit image %d's fields (use the materialised path)", i);
      fused = false;
    }
    (fused ? fin : min_).push_back(in[i]);
    (fused ? fout : mout).push_back(out[i]);
  }
  if ((s = ensure_stats(c, n))) return s;
  if (!fin.empty() && c->hist_path == 0) {
    std::vector<std::tuple<int, int, int, int>> key;
    for (size_t i = 0; i < fin.size(); ++i)
      key.emplace_back((int)fin[i].width, (int)fin[i].height, (int)fin[i].dtype, (int)fout[i].dtype);
    auto it = c->batch_choice.find(key);
    if (it == c->batch_choice.end()) {
      int choice = 1;
      if ((s = choose_batch_path(c, (int)fin.size(), fin.data(), fout.data(), st, (int)min_.size(), &choice)))
        return s;
      it = c->batch_choice.emplace(key, choice).first;
    }
    if (it->second == 2) {
      min_.insert(min_.end(), fin.begin(), fin.end());
      mout.insert(mout.end(), fout.begin(), fout.end());
      fin.clear();
      fout.clear();
    }
  }
  int64_t total = 0;
  ++c->calls;
  if (!fin.empty()) {
    mark(c, st, -1);
    s = forward_fused(c, (int)fin.size(), fin.data(), fout.data(), st, true);
    if (s) return s;
    total += c->launches;
    mark(c, st, ST_BATCH);
  }
  if (!min_.empty()) {
    mark(c, st, -1);
    s = forward_materialised_batch(c, (int)min_.size(), min_.data(), mout.data(), st, true, (int)fin.size());
    if (s) return s;
    total += c->launches;
    mark(c, st, ST_BATCH_MAT);
  }
  c->launches = total;
  return TM_OK;
}

extern "C" {

void tm_params_default(tm_params *p) {
  if (!p) return;
  memset(p, 0, sizeof *p);
  p->n_bins = 5;
  p->n_fields = 5;
  const int half[5] = {1024, 512, 256, 128, 64};
  for (int f = 0; f < TM_MAX_FIELDS; ++f) {
    p->rx[f] = p->ry[f] = f < 5 ? half[f] : 0;
    p->eps[f] = 0.1f;
    p->alpha[f] = 1.0f;
  }
  p->ld_min = 0.f;
  p->ld_max = 1.f;
  p->sat = 0.6f;
  p->flags = 0;
}

tm_status tm_params_pyramid(tm_params *p, int32_t width, int32_t height, int32_t n_fields,
                            int32_t n_bins) {
  if (!p || width < 1 || height < 1 || n_fields < 1 || n_fields > TM_MAX_FIELDS || n_bins < 1 ||
      n_bins > TM_MAX_BINS)
    return fail(nullptr, TM_EINVAL, "tm_params_pyramid: bad argument");
  tm_params_default(p);
  p->n_fields = n_fields;
  p->n_bins = n_bins;
  for (int f = 0; f < TM_MAX_FIELDS; ++f) {
    p->rx[f] = f < n_fields ? std::min(width >> (f + 1), TM_MAX_RADIUS) : 0;
    p->ry[f] = f < n_fields ? std::min(height >> (f + 1), TM_MAX_RADIUS) : 0;
  }
  return TM_OK;
}

tm_status tm_create(const tm_params *params, tm_ctx **out) {
  if (!out) return fail(nullptr, TM_EINVAL, "tm_create: out is NULL");
  *out = nullptr;
  std::string why;
  tm_status s = validate_params(params, why);
  if (s) return fail(nullptr, s, "tm_create: %s", why.c_str());
  tm_ctx *c = new (std::nothrow) tm_ctx();
  if (!c) return fail(nullptr, TM_ENOMEM, "tm_create: out of host memory");
  c->p = *params;
  *out = c;
  return TM_OK;
}

void tm_destroy(tm_ctx *c) {
  if (!c) return;
  if (c->ws || c->mws || c->stats || c->rr_stats || c->stage || c->djobs || c->gdjobs || !c->graphs.empty() || c->mgraph ||
      c->hslot[0])
    cudaDeviceSynchronize();
  drop_graph(c);
  for (auto &call : c->marks)
    for (auto &m : call) cudaEventDestroy(m.e);
  for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
  if (c->ws) cudaFree(c->ws);
  if (c->bws) cudaFree(c->bws);
  if (c->stats) cudaFree(c->stats);
  if (c->rr_stats) cudaFree(c->rr_stats);
  if (c->stage) cudaFree(c->stage);
  for (int k = 0; k < 2; ++k) {
    for (void *b : {c->hslot[k], c->oslot[k]})
      if (b) cudaFree(b);
    for (cudaEvent_t e : {c->hslot_free[k], c->hslot_full[k], c->oslot_free[k], c->oslot_full[k]})
      if (e) cudaEventDestroy(e);
  }
  for (cudaEvent_t e : {c->fwd_done, c->ext_done})
    if (e) cudaEventDestroy(e);
  for (cudaStream_t q : {c->copy_stream, c->fwd_stream})
    if (q) cudaStreamDestroy(q);
  if (c->djobs) cudaFree(c->djobs);
  if (c->ditems) cudaFree(c->ditems);
  if (c->graph_stream) cudaStreamDestroy(c->graph_stream);
  for (cudaStream_t q : {c->sweep_stream, c->int_stream})
    if (q) cudaStreamDestroy(q);
  for (cudaEvent_t e : {c->ov_fork, c->ov_sweep, c->ov_int})
    if (e) cudaEventDestroy(e);
  if (c->gdjobs) cudaFree(c->gdjobs);
  if (c->gditems) cudaFree(c->gditems);
  if (c->mws) cudaFree(c->mws);
  if (c->mdjobs) cudaFree(c->mdjobs);
  delete c;
}

const char *tm_last_error(const tm_ctx *c) {
  if (c) return c->err.c_str();
  std::lock_guard<std::mutex> g(g_create_mu);
  return g_create_err.c_str();
}

const char *tm_status_string(tm_status s) {
  switch (s) {
    case TM_OK: return "TM_OK";
    case TM_EINVAL: return "TM_EINVAL";
    case TM_ENOMEM: return "TM_ENOMEM";
    case TM_ECUDA: return "TM_ECUDA";
    case TM_EUNSUPPORTED: return "TM_EUNSUPPORTED";
    case TM_ETIMEOUT: return "TM_ETIMEOUT";
    case TM_ESTATE: return "TM_ESTATE";
  }
  return "TM_UNKNOWN";
}

tm_status tm_forward(tm_ctx *c, const tm_image *in, const tm_image *out, void *stream) {
  if (!c) return fail(nullptr, TM_EINVAL, "tm_forward: ctx is NULL");
  tm_status s;
  if ((s = validate_image(c, in, "in", true))) return s;
  if ((s = validate_image(c, out, "out", false))) return s;
  if (in->width != out->width || in->height != out->height)
    return fail(c, TM_EINVAL, "in is %dx%d but out is %dx%d", in->width, in->height, out->width,
                out->height);
  if (overlap(in, out)) return fail(c, TM_EINVAL, "in and out overlap");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((s = enter_caller(c, st))) return s;
  return leave_caller(c, st, forward_device(c, in, out, st));
}

tm_status tm_forward_host(tm_ctx *c, const tm_image *in, const tm_image *out, void *stream) {
  if (!c) return fail(nullptr, TM_EINVAL, "tm_forward_host: ctx is NULL");
  tm_status s;
  if ((s = validate_image(c, in, "in", true))) return s;
  if ((s = validate_image(c, out, "out", false))) return s;
  if (in->width != out->width || in->height != out->height)
    return fail(c, TM_EINVAL, "in and out sizes differ");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int W = in->width, H = in->height;
  const size_t in_row = 3 * (size_t)W * elem_size(in->dtype);
  const size_t out_row = 3 * (size_t)W * elem_size(out->dtype);
  const size_t in_bytes = align256(in_row * H), out_bytes = align256(out_row * H);
  if (c->stage_bytes < in_bytes + out_bytes) {
    if (c->stage) {
      TM_CUDA(c, cudaDeviceSynchronize());
      cudaFree(c->stage);
      c->stage = nullptr;
      c->stage_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&c->stage, in_bytes + out_bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(c, TM_ENOMEM, "staging buffer: %s", cudaGetErrorString(e));
    }
    c->stage_bytes = in_bytes + out_bytes;
  }
  tm_image din = *in, dout = *out;
  din.data = c->stage;
  din.pitch = 3LL * W;
  // A page-locked (pinned or registered) output buffer is addressable from
  // the device: the last kernel then stores the result straight into it over
  // the host link, overlapping the download with its own work instead of
  // following it with a copy. Pageable output goes through the staging copy.
  void *out_dev = nullptr;
  {
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, out->data) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
        pa.devicePointer != nullptr)
      out_dev = pa.devicePointer;
    cudaGetLastError();
  }
  if (out_dev) {
    dout.data = out_dev;
  } else {
    dout.data = static_cast<char *>(c->stage) + in_bytes;
    dout.pitch = 3LL * W;
  }
  if ((s = enter_caller(c, st))) return s;
  TM_CUDA(c, cudaMemcpy2DAsync(din.data, in_row, in->data, in->pitch * elem_size(in->dtype), in_row,
                               H, cudaMemcpyHostToDevice, st));
  if ((s = leave_caller(c, st, forward_device(c, &din, &dout, st)))) return s;
  if (!out_dev)
    TM_CUDA(c, cudaMemcpy2DAsync(out->data, out->pitch * elem_size(out->dtype), dout.data, out_row,
                                 out_row, H, cudaMemcpyDeviceToHost, st));
  TM_CUDA(c, cudaStreamSynchronize(st));
  return TM_OK;
}

static bool page_locked(const void *p) {
  cudaPointerAttributes pa{};
  const bool r = cudaPointerGetAttributes(&pa, p) == cudaSuccess && pa.type == cudaMemoryTypeHost;
  cudaGetLastError();
  return r;
}

// Two device buffers of at least `bytes` each (grown after the device is idle).
static tm_status grow_slots(tm_ctx *c, void **slot, size_t *have, size_t bytes, const char *what) {
  if (*have >= bytes) return TM_OK;
  if (slot[0]) TM_CUDA(c, cudaDeviceSynchronize());  // both slots may still be in use
  *have = 0;
  for (int k = 0; k < 2; ++k) {
    if (slot[k]) cudaFree(slot[k]);
    slot[k] = nullptr;
  }
  for (int k = 0; k < 2; ++k) {
    cudaError_t e = cudaMalloc(&slot[k], bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(c, TM_ENOMEM, "%s slots: %s", what, cudaGetErrorString(e));
    }
  }
  *have = bytes;
  return TM_OK;
}

tm_status tm_forward_host_async(tm_ctx *c, const tm_image *in, const tm_image *out, void *stream) {
  if (!c) return fail(nullptr, TM_EINVAL, "tm_forward_host_async: ctx is NULL");
  tm_status s;
  if ((s = validate_image(c, in, "in", true))) return s;
  if ((s = validate_image(c, out, "out", false))) return s;
  if (in->width != out->width || in->height != out->height)
    return fail(c, TM_EINVAL, "in and out sizes differ");
  if (!page_locked(in->data) || !page_locked(out->data))
    return fail(c, TM_EINVAL, "tm_forward_host_async needs page-locked in and out (use tm_forward_host)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int W = in->width, H = in->height;
  const size_t in_row = 3 * (size_t)W * elem_size(in->dtype);
  const size_t out_row = 3 * (size_t)W * elem_size(out->dtype);
  if ((s = grow_slots(c, c->hslot, &c->hslot_bytes, align256(in_row * H), "input"))) return s;
  if ((s = grow_slots(c, c->oslot, &c->oslot_bytes, align256(out_row * H), "output"))) return s;
  for (cudaStream_t *q : {&c->copy_stream, &c->fwd_stream})
    if (!*q) TM_CUDA(c, cudaStreamCreateWithFlags(q, cudaStreamNonBlocking));
  for (int k = 0; k < 2; ++k)
    for (cudaEvent_t *e : {&c->hslot_free[k], &c->hslot_full[k], &c->oslot_free[k], &c->oslot_full[k]})
      if (!*e) TM_CUDA(c, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  for (cudaEvent_t *e : {&c->fwd_done, &c->ext_done})
    if (!*e) TM_CUDA(c, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  const int k = c->hslot_next;
  c->hslot_next ^= 1;
  // upload k: after the forward that last read input slot k (a wait on an
  // event never recorded returns at once)
  TM_CUDA(c, cudaStreamWaitEvent(c->copy_stream, c->hslot_free[k], 0));
  TM_CUDA(c, cudaMemcpy2DAsync(c->hslot[k], in_row, in->data, in->pitch * elem_size(in->dtype), in_row, H,
                               cudaMemcpyHostToDevice, c->copy_stream));
  TM_CUDA(c, cudaEventRecord(c->hslot_full[k], c->copy_stream));
  // forward k: after upload k, the download that last read output slot k and
  // the last call on a caller's stream; it does not wait for download k-1
  const cudaStream_t fs = c->fwd_stream;
  TM_CUDA(c, cudaStreamWaitEvent(fs, c->hslot_full[k], 0));
  TM_CUDA(c, cudaStreamWaitEvent(fs, c->oslot_free[k], 0));
  if (c->ext_pending) {
    TM_CUDA(c, cudaStreamWaitEvent(fs, c->ext_done, 0));
    c->ext_pending = false;
  }
  tm_image din = *in, dout = *out;
  din.data = c->hslot[k];
  din.pitch = 3LL * W;
  dout.data = c->oslot[k];
  dout.pitch = 3LL * W;
  if ((s = forward_device(c, &din, &dout, fs))) return s;
  TM_CUDA(c, cudaEventRecord(c->hslot_free[k], fs));
  TM_CUDA(c, cudaEventRecord(c->oslot_full[k], fs));
  TM_CUDA(c, cudaEventRecord(c->fwd_done, fs));
  c->fwd_pending = true;
  // download k on the caller's stream, so that synchronising it covers the
  // upload, the forward and the download of every call made on it
  TM_CUDA(c, cudaStreamWaitEvent(st, c->oslot_full[k], 0));
  TM_CUDA(c, cudaMemcpy2DAsync(out->data, out->pitch * elem_size(out->dtype), c->oslot[k], out_row, out_row, H,
                               cudaMemcpyDeviceToHost, st));
  TM_CUDA(c, cudaEventRecord(c->oslot_free[k], st));
  return TM_OK;
}

tm_status tm_forward_batch(tm_ctx *c, int32_t n, const tm_image *in, const tm_image *out,
                           void *stream) {
  if (!c) return fail(nullptr, TM_EINVAL, "tm_forward_batch: ctx is NULL");
  if (n < 0) return fail(c, TM_EINVAL, "n = %d < 0", n);
  if (n == 0) { c->launches = 0; return TM_OK; }
  if (!in || !out) return fail(c, TM_EINVAL, "descriptor arrays are NULL");
  for (int i = 0; i < n; ++i) {
    tm_status s;
    char nm[32];
    snprintf(nm, sizeof nm, "in[%d]", i);
    if ((s = validate_image(c, &in[i], nm, true))) return s;
    snprintf(nm, sizeof nm, "out[%d]", i);
    if ((s = validate_image(c, &out[i], nm, false))) return s;
    if (in[i].width != out[i].width || in[i].height != out[i].height)
      return fail(c, TM_EINVAL, "image %d: in and out sizes differ", i);
    if (overlap(&in[i], &out[i])) return fail(c, TM_EINVAL, "image %d: in and out overlap", i);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  tm_status s;
  if ((s = enter_caller(c, st))) return s;
  return leave_caller(c, st, forward_batch(c, n, in, out, st));
}

tm_status tm_backward(tm_ctx *c, const tm_image *in, const tm_image *grad_out,
                      const tm_image *grad_in, float *grad_params, void *stream) {
  if (!c) return fail(nullptr, TM_EINVAL, "tm_backward: ctx is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  tm_status st;
  if ((st = enter_caller(c, s))) return st;
  return leave_caller(c, s, backward_images(c, 1, in, grad_out, grad_in, grad_params, s));
}

tm_status tm_backward_batch(tm_ctx *c, int32_t n, const tm_image *in, const tm_image *grad_out,
                            const tm_image *grad_in, float *grad_params, void *stream) {
  if (!c) return fail(nullptr, TM_EINVAL, "tm_backward_batch: ctx is NULL");
  if (n < 0) return fail(c, TM_EINVAL, "n = %d < 0", n);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n == 0) {
    c->launches = 0;
    if (grad_params) TM_CUDA(c, cudaMemsetAsync(grad_params, 0, sizeof(float) * (3 + 2 * c->p.n_fields), s));
    return TM_OK;
  }
  if (!in || !grad_out) return fail(c, TM_EINVAL, "descriptor arrays are NULL");
  tm_status st;
  if ((st = enter_caller(c, s))) return st;
  return leave_caller(c, s, backward_images(c, n, in, grad_out, grad_in, grad_params, s));
}

tm_status tm_integral_image(const int32_t *q, int32_t width, int32_t height, int64_t *s1,
                            int64_t *s2, void *stream) {
  if (!q || !s1 || !s2) return fail(nullptr, TM_EINVAL, "tm_integral_image: NULL pointer");
  if (width < 1 || height < 1) return fail(nullptr, TM_EINVAL, "tm_integral_image: bad size");
  if ((long long)width * height > (1LL << 31) - 1)
    return fail(nullptr, TM_EINVAL, "tm_integral_image: more than 2^31-1 elements");
  if (s1 == s2) return fail(nullptr, TM_EINVAL, "tm_integral_image: s1 == s2");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Job J{};
  J.in.W = width;
  J.in.H = height;
  J.q = const_cast<int32_t *>(q);
  J.s1 = reinterpret_cast<long long *>(s1);
  J.s2 = reinterpret_cast<long long *>(s2);
  integral_layout(width, height, SIZE_MAX, J.nseg, J.seg_rows);
  const size_t seg_bytes = 8 * integral_scratch_elems(width, height, J.nseg);
  void *scr = nullptr;
  cudaError_t e = cudaMallocAsync(&scr, align256(sizeof(Job)) + seg_bytes, st);
  if (e != cudaSuccess) { cudaGetLastError(); return fail(nullptr, TM_ENOMEM, "tm_integral_image: scratch"); }
  J.segtot = reinterpret_cast<long long *>(static_cast<char *>(scr) + align256(sizeof(Job)));
  put_jobs(&J, 1, static_cast<Job *>(scr), st);
  launch_integral_jobs(static_cast<Job *>(scr), 1, integral_tile_blocks(width, J.nseg),
                       integral_col_blocks(width), st);
  e = cudaGetLastError();
  cudaFreeAsync(scr, st);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "tm_integral_image");
  return TM_OK;
}

tm_status tm_integral_histogram(const uint8_t *bins, int32_t width, int32_t height,
                                int32_t n_bins, uint32_t *hk, void *stream) {
  if (!bins || !hk) return fail(nullptr, TM_EINVAL, "tm_integral_histogram: NULL pointer");
  if (width < 1 || height < 1) return fail(nullptr, TM_EINVAL, "tm_integral_histogram: bad size");
  if (n_bins < 1 || n_bins > TM_MAX_BINS)
    return fail(nullptr, TM_EINVAL, "tm_integral_histogram: n_bins outside 1..256");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void *scr = nullptr;
  size_t bytes = hist_scratch_bytes(width, height, n_bins);
  cudaError_t e = cudaMallocAsync(&scr, bytes, st);
  if (e != cudaSuccess) { cudaGetLastError(); return fail(nullptr, TM_ENOMEM, "tm_integral_histogram: scratch"); }
  launch_integral_histogram(bins, width, height, n_bins, false, hk, scr, st);
  e = cudaGetLastError();
  cudaFreeAsync(scr, st);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "tm_integral_histogram");
  return TM_OK;
}

tm_status tm_set_debug(tm_ctx *c, int32_t enable) {
  if (!c) return fail(nullptr, TM_EINVAL, "tm_set_debug: ctx is NULL");
  c->debug = enable ? 1 : 0;
  return TM_OK;
}

tm_status tm_debug_size(tm_ctx *c, int32_t what, size_t *bytes) {
  if (!c || !bytes) return fail(c, TM_EINVAL, "tm_debug_size: NULL argument");
  if (c->last_W == 0) return fail(c, TM_ESTATE, "no forward has run on this context");
  const size_t N = (size_t)c->last_W * c->last_H, s = c->p.n_fields;
  switch (what) {
    case TM_DBG_RANGE: *bytes = 8; break;
    case TM_DBG_THRESHOLDS: *bytes = 4 * (size_t)(c->p.n_bins - 1); break;
    case TM_DBG_BINS: *bytes = N; break;
    case TM_DBG_Q: *bytes = 4 * N; break;
    case TM_DBG_COUNTS: case TM_DBG_SIGMA2: case TM_DBG_WEIGHT: case TM_DBG_LF: *bytes = 4 * N * s; break;
    case TM_DBG_L: *bytes = 4 * N; break;
    case TM_DBG_QSHIFT: *bytes = 4; break;
    default: return fail(c, TM_EINVAL, "unknown debug export %d", what);
  }
  return TM_OK;
}

tm_status tm_debug_export(tm_ctx *c, int32_t what, void *dst, size_t bytes, void *stream) {
  size_t need = 0;
  tm_status s = tm_debug_size(c, what, &need);
  if (s) return s;
  if (!dst) return fail(c, TM_EINVAL, "dst is NULL");
  if (bytes < need) return fail(c, TM_EINVAL, "dst holds %zu bytes, %zu needed", bytes, need);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((s = enter_caller(c, st))) return s;
  const void *src = nullptr;
  switch (what) {
    case TM_DBG_RANGE: src = &(c->last_stats ? c->last_stats : c->stats)->imin; break;
    case TM_DBG_THRESHOLDS: src = (c->last_stats ? c->last_stats : c->stats)->thr; break;
    case TM_DBG_BINS: src = c->bins; break;
    case TM_DBG_Q: src = c->q; break;
    case TM_DBG_QSHIFT: {
      int32_t v = c->last_q;
      TM_CUDA(c, cudaMemcpyAsync(dst, &v, 4, cudaMemcpyHostToDevice, st));
      TM_CUDA(c, cudaStreamSynchronize(st));
      return TM_OK;
    }
    default:
      if (!c->dbg.l) return fail(c, TM_ESTATE, "debug planes were not kept (tm_set_debug before forward)");
      src = what == TM_DBG_COUNTS ? (const void *)c->dbg.cnt
            : what == TM_DBG_SIGMA2 ? (const void *)c->dbg.sigma2
            : what == TM_DBG_WEIGHT ? (const void *)c->dbg.weight
            : what == TM_DBG_LF ? (const void *)c->dbg.lf
                                : (const void *)c->dbg.l;
  }
  if (need) TM_CUDA(c, cudaMemcpyAsync(dst, src, need, cudaMemcpyDeviceToDevice, st));
  return leave_caller(c, st, TM_OK);
}

tm_status tm_set_option(tm_ctx *c, int32_t key, int64_t value) {
  if (!c) return fail(nullptr, TM_EINVAL, "tm_set_option: ctx is NULL");
  if (key == TM_OPT_STAGE_TIMING) {
    c->stage_timing = value ? 1 : 0;
    return TM_OK;
  }
  if (key == TM_OPT_REUSE_RANGE) {
    c->reuse_range = value ? 1 : 0;
    c->rr_valid = 0;
    return TM_OK;
  }
  if (key == TM_OPT_BACKWARD_REUSE) {
    if (c->bwd_reuse != (value ? 1 : 0)) {
      drop_graph(c);  // the cached batch graph keeps (or not) the window moments
      c->fwd_valid = false;
    }
    c->bwd_reuse = value ? 1 : 0;
    return TM_OK;
  }
  if (key == TM_OPT_SWEEP_TILES) {
    if (value < 0 || value > (1 << 20)) return fail(c, TM_EINVAL, "TM_OPT_SWEEP_TILES value %lld", (long long)value);
    c->sweep_tiles = (int)value;
    drop_graph(c);
    return TM_OK;
  }
  if (key == TM_OPT_SWEEP_WIDTH) {
    if (value != 0 && value != 256 && value != 512)
      return fail(c, TM_EINVAL, "TM_OPT_SWEEP_WIDTH value %lld (0, 256 or 512)", (long long)value);
    if (c->sweep_width != (int)value) {
      drop_graph(c);
      c->path_choice.clear();  // the timed path choices saw the other width
      c->batch_choice.clear();
    }
    c->sweep_width = (int)value;
    return TM_OK;
  }
  if (key == TM_OPT_HIST_PATH) {
    if (value < 0 || value > 2) return fail(c, TM_EINVAL, "TM_OPT_HIST_PATH value %lld", (long long)value);
    c->hist_path = (int)value;
    c->path_choice.clear();
    c->batch_choice.clear();
    return TM_OK;
  }
  return fail(c, TM_EINVAL, "unknown option %d", key);
}

int64_t tm_last_launch_count(const tm_ctx *c) { return c ? c->launches : 0; }

int32_t tm_stage_times(tm_ctx *c, float *ms, const char **names, int32_t cap) {
  if (!c || !ms || !names || cap < 0) {
    fail(c, TM_EINVAL, "tm_stage_times: bad argument");
    return -1;
  }
  for (auto &call : c->marks) {
    if (call.empty()) continue;
    bool ok = true;
    for (auto &m : call) ok = ok && cudaEventSynchronize(m.e) == cudaSuccess;  // marks on several streams
    if (!ok) {
      cudaGetLastError();
      fail(c, TM_ECUDA, "tm_stage_times: event synchronisation failed");
      return -1;
    }
    for (size_t i = 1; i < call.size(); ++i) {
      float t = 0.f;
      const size_t from = call[i].from >= 0 ? (size_t)call[i].from : i - 1;
      if (call[i].stage >= 0 && cudaEventElapsedTime(&t, call[from].e, call[i].e) == cudaSuccess)
        c->stage_ms[call[i].stage] += t;
    }
    for (auto &m : call) c->event_pool.push_back(m.e);
  }
  c->marks.clear();
  int32_t n = 0;
  for (int st = 0; st < ST_COUNT && n < cap; ++st)
    if (c->stage_ms[st] > 0.0) {
      ms[n] = (float)c->stage_ms[st];
      names[n] = kStageNames[st];
      ++n;
    }
  for (double &v : c->stage_ms) v = 0.0;
  return n;
}

}  // extern "C"
