// tm_lookup.cu -- per-pixel multi-field lookup, tone curve, fusion and colour.
//
// One thread per pixel. The Eq. 1 numerator of every field comes either from
// the materialised cumulative integral histogram (C_b = sum_{k < b} H_k, one
// box sum of the plane of the pixel's own bin, Eq. 9) or from the count
// planes written by the fused sweep. The window sums of q and q^2 are box sums
// of their integral images (Eq. 6), giving the exact window variance (Eq. 10);
// then Eq. 2, Eq. 4, the fusion of Eq. 3 and the colour restoration of Eq. 12.
// The fields are evaluated in one pass instead of the paper's per-scale loop
// (Section III-A).
#include "tm_kernels.cuh"

namespace tmk {
namespace {

// Running sums of the fusion of Eq. 3 over the fields.
struct Fusion {
  float wsum = 0.f, acc = 0.f, mean = 0.f;
};

// Field f of pixel (x, y) with Eq. 1 numerator cnt: Eq. 2 and Eq. 4 folded
// into the Eq. 3 sums (the same arithmetic as fuse_fields, one field at a
// time, so no per-field state is kept).
// mom (or null): receives the window's variance and mean of lhat for the
// backward (inv_scale = 2^-Q). kPlain: no debug planes and no literal area,
// and moments only under kMom (the other paths are then not compiled in);
// kSmall as for window_variance.
template <bool kPlain = false, bool kMom = false, int kSmall = -1>
__device__ __forceinline__ void fold_field(const DevParams &P, int f, int x, int y, int W, int H,
                                           unsigned cnt, const longlong2 *__restrict__ s12, int qbits,
                                           float inv_scale2, Fusion &fu, const DebugPlanes &dbg,
                                           float2 *mom = nullptr, float inv_scale = 0.f) {
  const WinMoments m = window_moments<!kPlain, kSmall>(P, f, x, y, W, H, s12, qbits, inv_scale2);
  const float rarea = m.rarea, var = m.var;
  if (kPlain ? kMom : mom != nullptr)
    mom[(size_t)f * W * H + (size_t)y * W + x] = make_float2(var, window_mean(m.q1, rarea, inv_scale));
  const float Pf = (float)cnt * rarea;                                  // Eq. 1
  const float Lf = fmaf(P.ld_max - P.ld_min, Pf, P.ld_min);             // Eq. 2
  const float Wf = __fdividef(P.alpha[f] * var, var + P.eps[f]);       // Eq. 4
  fu.wsum += Wf;
  fu.acc = fmaf(Wf, Lf, fu.acc);
  fu.mean += Lf;
  if (!kPlain && dbg.l) {
    const long long N = (long long)W * H, pix = (long long)y * W + x;
    dbg.cnt[f * N + pix] = cnt;
    dbg.sigma2[f * N + pix] = var;
    dbg.weight[f * N + pix] = Wf;
    dbg.lf[f * N + pix] = Lf;
  }
}

// Eq. 3 and Eq. 12 for one pixel from the folded sums. kDt: the dtype of
// both images when known at compile time (-1: read from the descriptors).
template <bool kPlain = false, int kDt = -1>
__device__ __forceinline__ void finish_pixel(const Image &in, const Image &out, const DevParams &P,
                                             int x, int y, const Fusion &fu, const DebugPlanes &dbg) {
  const float L = fu.wsum > 0.f ? __fdividef(fu.acc, fu.wsum)
                                : __fdividef(fu.mean, (float)P.n_fields);  // Eq. 3
  float r, g, b;
  load_rgb<kDt>(in, x, y, r, g, b);
  const float inv_i = __fdividef(1.f, luminance(r, g, b));
  store_rgb<kDt>(out, x, y, restore_channel(r, inv_i, P.sat, L), restore_channel(g, inv_i, P.sat, L),
                 restore_channel(b, inv_i, P.sat, L), (P.flags & kFlagSrgb) != 0);
  if (!kPlain && dbg.l) dbg.l[(long long)y * in.W + x] = L;
}

// Eight blocks per SM (32 registers, a few spilled at five fields and more)
// keep more corner loads in flight: at 12 MP with the five-field pyramid this
// ran 0.48 ms against 0.60 ms at five blocks per SM. kPlain: no debug planes
// and no literal area; kDt: the dtype of both images when they share it (-1:
// read from the descriptors).
template <int NF, bool kPlain, int kDt>
__global__ void __launch_bounds__(256, 8)
    k_lookup_materialised(Image in, Image out, DevParams P, const uint8_t *__restrict__ bins,
                          const unsigned *__restrict__ cplanes, const longlong2 *__restrict__ s12,
                          DebugPlanes dbg) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int W = in.W, H = in.H;
  if (x >= W || y >= H) return;
  const long long W1 = (long long)W + 1;
  const long long plane = W1 * ((long long)H + 1);
  // Eq. 1 numerator: box sum of C_t, t = b (strict) or b + 1 (inclusive);
  // C_0 = 0 and C_n is the whole (clipped) window
  const int t = bins[(long long)y * W + x] + ((P.flags & kFlagCdfIncl) ? 1 : 0);
  const unsigned *C = t > 0 && t < P.n_bins ? cplanes + (long long)(t - 1) * plane : nullptr;
  const float inv_scale2 = ldexpf(1.f, -2 * P.qbits);
  Fusion fu;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    unsigned cnt = 0u;
    Win w = window_of(P, f, x, y, W, H);
    if (C)
      cnt = __ldg(C + (long long)(w.y1 + 1) * W1 + w.x1 + 1) - __ldg(C + (long long)(w.y1 + 1) * W1 + w.x0) -
            __ldg(C + (long long)w.y0 * W1 + w.x1 + 1) + __ldg(C + (long long)w.y0 * W1 + w.x0);
    else if (t >= P.n_bins)
      cnt = (unsigned)((w.x1 - w.x0 + 1) * (w.y1 - w.y0 + 1));
    fold_field<kPlain>(P, f, x, y, W, H, cnt, s12, P.qbits, inv_scale2, fu, dbg);
  }
  finish_pixel<kPlain, kDt>(in, out, P, x, y, fu, dbg);
}

// Lookup from the sweep's count planes, over a batch of jobs: block ->
// (image, 32 x 8 pixel tile). NF = number of fields, so the field loop is
// straight-line code and the loads of all fields can be issued together.
// Eight blocks per SM (32 registers) keep more of those loads in flight.
// kPlain: no job has debug planes, every count plane is uint32, the literal
// area is off and every window is small (P.small_win; the window variance
// then takes its 32-bit conversions); then kMom: every job keeps its window
// moments (else
// none does). kDt: the dtype of every job's input and output when they all
// share one (-1: read from the descriptors). Specialising drops the paths a
// launch does not take: the compiler would otherwise predicate some of them
// into every pixel (at 12 MP the plain float32 variant took 0.191 ms against
// 0.247).
template <int NF, bool kPlain, int kDt, bool kMom = false>
__global__ void __launch_bounds__(256, 8) k_lookup_counts(DevParams P, const Job *__restrict__ jobs, int njobs) {
  const int j = find_job(jobs, njobs, kStLook, blockIdx.x);
  const Job &J = jobs[j];
  const int lb = blockIdx.x - J.b0[kStLook];
  const int W = J.in.W, H = J.in.H;
  const int bx = (W + 31) / 32;
  const int x = (lb % bx) * 32 + (threadIdx.x & 31);
  const int y = (lb / bx) * 8 + (threadIdx.x >> 5);
  if (x >= W || y >= H) return;
  const long long pix = (long long)y * W + x;
  const float inv_scale = ldexpf(1.f, -J.qbits);  // Q is per image
  const float inv_scale2 = inv_scale * inv_scale;
  Fusion fu;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const unsigned cnt = kPlain ? __ldg(reinterpret_cast<const unsigned *>(J.cnt + J.cnt_off[f]) + pix)
                                : load_count(J, f, pix);
    fold_field<kPlain, kMom, kPlain ? 1 : -1>(P, f, x, y, W, H, cnt, reinterpret_cast<const longlong2 *>(J.s1),
                                              J.qbits, inv_scale2, fu, J.dbg, J.mom, inv_scale);
  }
  finish_pixel<kPlain, kDt>(J.in, J.out, P, x, y, fu, J.dbg);
}

}  // namespace

template <bool kPlain, int kDt>
static void launch_mat(const Image &in, const Image &out, const DevParams &P, const uint8_t *bins,
                       const uint32_t *cplanes, const longlong2 *S12, const DebugPlanes &dbg, cudaStream_t s) {
  dim3 block(32, 8), grid((in.W + 31) / 32, (in.H + 7) / 8);
  switch (P.n_fields) {
#define TM_LOOKUP_MAT(nf)                                                                                       \
  case nf:                                                                                                      \
    k_lookup_materialised<nf, kPlain, kDt><<<grid, block, 0, s>>>(in, out, P, bins, cplanes, S12, dbg);        \
    break;
    TM_LOOKUP_MAT(1) TM_LOOKUP_MAT(2) TM_LOOKUP_MAT(3) TM_LOOKUP_MAT(4) TM_LOOKUP_MAT(5) TM_LOOKUP_MAT(6)
    TM_LOOKUP_MAT(7)
    default: k_lookup_materialised<8, kPlain, kDt><<<grid, block, 0, s>>>(in, out, P, bins, cplanes, S12, dbg); break;
#undef TM_LOOKUP_MAT
  }
}

int launch_lookup_materialised(const Image &in, const Image &out, const DevParams &P,
                               const uint8_t *bins, const uint32_t *cplanes, const int64_t *s12,
                               const DebugPlanes &dbg, cudaStream_t s) {
  const longlong2 *S12 = reinterpret_cast<const longlong2 *>(s12);
  const int dt = in.dtype == out.dtype ? in.dtype : -1;
  if (dbg.l || (P.flags & kFlagAreaLit))
    launch_mat<false, -1>(in, out, P, bins, cplanes, S12, dbg, s);
  else if (dt == kF32)
    launch_mat<true, kF32>(in, out, P, bins, cplanes, S12, dbg, s);
  else if (dt == kF16)
    launch_mat<true, kF16>(in, out, P, bins, cplanes, S12, dbg, s);
  else
    launch_mat<true, -1>(in, out, P, bins, cplanes, S12, dbg, s);
  return 1;
}

int lookup_blocks(int W, int H) { return ((W + 31) / 32) * ((H + 7) / 8); }

template <bool kPlain, int kDt, bool kMom = false>
static void launch_counts(const DevParams &P, const Job *jobs, int njobs, int blocks, cudaStream_t s) {
  switch (P.n_fields) {
    case 1: k_lookup_counts<1, kPlain, kDt, kMom><<<blocks, 256, 0, s>>>(P, jobs, njobs); break;
    case 2: k_lookup_counts<2, kPlain, kDt, kMom><<<blocks, 256, 0, s>>>(P, jobs, njobs); break;
    case 3: k_lookup_counts<3, kPlain, kDt, kMom><<<blocks, 256, 0, s>>>(P, jobs, njobs); break;
    case 4: k_lookup_counts<4, kPlain, kDt, kMom><<<blocks, 256, 0, s>>>(P, jobs, njobs); break;
    case 5: k_lookup_counts<5, kPlain, kDt, kMom><<<blocks, 256, 0, s>>>(P, jobs, njobs); break;
    case 6: k_lookup_counts<6, kPlain, kDt, kMom><<<blocks, 256, 0, s>>>(P, jobs, njobs); break;
    case 7: k_lookup_counts<7, kPlain, kDt, kMom><<<blocks, 256, 0, s>>>(P, jobs, njobs); break;
    default: k_lookup_counts<8, kPlain, kDt, kMom><<<blocks, 256, 0, s>>>(P, jobs, njobs); break;
  }
}

int launch_lookup_counts(const DevParams &P, const Job *jobs, int njobs, int blocks, bool plain, bool mom,
                         int dtype, cudaStream_t s) {
  if (!plain || !P.small_win || (P.flags & kFlagAreaLit) || (mom && dtype != kF32))
    launch_counts<false, -1>(P, jobs, njobs, blocks, s);
  else if (mom)
    launch_counts<true, kF32, true>(P, jobs, njobs, blocks, s);
  else if (dtype == kF32)
    launch_counts<true, kF32>(P, jobs, njobs, blocks, s);
  else if (dtype == kF16)
    launch_counts<true, kF16>(P, jobs, njobs, blocks, s);
  else
    launch_counts<true, -1>(P, jobs, njobs, blocks, s);
  return 1;
}

}  // namespace tmk
