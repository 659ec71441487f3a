// tm_common.cuh -- device-side definitions shared by the tone-mapping kernels.
//
// Pixel layout: interleaved RGB (HWC) with a row pitch in elements.
// Workspace planes: (H+1) x (W+1) row-major with a zero first row and column,
// so that the window [x0, x1] x [y0, y1] sums to
//   I(y1+1, x1+1) - I(y1+1, x0) - I(y0, x1+1) + I(y0, x0)      (Eq. 6, Eq. 9)
// i.e. Algorithm 1's corners x - (r + 1) and x + r shifted by one.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace tmk {

constexpr int kMaxFields = 8;
constexpr int kMaxBins = 256;
constexpr float kLumFloor = 1e-30f;

enum Dtype { kF32 = 0, kF16 = 1, kU8 = 2 };

// Kernel-argument copy of the operator parameters (paper notation).
struct DevParams {
  int n_bins;               // n (Eq. 7)
  int n_fields;             // s (Eq. 3)
  int rx[kMaxFields];       // half-widths (Algorithm 1 s_j.x)
  int ry[kMaxFields];       // half-heights (Algorithm 1 s_j.y)
  float eps[kMaxFields];    // epsilon of Eq. 4
  float alpha[kMaxFields];  // field weight multiplying Eq. 4
  float ld_min, ld_max;     // display range of Eq. 2
  float sat;                // Eq. 12
  int qbits;                // Q: q = round(2^Q lhat) - 2^(Q-1)
  int flags;                // TM_FLAG_* reading variants
  int small_win;            // 1: every unclipped window holds fewer than 2^18 pixels
};

// Reading variants (the TM_FLAG_* bits of tm_params.flags).
constexpr int kFlagCdfIncl = 1;  // Eq. 1 with <=
constexpr int kFlagAreaLit = 2;  // unclipped window area, zero padding
constexpr int kFlagVarLin = 4;   // Eq. 10 on i / imax
constexpr int kFlagSrgb = 8;     // sRGB-encoded uint8 output

// Per-image range state, resident in device memory. The range kernel reduces
// into min_bits/max_bits (luminance is positive, so float bits order like the
// values), and its last block finalises imin/imax, the bin edges and the
// constants of the quantised log, then re-arms the accumulators.
struct Stats {
  unsigned int min_bits;
  unsigned int max_bits;
  unsigned int blocks_done;
  int degenerate;           // imax == imin
  float imin, imax;
  float log2_scale;         // 2^Q / (log2 imax - log2 imin), 0 if degenerate
  float c0;                 // log2 of imin's significand (in [1, 2))
  int e0;                   // unbiased exponent of imin
  float lin_scale;          // 2^Q / imax (quantisation of i / imax)
  float lg_min;             // log2 imin (first guess of a bin)
  float bin_scale;          // n / (log2 imax - log2 imin), 0 if degenerate
  float thr[kMaxBins];      // thr[k-1]: lower edge of bin k, k = 1..n-1
};

struct Image {
  void *p;
  int W, H;
  long long pitch;          // elements
  int dtype;
};

// Debug planes written by the lookup kernels (each may be null).
struct DebugPlanes {
  unsigned *cnt;   // s * H * W
  float *sigma2;   // s * H * W
  float *weight;   // s * H * W
  float *lf;       // s * H * W
  float *l;        // H * W
};

// Tiling and shared-memory layout of the fused sweep over one image (host-
// computed). Tiles are strips of TX (512 or 256) columns cut into bands of TY
// rows; the bands of a strip form groups of K consecutive bands, each group
// one segment that a CTA sweeps while it can claim its next band.
struct SweepPlan {
  int W, H;
  int TX, TY, tiles_x, tiles_y;   // own tile size and grid of bands
  int K;                          // bands per group
  int Rx, Ry;                     // largest half-width / half-height (clipped to W-1 / H-1)
  int nch_max;                    // 32-column chunks of the widest swept row
  int bstride;                    // uint16 entries per threshold row of the in-chunk counts
  int kcap;                       // thresholds held in shared memory at once
  int cnt_wide;                   // bit f: field f's counts are uint32 (else uint16)
  size_t smem;                    // dynamic shared memory bytes
};

// Batched stages; every stage kernel of a batch maps its blocks to images
// through the per-image first-block offsets b0[stage].
enum StageId { kStRange = 0, kStPrep, kStRows, kStCols, kStLook, kNumStages };

// One image of a batch: its buffers and its share of every batched launch.
// 16-byte aligned, so that kernels can copy it with 16-byte loads.
struct alignas(16) Job {
  Image in, out;
  Stats *st;                // range state the bins and q are taken over
  Stats *st_next;           // streaming reuse: receives this image's own range (else null)
  uint8_t *bins;            // H*W bin map
  int32_t *q;               // H*W quantised log
  long long *s1, *s2;       // (H+1)*(W+1) integral images of q and q^2; with s_pair
                            //   interleaved: position i of both at s1[2i], s1[2i+1], s2 = s1 + 1
  long long *segtot;        // integral-image scratch, integral_scratch_elems(W, H, nseg)
  unsigned char *cnt;       // Eq. 1 numerators from the sweep: field f's H*W plane at
                            //   cnt + cnt_off[f], uint32 if bit f of cnt_wide, else uint16
  long long cnt_off[kMaxFields];
  int cnt_wide;
  uint16_t *grp;            // per row and 32-column group: smallest | largest << 8 bin
  float2 *mom;              // kept for the backward (else null): (variance, mean of lhat)
                            //   of field f's windows, plane f of H*W at mom + f*H*W
  DebugPlanes dbg;
  int qbits;
  int s_pair;               // 1: s1 and s2 interleaved (the forward's workspace)
  int nseg, seg_rows;       // integral images: row segments of the tiles
  int b0[kNumStages];       // first block of this job in each batched stage
  int itemA0, nitemA;       // the sweep queue's slots of this job's group starts (first phase)
  int itemB0, nitemB;       // and of its other bands (second phase)
  int *claim;               // tiles_x x tiles_y band claims (cleared by the prep stage)
  SweepPlan plan;           // sweep tiling of this image
};

static_assert(sizeof(Job) % 16 == 0, "jobs are copied in 16-byte words");

// Index of the job owning block `blk` of stage `st` (jobs sorted by b0).
__device__ __forceinline__ int find_job(const Job *jobs, int njobs, int st, int blk) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].b0[st] <= blk) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Largest window of field f (pixels), as a float (host and device).
__host__ __device__ __forceinline__ float window_max(const DevParams &P, int f, int W, int H) {
  return (float)min(2 * P.rx[f] + 1, W) * (float)min(2 * P.ry[f] + 1, H);
}

// Binary scale of a backward fixed-point plane whose largest |value| has bits
// `amax` and whose windows hold at most nmax pixels: every window sum of
// round(value x 2^shift) stays below 2^61 in magnitude.
__device__ __forceinline__ int fix_shift(unsigned amax, float nmax) {
  const float m = __uint_as_float(amax) * nmax;
  if (!(m > 0.f) || !(m < 3.0e38f)) return 0;
  int e;
  frexpf(m, &e);  // m < 2^e
  return 61 - e;
}

// Eq. 11 in float: fixed order, every product and sum rounded, no contraction.
__device__ __forceinline__ float luminance(float r, float g, float b) {
  float i = __fadd_rn(__fadd_rn(__fmul_rn(0.2126f, r), __fmul_rn(0.7152f, g)),
                      __fmul_rn(0.0722f, b));
  return fmaxf(i, kLumFloor);
}

// kDt: the image's dtype when known at compile time (-1: read from im).
template <int kDt = -1>
__device__ __forceinline__ void load_rgb(const Image &im, int x, int y, float &r,
                                         float &g, float &b) {
  long long o = (long long)y * im.pitch + 3LL * x;
  if ((kDt >= 0 ? kDt : im.dtype) == kF16) {
    const __half *p = static_cast<const __half *>(im.p) + o;
    r = __half2float(p[0]);
    g = __half2float(p[1]);
    b = __half2float(p[2]);
  } else {
    const float *p = static_cast<const float *>(im.p) + o;
    r = p[0];
    g = p[1];
    b = p[2];
  }
}

// sRGB transfer function (IEC 61966-2-1) on a value clamped to [0, 1].
__device__ __forceinline__ float srgb_encode(float c) {
  c = fminf(fmaxf(c, 0.f), 1.f);
  return c <= 0.0031308f ? 12.92f * c : 1.055f * powf(c, 1.f / 2.4f) - 0.055f;
}

template <int kDt = -1>
__device__ __forceinline__ void store_rgb(const Image &im, int x, int y, float r,
                                          float g, float b, bool srgb = false) {
  long long o = (long long)y * im.pitch + 3LL * x;
  const int dt = kDt >= 0 ? kDt : im.dtype;
  if (dt == kF32) {
    float *p = static_cast<float *>(im.p) + o;
    p[0] = r;
    p[1] = g;
    p[2] = b;
  } else if (dt == kF16) {
    __half *p = static_cast<__half *>(im.p) + o;
    p[0] = __float2half_rn(r);
    p[1] = __float2half_rn(g);
    p[2] = __float2half_rn(b);
  } else {
    uint8_t *p = static_cast<uint8_t *>(im.p) + o;
    if (srgb) {
      r = srgb_encode(r);
      g = srgb_encode(g);
      b = srgb_encode(b);
    }
    p[0] = (uint8_t)__float2int_rd(fminf(fmaxf(r, 0.f), 1.f) * 255.f + 0.5f);
    p[1] = (uint8_t)__float2int_rd(fminf(fmaxf(g, 0.f), 1.f) * 255.f + 0.5f);
    p[2] = (uint8_t)__float2int_rd(fminf(fmaxf(b, 0.f), 1.f) * 255.f + 0.5f);
  }
}

// Bin of a luminance (Section II-A): the number of edges at or below it. The
// first guess comes from the fast base-2 log, scaled to bins; the compares
// against the exact edges then settle it, so the result does not depend on
// the guess.
__device__ __forceinline__ int bin_of(float i, const float *thr, int n, float lg_min, float bin_scale) {
  int k = (int)((__log2f(i) - lg_min) * bin_scale);
  k = min(max(k, 0), n - 1);
  while (k > 0 && i < thr[k - 1]) --k;
  while (k < n - 1 && i >= thr[k]) ++k;
  return k;
}

// Quantised normalised log luminance: q = round(2^Q lhat) - 2^(Q-1), with
// lhat = (log2 i - log2 imin) / (log2 imax - log2 imin). The difference of
// logs is formed as exponent difference + significand-log difference and the
// product with the scale is kept as a float pair, so q is accurate to about
// one unit of 2^-Q.
__device__ __forceinline__ int quantise_log(float lum, const Stats &st, int qbits) {
  unsigned bits = __float_as_uint(lum);
  int e = (int)(bits >> 23) - 127;
  float m = __uint_as_float((bits & 0x7fffffu) | 0x3f800000u);
  float f = __log2f(m) - st.c0;  // m in [1, 2): absolute error near 2^-22
  float de = (float)(e - st.e0);
  float d_hi = de + f;                       // TwoSum(de, f)
  float bv = d_hi - de;
  float d_lo = (de - (d_hi - bv)) + (f - bv);
  float S = st.log2_scale;
  float p = S * d_hi;                        // TwoProduct(S, d_hi)
  float perr = fmaf(S, d_hi, -p);
  float tail = fmaf(S, d_lo, perr);
  float pi = rintf(p);
  float rem = (p - pi) + tail;
  int half = 1 << (qbits - 1);
  int q = (int)pi + __float2int_rn(rem) - half;
  return min(max(q, -half), half);
}

// Quantised linear luminance for the variance under TM_FLAG_VAR_LINEAR:
// q = round(2^Q i / imax) - 2^(Q-1).
__device__ __forceinline__ int quantise_lin(float lum, const Stats &st, int qbits) {
  const int half = 1 << (qbits - 1);
  const int q = __float2int_rn(lum * st.lin_scale) - half;
  return min(max(q, -half), half);
}

// Under TM_FLAG_AREA_LITERAL: the window sums of q and q^2 and the area of
// field f grow from the clipped window (area N) to the unclipped (2 rx + 1)
// (2 ry + 1), the missing pixels taking the value 0 (q = -2^(Q-1)). Exact in
// 64-bit arithmetic (Q is chosen for the unclipped area).
__device__ __forceinline__ void literal_area(const DevParams &P, int f, int qbits, long long &q1,
                                             long long &q2, unsigned long long &N) {
  if (!(P.flags & kFlagAreaLit)) return;
  const unsigned long long Nl = (unsigned long long)(2 * P.rx[f] + 1) * (unsigned long long)(2 * P.ry[f] + 1);
  const unsigned long long pad = Nl - N;
  const unsigned long long h = 1ull << (qbits - 1);
  q1 = (long long)((unsigned long long)q1 - pad * h);
  q2 = (long long)((unsigned long long)q2 + pad * (h * h));
  N = Nl;
}

// Window of field f around (x, y), clipped to the image.
struct Win {
  int x0, x1, y0, y1;
};
__device__ __forceinline__ Win window_of(const DevParams &P, int f, int x, int y,
                                         int W, int H) {
  Win w;
  w.x0 = max(x - P.rx[f], 0);
  w.x1 = min(x + P.rx[f], W - 1);
  w.y0 = max(y - P.ry[f], 0);
  w.y1 = min(y + P.ry[f], H - 1);
  return w;
}

// Integer <-> float conversions from 32-bit integer and FP32 operations. The
// 64-bit conversion instructions execute on the FP64 pipe, a small fraction
// of the FP32 rate on this part (about two results per clock per SM), and
// bounded the per-pixel kernels that used them.
//
// uint32 -> float, correctly rounded: each 16-bit half h is the exact float
// (2^23 + h) - 2^23, and one FMA joins them with a single rounding.
__device__ __forceinline__ float u32_to_float(unsigned x) {
  const float h = __uint_as_float(0x4B000000u | (x >> 16)) - 8388608.f;
  const float l = __uint_as_float(0x4B000000u | (x & 0xffffu)) - 8388608.f;
  return __fmaf_rn(h, 65536.f, l);
}

// uint64 -> float within one ulp (exact below 2^24, correctly rounded below
// 2^32): the 32-bit halves converted as above and joined by one FMA; the low
// half's rounding error is at most a quarter ulp of the result when the high
// half is nonzero.
__device__ __forceinline__ float u64_to_float(unsigned long long a) {
  const unsigned hi = (unsigned)(a >> 32);
  const float lo = u32_to_float((unsigned)a);
  return hi ? __fmaf_rn(u32_to_float(hi), 4294967296.f, lo) : lo;
}

// int64 -> float within one ulp (the magnitude as above, then the sign).
__device__ __forceinline__ float i64_to_float(long long s) {
  const float f = u64_to_float(s < 0 ? 0ull - (unsigned long long)s : (unsigned long long)s);
  return s < 0 ? -f : f;
}

// float -> int64, rounded to nearest with ties to even, for |y| < 2^62: at or
// above 2^23 a float is an integer (its significand shifted up); below,
// 2^23 + |y| rounds |y| to an integer in the last place.
__device__ __forceinline__ long long float_to_i64_rn(float y) {
  const unsigned bits = __float_as_uint(y);
  const int ex = (int)((bits >> 23) & 0xffu);
  const unsigned long long mag =
      ex >= 150 ? (unsigned long long)((bits & 0x7fffffu) | 0x800000u) << min(ex - 150, 40)
                : (unsigned long long)(__float_as_uint(fabsf(y) + 8388608.f) - 0x4B000000u);
  return (bits >> 31) ? -(long long)mag : (long long)mag;
}

// Window variance of q from its exact window sums s1 = sum q and s2 = sum q^2
// (modulo 2^64) over N pixels. With m the integer nearest a float estimate of
// the mean (within a few units of it) and d = s1 - m N,
//     T = sum (q - m)^2 = s2 - m (s1 + d)     exact in wrapping 64-bit arithmetic,
//     N^2 var = N T - d^2,
// so var = (T - d^2 / N) / N. T and d are exact; d^2 / N stays below a few N,
// so the one float subtraction loses at most a few bits whenever var >= 1
// unit^2, and far less than the quantisation step below that. rN = rounded
// 1/N; inv_scale2 = 2^-2Q converts to lhat units.
// Small windows (kSmall = 1, or small at run time with kSmall = -1: every
// window under 2^18 pixels) take the two 64-bit conversions that run on the
// slow FP64 pipe through 32-bit ones: |s1| <= 2^23 N < 2^41, so s1 / 2^10
// (rounded down) fits 31 bits and its float estimate of the mean is within
// 2^10 / N + 4 of it; then |d| <= 4.5 N + 2^10 < 2^31. The float error of
// T - d^2 / N grows to about 2^-24 (var + (m - mean)^2) unit^2, at most
// 2^-4 unit^2 (one-pixel windows), below the quantisation step.
template <int kSmall = -1>
__device__ __forceinline__ float window_variance(long long s1, long long s2, unsigned long long N,
                                                 float rN, float inv_scale2, bool small = false) {
  const bool sm = kSmall >= 0 ? kSmall != 0 : small;
  // |mean| <= 2^(Q-1) <= 2^23: the nearest integer fits 32 bits
  const int m = sm ? __float2int_rn(__int2float_rn((int)(s1 >> 10)) * (rN * 1024.f))
                   : __float2int_rn(__ll2float_rn(s1) * rN);
  const long long d = s1 - (long long)m * (long long)N;
  const unsigned long long T = (unsigned long long)s2 - (unsigned long long)((long long)m * (s1 + d));
  const float df = sm ? __int2float_rn((int)d) : __ll2float_rn(d);
  const float v = fmaf(-df * rN, df, __ull2float_rn(T)) * rN;
  return fmaxf(v, 0.f) * inv_scale2;
}

// Area of field f's window at (x, y) as a float: clipped to the image, or
// under TM_FLAG_AREA_LITERAL the unclipped (2 rx + 1)(2 ry + 1) (kLit =
// false: the caller guarantees that flag is off).
template <bool kLit = true>
__device__ __forceinline__ float window_area(const DevParams &P, int f, int x, int y, int W, int H) {
  if (kLit && (P.flags & kFlagAreaLit)) return (float)((unsigned)(2 * P.rx[f] + 1) * (unsigned)(2 * P.ry[f] + 1));
  const int x0 = max(x - P.rx[f], 0), x1 = min(x + P.rx[f], W - 1);
  const int y0 = max(y - P.ry[f], 0), y1 = min(y + P.ry[f], H - 1);
  return (float)((unsigned)(x1 - x0 + 1) * (unsigned)(y1 - y0 + 1));
}

// Window mean of lhat from the window sum of q (q = 2^Q lhat - 2^(Q-1), up
// to rounding), with explicit roundings so that every kernel gets the same
// bits.
__device__ __forceinline__ float window_mean(long long q1, float rarea, float inv_scale) {
  return __fmaf_rn(__fmul_rn(__ll2float_rn(q1), rarea), inv_scale, 0.5f);
}

// Window moments of field f at (x, y) from the interleaved integral images
// of q and q^2 (Eq. 6, one 16-byte load per corner): the fast reciprocal of
// the area (within 1 ulp), the variance (Eq. 10) and the window sum of q.
// Positions fit 32 bits: the image holds fewer than 2^31 pixels, so
// (W + 1)(H + 1) <= 2^32.
struct WinMoments {
  float rarea, var;
  long long q1;
};
// kLit = false: the caller guarantees TM_FLAG_AREA_LITERAL is off (the
// padding terms are then not compiled in); kSmall as for window_variance
// (-1: P.small_win).
template <bool kLit = true, int kSmall = -1>
__device__ __forceinline__ WinMoments window_moments(const DevParams &P, int f, int x, int y, int W, int H,
                                                     const longlong2 *__restrict__ s12, int qbits,
                                                     float inv_scale2) {
  const unsigned W1 = (unsigned)W + 1u;
  const int x0 = max(x - P.rx[f], 0), x1 = min(x + P.rx[f], W - 1);
  const int y0 = max(y - P.ry[f], 0), y1 = min(y + P.ry[f], H - 1);
  const unsigned rt = (unsigned)y0 * W1, rb = (unsigned)(y1 + 1) * W1;
  const longlong2 a = __ldg(s12 + (rt + (unsigned)x0)), b = __ldg(s12 + (rt + (unsigned)x1 + 1u));
  const longlong2 c = __ldg(s12 + (rb + (unsigned)x1 + 1u)), d = __ldg(s12 + (rb + (unsigned)x0));
  unsigned long long N = (unsigned long long)((unsigned)(x1 - x0 + 1) * (unsigned)(y1 - y0 + 1));
  long long q1 = (long long)((unsigned long long)c.x - (unsigned long long)d.x - (unsigned long long)b.x +
                             (unsigned long long)a.x);
  long long q2 = (long long)((unsigned long long)c.y - (unsigned long long)d.y - (unsigned long long)b.y +
                             (unsigned long long)a.y);
  if (kLit) literal_area(P, f, qbits, q1, q2, N);
  WinMoments m;
  m.rarea = __fdividef(1.f, (float)(unsigned)N);  // N <= 65535^2 < 2^32
  m.var = window_variance<kSmall>(q1, q2, N, m.rarea, inv_scale2, P.small_win != 0);
  m.q1 = q1;
  return m;
}

// Eq. 2, Eq. 4, Eq. 3 from per-field counts, reciprocal areas and variances.
// The Eq. 1 quotient is count x (1/N); the Eq. 4 and Eq. 3 quotients use the
// fast division (about 2 ulp).
__device__ __forceinline__ float fuse_fields(const DevParams &P, const unsigned *cnt,
                                             const float *rarea, const float *var,
                                             float *wout, float *lfout) {
  float wsum = 0.f, acc = 0.f, mean = 0.f;
  float span = P.ld_max - P.ld_min;
#pragma unroll
  for (int f = 0; f < kMaxFields; ++f) {
    if (f >= P.n_fields) break;
    float Pf = (float)cnt[f] * rarea[f];                                 // Eq. 1
    float Lf = fmaf(span, Pf, P.ld_min);                                 // Eq. 2
    float Wf = __fdividef(P.alpha[f] * var[f], var[f] + P.eps[f]);      // Eq. 4
    if (wout) wout[f] = Wf;
    if (lfout) lfout[f] = Lf;
    wsum += Wf;
    acc = fmaf(Wf, Lf, acc);
    mean += Lf;
  }
  return wsum > 0.f ? __fdividef(acc, wsum) : __fdividef(mean, (float)P.n_fields);  // Eq. 3
}

// Eq. 1 numerator of field f at pixel index pix from the sweep's count planes
// (J: a job holding cnt, cnt_off and cnt_wide).
template <class JobT>
__device__ __forceinline__ unsigned load_count(const JobT &J, int f, long long pix) {
  const unsigned char *pl = J.cnt + J.cnt_off[f];
  return ((J.cnt_wide >> f) & 1) ? __ldg(reinterpret_cast<const unsigned *>(pl) + pix)
                                 : (unsigned)__ldg(reinterpret_cast<const uint16_t *>(pl) + pix);
}

// Eq. 12 with the ratio clamped at zero; inv_i = 1 / i. The power is taken
// as exp2(sat * log2(rho)) on the special-function unit (relative error about
// 1e-7 for the ratios of real images); rho = 0 gives 0 (1 when sat = 0).
__device__ __forceinline__ float restore_channel(float C, float inv_i, float sat, float L) {
  const float rho = C * inv_i;
  if (!(rho > 0.f)) return sat == 0.f ? L : 0.f;
  return exp2f(sat * __log2f(rho)) * L;
}

}  // namespace tmk
