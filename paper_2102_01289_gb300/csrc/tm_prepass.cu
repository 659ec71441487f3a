// tm_prepass.cu -- luminance range, bin edges, bin map and quantised log.
//
// Section III Eq. 11 gives the luminance, Section II the logarithmic
// compression, Section II-A the n equal-width bins of the log over the
// image's value range. The range is a global reduction, so the input is read
// once here to find it and once more by every later stage.
//
// Pixels are read four at a time: twelve float samples as three 16-byte loads
// (or twelve halves as three 8-byte loads) when rows are aligned for it, with
// a scalar path for ragged row ends and unaligned images.
#include "tm_kernels.cuh"

namespace tmk {
namespace {

// Four consecutive pixels of row y starting at x (x + 3 < W), vector loads.
// kDt: the image's dtype when known at compile time (-1: read from im).
template <int kDt>
__device__ __forceinline__ void load4_vec(const Image &im, int x, int y, float r[4], float g[4],
                                          float b[4]) {
  const long long o = (long long)y * im.pitch + 3LL * x;
  float v[12];
  if ((kDt >= 0 ? kDt : im.dtype) == kF16) {
    const uint2 *p = reinterpret_cast<const uint2 *>(static_cast<const __half *>(im.p) + o);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const uint2 u = __ldg(p + k);
      const __half2 h0 = *reinterpret_cast<const __half2 *>(&u.x);
      const __half2 h1 = *reinterpret_cast<const __half2 *>(&u.y);
      v[4 * k + 0] = __low2float(h0);
      v[4 * k + 1] = __high2float(h0);
      v[4 * k + 2] = __low2float(h1);
      v[4 * k + 3] = __high2float(h1);
    }
  } else {
    const float4 *p = reinterpret_cast<const float4 *>(static_cast<const float *>(im.p) + o);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float4 f = __ldg(p + k);
      v[4 * k + 0] = f.x;
      v[4 * k + 1] = f.y;
      v[4 * k + 2] = f.z;
      v[4 * k + 3] = f.w;
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    r[i] = v[3 * i];
    g[i] = v[3 * i + 1];
    b[i] = v[3 * i + 2];
  }
}

// Up to four pixels of row y from x (n of them), scalar loads.
template <int kDt>
__device__ __forceinline__ void load4_scalar(const Image &im, int x, int y, int n, float r[4],
                                             float g[4], float b[4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (i < n) load_rgb<kDt>(im, x + i, y, r[i], g[i], b[i]);
    else r[i] = g[i] = b[i] = 1.f;
  }
}

template <int kDt>
__device__ __forceinline__ void load4(const Image &im, bool vec, int x, int y, int n, float r[4],
                                      float g[4], float b[4]) {
  if (vec && n == 4) load4_vec<kDt>(im, x, y, r, g, b);
  else load4_scalar<kDt>(im, x, y, n, r, g, b);
}

}  // namespace

// Rows of `im` can be read with the vector loads above.
__device__ __forceinline__ bool vec_ok(const Image &im) {
  const size_t es = im.dtype == kF16 ? 2 : 4;
  const size_t align = im.dtype == kF16 ? 8 : 16;
  return ((uintptr_t)im.p % align) == 0 && ((size_t)im.pitch * es) % align == 0;
}

// Fold a block's luminance range (float bits of its min and max) into *st;
// the block that arrives last (of nb) computes the bin edges and the
// quantisation constants in double precision and re-arms the accumulators for
// the next call, so no host round trip is needed. All threads of the block
// call this.
__device__ void commit_range(Stats *st, unsigned bmin, unsigned bmax, int nb, int n_bins, int qbits) {
  __shared__ unsigned smin[32], smax[32];
  __shared__ int last;
  bmin = __reduce_min_sync(0xffffffffu, bmin);
  bmax = __reduce_max_sync(0xffffffffu, bmax);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { smin[wid] = bmin; smax[wid] = bmax; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      bmin = min(bmin, smin[w]);
      bmax = max(bmax, smax[w]);
    }
    atomicMin(&st->min_bits, bmin);
    atomicMax(&st->max_bits, bmax);
    __threadfence();
    const unsigned ticket = atomicAdd(&st->blocks_done, 1u);
    last = (ticket == (unsigned)nb - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  volatile Stats *vs = st;
  const float imin = __uint_as_float(vs->min_bits);
  const float imax = __uint_as_float(vs->max_bits);
  const bool degenerate = !(imax > imin);
  // the FP64 logarithms, one warp each, so that their latencies overlap (the
  // FP64 pipe is slow on this part and this block is the kernel's tail)
  __shared__ double lg[5];
  const unsigned bits = __float_as_uint(imin);
  if ((threadIdx.x & 31) == 0) {
    switch (threadIdx.x >> 5) {
      case 0: lg[0] = log((double)imin); break;
      case 1: lg[1] = log((double)imax); break;
      case 2: lg[2] = log2((double)imin); break;
      case 3: lg[3] = log2((double)imax); break;
      case 4: lg[4] = log2((double)__uint_as_float((bits & 0x7fffffu) | 0x3f800000u)); break;
      default: break;
    }
  }
  __syncthreads();
  const double lmin = lg[0], lmax = lg[1];
  for (int k = 1 + threadIdx.x; k < n_bins; k += blockDim.x) {
    float edge = __int_as_float(0x7f800000);
    if (!degenerate) {
      const double t = exp(lmin + (lmax - lmin) * ((double)k / (double)n_bins));
      edge = __double2float_ru(t);  // smallest float >= t
    }
    st->thr[k - 1] = edge;
  }
  if (threadIdx.x == 0) {
    const double l2min = lg[2], l2max = lg[3];
    st->e0 = (int)(bits >> 23) - 127;
    st->c0 = (float)lg[4];
    st->log2_scale = degenerate ? 0.f : (float)(ldexp(1.0, qbits) / (l2max - l2min));
    st->lin_scale = (float)(ldexp(1.0, qbits) / (double)imax);
    st->lg_min = (float)l2min;
    st->bin_scale = degenerate ? 0.f : (float)((double)n_bins / (l2max - l2min));
    st->imin = imin;
    st->imax = imax;
    st->degenerate = degenerate ? 1 : 0;
    st->min_bits = 0x7f800000u;
    st->max_bits = 0u;
    st->blocks_done = 0u;
  }
}

// Range of Eq. 11 luminance, per image of the batch: block min/max folded
// into the image's Stats by commit_range. kDt: the dtype of every input when
// they share one (-1: read from the descriptors).
template <int kDt>
__global__ void __launch_bounds__(256) k_range(const Job *__restrict__ jobs, int njobs, int n_bins) {
  const int j = find_job(jobs, njobs, kStRange, blockIdx.x);
  const Job &J = jobs[j];
  const int lb = blockIdx.x - J.b0[kStRange];
  const int nb = (j + 1 < njobs ? jobs[j + 1].b0[kStRange] : (int)gridDim.x) - J.b0[kStRange];
  const Image in = J.in;
  const bool vec = vec_ok(in);
  Stats *st = J.st;
  unsigned bmin = 0x7f800000u, bmax = 0u;
  const int W = in.W, H = in.H;
  const int gpr = (W + 3) >> 2;  // groups of four pixels per row
  const int ng = gpr * H;        // fewer than 2^31 pixels
  const int stride = nb * blockDim.x;
  for (int g0 = lb * blockDim.x + threadIdx.x; g0 < ng; g0 += 2 * stride) {
    float r[2][4], gg[2][4], b[2][4];
    int n[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {  // two groups in flight per thread
      const int g = g0 + u * stride;
      n[u] = 0;
      if (g < ng) {
        const int y = g / gpr, x = (g - y * gpr) * 4;
        n[u] = min(4, W - x);
        load4<kDt>(in, vec, x, y, n[u], r[u], gg[u], b[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (i < n[u]) {
          const unsigned v = __float_as_uint(luminance(r[u][i], gg[u][i], b[u][i]));
          bmin = min(bmin, v);
          bmax = max(bmax, v);
        }
  }
  commit_range(st, bmin, bmax, nb, n_bins, J.qbits);
}

// Bin map (Section II-A, edges from k_range) and the quantised values whose
// window variance Eq. 10 takes: the normalised log, or i / imax under
// TM_FLAG_VAR_LINEAR. One thread per group of four pixels; rows are padded to
// whole 32-pixel groups so that eight consecutive lanes share one group,
// whose bin range (smallest | largest << 8) goes to J.grp for the sweep.
// kLin: TM_FLAG_VAR_LINEAR; kDt as in k_range.
template <bool kLin, int kDt>
__global__ void __launch_bounds__(256) k_prep(const Job *__restrict__ jobs, int njobs, int n_bins, int n_fields) {
  __shared__ float thr[kMaxBins];
  const int j = find_job(jobs, njobs, kStPrep, blockIdx.x);
  const Job &J = jobs[j];
  const int lb = blockIdx.x - J.b0[kStPrep];
  const int nb = (j + 1 < njobs ? jobs[j + 1].b0[kStPrep] : (int)gridDim.x) - J.b0[kStPrep];
  const Image in = J.in;
  const bool vec = vec_ok(in);
  const Stats *st = J.st;
  for (int k = threadIdx.x; k < n_bins - 1; k += blockDim.x) thr[k] = st->thr[k];
  Stats sst;  // only the three constants quantise_log reads
  sst.c0 = __ldg(&st->c0);
  sst.e0 = __ldg(&st->e0);
  sst.log2_scale = __ldg(&st->log2_scale);
  sst.lin_scale = __ldg(&st->lin_scale);
  const float lg_min = __ldg(&st->lg_min), bin_scale = __ldg(&st->bin_scale);
  __syncthreads();
  const int W = in.W, H = in.H, qbits = J.qbits;
  uint8_t *bins = J.bins;
  int32_t *q = J.q;
  const int G = (W + 31) >> 5;  // 32-pixel groups per row
  const int gpr = 8 * G;        // groups of four pixels per padded row
  const int ng = gpr * H;
  const int lane = threadIdx.x & 31;
  unsigned bmin = 0x7f800000u, bmax = 0u;  // this image's own range (streaming reuse)
  // whole warps iterate together (the group shuffles need all lanes)
  for (int g0 = lb * blockDim.x + (threadIdx.x & ~31); g0 < ng; g0 += nb * blockDim.x) {
    const int gi = g0 + lane;
    const int y = gi / gpr, x = (gi - y * gpr) * 4;
    const int n = gi < ng ? max(0, min(4, W - x)) : 0;
    int kmin = 256, kmax = -1;
    if (n > 0) {
      float r[4], g[4], b[4];
      load4<kDt>(in, vec, x, y, n, r, g, b);
      unsigned bq = 0;
      int qq[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float l = luminance(r[i], g[i], b[i]);
        const int bi = bin_of(l, thr, n_bins, lg_min, bin_scale);
        bq |= (unsigned)bi << (8 * i);
        qq[i] = kLin ? quantise_lin(l, sst, qbits) : quantise_log(l, sst, qbits);
        if (i < n) {
          bmin = min(bmin, __float_as_uint(l));
          bmax = max(bmax, __float_as_uint(l));
          kmin = min(kmin, bi);
          kmax = max(kmax, bi);
        }
      }
      const long long o = (long long)y * W + x;
      if (n == 4 && (o & 3) == 0) {
        *reinterpret_cast<unsigned *>(bins + o) = bq;
        *reinterpret_cast<int4 *>(q + o) = make_int4(qq[0], qq[1], qq[2], qq[3]);
        // the sweep adds its bands' contributions into zeroed count planes
        if (J.cnt)
          for (int f = 0; f < n_fields; ++f)
            *reinterpret_cast<int4 *>(J.cnt + J.cnt_off[f] + 4 * o) = make_int4(0, 0, 0, 0);
      } else {
        for (int i = 0; i < n; ++i) {
          bins[o + i] = (uint8_t)(bq >> (8 * i));
          q[o + i] = qq[i];
          if (J.cnt)
            for (int f = 0; f < n_fields; ++f) reinterpret_cast<unsigned *>(J.cnt + J.cnt_off[f])[o + i] = 0u;
        }
      }
    }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
      kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
    }
    if (J.grp && (lane & 7) == 0 && kmax >= 0) J.grp[(long long)y * G + (x >> 5)] = (uint16_t)(kmin | (kmax << 8));
  }
  // the sweep's band claims start cleared
  if (J.claim)
    for (int i = lb * blockDim.x + threadIdx.x; i < J.plan.tiles_x * J.plan.tiles_y; i += nb * blockDim.x)
      J.claim[i] = 0;
  // streaming reuse: the bins above used an earlier frame's range; this
  // frame's own range goes to st_next for the frame after
  if (J.st_next) commit_range(J.st_next, bmin, bmax, nb, n_bins, qbits);
}

int range_blocks(int W, int H, int num_sms, double share) {
  const long long groups = (long long)((W + 3) / 4) * H;
  long long b = (groups + 511) / 512;
  const long long cap = (long long)(4.0 * num_sms * share) + 1;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

int prep_blocks(int W, int H, int num_sms, double share) {
  const long long groups = (long long)8 * ((W + 31) / 32) * H;
  long long b = (groups + 255) / 256;
  const long long cap = (long long)(16.0 * num_sms * share) + 1;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

int input_dtype(const Job *jobs, int njobs) {
  int dt = njobs > 0 ? jobs[0].in.dtype : -1;
  for (int i = 1; i < njobs; ++i)
    if (jobs[i].in.dtype != dt) return -1;
  return dt;
}

void launch_range(const Job *jobs, int njobs, int blocks, int n_bins, int dtype, cudaStream_t s) {
  if (dtype == kF32) k_range<kF32><<<blocks, 256, 0, s>>>(jobs, njobs, n_bins);
  else if (dtype == kF16) k_range<kF16><<<blocks, 256, 0, s>>>(jobs, njobs, n_bins);
  else k_range<-1><<<blocks, 256, 0, s>>>(jobs, njobs, n_bins);
}

template <bool kLin>
static void launch_prep_lin(const Job *jobs, int njobs, int blocks, int n_bins, int n_fields, int dtype,
                            cudaStream_t s) {
  if (dtype == kF32) k_prep<kLin, kF32><<<blocks, 256, 0, s>>>(jobs, njobs, n_bins, n_fields);
  else if (dtype == kF16) k_prep<kLin, kF16><<<blocks, 256, 0, s>>>(jobs, njobs, n_bins, n_fields);
  else k_prep<kLin, -1><<<blocks, 256, 0, s>>>(jobs, njobs, n_bins, n_fields);
}

void launch_prep(const Job *jobs, int njobs, int blocks, int n_bins, int flags, int n_fields, int dtype,
                 cudaStream_t s) {
  if (flags & kFlagVarLin) launch_prep_lin<true>(jobs, njobs, blocks, n_bins, n_fields, dtype, s);
  else launch_prep_lin<false>(jobs, njobs, blocks, n_bins, n_fields, dtype, s);
}

}  // namespace tmk
