// tm_prepass.cu -- luminance range, bin edges, bin map and quantised log.
//
// Section III Eq. 11 gives the luminance, Section II the logarithmic
// compression, Section II-A the n equal-width bins of the log over the
// image's value range. The range is a global reduction, so the input is read
// once here to find it and once more by every later stage.
#include "tm_kernels.cuh"

namespace tmk {

// Range of Eq. 11 luminance. Block min/max are folded with unsigned atomics;
// the last block to finish computes the bin edges and the quantisation
// constants in double precision, then re-arms the accumulators for the next
// image, so no host round trip is needed between the stages.
__global__ void __launch_bounds__(256) k_range(Image in, Stats *st, int n_bins, int qbits) {
  __shared__ unsigned smin[8], smax[8];
  __shared__ int last;
  unsigned bmin = 0x7f800000u, bmax = 0u;
  const int W = in.W, H = in.H;
  for (int y = blockIdx.y; y < H; y += gridDim.y)
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < W; x += gridDim.x * blockDim.x) {
      float r, g, b;
      load_rgb(in, x, y, r, g, b);
      unsigned v = __float_as_uint(luminance(r, g, b));
      bmin = min(bmin, v);
      bmax = max(bmax, v);
    }
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
    unsigned ticket = atomicAdd(&st->blocks_done, 1u);
    last = (ticket == gridDim.x * gridDim.y - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  volatile Stats *vs = st;
  const float imin = __uint_as_float(vs->min_bits);
  const float imax = __uint_as_float(vs->max_bits);
  const bool degenerate = !(imax > imin);
  const double lmin = log((double)imin), lmax = log((double)imax);
  for (int k = 1 + threadIdx.x; k < n_bins; k += blockDim.x) {
    float edge = __int_as_float(0x7f800000);
    if (!degenerate) {
      double t = exp(lmin + (lmax - lmin) * ((double)k / (double)n_bins));
      edge = __double2float_ru(t);  // smallest float >= t
    }
    st->thr[k - 1] = edge;
  }
  if (threadIdx.x == 0) {
    unsigned bits = __float_as_uint(imin);
    st->e0 = (int)(bits >> 23) - 127;
    double m0 = (double)__uint_as_float((bits & 0x7fffffu) | 0x3f800000u);
    st->c0 = (float)log2(m0);
    st->log2_scale =
        degenerate ? 0.f : (float)(ldexp(1.0, qbits) / (log2((double)imax) - log2((double)imin)));
    st->imin = imin;
    st->imax = imax;
    st->degenerate = degenerate ? 1 : 0;
    st->min_bits = 0x7f800000u;
    st->max_bits = 0u;
    st->blocks_done = 0u;
  }
}

// Bin map (Section II-A, edges from k_range) and quantised normalised log.
__global__ void __launch_bounds__(256) k_prep(Image in, const Stats *st, int n_bins, int qbits,
                                               uint8_t *bins, int32_t *q) {
  __shared__ float thr[kMaxBins];
  __shared__ Stats sst;
  for (int k = threadIdx.x; k < n_bins - 1; k += blockDim.x) thr[k] = st->thr[k];
  if (threadIdx.x == 0) sst = *st;
  __syncthreads();
  const int W = in.W, H = in.H;
  for (int y = blockIdx.y; y < H; y += gridDim.y)
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < W; x += gridDim.x * blockDim.x) {
      float r, g, b;
      load_rgb(in, x, y, r, g, b);
      float i = luminance(r, g, b);
      long long o = (long long)y * W + x;
      bins[o] = (uint8_t)bin_of(i, thr, n_bins);
      q[o] = quantise_log(i, sst, qbits);
    }
}

void launch_range(const Image &in, Stats *st, int n_bins, int qbits, cudaStream_t s) {
  dim3 block(256);
  int gx = (in.W + 255) / 256;
  int gy = in.H < 1024 ? in.H : 1024;
  while ((long long)gx * gy > 4096 && gy > 1) gy = (gy + 1) / 2;
  k_range<<<dim3(gx, gy), block, 0, s>>>(in, st, n_bins, qbits);
}

void launch_prep(const Image &in, const Stats *st, int n_bins, int qbits, uint8_t *bins,
                 int32_t *q, cudaStream_t s) {
  dim3 block(256);
  int gx = (in.W + 255) / 256;
  int gy = in.H < 2048 ? in.H : 2048;
  k_prep<<<dim3(gx, gy), block, 0, s>>>(in, st, n_bins, qbits, bins, q);
}

}  // namespace tmk
