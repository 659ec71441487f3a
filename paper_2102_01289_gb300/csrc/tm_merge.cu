// tm_merge.cu -- the capture front-end of Section III: a WDR radiance map from
// several exposures by Debevec and Malik's method (the paper's application
// captures four exposures and recovers the WDR image this way before tone
// mapping it).
//
// For each channel of each pixel, with z_j the exposure's 8-bit value, g the
// channel's log inverse response (g(z) = ln of the sensor exposure that maps
// to z) and dt_j the exposure time:
//     ln E = sum_j w(z_j) (g(z_j) - ln dt_j) / sum_j w(z_j),
//     w(z) = z for z <= 127, 255 - z above (the hat weighting),
// and E = exp(ln E). Where every weight is zero (each exposure at 0 or 255),
// the shortest exposure's estimate is taken if it is saturated, else the
// longest's. The response table travels as a kernel parameter and is staged
// in shared memory (indexed by pixel value); nothing is allocated.
#include <cmath>

#include "tm.h"
#include "tm_host.h"
#include "tm_kernels.cuh"

using namespace tmk;

namespace {

constexpr int kMaxExposures = 8;
constexpr int kMT = 256;

struct MergeArgs {
  const uint8_t *ldr[kMaxExposures];  // HWC uint8, pitch_in elements per row
  float neg_log_t[kMaxExposures];     // -ln dt_j
  int n, shortest, longest;
  long long pitch_in;
  float g[3][256];                    // log inverse response per channel
};

__global__ void __launch_bounds__(kMT) k_merge(const __grid_constant__ MergeArgs a, Image out) {
  __shared__ float g[3][256];
  for (int i = threadIdx.x; i < 3 * 256; i += kMT) (&g[0][0])[i] = (&a.g[0][0])[i];
  __syncthreads();
  const int W = out.W, H = out.H;
  const long long N = (long long)W * H;
  for (long long p = (long long)blockIdx.x * kMT + threadIdx.x; p < N; p += (long long)gridDim.x * kMT) {
    const int y = (int)(p / W), x = (int)(p - (long long)y * W);
    const long long o = (long long)y * a.pitch_in + 3LL * x;
    float E[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float num = 0.f, den = 0.f;
      for (int j = 0; j < a.n; ++j) {
        const int z = __ldg(a.ldr[j] + o + c);
        const float w = (float)(z <= 127 ? z : 255 - z);
        num = fmaf(w, g[c][z] + a.neg_log_t[j], num);
        den += w;
      }
      float lnE;
      if (den > 0.f) {
        lnE = num / den;
      } else {
        const int j = __ldg(a.ldr[a.shortest] + o + c) == 255 ? a.shortest : a.longest;
        lnE = g[c][__ldg(a.ldr[j] + o + c)] + a.neg_log_t[j];
      }
      E[c] = expf(lnE);
    }
    store_rgb(out, x, y, E[0], E[1], E[2]);
  }
}

}  // namespace

extern "C" tm_status tm_merge_exposures(int32_t n, const uint8_t *const *ldr, const float *times,
                                        int32_t width, int32_t height, int64_t pitch,
                                        const float *log_response, const tm_image *out, void *stream) {
  if (n < 1 || n > kMaxExposures)
    return fail_noctx(TM_EINVAL, "tm_merge_exposures: 1 to 8 exposures");
  if (!ldr || !times || !log_response || !out || !out->data)
    return fail_noctx(TM_EINVAL, "tm_merge_exposures: null argument");
  if (width < 1 || height < 1 || (long long)width * height > (1LL << 31) - 1 || pitch < 3LL * width)
    return fail_noctx(TM_EINVAL, "tm_merge_exposures: bad size or pitch");
  if (out->width != width || out->height != height || out->pitch < 3LL * width ||
      (out->dtype != TM_F32 && out->dtype != TM_F16))
    return fail_noctx(TM_EINVAL, "tm_merge_exposures: out must be a float32 or float16 image of the same size");
  MergeArgs a{};
  a.n = n;
  a.pitch_in = pitch;
  for (int j = 0; j < n; ++j) {
    if (!ldr[j]) return fail_noctx(TM_EINVAL, "tm_merge_exposures: null exposure");
    if (!(times[j] > 0.f)) return fail_noctx(TM_EINVAL, "tm_merge_exposures: exposure times must be > 0");
    a.ldr[j] = ldr[j];
    a.neg_log_t[j] = (float)-std::log((double)times[j]);
    if (times[j] < times[a.shortest]) a.shortest = j;
    if (times[j] > times[a.longest]) a.longest = j;
  }
  for (int c = 0; c < 3; ++c)
    for (int z = 0; z < 256; ++z) {
      const float v = log_response[256 * c + z];
      if (!std::isfinite(v)) return fail_noctx(TM_EINVAL, "tm_merge_exposures: response table must be finite");
      a.g[c][z] = v;
    }
  Image o;
  o.p = out->data;
  o.W = width;
  o.H = height;
  o.pitch = out->pitch;
  o.dtype = out->dtype;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long N = (long long)width * height;
  const long long want = (N + kMT - 1) / kMT, cap = 8LL * (sms > 0 ? sms : 1);
  k_merge<<<(int)(want < cap ? want : cap), kMT, 0, static_cast<cudaStream_t>(stream)>>>(a, o);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_noctx(TM_ECUDA, "tm_merge_exposures: kernel launch failed");
  return TM_OK;
}
