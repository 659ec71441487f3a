// tm_lookup.cu -- per-pixel multi-field lookup over materialised structures.
//
// One thread per pixel. For every field the clipped window's four corners are
// read from the cumulative integral histogram plane of the pixel's own bin
// (C_b = sum_{k < b} H_k, so Eq. 1's numerator is one box sum, Eq. 9) and
// from the integral images of q and q^2 (Eq. 6); then Eq. 2, Eq. 4 with the
// exact window variance (Eq. 10), the fusion of Eq. 3 and the colour
// restoration of Eq. 12. The fields are evaluated in one pass instead of the
// paper's per-scale loop (Section III-A).
#include "tm_kernels.cuh"

namespace tmk {
namespace {

__global__ void __launch_bounds__(256)
    k_lookup_materialised(Image in, Image out, DevParams P, const uint8_t *__restrict__ bins,
                          const unsigned *__restrict__ cplanes, const long long *__restrict__ s1,
                          const long long *__restrict__ s2, DebugPlanes dbg) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int W = in.W, H = in.H;
  if (x >= W || y >= H) return;
  const long long W1 = (long long)W + 1;
  const long long plane = W1 * ((long long)H + 1);
  const long long pix = (long long)y * W + x;
  const int b = bins[pix];
  const unsigned *C = b > 0 ? cplanes + (long long)(b - 1) * plane : nullptr;
  const float inv_scale2 = ldexpf(1.f, -2 * P.qbits);

  unsigned cnt[kMaxFields];
  float area[kMaxFields], var[kMaxFields];
#pragma unroll
  for (int f = 0; f < kMaxFields; ++f) {
    if (f >= P.n_fields) break;
    Win w = window_of(P, f, x, y, W, H);
    const long long iA = (long long)w.y0 * W1 + w.x0;
    const long long iB = (long long)w.y0 * W1 + w.x1 + 1;
    const long long iC = (long long)(w.y1 + 1) * W1 + w.x1 + 1;
    const long long iD = (long long)(w.y1 + 1) * W1 + w.x0;
    const unsigned long long N = (unsigned long long)(w.x1 - w.x0 + 1) * (w.y1 - w.y0 + 1);
    cnt[f] = C ? (C[iC] - C[iD] - C[iB] + C[iA]) : 0u;
    long long q1 = (long long)((unsigned long long)s1[iC] - (unsigned long long)s1[iD] -
                               (unsigned long long)s1[iB] + (unsigned long long)s1[iA]);
    long long q2 = (long long)((unsigned long long)s2[iC] - (unsigned long long)s2[iD] -
                               (unsigned long long)s2[iB] + (unsigned long long)s2[iA]);
    area[f] = (float)N;
    var[f] = window_variance(q1, q2, area[f], N, inv_scale2);
  }
  float wv[kMaxFields], lf[kMaxFields];
  const float L = fuse_fields(P, cnt, area, var, wv, lf);
  float r, g, bb;
  load_rgb(in, x, y, r, g, bb);
  const float i = luminance(r, g, bb);
  store_rgb(out, x, y, restore_channel(r, i, P.sat, L), restore_channel(g, i, P.sat, L),
            restore_channel(bb, i, P.sat, L));
  if (dbg.l) {
    const long long N = (long long)W * H;
    dbg.l[pix] = L;
    for (int f = 0; f < P.n_fields; ++f) {
      dbg.cnt[f * N + pix] = cnt[f];
      dbg.sigma2[f * N + pix] = var[f];
      dbg.weight[f * N + pix] = wv[f];
      dbg.lf[f * N + pix] = lf[f];
    }
  }
}

}  // namespace

int launch_lookup_materialised(const Image &in, const Image &out, const DevParams &P,
                               const uint8_t *bins, const uint32_t *cplanes, const int64_t *s1,
                               const int64_t *s2, const DebugPlanes &dbg, cudaStream_t s) {
  dim3 block(32, 8), grid((in.W + 31) / 32, (in.H + 7) / 8);
  k_lookup_materialised<<<grid, block, 0, s>>>(in, out, P, bins, cplanes,
                                               reinterpret_cast<const long long *>(s1),
                                               reinterpret_cast<const long long *>(s2), dbg);
  return 1;
}

}  // namespace tmk
