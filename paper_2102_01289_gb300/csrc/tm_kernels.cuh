// tm_kernels.cuh -- host-side launchers of the tone-mapping kernels.
#pragma once

#include "tm_common.cuh"

namespace tmk {

// Stage a0: range of Eq. 11 luminance, bin edges, quantisation constants.
void launch_range(const Image &in, Stats *st, int n_bins, int qbits, cudaStream_t s);
// Stage a1: bin map (uint8) and quantised normalised log (int32).
void launch_prep(const Image &in, const Stats *st, int n_bins, int qbits, uint8_t *bins,
                 int32_t *q, cudaStream_t s);

// Stage a2 (Eq. 5): integral images of q and q^2, (H+1) x (W+1) int64.
// `scratch` holds at least integral_scratch_elems(W, H) int64 elements.
size_t integral_scratch_elems(int W, int H);
int launch_integral_image(const int32_t *q, int W, int H, int64_t *s1, int64_t *s2,
                          int64_t *scratch, cudaStream_t s);

// Stage a3 (Eq. 7-8): integral histogram planes, (H+1) x (W+1) uint32 each.
// cumulative = true: planes k = 1..n-1 hold the integral of [b < k];
// cumulative = false: planes k = 0..n-1 hold the integral of [b == k].
// `scratch` holds at least hist_scratch_elems(W, H, planes) uint32 elements.
size_t hist_scratch_elems(int W, int H, int planes);
int launch_integral_histogram(const uint8_t *bins, int W, int H, int n_bins, bool cumulative,
                              uint32_t *planes, uint32_t *scratch, cudaStream_t s);

// Debug planes written by the lookup kernels (each may be null).
struct DebugPlanes {
  unsigned *cnt;   // s * H * W
  float *sigma2;   // s * H * W
  float *weight;   // s * H * W
  float *lf;       // s * H * W
  float *l;        // H * W
};

// Stage a4 over materialised structures: per-pixel multi-field lookup, tone
// curve, fusion and colour restoration.
int launch_lookup_materialised(const Image &in, const Image &out, const DevParams &P,
                               const uint8_t *bins, const uint32_t *cplanes,
                               const int64_t *s1, const int64_t *s2, const DebugPlanes &dbg,
                               cudaStream_t s);

}  // namespace tmk
