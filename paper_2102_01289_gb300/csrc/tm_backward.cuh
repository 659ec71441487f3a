// tm_backward.cuh -- adjoint kernels of the forward operator.
#pragma once

#include "tm_kernels.cuh"

namespace tmk {

// Per-image accumulators of a backward call (cleared by its first launch:
// sums and maxima to 0, argmin / argmax to all ones).
struct BwdAcc {
  double lmin, lmax;              // dLoss/d ln imin, dLoss/d ln imax (times D)
  unsigned amax[2 * kMaxFields];  // float bits of max |u_f| (f) and max |v_f| (kMaxFields + f)
  unsigned long long argmin, argmax;
};

// Parameter-gradient sums of a backward call, over all its images:
// [d ld_min, d ld_max, d sat, d eps[s], d alpha[s]].
constexpr int kBwdParams = 3 + 2 * kMaxFields;

// One image of a backward batch: the forward intermediates the adjoint reads
// and the buffers it writes.
struct alignas(16) BwdJob {
  Image in;                     // the forward's input (float32 / float16 HWC)
  Image grad_out;               // float32 HWC
  Image grad_in;                // float32 HWC, p == nullptr to skip
  const Stats *st;              // the range state of the forward
  const int32_t *q;             // H*W quantised normalised log
  const longlong2 *s12;         // (H+1)*(W+1) integral images of q and q^2, interleaved
  const float2 *mom;            // the forward's window (variance, mean of lhat) per field, or
                                //   null: recomputed from s12
  const unsigned char *cnt;     // Eq. 1 numerators: plane f at cnt + cnt_off[f]
  long long cnt_off[kMaxFields];
  int cnt_wide;                 // bit f: plane f is uint32 (else uint16)
  int qbits;
  float *U, *V;                 // s x H x W: u_f = 2 dLoss/ds_f / N_f and u_f * mu_f
  float *gi_direct;             // H x W: dLoss/di through Eq. 12 directly
  const longlong2 *IUV;         // s pair planes of (H+1)*(W+1) positions: the fixed-point
                                //   integrals of u_f and v_f, interleaved
  BwdAcc *acc;
  int b0, b0_in;                // first block of this image in the two per-pixel launches
};
static_assert(sizeof(BwdJob) % 16 == 0, "jobs are copied in 16-byte words");

// Descriptors of a group: BwdJob[n] followed by FixJob[n], written by the
// setup launch from its kernel parameters (at most kBwdDescBytes per group).
constexpr int kBwdDescBytes = 24576;
constexpr int kBwdGroupMax = kBwdDescBytes / (int)(sizeof(BwdJob) + sizeof(FixJob));

// Blocks of the two per-pixel launches for one image.
int bwd_pixel_blocks(int W, int H);
int bwd_input_blocks(int W, int H);

// The adjoint of a group of n images given their forward intermediates, on
// one stream: launch_backward_setup (writes the group's descriptors `desc`,
// `bytes` of BwdJob[n] then FixJob[n], to device memory `dst`, clears the
// accumulators accs[n] and, first, the parameter sums gsum[kBwdParams]; -1
// if `bytes` exceeds kBwdDescBytes); launch_backward_pixel (per pixel: u_f,
// v_f, the direct gradients, the parameter sums; mom: every job's
// BwdJob::mom is set, else none is; plain: every job's input is float32 and
// its count planes uint32); launch_fix_integrals over the FixJobs
// (image i's reads U / V of job i and writes its IUV); launch_backward_input
// (the box sums back into the input, then the range terms and, when
// grad_params, device float[3 + 2s], is not null, the parameter gradients
// from gsum). Each returns its launches.
int launch_backward_setup(const void *desc, size_t bytes, void *dst, BwdAcc *accs, int n, double *gsum, bool first,
                          cudaStream_t s);
int launch_backward_pixel(const DevParams &P, const BwdJob *jobs, int n, int pix_blocks, bool mom, bool plain,
                          double *gsum, cudaStream_t s);
int launch_backward_input(const DevParams &P, const BwdJob *jobs, int n, int in_blocks, bool plain,
                          const double *gsum, float *grad_params, cudaStream_t s);

}  // namespace tmk
