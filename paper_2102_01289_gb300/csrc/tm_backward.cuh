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
  const unsigned char *cnt;     // Eq. 1 numerators: plane f at cnt + cnt_off[f]
  long long cnt_off[kMaxFields];
  int cnt_wide;                 // bit f: plane f is uint32 (else uint16)
  int qbits;
  float *U, *V;                 // s x H x W: u_f = 2 dLoss/ds_f / N_f and u_f * mu_f
  float *gi_direct;             // H x W: dLoss/di through Eq. 12 directly
  const longlong2 *IUV;         // s pair planes of (H+1)*(W+1) positions: the fixed-point
                                //   integrals of u_f and v_f, interleaved
  BwdAcc *acc;
  int b0;                       // first block of this image in the per-pixel launches
  int pad_;
};
static_assert(sizeof(BwdJob) % 16 == 0, "jobs are copied in 16-byte words");

// Blocks of the per-pixel launches for one image.
int bwd_pixel_blocks(int W, int H);

// The adjoint of a batch of images given their forward intermediates:
// `jobs` / `fix` (device, n each; the FixJob of image i reads U / V of job i
// and writes its IUV), `accs` (device, n), `gsum` (device, kBwdParams).
// first: clear gsum; grad_params (device float[3 + 2s]) or null: written
// from gsum at the end. Returns the number of launches.
int launch_backward(const DevParams &P, const BwdJob *jobs, const FixJob *fix, int n, int pix_blocks,
                    int tile_blocks, int col_blocks, BwdAcc *accs, double *gsum, bool first,
                    float *grad_params, cudaStream_t s);

}  // namespace tmk
