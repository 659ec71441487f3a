// tm_backward.cuh -- adjoint kernels of the forward operator.
#pragma once

#include "tm_kernels.cuh"

namespace tmk {

// FP64 accumulators of one backward call (cleared before it: sums to 0,
// argmin/argmax to all ones).
// g accumulates over the images of a batch; the fields from lmin on are per
// image (lmin .. amax cleared to 0, argmin / argmax to all ones).
struct BwdAcc {
  double g[3 + 2 * kMaxFields];   // [d ld_min, d ld_max, d sat, d eps[s], d alpha[s]]
  double lmin, lmax;              // dLoss/d ln imin, dLoss/d ln imax (times D)
  unsigned amax[2 * kMaxFields];  // float bits of max |u_f| (f) and max |v_f| (kMaxFields + f)
  unsigned long long argmin, argmax;
};

// Buffers of one backward call.
struct BwdJob {
  Image grad_out;      // float32 HWC
  Image grad_in;       // float32 HWC, p == nullptr to skip
  float *grad_params;  // device float[3 + 2s] or nullptr
  float *U, *V;        // s x H x W: u_f = 2 dLoss/ds_f / N_f and u_f * mu_f
  float *gi_direct;    // H x W: dLoss/di through Eq. 12 directly
  unsigned long long *IU, *IV;  // fixed-point integral planes of u_f and v_f: s planes of
                                //   (H+1) x (W+1) each, contiguous (IV = IU + s planes)
  unsigned long long *colscr;   // tile sums of the integral planes, fix_integral_scratch_elems(W, H, s)
  BwdAcc *acc;
};

// Launch the adjoint given the forward intermediates of `J` (bins, q, integral
// images, slab counts, range state). Returns the number of launches.
int launch_backward(const DevParams &P, const Job &J, const BwdJob &B, cudaStream_t s);

}  // namespace tmk
