// tm_backward.cu -- hand-written adjoint of the forward operator.
//
// With the bin map held fixed (bins are piecewise constant in the input), the
// output is a smooth function of the input RGB and of the parameters
// (min/max L_d, sat, eps_i, alpha_i). Loss gradient g = dLoss/d(out):
//   Eq. 12  out_c = rho_c^sat L, rho_c = C_c / i:
//           gL = sum_c g_c rho_c^sat; d/dsat; direct terms into C_c and i.
//   Eq. 3   L = sum W_f L_f / sum W_f: dL/dL_f = W_f / sum W, dL/dW_f =
//           (L_f - L) / sum W (equal weights when sum W = 0: no W terms).
//   Eq. 2   L_f = Ld_min + (Ld_max - Ld_min) P_f.
//   Eq. 4   W_f = alpha_f s_f / (s_f + eps_f), s_f the window variance.
//   Eq. 10  s_f(p) = (1/N) sum_{r in w_f(p)} (lhat_r - mu_f(p))^2, so
//           dLoss/dlhat_r = sum_f sum_{p : r in w_f(p)} (2 gs_f(p) / N_f(p))
//                           (lhat_r - mu_f(p))
//           = sum_f [lhat_r Box_f(u_f)(r) - Box_f(v_f)(r)],
//           u_f = 2 gs_f / N_f, v_f = u_f mu_f. The windows are symmetric, so
//           the adjoint of the window sum is the same clipped box sum around
//           r (the reversed scan of the integral image, Eq. 5-6). The box sums
//           of u and v come from integral images of u and v in 64-bit fixed
//           point, one binary scale per plane chosen from its largest |value|
//           so that every window sum fits in 62 bits; the sums are exact
//           modulo 2^64, so only the conversion to fixed point rounds.
//   lhat    = (ln i - ln imin) / D: dlhat/di = 1 / (i D), plus the range terms
//           through ln imin and ln imax, routed to the first pixel (raster
//           order) holding imin / imax.
//   Eq. 11  i = 0.2126 R + 0.7152 G + 0.0722 B (no gradient where floored).
// Per-pixel arithmetic is FP32 (FP64 throughput is a small fraction of FP32
// on this part). Parameter gradients are summed per block in FP32 and the
// block sums added into FP64 accumulators with one atomic each.
#include "tm_backward.cuh"

namespace tmk {
namespace {

constexpr int kBT = 256;
constexpr int kWarpsB = kBT / 32;

__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Per pixel: forward recomputation, Eq. 12/3/2/4 adjoints, u_f and v_f,
// direct gradients of the colour restoration, parameter partial sums and the
// largest |u_f|, |v_f| (for the fixed-point scales). NF = number of fields
// (so every per-field array lives in registers). Six blocks per SM (40
// registers at three fields, a few spilled): 2% faster per batch adjoint than
// the unbounded 61 registers at four blocks.
template <int NF>
__global__ void __launch_bounds__(kBT, 6) k_bwd_pixel(DevParams P, Job J, BwdJob B) {
  constexpr int kA = 3 + 2 * NF;  // [ld_min, ld_max, sat, eps[NF], alpha[NF]], the layout of BwdAcc::g
  __shared__ float sh[kA][kWarpsB];
  __shared__ unsigned shm[2 * NF][kWarpsB];
  const int W = J.in.W, H = J.in.H;
  const long long N = (long long)W * H;
  const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float acc[kA];
  unsigned amax[2 * NF];
#pragma unroll
  for (int k = 0; k < kA; ++k) acc[k] = 0.f;
#pragma unroll
  for (int k = 0; k < 2 * NF; ++k) amax[k] = 0u;
  if (pix < N) {
    const int y = (int)(pix / W), x = (int)(pix - (long long)y * W);
    const float inv_scale = ldexpf(1.f, -J.qbits);
    const float inv_scale2 = inv_scale * inv_scale;
    const long long W1 = (long long)W + 1;
    float Pf[NF], rarea[NF], var[NF], mu[NF], wv[NF], lf[NF];
    float wsum = 0.f, accL = 0.f, meanL = 0.f;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const unsigned cnt = load_count(J, f, pix);
      Win w = window_of(P, f, x, y, W, H);
      const long long iA = (long long)w.y0 * W1 + w.x0, iB = (long long)w.y0 * W1 + w.x1 + 1;
      const long long iC = (long long)(w.y1 + 1) * W1 + w.x1 + 1, iD = (long long)(w.y1 + 1) * W1 + w.x0;
      unsigned long long Nw = (unsigned long long)(w.x1 - w.x0 + 1) * (w.y1 - w.y0 + 1);
      const longlong2 *s12 = reinterpret_cast<const longlong2 *>(J.s1);  // interleaved (q, q^2) sums
      const longlong2 a = s12[iA], b = s12[iB], c = s12[iC], d = s12[iD];
      long long q1 = (long long)((unsigned long long)c.x - (unsigned long long)d.x - (unsigned long long)b.x +
                                 (unsigned long long)a.x);
      long long q2 = (long long)((unsigned long long)c.y - (unsigned long long)d.y - (unsigned long long)b.y +
                                 (unsigned long long)a.y);
      literal_area(P, f, J.qbits, q1, q2, Nw);  // Algorithm 1's area: zero padding
      rarea[f] = __frcp_rn((float)Nw);
      var[f] = window_variance(q1, q2, Nw, rarea[f], inv_scale2);
      mu[f] = (float)q1 * rarea[f] * inv_scale + 0.5f;  // mean of lhat
      // Eq. 1, 2, 4 and the sums of Eq. 3, as in the forward
      Pf[f] = (float)cnt * rarea[f];
      lf[f] = fmaf(P.ld_max - P.ld_min, Pf[f], P.ld_min);
      wv[f] = __fdividef(P.alpha[f] * var[f], var[f] + P.eps[f]);
      wsum += wv[f];
      accL = fmaf(wv[f], lf[f], accL);
      meanL += lf[f];
    }
    const float L = wsum > 0.f ? __fdividef(accL, wsum) : __fdividef(meanL, (float)NF);
    // Eq. 12
    float rgb[3];
    load_rgb(J.in, x, y, rgb[0], rgb[1], rgb[2]);
    const float pr = __fmul_rn(0.2126f, rgb[0]), pg = __fmul_rn(0.7152f, rgb[1]), pb = __fmul_rn(0.0722f, rgb[2]);
    const float raw = __fadd_rn(__fadd_rn(pr, pg), pb);
    const float i = fmaxf(raw, kLumFloor);
    const float inv_i = __frcp_rn(i);
    const float *go = static_cast<const float *>(B.grad_out.p) + (long long)y * B.grad_out.pitch + 3LL * x;
    float gL = 0.f, gi_direct = 0.f, gC[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float g = go[c];
      const float rho = rgb[c] * inv_i;
      gC[c] = 0.f;
      if (!(rho > 0.f)) {
        if (P.sat == 0.f) gL += g;
        continue;
      }
      const float rs = exp2f(P.sat * __log2f(rho));
      gL += g * rs;
      acc[2] += g * rs * __logf(rho) * L;
      gC[c] = g * P.sat * rs * L * inv_i / rho;
      gi_direct -= g * P.sat * rs * L * inv_i;
    }
    // Eq. 3, 2, 4
    const float rws = wsum > 0.f ? 1.f / wsum : 0.f;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const float dLdLf = wsum > 0.f ? wv[f] * rws : 1.f / (float)NF;
      const float dLdW = (lf[f] - L) * rws;
      acc[0] += gL * dLdLf * (1.f - Pf[f]);
      acc[1] += gL * dLdLf * Pf[f];
      const float gW = gL * dLdW;
      const float v = var[f], e = P.eps[f], a = P.alpha[f];
      const float den = (v + e) * (v + e);
      acc[3 + f] += gW * (-a * v / den);
      acc[3 + NF + f] += gW * (v / (v + e));
      const float gv = gW * a * e / den;
      const float u = 2.f * gv * rarea[f];
      const float vv = u * mu[f];
      B.U[f * N + pix] = u;
      B.V[f * N + pix] = vv;
      amax[f] = max(amax[f], __float_as_uint(fabsf(u)));
      amax[NF + f] = max(amax[NF + f], __float_as_uint(fabsf(vv)));
    }
    B.gi_direct[pix] = gi_direct;
    float *gin = static_cast<float *>(B.grad_in.p) + (long long)y * B.grad_in.pitch + 3LL * x;
    if (B.grad_in.p) {
      gin[0] = gC[0];
      gin[1] = gC[1];
      gin[2] = gC[2];
    }
    // first pixel (raster order) holding the range extremes
    if (i == J.st->imin) atomicMin(&B.acc->argmin, (unsigned long long)pix);
    if (i == J.st->imax) atomicMin(&B.acc->argmax, (unsigned long long)pix);
  }
  // block sums of the parameter partials and block maxima of |u|, |v|
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kA; ++k) {
    const float t = warp_sum(acc[k]);
    if (lane == 0) sh[k][wid] = t;
  }
#pragma unroll
  for (int k = 0; k < 2 * NF; ++k) {
    const unsigned t = __reduce_max_sync(0xffffffffu, amax[k]);
    if (lane == 0) shm[k][wid] = t;
  }
  __syncthreads();
  const int t = threadIdx.x;
  if (t < kA) {
    float sum = 0.f;
    for (int w = 0; w < kWarpsB; ++w) sum += sh[t][w];
    atomicAdd(&B.acc->g[t], (double)sum);
  } else if (t >= 32 && t < 32 + 2 * NF) {
    const int k = t - 32;
    unsigned m = 0u;
    for (int w = 0; w < kWarpsB; ++w) m = max(m, shm[k][w]);
    if (m) atomicMax(&B.acc->amax[k < NF ? k : kMaxFields + (k - NF)], m);
  }
}

// Per pixel: the adjoint of the window variances, through the normalised log,
// into the luminance and Eq. 11; range-term partial sums.
template <int NF>
__global__ void __launch_bounds__(kBT) k_bwd_input(DevParams P, Job J, BwdJob B) {
  __shared__ float sh[2][kWarpsB];
  const int W = J.in.W, H = J.in.H;
  const long long N = (long long)W * H;
  const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  // D = ln imax - ln imin = ln 2 x 2^Q / log2_scale (log2_scale = 2^Q / log2(imax / imin))
  const float l2s = J.st->log2_scale;
  const float D = J.st->imax > J.st->imin && l2s > 0.f ? 0.69314718f * ldexpf(1.f, J.qbits) / l2s : 0.f;
  float acc_lmin = 0.f, acc_lmax = 0.f;
  if (pix < N) {
    const int y = (int)(pix / W), x = (int)(pix - (long long)y * W);
    float r, g, b;
    load_rgb(J.in, x, y, r, g, b);
    const float raw = __fadd_rn(__fadd_rn(__fmul_rn(0.2126f, r), __fmul_rn(0.7152f, g)), __fmul_rn(0.0722f, b));
    float gi = B.gi_direct[pix];
    if (D > 0.f) {
      const long long W1 = (long long)W + 1, plane = W1 * ((long long)H + 1);
      const float lh = (float)J.q[pix] * ldexpf(1.f, -J.qbits) + 0.5f;
      float gl = 0.f;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        Win w = window_of(P, f, x, y, W, H);
        const long long iA = (long long)w.y0 * W1 + w.x0, iB = (long long)w.y0 * W1 + w.x1 + 1;
        const long long iC = (long long)(w.y1 + 1) * W1 + w.x1 + 1, iD = (long long)(w.y1 + 1) * W1 + w.x0;
        const unsigned long long *IU = B.IU + (long long)f * plane, *IV = B.IV + (long long)f * plane;
        const long long bu = (long long)(IU[iC] - IU[iD] - IU[iB] + IU[iA]);
        const long long bv = (long long)(IV[iC] - IV[iD] - IV[iB] + IV[iA]);
        const float nmax = window_max(P, f, W, H);
        const float fu = ldexpf(__ll2float_rn(bu), -fix_shift(B.acc->amax[f], nmax));
        const float fv = ldexpf(__ll2float_rn(bv), -fix_shift(B.acc->amax[kMaxFields + f], nmax));
        gl += lh * fu - fv;
      }
      const float i = fmaxf(raw, kLumFloor);
      gi += gl / (i * D);
      acc_lmin = gl * (lh - 1.f) / D;
      acc_lmax = -gl * lh / D;
    }
    // degenerate range: only the direct colour-restoration term reaches i
    if (B.grad_in.p && raw > kLumFloor) {
      float *gin = static_cast<float *>(B.grad_in.p) + (long long)y * B.grad_in.pitch + 3LL * x;
      gin[0] += 0.2126f * gi;
      gin[1] += 0.7152f * gi;
      gin[2] += 0.0722f * gi;
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  acc_lmin = warp_sum(acc_lmin);
  acc_lmax = warp_sum(acc_lmax);
  if (lane == 0) {
    sh[0][wid] = acc_lmin;
    sh[1][wid] = acc_lmax;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    float sum = 0.f;
    for (int w = 0; w < kWarpsB; ++w) sum += sh[threadIdx.x][w];
    atomicAdd(threadIdx.x == 0 ? &B.acc->lmin : &B.acc->lmax, (double)sum);
  }
}

// Range terms at the argmin / argmax pixels, and the parameter gradients.
__global__ void k_bwd_finish(DevParams P, Job J, BwdJob B) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int W = J.in.W;
  const float imin = J.st->imin, imax = J.st->imax;
  if (imax > imin && B.grad_in.p) {
    const unsigned long long idx[2] = {B.acc->argmin, B.acc->argmax};
    const double gterm[2] = {B.acc->lmin / (double)imin, B.acc->lmax / (double)imax};
    for (int k = 0; k < 2; ++k) {
      const long long pix = (long long)idx[k];
      const int y = (int)(pix / W), x = (int)(pix - (long long)y * W);
      float r, g, b;
      load_rgb(J.in, x, y, r, g, b);
      const float raw = __fadd_rn(__fadd_rn(__fmul_rn(0.2126f, r), __fmul_rn(0.7152f, g)), __fmul_rn(0.0722f, b));
      if (!(raw > kLumFloor)) continue;
      float *gin = static_cast<float *>(B.grad_in.p) + (long long)y * B.grad_in.pitch + 3LL * x;
      gin[0] += (float)(0.2126 * gterm[k]);
      gin[1] += (float)(0.7152 * gterm[k]);
      gin[2] += (float)(0.0722 * gterm[k]);
    }
  }
  if (B.grad_params)
    for (int k = 0; k < 3 + 2 * P.n_fields; ++k) B.grad_params[k] = (float)B.acc->g[k];
}

}  // namespace

int launch_backward(const DevParams &P, const Job &J, const BwdJob &B, cudaStream_t s) {
  const long long N = (long long)J.in.W * J.in.H;
  const int blocks = (int)((N + kBT - 1) / kBT);
  switch (P.n_fields) {
#define TM_BWD_PIXEL(nf) case nf: k_bwd_pixel<nf><<<blocks, kBT, 0, s>>>(P, J, B); break;
    TM_BWD_PIXEL(1) TM_BWD_PIXEL(2) TM_BWD_PIXEL(3) TM_BWD_PIXEL(4) TM_BWD_PIXEL(5) TM_BWD_PIXEL(6)
    TM_BWD_PIXEL(7) default: k_bwd_pixel<8><<<blocks, kBT, 0, s>>>(P, J, B); break;
#undef TM_BWD_PIXEL
  }
  const int W = J.in.W, H = J.in.H;
  // the integral planes of u_f and v_f in fixed point (IV = IU + s planes),
  // over tiles, one (u_f, v_f) pair per grid row
  float nmax[kMaxFields];
  for (int f = 0; f < P.n_fields; ++f) nmax[f] = window_max(P, f, W, H);
  const int nc = launch_fix_integrals(B.U, B.V, W, H, P.n_fields, B.acc->amax, nmax, B.IU,
                                      reinterpret_cast<long long *>(B.colscr), s);
  switch (P.n_fields) {
#define TM_BWD_INPUT(nf) case nf: k_bwd_input<nf><<<blocks, kBT, 0, s>>>(P, J, B); break;
    TM_BWD_INPUT(1) TM_BWD_INPUT(2) TM_BWD_INPUT(3) TM_BWD_INPUT(4) TM_BWD_INPUT(5) TM_BWD_INPUT(6)
    TM_BWD_INPUT(7) default: k_bwd_input<8><<<blocks, kBT, 0, s>>>(P, J, B); break;
#undef TM_BWD_INPUT
  }
  k_bwd_finish<<<1, 32, 0, s>>>(P, J, B);
  return 3 + nc;
}

}  // namespace tmk
