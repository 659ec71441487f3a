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
//           of u and v come from FP64 integral images.
//   lhat    = (ln i - ln imin) / D: dlhat/di = 1 / (i D), plus the range terms
//           through ln imin and ln imax, routed to the first pixel (raster
//           order) holding imin / imax.
//   Eq. 11  i = 0.2126 R + 0.7152 G + 0.0722 B (no gradient where floored).
// Parameter gradients are reduced in FP64 per block and added with atomics.
#include "tm_backward.cuh"

namespace tmk {
namespace {

constexpr int kBT = 256;

__device__ __forceinline__ double block_sum_d(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (int)(blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  return t;  // valid in thread 0
}

// Per pixel: forward recomputation, Eq. 12/3/2/4 adjoints, u_f and v_f,
// direct gradients of the colour restoration, parameter partial sums.
__global__ void __launch_bounds__(kBT) k_bwd_pixel(DevParams P, Job J, BwdJob B) {
  __shared__ double sh[32];
  const int W = J.in.W, H = J.in.H;
  const long long N = (long long)W * H;
  const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int s = P.n_fields;
  double acc_ld0 = 0.0, acc_ld1 = 0.0, acc_sat = 0.0, acc_eps[kMaxFields], acc_alpha[kMaxFields];
#pragma unroll
  for (int f = 0; f < kMaxFields; ++f) acc_eps[f] = acc_alpha[f] = 0.0;
  if (pix < N) {
    const int y = (int)(pix / W), x = (int)(pix - (long long)y * W);
    const SweepPlan &S = J.plan;
    const float inv_scale = ldexpf(1.f, -J.qbits);
    const float inv_scale2 = inv_scale * inv_scale;
    unsigned cnt[kMaxFields];
#pragma unroll
    for (int f = 0; f < kMaxFields; ++f) cnt[f] = 0u;
    for (int sl = 0; sl < S.nslabs; ++sl) {
      const int T = max(y + S.slab_a[sl] - 1, -1), Bb = min(y + S.slab_b[sl], H - 1);
      if (Bb > T) cnt[S.slab_field[sl]] += J.counts[sl * N + pix];
    }
    const long long W1 = (long long)W + 1;
    float area[kMaxFields], var[kMaxFields], mu[kMaxFields];
#pragma unroll
    for (int f = 0; f < kMaxFields; ++f) {
      if (f >= s) break;
      Win w = window_of(P, f, x, y, W, H);
      const long long iA = (long long)w.y0 * W1 + w.x0, iB = (long long)w.y0 * W1 + w.x1 + 1;
      const long long iC = (long long)(w.y1 + 1) * W1 + w.x1 + 1, iD = (long long)(w.y1 + 1) * W1 + w.x0;
      const unsigned long long Nw = (unsigned long long)(w.x1 - w.x0 + 1) * (w.y1 - w.y0 + 1);
      const long long q1 = (long long)((unsigned long long)J.s1[iC] - (unsigned long long)J.s1[iD] -
                                       (unsigned long long)J.s1[iB] + (unsigned long long)J.s1[iA]);
      const long long q2 = (long long)((unsigned long long)J.s2[iC] - (unsigned long long)J.s2[iD] -
                                       (unsigned long long)J.s2[iB] + (unsigned long long)J.s2[iA]);
      area[f] = (float)Nw;
      var[f] = window_variance(q1, q2, area[f], Nw, inv_scale2);
      mu[f] = (float)((double)q1 / (double)Nw) * inv_scale + 0.5f;  // mean of lhat
    }
    float wv[kMaxFields], lf[kMaxFields];
    const float L = fuse_fields(P, cnt, area, var, wv, lf);
    float wsum = 0.f;
    for (int f = 0; f < s; ++f) wsum += wv[f];
    // Eq. 12
    float rgb[3];
    load_rgb(J.in, x, y, rgb[0], rgb[1], rgb[2]);
    const float pr = __fmul_rn(0.2126f, rgb[0]), pg = __fmul_rn(0.7152f, rgb[1]), pb = __fmul_rn(0.0722f, rgb[2]);
    const float raw = __fadd_rn(__fadd_rn(pr, pg), pb);
    const float i = fmaxf(raw, kLumFloor);
    const float inv_i = __frcp_rn(i);
    const float *go = static_cast<const float *>(B.grad_out.p) + (long long)y * B.grad_out.pitch + 3LL * x;
    float gL = 0.f, gi_direct = 0.f, gC[3];
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
      acc_sat += (double)g * rs * __logf(rho) * L;
      gC[c] = g * P.sat * rs * L * inv_i / rho;
      gi_direct -= g * P.sat * rs * L * inv_i;
    }
    // Eq. 3, 2, 4
    const float span = P.ld_max - P.ld_min;
    for (int f = 0; f < s; ++f) {
      const float Pf = (float)cnt[f] / area[f];
      const float dLdLf = wsum > 0.f ? wv[f] / wsum : 1.f / (float)s;
      const float dLdW = wsum > 0.f ? (lf[f] - L) / wsum : 0.f;
      acc_ld0 += (double)gL * dLdLf * (1.f - Pf);
      acc_ld1 += (double)gL * dLdLf * Pf;
      const float gW = gL * dLdW;
      const float v = var[f], e = P.eps[f], a = P.alpha[f];
      const float den = (v + e) * (v + e);
      acc_eps[f] += (double)gW * (-a * v / den);
      acc_alpha[f] += (double)gW * (v / (v + e));
      const float gv = gW * a * e / den;
      const float u = 2.f * gv / area[f];
      B.U[f * N + pix] = u;
      B.V[f * N + pix] = u * mu[f];
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
  // parameter partial sums
  double t = block_sum_d(acc_ld0, sh);
  if (threadIdx.x == 0) atomicAdd(&B.acc->g[0], t);
  t = block_sum_d(acc_ld1, sh);
  if (threadIdx.x == 0) atomicAdd(&B.acc->g[1], t);
  t = block_sum_d(acc_sat, sh);
  if (threadIdx.x == 0) atomicAdd(&B.acc->g[2], t);
  for (int f = 0; f < s; ++f) {
    t = block_sum_d(acc_eps[f], sh);
    if (threadIdx.x == 0) atomicAdd(&B.acc->g[3 + f], t);
    t = block_sum_d(acc_alpha[f], sh);
    if (threadIdx.x == 0) atomicAdd(&B.acc->g[3 + s + f], t);
  }
}

// Row prefixes of the float planes u_f, v_f into FP64 integral planes.
__global__ void __launch_bounds__(kBT) k_rows_f64(const float *__restrict__ src, int W, int H,
                                                  double *__restrict__ dst) {
  __shared__ double wt[kBT / 32];
  const long long W1 = (long long)W + 1, plane = W1 * ((long long)H + 1);
  const int y = blockIdx.x, pl = blockIdx.y;
  const float *row = src + (long long)pl * W * H + (long long)y * W;
  double *P = dst + (long long)pl * plane;
  if (y == 0)
    for (long long x = threadIdx.x; x < W1; x += kBT) P[x] = 0.0;
  double *o = P + (long long)(y + 1) * W1;
  if (threadIdx.x == 0) o[0] = 0.0;
  double carry = 0.0;
  for (int base = 0; base < W; base += kBT) {
    const int x = base + threadIdx.x;
    const double v = x < W ? (double)row[x] : 0.0;
    double sc = v;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int off = 1; off < 32; off <<= 1) {
      const double nb = __shfl_up_sync(0xffffffffu, sc, off);
      if (lane >= off) sc += nb;
    }
    if (lane == 31) wt[wid] = sc;
    __syncthreads();
    double before = 0.0, total = 0.0;
    for (int k = 0; k < kBT / 32; ++k) {
      if (k < wid) before += wt[k];
      total += wt[k];
    }
    if (x < W) o[x + 1] = carry + before + sc;
    carry += total;
    __syncthreads();
  }
}

// Per pixel: the adjoint of the window variances, through the normalised log,
// into the luminance and Eq. 11; range-term partial sums.
__global__ void __launch_bounds__(kBT) k_bwd_input(DevParams P, Job J, BwdJob B) {
  __shared__ double sh[32];
  const int W = J.in.W, H = J.in.H;
  const long long N = (long long)W * H;
  const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const float imin = J.st->imin, imax = J.st->imax;
  const double D = imax > imin ? log((double)imax) - log((double)imin) : 0.0;
  double acc_lmin = 0.0, acc_lmax = 0.0;
  if (pix < N && D > 0.0) {
    const int y = (int)(pix / W), x = (int)(pix - (long long)y * W);
    const long long W1 = (long long)W + 1, plane = W1 * ((long long)H + 1);
    const double lh = (double)J.q[pix] * ldexp(1.0, -J.qbits) + 0.5;
    double gl = 0.0;
    for (int f = 0; f < P.n_fields; ++f) {
      Win w = window_of(P, f, x, y, W, H);
      const long long iA = (long long)w.y0 * W1 + w.x0, iB = (long long)w.y0 * W1 + w.x1 + 1;
      const long long iC = (long long)(w.y1 + 1) * W1 + w.x1 + 1, iD = (long long)(w.y1 + 1) * W1 + w.x0;
      const double *IU = B.IU + (long long)f * plane, *IV = B.IV + (long long)f * plane;
      const double bu = IU[iC] - IU[iD] - IU[iB] + IU[iA];
      const double bv = IV[iC] - IV[iD] - IV[iB] + IV[iA];
      gl += lh * bu - bv;
    }
    float r, g, b;
    load_rgb(J.in, x, y, r, g, b);
    const float raw = __fadd_rn(__fadd_rn(__fmul_rn(0.2126f, r), __fmul_rn(0.7152f, g)), __fmul_rn(0.0722f, b));
    const float i = fmaxf(raw, kLumFloor);
    const double gi = gl / ((double)i * D) + (double)B.gi_direct[pix];
    acc_lmin = gl * (lh - 1.0) / D;
    acc_lmax = -gl * lh / D;
    if (B.grad_in.p && raw > kLumFloor) {
      float *gin = static_cast<float *>(B.grad_in.p) + (long long)y * B.grad_in.pitch + 3LL * x;
      gin[0] += (float)(0.2126 * gi);
      gin[1] += (float)(0.7152 * gi);
      gin[2] += (float)(0.0722 * gi);
    }
  } else if (pix < N && B.grad_in.p) {
    // degenerate range: only the direct colour-restoration term reaches i
    const int y = (int)(pix / W), x = (int)(pix - (long long)y * W);
    float r, g, b;
    load_rgb(J.in, x, y, r, g, b);
    const float raw = __fadd_rn(__fadd_rn(__fmul_rn(0.2126f, r), __fmul_rn(0.7152f, g)), __fmul_rn(0.0722f, b));
    if (raw > kLumFloor) {
      const double gi = (double)B.gi_direct[pix];
      float *gin = static_cast<float *>(B.grad_in.p) + (long long)y * B.grad_in.pitch + 3LL * x;
      gin[0] += (float)(0.2126 * gi);
      gin[1] += (float)(0.7152 * gi);
      gin[2] += (float)(0.0722 * gi);
    }
  }
  double t = block_sum_d(acc_lmin, sh);
  if (threadIdx.x == 0) atomicAdd(&B.acc->lmin, t);
  t = block_sum_d(acc_lmax, sh);
  if (threadIdx.x == 0) atomicAdd(&B.acc->lmax, t);
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
  k_bwd_pixel<<<blocks, kBT, 0, s>>>(P, J, B);
  const int W = J.in.W, H = J.in.H;
  const long long plane = ((long long)W + 1) * ((long long)H + 1);
  dim3 rg(H, P.n_fields);
  k_rows_f64<<<rg, kBT, 0, s>>>(B.U, W, H, B.IU);
  k_rows_f64<<<rg, kBT, 0, s>>>(B.V, W, H, B.IV);
  // U and V integral planes are contiguous: one segmented column pass over 2s planes
  const int nc = launch_column_pass_f64(B.IU, plane, 2 * P.n_fields, W, H, B.colscr, s);
  k_bwd_input<<<blocks, kBT, 0, s>>>(P, J, B);
  k_bwd_finish<<<1, 32, 0, s>>>(P, J, B);
  return 5 + nc;
}

}  // namespace tmk
