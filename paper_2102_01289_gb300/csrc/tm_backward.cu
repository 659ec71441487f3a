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
// Every stage runs once over the whole batch (block -> image through
// BwdJob::b0), so a batch of small images fills the GPU as one large one.
// Per-pixel arithmetic is FP32 (FP64 throughput is a small fraction of FP32
// on this part). Parameter gradients are summed per block in FP32 and the
// block sums added into FP64 accumulators with one atomic each.
#include <algorithm>
#include <cstring>

#include "tm_backward.cuh"

namespace tmk {
namespace {

// Per-pixel launches: 32 x 8 threads, each thread kRowsPix (kRowsIn) rows 8
// apart, so a block covers a 32 x (8 kRowsPix) tile (the block's reductions
// are paid once per kRowsPix pixels of a thread).
constexpr int kBT = 256;
constexpr int kWarpsB = kBT / 32;
constexpr int kRowsPix = 4, kRowsIn = 4;
constexpr int kMinBlocksPix = 4, kMinBlocksIn = 5;

__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int find_bwd(const BwdJob *jobs, int n, bool input, int blk) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((input ? jobs[mid].b0_in : jobs[mid].b0) <= blk) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// The group's descriptors from the kernel parameters, cleared accumulators
// and block counter, and (first) cleared parameter sums.
struct DescPack {
  unsigned w[kBwdDescBytes / 4];
};
template <int Words>
struct SmallPack {
  unsigned w[Words];
};
template <class Pack>
__global__ void k_bwd_setup(const __grid_constant__ Pack p, int words, unsigned *dst, BwdAcc *accs, int n,
                            double *gsum, int first) {
  for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = p.w[i];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    BwdAcc &a = accs[i];
    a.lmin = a.lmax = 0.0;
    for (int k = 0; k < 2 * kMaxFields; ++k) a.amax[k] = 0u;
    a.argmin = a.argmax = ~0ull;
  }
  if (first && threadIdx.x < kBwdParams) gsum[threadIdx.x] = 0.0;
}

// Per pixel: forward recomputation, Eq. 12/3/2/4 adjoints, u_f and v_f,
// direct gradients of the colour restoration, parameter partial sums and the
// largest |u_f|, |v_f| (for the fixed-point scales). NF = number of fields
// (so every per-field array lives in registers).
// MOM: the window variances and means come from the forward's planes.
// kPlain: the literal area is off, every window is small (P.small_win),
// every count plane is uint32 and every input is float32 (the other paths are
// then not compiled in).
template <int NF, bool MOM, bool kPlain>
__global__ void __launch_bounds__(kBT, kMinBlocksPix) k_bwd_pixel(DevParams P, const BwdJob *__restrict__ jobs, int njobs,
                                                   double *__restrict__ gsum) {
  constexpr int kA = 3 + 2 * NF;  // [ld_min, ld_max, sat, eps[NF], alpha[NF]], the layout of gsum
  __shared__ float sh[kA][kWarpsB];
  __shared__ unsigned shm[2 * NF][kWarpsB];
  const BwdJob &J = jobs[find_bwd(jobs, njobs, false, blockIdx.x)];
  const int W = J.in.W, H = J.in.H;
  const int lb = blockIdx.x - J.b0, bx = (W + 31) / 32;
  const int x = (lb % bx) * 32 + (threadIdx.x & 31);
  const int ybase = (lb / bx) * (8 * kRowsPix) + (threadIdx.x >> 5);
  const size_t N = (size_t)W * H;
  const float inv_scale = ldexpf(1.f, -J.qbits);
  const float inv_scale2 = inv_scale * inv_scale;
  const float imin = J.st->imin, imax = J.st->imax;
  const float span = P.ld_max - P.ld_min;
  float acc[kA];
  unsigned amax[2 * NF];
#pragma unroll
  for (int k = 0; k < kA; ++k) acc[k] = 0.f;
#pragma unroll
  for (int k = 0; k < 2 * NF; ++k) amax[k] = 0u;
  if (x < W) {
#pragma unroll 1
    for (int r = 0; r < kRowsPix; ++r) {
      const int y = ybase + 8 * r;
      if (y >= H) break;
      const unsigned pix = (unsigned)y * (unsigned)W + (unsigned)x;
      float Pf[NF], rarea[NF], var[NF], mu[NF], wv[NF], lf[NF];
      float wsum = 0.f, accL = 0.f, meanL = 0.f;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const unsigned cnt = kPlain ? __ldg(reinterpret_cast<const unsigned *>(J.cnt + J.cnt_off[f]) + pix)
                                    : load_count(J, f, pix);
        if (MOM) {
          const float2 vm = __ldg(J.mom + f * N + pix);
          var[f] = vm.x;
          mu[f] = vm.y;
          rarea[f] = __fdividef(1.f, window_area<!kPlain>(P, f, x, y, W, H));
        } else {
          const WinMoments m = window_moments<!kPlain, kPlain ? 1 : -1>(P, f, x, y, W, H, J.s12, J.qbits,
                                                                        inv_scale2);
          rarea[f] = m.rarea;
          var[f] = m.var;
          mu[f] = window_mean(m.q1, m.rarea, inv_scale);
        }
        // Eq. 1, 2, 4 and the sums of Eq. 3, as in the forward
        Pf[f] = (float)cnt * rarea[f];
        lf[f] = fmaf(span, Pf[f], P.ld_min);
        wv[f] = __fdividef(P.alpha[f] * var[f], var[f] + P.eps[f]);
        wsum += wv[f];
        accL = fmaf(wv[f], lf[f], accL);
        meanL += lf[f];
      }
      const float L = wsum > 0.f ? __fdividef(accL, wsum) : __fdividef(meanL, (float)NF);
      // Eq. 12
      float rgb[3];
      load_rgb<kPlain ? kF32 : -1>(J.in, x, y, rgb[0], rgb[1], rgb[2]);
      const float raw =
          __fadd_rn(__fadd_rn(__fmul_rn(0.2126f, rgb[0]), __fmul_rn(0.7152f, rgb[1])), __fmul_rn(0.0722f, rgb[2]));
      const float i = fmaxf(raw, kLumFloor);
      const float inv_i = __fdividef(1.f, i);
      const float *go = static_cast<const float *>(J.grad_out.p) + (long long)y * J.grad_out.pitch + 3LL * x;
      float gL = 0.f, gi_direct = 0.f, gC[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float g = __ldg(go + c);
        const float rho = rgb[c] * inv_i;
        gC[c] = 0.f;
        if (!(rho > 0.f)) {
          if (P.sat == 0.f) gL += g;
          continue;
        }
        const float lg = __log2f(rho);
        const float grs = g * exp2f(P.sat * lg);  // g rho^sat
        gL += grs;
        acc[2] += grs * lg * (0.69314718f * L);  // d/dsat: g rho^sat ln(rho) L
        const float t = grs * P.sat * L;         // g sat rho^sat L = dLoss/d ln rho
        gC[c] = __fdividef(t, rgb[c]);
        gi_direct -= t * inv_i;
      }
      // Eq. 3, 2, 4
      const float rws = wsum > 0.f ? __fdividef(1.f, wsum) : 0.f;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const float dLdLf = wsum > 0.f ? wv[f] * rws : 1.f / (float)NF;
        const float gLf = gL * dLdLf;
        acc[0] += gLf * (1.f - Pf[f]);
        acc[1] += gLf * Pf[f];
        const float gW = gL * (lf[f] - L) * rws;
        const float v = var[f], e = P.eps[f], a = P.alpha[f];
        const float ve = v + e;
        const float rden = __fdividef(1.f, ve * ve);
        acc[3 + f] -= gW * a * v * rden;
        acc[3 + NF + f] += gW * v * ve * rden;
        const float u = 2.f * (gW * a * e * rden) * rarea[f];
        const float vv = u * mu[f];
        J.U[f * N + pix] = u;
        J.V[f * N + pix] = vv;
        amax[f] = max(amax[f], __float_as_uint(fabsf(u)));
        amax[NF + f] = max(amax[NF + f], __float_as_uint(fabsf(vv)));
      }
      J.gi_direct[pix] = gi_direct;
      if (J.grad_in.p) {
        float *gin = static_cast<float *>(J.grad_in.p) + (long long)y * J.grad_in.pitch + 3LL * x;
        gin[0] = gC[0];
        gin[1] = gC[1];
        gin[2] = gC[2];
      }
      // first pixel (raster order) holding the range extremes
      if (i == imin) atomicMin(&J.acc->argmin, (unsigned long long)pix);
      if (i == imax) atomicMin(&J.acc->argmax, (unsigned long long)pix);
    }
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
    atomicAdd(&gsum[t < 3 + NF ? t : kMaxFields + t - NF], (double)sum);  // gsum: eps[kMaxFields], alpha[...]
  } else if (t >= 32 && t < 32 + 2 * NF) {
    const int k = t - 32;
    unsigned m = 0u;
    for (int w = 0; w < kWarpsB; ++w) m = max(m, shm[k][w]);
    if (m) atomicMax(&J.acc->amax[k < NF ? k : kMaxFields + (k - NF)], m);
  }
}

// Range terms at each image's argmin / argmax pixels (block j: image j), and
// the parameter gradients (block 0).
__global__ void k_bwd_finish(DevParams P, const BwdJob *__restrict__ jobs, const double *gsum,
                             float *grad_params) {
  if (threadIdx.x == 0) {
    const BwdJob &J = jobs[blockIdx.x];
    const int W = J.in.W;
    const float imin = J.st->imin, imax = J.st->imax;
    const bool range = imax > imin && J.grad_in.p;
    const unsigned long long idx[2] = {J.acc->argmin, J.acc->argmax};
    const double gterm[2] = {J.acc->lmin / (double)imin, J.acc->lmax / (double)imax};
    for (int k = 0; k < 2 && range; ++k) {
      if (idx[k] >= (unsigned long long)W * (unsigned long long)J.in.H) continue;  // no pixel held it
      const long long pix = (long long)idx[k];
      const int y = (int)(pix / W), x = (int)(pix - (long long)y * W);
      float r, g, b;
      load_rgb(J.in, x, y, r, g, b);
      const float raw = __fadd_rn(__fadd_rn(__fmul_rn(0.2126f, r), __fmul_rn(0.7152f, g)), __fmul_rn(0.0722f, b));
      if (!(raw > kLumFloor)) continue;
      float *gin = static_cast<float *>(J.grad_in.p) + (long long)y * J.grad_in.pitch + 3LL * x;
      gin[0] += (float)(0.2126 * gterm[k]);
      gin[1] += (float)(0.7152 * gterm[k]);
      gin[2] += (float)(0.0722 * gterm[k]);
    }
  }
  if (grad_params && blockIdx.x == 0 && threadIdx.x == 0) {
    const int nf = P.n_fields;
    for (int k = 0; k < 3; ++k) grad_params[k] = (float)gsum[k];
    for (int f = 0; f < nf; ++f) {
      grad_params[3 + f] = (float)gsum[3 + f];
      grad_params[3 + nf + f] = (float)gsum[3 + kMaxFields + f];
    }
  }
}

// Per pixel: the adjoint of the window variances, through the normalised log,
// into the luminance and Eq. 11; range-term partial sums. kDt: the dtype of
// every input when known at compile time (-1: read from the descriptors).
template <int NF, int kDt>
__global__ void __launch_bounds__(kBT, kMinBlocksIn) k_bwd_input(DevParams P, const BwdJob *__restrict__ jobs, int njobs) {
  __shared__ float sh[2][kWarpsB];
  __shared__ float scale[2 * NF][2];  // 2^-shift of each fixed-point plane, as two factors
  const BwdJob &J = jobs[find_bwd(jobs, njobs, true, blockIdx.x)];
  const int W = J.in.W, H = J.in.H;
  if (threadIdx.x < 2 * NF) {
    const int k = threadIdx.x, f = k < NF ? k : k - NF;
    // 2^-shift (shift in [-67, 209]) as two normal factors, so that
    // float(sum) x hi x lo rounds once, like ldexpf(float(sum), -shift)
    const int sh_ = fix_shift(J.acc->amax[k < NF ? k : kMaxFields + f], window_max(P, f, W, H));
    const int h = sh_ / 2;
    scale[k][0] = ldexpf(1.f, -h);
    scale[k][1] = ldexpf(1.f, h - sh_);
  }
  __syncthreads();
  const int lb = blockIdx.x - J.b0_in, bx = (W + 31) / 32;
  const int x = (lb % bx) * 32 + (threadIdx.x & 31);
  const int ybase = (lb / bx) * (8 * kRowsIn) + (threadIdx.x >> 5);
  // D = ln imax - ln imin = ln 2 x 2^Q / log2_scale (log2_scale = 2^Q / log2(imax / imin))
  const float l2s = J.st->log2_scale;
  const float D = J.st->imax > J.st->imin && l2s > 0.f ? 0.69314718f * ldexpf(1.f, J.qbits) / l2s : 0.f;
  const float rD = D > 0.f ? 1.f / D : 0.f;
  const float inv_scale = ldexpf(1.f, -J.qbits);
  const unsigned W1 = (unsigned)W + 1u;
  const size_t plane = (size_t)W1 * ((size_t)H + 1);
  float acc_lmin = 0.f, acc_lmax = 0.f;
  if (x < W) {
#pragma unroll 1
    for (int r = 0; r < kRowsIn; ++r) {
      const int y = ybase + 8 * r;
      if (y >= H) break;
      const unsigned pix = (unsigned)y * (unsigned)W + (unsigned)x;
      float rc, gc, bc;
      load_rgb<kDt>(J.in, x, y, rc, gc, bc);
      const float raw = __fadd_rn(__fadd_rn(__fmul_rn(0.2126f, rc), __fmul_rn(0.7152f, gc)), __fmul_rn(0.0722f, bc));
      float gi = J.gi_direct[pix];
      if (D > 0.f) {
        const float lh = (float)J.q[pix] * inv_scale + 0.5f;
        float gl = 0.f;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          const int x0 = max(x - P.rx[f], 0), x1 = min(x + P.rx[f], W - 1);
          const int y0 = max(y - P.ry[f], 0), y1 = min(y + P.ry[f], H - 1);
          const unsigned rt = (unsigned)y0 * W1, rb = (unsigned)(y1 + 1) * W1;
          const longlong2 *I = J.IUV + f * plane;
          const longlong2 a = __ldg(I + (rt + (unsigned)x0)), b = __ldg(I + (rt + (unsigned)x1 + 1u));
          const longlong2 c = __ldg(I + (rb + (unsigned)x1 + 1u)), d = __ldg(I + (rb + (unsigned)x0));
          const long long bu = (long long)((unsigned long long)c.x - (unsigned long long)d.x -
                                           (unsigned long long)b.x + (unsigned long long)a.x);
          const long long bv = (long long)((unsigned long long)c.y - (unsigned long long)d.y -
                                           (unsigned long long)b.y + (unsigned long long)a.y);
          const float fu = i64_to_float(bu) * scale[f][0] * scale[f][1];
          const float fv = i64_to_float(bv) * scale[NF + f][0] * scale[NF + f][1];
          gl += lh * fu - fv;
        }
        const float i = fmaxf(raw, kLumFloor);
        gi += __fdividef(gl * rD, i);
        acc_lmin += gl * (lh - 1.f) * rD;
        acc_lmax -= gl * lh * rD;
      }
      // degenerate range: only the direct colour-restoration term reaches i
      if (J.grad_in.p && raw > kLumFloor) {
        float *gin = static_cast<float *>(J.grad_in.p) + (long long)y * J.grad_in.pitch + 3LL * x;
        gin[0] += 0.2126f * gi;
        gin[1] += 0.7152f * gi;
        gin[2] += 0.0722f * gi;
      }
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
    atomicAdd(threadIdx.x == 0 ? &J.acc->lmin : &J.acc->lmax, (double)sum);
  }
}

}  // namespace

int bwd_pixel_blocks(int W, int H) { return ((W + 31) / 32) * ((H + 8 * kRowsPix - 1) / (8 * kRowsPix)); }

int bwd_input_blocks(int W, int H) { return ((W + 31) / 32) * ((H + 8 * kRowsIn - 1) / (8 * kRowsIn)); }

int launch_backward_setup(const void *desc, size_t bytes, void *dst, BwdAcc *accs, int n, double *gsum, bool first,
                          cudaStream_t s) {
  const int words = (int)(bytes / 4);
  if (bytes > kBwdDescBytes || bytes % 4) return -1;
  if (bytes <= 4096) {
    SmallPack<1024> p;
    std::memcpy(p.w, desc, bytes);
    k_bwd_setup<<<1, 256, 0, s>>>(p, words, static_cast<unsigned *>(dst), accs, n, gsum, first ? 1 : 0);
  } else {
    DescPack p;
    std::memcpy(p.w, desc, bytes);
    k_bwd_setup<<<1, 256, 0, s>>>(p, words, static_cast<unsigned *>(dst), accs, n, gsum, first ? 1 : 0);
  }
  return 1;
}

template <bool MOM, bool kPlain>
static void launch_pixel(const DevParams &P, const BwdJob *jobs, int n, int pix_blocks, double *gsum,
                         cudaStream_t s) {
  switch (P.n_fields) {
#define TM_BWD_PIXEL(nf) \
  case nf: k_bwd_pixel<nf, MOM, kPlain><<<pix_blocks, kBT, 0, s>>>(P, jobs, n, gsum); break;
    TM_BWD_PIXEL(1) TM_BWD_PIXEL(2) TM_BWD_PIXEL(3) TM_BWD_PIXEL(4) TM_BWD_PIXEL(5) TM_BWD_PIXEL(6)
    TM_BWD_PIXEL(7) TM_BWD_PIXEL(8)
#undef TM_BWD_PIXEL
  }
}

int launch_backward_pixel(const DevParams &P, const BwdJob *jobs, int n, int pix_blocks, bool mom, bool plain,
                          double *gsum, cudaStream_t s) {
  plain = plain && P.small_win && !(P.flags & kFlagAreaLit);
  if (mom) {
    if (plain) launch_pixel<true, true>(P, jobs, n, pix_blocks, gsum, s);
    else launch_pixel<true, false>(P, jobs, n, pix_blocks, gsum, s);
  } else {
    if (plain) launch_pixel<false, true>(P, jobs, n, pix_blocks, gsum, s);
    else launch_pixel<false, false>(P, jobs, n, pix_blocks, gsum, s);
  }
  return 1;
}

template <int kDt>
static void launch_input(const DevParams &P, const BwdJob *jobs, int n, int in_blocks, cudaStream_t s) {
  switch (P.n_fields) {
#define TM_BWD_INPUT(nf) case nf: k_bwd_input<nf, kDt><<<in_blocks, kBT, 0, s>>>(P, jobs, n); break;
    TM_BWD_INPUT(1) TM_BWD_INPUT(2) TM_BWD_INPUT(3) TM_BWD_INPUT(4) TM_BWD_INPUT(5) TM_BWD_INPUT(6)
    TM_BWD_INPUT(7) TM_BWD_INPUT(8)
#undef TM_BWD_INPUT
  }
}

int launch_backward_input(const DevParams &P, const BwdJob *jobs, int n, int in_blocks, bool plain,
                          const double *gsum, float *grad_params, cudaStream_t s) {
  if (plain) launch_input<kF32>(P, jobs, n, in_blocks, s);
  else launch_input<-1>(P, jobs, n, in_blocks, s);
  k_bwd_finish<<<n, 32, 0, s>>>(P, jobs, gsum, grad_params);
  return 2;
}

}  // namespace tmk
