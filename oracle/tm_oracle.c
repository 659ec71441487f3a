/*
 * tm_oracle.c -- plain, slow FP64 CPU oracle for the local tone-mapping
 * operator of "Mobile-end Tone Mapping based on Integral Image and Integral
 * Histogram" (arXiv 2102.01289).
 *
 * TEST INFRASTRUCTURE, not product code: only the tests, the smoke check and
 * the benchmark's CPU-baseline / reference arm load this library. It shares no
 * code with the CUDA path.
 *
 * Every step follows the paper's definitions in the paper's order:
 *   Eq. 11  luminance            i = 0.2126 R + 0.7152 G + 0.0722 B
 *   Sec. II log compression      l = log i (normalised, see reading R2)
 *   Sec. II-A, Eq. 7  bins       n equal-width bins of l over its global range
 *   Eq. 5   integral image       I(x,y) = sum_{x'<=x, y'<=y} i(x',y')
 *   Eq. 6 / Eq. 9 box sums       four-corner combinations
 *   Eq. 8   integral histogram   H_k = integral image of the indicator h_k
 *   Eq. 1   windowed CDF         P = (1/T) sum_{b_i < b} f(b_i)
 *   Eq. 2   tone curve           L_w = min L_d + (max L_d - min L_d) P
 *   Eq. 10  local variance       (plain definition, reading R5)
 *   Eq. 4   weight               W = sigma^2 / (sigma^2 + eps)
 *   Eq. 3   fusion               L = sum W L_w / sum W
 *   Eq. 12  colour restoration   c_out = (C_in / L_in)^sat L_out
 *
 * Readings where the paper is silent or garbled:
 *   R1 luminance is evaluated in float, left to right, every product and sum
 *      rounded, then floored at 1e-30f.
 *   R2 l is normalised: lhat = (ln i - ln imin) / (ln imax - ln imin); lhat = 0
 *      when imax == imin.
 *   R3 bins are equal-width in l over the global range; the edge between bin
 *      k-1 and k is the smallest float >= exp(ln imin + (ln imax - ln imin) k/n)
 *      and a luminance on an edge belongs to the upper bin. Degenerate range:
 *      every pixel is in bin 0.
 *   R4 windows are centred and clipped to the image; T is the clipped area.
 *   R5 sigma^2 is the window variance of lhat, (1/T) sum (lhat - mean)^2
 *      (the printed Eq. 10 and Alg. 1 do not vanish on a constant window).
 *   R6 when sum W == 0 the fields are averaged with equal weights.
 *   R7 C_in / L_in is clamped at 0 before the power of Eq. 12.
 */
#include "tm_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Host threads for the per-pixel loops (pixels are independent: each is
 * computed exactly as in a single-threaded run). */
static int g_threads = 1;

void tmo_set_threads(int32_t n) { g_threads = n < 1 ? 1 : n; }

int32_t tmo_num_procs(void) {
#ifdef _OPENMP
  return omp_get_num_procs();
#else
  return 1;
#endif
}

static int thread_id(void) {
#ifdef _OPENMP
  return omp_get_thread_num();
#else
  return 0;
#endif
}

#define TMO_LUM_FLOOR 1e-30f

static const float K_R = 0.2126f, K_G = 0.7152f, K_B = 0.0722f; /* Eq. 11 */

float tmo_luminance(float r, float g, float b) {
  /* Built with -ffp-contract=off: each operation rounds to float (R1). */
  float pr = K_R * r;
  float pg = K_G * g;
  float pb = K_B * b;
  float i = (pr + pg) + pb;
  return i > TMO_LUM_FLOOR ? i : TMO_LUM_FLOOR;
}

void tmo_thresholds(float imin, float imax, int32_t n_bins, float *thr) {
  /* R3: equal-width bins of ln i between ln imin and ln imax (Sec. II-A). */
  if (!(imax > imin)) {
    for (int k = 1; k < n_bins; ++k) thr[k - 1] = INFINITY;
    return;
  }
  double lmin = log((double)imin), lmax = log((double)imax);
  for (int k = 1; k < n_bins; ++k) {
    double t = exp(lmin + (lmax - lmin) * ((double)k / (double)n_bins));
    float f = (float)t;
    if ((double)f < t) f = nextafterf(f, INFINITY); /* smallest float >= t */
    thr[k - 1] = f;
  }
}

static uint8_t bin_of(float i, const float *thr, int n_bins) {
  /* b = number of edges at or below i (an edge value goes to the upper bin). */
  int b = 0;
  for (int k = 1; k < n_bins; ++k)
    if (i >= thr[k - 1]) ++b;
  return (uint8_t)b;
}

int tmo_prepare(const float *rgb, int32_t W, int32_t H, int32_t n_bins,
                float *lum, float *imin, float *imax, float *thr,
                uint8_t *bins, double *lhat) {
  if (W <= 0 || H <= 0 || n_bins < 1 || n_bins > TMO_MAX_BINS) return -1;
  int64_t N = (int64_t)W * H;
  float lo = INFINITY, hi = -INFINITY;
  for (int64_t p = 0; p < N; ++p) {
    float i = tmo_luminance(rgb[3 * p], rgb[3 * p + 1], rgb[3 * p + 2]);
    lum[p] = i;
    if (i < lo) lo = i;
    if (i > hi) hi = i;
  }
  *imin = lo;
  *imax = hi;
  tmo_thresholds(lo, hi, n_bins, thr);
  double lmin = log((double)lo), D = log((double)hi) - lmin;
  for (int64_t p = 0; p < N; ++p) {
    bins[p] = bin_of(lum[p], thr, n_bins);
    lhat[p] = (hi > lo) ? (log((double)lum[p]) - lmin) / D : 0.0;
  }
  return 0;
}

void tmo_integral_i64(const int64_t *v, int32_t W, int32_t H, uint64_t *S) {
  /* Eq. 5 by the recurrence I(x,y) = i + I(x-1,y) + I(x,y-1) - I(x-1,y-1). */
  int64_t W1 = (int64_t)W + 1;
  memset(S, 0, sizeof(uint64_t) * (size_t)(W1 * ((int64_t)H + 1)));
  for (int64_t y = 0; y < H; ++y)
    for (int64_t x = 0; x < W; ++x)
      S[(y + 1) * W1 + x + 1] = (uint64_t)v[y * W + x] + S[(y + 1) * W1 + x] +
                                S[y * W1 + x + 1] - S[y * W1 + x];
}

void tmo_integral_f64(const double *v, int32_t W, int32_t H, double *S) {
  int64_t W1 = (int64_t)W + 1;
  memset(S, 0, sizeof(double) * (size_t)(W1 * ((int64_t)H + 1)));
  for (int64_t y = 0; y < H; ++y)
    for (int64_t x = 0; x < W; ++x)
      S[(y + 1) * W1 + x + 1] = v[y * W + x] + S[(y + 1) * W1 + x] +
                                S[y * W1 + x + 1] - S[y * W1 + x];
}

void tmo_integral_histogram(const uint8_t *bins, int32_t W, int32_t H,
                            int32_t n_bins, uint32_t *Hk) {
  /* Eq. 7 indicator planes h_k, Eq. 8 one integral image per plane. */
  int64_t W1 = (int64_t)W + 1, P = W1 * ((int64_t)H + 1);
  memset(Hk, 0, sizeof(uint32_t) * (size_t)(P * n_bins));
  for (int k = 0; k < n_bins; ++k) {
    uint32_t *S = Hk + (int64_t)k * P;
    for (int64_t y = 0; y < H; ++y)
      for (int64_t x = 0; x < W; ++x) {
        uint32_t h = (bins[y * W + x] == k) ? 1u : 0u;
        S[(y + 1) * W1 + x + 1] =
            h + S[(y + 1) * W1 + x] + S[y * W1 + x + 1] - S[y * W1 + x];
      }
  }
}

/* Window of field f around (x, y), clipped to the image (R4). */
typedef struct { int x0, x1, y0, y1; } win_t;

static win_t window_of(const tmo_params *p, int f, int x, int y, int W, int H) {
  win_t w;
  w.x0 = x - p->rx[f] < 0 ? 0 : x - p->rx[f];
  w.x1 = x + p->rx[f] > W - 1 ? W - 1 : x + p->rx[f];
  w.y0 = y - p->ry[f] < 0 ? 0 : y - p->ry[f];
  w.y1 = y + p->ry[f] > H - 1 ? H - 1 : y + p->ry[f];
  return w;
}

/* Eq. 9: count of bin k inside the window from the four corners of H_k. */
static uint32_t box_u32(const uint32_t *S, int W, win_t w) {
  int64_t W1 = (int64_t)W + 1;
  return S[((int64_t)w.y1 + 1) * W1 + w.x1 + 1] - S[((int64_t)w.y1 + 1) * W1 + w.x0] -
         S[(int64_t)w.y0 * W1 + w.x1 + 1] + S[(int64_t)w.y0 * W1 + w.x0];
}

/* Eq. 1 numerators alone, at every pixel and field: #{q in w_i(p) : b(q) < b(p)}
 * (b(q) <= b(p) under TMO_CDF_INCLUSIVE). Summing the window histogram of
 * Eq. 9 over the bins below b(p) is, by the linearity of the four-corner sum,
 * the box sum of the integral image of the indicator [b(q) < k], k = b(p)
 * (Eq. 7 summed over those bins, then Eq. 8). So one such integral image is
 * built per threshold k that some pixel needs, and read at those pixels.
 * cnt: s*H*W (field-major). Returns 0, -1 for bad parameters, -2 when out of
 * memory. */
int tmo_window_counts(const uint8_t *bins, int32_t W, int32_t H, const tmo_params *p,
                      uint32_t *cnt) {
  if (W < 1 || H < 1 || p->n_fields < 1 || p->n_fields > TMO_MAX_FIELDS || p->n_bins < 1 ||
      p->n_bins > TMO_MAX_BINS)
    return -1;
  const int s = p->n_fields, n = p->n_bins;
  const int incl = (p->flags & TMO_CDF_INCLUSIVE) ? 1 : 0;
  const int64_t W1 = (int64_t)W + 1, P = W1 * ((int64_t)H + 1), N = (int64_t)W * H;
  uint32_t *S = malloc(sizeof(uint32_t) * (size_t)P);
  if (!S) return -2;
  unsigned char used[TMO_MAX_BINS + 1];
  memset(used, 0, sizeof used);
  for (int64_t q = 0; q < N; ++q) used[bins[q] + incl] = 1;
  for (int k = 0; k <= n; ++k) {
    if (!used[k]) continue;
    memset(S, 0, sizeof(uint32_t) * (size_t)W1);
    for (int64_t y = 0; y < H; ++y) {
      S[(y + 1) * W1] = 0;
      for (int64_t x = 0; x < W; ++x) {
        uint32_t h = bins[y * W + x] < k ? 1u : 0u;
        S[(y + 1) * W1 + x + 1] = h + S[(y + 1) * W1 + x] + S[y * W1 + x + 1] - S[y * W1 + x];
      }
    }
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x) {
        int64_t q = (int64_t)y * W + x;
        if (bins[q] + incl != k) continue;
        for (int f = 0; f < s; ++f) cnt[f * N + q] = box_u32(S, W, window_of(p, f, x, y, W, H));
      }
  }
  free(S);
  return 0;
}

/* R5: variance over the window, as the mean of squared deviations. Summed
 * about the centre value c (the variance does not depend on the shift), which
 * keeps a constant window at exactly zero. T is the area the moments divide
 * by; when it exceeds the clipped window (TMO_AREA_LITERAL) the missing
 * pixels take part with the value `pad`. */
static void window_moments(const double *v, int W, win_t w, double c, double T, double pad,
                           double *mu, double *var) {
  double s1 = 0.0, s2 = 0.0;
  double Tc = (double)(w.x1 - w.x0 + 1) * (double)(w.y1 - w.y0 + 1);
  for (int y = w.y0; y <= w.y1; ++y)
    for (int x = w.x0; x <= w.x1; ++x) {
      double d = v[(int64_t)y * W + x] - c;
      s1 += d;
      s2 += d * d;
    }
  s1 += (T - Tc) * (pad - c);
  s2 += (T - Tc) * (pad - c) * (pad - c);
  double m = s1 / T;
  double r = s2 / T - m * m;
  *mu = c + m;
  *var = r > 0.0 ? r : 0.0;
}

/* Area of field f's window at a pixel: clipped (default) or the literal
 * (2 rx + 1)(2 ry + 1) of Algorithm 1. */
static uint32_t window_area(const tmo_params *p, int f, win_t w) {
  if (p->flags & TMO_AREA_LITERAL) return (uint32_t)(2 * p->rx[f] + 1) * (uint32_t)(2 * p->ry[f] + 1);
  return (uint32_t)((w.x1 - w.x0 + 1) * (w.y1 - w.y0 + 1));
}

/* Eq. 2, Eq. 4 and Eq. 3 for one pixel, from its per-field counts/moments. */
static double fuse(const tmo_params *p, const uint32_t *cnt, const uint32_t *area,
                   const double *var, double *weight, double *lf) {
  int s = p->n_fields;
  double wsum = 0.0, acc = 0.0, mean = 0.0;
  for (int f = 0; f < s; ++f) {
    double P = (double)cnt[f] / (double)area[f];                /* Eq. 1 */
    lf[f] = p->ld_min + (p->ld_max - p->ld_min) * P;            /* Eq. 2 */
    weight[f] = p->alpha[f] * var[f] / (var[f] + p->eps[f]);    /* Eq. 4 */
    wsum += weight[f];
    acc += weight[f] * lf[f];
    mean += lf[f];
  }
  return wsum > 0.0 ? acc / wsum : mean / (double)s;            /* Eq. 3, R6 */
}

/* Eq. 12 with R7 for one channel. */
static double restore(double C, double i, double sat, double L) {
  double rho = C / i;
  if (!(rho > 0.0)) rho = 0.0;
  return pow(rho, sat) * L;
}

static int params_ok(const tmo_params *p) {
  if (p->n_bins < 1 || p->n_bins > TMO_MAX_BINS) return 0;
  if (p->n_fields < 1 || p->n_fields > TMO_MAX_FIELDS) return 0;
  for (int f = 0; f < p->n_fields; ++f)
    if (p->rx[f] < 0 || p->ry[f] < 0 || p->rx[f] > 32767 || p->ry[f] > 32767 || !(p->eps[f] > 0.0))
      return 0;
  if (p->flags & ~(TMO_CDF_INCLUSIVE | TMO_AREA_LITERAL | TMO_VAR_LINEAR)) return 0;
  return 1;
}

/* ------------------------------------------------------------------------ */
/* Shared forward core: luminance in float (R1) or double, bins computed or  */
/* supplied, counts through the integral histogram (Eq. 8, Eq. 9), variance  */
/* by direct window sums.                                                    */

typedef struct {
  int W, H, s;
  int64_t N;
  double *lum;
  uint8_t *clamped;
  double imin, imax, lmin, D;
  int64_t argmin, argmax;
  uint8_t *bins;
  double *lhat;
  uint32_t *cnt, *area;
  double *mu, *var, *weight, *lf, *L, *wsum;
} core_t;

static void core_free(core_t *c) {
  free(c->lum); free(c->clamped); free(c->bins); free(c->lhat);
  free(c->cnt); free(c->area); free(c->mu); free(c->var);
  free(c->weight); free(c->lf); free(c->L); free(c->wsum);
  memset(c, 0, sizeof(*c));
}

/* range: NULL, or {imin, imax} to bin and normalise with instead of the
 * image's own range (streaming reuse of an earlier frame's range); the
 * normalised log is then clamped to [0, 1]. */
static int core_run(const double *rgb, int W, int H, const tmo_params *p,
                    int lum_f64, const uint8_t *fixed_bins, const float *range, core_t *c) {
  memset(c, 0, sizeof(*c));
  if (W <= 0 || H <= 0 || !params_ok(p)) return -1;
  int s = p->n_fields, n = p->n_bins;
  int64_t N = (int64_t)W * H;
  c->W = W; c->H = H; c->s = s; c->N = N;
  c->lum = malloc(sizeof(double) * N);
  c->clamped = malloc(N);
  c->bins = malloc(N);
  c->lhat = malloc(sizeof(double) * N);
  c->cnt = malloc(sizeof(uint32_t) * N * s);
  c->area = malloc(sizeof(uint32_t) * N * s);
  c->mu = malloc(sizeof(double) * N * s);
  c->var = malloc(sizeof(double) * N * s);
  c->weight = malloc(sizeof(double) * N * s);
  c->lf = malloc(sizeof(double) * N * s);
  c->L = malloc(sizeof(double) * N);
  c->wsum = malloc(sizeof(double) * N);
  if (!c->lum || !c->clamped || !c->bins || !c->lhat || !c->cnt || !c->area ||
      !c->mu || !c->var || !c->weight || !c->lf || !c->L || !c->wsum) {
    core_free(c);
    return -2;
  }
  /* Eq. 11 */
  double floor_v = (double)TMO_LUM_FLOOR;
  c->argmin = c->argmax = 0;
  for (int64_t q = 0; q < N; ++q) {
    double i, raw;
    if (lum_f64) {
      raw = 0.2126 * rgb[3 * q] + 0.7152 * rgb[3 * q + 1] + 0.0722 * rgb[3 * q + 2];
      i = raw > floor_v ? raw : floor_v;
    } else {
      float r = (float)rgb[3 * q], g = (float)rgb[3 * q + 1], b = (float)rgb[3 * q + 2];
      float pr = K_R * r, pg = K_G * g, pb = K_B * b;
      float fr = (pr + pg) + pb;
      raw = fr;
      i = tmo_luminance(r, g, b);
    }
    c->lum[q] = i;
    c->clamped[q] = raw > floor_v ? 0 : 1;
    if (i < c->lum[c->argmin]) c->argmin = q;
    if (i > c->lum[c->argmax]) c->argmax = q;
  }
  c->imin = c->lum[c->argmin];
  c->imax = c->lum[c->argmax];
  if (range) {
    c->imin = (double)range[0];
    c->imax = (double)range[1];
  }
  /* Sec. II-A bins (R3) */
  if (fixed_bins) {
    memcpy(c->bins, fixed_bins, N);
  } else {
    if (lum_f64) { core_free(c); return -1; }
    float thr[TMO_MAX_BINS];
    tmo_thresholds((float)c->imin, (float)c->imax, n, thr);
    for (int64_t q = 0; q < N; ++q) c->bins[q] = bin_of((float)c->lum[q], thr, n);
  }
  /* Sec. II log compression, normalised (R2) */
  c->lmin = log(c->imin);
  c->D = (c->imax > c->imin) ? log(c->imax) - c->lmin : 0.0;
  for (int64_t q = 0; q < N; ++q) {
    double l = c->D > 0.0 ? (log(c->lum[q]) - c->lmin) / c->D : 0.0;
    c->lhat[q] = l < 0.0 ? 0.0 : l > 1.0 ? 1.0 : l;  /* a no-op with the image's own range */
  }
  /* the values whose window variance Eq. 10 takes */
  const double *vdom = c->lhat;
  double *lin = NULL;
  if (p->flags & TMO_VAR_LINEAR) {
    lin = malloc(sizeof(double) * N);
    if (!lin) { core_free(c); return -2; }
    for (int64_t q = 0; q < N; ++q) lin[q] = c->lum[q] / c->imax;
    vdom = lin;
  }
  const int incl = (p->flags & TMO_CDF_INCLUSIVE) ? 1 : 0;
  /* Eq. 7-8 integral histogram */
  int64_t P = ((int64_t)W + 1) * ((int64_t)H + 1);
  uint32_t *Hk = malloc(sizeof(uint32_t) * P * n);
  if (!Hk) { free(lin); core_free(c); return -2; }
  tmo_integral_histogram(c->bins, W, H, n, Hk);
#pragma omp parallel for schedule(dynamic, 1) num_threads(g_threads)
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      int64_t q = (int64_t)y * W + x;
      uint32_t cnt[TMO_MAX_FIELDS], area[TMO_MAX_FIELDS];
      double var[TMO_MAX_FIELDS], wgt[TMO_MAX_FIELDS], lf[TMO_MAX_FIELDS];
      for (int f = 0; f < s; ++f) {
        win_t w = window_of(p, f, x, y, W, H);
        uint32_t k_count = 0;
        for (int k = 0; k < c->bins[q] + incl; ++k)    /* Eq. 1: b_i < b (or <=) */
          k_count += box_u32(Hk + (int64_t)k * P, W, w); /* Eq. 9 */
        cnt[f] = k_count;
        area[f] = window_area(p, f, w);
        double mu;
        window_moments(vdom, W, w, vdom[q], (double)area[f], 0.0, &mu, &var[f]);
        c->mu[f * N + q] = mu;
      }
      double L = fuse(p, cnt, area, var, wgt, lf);
      double ws = 0.0;
      for (int f = 0; f < s; ++f) {
        c->cnt[f * N + q] = cnt[f];
        c->area[f * N + q] = area[f];
        c->var[f * N + q] = var[f];
        c->weight[f * N + q] = wgt[f];
        c->lf[f * N + q] = lf[f];
        ws += wgt[f];
      }
      c->L[q] = L;
      c->wsum[q] = ws;
    }
  free(Hk);
  free(lin);
  return 0;
}

int tmo_forward_range(const float *rgb, int32_t W, int32_t H, const tmo_params *p,
                      const float *range, double *out, tmo_fields *fields) {
  if (W <= 0 || H <= 0) return -1;
  int64_t N = (int64_t)W * H;
  double *rgbd = malloc(sizeof(double) * 3 * N);
  if (!rgbd) return -2;
  for (int64_t q = 0; q < 3 * N; ++q) rgbd[q] = (double)rgb[q];
  core_t c;
  int rc = core_run(rgbd, W, H, p, 0, NULL, range, &c);
  free(rgbd);
  if (rc) return rc;
  for (int64_t q = 0; q < N; ++q)
    for (int ch = 0; ch < 3; ++ch)
      out[3 * q + ch] = restore((double)rgb[3 * q + ch], c.lum[q], p->sat, c.L[q]);
  if (fields) {
    int64_t sN = (int64_t)c.s * N;
    if (fields->cnt) memcpy(fields->cnt, c.cnt, sizeof(uint32_t) * sN);
    if (fields->area) memcpy(fields->area, c.area, sizeof(uint32_t) * sN);
    if (fields->mu) memcpy(fields->mu, c.mu, sizeof(double) * sN);
    if (fields->sigma2) memcpy(fields->sigma2, c.var, sizeof(double) * sN);
    if (fields->weight) memcpy(fields->weight, c.weight, sizeof(double) * sN);
    if (fields->lf) memcpy(fields->lf, c.lf, sizeof(double) * sN);
    if (fields->l) memcpy(fields->l, c.L, sizeof(double) * N);
  }
  core_free(&c);
  return 0;
}

int tmo_forward(const float *rgb, int32_t W, int32_t H, const tmo_params *p,
                double *out, tmo_fields *fields) {
  return tmo_forward_range(rgb, W, H, p, NULL, out, fields);
}

int tmo_forward_fixed_bins(const double *rgb, int32_t W, int32_t H,
                           const tmo_params *p, const uint8_t *bins,
                           double *out) {
  core_t c;
  int rc = core_run(rgb, W, H, p, 1, bins, NULL, &c);
  if (rc) return rc;
  for (int64_t q = 0; q < c.N; ++q)
    for (int ch = 0; ch < 3; ++ch)
      out[3 * q + ch] = restore(rgb[3 * q + ch], c.lum[q], p->sat, c.L[q]);
  core_free(&c);
  return 0;
}

int tmo_forward_pixels(const float *rgb, int32_t W, int32_t H,
                       const tmo_params *p, const int32_t *xs,
                       const int32_t *ys, int64_t K, double *out,
                       uint32_t *cnt_o, uint32_t *area_o, double *sigma2_o,
                       double *weight_o, double *lf_o) {
  if (W <= 0 || H <= 0 || !params_ok(p)) return -1;
  int64_t N = (int64_t)W * H;
  int s = p->n_fields;
  float *lum = malloc(sizeof(float) * N);
  uint8_t *bins = malloc(N);
  double *lhat = malloc(sizeof(double) * N);
  if (!lum || !bins || !lhat) { free(lum); free(bins); free(lhat); return -2; }
  float imin, imax, thr[TMO_MAX_BINS];
  tmo_prepare(rgb, W, H, p->n_bins, lum, &imin, &imax, thr, bins, lhat);
  if (p->flags & TMO_VAR_LINEAR)  /* the window variance of Eq. 10 on i / imax */
    for (int64_t q = 0; q < N; ++q) lhat[q] = (double)lum[q] / (double)imax;
  const int incl = (p->flags & TMO_CDF_INCLUSIVE) ? 1 : 0;
  for (int64_t k = 0; k < K; ++k)
    if (xs[k] < 0 || xs[k] >= W || ys[k] < 0 || ys[k] >= H) { free(lum); free(bins); free(lhat); return -1; }
#pragma omp parallel for schedule(dynamic, 64) num_threads(g_threads)
  for (int64_t k = 0; k < K; ++k) {
    int x = xs[k], y = ys[k];
    int64_t q = (int64_t)y * W + x;
    uint32_t cnt[TMO_MAX_FIELDS], area[TMO_MAX_FIELDS];
    double var[TMO_MAX_FIELDS], wgt[TMO_MAX_FIELDS], lf[TMO_MAX_FIELDS];
    for (int f = 0; f < s; ++f) {
      win_t w = window_of(p, f, x, y, W, H);
      uint32_t below = 0;                                 /* Eq. 1 by counting */
      for (int yy = w.y0; yy <= w.y1; ++yy)
        for (int xx = w.x0; xx <= w.x1; ++xx)
          if (bins[(int64_t)yy * W + xx] < bins[q] + incl) ++below;
      cnt[f] = below;
      area[f] = window_area(p, f, w);
      double mu;
      window_moments(lhat, W, w, lhat[q], (double)area[f], 0.0, &mu, &var[f]);
    }
    double L = fuse(p, cnt, area, var, wgt, lf);
    for (int ch = 0; ch < 3; ++ch)
      out[3 * k + ch] = restore((double)rgb[3 * q + ch], (double)lum[q], p->sat, L);
    for (int f = 0; f < s; ++f) {
      if (cnt_o) cnt_o[k * s + f] = cnt[f];
      if (area_o) area_o[k * s + f] = area[f];
      if (sigma2_o) sigma2_o[k * s + f] = var[f];
      if (weight_o) weight_o[k * s + f] = wgt[f];
      if (lf_o) lf_o[k * s + f] = lf[f];
    }
  }
  free(lum); free(bins); free(lhat);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Adjoint. With the bin map fixed, the output is a smooth function of the   */
/* input and of (ld_min, ld_max, sat, eps_i, alpha_i); the gradient is the   */
/* chain rule through Eq. 12, Eq. 3, Eq. 4, Eq. 2, the window variance, the  */
/* normalised log (including its dependence on the image range) and Eq. 11. */

int tmo_backward(const double *rgb, int32_t W, int32_t H, const tmo_params *p,
                 int32_t lum_f64, const uint8_t *bins, const double *grad_out,
                 double *grad_in, double *grad_params) {
  if (p->flags & TMO_VAR_LINEAR) return -3;  /* the adjoint covers the log-domain variance */
  core_t c;
  int rc = core_run(rgb, W, H, p, lum_f64, bins, NULL, &c);
  if (rc) return rc;
  int s = c.s;
  int64_t N = c.N;
  double *glhat = calloc(N, sizeof(double));
  double *gi = calloc(N, sizeof(double));
  if (!glhat || !gi) { free(glhat); free(gi); core_free(&c); return -2; }
  memset(grad_in, 0, sizeof(double) * 3 * N);
  memset(grad_params, 0, sizeof(double) * (3 + 2 * s));
  /* each host thread sums the window-variance adjoint and the parameter
   * gradients into its own copies, added up after the loop */
  const int nt = g_threads, npar = 3 + 2 * s;
  double *gl_all = calloc((size_t)N * nt, sizeof(double));
  double *gp_all = calloc((size_t)npar * nt, sizeof(double));
  if (!gl_all || !gp_all) { free(gl_all); free(gp_all); free(glhat); free(gi); core_free(&c); return -2; }
#pragma omp parallel num_threads(nt)
  {
  double *glt = gl_all + (int64_t)thread_id() * N;
  double *gpar = gp_all + (int64_t)thread_id() * npar;
  double *g_eps = gpar + 3, *g_alpha = gpar + 3 + s;
#pragma omp for schedule(dynamic, 1)
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      int64_t q = (int64_t)y * W + x;
      double i = c.lum[q], L = c.L[q];
      /* Eq. 12 */
      double gL = 0.0;
      for (int ch = 0; ch < 3; ++ch) {
        double C = rgb[3 * q + ch], g = grad_out[3 * q + ch];
        double rho = C / i;
        if (!(rho > 0.0)) {
          gL += g * pow(0.0, p->sat);
          continue;
        }
        double rs = pow(rho, p->sat);
        gL += g * rs;
        gpar[2] += g * rs * log(rho) * L;
        grad_in[3 * q + ch] += g * p->sat * pow(rho, p->sat - 1.0) * L / i;
        gi[q] += -g * p->sat * rs * L / i;
      }
      /* Eq. 3 */
      double ws = c.wsum[q];
      for (int f = 0; f < s; ++f) {
        int64_t fq = (int64_t)f * N + q;
        double dLdLf = ws > 0.0 ? c.weight[fq] / ws : 1.0 / (double)s;
        double dLdW = ws > 0.0 ? (c.lf[fq] - L) / ws : 0.0;
        double P = (double)c.cnt[fq] / (double)c.area[fq];
        gpar[0] += gL * dLdLf * (1.0 - P);               /* Eq. 2 */
        gpar[1] += gL * dLdLf * P;
        double gW = gL * dLdW;
        double v = c.var[fq], e = p->eps[f], a = p->alpha[f];
        double den = (v + e) * (v + e);
        g_eps[f] += gW * (-a * v / den);                          /* Eq. 4 */
        g_alpha[f] += gW * (v / (v + e));
        double gv = gW * a * e / den;
        if (gv == 0.0) continue;
        /* window variance: d var / d lhat_r = (2/T)(lhat_r - mean) */
        win_t w = window_of(p, f, x, y, W, H);
        double T = (double)c.area[fq], mu = c.mu[fq];
        for (int yy = w.y0; yy <= w.y1; ++yy)
          for (int xx = w.x0; xx <= w.x1; ++xx) {
            int64_t r = (int64_t)yy * W + xx;
            glt[r] += gv * (2.0 / T) * (c.lhat[r] - mu);
          }
      }
    }
  }
  for (int t = 0; t < nt; ++t) {
    for (int64_t q = 0; q < N; ++q) glhat[q] += gl_all[(int64_t)t * N + q];
    for (int k = 0; k < npar; ++k) grad_params[k] += gp_all[(int64_t)t * npar + k];
  }
  free(gl_all);
  free(gp_all);
  /* normalised log, including the range terms through ln imin and ln imax */
  if (c.D > 0.0) {
    double glmin = 0.0, glmax = 0.0;
    for (int64_t q = 0; q < N; ++q) {
      gi[q] += glhat[q] / (c.lum[q] * c.D);
      glmin += glhat[q] * (c.lhat[q] - 1.0) / c.D;
      glmax += glhat[q] * (-c.lhat[q] / c.D);
    }
    gi[c.argmin] += glmin / c.imin;
    gi[c.argmax] += glmax / c.imax;
  }
  /* Eq. 11 (no gradient where the floor is active) */
  for (int64_t q = 0; q < N; ++q) {
    if (c.clamped[q]) continue;
    grad_in[3 * q] += 0.2126 * gi[q];
    grad_in[3 * q + 1] += 0.7152 * gi[q];
    grad_in[3 * q + 2] += 0.0722 * gi[q];
  }
  free(glhat);
  free(gi);
  core_free(&c);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Capture front-end (Section III): the WDR image is recovered from several  */
/* exposures by Debevec and Malik's radiance-map merge. With g_c the log     */
/* inverse response of channel c (g_c(z) = ln of the sensor exposure X that  */
/* maps to pixel value z) and dt_j the exposure times, each channel of each  */
/* pixel takes the hat-weighted mean of the per-exposure log radiances:      */
/*   ln E = sum_j w(z_j) (g(z_j) - ln dt_j) / sum_j w(z_j),                  */
/*   w(z) = z for z <= 127, 255 - z above.                                   */
/* Reading (the merge is 0/0 when every exposure is at 0 or 255): the        */
/* shortest exposure's estimate when it is saturated, else the longest's.   */

static double merge_weight(int z) { return z <= 127 ? (double)z : (double)(255 - z); }

int tmo_merge_exposures(int32_t n, const uint8_t *const *ldr, const double *times,
                        int32_t W, int32_t H, const double *log_response, double *out) {
  if (n < 1 || W < 1 || H < 1) return -1;
  int shortest = 0, longest = 0;
  for (int j = 0; j < n; ++j) {
    if (!(times[j] > 0.0)) return -1;
    if (times[j] < times[shortest]) shortest = j;
    if (times[j] > times[longest]) longest = j;
  }
  int64_t N = (int64_t)W * H;
  for (int64_t p = 0; p < N; ++p)
    for (int c = 0; c < 3; ++c) {
      const double *g = log_response + 256 * c;
      double num = 0.0, den = 0.0;
      for (int j = 0; j < n; ++j) {
        int z = ldr[j][3 * p + c];
        double w = merge_weight(z);
        num += w * (g[z] - log(times[j]));
        den += w;
      }
      double lnE;
      if (den > 0.0) {
        lnE = num / den;
      } else {
        int j = ldr[shortest][3 * p + c] == 255 ? shortest : longest;
        lnE = g[ldr[j][3 * p + c]] - log(times[j]);
      }
      out[3 * p + c] = exp(lnE);
    }
  return 0;
}
