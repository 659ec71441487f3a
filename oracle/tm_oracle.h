/*
 * tm_oracle.h -- interface of the FP64 CPU oracle for the local tone-mapping
 * operator of "Mobile-end Tone Mapping based on Integral Image and Integral
 * Histogram" (arXiv 2102.01289).
 *
 * TEST INFRASTRUCTURE. This oracle is the plain, slow, obviously correct
 * statement of what the operator computes. Only the tests, the smoke check and
 * the benchmark's CPU-baseline / reference arm may load it; the product path
 * never does. It shares no code, header, table or constant generator with the
 * CUDA library.
 *
 * Conventions (all arrays row-major, caller-allocated):
 *   rgb      : H*W*3 interleaved (HWC) samples
 *   planes   : H*W scalars, index y*W + x
 *   integral : (H+1)*(W+1) with a zero first row and column; entry
 *              (y+1)*(W+1) + (x+1) holds the sum over x' <= x, y' <= y (Eq. 5)
 */
#ifndef TM_ORACLE_H
#define TM_ORACLE_H

#include <stdint.h>

#define TMO_MAX_FIELDS 8
#define TMO_MAX_BINS 256

/* Operator parameters, in the paper's notation (Section II-C, Section III). */
typedef struct {
  int32_t n_bins;              /* n: histogram bins (Eq. 7)            */
  int32_t n_fields;            /* s: receptive fields (Eq. 3)          */
  int32_t rx[TMO_MAX_FIELDS];  /* half-width of field i (Alg. 1 s_j.x) */
  int32_t ry[TMO_MAX_FIELDS];  /* half-height of field i (Alg. 1 s_j.y)*/
  double eps[TMO_MAX_FIELDS];  /* epsilon of Eq. 4 per field           */
  double alpha[TMO_MAX_FIELDS];/* field weight multiplying Eq. 4 (1 = paper) */
  double ld_min, ld_max;       /* min(L_d), max(L_d) of Eq. 2          */
  double sat;                  /* sat of Eq. 12                        */
  int32_t flags;               /* reading variants, TMO_* below (0 = defaults) */
} tmo_params;

/* Reading variants (0 selects the default readings):
 *   TMO_CDF_INCLUSIVE  Eq. 1 counts b(q) <= b(p) instead of b(q) < b(p).
 *   TMO_AREA_LITERAL   the window area is the unclipped (2 rx + 1)(2 ry + 1)
 *                      of Algorithm 1; pixels outside the image take part as
 *                      zeros (they are never counted by Eq. 1 and contribute
 *                      a normalised log of 0 to the window moments).
 *   TMO_VAR_LINEAR     Eq. 10 on the linear luminance normalised by the image
 *                      maximum, i / imax, instead of the normalised log. */
#define TMO_CDF_INCLUSIVE 1
#define TMO_AREA_LITERAL 2
#define TMO_VAR_LINEAR 4

/* Per-pixel, per-field intermediates (optional debug / backward state). */
typedef struct {
  uint32_t *cnt;    /* s*H*W: #{q in w_i : b(q) < b(p)} (Eq. 1 numerator)  */
  uint32_t *area;   /* s*H*W: T = |w_i| (clipped window area)               */
  double *mu;       /* s*H*W: window mean of the normalised log luminance   */
  double *sigma2;   /* s*H*W: window variance (Eq. 10, plain definition)    */
  double *weight;   /* s*H*W: W of Eq. 4                                     */
  double *lf;       /* s*H*W: L_{w_i} of Eq. 2                               */
  double *l;        /* H*W  : fused L of Eq. 3                               */
} tmo_fields;

/* Host threads of the per-pixel loops (default 1; the results do not depend
 * on it, up to the summation order of the adjoint's FP64 sums), and the number
 * of host cores. */
void tmo_set_threads(int32_t n);
int32_t tmo_num_procs(void);

/* Eq. 11 luminance in float, fixed order, each step rounded; floored. */
float tmo_luminance(float r, float g, float b);

/* Global pre-pass: luminance plane, its range, the n-1 bin thresholds, the bin
 * map and the normalised log luminance. Returns 0 on success. */
int tmo_prepare(const float *rgb, int32_t W, int32_t H, int32_t n_bins,
                float *lum, float *imin, float *imax, float *thr,
                uint8_t *bins, double *lhat);

/* Thresholds alone (n-1 floats) from a luminance range. */
void tmo_thresholds(float imin, float imax, int32_t n_bins, float *thr);

/* Eq. 5 integral image of an int64 plane, modulo 2^64. */
void tmo_integral_i64(const int64_t *v, int32_t W, int32_t H, uint64_t *S);

/* Eq. 5 integral image of a double plane. */
void tmo_integral_f64(const double *v, int32_t W, int32_t H, double *S);

/* Eq. 7-8 integral histogram: n planes of (H+1)*(W+1) uint32 counts. */
void tmo_integral_histogram(const uint8_t *bins, int32_t W, int32_t H,
                            int32_t n_bins, uint32_t *Hk);

/* Eq. 1 numerators only, every pixel and field (s*H*W, field-major), from
 * the integral image of [b(q) < k] per needed threshold k and Eq. 9 box sums;
 * no variance. Returns 0 on success. */
int tmo_window_counts(const uint8_t *bins, int32_t W, int32_t H, const tmo_params *p,
                      uint32_t *cnt);

/* Full forward over the image (counts through Eq. 9, variance by direct
 * window sums). out: H*W*3 doubles. fields: optional (NULL fields ignored). */
/* tmo_forward with bins and the normalised log taken over a given range
 * {imin, imax} (an earlier frame's) instead of the image's own; the
 * normalised log is clamped to [0, 1]. range == NULL is tmo_forward. */
int tmo_forward_range(const float *rgb, int32_t W, int32_t H, const tmo_params *p,
                      const float *range, double *out, tmo_fields *fields);

int tmo_forward(const float *rgb, int32_t W, int32_t H, const tmo_params *p,
                double *out, tmo_fields *fields);

/* Forward at K sampled pixels, every window statistic by direct loops.
 * out: K*3 doubles; cnt/area/sigma2/weight/lf: K*s (each nullable). */
int tmo_forward_pixels(const float *rgb, int32_t W, int32_t H,
                       const tmo_params *p, const int32_t *xs,
                       const int32_t *ys, int64_t K, double *out,
                       uint32_t *cnt, uint32_t *area, double *sigma2,
                       double *weight, double *lf);

/* Smooth forward for finite differences: double input, luminance in double
 * (no float rounding), bin map supplied by the caller and held fixed. */
int tmo_forward_fixed_bins(const double *rgb, int32_t W, int32_t H,
                           const tmo_params *p, const uint8_t *bins,
                           double *out);

/* Hand-written FP64 adjoint of the forward, bins held fixed.
 * grad_out: H*W*3; grad_in: H*W*3 (output);
 * grad_params: 3 + 2*s doubles (output) ordered
 *   [ld_min, ld_max, sat, eps[0..s-1], alpha[0..s-1]].
 * lum_f64 = 0: luminance as tmo_luminance (float); 1: in double (for finite
 * differences against tmo_forward_fixed_bins); bins: NULL = computed here. */
int tmo_backward(const double *rgb, int32_t W, int32_t H, const tmo_params *p,
                 int32_t lum_f64, const uint8_t *bins, const double *grad_out,
                 double *grad_in, double *grad_params);

/* Section III capture front-end: Debevec and Malik's radiance map from n
 * exposures. ldr: n pointers to H*W*3 uint8 (HWC) images; times: n exposure
 * times (> 0); log_response: 3 x 256 (channel-major), g_c(z) = ln of the
 * exposure that maps to value z. out: H*W*3 radiances. Weights: the hat
 * w(z) = z (z <= 127), 255 - z; where every weight is zero, the shortest
 * exposure's estimate if it is saturated, else the longest's. */
int tmo_merge_exposures(int32_t n, const uint8_t *const *ldr, const double *times,
                        int32_t W, int32_t H, const double *log_response, double *out);

#endif
