/*
 * tm.h -- C ABI of the GB300 (sm_103a) local tone-mapping library.
 *
 * The operator is the one of "Mobile-end Tone Mapping based on Integral Image
 * and Integral Histogram" (arXiv 2102.01289): every pixel is tone-mapped by
 * histogram adjustment (Eq. 1, Eq. 2) inside s centred receptive fields, the
 * fields are fused with variance weights (Eq. 3, Eq. 4, Eq. 10) and colour is
 * restored (Eq. 12). Window histograms and sums come from integral histograms
 * and integral images (Eq. 5-9). Luminance is Eq. 11.
 *
 * Conventions shared by every entry point
 *   - Images are interleaved RGB (HWC, 3 channels). tm_image.pitch is the
 *     number of ELEMENTS (not bytes) from the start of one row to the next and
 *     must be >= 3 * width. Pointers named "device" must be CUDA device (or
 *     managed) memory; "host" pointers are ordinary or pinned host memory.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *     stream. Entry points are stream-ordered and asynchronous unless stated.
 *   - Ownership: the caller owns every image and output buffer; a tm_ctx owns
 *     its device workspace (grown on demand, released by tm_destroy).
 *   - A tm_ctx is not thread-safe; use one per host thread, or serialise.
 *   - Errors: invalid arguments are rejected on the host before any launch and
 *     return TM_EINVAL (or TM_EUNSUPPORTED); no GPU work is issued then. CUDA
 *     failures return TM_ECUDA. tm_last_error() gives the message of the most
 *     recent failure on that context.
 */
#ifndef TM_H
#define TM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TM_ABI_VERSION 1
#define TM_MAX_FIELDS 8
#define TM_MAX_BINS 256
#define TM_MAX_RADIUS 32767

typedef enum tm_status {
  TM_OK = 0,
  TM_EINVAL = 1,        /* bad argument (null pointer, size, parameter)     */
  TM_ENOMEM = 2,        /* device or host allocation failed                 */
  TM_ECUDA = 3,         /* a CUDA runtime call or launch failed             */
  TM_EUNSUPPORTED = 4,  /* valid but unsupported combination (dtype pair)   */
  TM_ETIMEOUT = 5,      /* a bounded device-side wait gave up               */
  TM_ESTATE = 6         /* call not valid in the context's current state    */
} tm_status;

typedef enum tm_dtype {
  TM_F32 = 0,  /* float                                  */
  TM_F16 = 1,  /* IEEE half                               */
  TM_U8 = 2    /* uint8, output only: floor(255 c + 0.5) with c clamped to [0,1] */
} tm_dtype;

/* Operator parameters (copied by tm_create).
 *   n_bins    n of Section II-A / Eq. 7: equal-width bins of the log luminance
 *             over the image's range; 1..256. Paper default 5 (Section IV).
 *   n_fields  s of Eq. 3; 1..8. Paper default 5 (Section IV).
 *   rx, ry    half-sizes of field i: the window is [x-rx, x+rx] x [y-ry, y+ry]
 *             (Algorithm 1, corners x-(r+1) and x+r), clipped to the image.
 *             0..32767.
 *   eps       epsilon of Eq. 4 per field, > 0. Paper 0.1 (Section II-C).
 *   alpha     weight multiplying W of Eq. 4 per field, >= 0 (1 = the paper).
 *   ld_min, ld_max  min(L_d), max(L_d) of Eq. 2, ld_max >= ld_min.
 *   sat       colour saturation of Eq. 12, >= 0. Paper 0.6.
 *   flags     reading variants; 0 selects the defaults. A combination of
 *               TM_FLAG_CDF_INCLUSIVE  Eq. 1 counts b(q) <= b(p) (default <).
 *               TM_FLAG_AREA_LITERAL   window area (2 rx + 1)(2 ry + 1) of
 *                                      Algorithm 1, the pixels outside the
 *                                      image taking part as zeros (default:
 *                                      the window clipped to the image).
 *               TM_FLAG_VAR_LINEAR     Eq. 10 on i / imax (default: the
 *                                      normalised log). tm_backward rejects it.
 *               TM_FLAG_SRGB_U8        TM_U8 outputs are sRGB-encoded
 *                                      (IEC 61966-2-1) before quantisation.
 *             Other bits: TM_EINVAL.
 * Variance of Eq. 10 is taken over the normalised log luminance
 * (ln i - ln imin) / (ln imax - ln imin); it is the window variance. */
#define TM_FLAG_CDF_INCLUSIVE 1
#define TM_FLAG_AREA_LITERAL 2
#define TM_FLAG_VAR_LINEAR 4
#define TM_FLAG_SRGB_U8 8
typedef struct tm_params {
  int32_t n_bins;
  int32_t n_fields;
  int32_t rx[TM_MAX_FIELDS];
  int32_t ry[TM_MAX_FIELDS];
  float eps[TM_MAX_FIELDS];
  float alpha[TM_MAX_FIELDS];
  float ld_min;
  float ld_max;
  float sat;
  int32_t flags;
} tm_params;

typedef struct tm_image {
  void *data;       /* first sample of row 0 (device or host, per entry point) */
  int32_t width;    /* pixels per row, >= 1                                    */
  int32_t height;   /* rows, >= 1                                              */
  int64_t pitch;    /* elements between row starts, >= 3 * width              */
  int32_t dtype;    /* tm_dtype                                                */
} tm_image;

typedef struct tm_ctx tm_ctx;

/* Fill *p with the paper's quality setting (Section IV: n = 5, s = 5,
 * eps = 0.1) on its 2048 x 2048 example pyramid (Section II-C: field sizes
 * 2048, 1024, 512, 256, 128, i.e. half-sizes 1024, 512, 256, 128, 64),
 * alpha = 1, L_d = [0, 1], sat = 0.6 (Eq. 12). */
void tm_params_default(tm_params *p);

/* Fill *p with the paper's pyramid for a width x height image (Section II-C):
 * field i has size (width / 2^i) x (height / 2^i), i.e. half-sizes
 * rx = width >> (i+1), ry = height >> (i+1), so field 0 is as large as the
 * image and w_i / w_{i+1} = 2. Other members as tm_params_default.
 * n_fields 1..8, n_bins 1..256. */
tm_status tm_params_pyramid(tm_params *p, int32_t width, int32_t height,
                            int32_t n_fields, int32_t n_bins);

/* Validate *params and create a context (host only; no GPU work until the
 * first call that runs kernels). *out receives the context or NULL on error.
 * Errors: TM_EINVAL for a bad parameter, TM_ENOMEM. */
tm_status tm_create(const tm_params *params, tm_ctx **out);

/* Release the context and its device workspace. Synchronises the device
 * first. NULL is ignored. */
void tm_destroy(tm_ctx *ctx);

/* Message of the most recent failure on ctx ("" if none); valid until the
 * next call on ctx. A NULL ctx gives the message of the last tm_create. */
const char *tm_last_error(const tm_ctx *ctx);

/* Static name of a status code. */
const char *tm_status_string(tm_status s);

/* Forward operator on one image (Eq. 11 -> Eq. 12 over the whole path):
 * luminance, global range and bins, integral image, integral histogram, the
 * per-pixel multi-field lookup, fusion and colour restoration.
 *   in   device image, dtype TM_F32 or TM_F16.
 *   out  device image of the same width/height, dtype TM_F32, TM_F16 or TM_U8;
 *        must not overlap in.
 * Asynchronous on `stream`, except that with the automatic histogram path
 * (TM_OPT_HIST_PATH = 0, the default) the first call for an image size and
 * dtype pair times both paths and synchronises `stream` once. The context's
 * workspace is reused, so calls on one context must be ordered (same stream,
 * or synchronised). On the fused path, an (in, out) pair of descriptors that
 * comes back is captured in a CUDA graph of the context and replayed while
 * the same descriptors are passed (a replay reads the current pixel
 * contents); not with debug exports, stage timing or streaming range reuse
 * on. The context keeps six such graphs (batches' included). */
tm_status tm_forward(tm_ctx *ctx, const tm_image *in, const tm_image *out,
                     void *stream);

/* Same operator on host buffers: copies `in` to the device, runs tm_forward
 * and copies the result back into `out`, then synchronises `stream`. Host
 * buffers may be pageable; pinned buffers make the copies asynchronous. A
 * page-locked output buffer (cudaHostAlloc / cudaHostRegister) is written
 * directly by the last kernel over the host link instead of being copied
 * after it; the result is the same. */
tm_status tm_forward_host(tm_ctx *ctx, const tm_image *in_host,
                          const tm_image *out_host, void *stream);

/* tm_forward_host without the synchronisation, for streams of host images:
 * in_host and out_host must be page-locked (cudaHostAlloc / cudaHostRegister;
 * TM_EINVAL otherwise). Call k uploads in_host into device input slot k%2 on
 * an internal copy stream, runs the forward into device output slot k%2 on an
 * internal forward stream, and downloads that slot into out_host on `stream`.
 * So the upload of the next image, the forward of this one and the download
 * of the previous one run at the same time (the host link carries uploads
 * and downloads concurrently). Returns once the work is enqueued: in_host
 * must stay unchanged and out_host unread until `stream` has been
 * synchronised, which covers the upload, forward and download of every call
 * made on it. The upload is not ordered after earlier work on `stream` (write
 * in_host on the host). Other calls on the context wait for the pending
 * forwards before using the workspace, and the next forward waits for them.
 * Results are identical to tm_forward_host. */
tm_status tm_forward_host_async(tm_ctx *ctx, const tm_image *in_host,
                                const tm_image *out_host, void *stream);

/* Forward over n images of possibly different sizes. Images whose fields do
 * not fit the fused sweep take the materialised integral histogram; the
 * others take TM_OPT_HIST_PATH's path (automatic: the first batch of a given
 * list of sizes and dtype pairs times both batched passes on those images,
 * synchronising `stream` once, and keeps the faster for later batches).
 * The images on the fused path run as one batched pass: one launch per
 * stage, the sweep as one persistent launch over a shared queue of (image,
 * strip, row band) tiles. Those on the materialised path run as another:
 * the range, bin and integral-image stages once for all of them, then each
 * image's integral histogram and lookup. in[i], out[i] as for tm_forward
 * (host arrays of descriptors; the pixel data is on the device). n == 0 is a
 * no-op. Each pass is captured in a CUDA graph and replayed while the same
 * descriptors (pointers, sizes, pitches, dtypes) are passed; a replay reads
 * the current pixel contents. Results are bit-identical to per-image
 * tm_forward calls (both paths give the same outputs bit for bit). */
tm_status tm_forward_batch(tm_ctx *ctx, int32_t n, const tm_image *in,
                           const tm_image *out, void *stream);

/* Adjoint of tm_forward with the bin map held fixed (bins are piecewise
 * constant in the input). Recomputes the forward intermediates from `in`.
 *   grad_out    device image, TM_F32, dL/d(out).
 *   grad_in     device image, TM_F32, receives dL/d(in); NULL to skip.
 *   grad_params device float[3 + 2*s] receiving
 *               [d ld_min, d ld_max, d sat, d eps[0..s-1], d alpha[0..s-1]];
 *               NULL to skip. Overwritten, not accumulated. */
tm_status tm_backward(tm_ctx *ctx, const tm_image *in, const tm_image *grad_out,
                      const tm_image *grad_in, float *grad_params, void *stream);

/* tm_backward over n images of possibly different sizes: the forward
 * intermediates of all images are recomputed in one batched pass (as in
 * tm_forward_batch), then the adjoint runs one launch per stage over a group
 * of images at a time (up to 66 images, and a workspace under 4 GiB, per
 * group).
 *   in[i], grad_out[i]  host arrays of n device-image descriptors.
 *   grad_in             host array of n descriptors, or NULL to skip.
 *   grad_params         device float[3 + 2*s] receiving the SUM over the n
 *                       images (one shared parameter set); NULL to skip.
 *                       n == 0 writes zeros.
 * Per-image results equal tm_backward's, up to the summation order of the
 * floating-point block sums. Errors as tm_backward, with the image index in
 * the message. */
tm_status tm_backward_batch(tm_ctx *ctx, int32_t n, const tm_image *in, const tm_image *grad_out,
                            const tm_image *grad_in, float *grad_params, void *stream);

/* Eq. 5 on a caller-supplied integer plane: s1 = integral of q, s2 = integral
 * of q*q, both int64 modulo 2^64, (height+1) x (width+1) row-major with a zero
 * first row and column. q: device int32[height*width], |q| <= 2^23.
 * s1, s2: device int64 arrays. Standalone (no context). */
tm_status tm_integral_image(const int32_t *q, int32_t width, int32_t height,
                            int64_t *s1, int64_t *s2, void *stream);

/* tm_integral_image without any allocation (the paper has no counterpart).
 * For callers that must not allocate device memory once running: code under
 * a real-time or per-frame deadline that forbids allocator calls after
 * start-up, code running inside another framework's memory-pool or allocation
 * callbacks where re-entering the CUDA allocator is not allowed, and
 * processes that reserved all device memory up front. Same arguments, layout
 * and results as tm_integral_image; the scratch it needs (a 256-byte-aligned
 * job descriptor plus the tile sums: 16 bytes per column and row segment,
 * with row segments of 16 rows, doubled while the scratch would not fit, and
 * 16 bytes per row and 1024-column chunk) lives in a static device array of
 * 8 MiB that every GPU loading this library keeps until the process exits.
 *   - Every call looks the array's address up for the current device (a
 *     host-side lookup that allocates nothing); the first call on a device
 *     may load the library's device code, so make it before any stream
 *     capture.
 *   - Calls share the array: calls that overlap on the GPU (on different
 *     streams, or from several host threads without ordering) race.
 *   - Returns TM_EINVAL for bad arguments or a size whose scratch exceeds
 *     8 MiB (use tm_integral_image then), TM_ECUDA if a CUDA call fails;
 *     tm_last_error(NULL) then gives the reason. It never calls cudaMalloc,
 *     cudaFree or any allocating routine. */
tm_status tm_integral_image_noalloc(const int32_t *q, int32_t width, int32_t height,
                                    int64_t *s1, int64_t *s2, void *stream);

/* The capture front-end of Section III: the paper's application captures
 * four exposures and recovers the WDR image from them with Debevec and
 * Malik's radiance-map method before tone mapping it. For each channel c of
 * each pixel, with z_j its 8-bit value in exposure j, g_c the channel's log
 * inverse camera response (g_c(z) = ln of the sensor exposure that maps to
 * z) and dt_j the exposure times,
 *     ln E = sum_j w(z_j) (g_c(z_j) - ln dt_j) / sum_j w(z_j),
 *     w(z) = z for z <= 127, 255 - z above,
 * and out = E. Where every weight is zero (each exposure at 0 or 255) the
 * estimate of the shortest exposure is taken if it is saturated, else that
 * of the longest. The camera response is an input (the paper's capture data
 * and recovered curve are not available).
 *   n             exposures, 1..8.
 *   ldr           host array of n device pointers, each an HWC uint8 image of
 *                 width x height pixels with `pitch` elements per row.
 *   times         host array of n exposure times, > 0.
 *   log_response  host float[3 * 256], channel-major g_c(z); finite.
 *   out           device image, TM_F32 or TM_F16, width x height.
 * Standalone (no context), asynchronous on `stream`; allocates nothing.
 * Errors: TM_EINVAL for bad arguments (message in tm_last_error(NULL)). */
tm_status tm_merge_exposures(int32_t n, const uint8_t *const *ldr, const float *times, int32_t width,
                             int32_t height, int64_t pitch, const float *log_response,
                             const tm_image *out, void *stream);

/* Eq. 7-8 on a caller-supplied bin map: hk = n_bins planes, each the
 * (height+1) x (width+1) uint32 integral image of [bins == k] (zero first row
 * and column), plane-major. bins: device uint8[height*width], values < n_bins.
 * Standalone (no context). */
tm_status tm_integral_histogram(const uint8_t *bins, int32_t width,
                                int32_t height, int32_t n_bins, uint32_t *hk,
                                void *stream);

/* Debug exports (after a tm_forward on ctx with debug enabled). `what`:
 *   TM_DBG_RANGE      float[2]      imin, imax of Eq. 11 luminance
 *   TM_DBG_THRESHOLDS float[n-1]    bin edges (smallest float >= exact edge)
 *   TM_DBG_BINS       uint8[H*W]    bin map
 *   TM_DBG_Q          int32[H*W]    quantised normalised log luminance
 *   TM_DBG_COUNTS     uint32[s*H*W] #{q in w_i : b(q) < b(p)} (Eq. 1)
 *   TM_DBG_SIGMA2     float[s*H*W]  window variance (Eq. 10)
 *   TM_DBG_WEIGHT     float[s*H*W]  W of Eq. 4
 *   TM_DBG_LF         float[s*H*W]  L_{w_i} of Eq. 2
 *   TM_DBG_L          float[H*W]    fused L of Eq. 3
 *   TM_DBG_QSHIFT     int32[1]      Q: q = round(2^Q lhat) - 2^(Q-1)
 * dst is a device pointer of at least tm_debug_size() bytes. */
enum {
  TM_DBG_RANGE = 1,
  TM_DBG_THRESHOLDS = 2,
  TM_DBG_BINS = 3,
  TM_DBG_Q = 4,
  TM_DBG_COUNTS = 5,
  TM_DBG_SIGMA2 = 6,
  TM_DBG_WEIGHT = 7,
  TM_DBG_LF = 8,
  TM_DBG_L = 9,
  TM_DBG_QSHIFT = 10
};
tm_status tm_set_debug(tm_ctx *ctx, int32_t enable);
tm_status tm_debug_size(tm_ctx *ctx, int32_t what, size_t *bytes);
tm_status tm_debug_export(tm_ctx *ctx, int32_t what, void *dst, size_t bytes,
                          void *stream);

/* Tuning options.
 *   TM_OPT_HIST_PATH     0 = automatic (default), 1 = fused sliding sweep,
 *                        2 = materialised bin-major integral histogram.
 *                        Automatic: the first single-image forward of each
 *                        (width, height, input dtype, output dtype) on a
 *                        context runs both paths twice, timing the second
 *                        runs (it synchronises its stream once), and keeps
 *                        the faster; later forwards of that size take it
 *                        directly. Batches and tm_backward take the fused
 *                        path where it fits.
 *   TM_OPT_STAGE_TIMING  1 = record a CUDA event after every stage of each
 *                        forward/backward call on its stream (see
 *                        tm_stage_times); 0 = off (default).
 *   TM_OPT_REUSE_RANGE   1 = streaming video: tm_forward bins and
 *                        normalises each image with the luminance range of
 *                        the previous tm_forward on this context (same size),
 *                        and takes the image's own range for the next one
 *                        inside the bin pass, so the input is read once less.
 *                        The normalised log is clamped to [0, 1]. The first
 *                        image, and one whose size differs from the previous,
 *                        use their own range. A variant of the paper's method
 *                        (which takes each image's own range); off by default.
 *                        Batches and tm_backward always use each image's own
 *                        range.
 *   TM_OPT_BACKWARD_REUSE 1 = tm_backward / tm_backward_batch take the forward
 *                        intermediates (bin map, quantised log, integral
 *                        images, count planes) from the context's workspace
 *                        instead of recomputing them, when the last forward
 *                        call on the context ran the fused path, each image
 *                        over its own range, on the same image descriptors
 *                        (pointers, sizes, pitches, dtypes) in the same order.
 *                        The caller guarantees that the pixels of `in` have
 *                        not changed since that forward (an autograd function
 *                        holding its saved input does). Results are those of
 *                        the recomputation. While the option is on, the
 *                        forward's lookup also keeps each field's window
 *                        variance and mean of the normalised log (8 bytes per
 *                        field and pixel) for the backward to read.
 *                        0 = always recompute (default).
 *   TM_OPT_SWEEP_TILES   tuning: segments (groups of bands of one strip)
 *                        that the fused sweep cuts each image into, rounded
 *                        to whole strips; 0 = automatic (one wave of the
 *                        sweep's resident CTAs, shared among a batch's images
 *                        by pixel count). Results do not depend on it.
 *   TM_OPT_SWEEP_WIDTH   tuning: own columns of the fused sweep's strips,
 *                        256 (two CTAs of 512 threads per SM) or 512 (one
 *                        CTA of 1024 threads per SM; taken only where every
 *                        image of the call fits it, else 256); 0 = automatic
 *                        (512 where every image fits it). Other values are
 *                        TM_EINVAL. Results do not depend on it.
 */
enum {
  TM_OPT_HIST_PATH = 1,
  TM_OPT_STAGE_TIMING = 2,
  TM_OPT_REUSE_RANGE = 3,
  TM_OPT_BACKWARD_REUSE = 4,
  TM_OPT_SWEEP_TILES = 5,
  TM_OPT_SWEEP_WIDTH = 6
};
tm_status tm_set_option(tm_ctx *ctx, int32_t key, int64_t value);

/* Per-stage device time, summed over every call since the previous read,
 * with stage timing on. Writes up to `cap` entries: ms[i] milliseconds and
 * names[i] a static stage name. Synchronises with the last recorded event
 * and resets the sums. Returns the number of stages written, or -1 on error
 * (message in tm_last_error). */
int32_t tm_stage_times(tm_ctx *ctx, float *ms, const char **names, int32_t cap);

/* Number of kernels launched by the most recent forward/backward/batch call
 * on ctx (for launch accounting). */
int64_t tm_last_launch_count(const tm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* TM_H */
