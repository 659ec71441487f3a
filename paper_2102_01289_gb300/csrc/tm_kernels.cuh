// tm_kernels.cuh -- host-side launchers of the tone-mapping kernels.
//
// The forward stages run over a batch of jobs (one per image; a single image
// is a batch of one). Every launcher takes the device copy of the job array,
// the job count and the total number of blocks of its stage.
#pragma once

#include "tm_common.cuh"

namespace tmk {

// Stage a0: range of Eq. 11 luminance, bin edges, quantisation constants.
// dtype: the dtype every job's input shares, else -1.
void launch_range(const Job *jobs, int njobs, int blocks, int n_bins, int dtype, cudaStream_t s);
// Stage a1: bin map (uint8), quantised normalised log (int32), the per-row
// 32-column bin ranges (J.grp, when set) and zeroed count planes (J.cnt,
// when set: n_fields uint32 planes). dtype as for launch_range.
void launch_prep(const Job *jobs, int njobs, int blocks, int n_bins, int flags, int n_fields, int dtype,
                 cudaStream_t s);
// The dtype every job's input shares, else -1 (host).
int input_dtype(const Job *jobs, int njobs);
// Blocks of the range / prep stages for one image.
int range_blocks(int W, int H, int num_sms, double share);
int prep_blocks(int W, int H, int num_sms, double share);

// Stage a2 (Eq. 5): integral images of q and q^2, (H+1) x (W+1) int64, over
// tiles of row segments x column chunks. integral_layout picks the segments
// (J.nseg of J.seg_rows rows) whose scratch fits max_scratch_elems (the
// shortest such, at least 16 rows; at worst one segment). Per image:
// integral_tile_blocks(W, nseg) blocks of the tile launches (first block
// J.b0[kStRows]), integral_col_blocks(W) of the column-prefix launch
// (J.b0[kStCols]), and integral_scratch_elems(W, H, nseg) int64 elements of
// scratch at J.segtot. Returns the number of launches.
void integral_layout(int W, int H, size_t max_scratch_elems, int &nseg, int &seg_rows);
size_t integral_scratch_elems(int W, int H, int nseg);
int integral_tile_blocks(int W, int nseg);
int integral_col_blocks(int W);
int launch_integral_jobs(const Job *jobs, int njobs, int tile_blocks, int col_blocks, cudaStream_t s);

// The backward's integral planes (64-bit fixed point) of one image's `np`
// float plane pairs (u_p, v_p), each W x H: u_p scaled by 2^fix_shift(amax[p],
// nmax[p]) and v_p by 2^fix_shift(amax[kMaxFields + p], nmax[p]) (amax on the
// device), interleaved into pair plane p of dst ((H+1) x (W+1) positions of
// two int64). Over a batch: the image's first blocks in the tile and column
// launches are b0_tile and b0_col.
struct alignas(16) FixJob {
  const float *u, *v;
  const unsigned *amax;
  unsigned long long *dst;
  long long *scratch;        // fix_integral_scratch_elems(W, H, np, nseg) int64
  long long scratch_stride;  // per pair
  int W, H, nseg, seg_rows, np;
  int b0_tile, b0_col;
  float nmax[kMaxFields];
};
static_assert(sizeof(FixJob) % 16 == 0, "jobs are copied in 16-byte words");

// Row segments of an image in a batch of batch_pairs pairs in all; the scratch,
// tile blocks and column blocks of its np pairs; the three launches over a
// batch (returns 3).
void fix_layout(int W, int H, long long batch_pairs, int &nseg, int &seg_rows);
size_t fix_integral_scratch_elems(int W, int H, int pairs, int nseg);
int fix_tile_blocks(int W, int nseg, int pairs);
int fix_col_blocks(int W, int pairs);
int launch_fix_integrals(const FixJob *jobs, int n, int tile_blocks, int col_blocks, cudaStream_t s);

// Stage a3 (Eq. 7-8), materialised: integral histogram planes,
// (H+1) x (W+1) uint32 each (modulo 2^32, zero first row and column), over
// the integral images' tiles, two planes per tile task. cumulative = true:
// planes k = 1..n-1 hold the integral of [b < k]; cumulative = false: planes
// k = 0..n-1 the integral of [b == k]. `scratch` holds at least
// hist_scratch_bytes(W, H, planes) bytes. Returns the number of launches.
size_t hist_scratch_bytes(int W, int H, int planes);
int launch_integral_histogram(const uint8_t *bins, int W, int H, int n_bins, bool cumulative,
                              uint32_t *planes, void *scratch, cudaStream_t s);

// Stage a3', fused: plan of one image's sweep over strips of `width` (256 or
// 512) own columns (false if the fields do not fit: a swept row over 32
// chunks of 32 columns); segments: the groups of bands wanted for the image
// (its share of a wave). Count plane bytes of the plan (off[f]: byte offset
// of field f's plane). CTAs of the sweep that fit one SM at `smem` bytes of
// dynamic shared memory. The persistent launch over queue slots [0, nitems):
// every job's group starts (slots itemA0 ..), then the groups' other bands
// (itemB0 ..); every job's plan has the launch's width.
bool plan_sweep(const DevParams &P, int W, int H, int segments, size_t smem_limit, int width, SweepPlan &S);
size_t sweep_count_bytes(const DevParams &P, const SweepPlan &S, long long *off);
int sweep_ctas_per_sm(int n_fields, size_t smem, int width);
int launch_sweep(const DevParams &P, const Job *jobs, int njobs, int nitems, int *queue, size_t smem, int ctas,
                 int width, cudaStream_t s);

// Stage a4: per-pixel lookup, tone curve, fusion and colour restoration.
int lookup_blocks(int W, int H);
// plain: no job has debug planes to write and every job's count planes are
// uint32; mom: every job keeps its window moments (else none does); dtype:
// the dtype of every job's input and output when they all share one, else -1.
int launch_lookup_counts(const DevParams &P, const Job *jobs, int njobs, int blocks, bool plain, bool mom,
                         int dtype, cudaStream_t s);
int launch_lookup_materialised(const Image &in, const Image &out, const DevParams &P,
                               const uint8_t *bins, const uint32_t *cplanes, const int64_t *s12,
                               const DebugPlanes &dbg, cudaStream_t s);

}  // namespace tmk
