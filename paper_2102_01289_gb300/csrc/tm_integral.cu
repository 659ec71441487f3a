// tm_integral.cu -- integral images (Eq. 5) and integral histograms (Eq. 7-8).
//
// Both are two-pass: a row pass (block-wide scans, warp shuffles inside each
// warp) writes row prefixes into an (H+1) x (W+1) plane with a zero first row
// and column; a column pass then accumulates down the rows. The column pass is
// split into row segments: a first kernel sums each segment, a second one adds
// the sums of the segments above and scans its own segment. Integer
// arithmetic is modular (2^64 for q sums, 2^32 for counts), so box sums
// (Eq. 6, Eq. 9) are exact whatever the image size.
#include "tm_kernels.cuh"

namespace tmk {
namespace {

template <typename T, int NT>
__device__ __forceinline__ T block_exclusive_scan(T v, T *warp_tot, T &total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    T w = lane < NT / 32 ? warp_tot[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < NT / 32) warp_tot[lane] = w;
  }
  __syncthreads();
  T before = wid > 0 ? warp_tot[wid - 1] : T(0);
  total = warp_tot[NT / 32 - 1];
  __syncthreads();
  return before + x - v;
}

constexpr int kNT = 256;
constexpr int kItems = 8;
constexpr int kTile = kNT * kItems;

// Row prefixes of q and q^2 into rows 1..H of s1 / s2 (Eq. 5, first pass).
// Loads and stores go through shared memory so that global accesses are
// coalesced while each thread scans eight consecutive elements; the shared
// layouts are padded (9 slots per 8 elements) against bank conflicts.
__device__ __forceinline__ int pad9(int i) { return (i >> 3) * 9 + (i & 7); }

__global__ void __launch_bounds__(kNT) k_rows_q(const Job *__restrict__ jobs, int njobs) {
  __shared__ int32_t tile[kTile / 8 * 9];
  __shared__ long long out1[kTile / 8 * 9], out2[kTile / 8 * 9];
  __shared__ long long wt1[kNT / 32], wt2[kNT / 32];
  const int j = find_job(jobs, njobs, kStRows, blockIdx.x);
  const Job &J = jobs[j];
  const int y = blockIdx.x - J.b0[kStRows];
  const int W = J.in.W;
  const long long W1 = (long long)W + 1;
  long long *s1 = J.s1, *s2 = J.s2;
  if (y == 0)
    for (long long x = threadIdx.x; x < W1; x += kNT) s1[x] = 0, s2[x] = 0;
  const int32_t *row = J.q + (long long)y * W;
  long long *o1 = s1 + (long long)(y + 1) * W1;
  long long *o2 = s2 + (long long)(y + 1) * W1;
  if (threadIdx.x == 0) o1[0] = 0, o2[0] = 0;
  long long carry1 = 0, carry2 = 0;
  for (int base = 0; base < W; base += kTile) {
    for (int i = threadIdx.x; i < kTile; i += kNT) tile[pad9(i)] = base + i < W ? __ldg(row + base + i) : 0;
    __syncthreads();
    long long a1 = 0, a2 = 0, l1[kItems], l2[kItems];
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
      const long long v = tile[threadIdx.x * 9 + k];
      a1 += v;
      a2 += v * v;
      l1[k] = a1;
      l2[k] = a2;
    }
    long long t1, t2;
    const long long e1 = block_exclusive_scan<long long, kNT>(a1, wt1, t1) + carry1;
    const long long e2 = block_exclusive_scan<long long, kNT>(a2, wt2, t2) + carry2;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
      out1[threadIdx.x * 9 + k] = e1 + l1[k];
      out2[threadIdx.x * 9 + k] = e2 + l2[k];
    }
    __syncthreads();
    const int n = min(kTile, W - base);
    for (int i = threadIdx.x; i < n; i += kNT) {
      o1[base + i + 1] = out1[pad9(i)];
      o2[base + i + 1] = out2[pad9(i)];
    }
    carry1 += t1;
    carry2 += t2;
    __syncthreads();
  }
}

// Column pass over the integral images of the jobs: block -> (plane, segment,
// 128-column chunk) of its job. First kernel: segment sums.
__global__ void __launch_bounds__(128) k_colsum_jobs(const Job *__restrict__ jobs, int njobs) {
  const int j = find_job(jobs, njobs, kStCols, blockIdx.x);
  const Job &J = jobs[j];
  const int lb = blockIdx.x - J.b0[kStCols];
  const int cols = J.in.W + 1, rows = J.in.H + 1;
  const int chunks = (cols + 127) / 128;
  const int pl = lb / (chunks * J.nseg), rem = lb - pl * chunks * J.nseg;
  const int seg = rem / chunks, ch = rem - seg * chunks;
  const int c = ch * 128 + threadIdx.x;
  if (c >= cols) return;
  const long long *P = pl ? J.s2 : J.s1;
  const int r0 = 1 + seg * J.seg_rows, r1 = min(rows, r0 + J.seg_rows);
  long long acc = 0;
#pragma unroll 4
  for (int r = r0; r < r1; ++r) acc += P[(long long)r * cols + c];
  J.segtot[((long long)pl * J.nseg + seg) * cols + c] = acc;
}

// Second kernel: offset by the segments above, scan in place.
__global__ void __launch_bounds__(128) k_colscan_jobs(const Job *__restrict__ jobs, int njobs) {
  const int j = find_job(jobs, njobs, kStCols, blockIdx.x);
  const Job &J = jobs[j];
  const int lb = blockIdx.x - J.b0[kStCols];
  const int cols = J.in.W + 1, rows = J.in.H + 1;
  const int chunks = (cols + 127) / 128;
  const int pl = lb / (chunks * J.nseg), rem = lb - pl * chunks * J.nseg;
  const int seg = rem / chunks, ch = rem - seg * chunks;
  const int c = ch * 128 + threadIdx.x;
  if (c >= cols) return;
  long long *P = pl ? J.s2 : J.s1;
  long long acc = 0;
  for (int s = 0; s < seg; ++s) acc += J.segtot[((long long)pl * J.nseg + s) * cols + c];
  const int r0 = 1 + seg * J.seg_rows, r1 = min(rows, r0 + J.seg_rows);
#pragma unroll 4
  for (int r = r0; r < r1; ++r) {
    acc += P[(long long)r * cols + c];
    P[(long long)r * cols + c] = acc;
  }
}

// Row prefixes of bin indicators (Eq. 7) into rows 1..H of each plane.
__global__ void __launch_bounds__(kNT) k_rows_hist(const uint8_t *__restrict__ bins, int W, int H,
                                                   int k_begin, int n_planes, int per_block,
                                                   int cumulative, unsigned *planes,
                                                   long long plane_stride) {
  __shared__ uint8_t tile[kTile];
  __shared__ unsigned wt[kNT / 32];
  const long long W1 = (long long)W + 1;
  for (int y = blockIdx.x; y < H; y += gridDim.x) {
  const uint8_t *row = bins + (long long)y * W;
  const int p0 = blockIdx.y * per_block, p1 = min(p0 + per_block, n_planes);
  for (int pl = p0; pl < p1; ++pl) {
    const int k = k_begin + pl;
    unsigned *P = planes + pl * plane_stride;
    if (y == 0)
      for (long long x = threadIdx.x; x < W1; x += kNT) P[x] = 0;
    unsigned *o = P + (long long)(y + 1) * W1;
    if (threadIdx.x == 0) o[0] = 0;
    unsigned carry = 0;
    for (int base = 0; base < W; base += kTile) {
      for (int i = threadIdx.x; i < kTile; i += kNT) tile[i] = base + i < W ? row[base + i] : 0xff;
      __syncthreads();
      unsigned a = 0, l[kItems];
#pragma unroll
      for (int j = 0; j < kItems; ++j) {
        int b = tile[threadIdx.x * kItems + j];
        bool in_img = base + threadIdx.x * kItems + j < W;
        a += (in_img && (cumulative ? (b < k) : (b == k))) ? 1u : 0u;
        l[j] = a;
      }
      unsigned t;
      unsigned e = block_exclusive_scan<unsigned, kNT>(a, wt, t);
#pragma unroll
      for (int j = 0; j < kItems; ++j) {
        int x = base + threadIdx.x * kItems + j;
        if (x < W) o[x + 1] = carry + e + l[j];
      }
      carry += t;
      __syncthreads();
    }
  }
  }
}

// Column pass, first kernel: sum of each row segment of each column.
template <typename T>
__global__ void k_colsum(const T *__restrict__ base, long long plane_stride, int cols, int rows,
                         int seg_rows, int nseg, T *segtot) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int seg = blockIdx.y, pl = blockIdx.z;
  if (c >= cols) return;
  const T *P = base + pl * plane_stride;
  const int r0 = 1 + seg * seg_rows, r1 = min(rows, r0 + seg_rows);
  T acc = 0;
#pragma unroll 4
  for (int r = r0; r < r1; ++r) acc += P[(long long)r * cols + c];
  segtot[((long long)pl * nseg + seg) * cols + c] = acc;
}

// Column pass, second kernel: offset by the segments above, scan in place.
template <typename T>
__global__ void k_colscan(T *base, long long plane_stride, int cols, int rows, int seg_rows,
                          int nseg, const T *__restrict__ segtot) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int seg = blockIdx.y, pl = blockIdx.z;
  if (c >= cols) return;
  T *P = base + pl * plane_stride;
  T acc = 0;
  for (int s = 0; s < seg; ++s) acc += segtot[((long long)pl * nseg + s) * cols + c];
  const int r0 = 1 + seg * seg_rows, r1 = min(rows, r0 + seg_rows);
#pragma unroll 4
  for (int r = r0; r < r1; ++r) {
    acc += P[(long long)r * cols + c];
    P[(long long)r * cols + c] = acc;
  }
}

void segments(int cols, int H, int planes, int &nseg, int &seg_rows) {
  long long target = 160000;
  long long per = (long long)cols * planes;
  nseg = (int)((target + per - 1) / per);
  if (nseg < 1) nseg = 1;
  if (nseg > 64) nseg = 64;
  if (nseg > H) nseg = H;
  seg_rows = (H + nseg - 1) / nseg;
  nseg = (H + seg_rows - 1) / seg_rows;
}

template <typename T>
void column_pass(T *base, long long plane_stride, int planes, int W, int H, T *scratch,
                 cudaStream_t s) {
  const int cols = W + 1, rows = H + 1;
  int nseg, seg_rows;
  segments(cols, H, planes, nseg, seg_rows);
  dim3 block(128), grid((cols + 127) / 128, nseg, planes);
  if (nseg > 1) k_colsum<T><<<grid, block, 0, s>>>(base, plane_stride, cols, rows, seg_rows, nseg, scratch);
  k_colscan<T><<<grid, block, 0, s>>>(base, plane_stride, cols, rows, seg_rows, nseg, scratch);
}

}  // namespace

void column_segments(int W, int H, int planes, int &nseg, int &seg_rows) {
  segments(W + 1, H, planes, nseg, seg_rows);
}

int col_blocks(int W, int nseg) { return ((W + 1 + 127) / 128) * nseg * 2; }

int launch_integral_jobs(const Job *jobs, int njobs, int row_blocks, int colb, bool multi_seg,
                         cudaStream_t s) {
  k_rows_q<<<row_blocks, kNT, 0, s>>>(jobs, njobs);
  if (multi_seg) k_colsum_jobs<<<colb, 128, 0, s>>>(jobs, njobs);
  k_colscan_jobs<<<colb, 128, 0, s>>>(jobs, njobs);
  return multi_seg ? 3 : 2;
}

int launch_column_pass_u64(unsigned long long *base, long long plane_stride, int planes, int W, int H,
                           unsigned long long *scratch, cudaStream_t s) {
  int nseg, seg_rows;
  segments(W + 1, H, planes, nseg, seg_rows);
  column_pass<unsigned long long>(base, plane_stride, planes, W, H, scratch, s);
  return nseg > 1 ? 2 : 1;
}

size_t hist_scratch_elems(int W, int H, int planes) {
  int nseg, seg_rows;
  segments(W + 1, H, planes, nseg, seg_rows);
  return (size_t)planes * nseg * (W + 1);
}

int launch_integral_histogram(const uint8_t *bins, int W, int H, int n_bins, bool cumulative,
                              uint32_t *planes, uint32_t *scratch, cudaStream_t s) {
  const int k_begin = cumulative ? 1 : 0;
  const int n_planes = cumulative ? n_bins - 1 : n_bins;
  if (n_planes <= 0) return 0;
  const long long stride = ((long long)W + 1) * ((long long)H + 1);
  const int per_block = 8;
  dim3 grid(H < 65535 ? H : 65535, (n_planes + per_block - 1) / per_block);
  k_rows_hist<<<grid, kNT, 0, s>>>(bins, W, H, k_begin, n_planes, per_block, cumulative ? 1 : 0,
                                   planes, stride);
  int nseg, seg_rows;
  segments(W + 1, H, n_planes, nseg, seg_rows);
  column_pass<unsigned>(planes, stride, n_planes, W, H, scratch, s);
  return 1 + (nseg > 1 ? 2 : 1);
}

}  // namespace tmk
