// tm_integral.cu -- integral images (Eq. 5) and integral histograms (Eq. 7-8).
//
// The integral images of q and q^2 are built over tiles of kIR rows x kIC
// columns in three launches that read q twice and write each plane once:
//   1. per tile: the column sums of the tile's chunk-local row prefixes, each
//      row's chunk total, and the tile total;
//   2. per column: the exclusive prefix over the row segments of those column
//      sums plus the row totals of the chunks to the left (the value of the
//      plane just above each segment);
//   3. per tile: the row prefixes again, offset by the chunks to the left, and
//      accumulated down the tile from the column's offset, written once.
// The same tile kernels, templated on the source of their two planes, build
// the backward's fixed-point integral planes of (u_f, v_f) and the integral
// histograms (indicator planes of the bin map, two thresholds per tile
// task). Integer arithmetic is modular (2^64 in the sums, 2^32 in the
// histogram planes), so box sums (Eq. 6, Eq. 9) are exact whatever the image
// size or summation order.
#include <algorithm>
#include <cstdint>

#include "tm_kernels.cuh"

namespace tmk {
namespace {

constexpr int kItems = 8;  // consecutive columns per thread in a tile row

// Rows go through shared memory so that global accesses are coalesced while
// each thread scans eight consecutive elements; the shared layouts are padded
// (9 slots per 8 elements) against bank conflicts.
__device__ __forceinline__ int pad9(int i) { return (i >> 3) * 9 + (i & 7); }

// ---- integral images of q and q^2 over tiles ----
constexpr int kINT = 128;               // threads of a tile kernel
constexpr int kIC = kINT * kItems;      // columns of a tile (1024)
constexpr int kIR = 16;                 // rows of a tile (one row segment) unless scratch is tight
constexpr int kMidCols = 32;            // columns of a column-prefix block
constexpr int kMidGroups = 16;          // segment groups of a column-prefix block
constexpr int kMidPer = 8;              // segments of a group per batch

// One tiled integral task: two (H+1) x (W+1) int64 planes A and B of an
// image (row 0 and column 0 zero), with their scratch (int64): the tiles'
// column sums, rewritten in place by the column prefix (2 planes x nseg x W),
// the rows' chunk totals (2 x H x nchunk) and the tile totals
// (2 x nseg x nchunk). Row segments of seg_rows rows, nseg of them.
struct IntTask {
  int W, H, nseg, seg_rows, nchunk;
  long long *colsum, *rowsum, *tiletot;
};

__device__ __forceinline__ IntTask int_task(int W, int H, int nseg, int seg_rows, long long *scratch) {
  IntTask t;
  t.W = W;
  t.H = H;
  t.nseg = nseg;
  t.seg_rows = seg_rows;
  t.nchunk = (W + kIC - 1) / kIC;
  t.colsum = scratch;
  t.rowsum = t.colsum + 2LL * nseg * W;
  t.tiletot = t.rowsum + 2LL * H * t.nchunk;
  return t;
}

// Values of the planes: q and q^2 of the quantised log (Eq. 5 of q).
struct QSource {
  using Raw = int32_t;
  const int32_t *q;
  int W;
  __device__ __forceinline__ Raw load(int r, int c) const { return __ldg(q + (long long)r * W + c); }
  // columns c .. c + 3 of row r (zero past W); vec: rows are 16-byte aligned
  __device__ __forceinline__ void load4(int r, int c, bool vec, Raw *x) const {
    const int32_t *p = q + (size_t)r * W + c;
    if (vec && c + 3 < W) {
      const int4 v = __ldg(reinterpret_cast<const int4 *>(p));
      x[0] = v.x, x[1] = v.y, x[2] = v.z, x[3] = v.w;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) x[j] = c + j < W ? __ldg(p + j) : 0;
    }
  }
  __device__ __forceinline__ bool vec_ok() const {
    return (W & 3) == 0 && (reinterpret_cast<uintptr_t>(q) & 15) == 0;
  }
  // warp sums of a thread's four-element partial row sums: |q| <= 2^23, so a
  // partial sum of q fits 26 bits and one of q^2 splits into two 24-bit
  // parts, each summed exactly in 32 bits by the warp reduction
  __device__ __forceinline__ void warp_sums(long long &su, long long &sv) const {
    su = (long long)__reduce_add_sync(0xffffffffu, (int)su);
    const unsigned long long v = (unsigned long long)sv;
    const unsigned hi = __reduce_add_sync(0xffffffffu, (unsigned)(v >> 24));
    const unsigned lo = __reduce_add_sync(0xffffffffu, (unsigned)(v & 0xffffffu));
    sv = (long long)(((unsigned long long)hi << 24) + lo);
  }
  __device__ __forceinline__ Raw zero() const { return 0; }
  __device__ __forceinline__ void values(Raw x, long long &a, long long &b) const {
    a = x;
    b = (long long)x * x;
  }
};

// Values of the planes: two float planes in 64-bit fixed point, u x 2^sa and
// v x 2^sb rounded to nearest. Each power of two is applied as two float
// factors 2^h and 2^(s - h), h = s / 2 (s in [-67, 209], so both are normal):
// for s >= 0 no product leaves the normal range; for s < 0 only values that
// end below 2^-126 can round twice, and those convert to 0 either way, so
// the integers equal those of a single scaling.
struct FixSource {
  using Raw = float2;
  const float *u, *v;
  int W;
  float a_hi, a_lo, b_hi, b_lo;
  __device__ __forceinline__ Raw load(int r, int c) const {
    const long long o = (long long)r * W + c;
    return make_float2(__ldg(u + o), __ldg(v + o));
  }
  __device__ __forceinline__ Raw zero() const { return make_float2(0.f, 0.f); }
  __device__ __forceinline__ void load4(int r, int c, bool vec, Raw *x) const {
    const size_t o = (size_t)r * W + c;
    if (vec && c + 3 < W) {
      const float4 a = __ldg(reinterpret_cast<const float4 *>(u + o));
      const float4 b = __ldg(reinterpret_cast<const float4 *>(v + o));
      x[0] = make_float2(a.x, b.x), x[1] = make_float2(a.y, b.y);
      x[2] = make_float2(a.z, b.z), x[3] = make_float2(a.w, b.w);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) x[j] = c + j < W ? make_float2(__ldg(u + o + j), __ldg(v + o + j)) : zero();
    }
  }
  __device__ __forceinline__ bool vec_ok() const {
    return (W & 3) == 0 && ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(v)) & 15) == 0;
  }
  __device__ __forceinline__ void warp_sums(long long &su, long long &sv) const {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      su += __shfl_xor_sync(0xffffffffu, su, o);
      sv += __shfl_xor_sync(0xffffffffu, sv, o);
    }
  }
  // u through the hardware conversion (the FP64 pipe), v through the 32-bit
  // integer sequence (the ALU pipe): both give round-to-nearest-even, and the
  // split keeps either pipe from limiting the tile kernels
  __device__ __forceinline__ void values(Raw x, long long &a, long long &b) const {
    a = __float2ll_rn(x.x * a_hi * a_lo);
    b = float_to_i64_rn(x.y * b_hi * b_lo);
  }
};

__device__ __forceinline__ FixSource fix_source_of(const float *u, const float *v, int W, int sa, int sb) {
  return FixSource{u, v, W, ldexpf(1.f, sa / 2), ldexpf(1.f, sa - sa / 2), ldexpf(1.f, sb / 2),
                   ldexpf(1.f, sb - sb / 2)};
}

// Values of the planes: indicators of a bin map for thresholds k0 and k0 + 1,
// [b < k] (cumulative) or [b == k]; raw -1 stands for no pixel.
struct BinSource {
  using Raw = int;
  const uint8_t *bins;
  int W, k0, eq;
  __device__ __forceinline__ Raw load(int r, int c) const { return __ldg(bins + (long long)r * W + c); }
  __device__ __forceinline__ Raw zero() const { return -1; }
  __device__ __forceinline__ void values(Raw x, long long &a, long long &b) const {
    a = x >= 0 && (eq ? x == k0 : x < k0);
    b = x >= 0 && (eq ? x == k0 + 1 : x < k0 + 1);
  }
};

// Exclusive block scan of a pair of values with one set of barriers.
__device__ __forceinline__ void block_scan_pair(long long v1, long long v2, long long (*wt)[kINT / 32],
                                                long long &e1, long long &e2, long long &t1, long long &t2) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long x1 = v1, x2 = v2;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y1 = __shfl_up_sync(0xffffffffu, x1, o), y2 = __shfl_up_sync(0xffffffffu, x2, o);
    if (lane >= o) x1 += y1, x2 += y2;
  }
  if (lane == 31) wt[0][wid] = x1, wt[1][wid] = x2;
  __syncthreads();
  long long b1 = 0, b2 = 0;
#pragma unroll
  for (int w = 0; w < kINT / 32; ++w) {
    if (w < wid) b1 += wt[0][w], b2 += wt[1][w];
  }
  t1 = 0;
  t2 = 0;
#pragma unroll
  for (int w = 0; w < kINT / 32; ++w) t1 += wt[0][w], t2 += wt[1][w];
  e1 = b1 + x1 - v1;
  e2 = b2 + x2 - v2;
  __syncthreads();  // wt is rewritten by the next scan
}

// The thread's kItems strided raw elements (i = threadIdx.x + m kINT) of
// chunk [C0, C0 + nc) of row r; zero past the chunk.
template <class Src>
__device__ __forceinline__ void load_chunk_row(const Src &src, int r, int C0, int nc, typename Src::Raw *v) {
#pragma unroll
  for (int m = 0; m < kItems; ++m) {
    const int i = threadIdx.x + m * kINT;
    v[m] = i < nc ? src.load(r, C0 + i) : src.zero();
  }
}

// Chunk-local row prefixes of planes A and B of one row, given the thread's
// strided raw elements of it (load_chunk_row): thread-local running sums of
// its kItems consecutive columns (l1, l2) and the exclusive offsets of the
// thread (e1, e2); t1, t2 are the row's chunk totals. The row goes through
// shared memory so that the loads were coalesced and each thread scans
// consecutive columns.
template <class Src>
__device__ __forceinline__ void chunk_row_prefix(const Src &src, const typename Src::Raw *v,
                                                 typename Src::Raw *tile, long long (*wt)[kINT / 32],
                                                 long long *l1, long long *l2, long long &e1, long long &e2,
                                                 long long &t1, long long &t2) {
#pragma unroll
  for (int m = 0; m < kItems; ++m) tile[pad9(threadIdx.x + m * kINT)] = v[m];
  __syncthreads();
  long long a1 = 0, a2 = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    long long x1, x2;
    src.values(tile[threadIdx.x * 9 + k], x1, x2);
    a1 += x1;
    a2 += x2;
    l1[k] = a1;
    l2[k] = a2;
  }
  block_scan_pair(a1, a2, wt, e1, e2, t1, t2);  // its barriers also order the tile's reuse
}

// Launch 1: per tile (seg, k), the column sums of the chunk-local row
// prefixes, the rows' chunk totals and the tile totals. The column sum of the
// row prefixes at column c is the prefix, up to c, of the plain column sums
// (both are the sum of the values above and left of c in the tile), so the
// rows are only summed down each column and across each row (warp sums, no
// barrier per row); one block scan over the columns ends the tile. The row
// and tile totals of the last chunk column are read by no later launch (they
// only offset the chunks to their right), so its tiles skip them.
constexpr int kRowGroup = 16;  // rows whose warp partial sums are combined together
struct StatsSmem {
  long long col[2][kIC / 8 * 9];            // the tile's column sums, padded for the scan
  long long row[kRowGroup][2][kINT / 32];   // warp partial sums of a group of rows
  long long wt[2][kINT / 32];               // block scan
};

template <class Src>
__device__ __forceinline__ void int_stats_tile(const IntTask &X, const Src &src, int seg, int k, StatsSmem &sm) {
  const int W = X.W, H = X.H;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int R0 = seg * X.seg_rows, R1 = min(R0 + X.seg_rows, H), C0 = k * kIC, nc = min(kIC, W - C0);
  const bool totals = k + 1 < X.nchunk;  // block-uniform
  long long c1[kItems], c2[kItems];  // sums down the thread's strided columns threadIdx.x + m kINT
#pragma unroll
  for (int m = 0; m < kItems; ++m) c1[m] = c2[m] = 0;
  typename Src::Raw cur[kItems], nxt[kItems];
  load_chunk_row(src, R0, C0, nc, cur);
  for (int r = R0; r < R1; ++r) {
    if (r + 1 < R1) load_chunk_row(src, r + 1, C0, nc, nxt);  // in flight meanwhile
    long long s1 = 0, s2 = 0;
#pragma unroll
    for (int m = 0; m < kItems; ++m) {
      long long x1, x2;
      src.values(cur[m], x1, x2);
      c1[m] += x1;
      c2[m] += x2;
      s1 += x1;
      s2 += x2;
      cur[m] = nxt[m];
    }
    if (!totals) continue;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    const int g = (r - R0) % kRowGroup;
    if (lane == 0) {
      sm.row[g][0][wid] = s1;
      sm.row[g][1][wid] = s2;
    }
    if (g == kRowGroup - 1 || r == R1 - 1) {  // the group's row totals
      __syncthreads();
      if ((int)threadIdx.x <= g) {
        const int rr = r - g + (int)threadIdx.x;
        long long t1 = 0, t2 = 0;
#pragma unroll
        for (int w = 0; w < kINT / 32; ++w) t1 += sm.row[threadIdx.x][0][w], t2 += sm.row[threadIdx.x][1][w];
        X.rowsum[(long long)rr * X.nchunk + k] = t1;
        X.rowsum[((long long)H + rr) * X.nchunk + k] = t2;
      }
      __syncthreads();  // sm.row is rewritten by the next group
    }
  }
  // chunk-local column prefixes of the column sums: consecutive columns per thread
#pragma unroll
  for (int m = 0; m < kItems; ++m) {
    sm.col[0][pad9(threadIdx.x + m * kINT)] = c1[m];
    sm.col[1][pad9(threadIdx.x + m * kINT)] = c2[m];
  }
  __syncthreads();
  long long l1[kItems], l2[kItems], a1 = 0, a2 = 0;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    a1 += sm.col[0][threadIdx.x * 9 + i];
    a2 += sm.col[1][threadIdx.x * 9 + i];
    l1[i] = a1;
    l2[i] = a2;
  }
  long long e1, e2, t1, t2;
  block_scan_pair(a1, a2, sm.wt, e1, e2, t1, t2);
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const int c = C0 + threadIdx.x * kItems + i;
    if (c < W) {
      X.colsum[(long long)seg * W + c] = e1 + l1[i];
      X.colsum[((long long)X.nseg + seg) * W + c] = e2 + l2[i];
    }
  }
  if (threadIdx.x == 0 && totals) {
    X.tiletot[(long long)seg * X.nchunk + k] = t1;
    X.tiletot[((long long)X.nseg + seg) * X.nchunk + k] = t2;
  }
}

// Launch 2: for columns c0 .. c0 + kMidCols - 1 (of the image, one chunk),
// replace each segment's column sum by the plane value just above the
// segment: the sum, over the segments above, of their column sums plus the
// totals of their chunks left of c's chunk. The block's kMidGroups groups
// take kMidPer consecutive segments each per batch, with all loads of a batch
// in flight together.
constexpr int kMidBatch = kMidGroups * kMidPer;
__device__ __forceinline__ void int_mid_cols(const IntTask &X, int c0, long long (*part)[kMidGroups][kMidCols],
                                             long long (*leftT)[kMidBatch]) {
  const int W = X.W;
  const int lane = threadIdx.x % kMidCols, g = threadIdx.x / kMidCols;
  const int c = c0 + lane;
  const int k = c0 / kIC;  // the block's chunk (kMidCols divides kIC)
  long long carry1 = 0, carry2 = 0;
  for (int sb = 0; sb < X.nseg; sb += kMidBatch) {
    // totals of the batch's segments over the chunks left of k
    for (int t = threadIdx.x; t < 2 * kMidBatch; t += kMidCols * kMidGroups) {
      const int pl = t / kMidBatch, s = sb + t % kMidBatch;
      long long v = 0;
      if (s < X.nseg)
        for (int kk = 0; kk < k; ++kk) v += X.tiletot[((long long)pl * X.nseg + s) * X.nchunk + kk];
      leftT[pl][t % kMidBatch] = v;
    }
    __syncthreads();
    const int s0 = sb + g * kMidPer;
    long long v1[kMidPer], v2[kMidPer], sum1 = 0, sum2 = 0;
#pragma unroll
    for (int i = 0; i < kMidPer; ++i) {
      const int s = s0 + i;
      const bool ok = s < X.nseg && c < W;
      v1[i] = ok ? X.colsum[(long long)s * W + c] : 0;
      v2[i] = ok ? X.colsum[((long long)X.nseg + s) * W + c] : 0;
    }
#pragma unroll
    for (int i = 0; i < kMidPer; ++i) {
      if (s0 + i < X.nseg) {
        v1[i] += leftT[0][g * kMidPer + i];
        v2[i] += leftT[1][g * kMidPer + i];
      }
      sum1 += v1[i];
      sum2 += v2[i];
    }
    part[0][g][lane] = sum1;
    part[1][g][lane] = sum2;
    __syncthreads();
    long long run1 = carry1, run2 = carry2;
    for (int h = 0; h < g; ++h) run1 += part[0][h][lane], run2 += part[1][h][lane];
#pragma unroll
    for (int i = 0; i < kMidPer; ++i) {
      const int s = s0 + i;
      if (s < X.nseg && c < W) {
        X.colsum[(long long)s * W + c] = run1;
        X.colsum[((long long)X.nseg + s) * W + c] = run2;
      }
      run1 += v1[i];
      run2 += v2[i];
    }
    for (int h = 0; h < kMidGroups; ++h) carry1 += part[0][h][lane], carry2 += part[1][h][lane];
    __syncthreads();  // part and leftT are rewritten by the next batch
  }
}

// Launch 3: per tile, the full row prefixes (chunk-local prefix plus the
// row's totals of the chunks to the left) accumulated down the tile from the
// value above it, written to rows 1..H, columns 1..W of planes s1 and s2 (as
// OutT, modulo its range; s2 may be null); tiles of the first segment also
// write row 0, tiles of the first chunk column 0. Pair: the planes are
// interleaved (s2 = s1 + 1, two elements per position), and each position is
// written with one 16-byte store.
template <class Src, class OutT, bool Pair = false>
__device__ __forceinline__ void int_write_tile(const IntTask &X, const Src &src, OutT *s1, OutT *s2, int seg,
                                               int k, typename Src::Raw *tile, long long *out1, long long *out2,
                                               long long (*wt)[kINT / 32]) {
  const int W = X.W, H = X.H;
  const long long W1 = (long long)W + 1;
  const int R0 = seg * X.seg_rows, R1 = min(R0 + X.seg_rows, H), C0 = k * kIC, nc = min(kIC, W - C0);
  const bool two = s2 != nullptr;
  const long long os = Pair ? 2 : 1;  // elements per position (Pair: s2 = s1 + 1)
  if (seg == 0) {
    for (int i = threadIdx.x; i < nc; i += kINT) {
      s1[(C0 + 1 + i) * os] = 0;
      if (two) s2[(C0 + 1 + i) * os] = 0;
    }
    if (k == 0 && threadIdx.x == 0) {
      s1[0] = 0;
      if (two) s2[0] = 0;
    }
  }
  if (k == 0)
    for (int r = R0 + (int)threadIdx.x; r < R1; r += kINT) {
      s1[(r + 1) * W1 * os] = 0;
      if (two) s2[(r + 1) * W1 * os] = 0;
    }
  long long acc1[kItems], acc2[kItems];
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const int c = C0 + threadIdx.x * kItems + i;
    acc1[i] = c < W ? X.colsum[(long long)seg * W + c] : 0;
    acc2[i] = c < W ? X.colsum[((long long)X.nseg + seg) * W + c] : 0;
  }
  typename Src::Raw cur[kItems], nxt[kItems];
  load_chunk_row(src, R0, C0, nc, cur);
  for (int r = R0; r < R1; ++r) {
    if (r + 1 < R1) load_chunk_row(src, r + 1, C0, nc, nxt);  // in flight meanwhile
    long long L1 = 0, L2 = 0;  // the row's totals of the chunks to the left
    for (int kk = 0; kk < k; ++kk) {
      L1 += X.rowsum[(long long)r * X.nchunk + kk];
      L2 += X.rowsum[((long long)H + r) * X.nchunk + kk];
    }
    long long l1[kItems], l2[kItems], e1, e2, t1, t2;
    chunk_row_prefix(src, cur, tile, wt, l1, l2, e1, e2, t1, t2);
#pragma unroll
    for (int m = 0; m < kItems; ++m) cur[m] = nxt[m];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      acc1[i] += L1 + e1 + l1[i];
      acc2[i] += L2 + e2 + l2[i];
      out1[threadIdx.x * 9 + i] = acc1[i];
      out2[threadIdx.x * 9 + i] = acc2[i];
    }
    __syncthreads();
    if (Pair) {  // one 16-byte store per position
      longlong2 *o = reinterpret_cast<longlong2 *>(s1) + (long long)(r + 1) * W1 + C0 + 1;
      for (int i = threadIdx.x; i < nc; i += kINT) o[i] = make_longlong2(out1[pad9(i)], out2[pad9(i)]);
      __syncthreads();
      continue;
    }
    OutT *o1 = s1 + (long long)(r + 1) * W1 + C0 + 1;
    for (int i = threadIdx.x; i < nc; i += kINT) o1[i] = (OutT)out1[pad9(i)];
    if (two) {
      OutT *o2 = s2 + (long long)(r + 1) * W1 + C0 + 1;
      for (int i = threadIdx.x; i < nc; i += kINT) o2[i] = (OutT)out2[pad9(i)];
    }
    __syncthreads();  // out1 / out2 are rewritten by the next row
  }
}

// Launch 1 with each thread owning four consecutive columns of the chunk and
// kFSRows rows of loads in flight, 16 bytes at a time where the rows are
// 16-byte aligned: plain column sums down the segment, then one block scan
// over the columns; the same outputs as int_stats_tile.
constexpr int kFS = 256;    // threads of a four-column stats block
constexpr int kFSRows = 4;  // rows in flight per thread
static_assert(kFS * 4 == kIC, "a four-column stats block spans one chunk");

template <class Src>
__device__ __forceinline__ void int_stats4_tile(const IntTask &X, const Src &src, int seg, int k,
                                                long long (*rowp)[2][kFS / 32], long long (*wt)[kFS / 32]) {
  const int W = X.W, H = X.H;
  const int R0 = seg * X.seg_rows, R1 = min(R0 + X.seg_rows, H);
  const int c = k * kIC + 4 * (int)threadIdx.x;
  const bool vec = src.vec_ok();
  const bool totals = k + 1 < X.nchunk;  // block-uniform; see int_stats_tile
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long cu[4] = {0, 0, 0, 0}, cv[4] = {0, 0, 0, 0};
  for (int r0 = R0; r0 < R1; r0 += kFSRows) {
    typename Src::Raw raw[kFSRows][4];
#pragma unroll
    for (int i = 0; i < kFSRows; ++i) {
      if (r0 + i < R1) {
        src.load4(r0 + i, c, vec, raw[i]);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) raw[i][j] = src.zero();
      }
    }
#pragma unroll
    for (int i = 0; i < kFSRows; ++i) {
      long long su = 0, sv = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        long long x1, x2;
        src.values(raw[i][j], x1, x2);
        cu[j] += x1;
        cv[j] += x2;
        su += x1;
        sv += x2;
      }
      const int r = r0 + i;
      if (!totals || r >= R1) continue;  // block-uniform
      src.warp_sums(su, sv);
      const int g = (r - R0) % kRowGroup;
      if (lane == 0) {
        rowp[g][0][wid] = su;
        rowp[g][1][wid] = sv;
      }
      if (g == kRowGroup - 1 || r == R1 - 1) {  // the group's row totals
        __syncthreads();
        if ((int)threadIdx.x <= g) {
          const int rr = r - g + (int)threadIdx.x;
          long long t1 = 0, t2 = 0;
#pragma unroll
          for (int w = 0; w < kFS / 32; ++w) t1 += rowp[threadIdx.x][0][w], t2 += rowp[threadIdx.x][1][w];
          X.rowsum[(long long)rr * X.nchunk + k] = t1;
          X.rowsum[((long long)H + rr) * X.nchunk + k] = t2;
        }
        __syncthreads();  // rowp is rewritten by the next group
      }
    }
  }
  // chunk-local column prefixes of the column sums: the thread's four
  // columns, then an exclusive block scan over the threads
#pragma unroll
  for (int j = 1; j < 4; ++j) {
    cu[j] += cu[j - 1];
    cv[j] += cv[j - 1];
  }
  long long x1 = cu[3], x2 = cv[3];
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y1 = __shfl_up_sync(0xffffffffu, x1, o), y2 = __shfl_up_sync(0xffffffffu, x2, o);
    if (lane >= o) x1 += y1, x2 += y2;
  }
  if (lane == 31) wt[0][wid] = x1, wt[1][wid] = x2;
  __syncthreads();
  long long e1 = x1 - cu[3], e2 = x2 - cv[3], t1 = 0, t2 = 0;
#pragma unroll
  for (int w = 0; w < kFS / 32; ++w) {
    if (w < wid) e1 += wt[0][w], e2 += wt[1][w];
    t1 += wt[0][w];
    t2 += wt[1][w];
  }
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (c + j < W) {
      X.colsum[(long long)seg * W + c + j] = e1 + cu[j];
      X.colsum[((long long)X.nseg + seg) * W + c + j] = e2 + cv[j];
    }
  if (threadIdx.x == 0 && totals) {
    X.tiletot[(long long)seg * X.nchunk + k] = t1;
    X.tiletot[((long long)X.nseg + seg) * X.nchunk + k] = t2;
  }
}

// The q integrals of a batch of jobs: block -> job through the batched stage
// offsets, then the job's tile or column block.
__device__ __forceinline__ IntTask job_task(const Job &J) {
  return int_task(J.in.W, J.in.H, J.nseg, J.seg_rows, J.segtot);
}

__global__ void __launch_bounds__(kFS, 3) k_int_stats(const Job *__restrict__ jobs, int njobs) {
  __shared__ long long rowp[kRowGroup][2][kFS / 32];
  __shared__ long long wt[2][kFS / 32];
  const Job &J = jobs[find_job(jobs, njobs, kStRows, blockIdx.x)];
  const IntTask X = job_task(J);
  const int lb = blockIdx.x - J.b0[kStRows];
  const QSource src{J.q, J.in.W};
  int_stats4_tile(X, src, lb / X.nchunk, lb % X.nchunk, rowp, wt);
}

__global__ void __launch_bounds__(kMidCols * kMidGroups) k_int_mid(const Job *__restrict__ jobs, int njobs) {
  __shared__ long long part[2][kMidGroups][kMidCols];
  __shared__ long long leftT[2][kMidBatch];
  const Job &J = jobs[find_job(jobs, njobs, kStCols, blockIdx.x)];
  int_mid_cols(job_task(J), (blockIdx.x - J.b0[kStCols]) * kMidCols, part, leftT);
}

__global__ void __launch_bounds__(kINT, 4) k_int_write(const Job *__restrict__ jobs, int njobs) {
  __shared__ int32_t tile[kIC / 8 * 9];
  __shared__ long long out1[kIC / 8 * 9], out2[kIC / 8 * 9];
  __shared__ long long wt[2][kINT / 32];
  const Job &J = jobs[find_job(jobs, njobs, kStRows, blockIdx.x)];
  const IntTask X = job_task(J);
  const int lb = blockIdx.x - J.b0[kStRows];
  const QSource src{J.q, J.in.W};
  if (J.s_pair)
    int_write_tile<QSource, long long, true>(X, src, J.s1, J.s2, lb / X.nchunk, lb % X.nchunk, tile, out1, out2, wt);
  else
    int_write_tile(X, src, J.s1, J.s2, lb / X.nchunk, lb % X.nchunk, tile, out1, out2, wt);
}

// The backward's fixed-point integral planes of a batch of images: block ->
// image through FixJob::b0_tile / b0_col, then (pair p, tile) or (pair p,
// column block). Pair p of an image: planes u_p and v_p (each W x H), scaled
// by 2^fix_shift(amax[p], nmax[p]) and 2^fix_shift(amax[kMaxFields + p],
// nmax[p]) (the scales the backward converts back with), interleaved into
// the p-th pair plane of dst (two int64 per position); scratch per pair.
__device__ __forceinline__ int find_fix(const FixJob *jobs, int n, bool tiles, int blk) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((tiles ? jobs[mid].b0_tile : jobs[mid].b0_col) <= blk) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ IntTask fix_task(const FixJob &F, int p) {
  return int_task(F.W, F.H, F.nseg, F.seg_rows, F.scratch + (long long)p * F.scratch_stride);
}

__device__ __forceinline__ FixSource fix_source(const FixJob &F, int p) {
  const long long N = (long long)F.W * F.H;
  return fix_source_of(F.u + p * N, F.v + p * N, F.W, fix_shift(__ldg(F.amax + p), F.nmax[p]),
                       fix_shift(__ldg(F.amax + kMaxFields + p), F.nmax[p]));
}

__global__ void __launch_bounds__(kFS, 3) k_fix_stats(const FixJob *__restrict__ jobs, int n) {
  __shared__ long long rowp[kRowGroup][2][kFS / 32];
  __shared__ long long wt[2][kFS / 32];
  const FixJob &F = jobs[find_fix(jobs, n, true, blockIdx.x)];
  const int per = F.nseg * ((F.W + kIC - 1) / kIC), lb = blockIdx.x - F.b0_tile;
  const int p = lb / per, t = lb - p * per;
  const IntTask X = fix_task(F, p);
  int_stats4_tile(X, fix_source(F, p), t / X.nchunk, t % X.nchunk, rowp, wt);
}

__global__ void __launch_bounds__(kMidCols * kMidGroups) k_fix_mid(const FixJob *__restrict__ jobs, int n) {
  __shared__ long long part[2][kMidGroups][kMidCols];
  __shared__ long long leftT[2][kMidBatch];
  const FixJob &F = jobs[find_fix(jobs, n, false, blockIdx.x)];
  const int per = (F.W + kMidCols - 1) / kMidCols, lb = blockIdx.x - F.b0_col;
  const int p = lb / per;
  int_mid_cols(fix_task(F, p), (lb - p * per) * kMidCols, part, leftT);
}

__global__ void __launch_bounds__(kINT, 4) k_fix_write(const FixJob *__restrict__ jobs, int n) {
  __shared__ float2 tile[kIC / 8 * 9];
  __shared__ long long out1[kIC / 8 * 9], out2[kIC / 8 * 9];
  __shared__ long long wt[2][kINT / 32];
  const FixJob &F = jobs[find_fix(jobs, n, true, blockIdx.x)];
  const int per = F.nseg * ((F.W + kIC - 1) / kIC), lb = blockIdx.x - F.b0_tile;
  const int p = lb / per, t = lb - p * per;
  const IntTask X = fix_task(F, p);
  const long long plane = ((long long)F.W + 1) * ((long long)F.H + 1);
  long long *d = reinterpret_cast<long long *>(F.dst) + 2 * p * plane;
  int_write_tile<FixSource, long long, true>(X, fix_source(F, p), d, d + 1, t / X.nchunk, t % X.nchunk, tile,
                                             out1, out2, wt);
}

// Integral histogram planes (uint32, modulo 2^32) of a bin map over the same
// tiles: pair p = pair0 + blockIdx.y holds planes 2p and 2p + 1 of `planes`
// (thresholds k_begin + 2p and + 1; the second is skipped past n_planes),
// scratch per grid row.
struct HistPairs {
  const uint8_t *bins;
  uint32_t *planes;
  long long *scratch;
  size_t scratch_stride;
  int W, H, nseg, seg_rows, k_begin, n_planes, eq, pair0;
};

__device__ __forceinline__ IntTask hist_task(const HistPairs &Q) {
  return int_task(Q.W, Q.H, Q.nseg, Q.seg_rows, Q.scratch + (long long)blockIdx.y * Q.scratch_stride);
}

__device__ __forceinline__ BinSource hist_source(const HistPairs &Q) {
  return BinSource{Q.bins, Q.W, Q.k_begin + 2 * (Q.pair0 + (int)blockIdx.y), Q.eq};
}

__global__ void __launch_bounds__(kINT, 4) k_hist_stats(HistPairs Q) {
  __shared__ StatsSmem sm;
  const IntTask X = hist_task(Q);
  int_stats_tile(X, hist_source(Q), blockIdx.x / X.nchunk, blockIdx.x % X.nchunk, sm);
}

__global__ void __launch_bounds__(kMidCols * kMidGroups) k_hist_mid(HistPairs Q) {
  __shared__ long long part[2][kMidGroups][kMidCols];
  __shared__ long long leftT[2][kMidBatch];
  int_mid_cols(hist_task(Q), blockIdx.x * kMidCols, part, leftT);
}

__global__ void __launch_bounds__(kINT, 4) k_hist_write(HistPairs Q) {
  __shared__ int tile[kIC / 8 * 9];
  __shared__ long long out1[kIC / 8 * 9], out2[kIC / 8 * 9];
  __shared__ long long wt[2][kINT / 32];
  const IntTask X = hist_task(Q);
  const long long plane = ((long long)Q.W + 1) * ((long long)Q.H + 1);
  const int p = Q.pair0 + (int)blockIdx.y;
  uint32_t *a = Q.planes + 2LL * p * plane;
  uint32_t *b = 2 * p + 1 < Q.n_planes ? a + plane : nullptr;
  int_write_tile(X, hist_source(Q), a, b, blockIdx.x / X.nchunk, blockIdx.x % X.nchunk, tile, out1, out2, wt);
}

}  // namespace

void integral_layout(int W, int H, size_t max_scratch_elems, int &nseg, int &seg_rows) {
  // the shortest segments (most tiles) whose scratch fits, at least kIR rows
  seg_rows = kIR;
  for (;;) {
    nseg = (H + seg_rows - 1) / seg_rows;
    if (integral_scratch_elems(W, H, nseg) <= max_scratch_elems || seg_rows >= H) return;
    seg_rows = std::min(H, seg_rows * 2);
  }
}

size_t integral_scratch_elems(int W, int H, int nseg) {
  const long long nchunk = (W + kIC - 1) / kIC;
  return (size_t)(2LL * nseg * W + 2LL * H * nchunk + 2LL * nseg * nchunk);
}

int integral_tile_blocks(int W, int nseg) { return nseg * ((W + kIC - 1) / kIC); }

int integral_col_blocks(int W) { return (W + kMidCols - 1) / kMidCols; }

// Row segments of an image's fixed-point pairs in a batch whose pairs, over
// all images, number `batch_pairs`: short enough for about 2048 tiles over
// the batch, 4 to kIR rows.
void fix_layout(int W, int H, long long batch_pairs, int &nseg, int &seg_rows) {
  const long long tiles_per_row = batch_pairs * ((W + kIC - 1) / kIC);
  seg_rows = (int)std::min<long long>(kIR, std::max<long long>(4, H * tiles_per_row / 2048));
  nseg = (H + seg_rows - 1) / seg_rows;
}

size_t fix_integral_scratch_elems(int W, int H, int pairs, int nseg) {
  return (size_t)pairs * integral_scratch_elems(W, H, nseg);
}

int fix_tile_blocks(int W, int nseg, int pairs) { return pairs * integral_tile_blocks(W, nseg); }

int fix_col_blocks(int W, int pairs) { return pairs * integral_col_blocks(W); }

int launch_fix_integrals(const FixJob *jobs, int n, int tile_blocks, int col_blocks, cudaStream_t s) {
  k_fix_stats<<<tile_blocks, kFS, 0, s>>>(jobs, n);
  k_fix_mid<<<col_blocks, kMidCols * kMidGroups, 0, s>>>(jobs, n);
  k_fix_write<<<tile_blocks, kINT, 0, s>>>(jobs, n);
  return 3;
}

int launch_integral_jobs(const Job *jobs, int njobs, int tile_blocks, int col_blocks, cudaStream_t s) {
  k_int_stats<<<tile_blocks, kFS, 0, s>>>(jobs, njobs);
  k_int_mid<<<col_blocks, kMidCols * kMidGroups, 0, s>>>(jobs, njobs);
  k_int_write<<<tile_blocks, kINT, 0, s>>>(jobs, njobs);
  return 3;
}

constexpr int kHistPairs = 8;  // plane pairs per launch of the histogram tiles

size_t hist_scratch_bytes(int W, int H, int planes) {
  int nseg, seg_rows;
  integral_layout(W, H, SIZE_MAX, nseg, seg_rows);
  const int pairs = std::min((planes + 1) / 2, kHistPairs);
  return 8 * (size_t)std::max(pairs, 1) * integral_scratch_elems(W, H, nseg);
}

int launch_integral_histogram(const uint8_t *bins, int W, int H, int n_bins, bool cumulative,
                              uint32_t *planes, void *scratch, cudaStream_t s) {
  const int k_begin = cumulative ? 1 : 0;
  const int n_planes = cumulative ? n_bins - 1 : n_bins;
  if (n_planes <= 0) return 0;
  HistPairs Q{};
  Q.bins = bins;
  Q.planes = planes;
  Q.scratch = static_cast<long long *>(scratch);
  Q.W = W;
  Q.H = H;
  integral_layout(W, H, SIZE_MAX, Q.nseg, Q.seg_rows);
  Q.scratch_stride = integral_scratch_elems(W, H, Q.nseg);
  Q.k_begin = k_begin;
  Q.n_planes = n_planes;
  Q.eq = cumulative ? 0 : 1;
  const int pairs = (n_planes + 1) / 2;
  int n = 0;
  for (Q.pair0 = 0; Q.pair0 < pairs; Q.pair0 += kHistPairs) {  // groups share the scratch in turn
    const int g = std::min(kHistPairs, pairs - Q.pair0);
    const dim3 tiles(integral_tile_blocks(W, Q.nseg), g), cols(integral_col_blocks(W), g);
    k_hist_stats<<<tiles, kINT, 0, s>>>(Q);
    k_hist_mid<<<cols, kMidCols * kMidGroups, 0, s>>>(Q);
    k_hist_write<<<tiles, kINT, 0, s>>>(Q);
    n += 3;
  }
  return n;
}

}  // namespace tmk
