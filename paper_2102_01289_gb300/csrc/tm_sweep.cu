// tm_sweep.cu -- fused integral-histogram sweep: the Eq. 1 numerator of every
// field at every pixel, without materialising the integral histogram.
//
// For a threshold k, let C_k(u, v) be the integral histogram in cumulative
// form (Eq. 7-8 summed over the bins below k): the number of pixels (u', v')
// with u0 <= u' <= u, v0 < v' <= v and b(u', v') < k, over a segment-local
// origin (u0 - 1, v0). A pixel p = (x, y) with threshold k = b(p) (b(p) + 1
// under TM_FLAG_CDF_INCLUSIVE) needs, per field with half-sizes (rx, ry),
// the box sum of Eq. 9 over its clipped window [xl, xr] x [yt, yb]:
//     cnt = E(yb) - E(yt - 1),   E(v) = C_k(xr, v) - C_k(xl - 1, v).
// Each image is cut into strips of 512 (or 256) columns and bands of TY rows;
// K consecutive bands of a strip form a group. A CTA sweeps a segment: it
// starts on a band and runs on into the group's next bands while it claims
// them first. The sweep covers the strip's columns widened by the largest
// half-width on both sides, and only the segment's own rows, from an origin
// just above its first row. A window reaching above or below the segment
// takes its rows there from the other segments: each segment adds
// E(last row of the window in it) - E(row above the first) to the pixel's
// count, with 32-bit reductions into count planes cleared beforehand. After
// row v is taken in, windows opening at v + 1 subtract E(v) and windows
// closing on v add E(v); at the segment's last row every window reaching it
// and closing on it or below adds E(last row).
//
// The swept columns are cut into 32-column chunks aligned to the image, one
// warp lane per chunk. For every threshold k of the segment the
// shared-memory state is
//     C_k(u) = PT_k(c) + B_k(u) + (o + 1) m_k(c) + M_k (u - u0 + 1)
//                                                   (c = chunk of u, o = u - 32 c)
// where, over the rows swept so far,
//     m_k(c)  counts the rows in which all of chunk c lies below k,
//     B_k(u)  sums the in-chunk prefix counts #{u' in c, u' <= u : b < k} of
//             the rows in which chunk c holds bins on both sides of k,
//     PT_k(c) sums the counts below k of all chunks left of c, and
//     M_k     counts the rows whose every bin lies below k (applied lazily).
// So a row costs per-column work only where a bin edge crosses a chunk (one
// ballot and popcount per such threshold), plus one prefix over the chunks
// per threshold inside the row's bin range. PT and m share one word
// (21 + 11 bits: at most 2047 swept rows and 32 chunks), B fits 16 bits (32
// columns x 2047 rows), and every E is exact below 2^21.
//
// Per row the CTA runs two phases separated by barriers:
//   1. the corner events of the previous row (reading the state) and the
//      bins of this row into shared memory;
//   2. the state update of this row (B of the mixed chunks, PT and m), a warp
//      per threshold; the chunks' bin ranges come from the per-row group
//      summary of the bin pass.
// A segment whose own pixels use more thresholds than the shared memory
// holds is swept once per group of them (and then does not run on).
#include <algorithm>

#include "tm_kernels.cuh"

namespace tmk {
namespace {

constexpr int kMaxChunks = 32;      // 32-column chunks of a swept row
constexpr int kMaxRows = 2047;      // swept rows of a tile
constexpr unsigned kPTMask = (1u << 21) - 1;
constexpr int kPStride = 33;        // words per threshold row of PT | m << 21
// Bands per group: a segment starts on a group's first band and runs on into
// its next bands while no other CTA has taken them, so CTAs that finish early
// take the last bands of slow segments. Measured at 12 MP on 256-column strips
// (one wave of 304 groups) with 1, 3, 4, 6, 8 and 12 bands per group: the sweep
// took 0.480, 0.486, 0.469, 0.463, 0.453 and 0.466 ms (uniform tiles: 0.467).
// On 512-column strips (152 groups) the forward took 0.762, 0.749, 0.755 and
// 0.791 ms with 4, 6, 8 and 12: the integral images beside the sweep, which
// start as its CTAs run dry, end first with 6.
constexpr int kBandsPerGroup = 6;

// A strip has TX own columns (256 or 512) and its CTA 2 TX threads: threads
// t and t + TX take the top and bottom events of column t.
template <int TX>
struct Shape {
  static constexpr int NT = 2 * TX, Warps = NT / 32, ChunksPerWarp = kMaxChunks / Warps;
  // 256: two 512-thread CTAs per SM; 512: one 1024-thread CTA
  static constexpr int MinBlocks = TX == 256 ? 2 : 1;
  static_assert(ChunksPerWarp * Warps == kMaxChunks, "every chunk has a warp");
};

// The sweep's dynamic shared memory (named at file scope so that every access
// compiles to a shared-memory load or store).
extern __shared__ __align__(16) unsigned char g_smem[];

// Shared-memory layout of a CTA (byte offsets from the dynamic array):
//   PT     kcap x kPStride words   PT_k(c) | m_k(c) << 21
//   M      kcap words              rows whose bins all lie below k (lazy: such
//                                  a row adds u - u0 + 1 at every column u)
//   red    64 words                reductions
//   rowb   32 x 32 bytes           bins of the current swept row, by chunk
//   B      kcap x bstride uint16   in-chunk prefix counts of mixed rows
struct Lay {
  unsigned PT, M, red, rowb, B;
};

__host__ __device__ __forceinline__ Lay layout(int kcap) {
  Lay l;
  l.PT = 0;
  l.M = l.PT + (unsigned)kcap * kPStride * 4;
  l.red = l.M + (unsigned)kcap * 4;
  l.rowb = l.red + 64 * 4;
  l.B = l.rowb + kMaxChunks * 32;
  return l;
}

// E = C_k(jr) - C_k(jl) from the state of threshold row kk (jl = -1: the
// origin column, where C = 0). With M_k rows lying wholly below k, C_k(j)
// gains M_k (j + 1), so the pair gains M_k (jr - jl).
__device__ __forceinline__ unsigned pair_value(const unsigned *PT, const unsigned *M, const uint16_t *B, int bstride,
                                               int kk, int jr, int jl) {
  const unsigned *pr = PT + kk * kPStride;
  const uint16_t *br = B + kk * bstride;
  const unsigned wr = pr[jr >> 5];
  unsigned e = (wr & kPTMask) + (unsigned)br[jr] + (unsigned)((jr & 31) + 1) * (wr >> 21) +
               M[kk] * (unsigned)(jr - jl);
  if (jl >= 0) {
    const unsigned wl = pr[jl >> 5];
    e -= (wl & kPTMask) + (unsigned)br[jl] + (unsigned)((jl & 31) + 1) * (wl >> 21);
  }
  return e;
}

// One segment: band `band` of strip `strip` of job J, extended over the next
// bands of its group for as long as the CTA claims them first (a claim is
// one atomic exchange; a band taken by another CTA ends the segment). The
// sweep starts at the segment's first row (origin row Y0 - 1, where C = 0):
// a window reaching above or below the segment takes its rows there from
// the other segments, each adding E(last row of the window in the segment) -
// E(row above the first) to the pixel's count.
// kIncl: TM_FLAG_CDF_INCLUSIVE (the threshold is b + 1 instead of b).
template <int NF, int TX, bool kIncl>
__device__ __forceinline__ void sweep_tile(const DevParams &P, const Job &J, int strip, int band) {
  __shared__ int ext_sh, next_sh, ext_end_sh;  // the claim state lives in shared memory, off the registers
  unsigned char *const smem = g_smem;
  const SweepPlan &S = J.plan;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int W = S.W, H = S.H;
  constexpr int kNT = Shape<TX>::NT, kWarps = Shape<TX>::Warps, kChunksPerWarp = Shape<TX>::ChunksPerWarp;
  const int X0 = strip * TX, X1 = min(X0 + TX, W);
  const int Y0 = band * S.TY;
  int Y1 = min(Y0 + S.TY, H);
  // the group's bands from this one on; the rows the segment can reach
  const int gend = min((band / S.K + 1) * S.K, S.tiles_y);
  const int Yg = min(gend * S.TY, H);
  const int cL = max(X0 - S.Rx - 1, -1);
  const int cR = min(X1 - 1 + S.Rx, W - 1);
  const int g0 = (cL + 1) >> 5;
  const int nch = (cR >> 5) - g0 + 1;
  const int rL = Y0 - 1;  // origin row
  const int n = P.n_bins;
  constexpr int incl = kIncl ? 1 : 0;
  const int kcap = S.kcap, bstride = S.bstride;
  const Lay L = layout(kcap);
  unsigned *const sPT = reinterpret_cast<unsigned *>(smem + L.PT);
  unsigned *const sM = reinterpret_cast<unsigned *>(smem + L.M);
  int *const sred = reinterpret_cast<int *>(smem + L.red);
  uint8_t *const srow = smem + L.rowb;
  uint16_t *const sB = reinterpret_cast<uint16_t *>(smem + L.B);
  const uint8_t *__restrict__ bins = J.bins;
  const uint16_t *__restrict__ grp = J.grp;
  const int G = (W + 31) >> 5;
  // the count planes' bases, in shared memory (read per event, off the registers)
  __shared__ unsigned *pl[kMaxFields];
  if (tid < NF) pl[tid] = reinterpret_cast<unsigned *>(J.cnt + J.cnt_off[tid]);

  // ---- bin range of the pixels whose windows meet the segment (its own
  // columns, the rows the largest half-height reaches from the rows it can
  // extend over), from the per-row group summary of the bin pass ----
  {
    const int ya = max(Y0 - S.Ry, 0), yb = min(Yg + S.Ry, H);
    const int gx0 = X0 >> 5, ngx = ((X1 - 1) >> 5) - gx0 + 1;
    int bmin = 255, bmax = 0;
    for (int i = tid; i < (yb - ya) * ngx; i += kNT) {
      const int yy = i / ngx;
      const unsigned v = grp[(long long)(ya + yy) * G + gx0 + (i - yy * ngx)];
      bmin = min(bmin, (int)(v & 0xffu));
      bmax = max(bmax, (int)(v >> 8));
    }
    bmin = __reduce_min_sync(0xffffffffu, bmin);
    bmax = __reduce_max_sync(0xffffffffu, bmax);
    if (lane == 0) {
      sred[wid] = bmin;
      sred[32 + wid] = bmax;
    }
  }
  __syncthreads();
  int bmin = 255, bmax = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    bmin = min(bmin, sred[w]);
    bmax = max(bmax, sred[32 + w]);
  }
  const int klo = max(1, bmin + incl), khi = min(n - 1, bmax + incl);
  const int nK = max(0, khi - klo + 1);
  const int npass = max(1, (nK + kcap - 1) / kcap);
  // one pass: the segment may run on into its group's bands before gend as
  // it reaches them. Several passes each sweep the same rows, so the segment
  // claims the group's next bands (up to one taken by another CTA) now.
  if (tid == 0) {
    int nx = band + 1;
    if (npass > 1)
      while (nx < gend && atomicExch(J.claim + nx * S.tiles_x + strip, 1) == 0) ++nx;
    ext_sh = nx;
    next_sh = nx;
    ext_end_sh = npass == 1 ? gend : 0;
  }
  __syncthreads();
  Y1 = min(ext_sh * S.TY, H);

  // ---- the thread's event column: windows opening below a swept row
  // (tid < 256: subtract E) or closing on it (add E) ----
  const int xo = tid & (TX - 1);
  const bool is_close = tid >= TX;
  const int x = X0 + xo;
  const bool col_ok = x < X1;
  // per field: half-height, corner columns (relative to 32 g0; jl = -1 is the
  // origin), and the offset of the event pixel's row from the swept row
  int ry[NF], jr[NF], jl[NF], eoff[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    ry[f] = min(P.ry[f], H - 1);
    const int rx = min(P.rx[f], W - 1);
    jr[f] = min(x + rx, W - 1) - 32 * g0;
    jl[f] = max(x - rx, 0) - 1 - 32 * g0;
    eoff[f] = is_close ? -ry[f] : ry[f] + 1;
  }
  const unsigned lt = (1u << lane) - 1u, le = lt | (1u << lane);

  for (int pass = 0; pass < npass; ++pass) {
    const int kp0 = klo + pass * kcap;
    const int nKp = max(0, min(kcap, khi - kp0 + 1));
    const bool specials = pass == 0;  // thresholds 0 and n need no state: taken in the first pass
    __syncthreads();  // the previous pass (or tile) has finished reading the state
    for (int i = tid; i < nKp * kPStride; i += kNT) sPT[i] = 0u;
    for (int i = tid; i < nKp; i += kNT) sM[i] = 0u;
    {
      unsigned *b32 = reinterpret_cast<unsigned *>(sB);
      const int words = (nKp * bstride) >> 1;
      for (int i = tid; i < words; i += kNT) b32[i] = 0u;
    }
    // E at swept row v for threshold k = b + incl (corner columns cjr, cjl);
    // false when there is nothing to add: the threshold belongs to another
    // pass, or it is 0 (nothing lies below it)
    auto event_value = [&](int b, int cjr, int cjl, int v, unsigned &E) -> bool {
      const int k = b + incl, kk = k - kp0;
      if ((unsigned)kk < (unsigned)nKp) {
        E = pair_value(sPT, sM, sB, bstride, kk, cjr, cjl);
        return true;
      }
      if (!kIncl) return false;  // k <= n - 1 here: only k = 0 is left, or another pass
      // threshold n (the whole window) in the first pass
      E = (unsigned)(cjr - cjl) * (unsigned)(v - rL);
      return specials && k >= n;
    };
    // bins of a swept row, a warp per chunk (wid, wid + 16; 256 marks columns
    // past the image), and the chunks' bin ranges (lanes = chunks) from the
    // group summary of the bin pass; both loaded one row ahead
    int bcur[kChunksPerWarp], bnxt[kChunksPerWarp];
    unsigned gcur, gnxt = 0xffu;
#pragma unroll
    for (int q = 0; q < kChunksPerWarp; ++q) {
      const int c = wid + q * kWarps, col = 32 * (g0 + c) + lane;
      bcur[q] = (c < nch && col < W) ? (int)__ldg(bins + (long long)Y0 * W + col) : 256;
      bnxt[q] = 256;
    }
    gcur = lane < nch ? (unsigned)__ldg(grp + (long long)Y0 * G + g0 + lane) : 0xffu;
    // events of the pending row: act bit f = the thread's event of field f is
    // live; ebin = the bin of its pixel
    unsigned act = 0u;
    int ebin[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) ebin[f] = 0;
    for (int v = Y0; v <= Y1; ++v) {
      // at the current band's last row, claim the group's next band: if it
      // is ours, the segment runs on and this row takes regular events
      if (v == Y1 - 1) {  // block-uniform
        if (tid == 0) {
          const int nx = next_sh;
          ext_sh = nx < ext_end_sh && atomicExch(J.claim + nx * S.tiles_x + strip, 1) == 0;
          next_sh = nx + 1;
        }
        __syncthreads();
        if (ext_sh) Y1 = min(Y1 + J.plan.TY, H);
      }
      // ---- phase 1: events of row v - 1; bins of row v into shared memory ----
      const bool last = v >= Y1;
      // rows Y0 .. Y1 - 2 take the windows opening below them and those
      // closing on them; the band's last row is taken after the loop
      unsigned nact = 0u;
      int nbin[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const int y = v + eoff[f];
        const bool ok = v < Y1 - 1 && col_ok && (unsigned)y < (unsigned)H;
        nbin[f] = ok ? (int)__ldg(bins + (long long)y * W + x) : 0;
        nact |= (ok ? 1u : 0u) << f;
      }
      if (!last) {
#pragma unroll
        for (int q = 0; q < kChunksPerWarp; ++q) {
          const int c = wid + q * kWarps, col = 32 * (g0 + c) + lane;
          bnxt[q] = (c < nch && col < W && v + 1 < Y1) ? (int)__ldg(bins + (long long)(v + 1) * W + col) : 256;
        }
        gnxt = (lane < nch && v + 1 < Y1) ? (unsigned)__ldg(grp + (long long)(v + 1) * G + g0 + lane) : 0xffu;
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) {  // events of row v - 1
        if (!((act >> f) & 1u)) continue;
        unsigned E;
        if (event_value(ebin[f], jr[f], jl[f], v - 1, E))
          atomicAdd(pl[f] + ((long long)(v - 1 + eoff[f]) * W + x), is_close ? E : 0u - E);
      }
      if (last) break;
#pragma unroll
      for (int q = 0; q < kChunksPerWarp; ++q) {
        const int c = wid + q * kWarps;
        if (c < nch) srow[32 * c + lane] = (uint8_t)min(bcur[q], 255);
      }
      __syncthreads();
      // ---- phase 2: state update of row v, a warp per threshold (lanes =
      // chunks) ----
      act = nact;
#pragma unroll
      for (int f = 0; f < NF; ++f) ebin[f] = nbin[f];
      {
        const bool lc = lane < nch;
        const int cmin = lc ? (int)(gcur & 0xffu) : 256, cmax = lc ? (int)(gcur >> 8) : -1;
        const int rmin = __reduce_min_sync(0xffffffffu, cmin);
        const int rmax = __reduce_max_sync(0xffffffffu, cmax);
        // thresholds above every bin of the row: the lazy whole-row count
        if (wid == kWarps - 1)
          for (int kk = max(0, rmax + 1 - kp0) + lane; kk < nKp; kk += 32) sM[kk] += 1u;
        // thresholds inside the row's range: prefix over the chunks
        const int kk_hi = min(nKp - 1, rmax - kp0);
        for (int kk = max(0, rmin + 1 - kp0) + wid; kk <= kk_hi; kk += kWarps) {
          const int k = kp0 + kk;
          const bool below = lc && cmax < k;  // the chunk lies wholly below k
          const unsigned bm = __ballot_sync(0xffffffffu, below);
          unsigned mm = __ballot_sync(0xffffffffu, lc && cmin < k && k <= cmax);  // bins on both sides
          unsigned carry = 32u * (unsigned)__popc(bm & lt);
          while (mm) {
            const int c = __ffs(mm) - 1;
            mm &= mm - 1;
            // lanes = the columns of mixed chunk c: in-chunk prefix counts
            const int b = (32 * (g0 + c) + lane < W) ? (int)srow[32 * c + lane] : 256;
            const unsigned mask = __ballot_sync(0xffffffffu, b < k);
            uint16_t *bp = sB + kk * bstride + 32 * c + lane;
            *bp = (uint16_t)(*bp + __popc(mask & le));
            if (lane > c) carry += (unsigned)__popc(mask);
          }
          if (lc) sPT[kk * kPStride + lane] += carry + (below ? (1u << 21) : 0u);
        }
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < kChunksPerWarp; ++q) bcur[q] = bnxt[q];
      gcur = gnxt;
    }
    // the band's last row: every window that reaches it and closes on it or
    // below it adds E(Y1 - 1). Each thread walks its event column (the corner
    // columns are the ones its events use) over every other row, four rows at
    // a time
    const int vlast = Y1 - 1, par = is_close ? 1 : 0;
    if (col_ok) {
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const int ybeg = max(vlast - ry[f], 0), yend = min(vlast + ry[f], H - 1);
        for (int y0 = ybeg + par; y0 <= yend; y0 += 8) {
          int bb[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int y = y0 + 2 * u;
            bb[u] = y <= yend ? (int)__ldg(bins + (long long)y * W + x) : -1;
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (bb[u] < 0) continue;
            unsigned E;
            if (event_value(bb[u], jr[f], jl[f], vlast, E)) atomicAdd(pl[f] + ((long long)(y0 + 2 * u) * W + x), E);
          }
        }
      }
    }
  }
}

// The persistent sweep: CTAs pop queue slots until the queue runs dry. The
// first phase of the queue holds every job's group starts (band K g of each
// strip, jobs in their slot order), the second the groups' other bands, last
// bands first. A slot's band is swept unless a CTA running on from the band
// before has claimed it.
__device__ __forceinline__ void second_phase_band(const SweepPlan &S, int local, int &strip, int &band) {
  // bands with band % K == r, for r = K - 1 down to 1, each residue row-major
  for (int r = S.K - 1; r >= 1; --r) {
    const int nb = r < S.tiles_y ? (S.tiles_y - r + S.K - 1) / S.K : 0;
    const int cnt = nb * S.tiles_x;
    if (local < cnt) {
      strip = local % S.tiles_x;
      band = (local / S.tiles_x) * S.K + r;
      return;
    }
    local -= cnt;
  }
  strip = band = -1;
}

template <int NF, int TX, bool kIncl>
__global__ void __launch_bounds__(Shape<TX>::NT, Shape<TX>::MinBlocks)
    k_sweep(DevParams P, const Job *__restrict__ jobs, int njobs, int nitems, int *queue) {
  __shared__ int item_sh, job_sh, strip_sh, band_sh, won_sh;
  for (;;) {
    if (threadIdx.x == 0) {
      item_sh = atomicAdd(queue, 1);
      job_sh = -1;
    }
    __syncthreads();
    const int it = item_sh;
    if (it >= nitems) break;
    for (int j = threadIdx.x; j < njobs; j += Shape<TX>::NT)
      if ((jobs[j].itemA0 <= it && it < jobs[j].itemA0 + jobs[j].nitemA) ||
          (jobs[j].itemB0 <= it && it < jobs[j].itemB0 + jobs[j].nitemB))
        job_sh = j;
    __syncthreads();
    const int jb = job_sh;
    if (jb >= 0 && threadIdx.x == 0) {
      const Job &J = jobs[jb];
      int strip, band;
      if (it < J.itemA0 + J.nitemA && it >= J.itemA0) {
        const int local = it - J.itemA0;
        strip = local % J.plan.tiles_x;
        band = (local / J.plan.tiles_x) * J.plan.K;
      } else {
        second_phase_band(J.plan, it - J.itemB0, strip, band);
      }
      strip_sh = strip;
      band_sh = band;
      won_sh = band >= 0 && atomicExch(J.claim + band * J.plan.tiles_x + strip, 1) == 0;
    }
    __syncthreads();
    if (jb >= 0 && won_sh) sweep_tile<NF, TX, kIncl>(P, jobs[jb], strip_sh, band_sh);
    __syncthreads();  // the shared slot fields are rewritten for the next item
  }
}

size_t smem_for(int kcap, int bstride) { return layout(kcap).B + (size_t)kcap * bstride * 2; }

}  // namespace

bool plan_sweep(const DevParams &P, int W, int H, int segments, size_t smem_limit, int width, SweepPlan &S) {
  if (width != 256 && width != 512) return false;
  SweepPlan s{};
  s.W = W;
  s.H = H;
  int Rx = 0, Ry = 0;
  for (int f = 0; f < P.n_fields; ++f) {
    Rx = max(Rx, min(P.rx[f], W - 1));
    Ry = max(Ry, min(P.ry[f], H - 1));
  }
  s.Rx = Rx;
  s.Ry = Ry;
  s.TX = width;
  s.tiles_x = (W + width - 1) / width;
  // widest swept row: a strip of `width` columns widened by Rx + 1 on the left and
  // Rx on the right, rounded out to 32-column chunks
  int nch_max = 0;
  for (int strip = 0; strip < s.tiles_x; ++strip) {
    const int X0 = strip * width, X1 = min(X0 + width, W);
    const int cL = max(X0 - Rx - 1, -1), cR = min(X1 - 1 + Rx, W - 1);
    nch_max = max(nch_max, (cR >> 5) - ((cL + 1) >> 5) + 1);
  }
  if (nch_max > kMaxChunks) return false;
  s.nch_max = nch_max;
  s.bstride = 32 * nch_max + 2;  // an odd number of words per threshold row
  const int nthr = max(1, P.n_bins - 1);
  int kcap = nthr;
  while (kcap > 1 && smem_for(kcap, s.bstride) > smem_limit) --kcap;
  if (smem_for(kcap, s.bstride) > smem_limit) return false;
  s.kcap = kcap;
  s.smem = smem_for(kcap, s.bstride);
  // bands: kBandsPerGroup per segment of the target, each group of them at
  // most 2047 rows (a segment sweeps its own rows only)
  s.K = kBandsPerGroup;
  int bands = max(1, (s.K * segments + s.tiles_x - 1) / s.tiles_x);
  bands = min(bands, H);
  int TY = (H + bands - 1) / bands;
  if (TY > kMaxRows / s.K) TY = kMaxRows / s.K;
  s.TY = TY;
  s.tiles_y = (H + TY - 1) / TY;
  // count planes: uint32, the bands' contributions added into them
  s.cnt_wide = (1 << P.n_fields) - 1;
  S = s;
  return true;
}

size_t sweep_count_bytes(const DevParams &P, const SweepPlan &S, long long *off) {
  const size_t N = (size_t)S.W * S.H;
  size_t o = 0;
  for (int f = 0; f < kMaxFields; ++f) {
    if (off) off[f] = (long long)o;
    if (f < P.n_fields) o += N * (((S.cnt_wide >> f) & 1) ? 4 : 2);
    o = (o + 255) & ~(size_t)255;
  }
  return o;
}

template <int NF, int TX>
static int launch_nf(const DevParams &P, const Job *jobs, int njobs, int nitems, int *queue, size_t smem,
                     int ctas, cudaStream_t s) {
  const bool incl = (P.flags & kFlagCdfIncl) != 0;
  auto *k = incl ? k_sweep<NF, TX, true> : k_sweep<NF, TX, false>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -1;
  k<<<ctas, Shape<TX>::NT, smem, s>>>(P, jobs, njobs, nitems, queue);
  return 1;
}

template <int TX>
static int ctas_per_sm(int n_fields, size_t smem) {
  int per = 0;
  cudaError_t e;
  switch (n_fields) {
#define TM_OCC(nf)                                                                                          \
  case nf:                                                                                                  \
    e = cudaFuncSetAttribute(k_sweep<nf, TX, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (e == cudaSuccess)                                                                                   \
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep<nf, TX, false>, Shape<TX>::NT, smem); \
    break;
    TM_OCC(1) TM_OCC(2) TM_OCC(3) TM_OCC(4) TM_OCC(5) TM_OCC(6) TM_OCC(7) TM_OCC(8)
#undef TM_OCC
    default: return 0;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per;
}

template <int TX>
static int launch_width(const DevParams &P, const Job *jobs, int njobs, int nitems, int *queue, size_t smem,
                        int ctas, cudaStream_t s) {
  switch (P.n_fields) {
    case 1: return launch_nf<1, TX>(P, jobs, njobs, nitems, queue, smem, ctas, s);
    case 2: return launch_nf<2, TX>(P, jobs, njobs, nitems, queue, smem, ctas, s);
    case 3: return launch_nf<3, TX>(P, jobs, njobs, nitems, queue, smem, ctas, s);
    case 4: return launch_nf<4, TX>(P, jobs, njobs, nitems, queue, smem, ctas, s);
    case 5: return launch_nf<5, TX>(P, jobs, njobs, nitems, queue, smem, ctas, s);
    case 6: return launch_nf<6, TX>(P, jobs, njobs, nitems, queue, smem, ctas, s);
    case 7: return launch_nf<7, TX>(P, jobs, njobs, nitems, queue, smem, ctas, s);
    default: return launch_nf<8, TX>(P, jobs, njobs, nitems, queue, smem, ctas, s);
  }
}

int sweep_ctas_per_sm(int n_fields, size_t smem, int width) {
  return width == 512 ? ctas_per_sm<512>(n_fields, smem) : ctas_per_sm<256>(n_fields, smem);
}

int launch_sweep(const DevParams &P, const Job *jobs, int njobs, int nitems, int *queue, size_t smem, int ctas,
                 int width, cudaStream_t s) {
  cudaMemsetAsync(queue, 0, sizeof(int), s);
  return width == 512 ? launch_width<512>(P, jobs, njobs, nitems, queue, smem, ctas, s)
                      : launch_width<256>(P, jobs, njobs, nitems, queue, smem, ctas, s);
}

}  // namespace tmk
