// tm_fused.cu -- fused integral-histogram sweep and per-pixel lookup.
//
// The integral histogram (Eq. 7-8) is never materialised in HBM. Each CTA owns
// an output tile [X0, X1) x [Y0, Y1) and sweeps the rows of the tile plus the
// half-size of the largest field above and below it. For the current row v it
// keeps, in shared memory, the cumulative integral histogram row
//     C_k(u, v) = #{(u', v') : cL < u' <= u, rL < v' <= v, b(u', v') < k}
// for every column u of the tile widened by the largest half-width on both
// sides (cL, rL: the sweep origin), for every threshold k in the range of bins
// present in the CTA's region. It is stored as
//     C_k(u, v) = D_k(u) + (u - cL) * m_k
// where m_k counts the rows whose bins all lie below k (such a row adds 1 per
// column to C_k, so it only bumps m_k), and D_k accumulates the exact row
// prefixes of the other rows. A row whose bins all lie at or above k adds
// nothing. So a row only costs dense work for thresholds inside its own bin
// range; the arithmetic stays exact for any input.
//
// Dense work: one warp per pair of thresholds, one lane per 16-column segment;
// each lane counts its segment, a warp shuffle scan gives the segment
// prefixes, and each lane adds the running prefix into its 16 columns. Shared
// arrays are laid out with a stride of 17 words (bins: 5 words) per segment
// so the 32 lanes hit 32 different banks.
//
// Tiles are strips of TX columns cut into row ranges of near-equal cost,
// planned on the device from the bin map (k_strip_scan, k_plan_tiles); the
// sweep CTAs pop them from a queue.
//
// A pixel's Eq. 1 numerator for field i is one box sum of C_{b(p)} (Eq. 9):
//     (C(x+r, y+r) - C(x-r-1, y+r)) - (C(x+r, y-r-1) - C(x-r-1, y-r-1)).
// The two horizontal differences are taken when the sweep passes rows y-r-1
// and y+r; the first is parked in a per-slab ring in shared memory until the
// second arrives. Counts are kept modulo 2^16 (two thresholds per 32-bit word,
// added lane-wise); a field whose window can hold 2^16 pixels or more is split
// into row slabs each holding fewer, so every slab count is exact. Each
// completed slab count is written once (uint16 per pixel and slab); the
// per-pixel lookup kernel then evaluates Eq. 2-4, 10, 3 and 12.
#include <algorithm>

#include "tm_kernels.cuh"

namespace tmk {
namespace {

constexpr int kNT = 512;
constexpr int kWarps = kNT / 32;
constexpr int kSeg = 16;  // columns per segment
constexpr int kTaskMax = 4;  // corner-event tasks per thread (planner: events x TX <= kTaskMax x kNT)

__device__ __forceinline__ unsigned thr_inc(int b, int klo) {
  // thresholds klo (low half) and klo + 1 (high half): [b < k] each
  return b < klo ? 0x10001u : (b == klo ? 0x10000u : 0u);
}

// a + b + c in two independent 16-bit lanes, each modulo 2^16, when both
// halves of b + c are below 2^15: with a's top bits set aside no carry leaves
// a lane, and xor puts the top bits back.
__device__ __forceinline__ unsigned add16x2_small(unsigned a, unsigned b, unsigned c) {
  return ((a & 0x7fff7fffu) + b + c) ^ (a & 0x80008000u);
}

// Position of swept column i (i >= 1) in a 17-word-per-segment row.
__device__ __forceinline__ int dpos(int i) {
  const int c = i - 1;
  return 1 + (c >> 4) * 17 + (c & 15);
}

struct Smem {
  unsigned *D;       // nw_max x cstride   dense part of C
  unsigned *m;       // nw_max             rows entirely below each threshold pair
  unsigned *brow;    // 5 words per segment: bins of the swept row
  uint16_t *acc;     // ring_total x TX    parked top-corner differences
  uint8_t *bring;    // BR x TX            bins of the tile's own pixel rows
  int *red;          // 64                 reductions
};

__device__ __forceinline__ Smem carve(const SweepPlan &S, unsigned char *base) {
  Smem mm;
  size_t off = 0;
  mm.D = reinterpret_cast<unsigned *>(base + off);
  off += (size_t)S.nw_max * S.cstride * 4;
  mm.m = reinterpret_cast<unsigned *>(base + off);
  off += (size_t)S.nw_max * 4;
  mm.brow = reinterpret_cast<unsigned *>(base + off);
  off += (size_t)S.nseg_max * 5 * 4;
  mm.red = reinterpret_cast<int *>(base + off);
  off += 64 * 4;
  mm.acc = reinterpret_cast<uint16_t *>(base + off);
  off += (size_t)S.ring_total * S.TX * 2;
  mm.bring = base + off;
  return mm;
}

// One output tile [strip * TX, ..) x [Y0, Y1) of one image. lohi: the strip's
// per-row bin ranges. evt_buf: per event of the row (double buffered by row
// parity): pixel row offset, ring offset, bin-ring offset, rx.
__device__ __forceinline__ void sweep_tile(const DevParams &P, const SweepPlan &S,
                                           const uint8_t *__restrict__ bins,
                                           const uint16_t *__restrict__ lohi,
                                           uint16_t *__restrict__ counts, int strip, int Y0, int Y1,
                                           unsigned char *smem_raw, int (*evt_buf)[2 * kMaxSlabs][4]) {
  const Smem sm = carve(S, smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int W = S.W, H = S.H;
  const long long N = (long long)W * H;
  const int X0 = strip * S.TX, X1 = min(X0 + S.TX, W);
  Y1 = min(Y1, H);
  if (X0 >= W || Y0 >= Y1) return;
  const int TXc = X1 - X0;
  const int cL = max(X0 - S.Rx - 1, -1), cR = min(X1 - 1 + S.Rx, W - 1);
  const int text = cR - cL + 1;  // columns cL..cR; index 0 is the origin
  const int ncol = text - 1;     // swept columns 1..text-1
  const int nseg = (ncol + kSeg - 1) / kSeg;
  const int rL = max(Y0 - S.Ry - 1, -1), rR = min(Y1 - 1 + S.Ry, H - 1);
  const int ne = 2 * S.nslabs;

  // ---- bin range of the whole region, from the strip's per-row ranges ----
  int kmin = 255, kmax = 0;
  for (int r = rL + 1 + tid; r <= rR; r += kNT) {
    const int lh = __ldg(lohi + r);
    kmin = min(kmin, lh & 0xff);
    kmax = max(kmax, lh >> 8);
  }
  kmin = __reduce_min_sync(0xffffffffu, kmin);
  kmax = __reduce_max_sync(0xffffffffu, kmax);
  if (lane == 0) {
    sm.red[wid] = kmin;
    sm.red[32 + wid] = kmax;
  }
  __syncthreads();
  kmin = 255;
  kmax = 0;
  for (int w = 0; w < kWarps; ++w) {
    kmin = min(kmin, sm.red[w]);
    kmax = max(kmax, sm.red[32 + w]);
  }
  if (kmax < kmin) kmax = kmin = 0;
  // Eq. 1 reads C_{b} (strict) or C_{b+1} (TM_FLAG_CDF_INCLUSIVE) at the
  // corners: thresholds kmin+1 .. kmax + incl, two per word
  const int incl = (P.flags & kFlagCdfIncl) ? 1 : 0;
  const int nw = (kmax + incl - kmin + 1) >> 1;
  const int koff = kmin + 1 - incl;  // corner events read threshold b(p) + incl, stored at index k - kmin - 1

  for (int t = tid; t < nw * S.cstride; t += kNT) sm.D[t] = 0u;
  for (int t = tid; t < nw; t += kNT) sm.m[t] = 0u;
  for (int y = Y0; y < min(Y1, rL + S.Ry + 2); ++y)
    for (int x = tid; x < TXc; x += kNT) sm.bring[(y % S.BR) * S.TX + x] = bins[(long long)y * W + X0 + x];
  // per-event constants and ring positions, one thread per event: event e is
  // slab e/2, top corner (e even) or bottom corner (e odd); its pixel row
  // advances by one per swept row, so its ring slots advance by one too
  int ev_a = 0, ev_b = 0, ev_roff = 0, ev_rlen = 1, ev_rx = 0, ev_y = 0, ev_slot = 0, ev_bslot = 0;
  if (tid < ne) {
    const int s = tid >> 1;
    ev_a = S.slab_a[s];
    ev_b = S.slab_b[s];
    ev_roff = S.ring_off[s];
    ev_rlen = S.ring_len[s];
    ev_rx = P.rx[S.slab_field[s]];
    ev_y = (tid & 1) ? rL - ev_b : rL - ev_a + 1;  // pixel row of the event at v = rL
    ev_slot = ((ev_y % ev_rlen) + ev_rlen) % ev_rlen;
    ev_bslot = ((ev_y % S.BR) + S.BR) % S.BR;
  }
  // corner-event tasks of this thread, fixed for the tile: task t = tid + i kNT
  // is (event e, column xo), e-major so a warp shares one event; the shared
  // positions of the two columns it reads and its m multiplier are constant
  int tk_ex[kTaskMax], tk_pos[kTaskMax], tk_coef[kTaskMax];
  {
    const int ntask = ne * TXc;
#pragma unroll
    for (int i = 0; i < kTaskMax; ++i) {
      const int t = tid + i * kNT;
      tk_ex[i] = -1;
      tk_pos[i] = 0;
      tk_coef[i] = 0;
      if (t < ntask) {
        const int e = t / TXc, xo = t - e * TXc;
        const int rx = P.rx[S.slab_field[e >> 1]];
        const int x = X0 + xo;
        const int ir = min(x + rx, W - 1) - cL, il = max(x - rx - 1, -1) - cL;
        tk_ex[i] = xo | (e << 16);
        tk_pos[i] = (ir > 0 ? dpos(ir) : 0) | ((il > 0 ? dpos(il) : 0) << 16);  // position 0 holds 0
        tk_coef[i] = ir - il;
      }
    }
  }
  int yn_slot = ((rL + S.Ry + 2) % S.BR + S.BR) % S.BR;  // bring slot of the row entering at rL+1
  // bins of the first swept row and of the pixel row entering with it
  int pb = 255, pn = 0;
  int lh = rL + 1 <= rR ? __ldg(lohi + rL + 1) : 0;  // bin range of the next swept row
  if (rL + 1 <= rR) {
    if (tid < ncol) pb = __ldg(bins + (long long)(rL + 1) * W + cL + 1 + tid);
    const int yn = rL + 1 + S.Ry + 1;
    if (yn >= Y0 && yn < Y1 && tid < TXc) pn = __ldg(bins + (long long)yn * W + X0 + tid);
  }
  __syncthreads();

  const int pRy = S.Ry, pBR = S.BR, pTX = S.TX, pCs = S.cstride;
  for (int v = rL; v <= rR; ++v) {
    const bool burst = (v < 0) || (v == H - 1);
    if (v > rL) {
      // ---- row v into shared memory; fetch row v+1 for the next step ----
      uint8_t *bw = reinterpret_cast<uint8_t *>(sm.brow);
      if (tid < nseg * kSeg) bw[tid + 4 * (tid >> 4)] = tid < ncol ? (uint8_t)pb : (uint8_t)255;
      const int yn = v + pRy + 1;
      if (yn >= Y0 && yn < Y1 && tid < TXc) sm.bring[yn_slot * pTX + tid] = (uint8_t)pn;
      yn_slot = yn_slot + 1 == pBR ? 0 : yn_slot + 1;
      if (v + 1 <= rR) {
        if (tid < ncol) pb = __ldg(bins + (long long)(v + 1) * W + cL + 1 + tid);
        if (yn + 1 >= Y0 && yn + 1 < Y1 && tid < TXc) pn = __ldg(bins + (long long)(yn + 1) * W + X0 + tid);
      }
      const int lo = lh & 0xff, hi = lh >> 8;
      if (v + 1 <= rR) lh = __ldg(lohi + v + 1);
      const int j0 = min(nw, max(0, (lo - kmin) >> 1));
      const int j1 = min(nw, max(j0, (hi - kmin + 1) >> 1));
      int (*evt)[4] = evt_buf[v & 1];
      if (tid < ne) {
        ++ev_y;
        ev_slot = ev_slot + 1 == ev_rlen ? 0 : ev_slot + 1;
        ev_bslot = ev_bslot + 1 == pBR ? 0 : ev_bslot + 1;
        if (!burst) {
          const int T = max(ev_y + ev_a - 1, -1), B = min(ev_y + ev_b, H - 1);
          const bool valid = ev_y >= Y0 && ev_y < Y1 && B > T;
          evt[tid][0] = valid ? ev_y * W : -1;  // row offset of the pixel
          evt[tid][1] = (ev_roff + ev_slot) * pTX;
          evt[tid][2] = ev_bslot * pTX;
          evt[tid][3] = ev_rx;
        }
      }
      __syncthreads();
      // rows entirely below a threshold pair only bump its row count
      for (int j = j1 + tid; j < nw; j += kNT) sm.m[j] += 0x10001u;
      // ---- dense words: one warp per word, one lane per segment ----
      for (int j = j0 + wid; j < j1; j += kWarps) {
        const int klo = kmin + 1 + 2 * j;
        unsigned loc[kSeg];  // running increments within the lane's segment
        unsigned tot = 0;
        if (lane < nseg) {
          const unsigned *bp = sm.brow + lane * 5;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const unsigned w4 = bp[q];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              tot += thr_inc((int)__byte_perm(w4, 0u, 0x4440u + e), klo);
              loc[q * 4 + e] = tot;
            }
          }
        }
        unsigned pre = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned yv = __shfl_up_sync(0xffffffffu, pre, o);
          if (lane >= o) pre += yv;
        }
        if (lane < nseg) {
          const unsigned base = pre - tot;  // lanes stay below 2^15: one row of columns
          unsigned *row = sm.D + j * pCs + 1 + lane * 17;
#pragma unroll
          for (int c = 0; c < kSeg; ++c)
            row[c] = add16x2_small(row[c], loc[c], base);  // columns past the edge are never read
        }
      }
      __syncthreads();
    } else if (!burst) {
      int (*evt)[4] = evt_buf[v & 1];
      if (tid < ne) {
        const int T = max(ev_y + ev_a - 1, -1), B = min(ev_y + ev_b, H - 1);
        const bool valid = ev_y >= Y0 && ev_y < Y1 && B > T;
        evt[tid][0] = valid ? ev_y * W : -1;  // row offset of the pixel
        evt[tid][1] = (ev_roff + ev_slot) * pTX;
        evt[tid][2] = ev_bslot * pTX;
        evt[tid][3] = ev_rx;
      }
      __syncthreads();
    }

    // ---- corner events of row v: top corners park, bottom corners complete ----
    if (!burst) {
      const int4 *evt = reinterpret_cast<const int4 *>(evt_buf[v & 1]);
#pragma unroll
      for (int i = 0; i < kTaskMax; ++i) {
        if (tk_ex[i] < 0) continue;
        const int e = tk_ex[i] >> 16, xo = tk_ex[i] & 0xffff;
        const int4 ev = evt[e];  // pixel row offset, ring offset, bin-ring offset
        if (ev.x < 0) continue;
        const int kk = (int)sm.bring[ev.z + xo] - koff;  // threshold index of b(p) (+1 if inclusive)
        unsigned g = 0;
        if (kk >= 0) {
          const int j = kk >> 1, sh = (kk & 1) << 4;
          const unsigned *row = sm.D + j * pCs;
          const unsigned mk = sm.m[j] >> sh;  // bits above the lane drop out in the final mask
          const unsigned dr = row[tk_pos[i] & 0xffff], dl = row[tk_pos[i] >> 16];
          g = (dr >> sh) - (dl >> sh) + (unsigned)tk_coef[i] * mk;
        }
        uint16_t *ac = sm.acc + ev.y + xo;
        if (!(e & 1)) *ac = (uint16_t)g;
        else
          counts[(long long)(e >> 1) * N + (unsigned)(ev.x + X0 + xo)] = (uint16_t)(g - (unsigned)*ac);
      }
    } else {
      for (int pass = 0; pass < 2; ++pass) {  // tops, then bottoms
        for (int s = 0; s < S.nslabs; ++s) {
          const int a = S.slab_a[s], bb = S.slab_b[s];
          int ylo, yhi;
          if (pass == 0) {
            if (v >= 0) { ylo = v - a + 1; yhi = ylo + 1; }
            else { ylo = Y0; yhi = 1 - a; }
          } else {
            if (v < H - 1) { ylo = v - bb; yhi = ylo + 1; }
            else { ylo = H - 1 - bb; yhi = Y1; }
          }
          ylo = max(ylo, Y0);
          yhi = min(yhi, Y1);
          if (ylo >= yhi) continue;
          const int rx = P.rx[S.slab_field[s]];
          const int ntask = (yhi - ylo) * TXc;
          for (int t = tid; t < ntask; t += kNT) {
            const int yy = t / TXc;
            const int y = ylo + yy, xo = t - yy * TXc, x = X0 + xo;
            const int T = max(y + a - 1, -1), B = min(y + bb, H - 1);
            if (B <= T) continue;  // empty slab: counted as 0 by the lookup
            const int b = sm.bring[(y % pBR) * pTX + xo] + incl;
            unsigned g = 0;
            if (b > kmin) {
              const int kk = b - kmin - 1;
              const int j = kk >> 1, sh = (kk & 1) << 4;
              const int ir = min(x + rx, W - 1) - cL, il = max(x - rx - 1, -1) - cL;
              const unsigned *row = sm.D + j * pCs;
              const unsigned mk = (sm.m[j] >> sh) & 0xffffu;
              const unsigned dr = ir > 0 ? row[dpos(ir)] : 0u, dl = il > 0 ? row[dpos(il)] : 0u;
              g = ((dr >> sh) - (dl >> sh) + (unsigned)(ir - il) * mk) & 0xffffu;
            }
            uint16_t *ac = sm.acc + (size_t)(S.ring_off[s] + y % S.ring_len[s]) * pTX + xo;
            if (pass == 0) *ac = (uint16_t)g;
            else counts[(long long)s * N + (long long)y * W + x] = (uint16_t)((g - (unsigned)*ac) & 0xffffu);
          }
        }
        __syncthreads();  // a burst may park and complete the same slot
      }
    }
    // no barrier here: the next row only writes its own bin slots and event
    // descriptors before its first barrier, which every warp reaches after
    // finishing this row's events
  }
}

// Persistent sweep over a queue of (image, strip, Y0, Y1) items: each CTA pops
// the next item until the queue is drained (unused slots have image -1).
__global__ void __launch_bounds__(kNT, 1)
    k_sweep(DevParams P, const Job *__restrict__ jobs, const int4 *__restrict__ items, int nitems,
            int *queue) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) int evt_buf[2][2 * kMaxSlabs][4];
  __shared__ int item_sh;
  for (;;) {
    if (threadIdx.x == 0) item_sh = atomicAdd(queue, 1);
    __syncthreads();
    const int it = item_sh;
    __syncthreads();
    if (it >= nitems) break;
    const int4 t = items[it];
    if (t.x < 0) continue;
    const Job &J = jobs[t.x];
    sweep_tile(P, J.plan, J.bins, J.lohi + (long long)t.y * J.plan.H, J.counts, t.y, t.z, t.w, smem_raw,
               evt_buf);
    __syncthreads();  // the next item reuses shared memory
  }
}

size_t smem_bytes(const SweepPlan &S) {
  return (size_t)S.nw_max * S.cstride * 4 + (size_t)S.nw_max * 4 + (size_t)S.nseg_max * 20 + 64 * 4 +
         (size_t)S.ring_total * S.TX * 2 + (size_t)S.BR * S.TX + 16;
}

// ---- adaptive tile heights ----
//
// A tile's sweep time is close to linear in the rows it sweeps (its own rows
// plus Ry above and below), in the dense threshold words of those rows (about
// half the width of each row's bin range; rows with more words than warps
// take a second round) and in its corner-event tasks (2 per slab and pixel).
// Per-tile clock counters over seven tile shapes fit, in cycles, about 1490
// per swept row, 56 per word, 640 per row needing a second round and 17 per
// warp of event tasks, within a few percent on the costliest tiles. Rows
// crossing strong edges are several times costlier than flat ones, so
// uniform tiles leave most SMs idle while the tiles over the busiest content
// finish. Each strip is instead cut into tiles of near-equal cost, with no
// more tiles per image than the uniform plan used. Cost units are 8 cycles.
constexpr int kRowFix = 186;      // a swept row's fixed work (setup, barriers, dense base)
constexpr int kWordCost = 7;      // one dense threshold word of a row
constexpr int kRound2 = 80;       // a row with more dense words than warps
constexpr int kEvtTask = 2;       // one warp of corner-event tasks
constexpr int kPlanCap = 8192;    // prefix-sum entries of one image's plan (shared memory)
constexpr int kPlanStrips = 1024; // strips one plan can hold
constexpr int kScanWarps = 8;     // (strip, block) units per scan CTA
constexpr int kPlanThreads = 1024;

__device__ __forceinline__ int row_cost(int lo, int hi) {
  const int w = (hi - lo + 1) >> 1;
  return kRowFix + kWordCost * w + (w > kWarps ? kRound2 : 0);
}

// Event cost of one pixel row of strip `strip`: 2 tasks per slab and column.
__device__ __forceinline__ int event_cost(const SweepPlan &S, int strip) {
  const int txc = min(S.TX, S.W - strip * S.TX);
  return kEvtTask * 2 * S.nslabs * ((txc + 31) / 32);
}

// One warp per (strip, block of rb rows): bin range of each row over the
// strip's swept columns, and the block's summed row cost.
__global__ void __launch_bounds__(32 * kScanWarps) k_strip_scan(const Job *__restrict__ jobs, int njobs) {
  const int j = find_job(jobs, njobs, kStScan, blockIdx.x);
  const Job &J = jobs[j];
  const SweepPlan &S = J.plan;
  const int lane = threadIdx.x & 31;
  const int unit = (blockIdx.x - J.b0[kStScan]) * kScanWarps + (threadIdx.x >> 5);
  if (unit >= S.tiles_x * J.nb) return;
  const int strip = unit / J.nb, blk = unit - strip * J.nb;
  const int W = S.W, H = S.H;
  const int X0 = strip * S.TX, X1 = min(X0 + S.TX, W);
  const int c0 = max(X0 - S.Rx, 0), c1 = min(X1 - 1 + S.Rx, W - 1);  // the sweep's columns cL+1 .. cR
  const int r0 = blk * J.rb, r1 = min(r0 + J.rb, H);
  int cost = 0;
  // aligned 4-byte words covering columns c0..c1 of a row: the first starts up
  // to 3 bytes before c0 (not before the 256-byte aligned bin map), the last
  // ends up to 3 bytes after c1 (inside the workspace after the bin map);
  // bytes outside c0..c1 are skipped. Each lane loads its words of two rows
  // before reducing them, so the loads are in flight together.
  const int span = c1 - c0;  // column offsets 0 .. span are swept
  constexpr int kWpl = 4;    // words per lane and row held at once (512 columns)
  for (int r = r0; r < r1; r += 2) {
    unsigned w[2][kWpl];
    int lead[2], nwd[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint8_t *row = J.bins + (long long)min(r + h, r1 - 1) * W;
      lead[h] = (int)(reinterpret_cast<uintptr_t>(row + c0) & 3u);
      nwd[h] = (span + lead[h] + 4) >> 2;  // words covering offsets -lead .. span
      const unsigned *wp = reinterpret_cast<const unsigned *>(row + c0 - lead[h]);
#pragma unroll
      for (int q = 0; q < kWpl; ++q) {
        const int i = lane + 32 * q;
        w[h][q] = i < nwd[h] ? __ldg(wp + i) : 0u;
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (r + h >= r1) break;
      const uint8_t *row = J.bins + (long long)(r + h) * W;
      const unsigned *wp = reinterpret_cast<const unsigned *>(row + c0 - lead[h]);
      int lo = 255, hi = 0;
      auto take = [&](unsigned wv, int i) {
        const int first = 4 * i - lead[h];  // column offset of the word's byte 0
        if (first >= 0 && first + 3 <= span) {  // the whole word is swept
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int b = (int)__byte_perm(wv, 0u, 0x4440u + k);
            lo = min(lo, b);
            hi = max(hi, b);
          }
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (first + k >= 0 && first + k <= span) {
              const int b = (int)__byte_perm(wv, 0u, 0x4440u + k);
              lo = min(lo, b);
              hi = max(hi, b);
            }
        }
      };
#pragma unroll
      for (int q = 0; q < kWpl; ++q)
        if (lane + 32 * q < nwd[h]) take(w[h][q], lane + 32 * q);
      for (int i = lane + 32 * kWpl; i < nwd[h]; i += 32) take(__ldg(wp + i), i);  // spans over 512 columns
      lo = __reduce_min_sync(0xffffffffu, lo);
      hi = __reduce_max_sync(0xffffffffu, hi);
      if (lane == 0) J.lohi[(long long)strip * H + r + h] = (uint16_t)(lo | (hi << 8));
      cost += row_cost(lo, hi);
    }
  }
  if (lane == 0) J.bcost[unit] = cost;
}

// Cost of a tile over blocks [b0, b1) of one strip: the row costs of its
// blocks plus hb halo blocks on each side (clipped to the strip), and the
// event cost E of each of its own rows.
struct StripCost {
  const int *P;  // nb + 1 prefix sums of the block costs
  int nb, hb, rb, H, E;
  __device__ __forceinline__ int operator()(int b0, int b1) const {
    return P[min(b1 + hb, nb)] - P[max(b0 - hb, 0)] + E * (min(b1 * rb, H) - b0 * rb);
  }
};

// Greedy cut of one strip by one warp: each tile takes the most blocks whose
// cost stays within T (a single block always fits: T is at least the largest
// one-block cost). This gives the fewest tiles for T, because a tile's cost
// grows with its end and falls with its start. The end is searched among 32
// consecutive ends around the last tile's length first, then 32-way. With
// `out`, lane 0 writes the tiles as items. Returns the number of tiles.
__device__ int cut_strip(const StripCost cost, int T, int guess, int lane, int4 *out, int job, int strip) {
  const int nb = cost.nb;
  int b0 = 0, n = 0;
  while (b0 < nb) {
    int lo = b0 + 1, hi = nb;  // largest b1 in [lo, hi] with cost(b0, b1) <= T; lo fits
    {
      const int c_first = min(max(b0 + guess - 15, b0 + 1), nb);
      const unsigned ok = __ballot_sync(0xffffffffu, cost(b0, min(c_first + lane, nb)) <= T);
      const int k = __popc(ok);  // the fitting ends are a prefix: cost grows with b1
      if (k == 0) hi = c_first - 1;  // c_first > b0 + 1 here: b0 + 1 always fits
      else {
        lo = min(c_first + k - 1, nb);
        if (k < 32) hi = lo;  // the next end is the first that does not fit
      }
    }
    while (lo < hi) {
      const int step = (hi - lo + 31) / 32;
      const int cand = min(lo + (lane + 1) * step, hi);
      const unsigned ok = __ballot_sync(0xffffffffu, cost(b0, cand) <= T);
      const int k = __popc(ok);
      if (k == 0) hi = lo + step - 1;
      else {
        lo = min(lo + k * step, hi);
        if (k < 32) hi = min(lo + step - 1, hi);
      }
    }
    if (out && lane == 0) out[n] = make_int4(job, strip, b0 * cost.rb, min(lo * cost.rb, cost.H));
    ++n;
    guess = lo - b0;
    b0 = lo;
  }
  return n;
}

// One CTA per image: the smallest T (to within 1/64) for which the greedy
// cuts of all strips need at most J.nitem tiles (bisection), then the items
// of those cuts. Without the adaptive plan the uniform tiles of the static
// plan are written.
__global__ void __launch_bounds__(kPlanThreads, 1) k_plan_tiles(const Job *__restrict__ jobs, int4 *__restrict__ items) {
  __shared__ int pre[kPlanCap];
  __shared__ int first[kPlanStrips + 1];
  __shared__ int tries[kPlanStrips];
  __shared__ int red_lo, red_hi, red_n;
  __shared__ unsigned long long red_sum;
  const int job = blockIdx.x;
  const Job &J = jobs[job];
  const SweepPlan &S = J.plan;
  const int ns = S.tiles_x, H = S.H, nitem = J.nitem, item0 = J.item0;
  int4 *out = items + item0;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwarp = kPlanThreads / 32;
  if (!J.adaptive) {
    for (int i = tid; i < nitem; i += kPlanThreads) {
      const int strip = i % ns, ty = i / ns;
      out[i] = ty < S.tiles_y ? make_int4(job, strip, ty * S.TY, min((ty + 1) * S.TY, H)) : make_int4(-1, 0, 0, 0);
    }
    return;
  }
  const int nb = J.nb, rb = J.rb, hb = (S.Ry + rb - 1) / rb;
  const int ev_full = event_cost(S, 0), ev_last = event_cost(S, ns - 1);
  auto strip_cost = [&](int s) { return StripCost{pre + s * (nb + 1), nb, hb, rb, H, s + 1 < ns ? ev_full : ev_last}; };
  // block costs into shared memory (all loads in flight together), then a
  // prefix sum per strip (a warp per strip)
  for (int u = tid; u < ns * nb; u += kPlanThreads) {
    const int s = u / nb, b = u - s * nb;
    pre[s * (nb + 1) + b + 1] = __ldg(J.bcost + u);
  }
  if (tid == 0) {
    red_lo = 0;
    red_hi = 0;
    red_sum = 0ull;
  }
  __syncthreads();
  for (int s = wid; s < ns; s += nwarp) {
    int *P = pre + s * (nb + 1);
    if (lane == 0) P[0] = 0;
    int carry = 0;
    for (int b0 = 0; b0 < nb; b0 += 32) {
      int v = b0 + lane < nb ? P[b0 + lane + 1] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
      }
      if (b0 + lane < nb) P[b0 + lane + 1] = carry + v;
      carry += __shfl_sync(0xffffffffu, v, 31);
    }
  }
  __syncthreads();
  // bounds of T. Below: the costliest single block (with halo), and the mean
  // of the strips' costs over the tiles (every tiling's costliest tile is at
  // least that). Above: the costliest tile of the uniform tiling with its
  // bounds rounded down to blocks, which uses J.nitem tiles.
  int tlo = 0, thi = 0;
  const int tpb = S.tiles_y;  // uniform tiles per strip
  for (int s = wid; s < ns; s += nwarp) {
    const StripCost c = strip_cost(s);
    for (int b = lane; b < nb; b += 32) tlo = max(tlo, c(b, b + 1));
    for (int t = lane; t < tpb; t += 32) {
      const int b0 = (int)((long long)t * S.TY / rb), b1 = t + 1 < tpb ? (int)((long long)(t + 1) * S.TY / rb) : nb;
      if (b1 > b0) thi = max(thi, c(b0, b1));
    }
    if (lane == 0) atomicAdd(&red_sum, (unsigned long long)c.P[nb]);
  }
  tlo = __reduce_max_sync(0xffffffffu, tlo);
  thi = __reduce_max_sync(0xffffffffu, thi);
  if (lane == 0) {
    atomicMax(&red_lo, tlo);
    atomicMax(&red_hi, thi);
  }
  __syncthreads();
  tlo = max(red_lo, (int)((red_sum + nitem - 1) / nitem));
  thi = max(red_hi, tlo);
  const int guess = max(1, (int)((long long)nb * ns / nitem));  // mean tile length in blocks
  bool counted = false;  // first[1..ns] holds the tiles per strip at T = thi
  while (thi - tlo > (thi >> 6)) {
    const int T = tlo + (thi - tlo) / 2;
    if (tid == 0) red_n = 0;
    __syncthreads();
    for (int s = wid; s < ns; s += nwarp) {
      const int n = cut_strip(strip_cost(s), T, guess, lane, nullptr, 0, 0);
      if (lane == 0) {
        tries[s] = n;
        atomicAdd(&red_n, n);
      }
    }
    __syncthreads();
    const bool fits = red_n <= nitem;
    if (fits)
      for (int s = tid; s < ns; s += kPlanThreads) first[s + 1] = tries[s];
    __syncthreads();  // red_n and tries are read before the next pass rewrites them
    if (fits) {
      thi = T;
      counted = true;
    } else {
      tlo = T + 1;
    }
  }
  // tiles per strip at T = thi, their first slots, then the items
  if (!counted) {
    for (int s = wid; s < ns; s += nwarp) {
      const int n = cut_strip(strip_cost(s), thi, guess, lane, nullptr, 0, 0);
      if (lane == 0) first[s + 1] = n;
    }
    __syncthreads();
  }
  if (wid == 0) {  // exclusive scan of the tile counts: the strips' first slots
    int carry = 0;
    for (int s0 = 0; s0 < ns; s0 += 32) {
      int v = s0 + lane < ns ? first[s0 + lane + 1] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
      }
      if (s0 + lane < ns) first[s0 + lane + 1] = carry + v;
      carry += __shfl_sync(0xffffffffu, v, 31);
    }
    if (lane == 0) first[0] = 0;
  }
  __syncthreads();
  for (int s = wid; s < ns; s += nwarp) cut_strip(strip_cost(s), thi, guess, lane, out + first[s], job, s);
  for (int i = first[ns] + tid; i < nitem; i += kPlanThreads) out[i] = make_int4(-1, 0, 0, 0);
}

}  // namespace

bool plan_sweep(const DevParams &P, int W, int H, int num_sms, size_t smem_limit, SweepPlan &S) {
  SweepPlan best{};
  double best_cost = 1e300;
  int Rx = 0, Ry = 0;
  for (int f = 0; f < P.n_fields; ++f) {
    Rx = max(Rx, P.rx[f]);
    Ry = max(Ry, P.ry[f]);
  }
  SweepPlan base{};
  base.W = W;
  base.H = H;
  base.Rx = min(Rx, W);
  base.Ry = min(Ry, H);
  // slabs: split a field's rows evenly so that every slab holds < 2^16 pixels.
  // Row offsets beyond +-(H-1) never reach a row of the image, so a half-height
  // is clipped to H-1 first: the clipped window of every pixel is unchanged.
  int ns = 0;
  for (int f = 0; f < P.n_fields; ++f) {
    const long long wx = min(2LL * P.rx[f] + 1, (long long)W);
    const long long ry = min((long long)P.ry[f], (long long)H - 1);
    const long long rows = 2 * ry + 1;
    const long long cap = 65535LL / wx;
    if (cap < 1) return false;
    const long long pieces = (rows + cap - 1) / cap;
    const long long hs = (rows + pieces - 1) / pieces;
    for (long long a = -ry; a <= ry; a += hs) {
      if (ns >= kMaxSlabs) return false;
      base.slab_field[ns] = f;
      base.slab_a[ns] = (int)a;
      base.slab_b[ns] = (int)min(a + hs - 1, ry);
      ++ns;
    }
  }
  base.nslabs = ns;
  for (int f = 0, s = 0; f <= kMaxFields; ++f) {
    while (s < ns && base.slab_field[s] < f) ++s;
    base.field_slab0[f] = s;
  }
  int bmax = -(1 << 30), ring_total = 0;
  for (int s = 0; s < ns; ++s) {
    base.ring_len[s] = base.slab_b[s] - base.slab_a[s] + 2;
    base.ring_off[s] = ring_total;
    ring_total += base.ring_len[s];
    bmax = max(bmax, base.slab_b[s]);
  }
  base.ring_total = ring_total;
  base.bmax = bmax;
  base.BR = base.Ry + max(bmax, 0) + 3;
  base.nw_max = P.n_bins / 2 + 1;
  const int cand_tx[] = {32, 48, 64, 80, 96, 112, 128, 160, 192, 224, 256, 320, 384, 448, 512};
  for (int TX : cand_tx) {
    if (TX > W && TX != cand_tx[0]) continue;
    SweepPlan S2 = base;
    S2.TX = min(TX, W);
    S2.tiles_x = (W + S2.TX - 1) / S2.TX;
    const int text_max = min(S2.TX + 2 * S2.Rx + 2, W + 1);
    S2.nseg_max = (text_max - 1 + 15) / 16;
    if (S2.nseg_max > 32) continue;  // one lane per 16-column segment
    if (2 * ns * S2.TX > kTaskMax * kNT) continue;  // corner-event tasks held in registers
    S2.text_max = text_max;
    S2.cstride = (1 + 17 * S2.nseg_max) | 1;
    for (int tiles_y = 1; tiles_y <= H; tiles_y = tiles_y < 8 ? tiles_y + 1 : tiles_y + tiles_y / 4) {
      const int TY = (H + tiles_y - 1) / tiles_y;
      const int ty_n = (H + TY - 1) / TY;
      SweepPlan S3 = S2;
      S3.TY = TY;
      S3.tiles_y = ty_n;
      S3.rows_max = min(TY + 2 * S3.Ry + 2, H + 2);
      S3.smem = smem_bytes(S3);
      if (S3.smem > smem_limit) continue;
      const long long ctas = (long long)S3.tiles_x * ty_n;
      const long long waves = (ctas + num_sms - 1) / num_sms;
      const double rows = min(TY + 2.0 * S3.Ry + 1, H + 1.0);
      // swept columns x rows (dense work), per-row fixed cost, per-pixel work
      const double cost = waves * ((double)text_max * rows * 0.25 + 300.0 * rows + 2.0 * S3.TX * TY);
      if (cost < best_cost) {
        best_cost = cost;
        best = S3;
      }
      if (ctas > 8LL * num_sms) break;
    }
  }
  if (best_cost >= 1e299) return false;
  S = best;
  return true;
}

size_t sweep_count_elems(const SweepPlan &S) { return (size_t)S.nslabs * S.W * S.H; }

void sweep_cost_blocks(const SweepPlan &S, int &rb, int &nb, int &adaptive) {
  // the strips' prefix sums (nb + 1 each) must fit kPlanCap, and a strip's
  // cost must fit an int
  const int ns = S.tiles_x;
  const int nb_max = std::max(1, kPlanCap / std::max(ns, 1) - 1);
  rb = (S.H + nb_max - 1) / nb_max;
  nb = (S.H + rb - 1) / rb;
  const long long row_max = kRowFix + kWordCost * 128 + kRound2 + kEvtTask * 2LL * S.nslabs * ((S.TX + 31) / 32);
  adaptive = ns <= kPlanStrips && (long long)ns * (nb + 1) <= kPlanCap && (long long)S.H * row_max < (1LL << 31);
}

int strip_scan_blocks(const SweepPlan &S, int nb) { return (S.tiles_x * nb + kScanWarps - 1) / kScanWarps; }

int launch_sweep_plan(const Job *jobs, int njobs, int scan_blocks, int4 *items, cudaStream_t s) {
  k_strip_scan<<<scan_blocks, 32 * kScanWarps, 0, s>>>(jobs, njobs);
  k_plan_tiles<<<njobs, kPlanThreads, 0, s>>>(jobs, items);
  return 2;
}

int launch_sweep(const DevParams &P, const Job *jobs, const int4 *items, int nitems, int *queue,
                 size_t smem, int ctas, cudaStream_t s) {
  // dynamic shared memory beyond 48 KB needs the opt-in attribute (the static
  // shared memory of the kernel is covered by the planner's margin)
  cudaError_t e = cudaFuncSetAttribute(k_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return -1;
  cudaMemsetAsync(queue, 0, sizeof(int), s);
  k_sweep<<<ctas, kNT, smem, s>>>(P, jobs, items, nitems, queue);
  return 1;
}

}  // namespace tmk
