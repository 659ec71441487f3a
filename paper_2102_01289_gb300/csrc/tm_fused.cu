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
// A pixel's Eq. 1 numerator for field i is one box sum of C_{b(p)} (Eq. 9):
//     (C(x+r, y+r) - C(x-r-1, y+r)) - (C(x+r, y-r-1) - C(x-r-1, y-r-1)).
// The two horizontal differences are taken when the sweep passes rows y-r-1
// and y+r; the first is parked in a per-slab ring in shared memory until the
// second arrives. Counts are kept modulo 2^16 (two thresholds per 32-bit word,
// added lane-wise); a field whose window can hold 2^16 pixels or more is split
// into row slabs each holding fewer, so every slab count is exact. Each
// completed slab count is written once (uint16 per pixel and slab); the
// per-pixel lookup kernel then evaluates Eq. 2-4, 10, 3 and 12.
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
  uint8_t *rowlo;    // rows of the region: smallest bin of each swept row
  uint8_t *rowhi;    // largest bin of each swept row
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
  off += (size_t)S.BR * S.TX;
  mm.rowlo = base + off;
  off += (size_t)S.rows_max;
  mm.rowhi = base + off;
  return mm;
}

// One output tile of one image. evt_buf: per event of the row (double
// buffered by row parity): pixel row, ring offset, bin-ring offset, rx.
__device__ __forceinline__ void sweep_tile(const DevParams &P, const SweepPlan &S,
                                           const uint8_t *__restrict__ bins,
                                           uint16_t *__restrict__ counts, int tile,
                                           unsigned char *smem_raw, int (*evt_buf)[2 * kMaxSlabs][4]) {
  const Smem sm = carve(S, smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int W = S.W, H = S.H;
  const long long N = (long long)W * H;
  const int tx = tile % S.tiles_x, ty = tile / S.tiles_x;
  const int X0 = tx * S.TX, X1 = min(X0 + S.TX, W);
  const int Y0 = ty * S.TY, Y1 = min(Y0 + S.TY, H);
  if (X0 >= W || Y0 >= H) return;
  const int TXc = X1 - X0;
  const int cL = max(X0 - S.Rx - 1, -1), cR = min(X1 - 1 + S.Rx, W - 1);
  const int text = cR - cL + 1;  // columns cL..cR; index 0 is the origin
  const int ncol = text - 1;     // swept columns 1..text-1
  const int nseg = (ncol + kSeg - 1) / kSeg;
  const int rL = max(Y0 - S.Ry - 1, -1), rR = min(Y1 - 1 + S.Ry, H - 1);
  const int ne = 2 * S.nslabs;

  // ---- bin range of every swept row and of the whole region ----
  int kmin = 255, kmax = 0;
  for (int r = rL + 1 + wid; r <= rR; r += kWarps) {
    const uint8_t *row = bins + (long long)r * W;
    int lo = 255, hi = 0;
    for (int c = cL + 1 + lane; c <= cR; c += 32) {
      const int b = row[c];
      lo = min(lo, b);
      hi = max(hi, b);
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if (lane == 0) {
      sm.rowlo[r - rL - 1] = (uint8_t)lo;
      sm.rowhi[r - rL - 1] = (uint8_t)hi;
    }
    kmin = min(kmin, lo);
    kmax = max(kmax, hi);
  }
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
      const int lo = sm.rowlo[v - rL - 1], hi = sm.rowhi[v - rL - 1];
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

// Persistent sweep over a queue of (image, tile) items, longest first: each
// CTA pops the next item until the queue is drained.
__global__ void __launch_bounds__(kNT, 1)
    k_sweep(DevParams P, const Job *__restrict__ jobs, const int2 *__restrict__ items, int nitems,
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
    const int2 jt = items[it];
    const Job &J = jobs[jt.x];
    sweep_tile(P, J.plan, J.bins, J.counts, jt.y, smem_raw, evt_buf);
    __syncthreads();  // the next item reuses shared memory
  }
}

size_t smem_bytes(const SweepPlan &S) {
  return (size_t)S.nw_max * S.cstride * 4 + (size_t)S.nw_max * 4 + (size_t)S.nseg_max * 20 + 64 * 4 +
         (size_t)S.ring_total * S.TX * 2 + (size_t)S.BR * S.TX + 2 * (size_t)S.rows_max + 16;
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

int launch_sweep(const DevParams &P, const Job *jobs, const int2 *items, int nitems, int *queue,
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
