// tm_fused.cuh -- plan and launcher of the fused integral-histogram sweep.
#pragma once

#include "tm_kernels.cuh"

namespace tmk {

constexpr int kMaxSlabs = 16;

// Tiling and ring layout of one sweep launch (computed on the host).
struct SweepPlan {
  int W, H;
  int TX, TY, tiles_x, tiles_y;   // output tile and tile grid
  int Rx, Ry;                     // largest half-width / half-height
  int nslabs;                     // row slabs over all fields (each < 2^16 pixels)
  int slab_field[kMaxSlabs];      // field of each slab
  int slab_a[kMaxSlabs];          // first row offset of the slab (relative to y)
  int slab_b[kMaxSlabs];          // last row offset of the slab
  int ring_len[kMaxSlabs];        // rows of the parked-corner ring of each slab
  int ring_off[kMaxSlabs];        // first row of that ring in the shared ring array
  int ring_total;
  int bmax;                       // largest slab_b: a pixel row completes at y + bmax
  int LB;                         // pixel rows evaluated together
  int CR;                         // rows of the per-tile count ring
  int BR;                         // rows of the tile's own bin ring
  int nseg_max;                   // 16-column segments of the widest swept row (<= 32)
  int rows_max;                   // rows of the widest swept band
  int nw_max;                     // threshold words (two thresholds each) allocated
  int text_max;                   // widest tile row including both side bands
  int cstride;                    // words per threshold row in shared memory (odd)
  int seglen;                     // columns per scan segment
  size_t smem;                    // dynamic shared memory bytes
};

// Choose a tile shape for a W x H image (cost model: rows x widened columns
// swept per wave, plus per-pixel work). false if the fields do not fit.
bool plan_sweep(const DevParams &P, int W, int H, int num_sms, size_t smem_limit, SweepPlan &S);

// uint16 elements of the per-slab count planes (nslabs x H x W).
size_t sweep_count_elems(const SweepPlan &S);

// Fused sweep: per-slab Eq. 1 numerators of every pixel into `counts`.
int launch_sweep(const DevParams &P, const SweepPlan &S, const uint8_t *bins, uint16_t *counts,
                 cudaStream_t s);

// Stage a4 from the sweep's per-slab counts.
int launch_lookup_counts(const Image &in, const Image &out, const DevParams &P, const SweepPlan &S,
                         const uint16_t *counts, const int64_t *s1, const int64_t *s2,
                         const DebugPlanes &dbg, cudaStream_t s);

}  // namespace tmk
