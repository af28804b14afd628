// panel_common.cuh -- pieces shared by the LU panel kernels.
#pragma once

#include "common.cuh"

namespace harp {

// Compose the row interchanges of a factored panel from its pivot rows
// (called by one warp; every CTA of a cluster calls it on the same data).
//   piv_row[t]  panel row (0-based, below k0) chosen at step t; -1 when no
//               row was left
// Step t swaps position t with the position of its pivot row (LAPACK's
// ipiv: that position). Only the first nb positions and the pivot rows'
// positions are touched. A row below nb moves only when it is chosen, and
// the row displaced from position t is always one of the first nb rows, so
// the warp tracks two tables in registers, lane l holding entries l and
// l + 32: prow (the row at position v < nb) and rpos (the position of row
// v < nb). Writes ipiv[k0 + t] and, when rmap is given, the panel's net row
// move (count, then (destination, source) pairs) from CTA 0 only; sets
// dest[r] (the output position of local row r of the CTA owning panel rows
// r0 .. r0 + rows - 1) for the local rows that move.
__device__ __forceinline__ void panel_compose(const int* piv_row, int nb, int k0, int r0,
                                              int rows, int crank, int* ipiv, int* rmap,
                                              int* dest, int lane) {
  int prow0 = lane, prow1 = lane + 32, rpos0 = lane, rpos1 = lane + 32;
  const int pv0 = (lane < nb) ? piv_row[lane] : -1;
  const int pv1 = (lane + 32 < nb) ? piv_row[lane + 32] : -1;
  for (int t = 0; t < nb; ++t) {
    const int hi_t = t >> 5, ln_t = t & 31;
    const int p = __shfl_sync(0xffffffffu, hi_t ? pv1 : pv0, ln_t);
    if (p < 0) {  // no row left: the position keeps its row
      if (crank == 0 && lane == 0) ipiv[k0 + t] = k0 + t;
      continue;
    }
    const int jq = __shfl_sync(0xffffffffu, (p & 32) ? rpos1 : rpos0, p & 31);
    const int rt = __shfl_sync(0xffffffffu, hi_t ? prow1 : prow0, ln_t);
    const int j = (p < nb) ? jq : p;  // the pivot row's current position
    if (crank == 0 && lane == 0) ipiv[k0 + t] = k0 + j;
    if (lane == ln_t) (hi_t ? prow1 : prow0) = p;
    if (p < nb && lane == (p & 31)) ((p & 32) ? rpos1 : rpos0) = t;
    if (j != t) {  // row rt (below nb) moves to position j
      if (j < nb && lane == (j & 31)) ((j & 32) ? prow1 : prow0) = rt;
      if (lane == (rt & 31)) ((rt & 32) ? rpos1 : rpos0) = j;
    }
  }
  // the net row move of the panel for the other columns (rmap, when
  // given): position v < nb takes row prow[v]; a row v < nb that ended
  // at or beyond nb is listed after them
  const bool d0 = lane < nb && rpos0 >= nb, d1 = lane + 32 < nb && rpos1 >= nb;
  const unsigned b0 = __ballot_sync(0xffffffffu, d0), b1 = __ballot_sync(0xffffffffu, d1);
  const unsigned below = (1u << lane) - 1u;
  if (rmap && crank == 0) {
    if (lane == 0) rmap[0] = nb + __popc(b0) + __popc(b1);
    if (lane < nb) {
      rmap[1 + 2 * lane] = k0 + lane;
      rmap[2 + 2 * lane] = k0 + prow0;
    }
    if (lane + 32 < nb) {
      rmap[1 + 2 * (lane + 32)] = k0 + lane + 32;
      rmap[2 + 2 * (lane + 32)] = k0 + prow1;
    }
    if (d0) {
      const int q = nb + __popc(b0 & below);
      rmap[1 + 2 * q] = k0 + rpos0;
      rmap[2 + 2 * q] = k0 + lane;
    }
    if (d1) {
      const int q = nb + __popc(b0) + __popc(b1 & below);
      rmap[1 + 2 * q] = k0 + rpos1;
      rmap[2 + 2 * q] = k0 + lane + 32;
    }
  }
  // output positions of this CTA's rows that move
  if (lane < nb && prow0 >= r0 && prow0 < r0 + rows) dest[prow0 - r0] = lane;
  if (lane + 32 < nb && prow1 >= r0 && prow1 < r0 + rows) dest[prow1 - r0] = lane + 32;
  if (d0 && lane >= r0 && lane < r0 + rows) dest[lane - r0] = rpos0;
  if (d1 && lane + 32 >= r0 && lane + 32 < r0 + rows) dest[lane + 32 - r0] = rpos1;
}

}  // namespace harp
