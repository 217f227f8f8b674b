// Checked builds (nvcc -DPL_CHECKED, `python -m paper_2504_03909_b300.build
// --checked`): device-side bounds checks on gathered indices and table
// offsets, for runs where compute-sanitizer is not available.  A failed check
// skips the access and sets the check's bit in a per-translation-unit device
// word; paillier_sync ORs the words of every unit, clears them and reports
// PL_EDEVICE.  In the normal build PL_BOUNDS(ok, site) is `true` and costs
// nothing.
#pragma once

#include <cuda_runtime.h>

namespace pl {

// check sites (bit numbers of the word)
enum BoundsSite {
  kBoundsSample = 0,    // a sample index gathered from the sort (k_seg_product)
  kBoundsChunk = 1,     // a chunk partial read by k_combine
  kBoundsScatter = 2,   // a sorted position written by k_hist_scatter
  kBoundsTable = 3,     // a window-table entry of the exponentiation schedule
  kBoundsCluster = 4,   // a CKKS cluster exchange (rank, slice index)
  kBoundsSlot = 5,      // a CKKS slot permutation index
};

#ifdef PL_CHECKED
void register_bounds_reader(int (*read_and_clear)());
#endif

}  // namespace pl

#ifdef PL_CHECKED
namespace {
__device__ int g_pl_bounds;  // this translation unit's word

__device__ __forceinline__ bool pl_in_bounds(bool ok, int site) {
  if (!ok) atomicOr(&g_pl_bounds, 1 << site);
  return ok;
}

int pl_read_bounds() {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_pl_bounds, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (v) {
    const int z = 0;
    cudaMemcpyToSymbol(g_pl_bounds, &z, sizeof(int));
  }
  return v;
}

const bool g_pl_bounds_registered = (pl::register_bounds_reader(pl_read_bounds), true);
}  // namespace
#define PL_BOUNDS(ok, site) pl_in_bounds((ok), (site))
#else
#define PL_BOUNDS(ok, site) true
#endif
