// fixed_grid.cu -- the paper's own order of the points: the Fixed-Grid
// pseudo-sort (Alg. 1) over a dense histogram of the level-Ls cells, its
// bookmarks by a prefix sum of the histogram (Alg. 3), and the move of every
// point to bookmark + rank.
//
// Alg. 1 gives each point its cell and its rank among the points of the cell
// from the return value of one atomicAdd on the cell's histogram entry (the
// printed pseudocode re-reads the entry after the add, a race; the value the
// atomic returns is the rank).  The ranks, and so the order inside a cell,
// depend on the order in which the atomics land: the finishing sort that
// follows (finish_boxes) orders every level-Ls box by (key, index), so the
// build's output does not.  The histogram needs 8^Ls entries per set, so this
// path serves depths Ls <= 8 (the paper's own limit on a 4 GB GPU).
#include "fmm_internal.cuh"

namespace fmm {
namespace {

// Per tile of one set: Morton keys (stored for the move and the boxes),
// level-Ls cells, ranks from the histogram's atomics (Alg. 1).  Slot aux0 =
// the set's first histogram entry.
__global__ void __launch_bounds__(256) fg_count_kernel(const Seg* __restrict__ segs,
                                                       const Slot* __restrict__ slots,
                                                       uint32_t nslots, uint32_t* __restrict__ bins,
                                                       uint64_t* __restrict__ keys_out,
                                                       uint32_t* __restrict__ ranks_out,
                                                       DevStatus* st) {
  const Slot sl = slots[find_slot(slots, nslots, blockIdx.x)];
  const Seg& sg = segs[sl.seg];
  const uint64_t base = (uint64_t)(blockIdx.x - sl.unit0) * sg.tile;
  const uint32_t cnt = (uint32_t)((sg.n - base) < (uint64_t)sg.tile ? (sg.n - base) : sg.tile);
  const int shift = 63 - 3 * sg.Ls;
  uint32_t* const bin = bins + sl.aux0;
  uint64_t* const ko = keys_out + sg.base + base;
  uint32_t* const ro = ranks_out + sg.base + base;
  const float* xyz = sg.xyz + 3 * base;
  bool bad = false;
  for (uint32_t j = threadIdx.x; j < cnt; j += blockDim.x) {
    bool ok;
    const uint64_t k = morton_key(xyz[3 * j], xyz[3 * j + 1], xyz[3 * j + 2], &ok);
    bad |= !ok;
    const uint32_t cell = shift >= 63 ? 0u : (uint32_t)(k >> shift);
    ko[j] = k;
    ro[j] = atomicAdd(bin + cell, 1u);
  }
  if (bad) set_error(st, FMM_ERR_DOMAIN);
}

// Moves every point to its bookmark + rank.  `bins` holds the exclusive
// prefix sum over all sets' histograms; slot aux1 = the set's base minus the
// points of the sets before it.
__global__ void __launch_bounds__(256) fg_move_kernel(const Seg* __restrict__ segs,
                                                      const Slot* __restrict__ slots,
                                                      uint32_t nslots,
                                                      const uint32_t* __restrict__ bins,
                                                      const uint64_t* __restrict__ keys_in,
                                                      const uint32_t* __restrict__ ranks_in,
                                                      uint64_t* __restrict__ keys_out,
                                                      uint32_t* __restrict__ vals_out,
                                                      const DevStatus* st) {
  if (failed(st)) return;
  const Slot sl = slots[find_slot(slots, nslots, blockIdx.x)];
  const Seg& sg = segs[sl.seg];
  const uint64_t base = (uint64_t)(blockIdx.x - sl.unit0) * sg.tile;
  const uint32_t cnt = (uint32_t)((sg.n - base) < (uint64_t)sg.tile ? (sg.n - base) : sg.tile);
  const int shift = 63 - 3 * sg.Ls;
  const uint32_t* const bin = bins + sl.aux0;
  const uint32_t lo = sg.base, hi = sg.base + sg.n;
  for (uint32_t j = threadIdx.x; j < cnt; j += blockDim.x) {
    const uint64_t i = sg.base + base + j;
    const uint64_t k = keys_in[i];
    const uint32_t cell = shift >= 63 ? 0u : (uint32_t)(k >> shift);
    const uint32_t g = bin[cell] + sl.aux1 + ranks_in[i];
    if (g >= lo && g < hi) {  // inside the set's slots
      keys_out[g] = k;
      vals_out[g] = (uint32_t)(base + j);
    }
  }
}

}  // namespace

void launch_fg_count(const Seg* segs, const Slot* slots, uint32_t nslots, uint32_t ntiles,
                     uint32_t* bins, uint64_t* keys_out, uint32_t* ranks_out, DevStatus* st,
                     cudaStream_t s) {
  if (ntiles == 0) return;
  fg_count_kernel<<<ntiles, 256, 0, s>>>(segs, slots, nslots, bins, keys_out, ranks_out, st);
}

void launch_fg_move(const Seg* segs, const Slot* slots, uint32_t nslots, uint32_t ntiles,
                    const uint32_t* bins, const uint64_t* keys_in, const uint32_t* ranks_in,
                    uint64_t* keys_out, uint32_t* vals_out, DevStatus* st, cudaStream_t s) {
  if (ntiles == 0) return;
  fg_move_kernel<<<ntiles, 256, 0, s>>>(segs, slots, nslots, bins, keys_in, ranks_in, keys_out,
                                        vals_out, st);
}

}  // namespace fmm
