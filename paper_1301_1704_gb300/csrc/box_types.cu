// box_types.cu -- the source-box types of Alg. 6 (Sec. 3.2) for node J of a
// partition of the space at level l_par: DOMESTIC, EXPORT, IMPORT, ROOT or
// OTHERS for every source box of levels 2..L, from the source tree built
// against itself (its E4 lists are the M2L neighbours).
//
// Readings of the printed algorithm (the oracle takes the same): a box of
// level >= l_par is on J when its ancestor at l_par is owned by J; the
// children of an l_crit box that decide its type are its descendants at
// l_par; the IMPORT marks that one box's thread sets on another survive the
// final assignment (a box not on J is IMPORT when a box on J has it as an
// M2L neighbour, else OTHERS).  One thread per box, no races: a box reads its
// own E4 row instead of being written by its neighbours' threads.
#include "fmm_internal.cuh"

namespace fmm {
namespace {

// on[b] for the boxes of level l >= l_par: at l_par from the owners, deeper
// through the parent ranks.
__global__ void __launch_bounds__(256) on_node_kernel(const uint32_t* __restrict__ owner,
                                                      const uint32_t* __restrict__ parent,
                                                      const uint8_t* __restrict__ on_up,
                                                      uint32_t nbox, uint32_t node,
                                                      uint8_t* __restrict__ on) {
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nbox; b += gridDim.x * blockDim.x)
    on[b] = owner ? (owner[b] == node) : on_up[parent[b]];
}

// The boxes of l_crit: bit 0 = some descendant at l_par on J, bit 1 = some
// descendant off J.  Their children at l_par when l_crit < l_par (child
// ranges); the boxes themselves when l_crit = l_par (child = null).
__global__ void __launch_bounds__(256) child_sides_kernel(const uint32_t* __restrict__ child,
                                                          const uint8_t* __restrict__ on_par,
                                                          uint32_t nbox, uint8_t* __restrict__ sides) {
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nbox; b += gridDim.x * blockDim.x) {
    uint32_t s = 0;
    if (!child)
      s = on_par[b] ? 1u : 2u;
    else
      for (uint32_t c = child[b]; c < child[b + 1] && s != 3u; ++c) s |= on_par[c] ? 1u : 2u;
    sides[b] = (uint8_t)s;
  }
}

// The types of one level.  `sides` (levels <= l_crit) or `on` (deeper) give
// the boxes' relation to J.
__global__ void __launch_bounds__(256) box_type_kernel(const uint32_t* __restrict__ e4_off,
                                                       const uint32_t* __restrict__ e4_idx,
                                                       const uint8_t* __restrict__ sides,
                                                       const uint8_t* __restrict__ on,
                                                       uint32_t nbox, int mode,
                                                       uint8_t* __restrict__ type) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < nbox; k += gridDim.x * blockDim.x) {
    uint8_t t = FMM_BOX_DOMESTIC;
    if (mode == 1) {  // l_crit
      const uint32_t s = sides[k];
      if (!(s & 1u)) {
        t = FMM_BOX_IMPORT;
      } else if (s & 2u) {
        t = FMM_BOX_ROOT;
      } else {
        for (uint32_t j = e4_off[k]; j < e4_off[k + 1]; ++j)
          if (sides[e4_idx[j]] & 2u) {
            t = FMM_BOX_EXPORT;
            break;
          }
      }
    } else if (mode == 2) {  // deeper than l_crit
      const bool mine = on[k] != 0;
      bool across = false;  // an M2L neighbour on the other side of J's border
      for (uint32_t j = e4_off[k]; j < e4_off[k + 1] && !across; ++j)
        across = (on[e4_idx[j]] != 0) != mine;
      t = mine ? (across ? FMM_BOX_EXPORT : FMM_BOX_DOMESTIC)
               : (across ? FMM_BOX_IMPORT : FMM_BOX_OTHERS);
    }
    type[k] = t;
  }
}

uint32_t grid_for(uint32_t n) {
  uint32_t g = (n + 255) / 256;
  if (g > 152u * 8u) g = 152u * 8u;
  return g == 0 ? 1u : g;
}

}  // namespace

void launch_on_node(const uint32_t* owner, const uint32_t* parent, const uint8_t* on_up,
                    uint32_t nbox, uint32_t node, uint8_t* on, cudaStream_t s) {
  if (nbox == 0) return;
  on_node_kernel<<<grid_for(nbox), 256, 0, s>>>(owner, parent, on_up, nbox, node, on);
}

void launch_child_sides(const uint32_t* child, const uint8_t* on_par, uint32_t nbox,
                        uint8_t* sides, cudaStream_t s) {
  if (nbox == 0) return;
  child_sides_kernel<<<grid_for(nbox), 256, 0, s>>>(child, on_par, nbox, sides);
}

void launch_box_type(const uint32_t* e4_off, const uint32_t* e4_idx, const uint8_t* sides,
                     const uint8_t* on, uint32_t nbox, int mode, uint8_t* type, cudaStream_t s) {
  if (nbox == 0) return;
  box_type_kernel<<<grid_for(nbox), 256, 0, s>>>(e4_off, e4_idx, sides, on, nbox, mode, type);
}

}  // namespace fmm
