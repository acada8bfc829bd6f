// boxes.cu -- non-empty boxes, bookmarks, parents and children at every
// level (Alg. 3, Sec. 2.2), from keys sorted by their top 3*Lb bits.
//
// Alg. 3 scans a dense histogram of all 8^lmax boxes.  Here nothing dense is
// built: sorted point i opens a box at level l exactly when its level-l key
// differs from that of point i-1, i.e. for every l >= d_i where d_i is fixed
// by the highest bit in which the two keys differ.  One pass over the sorted
// keys therefore flags the box starts of all levels at once, and a
// multi-level prefix sum (one decoupled look-back chain per level) gives each
// start its rank at every level it opens.  The rank of a start is the box's
// index in SrcNonEmptyBoxIndex / RecvNonEmptyBoxIdx and its position is the
// bookmark.
#include "fmm_internal.cuh"

namespace fmm {

uint32_t boxes_tiles(uint32_t n) {
  const uint64_t t = ((uint64_t)n + kBoxTile - 1) / kBoxTile;
  return t == 0 ? 1u : (uint32_t)t;
}

__global__ void __launch_bounds__(kBoxThreads) boxes_kernel(const uint64_t* __restrict__ keys,
                                                            uint32_t n, int Lb, LevelArrays lv,
                                                            uint64_t* status, uint32_t* counter,
                                                            uint32_t* nbox, DevStatus* st,
                                                            uint64_t wait_ns, uint32_t ntiles) {
  constexpr int W = kBoxThreads / 32;
  __shared__ uint32_t s_tile;
  __shared__ uint64_t s_key[kBoxTile + 1];
  __shared__ uint32_t s_wtot[W][kLevels];
  __shared__ uint32_t s_texcl[kLevels];  // starts in all tiles before this one
  __shared__ uint32_t s_ttot[kLevels];   // starts in this tile

  __shared__ uint32_t s_abort;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    s_tile = atomicAdd(counter, 1u);
    s_abort = failed(st) ? 1u : 0u;
  }
  __syncthreads();
  if (s_abort) return;  // an earlier kernel failed: leave the outputs alone
  const uint32_t tile = s_tile;
  const int64_t base = (int64_t)tile * kBoxTile;
  for (int j = threadIdx.x; j < kBoxTile + 1; j += kBoxThreads) {
    const int64_t i = base - 1 + j;
    s_key[j] = (i >= 0 && i < (int64_t)n) ? keys[i] : 0ull;
  }
  __syncthreads();

  // d[k]: coarsest level at which item k opens a box (0xff: none <= Lb).
  const int hshift = 63 - 3 * Lb;
  uint32_t d[kBoxItems];
#pragma unroll
  for (int k = 0; k < kBoxItems; ++k) {
    const int j = threadIdx.x * kBoxItems + k;
    const int64_t i = base + j;
    uint32_t v = 0xffu;
    if (i < (int64_t)n) {
      if (i == 0) {
        v = 0;
      } else {
        const uint64_t x = (s_key[j + 1] ^ s_key[j]) >> hshift;
        if (x != 0) {
          const int h = 63 - __clzll((long long)x) + hshift;  // highest differing bit
          v = (uint32_t)((65 - h) / 3);
        }
      }
    }
    d[k] = v;
  }

  // Per level: lane counts, warp-inclusive scan, warp totals.
  uint32_t lex[kLevels];  // lane-exclusive prefix within the warp, per level
#pragma unroll
  for (int l = 0; l < kLevels; ++l) {
    lex[l] = 0;
    if (l <= Lb) {
      uint32_t c = 0;
#pragma unroll
      for (int k = 0; k < kBoxItems; ++k) c += (d[k] <= (uint32_t)l);
      uint32_t x = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      lex[l] = x - c;
      if (lane == 31) s_wtot[warp][l] = x;
    }
  }
  __syncthreads();

  // Thread l of warp 0 handles level l: warp prefixes, tile total, look-back.
  if (threadIdx.x <= (unsigned)Lb) {
    const int l = threadIdx.x;
    uint32_t run = 0;
    for (int w = 0; w < W; ++w) {
      const uint32_t c = s_wtot[w][l];
      s_wtot[w][l] = run;
      run += c;
    }
    s_ttot[l] = run;
    uint64_t* sw = status + (uint64_t)tile * kLevels + l;
    uint64_t prev = 0;
    if (tile == 0) {
      st_relaxed(sw, kFlagIncl | run);
    } else {
      st_relaxed(sw, kFlagAgg | run);
      prev = lookback(status + l, tile, kLevels, st, wait_ns);
      st_relaxed(sw, kFlagIncl | (prev + run));
    }
    s_texcl[l] = (uint32_t)prev;
  }
  __syncthreads();
  if (threadIdx.x <= (unsigned)Lb && tile > 0 && ld_relaxed_u32(&st->abort)) s_abort = 1;
  __syncthreads();
  if (s_abort) return;  // a wait gave up: ranks may be wrong, write nothing
  if (tile == ntiles - 1 && threadIdx.x == 0) {
    for (int l = 0; l <= Lb; ++l) {
      const uint32_t nb = s_texcl[l] + s_ttot[l];
      nbox[l] = nb;
      if (nb <= lv.cap[l]) lv.off[l][nb] = n;
      if (l >= 1 && s_texcl[l - 1] + s_ttot[l - 1] <= lv.cap[l - 1])
        lv.child[l - 1][s_texcl[l - 1] + s_ttot[l - 1]] = nb;
    }
  }

  // Running rank per level: starts before this thread's first item.
  uint32_t run[kLevels];
#pragma unroll
  for (int l = 0; l < kLevels; ++l)
    run[l] = (l <= Lb) ? s_texcl[l] + s_wtot[warp][l] + lex[l] : 0u;

#pragma unroll
  for (int k = 0; k < kBoxItems; ++k) {
    const uint32_t dk = d[k];
    if (dk <= (uint32_t)Lb) {
      const int j = threadIdx.x * kBoxItems + k;
      const uint32_t i = (uint32_t)(base + j);
      const uint64_t key = s_key[j + 1];
#pragma unroll
      for (int l = 0; l < kLevels; ++l) {
        if (l <= Lb && (uint32_t)l >= dk && run[l] < lv.cap[l]) {
          const uint32_t rank = run[l];
          lv.key[l][rank] = l == 0 ? 0ull : key >> (63 - 3 * l);
          lv.off[l][rank] = i;
          if (l >= 1) {
            const bool up_starts = dk <= (uint32_t)(l - 1);
            lv.parent[l][rank] = up_starts ? run[l - 1] : run[l - 1] - 1u;
            if (up_starts && run[l - 1] < lv.cap[l - 1]) lv.child[l - 1][run[l - 1]] = rank;
          }
        }
      }
#pragma unroll
      for (int l = 0; l < kLevels; ++l)
        if (l <= Lb && (uint32_t)l >= dk) ++run[l];
    }
  }
}

void launch_boxes(const uint64_t* keys, uint32_t n, int Lb, LevelArrays lv, uint64_t* status,
                  uint32_t* counter, uint32_t* nbox, DevStatus* st, uint64_t wait_ns,
                  cudaStream_t s) {
  const uint32_t t = boxes_tiles(n);
  boxes_kernel<<<t, kBoxThreads, 0, s>>>(keys, n, Lb, lv, status, counter, nbox, st, wait_ns, t);
}

// ---------------------------------------------------------------------------
// Child-occupancy mask of every box of levels 0..Lb-1: bit o is set when the
// child in octant o (x + 2y + 4z) is non-empty.  Lists use it to enumerate the
// children of a parent-level neighbour without reading their keys.
__global__ void occupancy_kernel(int Lb, LevelArrays lv, const uint32_t* __restrict__ nbox,
                                 const DevStatus* st) {
  const int l = blockIdx.y;
  if (l >= Lb || failed(st)) return;
  const uint32_t nb = nbox[l] < lv.cap[l] ? nbox[l] : lv.cap[l];
  const uint32_t* ch = lv.child[l];
  const uint64_t* ck = lv.key[l + 1];
  uint8_t* occ = lv.occ[l];
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
    uint32_t m = 0;
    const uint32_t c1 = ch[b + 1];
    for (uint32_t c = ch[b]; c < c1; ++c) m |= 1u << (uint32_t)(ck[c] & 7u);
    occ[b] = (uint8_t)m;
  }
}

void launch_occupancy(int Lb, LevelArrays lv, const uint32_t* nbox, uint32_t n,
                      const DevStatus* st, cudaStream_t s) {
  if (Lb < 1) return;
  uint32_t bx = (uint32_t)(((uint64_t)n + 255) / 256);
  if (bx > 152u * 4u) bx = 152u * 4u;
  if (bx == 0) bx = 1;
  occupancy_kernel<<<dim3(bx, Lb), 256, 0, s>>>(Lb, lv, nbox, st);
}

// Largest box occupancy of each level 0..Lb (cluster-size mode, Sec. 2.1).
__global__ void max_occupancy_kernel(int Lb, LevelArrays lv, const uint32_t* __restrict__ nbox,
                                     uint32_t* maxocc, const DevStatus* st) {
  const int l = blockIdx.y;
  if (l > Lb || failed(st)) return;
  const uint32_t nb = nbox[l] < lv.cap[l] ? nbox[l] : lv.cap[l];
  const uint32_t* off = lv.off[l];
  uint32_t m = 0;
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
    const uint32_t c = off[b + 1] - off[b];
    m = c > m ? c : m;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint32_t y = __shfl_xor_sync(0xffffffffu, m, o);
    m = y > m ? y : m;
  }
  if ((threadIdx.x & 31) == 0 && m) atomicMax(&maxocc[l], m);
}

void launch_max_occupancy(int Lb, LevelArrays lv, const uint32_t* nbox, uint32_t n,
                          uint32_t* maxocc, const DevStatus* st, cudaStream_t s) {
  uint32_t bx = (uint32_t)(((uint64_t)n + 255) / 256);
  if (bx > 152u * 4u) bx = 152u * 4u;
  if (bx == 0) bx = 1;
  max_occupancy_kernel<<<dim3(bx, Lb + 1), 256, 0, s>>>(Lb, lv, nbox, maxocc, st);
}

}  // namespace fmm
