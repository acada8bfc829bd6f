// boxes.cu -- non-empty boxes, bookmarks, parents and children at every
// level (Alg. 3, Sec. 2.2), from keys sorted by their top 3*Lb bits, fused
// with the finishing sort of the point order inside each box.
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

constexpr int kWin = kBoxTile + kBoxHalo;  // points held per tile
constexpr size_t kBoxSmem = sizeof(uint64_t) * (kWin + 1) + sizeof(uint32_t) * kWin;

// kLv: level slots held in registers (8 when Lb <= 7, else 22).
template <int kLv>
__global__ void __launch_bounds__(kBoxThreads) finish_boxes_kernel(
    const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals, uint32_t n, int Lb,
    int Ls, LevelArrays lv, uint32_t* __restrict__ perm, uint64_t* status, uint32_t* counter,
    uint32_t* nbox, DevStatus* st, uint64_t wait_ns, uint32_t ntiles) {
  constexpr int W = kBoxThreads / 32;
  __shared__ uint32_t s_tile, s_abort;
  __shared__ uint32_t s_wtot[W][kLevels];
  __shared__ uint32_t s_texcl[kLevels];  // box starts in all tiles before this one
  __shared__ uint32_t s_ttot[kLevels];   // box starts in this tile
  extern __shared__ __align__(16) uint64_t s_key[];  // s_key[j + 1] = key of point t0 + j
  uint32_t* s_val = reinterpret_cast<uint32_t*>(s_key + kWin + 1);

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    s_tile = atomicAdd(counter, 1u);
    s_abort = failed(st) ? 1u : 0u;
  }
  __syncthreads();
  if (s_abort) return;  // an earlier kernel failed: leave the outputs alone
  const uint32_t tile = s_tile;
  const int64_t t0 = (int64_t)tile * kBoxTile;
  const int64_t nn = n;
  for (int j = threadIdx.x; j < kWin + 1; j += kBoxThreads) {
    const int64_t i = t0 - 1 + j;
    s_key[j] = (i >= 0 && i < nn) ? keys[i] : 0ull;
  }
  for (int j = threadIdx.x; j < kWin; j += kBoxThreads) {
    const int64_t i = t0 + j;
    s_val[j] = i < nn ? vals[i] : 0u;
  }
  __syncthreads();

  // Box starts of levels 0..Lb.  d[k]: coarsest level at which item k
  // opens a box (0xff: none).  Items are blocked: thread t holds kBoxItems
  // consecutive points.
  const int hshift = 63 - 3 * Lb;
  uint32_t d[kBoxItems];
#pragma unroll
  for (int k = 0; k < kBoxItems; ++k) {
    const int j = threadIdx.x * kBoxItems + k;
    const int64_t i = t0 + j;
    uint32_t v = 0xffu;
    if (i < nn) {
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
  uint32_t lex[kLv];  // lane-exclusive prefix within the warp, per level
#pragma unroll
  for (int l = 0; l < kLv; ++l) {
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

  // Warp w handles levels w, w + 8, ...: warp prefixes and the tile total,
  // published at once as this tile's aggregate.
  for (int l = warp; l <= Lb; l += W) {
    if (lane == 0) {
      uint32_t run = 0;
      for (int w = 0; w < W; ++w) {
        const uint32_t c = s_wtot[w][l];
        s_wtot[w][l] = run;
        run += c;
      }
      s_ttot[l] = run;
      st_relaxed(status + (uint64_t)tile * kLevels + l, (tile == 0 ? kFlagIncl : kFlagAgg) | run);
    }
  }

  // Finishing sort inside the level-Ls boxes that START in this tile,
  // including their points in the halo past the tile's end; a box begun in an
  // earlier tile is finished by that tile.  In a box the points stand in index
  // order already.  It runs between publishing this tile's aggregate and
  // reading the earlier tiles', which gives them time to publish.
  {
    const int loS = 63 - 3 * Ls;
    const int jend = (int)((nn - t0) < kWin ? (nn - t0) : kWin);  // valid window points
    bool long_box = false;
    for (int j = threadIdx.x; j < jend; j += kBoxThreads) {
      const uint64_t k = s_key[j + 1];
      const uint64_t top = k >> loS;
      int a = j;
      while (a > 0 && (s_key[a] >> loS) == top) --a;  // s_key[a] is point a - 1
      if (a >= kBoxTile) continue;                                 // the next tile's box
      if (a == 0 && t0 > 0 && (s_key[0] >> loS) == top) continue;  // an earlier tile's box
      int b = j + 1;
      while (b < jend && (s_key[b + 1] >> loS) == top) ++b;
      if (b == jend && t0 + jend < nn) {
        long_box = true;  // runs past the window: the host redoes the order
        continue;
      }
      uint32_t r = 0;
      for (int q = a; q < b; ++q) {
        const uint64_t kq = s_key[q + 1];
        r += (kq < k) || (kq == k && q < j);
      }
      perm[t0 + a + r] = s_val[j];
    }
    if (long_box) atomicExch(&st->seg_long, 1u);
  }

  // Windowed look-back over the earlier tiles, one warp per level.
  for (int l = warp; l <= Lb; l += W) {
    uint64_t prev = 0;
    if (tile > 0) {
      prev = lookback_warp(status + l, tile, kLevels, st, wait_ns);
      if (lane == 0) st_relaxed(status + (uint64_t)tile * kLevels + l, kFlagIncl | (prev + s_ttot[l]));
    }
    if (lane == 0) s_texcl[l] = (uint32_t)prev;
  }
  __syncthreads();
  if (threadIdx.x == 0 && tile > 0 && ld_relaxed_u32(&st->abort)) s_abort = 1;
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

  uint32_t run[kLv];  // running rank per level: starts before the current item
#pragma unroll
  for (int l = 0; l < kLv; ++l) run[l] = (l <= Lb) ? s_texcl[l] + s_wtot[warp][l] + lex[l] : 0u;
#pragma unroll
  for (int k = 0; k < kBoxItems; ++k) {
    const uint32_t dk = d[k];
    if (dk <= (uint32_t)Lb) {
      const int j = threadIdx.x * kBoxItems + k;
      const uint32_t i = (uint32_t)(t0 + j);
      const uint64_t key = s_key[j + 1];
#pragma unroll
      for (int l = 0; l < kLv; ++l) {
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
      for (int l = 0; l < kLv; ++l)
        if (l <= Lb && (uint32_t)l >= dk) ++run[l];
    }
  }
}

void launch_finish_boxes(const uint64_t* keys, const uint32_t* vals, uint32_t n, int Lb, int Ls,
                         LevelArrays lv, uint32_t* perm, uint64_t* status, uint32_t* counter,
                         uint32_t* nbox, DevStatus* st, uint64_t wait_ns, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(finish_boxes_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kBoxSmem);
    cudaFuncSetAttribute(finish_boxes_kernel<kLevels>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBoxSmem);
    attr = true;
  }
  const uint32_t t = boxes_tiles(n);
  if (Lb < 8)
    finish_boxes_kernel<8><<<t, kBoxThreads, kBoxSmem, s>>>(keys, vals, n, Lb, Ls, lv, perm,
                                                             status, counter, nbox, st, wait_ns, t);
  else
    finish_boxes_kernel<kLevels><<<t, kBoxThreads, kBoxSmem, s>>>(
        keys, vals, n, Lb, Ls, lv, perm, status, counter, nbox, st, wait_ns, t);
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
