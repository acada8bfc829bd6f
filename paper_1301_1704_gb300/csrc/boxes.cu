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
// Shared memory: keys [kWin + 2] (u64: the two points before the tile, then
// the window, so that a bulk copy can start 16-byte aligned), then the
// per-point first differing levels [kWin] (u8, 16-byte aligned for vector
// reads), then the indices [kWin] (u32).
constexpr size_t kBoxDdOff = (sizeof(uint64_t) * (kWin + 2) + 15) & ~(size_t)15;
constexpr size_t kBoxValOff = kBoxDdOff + kWin;
constexpr size_t kBoxSmem = kBoxValOff + sizeof(uint32_t) * kWin;
static_assert(kWin % 16 == 0 && kBoxValOff % 16 == 0, "shared layout alignment");

// First level at which a key differs from the key before it (22: equal keys;
// the keys use bits 0..62, level l owns bits 63-3l .. 65-3l).
__device__ __forceinline__ uint32_t first_diff_level(uint64_t a, uint64_t b) {
  const uint64_t x = a ^ b;
  return x == 0 ? 22u : (uint32_t)((2 + __clzll((long long)x)) / 3);
}

__global__ void __launch_bounds__(kBoxThreads) finish_boxes_kernel(const Seg* __restrict__ segs,
                                                                   const Slot* __restrict__ slots,
                                                                   uint32_t nslots, DevStatus* st,
                                                                   uint64_t wait_ns) {
  constexpr int W = kBoxThreads / 32;
  __shared__ uint32_t s_tile, s_abort, s_ttot, s_texcl;
  __shared__ uint32_t s_wtot[W];
  __shared__ __align__(8) uint64_t s_bar;
  extern __shared__ __align__(16) uint64_t s_key[];  // s_key[j + 2] = key of point t0 + j
  uint64_t* const sk = s_key + 1;                     // sk[j + 1] = key of point t0 + j
  uint8_t* s_dd = reinterpret_cast<uint8_t*>(s_key) + kBoxDdOff;  // first differing level
  uint32_t* s_val = reinterpret_cast<uint32_t*>(reinterpret_cast<uint8_t*>(s_key) + kBoxValOff);

  const Seg& sg = segs[slots[find_slot(slots, nslots, blockIdx.x)].seg];
  const uint64_t* __restrict__ keys = sg.skeys;
  const uint32_t* __restrict__ vals = sg.svals;
  const uint32_t n = sg.n;
  const int Lb = sg.Lb, Ls = sg.Ls;
  const LevelArrays& lv = sg.lv;
  uint32_t* __restrict__ perm = sg.perm;
  uint64_t* status = sg.bstatus;
  const uint32_t ntiles = sg.btiles;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    s_tile = atomicAdd(&sg.tickets[0], 1u);
    s_abort = failed(st) ? 1u : 0u;
    mbar_init(&s_bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (s_abort) return;  // an earlier kernel failed: leave the outputs alone
  const uint32_t tile = s_tile;
  const int64_t t0 = (int64_t)tile * kBoxTile;
  const int64_t nn = n;
  const int jend = (int)((nn - t0) < kWin ? (nn - t0) : kWin);  // valid window points
  {
    // The window by bulk copy (TMA): keys of points [t0 - 2, t0 + jend) and
    // indices of [t0, t0 + jend).  Set bases are multiples of 4 slots and t0
    // of 4096, so both sources start 16-byte aligned; an odd key and up to
    // three indices at the end come by plain loads.  Slots outside the data
    // are never read (every use is bounded by jend).
    const int64_t g0 = t0 >= 2 ? t0 - 2 : 0;
    const uint32_t nk = (uint32_t)(t0 + jend - g0), nk_bulk = nk & ~1u;
    const uint32_t nv = (uint32_t)jend, nv_bulk = nv & ~3u;
    uint64_t* kdst = s_key + (g0 - (t0 - 2));
    if (threadIdx.x == 0) {
      mbar_expect_tx(&s_bar, nk_bulk * 8u + nv_bulk * 4u);
      if (nk_bulk) bulk_load(kdst, keys + g0, nk_bulk * 8u, &s_bar);
      if (nv_bulk) bulk_load(s_val, vals + t0, nv_bulk * 4u, &s_bar);
    }
    if (threadIdx.x == 32 && (nk & 1u)) kdst[nk - 1] = keys[g0 + nk - 1];
    if (threadIdx.x >= 64 && threadIdx.x < 64 + (nv - nv_bulk))
      s_val[nv_bulk + threadIdx.x - 64] = vals[t0 + nv_bulk + threadIdx.x - 64];
    const bool ok = mbar_wait(&s_bar, 0, st, wait_ns);
    if (__syncthreads_or(!ok)) {
      mbar_wait(&s_bar, 0, st, wait_ns);  // let the copy land before the block leaves
      return;
    }
  }
  // dd[j]: the point opens a box at every level >= dd[j].  Past the end of
  // the data every slot reads 0, which ends every box walk there.
  for (int j = threadIdx.x; j < kWin; j += kBoxThreads)
    s_dd[j] = (j >= jend || t0 + j == 0) ? 0u : (uint8_t)first_diff_level(sk[j + 1], sk[j]);
  __syncthreads();

  // Level-Lb box starts among this thread's points 8t .. 8t+7.
  uint32_t mask = 0;
  {
    static_assert(kBoxItems == 8, "one 8-byte read of the level bytes per thread");
    const uint2 w = *reinterpret_cast<const uint2*>(s_dd + threadIdx.x * kBoxItems);
    const uint64_t w64 = ((uint64_t)w.y << 32) | w.x;
#pragma unroll
    for (int k = 0; k < kBoxItems; ++k) {
      const uint32_t d = (uint32_t)(w64 >> (8 * k)) & 0xffu;
      if (threadIdx.x * kBoxItems + k < jend && d <= (uint32_t)Lb) mask |= 1u << k;
    }
  }
  const uint32_t c = __popc(mask);
  uint32_t x = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_wtot[warp] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int w = 0; w < W; ++w) {
      const uint32_t v = s_wtot[w];
      s_wtot[w] = run;
      run += v;
    }
    s_ttot = run;
    st_relaxed(status + tile, (tile == 0 ? kFlagIncl : kFlagAgg) | run);
  }

  // Finishing sort inside the level-Ls boxes that START in this tile,
  // including their points in the halo past the tile's end (a box begun in
  // an earlier tile is that tile's).  A point's rank counts the points of its
  // box that come before it in (full key, original index) order; the order
  // the radix passes left inside a box does not matter.  Each warp takes 32 consecutive
  // points; box bounds inside the warp come from one ballot of box starts.
  // This runs between publishing the aggregate and reading the earlier
  // tiles' words, which gives them time to publish.
  if (Ls >= kMaxLevel || sg.exact) {
    // Sorted with stable passes on all 63 key bits, or on exactly the bits
    // that the order asks for: the order is already final.
    const int own = jend < kBoxTile ? jend : kBoxTile;
    for (int j = threadIdx.x; j < own; j += kBoxThreads) perm[t0 + j] = s_val[j];
  } else {
    const uint32_t lt = lanemask_lt();
    bool long_box = false;
    const int lowbits = 63 - 3 * Ls;
    const uint64_t lowmask = lowbits >= 64 ? ~0ull : ((1ull << lowbits) - 1ull);
    for (int c0 = warp * 32; c0 < jend; c0 += W * 32) {
      const int j = c0 + lane;
      const bool in = j < jend;
      const bool start = in && s_dd[j] <= (uint32_t)Ls;
      const uint32_t f = __ballot_sync(0xffffffffu, start);
      int a;  // box start: last start at or before this lane, else walk back
      const uint32_t le = f & (lt | (1u << lane));
      if (le) {
        a = c0 + 31 - __clz(le);
      } else {
        a = c0;
        while (a > 0 && s_dd[a] > (uint32_t)Ls) --a;
      }
      int b;  // box end: next start after this lane, else walk on
      const uint32_t gt = f & ~(lt | (1u << lane));
      if (gt) {
        b = c0 + __ffs(gt) - 1;
      } else {
        b = c0 + 32;
        while (b < jend && s_dd[b] > (uint32_t)Ls) ++b;
        if (b > jend) b = jend;
      }
      if (!in) continue;
      if (a >= kBoxTile) continue;                                // the next tile's box
      if (a == 0 && t0 > 0 && s_dd[0] > (uint32_t)Ls) continue;  // an earlier tile's box
      if (b == jend && t0 + jend < nn) {
        long_box = true;  // runs past the window: the host redoes the order
        continue;
      }
      uint32_t r = 0;
      if (b - a > 1) {
        // within a box the top bits agree: order by (low key bits, index)
        const uint64_t mine = sk[j + 1] & lowmask;
        const uint32_t vj = s_val[j];
        for (int q = a; q < b; ++q) {
          const uint64_t kq = sk[q + 1] & lowmask;
          r += (kq < mine) || (kq == mine && s_val[q] < vj);
        }
      }
      perm[t0 + a + r] = s_val[j];
    }
    if (long_box) {
      atomicExch(&st->seg_long, 1u);
      atomicExch(sg.seg_long, 1u);
    }
  }

  // Windowed look-back over the earlier tiles.
  if (warp == 0) {
    uint64_t prev = 0;
    if (tile > 0) {
      prev = lookback_warp(status, tile, 1, st, wait_ns);
      if (lane == 0) st_relaxed(status + tile, kFlagIncl | (prev + s_ttot));
    }
    if (lane == 0) s_texcl = (uint32_t)prev;
  }
  __syncthreads();
  if (threadIdx.x == 0 && tile > 0 && ld_relaxed_u32(&st->abort)) s_abort = 1;
  __syncthreads();
  if (s_abort) return;  // a wait gave up: ranks may be wrong, write nothing
  if (tile == ntiles - 1 && threadIdx.x == 0) {
    const uint32_t nb = s_texcl + s_ttot;
    sg.nbox[Lb] = nb;
    if (nb <= lv.cap[Lb]) lv.off[Lb][nb] = n;
  }
  // Level-Lb keys and bookmarks.
  const int shift = 63 - 3 * Lb;
  uint32_t rank = s_texcl + s_wtot[warp] + (x - c);
  const uint32_t cap = lv.cap[Lb];
  while (mask) {
    const int k = __ffs(mask) - 1;
    mask &= mask - 1;
    const int j = threadIdx.x * kBoxItems + k;
    if (rank < cap) {
      lv.key[Lb][rank] = Lb == 0 ? 0ull : sk[j + 1] >> shift;
      lv.off[Lb][rank] = (uint32_t)(t0 + j);
    }
    ++rank;
  }
}

// Levels 0..Lb-1 (and the parents of the level-Lb boxes) from the level-Lb
// boxes: box b opens a level-l box exactly when its key differs from box
// b-1's in the level-l prefix.  A multi-level prefix sum over the boxes (one
// decoupled look-back chain per level) gives each start its rank.
// NL: a bound on the sets' box depths (Lb <= NL), so that the per-level
// loops, unrolled, cover only the levels in use.
// Four blocks an SM for trees up to level 8 (a few spilled registers): its
// look-back waits hide better; deeper trees keep their registers.
template <int NL>
__global__ void __launch_bounds__(kBoxThreads, NL <= 8 ? 4 : 1) coarse_boxes_kernel(const Seg* __restrict__ segs,
                                                                   const Slot* __restrict__ slots,
                                                                   uint32_t nslots, DevStatus* st,
                                                                   uint64_t wait_ns) {
  constexpr int W = kBoxThreads / 32;
  __shared__ uint32_t s_tile, s_abort;
  __shared__ uint32_t s_wtot[W][kLevels];
  __shared__ uint32_t s_texcl[kLevels];
  __shared__ uint32_t s_ttot[kLevels];
  __shared__ uint64_t s_key[kBoxTile + 1];  // s_key[j + 1] = level-Lb key of box t0 + j
  const Seg& sg = segs[slots[find_slot(slots, nslots, blockIdx.x)].seg];
  const int Lb = sg.Lb;
  const LevelArrays& lv = sg.lv;
  const uint32_t n = sg.n;
  uint64_t* status = sg.cstatus;
  uint32_t* nbox = sg.nbox;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    s_tile = atomicAdd(&sg.tickets[1], 1u);
    s_abort = failed(st) ? 1u : 0u;
  }
  __syncthreads();
  if (s_abort || Lb < 1) return;
  const uint32_t nb = nbox[Lb] < lv.cap[Lb] ? nbox[Lb] : lv.cap[Lb];
  const uint32_t ntiles = nb == 0 ? 1u : (nb + kBoxTile - 1) / kBoxTile;
  const uint32_t tile = s_tile;
  if (tile >= ntiles) return;  // the grid is sized for the capacity
  const int64_t t0 = (int64_t)tile * kBoxTile;
  const uint64_t* kLb = lv.key[Lb];
  const int up = 63 - 3 * Lb;  // level-Lb key -> full-key position
  for (int j = threadIdx.x; j < kBoxTile + 1; j += kBoxThreads) {
    const int64_t b = t0 - 1 + j;
    s_key[j] = (b >= 0 && b < (int64_t)nb) ? kLb[b] << up : 0ull;
  }
  __syncthreads();
  uint32_t dd[kBoxItems];
#pragma unroll
  for (int k = 0; k < kBoxItems; ++k) {
    const int j = threadIdx.x * kBoxItems + k;
    const int64_t b = t0 + j;
    dd[k] = b >= (int64_t)nb ? 0xffu : (b == 0 ? 0u : first_diff_level(s_key[j + 1], s_key[j]));
  }
  uint32_t lex[NL];
#pragma unroll
  for (int l = 0; l < NL; ++l) {
    lex[l] = 0;
    if (l < Lb) {
      uint32_t c = 0;
#pragma unroll
      for (int k = 0; k < kBoxItems; ++k) c += (dd[k] <= (uint32_t)l);
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
  for (int l = warp; l < Lb; l += W) {
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
    uint64_t prev = 0;
    if (tile > 0) {
      prev = lookback_warp(status + l, tile, kLevels, st, wait_ns);
      if (lane == 0)
        st_relaxed(status + (uint64_t)tile * kLevels + l, kFlagIncl | (prev + s_ttot[l]));
    }
    if (lane == 0) s_texcl[l] = (uint32_t)prev;
  }
  __syncthreads();
  if (threadIdx.x == 0 && tile > 0 && ld_relaxed_u32(&st->abort)) s_abort = 1;
  __syncthreads();
  if (s_abort) return;  // a wait gave up: ranks may be wrong, write nothing
  if (tile == ntiles - 1 && threadIdx.x == 0) {
    for (int l = 0; l < Lb; ++l) {
      const uint32_t c = s_texcl[l] + s_ttot[l];
      nbox[l] = c;
      if (c <= lv.cap[l]) lv.off[l][c] = n;
      if (c <= lv.cap[l]) lv.child[l][c] = l + 1 < Lb ? s_texcl[l + 1] + s_ttot[l + 1] : nb;
    }
  }
  uint32_t run[NL];
#pragma unroll
  for (int l = 0; l < NL; ++l) run[l] = (l < Lb) ? s_texcl[l] + s_wtot[warp][l] + lex[l] : 0u;
#pragma unroll
  for (int k = 0; k < kBoxItems; ++k) {
    const int j = threadIdx.x * kBoxItems + k;
    const int64_t b = t0 + j;
    if (b >= (int64_t)nb) continue;
    const uint32_t dk = dd[k];
    const uint64_t key = s_key[j + 1];
    // parent of the level-Lb box: the level-(Lb-1) box holding it
    if (Lb >= 1) {
      uint32_t pr = 0;
#pragma unroll
      for (int l = 0; l < NL; ++l)
        if (l == Lb - 1) pr = dk <= (uint32_t)l ? run[l] : run[l] - 1u;
      lv.parent[Lb][b] = pr;
      if (dk <= (uint32_t)(Lb - 1) && pr < lv.cap[Lb - 1]) lv.child[Lb - 1][pr] = (uint32_t)b;
    }
    if (dk < (uint32_t)Lb) {
      const uint32_t off = lv.off[Lb][b];
#pragma unroll
      for (int l = 0; l < NL; ++l) {
        if (l < Lb && (uint32_t)l >= dk && run[l] < lv.cap[l]) {
          const uint32_t rk = run[l];
          lv.key[l][rk] = l == 0 ? 0ull : key >> (63 - 3 * l);
          lv.off[l][rk] = off;
          if (l >= 1) {
            const bool up_starts = dk <= (uint32_t)(l - 1);
            lv.parent[l][rk] = up_starts ? run[l - 1] : run[l - 1] - 1u;
            if (up_starts && run[l - 1] < lv.cap[l - 1]) lv.child[l - 1][run[l - 1]] = rk;
          }
        }
      }
    }
#pragma unroll
    for (int l = 0; l < NL; ++l)
      if (l < Lb && (uint32_t)l >= dk) ++run[l];
  }
}

uint32_t coarse_tiles(uint32_t cap) {
  const uint64_t t = ((uint64_t)cap + kBoxTile - 1) / kBoxTile;
  return t == 0 ? 1u : (uint32_t)t;
}

void launch_finish_boxes(const Seg* segs, const Slot* slots, uint32_t nslots, uint32_t units,
                         DevStatus* st, uint64_t wait_ns, cudaStream_t s) {
  if (units == 0) return;
  // once per process (thread-safe static initialisation)
  static const bool attr = [] {
    cudaFuncSetAttribute(finish_boxes_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kBoxSmem);
    return true;
  }();
  (void)attr;
  finish_boxes_kernel<<<units, kBoxThreads, kBoxSmem, s>>>(segs, slots, nslots, st, wait_ns);
}

void launch_coarse_boxes(const Seg* segs, const Slot* slots, uint32_t nslots, uint32_t units,
                         int max_lb, DevStatus* st, uint64_t wait_ns, cudaStream_t s) {
  if (units == 0) return;
  if (max_lb <= 8)
    coarse_boxes_kernel<8><<<units, kBoxThreads, 0, s>>>(segs, slots, nslots, st, wait_ns);
  else if (max_lb <= 12)
    coarse_boxes_kernel<12><<<units, kBoxThreads, 0, s>>>(segs, slots, nslots, st, wait_ns);
  else if (max_lb <= 16)
    coarse_boxes_kernel<16><<<units, kBoxThreads, 0, s>>>(segs, slots, nslots, st, wait_ns);
  else
    coarse_boxes_kernel<kLevels><<<units, kBoxThreads, 0, s>>>(segs, slots, nslots, st, wait_ns);
}

// ---------------------------------------------------------------------------
// Child-occupancy byte of every box of levels 0..Lb-1 of the sets that serve
// as sources: bit o is set when the child in octant o (x + 2y + 4z) is
// non-empty.  Lists use it to enumerate the children of a parent-level
// neighbour without reading their keys.  A set owns a run of units (blocks)
// in proportion to its size; each unit takes a strided share of every level.
__global__ void __launch_bounds__(256) occupancy_kernel(const Seg* __restrict__ segs,
                                                        const Slot* __restrict__ slots,
                                                        uint32_t nslots, uint32_t unit_first,
                                                        const DevStatus* st) {
  if (failed(st)) return;
  const uint32_t unit = blockIdx.x + unit_first;
  const uint32_t k = find_slot(slots, nslots, unit);
  const Seg& sg = segs[slots[k].seg];
  const uint32_t u = unit - slots[k].unit0, units = slots[k].aux0;
  for (int l = 0; l < sg.Lb; ++l) {
    const uint32_t nb = sg.nbox[l] < sg.lv.cap[l] ? sg.nbox[l] : sg.lv.cap[l];
    const uint32_t* ch = sg.lv.child[l];
    const uint64_t* ck = sg.lv.key[l + 1];
    const uint32_t nbc = sg.nbox[l + 1] < sg.lv.cap[l + 1] ? sg.nbox[l + 1] : sg.lv.cap[l + 1];
    uint8_t* occ = sg.lv.occ[l];
    for (uint32_t b = u * blockDim.x + threadIdx.x; b < nb; b += units * blockDim.x) {
      uint32_t m = 0;
      const uint32_t c1 = ch[b + 1] < nbc ? ch[b + 1] : nbc;  // (never above nbc in a whole tree)
      for (uint32_t c = ch[b]; c < c1; ++c) m |= 1u << (uint32_t)(ck[c] & 7u);
      occ[b] = (uint8_t)m;
    }
  }
}

void launch_occupancy(const Seg* segs, const Slot* slots, uint32_t nslots, uint32_t units,
                      uint32_t unit_first, DevStatus* st, cudaStream_t s) {
  if (units == 0) return;
  occupancy_kernel<<<units, 256, 0, s>>>(segs, slots, nslots, unit_first, st);
}

uint32_t occupancy_units(uint32_t n) { return 1u + n / 16384u; }

// ---------------------------------------------------------------------------
// Cluster-size depth (Sec. 2.1: the smallest level whose boxes hold at most
// s points).  In an order sorted by the top 3*Ls key bits, a level-l box
// (l <= Ls) is a contiguous run, so it holds more than s points exactly when
// some sorted point i and point i + s share it, i.e. when their keys agree on
// the level-l prefix.  One pass over the pairs (i, i + s) therefore gives,
// for every set, D = max_i (deepest level shared by points i and i + s),
// capped at Ls; written as D + 1 by atomicMax into out[set] (zeroed, so 0
// means "no pair": the set has at most s points).  Units are sort tiles.
__global__ void __launch_bounds__(256) depth_kernel(const Seg* __restrict__ segs,
                                                    const Slot* __restrict__ slots,
                                                    uint32_t nslots, uint32_t s,
                                                    uint32_t* __restrict__ out,
                                                    const DevStatus* st) {
  if (failed(st)) return;
  const uint32_t k = find_slot(slots, nslots, blockIdx.x);
  const uint32_t set = slots[k].seg;
  const Seg& sg = segs[set];
  const uint64_t t0 = (uint64_t)(blockIdx.x - slots[k].unit0) * sg.tile;
  const uint64_t npairs = sg.n > s ? (uint64_t)sg.n - s : 0;
  const uint64_t* keys = sg.skeys;
  const uint32_t cap = (uint32_t)sg.Ls;
  uint32_t m = 0;
  for (uint64_t i = t0 + threadIdx.x; i < t0 + sg.tile && i < npairs; i += blockDim.x) {
    const uint32_t shared = first_diff_level(keys[i], keys[i + s]) - 1u;  // 0..21
    const uint32_t v = (shared < cap ? shared : cap) + 1u;
    m = v > m ? v : m;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint32_t y = __shfl_xor_sync(0xffffffffu, m, o);
    m = y > m ? y : m;
  }
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out + set, m);
}

void launch_depth(const Seg* segs, const Slot* slots, uint32_t nslots, uint32_t units, uint32_t s,
                  uint32_t* out, DevStatus* st, cudaStream_t stream) {
  if (units == 0) return;
  depth_kernel<<<units, 256, 0, stream>>>(segs, slots, nslots, s, out, st);
}

}  // namespace fmm
