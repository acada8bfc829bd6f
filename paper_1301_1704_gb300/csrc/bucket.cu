// bucket.cu -- the point order and every box level of a fixed-depth build,
// by bucketing the points on coarse cells (sort kind FMM_SORT_BUCKET).
//
// Alg. 1 orders the points with a histogram of the finest boxes, atomic
// ranks and one move; Alg. 3 scans that histogram for the bookmarks.  Here
// the same ideas are applied at a coarse level, where the histograms fit in
// shared memory, and inside each sub-cell, where the rest of the order is
// finished in shared memory by one block that also emits the boxes:
//
//   scatter  per tile of points: a histogram of the level-(bl + 1) cells,
//            the "sub-cells", in shared memory; one atomic per (tile,
//            non-empty sub-cell) reserves the tile's range inside the
//            sub-cell (Alg. 1's atomic ranks, taken per tile and sub-cell
//            instead of per point); then each point becomes one 8-byte item
//            -- the key bits below its sub-cell, left-aligned, over the point
//            index -- at the next slot of the tile's range in its sub-cell;
//   plan     per set: the prefix sum of the sub-cell counts -- their
//            bookmarks (Alg. 3) -- and the list of non-empty level-bl cells,
//            the "buckets", each with its 8 sub-cells;
//   boxes    per sub-cell, one block: a counting sort of its items on their
//            next key bits, whose group counts also give the non-empty boxes
//            of the next three levels with their ranks and bookmarks (Alg. 3
//            inside the sub-cell); each point's rank inside its group by (key
//            bits, index) -- the order (Morton key, original index) -- gives
//            its permutation entry; one decoupled look-back over the sub-cells
//            per level gives the sub-cell's first box ranks; deeper levels,
//            if any, come from the first differing level of the sorted items.
//
// Traffic per point: coordinates read once (12 bytes; the scatter's second
// read of a tile comes from L2), the item written and read once (8 + 8), the
// permutation written (4).
#include "fmm_internal.cuh"

namespace fmm {

namespace {

__device__ __forceinline__ uint32_t bk_cells(int bl) { return 1u << (3 * bl); }

// Bit i of v (v < 32) moved to bit 3i: the cell of level <= 5 from the top
// bits of the three cell coordinates.
__device__ __forceinline__ uint32_t spread5(uint32_t v) {
  return (v & 1u) | ((v & 2u) << 2) | ((v & 4u) << 4) | ((v & 8u) << 6) | ((v & 16u) << 8);
}

// Bit i of a 21-bit value moved to bit 3i, by five shift-or-mask steps
// (each halves the width of the bit groups still to be spread: 16, 8, 4, 2,
// 1 bits, the masks keeping every group at its place).
__device__ __forceinline__ uint64_t spread21(uint32_t x) {
  uint64_t v = x & 0x1fffffu;
  v = (v | (v << 32)) & 0x001f00000000ffffull;
  v = (v | (v << 16)) & 0x001f0000ff0000ffull;
  v = (v | (v << 8)) & 0x100f00f00f00f00full;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}
// The same key as morton_key (same quantisation).
__device__ __forceinline__ uint64_t spread_key(float x, float y, float z, bool* ok) {
  uint32_t qx, qy, qz;
  const bool a = quantize21(x, &qx), b = quantize21(y, &qy), c = quantize21(z, &qz);
  *ok = a && b && c;
  return spread21(qx) | (spread21(qy) << 1) | (spread21(qz) << 2);
}

// Cell of level bl (<= 5) of a point, and whether it lies in [0, 1]^3.
__device__ __forceinline__ uint32_t cell_of(float x, float y, float z, int bl, bool* ok) {
  uint32_t qx, qy, qz;
  const bool a = quantize21(x, &qx), b = quantize21(y, &qy), c = quantize21(z, &qz);
  *ok = a && b && c;
  const int sh = 21 - bl;
  return spread5(qx >> sh) | (spread5(qy >> sh) << 1) | (spread5(qz >> sh) << 2);
}

// First level at which two items of one sub-cell of level bl1 differ (22:
// not within the kept key bits).  The top three item bits are level bl1 + 1.
__device__ __forceinline__ uint32_t bk_diff_level(uint64_t a, uint64_t b, uint64_t keep, int bl1) {
  const uint64_t z = (a ^ b) & keep;
  if (z == 0) return 22u;
  const uint32_t d = (uint32_t)bl1 + 1u + (uint32_t)__clzll((long long)z) / 3u;
  return d < 22u ? d : 22u;
}

// Four 16-bit counters in a word: ones in fields a..b (b - a <= 3).
__device__ __forceinline__ uint64_t fields(int a, int b) {
  if (b < a) return 0ull;
  const uint64_t ones = 0x0001000100010001ull;
  return (ones >> (16 * (3 - (b - a)))) << (16 * a);
}
__device__ __forceinline__ uint32_t field(uint64_t w, int f) {
  return (uint32_t)(w >> (16 * f)) & 0xffffu;
}

}  // namespace

// ---------------------------------------------------------------------------
// plan: per set (one block each), the sub-cells' bookmarks and the buckets
// (the non-empty level-bl cells) with their sub-cells.
__global__ void __launch_bounds__(kBkPlanThreads) bucket_plan_kernel(const BkSet* __restrict__ bsets,
                                                                    DevStatus* st) {
  constexpr int W = kBkPlanThreads / 32;
  constexpr int kPer = kBkMaxCells / kBkPlanThreads;  // cells per thread, at most
  __shared__ uint64_t s_w[W];
  __shared__ uint32_t s_max[W];
  if (failed(st)) return;
  const BkSet& S = bsets[blockIdx.x];
  const uint32_t cells = bk_cells(S.bl);
  const uint32_t per = (cells + kBkPlanThreads - 1) / kBkPlanThreads;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t c0 = threadIdx.x * per;
  uint32_t v[kPer];
  uint64_t sum = 0;  // low 32 bits: points; high 32 bits: non-empty cells
  uint32_t mx = 0;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    v[k] = 0;
    if ((uint32_t)k < per && c0 + k < cells) {
      const uint4 lo = *reinterpret_cast<const uint4*>(S.sct + 8 * (c0 + k));
      const uint4 hi = *reinterpret_cast<const uint4*>(S.sct + 8 * (c0 + k) + 4);
      v[k] = lo.x + lo.y + lo.z + lo.w + hi.x + hi.y + hi.z + hi.w;
    }
    sum += (uint64_t)v[k] | ((uint64_t)(v[k] != 0) << 32);
    mx = v[k] > mx ? v[k] : mx;
  }
  uint64_t x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint32_t y = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = y > mx ? y : mx;
  }
  if (lane == 31) s_w[warp] = x;
  if (lane == 0) s_max[warp] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t run = 0;
    uint32_t m = 0;
    for (int w = 0; w < W; ++w) {
      const uint64_t c = s_w[w];
      s_w[w] = run;
      run += c;
      m = s_max[w] > m ? s_max[w] : m;
    }
    const uint32_t nbk = (uint32_t)(run >> 32);
    S.info[0] = nbk;
    S.info[1] = m;
    S.boff[nbk] = S.n;
  }
  __syncthreads();
  uint64_t e = s_w[warp] + x - sum;
  uint32_t off = (uint32_t)e, b = (uint32_t)(e >> 32);
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    if ((uint32_t)k < per && c0 + k < cells) {
      const uint32_t c = c0 + k;
      uint32_t so = off;  // the cell's sub-cells, in octant order
      for (int q = 0; q < 8; ++q) {
        const uint32_t n8 = S.sct[8 * c + q];
        if (v[k]) {
          S.soff[8 * b + q] = so;
          S.scnt[8 * b + q] = n8;
        }
        so += n8;
      }
      if (v[k]) {
        S.bcell[b] = c;
        S.boff[b] = off;
        ++b;
      }
      off += v[k];
    }
  }
}

// ---------------------------------------------------------------------------
// scatter: per tile of points, in one pass over the tile: the histogram of its
// sub-cells (level bl + 1) in shared memory; one atomic per (tile, non-empty
// sub-cell) on the sub-cell's total reserves the tile's range inside the
// sub-cell (Alg. 1's atomic ranks, taken per tile and sub-cell instead of per
// point); then each point (its coordinates read again, from L2) becomes one
// 8-byte item -- the key bits below its sub-cell, left-aligned, over the
// point index -- at the next slot of that range (a shared-memory atomic per
// point).  Sub-cell c's items occupy slots [c kBkCap, c kBkCap + count): the
// totals are not known while the tiles run, so every sub-cell has room for
// the most points one block sorts; a fuller sub-cell keeps only what fits
// (the boxes stage then stops the build and the host redoes the set by the
// radix path).  The order inside a sub-cell is left to the atomics: the
// boxes stage orders each sub-cell by whole item.  The stores of a warp land
// in many sub-cells, each a part of a 32-byte sector that the tile and its
// neighbours in tile order fill over time; one block an SM (few tiles in
// flight) and short tiles keep the partly written sectors few, so that most
// of them fill in L2 before they are evicted.
constexpr int kScThreads = 1024;
constexpr int kScGroups = 2;  // groups of 4 points a thread loads ahead

__global__ void __launch_bounds__(kScThreads, 1) bucket_scatter_kernel(
    const BkSet* __restrict__ bsets, const Slot* __restrict__ slots, uint32_t nslots,
    uint32_t t_first, DevStatus* st) {
  extern __shared__ uint32_t s_at[];  // per sub-cell: the tile's count, then its next slot
  if (failed(st)) return;
  const uint32_t unit = blockIdx.x + t_first;  // (a launch may start past unit 0)
  const Slot sl = slots[find_slot(slots, nslots, unit)];
  const BkSet& S = bsets[sl.seg];
  const uint32_t t = unit - sl.unit0;
  const int bl1 = S.bl + 1;
  const uint32_t subs = bk_cells(bl1);
  const int sh = 63 - 3 * bl1, lsh = 1 + 3 * bl1;
  const uint64_t keep1 = S.keep << 3;
  for (uint32_t c = threadIdx.x; c < subs; c += blockDim.x) s_at[c] = 0;
  __syncthreads();
  const uint64_t base = (uint64_t)t * S.tile;
  const uint32_t cnt = (uint32_t)((S.n - base) < (uint64_t)S.tile ? (S.n - base) : S.tile);
  const float* xyz = S.xyz + 3 * base;
  const bool vec = (reinterpret_cast<uintptr_t>(S.xyz) & 15u) == 0;
  const float4* v4 = reinterpret_cast<const float4*>(xyz);  // 4 points = 3 float4
  const uint32_t ng = vec ? cnt / 4 : 0u, done = 4 * ng;
  bool bad = false;

  // 1. the tile's histogram
  for (uint32_t g0 = 0; g0 < ng; g0 += kScGroups * kScThreads) {
    float4 a[kScGroups], b[kScGroups], c[kScGroups];
#pragma unroll
    for (int u = 0; u < kScGroups; ++u) {
      const uint32_t g = g0 + u * kScThreads + threadIdx.x;
      if (g < ng) {
        a[u] = __ldcg(v4 + 3 * g);
        b[u] = __ldcg(v4 + 3 * g + 1);
        c[u] = __ldcg(v4 + 3 * g + 2);
      }
    }
#pragma unroll
    for (int u = 0; u < kScGroups; ++u) {
      const uint32_t g = g0 + u * kScThreads + threadIdx.x;
      if (g < ng) {
        bool ok0, ok1, ok2, ok3;
        atomicAdd(&s_at[cell_of(a[u].x, a[u].y, a[u].z, bl1, &ok0)], 1u);
        atomicAdd(&s_at[cell_of(a[u].w, b[u].x, b[u].y, bl1, &ok1)], 1u);
        atomicAdd(&s_at[cell_of(b[u].z, b[u].w, c[u].x, bl1, &ok2)], 1u);
        atomicAdd(&s_at[cell_of(c[u].y, c[u].z, c[u].w, bl1, &ok3)], 1u);
        bad |= !(ok0 && ok1 && ok2 && ok3);
      }
    }
  }
  for (uint32_t j = done + threadIdx.x; j < cnt; j += kScThreads) {
    bool ok;
    atomicAdd(&s_at[cell_of(xyz[3 * j], xyz[3 * j + 1], xyz[3 * j + 2], bl1, &ok)], 1u);
    bad |= !ok;
  }
  if (bad) set_error(st, FMM_ERR_DOMAIN);
  __syncthreads();

  // 2. the tile's ranges: four atomics of a thread in flight together
  for (uint32_t c0 = 0; c0 < subs; c0 += 4 * kScThreads) {
    uint32_t hh[4], r[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint32_t c = c0 + u * kScThreads + threadIdx.x;
      hh[u] = c < subs ? s_at[c] : 0u;
      r[u] = hh[u] ? atomicAdd(&S.sct[c], hh[u]) : 0u;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint32_t c = c0 + u * kScThreads + threadIdx.x;
      if (hh[u]) s_at[c] = c * (uint32_t)kBkCap + r[u];
    }
  }
  __syncthreads();

  // 3. the items, each at the next slot of its sub-cell's range
  uint64_t* const items = S.items;
  auto put = [&](float x, float y, float z, uint32_t j) {
    bool ok;
    const uint64_t key = spread_key(x, y, z, &ok);
    const uint32_t sc = (uint32_t)(key >> sh);
    const uint32_t pos = atomicAdd(&s_at[sc], 1u);
    if (pos < (sc + 1u) * (uint32_t)kBkCap)  // (a sub-cell over its room keeps what fits)
      items[pos] = ((key << lsh) & keep1) | (uint32_t)(base + j);
  };
  for (uint32_t g0 = 0; g0 < ng; g0 += kScGroups * kScThreads) {
    float4 a[kScGroups], b[kScGroups], c[kScGroups];
#pragma unroll
    for (int u = 0; u < kScGroups; ++u) {
      const uint32_t g = g0 + u * kScThreads + threadIdx.x;
      if (g < ng) {
        a[u] = __ldcs(v4 + 3 * g);
        b[u] = __ldcs(v4 + 3 * g + 1);
        c[u] = __ldcs(v4 + 3 * g + 2);
      }
    }
#pragma unroll
    for (int u = 0; u < kScGroups; ++u) {
      const uint32_t g = g0 + u * kScThreads + threadIdx.x;
      if (g < ng) {
        put(a[u].x, a[u].y, a[u].z, 4 * g);
        put(a[u].w, b[u].x, b[u].y, 4 * g + 1);
        put(b[u].z, b[u].w, c[u].x, 4 * g + 2);
        put(c[u].y, c[u].z, c[u].w, 4 * g + 3);
      }
    }
  }
  for (uint32_t j = done + threadIdx.x; j < cnt; j += kScThreads)
    put(xyz[3 * j], xyz[3 * j + 1], xyz[3 * j + 2], j);
}

// ---------------------------------------------------------------------------
// boxes: one block per sub-cell, in sub-cell order (tickets).

// Block-wide sums of one packed word per thread: the exclusive prefix of
// this thread (returned) and the total (*tot).
template <int W>
__device__ __forceinline__ uint64_t block_scan64(uint64_t v, uint64_t* s_w, uint64_t* tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  if (warp == 0) {  // the warps' sums, scanned by one warp
    const uint64_t w = lane < W ? s_w[lane] : 0ull;
    uint64_t y = w;
#pragma unroll
    for (int o = 1; o < W; o <<= 1) {
      const uint64_t z = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += z;
    }
    if (lane < W) s_w[lane] = y - w;
    if (lane == W - 1) s_w[W] = y;
  }
  __syncthreads();
  const uint64_t r = s_w[warp] + x - v;
  *tot = s_w[W];
  __syncthreads();  // s_w is reused by the next call
  return r;
}

// Flags and exclusive ranks of the non-empty cells of the levels bl1 + m
// (m = 1 .. kBkHistLevels) inside a sub-cell: level m at [(8^m - 8) / 7, ...).
constexpr int kBkHistLevels = 3;
constexpr int kBkHistCells = 8 + 64 + 512;
__device__ __forceinline__ int hoff(int m) { return ((1 << (3 * m)) - 8) / 7; }

__global__ void __launch_bounds__(kBkThreads, 3) bucket_boxes_kernel(
    const BkSet* __restrict__ bsets, const Seg* __restrict__ segs, const Slot* __restrict__ slots,
    uint32_t nslots, uint32_t* ticket, DevStatus* st, uint64_t wait_ns) {
  constexpr int W = kBkThreads / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* B = reinterpret_cast<uint64_t*>(smem);          // the items, by group
  uint32_t* gs = reinterpret_cast<uint32_t*>(B + kBkCap);  // group counts, then starts [2^D + 1]
  uint16_t* ord = reinterpret_cast<uint16_t*>(gs + (1 << kBkGroupBits) + 4);  // sorted k: B[ord[k]]
  __shared__ uint32_t s_t, s_abort;
  __shared__ uint64_t s_w[W + 1];
  __shared__ uint32_t s_R[kLevels], s_C[kLevels];
  __shared__ __align__(8) uint8_t s_fl[kBkHistCells];  // non-empty flags
  __shared__ uint16_t s_pre[kBkHistCells];              // exclusive ranks
  __shared__ uint64_t* s_lkey[kLevels];                  // the output level arrays
  __shared__ uint32_t *s_loff[kLevels], *s_lpar[kLevels], *s_lchd[kLevels];
  __shared__ uint32_t s_lcap[kLevels];

  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) {
    s_t = atomicAdd(ticket, 1u);
    s_abort = failed(st) ? 1u : 0u;
  }
  __syncthreads();
  if (s_abort) return;  // an earlier kernel failed: leave the outputs alone
  const uint32_t t = s_t;
  const Slot sl = slots[find_slot(slots, nslots, t)];
  const BkSet& S = bsets[sl.seg];
  const uint32_t u = t - sl.unit0;  // sub-cell slot of the set: bucket b, octant j
  const uint32_t b = u >> 3, j = u & 7u;
  const uint32_t nbk = S.info[0];
  if (b >= nbk) return;  // past the set's last non-empty cell
  const Seg& G = segs[S.seg];
  const int bl = S.bl, bl1 = bl + 1, Lb = S.Lb, ib = S.ib, D = S.D;
  const uint64_t imask = (1ull << ib) - 1ull, keep1 = S.keep << 3;
  const uint32_t nsub = 8 * S.nslot;
  uint64_t* const status = S.status;  // [kLevels][nsub]: one chain of sub-cells per level
  const uint32_t n_j = S.scnt[u], offj = S.soff[u];
  const uint32_t cell = S.bcell[b], cell1 = cell * 8 + j;
  // a non-empty sub-cell precedes this one in the bucket
  const bool sib = __syncthreads_or(tid < (int)j && S.scnt[8 * b + tid] > 0);
  // The first point of the sub-cell opens a box at every level from the
  // first one at which it differs from the point before it in the set.
  uint32_t d0 = 0;
  if (sib) {
    d0 = (uint32_t)bl1;
  } else if (b > 0) {
    const uint32_t x = cell ^ S.bcell[b - 1];  // non-zero: distinct cells
    d0 = (uint32_t)bl - (uint32_t)(31 - __clz((int)x)) / 3u;
  }
  if (n_j > (uint32_t)kBkCap) {
    // More points than a block sorts: the host builds this set again by the
    // radix path.  The build stops here (later kernels see the status and
    // leave their outputs alone); empty counts are published so that later
    // sub-cells do not wait.
    if (tid == 0) {
      atomicOr(G.seg_long, 2u);
      atomicExch(&st->seg_long, 1u);
      set_error(st, kStatusBucketFull);
    }
    for (int l = tid; l <= Lb; l += kBkThreads)
      st_relaxed(status + (uint64_t)l * nsub + u, u == 0 ? kFlagIncl : kFlagAgg);
    return;
  }

  // The output level arrays, read once (their loads overlap the items').
  if (tid <= Lb) {
    s_lkey[tid] = G.lv.key[tid];
    s_loff[tid] = G.lv.off[tid];
    s_lpar[tid] = G.lv.parent[tid];
    s_lchd[tid] = G.lv.child[tid];
    s_lcap[tid] = G.lv.cap[tid];
  }
  uint32_t* const perm = G.perm;

  // 1. The sub-cell's items (all loads in flight together; kept in L2 for
  // the counting sort's scatter, which reads them again).
  const uint64_t* src = S.items + (uint64_t)cell1 * kBkCap;
  const uint32_t ng = 1u << D;
  const int gsh = 64 - D;
  uint32_t rk[kBkItems];
  {
    uint64_t v[kBkItems];
#pragma unroll
    for (int k = 0; k < kBkItems; ++k) {
      const uint32_t p = tid + k * kBkThreads;
      v[k] = p < n_j ? __ldcg(src + p) : 0ull;
    }
    for (uint32_t q = tid; q <= ng; q += kBkThreads) gs[q] = 0;
    __syncthreads();

    // 2. Group counts (the top D item bits) with each point's rank in its
    // group (an unstable counting sort), and the groups' starts.
#pragma unroll
    for (int k = 0; k < kBkItems; ++k) {
      const uint32_t p = tid + k * kBkThreads;
      if (p < n_j) rk[k] = atomicAdd(&gs[D ? (uint32_t)(v[k] >> gsh) : 0u], 1u);
    }
  }
  __syncthreads();
  {
    constexpr int kPer = ((1 << kBkGroupBits) + kBkThreads - 1) / kBkThreads;  // entries a thread
    uint32_t v[kPer], sum = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const uint32_t q = tid * kPer + k;
      v[k] = q < ng ? gs[q] : 0u;
      sum += v[k];
    }
    uint64_t tot;
    uint32_t e = (uint32_t)block_scan64<W>(sum, s_w, &tot);
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const uint32_t q = tid * kPer + k;
      if (q < ng) gs[q] = e;
      e += v[k];
    }
    if (tid == 0) gs[ng] = n_j;
  }
  __syncthreads();

  // 3. The boxes of levels bl1 + 1 .. lh from the group counts (Alg. 3 on
  // the sub-cell): a level-lh cell holds the groups [c << gpc, (c + 1) <<
  // gpc); its flag is set when they hold points, a coarser cell's when one
  // of its 8 children's is; ranks are exclusive counts of set flags.
  const int nm = (Lb - bl1) < kBkHistLevels ? (Lb - bl1) : kBkHistLevels;  // may be <= 0
  const int lh = bl1 + (nm > 0 ? nm : 0);
  const bool deep = Lb > lh;
  if (tid < kLevels) s_C[tid] = (tid <= Lb && tid <= bl1 && n_j > 0 && d0 <= (uint32_t)tid) ? 1u : 0u;
  if (nm > 0) {
    const int gpc = D - 3 * nm;  // group bits below a level-lh cell
    const uint32_t ncell = 1u << (3 * nm);
    if (tid < ncell) s_fl[hoff(nm) + tid] = gs[(tid + 1) << gpc] != gs[tid << gpc];
    __syncthreads();
    for (int m = nm - 1; m >= 1; --m) {
      if (tid < (1u << (3 * m)))
        s_fl[hoff(m) + tid] = *reinterpret_cast<const uint64_t*>(&s_fl[hoff(m + 1) + 8 * tid]) != 0;
      __syncthreads();
    }
    uint64_t c = 0;
    if (tid < ncell)
      for (int m = 1; m <= nm; ++m) {
        const int sh = 3 * (nm - m);
        if ((tid & ((1u << sh) - 1)) == 0) c += (uint64_t)s_fl[hoff(m) + (tid >> sh)] << (16 * (m - 1));
      }
    uint64_t tot;
    const uint64_t ex = block_scan64<W>(c, s_w, &tot);
    if (tid < ncell)
      for (int m = 1; m <= nm; ++m) {
        const int sh = 3 * (nm - m);
        if ((tid & ((1u << sh) - 1)) == 0) s_pre[hoff(m) + (tid >> sh)] = (uint16_t)field(ex, m - 1);
      }
    if (tid == 0)
      for (int m = 1; m <= nm; ++m) s_C[bl1 + m] = field(tot, m - 1);
  }
  __syncthreads();
  // the counts of levels <= lh are final: publish them before the sort
  if (tid <= lh && tid <= Lb)
    st_relaxed(status + (uint64_t)tid * nsub + u, (u == 0 ? kFlagIncl : kFlagAgg) | s_C[tid]);

  // 4. The sort: the counting sort's scatter, then each point's rank in its
  // group by the whole item (key bits, index).  A point's place in the
  // sub-cell is its group's start plus that rank: its permutation entry and
  // its sorted item are written from there.
#pragma unroll
  for (int k = 0; k < kBkItems; ++k) {
    const uint32_t p = tid + k * kBkThreads;
    if (p < n_j) {
      const uint64_t x = __ldcs(src + p);
      B[gs[D ? (uint32_t)(x >> gsh) : 0u] + rk[k]] = x;
    }
  }
  __syncthreads();
  const uint64_t hi = ~imask;
  for (uint32_t p = tid; p < n_j; p += kBkThreads) {
    const uint64_t x = B[p];
    const uint32_t g = D ? (uint32_t)(x >> gsh) : 0u;
    const uint32_t q0 = gs[g], q1 = gs[g + 1];
    uint32_t r = 0;
    for (uint32_t q = q0; q < q1; ++q) r += B[q] < x;
    perm[offj + q0 + r] = (uint32_t)(x & imask);
    ord[q0 + r] = (uint16_t)p;  // the sorted order
  }
  __syncthreads();
  // Items whose kept key bits tie are neighbours in the sorted order.
  bool tie = false;
  if (S.trunc)
    for (uint32_t p = tid + 1; p < n_j; p += kBkThreads) tie |= ((B[ord[p]] ^ B[ord[p - 1]]) & hi) == 0;
  if (S.trunc && __syncthreads_or(tie)) {
    // Points whose kept key bits tie but whose full keys may differ (keys
    // cut short to make room for the index): each tied run is put in (full
    // key, index) order by one thread, the full keys recomputed from the
    // coordinates, and the permutation is written again.  Rare: two points
    // in one cell of level about 17.
    for (uint32_t p = tid + 1; p < n_j; p += kBkThreads) {
      const uint64_t xm = B[ord[p - 1]];
      if (((B[ord[p]] ^ xm) & hi) != 0) continue;
      if (p >= 2 && ((B[ord[p - 2]] ^ xm) & hi) == 0) continue;  // not the run's second point
      const uint32_t q0 = p - 1;
      uint32_t e = p + 1;
      while (e < n_j && ((B[ord[e]] ^ xm) & hi) == 0) ++e;
      if (e - q0 > kBkTieRun) {
        atomicOr(G.seg_long, 1u);  // the host redoes this set's order with a full sort
        atomicExch(&st->seg_long, 1u);
        continue;
      }
      // insertion sort by (full key, index); the run starts in index order
      uint64_t kk[kBkTieRun];
      uint32_t ii[kBkTieRun];
      const uint32_t m = e - q0;
      for (uint32_t a2 = 0; a2 < m; ++a2) {
        const uint32_t i = (uint32_t)(B[ord[q0 + a2]] & imask);
        bool ok;
        const uint64_t kx = morton_key(S.xyz[3ull * i], S.xyz[3ull * i + 1], S.xyz[3ull * i + 2], &ok);
        uint32_t r = a2;
        while (r > 0 && (kk[r - 1] > kx || (kk[r - 1] == kx && ii[r - 1] > i))) {
          kk[r] = kk[r - 1];
          ii[r] = ii[r - 1];
          --r;
        }
        kk[r] = kx;
        ii[r] = i;
      }
      for (uint32_t a2 = 0; a2 < m; ++a2) perm[offj + q0 + a2] = ii[a2];
    }
  }
  __syncthreads();

  // 5. Levels deeper than lh (only for deep trees): box starts from the
  // first differing level of every sorted point, counted by groups of three
  // levels, each with the level above it (for the parents), in 16-bit
  // fields: thread tid owns the points [tid * ipt, tid * ipt + ipt).
  const uint32_t ipt = (n_j + kBkThreads - 1) / kBkThreads;
  const uint32_t p0 = tid * ipt, p1 = p0 + ipt < n_j ? p0 + ipt : n_j;
  // first differing level of sorted point p (the sub-cell's first: d0)
  auto ddl = [&](uint32_t p) -> int {
    return p == 0 ? (int)d0 : (int)bk_diff_level(B[ord[p]], B[ord[p - 1]], keep1, bl1);
  };
  if (deep) {
    for (int g0 = lh + 1; g0 <= Lb; g0 += 3) {
      const int g1 = g0 + 2 < Lb ? g0 + 2 : Lb;
      uint64_t c = 0;
      for (uint32_t p = p0; p < p1; ++p) {
        const int d = ddl(p);
        if (d <= g1) c += fields((d > g0 - 1 ? d : g0 - 1) - (g0 - 1), g1 - (g0 - 1));
      }
      uint64_t tot;
      block_scan64<W>(c, s_w, &tot);
      if (tid == 0)
        for (int l = g0; l <= g1; ++l) {
          s_C[l] = field(tot, l - (g0 - 1));
          st_relaxed(status + (uint64_t)l * nsub + u, (u == 0 ? kFlagIncl : kFlagAgg) | s_C[l]);
        }
    }
    __syncthreads();
  }

  // 6. Box ranks: a decoupled look-back over the set's sub-cells, per level.
  for (int l = tid >> 5; l <= Lb; l += W) {
    uint64_t* chain = status + (uint64_t)l * nsub;
    uint64_t prev = 0;
    if (u > 0) {
      prev = lookback_warp(chain, u, 1, st, wait_ns);
      if (lane == 0) st_relaxed(chain + u, kFlagIncl | (prev + s_C[l]));
    }
    if (lane == 0) s_R[l] = (uint32_t)prev;
  }
  __syncthreads();
  if (tid == 0 && u > 0 && ld_relaxed_u32(&st->abort)) s_abort = 1;
  __syncthreads();
  if (s_abort) return;  // a wait gave up: ranks may be wrong, write nothing

  // 7. Outputs: the set's totals (last sub-cell slot of the last bucket);
  // the boxes starting at point 0 at levels <= bl1; the boxes of levels
  // bl1 + 1 .. lh, one thread per cell; the deeper boxes.
  if (b == nbk - 1 && j == 7 && tid <= Lb) {
    const uint32_t tot = s_R[tid] + s_C[tid];
    G.nbox[tid] = tot;
    if (tot <= s_lcap[tid]) {
      s_loff[tid][tot] = S.n;
      if (tid < Lb) s_lchd[tid][tot] = s_R[tid + 1] + s_C[tid + 1];
    }
  }
  if (tid == 0 && n_j > 0) {
    const int top = Lb < bl1 ? Lb : bl1;
    for (int l = (int)d0; l <= top; ++l) {
      const uint32_t rank = s_R[l];
      if (rank >= s_lcap[l]) continue;
      s_lkey[l][rank] = (uint64_t)cell1 >> (3 * (bl1 - l));
      s_loff[l][rank] = offj;
      if (l >= 1) {
        const bool up = d0 <= (uint32_t)(l - 1);
        const uint32_t pr = up ? s_R[l - 1] : s_R[l - 1] - 1u;
        s_lpar[l][rank] = pr;
        if (up && pr < s_lcap[l - 1]) s_lchd[l - 1][pr] = rank;
      }
    }
  }
  if (nm > 0 && tid < (1u << (3 * nm))) {
    const int gpc = D - 3 * nm;
    for (int m = 1; m <= nm; ++m) {
      const int sh = 3 * (nm - m);
      if ((tid & ((1u << sh) - 1)) != 0) continue;
      const uint32_t c = tid >> sh;
      if (!s_fl[hoff(m) + c]) continue;
      const int l = bl1 + m;
      const uint32_t within = s_pre[hoff(m) + c];
      const uint32_t rank = s_R[l] + within;
      if (rank >= s_lcap[l]) continue;
      s_lkey[l][rank] = ((uint64_t)cell1 << (3 * m)) | c;
      s_loff[l][rank] = offj + gs[c << (gpc + 3 * (nm - m))];
      const uint32_t pr = m == 1 ? s_R[bl1] : s_R[l - 1] + s_pre[hoff(m - 1) + (c >> 3)];
      s_lpar[l][rank] = pr;
      // the first non-empty child of its parent starts the parent's children
      const uint32_t first = m == 1 ? 0u : s_pre[hoff(m) + (c & ~7u)];
      if (within == first && pr < s_lcap[l - 1]) s_lchd[l - 1][pr] = rank;
    }
  }
  if (deep) {
    for (int g0 = lh + 1; g0 <= Lb; g0 += 3) {
      const int g1 = g0 + 2 < Lb ? g0 + 2 : Lb;
      const int f0 = g0 - 1;  // field 0: the level above the group
      uint64_t c = 0;
      for (uint32_t p = p0; p < p1; ++p) {
        const int d = ddl(p);
        if (d <= g1) c += fields((d > f0 ? d : f0) - f0, g1 - f0);
      }
      uint64_t tot;
      uint64_t ex = block_scan64<W>(c, s_w, &tot);  // starts before this thread's first point
      for (uint32_t p = p0; p < p1; ++p) {
        const int d = ddl(p);
        if (d > g1) continue;
        const uint64_t x = B[ord[p]];
        for (int l = d > g0 ? d : g0; l <= g1; ++l) {
          const uint32_t rank = s_R[l] + field(ex, l - f0);
          if (rank >= s_lcap[l]) continue;
          s_lkey[l][rank] = ((uint64_t)cell1 << (3 * (l - bl1))) | (x >> (64 - 3 * (l - bl1)));
          s_loff[l][rank] = offj + p;
          const bool up = d <= l - 1;
          const uint32_t pr = s_R[l - 1] + field(ex, l - 1 - f0) - (up ? 0u : 1u);
          s_lpar[l][rank] = pr;
          if (up && pr < s_lcap[l - 1]) s_lchd[l - 1][pr] = rank;
        }
        ex += fields((d > f0 ? d : f0) - f0, g1 - f0);
      }
    }
  }
}

// ---------------------------------------------------------------------------
void launch_bucket_plan(const BkSet* bsets, uint32_t nsets, DevStatus* st, cudaStream_t s) {
  if (nsets == 0) return;
  bucket_plan_kernel<<<nsets, kBkPlanThreads, 0, s>>>(bsets, st);
}

void launch_bucket_scatter(const BkSet* bsets, const Slot* slots, uint32_t nslots, uint32_t t_first,
                           uint32_t tiles, int max_bl, DevStatus* st, cudaStream_t s) {
  if (tiles == 0) return;
  static const bool attr = [] {
    cudaFuncSetAttribute(bucket_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(uint32_t) * 8 * kBkMaxCells));
    return true;
  }();
  (void)attr;
  const size_t smem = sizeof(uint32_t) * 8 * (1u << (3 * max_bl));
  bucket_scatter_kernel<<<tiles, kScThreads, smem, s>>>(bsets, slots, nslots, t_first, st);
}

void launch_bucket_boxes(const BkSet* bsets, const Seg* segs, const Slot* slots, uint32_t nslots,
                         uint32_t units, int max_lb, uint32_t* ticket, DevStatus* st,
                         uint64_t wait_ns, cudaStream_t s) {
  if (units == 0) return;
  (void)max_lb;
  static const bool attr = [] {
    cudaFuncSetAttribute(bucket_boxes_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kBkSmem);
    return true;
  }();
  (void)attr;
  bucket_boxes_kernel<<<units * 8, kBkThreads, kBkSmem, s>>>(bsets, segs, slots, nslots, ticket, st,
                                                             wait_ns);
}

}  // namespace fmm
