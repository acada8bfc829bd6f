// sort.cu -- Morton keys and the deterministic point order.
//
// The paper orders points with a linear-time pseudo-sort (Alg. 1: a box
// histogram by atomicAdd, order inside a box left to the hardware).  Here the
// order is fixed to (Morton key, original index) and built in two steps:
//
//   1. a stable least-significant-digit radix sort of (key, index) pairs on
//      the top 3*Ls key bits (the level-Ls box key), one "onesweep" pass per
//      digit: every tile ranks its items by digit in shared memory, publishes
//      its digit counts and finds its global offsets by decoupled look-back
//      over the tiles before it, then scatters through shared memory so that
//      the stores of one digit are contiguous.  The first pass reads the
//      coordinates and forms the keys on the fly; the digit histograms of all
//      passes come from one upfront read of the coordinates.
//   2. a finishing sort inside each level-Ls box by the full key, fused with
//      the box construction (boxes.cu).
#include "fmm_internal.cuh"

namespace fmm {

SortPlan make_sort_plan(uint32_t n, int Ls) {
  SortPlan p;
  p.Ls = Ls;
  const int nbits = 3 * Ls;
  p.passes = nbits == 0 ? 0 : (nbits + 7) / 8;
  p.bits = p.passes == 0 ? 0 : (nbits + p.passes - 1) / p.passes;
  p.lo = 63 - nbits;
  p.ntiles = (uint32_t)(((uint64_t)n + kSortTile - 1) / kSortTile);
  return p;
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) keys_kernel(const float* __restrict__ xyz, uint32_t n,
                                                   uint64_t* __restrict__ keys, DevStatus* st) {
  bool bad = false;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    bool ok;
    keys[i] = morton_key(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], &ok);
    bad |= !ok;
  }
  if (bad) set_error(st, FMM_ERR_DOMAIN);
}

void launch_keys(const float* xyz, uint32_t n, uint64_t* keys, DevStatus* st, cudaStream_t s) {
  if (n == 0) return;
  uint32_t blocks = (uint32_t)(((uint64_t)n + 255) / 256);
  if (blocks > 152u * 16u) blocks = 152u * 16u;
  keys_kernel<<<blocks, 256, 0, s>>>(xyz, n, keys, st);
}

// ---------------------------------------------------------------------------
// Upfront histograms: one read of the coordinates gives the digit counts of
// every pass.  Four points per thread and step come in as three float4 loads
// (the coordinates must then be 16-byte aligned); block-private histograms
// in shared memory take plain atomics.
__device__ __forceinline__ void hist_point(float x, float y, float z, int passes, int bits,
                                           int lo, uint32_t mask, uint32_t* sh, bool* bad) {
  bool ok;
  const uint64_t key = morton_key(x, y, z, &ok);
  *bad |= !ok;
  for (int p = 0; p < passes; ++p)
    atomicAdd(&sh[p * kRadixMax + ((uint32_t)(key >> (lo + p * bits)) & mask)], 1u);
}

__global__ void __launch_bounds__(256) upfront_hist_kernel(const float* __restrict__ xyz,
                                                           uint32_t n, int passes, int bits,
                                                           int lo, bool vec,
                                                           uint32_t* __restrict__ hist,
                                                           DevStatus* st) {
  __shared__ uint32_t sh[8 * kRadixMax];
  for (int i = threadIdx.x; i < 8 * kRadixMax; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const uint32_t mask = (1u << bits) - 1u;
  bool bad = false;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t done = 0;
  if (vec) {
    const float4* v = reinterpret_cast<const float4*>(xyz);
    const uint64_t groups = n / 4;
    for (uint64_t g = tid; g < groups; g += stride) {
      const float4 a = __ldcs(v + 3 * g), b = __ldcs(v + 3 * g + 1), c = __ldcs(v + 3 * g + 2);
      hist_point(a.x, a.y, a.z, passes, bits, lo, mask, sh, &bad);
      hist_point(a.w, b.x, b.y, passes, bits, lo, mask, sh, &bad);
      hist_point(b.z, b.w, c.x, passes, bits, lo, mask, sh, &bad);
      hist_point(c.y, c.z, c.w, passes, bits, lo, mask, sh, &bad);
    }
    done = groups * 4;
  }
  for (uint64_t i = done + tid; i < n; i += stride)
    hist_point(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], passes, bits, lo, mask, sh, &bad);
  __syncthreads();
  const int radix = 1 << bits;
  for (int i = threadIdx.x; i < passes * kRadixMax; i += blockDim.x) {
    const int d = i % kRadixMax;
    if (d < radix && sh[i]) atomicAdd(&hist[i], sh[i]);
  }
  if (bad) set_error(st, FMM_ERR_DOMAIN);
}

void launch_upfront_hist(const float* xyz, uint32_t n, const SortPlan& p, uint32_t* hist,
                         DevStatus* st, cudaStream_t s) {
  if (n == 0 || p.passes == 0) return;
  const bool vec = ((uintptr_t)xyz & 15u) == 0;
  uint32_t blocks = (uint32_t)(((uint64_t)n / 4 + 255) / 256);
  if (blocks > 152u * 8u) blocks = 152u * 8u;
  if (blocks == 0) blocks = 1;
  upfront_hist_kernel<<<blocks, 256, 0, s>>>(xyz, n, p.passes, p.bits, p.lo, vec, hist, st);
}

// Exclusive scan of each pass's digit counts (one block, one warp per pass).
__global__ void digit_scan_kernel(uint32_t* hist, int passes, int radix) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp >= passes) return;
  uint32_t* h = hist + warp * kRadixMax;
  uint32_t carry = 0;
  for (int c = 0; c < radix; c += 32) {
    const uint32_t v = (c + lane < radix) ? h[c + lane] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (c + lane < radix) h[c + lane] = carry + x - v;
    carry += __shfl_sync(0xffffffffu, x, 31);
  }
}

void launch_digit_scan(const SortPlan& p, uint32_t* hist, cudaStream_t s) {
  if (p.passes == 0) return;
  digit_scan_kernel<<<1, 32 * 8, 0, s>>>(hist, p.passes, 1 << p.bits);
}

// ---------------------------------------------------------------------------
// One onesweep pass.  Shared memory: per-warp digit counters, then the tile
// reordered by digit as (key, index) so that each digit's run leaves as one
// contiguous store sequence.
constexpr size_t kSortSmem = sizeof(uint64_t) * kSortTile + sizeof(uint32_t) * kSortTile;

template <bool kFromXyz>
__global__ void __launch_bounds__(kSortThreads, 2) onesweep_kernel(
    const float* __restrict__ xyz, const uint64_t* __restrict__ keys_in,
    const uint32_t* __restrict__ vals_in, uint64_t* __restrict__ keys_out,
    uint32_t* __restrict__ vals_out, uint32_t n, int shift, int bits,
    const uint32_t* __restrict__ digit_base, uint64_t* status, uint32_t* counter,
    DevStatus* st, uint64_t wait_ns, int stall_tile) {
  constexpr int W = kSortThreads / 32;
  __shared__ uint32_t s_tile, s_abort;
  __shared__ uint32_t s_wcnt[W][kRadixMax];  // per-warp digit counts, then prefixes
  __shared__ uint32_t s_gbase[kRadixMax];    // global position of block slot 0, per digit
  __shared__ uint32_t s_wsum[W];
  extern __shared__ __align__(16) uint64_t s_keys[];
  uint32_t* s_vals = reinterpret_cast<uint32_t*>(s_keys + kSortTile);

  const uint32_t radix = 1u << bits, mask = radix - 1u;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < W * kRadixMax; i += kSortThreads) (&s_wcnt[0][0])[i] = 0;
  if (threadIdx.x == 0) {
    s_tile = atomicAdd(counter, 1u);
    s_abort = (!kFromXyz && failed(st)) ? 1u : 0u;
  }
  __syncthreads();
  if (s_abort) return;  // an earlier kernel failed: leave the outputs alone
  const uint32_t tile = s_tile;
  const uint64_t base = (uint64_t)tile * kSortTile;
  const uint64_t wbase = base + (uint64_t)warp * (kSortItems * 32);

  // Warp-striped load: item k of lane j is element wbase + 32k + j, so the
  // (k, lane) order below is the input order and ranking stays stable.
  // Values are fetched only when the tile is reordered (shorter live range);
  // in the first pass the value is the point index itself.
  uint64_t key[kSortItems];
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    const uint64_t i = wbase + k * 32 + lane;
    key[k] = 0;
    if (i < n) {
      if (kFromXyz) {
        bool ok;
        key[k] = morton_key(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], &ok);
      } else {
        key[k] = keys_in[i];
      }
    }
  }

  // Stable rank within the warp: peers with the same digit by match_any,
  // running per-warp digit counters in shared memory.
  const uint32_t lt = lanemask_lt();
  uint32_t pos[kSortItems];
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    const bool valid = wbase + k * 32 + lane < n;
    const uint32_t d = valid ? (uint32_t)(key[k] >> shift) & mask : 0xffffffffu;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t before = valid ? s_wcnt[warp][d] : 0u;
    __syncwarp();
    if (valid && (peers & lt) == 0) s_wcnt[warp][d] = before + __popc(peers);
    __syncwarp();
    pos[k] = before + __popc(peers & lt);
  }
  __syncthreads();

  // Digit totals of the tile (published at once as an aggregate); s_wcnt
  // becomes the per-warp exclusive prefix.
  uint32_t tot = 0;
  if (threadIdx.x < radix) {
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const uint32_t c = s_wcnt[w][threadIdx.x];
      s_wcnt[w][threadIdx.x] = tot;
      tot += c;
    }
    if ((int)tile != stall_tile)
      st_relaxed(status + (uint64_t)tile * radix + threadIdx.x,
                 (tile == 0 ? kFlagIncl : kFlagAgg) | (uint64_t)tot);
  }
  // Block-exclusive scan of the digit totals.
  uint32_t x = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_wsum[warp] = x;
  __syncthreads();
  if (threadIdx.x < 32) {
    const uint32_t v = lane < W ? s_wsum[lane] : 0u;
    uint32_t y = v;
#pragma unroll
    for (int o = 1; o < W; o <<= 1) {
      const uint32_t z = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += z;
    }
    if (lane < W) s_wsum[lane] = y - v;
  }
  __syncthreads();
  const uint32_t excl_blk = x - tot + s_wsum[warp];
  if (threadIdx.x < radix) {
    // s_wcnt[w][d] + excl_blk: block slot of warp w's first item of digit d
#pragma unroll
    for (int w = 0; w < W; ++w) s_wcnt[w][threadIdx.x] += excl_blk;
  }
  __syncthreads();

  // Reorder the tile by digit in shared memory (values are fetched here).
  // This work sits between publishing the aggregate and reading the earlier
  // tiles' words, which gives them time to publish.
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    const uint64_t i = wbase + k * 32 + lane;
    if (i < n) {
      const uint32_t d = (uint32_t)(key[k] >> shift) & mask;
      const uint32_t p = pos[k] + s_wcnt[warp][d];
      s_keys[p] = key[k];
      s_vals[p] = kFromXyz ? (uint32_t)i : vals_in[i];
    }
  }
  if (threadIdx.x < radix) {
    uint64_t prev = 0;
    if (tile > 0) {
      prev = lookback_thread<16>(status + threadIdx.x, tile, radix, st, wait_ns);
      if ((int)tile != stall_tile)
        st_relaxed(status + (uint64_t)tile * radix + threadIdx.x, kFlagIncl | (prev + tot));
    }
    s_gbase[threadIdx.x] = digit_base[threadIdx.x] + (uint32_t)prev - excl_blk;
  }
  __syncthreads();
  if (threadIdx.x < radix && tile > 0 && ld_relaxed_u32(&st->abort)) s_abort = 1;
  __syncthreads();
  if (s_abort) return;  // a wait gave up: offsets may be wrong, write nothing

  const uint32_t cnt = (uint32_t)((n - base) < (uint64_t)kSortTile ? (n - base) : kSortTile);
#pragma unroll 4
  for (int j = 0; j < kSortItems; ++j) {
    const uint32_t p = threadIdx.x + j * kSortThreads;
    if (p < cnt) {
      const uint64_t kk = s_keys[p];
      const uint32_t g = s_gbase[(uint32_t)(kk >> shift) & mask] + p;
      if (g < n) {
        keys_out[g] = kk;
        vals_out[g] = s_vals[p];
      }
    }
  }
}

void launch_onesweep_pass(int pass, const float* xyz, const uint64_t* keys_in,
                          const uint32_t* vals_in, uint64_t* keys_out, uint32_t* vals_out,
                          uint32_t n, const SortPlan& p, const uint32_t* digit_base,
                          uint64_t* status, uint32_t* counter, DevStatus* st, uint64_t wait_ns,
                          int stall_tile, cudaStream_t s) {
  if (n == 0) return;
  // once per process (thread-safe static initialisation)
  static const bool attr = [] {
    cudaFuncSetAttribute(onesweep_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kSortSmem);
    cudaFuncSetAttribute(onesweep_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kSortSmem);
    return true;
  }();
  (void)attr;
  const int shift = p.lo + pass * p.bits;
  if (pass == 0)
    onesweep_kernel<true><<<p.ntiles, kSortThreads, kSortSmem, s>>>(
        xyz, nullptr, nullptr, keys_out, vals_out, n, shift, p.bits, digit_base, status, counter,
        st, wait_ns, stall_tile);
  else
    onesweep_kernel<false><<<p.ntiles, kSortThreads, kSortSmem, s>>>(
        nullptr, keys_in, vals_in, keys_out, vals_out, n, shift, p.bits, digit_base, status,
        counter, st, wait_ns, -1);
}

// ---------------------------------------------------------------------------
// Reduce-then-scan passes over one or many point sets.  No tile waits for
// another: each tile's digit counts come from a separate read (of the
// coordinates for the first pass, of the keys for the later ones), one prefix
// sum over the counts -- laid out set after set, digit-major inside a set --
// gives every (set, digit, tile) its output start in the concatenated
// arrays, and the scatter kernel streams.

__device__ __forceinline__ void count_digit(uint64_t key, int shift, uint32_t* sh) {
  atomicAdd(&sh[(uint32_t)(key >> shift) & (kRadixMax - 1u)], 1u);
}

// kFromXyz (first pass): the keys are formed here from the coordinates and
// stored to keys_out (concatenated slots) for the scatter, which then reads 8
// bytes a point instead of forming each key a second time.
template <bool kFromXyz>
__global__ void __launch_bounds__(256) tile_hist_kernel(const Seg* __restrict__ segs,
                                                        const Slot* __restrict__ slots,
                                                        uint32_t nslots, int pass,
                                                        const uint64_t* __restrict__ keys,
                                                        uint64_t* __restrict__ keys_out,
                                                        uint32_t* __restrict__ hist,
                                                        TileRec* __restrict__ recs,
                                                        DevStatus* st) {
  __shared__ uint32_t sh[kRadixMax];
  for (int i = threadIdx.x; i < kRadixMax; i += blockDim.x) sh[i] = 0;
  const Slot sl = slots[find_slot(slots, nslots, blockIdx.x)];
  const Seg& sg = segs[sl.seg];
  const uint32_t t = blockIdx.x - sl.unit0;  // tile of the set
  const uint32_t n = sg.n;
  const int shift = sg.lo + kRadixBits * pass;
  const uint32_t tile = sg.tile;
  const uint64_t base = (uint64_t)t * tile;
  const uint32_t cnt = (uint32_t)((n - base) < (uint64_t)tile ? (n - base) : tile);
  if (threadIdx.x == 0) {
    TileRec r;
    r.xyz = sg.xyz ? sg.xyz + 3 * base : nullptr;
    r.first = sg.base + (uint32_t)base;
    r.local = (uint32_t)base;
    r.cnt = cnt;
    r.shift = (uint32_t)shift;
    r.hist = sl.aux0 + t;
    r.hstride = sg.ntiles;
    r.corr = sl.aux1;
    r.lo = sg.base;
    r.hi = sg.base + n;
    r.pad = 0;
    recs[blockIdx.x] = r;
  }
  __syncthreads();
  bool bad = false;
  if (kFromXyz) {
    const float* xyz = sg.xyz;
    uint64_t* ko = keys_out + sg.base + base;  // set bases: multiples of 4 slots
    uint32_t done = 0;
    if (((uintptr_t)xyz & 15u) == 0) {  // 4 points = 3 float4; tiles start at multiples of 4
      const float4* v = reinterpret_cast<const float4*>(xyz + 3 * base);
      ulonglong2* o = reinterpret_cast<ulonglong2*>(ko);
      for (uint32_t g = threadIdx.x; g < cnt / 4; g += blockDim.x) {
        const float4 a = __ldcs(v + 3 * g), b = __ldcs(v + 3 * g + 1), c = __ldcs(v + 3 * g + 2);
        bool ok0, ok1, ok2, ok3;
        const uint64_t k0 = morton_key(a.x, a.y, a.z, &ok0);
        const uint64_t k1 = morton_key(a.w, b.x, b.y, &ok1);
        const uint64_t k2 = morton_key(b.z, b.w, c.x, &ok2);
        const uint64_t k3 = morton_key(c.y, c.z, c.w, &ok3);
        count_digit(k0, shift, sh);
        count_digit(k1, shift, sh);
        count_digit(k2, shift, sh);
        count_digit(k3, shift, sh);
        o[2 * g] = make_ulonglong2(k0, k1);
        o[2 * g + 1] = make_ulonglong2(k2, k3);
        bad |= !(ok0 && ok1 && ok2 && ok3);
      }
      done = cnt & ~3u;
    }
    for (uint32_t j = done + threadIdx.x; j < cnt; j += blockDim.x) {
      const uint64_t i = base + j;
      bool ok;
      const uint64_t k = morton_key(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], &ok);
      count_digit(k, shift, sh);
      ko[j] = k;
      bad |= !ok;
    }
  } else {
    const uint64_t* k0 = keys + sg.base + base;  // set bases are multiples of 4 slots
    const ulonglong2* v = reinterpret_cast<const ulonglong2*>(k0);
    for (uint32_t g = threadIdx.x; g < cnt / 2; g += blockDim.x) {
      const ulonglong2 k = __ldcs(v + g);
      count_digit(k.x, shift, sh);
      count_digit(k.y, shift, sh);
    }
    if ((cnt & 1u) && threadIdx.x == 0) count_digit(k0[cnt - 1], shift, sh);
  }
  __syncthreads();
  for (uint32_t d = threadIdx.x; d < kRadixMax; d += blockDim.x)
    hist[sl.aux0 + (uint64_t)d * sg.ntiles + t] = sh[d];
  if (bad) set_error(st, FMM_ERR_DOMAIN);
}

void launch_tile_hist(int pass, const Seg* segs, const Slot* slots, uint32_t nslots,
                      uint32_t ntiles, uint32_t* hist, const uint64_t* keys, uint64_t* keys_out,
                      TileRec* recs, DevStatus* st, cudaStream_t s) {
  if (ntiles == 0) return;
  if (pass == 0)
    tile_hist_kernel<true><<<ntiles, 256, 0, s>>>(segs, slots, nslots, 0, nullptr, keys_out, hist,
                                                  recs, st);
  else
    tile_hist_kernel<false><<<ntiles, 256, 0, s>>>(segs, slots, nslots, pass, keys, nullptr, hist,
                                                   recs, st);
}

// Scatter of one pass, persistent: each block walks the tiles u = blockIdx.x,
// + gridDim.x, ... of all sets and, while it ranks and scatters one tile, a
// bulk copy (TMA) brings the next tile's input -- the keys the first pass's
// histogram kernel stored, then the (key, index) pairs of later passes --
// into the other half of a double buffer.  Partial tiles are read with plain
// loads.  Global output position of (set, digit, tile) = scanned offset + the
// slot's correction (set base minus the points of the sets before it in this
// pass).
// ITEMS: items per thread (the tile is kSortThreads * ITEMS points, a tuning
// knob); kFirst: the values are the points' indices (first pass); kStable:
// keep the input order inside a digit (every pass but an unstable first one).
template <int ITEMS>
constexpr size_t scatter_smem() {
  return 2 * (size_t)kSortThreads * ITEMS * 12;  // two buffers of keys + indices
}

template <int ITEMS, bool kFirst, bool kStable>
__global__ void __launch_bounds__(kSortThreads, ITEMS <= 7 ? 2 : 1) rts_scatter_kernel(
    const TileRec* __restrict__ recs, uint32_t ntiles, const uint64_t* __restrict__ keys_in,
    const uint32_t* __restrict__ vals_in, uint64_t* __restrict__ keys_out,
    uint32_t* __restrict__ vals_out, const uint32_t* __restrict__ offsets, bool bulk,
    DevStatus* st, uint64_t wait_ns) {
  constexpr int W = kSortThreads / 32;
  constexpr uint32_t mask = kRadixMax - 1u;
  constexpr uint32_t kTile = kSortThreads * ITEMS;
  constexpr uint32_t kInBytes = kTile * 12;
  constexpr uint32_t kCopyBytes = kFirst ? kTile * 8 : kInBytes;
  __shared__ uint32_t s_fail;
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ uint32_t s_wcnt[W][kRadixMax];  // per-warp digit counts, then block slots
  __shared__ uint32_t s_gbase[kRadixMax];    // global position of block slot 0, per digit
  __shared__ uint32_t s_wsum[W];
  extern __shared__ __align__(128) unsigned char s_in[];  // two input buffers

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = lanemask_lt();
  if (threadIdx.x == 0) {
    s_fail = failed(st) ? 1u : 0u;
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (s_fail) return;  // an earlier kernel failed (domain error): leave the outputs alone

  // Full tiles are read by bulk copy (set bases are multiples of 4 slots, so
  // their keys and indices start 16-byte aligned).
  auto is_bulk = [&](const TileRec& r) -> bool { return bulk && r.cnt == kTile; };
  auto issue = [&](const TileRec& r, int b) {  // thread 0 only
    unsigned char* dst = s_in + b * kInBytes;
    mbar_expect_tx(&s_bar[b], kCopyBytes);
    bulk_load(dst, keys_in + r.first, kTile * 8, &s_bar[b]);
    if (!kFirst) bulk_load(dst + kTile * 8, vals_in + r.first, kTile * 4, &s_bar[b]);
  };
  // bit b: parity of buffer b's barrier phase / a copy into buffer b is in flight
  uint32_t phase = 0u, pending = 0u;
  uint32_t u = blockIdx.x;
  TileRec rec;
  if (u < ntiles) {
    rec = recs[u];
    if (is_bulk(rec)) {
      if (threadIdx.x == 0) issue(rec, 0);
      pending |= 1u;
    }
  }
  for (int it = 0; u < ntiles; u += gridDim.x, ++it) {
    const int b = it & 1;
    unsigned char* buf = s_in + b * kInBytes;
    const TileRec r = rec;
    const uint32_t cnt = r.cnt;
    const int shift = (int)r.shift;
    const bool full = (pending >> b) & 1u;
    {
      const uint32_t un = u + gridDim.x;
      if (un < ntiles) {
        rec = recs[un];
        if (is_bulk(rec)) {
          if (threadIdx.x == 0) {
            fence_proxy_async();
            issue(rec, b ^ 1);
          }
          pending |= 1u << (b ^ 1);
        }
      }
    }
    const uint32_t my_off =
        threadIdx.x < kRadixMax
            ? __ldg(offsets + r.hist + (uint64_t)threadIdx.x * r.hstride) + r.corr
            : 0u;
    for (int i = threadIdx.x; i < W * kRadixMax; i += kSortThreads) (&s_wcnt[0][0])[i] = 0;
    bool ok = true;
    if (full) {
      ok = mbar_wait(&s_bar[b], (phase >> b) & 1u, st, wait_ns);
      phase ^= 1u << b;
      pending &= ~(1u << b);
    }
    if (__syncthreads_or(!ok)) {
      // a copy never completed: let any other copy land, then leave
      for (int k = 0; k < 2; ++k)
        if ((pending >> k) & 1u) mbar_wait(&s_bar[k], (phase >> k) & 1u, st, wait_ns);
      return;
    }

    // Items, warp-striped: item k of lane j is tile slot 32 * (ITEMS *
    // warp + k) + j, so (k, lane) order is the input order.  Values are point
    // indices local to the set.
    uint64_t key[ITEMS];
    uint32_t val[ITEMS];
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const uint32_t j = (uint32_t)warp * (ITEMS * 32) + k * 32 + lane;
      key[k] = 0;
      val[k] = r.local + j;
      if (j < cnt) {
        key[k] = full ? reinterpret_cast<const uint64_t*>(buf)[j] : keys_in[r.first + j];
        if (!kFirst)
          val[k] = full ? reinterpret_cast<const uint32_t*>(buf + kTile * 8)[j]
                        : vals_in[r.first + j];
      }
    }
    uint32_t pos[ITEMS];
    if (!kStable) {
      // First pass: there is no earlier order to keep, so the rank inside a
      // digit needs no stability -- one shared-memory atomic per item (the
      // paper's Alg. 1 takes box ranks the same way).  Counts go to warp 0's
      // row; the finishing sort orders points inside a box by (key, index).
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) {
        const bool valid = (uint32_t)warp * (ITEMS * 32) + k * 32 + lane < cnt;
        pos[k] = valid ? atomicAdd(&s_wcnt[0][(uint32_t)(key[k] >> shift) & mask], 1u) : 0u;
      }
    } else {
      // Stable rank inside the warp's run of items: the lanes holding the
      // same digit ("peers") come from one ballot per digit bit (a warp
      // multisplit, which keeps the slow match unit out of the loop); the
      // lowest peer adds their number to the warp's counter for the digit and
      // hands the old count to the others.  A warp takes its items in input
      // order, so count + peers below = rank among equal digits.
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) {
        const bool valid = (uint32_t)warp * (ITEMS * 32) + k * 32 + lane < cnt;
        const uint32_t d = (uint32_t)(key[k] >> shift) & mask;
        uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
        for (int b = 0; b < kRadixBits; ++b) {
          const bool bit = ((d >> b) & 1u) != 0u;
          const uint32_t bb = __ballot_sync(0xffffffffu, bit);
          peers &= bit ? bb : ~bb;
        }
        const int leader = valid ? __ffs(peers) - 1 : lane;
        uint32_t old = 0;
        if (valid && lane == leader) old = atomicAdd(&s_wcnt[warp][d], (uint32_t)__popc(peers));
        pos[k] = __shfl_sync(0xffffffffu, old, leader) + __popc(peers & lt);
      }
    }
    __syncthreads();
    uint32_t tot = 0;
    if (threadIdx.x < kRadixMax) {
#pragma unroll
      for (int w = 0; w < W; ++w) {
        const uint32_t c = s_wcnt[w][threadIdx.x];
        s_wcnt[w][threadIdx.x] = tot;
        tot += c;
      }
    }
    uint32_t x = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_wsum[warp] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
      const uint32_t v = lane < W ? s_wsum[lane] : 0u;
      uint32_t y = v;
#pragma unroll
      for (int o = 1; o < W; o <<= 1) {
        const uint32_t z = __shfl_up_sync(0xffffffffu, y, o);
        if (lane >= o) y += z;
      }
      if (lane < W) s_wsum[lane] = y - v;
    }
    __syncthreads();
    if (threadIdx.x < kRadixMax) {
      const uint32_t excl_blk = x - tot + s_wsum[warp];
#pragma unroll
      for (int w = 0; w < W; ++w) s_wcnt[w][threadIdx.x] += excl_blk;
      s_gbase[threadIdx.x] = my_off - excl_blk;
    }
    __syncthreads();
    // Reorder the tile by digit into the (now consumed) input buffer.
    uint64_t* r_keys = reinterpret_cast<uint64_t*>(buf);
    uint32_t* r_vals = reinterpret_cast<uint32_t*>(buf + kTile * 8);
    const int row = kStable ? warp : 0;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      if ((uint32_t)warp * (ITEMS * 32) + k * 32 + lane < cnt) {
        const uint32_t p = pos[k] + s_wcnt[row][(uint32_t)(key[k] >> shift) & mask];
        r_keys[p] = key[k];
        r_vals[p] = val[k];
      }
    }
    __syncthreads();
#pragma unroll 2
    for (int j = 0; j < ITEMS; ++j) {
      const uint32_t p = threadIdx.x + j * kSortThreads;
      if (p < cnt) {
        const uint64_t kk = r_keys[p];
        const uint32_t g = s_gbase[(uint32_t)(kk >> shift) & mask] + p;
        if (g >= r.lo && g < r.hi) {  // inside the set's slots
          keys_out[g] = kk;
          vals_out[g] = r_vals[p];
        }
      }
    }
    __syncthreads();  // the buffer is free for the copy issued next iteration
  }
}

namespace {

template <int ITEMS>
void scatter_items(int pass, const TileRec* recs, uint32_t ntiles, const uint64_t* keys_in,
                   const uint32_t* vals_in, uint64_t* keys_out, uint32_t* vals_out,
                   const uint32_t* offsets, bool stable, bool bulk, DevStatus* st,
                   uint64_t wait_ns, cudaStream_t s) {
  constexpr size_t smem = scatter_smem<ITEMS>();
  // once per process and instantiation (thread-safe static initialisation)
  static const int sms = [] {
    cudaFuncSetAttribute(rts_scatter_kernel<ITEMS, true, true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(rts_scatter_kernel<ITEMS, true, false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(rts_scatter_kernel<ITEMS, false, true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 152;
  }();
  uint32_t grid = (uint32_t)sms * (ITEMS <= 7 ? 2u : 1u);  // persistent: the resident blocks
  if (grid > ntiles) grid = ntiles;
  if (pass == 0) {
    if (stable)
      rts_scatter_kernel<ITEMS, true, true><<<grid, kSortThreads, smem, s>>>(
          recs, ntiles, keys_in, nullptr, keys_out, vals_out, offsets, bulk, st, wait_ns);
    else
      rts_scatter_kernel<ITEMS, true, false><<<grid, kSortThreads, smem, s>>>(
          recs, ntiles, keys_in, nullptr, keys_out, vals_out, offsets, bulk, st, wait_ns);
  } else {
    rts_scatter_kernel<ITEMS, false, true><<<grid, kSortThreads, smem, s>>>(
        recs, ntiles, keys_in, vals_in, keys_out, vals_out, offsets, bulk, st, wait_ns);
  }
}

}  // namespace

void launch_rts_scatter(int pass, uint32_t items, const TileRec* recs, uint32_t ntiles,
                        const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out,
                        uint32_t* vals_out, const uint32_t* offsets, bool stable, bool bulk,
                        DevStatus* st, uint64_t wait_ns, cudaStream_t s) {
  if (ntiles == 0) return;
  if (items == 4)
    scatter_items<4>(pass, recs, ntiles, keys_in, vals_in, keys_out, vals_out, offsets, stable,
                     bulk, st, wait_ns, s);
  else if (items == 7)
    scatter_items<7>(pass, recs, ntiles, keys_in, vals_in, keys_out, vals_out, offsets, stable,
                     bulk, st, wait_ns, s);
  else if (items == 8)
    scatter_items<8>(pass, recs, ntiles, keys_in, vals_in, keys_out, vals_out, offsets, stable,
                     bulk, st, wait_ns, s);
  else
    scatter_items<6>(pass, recs, ntiles, keys_in, vals_in, keys_out, vals_out, offsets, stable,
                     bulk, st, wait_ns, s);
}

}  // namespace fmm
