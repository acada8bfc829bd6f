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
//   2. a finishing sort inside each level-Ls box by the full key: boxes are
//      short (about 8 points at the benchmark sizes), so each point counts
//      the points of its box that precede it.  A box longer than the halo of
//      a tile is reported (seg_long) and the host redoes the set with the full
//      63-bit sort.
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
// every pass.  Warp-aggregated shared-memory atomics (match_any) keep hot
// digits of clustered inputs from serialising.
__global__ void __launch_bounds__(256) upfront_hist_kernel(const float* __restrict__ xyz,
                                                           uint32_t n, int passes, int bits,
                                                           int lo, uint32_t* __restrict__ hist,
                                                           DevStatus* st) {
  __shared__ uint32_t sh[8 * kRadixMax];
  for (int i = threadIdx.x; i < 8 * kRadixMax; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const uint32_t mask = (1u << bits) - 1u;
  const uint32_t lt = lanemask_lt();
  bool bad = false;
  for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x; i0 < n;
       i0 += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = i0 + threadIdx.x;
    const bool valid = i < n;
    uint64_t key = 0;
    if (valid) {
      bool ok;
      key = morton_key(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], &ok);
      bad |= !ok;
    }
    for (int p = 0; p < passes; ++p) {
      const uint32_t d = valid ? (uint32_t)(key >> (lo + p * bits)) & mask : 0xffffffffu;
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      if (valid && (peers & lt) == 0) atomicAdd(&sh[p * kRadixMax + d], (uint32_t)__popc(peers));
    }
  }
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
  uint32_t blocks = (uint32_t)(((uint64_t)n + 255) / 256);
  if (blocks > 152u * 8u) blocks = 152u * 8u;
  upfront_hist_kernel<<<blocks, 256, 0, s>>>(xyz, n, p.passes, p.bits, p.lo, hist, st);
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
// One onesweep pass.
template <bool kFromXyz>
__global__ void __launch_bounds__(kSortThreads) onesweep_kernel(
    const float* __restrict__ xyz, const uint64_t* __restrict__ keys_in,
    const uint32_t* __restrict__ vals_in, uint64_t* __restrict__ keys_out,
    uint32_t* __restrict__ vals_out, uint32_t n, int shift, int bits,
    const uint32_t* __restrict__ digit_base, uint64_t* status, uint32_t* counter,
    DevStatus* st, uint64_t wait_ns, int stall_tile) {
  constexpr int W = kSortThreads / 32;
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_wcnt[W][kRadixMax];  // per-warp digit counts, then prefixes
  __shared__ uint32_t s_doff[kRadixMax];     // block-exclusive digit offsets
  __shared__ uint32_t s_gbase[kRadixMax];    // global position of block slot 0, per digit
  __shared__ uint32_t s_wsum[W];
  __shared__ __align__(16) uint64_t s_buf[kSortTile];

  const uint32_t radix = 1u << bits, mask = radix - 1u;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ uint32_t s_abort;
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
  uint64_t key[kSortItems];
  uint32_t val[kSortItems];
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    const uint64_t i = wbase + k * 32 + lane;
    key[k] = 0;
    val[k] = 0;
    if (i < n) {
      if (kFromXyz) {
        bool ok;
        key[k] = morton_key(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], &ok);
        val[k] = (uint32_t)i;
      } else {
        key[k] = keys_in[i];
        val[k] = vals_in[i];
      }
    }
  }

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

  // Digit totals of the tile; s_wcnt becomes the per-warp exclusive prefix.
  uint32_t tot = 0;
  if (threadIdx.x < radix) {
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const uint32_t c = s_wcnt[w][threadIdx.x];
      s_wcnt[w][threadIdx.x] = tot;
      tot += c;
    }
    const bool stalled = (int)tile == stall_tile;
    if (!stalled)
      st_relaxed(status + base / kSortTile * radix + threadIdx.x,
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
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int w = 0; w < W; ++w) {
      const uint32_t c = s_wsum[w];
      s_wsum[w] = run;
      run += c;
    }
  }
  __syncthreads();
  const uint32_t excl_blk = x - tot + s_wsum[warp];
  if (threadIdx.x < radix) {
    s_doff[threadIdx.x] = excl_blk;
    uint64_t prev = 0;
    if (tile > 0) {
      prev = lookback(status + threadIdx.x, tile, radix, st, wait_ns);
      if ((int)tile != stall_tile)
        st_relaxed(status + (uint64_t)tile * radix + threadIdx.x, kFlagIncl | (prev + tot));
    }
    s_gbase[threadIdx.x] = digit_base[threadIdx.x] + (uint32_t)prev - excl_blk;
  }
  __syncthreads();
  if (threadIdx.x < radix && tile > 0 && ld_relaxed_u32(&st->abort)) s_abort = 1;
  __syncthreads();
  if (s_abort) return;  // a wait gave up: offsets may be wrong, write nothing

  // Scatter through shared memory: keys first, then values.
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    if (wbase + k * 32 + lane < n) {
      const uint32_t d = (uint32_t)(key[k] >> shift) & mask;
      pos[k] += s_doff[d] + s_wcnt[warp][d];
      s_buf[pos[k]] = key[k];
    }
  }
  __syncthreads();
  const uint32_t cnt = (uint32_t)((n - base) < (uint64_t)kSortTile ? (n - base) : kSortTile);
  uint32_t gdst[kSortItems];
#pragma unroll
  for (int j = 0; j < kSortItems; ++j) {
    const uint32_t p = threadIdx.x + j * kSortThreads;
    gdst[j] = 0;
    if (p < cnt) {
      const uint64_t kk = s_buf[p];
      const uint32_t d = (uint32_t)(kk >> shift) & mask;
      gdst[j] = s_gbase[d] + p;
      if (gdst[j] < n) keys_out[gdst[j]] = kk;
    }
  }
  __syncthreads();
  uint32_t* s_vbuf = reinterpret_cast<uint32_t*>(s_buf);
#pragma unroll
  for (int k = 0; k < kSortItems; ++k)
    if (wbase + k * 32 + lane < n) s_vbuf[pos[k]] = val[k];
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kSortItems; ++j) {
    const uint32_t p = threadIdx.x + j * kSortThreads;
    if (p < cnt && gdst[j] < n) vals_out[gdst[j]] = s_vbuf[p];
  }
}

void launch_onesweep_pass(int pass, const float* xyz, const uint64_t* keys_in,
                          const uint32_t* vals_in, uint64_t* keys_out, uint32_t* vals_out,
                          uint32_t n, const SortPlan& p, const uint32_t* digit_base,
                          uint64_t* status, uint32_t* counter, DevStatus* st, uint64_t wait_ns,
                          int stall_tile, cudaStream_t s) {
  if (n == 0) return;
  const int shift = p.lo + pass * p.bits;
  if (pass == 0)
    onesweep_kernel<true><<<p.ntiles, kSortThreads, 0, s>>>(
        xyz, nullptr, nullptr, keys_out, vals_out, n, shift, p.bits, digit_base, status, counter,
        st, wait_ns, stall_tile);
  else
    onesweep_kernel<false><<<p.ntiles, kSortThreads, 0, s>>>(
        nullptr, keys_in, vals_in, keys_out, vals_out, n, shift, p.bits, digit_base, status,
        counter, st, wait_ns, -1);
}

// ---------------------------------------------------------------------------
// Finishing sort inside level-Ls boxes.  A block owns kSegTile points and
// loads kSegHalo more on each side, so every box of at most kSegHalo points
// that touches the tile is entirely in shared memory.  Each point finds its
// box by walking to equal top bits on both sides, counts the points of the box
// that precede it in (full key, index) order -- inside a box the points
// already stand in index order -- and writes its index there.
__global__ void __launch_bounds__(kSegThreads) segment_finish_kernel(
    const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals, uint32_t n, int lo,
    uint32_t* __restrict__ perm, DevStatus* st) {
  constexpr int W = kSegTile + 2 * kSegHalo;
  __shared__ uint64_t s_key[W];
  __shared__ uint32_t s_val[W];
  if (__syncthreads_or(threadIdx.x == 0 && failed(st))) return;  // uniform
  const int64_t w0 = (int64_t)blockIdx.x * kSegTile - kSegHalo;
  for (int j = threadIdx.x; j < W; j += kSegThreads) {
    const int64_t i = w0 + j;
    if (i >= 0 && i < (int64_t)n) {
      s_key[j] = keys[i];
      s_val[j] = vals[i];
    }
  }
  __syncthreads();
  const int jlo = (int)((w0 < 0 ? 0 : w0) - w0);                              // first valid slot
  const int jhi = (int)(((w0 + W) > (int64_t)n ? (int64_t)n : (w0 + W)) - w0);  // one past last
  bool long_box = false;
  for (int j = kSegHalo + threadIdx.x; j < kSegHalo + kSegTile; j += kSegThreads) {
    if (j >= jhi) break;
    const uint64_t k = s_key[j];
    const uint64_t top = k >> lo;
    int a = j;
    while (a > jlo && (s_key[a - 1] >> lo) == top) --a;
    int b = j + 1;
    while (b < jhi && (s_key[b] >> lo) == top) ++b;
    if ((a == jlo && w0 + a > 0) || (b == jhi && w0 + b < (int64_t)n)) {
      long_box = true;  // the box runs past the loaded window
      continue;
    }
    uint32_t r = 0;
    for (int q = a; q < b; ++q) {
      const uint64_t kq = s_key[q];
      r += (kq < k) || (kq == k && q < j);
    }
    perm[w0 + a + r] = s_val[j];
  }
  if (long_box) atomicExch(&st->seg_long, 1u);
}

void launch_segment_finish(const uint64_t* keys, const uint32_t* vals, uint32_t n, int Ls,
                           uint32_t* perm, DevStatus* st, cudaStream_t s) {
  if (n == 0) return;
  const uint32_t blocks = (uint32_t)(((uint64_t)n + kSegTile - 1) / kSegTile);
  segment_finish_kernel<<<blocks, kSegThreads, 0, s>>>(keys, vals, n, 63 - 3 * Ls, perm, st);
}

}  // namespace fmm
