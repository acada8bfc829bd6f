// fmm_internal.cuh -- device helpers and kernel launchers shared by the
// library's translation units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fmmds.h"

namespace fmm {

constexpr int kMaxLevel = FMM_MAX_LEVEL;
constexpr int kLevels = FMM_LEVELS;

// ---------------------------------------------------------------------------
// Device status word.  `code` keeps the first error (fmm_status); `seg_long`
// records that a box was too long for the in-tile finishing sort.
struct DevStatus {
  uint32_t code;
  uint32_t seg_long;
  uint32_t abort;  // set by the first wait that gives up, seen by the others
  uint32_t pad;
};

// Internal code (never returned by the ABI): a bucket held more points than
// a block sorts; the build stops and the host builds again with the radix
// path for the sets concerned.
constexpr uint32_t kStatusBucketFull = 0x100u;

__device__ __forceinline__ void set_error(DevStatus* st, uint32_t code) {
  atomicCAS(&st->code, 0u, code);
}

// True once an earlier kernel (or an earlier block) has recorded an error;
// later kernels then leave their outputs alone.
__device__ __forceinline__ bool failed(const DevStatus* st) {
  return *(volatile const uint32_t*)&st->code != 0u;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------------------
// Morton code.  The 21 bits of a cell coordinate are spread three apart with
// the usual shift-and-mask ladder (each step doubles the gap between groups
// of bits: 16 -> 8 -> 4 -> 2 -> 1 bit groups); compact3 undoes it.
__device__ __forceinline__ uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0x1fffffu;
  x = (x | (x << 32)) & 0x001f00000000ffffull;
  x = (x | (x << 16)) & 0x001f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

__device__ __forceinline__ uint32_t compact3(uint64_t x) {
  x &= 0x1249249249249249ull;
  x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
  x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
  x = (x ^ (x >> 8)) & 0x001f0000ff0000ffull;
  x = (x ^ (x >> 16)) & 0x001f00000000ffffull;
  x = (x ^ (x >> 32)) & 0x1fffffull;
  return (uint32_t)x;
}

// Cell of one coordinate at level 21; false if outside [0, 1] or NaN.
__device__ __forceinline__ bool quantize21(float x, uint32_t* q) {
  bool ok = (x >= 0.0f) && (x <= 1.0f);
  float t = ok ? x * 2097152.0f : 0.0f;  // exact: power-of-two scale
  uint32_t v = (uint32_t)t;
  *q = v > 0x1fffffu ? 0x1fffffu : v;
  return ok;
}

__device__ __forceinline__ uint64_t morton_key(float x, float y, float z, bool* ok) {
  uint32_t qx, qy, qz;
  bool a = quantize21(x, &qx), b = quantize21(y, &qy), c = quantize21(z, &qz);
  *ok = a && b && c;
  return spread3(qx) | (spread3(qy) << 1) | (spread3(qz) << 2);
}

// ---------------------------------------------------------------------------
// Decoupled look-back words: 2 flag bits over a 62-bit value.
constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagIncl = 2ull << 62;
constexpr uint64_t kValMask = (1ull << 62) - 1;

__device__ __forceinline__ void st_relaxed(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Bounded wait step shared by the look-back loops: returns true when the
// caller must give up (time limit reached, or another thread gave up first).
struct WaitClock {
  uint64_t t0 = 0;
  uint32_t spins = 0;
  __device__ __forceinline__ bool expired(DevStatus* st, uint64_t wait_ns) {
    ++spins;
    if (spins <= 32) return false;
    if (t0 == 0) t0 = global_timer_ns();
    __nanosleep(spins > 1024 ? 1000 : 64);
    if ((spins & 31) != 0) return false;
    if (ld_relaxed_u32(&st->abort) != 0) return true;
    if (global_timer_ns() - t0 > wait_ns) {
      set_error(st, FMM_ERR_TIMEOUT);
      atomicExch(&st->abort, 1u);
      return true;
    }
    return false;
  }
};

// Exclusive prefix of tile `tile` for one counter, one thread: the words
// status[j * stride] of the tiles j < tile are read kWin at a time (independent
// loads), aggregates are summed back to the first inclusive prefix.
template <int kWin>
__device__ __forceinline__ uint64_t lookback_thread(const uint64_t* status, uint32_t tile,
                                                    uint32_t stride, DevStatus* st,
                                                    uint64_t wait_ns) {
  uint64_t excl = 0;
  int64_t j = (int64_t)tile - 1;
  WaitClock clk;
  while (j >= 0) {
    uint64_t w[kWin];
#pragma unroll
    for (int i = 0; i < kWin; ++i)
      w[i] = (j - i >= 0) ? ld_relaxed(status + (uint64_t)(j - i) * stride) : kFlagIncl;
    int used = 0;
    bool done = false, stall = false;
#pragma unroll
    for (int i = 0; i < kWin; ++i) {
      if (done || stall) continue;
      const uint64_t f = w[i] & ~kValMask;
      if (f == 0) {
        stall = true;
      } else {
        excl += (j - i >= 0) ? (w[i] & kValMask) : 0;
        ++used;
        if (f == kFlagIncl) done = true;
      }
    }
    if (done) break;
    j -= used;
    if (stall && clk.expired(st, wait_ns)) break;
  }
  return excl;
}

// The same for one counter with a whole warp: lane i reads tile j - i, so 32
// predecessors are examined per round trip.  All lanes return the result.
__device__ __forceinline__ uint64_t lookback_warp(const uint64_t* status, uint32_t tile,
                                                  uint32_t stride, DevStatus* st,
                                                  uint64_t wait_ns) {
  const int lane = threadIdx.x & 31;
  uint64_t excl = 0;
  int64_t j = (int64_t)tile - 1;
  WaitClock clk;
  while (j >= 0) {
    const int64_t t = j - lane;
    const uint64_t w = t >= 0 ? ld_relaxed(status + (uint64_t)t * stride) : kFlagIncl;
    const uint64_t f = w & ~kValMask;
    const uint32_t not_ready = __ballot_sync(0xffffffffu, f == 0);
    const uint32_t incl = __ballot_sync(0xffffffffu, f == kFlagIncl);
    // lanes below the first blocking word (not ready, or inclusive) are usable
    const uint32_t stop = not_ready | incl;
    const int first = stop ? __ffs(stop) - 1 : 32;
    const bool take_incl = first < 32 && ((incl >> first) & 1u);  // stop word is inclusive
    const int upto = take_incl ? first + 1 : first;
    uint64_t v = (lane < upto && t >= 0) ? (w & kValMask) : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    excl += v;
    if (take_incl) break;
    j -= upto;
    if (upto == 0 && clk.expired(st, wait_ns)) break;
  }
  return excl;
}

// Store v when `word` is non-zero, as one predicated instruction (streaming
// cache hint): no branch around it.
__device__ __forceinline__ void st_cs_if(uint32_t* p, uint32_t v, uint32_t word) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.global.cs.u32 [%0], %1;\n\t}"
      ::"l"(p), "r"(v), "r"(word)
      : "memory");
}
// ... and when `word` is zero.
__device__ __forceinline__ void st_cs_if_zero(uint32_t* p, uint32_t v, uint32_t word) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.eq.u32 q, %2, 0;\n\t@q st.global.cs.u32 [%0], %1;\n\t}"
      ::"l"(p), "r"(v), "r"(word)
      : "memory");
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (TMA, untiled) into shared memory, completed on an
// mbarrier.  Addresses and sizes must be multiples of 16 bytes.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Orders this thread's earlier shared-memory accesses before later bulk
// copies into the same memory.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
          smem_u32(bar)),
      "r"(bytes)
      : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 "
      "%0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for phase `parity` of an mbarrier; false after wait_ns (or
// once another thread gave up), with FMM_ERR_TIMEOUT recorded.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, DevStatus* st,
                                          uint64_t wait_ns) {
  WaitClock clk;
  while (!mbar_try_wait(bar, parity))
    if (clk.expired(st, wait_ns)) return false;
  return true;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// ---------------------------------------------------------------------------
// Per-level device views of one point set.
struct LevelArrays {
  uint32_t cap[kLevels];  // allocated boxes per level (writes are bounded by it)
  uint64_t* key[kLevels];
  uint32_t* off[kLevels];
  uint32_t* parent[kLevels];
  uint32_t* child[kLevels];
  uint8_t* occ[kLevels];
};

// One point set of a build ("segment").  A build holds one or two (sources,
// receivers) or, batched, many; their points are concatenated in the sort
// arrays, everything else is per set.  Device-resident; built on the host.
struct Seg {
  const float* xyz;  // [n][3]
  uint32_t n;
  uint32_t base;      // first slot of this set in the concatenated sort arrays
  int Ls, Lb;         // sort depth (top 3*Ls key bits), box depth
  int passes, lo;     // radix passes of 8 bits, lowest sorted key bit
  int exact;          // sorted on exactly the top 3*Ls bits with stable passes: the
                      // order is final, no finishing sort (box-key order)
  uint32_t tile;      // points of a sort tile (kSortThreads x items per thread)
  uint32_t ntiles;    // sort tiles
  uint32_t btiles;    // finishing / finest-box tiles
  uint32_t* perm;
  float* sorted;          // SortedSrc / SortedRecv [n][3], or null
  const uint64_t* skeys;  // this set's keys after the last pass (concatenated array + base)
  const uint32_t* svals;  // ... and point indices (local to the set)
  LevelArrays lv;
  uint64_t* bstatus;  // [btiles] look-back words of the finest level
  uint64_t* cstatus;  // [coarse tiles][kLevels]
  uint32_t* tickets;  // [2]: finishing tiles, coarse tiles
  uint32_t* nbox;     // [kLevels] box counts
  uint32_t* seg_long; // set when a box outruns the finishing window
};

// A range of work units of one launch that belongs to one set.
struct Slot {
  uint32_t seg;    // set index
  uint32_t unit0;  // first work unit (tile, or level-major unit) of the range
  uint32_t aux0;   // per-kernel: first histogram entry, ...
  uint32_t aux1;   // per-kernel: position correction, ...
};

// What the scatter of one radix pass needs about one tile, written by the
// pass's histogram kernel so that the scatter reads one record per tile
// instead of searching the slot table and the set descriptor.
struct alignas(16) TileRec {
  const float* xyz;  // the tile's first point (first pass)
  uint32_t first;    // the tile's first slot in the concatenated sort arrays
  uint32_t local;    // its first point index within the set
  uint32_t cnt;      // points in the tile
  uint32_t shift;    // lowest key bit of this pass's digit
  uint32_t hist;     // scanned offset of (digit 0, tile); digit d at hist + d * hstride
  uint32_t hstride;
  uint32_t corr;     // added to scanned offsets: set base minus earlier sets' points
  uint32_t lo, hi;   // the set's slots [lo, hi)
  uint32_t pad;
};
static_assert(sizeof(TileRec) == 48, "TileRec layout");

// Slot holding work unit u: slots[k].unit0 <= u < slots[k+1].unit0.
__device__ __forceinline__ uint32_t find_slot(const Slot* slots, uint32_t nslots, uint32_t u) {
  uint32_t lo = 0, hi = nslots;  // answer in [lo, hi)
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (slots[mid].unit0 <= u)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// One (sources, receivers) pair whose E2 / E4 lists are built.  The list
// arrays of a level are shared by all jobs of a build: counts go to the
// job's region of the level's work array (scanned once for all jobs), list
// entries to one array in job order; each job's row starts come out rebased
// to its own lists.
struct Job {
  uint32_t src, recv;  // set indices
  int L;               // lists at levels 2..L
  uint32_t pad;
  uint32_t region[kLevels];     // first entry of the job in the level's work array
  uint32_t* out2[kLevels];      // rebased E2 row starts [nbox_recv + 1]
  uint32_t* out4[kLevels];      // rebased E4 row starts
};

// Per-level arrays shared by the jobs of a build.
struct ListLevel {
  uint32_t* work2;   // counts, then global row starts (all jobs)
  uint32_t* work4;
  uint32_t* idx2;    // list entries (all jobs)
  uint32_t* idx4;
  uint8_t* code2;    // per E2 entry: (dx+1) + 3(dy+1) + 9(dz+1), the source box's offset
                     // from the receiver box; for the next level (null at the last one)
  uint32_t* jprefix; // [njobs + 1] parents (receiver boxes at l-1) before each job
  uint64_t* base;    // [njobs][2] first E2 / E4 entry of each job
  uint64_t* nnz;     // [njobs][2] E2 / E4 entries of each job
  uint64_t* total;   // [2] scanned totals of the level (capacity check)
};

// One point set on the bucket path (bucket.cu): the points are bucketed on
// the sub-cells (level bl + 1) of the cells of level bl, in one pass, and
// each sub-cell is sorted, and its boxes emitted, by one block.
// Device-resident; built on the host.
struct BkSet {
  const float* xyz;  // [n][3]
  uint32_t n;
  int bl;            // cell level of the buckets (0..4)
  int Lb;            // box depth
  int ib;            // bits of the point index at the bottom of an item
  int D;             // group bits of a sub-cell's counting sort
  int trunc;         // items hold fewer key bits than lie below the cell
  uint64_t keep;     // key bits an item keeps (box-key order: down to Lb only)
  uint32_t tile;     // points of a scatter tile
  uint32_t ntiles;
  uint32_t* sct;     // [8^(bl+1)] points per sub-cell (zeroed before the scatter)
  uint32_t* bcell;   // [nslot] non-empty cells, ascending
  uint32_t* boff;    // [nslot + 1] their bookmarks
  uint32_t* info;    // [4]: non-empty cells, largest cell
  uint64_t* items;   // [8^(bl+1)][kBkCap] the points' items, sub-cell c's from slot c kBkCap
  uint32_t* soff;    // [8 * nslot] sub-cell bookmarks
  uint32_t* scnt;    // [8 * nslot] sub-cell sizes
  uint64_t* status;  // [kLevels][8 * nslot] look-back words of the box ranks (zeroed)
  uint32_t nslot;    // min(8^bl, n): bucket slots
  uint32_t seg;      // the set's index among the build's sets (its Seg)
};

// ---------------------------------------------------------------------------
// Tunables of the kernels.
constexpr int kSortThreads = 512;
constexpr int kSortItems = 6;
constexpr int kSortTile = kSortThreads * kSortItems;  // 3072
constexpr int kRadixBits = 8;
constexpr int kRadixMax = 1 << kRadixBits;

constexpr int kBoxThreads = 512;
constexpr int kBoxItems = 8;
constexpr int kBoxTile = kBoxThreads * kBoxItems;  // 4096
constexpr int kBoxHalo = 256;  // a box the finishing sort handles ends within it

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

constexpr int kListThreads = 256;

constexpr int kBkPlanThreads = 1024;
constexpr int kBkThreads = 512;                     // a sub-cell's block (8 sub-cells a bucket)
constexpr int kBkItems = 12;
constexpr int kBkCap = kBkThreads * kBkItems;       // 6144 points sorted by one block
constexpr int kBkGroupBits = 11;                    // groups of a sub-cell's counting sort
constexpr int kBkMaxLevel = 4;                      // bucket cells of level 4 at most
constexpr int kBkMaxCells = 1 << (3 * kBkMaxLevel);  // 4096
constexpr uint32_t kBkTieRun = 32;                  // longest run of tied items one thread orders
constexpr size_t kBkSmem = sizeof(uint64_t) * kBkCap + sizeof(uint32_t) * ((1 << kBkGroupBits) + 4) +
                           sizeof(uint16_t) * kBkCap;

// Radix passes (8-bit digits) that sort the top 3*Ls key bits.
__host__ __device__ inline int passes_for(int Ls) { return (3 * Ls + kRadixBits - 1) / kRadixBits; }

// ---------------------------------------------------------------------------
// Launchers (host side).  All asynchronous on `s`.  `segs` / `jobs` and the
// slot tables are device pointers.

// Reduce-then-scan radix pass p over the sets of `slots` (units = sort tiles;
// aux0 = first histogram entry of the set, aux1 = scan-to-slot correction):
// per-tile digit histograms, digit-major per set, set after set.
// Per-tile digit counts of pass p, and the tiles' records for the scatter.
// Pass 0 forms the keys from the coordinates and stores them to keys_out;
// later passes read `keys`.
void launch_tile_hist(int pass, const Seg* segs, const Slot* slots, uint32_t nslots,
                      uint32_t ntiles, uint32_t* hist, const uint64_t* keys, uint64_t* keys_out,
                      TileRec* recs, DevStatus* st, cudaStream_t s);
// Scatter of pass p from (keys_in, vals_in) -- pass 0: the keys pass 0's
// histogram stored, values = point indices -- to (keys_out, vals_out)
// (concatenated arrays).  stable = false only for a first pass that a
// finishing sort follows.
void launch_rts_scatter(int pass, uint32_t items, const TileRec* recs, uint32_t ntiles,
                        const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out,
                        uint32_t* vals_out, const uint32_t* offsets, bool stable, bool bulk,
                        DevStatus* st, uint64_t wait_ns, cudaStream_t s);

// Onesweep pass over one set (keys_in / keys_out point at the set's slots).
struct SortPlan {
  int Ls, passes, bits, lo;
  uint32_t ntiles;
};
SortPlan make_sort_plan(uint32_t n, int Ls);
void launch_upfront_hist(const float* xyz, uint32_t n, const SortPlan& p, uint32_t* hist,
                         DevStatus* st, cudaStream_t s);
void launch_digit_scan(const SortPlan& p, uint32_t* hist, cudaStream_t s);
void launch_onesweep_pass(int pass, const float* xyz, const uint64_t* keys_in,
                          const uint32_t* vals_in, uint64_t* keys_out, uint32_t* vals_out,
                          uint32_t n, const SortPlan& p, const uint32_t* digit_base,
                          uint64_t* status, uint32_t* counter, DevStatus* st, uint64_t wait_ns,
                          int stall_tile, cudaStream_t s);

// Finishing sort inside level-Ls boxes (-> perm) and the finest level Lb of
// every set of `slots` (units = box tiles).
void launch_finish_boxes(const Seg* segs, const Slot* slots, uint32_t nslots, uint32_t units,
                         DevStatus* st, uint64_t wait_ns, cudaStream_t s);
// Levels 0..Lb-1, parents of level Lb, children of level Lb-1 (units =
// coarse tiles by capacity).
void launch_coarse_boxes(const Seg* segs, const Slot* slots, uint32_t nslots, uint32_t units,
                         int max_lb, DevStatus* st, uint64_t wait_ns, cudaStream_t s);
// Child-occupancy bytes (sets flagged in `which`, grid y = set) and largest
// occupancy per level.
// Sorted points (xyz[perm[j]]) of the sets with `sorted` set; units: finishing tiles.
void launch_sorted_xyz(const Seg* segs, const Slot* slots, uint32_t nslots, uint32_t units,
                       DevStatus* st, cudaStream_t s);
void launch_sorted_xyz_one(const uint32_t* perm, const float* xyz, uint32_t n, float* out,
                           cudaStream_t s);
// Alg. 2 over all receiver boxes of a level: E2 source-point counts, then the copy.
void launch_e2_count(const uint32_t* e2_off, const uint32_t* e2_idx, const uint32_t* src_off,
                     uint32_t nrecv, uint32_t* out, DevStatus* st, cudaStream_t s);
void launch_e2_gather(const uint32_t* e2_off, const uint32_t* e2_idx, const uint32_t* src_off,
                      const float* sorted_src, const uint32_t* off, uint32_t nrecv, float* out,
                      cudaStream_t s);
// Fixed-Grid pseudo-sort (Alg. 1, 3): keys, cells and atomic ranks per tile
// (slot aux0: the set's first histogram entry), then the move to bookmark +
// rank (slot aux1: the set's base minus the points of earlier sets).
void launch_fg_count(const Seg* segs, const Slot* slots, uint32_t nslots, uint32_t ntiles,
                     uint32_t* bins, uint64_t* keys_out, uint32_t* ranks_out, DevStatus* st,
                     cudaStream_t s);
void launch_fg_move(const Seg* segs, const Slot* slots, uint32_t nslots, uint32_t ntiles,
                    const uint32_t* bins, const uint64_t* keys_in, const uint32_t* ranks_in,
                    uint64_t* keys_out, uint32_t* vals_out, DevStatus* st, cudaStream_t s);
// Alg. 6 box types (box_types.cu): on-J flags of a level (from the owners
// at lpar, or through the parents), the child sides of the lcrit boxes, and
// the types of a level (mode 0: DOMESTIC; 1: lcrit; 2: deeper).
void launch_on_node(const uint32_t* owner, const uint32_t* parent, const uint8_t* on_up,
                    uint32_t nbox, uint32_t node, uint8_t* on, cudaStream_t s);
void launch_child_sides(const uint32_t* child, const uint8_t* on_par, uint32_t nbox,
                        uint8_t* sides, cudaStream_t s);
void launch_box_type(const uint32_t* e4_off, const uint32_t* e4_idx, const uint8_t* sides,
                     const uint8_t* on, uint32_t nbox, int mode, uint8_t* type, cudaStream_t s);
// Child-occupancy bytes of the slots' sets (slot aux0 = the set's units):
// the launch covers units [unit_first, unit_first + units).
void launch_occupancy(const Seg* segs, const Slot* slots, uint32_t nslots, uint32_t units,
                      uint32_t unit_first, DevStatus* st, cudaStream_t s);
uint32_t occupancy_units(uint32_t n);
// Cluster-size depth per set (units: sort tiles of the slots' sets); out[set]
// = 1 + deepest level shared by sorted points i and i + s, capped at Ls.
void launch_depth(const Seg* segs, const Slot* slots, uint32_t nslots, uint32_t units, uint32_t s,
                  uint32_t* out, DevStatus* st, cudaStream_t stream);
uint32_t coarse_tiles(uint32_t cap);

// Exclusive scan of u32 counts in place (count entries at data[0..count)),
// writes data[count] = total (low 32 bits) and total64 (if not null); flags
// FMM_ERR_CAPACITY if the total needs more than 32 bits.  `count` is read
// from device memory (*count_dev) and bounded by cap; count_dev == null
// means count = cap.
void launch_scan_u32(uint32_t* data, const uint32_t* count_dev, uint32_t cap, uint64_t* status,
                     uint32_t* counter, uint64_t* total64, DevStatus* st, uint64_t wait_ns,
                     cudaStream_t s);
// The same for two arrays of cap entries each, in one launch.
void launch_scan_u32_pair(uint32_t* data0, uint64_t* status0, uint64_t* total0, uint32_t* data1,
                          uint64_t* status1, uint64_t* total1, uint32_t cap, uint32_t* counter,
                          DevStatus* st, uint64_t wait_ns, cudaStream_t s);
uint32_t scan_tiles(uint32_t cap);

// Lists of level l for every job.  jprefix of the level is computed first
// (parents before each job; 0 for jobs whose L < l).
// lvls: device array of kLevels ListLevel (level l and its parent level l-1
// are read).
void launch_job_prefix(const Seg* segs, const Job* jobs, uint32_t njobs, int l,
                       const ListLevel* lvls, DevStatus* st, cudaStream_t s);
// Whether list_count computes the per-job prefix itself (small builds), so
// that no job_prefix launch is needed.
bool job_prefix_in_count(uint32_t njobs);
void launch_list_count(const Seg* segs, const Job* jobs, uint32_t njobs, int l,
                       const ListLevel* lvls, DevStatus* st, cudaStream_t s);
void launch_list_fill(const Seg* segs, const Job* jobs, uint32_t njobs, int l,
                      const ListLevel* lvls, bool codes, DevStatus* st, cudaStream_t s);

// Bucket path (bucket.cu).  count and scatter: units = tiles of the slots'
// sets (slot seg = BkSet index); plan: one block per set; split: units =
// bucket slots (slot unit0 = the set's first bucket slot); boxes: units =
// bucket slots as for split, 8 blocks each (one per sub-cell), taken in
// order by ticket (slot unit0 = the set's first sub-cell slot).
void launch_bucket_plan(const BkSet* bsets, uint32_t nsets, DevStatus* st, cudaStream_t s);
// Tiles [t_first, t_first + tiles) of the launch's units.
void launch_bucket_scatter(const BkSet* bsets, const Slot* slots, uint32_t nslots, uint32_t t_first,
                           uint32_t tiles, int max_bl, DevStatus* st, cudaStream_t s);
void launch_bucket_boxes(const BkSet* bsets, const Seg* segs, const Slot* slots, uint32_t nslots,
                         uint32_t units, int max_lb, uint32_t* ticket, DevStatus* st,
                         uint64_t wait_ns, cudaStream_t s);

// Morton keys of n points (public fmm_morton_keys).
void launch_keys(const float* xyz, uint32_t n, uint64_t* keys, DevStatus* st, cudaStream_t s);

}  // namespace fmm
