// noalloc.cu -- fmm_exclusive_scan_noalloc: the prefix sum that turns
// per-box list counts into CSR row starts, for callers that cannot allocate
// device memory.
//
// Its only scratch (the look-back words of the tiles, a tile counter and a
// status word) is one file-scope __device__ array of fixed size, reserved on
// every GPU that loads this library for as long as the process lives.  Host
// code cannot use the array's name as a device address, so the first call on
// each device looks its address up with cudaGetSymbolAddress (with that
// device current) and caches it.
#include <cstddef>
#include <mutex>

#include "fmm_internal.cuh"

namespace fmm {
namespace {

constexpr uint32_t kNaMaxTiles = (FMM_NOALLOC_SCAN_MAX + kScanTile - 1) / kScanTile;

struct NoAllocScratch {
  uint64_t status[kNaMaxTiles];  // one look-back word per tile
  uint32_t counter;              // tile ticket
  uint32_t pad;
  DevStatus st;                  // bounded-wait status
};

constexpr int kMaxDevices = 64;
std::mutex g_mu;
NoAllocScratch* g_addr[kMaxDevices] = {};

}  // namespace
}  // namespace fmm

// The scratch: 128 KiB + 32 bytes on every device, laid out as NoAllocScratch.
constexpr size_t kNaWords = sizeof(fmm::NoAllocScratch) / sizeof(uint64_t);
static_assert(sizeof(fmm::NoAllocScratch) % sizeof(uint64_t) == 0, "scratch layout");
static __device__ __align__(256) uint64_t g_noalloc_scratch[kNaWords];

namespace fmm {
namespace {

// Out-of-place exclusive scan of counts[0..n) into offsets[0..n], with
// offsets[n] = total (low 32 bits) and *total = the 64-bit total.  The sums
// of a thread, a warp and a tile are kept in 64 bits, so a tile whose counts
// add up past 2^32 still gives the exact total.  If a bounded wait gives up,
// offsets[n] = 0xffffffff and *total = all ones (a real total is below 2^58).
__global__ void __launch_bounds__(kScanThreads) scan_noalloc_kernel(const uint32_t* counts,
                                                                   uint32_t n, uint32_t* offsets,
                                                                   uint64_t* total,
                                                                   NoAllocScratch* sc,
                                                                   uint64_t wait_ns) {
  constexpr int W = kScanThreads / 32;
  __shared__ uint32_t s_tile;
  __shared__ uint64_t s_wsum[W];
  __shared__ uint64_t s_prev;
  const uint32_t ntiles = n == 0 ? 1u : (uint32_t)(((uint64_t)n + kScanTile - 1) / kScanTile);
  if (threadIdx.x == 0) s_tile = atomicAdd(&sc->counter, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t i0 = (uint64_t)tile * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint64_t sum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (i0 + k < n) ? counts[i0 + k] : 0u;
    sum += v[k];
  }
  uint64_t x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint64_t run = 0;
    if (lane == 0) {
      for (int w = 0; w < W; ++w) {
        const uint64_t c = s_wsum[w];
        s_wsum[w] = run;
        run += c;
      }
    }
    run = __shfl_sync(0xffffffffu, run, 0);
    uint64_t prev = 0;
    if (tile == 0) {
      if (lane == 0) st_relaxed(sc->status, kFlagIncl | run);
    } else {
      if (lane == 0) st_relaxed(sc->status + tile, kFlagAgg | run);
      prev = lookback_warp(sc->status, tile, 1, &sc->st, wait_ns);
      if (lane == 0) st_relaxed(sc->status + tile, kFlagIncl | (prev + run));
    }
    if (lane == 0) {
      s_prev = prev;
      if (tile == ntiles - 1) {
        const bool gave_up = ld_relaxed_u32(&sc->st.abort) != 0;
        const uint64_t t = prev + run;
        offsets[n] = gave_up ? 0xffffffffu : (uint32_t)t;
        if (total) *total = gave_up ? ~0ull : t;
      }
    }
  }
  __syncthreads();
  uint64_t off = s_prev + s_wsum[warp] + (x - sum);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (i0 + k < n) offsets[i0 + k] = (uint32_t)off;
    off += v[k];
  }
}

// Device address of the scratch on `dev` (looked up once per device, with
// that device current).
NoAllocScratch* scratch_of(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    g_addr[dev] = static_cast<NoAllocScratch*>(p);
  }
  return g_addr[dev];
}

}  // namespace
}  // namespace fmm

extern "C" int fmm_exclusive_scan_noalloc(const uint32_t* counts, uint32_t n, uint32_t* offsets,
                                          uint64_t* total, void* stream) {
  using namespace fmm;
  if (!offsets || (n > 0 && !counts) || n > FMM_NOALLOC_SCAN_MAX) return FMM_ERR_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return FMM_ERR_CUDA;
  }
  NoAllocScratch* sc = scratch_of(dev);
  if (!sc) return FMM_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint32_t ntiles = n == 0 ? 1u : (uint32_t)(((uint64_t)n + kScanTile - 1) / kScanTile);
  // Everything the scan reads before writing starts at zero: the look-back
  // words of the tiles in use, the ticket and the status word.
  if (cudaMemsetAsync(sc->status, 0, sizeof(uint64_t) * ntiles, s) != cudaSuccess ||
      cudaMemsetAsync(&sc->counter, 0,
                      sizeof(NoAllocScratch) - offsetof(NoAllocScratch, counter), s) !=
          cudaSuccess) {
    cudaGetLastError();
    return FMM_ERR_CUDA;
  }
  scan_noalloc_kernel<<<ntiles, kScanThreads, 0, s>>>(counts, n, offsets, total, sc,
                                                      2000ull * 1000000ull);
  if (cudaGetLastError() != cudaSuccess) return FMM_ERR_CUDA;
  return FMM_OK;
}
