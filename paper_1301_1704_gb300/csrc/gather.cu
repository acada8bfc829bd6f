// gather.cu -- the sorted point arrays (SortedSrc / SortedRecv, Sec. 2.1)
// and Alg. 2 (Access-Source-E2-neighborhood) for all receiver boxes of a
// level at once: the consumer side of the CSR chain NeighborBookmark ->
// NeighborList -> SrcBookmark -> SortedSrc.
#include "fmm_internal.cuh"

namespace fmm {
namespace {

// Point j of each set's sorted array is input point perm[j].  Units are the
// finishing tiles of kBoxTile points.
__global__ void __launch_bounds__(256) sorted_xyz_kernel(const Seg* __restrict__ segs,
                                                         const Slot* __restrict__ slots,
                                                         uint32_t nslots, const DevStatus* st) {
  if (failed(st)) return;
  const Slot sl = slots[find_slot(slots, nslots, blockIdx.x)];
  const Seg& sg = segs[sl.seg];
  // A set whose boxes outran the finishing window has an incomplete
  // permutation until the host redoes its order (and then its points).
  if (!sg.sorted || *sg.seg_long) return;
  const uint64_t t0 = (uint64_t)(blockIdx.x - sl.unit0) * kBoxTile;
  const uint64_t t1 = t0 + kBoxTile < sg.n ? t0 + kBoxTile : sg.n;
  for (uint64_t j = t0 + threadIdx.x; j < t1; j += blockDim.x) {
    const uint64_t i = sg.perm[j];
    if (i >= sg.n) continue;  // never for a complete permutation
    sg.sorted[3 * j] = sg.xyz[3 * i];
    sg.sorted[3 * j + 1] = sg.xyz[3 * i + 1];
    sg.sorted[3 * j + 2] = sg.xyz[3 * i + 2];
  }
}

// Number of E2 source points of each receiver box.
__global__ void __launch_bounds__(256) e2_count_kernel(const uint32_t* __restrict__ e2_off,
                                                       const uint32_t* __restrict__ e2_idx,
                                                       const uint32_t* __restrict__ src_off,
                                                       uint32_t nrecv, uint32_t* __restrict__ out,
                                                       DevStatus* st) {
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < nrecv;
       r += gridDim.x * blockDim.x) {
    uint64_t c = 0;
    for (uint32_t j = e2_off[r]; j < e2_off[r + 1]; ++j) {
      const uint32_t v = e2_idx[j];
      c += src_off[v + 1] - src_off[v];
    }
    if (c >> 32) set_error(st, FMM_ERR_CAPACITY);
    out[r] = (uint32_t)c;
  }
}

// One warp per receiver box: its E2 source boxes in list order, each a
// contiguous run of sorted points copied with coalesced float loads.
__global__ void __launch_bounds__(256) e2_gather_kernel(const uint32_t* __restrict__ e2_off,
                                                        const uint32_t* __restrict__ e2_idx,
                                                        const uint32_t* __restrict__ src_off,
                                                        const float* __restrict__ sorted_src,
                                                        const uint32_t* __restrict__ off,
                                                        uint32_t nrecv, float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nrecv; r += nw) {
    uint64_t w = 3ull * off[r];
    for (uint32_t j = e2_off[r]; j < e2_off[r + 1]; ++j) {
      const uint32_t v = e2_idx[j];
      const uint64_t a = 3ull * src_off[v], b = 3ull * src_off[v + 1];
      for (uint64_t k = a + lane; k < b; k += 32) out[w + (k - a)] = sorted_src[k];
      w += b - a;
    }
  }
}

// One set's sorted points (after its permutation was replaced).
__global__ void __launch_bounds__(256) sorted_xyz_one_kernel(const uint32_t* __restrict__ perm,
                                                             const float* __restrict__ xyz,
                                                             uint32_t n, float* __restrict__ out) {
  for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n;
       j += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = perm[j];
    if (i >= n) continue;  // never for a complete permutation
    out[3 * j] = xyz[3 * i];
    out[3 * j + 1] = xyz[3 * i + 1];
    out[3 * j + 2] = xyz[3 * i + 2];
  }
}

}  // namespace

void launch_sorted_xyz_one(const uint32_t* perm, const float* xyz, uint32_t n, float* out,
                           cudaStream_t s) {
  if (n == 0) return;
  uint32_t grid = (n + 255) / 256;
  if (grid > 152u * 8u) grid = 152u * 8u;
  sorted_xyz_one_kernel<<<grid, 256, 0, s>>>(perm, xyz, n, out);
}

void launch_sorted_xyz(const Seg* segs, const Slot* slots, uint32_t nslots, uint32_t units,
                       DevStatus* st, cudaStream_t s) {
  if (units == 0) return;
  sorted_xyz_kernel<<<units, 256, 0, s>>>(segs, slots, nslots, st);
}

void launch_e2_count(const uint32_t* e2_off, const uint32_t* e2_idx, const uint32_t* src_off,
                     uint32_t nrecv, uint32_t* out, DevStatus* st, cudaStream_t s) {
  if (nrecv == 0) return;
  uint32_t grid = (nrecv + 255) / 256;
  if (grid > 152u * 8u) grid = 152u * 8u;
  e2_count_kernel<<<grid, 256, 0, s>>>(e2_off, e2_idx, src_off, nrecv, out, st);
}

void launch_e2_gather(const uint32_t* e2_off, const uint32_t* e2_idx, const uint32_t* src_off,
                      const float* sorted_src, const uint32_t* off, uint32_t nrecv, float* out,
                      cudaStream_t s) {
  if (nrecv == 0) return;
  uint32_t grid = (nrecv + 7) / 8;  // 8 warps a block
  if (grid > 152u * 16u) grid = 152u * 16u;
  e2_gather_kernel<<<grid, 256, 0, s>>>(e2_off, e2_idx, src_off, sorted_src, off, nrecv, out);
}

}  // namespace fmm
