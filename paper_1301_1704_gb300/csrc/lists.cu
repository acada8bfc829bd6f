// lists.cu -- E2 neighbour lists and E4 (M2L) interaction lists, levels 2..L.
//
// Alg. 4 builds E2 by a search of the 27 cells around each receiver box.  Here
// both lists come from the level above, with no search: the children of the
// source boxes in E2(parent(r), l-1) are exactly E2(r, l) + E4(r, l) (Sec. 1.4
// item 4, E4 = E2(parent) minus E2).  The level-2 case uses the fact that all
// level-1 boxes touch, so E2 at level 1 is "every non-empty source box".
//
// For a parent-level neighbour Q at offset delta (per axis -1, 0, +1) from
// parent(r), and r in octant rho of its parent, a child of Q in octant o is in
// E2(r) iff on every axis |2 delta + o - rho| <= 1, i.e.
//     delta = 0: any child bit;  delta = +1: bit 0, only if rho = 1;
//     delta = -1: bit 1, only if rho = 0.
// So E2 children of Q = occ(Q) & mask(delta, rho) and the E4 children are the
// rest of occ(Q), where occ(Q) is Q's child-occupancy byte.  A child's rank is
// child(Q) + popc(occ(Q) below its octant), so neither list reads child keys,
// and walking Q in ascending rank, children in ascending octant, yields
// ascending ranks.
//
// One warp handles one parent box p: lane k takes the k-th entry Q_k of
// E2(p) (at most 27), and the warp serves every receiver child r of p.
// Counting and filling are two kernels around a prefix sum of the counts.
#include <type_traits>

#include "fmm_internal.cuh"

namespace fmm {

constexpr int kListWarps = kListThreads / 32;
// Builds of at most this many jobs get their per-job prefix inside list_count.
constexpr uint32_t kLocalJobs = 1024;

__device__ __forceinline__ uint32_t axis_mask(int delta, uint32_t rho_bit, uint32_t lo_oct,
                                              uint32_t hi_oct) {
  // lo_oct / hi_oct: octants with child bit 0 / 1 on this axis.
  if (delta == 0) return lo_oct | hi_oct;
  if (delta == 1) return rho_bit ? lo_oct : 0u;
  return rho_bit ? 0u : hi_oct;  // delta == -1
}

__device__ __forceinline__ uint32_t e2_child_mask(int dx, int dy, int dz, uint32_t rho) {
  return axis_mask(dx, rho & 1u, 0x55u, 0xaau) & axis_mask(dy, (rho >> 1) & 1u, 0x33u, 0xccu) &
         axis_mask(dz, (rho >> 2) & 1u, 0x0fu, 0xf0u);
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ uint32_t warp_excl(uint32_t v, int lane) {
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x - v;
}

// Everything one warp needs to serve the parents of one job at level l.
struct ListCtx {
  uint32_t nsrc1;              // non-empty source boxes at level 1 (level 2 only)
  const uint64_t* rkey_up;     // receiver keys, level l-1
  const uint32_t* rchild_up;   // receiver children, level l-1
  const uint64_t* rkey;        // receiver keys, level l
  const uint32_t* e2_off_up;   // the job's E2 row starts, level l-1 (rebased)
  const uint32_t* e2_idx_up;   // the job's E2 entries, level l-1
  const uint8_t* e2_code_up;   // ... and their offset codes (see list_fill), or null
  const uint64_t* skey_up;     // source keys, level l-1
  const uint32_t* schild_up;   // source children, level l-1
  const uint8_t* socc_up;      // source child occupancy, level l-1
  uint32_t region;             // the job's first entry in the level's work arrays
  uint32_t nrecv;              // receiver boxes of the job at level l
  uint32_t np;                 // parents (receiver boxes at l-1) of the job
};

__device__ __forceinline__ ListCtx make_ctx(const Seg* segs, const Job& J, int l,
                                            const ListLevel* lvls, uint32_t jidx) {
  const Seg& S = segs[J.src];
  const Seg& R = segs[J.recv];
  ListCtx c;
  c.nsrc1 = S.nbox[1];
  c.rkey_up = R.lv.key[l - 1];
  c.rchild_up = R.lv.child[l - 1];
  c.rkey = R.lv.key[l];
  c.e2_off_up = l >= 3 ? J.out2[l - 1] : nullptr;
  c.e2_idx_up = l >= 3 ? lvls[l - 1].idx2 + lvls[l - 1].base[2 * jidx] : nullptr;
  c.e2_code_up = (l >= 3 && lvls[l - 1].code2) ? lvls[l - 1].code2 + lvls[l - 1].base[2 * jidx]
                                               : nullptr;
  c.skey_up = S.lv.key[l - 1];
  c.schild_up = S.lv.child[l - 1];
  c.socc_up = S.lv.occ[l - 1];
  c.region = J.region[l];
  c.nrecv = R.nbox[l];
  c.np = 0;
  return c;
}

// Per-lane view of one parent-level neighbour.
struct Neighbour {
  int dx, dy, dz;
  uint32_t occ;
  uint32_t child;
};

__device__ __forceinline__ Neighbour load_neighbour(const ListCtx& a, int l, uint32_t p, int lane) {
  Neighbour q{0, 0, 0, 0u, 0u};
  uint32_t m, first;
  if (l == 2) {
    first = 0;
    m = a.nsrc1;
  } else {
    first = a.e2_off_up[p];
    m = a.e2_off_up[p + 1] - first;
  }
  if ((uint32_t)lane < m) {
    const uint32_t Q = (l == 2) ? (uint32_t)lane : a.e2_idx_up[first + lane];
    if (a.e2_code_up) {
      // the offset of Q from p, written with the entry: (dx+1) + 3(dy+1) + 9(dz+1)
      const uint32_t code = a.e2_code_up[first + lane];
      const uint32_t z = code / 9u, rem = code - 9u * z, y = rem / 3u;
      q.dx = (int)(rem - 3u * y) - 1;
      q.dy = (int)y - 1;
      q.dz = (int)z - 1;
    } else {
      const uint64_t pk = a.rkey_up[p];
      const uint64_t qk = a.skey_up[Q];
      q.dx = (int)compact3(qk) - (int)compact3(pk);
      q.dy = (int)compact3(qk >> 1) - (int)compact3(pk >> 1);
      q.dz = (int)compact3(qk >> 2) - (int)compact3(pk >> 2);
    }
    q.occ = a.socc_up[Q];
    q.child = a.schild_up[Q];
  }
  return q;
}

// Job holding global parent g: jp[j] <= g < jp[j + 1].
__device__ __forceinline__ uint32_t find_job(const uint32_t* jp, uint32_t njobs, uint32_t g) {
  uint32_t lo = 0, hi = njobs;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (jp[mid] <= g)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// Parents before each job at level l (0 for jobs whose lists stop below l).
__global__ void job_prefix_kernel(const Seg* __restrict__ segs, const Job* __restrict__ jobs,
                                  uint32_t njobs, int l, const ListLevel* lvls, DevStatus* st) {
  __shared__ uint32_t s_carry, s_wsum[32];
  if (failed(st)) return;
  const ListLevel& LV = lvls[l];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (uint32_t c = 0; c < njobs; c += blockDim.x) {
    const uint32_t j = c + threadIdx.x;
    uint32_t np = 0;
    if (j < njobs && jobs[j].L >= l) {
      const Seg& R = segs[jobs[j].recv];
      np = R.nbox[l - 1];
      if (R.nbox[l] == 0) {
        jobs[j].out2[l][0] = 0;
        jobs[j].out4[l][0] = 0;
      }
    }
    uint32_t x = np;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_wsum[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t run = s_carry;
      for (int w = 0; w < nw; ++w) {
        const uint32_t v = s_wsum[w];
        s_wsum[w] = run;
        run += v;
      }
      s_carry = run;
    }
    __syncthreads();
    if (j < njobs) LV.jprefix[j] = s_wsum[warp] + x - np;
    __syncthreads();
  }
  if (threadIdx.x == 0) LV.jprefix[njobs] = s_carry;
}

void launch_job_prefix(const Seg* segs, const Job* jobs, uint32_t njobs, int l,
                       const ListLevel* lvls, DevStatus* st, cudaStream_t s) {
  job_prefix_kernel<<<1, 1024, 0, s>>>(segs, jobs, njobs, l, lvls, st);
}

bool job_prefix_in_count(uint32_t njobs) { return njobs <= kLocalJobs; }

// Each block takes a contiguous run of the level's parents (over all jobs),
// dealt round-robin to its warps: a warp changes jobs only where the run
// crosses a job boundary, and the warps of a block work on neighbouring
// parents, whose list stores land close together.
struct BlockRange {
  uint32_t g0, g1;
};

__device__ __forceinline__ BlockRange block_range(uint32_t total) {
  const uint32_t per = (uint32_t)(((uint64_t)total + gridDim.x - 1) / gridDim.x);
  const uint64_t a = (uint64_t)blockIdx.x * per, b = a + per;
  return BlockRange{(uint32_t)(a < total ? a : total), (uint32_t)(b < total ? b : total)};
}

// Parents before each job at level l, computed by the whole block into s_jp
// (njobs <= kLocalJobs; s_jp[kLocalJobs] = the level's total).  Block 0 also
// publishes them in `jprefix_out` for the fill kernel and starts the rows of
// jobs with no receiver box at level l, as job_prefix_kernel does for larger
// builds.

__device__ void block_job_prefix(const Seg* __restrict__ segs, const Job* __restrict__ jobs,
                                 uint32_t njobs, int l, uint32_t* s_jp, uint32_t* s_wsum,
                                 uint32_t* jprefix_out) {
  constexpr int kPer = kLocalJobs / kListThreads;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t v[kPer], sum = 0;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const uint32_t j = threadIdx.x * kPer + k;
    v[k] = 0;
    if (j < njobs && jobs[j].L >= l) {
      const Seg& R = segs[jobs[j].recv];
      v[k] = R.nbox[l - 1];
      if (blockIdx.x == 0 && R.nbox[l] == 0) {
        jobs[j].out2[l][0] = 0;
        jobs[j].out4[l][0] = 0;
      }
    }
    sum += v[k];
  }
  uint32_t x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_wsum[warp] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int w = 0; w < kListWarps; ++w) {
      const uint32_t c = s_wsum[w];
      s_wsum[w] = run;
      run += c;
    }
    s_jp[kLocalJobs] = run;
  }
  __syncthreads();
  uint32_t off = s_wsum[warp] + x - sum;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    s_jp[threadIdx.x * kPer + k] = off;
    off += v[k];
  }
  __syncthreads();
  if (blockIdx.x == 0)
    for (uint32_t j = threadIdx.x; j <= njobs; j += blockDim.x)
      jprefix_out[j] = j < kLocalJobs ? s_jp[j] : s_jp[kLocalJobs];
}

// Counts: per receiver child r of parent p, |E2(r)| = sum over the parent's
// neighbours Q of popc(occ(Q) & mask(delta_Q, rho_r)), and |E2| + |E4| = the
// number of non-empty children of all Q.  The eight possible sibling octants
// are counted at once: byte rho of a packed pair of words.  The kernel waits
// on chains of dependent loads (row start, entry, occupancy): eight blocks an
// SM keep more parents in flight.
__global__ void __launch_bounds__(kListThreads, 8) list_count_kernel(const Seg* __restrict__ segs,
                                                                 const Job* __restrict__ jobs,
                                                                 uint32_t njobs, int l,
                                                                 const ListLevel* lvls,
                                                                 DevStatus* st) {
  __shared__ uint32_t s_jp[kLocalJobs + 1];
  __shared__ uint32_t s_wsum[kListWarps];
  if (failed(st)) return;  // set before this launch: the same for every thread
  const int lane = threadIdx.x & 31;
  // The level's arrays in registers: stores through them must not force
  // reloads of the descriptor.
  uint32_t* const work2 = lvls[l].work2;
  uint32_t* const work4 = lvls[l].work4;
  const uint32_t* jprefix = lvls[l].jprefix;
  if (njobs <= kLocalJobs) {  // the per-job prefix here, not in its own launch
    block_job_prefix(segs, jobs, njobs, l, s_jp, s_wsum, lvls[l].jprefix);
    jprefix = s_jp;
  }
  const uint32_t total = njobs <= kLocalJobs ? s_jp[kLocalJobs] : jprefix[njobs];
  const BlockRange br = block_range(total);
  uint32_t j = 0, jstart = 0, jend = 0;
  ListCtx a{};
  for (uint32_t g = br.g0 + (threadIdx.x >> 5); g < br.g1; g += blockDim.x >> 5) {
    if (g >= jend) {  // g only grows: look its job up when it leaves the current one
      j = find_job(jprefix, njobs, g);
      a = make_ctx(segs, jobs[j], l, lvls, j);
      jstart = jprefix[j];
      jend = jprefix[j + 1];
    }
    const uint32_t p = g - jstart;
    const Neighbour q = load_neighbour(a, l, p, lane);
    uint32_t lo = 0, hi = 0;  // byte rho: popc(occ & mask(delta, rho))
    {
      // mask(delta, rho) factors by axis into masks chosen by rho's bits
      const uint32_t mx0 = axis_mask(q.dx, 0u, 0x55u, 0xaau), mx1 = axis_mask(q.dx, 1u, 0x55u, 0xaau);
      const uint32_t my0 = axis_mask(q.dy, 0u, 0x33u, 0xccu), my1 = axis_mask(q.dy, 1u, 0x33u, 0xccu);
      const uint32_t mz0 = axis_mask(q.dz, 0u, 0x0fu, 0xf0u), mz1 = axis_mask(q.dz, 1u, 0x0fu, 0xf0u);
#pragma unroll
      for (uint32_t rho = 0; rho < 8; ++rho) {
        const uint32_t m = ((rho & 1) ? mx1 : mx0) & ((rho & 2) ? my1 : my0) & ((rho & 4) ? mz1 : mz0);
        const uint32_t cnt = (uint32_t)__popc(q.occ & m);
        if (rho < 4)
          lo |= cnt << (8 * rho);
        else
          hi |= cnt << (8 * (rho - 4));
      }
    }
    const uint32_t tot = warp_sum(__popc(q.occ));
    lo = warp_sum(lo);
    hi = warp_sum(hi);
    const uint32_t c0 = a.rchild_up[p];
    const uint32_t c1 = min(a.rchild_up[p + 1], c0 + 8u);  // (at most 8 in a whole tree)
    const uint32_t r = c0 + lane;
    if (r < c1) {
      const uint32_t rho = (uint32_t)(a.rkey[r] & 7u);
      const uint32_t n2 = ((rho < 4 ? lo : hi) >> (8 * (rho & 3))) & 0xffu;
      work2[a.region + r] = n2;
      work4[a.region + r] = tot - n2;
    }
  }
}

// Fill: per parent p, the candidate list C -- the non-empty children of p's
// neighbours in ascending rank -- is built once in shared memory with, per
// candidate, the byte of sibling octants rho whose E2 it belongs to.  Because
// the E2 condition |2 delta + o - rho| <= 1 is symmetric under
// (delta, o, rho) -> (-delta, rho, o), that byte is e2_child_mask(-delta, o).
// Every receiver child then splits C by one ballot per 32 candidates: its E2
// and E4 lists come out in ascending order as contiguous, coalesced stores.
// Row starts are written rebased to the job's own lists.
constexpr int kCand = 27 * 8;  // at most 27 neighbours x 8 children
constexpr int kNear = 64;      // candidates in some sibling's E2: the 4x4x4 block
constexpr uint32_t kStage = 4 * 189 + 4;  // four E4 lists, and up to 3 entries of alignment
constexpr uint32_t kStageMin = 128;       // candidates of a parent whose E4 lists are staged
constexpr uint32_t kStageJob = 1u << 25;  // E4 entries of a job's level whose lists are staged

// A warp's current job in the fill kernel.
struct WarpJob {
  ListCtx a;
  uint32_t* out2;  // the job's row starts, level l
  uint32_t* out4;
  uint32_t G2, G4;  // the job's first entries in the level's lists
  uint32_t j, jstart, jend;
  uint32_t big;     // the job's E4 lists at this level outgrow L2
};

// kCodes: also write the E2 entries' offset codes for the next level (every
// level but the last).
template <bool kCodes>
__global__ void __launch_bounds__(kListThreads, 4) list_fill_kernel(const Seg* __restrict__ segs,
                                                                const Job* __restrict__ jobs,
                                                                uint32_t njobs, int l,
                                                                const ListLevel* lvls,
                                                                DevStatus* st) {
  __shared__ uint32_t s_rank[kListWarps][kCand];
  // per candidate: its sibling byte, and above it (lane of its neighbour) * 8 + octant
  __shared__ uint16_t s_sib[kListWarps][kCand];
  __shared__ uint32_t s_nrank[kListWarps][kNear];
  __shared__ uint16_t s_nsib[kListWarps][kNear];
  __shared__ WarpJob s_job[kListWarps];
  __shared__ __align__(16) uint32_t s_stage[kListWarps][kStage];  // E4 lists of four siblings
  if (failed(st)) return;  // set before this launch: the same for every thread
  const ListLevel& LV = lvls[l];
  if ((LV.total[0] >> 32) != 0 || (LV.total[1] >> 32) != 0) return;  // capacity error set
  // The level's arrays in registers: the list stores must not force reloads
  // of the descriptor.
  const uint32_t* const jprefix = LV.jprefix;
  const uint32_t* const work2 = LV.work2;
  const uint32_t* const work4 = LV.work4;
  uint32_t* const idx2 = LV.idx2;
  uint32_t* const idx4 = LV.idx4;
  uint64_t* const lbase = LV.base;
  uint64_t* const lnnz = LV.nnz;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = lanemask_lt();
  uint32_t* crank = s_rank[warp];
  uint16_t* csib = s_sib[warp];
  uint32_t* nrank = s_nrank[warp];
  uint16_t* nsibm = s_nsib[warp];
  uint32_t* stage = s_stage[warp];
  uint8_t* const code2 = LV.code2;
  const uint32_t npar = jprefix[njobs];
  const BlockRange br = block_range(npar);
  // The warp's current job lives in shared memory, not in registers: the
  // list loops below need the registers for the eight siblings' cursors.
  WarpJob& J = s_job[warp];
  uint32_t jend = 0;
  for (uint32_t g = br.g0 + warp; g < br.g1; g += kListWarps) {
    if (g >= jend) {  // g only grows: look its job up when it leaves the current one
      if (lane == 0) {
        const uint32_t j = find_job(jprefix, njobs, g);
        J.a = make_ctx(segs, jobs[j], l, lvls, j);
        J.j = j;
        J.jstart = jprefix[j];
        J.jend = jprefix[j + 1];
        J.out2 = jobs[j].out2[l];
        J.out4 = jobs[j].out4[l];
        J.G2 = work2[J.a.region];
        J.G4 = work4[J.a.region];
        J.big = work4[J.a.region + J.a.nrecv] - J.G4 >= kStageJob;
      }
      __syncwarp();
      jend = J.jend;
    }
    const uint32_t p = g - J.jstart;
    const uint32_t region = J.a.region, G2 = J.G2, G4 = J.G4;
    const bool big = J.big != 0;
    uint32_t* const out2 = J.out2;
    uint32_t* const out4 = J.out4;
    // The receiver children of p (at most 8): lane j fetches child j's octant
    // and list starts up front, so their loads overlap the neighbour loads.
    const uint32_t c0 = J.a.rchild_up[p];
    const uint32_t c1 = min(J.a.rchild_up[p + 1], c0 + 8u);  // (at most 8 in a whole tree)
    uint32_t my_rho = 0, my_o2 = 0, my_o4 = 0;
    if (c0 + lane < c1) {
      my_rho = (uint32_t)(J.a.rkey[c0 + lane] & 7u);
      my_o2 = work2[region + c0 + lane];
      my_o4 = work4[region + c0 + lane];
      out2[c0 + lane] = my_o2 - G2;
      out4[c0 + lane] = my_o4 - G4;
    }
    if (g + 1 == jend) {  // the job's last parent closes its rows
      const uint32_t nrecv = J.a.nrecv, j = J.j;
      const uint32_t e2 = work2[region + nrecv], e4 = work4[region + nrecv];
      if (lane == 0) {
        out2[nrecv] = e2 - G2;
        out4[nrecv] = e4 - G4;
        lbase[2 * j] = G2;
        lbase[2 * j + 1] = G4;
        lnnz[2 * j] = e2 - G2;
        lnnz[2 * j + 1] = e4 - G4;
      }
    }
    const Neighbour q = load_neighbour(J.a, l, p, lane);
    const uint32_t nsib = c1 - c0;
    // this lane's neighbour's part of the position sum P (see the E2 loop)
    const int pbase = (2 * q.dx + 1) + 3 * (2 * q.dy + 1) + 9 * (2 * q.dz + 1);

    // Candidates C (children of p's neighbours, ascending rank) and the near
    // candidates (those in some sibling's E2), each with its sibling byte.
    const uint32_t nc = __popc(q.occ);
    uint32_t e = warp_excl(nc, lane);
    const uint32_t total = __shfl_sync(0xffffffffu, e + nc, 31);
    {
      // The sibling byte of child o of this neighbour factors by axis: bit
      // rho is set iff axis_mask(-delta, o's bit, ...) holds on every axis.
      // Branch-free over the eight octants (predicated stores).
      const uint32_t mx0 = axis_mask(-q.dx, 0u, 0x55u, 0xaau), mx1 = axis_mask(-q.dx, 1u, 0x55u, 0xaau);
      const uint32_t my0 = axis_mask(-q.dy, 0u, 0x33u, 0xccu), my1 = axis_mask(-q.dy, 1u, 0x33u, 0xccu);
      const uint32_t mz0 = axis_mask(-q.dz, 0u, 0x0fu, 0xf0u), mz1 = axis_mask(-q.dz, 1u, 0x0fu, 0xf0u);
      uint32_t rank = q.child;
      const uint32_t lane8 = (uint32_t)lane << 11;  // (lane * 8) << 8
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        if ((q.occ >> o) & 1u) {
          crank[e] = rank++;
          csib[e] = (uint16_t)((((o & 1) ? mx1 : mx0) & ((o & 2) ? my1 : my0) & ((o & 4) ? mz1 : mz0)) |
                               lane8 | ((uint32_t)o << 8));
          ++e;
        }
      }
    }
    __syncwarp();
    uint32_t nnear = 0;
    for (uint32_t c = 0; c < total; c += 32) {
      const uint32_t i = c + lane;
      const uint32_t sb16 = i < total ? csib[i] : 0u;
      const bool near = (sb16 & 0xffu) != 0u;
      const uint32_t bn = __ballot_sync(0xffffffffu, near);
      if (near) {
        const uint32_t k = nnear + __popc(bn & lt);
        nrank[k] = crank[i];
        nsibm[k] = (uint16_t)sb16;
      }
      nnear += __popc(bn);
    }
    __syncwarp();

    uint32_t sbit[8], w2[8], w4[8];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      sbit[jj] = 1u << __shfl_sync(0xffffffffu, my_rho, jj);
      w2[jj] = __shfl_sync(0xffffffffu, my_o2, jj);
      w4[jj] = __shfl_sync(0xffffffffu, my_o4, jj);
    }
    // E2 of sibling jj: the near candidates whose byte has bit rho_jj; E4:
    // the candidates without it.  A parent with all eight children runs the
    // eight siblings as straight-line code; otherwise absent siblings (the
    // same for the whole warp) are skipped.
    auto emit = [&](auto all_tag) {
      constexpr bool kAll = decltype(all_tag)::value;
      for (uint32_t c = 0; c < nnear; c += 32) {
        const uint32_t i = c + lane;
        const uint32_t v = i < nnear ? nrank[i] : 0u;
        const uint32_t sb16 = i < nnear ? nsibm[i] : 0u;
        const uint32_t sb = sb16 & 0xffu;
        // Position of the candidate, child o of the neighbour at delta, among
        // the parent's children: p = 2 delta + o per axis; P = sum over axes of
        // 3^axis (p + 1).  Minus the sibling's (rx + 3 ry + 9 rz) it is the
        // entry's offset code (dx+1) + 3(dy+1) + 9(dz+1) from that sibling.
        uint32_t P = 0;
        if (kCodes) {
          const uint32_t cq = sb16 >> 8, o = cq & 7u;
          P = (uint32_t)__shfl_sync(0xffffffffu, pbase, (int)(cq >> 3)) + (o & 1u) +
              3u * ((o >> 1) & 1u) + 9u * (o >> 2);
        }
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          if (kAll || (uint32_t)jj < nsib) {
            const uint32_t hit = sb & sbit[jj];
            const uint32_t b2 = __ballot_sync(0xffffffffu, hit != 0u);
            const uint32_t at = w2[jj] + __popc(b2 & lt);
            st_cs_if(idx2 + at, v, hit);
            if (kCodes) {
              const uint32_t rho = __ffs(sbit[jj]) - 1u;
              const uint32_t R = (rho & 1u) + 3u * ((rho >> 1) & 1u) + 9u * (rho >> 2);
              if (hit) code2[at] = (uint8_t)(P - R);
            }
            w2[jj] += __popc(b2);
          }
        }
      }
      // E4.  Where a job's E4 lists of the level outgrow L2, a parent with all eight
      // children and many candidates gathers its E4 lists four siblings at a
      // time in the warp's stage (they are adjacent in idx4; the stage is
      // aligned like idx4) and writes them as whole 16-byte vectors, so that
      // DRAM sees whole sectors; elsewhere the entries are stored directly
      // (partial writes merge in L2 there).
      if (kAll && big && total >= kStageMin) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint32_t a0 = w4[4 * h], sb0 = a0 & ~3u;
          for (uint32_t c = 0; c < total; c += 32) {
            const uint32_t i = c + lane;
            const uint32_t v = i < total ? crank[i] : 0u;
            const uint32_t sb = i < total ? (csib[i] & 0xffu) : 0xffu;  // past the end: never stored
#pragma unroll
            for (int jj = 4 * h; jj < 4 * h + 4; ++jj) {
              const uint32_t hit = sb & sbit[jj];
              const uint32_t b4 = __ballot_sync(0xffffffffu, hit == 0u);
              const uint32_t at = w4[jj] + __popc(b4 & lt) - sb0;
              if (hit == 0u && at < kStage) stage[at] = v;
              w4[jj] += __popc(b4);
            }
          }
          __syncwarp();
          // the half's entries [a0, a1): head and tail one by one, the rest
          // as 16-byte vectors
          const uint32_t a1 = w4[4 * h + 3];
          const uint32_t v0 = min((a0 + 3u) & ~3u, a1), v1 = max(a1 & ~3u, v0);
          if ((uint32_t)lane < v0 - a0) __stcs(idx4 + a0 + lane, stage[a0 + lane - sb0]);
          if ((uint32_t)lane < a1 - v1) __stcs(idx4 + v1 + lane, stage[v1 + lane - sb0]);
          for (uint32_t e = v0 + 4u * lane; e < v1; e += 128u)
            __stcs(reinterpret_cast<uint4*>(idx4 + e),
                   *reinterpret_cast<const uint4*>(stage + (e - sb0)));
          __syncwarp();
        }
      } else {
        for (uint32_t c = 0; c < total; c += 32) {
          const uint32_t i = c + lane;
          const uint32_t v = i < total ? crank[i] : 0u;
          const uint32_t sb = i < total ? (csib[i] & 0xffu) : 0xffu;  // past the end: never stored
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            if (kAll || (uint32_t)jj < nsib) {
              const uint32_t hit = sb & sbit[jj];
              const uint32_t b4 = __ballot_sync(0xffffffffu, hit == 0u);
              st_cs_if_zero(idx4 + w4[jj] + __popc(b4 & lt), v, hit);
              w4[jj] += __popc(b4);
            }
          }
        }
      }
    };
    if (nsib == 8)
      emit(std::true_type{});
    else
      emit(std::false_type{});
    __syncwarp();
  }
}

void launch_list_count(const Seg* segs, const Job* jobs, uint32_t njobs, int l,
                       const ListLevel* lvls, DevStatus* st, cudaStream_t s) {
  list_count_kernel<<<152u * 8u, kListThreads, 0, s>>>(segs, jobs, njobs, l, lvls, st);
}

void launch_list_fill(const Seg* segs, const Job* jobs, uint32_t njobs, int l,
                      const ListLevel* lvls, bool codes, DevStatus* st, cudaStream_t s) {
  if (codes)
    list_fill_kernel<true><<<152u * 8u, kListThreads, 0, s>>>(segs, jobs, njobs, l, lvls, st);
  else
    list_fill_kernel<false><<<152u * 8u, kListThreads, 0, s>>>(segs, jobs, njobs, l, lvls, st);
}

// ---------------------------------------------------------------------------
// Exclusive prefix sum of u32 counts in place, single pass with decoupled
// look-back (the CSR row starts NeighborBookmark of Alg. 4).
__host__ __device__ inline uint32_t scan_tiles_of(uint32_t cap) {
  const uint64_t t = ((uint64_t)cap + kScanTile - 1) / kScanTile;
  return t == 0 ? 1u : (uint32_t)t;
}

uint32_t scan_tiles(uint32_t cap) { return scan_tiles_of(cap); }

// Up to two arrays of the same length in one launch (the E2 and E4 counts of
// a level): tickets [0, need) scan the first, [need, 2 need) the second, each
// with its own look-back words and total.
struct ScanArray {
  uint32_t* data;
  uint64_t* status;
  uint64_t* total64;
};

__global__ void __launch_bounds__(kScanThreads) scan_u32_kernel(ScanArray a0, ScanArray a1,
                                                               const uint32_t* count_dev,
                                                               uint32_t cap, uint32_t* counter,
                                                               DevStatus* st, uint64_t wait_ns) {
  constexpr int W = kScanThreads / 32;
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_wsum[W];
  __shared__ uint64_t s_prev;
  const uint32_t count = (count_dev && *count_dev < cap) ? *count_dev : cap;
  const uint32_t need = scan_tiles_of(count);
  if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1u);
  __syncthreads();
  const uint32_t ticket = s_tile;
  const bool second = ticket >= need;
  if (second && (a1.data == nullptr || ticket >= 2 * need)) return;
  const uint32_t tile = second ? ticket - need : ticket;
  uint32_t* const data = second ? a1.data : a0.data;
  uint64_t* const status = second ? a1.status : a0.status;
  uint64_t* const total64 = second ? a1.total64 : a0.total64;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t i0 = (uint64_t)tile * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t sum = 0;
  // A thread's items are consecutive: four 16-byte loads (and stores) when
  // the array is 16-byte aligned and all of them are in range.
  const bool vec = ((reinterpret_cast<uintptr_t>(data) & 15u) == 0) && i0 + kScanItems <= count;
  if (vec) {
    const uint4* p4 = reinterpret_cast<const uint4*>(data + i0);
#pragma unroll
    for (int k = 0; k < kScanItems / 4; ++k) {
      const uint4 q = p4[k];
      v[4 * k] = q.x;
      v[4 * k + 1] = q.y;
      v[4 * k + 2] = q.z;
      v[4 * k + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) v[k] = (i0 + k < count) ? data[i0 + k] : 0u;
  }
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) sum += v[k];
  uint32_t x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t run = 0;
    if (lane == 0) {
      for (int w = 0; w < W; ++w) {
        const uint32_t c = s_wsum[w];
        s_wsum[w] = run;
        run += c;
      }
    }
    run = __shfl_sync(0xffffffffu, run, 0);
    uint64_t prev = 0;
    if (tile == 0) {
      if (lane == 0) st_relaxed(status, kFlagIncl | run);
    } else {
      if (lane == 0) st_relaxed(status + tile, kFlagAgg | run);
      prev = lookback_warp(status, tile, 1, st, wait_ns);
      if (lane == 0) st_relaxed(status + tile, kFlagIncl | (prev + run));
    }
    if (lane == 0) {
      s_prev = prev;
      if (tile == need - 1) {
        const uint64_t total = prev + run;
        if (total64) *total64 = total;
        data[count] = (uint32_t)total;
        if (total >> 32) set_error(st, FMM_ERR_CAPACITY);
      }
    }
  }
  __syncthreads();
  uint64_t off = s_prev + s_wsum[warp] + (x - sum);
  if (vec) {
    uint4* p4 = reinterpret_cast<uint4*>(data + i0);
#pragma unroll
    for (int k = 0; k < kScanItems / 4; ++k) {
      uint4 q;
      q.x = (uint32_t)off;
      off += v[4 * k];
      q.y = (uint32_t)off;
      off += v[4 * k + 1];
      q.z = (uint32_t)off;
      off += v[4 * k + 2];
      q.w = (uint32_t)off;
      off += v[4 * k + 3];
      p4[k] = q;
    }
  } else {
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      if (i0 + k < count) data[i0 + k] = (uint32_t)off;
      off += v[k];
    }
  }
}

void launch_scan_u32(uint32_t* data, const uint32_t* count_dev, uint32_t cap, uint64_t* status,
                     uint32_t* counter, uint64_t* total64, DevStatus* st, uint64_t wait_ns,
                     cudaStream_t s) {
  scan_u32_kernel<<<scan_tiles(cap), kScanThreads, 0, s>>>(ScanArray{data, status, total64},
                                                           ScanArray{nullptr, nullptr, nullptr},
                                                           count_dev, cap, counter, st, wait_ns);
}

void launch_scan_u32_pair(uint32_t* data0, uint64_t* status0, uint64_t* total0, uint32_t* data1,
                          uint64_t* status1, uint64_t* total1, uint32_t cap, uint32_t* counter,
                          DevStatus* st, uint64_t wait_ns, cudaStream_t s) {
  scan_u32_kernel<<<2 * scan_tiles(cap), kScanThreads, 0, s>>>(
      ScanArray{data0, status0, total0}, ScanArray{data1, status1, total1}, nullptr, cap, counter,
      st, wait_ns);
}

}  // namespace fmm
