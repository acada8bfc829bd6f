// api.cu -- the C ABI (include/fmmds.h): context, arena, and the build
// pipeline of Alg. 5 on one stream.
//
// Per set (sources, then receivers; once if both are the same array):
//   upfront digit histograms -> digit offsets -> onesweep passes (the first
//   one forms the Morton keys from the coordinates) -> finishing sort inside
//   boxes (permutation) fused with the boxes of all levels -> child
//   occupancy.
// Then, after one read-back of the box counts (for list capacities and the
// cluster-size level), for l = 2..L: list counts -> two prefix sums -> fill.
// A final read-back returns sizes and the device status word.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fmm_internal.cuh"

using namespace fmm;

namespace {

struct Chunk {
  void* ptr;
  size_t bytes;
};

struct PendingTime {
  const char* name;
  cudaEvent_t a, b;
};

struct TimeAcc {
  std::string name;
  uint64_t launches;
  double ms;
};

// Arrays of one point set.
struct SetArrays {
  uint32_t n = 0;
  const float* xyz = nullptr;
  uint32_t* perm = nullptr;
  LevelArrays lv{};
  uint32_t* nbox_dev = nullptr;    // [kLevels]
  uint32_t* maxocc_dev = nullptr;  // [kLevels]
  uint32_t cap[kLevels] = {};
  uint64_t* skeys = nullptr;  // keys sorted by the top 3*Ls bits
  uint32_t* svals = nullptr;
  int Ls = 0;
};

}  // namespace

struct fmm_ctx {
  int device = 0;
  fmm_alloc_fn alloc = nullptr;
  fmm_free_fn free_fn = nullptr;
  void* user = nullptr;
  std::vector<Chunk> chunks;
  size_t cur = 0, off = 0;
  size_t peak_request = 0;
  DevStatus* st = nullptr;          // persistent device status word
  void* host_buf = nullptr;         // pinned read-back buffer
  cudaStream_t stream = nullptr;    // stream of the call in progress
  bool timing = false;
  std::vector<PendingTime> pending;
  std::vector<cudaEvent_t> event_pool;
  std::vector<TimeAcc> acc;
  uint64_t launches = 0;
  uint64_t last_launches = 0;
  fmm_tuning tuning{FMM_SORT_RTS};
};

namespace {

constexpr size_t kHostBuf = 1 << 16;
// Largest list capacity (bytes) reserved from the box-count bounds alone;
// above it the box counts are read back first.
constexpr uint64_t kAsyncListBytes = 16ull << 30;
constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

void* raw_alloc(fmm_ctx* c, size_t bytes) {
  if (c->alloc) return c->alloc(bytes, (void*)c->stream, c->user);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void raw_free(fmm_ctx* c, void* p, size_t bytes) {
  if (!p) return;
  if (c->free_fn)
    c->free_fn(p, bytes, (void*)c->stream, c->user);
  else
    cudaFree(p);
}

void arena_release(fmm_ctx* c) {
  for (auto& ch : c->chunks) raw_free(c, ch.ptr, ch.bytes);
  c->chunks.clear();
  c->cur = c->off = 0;
}

// Starts a build: outputs of the previous build are dropped.  Several chunks
// left by a growing build are merged into one.
int arena_reset(fmm_ctx* c, size_t expect) {
  size_t total = 0;
  for (auto& ch : c->chunks) total += ch.bytes;
  if (c->chunks.size() > 1 || total < expect) {
    const size_t want = std::max(total, expect);
    arena_release(c);
    if (want) {
      void* p = raw_alloc(c, want);
      if (!p) return FMM_ERR_OOM;
      c->chunks.push_back({p, want});
    }
  }
  c->cur = c->off = 0;
  return FMM_OK;
}

template <class T>
T* arena_get(fmm_ctx* c, size_t count, int* err) {
  const size_t bytes = align_up(std::max<size_t>(count * sizeof(T), 1));
  while (c->cur < c->chunks.size()) {
    Chunk& ch = c->chunks[c->cur];
    if (c->off + bytes <= ch.bytes) {
      T* p = reinterpret_cast<T*>(static_cast<char*>(ch.ptr) + c->off);
      c->off += bytes;
      return p;
    }
    ++c->cur;
    c->off = 0;
  }
  size_t grow = 0;
  for (auto& ch : c->chunks) grow += ch.bytes;
  const size_t want = std::max(bytes, std::max<size_t>(grow, 64u << 20));
  void* p = raw_alloc(c, want);
  if (!p) {
    *err = FMM_ERR_OOM;
    return nullptr;
  }
  c->chunks.push_back({p, want});
  c->cur = c->chunks.size() - 1;
  c->off = bytes;
  return reinterpret_cast<T*>(p);
}

cudaEvent_t get_event(fmm_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

// Wraps one kernel launch: counts it and, with timing on, brackets it with
// events on the build's stream.
struct Launch {
  fmm_ctx* c;
  const char* name;
  cudaEvent_t a = nullptr;
  Launch(fmm_ctx* ctx, const char* nm) : c(ctx), name(nm) {
    ++c->launches;
    if (c->timing) {
      a = get_event(c);
      cudaEventRecord(a, c->stream);
    }
  }
  ~Launch() {
    if (c->timing) {
      cudaEvent_t b = get_event(c);
      cudaEventRecord(b, c->stream);
      c->pending.push_back({name, a, b});
    }
  }
};

void collect_times(fmm_ctx* c) {
  for (auto& p : c->pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    auto it = std::find_if(c->acc.begin(), c->acc.end(),
                           [&](const TimeAcc& t) { return t.name == p.name; });
    if (it == c->acc.end()) {
      c->acc.push_back({p.name, 0, 0.0});
      it = c->acc.end() - 1;
    }
    it->launches += 1;
    it->ms += ms;
    c->event_pool.push_back(p.a);
    c->event_pool.push_back(p.b);
  }
  c->pending.clear();
}

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return FMM_OK;
  cudaGetLastError();
  return FMM_ERR_CUDA;
}

#define FMM_TRY(expr)             \
  do {                            \
    int _s = (expr);              \
    if (_s != FMM_OK) return _s;  \
  } while (0)

#define FMM_CUDA(expr) FMM_TRY(cuda_status(expr))

uint64_t min_u64(uint64_t a, uint64_t b) { return a < b ? a : b; }

// Capacity of level l for n points: at most min(n, 8^l) non-empty boxes.
uint32_t level_cap(uint32_t n, int l) {
  const uint64_t full = l >= 11 ? ~0ull : (1ull << (3 * l));
  return (uint32_t)min_u64(n, full);
}

// Sort depth: at least the tree depth, and deep enough that a box averages
// about 8 points, which keeps the finishing sort short; then as deep as the
// radix passes it needs allow at 8 bits per pass (3 passes sort 24 bits:
// level 8 costs no more than level 7).
int sort_level(uint32_t n, int L) {
  int lvl = 1;
  while (lvl < kMaxLevel && ((uint64_t)n >> (3 * lvl)) > 8) ++lvl;
  lvl = std::max(std::max(lvl, L), 1);
  const int passes = (3 * lvl + 7) / 8;
  return std::min(kMaxLevel, std::max(lvl, 8 * passes / 3));
}

uint64_t wait_ns_of(const fmm_params& p) {
  return (uint64_t)(p.wait_ms ? p.wait_ms : 2000u) * 1000000ull;
}

// Radix passes over the (key, index) pairs of one set: the first pass forms
// the keys from the coordinates.  Output in (*kout, *vout); with
// vals_last != null the last pass writes its values there instead.
int sort_pairs(fmm_ctx* c, const SortPlan& plan, const float* xyz, uint32_t n, bool stall,
               uint64_t wait_ns, uint64_t* ka, uint32_t* va, uint64_t* kb, uint32_t* vb,
               uint32_t* vals_last, uint64_t** kout, uint32_t** vout) {
  cudaStream_t s = c->stream;
  int err = FMM_OK;
  *kout = nullptr;
  *vout = nullptr;
  if (n == 0 || plan.passes == 0) return FMM_OK;
  const uint32_t radix = 1u << plan.bits;
  // The bounded-wait test needs a look-back pass: it always takes onesweep.
  const bool onesweep = stall || c->tuning.sort_kind == FMM_SORT_ONESWEEP;
  uint32_t* hist = nullptr;
  uint64_t* sstatus = nullptr;
  uint32_t* counters = nullptr;
  size_t per_pass = 0;
  if (onesweep) {
    per_pass = (size_t)plan.ntiles * radix;
    const size_t zb = align_up(sizeof(uint32_t) * 8 * kRadixMax) +
                      align_up(sizeof(uint64_t) * per_pass * plan.passes) +
                      align_up(sizeof(uint32_t) * 16);
    char* z = arena_get<char>(c, zb, &err);
    if (err) return err;
    FMM_CUDA(cudaMemsetAsync(z, 0, zb, s));
    hist = reinterpret_cast<uint32_t*>(z);
    sstatus = reinterpret_cast<uint64_t*>(z + align_up(sizeof(uint32_t) * 8 * kRadixMax));
    counters = reinterpret_cast<uint32_t*>(z + align_up(sizeof(uint32_t) * 8 * kRadixMax) +
                                           align_up(sizeof(uint64_t) * per_pass * plan.passes));
    {
      Launch L(c, "upfront_hist");
      launch_upfront_hist(xyz, n, plan, hist, c->st, s);
    }
    Launch L(c, "digit_scan");
    launch_digit_scan(plan, hist, s);
  } else {
    per_pass = (size_t)radix * plan.ntiles;  // digit-major tile histogram
    const uint32_t stiles = scan_tiles((uint32_t)per_pass);
    const size_t zb = align_up(sizeof(uint64_t) * stiles) * plan.passes +
                      align_up(sizeof(uint32_t) * 16);
    char* z = arena_get<char>(c, zb, &err);
    hist = arena_get<uint32_t>(c, (per_pass + 1) * plan.passes, &err);
    if (err) return err;
    FMM_CUDA(cudaMemsetAsync(z, 0, zb, s));
    sstatus = reinterpret_cast<uint64_t*>(z);
    counters = reinterpret_cast<uint32_t*>(z + align_up(sizeof(uint64_t) * stiles) * plan.passes);
  }
  uint64_t* kin = nullptr;
  uint32_t* vin = nullptr;
  for (int p = 0; p < plan.passes; ++p) {
    uint64_t* ko = (p & 1) ? kb : ka;
    uint32_t* vo = (p & 1) ? vb : va;
    if (vals_last && p == plan.passes - 1) vo = vals_last;
    if (onesweep) {
      Launch L(c, "onesweep");
      launch_onesweep_pass(p, xyz, kin, vin, ko, vo, n, plan, hist + p * kRadixMax,
                           sstatus + (size_t)p * per_pass, counters + p, c->st, wait_ns,
                           (stall && p == 0 && plan.ntiles > 2) ? 1 : -1, s);
    } else {
      uint32_t* h = hist + (per_pass + 1) * p;
      const uint32_t stiles = scan_tiles((uint32_t)per_pass);
      {
        Launch L(c, "tile_hist");
        launch_tile_hist(p, xyz, kin, n, plan, h, c->st, s);
      }
      {
        Launch L(c, "scan");
        launch_scan_u32(h, nullptr, (uint32_t)per_pass, sstatus + (size_t)stiles * p,
                        counters + p, nullptr, c->st, wait_ns, s);
      }
      Launch L(c, "rts_scatter");
      // The first pass may leave equal digits in any order when a finishing
      // sort follows; the full-key fallback writes the order directly.
      launch_rts_scatter(p, xyz, kin, vin, ko, vo, n, plan, h, vals_last != nullptr || p > 0,
                         c->st, wait_ns, s);
    }
    kin = ko;
    vin = vo;
  }
  *kout = kin;
  *vout = vin;
  return FMM_OK;
}

// Keys, order, boxes of levels 0..Lb and (sources) occupancy for one set.
int build_set(fmm_ctx* c, SetArrays* S, int Lb, bool need_occ, bool stall, uint64_t wait_ns,
              bool full_sort) {
  cudaStream_t s = c->stream;
  int err = FMM_OK;
  const uint32_t n = S->n;
  S->Ls = full_sort ? kMaxLevel : std::max(sort_level(n, Lb), Lb);
  const SortPlan plan = make_sort_plan(n, S->Ls);

  // Zero-initialised scratch of the box pass: look-back words, tile counter,
  // box counts.
  const uint32_t btiles = boxes_tiles(n);
  const uint32_t ctiles = coarse_tiles(level_cap(n, Lb));
  const size_t zero_bytes = align_up(sizeof(uint64_t) * (size_t)btiles) +
                            align_up(sizeof(uint64_t) * (size_t)ctiles * kLevels) +
                            align_up(sizeof(uint32_t) * 16) +
                            align_up(sizeof(uint32_t) * kLevels * 2);
  char* z = arena_get<char>(c, zero_bytes, &err);
  if (!z) return err;
  FMM_CUDA(cudaMemsetAsync(z, 0, zero_bytes, s));
  uint64_t* bstatus = reinterpret_cast<uint64_t*>(z);
  z += align_up(sizeof(uint64_t) * (size_t)btiles);
  uint64_t* cstatus = reinterpret_cast<uint64_t*>(z);
  z += align_up(sizeof(uint64_t) * (size_t)ctiles * kLevels);
  uint32_t* counters = reinterpret_cast<uint32_t*>(z);
  z += align_up(sizeof(uint32_t) * 16);
  S->nbox_dev = reinterpret_cast<uint32_t*>(z);
  S->maxocc_dev = S->nbox_dev + kLevels;

  uint64_t* ka = arena_get<uint64_t>(c, n, &err);
  uint32_t* va = arena_get<uint32_t>(c, n, &err);
  uint64_t* kb = arena_get<uint64_t>(c, n, &err);
  uint32_t* vb = arena_get<uint32_t>(c, n, &err);
  if (!S->perm) S->perm = arena_get<uint32_t>(c, n, &err);
  if (err) return err;
  uint64_t* kin = nullptr;
  uint32_t* vin = nullptr;
  FMM_TRY(sort_pairs(c, plan, S->xyz, n, stall, wait_ns, ka, va, kb, vb, nullptr, &kin, &vin));
  S->skeys = kin;
  S->svals = vin;

  // Boxes of levels 0..Lb, fused with the finishing sort (permutation).
  for (int l = 0; l <= Lb; ++l) {
    S->cap[l] = level_cap(n, l);
    S->lv.cap[l] = S->cap[l];
    S->lv.key[l] = arena_get<uint64_t>(c, S->cap[l], &err);
    S->lv.off[l] = arena_get<uint32_t>(c, (size_t)S->cap[l] + 1, &err);
    S->lv.parent[l] = arena_get<uint32_t>(c, S->cap[l], &err);
    if (l < Lb) S->lv.child[l] = arena_get<uint32_t>(c, (size_t)S->cap[l] + 1, &err);
    if (l < Lb && need_occ) S->lv.occ[l] = arena_get<uint8_t>(c, S->cap[l], &err);
  }
  if (err) return err;
  {
    Launch L(c, "finish_boxes");
    launch_finish_boxes(kin ? kin : ka, vin ? vin : va, n, Lb, S->Ls, S->lv, S->perm, bstatus,
                        counters + 15, S->nbox_dev, c->st, wait_ns, s);
  }
  if (Lb >= 1) {
    Launch L(c, "coarse_boxes");
    launch_coarse_boxes(Lb, S->lv, n, cstatus, counters + 14, S->nbox_dev, c->st, wait_ns, s);
  }
  if (need_occ && Lb >= 1) {
    Launch L(c, "occupancy");
    launch_occupancy(Lb, S->lv, S->nbox_dev, n, c->st, s);
  }
  return FMM_OK;
}

// Redoes the order of one set with the full 63-bit sort (a box was longer
// than the finishing sort's window).  Only the permutation changes.
int full_sort_perm(fmm_ctx* c, SetArrays* S, uint64_t wait_ns) {
  int err = FMM_OK;
  const uint32_t n = S->n;
  const SortPlan plan = make_sort_plan(n, kMaxLevel);
  uint64_t* ka = arena_get<uint64_t>(c, n, &err);
  uint32_t* va = arena_get<uint32_t>(c, n, &err);
  uint64_t* kb = arena_get<uint64_t>(c, n, &err);
  uint32_t* vb = arena_get<uint32_t>(c, n, &err);
  if (err) return err;
  uint64_t* kout;
  uint32_t* vout;
  return sort_pairs(c, plan, S->xyz, n, false, wait_ns, ka, va, kb, vb, S->perm, &kout, &vout);
}

struct SetReadback {
  uint32_t nbox[kLevels];
  uint32_t maxocc[kLevels];
};

struct Readback {
  DevStatus st;
  SetReadback set[2];
  uint64_t nnz[kLevels][2];
};

void fill_side(const SetArrays& S, int L, const uint32_t* nbox, uint32_t* out_nbox,
               const uint64_t** key, const uint32_t** off, const uint32_t** parent,
               const uint32_t** child, const uint32_t** perm) {
  *perm = S.perm;
  for (int l = 0; l < kLevels; ++l) {
    const bool in = l <= L;
    out_nbox[l] = in ? nbox[l] : 0;
    key[l] = in ? S.lv.key[l] : nullptr;
    off[l] = in ? S.lv.off[l] : nullptr;
    parent[l] = (in && l >= 1) ? S.lv.parent[l] : nullptr;
    child[l] = (l < L) ? S.lv.child[l] : nullptr;
  }
}

int do_build(fmm_ctx* c, const float* src, uint32_t N, const float* recv, uint32_t M,
             const fmm_params& prm, fmm_tree* out) {
  cudaStream_t s = c->stream;
  int err = FMM_OK;
  const uint64_t wait_ns = wait_ns_of(prm);
  const bool stall = (prm.flags & FMM_FLAG_TEST_STALL) != 0;
  const bool aliased = (src == recv) && (N == M);
  const bool smode = prm.L < 0;

  uint64_t expect = 0;
  fmm_query_workspace(N, M, prm, &expect);
  FMM_TRY(arena_reset(c, c->peak_request > expect ? c->peak_request : expect));
  FMM_CUDA(cudaMemsetAsync(c->st, 0, sizeof(DevStatus), s));

  SetArrays S[2];
  S[0].n = N;
  S[1].n = M;
  S[0].xyz = src;
  S[1].xyz = recv;
  if (prm.flags & FMM_FLAG_HOST_INPUT) {
    for (int k = 0; k < (aliased ? 1 : 2); ++k) {
      float* d = arena_get<float>(c, (size_t)S[k].n * 3, &err);
      if (err) return err;
      if (S[k].n)
        FMM_CUDA(cudaMemcpyAsync(d, S[k].xyz, sizeof(float) * 3 * S[k].n,
                                 cudaMemcpyHostToDevice, s));
      S[k].xyz = d;
    }
    if (aliased) S[1].xyz = S[0].xyz;
  }

  // In cluster-size mode the boxes are built down to the sort depth of the
  // larger set; the level is picked from their occupancy.
  const int Lb = smode ? std::max(sort_level(std::max(N, M), 2), 2) : prm.L;
  FMM_TRY(build_set(c, &S[0], Lb, true, stall, wait_ns, false));
  if (aliased) {
    S[1] = S[0];
  } else {
    FMM_TRY(build_set(c, &S[1], Lb, false, false, wait_ns, false));
  }
  if (smode) {
    for (int k = 0; k < (aliased ? 1 : 2); ++k) {
      Launch Lq(c, "max_occupancy");
      launch_max_occupancy(Lb, S[k].lv, S[k].nbox_dev, S[k].n, S[k].maxocc_dev, c->st, s);
    }
  }

  // With a fixed level and list capacities bounded by the box capacities
  // (27 and 189 per receiver box), everything is launched without waiting
  // for the box counts; otherwise read them back first.
  Readback* hb = static_cast<Readback*>(c->host_buf);
  Readback rb1{};
  uint64_t list_bound = 0;
  if (!smode)
    for (int l = 2; l <= prm.L; ++l) list_bound += 4ull * (2 + 27 + 189) * level_cap(M, l);
  const bool async_lists = !smode && list_bound <= kAsyncListBytes;
  if (!async_lists) {
    FMM_CUDA(cudaMemcpyAsync(&hb->st, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    for (int k = 0; k < 2; ++k)
      FMM_CUDA(cudaMemcpyAsync(&hb->set[k], S[k].nbox_dev, sizeof(SetReadback),
                               cudaMemcpyDeviceToHost, s));
    FMM_CUDA(cudaStreamSynchronize(s));
    if (hb->st.code) return (int)hb->st.code;
    rb1 = *hb;
  } else {
    for (int l = 0; l <= prm.L; ++l) {
      rb1.set[0].nbox[l] = level_cap(N, l);
      rb1.set[1].nbox[l] = level_cap(M, l);
    }
  }

  int L = prm.L;
  uint32_t s_unmet = 0;
  if (smode) {
    L = -1;
    for (int l = 2; l <= Lb; ++l) {
      if (rb1.set[0].maxocc[l] <= prm.s && rb1.set[1].maxocc[l] <= prm.s) {
        L = l;
        break;
      }
    }
    if (L < 0) {
      // Not met down to the sort depth: rebuild with the full 63-bit order
      // and every level.
      FMM_CUDA(cudaMemsetAsync(c->st, 0, sizeof(DevStatus), s));
      SetArrays T[2];
      T[0].n = N;
      T[1].n = M;
      T[0].xyz = S[0].xyz;
      T[1].xyz = S[1].xyz;
      FMM_TRY(build_set(c, &T[0], kMaxLevel, true, false, wait_ns, true));
      if (aliased)
        T[1] = T[0];
      else
        FMM_TRY(build_set(c, &T[1], kMaxLevel, false, false, wait_ns, true));
      for (int k = 0; k < (aliased ? 1 : 2); ++k) {
        Launch Lq(c, "max_occupancy");
        launch_max_occupancy(kMaxLevel, T[k].lv, T[k].nbox_dev, T[k].n, T[k].maxocc_dev, c->st,
                             s);
      }
      FMM_CUDA(cudaMemcpyAsync(&hb->st, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
      for (int k = 0; k < 2; ++k)
        FMM_CUDA(cudaMemcpyAsync(&hb->set[k], T[k].nbox_dev, sizeof(SetReadback),
                                 cudaMemcpyDeviceToHost, s));
      FMM_CUDA(cudaStreamSynchronize(s));
      if (hb->st.code) return (int)hb->st.code;
      rb1 = *hb;
      S[0] = T[0];
      S[1] = T[1];
      L = kMaxLevel;
      s_unmet = 1;
      for (int l = 2; l <= kMaxLevel; ++l) {
        if (rb1.set[0].maxocc[l] <= prm.s && rb1.set[1].maxocc[l] <= prm.s) {
          L = l;
          s_unmet = 0;
          break;
        }
      }
    }
  }
  if (!async_lists && rb1.st.seg_long) {
    // A box outran the finishing sort: redo the order(s) with all 63 bits.
    for (int k = 0; k < (aliased ? 1 : 2); ++k) FMM_TRY(full_sort_perm(c, &S[k], wait_ns));
    if (aliased) S[1].perm = S[0].perm;
  }

  // Lists, levels 2..L.
  uint32_t* lst_off[2][kLevels] = {};
  uint32_t* lst_idx[2][kLevels] = {};
  uint64_t* nnz_dev = arena_get<uint64_t>(c, (size_t)kLevels * 2, &err);
  if (err) return err;
  FMM_CUDA(cudaMemsetAsync(nnz_dev, 0, sizeof(uint64_t) * kLevels * 2, s));
  for (int l = 2; l <= L; ++l) {
    const uint32_t nr = rb1.set[1].nbox[l];
    lst_off[0][l] = arena_get<uint32_t>(c, (size_t)nr + 1, &err);
    lst_off[1][l] = arena_get<uint32_t>(c, (size_t)nr + 1, &err);
    lst_idx[0][l] = arena_get<uint32_t>(c, (size_t)nr * 27, &err);
    lst_idx[1][l] = arena_get<uint32_t>(c, (size_t)nr * 189, &err);
    const uint32_t tiles = scan_tiles(nr);
    const size_t zb = align_up(sizeof(uint64_t) * tiles) * 2 + align_up(sizeof(uint32_t) * 2);
    char* z = arena_get<char>(c, zb, &err);
    if (err) return err;
    FMM_CUDA(cudaMemsetAsync(z, 0, zb, s));
    uint64_t* st2 = reinterpret_cast<uint64_t*>(z);
    uint64_t* st4 = reinterpret_cast<uint64_t*>(z + align_up(sizeof(uint64_t) * tiles));
    uint32_t* cnt = reinterpret_cast<uint32_t*>(z + 2 * align_up(sizeof(uint64_t) * tiles));

    ListArgs a{};
    a.l = l;
    a.nbox_recv = S[1].nbox_dev;
    a.nbox_src = S[0].nbox_dev;
    a.rkey_up = S[1].lv.key[l - 1];
    a.rchild_up = S[1].lv.child[l - 1];
    a.rkey = S[1].lv.key[l];
    a.e2_off_up = l >= 3 ? lst_off[0][l - 1] : nullptr;
    a.e2_idx_up = l >= 3 ? lst_idx[0][l - 1] : nullptr;
    a.skey_up = S[0].lv.key[l - 1];
    a.schild_up = S[0].lv.child[l - 1];
    a.socc_up = S[0].lv.occ[l - 1];
    a.e2_off = lst_off[0][l];
    a.e4_off = lst_off[1][l];
    a.e2_idx = lst_idx[0][l];
    a.e4_idx = lst_idx[1][l];
    a.nnz = nnz_dev + 2 * l;
    const uint32_t np = rb1.set[1].nbox[l - 1];
    {
      Launch Lk(c, "list_count");
      launch_list_count(a, np, c->st, s);
    }
    {
      Launch Lk(c, "scan");
      launch_scan_u32(a.e2_off, S[1].nbox_dev + l, nr, st2, cnt, nnz_dev + 2 * l, c->st, wait_ns,
                      s);
    }
    {
      Launch Lk(c, "scan");
      launch_scan_u32(a.e4_off, S[1].nbox_dev + l, nr, st4, cnt + 1, nnz_dev + 2 * l + 1, c->st,
                      wait_ns, s);
    }
    {
      Launch Lk(c, "list_fill");
      launch_list_fill(a, np, c->st, s);
    }
  }
  FMM_CUDA(cudaGetLastError());
  FMM_CUDA(cudaMemcpyAsync(&hb->st, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  FMM_CUDA(cudaMemcpyAsync(hb->nnz, nnz_dev, sizeof(uint64_t) * kLevels * 2,
                           cudaMemcpyDeviceToHost, s));
  if (async_lists)
    for (int k = 0; k < 2; ++k)
      FMM_CUDA(cudaMemcpyAsync(&hb->set[k], S[k].nbox_dev, sizeof(SetReadback),
                               cudaMemcpyDeviceToHost, s));
  FMM_CUDA(cudaStreamSynchronize(s));
  if (hb->st.code) return (int)hb->st.code;
  if (async_lists) {
    for (int k = 0; k < 2; ++k) rb1.set[k] = hb->set[k];
    if (hb->st.seg_long) {
      // A box outran the finishing sort: redo the order(s) with all 63 bits.
      for (int k = 0; k < (aliased ? 1 : 2); ++k) FMM_TRY(full_sort_perm(c, &S[k], wait_ns));
      if (aliased) S[1].perm = S[0].perm;
      FMM_CUDA(cudaMemcpyAsync(&hb->st, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
      FMM_CUDA(cudaStreamSynchronize(s));
      if (hb->st.code) return (int)hb->st.code;
    }
  }

  std::memset(out, 0, sizeof(*out));
  out->L = L;
  out->s_unmet = s_unmet;
  out->n_src = N;
  out->n_recv = M;
  fill_side(S[0], L, rb1.set[0].nbox, out->nbox_src, out->key_src, out->off_src, out->parent_src,
            out->child_src, &out->perm_src);
  fill_side(S[1], L, rb1.set[1].nbox, out->nbox_recv, out->key_recv, out->off_recv, out->parent_recv,
            out->child_recv, &out->perm_recv);
  for (int l = 2; l <= L; ++l) {
    out->nnz_e2[l] = hb->nnz[l][0];
    out->nnz_e4[l] = hb->nnz[l][1];
    out->e2_off[l] = lst_off[0][l];
    out->e4_off[l] = lst_off[1][l];
    out->e2_idx[l] = lst_idx[0][l];
    out->e4_idx[l] = lst_idx[1][l];
  }
  size_t used = 0;
  for (size_t i = 0; i < c->chunks.size(); ++i) used += c->chunks[i].bytes;
  c->peak_request = std::max(c->peak_request, used);
  return FMM_OK;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" {

int fmm_create(fmm_ctx** ctx, int device, fmm_alloc_fn alloc, fmm_free_fn free_fn, void* user) {
  if (!ctx || (alloc == nullptr) != (free_fn == nullptr)) return FMM_ERR_ARG;
  *ctx = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return FMM_ERR_CUDA;
  }
  if (device < 0 || device >= ndev) return FMM_ERR_ARG;
  DeviceGuard g(device);
  fmm_ctx* c = new fmm_ctx();
  c->device = device;
  c->alloc = alloc;
  c->free_fn = free_fn;
  c->user = user;
  if (cudaMalloc(&c->st, sizeof(DevStatus)) != cudaSuccess ||
      cudaMallocHost(&c->host_buf, kHostBuf) != cudaSuccess) {
    cudaGetLastError();
    if (c->st) cudaFree(c->st);
    delete c;
    return FMM_ERR_CUDA;
  }
  static_assert(sizeof(Readback) <= kHostBuf, "read-back buffer");
  *ctx = c;
  return FMM_OK;
}

int fmm_destroy(fmm_ctx* c) {
  if (!c) return FMM_ERR_ARG;
  DeviceGuard g(c->device);
  cudaDeviceSynchronize();
  arena_release(c);
  for (auto& p : c->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : c->event_pool) cudaEventDestroy(e);
  cudaFree(c->st);
  cudaFreeHost(c->host_buf);
  delete c;
  return FMM_OK;
}

int fmm_query_workspace(uint32_t N, uint32_t M, fmm_params p, uint64_t* bytes) {
  if (!bytes) return FMM_ERR_ARG;
  if (p.L > kMaxLevel || p.L < -1 || (p.L == -1 && p.s == 0)) return FMM_ERR_LEVEL;
  const int L = p.L >= 0 ? p.L : std::max(sort_level(std::max(N, M), 2), 2);
  uint64_t total = 1 << 20;
  const uint32_t ns[2] = {N, M};
  for (int k = 0; k < 2; ++k) {
    const uint64_t n = ns[k];
    if (p.flags & FMM_FLAG_HOST_INPUT) total += align_up(12 * n);
    total += 4 * align_up(12 * n + 8) / 2 + align_up(4 * n) + (8u << 20);
    total += (n / kSortTile + 1) * 256 * 8 * 8;
    for (int l = 0; l <= L; ++l) total += 4 * align_up(8ull * level_cap(ns[k], l) + 8);
  }
  for (int l = 2; l <= L; ++l) total += align_up(4ull * (2 + 27 + 189) * level_cap(M, l) + 64) + 4096;
  *bytes = total;
  return FMM_OK;
}

int fmm_build(fmm_ctx* c, const float* src_xyz, uint32_t N, const float* recv_xyz, uint32_t M,
              fmm_params params, fmm_tree* out, void* stream) {
  if (!c || !out) return FMM_ERR_ARG;
  if ((N > 0 && !src_xyz) || (M > 0 && !recv_xyz)) return FMM_ERR_ARG;
  if (params.flags & ~(FMM_FLAG_HOST_INPUT | FMM_FLAG_TEST_STALL)) return FMM_ERR_ARG;
  if (params.L > kMaxLevel || params.L < -1 || (params.L == -1 && params.s == 0))
    return FMM_ERR_LEVEL;
  DeviceGuard g(c->device);
  c->stream = static_cast<cudaStream_t>(stream);
  const uint64_t l0 = c->launches;
  int st = do_build(c, src_xyz, N, recv_xyz, M, params, out);
  if (st != FMM_OK) {
    cudaStreamSynchronize(c->stream);
    cudaGetLastError();
  }
  if (c->timing) collect_times(c);
  c->last_launches = c->launches - l0;
  return st;
}

int fmm_morton_keys(fmm_ctx* c, const float* xyz, uint32_t n, uint64_t* keys, void* stream) {
  if (!c || (n > 0 && (!xyz || !keys))) return FMM_ERR_ARG;
  DeviceGuard g(c->device);
  c->stream = static_cast<cudaStream_t>(stream);
  cudaStream_t s = c->stream;
  FMM_CUDA(cudaMemsetAsync(c->st, 0, sizeof(DevStatus), s));
  {
    Launch L(c, "keys");
    launch_keys(xyz, n, keys, c->st, s);
  }
  Readback* hb = static_cast<Readback*>(c->host_buf);
  FMM_CUDA(cudaMemcpyAsync(&hb->st, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  FMM_CUDA(cudaStreamSynchronize(s));
  if (c->timing) collect_times(c);
  return (int)hb->st.code;
}

int fmm_set_tuning(fmm_ctx* c, const fmm_tuning* t) {
  if (!c || !t || t->sort_kind > FMM_SORT_ONESWEEP) return FMM_ERR_ARG;
  c->tuning = *t;
  return FMM_OK;
}

int fmm_get_tuning(fmm_ctx* c, fmm_tuning* t) {
  if (!c || !t) return FMM_ERR_ARG;
  *t = c->tuning;
  return FMM_OK;
}

int fmm_set_timing(fmm_ctx* c, int enable) {
  if (!c) return FMM_ERR_ARG;
  c->timing = enable != 0;
  return FMM_OK;
}

int fmm_reset_timing(fmm_ctx* c) {
  if (!c) return FMM_ERR_ARG;
  c->acc.clear();
  return FMM_OK;
}

int fmm_get_timing(fmm_ctx* c, fmm_kernel_time* out, int max_entries, int* n_entries) {
  if (!c || !n_entries || (max_entries > 0 && !out)) return FMM_ERR_ARG;
  const int n = (int)c->acc.size();
  *n_entries = n;
  for (int i = 0; i < n && i < max_entries; ++i) {
    std::memset(out[i].name, 0, sizeof(out[i].name));
    std::strncpy(out[i].name, c->acc[i].name.c_str(), sizeof(out[i].name) - 1);
    out[i].launches = c->acc[i].launches;
    out[i].total_ms = c->acc[i].ms;
  }
  return FMM_OK;
}

int fmm_last_launch_count(fmm_ctx* c, uint64_t* launches) {
  if (!c || !launches) return FMM_ERR_ARG;
  *launches = c->last_launches;
  return FMM_OK;
}

const char* fmm_status_string(int status) {
  switch (status) {
    case FMM_OK: return "ok";
    case FMM_ERR_ARG: return "invalid argument";
    case FMM_ERR_DOMAIN: return "coordinate outside [0, 1] or NaN";
    case FMM_ERR_LEVEL: return "invalid level or cluster size";
    case FMM_ERR_OOM: return "device allocation failed";
    case FMM_ERR_TIMEOUT: return "a bounded device-side wait expired";
    case FMM_ERR_CUDA: return "CUDA runtime error";
    case FMM_ERR_CAPACITY: return "a list holds 2^32 or more entries";
    default: return "unknown status";
  }
}

}  // extern "C"
