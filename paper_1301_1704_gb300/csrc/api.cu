// api.cu -- the C ABI (include/fmmds.h): context, arena, and the build
// pipeline of Alg. 5 on one stream, for one (Src, Recv) pair or a batch.
//
// A build is a list of point sets (sources and receivers; a set given as both
// is built once) and a list of jobs (source set, receiver set) whose lists
// are wanted.  Every stage covers all sets in one launch:
//   radix passes (per-tile digit histograms -> one prefix sum -> scatter; the
//   first pass forms the Morton keys from the coordinates) -> finishing sort
//   inside boxes + finest boxes -> coarser boxes -> child occupancy;
// then for l = 2..L: job prefix -> list counts -> two prefix sums -> fill.
// The host synchronises once at the end, and also: in cluster-size mode after
// the sort (to learn each set's depth) and after the full-key sort of the sets
// that need one; when the list capacity bound is too large, after the boxes.
// In graph mode (fmm_set_graphs) the launches of a fixed-depth build up to its
// first host synchronisation are captured into a CUDA graph, which updates
// the executable graph kept from the previous build and is launched.
#include <algorithm>
#include <functional>
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

// Host input of a pipelined build: at most kPipeSets sets, each copied in at
// most kCopyChunks pieces of whole 2^16-point blocks.
constexpr uint32_t kPipeSets = 4;
constexpr uint32_t kCopyChunks = 8;
constexpr uint64_t kCopyGrain = 1u << 16;

uint64_t copy_chunk_points(uint64_t n) {
  const uint64_t per = (n + kCopyChunks - 1) / kCopyChunks;
  return std::max<uint64_t>(kCopyGrain, (per + kCopyGrain - 1) / kCopyGrain * kCopyGrain);
}

}  // namespace

struct fmm_ctx {
  int device = 0;
  fmm_alloc_fn alloc = nullptr;
  fmm_free_fn free_fn = nullptr;
  void* user = nullptr;
  std::vector<Chunk> chunks;
  size_t cur = 0, off = 0;
  size_t peak_request = 0;
  DevStatus* st = nullptr;        // persistent device status word
  void* up_buf = nullptr;         // pinned staging of descriptor uploads
  size_t up_bytes = 0, up_cursor = 0;
  void* rb_buf = nullptr;         // pinned read-back buffer
  size_t rb_bytes = 0;
  cudaStream_t stream = nullptr;  // stream of the call in progress
  bool timing = false;
  std::vector<PendingTime> pending;
  std::vector<cudaEvent_t> event_pool;
  std::vector<TimeAcc> acc;
  uint64_t launches = 0;
  uint64_t last_launches = 0;
  fmm_tuning tuning{FMM_SORT_BUCKET, 6};
  // graph mode
  bool graphs = false;         // capture builds (after the first) into CUDA graphs
  bool warm = false;           // a build has run eagerly on this context
  bool graph_build = false;    // the build in progress captures its stream work
  bool capturing = false;      // the stream is being captured
  uint32_t seg = 0;            // next segment of the build in progress
  std::vector<cudaGraphExec_t> gexec;  // executable graph per segment
  uint64_t graph_launches = 0, graph_instantiations = 0;
  // The legacy default stream cannot be captured: graph builds called on it
  // run on this stream, after an event that orders them behind the caller's
  // earlier work.
  cudaStream_t gstream = nullptr;
  cudaEvent_t gevent = nullptr;
  // host-input copies of a pipelined build (see do_builds_on): the copy
  // stream, the event that orders it behind the build stream, and one event
  // per copied piece (set k's piece j: k * kCopyChunks + j)
  cudaStream_t cstream = nullptr;
  cudaEvent_t cevent = nullptr;
  cudaEvent_t chunk_ev[kPipeSets * kCopyChunks] = {};
  // sets of the build in progress kept off the bucket path (a bucket of
  // theirs was too full for one block)
  std::vector<uint8_t> no_bucket;
  // Point sets (input pointer, size) whose bucket was too full for one block
  // in an earlier build on this context: they take the radix path directly,
  // saving the stopped attempt (resident time-stepped systems keep their
  // pointer and their clumps).  Cleared when the tuning changes.
  std::vector<std::pair<const float*, uint32_t>> full_sets;
};

namespace {

constexpr size_t kAlign = 256;
// Largest list capacity (bytes) reserved from the box-count bounds alone;
// above it the box counts are read back first.
constexpr uint64_t kAsyncListBytes = 16ull << 30;

size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

// ---- graph mode: segments of a build's stream work.
int cap_begin(fmm_ctx* c) {
  if (!c->graph_build || c->capturing) return FMM_OK;
  if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    c->graph_build = false;  // the rest of the build runs eagerly
    return FMM_OK;
  }
  c->capturing = true;
  return FMM_OK;
}

// Ends the segment being captured, if any: its graph updates the executable
// graph of the same segment of the previous build (or replaces it when the
// shape changed) and is launched.
int cap_end(fmm_ctx* c) {
  if (!c->capturing) return FMM_OK;
  c->capturing = false;
  cudaGraph_t g = nullptr;
  if (cudaStreamEndCapture(c->stream, &g) != cudaSuccess || g == nullptr) {
    cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    return FMM_ERR_CUDA;
  }
  size_t nodes = 0;
  int st = FMM_OK;
  if (cudaGraphGetNodes(g, nullptr, &nodes) != cudaSuccess) {
    cudaGetLastError();
    st = FMM_ERR_CUDA;
  } else if (nodes > 0) {
    const uint32_t k = c->seg++;
    if (c->gexec.size() <= k) c->gexec.resize(k + 1, nullptr);
    cudaGraphExec_t& ex = c->gexec[k];
    if (ex) {
      cudaGraphExecUpdateResultInfo info;
      if (cudaGraphExecUpdate(ex, g, &info) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphExecDestroy(ex);
        ex = nullptr;
      }
    }
    if (!ex) {
      if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
        cudaGetLastError();
        ex = nullptr;
        st = FMM_ERR_CUDA;
      } else {
        ++c->graph_instantiations;
      }
    }
    if (ex) {
      if (cudaGraphLaunch(ex, c->stream) != cudaSuccess) {
        cudaGetLastError();
        st = FMM_ERR_CUDA;
      } else {
        ++c->graph_launches;
      }
    }
  }
  cudaGraphDestroy(g);
  return st;
}

// Drops the segment being captured (a build that fails): its work never runs.
void cap_abort(fmm_ctx* c) {
  c->graph_build = false;
  if (!c->capturing) return;
  c->capturing = false;
  cudaGraph_t g = nullptr;
  cudaStreamEndCapture(c->stream, &g);
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
}

// A host synchronisation inside a build: the segment captured so far is
// launched first.  What follows the first one (read-backs, the rare re-sorts)
// runs eagerly.
int build_sync(fmm_ctx* c) {
  const int st = cap_end(c);
  c->graph_build = false;
  if (st != FMM_OK) return st;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
    cudaGetLastError();
    return FMM_ERR_CUDA;
  }
  return FMM_OK;
}

void* raw_alloc(fmm_ctx* c, size_t bytes) {
  // no allocation inside a captured segment: it is launched first, and the
  // rest of the build runs eagerly
  if (c->capturing) {
    const int st = cap_end(c);
    c->graph_build = false;
    if (st != FMM_OK) return nullptr;
  }
  void* p = nullptr;
  if (c->alloc) {
    p = c->alloc(bytes, (void*)c->stream, c->user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
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

// Pinned host buffers (grown on demand; the caller has synchronised the
// stream when a buffer in use could be replaced).
int pinned_reserve(void** buf, size_t* have, size_t bytes) {
  if (bytes <= *have) return FMM_OK;
  if (*buf) cudaFreeHost(*buf);
  *buf = nullptr;
  *have = 0;
  // whole 256-byte blocks: the upload kernel reads whole words past a size
  const size_t want = align_up(std::max<size_t>(bytes, 1 << 20));
  if (cudaMallocHost(buf, want) != cudaSuccess) {
    cudaGetLastError();
    return FMM_ERR_OOM;
  }
  *have = want;
  return FMM_OK;
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

// Small transfers of a build done by the SMs, not the copy engines: on the
// copy engines they would queue behind a large host copy of another set's
// coordinates (a pipelined host-input build) and stall the stage they feed.
// Zeroes up to two word ranges (16-byte aligned starts) in one launch.
__global__ void __launch_bounds__(256) zero_words_kernel(uint32_t* __restrict__ p0, uint64_t w0,
                                                         uint32_t* __restrict__ p1, uint64_t w1) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t t0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    uint32_t* const p = r ? p1 : p0;
    const uint64_t words = r ? w1 : w0;
    const uint64_t n16 = words / 4;
    uint4* q = reinterpret_cast<uint4*>(p);
    for (uint64_t i = t0; i < n16; i += stride) q[i] = make_uint4(0u, 0u, 0u, 0u);
    if (blockIdx.x == 0 && threadIdx.x < words - 4 * n16) p[4 * n16 + threadIdx.x] = 0u;
  }
}

__global__ void __launch_bounds__(256) copy_words_kernel(const uint32_t* __restrict__ src,
                                                          uint32_t* __restrict__ dst,
                                                          uint64_t words) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < words; i += stride)
    dst[i] = src[i];
}

uint32_t small_grid(uint64_t items) {
  const uint64_t g = (items + 255) / 256;
  return (uint32_t)(g == 0 ? 1 : (g > 152u * 4u ? 152u * 4u : g));
}

// Zeroes [p0, p0 + b0) and [p1, p1 + b1) on the build's stream (16-byte
// aligned starts, whole words).
int dev_zero2(fmm_ctx* c, void* p0, size_t b0, void* p1, size_t b1) {
  if (b0 == 0 && b1 == 0) return FMM_OK;
  if (b0 % 4 != 0 || b1 % 4 != 0 || (reinterpret_cast<uintptr_t>(p0) & 15) != 0 ||
      (reinterpret_cast<uintptr_t>(p1) & 15) != 0)
    return FMM_ERR_ARG;
  Launch L(c, "zero");
  const uint64_t w0 = b0 / 4, w1 = b1 / 4;
  zero_words_kernel<<<small_grid(std::max(w0, w1) / 4), 256, 0, c->stream>>>(
      static_cast<uint32_t*>(p0), w0, static_cast<uint32_t*>(p1), w1);
  return cudaGetLastError() == cudaSuccess ? FMM_OK : FMM_ERR_CUDA;
}

// Zeroes `bytes` (a multiple of 4) at p (16-byte aligned).
int dev_zero(fmm_ctx* c, void* p, size_t bytes) { return dev_zero2(c, p, bytes, nullptr, 0); }

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
  const int passes = passes_for(lvl);
  return std::min(kMaxLevel, std::max(lvl, 8 * passes / 3));
}

uint64_t wait_ns_of(const fmm_params& p) {
  return (uint64_t)(p.wait_ms ? p.wait_ms : 2000u) * 1000000ull;
}

// ---------------------------------------------------------------------------
// Host bookkeeping of a build.

struct SetPlan {
  const float* xyz = nullptr;
  const float* orig = nullptr;  // the caller's pointer to the points
  uint32_t n = 0;
  int Lb = 0, Ls = 0;
  bool full = false;      // sort all 63 bits (the order needs no finishing window)
  bool exact = false;     // box-key order: exactly the top 3*Ls bits, stable passes
  bool want_sorted = false;  // also the points in sorted order
  bool need_occ = false;  // used as a source
  uint32_t depth = 0;     // cluster-size mode: 1 + deepest level shared by points i, i + s
  bool bucket = false;    // ordered and boxed by the bucket path (bucket.cu)
  Seg dev{};              // the device descriptor
  uint32_t cap[kLevels] = {};
};

struct JobPlan {
  uint32_t src = 0, recv = 0;
  int L = 0;
  uint32_t s_unmet = 0;
  Job dev{};
  uint32_t cap[kLevels] = {};  // receiver capacity per list level
};

// Sizes read back at the end of a build.
struct Readback {
  DevStatus st{};
  std::vector<uint32_t> nbox;      // [nsets][kLevels] box counts
  std::vector<uint32_t> seg_long;  // [nsets]
  std::vector<uint64_t> list;      // [kLevels][njobs][4]: base E2, base E4, nnz E2, nnz E4
  std::vector<uint32_t*> idx;      // [kLevels][2]: the level's E2 / E4 entry arrays
};

// Device tables of the sort stage.
struct SortMem {
  Seg* segs = nullptr;  // descriptors of the sorted sets (sort fields and skeys / svals)
  Slot* pass_slots[8] = {};
  uint32_t pass_nslots[8] = {}, pass_tiles[8] = {};
  uint32_t* pass_hist[8] = {};
  TileRec* pass_recs[8] = {};
  size_t pass_hist_len[8] = {};
  uint64_t* pass_scan[8] = {};
  uint32_t* pass_cnt = nullptr;  // scan tickets, one per pass
  uint64_t* ka = nullptr;
  uint32_t* va = nullptr;
  uint64_t* kb = nullptr;
  uint32_t* vb = nullptr;
  int max_passes = 0;
};

// Device tables of the box and list stages.
struct BuildMem {
  Seg* segs = nullptr;
  Job* jobs = nullptr;
  ListLevel* lvls = nullptr;
  Slot* fin_slots = nullptr;
  Slot* crs_slots = nullptr;
  Slot* occ_slots = nullptr;
  Slot* sx_slots = nullptr;
  uint32_t fin_units = 0, crs_units = 0, occ_units = 0;
};

// Host image of one upload: descriptors and slot tables, 256-byte aligned.
struct Upload {
  std::vector<unsigned char> bytes;
  template <class T>
  size_t add(const T* p, size_t count) {
    const size_t at = (bytes.size() + 255) & ~(size_t)255;
    bytes.resize(at + sizeof(T) * count);
    if (count) std::memcpy(bytes.data() + at, p, sizeof(T) * count);
    return at;
  }
};

// Copies `up` to fresh device memory on the build's stream; returns the
// device address of its first byte.
char* upload(fmm_ctx* c, const Upload& up, int* err) {
  const size_t need = up.bytes.size();
  char* dev = arena_get<char>(c, need + 256, err);
  if (*err) return nullptr;
  if (c->up_cursor + need > c->up_bytes) {
    // every earlier copy from the staging buffer must have landed
    *err = build_sync(c);
    if (*err) return nullptr;
    c->up_cursor = 0;
    if (need > c->up_bytes) {
      *err = pinned_reserve(&c->up_buf, &c->up_bytes, 2 * need);
      if (*err) return nullptr;
    }
  }
  char* h = static_cast<char*>(c->up_buf) + c->up_cursor;
  std::memcpy(h, up.bytes.data(), need);
  // the device reads the pinned staging buffer directly (see copy_words_kernel)
  void* hd = nullptr;
  if (cudaHostGetDevicePointer(&hd, h, 0) != cudaSuccess) {
    cudaGetLastError();
    *err = FMM_ERR_CUDA;
    return nullptr;
  }
  {
    Launch L(c, "upload");
    const uint64_t words = (need + 3) / 4;  // the staging buffer and the arena block hold the rounding
    copy_words_kernel<<<small_grid(words), 256, 0, c->stream>>>(static_cast<const uint32_t*>(hd),
                                                                 reinterpret_cast<uint32_t*>(dev),
                                                                 words);
  }
  if (cudaGetLastError() != cudaSuccess) {
    *err = FMM_ERR_CUDA;
    return nullptr;
  }
  c->up_cursor += (need + 255) & ~(size_t)255;
  return dev;
}

struct SortTables {
  std::vector<Slot> slots[8];
  uint32_t tiles[8] = {};
  size_t hist_len[8] = {};
};

// Radix pass p covers the sets with more than p passes.  Per participating
// set: its first tile, its first histogram entry and the correction from
// scanned positions (which count only participating points) to its slots.
SortTables plan_sort(const std::vector<SetPlan*>& sets) {
  SortTables t;
  for (int p = 0; p < 8; ++p) {
    uint32_t tiles = 0, compact = 0;
    size_t hist = 0;
    for (uint32_t id = 0; id < sets.size(); ++id) {
      const SetPlan& s = *sets[id];
      if (s.n == 0 || s.dev.passes <= p) continue;
      Slot sl;
      sl.seg = id;
      sl.unit0 = tiles;
      sl.aux0 = (uint32_t)hist;
      sl.aux1 = s.dev.base - compact;
      t.slots[p].push_back(sl);
      tiles += s.dev.ntiles;
      hist += (size_t)kRadixMax * s.dev.ntiles;
      compact += s.n;
    }
    t.tiles[p] = tiles;
    t.hist_len[p] = hist;
  }
  return t;
}

// Radix passes of every set.  Pass p reads buffer (p-1)&1 (the coordinates
// for p = 0) and writes buffer p&1; a set's result stays in buffer
// (passes-1)&1 at its base.
int run_sort(fmm_ctx* c, std::vector<SetPlan*>& sets, SortMem& m, bool stall, uint64_t wait_ns) {
  cudaStream_t s = c->stream;
  int err = FMM_OK;
  bool any_full = false;  // a set sorted in full (or exactly) keeps every pass stable
  bool any_exact = false;
  for (auto* sp : sets) {
    any_full |= sp->full || sp->exact;
    any_exact |= sp->exact;
  }
  const bool onesweep = stall || (c->tuning.sort_kind == FMM_SORT_ONESWEEP && !any_exact);
  if (onesweep) {
    // One set at a time, one kernel per pass (decoupled look-back).
    for (auto* sp : sets) {
      if (sp->n == 0) continue;
      const SortPlan plan = make_sort_plan(sp->n, sp->Ls);
      const uint32_t radix = 1u << plan.bits;
      const size_t per_pass = (size_t)plan.ntiles * radix;
      const size_t zb = align_up(sizeof(uint32_t) * 8 * kRadixMax) +
                        align_up(sizeof(uint64_t) * per_pass * plan.passes) +
                        align_up(sizeof(uint32_t) * 16);
      char* z = arena_get<char>(c, zb, &err);
      if (err) return err;
      FMM_TRY(dev_zero(c, z, zb));
      uint32_t* hist = reinterpret_cast<uint32_t*>(z);
      uint64_t* sstatus =
          reinterpret_cast<uint64_t*>(z + align_up(sizeof(uint32_t) * 8 * kRadixMax));
      uint32_t* counters = reinterpret_cast<uint32_t*>(
          z + align_up(sizeof(uint32_t) * 8 * kRadixMax) +
          align_up(sizeof(uint64_t) * per_pass * plan.passes));
      {
        Launch L(c, "upfront_hist");
        launch_upfront_hist(sp->xyz, sp->n, plan, hist, c->st, s);
      }
      {
        Launch L(c, "digit_scan");
        launch_digit_scan(plan, hist, s);
      }
      const uint32_t b0 = sp->dev.base;
      for (int p = 0; p < plan.passes; ++p) {
        uint64_t* ko = ((p & 1) ? m.kb : m.ka) + b0;
        uint32_t* vo = ((p & 1) ? m.vb : m.va) + b0;
        const uint64_t* ki = ((p & 1) ? m.ka : m.kb) + b0;
        const uint32_t* vi = ((p & 1) ? m.va : m.vb) + b0;
        Launch L(c, "onesweep");
        launch_onesweep_pass(p, sp->xyz, ki, vi, ko, vo, sp->n, plan, hist + p * kRadixMax,
                             sstatus + (size_t)p * per_pass, counters + p, c->st, wait_ns,
                             (stall && p == 0 && plan.ntiles > 2) ? 1 : -1, s);
      }
    }
    return FMM_OK;
  }
  for (int p = 0; p < m.max_passes; ++p) {
    if (m.pass_tiles[p] == 0) continue;
    const uint64_t* kin = (p & 1) ? m.ka : m.kb;
    const uint32_t* vin = (p & 1) ? m.va : m.vb;
    uint64_t* kout = (p & 1) ? m.kb : m.ka;
    uint32_t* vout = (p & 1) ? m.vb : m.va;
    {
      // pass 0 stores the keys in buffer b, which pass 0's scatter then reads
      Launch L(c, "tile_hist");
      launch_tile_hist(p, m.segs, m.pass_slots[p], m.pass_nslots[p], m.pass_tiles[p],
                       m.pass_hist[p], kin, p == 0 ? m.kb : nullptr, m.pass_recs[p], c->st, s);
    }
    {
      Launch L(c, "scan");
      launch_scan_u32(m.pass_hist[p], nullptr, (uint32_t)m.pass_hist_len[p], m.pass_scan[p],
                      m.pass_cnt + p, nullptr, c->st, wait_ns, s);
    }
    // The first pass may leave equal digits in any order when a finishing
    // sort follows; sets sorted in full keep every pass stable.
    Launch L(c, "rts_scatter");
    launch_rts_scatter(p, c->tuning.sort_items, m.pass_recs[p], m.pass_tiles[p], kin, vin, kout,
                       vout, m.pass_hist[p], any_full || p > 0, true, c->st, wait_ns, s);
  }
  return FMM_OK;
}

// The Fixed-Grid pseudo-sort of `sets` (Alg. 1, 3): keys, cells and atomic
// ranks into (kb, vb), one prefix sum over all sets' histograms, the move
// into (ka, va).  The order inside a level-Ls cell is left to the finishing
// sort.
int fixed_grid_sort(fmm_ctx* c, std::vector<SetPlan*>& sets, SortMem& m, uint64_t cells,
                    uint64_t wait_ns) {
  cudaStream_t s = c->stream;
  int err = FMM_OK;
  std::vector<Slot> slots;
  uint32_t tiles = 0, compact = 0, bin0 = 0;
  for (uint32_t id = 0; id < sets.size(); ++id) {
    SetPlan& sp = *sets[id];
    Seg& d = sp.dev;
    d.passes = sp.n ? 1 : 0;
    d.skeys = m.ka + d.base;
    d.svals = m.va + d.base;
    if (sp.n == 0) continue;
    slots.push_back(Slot{id, tiles, bin0, d.base - compact});
    tiles += d.ntiles;
    compact += sp.n;
    bin0 += 1u << (3 * sp.Ls);
  }
  const size_t zb = align_up(sizeof(uint32_t) * (cells + 1)) +
                    align_up(sizeof(uint64_t) * scan_tiles((uint32_t)cells)) +
                    align_up(sizeof(uint32_t) * 4);
  char* z = arena_get<char>(c, zb, &err);
  if (err) return err;
  uint32_t* bins = reinterpret_cast<uint32_t*>(z);
  uint64_t* status = reinterpret_cast<uint64_t*>(z + align_up(sizeof(uint32_t) * (cells + 1)));
  uint32_t* counter = reinterpret_cast<uint32_t*>(
      reinterpret_cast<char*>(status) + align_up(sizeof(uint64_t) * scan_tiles((uint32_t)cells)));
  Upload up;
  std::vector<Seg> segs_host(sets.size());
  for (size_t i = 0; i < sets.size(); ++i) segs_host[i] = sets[i]->dev;
  const size_t o_segs = up.add(segs_host.data(), segs_host.size());
  const size_t o_slots = up.add(slots.data(), slots.size());
  char* dev = upload(c, up, &err);
  if (err) return err;
  m.segs = reinterpret_cast<Seg*>(dev + o_segs);
  // the depth stage walks the sort's tiles through pass 0's slot table
  m.max_passes = 1;
  m.pass_slots[0] = reinterpret_cast<Slot*>(dev + o_slots);
  m.pass_nslots[0] = (uint32_t)slots.size();
  m.pass_tiles[0] = tiles;
  FMM_TRY(dev_zero(c, z, zb));
  {
    Launch L(c, "fg_count");
    launch_fg_count(m.segs, m.pass_slots[0], m.pass_nslots[0], tiles, bins, m.kb, m.vb, c->st, s);
  }
  {
    Launch L(c, "scan");
    launch_scan_u32(bins, nullptr, (uint32_t)cells, status, counter, nullptr, c->st, wait_ns, s);
  }
  {
    Launch L(c, "fg_move");
    launch_fg_move(m.segs, m.pass_slots[0], m.pass_nslots[0], tiles, bins, m.kb, m.vb, m.ka, m.va,
                   c->st, s);
  }
  FMM_CUDA(cudaGetLastError());
  return FMM_OK;
}

// Sort stage: orders the points of `sets` by the top 3 * Ls bits of their
// keys (all 63 for full sets) into fresh concatenated arrays and points each
// set's skeys / svals there.  Only the sort fields of the descriptors change.
int sort_sets(fmm_ctx* c, std::vector<SetPlan*>& sets, bool stall, uint64_t wait_ns, SortMem* out) {
  int err = FMM_OK;
  SortMem& m = *out;
  m = SortMem{};
  uint64_t slots_total = 0;
  for (auto* sp : sets) {
    if (sp->full) sp->Ls = kMaxLevel;
    Seg& d = sp->dev;
    d.xyz = sp->xyz;
    d.n = sp->n;
    d.base = (uint32_t)slots_total;
    d.Ls = sp->Ls;
    // an exact sort of 0 bits still takes one pass: it forms the keys, and
    // its digit (bits 63..70 of a 63-bit key) is zero for every point
    d.passes = sp->n ? std::max(passes_for(sp->Ls), sp->exact ? 1 : 0) : 0;
    d.lo = 63 - 3 * sp->Ls;
    d.exact = sp->exact ? 1 : 0;
    d.tile = kSortThreads * c->tuning.sort_items;
    d.ntiles = (uint32_t)(((uint64_t)sp->n + d.tile - 1) / d.tile);
    slots_total += ((uint64_t)sp->n + 3) & ~3ull;  // set bases stay 16-byte aligned
    if (slots_total >= (1ull << 32)) return FMM_ERR_ARG;
    m.max_passes = std::max(m.max_passes, d.passes);
  }
  const size_t nslot = (size_t)slots_total + 4;
  m.ka = arena_get<uint64_t>(c, nslot, &err);
  m.va = arena_get<uint32_t>(c, nslot, &err);
  m.kb = arena_get<uint64_t>(c, nslot, &err);
  m.vb = arena_get<uint32_t>(c, nslot, &err);
  if (err) return err;

  // The Fixed-Grid pseudo-sort, when chosen and every set's dense histogram
  // (8^Ls cells) fits.
  if (c->tuning.sort_kind == FMM_SORT_FIXED_GRID && !stall) {
    bool ok = true;
    uint64_t cells = 0;
    for (auto* sp : sets) {
      ok &= !sp->full && !sp->exact && sp->Ls <= 8;
      if (sp->n) cells += 1ull << (3 * std::min(sp->Ls, 8));
    }
    if (ok && cells <= (1ull << 28)) return fixed_grid_sort(c, sets, m, cells, wait_ns);
  }

  for (auto* sp : sets) {
    Seg& d = sp->dev;
    const int last = d.passes > 0 ? (d.passes - 1) & 1 : 0;
    d.skeys = (last ? m.kb : m.ka) + d.base;
    d.svals = (last ? m.vb : m.va) + d.base;
  }
  SortTables tab = plan_sort(sets);

  // Zero-initialised words: per pass scan words and scan tickets.
  size_t zero_bytes = 0;
  size_t scan_off[8] = {};
  for (int p = 0; p < m.max_passes; ++p) {
    scan_off[p] = zero_bytes;
    zero_bytes += align_up(sizeof(uint64_t) * scan_tiles((uint32_t)tab.hist_len[p]));
  }
  const size_t cnt_off = zero_bytes;
  zero_bytes += align_up(sizeof(uint32_t) * 16);
  char* zero = arena_get<char>(c, zero_bytes, &err);
  if (err) return err;
  m.pass_cnt = reinterpret_cast<uint32_t*>(zero + cnt_off);
  for (int p = 0; p < m.max_passes; ++p) {
    m.pass_scan[p] = reinterpret_cast<uint64_t*>(zero + scan_off[p]);
    m.pass_hist[p] = arena_get<uint32_t>(c, tab.hist_len[p] + 1, &err);
    m.pass_recs[p] = arena_get<TileRec>(c, tab.tiles[p], &err);
    m.pass_hist_len[p] = tab.hist_len[p];
    m.pass_tiles[p] = tab.tiles[p];
    m.pass_nslots[p] = (uint32_t)tab.slots[p].size();
  }
  if (err) return err;

  Upload up;
  std::vector<Seg> segs_host(sets.size());
  for (size_t i = 0; i < sets.size(); ++i) segs_host[i] = sets[i]->dev;
  const size_t o_segs = up.add(segs_host.data(), segs_host.size());
  size_t o_pass[8] = {};
  for (int p = 0; p < m.max_passes; ++p)
    o_pass[p] = up.add(tab.slots[p].data(), tab.slots[p].size());
  char* dev = upload(c, up, &err);
  if (err) return err;
  m.segs = reinterpret_cast<Seg*>(dev + o_segs);
  for (int p = 0; p < m.max_passes; ++p)
    m.pass_slots[p] = reinterpret_cast<Slot*>(dev + o_pass[p]);
  FMM_TRY(dev_zero(c, zero, zero_bytes));
  return run_sort(c, sets, m, stall, wait_ns);
}

// Cluster-size depth of each sorted set (see depth_kernel), read back into
// SetPlan::depth; also returns the build's status word.
int depth_sets(fmm_ctx* c, std::vector<SetPlan*>& sets, const SortMem& m, uint32_t s_cluster,
               DevStatus* st_out) {
  cudaStream_t s = c->stream;
  int err = FMM_OK;
  const size_t nsets = sets.size();
  uint32_t* dout = arena_get<uint32_t>(c, nsets, &err);
  if (err) return err;
  FMM_TRY(dev_zero(c, dout, sizeof(uint32_t) * nsets));
  {
    Launch L(c, "depth");
    launch_depth(m.segs, m.pass_slots[0], m.pass_nslots[0], m.pass_tiles[0], s_cluster, dout,
                 c->st, s);
  }
  const size_t need = 64 + sizeof(uint32_t) * nsets;
  FMM_TRY(build_sync(c));  // the read-back buffer may be replaced
  FMM_TRY(pinned_reserve(&c->rb_buf, &c->rb_bytes, need));
  char* h = static_cast<char*>(c->rb_buf);
  FMM_CUDA(cudaMemcpyAsync(h, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  FMM_CUDA(cudaMemcpyAsync(h + 64, dout, sizeof(uint32_t) * nsets, cudaMemcpyDeviceToHost, s));
  FMM_TRY(build_sync(c));
  std::memcpy(st_out, h, sizeof(DevStatus));
  const uint32_t* hd = reinterpret_cast<const uint32_t*>(h + 64);
  for (size_t i = 0; i < nsets; ++i) sets[i]->depth = hd[i];
  return FMM_OK;
}

// ---- bucket path (bucket.cu) ----------------------------------------------

// Device tables of the bucket path of a build.
struct BucketMem {
  BkSet* bsets = nullptr;            // descriptors, one per bucket set
  std::vector<BkSet> host;           // ... and their host copies
  Slot* tile_slots = nullptr;        // count / scatter units of all bucket sets
  uint32_t tiles = 0;
  Slot* one_slots = nullptr;         // per bucket set k: Slot{k, 0} (one-set launches)
  Slot* box_slots = nullptr;         // sub-cell slots (8 a bucket slot)
  uint32_t units = 0;                // bucket slots
  uint32_t* ticket = nullptr;         // sub-cell tickets of an all-sets boxes launch
  uint32_t* set_tickets = nullptr;    // ... and of one-set launches, one per set
  int max_bl = 0, max_lb = 0;
  uint32_t count() const { return (uint32_t)host.size(); }
};

// Bucket parameters of a set of n points boxed to depth Lb; false when the
// bucket path cannot take it (too many points for level-4 buckets, more box
// levels below the sub-cells than an item keeps, or a box-key order whose
// boxes would span several sub-cells).
// Cell level of the buckets of n points: the mean sub-cell at most 3/4 of
// what one block sorts; -1 when even level-4 buckets are too few.
int bucket_level(uint64_t n) {
  const uint64_t avg = (uint64_t)kBkCap * 3 / 4;
  int bl = 0;
  while (bl < kBkMaxLevel && n > (avg << (3 * (bl + 1)))) ++bl;
  return n > (avg << (3 * (bl + 1))) ? -1 : bl;
}

bool bucket_params(uint32_t n, int Lb, bool exact, BkSet* b) {
  std::memset(b, 0, sizeof(*b));
  if (n == 0) return false;
  const int bl = bucket_level(n);
  if (bl < 0) return false;
  const int ib = n <= 1 ? 1 : 32 - __builtin_clz(n - 1);
  const int kept = 61 - ib;  // key bits an item keeps below the sub-cell
  const int below = Lb - bl - 1;
  if (below > 0 && 3 * below > kept) return false;
  if (exact && below < 0) return false;
  b->n = n;
  b->bl = bl;
  b->Lb = Lb;
  b->ib = ib;
  if (exact) {
    b->keep = ~0ull << (64 - 3 * (Lb - bl));  // levels bl+1 .. Lb
    b->D = std::min(kBkGroupBits, 3 * below);
    b->trunc = 0;
  } else {
    b->keep = ~((1ull << ib) - 1ull);
    b->D = std::min(kBkGroupBits, std::min(kept, 60 - 3 * bl));
    b->trunc = 63 - 3 * bl > 64 - ib ? 1 : 0;
  }
  const uint32_t cells = 1u << (3 * bl);
  b->tile = std::max<uint32_t>(8192u, cells * 32u);
  b->ntiles = (uint32_t)(((uint64_t)n + b->tile - 1) / b->tile);
  b->nslot = std::min<uint32_t>(cells, n);
  return true;
}

// Allocates and uploads the bucket path's tables for the sets flagged
// `bucket` (their BkSet parameters come from bucket_params).
int bucket_setup(fmm_ctx* c, std::vector<SetPlan>& sets, BucketMem* bm) {
  int err = FMM_OK;
  BucketMem& m = *bm;
  std::vector<Slot> tile_slots, one, box_slots;
  size_t zero_bytes = align_up(sizeof(uint32_t) * (1 + sets.size()));  // the tickets
  std::vector<size_t> zoff;
  for (uint32_t i = 0; i < sets.size(); ++i) {
    SetPlan& sp = sets[i];
    if (!sp.bucket) continue;
    BkSet b;
    bucket_params(sp.n, sp.Lb, sp.exact, &b);
    b.xyz = sp.xyz;
    b.seg = i;
    const uint32_t k = (uint32_t)m.host.size();
    tile_slots.push_back(Slot{k, m.tiles, 0, 0});
    one.push_back(Slot{k, 0, 0, 0});
    box_slots.push_back(Slot{k, 8 * m.units, 0, 0});
    m.tiles += b.ntiles;
    m.units += b.nslot;
    m.max_bl = std::max(m.max_bl, b.bl);
    m.max_lb = std::max(m.max_lb, b.Lb);
    zoff.push_back(zero_bytes);
    zero_bytes += align_up(sizeof(uint32_t) * 8 * (1u << (3 * b.bl))) + align_up(sizeof(uint32_t) * 4) +
                  align_up(sizeof(uint64_t) * kLevels * 8 * b.nslot);
    m.host.push_back(b);
    // the set's Seg fields the later stages read
    Seg& d = sp.dev;
    d.xyz = sp.xyz;
    d.n = sp.n;
    d.Ls = sp.Lb;
    d.exact = sp.exact ? 1 : 0;
  }
  if (m.host.empty()) return FMM_OK;
  char* zero = arena_get<char>(c, zero_bytes, &err);
  if (err) return err;
  m.ticket = reinterpret_cast<uint32_t*>(zero);
  m.set_tickets = m.ticket + 1;
  for (uint32_t k = 0; k < m.count(); ++k) {
    BkSet& b = m.host[k];
    const uint32_t subs = 8u << (3 * b.bl);
    char* z = zero + zoff[k];
    b.sct = reinterpret_cast<uint32_t*>(z);
    z += align_up(sizeof(uint32_t) * subs);
    b.info = reinterpret_cast<uint32_t*>(z);
    z += align_up(sizeof(uint32_t) * 4);
    b.status = reinterpret_cast<uint64_t*>(z);
    b.bcell = arena_get<uint32_t>(c, b.nslot, &err);
    b.boff = arena_get<uint32_t>(c, (size_t)b.nslot + 1, &err);
    b.items = arena_get<uint64_t>(c, (size_t)subs * kBkCap, &err);
    b.soff = arena_get<uint32_t>(c, 8ull * b.nslot, &err);
    b.scnt = arena_get<uint32_t>(c, 8ull * b.nslot, &err);
    if (err) return err;
  }
  Upload up;
  const size_t o_b = up.add(m.host.data(), m.host.size());
  const size_t o_t = up.add(tile_slots.data(), tile_slots.size());
  const size_t o_o = up.add(one.data(), one.size());
  const size_t o_x = up.add(box_slots.data(), box_slots.size());
  char* dev = upload(c, up, &err);
  if (err) return err;
  m.bsets = reinterpret_cast<BkSet*>(dev + o_b);
  m.tile_slots = reinterpret_cast<Slot*>(dev + o_t);
  m.one_slots = reinterpret_cast<Slot*>(dev + o_o);
  m.box_slots = reinterpret_cast<Slot*>(dev + o_x);
  return dev_zero(c, zero, zero_bytes);
}

// Scatter of tiles [t0, t1) of bucket set k (one-set slot {k, 0}), or of
// every tile of all bucket sets (k < 0).
int bucket_scatter(fmm_ctx* c, const BucketMem& m, int k, uint32_t t0, uint32_t t1) {
  const Slot* slots = k < 0 ? m.tile_slots : m.one_slots + k;
  const uint32_t nsl = k < 0 ? m.count() : 1u;
  const int max_bl = k < 0 ? m.max_bl : m.host[k].bl;
  if (t1 > t0) {
    Launch L(c, "bucket_scatter");
    launch_bucket_scatter(m.bsets, slots, nsl, t0, t1 - t0, max_bl, c->st, c->stream);
  }
  return cuda_status(cudaGetLastError());
}

// Plan of bucket set k, or of all bucket sets (k < 0), once scattered.
int bucket_plan(fmm_ctx* c, const BucketMem& m, int k) {
  Launch L(c, "bucket_plan");
  launch_bucket_plan(k < 0 ? m.bsets : m.bsets + k, k < 0 ? m.count() : 1u, c->st, c->stream);
  return cuda_status(cudaGetLastError());
}

// scatter -> plan of bucket set k, or of all bucket sets (k < 0).
int bucket_sort(fmm_ctx* c, const BucketMem& m, int k) {
  FMM_TRY(bucket_scatter(c, m, k, 0, k < 0 ? m.tiles : m.host[k].ntiles));
  return bucket_plan(c, m, k);
}

// The boxes of bucket set k alone (its own tickets), into the outputs `segs`
// of the build.
int bucket_boxes_one(fmm_ctx* c, const BucketMem& bm, const Seg* segs, uint32_t k,
                     uint64_t wait_ns) {
  Launch L(c, "bucket_boxes");
  launch_bucket_boxes(bm.bsets, segs, bm.one_slots + k, 1, bm.host[k].nslot, bm.max_lb,
                      bm.set_tickets + k, c->st, wait_ns, c->stream);
  return cuda_status(cudaGetLastError());
}

// Box and list stages of a build over sorted `sets` (SetPlan::Lb and
// JobPlan::L fixed).
// `early`, when given, runs once the outputs are allocated and cleared, in
// place of the all-sets bucket boxes and occupancy launches: the pipelined
// host-input build copies, sorts and boxes its bucket sets one at a time
// there, calling its second argument with each set once that set is boxed.
using EarlyFn = std::function<int(const Seg*, const std::function<int(uint32_t)>&)>;
int run_build(fmm_ctx* c, std::vector<SetPlan>& sets, std::vector<JobPlan>& jobs,
              const fmm_params& prm, const BucketMem& bm, Readback* rb,
              const EarlyFn* early = nullptr) {
  cudaStream_t s = c->stream;
  int err = FMM_OK;
  const uint64_t wait_ns = wait_ns_of(prm);
  const uint32_t nsets = (uint32_t)sets.size(), njobs = (uint32_t)jobs.size();
  BuildMem m;

  for (auto& sp : sets) {
    sp.dev.Lb = sp.Lb;
    sp.dev.btiles =
        std::max<uint32_t>(1, (uint32_t)(((uint64_t)sp.n + kBoxTile - 1) / kBoxTile));
    for (int l = 0; l <= sp.Lb; ++l) sp.cap[l] = level_cap(sp.n, l);
  }

  // Zero-initialised words: every set's tickets, box counts and long-box
  // flag side by side (one read-back copy for all sets), then per set its
  // look-back words.
  constexpr size_t kSetWords = 2 + kLevels + 1;
  size_t zero_bytes = align_up(sizeof(uint32_t) * kSetWords * nsets);
  std::vector<size_t> zoff(nsets);
  for (uint32_t i = 0; i < nsets; ++i) {
    zoff[i] = zero_bytes;
    zero_bytes += align_up(sizeof(uint64_t) * sets[i].dev.btiles) +
                  align_up(sizeof(uint64_t) * coarse_tiles(sets[i].cap[sets[i].Lb]) * kLevels);
  }
  char* zero = arena_get<char>(c, std::max<size_t>(zero_bytes, 1), &err);
  if (err) return err;
  uint32_t* const set_words = reinterpret_cast<uint32_t*>(zero);

  // Per-set outputs.
  for (uint32_t i = 0; i < nsets; ++i) {
    SetPlan& sp = sets[i];
    Seg& d = sp.dev;
    char* z = zero + zoff[i];
    d.bstatus = reinterpret_cast<uint64_t*>(z);
    z += align_up(sizeof(uint64_t) * d.btiles);
    d.cstatus = reinterpret_cast<uint64_t*>(z);
    z += align_up(sizeof(uint64_t) * coarse_tiles(sp.cap[sp.Lb]) * kLevels);
    d.tickets = set_words + (size_t)i * kSetWords;
    d.nbox = d.tickets + 2;
    d.seg_long = d.nbox + kLevels;
    d.perm = arena_get<uint32_t>(c, sp.n, &err);
    d.sorted = sp.want_sorted ? arena_get<float>(c, 3ull * sp.n, &err) : nullptr;
    std::memset(&d.lv, 0, sizeof(d.lv));
    for (int l = 0; l <= sp.Lb; ++l) {
      d.lv.cap[l] = sp.cap[l];
      d.lv.key[l] = arena_get<uint64_t>(c, sp.cap[l], &err);
      d.lv.off[l] = arena_get<uint32_t>(c, (size_t)sp.cap[l] + 1, &err);
      d.lv.parent[l] = arena_get<uint32_t>(c, sp.cap[l], &err);
      if (l < sp.Lb) d.lv.child[l] = arena_get<uint32_t>(c, (size_t)sp.cap[l] + 1, &err);
      if (l < sp.Lb && sp.need_occ) d.lv.occ[l] = arena_get<uint8_t>(c, sp.cap[l], &err);
    }
    if (err) return err;
  }

  // Box-stage slots (the bucket path emits its sets' boxes itself; every
  // set's finishing tiles serve the sorted points).
  std::vector<Slot> fin, crs, occ, sx;
  uint32_t sx_units = 0;
  for (uint32_t i = 0; i < nsets; ++i) {
    sx.push_back(Slot{i, sx_units, 0, 0});
    sx_units += sets[i].dev.btiles;
    if (!sets[i].bucket) {
      fin.push_back(Slot{i, m.fin_units, 0, 0});
      m.fin_units += sets[i].dev.btiles;
    }
    if (sets[i].Lb >= 1 && !sets[i].bucket) {
      crs.push_back(Slot{i, m.crs_units, 0, 0});
      m.crs_units += coarse_tiles(sets[i].cap[sets[i].Lb]);
    }
    if (sets[i].Lb >= 1 && sets[i].need_occ) {
      const uint32_t u = occupancy_units(sets[i].n);
      occ.push_back(Slot{i, m.occ_units, u, 0});
      m.occ_units += u;
    }
  }

  // ---- lists: capacities from the box-count bounds when they fit.
  int Lmax = 0;
  for (auto& jp : jobs) Lmax = std::max(Lmax, jp.L);
  uint64_t list_bound = 0;
  for (auto& jp : jobs)
    for (int l = 2; l <= jp.L; ++l) list_bound += 4ull * (2 + 27 + 189) * sets[jp.recv].cap[l];
  const bool async_lists = list_bound <= kAsyncListBytes;

  std::vector<ListLevel> lvls(kLevels);
  std::memset(lvls.data(), 0, sizeof(ListLevel) * kLevels);
  auto upload_all = [&](bool with_lists) -> int {
    Upload up;
    std::vector<Seg> segs_host(nsets);
    for (uint32_t i = 0; i < nsets; ++i) segs_host[i] = sets[i].dev;
    const size_t o_segs = up.add(segs_host.data(), nsets);
    const size_t o_fin = up.add(fin.data(), fin.size());
    const size_t o_crs = up.add(crs.data(), crs.size());
    const size_t o_occ = up.add(occ.data(), occ.size());
    const size_t o_sx = up.add(sx.data(), sx.size());
    size_t o_jobs = 0, o_lvls = 0;
    std::vector<Job> jobs_host(njobs);
    if (with_lists) {
      for (uint32_t j = 0; j < njobs; ++j) jobs_host[j] = jobs[j].dev;
      o_jobs = up.add(jobs_host.data(), njobs);
      o_lvls = up.add(lvls.data(), kLevels);
    }
    char* dev = upload(c, up, &err);
    if (err) return err;
    m.segs = reinterpret_cast<Seg*>(dev + o_segs);
    m.fin_slots = reinterpret_cast<Slot*>(dev + o_fin);
    m.crs_slots = reinterpret_cast<Slot*>(dev + o_crs);
    m.occ_slots = reinterpret_cast<Slot*>(dev + o_occ);
    m.sx_slots = reinterpret_cast<Slot*>(dev + o_sx);
    if (with_lists) {
      m.jobs = reinterpret_cast<Job*>(dev + o_jobs);
      m.lvls = reinterpret_cast<ListLevel*>(dev + o_lvls);
    }
    return FMM_OK;
  };

  // List arrays (per level, shared by the jobs) and per-job row starts.
  std::vector<size_t> work_len(kLevels, 0), zo_scan(kLevels, 0);
  char* list_zero = nullptr;
  size_t list_zero_bytes = 0;
  auto plan_lists = [&]() -> int {
    for (auto& jp : jobs) {
      std::memset(&jp.dev, 0, sizeof(jp.dev));
      jp.dev.src = jp.src;
      jp.dev.recv = jp.recv;
      jp.dev.L = jp.L;
    }
    std::vector<size_t> zo(kLevels, 0), i2(kLevels, 0), i4(kLevels, 0);
    for (int l = 2; l <= Lmax; ++l) {
      size_t run = 0;
      for (auto& jp : jobs) {
        if (jp.L < l) continue;
        jp.dev.region[l] = (uint32_t)run;
        run += (size_t)jp.cap[l] + 1;
        i2[l] += 27ull * jp.cap[l];
        i4[l] += 189ull * jp.cap[l];
      }
      if (run >= (1ull << 32)) return FMM_ERR_CAPACITY;
      work_len[l] = run;
      zo[l] = list_zero_bytes;
      // work arrays hold run + 1 entries: the scan writes its total at [run]
      list_zero_bytes += 2 * align_up(sizeof(uint32_t) * (run + 1)) +
                         2 * align_up(sizeof(uint64_t) * scan_tiles((uint32_t)run)) +
                         align_up(sizeof(uint32_t) * 2) +
                         2 * align_up(sizeof(uint64_t) * 2 * njobs) + align_up(sizeof(uint64_t) * 2);
    }
    list_zero = arena_get<char>(c, std::max<size_t>(list_zero_bytes, 1), &err);
    if (err) return err;
    for (int l = 2; l <= Lmax; ++l) {
      char* z = list_zero + zo[l];
      const size_t run = work_len[l];
      ListLevel& LV = lvls[l];
      LV.work2 = reinterpret_cast<uint32_t*>(z);
      z += align_up(sizeof(uint32_t) * (run + 1));
      LV.work4 = reinterpret_cast<uint32_t*>(z);
      z += align_up(sizeof(uint32_t) * (run + 1));
      zo_scan[l] = (size_t)(z - list_zero);
      z += 2 * align_up(sizeof(uint64_t) * scan_tiles((uint32_t)run)) + align_up(sizeof(uint32_t) * 2);
      LV.base = reinterpret_cast<uint64_t*>(z);
      z += align_up(sizeof(uint64_t) * 2 * njobs);
      LV.nnz = reinterpret_cast<uint64_t*>(z);
      z += align_up(sizeof(uint64_t) * 2 * njobs);
      LV.total = reinterpret_cast<uint64_t*>(z);
      LV.idx2 = arena_get<uint32_t>(c, i2[l], &err);
      LV.idx4 = arena_get<uint32_t>(c, i4[l], &err);
      LV.code2 = l < Lmax ? arena_get<uint8_t>(c, i2[l], &err) : nullptr;
      LV.jprefix = arena_get<uint32_t>(c, (size_t)njobs + 1, &err);
      for (auto& jp : jobs) {
        if (jp.L < l) continue;
        jp.dev.out2[l] = arena_get<uint32_t>(c, (size_t)jp.cap[l] + 1, &err);
        jp.dev.out4[l] = arena_get<uint32_t>(c, (size_t)jp.cap[l] + 1, &err);
      }
      if (err) return err;
    }
    return FMM_OK;
  };

  if (async_lists) {
    for (auto& jp : jobs)
      for (int l = 2; l <= jp.L; ++l) jp.cap[l] = sets[jp.recv].cap[l];
    FMM_TRY(plan_lists());
  }
  FMM_TRY(upload_all(async_lists));
  FMM_TRY(dev_zero2(c, zero, zero_bytes, async_lists ? list_zero : nullptr,
                    async_lists ? list_zero_bytes : 0));

  if (early) {
    // a set's child occupancy needs only that set's boxes
    const std::function<int(uint32_t)> boxed = [&](uint32_t set) -> int {
      for (const Slot& o : occ)
        if (o.seg == set) {
          Launch L(c, "occupancy");
          launch_occupancy(m.segs, m.occ_slots, (uint32_t)occ.size(), o.aux0, o.unit0, c->st, s);
        }
      return FMM_OK;
    };
    FMM_TRY((*early)(m.segs, boxed));
  }

  // ---- boxes, occupancy.
  if (bm.units && !early) {
    Launch L(c, "bucket_boxes");
    launch_bucket_boxes(bm.bsets, m.segs, bm.box_slots, bm.count(), bm.units, bm.max_lb, bm.ticket,
                        c->st, wait_ns, s);
  }
  if (m.fin_units) {
    Launch L(c, "finish_boxes");
    launch_finish_boxes(m.segs, m.fin_slots, (uint32_t)fin.size(), m.fin_units, c->st, wait_ns, s);
  }
  bool any_sorted = false;
  for (auto& sp : sets) any_sorted |= sp.want_sorted;
  if (any_sorted) {
    Launch L(c, "sorted_xyz");
    launch_sorted_xyz(m.segs, m.sx_slots, (uint32_t)sx.size(), sx_units, c->st, s);
  }
  if (m.crs_units) {
    int max_lb = 0;
    for (auto& sp : sets) max_lb = std::max(max_lb, sp.Lb);
    Launch L(c, "coarse_boxes");
    launch_coarse_boxes(m.segs, m.crs_slots, (uint32_t)crs.size(), m.crs_units, max_lb, c->st,
                        wait_ns, s);
  }
  if (m.occ_units && !early) {
    Launch L(c, "occupancy");
    launch_occupancy(m.segs, m.occ_slots, (uint32_t)occ.size(), m.occ_units, 0, c->st, s);
  }

  auto read_sets = [&](bool lists) -> int {
    const size_t list_words = lists ? 4 * (size_t)njobs * kLevels : 0;
    const size_t need = 64 + sizeof(uint32_t) * nsets * kSetWords + 16 + sizeof(uint64_t) * list_words;
    FMM_TRY(build_sync(c));  // the read-back buffer may be replaced
    FMM_TRY(pinned_reserve(&c->rb_buf, &c->rb_bytes, need));
    char* h = static_cast<char*>(c->rb_buf);
    FMM_CUDA(cudaMemcpyAsync(h, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    uint32_t* hn = reinterpret_cast<uint32_t*>(h + 64);
    FMM_CUDA(cudaMemcpyAsync(hn, set_words, sizeof(uint32_t) * nsets * kSetWords,
                             cudaMemcpyDeviceToHost, s));
    uint64_t* hl = reinterpret_cast<uint64_t*>(
        (reinterpret_cast<uintptr_t>(hn + (size_t)nsets * kSetWords) + 15) & ~(uintptr_t)15);
    if (lists)
      for (int l = 2; l <= Lmax; ++l) {
        FMM_CUDA(cudaMemcpyAsync(hl + (size_t)l * njobs * 4, lvls[l].base,
                                 sizeof(uint64_t) * 2 * njobs, cudaMemcpyDeviceToHost, s));
        FMM_CUDA(cudaMemcpyAsync(hl + (size_t)l * njobs * 4 + 2 * njobs, lvls[l].nnz,
                                 sizeof(uint64_t) * 2 * njobs, cudaMemcpyDeviceToHost, s));
      }
    FMM_TRY(build_sync(c));
    std::memcpy(&rb->st, h, sizeof(DevStatus));
    rb->nbox.assign((size_t)nsets * kLevels, 0);
    rb->seg_long.assign(nsets, 0);
    for (uint32_t i = 0; i < nsets; ++i) {
      std::memcpy(&rb->nbox[(size_t)i * kLevels], hn + (size_t)i * kSetWords + 2,
                  sizeof(uint32_t) * kLevels);
      rb->seg_long[i] = hn[(size_t)i * kSetWords + 2 + kLevels];
    }
    if (lists) {
      rb->list.assign((size_t)kLevels * njobs * 4, 0);
      for (int l = 2; l <= Lmax; ++l)
        for (uint32_t j = 0; j < njobs; ++j) {
          if (jobs[j].L < l) continue;
          const uint64_t* b = hl + (size_t)l * njobs * 4;
          uint64_t* o = &rb->list[((size_t)l * njobs + j) * 4];
          o[0] = b[2 * j];
          o[1] = b[2 * j + 1];
          o[2] = b[2 * njobs + 2 * j];
          o[3] = b[2 * njobs + 2 * j + 1];
        }
    }
    return FMM_OK;
  };

  if (!async_lists) {
    FMM_TRY(read_sets(false));
    if (rb->st.code) return (int)rb->st.code;
    for (auto& jp : jobs)
      for (int l = 2; l <= jp.L; ++l) jp.cap[l] = rb->nbox[(size_t)jp.recv * kLevels + l];
    FMM_TRY(plan_lists());
    FMM_TRY(upload_all(true));
    FMM_TRY(dev_zero(c, list_zero, list_zero_bytes));
  }

  // ---- lists, levels 2..Lmax.
  for (int l = 2; l <= Lmax; ++l) {
    char* zs = list_zero + zo_scan[l];
    const size_t sw = align_up(sizeof(uint64_t) * scan_tiles((uint32_t)work_len[l]));
    uint64_t* st2 = reinterpret_cast<uint64_t*>(zs);
    uint64_t* st4 = reinterpret_cast<uint64_t*>(zs + sw);
    uint32_t* cnt = reinterpret_cast<uint32_t*>(zs + 2 * sw);
    if (!job_prefix_in_count(njobs)) {
      Launch Lk(c, "job_prefix");
      launch_job_prefix(m.segs, m.jobs, njobs, l, m.lvls, c->st, s);
    }
    {
      Launch Lk(c, "list_count");
      launch_list_count(m.segs, m.jobs, njobs, l, m.lvls, c->st, s);
    }
    {
      Launch Lk(c, "scan");
      launch_scan_u32_pair(lvls[l].work2, st2, lvls[l].total, lvls[l].work4, st4,
                           lvls[l].total + 1, (uint32_t)work_len[l], cnt, c->st, wait_ns, s);
    }
    {
      Launch Lk(c, "list_fill");
      launch_list_fill(m.segs, m.jobs, njobs, l, m.lvls, lvls[l].code2 != nullptr, c->st, s);
    }
  }
  FMM_CUDA(cudaGetLastError());

  // ---- sizes and status.
  FMM_TRY(read_sets(true));
  if (rb->st.code) return (int)rb->st.code;
  rb->idx.assign((size_t)kLevels * 2, nullptr);
  for (int l = 2; l <= Lmax; ++l) {
    rb->idx[2 * l] = lvls[l].idx2;
    rb->idx[2 * l + 1] = lvls[l].idx4;
  }
  return FMM_OK;
}

// Redoes the order of the flagged sets with the full 63-bit sort (a box was
// longer than the finishing window).  Only their permutations change.
int full_sort_perms(fmm_ctx* c, std::vector<SetPlan>& sets, const std::vector<uint32_t>& ids,
                    const fmm_params& prm) {
  if (ids.empty()) return FMM_OK;
  std::vector<SetPlan> sub(ids.size());
  std::vector<SetPlan*> ps;
  for (size_t k = 0; k < ids.size(); ++k) {
    sub[k].xyz = sets[ids[k]].xyz;
    sub[k].n = sets[ids[k]].n;
    sub[k].full = true;
    ps.push_back(&sub[k]);
  }
  SortMem sm;
  FMM_TRY(sort_sets(c, ps, false, wait_ns_of(prm), &sm));
  // Every pass of a full sort is stable: the values of the last pass are the
  // order by (key, index).
  cudaStream_t s = c->stream;
  for (size_t k = 0; k < ids.size(); ++k) {
    const Seg& d = sets[ids[k]].dev;
    FMM_CUDA(cudaMemcpyAsync(d.perm, sub[k].dev.svals, sizeof(uint32_t) * sub[k].n,
                             cudaMemcpyDeviceToDevice, s));
    if (d.sorted) {
      Launch L(c, "sorted_xyz");
      launch_sorted_xyz_one(d.perm, d.xyz, sub[k].n, d.sorted, s);
    }
  }
  FMM_TRY(build_sync(c));
  return FMM_OK;
}

void fill_tree(const std::vector<SetPlan>& sets, const JobPlan& J, const Readback& rb,
               uint32_t ji, uint32_t njobs, fmm_tree* out) {
  std::memset(out, 0, sizeof(*out));
  const int L = J.L;
  const SetPlan& S = sets[J.src];
  const SetPlan& R = sets[J.recv];
  out->L = L;
  out->s_unmet = J.s_unmet;
  out->n_src = S.n;
  out->n_recv = R.n;
  const SetPlan* side[2] = {&S, &R};
  const uint32_t idx[2] = {J.src, J.recv};
  for (int k = 0; k < 2; ++k) {
    const Seg& d = side[k]->dev;
    const uint32_t* nb = &rb.nbox[(size_t)idx[k] * kLevels];
    uint32_t* onb = k ? out->nbox_recv : out->nbox_src;
    const uint64_t** okey = k ? out->key_recv : out->key_src;
    const uint32_t** ooff = k ? out->off_recv : out->off_src;
    const uint32_t** opar = k ? out->parent_recv : out->parent_src;
    const uint32_t** ochi = k ? out->child_recv : out->child_src;
    (k ? out->perm_recv : out->perm_src) = d.perm;
    (k ? out->sorted_recv : out->sorted_src) = d.sorted;
    for (int l = 0; l <= L; ++l) {
      onb[l] = nb[l];
      okey[l] = d.lv.key[l];
      ooff[l] = d.lv.off[l];
      opar[l] = l >= 1 ? d.lv.parent[l] : nullptr;
      ochi[l] = l < L ? d.lv.child[l] : nullptr;
    }
  }
  for (int l = 2; l <= L; ++l) {
    const uint64_t* o = &rb.list[((size_t)l * njobs + ji) * 4];
    out->nnz_e2[l] = o[2];
    out->nnz_e4[l] = o[3];
    out->e2_off[l] = J.dev.out2[l];
    out->e4_off[l] = J.dev.out4[l];
    out->e2_idx[l] = rb.idx[2 * l] + o[0];
    out->e4_idx[l] = rb.idx[2 * l + 1] + o[1];
  }
}

struct PairIn {
  const float* src;
  uint32_t N;
  const float* recv;
  uint32_t M;
  int L;  // own depth, or -1: the call's params
};

int query_workspace(uint32_t N, uint32_t M, const fmm_params& p, uint64_t* bytes);
void workspace_parts(uint32_t N, uint32_t M, const fmm_params& p, uint64_t* bytes,
                     uint64_t* list_bytes);

// The build of one or many (Src, Recv) pairs, outputs in outs[].
int do_builds_on(fmm_ctx* c, const PairIn* pairs, uint32_t npairs, const fmm_params& prm,
                 fmm_tree* outs) {
  cudaStream_t s = c->stream;
  int err = FMM_OK;
  const bool stall = (prm.flags & FMM_FLAG_TEST_STALL) != 0;
  const bool host_in = (prm.flags & FMM_FLAG_HOST_INPUT) != 0;
  const bool box_order = (prm.flags & FMM_FLAG_BOX_ORDER) != 0;
  const uint64_t wait_ns = wait_ns_of(prm);

  // The sort stage concatenates every distinct set (each rounded up to 4
  // points) and indexes the result with 32-bit offsets.
  uint64_t points = 0;
  for (uint32_t k = 0; k < npairs; ++k) {
    const bool aliased = pairs[k].src == pairs[k].recv && pairs[k].N == pairs[k].M;
    points += ((uint64_t)pairs[k].N + 3) & ~3ull;
    if (!aliased) points += ((uint64_t)pairs[k].M + 3) & ~3ull;
  }
  if (points >= (1ull << 32)) return FMM_ERR_ARG;

  // Arena reserved up front: the lists' capacity bound only while it is
  // reserved as such (above kAsyncListBytes the lists are sized from the box
  // counts and the arena grows by what they need).
  uint64_t expect = 0, list_expect = 0;
  for (uint32_t k = 0; k < npairs; ++k) {
    uint64_t b = 0, lb = 0;
    fmm_params pk = prm;
    if (pairs[k].L >= 0) pk.L = pairs[k].L;
    workspace_parts(pairs[k].N, pairs[k].M, pk, &b, &lb);
    expect += b;
    list_expect += lb;
  }
  expect += std::min<uint64_t>(list_expect, kAsyncListBytes);
  FMM_TRY(arena_reset(c, c->peak_request > expect ? c->peak_request : expect));
  c->up_cursor = 0;
  c->seg = 0;
  FMM_TRY(cap_begin(c));
  FMM_TRY(dev_zero(c, c->st, sizeof(DevStatus)));

  // Sets (the same array given as a pair's sources and receivers is one set)
  // and jobs.
  std::vector<SetPlan> sets;
  std::vector<JobPlan> jobs(npairs);
  auto add_set = [&](const float* p, uint32_t n) {
    SetPlan sp;
    sp.xyz = p;
    sp.orig = p;
    sp.n = n;
    sets.push_back(sp);
    return (uint32_t)sets.size() - 1;
  };
  for (uint32_t k = 0; k < npairs; ++k) {
    const bool aliased = pairs[k].src == pairs[k].recv && pairs[k].N == pairs[k].M;
    jobs[k].src = add_set(pairs[k].src, pairs[k].N);
    jobs[k].recv = aliased ? jobs[k].src : add_set(pairs[k].recv, pairs[k].M);
    sets[jobs[k].src].need_occ = true;
  }
  // Host input: the coordinates are copied to the arena.  A fixed-depth
  // build of a few sets copies them one set at a time on a copy stream and
  // sorts each set as soon as it has landed, so that the next set's copy runs
  // under that sort; otherwise every copy precedes the build.
  bool all_fixed = true;
  for (uint32_t k = 0; k < npairs; ++k) all_fixed &= (pairs[k].L >= 0 ? pairs[k].L : prm.L) >= 0;
  const bool pipelined =
      host_in && !stall && all_fixed && sets.size() >= 2 && sets.size() <= kPipeSets;
  std::vector<const float*> host_xyz(sets.size(), nullptr);
  if (pipelined && !c->cstream) {
    bool ok = cudaStreamCreateWithFlags(&c->cstream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&c->cevent, cudaEventDisableTiming) == cudaSuccess;
    for (auto& e : c->chunk_ev)
      ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      return FMM_ERR_CUDA;
    }
  }
  // Pinned (page-locked or registered) inputs are copied in full at once, in
  // pieces whose events the sort waits on; a pageable copy holds the host
  // until it is done, so each piece of one is issued just before the work
  // that needs it.
  bool upfront = pipelined;
  for (size_t i = 0; upfront && i < sets.size(); ++i) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, sets[i].xyz) != cudaSuccess) {
      cudaGetLastError();
      upfront = false;
    } else {
      upfront = a.type == cudaMemoryTypeHost;
    }
  }
  const auto chunks_of = [&](uint64_t n) -> uint32_t {
    return (uint32_t)((n + copy_chunk_points(n) - 1) / copy_chunk_points(n));
  };
  const auto chunk_end = [&](uint64_t n, uint32_t j) -> uint64_t {
    return std::min<uint64_t>(n, copy_chunk_points(n) * (j + 1));
  };
  const auto copy_chunk = [&](uint32_t k, uint32_t j) -> int {
    const uint64_t n = sets[k].n, p0 = j ? chunk_end(n, j - 1) : 0, p1 = chunk_end(n, j);
    FMM_CUDA(cudaMemcpyAsync(const_cast<float*>(sets[k].xyz) + 3 * p0, host_xyz[k] + 3 * p0,
                             sizeof(float) * 3 * (p1 - p0), cudaMemcpyHostToDevice,
                             c->cstream));
    FMM_CUDA(cudaEventRecord(c->chunk_ev[k * kCopyChunks + j], c->cstream));
    return FMM_OK;
  };
  // Piece j of set k is on the device for the build stream's next launches.
  const auto land = [&](uint32_t k, uint32_t j) -> int {
    if (!upfront) FMM_TRY(copy_chunk(k, j));
    FMM_CUDA(cudaStreamWaitEvent(s, c->chunk_ev[k * kCopyChunks + j], 0));
    return FMM_OK;
  };
  if (host_in) {
    for (size_t i = 0; i < sets.size(); ++i) {
      SetPlan& sp = sets[i];
      float* d = arena_get<float>(c, (size_t)sp.n * 3, &err);
      if (err) return err;
      host_xyz[i] = sp.xyz;
      if (sp.n && !pipelined)
        FMM_CUDA(cudaMemcpyAsync(d, sp.xyz, sizeof(float) * 3 * sp.n, cudaMemcpyHostToDevice, s));
      sp.xyz = d;
    }
    if (pipelined) {  // the copies start after the build stream's earlier work
      FMM_CUDA(cudaEventRecord(c->cevent, s));
      FMM_CUDA(cudaStreamWaitEvent(c->cstream, c->cevent, 0));
      if (upfront)
        for (uint32_t k = 0; k < sets.size(); ++k)
          for (uint32_t j = 0; j < chunks_of(sets[k].n); ++j) FMM_TRY(copy_chunk(k, j));
    }
  }
  std::vector<SetPlan*> all;
  for (auto& sp : sets) {
    sp.want_sorted = (prm.flags & FMM_FLAG_SORTED_XYZ) != 0;
    all.push_back(&sp);
  }

  // Jobs of fixed depth (their own, or the call's L) and cluster-size jobs
  // (L = -1).  Sort depth: at least every fixed depth the set serves, and deep
  // enough that a box averages a few points, which keeps the finishing sort
  // short.
  std::vector<int> fixed_lb(sets.size(), -1);
  std::vector<uint8_t> in_smode(sets.size(), 0);
  bool any_smode = false;
  for (uint32_t k = 0; k < npairs; ++k) {
    JobPlan& jp = jobs[k];
    jp.L = pairs[k].L >= 0 ? pairs[k].L : prm.L;
    if (jp.L >= 0) {
      fixed_lb[jp.src] = std::max(fixed_lb[jp.src], jp.L);
      fixed_lb[jp.recv] = std::max(fixed_lb[jp.recv], jp.L);
    } else {
      in_smode[jp.src] = in_smode[jp.recv] = 1;
      any_smode = true;
    }
  }
  for (uint32_t i = 0; i < sets.size(); ++i) {
    SetPlan& sp = sets[i];
    const int lb = std::max(fixed_lb[i], in_smode[i] ? 2 : 0);
    if (box_order && !in_smode[i]) {
      sp.Ls = lb;  // exactly the box bits
      sp.exact = true;
    } else {
      sp.Ls = std::max(sort_level(sp.n, lb), lb);
    }
    // The bucket path (sort kind FMM_SORT_BUCKET) takes fixed-depth sets it
    // can hold; the others, and every set after a bucket overflowed, take
    // the radix passes.
    BkSet probe;
    const bool was_full =
        std::find(c->full_sets.begin(), c->full_sets.end(), std::make_pair(sp.orig, sp.n)) !=
        c->full_sets.end();
    sp.bucket = c->tuning.sort_kind == FMM_SORT_BUCKET && !stall && !in_smode[i] && !was_full &&
                !(i < c->no_bucket.size() && c->no_bucket[i]) &&
                bucket_params(sp.n, lb, sp.exact, &probe);
    if (sp.bucket) {
      sp.Lb = lb;
      sp.Ls = lb;
    }
  }
  std::vector<SetPlan*> lsd;
  for (auto& sp : sets)
    if (!sp.bucket) lsd.push_back(&sp);
  BucketMem bm;
  FMM_TRY(bucket_setup(c, sets, &bm));
  // A pipelined build whose sets all take the bucket path also boxes each
  // set as soon as it is sorted (inside run_build, once the outputs exist),
  // so that the sources' box stage runs under the receivers' copy too.
  const bool early_boxes = pipelined && bm.count() == sets.size();
  {
    SortMem sm;
    if (early_boxes) {
      // (sorted and boxed in run_build)
    } else if (pipelined) {
      // set i's copy, then its sort behind its pieces' events; a pageable
      // set i+1 is copied after sort i's launches
      uint32_t kb = 0;
      for (uint32_t i = 0; i < sets.size(); ++i) {
        SetPlan& sp = sets[i];
        for (uint32_t j = 0; j < chunks_of(sp.n); ++j) FMM_TRY(land(i, j));
        if (sp.bucket) {
          FMM_TRY(bucket_sort(c, bm, (int)kb++));
        } else {
          std::vector<SetPlan*> one{&sp};
          SortMem si;
          FMM_TRY(sort_sets(c, one, false, wait_ns, &si));
        }
      }
    } else {
      if (bm.count()) FMM_TRY(bucket_sort(c, bm, -1));
      if (!lsd.empty()) FMM_TRY(sort_sets(c, lsd, stall, wait_ns, &sm));
    }
    if (any_smode) {
      // Cluster-size mode (Sec. 2.1): the deepest level at which s + 1 sorted
      // points still share a box, per set; sets whose boxes are still too
      // full at the sort depth are sorted on all key bits and measured again.
      std::vector<SetPlan*> ss;
      for (uint32_t i = 0; i < sets.size(); ++i)
        if (in_smode[i]) ss.push_back(&sets[i]);
      // (measured over all sorted sets: the sort's descriptors are in that order)
      DevStatus st{};
      FMM_TRY(depth_sets(c, lsd, sm, prm.s, &st));
      if (st.code) return (int)st.code;
      // A set still too full at its sort depth is sorted three levels deeper
      // (one or two more radix passes) and measured again; only if that is not
      // deep enough either, on all key bits.
      for (int round = 0; round < 2; ++round) {
        std::vector<SetPlan*> deep;
        for (auto* sp : ss)
          if (!sp->full && sp->depth > (uint32_t)sp->Ls) {
            if (round == 0 && sp->Ls + 3 < kMaxLevel)
              sp->Ls += 3;
            else
              sp->full = true;
            deep.push_back(sp);
          }
        if (deep.empty()) break;
        SortMem sd;
        FMM_TRY(sort_sets(c, deep, false, wait_ns, &sd));
        FMM_TRY(depth_sets(c, deep, sd, prm.s, &st));
        if (st.code) return (int)st.code;
      }
      // A job's depth: the smallest L >= 2 at which neither set has a box of
      // more than s points; level 21 with s_unmet when no level has.
      for (auto& jp : jobs) {
        if (jp.L >= 0) continue;
        const uint32_t d = std::max(sets[jp.src].depth, sets[jp.recv].depth);
        if (d > (uint32_t)kMaxLevel) {
          jp.L = kMaxLevel;
          jp.s_unmet = 1;
        } else {
          jp.L = std::max(2, (int)d);
        }
      }
    }
  }
  for (auto& sp : sets) sp.Lb = 0;
  for (auto& jp : jobs) {
    sets[jp.src].Lb = std::max(sets[jp.src].Lb, jp.L);
    sets[jp.recv].Lb = std::max(sets[jp.recv].Lb, jp.L);
  }
  // A set paired with a deeper one needs its order to that depth; in the
  // box-key order every set is sorted on exactly its box bits.
  std::vector<SetPlan*> resort;
  for (auto& sp : sets) {
    if (sp.bucket) continue;  // ordered to its box depth already
    if (box_order) {
      if (!sp.exact || sp.Ls != sp.Lb) {
        sp.Ls = sp.Lb;
        sp.exact = true;
        sp.full = false;
        resort.push_back(&sp);
      }
    } else if (sp.Lb > sp.Ls) {
      sp.Ls = std::max(sort_level(sp.n, sp.Lb), sp.Lb);
      resort.push_back(&sp);
    }
  }
  if (!resort.empty()) {
    SortMem sr;
    FMM_TRY(sort_sets(c, resort, false, wait_ns, &sr));
  }

  Readback rb;
  // A scatter tile needs only its own points, so the tiles of each copied
  // piece are scattered as soon as it has landed, and only the last piece's
  // scatter, the plan and the boxes follow the set's copy.
  const EarlyFn copy_sort_box = [&](const Seg* segs,
                                    const std::function<int(uint32_t)>& boxed) -> int {
    for (uint32_t k = 0; k < sets.size(); ++k) {
      const uint64_t n = sets[k].n;
      const BkSet& b = bm.host[k];
      const uint32_t nch = chunks_of(n);
      uint32_t t_done = 0;
      for (uint32_t j = 0; j < nch; ++j) {
        FMM_TRY(land(k, j));
        // tiles wholly inside the pieces landed so far
        const uint32_t t_hi = j + 1 == nch ? b.ntiles : (uint32_t)(chunk_end(n, j) / b.tile);
        if (t_hi > t_done) {
          FMM_TRY(bucket_scatter(c, bm, (int)k, t_done, t_hi));
          t_done = t_hi;
        }
      }
      FMM_TRY(bucket_plan(c, bm, (int)k));
      FMM_TRY(bucket_boxes_one(c, bm, segs, k, wait_ns));
      FMM_TRY(boxed(k));
    }
    return FMM_OK;
  };
  const int rs = run_build(c, sets, jobs, prm, bm, &rb, early_boxes ? &copy_sort_box : nullptr);
  // A bucket too full for one block (status kStatusBucketFull; the sets
  // carry bit 2): the build stopped there; build again with those sets on
  // the radix path.
  if (rs == (int)kStatusBucketFull) {
    if (c->no_bucket.size() < sets.size()) c->no_bucket.resize(sets.size(), 0);
    bool any = false;
    for (uint32_t i = 0; i < sets.size(); ++i)
      if (rb.seg_long[i] & 2u) {
        c->no_bucket[i] = 1;
        any = true;
        const auto key = std::make_pair(sets[i].orig, sets[i].n);
        if (std::find(c->full_sets.begin(), c->full_sets.end(), key) == c->full_sets.end()) {
          if (c->full_sets.size() >= 1024) c->full_sets.erase(c->full_sets.begin());
          c->full_sets.push_back(key);
        }
      }
    if (!any) return FMM_ERR_CUDA;  // (cannot happen: the status comes with the bit)
    cap_abort(c);
    c->graph_build = false;
    return do_builds_on(c, pairs, npairs, prm, outs);
  }
  FMM_TRY(rs);
  // Boxes that outran the finishing window, or runs of points tied in an
  // item's key bits too long for one thread (bit 1): redo those orders in
  // full.
  std::vector<uint32_t> longs;
  for (uint32_t i = 0; i < sets.size(); ++i)
    if (rb.seg_long[i]) longs.push_back(i);
  FMM_TRY(full_sort_perms(c, sets, longs, prm));

  for (uint32_t j = 0; j < npairs; ++j) fill_tree(sets, jobs[j], rb, j, npairs, &outs[j]);
  FMM_TRY(cap_end(c));  // nothing is left to capture after the last read-back
  c->graph_build = false;
  c->warm = true;
  size_t used = 0;
  for (size_t i = 0; i < c->chunks.size(); ++i) used += c->chunks[i].bytes;
  c->peak_request = std::max(c->peak_request, used);
  return FMM_OK;
}

// A build, in graph mode when the context asks for it: a fixed-depth build
// (no cluster-size job), from the second build of a context on (the first
// one grows the arena and the staging buffers), and not with timing, the
// stall test or copies from the caller's host memory.  Its launches up to the
// first host synchronisation -- the whole build but the read-back, unless
// the list capacity is too large to reserve up front -- are one graph.
int do_builds(fmm_ctx* c, const PairIn* pairs, uint32_t npairs, const fmm_params& prm,
              fmm_tree* outs) {
  const uint32_t f = prm.flags;
  bool fixed = true;
  for (uint32_t k = 0; k < npairs; ++k) fixed &= (pairs[k].L >= 0 ? pairs[k].L : prm.L) >= 0;
  c->graph_build = c->graphs && c->warm && fixed && !c->timing &&
                   !(f & FMM_FLAG_TEST_STALL) && !(f & FMM_FLAG_HOST_INPUT);
  const cudaStream_t caller = c->stream;
  bool moved = false;
  if (c->graph_build && (caller == nullptr || caller == cudaStreamLegacy)) {
    if (!c->gstream &&
        (cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking) != cudaSuccess ||
         cudaEventCreateWithFlags(&c->gevent, cudaEventDisableTiming) != cudaSuccess)) {
      cudaGetLastError();
      if (c->gstream) cudaStreamDestroy(c->gstream);
      c->gstream = nullptr;
      c->graph_build = false;
    }
    if (c->graph_build) {
      FMM_CUDA(cudaEventRecord(c->gevent, caller));
      FMM_CUDA(cudaStreamWaitEvent(c->gstream, c->gevent, 0));
      c->stream = c->gstream;
      moved = true;
    }
  }
  c->no_bucket.clear();
  const int st = do_builds_on(c, pairs, npairs, prm, outs);
  c->no_bucket.clear();
  cap_abort(c);  // a build that failed inside a captured segment
  if (moved) {
    if (st != FMM_OK) cudaStreamSynchronize(c->stream);
    c->stream = caller;
  }
  return st;
}

// Arena bytes of a build of N sources and M receivers: everything but the
// lists (*bytes), and the lists' capacity bound (*list_bytes).
void workspace_parts(uint32_t N, uint32_t M, const fmm_params& p, uint64_t* bytes,
                     uint64_t* list_bytes) {
  const int L = p.L >= 0 ? p.L : std::max(sort_level(std::max(N, M), 2), 2);
  uint64_t total = 64 << 10;
  const uint32_t ns[2] = {N, M};
  for (int k = 0; k < 2; ++k) {
    const uint64_t n = ns[k];
    if (p.flags & FMM_FLAG_HOST_INPUT) total += align_up(12 * n);
    total += 2 * align_up(12 * n + 48) + align_up(4 * n) + (16 << 10);
    // the bucket path's sub-cells each have room for what one block sorts:
    // its items can outgrow the radix passes' arrays
    const int bl = n ? bucket_level(n) : -1;
    if (bl >= 0) {
      const uint64_t subs = 8ull << (3 * bl);
      const uint64_t bk = subs * (8ull * kBkCap + 8ull * kLevels + 64) + (64 << 10);
      const uint64_t rx = 2 * align_up(12 * n + 48);
      if (bk > rx) total += bk - rx;
    }
    const uint64_t tiles = n / (kSortThreads * 4) + 1;  // the smallest tile
    total += tiles * kRadixMax * 4 * 3 + (n / kBoxTile + 1) * 8 * (1 + kLevels);
    total += tiles * sizeof(TileRec) * 8 + 8 * 256;  // tile records, 8 passes
    for (int l = 0; l <= L; ++l) total += align_up(21ull * level_cap(ns[k], l) + 8) + 1024;
  }
  uint64_t lists = 0;
  for (int l = 2; l <= L; ++l) lists += align_up(4ull * (4 + 27 + 189) * level_cap(M, l) + 64) + 4096;
  *bytes = total;
  *list_bytes = lists;
}

int query_workspace(uint32_t N, uint32_t M, const fmm_params& p, uint64_t* bytes) {
  uint64_t rest = 0, lists = 0;
  workspace_parts(N, M, p, &rest, &lists);
  *bytes = rest + lists;
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

int check_params(const fmm_params& p) {
  if (p.flags & ~(FMM_FLAG_HOST_INPUT | FMM_FLAG_TEST_STALL | FMM_FLAG_BOX_ORDER |
                  FMM_FLAG_SORTED_XYZ))
    return FMM_ERR_ARG;
  if (p.L > kMaxLevel || p.L < -1 || (p.L == -1 && p.s == 0)) return FMM_ERR_LEVEL;
  return FMM_OK;
}

int finish_call(fmm_ctx* c, int st, uint64_t l0) {
  cap_abort(c);  // a build that failed inside a captured segment
  if (st != FMM_OK) {
    cudaStreamSynchronize(c->stream);
    cudaGetLastError();
  }
  if (c->timing) collect_times(c);
  c->last_launches = c->launches - l0;
  return st;
}

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
      pinned_reserve(&c->up_buf, &c->up_bytes, 1 << 20) != FMM_OK ||
      pinned_reserve(&c->rb_buf, &c->rb_bytes, 1 << 16) != FMM_OK) {
    cudaGetLastError();
    if (c->st) cudaFree(c->st);
    if (c->up_buf) cudaFreeHost(c->up_buf);
    delete c;
    return FMM_ERR_CUDA;
  }
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
  for (auto ex : c->gexec)
    if (ex) cudaGraphExecDestroy(ex);
  if (c->gevent) cudaEventDestroy(c->gevent);
  if (c->gstream) cudaStreamDestroy(c->gstream);
  if (c->cevent) cudaEventDestroy(c->cevent);
  for (auto e : c->chunk_ev)
    if (e) cudaEventDestroy(e);
  if (c->cstream) cudaStreamDestroy(c->cstream);
  cudaFree(c->st);
  if (c->up_buf) cudaFreeHost(c->up_buf);
  if (c->rb_buf) cudaFreeHost(c->rb_buf);
  delete c;
  return FMM_OK;
}

int fmm_query_workspace(uint32_t N, uint32_t M, fmm_params p, uint64_t* bytes) {
  if (!bytes) return FMM_ERR_ARG;
  if (p.L > kMaxLevel || p.L < -1 || (p.L == -1 && p.s == 0)) return FMM_ERR_LEVEL;
  return query_workspace(N, M, p, bytes);
}

int fmm_query_sizes(uint32_t N, uint32_t M, fmm_params p, fmm_sizes* out) {
  if (!out) return FMM_ERR_ARG;
  FMM_TRY(check_params(p));
  std::memset(out, 0, sizeof(*out));
  FMM_TRY(query_workspace(N, M, p, &out->workspace_bytes));
  const int L = p.L >= 0 ? p.L : kMaxLevel;
  for (int l = 0; l <= L; ++l) {
    out->max_nbox_src[l] = level_cap(N, l);
    out->max_nbox_recv[l] = level_cap(M, l);
    if (l >= 2) {
      out->max_nnz_e2[l] = 27ull * level_cap(M, l);
      out->max_nnz_e4[l] = 189ull * level_cap(M, l);
    }
  }
  return FMM_OK;
}

int fmm_build(fmm_ctx* c, const float* src_xyz, uint32_t N, const float* recv_xyz, uint32_t M,
              fmm_params params, fmm_tree* out, void* stream) {
  if (!c || !out) return FMM_ERR_ARG;
  if ((N > 0 && !src_xyz) || (M > 0 && !recv_xyz)) return FMM_ERR_ARG;
  FMM_TRY(check_params(params));
  DeviceGuard g(c->device);
  c->stream = static_cast<cudaStream_t>(stream);
  const uint64_t l0 = c->launches;
  const PairIn pin{src_xyz, N, recv_xyz, M, -1};
  return finish_call(c, do_builds(c, &pin, 1, params, out), l0);
}

int fmm_build_batched(fmm_ctx* c, const fmm_set* sets, uint32_t nsets, fmm_params params,
                      fmm_tree* outs, void* stream) {
  if (!c || (nsets > 0 && (!sets || !outs))) return FMM_ERR_ARG;
  FMM_TRY(check_params(params));
  if (params.flags & FMM_FLAG_TEST_STALL) return FMM_ERR_ARG;
  for (uint32_t k = 0; k < nsets; ++k) {
    if ((sets[k].N > 0 && !sets[k].src) || (sets[k].M > 0 && !sets[k].recv)) return FMM_ERR_ARG;
    if (sets[k].L < FMM_SET_PARAMS_L || sets[k].L > kMaxLevel) return FMM_ERR_LEVEL;
  }
  if (nsets == 0) return FMM_OK;
  DeviceGuard g(c->device);
  c->stream = static_cast<cudaStream_t>(stream);
  const uint64_t l0 = c->launches;
  std::vector<PairIn> pins(nsets);
  for (uint32_t k = 0; k < nsets; ++k)
    pins[k] = {sets[k].src, sets[k].N, sets[k].recv, sets[k].M, sets[k].L};
  return finish_call(c, do_builds(c, pins.data(), nsets, params, outs), l0);
}

int fmm_e2_source_offsets(fmm_ctx* c, const fmm_tree* t, int level, uint32_t* off,
                          uint64_t* total, void* stream) {
  if (!c || !t || !off || !total) return FMM_ERR_ARG;
  if (level < 2 || level > t->L) return FMM_ERR_LEVEL;
  DeviceGuard g(c->device);
  c->stream = static_cast<cudaStream_t>(stream);
  cudaStream_t s = c->stream;
  const uint32_t nrecv = t->nbox_recv[level];
  int err = FMM_OK;
  const size_t zb = align_up(sizeof(uint64_t) * scan_tiles(nrecv)) + align_up(sizeof(uint64_t)) +
                    align_up(sizeof(uint32_t));
  char* z = arena_get<char>(c, zb, &err);
  if (err) return err;
  uint64_t* status = reinterpret_cast<uint64_t*>(z);
  uint64_t* total64 = reinterpret_cast<uint64_t*>(z + align_up(sizeof(uint64_t) * scan_tiles(nrecv)));
  uint32_t* counter = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(total64) +
                                                  align_up(sizeof(uint64_t)));
  FMM_CUDA(cudaMemsetAsync(z, 0, zb, s));
  FMM_CUDA(cudaMemsetAsync(c->st, 0, sizeof(DevStatus), s));
  {
    Launch L(c, "e2_count");
    launch_e2_count(t->e2_off[level], t->e2_idx[level], t->off_src[level], nrecv, off, c->st, s);
  }
  {
    Launch L(c, "scan");
    launch_scan_u32(off, nullptr, nrecv, status, counter, total64, c->st, wait_ns_of(fmm_params{}),
                    s);
  }
  char* h = static_cast<char*>(c->rb_buf);
  FMM_CUDA(cudaMemcpyAsync(h, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  FMM_CUDA(cudaMemcpyAsync(h + 64, total64, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  FMM_CUDA(cudaStreamSynchronize(s));
  if (c->timing) collect_times(c);
  DevStatus st;
  std::memcpy(&st, h, sizeof(st));
  std::memcpy(total, h + 64, sizeof(uint64_t));
  if (st.code) return (int)st.code;
  return (*total >> 32) ? FMM_ERR_CAPACITY : FMM_OK;
}

int fmm_box_types(fmm_ctx* c, const fmm_tree* t, int lpar, const uint32_t* owner, uint32_t node,
                  uint8_t* const* types, void* stream) {
  if (!c || !t || !types) return FMM_ERR_ARG;
  if (lpar < 2 || lpar > t->L) return FMM_ERR_LEVEL;
  if (t->perm_src != t->perm_recv || (t->nbox_src[lpar] > 0 && !owner)) return FMM_ERR_ARG;
  for (int l = 2; l <= t->L; ++l)
    if (!types[l] && t->nbox_src[l] > 0) return FMM_ERR_ARG;
  DeviceGuard g(c->device);
  c->stream = static_cast<cudaStream_t>(stream);
  cudaStream_t s = c->stream;
  int err = FMM_OK;
  const int L = t->L, lcrit = std::max(lpar - 1, 2);
  std::vector<uint8_t*> on(kLevels, nullptr);
  for (int l = lpar; l <= L; ++l) {
    on[l] = arena_get<uint8_t>(c, t->nbox_src[l], &err);
    if (err) return err;
    Launch Lk(c, "box_types");
    launch_on_node(l == lpar ? owner : nullptr, t->parent_src[l], on[l - 1], t->nbox_src[l], node,
                   on[l], s);
  }
  uint8_t* sides = nullptr;
  if (lcrit < lpar) {
    sides = arena_get<uint8_t>(c, t->nbox_src[lcrit], &err);
    if (err) return err;
    Launch Lk(c, "box_types");
    launch_child_sides(t->child_src[lcrit], on[lpar], t->nbox_src[lcrit], sides, s);
  }
  for (int l = 2; l <= L; ++l) {
    Launch Lk(c, "box_types");
    if (l < lcrit) {
      launch_box_type(nullptr, nullptr, nullptr, nullptr, t->nbox_src[l], 0, types[l], s);
    } else if (l == lcrit && lcrit < lpar) {
      launch_box_type(t->e4_off[l], t->e4_idx[l], sides, nullptr, t->nbox_src[l], 1, types[l], s);
    } else if (l == lcrit) {  // lcrit = lpar = 2: a box's own ownership decides
      // its descendants at lpar are itself: bit 0 on J, bit 1 off J
      uint8_t* sd = arena_get<uint8_t>(c, t->nbox_src[l], &err);
      if (err) return err;
      launch_child_sides(nullptr, on[l], t->nbox_src[l], sd, s);
      launch_box_type(t->e4_off[l], t->e4_idx[l], sd, nullptr, t->nbox_src[l], 1, types[l], s);
    } else {
      launch_box_type(t->e4_off[l], t->e4_idx[l], nullptr, on[l], t->nbox_src[l], 2, types[l], s);
    }
  }
  FMM_CUDA(cudaGetLastError());
  return FMM_OK;
}

int fmm_gather_e2_sources(fmm_ctx* c, const fmm_tree* t, int level, const float* sorted_src,
                          const uint32_t* off, float* out, void* stream) {
  if (!c || !t || !off || (!sorted_src && t->n_src > 0)) return FMM_ERR_ARG;
  if (level < 2 || level > t->L) return FMM_ERR_LEVEL;
  DeviceGuard g(c->device);
  c->stream = static_cast<cudaStream_t>(stream);
  {
    Launch L(c, "e2_gather");
    launch_e2_gather(t->e2_off[level], t->e2_idx[level], t->off_src[level], sorted_src, off,
                     t->nbox_recv[level], out, c->stream);
  }
  FMM_CUDA(cudaGetLastError());
  return FMM_OK;
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
  DevStatus* h = static_cast<DevStatus*>(c->rb_buf);
  FMM_CUDA(cudaMemcpyAsync(h, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  FMM_CUDA(cudaStreamSynchronize(s));
  if (c->timing) collect_times(c);
  return (int)h->code;
}

int fmm_set_tuning(fmm_ctx* c, const fmm_tuning* t) {
  if (!c || !t || t->sort_kind > FMM_SORT_BUCKET) return FMM_ERR_ARG;
  const uint32_t items = t->sort_items ? t->sort_items : 6;
  if (items != 4 && items != 6 && items != 7 && items != 8) return FMM_ERR_ARG;
  c->tuning = *t;
  c->full_sets.clear();
  c->tuning.sort_items = items;
  return FMM_OK;
}

int fmm_autotune(fmm_ctx* c, const fmm_set* sets, uint32_t nsets, fmm_params params,
                 uint32_t trials, fmm_tuning* best, double* best_ms, void* stream) {
  if (!c || !best || nsets == 0 || !sets || trials == 0) return FMM_ERR_ARG;
  FMM_TRY(check_params(params));
  if (params.flags & FMM_FLAG_TEST_STALL) return FMM_ERR_ARG;
  DeviceGuard g(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<fmm_tree> outs(nsets);
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    cudaGetLastError();
    return FMM_ERR_CUDA;
  }
  const fmm_tuning saved = c->tuning;
  fmm_tuning win = saved;
  double win_ms = 1e300;
  int st = FMM_OK;
  const uint32_t kinds[4] = {FMM_SORT_BUCKET, FMM_SORT_RTS, FMM_SORT_ONESWEEP, FMM_SORT_FIXED_GRID};
  const uint32_t items[4] = {4, 6, 7, 8};
  // a cluster-size build orders its points by the radix passes whatever the
  // kind (the bucket path needs the depth before it sorts)
  bool fixed = params.L >= 0;
  for (uint32_t k = 0; k < nsets; ++k) fixed &= params.L >= 0 || sets[k].L >= 0;
  for (uint32_t kind : kinds) {
    for (uint32_t it : items) {
      if (kind == FMM_SORT_ONESWEEP && it != 6) continue;  // onesweep keeps its own tile
      if (kind == FMM_SORT_BUCKET && (it != 6 || !fixed)) continue;  // no radix tile
      c->tuning = fmm_tuning{kind, it};
      c->full_sets.clear();
      std::vector<double> ms;
      for (uint32_t r = 0; r <= trials && st == FMM_OK; ++r) {
        cudaEventRecord(a, s);
        st = fmm_build_batched(c, sets, nsets, params, outs.data(), stream);
        cudaEventRecord(b, s);
        if (st == FMM_OK && cudaEventSynchronize(b) != cudaSuccess) st = FMM_ERR_CUDA;
        float t = 0.f;
        if (st == FMM_OK && r > 0) {  // the first build of a choice warms up
          cudaEventElapsedTime(&t, a, b);
          ms.push_back(t);
        }
      }
      if (st != FMM_OK) break;
      std::sort(ms.begin(), ms.end());
      const double med = ms[ms.size() / 2];
      if (med < win_ms) {
        win_ms = med;
        win = c->tuning;
      }
    }
    if (st != FMM_OK) break;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  c->tuning = st == FMM_OK ? win : saved;
  c->full_sets.clear();
  if (st != FMM_OK) return st;
  *best = win;
  if (best_ms) *best_ms = win_ms;
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

int fmm_set_graphs(fmm_ctx* c, int enable) {
  if (!c) return FMM_ERR_ARG;
  DeviceGuard g(c->device);
  c->graphs = enable != 0;
  if (!c->graphs) {
    for (auto& ex : c->gexec)
      if (ex) cudaGraphExecDestroy(ex);
    c->gexec.clear();
  }
  return FMM_OK;
}

int fmm_graph_stats(fmm_ctx* c, uint64_t* launches, uint64_t* instantiations) {
  if (!c || !launches || !instantiations) return FMM_ERR_ARG;
  *launches = c->graph_launches;
  *instantiations = c->graph_instantiations;
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
    case FMM_PENDING: return "the request is not done yet";
    default: return "unknown status";
  }
}

}  // extern "C"
