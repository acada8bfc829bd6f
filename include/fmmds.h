/* fmmds.h -- C ABI of the GB300 FMM data-structure builder.
 *
 * The library builds the data structures of the fast multipole method for a
 * set of sources and a set of receivers in the unit cube, following
 * Q. Hu, N. A. Gumerov, R. Duraiswami, "Parallel algorithms for constructing
 * data structures for fast multipole methods" (arXiv:1301.1704):
 *
 *   Alg. 5 (Build-fmm-data-structures) takes Src[] and Recv[] and returns the
 *   sorted-point permutation (RecvPermutationIdx), the bookmarks
 *   (Src/RecvBookmark), the Morton keys of the non-empty boxes
 *   (SrcNonEmptyBoxIndex) and the E2 neighbour lists in CSR form
 *   (NeighborBookmark / NeighborList, Alg. 4).  This library returns those at
 *   every level 0..L, plus parent ranks, child ranges and the E4 (M2L)
 *   interaction lists (Sec. 1.4 item 4) at every level 2..L.
 *
 * Conventions (the paper leaves these open; Sec. 1.4, Sec. 2):
 *   - coordinates are float32, row-major [n][3] (x, y, z), each in [0, 1];
 *     a coordinate < 0, > 1 or NaN is an error (FMM_ERR_DOMAIN); 1.0 belongs
 *     to the last cell;
 *   - cell of a coordinate at level 21: min(floor(x * 2^21), 2^21 - 1);
 *     Morton key: bit k of the x / y / z cell goes to bit 3k / 3k+1 / 3k+2
 *     (63-bit key); the level-l key of a point is key >> 3(21 - l);
 *   - points are ordered by (Morton key, original index): unique and
 *     deterministic (the paper's pseudo-sort allows any order inside a box);
 *   - all box ranks, bookmarks and list entries are uint32 ("all the
 *     integers ... are stored as unsigned int", Sec. 2);
 *   - E2(r) holds the non-empty source boxes at max-norm distance <= 1 from
 *     receiver box r, r itself included (at most 27); E4(r) the non-empty
 *     source boxes whose parent touches r's parent but that are not in E2(r)
 *     (at most 6^3 - 3^3 = 189).  Both ascending by source-box rank; no
 *     periodic images.
 *
 * Errors: every call returns an fmm_status.  Device-side checks (domain,
 * capacity, bounded waits) report through a status word read at the end of
 * the call; no kernel traps.  After an error the outputs are undefined but
 * the context stays usable.
 *
 * Threading: a context may be used by one host thread at a time.
 */
#ifndef FMMDS_H
#define FMMDS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FMM_MAX_LEVEL 21
#define FMM_LEVELS 22 /* levels 0..21 */

typedef enum fmm_status {
  FMM_OK = 0,
  FMM_ERR_ARG = 1,      /* null pointer, bad size, bad flag */
  FMM_ERR_DOMAIN = 2,   /* a coordinate < 0, > 1 or NaN */
  FMM_ERR_LEVEL = 3,    /* L > 21, L < -1, or L == -1 with s == 0 */
  FMM_ERR_OOM = 4,      /* the allocator returned NULL */
  FMM_ERR_TIMEOUT = 5,  /* a bounded device-side wait expired */
  FMM_ERR_CUDA = 6,     /* a CUDA runtime call failed */
  FMM_ERR_CAPACITY = 7  /* a list of one level holds 2^32 or more entries */
} fmm_status;

/* Device allocator used for the context's arena (for instance PyTorch's
 * caching allocator).  `stream` is the cudaStream_t of the call in
 * progress.  Returning NULL makes the call fail with FMM_ERR_OOM. */
typedef void* (*fmm_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*fmm_free_fn)(void* ptr, size_t bytes, void* stream, void* user);

/* Build flags. */
#define FMM_FLAG_HOST_INPUT 0x1u   /* src/recv point to host memory (pinned or
                                      pageable); the call copies them to the
                                      device on its stream */
#define FMM_FLAG_TEST_STALL 0x80000000u /* test only: one tile of the first
                                      sort pass never publishes, so the
                                      bounded wait must end with
                                      FMM_ERR_TIMEOUT */

/* Problem statement of Alg. 5 / Sec. 2.1: a maximal level L (0..21), or a
 * cluster size s (L = -1, s >= 1): the smallest L >= 2 at which no finest
 * box of either set holds more than s points (capped at 21, see
 * fmm_tree.s_unmet). */
typedef struct fmm_params {
  int L;
  uint32_t s;
  uint32_t flags;
  uint32_t wait_ms; /* limit of each device-side wait; 0 = 2000 ms */
} fmm_params;

/* Result of a build.  All array pointers are DEVICE pointers into the
 * context's arena; they stay valid until the next build on the same context
 * or fmm_destroy.  Entries for levels outside 0..L (lists: 2..L) are NULL/0.
 *
 *   perm_*[j]           original index of the j-th sorted point  [n]
 *   key_*[l][b]         level-l Morton key of non-empty box b, ascending
 *   off_*[l][b]         first sorted point of box b; off[l][nbox] = n
 *   parent_*[l][b]      rank of b's parent at level l-1 (l >= 1)
 *   child_*[l][b]       first child rank at level l+1; child[l][nbox] =
 *                       nbox[l+1] (l < L)
 *   e2_off[l][r], e4_off[l][r]  CSR row starts for receiver box r, length
 *                       nbox_recv[l] + 1
 *   e2_idx[l], e4_idx[l] source-box ranks (level l), nnz_e2[l] / nnz_e4[l]
 */
typedef struct fmm_tree {
  int L;
  uint32_t s_unmet; /* 1 if cluster-size mode could not meet s at L = 21 */
  uint32_t n_src, n_recv;
  const uint32_t* perm_src;
  const uint32_t* perm_recv;
  uint32_t nbox_src[FMM_LEVELS];
  uint32_t nbox_recv[FMM_LEVELS];
  const uint64_t* key_src[FMM_LEVELS];
  const uint64_t* key_recv[FMM_LEVELS];
  const uint32_t* off_src[FMM_LEVELS];
  const uint32_t* off_recv[FMM_LEVELS];
  const uint32_t* parent_src[FMM_LEVELS];
  const uint32_t* parent_recv[FMM_LEVELS];
  const uint32_t* child_src[FMM_LEVELS];
  const uint32_t* child_recv[FMM_LEVELS];
  uint64_t nnz_e2[FMM_LEVELS];
  uint64_t nnz_e4[FMM_LEVELS];
  const uint32_t* e2_off[FMM_LEVELS];
  const uint32_t* e2_idx[FMM_LEVELS];
  const uint32_t* e4_off[FMM_LEVELS];
  const uint32_t* e4_idx[FMM_LEVELS];
} fmm_tree;

typedef struct fmm_ctx fmm_ctx;

/* Creates a context bound to CUDA device `device`.  alloc/free may both be
 * NULL (the library then uses cudaMalloc/cudaFree); `user` is passed back to
 * them.  The context owns its arena; fmm_destroy releases it. */
int fmm_create(fmm_ctx** ctx, int device, fmm_alloc_fn alloc, fmm_free_fn free_fn, void* user);

/* Releases the context and every array of its last build. */
int fmm_destroy(fmm_ctx* ctx);

/* Alg. 5 for one (Src, Recv) pair.  src_xyz [N][3] and recv_xyz [M][3] are
 * device pointers (host pointers with FMM_FLAG_HOST_INPUT), caller-owned and
 * read-only; they must stay valid until the call returns.  src_xyz may equal
 * recv_xyz (N == M).  N or M may be 0.  Work runs on `stream`
 * (cudaStream_t, NULL = legacy default stream); the call returns after the
 * stream has finished the build, with *out filled. */
int fmm_build(fmm_ctx* ctx, const float* src_xyz, uint32_t N, const float* recv_xyz,
              uint32_t M, fmm_params params, fmm_tree* out, void* stream);

/* One (Src, Recv) pair of a batched build. */
typedef struct fmm_set {
  const float* src;
  uint32_t N;
  const float* recv;
  uint32_t M;
} fmm_set;

/* Alg. 5 for nsets independent pairs at once: every stage (radix passes,
 * boxes, lists) covers all sets in one kernel launch, so many small builds
 * cost about as many launches as one.  Same conventions as fmm_build per
 * set; params apply to every set (in cluster-size mode each set gets its own
 * L).  outs[k] receives set k's tree, with values local to the set (point
 * indices, box ranks and list entries as if the set were built alone); all
 * arrays live in the context's arena until its next build.  Inputs must not
 * overlap partially: a set's src and recv may be the same array (N == M).
 * FMM_FLAG_TEST_STALL is not accepted here. */
int fmm_build_batched(fmm_ctx* ctx, const fmm_set* sets, uint32_t nsets, fmm_params params,
                      fmm_tree* outs, void* stream);

/* Sec. 2 "BoxIndex" + Sec. 1.4 interleave: the 63-bit Morton keys of n
 * points in input order.  xyz [n][3] and keys [n] are device pointers owned
 * by the caller.  Asynchronous on `stream`; returns FMM_ERR_DOMAIN (after a
 * stream synchronisation) if a coordinate is outside [0, 1]. */
int fmm_morton_keys(fmm_ctx* ctx, const float* xyz, uint32_t n, uint64_t* keys, void* stream);

/* Upper bound of the arena bytes one build of this size needs. */
int fmm_query_workspace(uint32_t N, uint32_t M, fmm_params params, uint64_t* bytes);

/* Tuning of a context (the autotuner's knobs).  sort_kind selects how each
 * radix pass finds its output positions:
 *   FMM_SORT_RTS       per-tile digit histograms, one prefix sum, then a
 *                      scatter with no waiting between tiles (default);
 *   FMM_SORT_ONESWEEP  one kernel per pass, each tile finds its offsets by
 *                      decoupled look-back over the earlier tiles.
 * Both give the same result.  FMM_ERR_ARG for an unknown kind. */
#define FMM_SORT_RTS 0u
#define FMM_SORT_ONESWEEP 1u
typedef struct fmm_tuning {
  uint32_t sort_kind;
} fmm_tuning;

int fmm_set_tuning(fmm_ctx* ctx, const fmm_tuning* tuning);
int fmm_get_tuning(fmm_ctx* ctx, fmm_tuning* tuning);

/* Per-kernel timing with CUDA events on the build's stream (off by
 * default).  Each entry: kernel name, launches and summed milliseconds since
 * the last reset. */
typedef struct fmm_kernel_time {
  char name[32];
  uint64_t launches;
  double total_ms;
} fmm_kernel_time;

int fmm_set_timing(fmm_ctx* ctx, int enable);
int fmm_get_timing(fmm_ctx* ctx, fmm_kernel_time* out, int max_entries, int* n_entries);
int fmm_reset_timing(fmm_ctx* ctx);

/* Number of kernels launched by the last fmm_build on this context. */
int fmm_last_launch_count(fmm_ctx* ctx, uint64_t* launches);

/* Exclusive prefix sum of n uint32 counts that allocates nothing.  The paper
 * has no counterpart: this serves callers that must not allocate device
 * memory while they run -- for example a time-stepping loop that reserved
 * all device memory up front, or code running where the CUDA allocator may
 * not be called -- and that want the CSR row starts of their own per-box list
 * counts (the role of NeighborBookmark).
 *
 *   counts  [n] device, read-only; offsets [n + 1] device: offsets[i] = sum
 *   of counts[0..i), offsets[n] = the total (low 32 bits); total: optional
 *   device uint64 receiving the full total (all ones if a bounded device-side
 *   wait gave up).  Both buffers are the caller's.
 *
 * n must not exceed FMM_NOALLOC_SCAN_MAX (FMM_ERR_ARG otherwise).  The only
 * scratch is a fixed static device array (about 128 KiB) that every GPU
 * loading this library keeps until the process exits; the call allocates
 * nothing (no cudaMalloc, no allocator callback) and clears the part of the
 * scratch it uses on `stream` before its kernel runs.  The first call on a
 * device looks up that array's device address (once per device, with the
 * device current): make that first call before any stream capture.  All calls
 * share the one array, which keeps the last call's contents, so calls that
 * overlap on the GPU (on different streams, or from several threads) race
 * and give wrong results: order them.  Asynchronous on `stream`; returns
 * after launching.  Runs on the current device. */
#define FMM_NOALLOC_SCAN_MAX (1u << 26)
int fmm_exclusive_scan_noalloc(const uint32_t* counts, uint32_t n, uint32_t* offsets,
                               uint64_t* total, void* stream);

/* Static description of a status code. */
const char* fmm_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* FMMDS_H */
