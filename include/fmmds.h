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
  FMM_ERR_CAPACITY = 7, /* a list of one level holds 2^32 or more entries */
  FMM_PENDING = 8       /* fmm_server_poll only: the request is not done yet */
} fmm_status;

/* Device allocator used for the context's arena (for instance PyTorch's
 * caching allocator).  `stream` is the cudaStream_t of the call in
 * progress.  Returning NULL makes the call fail with FMM_ERR_OOM. */
typedef void* (*fmm_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*fmm_free_fn)(void* ptr, size_t bytes, void* stream, void* user);

/* Build flags. */
#define FMM_FLAG_HOST_INPUT 0x1u   /* src/recv point to host memory (pinned or
                                      pageable); the call copies them to the
                                      device after its stream's earlier work
                                      (on an internal copy stream that its
                                      stream then waits on, so that the copies
                                      overlap the sort of the sets already
                                      landed) */
#define FMM_FLAG_BOX_ORDER 0x2u    /* order the points by (level-L box key,
                                      original index) instead of (full key,
                                      original index): the order inside a box
                                      that Sec. 2.1 leaves free, taken as input
                                      order; only the permutations differ */
#define FMM_FLAG_SORTED_XYZ 0x4u   /* also return the points in sorted
                                      order (fmm_tree.sorted_src/_recv) */
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
  /* SortedSrc / SortedRecv (Sec. 2.1): float32 [n][3], point j = input
   * point perm[j]; only with FMM_FLAG_SORTED_XYZ, else NULL. */
  const float* sorted_src;
  const float* sorted_recv;
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
 * recv_xyz (N == M).  N or M may be 0.  N and M, each rounded up to a
 * multiple of 4 (once when the sets are the same array), must add up to less
 * than 2^32; FMM_ERR_ARG otherwise (in a batched build: over all distinct
 * sets).  Work runs on `stream` (cudaStream_t, NULL = legacy default
 * stream); the call returns after the stream has finished the build, with
 * *out filled. */
int fmm_build(fmm_ctx* ctx, const float* src_xyz, uint32_t N, const float* recv_xyz,
              uint32_t M, fmm_params params, fmm_tree* out, void* stream);

/* One (Src, Recv) pair of a batched build.  L: the pair's own tree depth
 * (0..21), or FMM_SET_PARAMS_L (-1) to take it from the call's params (fixed
 * L, or cluster-size mode). */
#define FMM_SET_PARAMS_L (-1)
typedef struct fmm_set {
  const float* src;
  uint32_t N;
  const float* recv;
  uint32_t M;
  int32_t L;
} fmm_set;

/* Alg. 5 for nsets independent pairs at once: every stage (radix passes,
 * boxes, lists) covers all sets in one kernel launch, so many small builds
 * cost about as many launches as one.  Same conventions as fmm_build per
 * set; params apply to every set whose L is FMM_SET_PARAMS_L (in cluster-size
 * mode each such set gets its own L); a set's own L (0..21) overrides them,
 * and FMM_ERR_LEVEL is returned for an L above 21 or below -1.
 * outs[k] receives set k's tree, with values local to the set (point
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

/* Sizes of one build known before it runs (Alg. 5's outputs, Sec. 2.1):
 * the arena bound of fmm_query_workspace, and per level l the largest
 * possible number of non-empty boxes, min(n, 8^l), of each set and the
 * largest possible list sizes, 27 and 189 entries per receiver box (E2
 * includes the box itself; E4 = the 6^3 children of the parent's neighbours
 * less the 3^3 of E2).  With L = -1 (cluster-size mode) the level bounds are
 * given for every level 0..21.  The tree a build returns holds the exact
 * sizes (nbox_*, nnz_*). */
typedef struct fmm_sizes {
  uint64_t workspace_bytes;
  uint32_t max_nbox_src[FMM_LEVELS], max_nbox_recv[FMM_LEVELS];
  uint64_t max_nnz_e2[FMM_LEVELS], max_nnz_e4[FMM_LEVELS];  /* 0 at levels 0, 1 */
} fmm_sizes;
int fmm_query_sizes(uint32_t N, uint32_t M, fmm_params params, fmm_sizes* out);

/* Tuning of a context (the autotuner's knobs).  sort_kind selects how the
 * points are ordered before the finishing sort inside the boxes:
 *   FMM_SORT_RTS         LSD radix passes, each: per-tile digit histograms,
 *                        one prefix sum, then a scatter with no waiting
 *                        between tiles;
 *   FMM_SORT_ONESWEEP    radix passes, one kernel each, every tile finding
 *                        its offsets by decoupled look-back over the earlier
 *                        tiles;
 *   FMM_SORT_FIXED_GRID  the paper's Fixed-Grid pseudo-sort (Alg. 1): a dense
 *                        histogram of the level-Ls cells with atomic ranks,
 *                        its prefix sum as the bookmarks (Alg. 3), one move;
 *                        used when every set's sort depth is at most 8 and
 *                        the histograms hold at most 2^28 cells (else RTS).
 *   FMM_SORT_BUCKET      fixed-depth builds: the points are bucketed on
 *                        coarse cells in one pass (a histogram in shared
 *                        memory and atomic ranks per tile, the cells' prefix
 *                        sum as their bookmarks -- Alg. 1 and 3 at a coarse
 *                        level), then each cell is sorted in shared memory
 *                        by one block, which also emits the boxes of every
 *                        level; a set whose cell is too full for one block (the
 *                        build is then redone, and the context builds the
 *                        same input pointer and size by the radix passes
 *                        directly until its tuning changes), and every
 *                        cluster-size build, takes FMM_SORT_RTS (default).
 * All give the same result.  FMM_ERR_ARG for an unknown kind. */
#define FMM_SORT_RTS 0u
#define FMM_SORT_ONESWEEP 1u
#define FMM_SORT_FIXED_GRID 2u
#define FMM_SORT_BUCKET 3u
/* sort_items: points per thread of a radix tile (4, 6, 7 or 8; 0 = 6): the
 * tile of the histogram, scatter, depth and Fixed-Grid kernels is 512 x
 * sort_items points.  Larger tiles mean fewer tiles and histogram entries but
 * one resident scatter block per SM instead of two at 8. */
typedef struct fmm_tuning {
  uint32_t sort_kind;
  uint32_t sort_items;
} fmm_tuning;

int fmm_set_tuning(fmm_ctx* ctx, const fmm_tuning* tuning);
int fmm_get_tuning(fmm_ctx* ctx, fmm_tuning* tuning);

/* The autotuner: times `trials` builds of `sets` (as fmm_build_batched with
 * `params`) for every sort kind x items-per-thread choice, after one warm-up
 * build each, with CUDA events on `stream`; keeps the one with the smallest
 * median time as the context's tuning and returns it in *best (and its median
 * in *best_ms).  Every candidate gives the same result, so the choice only
 * changes speed.  The context's arena holds the last candidate's outputs
 * afterwards. */
int fmm_autotune(fmm_ctx* ctx, const fmm_set* sets, uint32_t nsets, fmm_params params,
                 uint32_t trials, fmm_tuning* best, double* best_ms, void* stream);

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

/* Graph mode (off by default).  When enabled, every fixed-depth build on the
 * context after its first one records its launches up to its first host
 * synchronisation -- sort, boxes and lists, everything but the read-back of
 * the sizes (and the rare full-key re-sort of over-full boxes) -- into one
 * CUDA graph, which updates the executable graph kept from the previous build
 * (or replaces it when the work changed shape) and is launched.  A
 * time-stepping caller that rebuilds from the same device buffers with new
 * coordinates launches one graph per build instead of some thirty kernels.
 * Results are identical to the eager build.  Cluster-size builds, builds with
 * per-kernel timing, with FMM_FLAG_HOST_INPUT or with the stall test flag run
 * eagerly.  Disabling frees the kept graph.  Errors: FMM_ERR_ARG for a null
 * context. */
int fmm_set_graphs(fmm_ctx* ctx, int enable);

/* Graphs launched and graphs instantiated (not just updated) by builds on
 * this context since its creation. */
int fmm_graph_stats(fmm_ctx* ctx, uint64_t* launches, uint64_t* instantiations);

/* Exclusive prefix sum of n uint32 counts that allocates nothing.  The paper
 * has no counterpart: this serves callers that must not allocate device
 * memory while they run -- for example a time-stepping loop that reserved
 * all device memory up front, or code running where the CUDA allocator may
 * not be called -- and that want the CSR row starts of their own per-box list
 * counts (the role of NeighborBookmark).
 *
 *   counts  [n] device, read-only; offsets [n + 1] device: offsets[i] = sum
 *   of counts[0..i) (low 32 bits), offsets[n] = the total (low 32 bits);
 *   total: optional device uint64 receiving the full 64-bit total.  All
 *   buffers are the caller's.  If a bounded device-side wait gives up (the
 *   GPU did not schedule an earlier tile within 2 s), offsets[n] is set to
 *   0xffffffff and *total to all ones; only `total` tells that apart from a
 *   real total, so a caller that must detect the failure passes `total`
 *   (a real total is below 2^58).
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

/* ---- Alg. 2: the source points of every receiver box's E2 neighbourhood.
 *
 * For receiver box i of `level` (2..tree->L), Alg. 2 walks its neighbour
 * list NeighborList[NeighborBookmark[i] .. NeighborBookmark[i+1]) and, for
 * each source box v there, copies SortedSrc[SrcBookmark[v] ..
 * SrcBookmark[v+1]).  These two calls do it for all receiver boxes at once:
 *
 * fmm_e2_source_offsets writes off[i] = number of E2 source points of the
 * receiver boxes before i (off [nbox_recv[level] + 1], device, caller-owned;
 * off[nbox] = the total) and *total (host) = the total; FMM_ERR_CAPACITY if
 * it reaches 2^32.  Synchronises `stream`.
 *
 * fmm_gather_e2_sources then copies the points: box i's occupy out[off[i] ..
 * off[i+1]) ([total][3] float32, device, caller-owned), neighbour boxes in
 * list order, points inside a box in sorted order.  sorted_src is the tree's
 * sorted_src (FMM_FLAG_SORTED_XYZ) or any [N][3] float32 array in that
 * order.  Asynchronous on `stream`.
 *
 * The tree must come from the last build of `ctx` (its arrays live in the
 * arena); FMM_ERR_LEVEL for a level outside 2..L. */
int fmm_e2_source_offsets(fmm_ctx* ctx, const fmm_tree* tree, int level, uint32_t* off,
                          uint64_t* total, void* stream);
int fmm_gather_e2_sources(fmm_ctx* ctx, const fmm_tree* tree, int level, const float* sorted_src,
                          const uint32_t* off, float* out, void* stream);

/* ---- Alg. 6: source-box types for node J of a partition (Sec. 3.2).
 *
 * The space is split among nodes at level lpar (2..L): owner[b] is the node
 * of source box b of that level (device, [nbox_src[lpar]]).  With the
 * critical level lcrit = max(lpar - 1, 2), every source box of levels 2..L
 * gets a type (types[l] device, [nbox_src[l]], caller-owned, for l = 2..L):
 *   levels < lcrit: DOMESTIC;
 *   lcrit: IMPORT if none of its descendants at lpar is owned by J, else ROOT
 *          if some is not, else EXPORT if an M2L neighbour (E4 entry) has a
 *          descendant at lpar not owned by J, else DOMESTIC;
 *   deeper: a box "on J" (its ancestor at lpar owned by J) is EXPORT if an
 *          M2L neighbour is not on J, else DOMESTIC; a box not on J is IMPORT
 *          if an M2L neighbour is on J, else OTHERS.
 * (Readings: ownership is read at lpar, and the IMPORT marks the printed
 * algorithm sets from other boxes' threads are kept.)  The tree must be a
 * build of the sources against themselves (the same array as src and recv,
 * with lists), the last build of ctx.  Asynchronous on `stream`; scratch
 * from the arena.  FMM_ERR_LEVEL for lpar outside 2..L, FMM_ERR_ARG for a
 * tree that is not built against itself. */
#define FMM_BOX_DOMESTIC 0
#define FMM_BOX_EXPORT 1
#define FMM_BOX_IMPORT 2
#define FMM_BOX_ROOT 3
#define FMM_BOX_OTHERS 4
int fmm_box_types(fmm_ctx* ctx, const fmm_tree* tree, int lpar, const uint32_t* owner,
                  uint32_t node, uint8_t* const* types, void* stream);

/* ---- Served dynamic rebuilds ---------------------------------------------
 *
 * Dynamic problems rebuild the structure every time step (Sec. 1).  The
 * server keeps time-stepped point systems resident on the device.  A request
 * advances one system by one step: every point moves by an independent
 * N(0, sigma^2) step per axis, sigma = sigma_scale * 2^-L, reflecting at the
 * cube walls (fmm_displace), and the system's structure is rebuilt at its
 * fixed depth L (aliased sources = receivers).  Requests to one system run in
 * arrival order, one at a time.  Workers (each with its own context and
 * stream, so their builds overlap on the device) take, whenever they free
 * up, every waiting system they can -- oldest request first, at most
 * max_batch, while the systems' workspace estimates fit the worker's share
 * of the memory budget (always at least one) -- and build them in one
 * batched build (continuous batching).  A step's result depends only on the
 * system's state and step number, never on its batch. */

/* One time step of n points in place (xyz [n][3], device): point i, axis
 * x / y / z, moves by sigma * z_i with standard normal draws from
 * Philox4x32-10 (Salmon et al., SC'11) at counter (i, step low, step high, 0)
 * and key (seed low, seed high): output words r0..r3 give uniforms
 * u_k = (floor(r_k / 2^9) + 1/2) * 2^-23 and Box-Muller normals
 * z_x = sqrt(-2 ln u0) cos(2 pi u1), z_y = sqrt(-2 ln u0) sin(2 pi u1),
 * z_z = sqrt(-2 ln u2) cos(2 pi u3); then x < 0 -> -x, x > 1 -> 2 - x.
 * float32 arithmetic.  Asynchronous on `stream`; runs on the current device. */
int fmm_displace(float* xyz, uint32_t n, uint64_t seed, uint64_t step, float sigma, void* stream);

typedef struct fmm_server fmm_server;

#define FMM_SERVER_DIGEST 0x1u /* hash every result (for equivalence tests) */

typedef struct fmm_server_params {
  uint32_t workers;    /* concurrent batched builds, >= 1 */
  uint32_t max_batch;  /* systems per batched build, >= 1 (1: one build per request) */
  uint64_t mem_budget; /* workspace bytes shared by the workers; 0: 80% of the
                          device memory free at creation */
  uint32_t flags;      /* FMM_SERVER_DIGEST */
} fmm_server_params;

/* Outcome of one request.  Times in seconds on the server's clock (steady,
 * zero at creation): arrival (for a trace: the scheduled arrival), start of
 * its batch, completion (the batch's results read back). */
typedef struct fmm_request_info {
  uint64_t id;
  uint32_t system;
  uint32_t status;     /* fmm_status of the step */
  uint64_t step;       /* the system's step count after this request */
  double t_arrival, t_start, t_done;
  uint32_t batch_size; /* systems built in the same batched build */
  uint32_t worker;
  uint64_t points;     /* points of the system */
  uint64_t nnz_e2, nnz_e4; /* list entries over all levels */
  uint64_t digest;     /* FMM_SERVER_DIGEST: hash of every output array, else 0 */
} fmm_request_info;

/* Creates a server on `device` and starts its worker threads. */
int fmm_server_create(fmm_server** srv, int device, const fmm_server_params* params);
/* Finishes every queued request, stops the workers, frees everything. */
int fmm_server_destroy(fmm_server* srv);
/* Adds a system of n points (xyz [n][3] float32: host memory if `host`,
 * else device), copied into the server; depth L (0..21) and step size
 * sigma_scale * 2^-L are fixed for its life; seed keys its random steps.
 * The system starts at step 0.  FMM_ERR_DOMAIN for a coordinate outside
 * [0, 1]. */
int fmm_server_add_system(fmm_server* srv, const float* xyz, uint32_t n, int host, int L,
                          float sigma_scale, uint64_t seed, uint32_t* system);
/* Queues one step of `system` (arrival: now). */
int fmm_server_submit(fmm_server* srv, uint32_t system, uint64_t* request_id);
/* Blocks until the request is done. */
int fmm_server_wait(fmm_server* srv, uint64_t request_id, fmm_request_info* info);
/* Does not block: FMM_PENDING while the request is queued or running (info
 * untouched); once it is done, the same as fmm_server_wait. */
int fmm_server_poll(fmm_server* srv, uint64_t request_id, fmm_request_info* info);
/* Open-loop replay: request k arrives at (call time + arrival_s[k]) for
 * system[k] (arrival_s ascending); blocks until every request is done and
 * fills info[k]. */
int fmm_server_run_trace(fmm_server* srv, const double* arrival_s, const uint32_t* system,
                         uint32_t count, fmm_request_info* info);
/* Copies a system's current points to host memory (xyz [n][3]); the system
 * must have no request queued or running (FMM_ERR_ARG otherwise). */
int fmm_server_points(fmm_server* srv, uint32_t system, float* host_xyz);
/* The system's latest tree: the served build's own output while the worker
 * that built it has not taken another batch, else a rebuild of the same
 * points on a context of the server's own (a build depends on the points and
 * L alone).  The device arrays stay valid until the next request is submitted
 * or the next fmm_server_tree call.  FMM_ERR_ARG if the system has no result
 * yet or has a request queued or running. */
int fmm_server_tree(fmm_server* srv, uint32_t system, fmm_tree* out);

/* Static description of a status code. */
const char* fmm_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* FMMDS_H */
