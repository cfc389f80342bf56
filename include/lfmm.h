/* lfmm.h - C ABI of the GB300 lattice fast multipole method library (liblfmm.so).
 *
 * The library evaluates the lattice sum
 *
 *     u(m) = sum_n phi(m - n) f(n),     m, n in Z^2                (eq. 1.7 / eq. 2.1)
 *
 * for finitely many source points n (charges f) and target points m, where phi
 * is the fundamental solution of the 5-point discrete Laplacian A (eq. 1.2),
 * normalised by the Fourier integral eq. 1.8 so that phi(0) = 0 and
 * A phi = delta_0.  The evaluation is the lattice FMM of Sec. 8: a uniform
 * quadtree (Sec. 6), skeleton-based outgoing/incoming expansions (Sec. 4-5),
 * the translation operators T_ofs, T_ofo, T_ifo, T_ifi, T_tfi (Sec. 7), and a
 * direct near field from a tabulated phi (Sec. 2, Sec. 3).
 *
 * Conventions
 *  - Every entry point returns an int status (LFMM_OK = 0 on success); nothing
 *    throws across this boundary and nothing exits the process.
 *    lfmm_last_error() gives a human-readable detail for the calling thread.
 *  - Coordinates are int32 pairs interleaved (x0, y0, x1, y1, ...).
 *  - Any array argument may live in host memory (pageable or pinned) or in
 *    device memory of the current CUDA device; the library detects which with
 *    cudaPointerGetAttributes and copies host data through its own buffers.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *    enqueued on it; when an output is a host pointer the call returns after
 *    the result has been copied back, otherwise it returns asynchronously.
 *  - The caller keeps ownership of all arrays it passes.  A plan owns copies of
 *    the (sorted) coordinates, the tree, and its workspaces; the per-level
 *    operators and the phi table live in a process-wide cache shared by plans.
 *  - A plan may be used from one thread at a time; concurrent lfmm_eval calls
 *    on one plan race on its workspaces.
 */
#ifndef LFMM_H
#define LFMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------- */
#define LFMM_OK 0
#define LFMM_EINVAL 1        /* invalid argument (NULL, n < 0, extent > 2^30, bad opts) */
#define LFMM_ENOMEM 2        /* device or host allocation failed; nothing leaked       */
#define LFMM_ECUDA 3         /* a CUDA runtime call failed (detail in lfmm_last_error)  */
#define LFMM_ETIMEOUT 4      /* a bounded device-side wait gave up                      */
#define LFMM_EUNSUPPORTED 5  /* valid request this build does not handle                */
#define LFMM_EINTERNAL 6     /* internal consistency check failed                       */
#define LFMM_EBUSY 7         /* a server refused or shed a request (overload policy)    */
#define LFMM_ECANCELED 8     /* a queued server request was cancelled                   */

/* ---- precision paths ------------------------------------------------------------- */
/* LFMM_FP64: every step in binary64 (the plain path, relative error <= 1e-10 at p >= 16).
 * LFMM_MIXED: near field, expansions and translations in binary32, charges rounded
 *   to binary32, the per-target sum of near and far parts in binary64 (<= 1e-6). */
#define LFMM_FP64 0   /* every step in binary64                                         */
#define LFMM_MIXED 1  /* binary32 near and far field, compensated charge channel, TF32    */
                      /* tensor-core M2L; binary64 final sum (relative error ~1e-7)       */
#define LFMM_DF 2     /* binary64 inputs and outputs, every step in float-float pairs     */
                      /* (~48 bits) on the FP32 pipes: binary64-level accuracy at a       */
                      /* fraction of the binary64 pipe's cost                             */

typedef struct lfmm_plan lfmm_plan;

typedef struct lfmm_opts {
    int32_t precision;        /* LFMM_FP64, LFMM_MIXED or LFMM_DF                             */
    int32_t p;                /* expansion order, 2 <= p <= 17; skeleton size P = 4(p-1)        */
                              /* (Table 4.1: P ~ 27 gives 1e-8, P ~ 49 gives 1e-13)           */
    int32_t leaf_size;        /* N_leaf of Sec. 6: the leaf level is the coarsest level whose  */
                              /* boxes hold at most N_leaf sources and at most N_leaf targets  */
    int32_t max_leaf_side;    /* largest leaf side in lattice cells, a power of 2 in [1, 32]   */
    int32_t proxies_per_edge; /* proxy points per edge of the proxy ring of Sec. 5 (>= 8);     */
                              /* the remark of Sec. 5 finds 40 enough for 1e-10               */
    int32_t tc_min_level;     /* mixed path: tree levels >= this run M2L on the tensor cores  */
                              /* (0 = default 6; a value > 30 disables them); pruned storage  */
                              /* and forests: every list level of >= 1024 boxes runs there    */
                              /* unless this is > 30                                          */
    int32_t tree;             /* LFMM_TREE_AUTO, LFMM_TREE_UNIFORM or LFMM_TREE_PRUNED         */
    int32_t flags;            /* bitwise OR of LFMM_FLAG_* (0: none)                           */
    /* M2L tiling (0 everywhere: the library's rules; lfmm_autotune picks these).  They    */
    /* change how the interaction-list GEMM of Sec. 8.2 step 3 is cut into tiles, not    */
    /* what it computes: results differ at most by rounding (summation order).            */
    int32_t m2l_tile;         /* tensor-core M2L: target tile width in boxes, 16, 32, 64 or    */
                              /* 128 (a tile is 128 boxes of one parity class, as wide as    */
                              /* this and the class row allow); 0: as wide as possible       */
    int32_t m2l_stages;       /* tensor-core M2L: depth of the TMA ring, 2, 3 or 4 (0: 3)      */
    int32_t m2l_split;        /* coarse-level and list M2L kernels: chunks the 27 interaction  */
                              /* offsets are split into, 1 .. 9 (0: by the number of tiles); */
                              /* list levels whose 32-box tiles fill the GPU three times over */
                              /* are never split                                              */
    int32_t reserved;         /* must be 0                                                     */
} lfmm_opts;

/* Evaluate through a CUDA graph: the first lfmm_eval / lfmm_eval_parts of a plan records
 * its kernel launches (stream capture on a plan-owned stream, nothing runs) into a graph,
 * which that call and every later one with the same device argument pointers launch on
 * the caller's stream in one call; new pointers re-record it (the executable graph is
 * updated in place when possible).  Host f / u are staged through plan-owned device
 * buffers, so they reuse the graph too.  Results are bit-identical to the eager
 * launches.  While phase profiling is on (lfmm_profile_enable) evaluation is eager, so
 * that each phase can be timed. */
#define LFMM_FLAG_GRAPH 1
/* Run the whole evaluation on the caller's stream, one kernel after the other.  By
 * default the near field (P2P) runs on a second stream beside the far-field sweeps and
 * the two are joined by one elementwise sum; serial order gives each kernel the whole
 * device, so per-phase timings (lfmm_profile_*) measure each kernel alone.  Results
 * are bit-identical either way. */
#define LFMM_FLAG_SERIAL 2
/* Pruned trees and forests: run the upward sweep (P2M of every leaf, then M2M level by
 * level) of all problems as one persistent cooperative launch, and the downward sweep
 * (M2L + L2L, coarse to fine) as one persistent cooperative launch over the levels that
 * run on the CUDA cores (blocks take work from per-level queues, bounded grid barriers
 * between levels), followed by one tensor-core launch per finer level (mixed path,
 * levels of at least 1,024 boxes, as in the default form).  The results are
 * bit-identical either way; on the 4,096-problem forest the two forms measured within
 * 1 % of each other (per-level launches slightly ahead), and per-level launches are the
 * default. */
#define LFMM_FLAG_PERSISTENT 4

/* Tree storage.  UNIFORM: every box of every level is stored (Sec. 6), the layout for
 * points that fill their root box.  PRUNED: the same levels and boxes, but only boxes
 * with a source or target below them are kept, each with explicit parent, children and
 * interaction list; the layout for clustered points, whose leaf level is set by the
 * densest cluster.  AUTO picks PRUNED when more than half of the leaves are empty. */
#define LFMM_TREE_AUTO 0
#define LFMM_TREE_UNIFORM 1
#define LFMM_TREE_PRUNED 2

/* Fill opts with the defaults: LFMM_MIXED, p = 8, leaf_size = 64, max_leaf_side = 32,
 * proxies_per_edge = 64, tc_min_level = 0, tree = LFMM_TREE_AUTO, flags = 0, M2L tiling
 * by the library's rules (m2l_tile = m2l_stages = m2l_split = 0). */
void lfmm_opts_default(lfmm_opts* opts);

/* Build a plan for fixed source and target locations (Sec. 8.1 precomputation):
 * root box, uniform quadtree with leaf level chosen by N_leaf (Sec. 6), points
 * bucketed by leaf in Morton order, and the per-level skeletons and translation
 * operators of the model boxes (Sec. 8.1 steps 3-4, Remark 8.2), which are cached
 * process-wide by (leaf side, P, proxies per edge, precision).
 *   plan     out: the new plan, or NULL on failure
 *   src_xy   2*n_src int32 (host or device); n_src >= 1
 *   tgt_xy   2*n_tgt int32 (host or device); n_tgt >= 1
 *   opts     NULL for the defaults
 *   stream   cudaStream_t for all device work
 * The points must span at most 2^30 lattice cells per axis (LFMM_EINVAL).
 * Duplicate points are allowed (the sum is linear).  Synchronises `stream` twice
 * (the root box and the leaf level are read back to size the workspaces).  Uniform
 * storage without LFMM_FLAG_SERIAL buckets the targets on a plan-owned second stream
 * behind the work queued on `stream`; every later call that reads them (evaluation on
 * any stream, graph replay, lfmm_plan_destroy) waits for it. */
int lfmm_plan_create(lfmm_plan** plan, const int32_t* src_xy, int64_t n_src,
                     const int32_t* tgt_xy, int64_t n_tgt, const lfmm_opts* opts, void* stream);

/* A forest: n_problems independent problems in one plan, evaluated together.  Problem
 * i owns sources src_xy[2 src_offsets[i] .. 2 src_offsets[i+1]) and targets likewise;
 * every problem needs at least one source and one target.  All problems share the leaf
 * side (the largest power of two <= opts.max_leaf_side at which no leaf of any problem
 * holds more than opts.leaf_size sources or targets), hence the model-box operators of
 * every level; each has its own root box and leaf level.  Boxes are stored pruned (see
 * LFMM_TREE_PRUNED) and every sweep covers all problems in one launch per level.
 *   src_offsets, tgt_offsets  n_problems + 1 int64 in HOST memory, offsets[0] = 0,
 *                             non-decreasing, offsets[n_problems] = the point count
 * lfmm_eval on the plan takes f for all sources and writes u for all targets, both in
 * the concatenated order.  Synchronises `stream` (several times). */
int lfmm_forest_create(lfmm_plan** plan, const int32_t* src_xy, const int64_t* src_offsets,
                       const int32_t* tgt_xy, const int64_t* tgt_offsets, int64_t n_problems,
                       const lfmm_opts* opts, void* stream);

/* Apply the plan (Sec. 8.2): u[i] = sum_j phi(tgt_i - src_j) f[j] for all targets,
 * in the caller's target order.  f: n_src doubles, u: n_tgt doubles (host or device).
 * A coincident source contributes phi(0) = 0.  If sum(f) != 0 the result keeps the
 * normalisation phi(0) = 0 of eq. 1.8. */
int lfmm_eval(lfmm_plan* plan, const double* f, double* u, void* stream);

/* As lfmm_eval but returns the two parts separately: u_near (same and adjacent
 * leaves, eq. 2.2) and u_far (everything else, eq. 2.4, through the expansions). */
int lfmm_eval_parts(lfmm_plan* plan, const double* f, double* u_near, double* u_far, void* stream);

/* Release a plan (NULL is a no-op).  Waits for the plan's outstanding work. */
int lfmm_plan_destroy(lfmm_plan* plan);

/* Apply the plan to k charge vectors at once: U[r n_tgt + i] = sum_j phi(tgt_i - src_j)
 * F[r n_src + j] for r < k (vector-major layouts, host or device, k in [1, 4096]).
 * Each vector's result is bit-identical to lfmm_eval on the same plan; the near field of
 * four vectors shares every table lookup (a uniform plan with a far field; forests and
 * trees without a far field evaluate the vectors one after another).  The per-vector
 * buffers grow with the largest k seen and stay with the plan.  Evaluates eagerly (the
 * graph flag applies to lfmm_eval). */
int lfmm_eval_multi(lfmm_plan* plan, const double* F, int32_t k, double* U, void* stream);

/* One-shot solve: lfmm_plan_create + lfmm_eval + lfmm_plan_destroy in one call, for
 * points that are solved once.  Host inputs are uploaded first (coordinates on
 * `stream`); the upload of a host f runs on a second stream behind them, overlapping
 * the tree build.  A host u is filled when the call returns (it synchronises `stream`);
 * a device u is ready in stream order.  Arguments as for the three calls. */
int lfmm_solve(const int32_t* src_xy, int64_t n_src, const int32_t* tgt_xy, int64_t n_tgt, const double* f,
               double* u, const lfmm_opts* opts, void* stream);

/* Replace the plan's LFMM_FLAG_* bits (graph replay, serial order) for later
 * evaluations; clearing LFMM_FLAG_GRAPH releases the recorded graph.  Work already
 * queued is not affected. */
int lfmm_plan_set_flags(lfmm_plan* plan, int32_t flags);

/* Synchronise `stream` and report device-side failures of the plan's kernels since the
 * last call: LFMM_ETIMEOUT if a bounded wait inside a kernel gave up (an mbarrier wait of
 * the tensor-core M2L or a grid barrier of the fused coarse-level kernels; the affected
 * results are not valid), else LFMM_OK.  Clears the status. */
int lfmm_plan_status(lfmm_plan* plan, void* stream);

/* Bound of the plan's device-side waits (the grid barriers of the cooperative coarse-level
 * kernels and the mbarrier polls of the tensor-core M2L), in polls; 0 restores the
 * defaults (about 2^24 polls, a second or more).  An expired wait records LFMM_ETIMEOUT
 * for lfmm_plan_status and lets the kernel finish with invalid results instead of
 * hanging; the tensor-core kernel still waits, with the default bound, for the copies and
 * products it has issued before it frees its tensor memory and exits.  A small bound
 * turns slow progress into timeouts: it is meant for tests of the timeout path and for
 * callers that prefer a fast failure.  Enqueued on the plan's last stream. */
int lfmm_plan_set_wait_budget(lfmm_plan* plan, int32_t polls);

/* Test hook for the timeout path: sets the arrival count of the plan's grid barrier far
 * beyond any grid size, so that no arrival completes the next barrier, as if blocks of
 * the next cooperative kernel never arrived.  Every block then waits its poll budget out
 * at each barrier of the evaluation, which records LFMM_ETIMEOUT.
 * lfmm_plan_status reports it and puts the barrier words back to zero, after which the
 * plan evaluates normally again.  Enqueued on the plan's last stream. */
int lfmm_plan_inject_barrier_stall(lfmm_plan* plan);

typedef struct lfmm_plan_info {
    int64_t n_src, n_tgt;
    int64_t x0, y0;           /* lower-left corner of the root box                       */
    int32_t K;                /* root side 2^K                                          */
    int32_t L;                /* leaf level; 4^L leaves of side 2^(K-L)                  */
    int32_t leaf_side;
    int32_t P;                /* skeleton size of the leaf model box                     */
    int32_t P_pad;            /* padded expansion length in device arrays (32 or 64)     */
    int32_t precision;
    int32_t max_leaf_src;     /* largest number of sources in one leaf                   */
    int32_t max_leaf_tgt;
    int64_t device_bytes;     /* device memory owned by the plan (not the shared cache)  */
    int32_t tree;             /* LFMM_TREE_UNIFORM or LFMM_TREE_PRUNED (forests: PRUNED) */
    int32_t n_problems;       /* 1, or the number of problems of a forest                */
    int64_t n_boxes;          /* boxes holding expansions (levels >= 2; pruned: leaves)  */
} lfmm_plan_info;

int lfmm_plan_get_info(const lfmm_plan* plan, lfmm_plan_info* info);

const char* lfmm_status_string(int status);
/* Detail of the last failure on the calling thread ("" if none). */
const char* lfmm_last_error(void);

/* ---- serving ----------------------------------------------------------------------- */
/* A request loop for solves that arrive over time (different point sets and counts).
 * The server runs n_slots requests at once, each on its own worker thread and CUDA
 * stream; requests wait in arrival order and the oldest is admitted as soon as a slot
 * is free and its estimated device footprint fits beside the running ones, within
 * hbm_budget_bytes and the device's free memory (memory the stream-ordered pool holds
 * unused counts as free).  Requests at binary64-level tolerance may hold at most
 * n_slots - max(1, n_slots/4) slots; while they fill those, later mixed requests may
 * pass them.  An admitted request builds its plan, evaluates and frees
 * the plan on its stream, overlapping on the device with the others.  The model-box
 * operators and phi tables stay resident (process-wide cache).  A request's result is
 * independent of the requests that run beside it. */
typedef struct lfmm_server lfmm_server;

typedef struct lfmm_request {
    const int32_t* src_xy;    /* 2*n_src int32, host or device; owned by the caller until  */
    int64_t n_src;            /* lfmm_server_wait returns                                  */
    const int32_t* tgt_xy;
    int64_t n_tgt;
    const double* f;          /* n_src, host or device                                     */
    double* u;                /* n_tgt result, host or device                              */
    double tol;               /* requested relative error: >= 1e-6 runs the mixed path at  */
                              /* p = 8, smaller values the float-float path (LFMM_DF) at   */
                              /* p = 16 with leaves of up to 192 points                    */
} lfmm_request;

typedef struct lfmm_request_stats {
    int32_t status;           /* the request's own status                                   */
    int32_t precision;        /* LFMM_MIXED or LFMM_DF                                      */
    double queue_ms;          /* submit -> admission                                        */
    double run_ms;            /* admission -> result in u                                   */
    double total_ms;          /* submit -> result in u (latency)                            */
    int64_t device_bytes;     /* device memory of the request's plan                        */
} lfmm_request_stats;

/* n_slots in [1, 64]; hbm_budget_bytes = 0 for 80 % of the device memory available at
 * creation.  Uses the current device. */
int lfmm_server_create(lfmm_server** server, int32_t n_slots, int64_t hbm_budget_bytes);
/* Queue a request (returns at once); *ticket identifies it for lfmm_server_wait. */
int lfmm_server_submit(lfmm_server* server, const lfmm_request* req, int64_t* ticket);
/* Block until the request is done; fills *stats (may be NULL) and returns its status.
 * Each ticket can be waited for once. */
int lfmm_server_wait(lfmm_server* server, int64_t ticket, lfmm_request_stats* stats);
/* Finish the queued requests, stop the workers and free the server (NULL: no-op). */
int lfmm_server_destroy(lfmm_server* server);
/* Overload policy.  max_pending > 0 bounds the requests waiting for admission:
 * lfmm_server_submit refuses a request beyond it with LFMM_EBUSY (no ticket is issued).
 * max_queue_ms > 0 is a latency budget for the wait before admission.  At submit, the
 * server predicts the wait (the run times it has measured for requests of the same path
 * and size, summed over the queued requests and divided by the slots) and refuses the
 * request with LFMM_EBUSY when that exceeds the budget; a queued request that has waited
 * longer than the budget anyway is shed when the server next considers its queue (at
 * every submit and whenever a slot frees) and completes with LFMM_EBUSY (its ticket must
 * still be waited for).  0 disables either limit (the default: every request is
 * eventually served). */
int lfmm_server_set_limits(lfmm_server* server, int32_t max_pending, double max_queue_ms);
/* Cancel a request that is still waiting for admission: it leaves the queue and
 * completes with LFMM_ECANCELED (its ticket must still be waited for).  A request that
 * has been admitted runs to the end: LFMM_EINVAL, and the request is not affected. */
int lfmm_server_cancel(lfmm_server* server, int64_t ticket);

/* ---- autotuner ---------------------------------------------------------------------- */
/* Picks the expansion order p, the leaf size N_leaf and the tensor-core levels for a
 * point set (or a forest of point sets) and a required accuracy, by measurement on the
 * device.  The paper fixes none of these (it reports the error for chosen P, Table 4.1,
 * and times one leaf size, Sec. 9); the choice is the fastest configuration whose error
 * meets the request:
 *   1. precision: LFMM_MIXED when tol >= 1e-6, else LFMM_DF;
 *   2. reference: the same points evaluated by LFMM_DF at p = 16 (rel. error ~1e-13)
 *      for a fixed pseudo-random zero-sum charge vector;
 *   3. p: the smallest candidate (MIXED: 4..9, DF: 10, 12, 14, 16, 17) whose max-norm
 *      relative error against the reference is <= tol / 2 at leaf size 64;
 *   4. N_leaf (MIXED: 32, 64, 128; DF: 64, 128, 192) and then, for MIXED, the first
 *      tensor-core level (the leaf level, the one above it, or none): the smallest
 *      median time of plan creation + evaluation over three timed steps; a candidate
 *      whose error exceeds tol / 2 is skipped;
 * Results are cached process-wide by (precision, decade of tol, ceil(log2) of the
 * source and target counts, ceil(log2) of the problem count, tree storage); a cached
 * entry is returned without measuring (result->from_cache = 1).
 *   src_offsets, tgt_offsets  NULL with n_problems = 1 for one problem, else as for
 *                             lfmm_forest_create (host memory)
 *   tol                       required max-norm relative error, in [1e-13, 1e-2]
 *   base                      NULL for the defaults; its max_leaf_side, proxies_per_edge
 *                             and tree are kept, its flags copied to the result
 *   result                    out: the chosen options and their measurements
 * Runs on `stream` and synchronises it; the plans it builds are destroyed before it
 * returns. */
typedef struct lfmm_tune_result {
    lfmm_opts opts;           /* the chosen options                                        */
    double rel_err;           /* their error against the reference evaluation             */
    double ms;                /* their median plan create + eval time (ms)                 */
    int32_t candidates;       /* configurations measured (0 when from the cache)           */
    int32_t from_cache;
} lfmm_tune_result;

int lfmm_autotune(const int32_t* src_xy, int64_t n_src, const int64_t* src_offsets,
                  const int32_t* tgt_xy, int64_t n_tgt, const int64_t* tgt_offsets, int64_t n_problems,
                  double tol, const lfmm_opts* base, lfmm_tune_result* result, void* stream);
/* Forget every cached tuning result. */
int lfmm_tune_cache_clear(void);
/* Write the cache to `path` (one text line per entry) / merge entries from such a file
 * (LFMM_EINVAL on a malformed line; entries before it are kept). */
int lfmm_tune_cache_save(const char* path);
int lfmm_tune_cache_load(const char* path);

/* ---- plan shape without allocation -------------------------------------------------- */
/* The paper has no counterpart: this is a service entry point for callers that cannot
 * allocate device memory when they have to decide about a problem - an admission
 * controller sizing a request before committing memory to it, host code running while
 * a stream is being captured into a CUDA graph (where allocation calls are illegal), or
 * a process whose device memory belongs to another allocator.
 *
 * Fills *info with what lfmm_plan_create would produce for these points and opts: root
 * corner and K, leaf level L and leaf side, largest leaf occupancies, P and P_pad, and
 * device_bytes = the device memory the plan would own when its coordinates are given
 * in device memory, and the storage the plan would pick (info->tree).  For pruned
 * storage, device_bytes and n_boxes are those of the uniform layout (upper bounds).
 * Calls no cudaMalloc/cudaFree or any allocating routine.
 *   src_xy, tgt_xy  8-byte aligned DEVICE memory (LFMM_EINVAL otherwise)
 *   stream          the work runs on it; the call synchronises it (results go to the host)
 * Limits: the leaf-count scratch is a static device array of LFMM_NOALLOC_SCRATCH_BYTES
 * (every GPU that loads the library holds it until the process exits); trees that need
 * counting below level 10 (more than 4^10 boxes per level) are rejected with
 * LFMM_EINVAL and a message saying so.  The first call on a device resolves the
 * array's device address (cudaGetSymbolAddress) and should be made before any stream
 * capture.  Calls share the array: concurrent calls (other streams or threads) race
 * and must be serialised by the caller. */
#define LFMM_NOALLOC_SCRATCH_BYTES (4 * (2 * (1 << 20) + 2 * (1 << 18) + 64))
int lfmm_plan_shape_noalloc(const int32_t* src_xy, int64_t n_src, const int32_t* tgt_xy,
                            int64_t n_tgt, const lfmm_opts* opts, lfmm_plan_info* info,
                            void* stream);

/* ---- device memory accounting and allocation-failure injection --------------------- */
/* Bytes in use in the current device's default stream-ordered memory pool, from which
 * the library takes plan memory and temporaries (the shared operator cache is separate).
 * With no plan alive and no call in flight it returns to its earlier value: a failed
 * call leaks nothing. */
int lfmm_pool_used_bytes(int64_t* bytes);
/* Test hook: the nth device allocation the library makes from now on (n >= 1; plans,
 * temporaries and staging buffers, any thread) fails as if the device were out of
 * memory, so that the caller sees LFMM_ENOMEM; the hook disarms itself after that
 * allocation.  n = 0 disarms it.  Process-wide. */
int lfmm_fault_inject_alloc(int64_t nth);

/* ---- tracing ---------------------------------------------------------------------- */
/* Phases timed by the profiler with CUDA events recorded on the stream each phase is
 * enqueued on (plan create: TREE, OPERATORS; eval: the sweeps of Sec. 8.2). */
#define LFMM_PHASE_TREE 0       /* root box, leaf level, leaf buckets (Sec. 6)          */
#define LFMM_PHASE_OPERATORS 1  /* model-box operator cache lookup / upload (Sec. 8.1)  */
#define LFMM_PHASE_P2M 2        /* step 1: T_ofs                                        */
#define LFMM_PHASE_M2M 3        /* step 2: T_ofo                                        */
#define LFMM_PHASE_M2L 4        /* steps 3-4: T_ifo and T_ifi (SIMT kernels)            */
#define LFMM_PHASE_P2P 5        /* step 5: near field, T_tfi, binary64 final sum        */
#define LFMM_PHASE_COPY 6       /* host<->device copies of coordinates, f and u         */
#define LFMM_PHASE_M2L_TC 7     /* steps 3-4 on the tensor cores (fp32 levels, P <= 32) */
#define LFMM_PHASE_L2P 8        /* step 5 far part and final sum, when the near field   */
                                /* runs concurrently with the far-field sweeps          */
#define LFMM_NUM_PHASES 9

/* Turn per-phase timing on (1) or off (0).  While on, every create/eval synchronises its
 * stream once at the end to read the events.  Process-wide. */
int lfmm_profile_enable(int enable);
/* ms[i], launches[i] (either may be NULL; LFMM_NUM_PHASES entries) accumulated since the
 * last reset; reset != 0 clears them after reading. */
int lfmm_profile_read(double* ms, int64_t* launches, int reset);
/* Total kernels this library has launched in the process (always counted). */
int64_t lfmm_launch_count(void);

/* ---- host-side views of the precomputation (no GPU needed) ------------------------- */

/* The library's phi on the packed octant 0 <= lo <= hi <= R, entry hi*(hi+1)/2 + lo,
 * computed by the one-dimensional integral of Remark 3.1 (t1 integrated in closed
 * form, composite Gauss-Legendre in t2).  1 <= R <= 256; out holds (R+1)(R+2)/2 doubles. */
int lfmm_phi_table(int32_t R, double* out);
/* phi near the origin for a symmetric lattice operator with constant coefficients,
 * by the two-dimensional quadrature of Sec. 3.2 on the GPU (boxes of about one
 * oscillation with 20 x 20 Gauss-Legendre rules next to the centre and 14 x 14 further
 * out, the singular centre box as a sum of annuli with Richardson extrapolation).  The operator is
 *   (A u)(m) = sum_k w[k] (2 u(m) - u(m + d_k) - u(m - d_k)),  d_k = (d[2k], d[2k+1]),
 * with 1 <= n_terms <= 8 distinct offsets (no two opposite), |d| <= 64, w[k] > 0, and two
 * offsets of determinant +-1 (so that the symbol vanishes only at 0); the 5-point
 * operator of eq. 1.2 is d = {1,0, 0,1}, w = {1, 1}.  Then A phi = delta_0, phi(0) = 0.
 * With Q = sum_k w[k] d_k d_k', c = sqrt(det Q) / max(Q_11, Q_22) must be >= 1/8 (the
 * pieces near the origin are split ceil(1/c) times per side; c = 1 for eq. 1.2).
 * out: (2R+1)^2 doubles (host or device), out[(y + R)(2R+1) + x + R] = phi(x, y);
 * R in [1, 64].  Runs on `stream` (this one needs the GPU); a host `out` is filled when
 * the call returns.  LFMM_EINVAL for arguments outside these ranges (checked before any
 * launch), LFMM_ECUDA for a failed launch or copy. */
int lfmm_phi_quadrature(const int32_t* d, const double* w, int32_t n_terms, int32_t R, double* out, void* stream);

/* phi at n integer offsets d = (dx0, dy0, dx1, dy1, ...): the table above for
 * |d|_inf <= 128, the asymptotic expansion eq. 3.1 beyond. */
int lfmm_phi(const int64_t* d, int64_t n, double* out);

/* Skeleton of the model box `level_above_leaf` levels above a leaf of side
 * leaf_side (box side leaf_side * 2^level_above_leaf, lower-left corner at 0):
 * xy receives up to 2*64 int32, *count the skeleton size (Sec. 5, Sec. 8.1 step 3). */
int lfmm_model_skeleton(int32_t leaf_side, int32_t p, int32_t proxies_per_edge,
                        int32_t level_above_leaf, int32_t* xy, int32_t* count);

/* Leaf outgoing-from-sources operator for the dense leaf box (Remark 8.2):
 * out receives count x leaf_side^2 doubles, row-major, column j the lattice point
 * (j % leaf_side, j / leaf_side).  T_tfi is its transpose (Sec. 7). */
int lfmm_model_tofs(int32_t leaf_side, int32_t p, int32_t proxies_per_edge, double* out);

/* Parent-from-children interpolation S of Sec. 7 at `level_above_leaf` >= 1:
 * out receives count_parent x (4 * count_child) doubles, row-major; column block i
 * (children in Morton order (0,0),(1,0),(0,1),(1,1)) is T_ofo for child i, and its
 * transpose is T_ifi. */
int lfmm_model_s(int32_t leaf_side, int32_t p, int32_t proxies_per_edge,
                 int32_t level_above_leaf, double* out);

#ifdef __cplusplus
}
#endif

#endif /* LFMM_H */
