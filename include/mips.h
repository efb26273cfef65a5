/*
 * mips.h -- C ABI of libmips: exact batch top-K maximum inner product
 * search on one GB300 GPU (sm_103a).
 *
 * The operation (Sec. II-B, "Problem Statement: Batch Exact MIPS"): given
 * user vectors U (|U| x f) and item vectors I (|I| x f), return for every
 * user u the K items i with the largest u^T i.
 *
 * Result semantics shared by every entry point below:
 *   - out_idx[u * K + k] (int32) and out_score[u * K + k] (double) list the
 *     user's K best items, best first.  Items rank by u^T i of the FP32
 *     inputs, descending; equal scores rank by the smaller item index.
 *   - Indices equal those of the FP64 definition (sequential sum of the
 *     exact FP32 products, full sort per user) exactly, ties included:
 *     whenever two candidates are closer than the rescore's error bound the
 *     library recomputes them with exactly that FP64 arithmetic.
 *   - Scores are the exact inner product to within 2e-10 relative to
 *     ||u|| ||i|| (compensated FP32 arithmetic), or the FP64 definition's
 *     value itself for users resolved by the tie check.
 *
 * Conventions:
 *   - Matrices are row-major FP32, row r at ptr + r * f.
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous on it; argument errors return at
 *     once, device-side errors (non-finite input, a timed-out wait) are
 *     reported by mips_sync() or by the next call on the same index.
 *   - Device pointers must be valid on the index's device until the stream
 *     has reached the end of the call.  The caller owns every buffer it
 *     passes; the index owns its own copies and workspace.
 *   - An index is not thread-safe: serialise calls on one handle.
 *   - No C++ exception crosses this boundary.
 *   - Status codes: MIPS_ERR_ARG for null pointers, n <= 0, f < 1,
 *     K < 1 or K > n_items, unsupported sizes; MIPS_ERR_NOMEM when device
 *     memory runs out; MIPS_ERR_CUDA for any other CUDA failure;
 *     MIPS_ERR_NONFINITE when an input row holds NaN or Inf;
 *     MIPS_ERR_TIMEOUT when a bounded wait in a kernel gave up.
 *     mips_last_error() returns a message for the calling thread.
 */
#ifndef MIPS_H_
#define MIPS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mips_index_s* mips_index_t; /* opaque; owned by the library */

typedef enum {
  MIPS_OK = 0,
  MIPS_ERR_ARG = 1,
  MIPS_ERR_NOMEM = 2,
  MIPS_ERR_CUDA = 3,
  MIPS_ERR_TIMEOUT = 4,
  MIPS_ERR_OVERFLOW = 5,
  MIPS_ERR_UNIMPLEMENTED = 6,
  MIPS_ERR_NONFINITE = 7
} mips_status;

/* Arithmetic of the candidate (filter) pass of the blocked multiply. */
typedef enum {
  MIPS_FP32 = 0,     /* FP32 CUDA-core dot products */
  MIPS_BF16 = 1,     /* BF16 operands on tcgen05 tensor cores, FP32 accumulate */
  MIPS_FP8_E4M3 = 2  /* FP8 E4M3 operands on tcgen05 (kind::f8f6f4), FP32 accumulate: users scaled
                      * per row, items by one scale, bound columns rounded up (the same exact
                      * top-K, a looser candidate filter than BF16) */
} mips_dtype;

typedef struct {
  int dtype;          /* mips_dtype of the candidate pass (default MIPS_BF16) */
  int kmeans_iters;   /* Lloyd iterations for Maximus (Sec. III-D: i = 3) */
  int block_items;    /* Maximus item block B; 0 = library default */
  double sample_frac; /* Optimus user sample fraction (Sec. IV: 0.005) */
  int autotune;       /* reserved */
  uint64_t seed;      /* seed of the k-means initial centroids and samples */
  int kmeans_spherical; /* 1: spherical k-means (Sec. III-A): unit-length centroids, largest cosine */
} mips_options;

/* Fill *opt with the defaults listed above. */
void mips_default_options(mips_options* opt);

/*
 * Build an index over n_items item vectors of dimension f
 * (items_dev: device FP32 [n_items][f]; read during the call only).
 * clusters = |C| for Maximus (Sec. III-A; Algorithm 1 input "# clusters"),
 * fixed here and used by mips_topk_maximus.  The index copies the items
 * (FP32 master + quantised copies + per-item bounds); the caller may free
 * items_dev once the stream has passed this call.
 * Limits: 1 <= f <= 128, 1 <= n_items < 2^31, 1 <= clusters <= 4096;
 * options: 0 <= kmeans_iters <= 100, block_items >= 0, 0 < sample_frac <= 1,
 * kmeans_spherical 0 or 1, dtype one of mips_dtype (else MIPS_ERR_ARG).
 * *out receives the handle; free it with mips_free_index.
 */
mips_status mips_build_index(const float* items_dev, int64_t n_items, int f, int clusters,
                             const mips_options* opt, void* stream, mips_index_t* out);

/*
 * Blocked matrix multiply with fused top-K selection (Sec. II-C, "BMM"):
 * every user against every item, nothing pruned.
 * users_dev: device FP32 [n_users][f]; out_idx_dev: device int32
 * [n_users][K]; out_score_dev: device double [n_users][K].
 * 1 <= K <= min(n_items, 128).
 */
mips_status mips_topk(mips_index_t idx, const float* users_dev, int64_t n_users, int K,
                      int32_t* out_idx_dev, double* out_score_dev, void* stream);

/*
 * The Maximus index (Sec. III, Algorithm 1): cluster these users with
 * k-means into the index's |C| clusters, compute theta_b per cluster and
 * the per-cluster item lists ordered by CBound (Eq. appx_bound), then walk
 * each cluster's list in blocks for all of its users, stopping when no
 * remaining item can enter any user's top-K.  Same arguments and result
 * as mips_topk; the result is identical to mips_topk's (Theorem "exact").
 */
mips_status mips_topk_maximus(mips_index_t idx, const float* users_dev, int64_t n_users, int K,
                              int32_t* out_idx_dev, double* out_score_dev, void* stream);

/*
 * Dynamic users (Sec. III-E, "Practical Usage"): run k-means (the index's
 * kmeans_iters Lloyd iterations, initial centroids a seeded draw of users)
 * on these users (device FP32 [n_users][f], read during the call only) and
 * keep the min(|C|, n_users) centroids in the index.  Afterwards every
 * Maximus call on this index (mips_topk_maximus, mips_select, graphs,
 * servers and worker handles created later) assigns its users to these
 * centroids with one assignment step instead of clustering them; theta_b,
 * the bounds and the lists are still those of the call's users, and only
 * the clusters that receive users are walked.  The result stays exact
 * whatever the centroids.  mips_autotune then tunes B only.
 * users_dev = NULL with n_users = 0 drops the fitted centroids (clustering
 * per call again).  Errors: MIPS_ERR_ARG (null index, null users with
 * n_users != 0, n_users < 0 or >= 2^31), MIPS_ERR_NOMEM, MIPS_ERR_CUDA.
 * Asynchronous on stream; the index owns the centroid buffer.
 */
mips_status mips_fit_clusters(mips_index_t idx, const float* users_dev, int64_t n_users, void* stream);

/* Report of one Optimus decision (Sec. IV, "Overhead of Optimizer"). */
typedef struct {
  int choice;           /* 0 = blocked multiply, 1 = Maximus */
  double t_build;       /* C_I: seconds of Maximus construction on the sample */
  double q_user;        /* Q_I: Maximus seconds per user (sample) */
  double m_user;        /* M_I: blocked-multiply seconds per user (sample) */
  int64_t sample_users; /* s */
  double est_index;     /* predicted seconds: C_I + n * Q_I */
  double est_bmm;       /* predicted seconds: n * M_I */
} mips_select_report;

/*
 * Optimus (Sec. IV): time a random user sample on both paths, extrapolate
 * to all users, finish the remaining users with the faster one and reuse
 * the sample's results.  Full results land in out_idx_dev/out_score_dev.
 * This call synchronises the stream (it reads the sample's timings).
 * rep may be NULL.
 */
mips_status mips_select(mips_index_t idx, const float* users_dev, int64_t n_users, int K,
                        int32_t* out_idx_dev, double* out_score_dev, void* stream,
                        mips_select_report* rep);

/* One arm of mips_select_arms: a candidate pass (the dtype of one of the
 * given indexes) with one method. */
typedef struct {
  int index;        /* position of its index in the indexes argument */
  int dtype;        /* mips_dtype of that index */
  int method;       /* 0 blocked multiply (mips_topk), 1 Maximus (mips_topk_maximus) */
  int rounds;       /* timings of the sample taken */
  double est_mean;  /* predicted seconds for all n_users, mean over its timings */
  double est_ci;    /* half-width of the 95% confidence interval of that mean
                     * (Student t, rounds - 1 degrees of freedom; 0 below 2 rounds) */
  int dropped;      /* 1: no longer timed once its interval lay above the best arm's */
} mips_arm_report;

#define MIPS_MAX_ARMS 16

typedef struct {
  int n_arms;
  mips_arm_report arm[MIPS_MAX_ARMS];
  int choice;             /* arm that finished the remaining users */
  int separated;          /* 1: the chosen arm's interval lay below every other arm's */
  int rounds;             /* rounds run (every live arm timed once per round) */
  int64_t sample_users;   /* users in the timed sample */
  double t_sample;        /* seconds of device time spent timing arms on the sample */
  double t_total;         /* seconds of device time of the whole call */
} mips_arms_report;

/*
 * Multi-arm Optimus (Sec. IV, with more arms than the paper's two): the arms
 * are every given index (built on the same items, e.g. with the FP32, BF16
 * and FP8 candidate passes) times {blocked multiply, Maximus}.  A seeded
 * user sample (as mips_select's) is timed on every arm in rounds; each
 * timing is extrapolated to all users (blocked multiply: per user;
 * Maximus: the sample's k-means per user, bounds and sort once, the rest
 * per user).  The paper's early stop, a t-test on per-user times, does not
 * apply to arms that batch users, as all of these do; instead, after every
 * round from the third on, an arm whose interval lies above the best arm's
 * is dropped, and the rounds stop once the best arm's interval lies below
 * every remaining one (or after max_rounds, 3..16; 0 = 6).  The chosen arm's
 * sample results are kept and it computes the remaining users; every arm
 * is exact, so any choice gives the same top-K.  Synchronises the stream.
 * Every index must hold the same items (not checked: same f and n_items
 * are) and live on the current device; the call runs on indexes[0]'s
 * stream order (the others' earlier calls are waited for).  rep may be NULL.
 */
mips_status mips_select_arms(const mips_index_t* indexes, int n_indexes, const float* users_dev, int64_t n_users,
                             int K, int max_rounds, int32_t* out_idx_dev, double* out_score_dev, void* stream,
                             mips_arms_report* rep);

/* Result of mips_autotune. */
typedef struct {
  int clusters;            /* chosen |C|, now the index's */
  int block_items;         /* chosen item block B, now the index's */
  int64_t sample_users;    /* users in the timed sample */
  int n_tried;             /* candidates timed (at most 32) */
  int tried_clusters[32];  /* |C| of candidate t (for all n_users) */
  int tried_block[32];     /* B of candidate t */
  double tried_est[32];    /* predicted seconds of candidate t for all n_users */
  double t_tune;           /* seconds spent tuning (wall clock) */
} mips_tune_report;

/*
 * Autotuner for Maximus: picks the cluster count |C| and the item block B
 * (Sec. III-A, III-D) for these users by timing Maximus on a seeded user
 * sample (n_users / 8 users, at least two waves of 128-user tiles per SM)
 * for |C| in {16, ..., 1024} (at most n_users / 32) and B in {1024, 4096,
 * 16384}.  The sample runs with |C| scaled by sample / n_users, so that it
 * has the full run's users per cluster; the prediction for all users
 * scales the sample's k-means and per-user stages by n_users / sample and
 * k-means and the (cluster, item) bound and sort stages by the |C| ratio.
 * The best pair becomes the index's (later Maximus calls use it).
 * Synchronises the stream; rep may be NULL.  Errors as mips_topk.
 */
mips_status mips_autotune(mips_index_t idx, const float* users_dev, int64_t n_users, int K,
                          void* stream, mips_tune_report* rep);

/*
 * mips_topk (method 0) or mips_topk_maximus (method 1) through a CUDA
 * graph: the first call with a given (method, users_dev, n_users, K,
 * out_idx_dev, out_score_dev) runs the plain call and then captures the
 * same call into a graph held by the index; later calls with the same
 * arguments replay it with one cudaGraphLaunch on `stream` (the inputs
 * are read afresh, so new user values at the same address give new
 * results).  A graph is dropped once the index's workspace is reallocated
 * by a larger call; the index keeps at most 8.  The legacy default stream
 * (NULL) cannot be captured: the call then runs plain.  Same result
 * semantics, ownership and errors as mips_topk; method outside {0, 1}:
 * MIPS_ERR_ARG.  No counterpart in the paper (one grouped launch per pass
 * and the whole call in one graph are GPU forms of its batching).
 */
mips_status mips_topk_graph(mips_index_t idx, const float* users_dev, int64_t n_users, int K,
                            int method, int32_t* out_idx_dev, double* out_score_dev,
                            void* stream);

/*
 * Serving: a request loop over one index with continuous batching.
 * Requests (host user rows, any K) queue in arrival order; a scheduler
 * thread forms a batch from the oldest request and the requests after it
 * whose K falls in the same class (1; 2..10; 11..32; 33..128), up to
 * max_batch_users users, runs it with the batch's largest K (each request
 * keeps its own first K: the ranking is a strict order, so its top-K is the
 * prefix of a larger K's) and starts it as soon as one of `slots` stream
 * slots is free and the batch fits the memory budget next to the batches in
 * flight.  Each slot owns a worker handle of the index (shared item arrays,
 * own workspace), pinned staging and a stream, so batches overlap: one's
 * copies and rescore with another's score kernel.  A completion thread
 * scatters each batch's results to its requests' host buffers.  Results
 * are those of mips_topk / mips_topk_maximus on the request alone
 * (exact, so independent of the batch).  No counterpart in the paper,
 * which scores offline batches (Sec. II-C); this is the serving form of
 * its user batching.
 */
typedef struct mips_server_s* mips_server_t;

typedef struct {
  int method;              /* 0 = blocked multiply (mips_topk), 1 = Maximus */
  int slots;               /* batches in flight at once (1..8), one stream each */
  int64_t max_batch_users; /* users per batch; a larger request runs alone */
  int64_t mem_budget;      /* device bytes the batches in flight may hold (0 = unlimited): a batch is
                            * admitted only if its bytes (its call's workspace, computed by that call's
                            * own layout, plus its buffers) fit beside those in flight, or nothing is
                            * in flight; while the slots hold more than this, a slot frees its
                            * workspace and buffers after each batch */
} mips_server_options;

typedef struct {
  double t_submit;      /* seconds since the server started */
  double t_start;       /* its batch was launched */
  double t_done;        /* its results were in its host buffers */
  int64_t batch;        /* id of the batch that served it */
  int64_t batch_users;  /* users in that batch */
  int batch_K;          /* K the batch ran with */
  int slot;             /* stream slot of the batch */
  int64_t batch_bytes;    /* device bytes its batch was admitted with: the workspace its call lays out
                           * plus the batch's user rows and results */
  int64_t batch_ws_bytes; /* workspace bytes that call actually took (equal to the admitted workspace) */
  int64_t inflight_bytes; /* admitted bytes of every batch in flight when its batch started, its own included:
                           * never above mem_budget when mem_budget is at least one batch */
} mips_request_info;

/* Creates the server (its threads, streams, worker handles).  The index
 * must outlive the server.  opt NULL: method 0, 2 slots, 8192 users, no
 * budget.  Errors: MIPS_ERR_ARG (bad options), MIPS_ERR_CUDA/NOMEM. */
mips_status mips_server_create(mips_index_t idx, const mips_server_options* opt, mips_server_t* out);

/* Queues a request: users_host [n_users][f] float; results to
 * out_idx_host / out_score_host [n_users][K].  The three host buffers
 * must stay valid until mips_server_wait returns for the request.
 * Returns at once; *request_id identifies it.  Errors: MIPS_ERR_ARG (K out
 * of [1, min(n_items, 128)], n_users < 1, null pointers, server stopped). */
mips_status mips_server_submit(mips_server_t srv, const float* users_host, int64_t n_users, int K,
                               int32_t* out_idx_host, double* out_score_host, int64_t* request_id);

/* Waits until the request is done or timeout_s passes (MIPS_ERR_TIMEOUT;
 * the request stays queued).  info may be NULL.  A failed batch reports its
 * error to each of its requests. */
mips_status mips_server_wait(mips_server_t srv, int64_t request_id, double timeout_s, mips_request_info* info);

/* Finishes the queued and running requests, stops the threads and frees
 * the server's resources. */
mips_status mips_server_destroy(mips_server_t srv);

/*
 * Host-memory variant of mips_topk (method 0) / mips_topk_maximus
 * (method 1) / mips_select (method 2): copies users_host to the device,
 * runs the method and copies the results back, then synchronises `stream`.
 * Host buffers are used as given (pinned memory gives asynchronous copies).
 * Same result semantics as the device entry points.  Method 0 with at least
 * 131,072 users runs in up to eight user chunks whose copies (on a stream the
 * index owns) overlap the other chunks' compute on `stream`; mips_get_stats
 * then reports the last chunk.
 */
mips_status mips_topk_host(mips_index_t idx, const float* users_host, int64_t n_users, int K,
                           int method, int32_t* out_idx_host, double* out_score_host,
                           void* stream);

/* Wait for `stream` and report any device-side error raised by this
 * index's kernels since the last check (the error word is then cleared). */
mips_status mips_sync(mips_index_t idx, void* stream);

/* Counters of the last completed call (synchronises the index's work). */
typedef struct {
  uint64_t cand_emitted;   /* candidates the score kernels emitted */
  uint64_t cand_rescored;  /* candidates with upper bound >= final threshold */
  uint64_t users_overflow; /* users whose candidate list overflowed (exhaustive rescore) */
  uint64_t users_fp64;     /* users decided by the FP64 tie check */
  uint64_t pairs_scored;   /* (user, item) pairs scored by the Maximus walk */
  uint64_t blocks_walked;  /* item blocks the Maximus walk processed */
  int64_t n_users;         /* users in the last call */
  int clusters;            /* |C| of the last Maximus call */
  int dtype;               /* candidate-pass dtype used */
  int launches;            /* kernels the last call launched */
  int pad_;
  /* per-stage device time of the last call in milliseconds (CUDA events
   * recorded on the call's stream; 0 for stages it did not run) */
  double ms_prep;          /* quantisation / packing of the users */
  double ms_score;         /* fused score + select (blocked multiply) */
  double ms_rescore;       /* exact rescore + final top-K */
  double ms_kmeans;        /* Maximus: k-means iterations */
  double ms_bounds;        /* Maximus: theta_b + CBound for every (cluster, item) */
  double ms_sort;          /* Maximus: per-cluster list sort + user grouping */
  double ms_walk;          /* Maximus: grouped walk (score + select) */
  double ms_total;         /* whole call */
  uint64_t select_slow;    /* select slow-path entries (warp x 64-score chunk), BF16 path */
  double ms_kernel;        /* device time of the call's dominant kernel alone: the fused score + select
                            * launch of a blocked multiply, or the sum of the Maximus walk's two launches
                            * (first block, then the rest), without the work between them (CUDA events
                            * around the launches; the first two launches of a call are counted) */
} mips_stats;
mips_status mips_get_stats(mips_index_t idx, mips_stats* out);

/*
 * Read-only view of an internal device array of the index, for tests and
 * inspection: name is one of "perm" (int32 [n_items], sorted position ->
 * item id), "item_nrm" (float [n_items], upper bounds of ||i||, sorted
 * order), and after a Maximus call "assign" (int32 [n_users]), "centroids"
 * (float [C][f]), "cos_b" (float [C], lower bound of cos theta_b),
 * "bound_sorted" (float [C][n_items], CBound upper bounds in list order),
 * "list" (int32 [C][n_items], sorted item positions in list order),
 * "visited" (int32 [n_users], items scored per user), and after
 * mips_fit_clusters "fit_centroids" (float [C_fit][f]).  *dev_ptr and
 * *bytes describe the array; it stays valid until the next call on idx.
 */
mips_status mips_get_buffer(mips_index_t idx, const char* name, const void** dev_ptr,
                            int64_t* bytes);

/*
 * Exact top-K without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc/cudaFree
 * -- code running inside a custom device allocator or an out-of-memory
 * handler (the allocator must not be re-entered), a latency-critical path
 * where cudaFree's device-wide synchronisation is unacceptable, or a
 * process whose whole memory budget is owned by someone else.
 *
 * It runs the FP32 blocked multiply with fused select and the exact
 * rescore (the same kernels, and the same result semantics, as mips_topk on
 * an MIPS_FP32 index) directly on the caller's buffers: items_dev FP32
 * [n_items][f], users_dev FP32 [n_users][f], out_idx_dev int32 [n_users][K],
 * out_score_dev double [n_users][K], all device memory owned by the caller.
 * No index is needed and none of its state is used.
 *
 * Scratch comes from one static device array of 32 MiB per GPU, reserved
 * when the library's code is loaded on that GPU and held until the process
 * exits.  A call needs 8 n_items + n_users (28 + 28 cap) bytes of it plus
 * at most 5 KiB of counters and alignment padding, where cap = max(4K + 96,
 * K (2 + ln(n_items / K)) + 96) is the candidate slots per user (K = 10:
 * about 6,200 users against 17,770 items); larger calls return
 * MIPS_ERR_ARG (split the users).  A user whose candidates overflow its
 * slots is scored exhaustively (still exact, slower).  Limits as
 * mips_topk: 1 <= f <= 128, 1 <= K <= min(n_items, 128).
 *
 * All calls share that array and it keeps the last call's contents (each
 * call clears the counters that must start at zero).  Calls that overlap on
 * the GPU -- on two streams or from two host threads -- race on it and
 * return wrong results: serialise them.
 *
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  The call returns after `stream` has finished
 * it, and reports non-finite input as MIPS_ERR_NONFINITE.
 */
mips_status mips_topk_noalloc(const float* items_dev, int64_t n_items, const float* users_dev, int64_t n_users,
                              int f, int K, int32_t* out_idx_dev, double* out_score_dev, void* stream);

/*
 * Test hook of the bounded device waits (no counterpart in the paper; it
 * exists for the library's own tests).  Every wait inside the tensor-core
 * score kernel gives up after a limit, raises a timeout, lets the other
 * roles drain their copies and MMAs, frees the tensor memory and exits, so
 * the context stays usable.  After this call, the next blocked-multiply
 * launch of that kernel in this process (a BF16 mips_topk call) publishes
 * no work item: its MMA issuers and select warps wait for one until wait_ns
 * nanoseconds pass, and the call's mips_sync reports MIPS_ERR_TIMEOUT (the
 * call's rescore then finds empty candidate lists).  One launch only;
 * later launches are unaffected.  Errors: MIPS_ERR_ARG unless
 * 1e5 <= wait_ns <= 1e9.
 */
mips_status mips_test_expire_next_wait(int64_t wait_ns);

/* Release the index and everything it allocated.  NULL is a no-op. */
void mips_free_index(mips_index_t idx);

/* Thread-local message describing the last failed call ("" if none). */
const char* mips_last_error(void);

/* Library version, major * 10000 + minor * 100 + patch. */
int mips_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MIPS_H_ */
