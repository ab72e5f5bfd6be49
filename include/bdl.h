/*
 * bdl.h -- C ABI of the GB300 (sm_103a) BDL-tree: a batch-dynamic forest of
 * static kd-trees after Yesantharao, Wang, Dhulipala & Shun, "Parallel
 * Batch-Dynamic kd-Trees" (arXiv 2112.06188).
 *
 * The library keeps the log-structured set of static kd-trees (Sec. III-D)
 * resident in device memory and exposes the three batch operations of the
 * paper -- Insert_L (Alg. 3), Erase_L (Alg. 4) and kNN_L (Alg. 5) -- plus
 * construction (Alg. 1 applied to the first batch).  Every step runs in CUDA
 * kernels; there is no CPU fallback.
 *
 * Conventions shared by every entry point
 *  - Points are int32 coordinates on the grid [0, 2^20), `dim` per point,
 *    row-major [n][dim].  Squared distances are exact int64; ties are broken
 *    by point id, so results are deterministic.
 *  - Ids are int32, assigned 0, 1, 2, ... in insertion order across
 *    bdl_create and bdl_insert; at most 2^31 - 1 ids per forest.
 *  - Data pointers marked _dev are device pointers owned by the caller; the
 *    library only reads inputs and writes outputs through them.  Results are
 *    valid once `stream` has completed.  Pointers marked _host are host memory.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  All work
 *    of a call is ordered on it; calls that need a count back from the device
 *    (insert validation, erase) synchronise it before they return.
 *  - Calls on one forest must not overlap (serialise them on one stream or
 *    one thread).  Distinct forests are independent.
 *  - Every function returns a bdl_status.  On BDL_EINVAL and BDL_ENOMEM the
 *    forest is left as it was, except where a function says otherwise.
 *    bdl_last_error() describes the last failure of the calling thread.
 *  - Device memory of the forest comes from a CUDA stream-ordered memory pool
 *    owned by the library (one per device), optionally capped per forest by
 *    bdl_config.hbm_budget_bytes.
 *  - Kernels check their indexes: one that finds an index outside its buffers
 *    skips the access and sets a bit in the forest's device error word (1 child
 *    slot, 2 leaf range, 4 traversal stack, 8 partition, 16 gather, 32 a packed
 *    k-NN record's live count differs from its node's).  bdl_insert and
 *    bdl_erase read the word at the waits they make and return BDL_EINTERNAL
 *    when a bit is set, with the bits in bdl_last_error(); bdl_poll_error reads
 *    it on demand.  With the environment variable BDL_DEBUG_CHECK=1 (read at
 *    bdl_create) every call also waits for its own kernels and checks the word.
 *  - Builds: the on-chip subtrees run one CTA per SM; a build gives trees with
 *    fewer global levels than its deepest tree extra ones when that shortens
 *    an estimated schedule of the subtree CTAs on the device's SMs
 *    (BDL_BUILD_SLOTS=n, read at every build, schedules on n slots instead).
 *    The trees are the same either way.
 *  - Memory: without an hbm budget, static trees are laid out for their
 *    level's capacity X*2^level and each level keeps the block of its last
 *    cleared tree for the level's next tree (no allocation per carry); those
 *    blocks stay the forest's until bdl_destroy.  With a budget, trees take
 *    exactly their size and nothing is kept.
 */
#ifndef BDL_H
#define BDL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bdl_forest bdl_forest;        /* opaque, library-owned */
typedef struct CUstream_st *bdl_stream_t;    /* same type as cudaStream_t */

typedef enum {
    BDL_OK = 0,
    BDL_EINVAL = 1,     /* bad argument: dim, sizes, k, coordinates, ids */
    BDL_ENOMEM = 2,     /* device allocation failed or hbm budget exceeded */
    BDL_ECUDA = 3,      /* a CUDA runtime call failed (message in bdl_last_error) */
    BDL_ETIMEOUT = 4,   /* a bounded device wait gave up */
    BDL_EINTERNAL = 5   /* an internal consistency check failed */
} bdl_status;

typedef struct {
    int32_t leaf_size;          /* L: points per leaf, 2..64; default 16 (Sec. V-D) */
    int32_t buffer_size;        /* X: buffer capacity and tree unit, 2..16384;
                                   default 1024 (Sec. V-D); tree i holds up to X*2^i */
    int32_t bloom_bits_per_key; /* bloom filter size, 1..64 bits per point; default 16 (Sec. V-A) */
    int32_t bloom_hashes;       /* bits set per key; must be 8 (split-block filter) */
    uint64_t hash_seed;         /* bloom hash seed; default 0x5EED */
    int64_t hbm_budget_bytes;   /* cap on the forest's device memory; 0 = none */
    int32_t split_rule;         /* BDL_SPLIT_OBJECT (default): split at the median point
                                   (Alg. 1); BDL_SPLIT_SPATIAL: split at the midpoint of the
                                   points' extent, v = floor((min + max) / 2), coordinates <= v
                                   to the left (Sec. V-C).  k-NN results are the same. */
    int32_t reserved_;          /* 0 */
} bdl_config;

enum { BDL_SPLIT_OBJECT = 0, BDL_SPLIT_SPATIAL = 1 };

/* Fill *cfg with the defaults above. */
void bdl_default_config(bdl_config *cfg);

/* Construction (Sec. IV-B1 with F = 0, i.e. Alg. 1 on the trees Alg. 3 plans):
 * a new forest of `dim`-dimensional points (1 <= dim <= 16) holding the n
 * points pts_dev[n][dim] (n may be 0), with ids 0..n-1 written to
 * out_ids_dev[n] when it is not NULL.  cfg NULL = defaults.  On success
 * *out is the new forest (free it with bdl_destroy); on failure *out = NULL. */
int bdl_create(int dim, const bdl_config *cfg, const int32_t *pts_dev, int64_t n,
               int32_t *out_ids_dev, bdl_stream_t stream, bdl_forest **out);

/* Insert_L (Alg. 3): add the n points pts_dev[n][dim]; their ids (next
 * consecutive ids) go to out_ids_dev[n] when it is not NULL.  The buffer takes
 * the overflow (Sec. IV-B1), trees are merged by binary-counter carry
 * F_new = F + (b + n) / X and the new trees are rebuilt with median splits in
 * vEB layout (Alg. 1).  A coordinate outside [0, 2^20) gives BDL_EINVAL and
 * leaves the forest unchanged.  Waits once, before returning, for the
 * validation of the coordinates (the new trees are built meanwhile on grid-
 * clamped values and installed only if every coordinate was on the grid). */
int bdl_insert(bdl_forest *f, const int32_t *pts_dev, int64_t n, int32_t *out_ids_dev,
               bdl_stream_t stream);

/* Erase_L (Alg. 4): erase the points whose ids are in ids_dev[n].  Ids that
 * are not live (never inserted, already erased, negative, repeated in the
 * batch) are ignored; *out_n_erased_host (may be NULL) receives the number of
 * points erased.  Each nonempty tree is filtered by its bloom filter (built
 * lazily, Sec. V-A); matches are tombstoned (Alg. 2); trees left below half
 * of their capacity X*2^i are emptied and their points reinserted through
 * Insert_L with their ids kept.  Synchronises `stream`.  If the reinsertion
 * cannot get memory the erase itself stays applied, the affected trees stay
 * in place (still exact for queries) and BDL_ENOMEM is returned. */
int bdl_erase(bdl_forest *f, const int32_t *ids_dev, int64_t n, int64_t *out_n_erased_host,
              bdl_stream_t stream);

/* kNN_L (Alg. 5): for each of the m queries q_dev[m][dim] the k nearest
 * live points, 1 <= k <= 32.  Query coordinates must lie on the grid
 * [0, 2^20) like the points (the query path does no device-to-host check;
 * rows of other queries are unspecified).  Row i of
 * out_ids_dev[m][k] / out_d2_dev[m][k] lists them by increasing (squared
 * distance, id); when fewer than k points are live the row is padded with
 * id -1 and d2 INT64_MAX.  A query equal to a live point returns it at d2 0.
 * Trees are searched largest first (Sec. V-B), then the buffer. */
int bdl_knn(bdl_forest *f, const int32_t *q_dev, int64_t m, int k, int32_t *out_ids_dev,
            int64_t *out_d2_dev, bdl_stream_t stream);

/* kNN_L like bdl_knn, for callers that cannot allocate device memory while
 * they query: for example a process whose free device memory is already held
 * by another allocator, so that a new allocation would fail, or a request
 * path that must not wait on a memory pool.  bdl_knn takes scratch for the
 * query ordering from the library's pool, and it may rebuild the buffer's
 * kd-tree.  This call does neither.  (The paper has no counterpart; it is an
 * interface choice of this library.)
 *  - Scratch lives in one fixed device array of 8 MiB + 4 KiB that every GPU
 *    loading the library holds until the process exits.
 *  - m is at most 1,048,576; larger batches return BDL_EINVAL.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  - Every call shares the one array and leaves its contents behind: calls
 *    whose work can overlap on the GPU (other streams, other forests on the
 *    same device) race with each other and must be ordered by the caller.
 *  - If the buffer changed since the last bdl_knn, its points are scanned
 *    instead of searched; results are the same as bdl_knn's. */
int bdl_knn_noalloc(bdl_forest *f, const int32_t *q_dev, int64_t m, int k, int32_t *out_ids_dev,
                    int64_t *out_d2_dev, bdl_stream_t stream);

/* Launch shape of f's k-NN kernel (a tuning knob of this library; the paper's
 * kNN_L, Alg. 5, has none): block_threads in {64, 128, 256} (0 = the default
 * 128; a block is halved while its k top-k slots per thread, 12 bytes each,
 * would pass 48 KB of shared memory) and queries_per_warp in {32, 64, 128}
 * (0 = the default 32): each warp answers that many consecutive queries in
 * the order the call processes them, 32 at a time.  Used by bdl_knn,
 * bdl_knn_noalloc, bdl_knn_count, and by the batched calls and plans whose
 * forests[0] is f (a plan keeps the shape it was made with).  Results do not
 * depend on the shape.  Other values: BDL_EINVAL, shape unchanged.  Host
 * only; no device work. */
int bdl_set_knn_shape(bdl_forest *f, int block_threads, int queries_per_warp);

/* ---------------------------------------------------------------------
 * Batched forests: one call runs the same operation on nf independent
 * forests (nf >= 0) of possibly different sizes, sharing kernel launches and
 * host synchronisations instead of issuing nf separate calls.  Forest i gets
 * exactly the result the single-forest call on it would give.  The arrays
 * (forests, per-forest pointers, sizes) are host arrays of length nf; the
 * pointers in them are device pointers as in the single-forest calls.  All
 * forests must live on the same device and (insert, erase) be distinct.
 * Forests of different dimensions may be mixed (one launch per dimension).
 * (The paper treats one forest; batching many is an interface choice of
 * this library.)
 * --------------------------------------------------------------------- */

/* bdl_insert on every forest i with pts_dev[i][n[i]][dim_i] and
 * out_ids_dev[i] (NULL entries allowed).  All or nothing: on BDL_EINVAL (a
 * coordinate off the grid anywhere, a bad size, a repeated forest) or
 * BDL_ENOMEM no forest changes.  Synchronises `stream` once. */
int bdl_insert_batch(bdl_forest *const *forests, int nf, const int32_t *const *pts_dev,
                     const int64_t *n, int32_t *const *out_ids_dev, bdl_stream_t stream);

/* bdl_erase on every forest i with ids_dev[i][n[i]]; out_n_erased_host[i]
 * (array may be NULL) receives forest i's count.  Argument errors change no
 * forest; a failed reinsertion behaves as in bdl_erase for the forests it
 * hits and the call returns the first such status. */
int bdl_erase_batch(bdl_forest *const *forests, int nf, const int32_t *const *ids_dev,
                    const int64_t *n, int64_t *out_n_erased_host, bdl_stream_t stream);

/* bdl_knn on every forest i with q_dev[i][m[i]][dim_i] into
 * out_ids_dev[i][m[i]][k] / out_d2_dev[i][m[i]][k]; one k for all.  A forest
 * may appear more than once. */
int bdl_knn_batch(bdl_forest *const *forests, int nf, const int32_t *const *q_dev, const int64_t *m,
                  int k, int32_t *const *out_ids_dev, int64_t *const *out_d2_dev,
                  bdl_stream_t stream);

/* A prepared kNN_L over forests[nf] (a forest may appear more than once):
 * the job tables and the query-ordering scratch are made once, in device
 * memory the plan owns (charged to forests[0]), so that
 * bdl_knn_plan_launch issues kernels and memsets only -- on any stream,
 * inside a CUDA graph capture too.  Every launch answers the queries that
 * q_dev[i] holds when it runs (contents may change between launches, the
 * pointers and sizes may not) against the forests as they were when the
 * plan was made; a launch after an insert or erase on any of them returns
 * BDL_EINVAL and launches nothing.  (A captured graph replays without that
 * check: do not replay it after changing the forests.)  Results equal
 * bdl_knn_batch's.  Destroy the plan before its forests. */
typedef struct bdl_knn_plan bdl_knn_plan;
int bdl_knn_plan_create(bdl_forest *const *forests, int nf, const int32_t *const *q_dev,
                        const int64_t *m, int k, int32_t *const *out_ids_dev,
                        int64_t *const *out_d2_dev, bdl_stream_t stream, bdl_knn_plan **out);
int bdl_knn_plan_launch(bdl_knn_plan *plan, bdl_stream_t stream);
/* Waits for the device, then frees the plan's memory.  NULL is a no-op. */
int bdl_knn_plan_destroy(bdl_knn_plan *plan);

/* ---------------------------------------------------------------------
 * Serving: a request server that keeps one forest resident and takes
 * insert / erase / k-NN requests from host memory as they arrive.
 * Requests take effect in submission order with exactly the results the
 * plain calls give when issued one by one in that order; the server batches
 * them for the device as they arrive (continuous batching):
 *  - consecutive k-NN requests go out as one k-NN launch: with one k up to
 *    max_group_queries queries, with different k up to 32,768 queries in all
 *    (launched with the largest k, each request's rows cut to its own k --
 *    the k nearest by (d2, id) are the first k of the larger list);
 *  - consecutive inserts go out as one Insert_L of their concatenated points
 *    (same ids, same live set);
 *  - consecutive erases go out as one Erase_L of all their ids, marked
 *    request by request in order, so that each request's count is the number
 *    of its ids that were live after the erases before it (an id named twice
 *    counts for the first request).
 * A request is admitted -- its device buffers allocated and its input
 * copied in -- only while fewer than max_inflight requests are in flight and
 * their buffers fit in staging_budget_bytes; inputs of later requests and
 * outputs of earlier ones are copied while the current group computes (use
 * pinned host buffers for that overlap).  The forest's own memory stays
 * capped by its bdl_config.hbm_budget_bytes.  While a server is alive the
 * caller must not use its forest directly.  (The paper has no serving layer;
 * this interface is a choice of this library.)
 * --------------------------------------------------------------------- */

typedef struct bdl_server bdl_server;        /* opaque, library-owned */

typedef enum { BDL_REQ_INSERT = 0, BDL_REQ_ERASE = 1, BDL_REQ_KNN = 2 } bdl_request_kind;

typedef struct {
    int32_t kind;               /* bdl_request_kind */
    int32_t k;                  /* k-NN: 1..32 */
    int64_t n;                  /* points, ids or queries */
    const int32_t *in_host;     /* insert: [n][dim] points; erase: [n] ids; k-NN: [n][dim]
                                   queries.  Read until the request completes. */
    int32_t *out_ids_host;      /* insert: [n] new ids (may be NULL); k-NN: [n][k] */
    int64_t *out_d2_host;       /* k-NN: [n][k] */
} bdl_request;

typedef struct {
    int32_t status;             /* bdl_status of the request */
    int32_t kind;
    int32_t done;               /* 1 once completed */
    int32_t pad_;
    uint64_t ticket;
    int64_t n_done;             /* insert: points inserted; erase: points erased; k-NN: queries */
    int64_t group;              /* index of the device group it ran in */
    double t_submit_ms;         /* host clock, ms since the server was created */
    double t_start_ms;          /* its group started on the host */
    double t_done_ms;           /* its outputs were in host memory */
} bdl_result;

typedef struct {
    int32_t max_inflight;       /* admitted, not completed; default 64 */
    int32_t serial;             /* 1 = one request at a time, no batching (comparison path) */
    int64_t staging_budget_bytes; /* device bytes of the requests in flight; default 1 GiB */
    int64_t max_group_queries;  /* k-NN queries per launch; default 2^20 */
    int64_t max_group_points;   /* points per merged insert, ids per merged erase; default 2^21 */
} bdl_server_config;

/* Fill *cfg with the defaults above. */
void bdl_server_default_config(bdl_server_config *cfg);

/* Start a server on forest f (cfg NULL = defaults); it runs host threads of
 * its own and three CUDA streams on f's device. */
int bdl_server_create(bdl_forest *f, const bdl_server_config *cfg, bdl_server **out);

/* Queue a request (never blocks on the device); *out_ticket identifies it.
 * The request struct is copied; the buffers it points to are not. */
int bdl_server_submit(bdl_server *s, const bdl_request *req, uint64_t *out_ticket);

/* Wait for a request to complete and collect its result (once per ticket). */
int bdl_server_wait(bdl_server *s, uint64_t ticket, bdl_result *out_host);

/* Wait until every submitted request has completed. */
int bdl_server_drain(bdl_server *s);

/* The server's clock: ms since it was created (the clock of bdl_result's
 * timestamps). */
double bdl_server_now_ms(const bdl_server *s);

/* Device groups run so far. */
int bdl_server_stats(const bdl_server *s, int64_t *out_groups_host);

/* Finish every submitted request, stop the threads and free the server (not
 * the forest).  NULL is a no-op. */
int bdl_server_destroy(bdl_server *s);

/* Number of live points (host-side count, no device access). */
int bdl_size(const bdl_forest *f, int64_t *out_live_host);

/* The id the next inserted point will get, i.e. the number of ids assigned
 * so far (host-side value, no device access).  After a successful insert of
 * n points the ids were next_id - n .. next_id - 1. */
int bdl_next_id(const bdl_forest *f, int64_t *out_next_id_host);

/* Free the forest and all its device memory (waits for its pending work).
 * NULL is a no-op. */
int bdl_destroy(bdl_forest *f);

/* Static description of a status code. */
const char *bdl_status_string(int status);

/* Description of the last failure on the calling thread ("" if none). */
const char *bdl_last_error(void);

/* ---------------------------------------------------------------------
 * Introspection (tests, benchmarks).  All outputs are host memory; these
 * calls synchronise `stream`.
 * --------------------------------------------------------------------- */

/* Bitmask F of the nonempty static trees (bit i = tree of capacity X*2^i)
 * and the number of points in the buffer. */
int bdl_tree_mask(const bdl_forest *f, uint64_t *out_mask_host, int64_t *out_buffer_n_host);

/* The buffer's ids (ascending), at most `cap` of them; *out_n = count. */
int bdl_buffer_ids(const bdl_forest *f, int32_t *out_ids_host, int64_t cap, int64_t *out_n_host,
                   bdl_stream_t stream);

/* info[0..5] = stored points, live points, split levels h, node count
 * 2^(h+1)-1, bloom blocks (0 if not built), level.  BDL_EINVAL if tree
 * `level` is empty. */
int bdl_tree_info(const bdl_forest *f, int level, int64_t *info_host);

/* Copy tree `level` to the host.  Nodes are in vEB order (Alg. 1):
 *   key[nn]        split key (coordinate << 31 | id) of internal nodes, 0 for leaves
 *   child[nn][2]   vEB slots of the left/right child; leaves: (-1 - leaf index, 0)
 *   box[nn][2*dim] lo[dim], hi[dim] of the points below the node
 *   live[nn]       live points below the node
 *   leaf_off[2^h + 1] point range of each leaf (leaf index = position at depth h)
 *   ids[size]      point ids in leaf order; an erased point is stored as id | 0x80000000
 * Any pointer may be NULL. */
int bdl_tree_export(const bdl_forest *f, int level, int64_t *key_host, int32_t *child_host,
                    int32_t *box_host, int32_t *live_host, int32_t *leaf_off_host,
                    int32_t *ids_host, bdl_stream_t stream);

/* The bloom filter words of tree `level` (blocks * 8 uint32, see
 * bdl_tree_info); BDL_EINVAL if it has not been built. */
int bdl_bloom_export(const bdl_forest *f, int level, uint32_t *words_host, bdl_stream_t stream);

/* kNN_L like bdl_knn, run by the counting instance of the kernel (a plain
 * one-lane walk of the binary nodes with the same pruning rule, Alg. 5 /
 * Sec. IV-A3), which returns the same rows and adds, with device atomics,
 * the tree nodes it visits to counts_dev[0], the live leaf points it examines
 * to counts_dev[1] and the queries to counts_dev[2].  counts_dev is a device
 * array of three uint64 (8-byte aligned) owned by the caller, who zeroes it;
 * nothing is waited for.  Measurement only: these counts give the
 * algorithmic bytes of a k-NN launch (4d + 12k per query, 32 per node, one
 * record per leaf point).  Under profiling its launches are reported as
 * "k_knn_count", apart from the timed instance "k_knn". */
int bdl_knn_count(bdl_forest *f, const int32_t *q_dev, int64_t m, int k, int32_t *out_ids_dev,
                  int64_t *out_d2_dev, uint64_t *counts_dev, bdl_stream_t stream);

/* Wait for `stream` and read the forest's device error word (bit codes as
 * in the conventions above) into *out_bits_host (may be NULL): BDL_OK if no
 * bit is set, else BDL_EINTERNAL.  The word is sticky.  bdl_insert and
 * bdl_erase read it at the waits they make anyway (insert: the word as it
 * stood before the call's own kernels; erase: after them) and fail with
 * BDL_EINTERNAL when it is set; this call is the poll for k-NN callers, whose
 * calls never wait. */
int bdl_poll_error(const bdl_forest *f, uint64_t *out_bits_host, bdl_stream_t stream);

/* Totals over every bdl_knn call of this forest since the last reset when
 * counting is on: out[0] = tree nodes visited, out[1] = leaf points examined,
 * out[2] = queries.  bdl_knn_stats(f, 1/0, NULL) switches counting on/off and
 * resets.  While counting is on, k-NN runs a counting instance of the kernel
 * (the same rows, from a plain one-lane walk of the binary nodes, with
 * atomics): meant for measurement runs only. */
int bdl_knn_stats(bdl_forest *f, int enable, int64_t *out_host);

/* Number of kernels this library has launched in the process. */
uint64_t bdl_launch_count(void);

/* Live per-kernel timing for measurement runs: while enabled, every kernel
 * launch is bracketed by CUDA events on its own stream.  bdl_profile(1/0)
 * switches it on/off and clears the records; bdl_profile_read waits for the
 * recorded events and fills, per kernel id < cap, the summed device time in
 * ms and the launch count since the last call, then clears the records. */
int bdl_profile(int enable);
int bdl_profile_read(double *ms_host, int64_t *launches_host, int cap);
/* bdl_profile_read plus, per kernel, the summed algorithmic bytes of the
 * recorded launches (bytes_host may be NULL): the least DRAM traffic the
 * launch's work implies, computed by the library from the sizes it knows when
 * it launches (records per level, ids, points), for the roofline fraction
 * achieved = bytes / time.  Per record of d coordinates: the global build
 * levels' histogram and candidate passes read its split coordinate (4 B) and
 * the partition reads and writes it ((d + 1) words each way); the on-chip
 * subtree build reads it from staging and writes it in leaf order, plus every
 * node below the global levels (16-byte node, 2d-word box, live count) and
 * the leaf offsets; per erased id (batch length): 4d for its coordinates, a
 * 32-byte bloom block per tree and a descent (16 B per level and the leaf's
 * records) of a tree chosen in proportion to the trees' sizes; per bloom key
 * 4 + 32.  Kernels without a stated figure (k_knn among them: its bytes come
 * from bdl_knn_count) report 0. */
int bdl_profile_read_bytes(double *ms_host, int64_t *launches_host, double *bytes_host, int cap);

/* The recorded launches since profiling was switched on or last read, in
 * launch order (a trace, for finding the gaps between kernels): per launch i <
 * cap its kernel id, the device times of its start and end events in ms from
 * the first recorded launch's start (launches on several streams share that
 * origin), and its algorithmic bytes.  *out_n = launches recorded.  Waits
 * for the events; does not clear the records (bdl_profile_read does). */
int bdl_profile_timeline(int32_t *kid_host, double *start_ms_host, double *end_ms_host, double *bytes_host,
                         int cap, int *out_n_host);

/* Kernel ids are 0 .. bdl_kernel_count()-1; bdl_kernel_name gives each one's
 * name (e.g. "k_knn"). */
int bdl_kernel_count(void);
const char *bdl_kernel_name(int id);

#ifdef __cplusplus
}
#endif

#endif /* BDL_H */
