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
} bdl_config;

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
 * leaves the forest unchanged.  Synchronises `stream` once (validation). */
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

/* Number of live points (host-side count, no device access). */
int bdl_size(const bdl_forest *f, int64_t *out_live_host);

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

/* Totals over every bdl_knn call of this forest since the last reset when
 * counting is on: out[0] = tree nodes visited, out[1] = leaf points examined,
 * out[2] = queries.  bdl_knn_stats(f, 1/0, NULL) switches counting on/off and
 * resets; counting adds atomics and is meant for measurement runs only. */
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

/* Kernel ids are 0 .. bdl_kernel_count()-1; bdl_kernel_name gives each one's
 * name (e.g. "k_knn"). */
int bdl_kernel_count(void);
const char *bdl_kernel_name(int id);

#ifdef __cplusplus
}
#endif

#endif /* BDL_H */
