// bdl_internal.cuh -- types and device helpers shared by the CUDA translation
// units of the BDL-tree library (forest.cu, build.cu, erase.cu, knn.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/bdl.h"

namespace bdl {

constexpr int kMaxDim = 16;
constexpr int kMaxLevel = 40;          // trees 0..39; ids < 2^31 keep us far below
constexpr int kMaxK = 32;
constexpr int kCoordBits = 20;         // grid [0, 2^20)
constexpr int kKeyBits = 51;           // composite key: coord << 31 | id
constexpr uint32_t kTomb = 0x80000000u;  // erased point: id | kTomb (negative int32)
constexpr int kHistBins = 2048;        // 11-bit digit of the global median search
constexpr int kHistShift = kCoordBits - 11;

extern std::atomic<uint64_t> g_launches;

// Every kernel launch of the library goes through a KScope: it counts the
// launch and, while profiling is on, brackets it with CUDA events on the
// launching stream so per-kernel device times can be read back, together
// with the launch's algorithmic bytes (the minimum DRAM traffic its work
// implies, computed from the sizes the host knows at launch; 0 where not
// stated).
enum KernelId : int {
  kK_build_levels,
  kK_subtree,
  kK_build_finish,
  kK_sort_small,
  kK_erase_mark,
  kK_bloom_build,
  kK_erase_locate,
  kK_buffer_compact,
  kK_mark_ids,
  kK_popc_blocks,
  kK_scan_bsum,
  kK_emit_ids,
  kK_knn,
  kK_pack_nodes,
  kK_qsort,
  kK_fill,
  kK_pack_lives,
  kK_put_blob,
  kK_sp_gather,
  kK_sp_minmax,
  kK_sp_scatter,
  kK_sp_split,
  kK_sp_box,
  kK_knn_count,
  kK_small_copy,
  kKernelCount
};
extern const char *const kKernelNames[kKernelCount];
struct KScope {
  KScope(int kid, cudaStream_t s, double bytes = 0);
  ~KScope();
  int rec;
  cudaStream_t s;
};

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------

// Composite split key in one dimension (coordinate, ties by id): Sec. IV-A1
// needs a strict order so that every node splits its points exactly in half.
__host__ __device__ inline uint64_t comp_key(int32_t coord, int32_t id) {
  return ((uint64_t)(uint32_t)coord << 31) | (uint64_t)(uint32_t)id;
}

// Smallest power of two >= l/2: levels of the bottom part of a vEB split.
__host__ __device__ inline int veb_bottom(int l) {
  int lb = 1;
  while (2 * lb < l) lb *= 2;
  return lb;
}

// Slot of node (depth t, index i at that depth) in the vEB layout of a
// complete tree with l levels (Alg. 1): the top l_t levels come first, then
// the 2^l_t bottom trees of l_b levels, each laid out recursively.
__host__ __device__ inline int64_t veb_slot(int l, int t, int64_t i) {
  int64_t off = 0;
  while (l > 1) {
    int lb = veb_bottom(l);
    int lt = l - lb;
    if (t < lt) {
      l = lt;
    } else {
      int tt = t - lt;
      int64_t j = i >> tt;
      off += (((int64_t)1 << lt) - 1) + j * (((int64_t)1 << lb) - 1);
      i &= ((int64_t)1 << tt) - 1;
      t = tt;
      l = lb;
    }
  }
  return off;
}

// Point range of segment `idx` at depth t of a tree over s points, where every
// split gives the left child ceil(m/2) points.  O(t).
__host__ __device__ inline void seg_range(int64_t s, int t, int64_t idx, int64_t &start,
                                          int64_t &size) {
  start = 0;
  size = s;
  for (int u = t - 1; u >= 0; --u) {
    int64_t l = (size + 1) >> 1;
    if ((idx >> u) & 1) {
      start += l;
      size -= l;
    } else {
      size = l;
    }
  }
}

// Segment at depth t that holds position p (0 <= p < s).  O(t).
__host__ __device__ inline int64_t seg_of(int64_t s, int t, int64_t p, int64_t &start,
                                          int64_t &size) {
  start = 0;
  size = s;
  int64_t idx = 0;
  for (int u = 0; u < t; ++u) {
    int64_t l = (size + 1) >> 1;
    if (p < start + l) {
      size = l;
      idx = 2 * idx;
    } else {
      start += l;
      size -= l;
      idx = 2 * idx + 1;
    }
  }
  return idx;
}

// Split levels of a tree over s points with leaves of at most L points:
// h = ceil(log2(ceil(s / L))).
__host__ __device__ inline int tree_height(int64_t s, int L) {
  int64_t nl = (s + L - 1) / L;
  int h = 0;
  while (((int64_t)1 << h) < nl) h++;
  return h;
}

// SplitMix64 output function (Steele, Lea & Flood 2014) applied to x.
__host__ __device__ inline uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Split-block bloom filter position of an id: block and one bit per word.
__host__ __device__ inline void bloom_hash(uint64_t seed, int64_t blocks, int32_t id,
                                           int64_t &blk, uint64_t &bits) {
  uint64_t h1 = splitmix64(seed ^ (uint64_t)(uint32_t)id);
  bits = splitmix64(h1);
  blk = (int64_t)(h1 & (uint64_t)(blocks - 1));
}

__device__ inline uint32_t bloom_word_bit(uint64_t bits, int w) {
  return 1u << ((bits >> (5 * w)) & 31u);
}

// ---------------------------------------------------------------------------
// device views
// ---------------------------------------------------------------------------

// One tree node (16 bytes, one sector per visit): the split key of an
// internal node and the slots of its children; a leaf has key 0 and
// l = -1 - (leaf index), r = 0.
struct __align__(16) Node {
  uint64_t key;
  int32_t l, r;
};

// Ints of one point record in a tree: dim coordinates, the id, padding to a
// multiple of 16 bytes (so a 3-D point is one int4: x, y, z, id).
__host__ __device__ constexpr int rec_ints(int dim) { return (dim + 1 + 3) / 4 * 4; }

// Packed k-NN node records.  A tree with h internal levels has one record
// for the root and one for every internal node at a depth t with h - t even
// (t > 0); a record describes its node's four descendants two levels down
// (the root of an odd h: its two children), each an internal node that has a
// record of its own or a leaf.  Ints of a record: the four entries' codes
// (record slot, or -1 - leaf index), their live counts, then per coordinate
// c the four entries' low bounds and the four high bounds, so that one
// 16-byte load gives one bound of every entry.  32-byte aligned for every dim.
__host__ __device__ constexpr int packed_node_ints(int dim) { return 8 + 8 * dim; }

__host__ __device__ inline int64_t quad_count(int H) {   // (4^H - 1) / 3 nodes in H 4-ary levels
  return (((int64_t)1 << (2 * H)) - 1) / 3;
}

// Position of node (level u, index i) in the vEB order of a complete 4-ary
// tree of H levels, split into top and bottom levels as veb_slot does.
__host__ __device__ inline int64_t veb4_slot(int H, int u, int64_t i) {
  int64_t off = 0;
  while (H > 1) {
    const int Hb = veb_bottom(H);
    const int Ht = H - Hb;
    if (u < Ht) {
      H = Ht;
    } else {
      const int uu = u - Ht;
      const int64_t j = i >> (2 * uu);
      off += quad_count(Ht) + j * quad_count(Hb);
      i &= ((int64_t)1 << (2 * uu)) - 1;
      u = uu;
      H = Hb;
    }
  }
  return off;
}

// Records of a tree with h internal levels.
__host__ __device__ inline int64_t packed_nrec(int h) {
  if (h <= 0) return 0;
  if (h & 1) return 1 + 2 * quad_count((h - 1) / 2);
  return quad_count(h / 2);
}

// Levels from the record of a node at depth t down to its entries.
__host__ __device__ inline int packed_step(int h, int t) { return ((h & 1) && t == 0) ? 1 : 2; }

// Slot of the record of the node at depth t, index i.  Even h: the records
// form one complete 4-ary tree, in vEB order.  Odd h: the root's record, then
// the 4-ary trees under its two children, each in vEB order.
__host__ __device__ inline int64_t packed_slot(int h, int t, int64_t i) {
  if (!(h & 1)) return veb4_slot(h / 2, t / 2, i);
  if (t == 0) return 0;
  const int64_t sub = i >> (t - 1), il = i & (((int64_t)1 << (t - 1)) - 1);
  return 1 + sub * quad_count((h - 1) / 2) + veb4_slot((h - 1) / 2, (t - 1) / 2, il);
}

// The g-th record in level order: depth t and index i of its node.
__host__ __device__ inline void packed_record_of(int h, int64_t g, int &t, int64_t &i) {
  const int odd = h & 1;
  if (odd && g == 0) {
    t = 0;
    i = 0;
    return;
  }
  int64_t y = odd ? g - 1 : g;
  int u = 0;
  while (y >= ((int64_t)(1 + odd) << (2 * u))) {   // 2 * 4^u (odd h) or 4^u nodes on level u
    y -= (int64_t)(1 + odd) << (2 * u);
    ++u;
  }
  t = 2 * u + odd;
  i = y;
}

struct TreeView {          // one static tree, device pointers
  int32_t *pts;            // [size][rec_ints(dim)]: coordinates, id (erased: id | kTomb)
  const Node *node;        // [nnodes]
  const int32_t *box;      // [nnodes][2*dim]
  int32_t *live;           // [nnodes]
  const int32_t *leaf_off; // [2^h + 1]
  const uint32_t *bloom;   // [blocks * 8] or nullptr
  int32_t *pk;             // packed k-NN node records (packed_slot order)
  int64_t size;
  int64_t nnodes;
  int64_t bloom_blocks;
  int32_t h;
  int32_t level;
};

struct ForestView {        // what the k-NN and erase kernels see
  int ntrees;              // nonempty trees, largest first
  TreeView tree[kMaxLevel];
  const int32_t *idtab;    // [id][dim]
  const int32_t *buf;      // buffer ids
  int64_t nbuf;
  int dim;
  unsigned long long *err; // device error word (bit codes below), never null
};

// Device error codes: a kernel that finds an index outside its buffers
// records one of these bits and skips the access instead of faulting.
enum : unsigned long long {
  kErrChild = 1,       // child slot outside the node array
  kErrLeaf = 2,        // leaf range outside the point array
  kErrStack = 4,       // traversal stack full
  kErrPartition = 8,   // partition destination outside its segment
  kErrGather = 16,     // gather destination outside its tree
  kErrLiveCount = 32,  // a packed record's live count differs from its node's (debug check)
  kErrBarrier = 64,    // a grid barrier of a cooperative kernel waited too long and gave up
};

// Grid-wide barrier of a cooperative launch (every block resident at once):
// bar[0] counts the blocks that arrived, bar[1] is the generation the last
// arrival advances.  Writes before the barrier are visible after it (block
// barrier, then a device-scope fence by the arriving thread, cumulative over
// the block's writes, and another after the wait).  The wait is bounded:
// after kBarrierPolls polls (about a second) the block sets kErrBarrier in
// *err and goes on, so a lost block never hangs the GPU; the call then fails
// with BDL_EINTERNAL.
constexpr unsigned kBarrierPolls = 1u << 24;
__device__ __forceinline__ void grid_barrier(unsigned *bar, unsigned long long *err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned polls = 0;
      while (*gen == g) {
        if (++polls > kBarrierPolls) {
          atomicOr(err, kErrBarrier);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// host-side state
// ---------------------------------------------------------------------------

struct Tree {
  int level = 0;
  int64_t size = 0, live = 0;
  int h = 0;
  int64_t nnodes = 0, nleaves = 0;
  int64_t room = 0;        // points the arrays have room for (>= size)
  void *block = nullptr;   // one pool allocation holding the arrays below
  size_t bytes = 0;
  int32_t *pts = nullptr;      // [size][rec_ints(dim)] in leaf order
  int32_t *box = nullptr, *live_nodes = nullptr, *leaf_off = nullptr;
  Node *node = nullptr;        // [nnodes], vEB order
  int32_t *pk = nullptr;       // packed k-NN node records, packed_nrec(h) of them
  uint32_t *bloom = nullptr;   // the bloom filter once built (lazily), else nullptr
  uint32_t *bloom_room = nullptr;  // its place in the block (static trees)
  int64_t bloom_room_blocks = 0;
  int64_t bloom_blocks = 0;
  size_t bloom_bytes = 0;
};

// Where a pool of point ids comes from (Sec. IV-B1): the forest's sorted
// buffer ids, then either an explicit id array or a range of new ids.
struct PoolSrc {
  const int32_t *buf;      // sorted buffer ids (nbuf of them)
  int64_t nbuf;
  const int32_t *arr;      // explicit ids, or nullptr for a range
  int64_t first;           // first id of the range
};

// One tree to build: its outputs and where its input points come from --
// the live records of cleared trees (from_cleared of them, listed as
// ClearedSrc entries) followed by entries [pool_lo, pool_lo + s - from_cleared)
// of its forest's pool.  Trees of different forests can share one build.
struct BuildTree {
  Tree *tree;
  int64_t s;
  int h;
  int64_t from_cleared;
  PoolSrc pool;
  int64_t pool_lo;
  const int32_t *idtab;    // the forest's id table
  unsigned long long *err; // the forest's error word
  int64_t base = 0;        // set by build_trees: first staging position
  int g = 0;               // set by build_trees: levels split by the global kernels
};

struct Scratch;            // allocation helper (forest.cu)

// Launch shape of the k-NN kernels (results do not depend on it): threads
// per block (64, 128 or 256; halved while k slots per thread would pass 48 KB
// of shared memory) and queries per warp (32, 64 or 128: a warp answers that
// many consecutive queries of its job, 32 at a time).
struct KnnShape {
  int block = 128;
  int qpw = 32;
};
}  // namespace bdl

struct bdl_forest {
  int dim = 0;
  bdl_config cfg{};
  int device = 0;
  cudaMemPool_t pool = nullptr;
  int32_t *idtab = nullptr;      // [id_cap][dim]
  uint32_t *alive = nullptr;     // [id_cap / 32]
  int64_t id_cap = 0, next_id = 0;
  int32_t *buf = nullptr;        // [X] ascending ids
  int32_t *buf_spare = nullptr;  // [X] the previous buffer, reused as the next one
  int64_t nbuf = 0;
  bdl::Tree *trees[bdl::kMaxLevel] = {};
  bdl::Tree *btree = nullptr;    // kd-tree over the buffer's points (k-NN only), built lazily
  bool buf_dirty = true;         // the buffer changed since btree was built
  uint64_t F = 0;
  int64_t live = 0;              // host mirror of the live count
  int64_t bytes_in_use = 0;
  int64_t *pinned = nullptr;     // pinned host scratch [kPinnedWords]: [0, kPinnedFlags) insert
                                 // flags, [kPinnedErr] the error word
  int64_t *pinned_dev = nullptr; // its device address (mapped page-locked memory)
  int64_t *dev_small = nullptr;  // small device scratch for counts / flags
  unsigned long long *err = nullptr;  // device error word (inside dev_small)
  bool debug_check = false;      // BDL_DEBUG_CHECK=1: sync and check err after each call
  unsigned long long *knn_stats = nullptr;  // [3] device counters, or nullptr
  uint64_t version = 0;          // bumped by every change of the trees or the buffer
  cudaEvent_t ev_flags = nullptr;  // recorded behind the insert flags' copy
  bdl::KnnShape knn_shape;         // launch shape of its k-NN calls
  // per static-tree level: the block of the level's last cleared tree, kept
  // for its next tree (forests without an hbm budget; freed by bdl_destroy)
  struct SpareBlock {
    void *block = nullptr;
    size_t bytes = 0;
    int64_t room = 0;
  } spare[bdl::kMaxLevel];
};

namespace bdl {

// ---- forest.cu ----
int set_error(int status, const std::string &msg);
int cuda_check(cudaError_t e, const char *what);
int dev_alloc(bdl_forest *f, void **p, size_t bytes, cudaStream_t s);
void dev_free(bdl_forest *f, void *p, size_t bytes, cudaStream_t s);
// Copy a launch table from host memory (any kind) to 16-byte aligned device
// memory, ordered on `s`, without making the host wait for the stream; the
// source may be reused when this returns.  Legal while `s` is capturing.
int h2d(void *dst, const void *src, size_t bytes, cudaStream_t s);
// A small copy between device memory and page-locked host memory (which the
// device reaches directly, unified addressing), done by a kernel on `s`
// instead of a copy engine: the caller's own large transfers queued on the
// copy engines cannot delay it.
int small_copy(void *dst, const void *src, size_t bytes, cudaStream_t s);
// Zero a device buffer with a kernel (not a copy-engine memset), for the
// same reason.
int small_zero(void *dst, size_t bytes, cudaStream_t s);
// Page-locked host scratch for readbacks, from a pool (returned by
// pinned_put); nullptr if none can be had.
void *pinned_get(size_t bytes);
void pinned_put(void *p);
// The device address of mapped page-locked host memory (nullptr if none).
void *mapped(void *host);
ForestView forest_view(const bdl_forest *f);
// The view k-NN uses: the static trees plus the buffer's kd-tree.  With
// build = true a stale buffer tree is rebuilt first (this allocates); with
// build = false a stale one is left alone and the buffer is scanned instead.
ForestView knn_view(bdl_forest *f, bool build, cudaStream_t s);
// BDL_DEBUG_CHECK: wait for the call's kernels and report a bounds-check hit.
int finish_call(bdl_forest *f, cudaStream_t s, int status);
constexpr int64_t kSortMinQueries = 1 << 15;   // smaller batches run in input order ...
constexpr int64_t kBatchSortMinQueries = 1 << 12;   // ... unless a batched call's small jobs
                                                   // hold this many queries together
constexpr size_t kPinnedWords = 2048;          // a forest's pinned scratch, in int64 words
constexpr size_t kPinnedFlags = 2040;          // insert-validation flags that fit in it
constexpr size_t kPinnedErr = 2044;            // where the error word is read back
constexpr int kBufOutWords = kMaxLevel + 2;    // per forest: buffer size, root live counts, error word
int smem_subtree_capacity(int dim);

// Erase_L on one forest for several id lists in order (the server's merged
// erase requests): an id counts for the first list that names it, so
// counts[r] is what list r would erase in a call of its own after the lists
// before it.  One bloom build, descent launch and wait for all of them.
int erase_lists(bdl_forest *f, const std::vector<const int32_t *> &ids, const std::vector<int64_t> &n,
                int64_t *counts, cudaStream_t s);

// ---- build.cu ----
struct ClearedSrc {        // a cleared tree whose live points join a new tree
  const int32_t *pts;      // point records
  int64_t size;
  int32_t dst;             // index into the BuildTree list
};
// Gather the points of the new trees (of any number of forests with the same
// dim) into staging and build all of them in shared launches.  Scratch is
// charged to forest `af`.
// The object-median (Alg. 1, build.cu) and spatial-median (Sec. V-C,
// spatial.cu) builds; build_trees picks by af's splitting rule, and every
// tree in one call must come from forests with that rule.
int build_trees_object(bdl_forest *af, int dim, std::vector<BuildTree> &bt,
                       const std::vector<ClearedSrc> &cl, cudaStream_t s);
int build_trees_spatial(bdl_forest *af, int dim, std::vector<BuildTree> &bt,
                        const std::vector<ClearedSrc> &cl, cudaStream_t s);
int build_trees(bdl_forest *af, int dim, std::vector<BuildTree> &bt,
                const std::vector<ClearedSrc> &cl, cudaStream_t s);
// Sort each list (ids[n], n <= 16384) ascending, one CTA per list, in one
// launch; the list table goes to `table` (sort_small_table_bytes of device memory).
struct SortList {
  int32_t *ids;
  int32_t n, np2;
};
size_t sort_small_table_bytes(size_t nlists);
int launch_sort_small_many(const std::vector<SortList> &lists, void *table, cudaStream_t s);

// ---- erase.cu ----
// One forest's deduplicated erase list in an erase launch.
struct EraseCall {
  const ForestView *fv;
  const int32_t *list;     // ids to erase (each live, each once)
  int64_t n;
  uint64_t seed;           // the forest's bloom hash seed
  const int64_t *n_dev;    // if set: the list's length on the device (<= n)
  int records;             // 1: also keep the packed k-NN records' live counts current
};
struct EraseJob {          // device form of an EraseCall
  const TreeView *trees;
  int32_t ntrees, dim;
  const int32_t *idtab;
  unsigned long long *err;
  const int32_t *list;
  int64_t n;
  uint64_t seed;
  const int64_t *n_dev;
  int32_t records;
};
size_t erase_table_bytes(const std::vector<EraseCall> &calls);
// Bloom probe, descent and tombstone for every call in one launch; the job
// table goes to `table` (erase_table_bytes of device memory).
int launch_erase_jobs(const std::vector<EraseCall> &calls, void *table,
                      cudaStream_t s);
// The live ids of trees `trees` of forest f in increasing order, n of them,
// into out -- for many forests in shared launches.
struct LiveCollect {
  bdl_forest *f;
  std::vector<Tree *> trees;
  int64_t n;
  int32_t *out;
};
int collect_sorted_live(const std::vector<LiveCollect> &jobs, cudaStream_t s);

// Table-driven helpers (one launch for many forests or trees).
enum FillKind : int32_t { kFillAppend = 0, kFillPoolTail = 1, kFillIota = 2, kFillAlive = 3, kFillZero = 4 };
struct FillSeg {           // `count` work items of one kind
  int32_t kind, pad_;
  int64_t count;
  const int32_t *src;      // append: coordinates in
  int32_t *dst;            // append / pool tail / iota: out
  unsigned long long *flag;  // append: set to 1 on a coordinate off the grid
  const int32_t *buf;      // pool tail: the forest's pool ...
  int64_t nbuf;
  const int32_t *arr;
  int64_t first;           // pool tail: range start; iota / alive: first id
  int64_t from;            // pool tail: first pool entry copied
  uint32_t *alive;         // alive: the forest's bitmap
  const unsigned long long *errw;  // append: the forest's device error word; a set word
                                   // sets bit 1 of *flag and its bits from bit 8 on
};
struct MarkSeg {           // one erase list of one forest
  uint32_t *alive;
  int64_t next_id;
  const int32_t *ids;
  int64_t n;
  int32_t *list;           // out: owned ids
  int64_t *count;          // out: how many
  int64_t *total;          // out: the forest's count over all its lists (may alias count)
};
struct TreeSeg {           // one tree: bloom builds, record packing, live refreshes
  const int32_t *pts;
  int64_t size;
  int32_t dim, h;
  uint32_t *bloom;
  int64_t blocks;
  const Node *node;
  const int32_t *box;
  const int32_t *live;
  int32_t *pk;
  uint64_t seed;           // bloom hash seed (bloom builds)
  const int64_t *gate;     // bloom builds: skipped when *gate == 0 (nullptr: always built)
  unsigned long long *err; // live refreshes: compare and flag instead of write (debug check)
};
struct BufSeg {            // one forest's buffer and roots
  int32_t *buf;
  int64_t nbuf;
  const uint32_t *alive;
  int64_t *out;            // out[0] = new nbuf, out[1 + t] = live count of tree t,
                           // out[kMaxLevel + 1] = the forest's device error word
  const unsigned long long *errw;
  int32_t ntrees, pad_;
  const int32_t *roots[kMaxLevel];
};
size_t table_bytes(size_t nseg, size_t seg_size);
int launch_fill_many(const std::vector<FillSeg> &segs, void *table, cudaStream_t s);
int launch_erase_mark_many(const std::vector<MarkSeg> &segs, void *table, cudaStream_t s);
int launch_bloom_build_many(const std::vector<TreeSeg> &segs, void *table,
                            cudaStream_t s);
int launch_pack_lives_many(const std::vector<TreeSeg> &segs, void *table, cudaStream_t s);
int launch_buffer_compact_many(const std::vector<BufSeg> &segs, void *table, cudaStream_t s);

// ---- knn.cu ----
// One forest's query batch in a k-NN launch.
struct KnnCall {
  const ForestView *fv;
  const int32_t *q;        // [m][dim]
  const int32_t *perm;     // processing order, or nullptr
  int64_t m;
  int32_t *oi;             // [m][k]
  int64_t *od;
};
// Device form of a KnnCall (the kernel reads these from a table).
struct KnnJob {
  const TreeView *trees;
  int32_t ntrees, dim;
  const int32_t *idtab;
  const int32_t *buf;
  int64_t nbuf;
  unsigned long long *err;
  const int32_t *q;
  const int32_t *perm;
  int64_t m;
  int32_t *oi;
  int64_t *od;
};
// Device bytes the job table of `calls` needs (0 for a single call, whose job
// travels as kernel parameters; `table` may then be null).
size_t knn_table_bytes(const std::vector<KnnCall> &calls);
// The table path in two halves (prepared k-NN plans): upload the job table of
// `calls` (knn_table_bytes_always bytes at `table`; *warps = warps to launch),
// then launch it as often as wanted.
size_t knn_table_bytes_always(const std::vector<KnnCall> &calls);
int upload_knn_table(const std::vector<KnnCall> &calls, void *table, int64_t *warps, int qpw,
                     cudaStream_t s);
int launch_knn_table(const void *table, int njobs, int64_t warps, int dim, int k, const KnnShape &sh,
                     unsigned long long *stats, cudaStream_t s);
// k-NN for every call (all of dimension `dim`) in one launch; the job table
// is uploaded to `table` (knn_table_bytes of device memory) on stream s.
int launch_knn_jobs(const std::vector<KnnCall> &calls, int dim, int k, const KnnShape &sh, void *table,
                    unsigned long long *stats, cudaStream_t s);
// The packed k-NN records of many trees (Sec. V-B's per-node data, laid out
// for the query kernel): table entries and their work prefix ...
void pack_nodes_entries(const std::vector<Tree *> &trees, int dim, std::vector<TreeSeg> &segs,
                        std::vector<int64_t> &pre);
// ... and one launch over a device copy of them (pre[nseg] = total).
void launch_pack_nodes(const TreeSeg *segs, const int64_t *pre, int nseg, int64_t total, cudaStream_t s);
// Spatial order for the small jobs of a batched call (all of one dimension,
// perm unset): one counting sort over all their queries keyed by (job rank,
// Morton prefix), which sets each call's perm; scratch of
// batch_query_sort_bytes().  Does nothing for fewer than two jobs.
size_t batch_query_sort_bytes(const std::vector<KnnCall> &calls);
int batch_query_sort(std::vector<KnnCall> &calls, void *scratch, size_t bytes, cudaStream_t s);
// Spatial order of the queries (counting sort on a Morton prefix of their
// coordinates): perm[m] gets query indices; scratch of query_sort_bytes().
size_t query_sort_bytes(int64_t m, int dim);
void launch_query_sort(const int32_t *q, int64_t m, int dim, void *scratch, int32_t *perm,
                       cudaStream_t s);
// The same order for the points named by ids[m] (coordinates in coords):
// out[m] receives the ids themselves, reordered.  With m_dev, only the first
// min(*m_dev, m) ids are sorted (a count still on the device); out's tail past
// them is left as it was.
void launch_point_sort(const int32_t *coords, const int32_t *ids, int64_t m, int dim,
                       void *scratch, int32_t *out, cudaStream_t s,
                       const int64_t *m_dev = nullptr);

}  // namespace bdl

