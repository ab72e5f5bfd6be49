// forest.cu -- host side of the BDL-tree library: the log structure
// (Sec. III-D), the planner of Insert_L (Alg. 3) and Erase_L (Alg. 4), device
// memory, and the C ABI declared in include/bdl.h.
//
// Readings of the paper that the planner implements (same as the serial
// oracle, written independently):
//  * buffer overflow (Sec. IV-B1): the pool is the buffer's ids (ascending)
//    followed by the batch; the last (b + n) mod X pool entries become the new
//    buffer, the first q*X (q = floor((b + n) / X)) feed the new trees;
//  * F_new = F + q; every cleared tree (in F, not in F_new) merges into the
//    smallest new tree above it, and new tree j takes cap_j minus the
//    capacities of its cleared trees from the pool, new trees in increasing j;
//  * after an erase batch, trees with live < X*2^i / 2 are emptied and their
//    live points reinserted in ascending id order, keeping their ids.
#include "bdl_internal.cuh"

#include <algorithm>
#include <cstring>
#include <mutex>

namespace bdl {

std::atomic<uint64_t> g_launches{0};
static thread_local std::string g_err;

const char *const kKernelNames[kKernelCount] = {
    "k_gather_cleared",
    "k_gather_pool",
    "k_level_hist",
    "k_level_bucket",
    "k_level_collect",
    "k_level_select",
    "k_level_partition",
    "k_subtree",
    "k_box_up",
    "k_pool_tail",
    "k_sort_small",
    "k_append_validate",
    "k_set_alive",
    "k_iota",
    "k_erase_mark",
    "k_bloom_build",
    "k_erase_locate",
    "k_buffer_compact",
    "k_gather_roots",
    "k_mark_ids",
    "k_popc_blocks",
    "k_scan_bsum",
    "k_emit_ids",
    "k_knn",
    "k_pack_nodes",
    "k_qsort",
};

// ---- live per-kernel timing (CUDA events on the launching stream) ----
struct ProfRec {
  int kid;
  cudaEvent_t a, b;
};
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<ProfRec> g_prof;
static std::vector<cudaEvent_t> g_ev_free;

static cudaEvent_t take_event() {
  if (!g_ev_free.empty()) {
    cudaEvent_t e = g_ev_free.back();
    g_ev_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

KScope::KScope(int kid, cudaStream_t st) : rec(-1), s(st) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!g_prof_on) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  ProfRec r{kid, take_event(), take_event()};
  cudaEventRecord(r.a, s);
  g_prof.push_back(r);
  rec = (int)g_prof.size() - 1;
}

KScope::~KScope() {
  if (rec < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (rec < (int)g_prof.size()) cudaEventRecord(g_prof[rec].b, s);
}

static void prof_reset() {
  for (auto &r : g_prof) {
    g_ev_free.push_back(r.a);
    g_ev_free.push_back(r.b);
  }
  g_prof.clear();
}

int set_error(int status, const std::string &msg) {
  g_err = msg;
  return status;
}

int cuda_check(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return BDL_OK;
  cudaGetLastError();
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? BDL_ENOMEM : BDL_ECUDA;
}

static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[128];

static int get_pool(int dev, cudaMemPool_t *out) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (dev < 0 || dev >= 128) return set_error(BDL_EINVAL, "device index out of range");
  if (!g_pools[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p;
    int st = cuda_check(cudaMemPoolCreate(&p, &props), "cudaMemPoolCreate");
    if (st) return st;
    uint64_t thr = UINT64_MAX;   // keep freed memory cached in the pool
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr);
    g_pools[dev] = p;
  }
  *out = g_pools[dev];
  return BDL_OK;
}

int dev_alloc(bdl_forest *f, void **p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  if (bytes == 0) bytes = 256;
  if (f->cfg.hbm_budget_bytes > 0 && f->bytes_in_use + (int64_t)bytes > f->cfg.hbm_budget_bytes)
    return set_error(BDL_ENOMEM, "hbm budget exceeded");
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, f->pool, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return set_error(BDL_ENOMEM, std::string("device allocation failed: ") + cudaGetErrorString(e));
  }
  f->bytes_in_use += (int64_t)bytes;
  return BDL_OK;
}

void dev_free(bdl_forest *f, void *p, size_t bytes, cudaStream_t s) {
  if (!p) return;
  if (bytes == 0) bytes = 256;
  cudaFreeAsync(p, s);
  f->bytes_in_use -= (int64_t)bytes;
}

static size_t a256(size_t x) { return (x + 255) / 256 * 256; }

static void free_tree(bdl_forest *f, Tree *t, cudaStream_t s) {
  if (!t) return;
  dev_free(f, t->block, t->bytes, s);
  dev_free(f, t->bloom, t->bloom_bytes, s);
  delete t;
}

static int alloc_tree(bdl_forest *f, int level, int64_t size, cudaStream_t s, Tree **out) {
  Tree *t = new Tree();
  t->level = level;
  t->size = size;
  t->live = size;
  t->h = tree_height(size, f->cfg.leaf_size);
  t->nnodes = ((int64_t)2 << t->h) - 1;
  t->nleaves = (int64_t)1 << t->h;
  size_t b_pts = a256((size_t)rec_ints(f->dim) * size * 4),
         b_node = a256((size_t)t->nnodes * 16),
         b_box = a256((size_t)t->nnodes * 2 * f->dim * 4), b_live = a256((size_t)t->nnodes * 4),
         b_leaf = a256((size_t)(t->nleaves + 1) * 4),
         b_pk = a256((size_t)(t->nleaves - 1) * packed_node_ints(f->dim) * 4);
  t->bytes = b_pts + b_node + b_box + b_live + b_leaf + b_pk;
  int st = dev_alloc(f, &t->block, t->bytes, s);
  if (st) {
    delete t;
    return st;
  }
  char *p = (char *)t->block;
  t->pts = (int32_t *)p; p += b_pts;
  t->node = (Node *)p; p += b_node;
  t->box = (int32_t *)p; p += b_box;
  t->live_nodes = (int32_t *)p; p += b_live;
  t->leaf_off = (int32_t *)p; p += b_leaf;
  t->pk = (int32_t *)p;
  // unwritten nodes read as leaf 0 (children -1, -1): never outside the arrays
  cudaMemsetAsync(t->node, 0xff, (size_t)t->nnodes * 16, s);
  *out = t;
  return BDL_OK;
}

ForestView forest_view(const bdl_forest *f) {
  ForestView v;
  memset(&v, 0, sizeof(v));
  v.dim = f->dim;
  v.idtab = f->idtab;
  v.buf = f->buf;
  v.nbuf = f->nbuf;
  v.err = f->err;
  int n = 0;
  for (int i = kMaxLevel - 1; i >= 0; --i) {
    const Tree *t = f->trees[i];
    if (!t) continue;
    TreeView &tv = v.tree[n++];
    tv.pts = t->pts;
    tv.node = t->node;
    tv.box = t->box;
    tv.live = t->live_nodes;
    tv.leaf_off = t->leaf_off;
    tv.bloom = t->bloom;
    tv.pk = t->pk;
    tv.bloom_blocks = t->bloom_blocks;
    tv.size = t->size;
    tv.nnodes = t->nnodes;
    tv.h = t->h;
    tv.level = t->level;
  }
  v.ntrees = n;
  return v;
}

// Make the forest's device current for the duration of a call.
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

static int sync_read(bdl_forest *f, const int64_t *dev, int64_t n, cudaStream_t s) {
  int st = cuda_check(cudaMemcpyAsync(f->pinned, dev, (size_t)n * 8, cudaMemcpyDeviceToHost, s),
                      "cudaMemcpyAsync");
  if (st) return st;
  return cuda_check(cudaStreamSynchronize(s), "cudaStreamSynchronize");
}

static int ensure_id_capacity(bdl_forest *f, int64_t need, cudaStream_t s) {
  if (need <= f->id_cap) return BDL_OK;
  int64_t cap = std::max<int64_t>(f->id_cap, 1024);
  while (cap < need) cap *= 2;
  cap = (cap + 31) / 32 * 32;
  void *tab = nullptr, *alv = nullptr;
  int st = dev_alloc(f, &tab, (size_t)cap * f->dim * 4, s);
  if (st) return st;
  st = dev_alloc(f, &alv, (size_t)cap / 8, s);
  if (st) {
    dev_free(f, tab, (size_t)cap * f->dim * 4, s);
    return st;
  }
  cudaMemsetAsync(alv, 0, (size_t)cap / 8, s);
  if (f->id_cap) {
    cudaMemcpyAsync(tab, f->idtab, (size_t)f->next_id * f->dim * 4, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(alv, f->alive, (size_t)(f->next_id + 31) / 32 * 4, cudaMemcpyDeviceToDevice, s);
    dev_free(f, f->idtab, (size_t)f->id_cap * f->dim * 4, s);
    dev_free(f, f->alive, (size_t)f->id_cap / 8, s);
  }
  f->idtab = (int32_t *)tab;
  f->alive = (uint32_t *)alv;
  f->id_cap = cap;
  return cuda_check(cudaGetLastError(), "id table growth");
}

// Insert_L (Alg. 3) of the pool = sorted buffer ++ P, with n = |P|.
static int insert_pool(bdl_forest *f, const int32_t *arr, int64_t first, int64_t n, cudaStream_t s) {
  if (n == 0) return BDL_OK;
  const int64_t X = f->cfg.buffer_size;
  const int64_t t = f->nbuf + n, q = t / X, rem = t % X;
  PoolSrc pool{f->buf, f->nbuf, arr, first};
  if (q == 0) {
    // everything fits in the buffer
    launch_pool_tail(pool, f->nbuf, n, f->buf + f->nbuf, s);
    if (arr) launch_sort_small(f->buf, t, s);
    f->nbuf = t;
    f->buf_dirty = true;
    return cuda_check(cudaGetLastError(), "buffer append");
  }
  const uint64_t Fnew = f->F + (uint64_t)q;
  const uint64_t newt = Fnew & ~f->F, cleared = f->F & ~Fnew;
  if (Fnew >> kMaxLevel) return set_error(BDL_EINVAL, "forest too large");

  std::vector<BuildTree> bt;
  std::vector<ClearedSrc> cl;
  std::vector<int64_t> pool_lo, from_cleared;
  int64_t pos = 0;
  int prev = -1;
  int st = BDL_OK;
  for (int j = 0; j < kMaxLevel && !st; ++j) {
    if (!((newt >> j) & 1)) continue;
    int64_t capsum = 0, livesum = 0;
    for (int i = prev + 1; i < j; ++i) {
      if (!((cleared >> i) & 1)) continue;
      Tree *ct = f->trees[i];
      capsum += X << i;
      livesum += ct->live;
      cl.push_back(ClearedSrc{ct->pts, ct->size, (int32_t)bt.size()});
    }
    int64_t shortfall = (X << j) - capsum;
    Tree *nt = nullptr;
    st = alloc_tree(f, j, livesum + shortfall, s, &nt);
    if (st) break;
    bt.push_back(BuildTree{nt, 0, livesum + shortfall, nt->h, 0});
    pool_lo.push_back(pos);
    from_cleared.push_back(livesum);
    pos += shortfall;
    prev = j;
  }
  void *newbuf = nullptr;
  if (!st) st = dev_alloc(f, &newbuf, (size_t)X * 4, s);
  if (!st && pos != q * X) st = set_error(BDL_EINTERNAL, "planner: pool split mismatch");
  if (!st) {
    pool_lo.push_back(pos);
    st = build_trees(f, bt, cl, pool, pool_lo, from_cleared, s);
  }
  if (st) {
    for (auto &b : bt) free_tree(f, b.tree, s);
    dev_free(f, newbuf, (size_t)X * 4, s);
    return st;
  }
  launch_pool_tail(pool, q * X, rem, (int32_t *)newbuf, s);
  if (arr && rem > 1) launch_sort_small((int32_t *)newbuf, rem, s);
  for (int i = 0; i < kMaxLevel; ++i)
    if ((cleared >> i) & 1) {
      free_tree(f, f->trees[i], s);
      f->trees[i] = nullptr;
    }
  for (auto &b : bt) f->trees[b.tree->level] = b.tree;
  dev_free(f, f->buf, (size_t)X * 4, s);
  f->buf = (int32_t *)newbuf;
  f->nbuf = rem;
  f->buf_dirty = true;
  f->F = Fnew;
  return cuda_check(cudaGetLastError(), "insert");
}

ForestView knn_view(bdl_forest *f, bool build, cudaStream_t s) {
  // the buffer's points get a small kd-tree of their own (the paper's buffer
  // tree), rebuilt when the buffer changed; without it they are scanned
  if (build && f->buf_dirty) {
    free_tree(f, f->btree, s);
    f->btree = nullptr;
    if (f->nbuf > 0) {
      Tree *bt = nullptr;
      if (alloc_tree(f, kMaxLevel, f->nbuf, s, &bt) == BDL_OK) {
        std::vector<BuildTree> b{BuildTree{bt, 0, f->nbuf, bt->h, 0}};
        PoolSrc pool{f->buf, f->nbuf, nullptr, 0};
        if (build_trees(f, b, {}, pool, {0, f->nbuf}, {0}, s) == BDL_OK) f->btree = bt;
        else free_tree(f, bt, s);
      }
    }
    f->buf_dirty = false;
  }
  ForestView fv = forest_view(f);
  if (f->btree && !f->buf_dirty && fv.ntrees < kMaxLevel) {
    TreeView &tv = fv.tree[fv.ntrees++];
    const Tree *t = f->btree;
    memset(&tv, 0, sizeof(tv));
    tv.pts = t->pts;
    tv.node = t->node;
    tv.box = t->box;
    tv.live = t->live_nodes;
    tv.leaf_off = t->leaf_off;
    tv.pk = t->pk;
    tv.size = t->size;
    tv.nnodes = t->nnodes;
    tv.h = t->h;
    tv.level = t->level;
    fv.nbuf = 0;
  }
  return fv;
}

// With BDL_DEBUG_CHECK=1 every call waits for its kernels and fails with
// BDL_EINTERNAL if one of them recorded an out-of-range index.
static int finish(bdl_forest *f, cudaStream_t s, int st) {
  if (st || !f->debug_check) return st;
  st = cuda_check(cudaMemcpyAsync(f->pinned + 500, f->err, 8, cudaMemcpyDeviceToHost, s), "copy");
  if (!st) st = cuda_check(cudaStreamSynchronize(s), "sync");
  if (st) return st;
  if (f->pinned[500])
    return set_error(BDL_EINTERNAL, "device bounds check failed, code " + std::to_string(f->pinned[500]));
  return BDL_OK;
}

int finish_call(bdl_forest *f, cudaStream_t s, int st) { return finish(f, s, st); }

static int check_config(const bdl_config &c) {
  if (c.leaf_size < 2 || c.leaf_size > 64) return set_error(BDL_EINVAL, "leaf_size must be in 2..64");
  if (c.buffer_size < 2 || c.buffer_size > 16384)
    return set_error(BDL_EINVAL, "buffer_size must be in 2..16384");
  if (c.bloom_bits_per_key < 1 || c.bloom_bits_per_key > 64)
    return set_error(BDL_EINVAL, "bloom_bits_per_key must be in 1..64");
  if (c.bloom_hashes != 8) return set_error(BDL_EINVAL, "bloom_hashes must be 8");
  if (c.hbm_budget_bytes < 0) return set_error(BDL_EINVAL, "hbm_budget_bytes must be >= 0");
  return BDL_OK;
}

}  // namespace bdl

using namespace bdl;

extern "C" {

void bdl_default_config(bdl_config *cfg) {
  if (!cfg) return;
  cfg->leaf_size = 16;
  cfg->buffer_size = 1024;
  cfg->bloom_bits_per_key = 16;
  cfg->bloom_hashes = 8;
  cfg->hash_seed = 0x5EED;
  cfg->hbm_budget_bytes = 0;
}

const char *bdl_status_string(int st) {
  switch (st) {
    case BDL_OK: return "ok";
    case BDL_EINVAL: return "invalid argument";
    case BDL_ENOMEM: return "out of device memory or over the hbm budget";
    case BDL_ECUDA: return "CUDA error";
    case BDL_ETIMEOUT: return "device wait timed out";
    case BDL_EINTERNAL: return "internal error";
    default: return "unknown status";
  }
}

const char *bdl_last_error(void) { return g_err.c_str(); }

uint64_t bdl_launch_count(void) { return g_launches.load(); }

int bdl_profile(int enable) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  prof_reset();
  g_prof_on = enable != 0;
  return BDL_OK;
}

int bdl_profile_read(double *ms, int64_t *launches, int cap) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (int i = 0; i < cap && i < kKernelCount; ++i) {
    if (ms) ms[i] = 0;
    if (launches) launches[i] = 0;
  }
  for (auto &r : g_prof) {
    int st = cuda_check(cudaEventSynchronize(r.b), "cudaEventSynchronize");
    if (st) return st;
    float t = 0;
    st = cuda_check(cudaEventElapsedTime(&t, r.a, r.b), "cudaEventElapsedTime");
    if (st) return st;
    if (r.kid < cap) {
      if (ms) ms[r.kid] += t;
      if (launches) launches[r.kid] += 1;
    }
  }
  prof_reset();
  return BDL_OK;
}

int bdl_kernel_count(void) { return kKernelCount; }

const char *bdl_kernel_name(int id) { return id >= 0 && id < kKernelCount ? kKernelNames[id] : ""; }

int bdl_insert(bdl_forest *f, const int32_t *pts, int64_t n, int32_t *out_ids, bdl_stream_t stream) {
  if (!f) return set_error(BDL_EINVAL, "forest is NULL");
  if (n < 0) return set_error(BDL_EINVAL, "n < 0");
  if (n == 0) return BDL_OK;
  if (!pts) return set_error(BDL_EINVAL, "pts is NULL");
  if (f->next_id + n > (int64_t)INT32_MAX) return set_error(BDL_EINVAL, "id space (2^31 - 1) exhausted");
  cudaStream_t s = (cudaStream_t)stream;
  DeviceGuard g(f->device);
  int st = ensure_id_capacity(f, f->next_id + n, s);
  if (st) return st;
  cudaMemsetAsync(f->dev_small, 0, 8, s);
  launch_append_validate(pts, n, f->dim, f->idtab + f->next_id * f->dim, f->dev_small, s);
  st = sync_read(f, f->dev_small, 1, s);
  if (st) return st;
  if (f->pinned[0]) return set_error(BDL_EINVAL, "coordinate outside [0, 2^20)");
  const int64_t first = f->next_id;
  st = insert_pool(f, nullptr, first, n, s);
  if (st) return st;
  launch_set_alive(f->alive, first, n, s);
  launch_iota(out_ids, first, n, s);
  f->next_id += n;
  f->live += n;
  return finish(f, s, cuda_check(cudaGetLastError(), "insert"));
}

int bdl_create(int dim, const bdl_config *cfg, const int32_t *pts, int64_t n, int32_t *out_ids,
               bdl_stream_t stream, bdl_forest **out) {
  if (!out) return set_error(BDL_EINVAL, "out is NULL");
  *out = nullptr;
  if (dim < 1 || dim > kMaxDim) return set_error(BDL_EINVAL, "dim must be in 1..16");
  bdl_config c;
  bdl_default_config(&c);
  if (cfg) c = *cfg;
  int st = check_config(c);
  if (st) return st;
  bdl_forest *f = new bdl_forest();
  f->dim = dim;
  f->cfg = c;
  cudaStream_t s = (cudaStream_t)stream;
  st = cuda_check(cudaGetDevice(&f->device), "cudaGetDevice");
  if (!st) st = get_pool(f->device, &f->pool);
  if (!st) st = cuda_check(cudaMallocHost((void **)&f->pinned, 4096), "cudaMallocHost");
  void *small = nullptr;
  if (!st) st = dev_alloc(f, &small, 4096, s);
  f->dev_small = (int64_t *)small;
  if (!st) {
    f->err = (unsigned long long *)(f->dev_small + 256);
    cudaMemsetAsync(small, 0, 4096, s);
    const char *dbg = getenv("BDL_DEBUG_CHECK");
    f->debug_check = dbg && dbg[0] == '1';
  }
  void *buf = nullptr;
  if (!st) st = dev_alloc(f, &buf, (size_t)c.buffer_size * 4, s);
  f->buf = (int32_t *)buf;
  if (!st) st = ensure_id_capacity(f, std::max<int64_t>(n, 1024), s);
  if (!st && n > 0) st = bdl_insert(f, pts, n, out_ids, stream);
  if (st) {
    std::string keep = g_err;
    bdl_destroy(f);
    g_err = keep;
    return st;
  }
  *out = f;
  return BDL_OK;
}

int bdl_erase(bdl_forest *f, const int32_t *ids, int64_t n, int64_t *out_n, bdl_stream_t stream) {
  if (out_n) *out_n = 0;
  if (!f) return set_error(BDL_EINVAL, "forest is NULL");
  if (n < 0) return set_error(BDL_EINVAL, "n < 0");
  if (n == 0 || f->next_id == 0) return BDL_OK;
  if (!ids) return set_error(BDL_EINVAL, "ids is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  DeviceGuard g(f->device);
  void *list = nullptr;
  int st = dev_alloc(f, &list, (size_t)n * 4, s);
  if (st) return st;
  // 1. dedup against the live set
  cudaMemsetAsync(f->dev_small, 0, 8, s);
  launch_erase_mark(f->alive, f->next_id, ids, n, (int32_t *)list, f->dev_small, s);
  st = sync_read(f, f->dev_small, 1, s);
  if (st) { dev_free(f, list, (size_t)n * 4, s); return st; }
  const int64_t ne = f->pinned[0];
  if (out_n) *out_n = ne;
  if (ne == 0) {
    dev_free(f, list, (size_t)n * 4, s);
    return BDL_OK;
  }
  f->live -= ne;
  // 2. lazily build the bloom filter of every nonempty tree (Sec. V-A)
  for (int i = 0; i < kMaxLevel && !st; ++i) {
    Tree *t = f->trees[i];
    if (!t || t->live == 0 || t->bloom) continue;
    int64_t need = (t->size * f->cfg.bloom_bits_per_key + 255) / 256, blocks = 1;
    while (blocks < need) blocks *= 2;
    void *b = nullptr;
    st = dev_alloc(f, &b, (size_t)blocks * 32, s);
    if (st) break;
    t->bloom = (uint32_t *)b;
    t->bloom_blocks = blocks;
    t->bloom_bytes = (size_t)blocks * 32;
    cudaMemsetAsync(t->bloom, 0, t->bloom_bytes, s);
    launch_bloom_build(t, f->dim, f->cfg.hash_seed, s);
  }
  if (st) { dev_free(f, list, (size_t)n * 4, s); return st; }
  // 3. probe, descend, tombstone (Alg. 2 per tree, all trees in one launch);
  //    large batches descend in spatial order so neighbouring threads share paths
  ForestView fv = forest_view(f);
  const int32_t *order = (const int32_t *)list;
  void *sorted = nullptr;
  size_t sorted_bytes = 0;
  if (ne >= kSortMinQueries) {
    sorted_bytes = a256((size_t)ne * 4) + query_sort_bytes(ne, f->dim);
    if (dev_alloc(f, &sorted, sorted_bytes, s) == BDL_OK) {
      launch_point_sort(f->idtab, (const int32_t *)list, ne, f->dim,
                        (char *)sorted + a256((size_t)ne * 4), (int32_t *)sorted, s);
      order = (const int32_t *)sorted;
    } else {
      sorted = nullptr;   // same result in input order
    }
  }
  launch_erase_locate(fv, f->cfg.hash_seed, order, ne, s);
  if (sorted) dev_free(f, sorted, sorted_bytes, s);
  for (int i = 0; i < kMaxLevel; ++i)   // live counts changed: refresh the k-NN records
    if (f->trees[i]) launch_pack_lives(f->trees[i], f->dim, s);
  // 4. the buffer
  launch_buffer_compact(f->buf, f->nbuf, f->alive, f->dev_small, s);
  launch_gather_roots(fv, f->dev_small + 1, s);
  st = sync_read(f, f->dev_small, 1 + fv.ntrees, s);
  dev_free(f, list, (size_t)n * 4, s);
  if (st) return st;
  if (f->pinned[0] != f->nbuf) f->buf_dirty = true;
  f->nbuf = f->pinned[0];
  for (int j = 0; j < fv.ntrees; ++j) f->trees[fv.tree[j].level]->live = f->pinned[1 + j];
  // 5. trees below half capacity (Alg. 4 lines 3-4)
  std::vector<Tree *> low;
  int64_t nr = 0;
  for (int i = 0; i < kMaxLevel; ++i) {
    Tree *t = f->trees[i];
    if (t && 2 * t->live < ((int64_t)f->cfg.buffer_size << i)) {
      low.push_back(t);
      nr += t->live;
    }
  }
  if (low.empty()) return finish(f, s, cuda_check(cudaGetLastError(), "erase"));
  void *R = nullptr;
  st = dev_alloc(f, &R, (size_t)std::max<int64_t>(nr, 1) * 4, s);
  if (!st) st = collect_sorted_live(f, low, nr, (int32_t *)R, s);
  if (st) {
    dev_free(f, R, (size_t)std::max<int64_t>(nr, 1) * 4, s);
    return st;
  }
  uint64_t Fsave = f->F;
  Tree *saved[kMaxLevel];
  memcpy(saved, f->trees, sizeof(saved));
  for (Tree *t : low) {
    f->trees[t->level] = nullptr;
    f->F &= ~((uint64_t)1 << t->level);
  }
  st = insert_pool(f, (const int32_t *)R, 0, nr, s);
  if (st) {
    // reinsertion failed: keep the emptied trees where they were (still exact)
    f->F = Fsave;
    memcpy(f->trees, saved, sizeof(saved));
  } else {
    for (Tree *t : low) free_tree(f, t, s);
  }
  dev_free(f, R, (size_t)std::max<int64_t>(nr, 1) * 4, s);
  if (st) return st;
  return finish(f, s, cuda_check(cudaGetLastError(), "erase"));
}

int bdl_knn(bdl_forest *f, const int32_t *q, int64_t m, int k, int32_t *out_ids, int64_t *out_d2,
            bdl_stream_t stream) {
  if (!f) return set_error(BDL_EINVAL, "forest is NULL");
  if (k < 1 || k > kMaxK) return set_error(BDL_EINVAL, "k must be in 1..32");
  if (m < 0) return set_error(BDL_EINVAL, "m < 0");
  if (m == 0) return BDL_OK;
  if (!q || !out_ids || !out_d2) return set_error(BDL_EINVAL, "NULL pointer");
  DeviceGuard g(f->device);
  cudaStream_t s = (cudaStream_t)stream;
  ForestView fv = knn_view(f, true, s);
  // large batches run in spatial order so that neighbouring threads walk
  // neighbouring paths; results are written back in input order
  void *scratch = nullptr;
  size_t sbytes = 0;
  int32_t *perm = nullptr;
  if (m >= kSortMinQueries) {
    sbytes = query_sort_bytes(m, f->dim);
    if (dev_alloc(f, &scratch, sbytes, s) == BDL_OK) {
      perm = (int32_t *)scratch;
      launch_query_sort(q, m, f->dim, (char *)scratch + ((size_t)m * 4 + 255) / 256 * 256, perm, s);
    } else {
      scratch = nullptr;   // fall back to input order (same results)
    }
  }
  int st = launch_knn(fv, q, perm, m, k, out_ids, out_d2, f->knn_stats, s);
  if (scratch) dev_free(f, scratch, sbytes, s);
  return finish(f, s, st);
}

int bdl_size(const bdl_forest *f, int64_t *out) {
  if (!f || !out) return set_error(BDL_EINVAL, "NULL pointer");
  *out = f->live;
  return BDL_OK;
}

int bdl_destroy(bdl_forest *f) {
  if (!f) return BDL_OK;
  DeviceGuard g(f->device);
  cudaDeviceSynchronize();
  cudaStream_t s = 0;
  for (int i = 0; i < kMaxLevel; ++i) free_tree(f, f->trees[i], s);
  free_tree(f, f->btree, s);
  if (f->id_cap) {
    dev_free(f, f->idtab, (size_t)f->id_cap * f->dim * 4, s);
    dev_free(f, f->alive, (size_t)f->id_cap / 8, s);
  }
  dev_free(f, f->buf, (size_t)f->cfg.buffer_size * 4, s);
  dev_free(f, f->dev_small, 4096, s);
  if (f->knn_stats) dev_free(f, f->knn_stats, 64, s);
  cudaStreamSynchronize(s);
  if (f->pinned) cudaFreeHost(f->pinned);
  delete f;
  return cuda_check(cudaGetLastError(), "destroy");
}

int bdl_tree_mask(const bdl_forest *f, uint64_t *mask, int64_t *nbuf) {
  if (!f) return set_error(BDL_EINVAL, "forest is NULL");
  if (mask) *mask = f->F;
  if (nbuf) *nbuf = f->nbuf;
  return BDL_OK;
}

int bdl_buffer_ids(const bdl_forest *f, int32_t *out, int64_t cap, int64_t *out_n, bdl_stream_t stream) {
  if (!f) return set_error(BDL_EINVAL, "forest is NULL");
  if (out_n) *out_n = f->nbuf;
  int64_t n = std::min(cap, f->nbuf);
  if (n <= 0 || !out) return BDL_OK;
  DeviceGuard g(f->device);
  cudaStream_t s = (cudaStream_t)stream;
  int st = cuda_check(cudaMemcpyAsync(out, f->buf, (size_t)n * 4, cudaMemcpyDeviceToHost, s), "copy");
  if (st) return st;
  return cuda_check(cudaStreamSynchronize(s), "sync");
}

int bdl_tree_info(const bdl_forest *f, int level, int64_t *info) {
  if (!f || !info) return set_error(BDL_EINVAL, "NULL pointer");
  if (level < 0 || level >= kMaxLevel || !f->trees[level]) return set_error(BDL_EINVAL, "empty tree");
  const Tree *t = f->trees[level];
  info[0] = t->size;
  info[1] = t->live;
  info[2] = t->h;
  info[3] = t->nnodes;
  info[4] = t->bloom ? t->bloom_blocks : 0;
  info[5] = t->level;
  return BDL_OK;
}

int bdl_tree_export(const bdl_forest *f, int level, int64_t *key, int32_t *child, int32_t *box,
                    int32_t *live, int32_t *leaf_off, int32_t *ids, bdl_stream_t stream) {
  if (!f) return set_error(BDL_EINVAL, "forest is NULL");
  if (level < 0 || level >= kMaxLevel || !f->trees[level]) return set_error(BDL_EINVAL, "empty tree");
  const Tree *t = f->trees[level];
  DeviceGuard g(f->device);
  cudaStream_t s = (cudaStream_t)stream;
  int st = BDL_OK;
  auto cp = [&](void *dst, const void *src, size_t bytes) {
    if (dst && !st) st = cuda_check(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s), "copy");
  };
  std::vector<Node> nodes;
  if ((key || child) && !st) {
    nodes.resize((size_t)t->nnodes);
    cp(nodes.data(), t->node, nodes.size() * sizeof(Node));
  }
  cp(box, t->box, (size_t)t->nnodes * 2 * f->dim * 4);
  cp(live, t->live_nodes, (size_t)t->nnodes * 4);
  cp(leaf_off, t->leaf_off, (size_t)(t->nleaves + 1) * 4);
  std::vector<int32_t> recs;
  const int rs = rec_ints(f->dim);
  if (ids && !st) {
    recs.resize((size_t)t->size * rs);
    cp(recs.data(), t->pts, recs.size() * 4);
  }
  if (st) return st;
  st = cuda_check(cudaStreamSynchronize(s), "sync");
  if (!st && ids)
    for (int64_t j = 0; j < t->size; ++j) ids[j] = recs[(size_t)j * rs + f->dim];
  if (!st && (key || child))
    for (int64_t v = 0; v < t->nnodes; ++v) {
      if (key) key[v] = (int64_t)nodes[(size_t)v].key;
      if (child) { child[2 * v] = nodes[(size_t)v].l; child[2 * v + 1] = nodes[(size_t)v].r; }
    }
  return st;
}

int bdl_bloom_export(const bdl_forest *f, int level, uint32_t *words, bdl_stream_t stream) {
  if (!f || !words) return set_error(BDL_EINVAL, "NULL pointer");
  if (level < 0 || level >= kMaxLevel || !f->trees[level] || !f->trees[level]->bloom)
    return set_error(BDL_EINVAL, "no bloom filter");
  const Tree *t = f->trees[level];
  DeviceGuard g(f->device);
  cudaStream_t s = (cudaStream_t)stream;
  int st = cuda_check(cudaMemcpyAsync(words, t->bloom, t->bloom_bytes, cudaMemcpyDeviceToHost, s), "copy");
  if (st) return st;
  return cuda_check(cudaStreamSynchronize(s), "sync");
}

int bdl_knn_stats(bdl_forest *f, int enable, int64_t *out) {
  if (!f) return set_error(BDL_EINVAL, "forest is NULL");
  DeviceGuard g(f->device);
  if (out) {
    if (f->knn_stats) {
      unsigned long long h[3];
      int st = cuda_check(cudaMemcpy(h, f->knn_stats, sizeof(h), cudaMemcpyDeviceToHost), "copy");
      if (st) return st;
      for (int i = 0; i < 3; ++i) out[i] = (int64_t)h[i];
    } else {
      out[0] = out[1] = out[2] = 0;
    }
    return BDL_OK;
  }
  if (enable && !f->knn_stats) {
    void *p = nullptr;
    int st = dev_alloc(f, &p, 64, 0);
    if (st) return st;
    f->knn_stats = (unsigned long long *)p;
  }
  if (!enable && f->knn_stats) {
    cudaDeviceSynchronize();
    dev_free(f, f->knn_stats, 64, 0);
    f->knn_stats = nullptr;
    return cuda_check(cudaDeviceSynchronize(), "sync");
  }
  if (f->knn_stats) {
    int st = cuda_check(cudaMemset(f->knn_stats, 0, 64), "memset");
    if (st) return st;
  }
  return cuda_check(cudaDeviceSynchronize(), "sync");
}

}  // extern "C"
