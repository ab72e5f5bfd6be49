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
    "k_build_levels",
    "k_subtree",
    "k_build_finish",
    "k_sort_small",
    "k_erase_mark",
    "k_bloom_build",
    "k_erase_locate",
    "k_buffer_compact",
    "k_mark_ids",
    "k_popc_blocks",
    "k_scan_bsum",
    "k_emit_ids",
    "k_knn",
    "k_pack_nodes",
    "k_qsort",
    "k_fill",
    "k_pack_lives",
    "k_put_blob",
    "k_sp_gather",
    "k_sp_minmax",
    "k_sp_scatter",
    "k_sp_split",
    "k_sp_box",
    "k_knn_count",
    "k_small_copy",
};

// ---- live per-kernel timing (CUDA events on the launching stream) ----
struct ProfRec {
  int kid;
  cudaEvent_t a, b;
  double bytes;    // algorithmic bytes of the launch (0: not stated)
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

KScope::KScope(int kid, cudaStream_t st, double bytes) : rec(-1), s(st) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!g_prof_on) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  ProfRec r{kid, take_event(), take_event(), bytes};
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

// ---------------------------------------------------------------------------
// Host -> device copies of small launch tables
// ---------------------------------------------------------------------------
//
// A copy from pageable memory may make the host wait for the stream, and a
// stream that is being captured into a CUDA graph cannot take it at all.  So
// tables go through a pinned ring (one per device; a region is reused only
// after the event recorded behind its copy has completed), and while the
// stream is capturing they travel as kernel parameters instead, which the
// graph keeps by value.

namespace {

constexpr size_t kRingBytes = (size_t)16 << 20;
constexpr int kBlobWords = 1024;                      // 16 KB of parameters

struct Blob {
  uint4 w[kBlobWords];
};

__global__ void k_put_blob(const Blob b, unsigned char *dst, int bytes) {
  const int full = bytes / 16;
  uint4 *d = (uint4 *)dst;
  for (int i = threadIdx.x; i < full; i += blockDim.x) d[i] = b.w[i];
  const unsigned char *src = (const unsigned char *)b.w;
  for (int i = full * 16 + threadIdx.x; i < bytes; i += blockDim.x) dst[i] = src[i];
}

struct Ring {
  unsigned char *base = nullptr;
  unsigned char *dbase = nullptr;   // its device address
  size_t head = 0;
  struct Use {
    size_t off, len;
    cudaEvent_t ev;
  };
  std::vector<Use> busy;
  std::vector<cudaEvent_t> spare;
};
std::mutex g_ring_mu;
Ring g_ring[128];

}  // namespace

namespace {

// Word-wise copy between device-accessible buffers (8-byte words when both
// ends are 8-byte aligned, bytes otherwise).
__global__ void k_small_copy(const unsigned char *src, unsigned char *dst, size_t bytes) {
  const size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x, step = (size_t)gridDim.x * blockDim.x;
  if ((((uintptr_t)src | (uintptr_t)dst) & 7) == 0) {
    const size_t nw = bytes / 8;
    const uint64_t *s8 = (const uint64_t *)src;
    uint64_t *d8 = (uint64_t *)dst;
    for (size_t i = i0; i < nw; i += step) d8[i] = s8[i];
    for (size_t i = nw * 8 + i0; i < bytes; i += step) dst[i] = src[i];
  } else {
    for (size_t i = i0; i < bytes; i += step) dst[i] = src[i];
  }
}

// Zero fill of a device buffer (8-byte words when aligned).
__global__ void k_zero(unsigned char *dst, size_t bytes) {
  const size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x, step = (size_t)gridDim.x * blockDim.x;
  if (((uintptr_t)dst & 7) == 0) {
    const size_t nw = bytes / 8;
    uint64_t *d8 = (uint64_t *)dst;
    for (size_t i = i0; i < nw; i += step) d8[i] = 0;
    for (size_t i = nw * 8 + i0; i < bytes; i += step) dst[i] = 0;
  } else {
    for (size_t i = i0; i < bytes; i += step) dst[i] = 0;
  }
}

std::mutex g_pin_mu;
std::vector<std::pair<void *, size_t>> g_pin_free;   // page-locked buffers not in use
std::vector<std::pair<void *, size_t>> g_pin_used;

}  // namespace

// Page-locked, device-mapped host memory, and the address kernels use for it.
static int host_alloc_mapped(void **p, size_t bytes) {
  return cuda_check(cudaHostAlloc(p, bytes, cudaHostAllocMapped | cudaHostAllocPortable), "cudaHostAlloc");
}

void *mapped(void *host) {
  void *d = nullptr;
  if (cudaHostGetDevicePointer(&d, host, 0) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return d;
}

int small_copy(void *dst, const void *src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return BDL_OK;
  const size_t words = (bytes + 7) / 8;
  const unsigned blocks = (unsigned)std::min<size_t>((words + 255) / 256, 64);
  KScope ks_(kK_small_copy, s);
  k_small_copy<<<blocks, 256, 0, s>>>((const unsigned char *)src, (unsigned char *)dst, bytes);
  return cuda_check(cudaGetLastError(), "small copy");
}

int small_zero(void *dst, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return BDL_OK;
  const size_t words = (bytes + 7) / 8;
  const unsigned blocks = (unsigned)std::min<size_t>((words + 255) / 256, 2048);
  KScope ks_(kK_small_copy, s);
  k_zero<<<blocks, 256, 0, s>>>((unsigned char *)dst, bytes);
  return cuda_check(cudaGetLastError(), "zero fill");
}

void *pinned_get(size_t bytes) {
  std::lock_guard<std::mutex> lk(g_pin_mu);
  for (size_t i = 0; i < g_pin_free.size(); ++i)
    if (g_pin_free[i].second >= bytes) {
      auto b = g_pin_free[i];
      g_pin_free.erase(g_pin_free.begin() + (long)i);
      g_pin_used.push_back(b);
      return b.first;
    }
  size_t sz = 4096;
  while (sz < bytes) sz *= 2;
  void *p = nullptr;
  if (host_alloc_mapped(&p, sz) != BDL_OK) return nullptr;
  g_pin_used.push_back({p, sz});
  return p;
}

void pinned_put(void *p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pin_mu);
  for (size_t i = 0; i < g_pin_used.size(); ++i)
    if (g_pin_used[i].first == p) {
      g_pin_free.push_back(g_pin_used[i]);
      g_pin_used.erase(g_pin_used.begin() + (long)i);
      return;
    }
}

int h2d(void *dst, const void *src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return BDL_OK;
  if (((uintptr_t)dst & 15) != 0) return set_error(BDL_EINTERNAL, "table not 16-byte aligned");
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  int st = cuda_check(cudaStreamIsCapturing(s, &cs), "cudaStreamIsCapturing");
  if (st) return st;
  if (cs != cudaStreamCaptureStatusNone) {
    for (size_t o = 0; o < bytes; o += sizeof(Blob)) {
      Blob b;
      const size_t n = std::min(sizeof(Blob), bytes - o);
      memcpy(b.w, (const unsigned char *)src + o, n);
      KScope ks_(kK_put_blob, s);
      k_put_blob<<<1, 256, 0, s>>>(b, (unsigned char *)dst + o, (int)n);
    }
    return cuda_check(cudaGetLastError(), "table upload");
  }
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 128) return set_error(BDL_EINVAL, "device index out of range");
  const size_t len = a256(bytes);
  if (len > kRingBytes)   // larger than the ring: plain copy
    return cuda_check(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s), "table upload");
  std::lock_guard<std::mutex> lk(g_ring_mu);
  Ring &R = g_ring[dev];
  if (!R.base) {
    st = host_alloc_mapped((void **)&R.base, kRingBytes);
    if (st) return st;
    R.dbase = (unsigned char *)mapped(R.base);
    if (!R.dbase) {
      cudaFreeHost(R.base);
      R.base = nullptr;
      return set_error(BDL_ECUDA, "table ring is not device-mapped");
    }
  }
  if (R.head + len > kRingBytes) R.head = 0;
  const size_t lo = R.head, hi = R.head + len;
  for (size_t i = 0; i < R.busy.size();) {   // wait for the copies that used this region
    const Ring::Use &u = R.busy[i];
    if (u.off < hi && lo < u.off + u.len) {
      st = cuda_check(cudaEventSynchronize(u.ev), "cudaEventSynchronize(table ring)");
      if (st) return st;
      R.spare.push_back(u.ev);
      R.busy.erase(R.busy.begin() + (long)i);
    } else {
      ++i;
    }
  }
  memcpy(R.base + lo, src, bytes);
  st = small_copy(dst, R.dbase + lo, bytes, s);   // not behind the caller's transfers on a copy engine
  if (st) return st;
  cudaEvent_t ev = nullptr;
  if (!R.spare.empty()) {
    ev = R.spare.back();
    R.spare.pop_back();
  } else {
    st = cuda_check(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "cudaEventCreate");
    if (st) {
      cudaStreamSynchronize(s);   // no event to guard the region: wait here instead
      return st;
    }
  }
  st = cuda_check(cudaEventRecord(ev, s), "cudaEventRecord");
  if (st) {
    cudaStreamSynchronize(s);
    R.spare.push_back(ev);
    return st;
  }
  R.busy.push_back(Ring::Use{lo, len, ev});
  R.head = hi;
  return BDL_OK;
}

// Static trees of a forest without an hbm budget are laid out for their
// level's capacity X * 2^level (the most a tree of that level holds), so a
// cleared tree's block can serve its level's next tree: it is kept as the
// level's spare instead of going back to the pool.  The binary counter
// clears a level and later fills it again, so after the first carries a
// step allocates almost nothing (a batched step over hundreds of forests
// otherwise makes a pool call per new tree and per cleared one).  Reuse is
// ordered like the buffer's spare: a forest's calls are ordered on one stream.
static bool keeps_spares(const bdl_forest *f, int level) {
  return level < kMaxLevel && f->cfg.hbm_budget_bytes == 0;
}

static void free_tree(bdl_forest *f, Tree *t, cudaStream_t s) {
  if (!t) return;
  if (keeps_spares(f, t->level) && !f->spare[t->level].block &&
      t->room >= ((int64_t)f->cfg.buffer_size << t->level)) {
    f->spare[t->level] = bdl_forest::SpareBlock{t->block, t->bytes, t->room};   // still the forest's memory
    delete t;
    return;
  }
  dev_free(f, t->block, t->bytes, s);   // the bloom filter, if any, lives in the block
  delete t;
}

// Blocks of the split-block bloom filter of a tree of `size` points: the
// smallest power of two with at least bits_per_key bits per point (Sec. V-A).
static int64_t bloom_blocks_for(const bdl_forest *f, int64_t size) {
  const int64_t need = (size * f->cfg.bloom_bits_per_key + 255) / 256;
  int64_t blocks = 1;
  while (blocks < need) blocks *= 2;
  return blocks;
}

// Set a tree's shape for `size` points (its arrays must have room for it).
static void shape_tree(const bdl_forest *f, Tree *t, int64_t size) {
  t->size = size;
  t->live = size;
  t->h = tree_height(size, f->cfg.leaf_size);
  t->nnodes = ((int64_t)2 << t->h) - 1;
  t->nleaves = (int64_t)1 << t->h;
}

// A tree of `size` points whose arrays have room for up to `room` points
// (room >= size; the buffer's tree is laid out for a full buffer and reused).
static int alloc_tree(bdl_forest *f, int level, int64_t size, cudaStream_t s, Tree **out, int64_t room = 0) {
  room = std::max(room, size);
  bdl_forest::SpareBlock *sp = nullptr;
  if (keeps_spares(f, level)) {
    room = std::max(room, (int64_t)f->cfg.buffer_size << level);
    sp = &f->spare[level];
    if (sp->block && sp->room < room) {   // too small for this tree: back to the pool
      dev_free(f, sp->block, sp->bytes, s);
      sp->block = nullptr;
    }
    if (sp->block) room = sp->room;
  }
  Tree *t = new Tree();
  t->level = level;
  shape_tree(f, t, room);               // the layout is that of the largest shape
  t->room = room;
  size_t b_pts = a256((size_t)rec_ints(f->dim) * room * 4),
         b_node = a256((size_t)t->nnodes * 16),
         b_box = a256((size_t)t->nnodes * 2 * f->dim * 4), b_live = a256((size_t)t->nnodes * 4),
         b_leaf = a256((size_t)(t->nleaves + 1) * 4),
         b_pk = a256((size_t)packed_nrec(t->h) * packed_node_ints(f->dim) * 4);
  shape_tree(f, t, size);
  // a static tree's bloom filter (Sec. V-A) is built lazily but its room is
  // part of the block, so building it needs no allocation (the room is sized
  // for the layout's capacity, the filter for the tree's size)
  const int64_t blocks = level < kMaxLevel ? bloom_blocks_for(f, size) : 0;
  const int64_t room_blocks = level < kMaxLevel ? bloom_blocks_for(f, sp ? room : size) : 0;
  const size_t b_bloom = a256((size_t)room_blocks * 32);
  t->bytes = b_pts + b_node + b_box + b_live + b_leaf + b_pk + b_bloom;
  if (sp && sp->block && sp->bytes == t->bytes) {
    t->block = sp->block;
    sp->block = nullptr;
  } else {
    if (sp && sp->block) {   // (a layout of the same room has the same bytes)
      dev_free(f, sp->block, sp->bytes, s);
      sp->block = nullptr;
    }
    const int st = dev_alloc(f, &t->block, t->bytes, s);
    if (st) {
      delete t;
      return st;
    }
  }
  char *p = (char *)t->block;
  t->pts = (int32_t *)p; p += b_pts;
  t->node = (Node *)p; p += b_node;
  t->box = (int32_t *)p; p += b_box;
  t->live_nodes = (int32_t *)p; p += b_live;
  t->leaf_off = (int32_t *)p; p += b_leaf;
  t->pk = (int32_t *)p; p += b_pk;
  t->bloom_room = blocks ? (uint32_t *)p : nullptr;
  t->bloom_room_blocks = blocks;
  // Every build writes every node.  Under BDL_DEBUG_CHECK the node array starts
  // filled with -1 anyway, so that a node a build failed to write reads the
  // same each time; without it such a node could only trip the kernels' own
  // index checks, which never step outside the arrays.
  if (f->debug_check) cudaMemsetAsync(t->node, 0xff, (size_t)t->nnodes * 16, s);
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

// ---------------------------------------------------------------------------
// Insert_L (Alg. 3), planned per forest, built for many forests at once
// ---------------------------------------------------------------------------

// One forest's Insert_L of the pool = sorted buffer ++ P (|P| = n).
struct InsertPlan {
  bdl_forest *f = nullptr;
  PoolSrc pool{};
  int64_t n = 0, t = 0, q = 0, rem = 0;
  uint64_t Fnew = 0, cleared = 0;
  std::vector<Tree *> built;     // new trees, allocated, built by build_trees
  void *newbuf = nullptr;        // the new buffer (q > 0)
};

// Plan the carry and allocate the new trees; their BuildTree / ClearedSrc
// entries are appended to bt / cl (indices of cl.dst refer to bt).
static int plan_insert(bdl_forest *f, const PoolSrc &pool, int64_t n, InsertPlan &ip,
                       std::vector<BuildTree> &bt, std::vector<ClearedSrc> &cl, cudaStream_t s) {
  const int64_t X = f->cfg.buffer_size;
  ip.f = f;
  ip.pool = pool;
  ip.n = n;
  ip.t = f->nbuf + n;
  ip.q = ip.t / X;
  ip.rem = ip.t % X;
  if (ip.q == 0) return BDL_OK;                 // everything fits in the buffer
  ip.Fnew = f->F + (uint64_t)ip.q;
  const uint64_t newt = ip.Fnew & ~f->F;
  ip.cleared = f->F & ~ip.Fnew;
  if (ip.Fnew >> kMaxLevel) return set_error(BDL_EINVAL, "forest too large");
  int64_t pos = 0;
  int prev = -1;
  for (int j = 0; j < kMaxLevel; ++j) {
    if (!((newt >> j) & 1)) continue;
    int64_t capsum = 0, livesum = 0;
    const int32_t dst = (int32_t)bt.size();
    for (int i = prev + 1; i < j; ++i) {
      if (!((ip.cleared >> i) & 1)) continue;
      Tree *ct = f->trees[i];
      capsum += X << i;
      livesum += ct->live;
      cl.push_back(ClearedSrc{ct->pts, ct->size, dst});
    }
    const int64_t shortfall = (X << j) - capsum;
    Tree *nt = nullptr;
    int st = alloc_tree(f, j, livesum + shortfall, s, &nt);
    if (st) return st;
    ip.built.push_back(nt);
    BuildTree b;
    b.tree = nt;
    b.s = livesum + shortfall;
    b.h = nt->h;
    b.from_cleared = livesum;
    b.pool = pool;
    b.pool_lo = pos;
    b.idtab = f->idtab;
    b.err = f->err;
    bt.push_back(b);
    pos += shortfall;
    prev = j;
  }
  if (pos != ip.q * X) return set_error(BDL_EINTERNAL, "planner: pool split mismatch");
  // the new buffer: the forest's spare one (the buffer before last, kept
  // instead of freed), else a new allocation
  if (f->buf_spare) {
    ip.newbuf = f->buf_spare;
    f->buf_spare = nullptr;
    return BDL_OK;
  }
  return dev_alloc(f, &ip.newbuf, (size_t)X * 4, s);
}

// Undo a plan that will not be committed.
static void drop_plan(InsertPlan &ip, cudaStream_t s) {
  for (Tree *t : ip.built) free_tree(ip.f, t, s);
  ip.built.clear();
  if (ip.newbuf) {
    if (!ip.f->buf_spare) ip.f->buf_spare = (int32_t *)ip.newbuf;
    else dev_free(ip.f, ip.newbuf, (size_t)ip.f->cfg.buffer_size * 4, s);
  }
  ip.newbuf = nullptr;
}

// The new buffer (the pool's tail, Sec. IV-B1) as a fill segment.
static FillSeg tail_fill(const InsertPlan &ip) {
  FillSeg g;
  memset(&g, 0, sizeof(g));
  g.kind = kFillPoolTail;
  g.buf = ip.pool.buf;
  g.nbuf = ip.pool.nbuf;
  g.arr = ip.pool.arr;
  g.first = ip.pool.first;
  if (ip.q == 0) {               // append P after the buffer
    g.from = ip.f->nbuf;
    g.count = ip.n;
    g.dst = ip.f->buf + ip.f->nbuf;
  } else {
    g.from = ip.q * ip.f->cfg.buffer_size;
    g.count = ip.rem;
    g.dst = (int32_t *)ip.newbuf;
  }
  return g;
}

// A list to sort, given its length.
static SortList sort_list(int32_t *ids, int64_t n) {
  int np2 = 1;
  while (np2 < n) np2 <<= 1;
  return SortList{ids, (int32_t)n, np2};
}

// After the build and the tail fill: free cleared trees and the old buffer,
// install the new trees.  A buffer that took reinserted ids is added to
// `sorts` (it must stay in ascending id order).
static void commit_insert(InsertPlan &ip, std::vector<SortList> &sorts, cudaStream_t s) {
  bdl_forest *f = ip.f;
  const int64_t X = f->cfg.buffer_size;
  if (ip.pool.arr) {             // reinserted ids: keep the buffer sorted
    if (ip.q == 0 && ip.t > 1) sorts.push_back(sort_list(f->buf, ip.t));
    else if (ip.q > 0 && ip.rem > 1) sorts.push_back(sort_list((int32_t *)ip.newbuf, ip.rem));
  }
  if (ip.q == 0) {
    f->nbuf = ip.t;
  } else {
    for (int i = 0; i < kMaxLevel; ++i)
      if ((ip.cleared >> i) & 1) {
        free_tree(f, f->trees[i], s);
        f->trees[i] = nullptr;
      }
    for (Tree *t : ip.built) f->trees[t->level] = t;
    // the old buffer becomes the spare (its last readers are earlier on the
    // stream than any writer of the next insert)
    if (!f->buf_spare) f->buf_spare = f->buf;
    else dev_free(f, f->buf, (size_t)X * 4, s);
    f->buf = (int32_t *)ip.newbuf;
    f->nbuf = ip.rem;
    f->F = ip.Fnew;
  }
  f->buf_dirty = true;
  f->version++;
  ip.built.clear();
  ip.newbuf = nullptr;
}

// Trees of forests in one class are built together: same dimension, same
// splitting rule (Sec. V-C).
static int build_class(const bdl_forest *f) { return 2 * f->dim + (f->cfg.split_rule == BDL_SPLIT_SPATIAL); }

// Per-call device scratch for small tables, charged to one forest.
struct Temp {
  bdl_forest *f;
  cudaStream_t s;
  std::vector<std::pair<void *, size_t>> blocks;
  Temp(bdl_forest *f_, cudaStream_t s_) : f(f_), s(s_) {}
  int get(size_t bytes, void **p) {
    int st = dev_alloc(f, p, bytes, s);
    if (!st) blocks.push_back({*p, bytes});
    return st;
  }
  ~Temp() {
    for (auto &b : blocks) dev_free(f, b.first, b.second, s);
  }
};

// Build the planned trees of many forests, grouped by dimension, then fill
// the new buffers and commit.  Plans with q == 0 only fill.
// Device work of the plans: build every new tree (one build per class) and
// write the new buffers.  On failure every plan is dropped.
static int build_planned(std::vector<InsertPlan> &plans, std::vector<BuildTree> &bt,
                         std::vector<ClearedSrc> &cl, std::vector<int> &bt_plan, Temp &tmp,
                         cudaStream_t s) {
  int st = BDL_OK;
  // one build per (dimension, splitting rule) present
  std::vector<int> classes;
  for (auto &b : bt) {
    int d = build_class(plans[bt_plan[&b - bt.data()]].f);
    if (std::find(classes.begin(), classes.end(), d) == classes.end()) classes.push_back(d);
  }
  for (int d : classes) {
    if (st) break;
    std::vector<BuildTree> g;
    std::vector<int> remap(bt.size(), -1);
    bdl_forest *charge = nullptr;
    for (size_t j = 0; j < bt.size(); ++j) {
      bdl_forest *f = plans[bt_plan[j]].f;
      if (build_class(f) != d) continue;
      if (!charge) charge = f;
      remap[j] = (int)g.size();
      g.push_back(bt[j]);
    }
    std::vector<ClearedSrc> gc;
    for (auto &c : cl)
      if (remap[c.dst] >= 0) gc.push_back(ClearedSrc{c.pts, c.size, remap[c.dst]});
    st = build_trees(charge, charge->dim, g, gc, s);
  }
  std::vector<FillSeg> fills;
  for (auto &ip : plans)
    if (ip.f && (ip.q > 0 ? ip.rem > 0 : ip.n > 0)) fills.push_back(tail_fill(ip));
  void *table = nullptr;
  if (!st && !fills.empty()) st = tmp.get(table_bytes(fills.size(), sizeof(FillSeg)), &table);
  if (!st && !fills.empty()) st = launch_fill_many(fills, table, s);
  if (st)
    for (auto &ip : plans) drop_plan(ip, s);
  return st;
}

// Install built plans: the given fills (alive bits, ids out) on the device,
// then the trees and buffers on the host.
static int commit_planned(std::vector<InsertPlan> &plans, std::vector<FillSeg> fills, Temp &tmp,
                          cudaStream_t s) {
  int st = BDL_OK;
  void *table = nullptr;
  if (!fills.empty()) st = tmp.get(table_bytes(fills.size(), sizeof(FillSeg)), &table);
  if (!st && !fills.empty()) st = launch_fill_many(fills, table, s);
  if (st) {
    for (auto &ip : plans) drop_plan(ip, s);
    return st;
  }
  std::vector<SortList> sorts;
  for (auto &ip : plans)
    if (ip.f) commit_insert(ip, sorts, s);
  if (sorts.empty()) return BDL_OK;
  void *st_tab = nullptr;
  st = tmp.get(sort_small_table_bytes(sorts.size()), &st_tab);
  if (!st) st = launch_sort_small_many(sorts, st_tab, s);
  return st;
}

static int build_and_commit(std::vector<InsertPlan> &plans, std::vector<BuildTree> &bt,
                            std::vector<ClearedSrc> &cl, std::vector<int> &bt_plan,
                            std::vector<FillSeg> extra_fills, Temp &tmp, cudaStream_t s) {
  const int st = build_planned(plans, bt, cl, bt_plan, tmp, s);
  if (st) return st;
  return commit_planned(plans, std::move(extra_fills), tmp, s);
}

// The buffer's points get a small kd-tree of their own for k-NN (the paper's
// buffer tree), rebuilt when the buffer changed -- for many forests in shared
// build launches.  A forest whose rebuild cannot get memory keeps scanning.
static void refresh_btrees(bdl_forest *const *F, int nf, cudaStream_t s) {
  std::vector<BuildTree> bt;
  std::vector<int> owner;
  for (int i = 0; i < nf; ++i) {
    bdl_forest *f = F[i];
    if (!f->buf_dirty) continue;
    f->buf_dirty = false;
    f->version++;
    // the tree's arrays have room for a full buffer and are rebuilt in place
    // (earlier readers are earlier on the stream)
    Tree *t = f->btree;
    f->btree = nullptr;
    if (f->nbuf == 0) {
      free_tree(f, t, s);
      continue;
    }
    if (t) {
      shape_tree(f, t, f->nbuf);
    } else if (alloc_tree(f, kMaxLevel, f->nbuf, s, &t, f->cfg.buffer_size) != BDL_OK) {
      continue;
    }
    BuildTree b;
    b.tree = t;
    b.s = f->nbuf;
    b.h = t->h;
    b.from_cleared = 0;
    b.pool = PoolSrc{f->buf, f->nbuf, nullptr, 0};
    b.pool_lo = 0;
    b.idtab = f->idtab;
    b.err = f->err;
    bt.push_back(b);
    owner.push_back(i);
  }
  std::vector<int> classes;
  for (size_t j = 0; j < bt.size(); ++j) {
    const int c = build_class(F[owner[j]]);
    if (std::find(classes.begin(), classes.end(), c) == classes.end()) classes.push_back(c);
  }
  for (int d : classes) {
    std::vector<BuildTree> g;
    std::vector<int> who;
    for (size_t j = 0; j < bt.size(); ++j)
      if (build_class(F[owner[j]]) == d) { g.push_back(bt[j]); who.push_back(owner[j]); }
    const bool ok = build_trees(F[who[0]], F[who[0]]->dim, g, {}, s) == BDL_OK;
    for (size_t j = 0; j < g.size(); ++j) {
      if (ok) F[who[j]]->btree = g[j].tree;
      else free_tree(F[who[j]], g[j].tree, s);
    }
  }
}

ForestView knn_view(bdl_forest *f, bool build, cudaStream_t s) {
  if (build && f->buf_dirty) refresh_btrees(&f, 1, s);
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

static bool same_device(bdl_forest *const *F, int nf) {
  for (int i = 1; i < nf; ++i)
    if (!F[i] || F[i]->device != F[0]->device) return false;
  return true;
}

static bool distinct(bdl_forest *const *F, int nf) {
  std::vector<bdl_forest *> v(F, F + nf);
  std::sort(v.begin(), v.end());
  return std::adjacent_find(v.begin(), v.end()) == v.end();
}

// Insert_L on nf forests: one validation pass and one host sync for all, one
// build per dimension for every new tree, table-driven fills.  All or nothing:
// on EINVAL / ENOMEM no forest changes.
static int insert_many(bdl_forest *const *F, int nf, const int32_t *const *pts, const int64_t *n,
                       int32_t *const *out_ids, cudaStream_t s) {
  for (int i = 0; i < nf; ++i) {
    if (!F[i]) return set_error(BDL_EINVAL, "forest is NULL");
    if (n[i] < 0) return set_error(BDL_EINVAL, "n < 0");
    if (n[i] > 0 && !pts[i]) return set_error(BDL_EINVAL, "pts is NULL");
    if (F[i]->next_id + n[i] > (int64_t)INT32_MAX)
      return set_error(BDL_EINVAL, "id space (2^31 - 1) exhausted");
  }
  if (!same_device(F, nf)) return set_error(BDL_EINVAL, "forests on different devices");
  if (!distinct(F, nf)) return set_error(BDL_EINVAL, "a forest appears twice");
  int st = BDL_OK;
  for (int i = 0; i < nf && !st; ++i)
    if (n[i] > 0) st = ensure_id_capacity(F[i], F[i]->next_id + n[i], s);
  if (st) return st;
  Temp tmp(F[0], s);
  // 1. append the coordinates to the id tables and check them (one pass)
  std::vector<FillSeg> app;
  for (int i = 0; i < nf; ++i) {
    if (n[i] == 0) continue;
    FillSeg g;
    memset(&g, 0, sizeof(g));
    g.kind = kFillAppend;
    g.count = n[i] * F[i]->dim;
    g.src = pts[i];
    g.dst = F[i]->idtab + F[i]->next_id * F[i]->dim;
    g.errw = F[i]->err;            // the flags also carry the error word of earlier work
    app.push_back(g);
  }
  if (app.empty()) return BDL_OK;
  void *flags = nullptr, *table = nullptr;
  st = tmp.get(app.size() * 8, &flags);
  if (!st) st = tmp.get(table_bytes(app.size(), sizeof(FillSeg)), &table);
  if (st) return st;
  for (size_t j = 0; j < app.size(); ++j) app[j].flag = (unsigned long long *)flags + j;
  small_zero(flags, app.size() * 8, s);
  st = launch_fill_many(app, table, s);
  // The append stores off-grid coordinates clamped onto the grid and flags
  // them.  With room for the flags in the forest's pinned scratch, the build
  // goes ahead without waiting: it only ever sees grid coordinates, and its
  // result is installed after the flags have come back clean (else dropped:
  // nothing it wrote is reachable from the forest).  Without room, wait first.
  int64_t *hf = F[0]->pinned;
  const bool ahead = app.size() <= kPinnedFlags;
  std::vector<int64_t> hf_big;
  if (!ahead) {
    hf_big.resize(app.size());
    hf = hf_big.data();
  }
  if (!st && ahead) st = small_copy(F[0]->pinned_dev, flags, app.size() * 8, s);   // the forest's mapped scratch
  if (!st && !ahead) st = cuda_check(cudaMemcpyAsync(hf, flags, app.size() * 8, cudaMemcpyDeviceToHost, s), "copy");
  if (!st && ahead) {
    if (!F[0]->ev_flags) st = cuda_check(cudaEventCreateWithFlags(&F[0]->ev_flags, cudaEventDisableTiming),
                                         "cudaEventCreate");
    if (!st) st = cuda_check(cudaEventRecord(F[0]->ev_flags, s), "cudaEventRecord");
  }
  if (!st && !ahead) st = cuda_check(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  if (st) return st;
  // flag bit 0: a coordinate off the grid; bit 1: the forest's device error
  // word was set by earlier work (a kernel found an index outside its
  // buffers), whose bits follow from bit 8 on
  auto off_grid = [&]() {
    for (size_t j = 0; j < app.size(); ++j)
      if (hf[j] & 1) return true;
    return false;
  };
  auto dev_error = [&]() {
    for (size_t j = 0; j < app.size(); ++j)
      if (hf[j] & 2) return true;
    return false;
  };
  auto dev_error_msg = [&]() {
    uint64_t bits = 0;
    for (size_t j = 0; j < app.size(); ++j) bits |= (uint64_t)hf[j] >> 8;
    return std::string("device error word set by earlier work, code ") + std::to_string(bits);
  };
  if (!ahead && dev_error()) return set_error(BDL_EINTERNAL, dev_error_msg());
  if (!ahead && off_grid()) return set_error(BDL_EINVAL, "coordinate outside [0, 2^20)");
  // 2. plan every forest (Alg. 3), allocating the new trees
  std::vector<InsertPlan> plans(nf);
  std::vector<BuildTree> bt;
  std::vector<ClearedSrc> cl;
  std::vector<int> bt_plan;
  for (int i = 0; i < nf && !st; ++i) {
    if (n[i] == 0) continue;
    st = plan_insert(F[i], PoolSrc{F[i]->buf, F[i]->nbuf, nullptr, F[i]->next_id}, n[i], plans[i], bt, cl, s);
    bt_plan.resize(bt.size(), i);
  }
  if (st) {
    for (auto &ip : plans)
      if (ip.f) drop_plan(ip, s);
    if (ahead) cudaEventSynchronize(F[0]->ev_flags);   // the flags' copy targets pinned scratch
    return st;
  }
  // 3. build and new buffers; then, once the coordinates are known to be on
  //    the grid, alive bits, ids out and the commit
  std::vector<FillSeg> post;
  for (int i = 0; i < nf; ++i) {
    if (n[i] == 0) continue;
    FillSeg g;
    memset(&g, 0, sizeof(g));
    g.kind = kFillAlive;
    g.first = F[i]->next_id;
    g.count = n[i];
    g.alive = F[i]->alive;
    post.push_back(g);
    if (out_ids[i]) {
      g.kind = kFillIota;
      g.dst = out_ids[i];
      g.alive = nullptr;
      post.push_back(g);
    }
  }
  st = build_planned(plans, bt, cl, bt_plan, tmp, s);
  if (ahead) {
    const int es = cuda_check(cudaEventSynchronize(F[0]->ev_flags), "cudaEventSynchronize");
    if (!st) st = es;
    if (!st && (off_grid() || dev_error())) {
      for (auto &ip : plans)
        if (ip.f) drop_plan(ip, s);
      if (dev_error()) return set_error(BDL_EINTERNAL, dev_error_msg());
      return set_error(BDL_EINVAL, "coordinate outside [0, 2^20)");
    }
  }
  if (st) return st;   // (a failed build has dropped its plans)
  st = commit_planned(plans, post, tmp, s);
  if (st) return st;
  for (int i = 0; i < nf; ++i) {
    F[i]->next_id += n[i];
    F[i]->live += n[i];
  }
  return cuda_check(cudaGetLastError(), "insert");
}

static int reinsert_low(const std::vector<bdl_forest *> &fs, cudaStream_t s);
static int finish(bdl_forest *f, cudaStream_t s, int st);

// One id list of one forest in an erase call.
struct EraseList {
  int forest;              // index into the call's forests
  const int32_t *ids;
  int64_t n;
};

// Erase_L on nf distinct forests, each erasing its lists in the order given
// (one list per forest for the plain calls; the server's merged requests give
// several): one marking pass per rank of list -- a forest's list r is marked
// after its list r - 1, so an id counts for the first list that names it --
// whose counts stay on the device, lazily built blooms, one descent launch,
// the k-NN records' live counts (refreshed, or kept on the descent paths of
// small batches), one buffer compaction, one host sync for the counts;
// reinsertion of trees below half then runs for all forests together
// (Alg. 4).  out_list[j] receives list j's count.
static int erase_core(bdl_forest *const *F, int nf, const std::vector<EraseList> &L, int64_t *out_list,
                      cudaStream_t s) {
  const size_t nl = L.size();
  for (size_t j = 0; j < nl; ++j)
    if (out_list) out_list[j] = 0;
  Temp tmp(F[0], s);
  // 1. dedup against the live sets, list rank by list rank
  std::vector<int64_t> fsum(nf, 0);
  for (const auto &e : L) fsum[e.forest] += e.n;
  std::vector<int> fa(nf, -1), act_forest;   // forest -> active index
  for (int i = 0; i < nf; ++i)
    if (fsum[i] > 0 && F[i]->next_id > 0) {
      fa[i] = (int)act_forest.size();
      act_forest.push_back(i);
    }
  if (act_forest.empty()) return BDL_OK;
  const size_t na = act_forest.size();
  std::vector<int> use;                      // lists taking part
  int64_t total = 0;
  for (size_t j = 0; j < nl; ++j)
    if (L[j].n > 0 && fa[L[j].forest] >= 0) use.push_back((int)j), total += L[j].n;
  // device counts: one per list taking part, then one total per active forest
  void *lists = nullptr, *counts = nullptr, *table = nullptr;
  int st = tmp.get((size_t)total * 4, &lists);
  if (!st) st = tmp.get((use.size() + na) * 8, &counts);
  if (!st) st = tmp.get(table_bytes(use.size(), sizeof(MarkSeg)), &table);
  if (st) return st;
  int64_t *lcount = (int64_t *)counts;                 // [use.size()]
  int64_t *ftotal = lcount + use.size();               // [na]
  std::vector<int32_t *> lptr(use.size());
  std::vector<int> rank(use.size()), seen(nf, 0);
  int64_t off = 0;
  int nrank = 0;
  for (size_t u = 0; u < use.size(); ++u) {
    const EraseList &e = L[use[u]];
    lptr[u] = (int32_t *)lists + off;
    off += e.n;
    rank[u] = seen[e.forest]++;
    nrank = std::max(nrank, rank[u] + 1);
  }
  small_zero(counts, (use.size() + na) * 8, s);
  for (int r = 0; r < nrank && !st; ++r) {
    std::vector<MarkSeg> mk;
    for (size_t u = 0; u < use.size(); ++u) {
      if (rank[u] != r) continue;
      const EraseList &e = L[use[u]];
      bdl_forest *f = F[e.forest];
      const bool alone = seen[e.forest] == 1;
      mk.push_back(MarkSeg{f->alive, f->next_id, e.ids, e.n, lptr[u], lcount + u,
                           alone ? lcount + u : ftotal + fa[e.forest]});
    }
    st = launch_erase_mark_many(mk, table, s);   // stream order: the table is reused after the launch read it
  }
  if (st) return st;
  // a forest's count on the device: its list's, or the total over its lists
  std::vector<const int64_t *> ne_dev(na);
  for (size_t u = 0; u < use.size(); ++u) {
    const int i = L[use[u]].forest;
    ne_dev[fa[i]] = seen[i] == 1 ? lcount + u : ftotal + fa[i];
  }
  // Every forest with a nonempty batch takes part from here on without a wait
  // for the counts: the launches are sized by the batch lengths and read the
  // counts on the device, and a forest whose batch erased nothing is left as
  // it was (its new blooms are skipped on the device and unmarked after the
  // sync below).
  // 2. lazily build the bloom filter of every nonempty tree (Sec. V-A)
  std::vector<TreeSeg> blooms;
  std::vector<FillSeg> zeros;
  std::vector<std::pair<int, Tree *>> fresh;   // (active index, tree) of the blooms built here
  for (size_t a = 0; a < na; ++a) {
    bdl_forest *f = F[act_forest[a]];
    for (int i = 0; i < kMaxLevel && !st; ++i) {
      Tree *t = f->trees[i];
      if (!t || t->live == 0 || t->bloom) continue;
      const int64_t blocks = t->bloom_room_blocks;
      if (!t->bloom_room || blocks != bloom_blocks_for(f, t->size)) {
        st = set_error(BDL_EINTERNAL, "tree without bloom room");
        break;
      }
      t->bloom = t->bloom_room;
      t->bloom_blocks = blocks;
      t->bloom_bytes = (size_t)blocks * 32;
      fresh.emplace_back((int)a, t);
      FillSeg z;                     // zeroed in one launch with the others
      memset(&z, 0, sizeof(z));
      z.kind = kFillZero;
      z.count = blocks * 8;
      z.dst = (int32_t *)t->bloom;
      zeros.push_back(z);
      TreeSeg g;
      memset(&g, 0, sizeof(g));
      g.pts = t->pts;
      g.size = t->size;
      g.dim = f->dim;
      g.bloom = t->bloom;
      g.blocks = blocks;
      g.seed = f->cfg.hash_seed;
      g.gate = ne_dev[a];             // built only if the batch erases something
      blooms.push_back(g);
    }
  }
  if (st) return st;
  if (!zeros.empty()) {
    void *zt = nullptr;
    st = tmp.get(table_bytes(zeros.size(), sizeof(FillSeg)), &zt);
    if (!st) st = launch_fill_many(zeros, zt, s);
    if (st) return st;
  }
  if (!blooms.empty()) {
    void *bt = nullptr;
    st = tmp.get(table_bytes(blooms.size(), sizeof(TreeSeg)), &bt);
    if (!st) st = launch_bloom_build_many(blooms, bt, s);
    if (st) return st;
  }
  // 3. probe, descend, tombstone (Alg. 2 on every tree of every forest, one
  //    launch, one job per list); a large list descends in spatial order
  std::vector<ForestView> views(na);
  std::vector<EraseCall> calls;
  // The packed k-NN records' live counts: a small batch (under 1/128 of the
  // forest) updates them on its descent paths, a larger one has every record
  // refreshed from the nodes afterwards, whichever touches less.
  std::vector<int> incremental(na);
  for (size_t a = 0; a < na; ++a) {
    const bdl_forest *f = F[act_forest[a]];
    incremental[a] = fsum[act_forest[a]] * 128 < f->live;
    views[a] = forest_view(f);
  }
  for (size_t u = 0; u < use.size(); ++u) {
    const int i = L[use[u]].forest, a = fa[i];
    bdl_forest *f = F[i];
    const int32_t *order = lptr[u];
    const int64_t nj = L[use[u]].n;   // the owned ids are the first lcount[u] of the list
    if (nj >= kSortMinQueries) {
      void *sorted = nullptr;
      if (tmp.get(a256((size_t)nj * 4) + query_sort_bytes(nj, f->dim), &sorted) == BDL_OK) {
        launch_point_sort(f->idtab, lptr[u], nj, f->dim, (char *)sorted + a256((size_t)nj * 4),
                          (int32_t *)sorted, s, lcount + u);
        order = (const int32_t *)sorted;
      }
    }
    calls.push_back(EraseCall{&views[a], order, nj, f->cfg.hash_seed, lcount + u, incremental[a]});
  }
  {
    void *et = nullptr;
    st = tmp.get(erase_table_bytes(calls), &et);
    if (!st) st = launch_erase_jobs(calls, et, s);
    if (st) return st;
  }
  // 4. the records' live counts (refreshed, or checked in debug runs when the
  //    descent kept them); compact the buffers; counts back
  std::vector<TreeSeg> lives;
  std::vector<BufSeg> bufs;
  void *outs = nullptr;
  st = tmp.get(na * kBufOutWords * 8, &outs);
  if (st) return st;
  for (size_t a = 0; a < na; ++a) {
    bdl_forest *f = F[act_forest[a]];
    BufSeg b;
    memset(&b, 0, sizeof(b));
    b.buf = f->buf;
    b.nbuf = f->nbuf;
    b.alive = f->alive;
    b.out = (int64_t *)outs + a * kBufOutWords;
    b.errw = f->err;
    for (int i = kMaxLevel - 1; i >= 0; --i) {
      Tree *t = f->trees[i];
      if (!t) continue;
      b.roots[b.ntrees++] = t->live_nodes;
      if (incremental[a] && !f->debug_check) continue;
      TreeSeg g;
      memset(&g, 0, sizeof(g));
      g.dim = f->dim;
      g.h = t->h;
      g.node = t->node;
      g.live = t->live_nodes;
      g.pk = t->pk;
      g.err = incremental[a] ? f->err : nullptr;
      lives.push_back(g);
    }
    bufs.push_back(b);
  }
  void *lt = nullptr, *bt2 = nullptr;
  if (!lives.empty()) {
    st = tmp.get(table_bytes(lives.size(), sizeof(TreeSeg)), &lt);
    if (!st) st = launch_pack_lives_many(lives, lt, s);
    if (st) return st;
  }
  st = tmp.get(table_bytes(bufs.size(), sizeof(BufSeg)), &bt2);
  if (!st) st = launch_buffer_compact_many(bufs, bt2, s);
  // counts back through page-locked scratch written by a kernel (not behind
  // the caller's transfers on a copy engine)
  const size_t nho = na * kBufOutWords, nhc = use.size() + na;
  struct PinGuard {
    void *p;
    ~PinGuard() { pinned_put(p); }
  } pin{pinned_get((nho + nhc) * 8)};
  std::vector<int64_t> ho_v, hc_v;
  int64_t *ho, *hc;
  int64_t *pin_dev = pin.p ? (int64_t *)mapped(pin.p) : nullptr;
  if (pin_dev) {
    ho = (int64_t *)pin.p;
    hc = ho + nho;
    if (!st) st = small_copy(pin_dev, outs, nho * 8, s);
    if (!st) st = small_copy(pin_dev + nho, counts, nhc * 8, s);
  } else {
    ho_v.resize(nho);
    hc_v.resize(nhc);
    ho = ho_v.data();
    hc = hc_v.data();
    if (!st) st = cuda_check(cudaMemcpyAsync(ho, outs, nho * 8, cudaMemcpyDeviceToHost, s), "copy");
    if (!st) st = cuda_check(cudaMemcpyAsync(hc, counts, nhc * 8, cudaMemcpyDeviceToHost, s), "copy");
  }
  if (!st) st = cuda_check(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  if (st) return st;
  // 5. new counts; trees below half capacity are emptied and their points
  //    reinserted (Alg. 4), all forests' reinsertions built together
  std::vector<int64_t> ne(na, 0);
  for (size_t u = 0; u < use.size(); ++u) {
    if (out_list) out_list[use[u]] = hc[u];
    ne[fa[L[use[u]].forest]] += hc[u];
  }
  std::vector<bdl_forest *> touched;
  int64_t dev_err = 0;
  for (size_t a = 0; a < na; ++a) {
    bdl_forest *f = F[act_forest[a]];
    f->live -= ne[a];
    const int64_t *o = &ho[a * kBufOutWords];
    dev_err |= o[kMaxLevel + 1];
    if (ne[a] == 0) continue;   // nothing erased: counts and trees as they were
    f->version++;
    if (o[0] != f->nbuf) f->buf_dirty = true;
    f->nbuf = o[0];
    int r = 0;
    for (int i = kMaxLevel - 1; i >= 0; --i)
      if (f->trees[i]) f->trees[i]->live = o[1 + r++];
    touched.push_back(f);
  }
  // a forest whose batch erased nothing had its new blooms skipped on the
  // device: they stay unbuilt, as if the erase had not reached the forest
  for (const auto &ft : fresh)
    if (ne[ft.first] == 0) {
      ft.second->bloom = nullptr;
      ft.second->bloom_blocks = 0;
      ft.second->bloom_bytes = 0;
    }
  // a kernel of this call or an earlier one found an index outside its
  // buffers: the counts above are applied, the rebuilds are not attempted
  if (dev_err)
    return set_error(BDL_EINTERNAL, "device bounds check failed, code " + std::to_string(dev_err));
  st = reinsert_low(touched, s);
  if (st) return st;
  return cuda_check(cudaGetLastError(), "erase");
}

// Erase_L on nf distinct forests, one id list each.
static int erase_many(bdl_forest *const *F, int nf, const int32_t *const *ids, const int64_t *n,
                      int64_t *out_n, cudaStream_t s) {
  for (int i = 0; i < nf; ++i) {
    if (out_n) out_n[i] = 0;
    if (!F[i]) return set_error(BDL_EINVAL, "forest is NULL");
    if (n[i] < 0) return set_error(BDL_EINVAL, "n < 0");
    if (n[i] > 0 && !ids[i]) return set_error(BDL_EINVAL, "ids is NULL");
  }
  if (!same_device(F, nf)) return set_error(BDL_EINVAL, "forests on different devices");
  if (!distinct(F, nf)) return set_error(BDL_EINVAL, "a forest appears twice");
  std::vector<EraseList> L;
  for (int i = 0; i < nf; ++i) L.push_back(EraseList{i, ids[i], n[i]});
  return erase_core(F, nf, L, out_n, s);
}

int erase_lists(bdl_forest *f, const std::vector<const int32_t *> &ids, const std::vector<int64_t> &n,
                int64_t *counts, cudaStream_t s) {
  if (!f) return set_error(BDL_EINVAL, "forest is NULL");
  std::vector<EraseList> L;
  for (size_t j = 0; j < ids.size(); ++j) {
    if (counts) counts[j] = 0;
    if (n[j] < 0) return set_error(BDL_EINVAL, "n < 0");
    if (n[j] > 0 && !ids[j]) return set_error(BDL_EINVAL, "ids is NULL");
    L.push_back(EraseList{0, ids[j], n[j]});
  }
  DeviceGuard g(f->device);
  return finish(f, s, erase_core(&f, 1, L, counts, s));
}

// Alg. 4's rebuild step for the given forests: every tree with fewer live
// points than half its capacity X*2^i is emptied, and its live points are
// reinserted through Insert_L in ascending id order, keeping their ids.  The
// forests' new trees are built in shared launches.  If that cannot get
// memory, the emptied trees stay where they were (queries remain exact).
static int reinsert_low(const std::vector<bdl_forest *> &fs, cudaStream_t s) {
  struct Low {
    bdl_forest *f;
    std::vector<Tree *> trees;
    int64_t nr;
    void *R;
    uint64_t Fsave;
    Tree *saved[kMaxLevel];
  };
  std::vector<Low> lows;
  for (bdl_forest *f : fs) {
    Low L;
    L.f = f;
    L.nr = 0;
    L.R = nullptr;
    for (int i = 0; i < kMaxLevel; ++i) {
      Tree *t = f->trees[i];
      if (t && 2 * t->live < ((int64_t)f->cfg.buffer_size << i)) {
        L.trees.push_back(t);
        L.nr += t->live;
      }
    }
    if (!L.trees.empty()) lows.push_back(std::move(L));
  }
  if (lows.empty()) return BDL_OK;
  int st = BDL_OK;
  std::vector<LiveCollect> jobs;
  for (auto &L : lows) {
    if (st) break;
    st = dev_alloc(L.f, &L.R, (size_t)std::max<int64_t>(L.nr, 1) * 4, s);
    jobs.push_back(LiveCollect{L.f, L.trees, L.nr, (int32_t *)L.R});
  }
  if (!st) st = collect_sorted_live(jobs, s);   // every forest's ids in shared launches
  std::vector<InsertPlan> plans(lows.size());
  std::vector<BuildTree> bt;
  std::vector<ClearedSrc> cl;
  std::vector<int> bt_plan;
  if (!st) {
    for (size_t j = 0; j < lows.size(); ++j) {
      Low &L = lows[j];
      L.Fsave = L.f->F;
      memcpy(L.saved, L.f->trees, sizeof(L.saved));
      for (Tree *t : L.trees) {
        L.f->trees[t->level] = nullptr;
        L.f->F &= ~((uint64_t)1 << t->level);
      }
    }
    for (size_t j = 0; j < lows.size() && !st; ++j) {
      Low &L = lows[j];
      if (L.nr == 0) continue;
      st = plan_insert(L.f, PoolSrc{L.f->buf, L.f->nbuf, (const int32_t *)L.R, 0}, L.nr, plans[j], bt,
                       cl, s);
      bt_plan.resize(bt.size(), (int)j);
    }
    if (st) {
      for (auto &ip : plans)
        if (ip.f) drop_plan(ip, s);
    } else {
      Temp tmp(lows[0].f, s);
      st = build_and_commit(plans, bt, cl, bt_plan, {}, tmp, s);
    }
    for (auto &L : lows) {
      if (st) {                    // put the emptied trees back
        L.f->F = L.Fsave;
        memcpy(L.f->trees, L.saved, sizeof(L.saved));
      } else {
        for (Tree *t : L.trees) free_tree(L.f, t, s);
      }
    }
  }
  for (auto &L : lows)
    if (L.R) dev_free(L.f, L.R, (size_t)std::max<int64_t>(L.nr, 1) * 4, s);
  return st;
}

// kNN_L on nf forests: stale buffer trees rebuilt in shared builds, then one
// k-NN launch per dimension over every forest's queries.
static int knn_many(bdl_forest *const *F, int nf, const int32_t *const *q, const int64_t *m, int k,
                    int32_t *const *oi, int64_t *const *od, cudaStream_t s,
                    unsigned long long *counts = nullptr) {
  if (k < 1 || k > kMaxK) return set_error(BDL_EINVAL, "k must be in 1..32");
  for (int i = 0; i < nf; ++i) {
    if (!F[i]) return set_error(BDL_EINVAL, "forest is NULL");
    if (m[i] < 0) return set_error(BDL_EINVAL, "m < 0");
    if (m[i] > 0 && (!q[i] || !oi[i] || !od[i])) return set_error(BDL_EINVAL, "NULL pointer");
  }
  if (!same_device(F, nf)) return set_error(BDL_EINVAL, "forests on different devices");
  Temp tmp(F[0], s);
  // large batches run in spatial order so that neighbouring threads walk
  // neighbouring paths; results are written back in input order.  The sorts
  // need nothing from the forests, so they go first and the device sorts
  // while the host plans the buffer trees' rebuilds.
  std::vector<int32_t *> perm(nf, nullptr);
  for (int i = 0; i < nf; ++i) {
    if (m[i] < kSortMinQueries || counts) continue;   // the counting walk is per lane: no order needed
    void *scratch = nullptr;
    if (tmp.get(query_sort_bytes(m[i], F[i]->dim), &scratch) == BDL_OK) {
      perm[i] = (int32_t *)scratch;
      launch_query_sort(q[i], m[i], F[i]->dim, (char *)scratch + a256((size_t)m[i] * 4), perm[i], s);
    }
  }
  refresh_btrees(F, nf, s);
  std::vector<ForestView> views(nf);
  std::vector<KnnCall> calls;
  for (int i = 0; i < nf; ++i) {
    if (m[i] == 0) continue;
    views[i] = knn_view(F[i], false, s);
    calls.push_back(KnnCall{&views[i], q[i], perm[i], m[i], oi[i], od[i]});
  }
  int st = BDL_OK;
  std::vector<int> dims;
  for (auto &c : calls)
    if (std::find(dims.begin(), dims.end(), c.fv->dim) == dims.end()) dims.push_back(c.fv->dim);
  for (int d : dims) {
    std::vector<KnnCall> g;
    unsigned long long *stats = nullptr;
    for (auto &c : calls)
      if (c.fv->dim == d) g.push_back(c);
    for (int i = 0; i < nf; ++i)
      if (F[i]->dim == d && F[i]->knn_stats) stats = F[i]->knn_stats;
    if (counts) stats = counts;
    // the jobs too small for a sort of their own share one (job, Morton) sort
    if (!counts) {
      std::vector<int> small;
      int64_t msum = 0;
      for (size_t j = 0; j < g.size(); ++j)
        if (!g[j].perm && g[j].m > 0) small.push_back((int)j), msum += g[j].m;
      if (small.size() >= 2 && msum >= kBatchSortMinQueries) {
        std::vector<KnnCall> sg;
        for (int j : small) sg.push_back(g[j]);
        void *scr = nullptr;
        const size_t bytes = batch_query_sort_bytes(sg);
        if (tmp.get(bytes, &scr) == BDL_OK && batch_query_sort(sg, scr, bytes, s) == BDL_OK)
          for (size_t j = 0; j < small.size(); ++j) g[small[j]].perm = sg[j].perm;
      }
    }
    void *table = nullptr;
    const size_t tb = knn_table_bytes(g);
    if (tb) st = tmp.get(tb, &table);
    if (!st) st = launch_knn_jobs(g, d, k, F[0]->knn_shape, table, stats, s);
    if (st) return st;
  }
  return BDL_OK;
}

}  // namespace bdl

// A prepared kNN_L over many forests: job tables and sort scratch live in
// device memory owned by the plan, so a launch is kernels only.
struct bdl_knn_plan {
  std::vector<bdl_forest *> F;
  std::vector<uint64_t> version;   // of each forest when the plan was made
  int device = 0, k = 0;
  struct Part {
    int dim, njobs;
    int64_t warps;
    void *table;
    unsigned long long *stats;
    bdl::KnnShape shape;
  };
  struct Sort {
    const int32_t *q;
    int64_t m;
    int dim;
    int32_t *perm;
    void *scratch;
  };
  std::vector<Part> parts;
  std::vector<Sort> sorts;
  bdl_forest *charge = nullptr;
  void *block = nullptr;
  size_t bytes = 0;
};

namespace bdl {

static int knn_plan_make(bdl_forest *const *F, int nf, const int32_t *const *q, const int64_t *m, int k,
                         int32_t *const *oi, int64_t *const *od, cudaStream_t s, bdl_knn_plan *P) {
  if (k < 1 || k > kMaxK) return set_error(BDL_EINVAL, "k must be in 1..32");
  if (nf < 1) return set_error(BDL_EINVAL, "a plan needs at least one forest");
  for (int i = 0; i < nf; ++i) {
    if (!F[i]) return set_error(BDL_EINVAL, "forest is NULL");
    if (m[i] < 0) return set_error(BDL_EINVAL, "m < 0");
    if (m[i] > 0 && (!q[i] || !oi[i] || !od[i])) return set_error(BDL_EINVAL, "NULL pointer");
  }
  if (!same_device(F, nf)) return set_error(BDL_EINVAL, "forests on different devices");
  refresh_btrees(F, nf, s);
  std::vector<ForestView> views(nf);
  std::vector<KnnCall> calls;
  size_t sort_bytes = 0;
  for (int i = 0; i < nf; ++i) {
    if (m[i] == 0) continue;
    views[i] = knn_view(F[i], false, s);
    if (m[i] >= kSortMinQueries) sort_bytes += a256(query_sort_bytes(m[i], F[i]->dim));
    calls.push_back(KnnCall{&views[i], q[i], nullptr, m[i], oi[i], od[i]});
  }
  std::vector<int> dims;
  for (auto &c : calls)
    if (std::find(dims.begin(), dims.end(), c.fv->dim) == dims.end()) dims.push_back(c.fv->dim);
  std::vector<std::vector<KnnCall>> groups;
  size_t table_bytes = 0;
  for (int d : dims) {
    std::vector<KnnCall> g;
    for (auto &c : calls)
      if (c.fv->dim == d) g.push_back(c);
    table_bytes += a256(knn_table_bytes_always(g));
    groups.push_back(std::move(g));
  }
  P->bytes = std::max<size_t>(table_bytes + sort_bytes, 256);
  P->charge = F[0];
  int st = dev_alloc(F[0], &P->block, P->bytes, s);
  if (st) return st;
  char *p = (char *)P->block;
  // sort scratch first: its permutation is part of the jobs
  for (auto &c : calls) {
    if (c.m < kSortMinQueries) continue;
    bdl_knn_plan::Sort so{c.q, c.m, c.fv->dim, (int32_t *)p, p + a256((size_t)c.m * 4)};
    P->sorts.push_back(so);
    p += a256(query_sort_bytes(c.m, c.fv->dim));
  }
  for (auto &g : groups)
    for (auto &c : g)
      for (auto &so : P->sorts)
        if (so.q == c.q && so.m == c.m) c.perm = so.perm;
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    const int d = dims[gi];
    unsigned long long *stats = nullptr;
    for (int i = 0; i < nf; ++i)
      if (F[i]->dim == d && F[i]->knn_stats) stats = F[i]->knn_stats;
    bdl_knn_plan::Part part{d, (int)groups[gi].size(), 0, p, stats, F[0]->knn_shape};
    st = upload_knn_table(groups[gi], p, &part.warps, part.shape.qpw, s);
    if (st) return st;
    p += a256(knn_table_bytes_always(groups[gi]));
    P->parts.push_back(part);
  }
  P->F.assign(F, F + nf);
  for (int i = 0; i < nf; ++i) P->version.push_back(F[i]->version);
  P->device = F[0]->device;
  P->k = k;
  return cuda_check(cudaGetLastError(), "k-NN plan");
}

static int knn_plan_launch(bdl_knn_plan *P, cudaStream_t s) {
  for (size_t i = 0; i < P->F.size(); ++i)
    if (P->F[i]->version != P->version[i])
      return set_error(BDL_EINVAL, "a forest changed since the k-NN plan was made");
  for (auto &so : P->sorts) launch_query_sort(so.q, so.m, so.dim, so.scratch, so.perm, s);
  for (auto &part : P->parts) {
    const int st = launch_knn_table(part.table, part.njobs, part.warps, part.dim, P->k, part.shape, part.stats, s);
    if (st) return st;
  }
  return BDL_OK;
}

// With BDL_DEBUG_CHECK=1 every call waits for its kernels and fails with
// BDL_EINTERNAL if one of them recorded an out-of-range index.
static int finish(bdl_forest *f, cudaStream_t s, int st) {
  if (st || !f->debug_check) return st;
  st = small_copy(f->pinned_dev + kPinnedErr, f->err, 8, s);
  if (!st) st = cuda_check(cudaStreamSynchronize(s), "sync");
  if (st) return st;
  if (f->pinned[kPinnedErr])
    return set_error(BDL_EINTERNAL, "device bounds check failed, code " + std::to_string(f->pinned[kPinnedErr]));
  return BDL_OK;
}

int finish_call(bdl_forest *f, cudaStream_t s, int st) { return finish(f, s, st); }

static int finish_many(bdl_forest *const *F, int nf, cudaStream_t s, int st) {
  for (int i = 0; i < nf && !st; ++i)
    if (F[i]) st = finish(F[i], s, st);
  return st;
}

static int check_config(const bdl_config &c) {
  if (c.leaf_size < 2 || c.leaf_size > 64) return set_error(BDL_EINVAL, "leaf_size must be in 2..64");
  if (c.buffer_size < 2 || c.buffer_size > 16384)
    return set_error(BDL_EINVAL, "buffer_size must be in 2..16384");
  if (c.bloom_bits_per_key < 1 || c.bloom_bits_per_key > 64)
    return set_error(BDL_EINVAL, "bloom_bits_per_key must be in 1..64");
  if (c.bloom_hashes != 8) return set_error(BDL_EINVAL, "bloom_hashes must be 8");
  if (c.hbm_budget_bytes < 0) return set_error(BDL_EINVAL, "hbm_budget_bytes must be >= 0");
  if (c.split_rule != BDL_SPLIT_OBJECT && c.split_rule != BDL_SPLIT_SPATIAL)
    return set_error(BDL_EINVAL, "split_rule must be BDL_SPLIT_OBJECT or BDL_SPLIT_SPATIAL");
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
  cfg->split_rule = BDL_SPLIT_OBJECT;
  cfg->reserved_ = 0;
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
  return bdl_profile_read_bytes(ms, launches, nullptr, cap);
}

int bdl_profile_read_bytes(double *ms, int64_t *launches, double *bytes, int cap) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (int i = 0; i < cap && i < kKernelCount; ++i) {
    if (ms) ms[i] = 0;
    if (launches) launches[i] = 0;
    if (bytes) bytes[i] = 0;
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
      if (bytes) bytes[r.kid] += r.bytes;
    }
  }
  prof_reset();
  return BDL_OK;
}

int bdl_profile_timeline(int32_t *kid, double *start_ms, double *end_ms, double *bytes, int cap, int *out_n) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (out_n) *out_n = (int)g_prof.size();
  const int n = std::min(cap, (int)g_prof.size());
  for (int i = 0; i < n; ++i) {
    const ProfRec &r = g_prof[i];
    int st = cuda_check(cudaEventSynchronize(r.b), "cudaEventSynchronize");
    if (st) return st;
    float a = 0, b = 0;
    st = cuda_check(cudaEventElapsedTime(&a, g_prof[0].a, r.a), "cudaEventElapsedTime");
    if (!st) st = cuda_check(cudaEventElapsedTime(&b, g_prof[0].a, r.b), "cudaEventElapsedTime");
    if (st) return st;
    if (kid) kid[i] = r.kid;
    if (start_ms) start_ms[i] = a;
    if (end_ms) end_ms[i] = b;
    if (bytes) bytes[i] = r.bytes;
  }
  return BDL_OK;
}

int bdl_kernel_count(void) { return kKernelCount; }

const char *bdl_kernel_name(int id) { return id >= 0 && id < kKernelCount ? kKernelNames[id] : ""; }

int bdl_insert(bdl_forest *f, const int32_t *pts, int64_t n, int32_t *out_ids, bdl_stream_t stream) {
  return bdl_insert_batch(&f, 1, &pts, &n, &out_ids, stream);
}

int bdl_insert_batch(bdl_forest *const *forests, int nf, const int32_t *const *pts, const int64_t *n,
                     int32_t *const *out_ids, bdl_stream_t stream) {
  if (nf < 0 || (nf > 0 && (!forests || !pts || !n || !out_ids))) return set_error(BDL_EINVAL, "NULL array");
  if (nf == 0) return BDL_OK;
  if (!forests[0]) return set_error(BDL_EINVAL, "forest is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  DeviceGuard g(forests[0]->device);
  return finish_many(forests, nf, s, insert_many(forests, nf, pts, n, out_ids, s));
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
  if (!st) st = host_alloc_mapped((void **)&f->pinned, kPinnedWords * 8);
  if (!st) {
    f->pinned_dev = (int64_t *)mapped(f->pinned);
    if (!f->pinned_dev) st = set_error(BDL_ECUDA, "page-locked scratch is not device-mapped");
  }
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
  return bdl_erase_batch(&f, 1, &ids, &n, out_n, stream);
}

int bdl_erase_batch(bdl_forest *const *forests, int nf, const int32_t *const *ids, const int64_t *n,
                    int64_t *out_n, bdl_stream_t stream) {
  if (nf < 0 || (nf > 0 && (!forests || !ids || !n))) return set_error(BDL_EINVAL, "NULL array");
  if (nf == 0) return BDL_OK;
  if (!forests[0]) {
    if (out_n)
      for (int i = 0; i < nf; ++i) out_n[i] = 0;
    return set_error(BDL_EINVAL, "forest is NULL");
  }
  cudaStream_t s = (cudaStream_t)stream;
  DeviceGuard g(forests[0]->device);
  return finish_many(forests, nf, s, erase_many(forests, nf, ids, n, out_n, s));
}

int bdl_knn(bdl_forest *f, const int32_t *q, int64_t m, int k, int32_t *out_ids, int64_t *out_d2,
            bdl_stream_t stream) {
  return bdl_knn_batch(&f, 1, &q, &m, k, &out_ids, &out_d2, stream);
}

int bdl_knn_batch(bdl_forest *const *forests, int nf, const int32_t *const *q, const int64_t *m, int k,
                  int32_t *const *out_ids, int64_t *const *out_d2, bdl_stream_t stream) {
  if (nf < 0 || (nf > 0 && (!forests || !q || !m || !out_ids || !out_d2)))
    return set_error(BDL_EINVAL, "NULL array");
  if (nf == 0) return BDL_OK;
  if (!forests[0]) return set_error(BDL_EINVAL, "forest is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  DeviceGuard g(forests[0]->device);
  return finish_many(forests, nf, s, knn_many(forests, nf, q, m, k, out_ids, out_d2, s));
}

int bdl_knn_count(bdl_forest *f, const int32_t *q, int64_t m, int k, int32_t *out_ids, int64_t *out_d2,
                  uint64_t *counts_dev, bdl_stream_t stream) {
  if (!f) return set_error(BDL_EINVAL, "forest is NULL");
  if (!counts_dev || ((uintptr_t)counts_dev & 7)) return set_error(BDL_EINVAL, "counts_dev must be an aligned device pointer");
  cudaStream_t s = (cudaStream_t)stream;
  DeviceGuard g(f->device);
  return finish(f, s, knn_many(&f, 1, &q, &m, k, &out_ids, &out_d2, s, (unsigned long long *)counts_dev));
}

int bdl_poll_error(const bdl_forest *f, uint64_t *out_bits, bdl_stream_t stream) {
  if (!f) return set_error(BDL_EINVAL, "forest is NULL");
  DeviceGuard g(f->device);
  cudaStream_t s = (cudaStream_t)stream;
  int st = small_copy(f->pinned_dev + kPinnedErr, f->err, 8, s);
  if (!st) st = cuda_check(cudaStreamSynchronize(s), "sync");
  if (st) return st;
  const uint64_t bits = (uint64_t)f->pinned[kPinnedErr];
  if (out_bits) *out_bits = bits;
  if (bits) return set_error(BDL_EINTERNAL, "device bounds check failed, code " + std::to_string(bits));
  return BDL_OK;
}

int bdl_knn_plan_create(bdl_forest *const *forests, int nf, const int32_t *const *q, const int64_t *m, int k,
                        int32_t *const *out_ids, int64_t *const *out_d2, bdl_stream_t stream,
                        bdl_knn_plan **out) {
  if (!out) return set_error(BDL_EINVAL, "out is NULL");
  *out = nullptr;
  if (nf < 1 || !forests || !q || !m || !out_ids || !out_d2) return set_error(BDL_EINVAL, "NULL array");
  if (!forests[0]) return set_error(BDL_EINVAL, "forest is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  DeviceGuard g(forests[0]->device);
  bdl_knn_plan *P = new bdl_knn_plan();
  int st = knn_plan_make(forests, nf, q, m, k, out_ids, out_d2, s, P);
  if (!st) st = finish_many(forests, nf, s, st);
  if (st) {
    if (P->block) dev_free(P->charge, P->block, P->bytes, s);
    delete P;
    return st;
  }
  *out = P;
  return BDL_OK;
}

int bdl_knn_plan_launch(bdl_knn_plan *plan, bdl_stream_t stream) {
  if (!plan) return set_error(BDL_EINVAL, "plan is NULL");
  DeviceGuard g(plan->device);
  return knn_plan_launch(plan, (cudaStream_t)stream);
}

int bdl_knn_plan_destroy(bdl_knn_plan *plan) {
  if (!plan) return BDL_OK;
  DeviceGuard g(plan->device);
  cudaDeviceSynchronize();   // no launch of the plan may still be running
  if (plan->block) dev_free(plan->charge, plan->block, plan->bytes, 0);
  const int st = cuda_check(cudaStreamSynchronize(0), "sync");
  delete plan;
  return st;
}

int bdl_size(const bdl_forest *f, int64_t *out) {
  if (!f || !out) return set_error(BDL_EINVAL, "NULL pointer");
  *out = f->live;
  return BDL_OK;
}

int bdl_next_id(const bdl_forest *f, int64_t *out) {
  if (!f || !out) return set_error(BDL_EINVAL, "NULL pointer");
  *out = f->next_id;
  return BDL_OK;
}

int bdl_destroy(bdl_forest *f) {
  if (!f) return BDL_OK;
  DeviceGuard g(f->device);
  cudaDeviceSynchronize();
  cudaStream_t s = 0;
  for (int i = 0; i < kMaxLevel; ++i) free_tree(f, f->trees[i], s);
  free_tree(f, f->btree, s);
  for (auto &sp : f->spare)
    if (sp.block) dev_free(f, sp.block, sp.bytes, s);
  if (f->id_cap) {
    dev_free(f, f->idtab, (size_t)f->id_cap * f->dim * 4, s);
    dev_free(f, f->alive, (size_t)f->id_cap / 8, s);
  }
  dev_free(f, f->buf, (size_t)f->cfg.buffer_size * 4, s);
  dev_free(f, f->buf_spare, (size_t)f->cfg.buffer_size * 4, s);
  dev_free(f, f->dev_small, 4096, s);
  if (f->knn_stats) dev_free(f, f->knn_stats, 64, s);
  cudaStreamSynchronize(s);
  if (f->ev_flags) cudaEventDestroy(f->ev_flags);
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

int bdl_set_knn_shape(bdl_forest *f, int block_threads, int queries_per_warp) {
  if (!f) return set_error(BDL_EINVAL, "forest is NULL");
  const int b = block_threads ? block_threads : 128, q = queries_per_warp ? queries_per_warp : 32;
  if (b != 64 && b != 128 && b != 256) return set_error(BDL_EINVAL, "block_threads must be 64, 128 or 256");
  if (q != 32 && q != 64 && q != 128) return set_error(BDL_EINVAL, "queries_per_warp must be 32, 64 or 128");
  f->knn_shape.block = b;
  f->knn_shape.qpw = q;
  return BDL_OK;
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
