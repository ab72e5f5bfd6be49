// erase.cu -- Erase_L (Alg. 4) device work: id bookkeeping, the lazily built
// per-tree bloom filters (Sec. V-A), the per-id descent that finds and
// tombstones each point (Alg. 2), and the ordered gather of the points of the
// trees that fell below half capacity.
//
// GPU design: instead of partitioning the erase batch around every split
// (Alg. 2), each erased id descends on its own -- the composite split key
// gives every point a unique root-to-leaf path -- and marks its leaf entry.
// The collapse of emptied subtrees is kept as per-node live counts, which the
// descent decrements along the path with warp-aggregated atomics.
#include "bdl_internal.cuh"

namespace bdl {

namespace {

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// K6b + K7: for each erased id and each tree (largest first) probe the bloom
// filter (one 32-byte sector); on a hit descend by the composite key to the
// unique leaf, find the id, tombstone it and decrement the live counts along
// the path.  A live id that no tree holds is in the buffer.
// REC: some job keeps its packed k-NN records' live counts (the instance
// without that code is used when none does)
template <bool REC>
__global__ void k_erase_locate(const EraseJob *jobs, const int64_t *job_warp, int njobs) {
  // every warp belongs to one job (one forest's erase list)
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= job_warp[njobs]) return;
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (job_warp[mid] <= w) lo = mid;
    else hi = mid - 1;
  }
  const EraseJob &F = jobs[lo];
  const int lane = threadIdx.x & 31;
  const int64_t i = (w - job_warp[lo]) * 32 + lane;
  const int64_t n = F.n_dev ? min(*F.n_dev, F.n) : F.n;
  bool pending = i < n;
  int32_t id = pending ? F.list[i] : 0;
  const int32_t *xq = F.idtab + (int64_t)id * F.dim;
  int32_t path[kMaxLevel + 2];
  // all bloom probes first: independent 32-byte loads, one per tree
  uint64_t maybe_mask = 0;
  if (pending) {
    for (int ti = 0; ti < F.ntrees; ++ti) {
      const TreeView &T = F.trees[ti];
      bool maybe = true;
      if (T.bloom) {
        int64_t blk;
        uint64_t bits;
        bloom_hash(F.seed, T.bloom_blocks, id, blk, bits);
        const uint4 *bw = reinterpret_cast<const uint4 *>(T.bloom + blk * 8);
        uint4 a = bw[0], b = bw[1];
        uint32_t wv[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
        for (int w = 0; w < 8; ++w) maybe = maybe && (wv[w] & bloom_word_bit(bits, w));
      }
      maybe_mask |= (uint64_t)maybe << ti;
    }
  }
  // Each lane walks its own maybe-trees, largest first, until it finds its
  // id: the lanes of a warp descend different trees at the same time (an id
  // is in one tree; the warp's ids are spread over several).
  bool found = false;
  int fti = 0;            // the tree that held the id
  int64_t leaf_at = 0;    // its leaf's index among that tree's 2^h leaves
  uint64_t mm = pending ? maybe_mask : 0;
  while (mm) {
    const int ti = __ffsll((long long)mm) - 1;
    mm &= mm - 1;
    const TreeView &T = F.trees[ti];
    int v = 0, depth = 0;
    Node nd;
    bool ok = true;
    while (true) {
      path[depth] = v;
      nd = T.node[v];
      if (nd.l < 0) break;
      uint64_t key = comp_key(xq[depth % F.dim], id);
      v = key > nd.key ? nd.r : nd.l;
      depth++;
      if (v < 0 || v >= T.nnodes || depth > T.h) { ok = false; break; }
    }
    const int leaf = -1 - nd.l;
    int a = 0, z = 0;
    if (ok && leaf < ((int64_t)1 << T.h)) {
      a = T.leaf_off[leaf];
      z = T.leaf_off[leaf + 1];
      if (a < 0 || z > T.size || a > z) { a = z = 0; atomicOr(F.err, kErrLeaf); }
    } else {
      atomicOr(F.err, kErrChild);
    }
    const int rs = rec_ints(F.dim);
    for (int j = a; j < z; ++j) {
      int32_t *slot = T.pts + (int64_t)j * rs + F.dim;
      if (*slot == id) {
        *slot = (int32_t)((uint32_t)id | kTomb);
        found = true;
        break;
      }
    }
    if (found) {
      fti = ti;
      leaf_at = leaf;
      break;
    }
  }
  // live counts on the path: the nodes', and (when the job keeps them) the
  // packed k-NN record entries' for the nodes that are entries (depth d >= 1
  // with h - d even: entry (i & 3) of the record two levels up, or (i & 1) of
  // the root's record for d = 1); lanes at the same node of the same tree add
  // up their counts first
  const int fh = found ? F.trees[fti].h : -1;
  const int maxh = __reduce_max_sync(0xffffffffu, fh);
  const int rec = packed_node_ints(F.dim);
  for (int d = 0; d <= maxh; ++d) {
    const bool act = d <= fh;
    const unsigned am = __ballot_sync(0xffffffffu, act);
    if (!act) continue;
    const int v = path[d];
    const unsigned peers = __match_any_sync(am, ((unsigned long long)fti << 32) | (uint32_t)v);
    if (lane == __ffs(peers) - 1) {
      const TreeView &T = F.trees[fti];
      const int cnt = __popc(peers);
      atomicSub(&T.live[v], cnt);
      if (REC && F.records && d >= 1 && ((T.h - d) & 1) == 0) {
        const int e = d == 1 ? 1 : 2;
        const int64_t at = leaf_at >> (T.h - d);   // the node's index at depth d
        const int64_t r = packed_slot(T.h, d - e, at >> e);
        atomicSub(&T.pk[r * rec + 4 + (int)(at & ((1 << e) - 1))], cnt);
      }
    }
  }
}

// Ordered gather, for many forests at once: mark the live ids of the given
// trees in their forest's bitmap, then emit each forest's marked ids in
// increasing order through a prefix sum of per-word popcounts.

// One tree whose live ids are marked in its forest's bitmap.
struct MarkTree {
  const int32_t *pts;
  int64_t size;
  int32_t dim, pad_;
  uint32_t *bm;
};

// One forest's bitmap and output.
struct BitForest {
  const uint32_t *bm;
  int64_t nwords;
  int64_t *bsum;           // [blocks] popcount of each scan block, then its exclusive prefix
  int64_t nb;
  int32_t *out;
  int64_t nout;
  unsigned long long *err;
};

__device__ __forceinline__ int find_pre(const int64_t *pre, int n, int64_t x) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// thread per record of the trees (tree j owns records pre[j] .. pre[j+1]-1)
__global__ void k_mark_ids_many(const MarkTree *t, const int64_t *pre, int nt) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= pre[nt]) return;
  const int j = find_pre(pre, nt, x);
  const MarkTree &T = t[j];
  const int32_t id = T.pts[(x - pre[j]) * rec_ints(T.dim) + T.dim];
  if (id >= 0) atomicOr(&T.bm[id >> 5], 1u << (id & 31));
}

constexpr int kScanBlock = 1024;
constexpr int kScanWords = 4;   // words per thread

__device__ int block_excl_scan(int v, int *tot) {
  __shared__ int ws[33];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int inc = v;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  __syncthreads();
  if (lane == 31) ws[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int nw = blockDim.x >> 5;
    int x = lane < nw ? ws[lane] : 0, xi = x;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, xi, o);
      if (lane >= o) xi += y;
    }
    if (lane < nw) ws[lane] = xi - x;
    if (lane == nw - 1) ws[32] = xi;   // total (nw <= 32)
  }
  __syncthreads();
  int r = inc - v + ws[warp];
  *tot = ws[32];
  return r;
}

// Scan block bb of all forests' bitmaps (forest j owns blocks pre[j] ..
// pre[j+1]-1): its popcount.
__global__ void k_popc_blocks_many(const BitForest *f, const int64_t *pre, int nf) {
  const int j = find_pre(pre, nf, blockIdx.x);
  const BitForest &F = f[j];
  const int64_t b = blockIdx.x - pre[j];
  const int64_t w0 = (b * kScanBlock + threadIdx.x) * kScanWords;
  int c = 0;
  for (int k = 0; k < kScanWords; ++k)
    if (w0 + k < F.nwords) c += __popc(F.bm[w0 + k]);
  int tot;
  block_excl_scan(c, &tot);
  if (threadIdx.x == 0) F.bsum[b] = tot;
}

// One CTA per forest: exclusive prefix of its blocks' popcounts.
__global__ void k_scan_bsum_many(const BitForest *f) {
  __shared__ int64_t carry;
  const BitForest &F = f[blockIdx.x];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t a = 0; a < F.nb; a += blockDim.x) {
    int64_t j = a + threadIdx.x;
    int v = j < F.nb ? (int)F.bsum[j] : 0;
    int tot;
    int e = block_excl_scan(v, &tot);
    if (j < F.nb) F.bsum[j] = carry + e;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
}

// Scan block bb of all forests' bitmaps: its ids, in order, to the forest's output.
__global__ void k_emit_ids_many(const BitForest *f, const int64_t *pre, int nf) {
  const int j = find_pre(pre, nf, blockIdx.x);
  const BitForest &F = f[j];
  const int64_t b = blockIdx.x - pre[j];
  const int64_t w0 = (b * kScanBlock + threadIdx.x) * kScanWords;
  uint32_t wv[kScanWords];
  int c = 0;
  for (int k = 0; k < kScanWords; ++k) {
    wv[k] = w0 + k < F.nwords ? F.bm[w0 + k] : 0u;
    c += __popc(wv[k]);
  }
  int tot;
  int64_t pos = F.bsum[b] + block_excl_scan(c, &tot);
  for (int k = 0; k < kScanWords; ++k) {
    uint32_t x = wv[k];
    while (x) {
      int bt = __ffs(x) - 1;
      if (pos < F.nout) F.out[pos] = (int32_t)(((w0 + k) << 5) + bt);
      else atomicOr(F.err, kErrGather);
      pos++;
      x &= x - 1;
    }
  }
}

}  // namespace

size_t erase_table_bytes(const std::vector<EraseCall> &calls) {
  size_t n = calls.size(), views = 0;
  for (const auto &c : calls) views += (size_t)c.fv->ntrees;
  return n * sizeof(EraseJob) + (n + 1) * 8 + views * sizeof(TreeView) + 64;
}

int launch_erase_jobs(const std::vector<EraseCall> &calls, void *table,
                      cudaStream_t s) {
  const size_t n = calls.size();
  std::vector<unsigned char> img(erase_table_bytes(calls));
  EraseJob *jobs = (EraseJob *)img.data();
  int64_t *warp = (int64_t *)(img.data() + n * sizeof(EraseJob));
  const size_t views_off = n * sizeof(EraseJob) + (n + 1) * 8;
  TreeView *views = (TreeView *)(img.data() + views_off);
  size_t v = 0;
  warp[0] = 0;
  for (size_t j = 0; j < n; ++j) {
    const EraseCall &c = calls[j];
    EraseJob &J = jobs[j];
    memset(&J, 0, sizeof(J));
    J.trees = (const TreeView *)((char *)table + views_off) + v;
    J.ntrees = c.fv->ntrees;
    J.dim = c.fv->dim;
    J.idtab = c.fv->idtab;
    J.err = c.fv->err;
    J.list = c.list;
    J.seed = c.seed;
    J.n = c.fv->ntrees ? c.n : 0;
    J.n_dev = c.n_dev;
    J.records = c.records;
    for (int t = 0; t < c.fv->ntrees; ++t) views[v++] = c.fv->tree[t];
    warp[j + 1] = warp[j] + (J.n + 31) / 32;
  }
  if (warp[n] == 0) return BDL_OK;
  int st = h2d(table, img.data(), img.size(), s);
  if (st) return st;
  bool rec = false;
  for (const auto &c : calls) rec = rec || c.records;
  // algorithmic bytes per erased id: its coordinates (4d), one 32-byte bloom
  // block per tree, and the descent of the tree that holds it -- one 16-byte
  // node per level and its leaf's records -- weighted by the trees' sizes
  // (the ids of a batch are spread over the trees in proportion to them);
  // the batch length stands for the count of ids the alive filter keeps
  double eb = 0;
  for (const auto &c : calls) {
    const ForestView &fv = *c.fv;
    double tot = 0, desc = 0;
    for (int t = 0; t < fv.ntrees; ++t) tot += (double)fv.tree[t].size;
    for (int t = 0; t < fv.ntrees && tot > 0; ++t) {
      const TreeView &T = fv.tree[t];
      const double leaf = (double)T.size / (double)((int64_t)1 << T.h);
      desc += (double)T.size / tot * (16.0 * (T.h + 1) + 4.0 * rec_ints(fv.dim) * leaf);
    }
    eb += (double)(fv.ntrees ? c.n : 0) * (4.0 * fv.dim + 32.0 * fv.ntrees + desc);
  }
  KScope ks_(kK_erase_locate, s, eb);
  const unsigned grid = (unsigned)cdiv(warp[n] * 32, 128);
  const EraseJob *djobs = (const EraseJob *)table;
  const int64_t *jw = (const int64_t *)((char *)table + n * sizeof(EraseJob));
  if (rec)
    k_erase_locate<true><<<grid, 128, 0, s>>>(djobs, jw, (int)n);
  else
    k_erase_locate<false><<<grid, 128, 0, s>>>(djobs, jw, (int)n);
  return cuda_check(cudaGetLastError(), "erase kernel");
}

int collect_sorted_live(const std::vector<LiveCollect> &jobs, cudaStream_t s) {
  std::vector<BitForest> bf;
  std::vector<MarkTree> mt;
  std::vector<int64_t> fpre{0}, tpre{0};
  size_t bytes = 0;
  for (const auto &J : jobs) {
    if (J.n <= 0) continue;
    const int64_t nwords = (J.f->next_id + 31) >> 5;
    const int64_t nb = cdiv(nwords, (int64_t)kScanBlock * kScanWords);
    bytes += ((size_t)nwords * 4 + 255) / 256 * 256 + ((size_t)nb * 8 + 255) / 256 * 256;
  }
  if (bytes == 0) return BDL_OK;
  bdl_forest *charge = nullptr;
  for (const auto &J : jobs)
    if (J.n > 0) { charge = J.f; break; }
  void *blk = nullptr;
  int st = dev_alloc(charge, &blk, bytes, s);
  if (st) return st;
  char *p = (char *)blk;
  size_t bm_bytes = 0;
  for (const auto &J : jobs) {
    if (J.n <= 0) continue;
    const int64_t nwords = (J.f->next_id + 31) >> 5;
    const int64_t nb = cdiv(nwords, (int64_t)kScanBlock * kScanWords);
    BitForest F;
    F.bm = (const uint32_t *)p;
    p += ((size_t)nwords * 4 + 255) / 256 * 256;
    bm_bytes = (size_t)(p - (char *)blk);
    F.nwords = nwords;
    F.bsum = nullptr;
    F.nb = nb;
    F.out = J.out;
    F.nout = J.n;
    F.err = J.f->err;
    for (Tree *t : J.trees) {
      mt.push_back(MarkTree{t->pts, t->size, J.f->dim, 0, (uint32_t *)F.bm});
      tpre.push_back(tpre.back() + t->size);
    }
    bf.push_back(F);
    fpre.push_back(fpre.back() + nb);
  }
  for (auto &F : bf) {   // the block sums after all bitmaps
    F.bsum = (int64_t *)p;
    p += ((size_t)F.nb * 8 + 255) / 256 * 256;
  }
  // tables: [MarkTree][tree prefix][BitForest][block prefix]
  std::vector<unsigned char> img;
  auto put = [&](const void *src, size_t n) {
    size_t off = (img.size() + 255) / 256 * 256;
    img.resize(off + std::max<size_t>(n, 8));
    memcpy(img.data() + off, src, n);
    return off;
  };
  const size_t o_mt = put(mt.data(), mt.size() * sizeof(MarkTree)), o_tp = put(tpre.data(), tpre.size() * 8),
               o_bf = put(bf.data(), bf.size() * sizeof(BitForest)), o_fp = put(fpre.data(), fpre.size() * 8);
  void *tab = nullptr;
  st = dev_alloc(charge, &tab, img.size(), s);
  if (st) {
    dev_free(charge, blk, bytes, s);
    return st;
  }
  st = h2d(tab, img.data(), img.size(), s);
  if (!st) st = small_zero(blk, bm_bytes, s);
  const char *T = (const char *)tab;
  const int nt = (int)mt.size(), nf = (int)bf.size();
  if (!st && tpre.back() > 0) {
    KScope ks_(kK_mark_ids, s);
    k_mark_ids_many<<<(unsigned)cdiv(tpre.back(), 256), 256, 0, s>>>((const MarkTree *)(T + o_mt),
                                                                     (const int64_t *)(T + o_tp), nt);
  }
  if (!st) {
    { KScope ks_(kK_popc_blocks, s);
      k_popc_blocks_many<<<(unsigned)fpre.back(), kScanBlock, 0, s>>>((const BitForest *)(T + o_bf),
                                                                      (const int64_t *)(T + o_fp), nf); }
    { KScope ks_(kK_scan_bsum, s);
      k_scan_bsum_many<<<(unsigned)nf, 1024, 0, s>>>((const BitForest *)(T + o_bf)); }
    { KScope ks_(kK_emit_ids, s);
      k_emit_ids_many<<<(unsigned)fpre.back(), kScanBlock, 0, s>>>((const BitForest *)(T + o_bf),
                                                                   (const int64_t *)(T + o_fp), nf); }
  }
  if (!st) st = cuda_check(cudaGetLastError(), "collect_sorted_live");
  dev_free(charge, tab, img.size(), s);
  dev_free(charge, blk, bytes, s);
  return st;
}

}  // namespace bdl

// ---------------------------------------------------------------------------
// Table-driven helpers: one launch serves many forests (or trees).  Each
// table entry owns a contiguous range of the launch's work items; a thread
// finds its entry by binary search over the range prefix.
// ---------------------------------------------------------------------------

namespace bdl {

namespace {

__device__ __forceinline__ int seg_find(const int64_t *pre, int n, int64_t x) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int32_t pool_entry(const FillSeg &g, int64_t k) {
  if (k < g.nbuf) return g.buf[k];
  return g.arr ? g.arr[k - g.nbuf] : (int32_t)(g.first + (k - g.nbuf));
}

__global__ void k_fill_many(const FillSeg *segs, const int64_t *pre, int nseg) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= pre[nseg]) return;
  const int j = seg_find(pre, nseg, x);
  const FillSeg &g = segs[j];
  const int64_t i = x - pre[j];
  switch (g.kind) {
    case kFillAppend: {            // copy coordinates into the id table, check the grid
      const int32_t v = g.src[i];
      // an off-grid value is flagged and stored clamped, so that work started
      // before the flag is read back only ever sees grid coordinates
      g.dst[i] = min(max(v, 0), (1 << kCoordBits) - 1);
      if (v < 0 || v >= (1 << kCoordBits)) atomicOr(g.flag, 1ull);
      if (i == 0 && g.errw && *g.errw) atomicOr(g.flag, 2ull | (*g.errw << 8));   // with the word's bits
      break;
    }
    case kFillPoolTail: g.dst[i] = pool_entry(g, g.from + i); break;
    case kFillIota: g.dst[i] = (int32_t)(g.first + i); break;
    case kFillZero: g.dst[i] = 0; break;
    case kFillAlive: {   // consecutive ids: the lanes on one word OR their bits first
      const int64_t id = g.first + i;
      uint32_t *wd = &g.alive[id >> 5];
      const unsigned peers = __match_any_sync(__activemask(), (unsigned long long)wd);
      const unsigned bits = __reduce_or_sync(peers, 1u << (id & 31));
      if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicOr(wd, bits);
      break;
    }
  }
}

// Erase marking for many forests: entries are warp-aligned, so the warp's
// aggregated append stays inside one forest's list.
__global__ void k_erase_mark_many(const MarkSeg *segs, const int64_t *pre_warp, int nseg) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= pre_warp[nseg]) return;
  const int j = seg_find(pre_warp, nseg, w);
  const MarkSeg &g = segs[j];
  const int lane = threadIdx.x & 31;
  const int64_t i = (w - pre_warp[j]) * 32 + lane;
  bool own = false;
  int32_t id = -1;
  if (i < g.n) {
    id = g.ids[i];
    if (id >= 0 && id < g.next_id) {
      const uint32_t bit = 1u << (id & 31);
      own = (atomicAnd(&g.alive[id >> 5], ~bit) & bit) != 0;
    }
  }
  const unsigned m = __ballot_sync(0xffffffffu, own);
  if (!m) return;
  unsigned long long base = 0;
  if (lane == __ffs(m) - 1) {
    base = atomicAdd((unsigned long long *)g.count, (unsigned long long)__popc(m));
    if (g.total != g.count) atomicAdd((unsigned long long *)g.total, (unsigned long long)__popc(m));
  }
  base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
  if (own) g.list[base + __popc(m & ((1u << lane) - 1))] = id;
}

__global__ void k_bloom_build_many(const TreeSeg *segs, const int64_t *pre, int nseg) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= pre[nseg]) return;
  const int j = seg_find(pre, nseg, x);
  const TreeSeg &g = segs[j];
  if (g.gate && *g.gate == 0) return;   // its forest's batch erased nothing
  const int32_t id = g.pts[(x - pre[j]) * rec_ints(g.dim) + g.dim];
  if (id < 0) return;
  int64_t blk;
  uint64_t bits;
  bloom_hash(g.seed, g.blocks, id, blk, bits);
  // the block's eight words as four 64-bit halves: four atomics per key
  unsigned long long *b64 = reinterpret_cast<unsigned long long *>(g.bloom + blk * 8);
  for (int w = 0; w < 4; ++w)
    atomicOr(&b64[w], (unsigned long long)bloom_word_bit(bits, 2 * w) |
                          ((unsigned long long)bloom_word_bit(bits, 2 * w + 1) << 32));
}

// One thread per packed k-NN record of many trees (pre[j] .. pre[j+1]-1 are
// tree j's records in level order): its entries' live counts from the nodes'.
// With segs[j].err set, compare instead of copy and flag a difference (the
// erase keeps both up to date; this is the debug check of that).
__global__ void k_pack_lives_many(const TreeSeg *segs, const int64_t *pre, int nseg) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= pre[nseg]) return;
  const int j = seg_find(pre, nseg, x);
  const TreeSeg &g = segs[j];
  int t;
  int64_t i;
  packed_record_of(g.h, x - pre[j], t, i);   // the record's node, and its entries two levels
  const int st = packed_step(g.h, t);        // down (one for an odd tree's root)
  int4 lv = make_int4(0, 0, 0, 0);
  lv.x = g.live[veb_slot(g.h + 1, t + st, (i << st) + 0)];
  lv.y = g.live[veb_slot(g.h + 1, t + st, (i << st) + 1)];
  if (st == 2) {
    lv.z = g.live[veb_slot(g.h + 1, t + st, (i << st) + 2)];
    lv.w = g.live[veb_slot(g.h + 1, t + st, (i << st) + 3)];
  }
  int4 *dst = reinterpret_cast<int4 *>(g.pk + packed_slot(g.h, t, i) * packed_node_ints(g.dim) + 4);
  if (!g.err) {
    *dst = lv;
  } else {
    const int4 have = *dst;
    if (have.x != lv.x || have.y != lv.y || have.z != lv.z || have.w != lv.w) atomicOr(g.err, kErrLiveCount);
  }
}

// One CTA per forest: keep its buffer ids that are still alive, in order;
// then the live counts of its tree roots.
__global__ void k_buffer_compact_many(const BufSeg *segs) {
  __shared__ int wsum[32];
  __shared__ int base;
  const BufSeg &g = segs[blockIdx.x];
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t a = 0; a < g.nbuf; a += blockDim.x) {
    const int64_t j = a + threadIdx.x;
    const int32_t id = j < g.nbuf ? g.buf[j] : -1;
    const bool keep = j < g.nbuf && ((g.alive[id >> 5] >> (id & 31)) & 1);
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) wsum[warp] = __popc(m);
    __syncthreads();
    int pre = 0, tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      if (w < warp) pre += wsum[w];
      tot += wsum[w];
    }
    const int dst = base + pre + __popc(m & ((1u << lane) - 1));
    __syncthreads();
    if (keep) g.buf[dst] = id;
    __syncthreads();
    if (threadIdx.x == 0) base += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    g.out[0] = base;
    g.out[kMaxLevel + 1] = g.errw ? (int64_t)*g.errw : 0;
  }
  for (int t = threadIdx.x; t < g.ntrees; t += blockDim.x) g.out[1 + t] = g.roots[t][0];
}

template <class T>
int upload_table(const std::vector<T> &segs, const std::vector<int64_t> &pre, void *dev,
                 cudaStream_t s) {
  std::vector<unsigned char> img(table_bytes(segs.size(), sizeof(T)));
  memcpy(img.data(), segs.data(), segs.size() * sizeof(T));
  memcpy(img.data() + (segs.size() * sizeof(T) + 255) / 256 * 256, pre.data(), pre.size() * 8);
  return h2d(dev, img.data(), img.size(), s);
}

template <class T>
const int64_t *table_pre(const std::vector<T> &segs, const void *dev) {
  return (const int64_t *)((const char *)dev + (segs.size() * sizeof(T) + 255) / 256 * 256);
}

}  // namespace

size_t table_bytes(size_t nseg, size_t seg_size) {
  return (nseg * seg_size + 255) / 256 * 256 + (nseg + 1) * 8 + 64;
}

int launch_fill_many(const std::vector<FillSeg> &segs, void *table, cudaStream_t s) {
  std::vector<int64_t> pre(segs.size() + 1, 0);
  for (size_t j = 0; j < segs.size(); ++j) pre[j + 1] = pre[j] + segs[j].count;
  if (pre.back() == 0) return BDL_OK;
  int st = upload_table(segs, pre, table, s);
  if (st) return st;
  KScope ks_(kK_fill, s);
  k_fill_many<<<(unsigned)cdiv(pre.back(), 256), 256, 0, s>>>((const FillSeg *)table,
                                                               table_pre(segs, table), (int)segs.size());
  return cuda_check(cudaGetLastError(), "fill kernel");
}

int launch_erase_mark_many(const std::vector<MarkSeg> &segs, void *table, cudaStream_t s) {
  std::vector<int64_t> pre(segs.size() + 1, 0);
  for (size_t j = 0; j < segs.size(); ++j) pre[j + 1] = pre[j] + (segs[j].n + 31) / 32;
  if (pre.back() == 0) return BDL_OK;
  int st = upload_table(segs, pre, table, s);
  if (st) return st;
  KScope ks_(kK_erase_mark, s);
  k_erase_mark_many<<<(unsigned)cdiv(pre.back() * 32, 256), 256, 0, s>>>(
      (const MarkSeg *)table, table_pre(segs, table), (int)segs.size());
  return cuda_check(cudaGetLastError(), "erase mark kernel");
}

int launch_bloom_build_many(const std::vector<TreeSeg> &segs, void *table,
                            cudaStream_t s) {
  std::vector<int64_t> pre(segs.size() + 1, 0);
  for (size_t j = 0; j < segs.size(); ++j) pre[j + 1] = pre[j] + segs[j].size;
  if (pre.back() == 0) return BDL_OK;
  int st = upload_table(segs, pre, table, s);
  if (st) return st;
  // algorithmic bytes per point: its id and one 32-byte block
  KScope ks_(kK_bloom_build, s, (double)pre.back() * 36.0);
  k_bloom_build_many<<<(unsigned)cdiv(pre.back(), 256), 256, 0, s>>>(
      (const TreeSeg *)table, table_pre(segs, table), (int)segs.size());
  return cuda_check(cudaGetLastError(), "bloom kernel");
}

int launch_pack_lives_many(const std::vector<TreeSeg> &segs, void *table, cudaStream_t s) {
  std::vector<int64_t> pre(segs.size() + 1, 0);
  for (size_t j = 0; j < segs.size(); ++j) pre[j + 1] = pre[j] + packed_nrec(segs[j].h);
  if (pre.back() == 0) return BDL_OK;
  int st = upload_table(segs, pre, table, s);
  if (st) return st;
  KScope ks_(kK_pack_lives, s);
  k_pack_lives_many<<<(unsigned)cdiv(pre.back(), 256), 256, 0, s>>>(
      (const TreeSeg *)table, table_pre(segs, table), (int)segs.size());
  return cuda_check(cudaGetLastError(), "pack lives kernel");
}

int launch_buffer_compact_many(const std::vector<BufSeg> &segs, void *table, cudaStream_t s) {
  if (segs.empty()) return BDL_OK;
  std::vector<int64_t> pre(segs.size() + 1, 0);
  int st = upload_table(segs, pre, table, s);
  if (st) return st;
  KScope ks_(kK_buffer_compact, s);
  k_buffer_compact_many<<<(unsigned)segs.size(), 1024, 0, s>>>((const BufSeg *)table);
  return cuda_check(cudaGetLastError(), "buffer compact kernel");
}

}  // namespace bdl
