// spatial.cu -- construction of the static kd-trees of one Insert_L with the
// spatial-median splitting rule of Sec. V-C: a node splits its points at the
// midpoint v = floor((min + max) / 2) of their coordinates in its dimension,
// points with coordinate <= v to the left (reading G12).  The trees keep the
// shape of the object-median trees (h split levels, nodes in vEB slots), so
// queries and erases run on them unchanged; only the build differs.
//
// GPU design: the sizes of a node's children now depend on the data, so the
// build carries each segment's bounds in arrays instead of closed form.  All
// new trees of one dimension advance level by level together; the trees are
// ordered by height, so the trees still splitting at level t are a prefix of
// that order and so are their records in the staging buffer.  A record's
// segment at level t is s = j * 2^t + i (tree j, node i of depth t), and its
// child's is 2s or 2s + 1.  Per level:
//   k_sp_minmax  -- min and max of the split coordinate per segment (block-,
//                   then warp-aggregated atomics), for the first level only;
//   k_sp_scatter -- left records fill the child's range from its start, right
//                   ones from its end (aggregated atomic cursors); records of
//                   a tree whose children are leaves go straight to the tree;
//                   the others also give their child segment's min and max of
//                   the next level's split coordinate, so that level needs no
//                   pass of its own;
//   k_sp_split   -- the node's key and children, the children's bounds, and
//                   the leaf offsets of trees that end here.
// Order inside a child is not kept (the sets are what the rule fixes).  Then
// leaf boxes, boxes bottom-up and the packed k-NN records.
#include "bdl_internal.cuh"

#include <algorithm>
#include <numeric>

namespace bdl {

namespace {

constexpr int kT = 256;   // threads per block of the record passes

struct SpTree {           // one tree of a spatial build, as the kernels see it
  Node *node;
  int32_t *box, *live, *leaf_off, *pts;
  int64_t toff, size;     // first staging position, points
  int64_t from_cleared;   // records that come from cleared trees (first in the tree)
  int32_t h, pad_;
  unsigned long long *err;
};

struct SpGather {         // one source of a tree's points
  const int32_t *src;     // a cleared tree's records (live ones move), or nullptr: a pool chunk
  int64_t count;
  const int32_t *pbuf;    // pool chunk: the forest's pool (sorted buffer ids, then ids)
  int64_t pnbuf;
  const int32_t *parr;
  int64_t pfirst, pool_lo;
  const int32_t *idtab;
  int64_t dst0;           // pool chunk: first position inside its tree
  int32_t tree, pad_;
};

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
size_t al256(size_t x) { return (x + 255) / 256 * 256; }

__device__ __forceinline__ int find_entry(const int64_t *pre, int n, int64_t x) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void copy_rec(int32_t *dst, const int32_t *src, int rs) {
  for (int c = 0; c < rs; c += 4)
    *reinterpret_cast<int4 *>(dst + c) = *reinterpret_cast<const int4 *>(src + c);
}

// Gather: the live records of the cleared trees (any order) and the pool
// chunks (in order behind them) into staging -- or, for a tree that is a
// single leaf, straight into the tree.  Level-0 segment of a record = its tree.
__global__ void k_sp_gather(const SpGather *G, const int64_t *pre, int ng, const SpTree *T, int dim,
                            int32_t *stg, int32_t *seg, unsigned long long *cursor) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool act = x < pre[ng];
  const int j = act ? find_entry(pre, ng, x) : 0;
  const SpGather &g = G[j];
  const int64_t i = x - pre[j];
  const int rs = rec_ints(dim);
  int32_t r[rec_ints(kMaxDim)];
  bool keep = false;
  int tree = g.tree;
  if (act) {
    if (g.src) {
      const int32_t *src = g.src + i * rs;
      for (int c = 0; c < rs; ++c) r[c] = src[c];
      keep = r[dim] >= 0;               // tombstoned records stay behind
    } else {
      const int64_t k = g.pool_lo + i;
      const int32_t id = k < g.pnbuf ? g.pbuf[k] : (g.parr ? g.parr[k - g.pnbuf] : (int32_t)(g.pfirst + (k - g.pnbuf)));
      for (int c = 0; c < rs; ++c) r[c] = 0;
      for (int c = 0; c < dim; ++c) r[c] = g.idtab[(int64_t)id * dim + c];
      r[dim] = id;
      keep = true;
    }
  }
  // positions: cleared records take the next free slot of their tree (warp-
  // aggregated per tree), pool records a fixed slot after them
  int64_t pos = 0;
  const bool from_cleared = act && keep && g.src;
  const unsigned cm = __ballot_sync(0xffffffffu, from_cleared);
  if (from_cleared) {
    const unsigned peers = __match_any_sync(cm, tree);
    const int leader = __ffs(peers) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(&cursor[tree], (unsigned long long)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    pos = (int64_t)base + __popc(peers & ((1u << lane) - 1));
  } else if (act && keep) {
    pos = g.dst0 + i;
  }
  if (!(act && keep)) return;
  const SpTree &tr = T[tree];
  if (pos < 0 || pos >= (g.src ? tr.from_cleared : tr.size)) {
    atomicOr(tr.err, kErrGather);
    return;
  }
  if (tr.h == 0) {
    for (int c = 0; c < rs; c += 4)
      *reinterpret_cast<int4 *>(tr.pts + pos * rs + c) = make_int4(r[c], r[c + 1], r[c + 2], r[c + 3]);
  } else {
    const int64_t p = tr.toff + pos;
    for (int c = 0; c < rs; c += 4)
      *reinterpret_cast<int4 *>(stg + p * rs + c) = make_int4(r[c], r[c + 1], r[c + 2], r[c + 3]);
    seg[p] = tree;
  }
}

// Level-0 bounds of every splitting tree; the leaf-offset sentinels; the
// single leaf of a tree with h = 0.
__global__ void k_sp_roots(const SpTree *T, int ntree, int64_t *lo, int32_t *n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ntree) return;
  const SpTree &tr = T[j];
  tr.leaf_off[(int64_t)1 << tr.h] = (int32_t)tr.size;
  if (tr.h == 0) {
    tr.leaf_off[0] = 0;
    tr.node[0] = Node{0, -1, 0};
  } else {
    lo[j] = tr.toff;
    n[j] = (int32_t)tr.size;
  }
}

// Cursors of the N segments of this level; empty bounds for the Nb segments
// whose min and max are gathered next (by k_sp_minmax or by the scatter).
__global__ void k_sp_level_init(int64_t N, uint32_t *curL, uint32_t *curR, int64_t Nb, int32_t *mn,
                                int32_t *mx) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < N) {
    curL[s] = 0;
    curR[s] = 0;
  }
  if (s < Nb) {
    mn[s] = INT32_MAX;
    mx[s] = INT32_MIN;
  }
}

__global__ void __launch_bounds__(kT) k_sp_minmax(const int32_t *stg, const int32_t *seg, int64_t A, int rs,
                                                  int c, int32_t *mn, int32_t *mx) {
  __shared__ int32_t s_mn[kT / 32], s_mx[kT / 32];
  const int64_t p0 = (int64_t)blockIdx.x * kT;
  const int64_t p = p0 + threadIdx.x;
  const bool act = p < A;
  const int s = act ? seg[p] : -1;
  const int32_t x = act ? stg[p * rs + c] : 0;
  const int s0 = seg[p0];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int32_t xl = act ? x : INT32_MAX, xh = act ? x : INT32_MIN;
  if (__syncthreads_and(!act || s == s0)) {
    // the whole block in one segment: one atomic pair
    const int32_t wl = __reduce_min_sync(0xffffffffu, xl), wh = __reduce_max_sync(0xffffffffu, xh);
    if (lane == 0) {
      s_mn[warp] = wl;
      s_mx[warp] = wh;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int32_t a = s_mn[0], b = s_mx[0];
      for (int w = 1; w < kT / 32; ++w) {
        a = min(a, s_mn[w]);
        b = max(b, s_mx[w]);
      }
      atomicMin(&mn[s0], a);
      atomicMax(&mx[s0], b);
    }
    return;
  }
  const int ws = __shfl_sync(0xffffffffu, s, 0);
  if (__all_sync(0xffffffffu, !act || s == ws)) {
    const int32_t wl = __reduce_min_sync(0xffffffffu, xl), wh = __reduce_max_sync(0xffffffffu, xh);
    if (lane == 0 && ws >= 0) {
      atomicMin(&mn[ws], wl);
      atomicMax(&mx[ws], wh);
    }
    return;
  }
  if (act) {
    atomicMin(&mn[s], x);
    atomicMax(&mx[s], x);
  }
}

// Left records fill [lo, lo + nl) from the start, right ones [lo + nl, lo + m)
// from the end, so neither side needs the other's count first.
__global__ void __launch_bounds__(kT) k_sp_scatter(const int32_t *stg, const int32_t *seg, int64_t A, int dim,
                                                   int c, int t, const int32_t *mn, const int32_t *mx,
                                                   const int64_t *lo, const int32_t *n, uint32_t *curL,
                                                   uint32_t *curR, const SpTree *T, int32_t *stg_out,
                                                   int32_t *seg_out, int32_t *mn_next, int32_t *mx_next) {
  __shared__ uint32_t s_cnt[2][kT / 32];
  __shared__ uint32_t s_base[2];
  __shared__ int32_t s_bnd[4][kT / 32];   // per warp: left min, left max, right min, right max
  const int rs = rec_ints(dim);
  const int64_t p0 = (int64_t)blockIdx.x * kT;
  const int64_t p = p0 + threadIdx.x;
  const bool act = p < A;
  const int s = act ? seg[p] : -1;
  const int s0 = seg[p0];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int32_t x = act ? stg[p * rs + c] : 0;
  const bool left = act && x <= ((act ? mn[s] + mx[s] : 0) >> 1);
  const bool right = act && !left;
  const unsigned lt_mask = (1u << lane) - 1;
  // the next level's split coordinate, for the records whose children split on
  const int cn = (t + 1) % dim;
  const bool more = act && t + 2 <= T[s >> t].h;
  const int32_t xn = more ? stg[p * rs + cn] : 0;
  uint32_t rank = 0;
  if (__syncthreads_and(!act || s == s0)) {
    const unsigned bl = __ballot_sync(0xffffffffu, left), br = __ballot_sync(0xffffffffu, right);
    const int32_t lmn = __reduce_min_sync(0xffffffffu, more && left ? xn : INT32_MAX);
    const int32_t lmx = __reduce_max_sync(0xffffffffu, more && left ? xn : INT32_MIN);
    const int32_t rmn = __reduce_min_sync(0xffffffffu, more && right ? xn : INT32_MAX);
    const int32_t rmx = __reduce_max_sync(0xffffffffu, more && right ? xn : INT32_MIN);
    if (lane == 0) {
      s_cnt[0][warp] = __popc(bl);
      s_cnt[1][warp] = __popc(br);
      s_bnd[0][warp] = lmn;
      s_bnd[1][warp] = lmx;
      s_bnd[2][warp] = rmn;
      s_bnd[3][warp] = rmx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t tl = 0, tr = 0;
      int32_t a0 = INT32_MAX, a1 = INT32_MIN, a2 = INT32_MAX, a3 = INT32_MIN;
      for (int w = 0; w < kT / 32; ++w) {
        const uint32_t a = s_cnt[0][w], b = s_cnt[1][w];
        s_cnt[0][w] = tl;
        s_cnt[1][w] = tr;
        tl += a;
        tr += b;
        a0 = min(a0, s_bnd[0][w]);
        a1 = max(a1, s_bnd[1][w]);
        a2 = min(a2, s_bnd[2][w]);
        a3 = max(a3, s_bnd[3][w]);
      }
      s_base[0] = tl ? atomicAdd(&curL[s0], tl) : 0;
      s_base[1] = tr ? atomicAdd(&curR[s0], tr) : 0;
      if (a0 <= a1) {
        atomicMin(&mn_next[2 * s0], a0);
        atomicMax(&mx_next[2 * s0], a1);
      }
      if (a2 <= a3) {
        atomicMin(&mn_next[2 * s0 + 1], a2);
        atomicMax(&mx_next[2 * s0 + 1], a3);
      }
    }
    __syncthreads();
    rank = left ? s_base[0] + s_cnt[0][warp] + __popc(bl & lt_mask)
                : s_base[1] + s_cnt[1][warp] + __popc(br & lt_mask);
  } else {
    // groups of lanes with the same (segment, side)
    const int key = act ? 2 * s + (left ? 0 : 1) : -1 - lane;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (act && lane == leader) base = atomicAdd(left ? &curL[s] : &curR[s], (uint32_t)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    rank = base + __popc(peers & lt_mask);
    // the group's bounds of the next coordinate (every lane of a group is in
    // the same tree, so `more` is the same for all of them)
    const int32_t gmn = __reduce_min_sync(peers, more ? xn : INT32_MAX);
    const int32_t gmx = __reduce_max_sync(peers, more ? xn : INT32_MIN);
    if (more && lane == leader) {
      atomicMin(&mn_next[2 * s + (left ? 0 : 1)], gmn);
      atomicMax(&mx_next[2 * s + (left ? 0 : 1)], gmx);
    }
  }
  if (!act) return;
  const int j = s >> t;
  const SpTree &tr = T[j];
  const int64_t m = n[s];
  if ((int64_t)rank >= m) {
    atomicOr(tr.err, kErrPartition);
    return;
  }
  const int64_t pos = left ? lo[s] + rank : lo[s] + m - 1 - rank;
  if (t + 1 == tr.h) {                    // the children are leaves: into the tree
    copy_rec(tr.pts + (pos - tr.toff) * rs, stg + p * rs, rs);
  } else {
    copy_rec(stg_out + pos * rs, stg + p * rs, rs);
    seg_out[pos] = 2 * s + (left ? 0 : 1);
  }
}

// Per segment: the node's key and children, the children's bounds for the
// next level, or the leaves' offsets and records when the children are leaves.
__global__ void k_sp_split(int t, int64_t N, const int32_t *mn, const int32_t *mx, const int64_t *lo,
                           const int32_t *n, const uint32_t *curL, const uint32_t *curR, const SpTree *T,
                           int64_t *lo_next, int32_t *n_next) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  const int j = (int)(s >> t);
  const int64_t i = s & (((int64_t)1 << t) - 1);
  const SpTree &tr = T[j];
  const int64_t m = n[s];
  const int64_t nl = curL[s];
  if (nl + (int64_t)curR[s] != m) atomicOr(tr.err, kErrPartition);
  const int64_t v = m > 0 ? ((int64_t)mn[s] + (int64_t)mx[s]) >> 1 : 0;
  const int l = tr.h + 1;
  const int64_t cl = veb_slot(l, t + 1, 2 * i), cr = veb_slot(l, t + 1, 2 * i + 1);
  tr.node[veb_slot(l, t, i)] = Node{(uint64_t)((v << 31) | 0x7FFFFFFF), (int32_t)cl, (int32_t)cr};
  if (t + 1 == tr.h) {
    tr.leaf_off[2 * i] = (int32_t)(lo[s] - tr.toff);
    tr.leaf_off[2 * i + 1] = (int32_t)(lo[s] + nl - tr.toff);
    tr.node[cl] = Node{0, (int32_t)(-1 - 2 * i), 0};
    tr.node[cr] = Node{0, (int32_t)(-2 - 2 * i), 0};
  } else {
    lo_next[2 * s] = lo[s];
    n_next[2 * s] = (int32_t)nl;
    lo_next[2 * s + 1] = lo[s] + nl;
    n_next[2 * s + 1] = (int32_t)(m - nl);
  }
}

// Box and live count of every leaf (one thread per leaf; an empty leaf gets
// the empty box [INT32_MAX, INT32_MIN]).
__global__ void k_sp_leaf_box(const SpTree *T, const int64_t *pre, int ntree, int dim) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= pre[ntree]) return;
  const int j = find_entry(pre, ntree, x);
  const SpTree &tr = T[j];
  const int64_t leaf = x - pre[j];
  const int rs = rec_ints(dim);
  int32_t lo[kMaxDim], hi[kMaxDim];
  for (int c = 0; c < dim; ++c) {
    lo[c] = INT32_MAX;
    hi[c] = INT32_MIN;
  }
  const int64_t a = tr.leaf_off[leaf], b = tr.leaf_off[leaf + 1];
  if (a < 0 || b > tr.size || a > b) {
    atomicOr(tr.err, kErrLeaf);
    return;
  }
  for (int64_t r = a; r < b; ++r)
    for (int c = 0; c < dim; ++c) {
      const int32_t v = tr.pts[r * rs + c];
      lo[c] = min(lo[c], v);
      hi[c] = max(hi[c], v);
    }
  const int64_t v = veb_slot(tr.h + 1, tr.h, leaf);
  for (int c = 0; c < dim; ++c) {
    tr.box[v * 2 * dim + c] = lo[c];
    tr.box[v * 2 * dim + dim + c] = hi[c];
  }
  tr.live[v] = (int32_t)(b - a);
}

// Boxes and live counts of the nodes of depth t from their children.
__global__ void k_sp_box_up(const SpTree *T, int t, int64_t N, int dim) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  const int j = (int)(s >> t);
  const int64_t i = s & (((int64_t)1 << t) - 1);
  const SpTree &tr = T[j];
  const int l = tr.h + 1;
  const int64_t v = veb_slot(l, t, i), a = veb_slot(l, t + 1, 2 * i), b = veb_slot(l, t + 1, 2 * i + 1);
  for (int c = 0; c < dim; ++c) {
    tr.box[v * 2 * dim + c] = min(tr.box[a * 2 * dim + c], tr.box[b * 2 * dim + c]);
    tr.box[v * 2 * dim + dim + c] = max(tr.box[a * 2 * dim + dim + c], tr.box[b * 2 * dim + dim + c]);
  }
  tr.live[v] = tr.live[a] + tr.live[b];
}

}  // namespace

int build_trees_spatial(bdl_forest *af, int dim, std::vector<BuildTree> &bt, const std::vector<ClearedSrc> &cl,
                        cudaStream_t s) {
  if (bt.empty()) return BDL_OK;
  const int ntree = (int)bt.size();
  // trees by height, tallest first: the trees still splitting at a level are a prefix
  std::vector<int> order(ntree);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return bt[a].h > bt[b].h; });
  std::vector<int> rank_of(ntree);
  for (int r = 0; r < ntree; ++r) rank_of[order[r]] = r;
  std::vector<SpTree> tr(ntree);
  int64_t S = 0;
  int hmax = 0;
  for (int r = 0; r < ntree; ++r) {
    const BuildTree &b = bt[order[r]];
    SpTree &x = tr[r];
    memset(&x, 0, sizeof(x));
    x.node = b.tree->node;
    x.box = b.tree->box;
    x.live = b.tree->live_nodes;
    x.leaf_off = b.tree->leaf_off;
    x.pts = b.tree->pts;
    x.size = b.s;
    x.from_cleared = b.from_cleared;
    x.h = b.h;
    x.err = b.err;
    x.toff = S;
    if (b.h > 0) S += b.s;
    hmax = std::max(hmax, b.h);
  }
  std::vector<int> nact(hmax + 1, 0);     // trees still splitting at level t
  for (int t = 0; t <= hmax; ++t)
    for (int r = 0; r < ntree; ++r)
      if (tr[r].h > t) nact[t]++;
  int64_t Nmax = 1, leaves = 0;
  for (int t = 0; t < hmax; ++t) Nmax = std::max(Nmax, (int64_t)nact[t] << t);
  std::vector<int64_t> leaf_pre(1, 0);
  for (int r = 0; r < ntree; ++r) leaf_pre.push_back(leaf_pre.back() + ((int64_t)1 << tr[r].h));
  leaves = leaf_pre.back();
  // gather sources: cleared trees' records, then each tree's pool chunk
  std::vector<SpGather> ga;
  std::vector<int64_t> gpre(1, 0);
  for (const ClearedSrc &c : cl) {
    SpGather g;
    memset(&g, 0, sizeof(g));
    g.src = c.pts;
    g.count = c.size;
    g.tree = rank_of[c.dst];
    ga.push_back(g);
    gpre.push_back(gpre.back() + c.size);
  }
  for (int k = 0; k < ntree; ++k) {
    const BuildTree &b = bt[k];
    SpGather g;
    memset(&g, 0, sizeof(g));
    g.count = b.s - b.from_cleared;
    g.pbuf = b.pool.buf;
    g.pnbuf = b.pool.nbuf;
    g.parr = b.pool.arr;
    g.pfirst = b.pool.first;
    g.pool_lo = b.pool_lo;
    g.idtab = b.idtab;
    g.dst0 = b.from_cleared;
    g.tree = rank_of[k];
    ga.push_back(g);
    gpre.push_back(gpre.back() + g.count);
  }
  // ---- one device block: staging, per-level arrays, tables ----
  const int rs = rec_ints(dim);
  const size_t b_stg = al256((size_t)std::max<int64_t>(S, 1) * rs * 4);
  const size_t b_seg = al256((size_t)std::max<int64_t>(S, 1) * 4);
  const size_t b_i32 = al256((size_t)Nmax * 4), b_i64 = al256((size_t)Nmax * 8);
  const size_t b_tr = al256(ntree * sizeof(SpTree)), b_ga = al256(ga.size() * sizeof(SpGather));
  const size_t b_gpre = al256(gpre.size() * 8), b_lpre = al256(leaf_pre.size() * 8);
  const size_t b_cur = al256((size_t)ntree * 8);
  std::vector<TreeSeg> pk;
  std::vector<int64_t> pk_pre;
  {
    std::vector<Tree *> trees;
    for (auto &b : bt) trees.push_back(b.tree);
    pack_nodes_entries(trees, dim, pk, pk_pre);
  }
  const size_t b_pk = al256(pk.size() * sizeof(TreeSeg)), b_pkpre = al256(pk_pre.size() * 8);
  const size_t total = 2 * b_stg + 2 * b_seg + 6 * b_i32 + 2 * (b_i64 + b_i32) + b_tr + b_ga + b_gpre + b_lpre +
                       b_cur + b_pk + b_pkpre;
  void *block = nullptr;
  int st = dev_alloc(af, &block, total, s);
  if (st) return st;
  unsigned char *p = (unsigned char *)block;
  auto take = [&](size_t bytes) {
    void *q = p;
    p += bytes;
    return q;
  };
  int32_t *stg[2], *seg[2];
  stg[0] = (int32_t *)take(b_stg);
  stg[1] = (int32_t *)take(b_stg);
  seg[0] = (int32_t *)take(b_seg);
  seg[1] = (int32_t *)take(b_seg);
  int32_t *mn[2], *mx[2];   // split-coordinate bounds of this level's and the next level's segments
  mn[0] = (int32_t *)take(b_i32);
  mx[0] = (int32_t *)take(b_i32);
  mn[1] = (int32_t *)take(b_i32);
  mx[1] = (int32_t *)take(b_i32);
  uint32_t *curL = (uint32_t *)take(b_i32), *curR = (uint32_t *)take(b_i32);
  int64_t *lo[2];
  int32_t *nn[2];
  lo[0] = (int64_t *)take(b_i64);
  nn[0] = (int32_t *)take(b_i32);
  lo[1] = (int64_t *)take(b_i64);
  nn[1] = (int32_t *)take(b_i32);
  SpTree *d_tr = (SpTree *)take(b_tr);
  SpGather *d_ga = (SpGather *)take(b_ga);
  int64_t *d_gpre = (int64_t *)take(b_gpre), *d_lpre = (int64_t *)take(b_lpre);
  unsigned long long *cursor = (unsigned long long *)take(b_cur);
  TreeSeg *d_pk = (TreeSeg *)take(b_pk);
  int64_t *d_pkpre = (int64_t *)take(b_pkpre);
  st = h2d(d_tr, tr.data(), ntree * sizeof(SpTree), s);
  if (!st) st = h2d(d_ga, ga.data(), ga.size() * sizeof(SpGather), s);
  if (!st) st = h2d(d_gpre, gpre.data(), gpre.size() * 8, s);
  if (!st) st = h2d(d_lpre, leaf_pre.data(), leaf_pre.size() * 8, s);
  if (!st && !pk.empty()) st = h2d(d_pk, pk.data(), pk.size() * sizeof(TreeSeg), s);
  if (!st) st = h2d(d_pkpre, pk_pre.data(), pk_pre.size() * 8, s);
  if (!st) st = small_zero(cursor, b_cur, s);
  if (st) {
    dev_free(af, block, total, s);
    return st;
  }
  // ---- gather, roots ----
  if (gpre.back() > 0) {
    KScope ks_(kK_sp_gather, s);
    k_sp_gather<<<(unsigned)cdiv(gpre.back(), kT), kT, 0, s>>>(d_ga, d_gpre, (int)ga.size(), d_tr, dim, stg[0],
                                                               seg[0], cursor);
  }
  {
    KScope ks_(kK_sp_split, s);
    k_sp_roots<<<(unsigned)cdiv(ntree, 128), 128, 0, s>>>(d_tr, ntree, lo[0], nn[0]);
  }
  // ---- levels ----
  for (int t = 0; t < hmax; ++t) {
    const int64_t N = (int64_t)nact[t] << t;
    const int64_t A = tr[nact[t] - 1].toff + tr[nact[t] - 1].size;   // records still splitting
    const int c = t % dim;
    const int cur = t & 1, nxt = cur ^ 1;
    if (t == 0) {   // the first level's bounds by a pass of their own; later ones come from the scatter
      KScope ks_(kK_sp_minmax, s);
      k_sp_level_init<<<(unsigned)cdiv(N, 256), 256, 0, s>>>(0, curL, curR, N, mn[cur], mx[cur]);
      k_sp_minmax<<<(unsigned)cdiv(A, kT), kT, 0, s>>>(stg[cur], seg[cur], A, rs, c, mn[cur], mx[cur]);
    }
    const int64_t Nn = t + 1 < hmax ? (int64_t)nact[t + 1] << (t + 1) : 0;
    {
      KScope ks_(kK_sp_minmax, s);
      k_sp_level_init<<<(unsigned)cdiv(std::max(N, Nn), 256), 256, 0, s>>>(N, curL, curR, Nn, mn[nxt], mx[nxt]);
    }
    {
      KScope ks_(kK_sp_scatter, s);
      k_sp_scatter<<<(unsigned)cdiv(A, kT), kT, 0, s>>>(stg[cur], seg[cur], A, dim, c, t, mn[cur], mx[cur], lo[cur],
                                                        nn[cur], curL, curR, d_tr, stg[nxt], seg[nxt], mn[nxt],
                                                        mx[nxt]);
    }
    {
      KScope ks_(kK_sp_split, s);
      k_sp_split<<<(unsigned)cdiv(N, 256), 256, 0, s>>>(t, N, mn[cur], mx[cur], lo[cur], nn[cur], curL, curR, d_tr,
                                                       lo[nxt], nn[nxt]);
    }
  }
  // ---- boxes, live counts, packed records ----
  {
    KScope ks_(kK_sp_box, s);
    k_sp_leaf_box<<<(unsigned)cdiv(leaves, 128), 128, 0, s>>>(d_tr, d_lpre, ntree, dim);
  }
  for (int t = hmax - 1; t >= 0; --t) {
    const int64_t N = (int64_t)nact[t] << t;
    KScope ks_(kK_sp_box, s);
    k_sp_box_up<<<(unsigned)cdiv(N, 256), 256, 0, s>>>(d_tr, t, N, dim);
  }
  launch_pack_nodes(d_pk, d_pkpre, (int)pk.size(), pk_pre.back(), s);
  const int err = cuda_check(cudaGetLastError(), "spatial build kernels");
  dev_free(af, block, total, s);
  return err;
}

}  // namespace bdl
