// build.cu -- batched construction of the static kd-trees of one Insert_L
// (Alg. 3 line 5): gather the points of every new tree, then build all of them
// together with median splits in vEB layout (Alg. 1).
//
// GPU design (level-synchronous instead of Alg. 1's recursion):
//  * Every new tree is a complete tree with h = ceil(log2(ceil(s/L))) split
//    levels; the segment of points under node (depth t, index i) is fixed by
//    s alone (left child = ceil(m/2) points), so all trees advance depth by
//    depth in shared launches.
//  * Global levels (segments larger than one CTA's shared memory): an 11-bit
//    histogram of the split coordinate per segment, a per-segment bucket
//    search, a candidate gather of the median's bucket, an exact radix select
//    on the candidates' (low coordinate bits, id) key, and a partition pass
//    that moves whole records into the other staging buffer.
//  * Once segments fit in shared memory, one CTA builds each remaining
//    subtree entirely on chip (radix select on the composite key with
//    per-level digit widths; a bitonic sort across one warp for segments
//    <= 64 points),
//    writes leaves, bounding boxes and live counts, and stores the points in
//    leaf order.
//  * Node slots follow the vEB layout in closed form (veb_slot), children are
//    stored explicitly, boxes of the global-level nodes are merged bottom-up.
#include "bdl_internal.cuh"

#include <algorithm>
#include <cstdlib>
#include <functional>
#include <mutex>
#include <queue>

namespace bdl {

namespace {

constexpr int kItems = 8;          // records per thread in the tiled kernels
constexpr int kSubThreads = 1024;  // threads of the subtree kernel
constexpr int kSmallSubThreads = 256;   // threads of its instance for small subtrees
constexpr int kSmallSub = 2048;         // subtrees below this many records take that instance
constexpr int kWarpMode = 64;      // segments this small are sorted by one warp

struct SegState {
  unsigned long long cand_n;   // candidates gathered
  unsigned long long lcur;     // records placed left / right
  unsigned long long rcur;
  uint64_t median;             // composite key of the median
  int64_t rank;                // 1-based rank of the median inside its bucket
  int32_t bucket;              // top-11-bit bucket of the split coordinate
  int32_t nbucket;
};

struct NodeOut {               // where a tree's arrays go
  int32_t *pts, *box, *live, *leaf_off;
  Node *node;
};

// One tree of a build, as the kernels see it (in device memory).  The trees
// of one build may come from different forests: each carries its own pool,
// id table and error word.
struct DTree {
  int64_t base, s;             // first staging position, points
  int32_t h, g;                // split levels, levels split by the global kernels
  int32_t sel, pad_;           // staging buffer holding the tree after its global levels
  NodeOut out;
  int64_t from_cleared;        // records gathered from cleared trees (they come first)
  int64_t pool_lo;             // first pool entry of the tree's chunk
  const int32_t *pbuf;         // owning forest's pool: sorted buffer ids ...
  int64_t pnbuf;
  const int32_t *parr;         // ... then explicit ids, or a range from pfirst
  int64_t pfirst;
  const int32_t *idtab;        // owning forest's id table
  unsigned long long *err;     // owning forest's error word
};

struct DCleared {              // a cleared tree whose live records join tree `dst`
  const int32_t *pts;
  int64_t size;
  int32_t dst, pad_;
};

// Largest j in [0, n) with pre[j] <= x, for a prefix array pre[0..n] that
// starts at 0 and has pre[n] > x (empty entries are skipped).
__device__ __forceinline__ int find_le(const int64_t *pre, int n, int64_t x) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

struct LvTree {                // one tree at one global level
  int64_t base, s, seg_off, tile_off;
  int64_t next_seg;            // its first segment at the next global level, or -1 if it has none
  int32_t t, c, h;
  NodeOut out;
  unsigned long long *err;
};

struct LvParams {              // one global level
  int nact, dim, tile, it;
  int64_t S;
  const int32_t *src;
  int32_t *dst;
  uint32_t *hist;              // this level's per-segment histograms (filled by the level before)
  SegState *seg;               // this level's segment states
  uint32_t *hist_next;         // the next level's (accumulated by this level's partition)
  SegState *seg_next;          // the next level's (cleared by this level's partition)
  int64_t nseg_next;
  uint64_t *cand;
  LvTree one;                  // the level's tree when nact == 1 (no memory lookups)
  const LvTree *lt;            // [nact] the level's trees
  const int64_t *act_seg;      // [nact + 1] segment prefix
  const int64_t *act_tile;     // [nact + 1] tile prefix
};

// The level's tree that owns tile b / segment g (a reference into the
// level's descriptor in device memory: fields are loaded where used).
__device__ __forceinline__ const LvTree &tree_by_tile(const LvParams &P, int64_t b) {
  return P.nact == 1 ? P.one : P.lt[find_le(P.act_tile, P.nact, b)];
}

__device__ __forceinline__ const LvTree &tree_by_seg(const LvParams &P, int64_t g) {
  return P.nact == 1 ? P.one : P.lt[find_le(P.act_seg, P.nact, g)];
}

// ---------------------------------------------------------------------------
// K5: gather the points of each new tree into the staging arrays
// ---------------------------------------------------------------------------

struct GatherParams {
  int nsrc, ntrees, dim;
  int64_t S;
  int32_t *stg;                       // staging A: [dim+1][S]
  unsigned long long *cursor;         // per tree: records placed from cleared trees
  const DTree *tree;
  const DCleared *cl;
  const int64_t *cl_blk;              // [nsrc + 1] block prefix of the cleared sources
  const int64_t *pool_off;            // [ntrees + 1] prefix of the pool chunk sizes
};

__device__ __forceinline__ int32_t pool_id(const int32_t *buf, int64_t nbuf, const int32_t *arr,
                                           int64_t first, int64_t k) {
  if (k < nbuf) return buf[k];
  return arr ? arr[k - nbuf] : (int32_t)(first + (k - nbuf));
}

// Records [b * blockDim.x, (b + 1) * blockDim.x) of the cleared sources: the
// live ones are appended to their new tree's staging range (one atomic per
// block and tree).
__device__ void gather_cleared(const GatherParams &P, int64_t b) {
  __shared__ int wsum[32];
  __shared__ unsigned long long sbase;
  const int src = find_le(P.cl_blk, P.nsrc, b);
  const DCleared C = P.cl[src];
  int64_t p = (int64_t)(b - P.cl_blk[src]) * blockDim.x + threadIdx.x;
  bool ok = p < C.size;
  const int rs = rec_ints(P.dim);
  int32_t id = ok ? C.pts[p * rs + P.dim] : -1;
  bool live = ok && id >= 0;
  // block-exclusive count of live records
  unsigned bal = __ballot_sync(0xffffffffu, live);
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int wpre = __popc(bal & ((1u << lane) - 1));
  if (lane == 0) wsum[warp] = __popc(bal);
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { int v = wsum[w]; wsum[w] = acc; acc += v; }
    sbase = atomicAdd(&P.cursor[C.dst], (unsigned long long)acc);
  }
  __syncthreads();
  if (!live) return;
  const DTree &T = P.tree[C.dst];
  int64_t rel = (int64_t)sbase + wsum[warp] + wpre;
  if (rel >= T.from_cleared) {   // more live records than the plan counted
    atomicOr(T.err, kErrGather);
    return;
  }
  int64_t dst = T.base + rel;
  for (int c = 0; c < P.dim; ++c) P.stg[c * P.S + dst] = C.pts[p * rs + c];
  P.stg[P.dim * P.S + dst] = id;
}

// Pool entry k of the new trees (the batch's points, by id).
__device__ void gather_pool(const GatherParams &P, int64_t k) {
  const int j = find_le(P.pool_off, P.ntrees, k);
  const DTree &T = P.tree[j];
  const int64_t i = k - P.pool_off[j];
  int32_t id = pool_id(T.pbuf, T.pnbuf, T.parr, T.pfirst, T.pool_lo + i);
  int64_t dst = T.base + T.from_cleared + i;
  const int32_t *src = T.idtab + (int64_t)id * P.dim;
  for (int c = 0; c < P.dim; ++c) P.stg[c * P.S + dst] = src[c];
  P.stg[P.dim * P.S + dst] = id;
}

// ---------------------------------------------------------------------------
// K1 global levels: histogram, bucket search, candidate gather, exact select
// ---------------------------------------------------------------------------

struct TileSegs {
  int64_t p0, p1;          // tile [p0, p1) relative to the tree
  int64_t idx0, st0, sz0;  // first segment
  int64_t st1, sz1;        // second segment (sz1 = 0 if none)
};

__device__ __forceinline__ TileSegs tile_segs(const LvParams &P, const LvTree &T, int64_t b) {
  TileSegs g;
  g.p0 = (b - T.tile_off) * P.tile;
  g.p1 = min(g.p0 + (int64_t)P.tile, T.s);
  g.idx0 = seg_of(T.s, T.t, g.p0, g.st0, g.sz0);
  g.sz1 = 0;
  g.st1 = g.st0 + g.sz0;
  if (g.p1 > g.st1) seg_range(T.s, T.t, g.idx0 + 1, g.st1, g.sz1);
  return g;
}

// Eight consecutive ints from x[p] (x + p is 32-byte aligned when p is a
// multiple of 8); positions at or past `end` are not read.
__device__ __forceinline__ void load8(const int32_t *x, int64_t p, int64_t end, int32_t v[kItems]) {
  if (p + kItems <= end) {
    const int4 a = reinterpret_cast<const int4 *>(x + p)[0];
    const int4 b = reinterpret_cast<const int4 *>(x + p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  } else {
#pragma unroll
    for (int j = 0; j < kItems; ++j) v[j] = p + j < end ? x[p + j] : 0;
  }
}

// Tile b of the level: 11-bit histogram of the split coordinate, per segment.
__device__ void level_hist(const LvParams &P, int64_t b, uint32_t (*h)[kHistBins]) {
  const LvTree &T = tree_by_tile(P, b);
  TileSegs g = tile_segs(P, T, b);
  for (int i = threadIdx.x; i < 2 * kHistBins; i += blockDim.x) (&h[0][0])[i] = 0;
  __syncthreads();
  const int32_t *x = P.src + T.c * P.S + T.base;
  const int64_t pb = g.p0 + (int64_t)threadIdx.x * kItems;   // kCoopThreads * kItems = tile
  int32_t cv[kItems];
  load8(x, pb, g.p1, cv);
#pragma unroll
  for (int j = 0; j < kItems; ++j)
    if (pb + j < g.p1) atomicAdd(&h[pb + j >= g.st1][cv[j] >> kHistShift], 1u);
  __syncthreads();
  uint32_t *h0 = P.hist + (T.seg_off + g.idx0) * kHistBins;
  for (int i = threadIdx.x; i < kHistBins; i += blockDim.x) {
    uint32_t v = h[0][i];
    if (v) atomicAdd(&h0[i], v);
    if (g.sz1) {
      v = h[1][i];
      if (v) atomicAdd(&h0[kHistBins + i], v);
    }
  }
}

// The bin of a kHistBins-bin histogram h that holds the r-th smallest entry
// (1-based), and how many entries lie in the bins before it; block-wide,
// kCoopThreads threads, 4 bins each.
__device__ void hist_rank_bin(const uint32_t *h, uint32_t r, int *out_bin, uint32_t *out_below,
                              uint32_t *out_cnt) {
  __shared__ uint32_t wsum[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int per = kHistBins / blockDim.x;   // 4
  uint32_t v[4] = {0, 0, 0, 0}, sum = 0;
  if (per == 4) {
    const uint4 q = reinterpret_cast<const uint4 *>(h)[threadIdx.x];
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    sum = q.x + q.y + q.z + q.w;
  }
  uint32_t inc = sum;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  uint32_t base = 0;
  for (int w = 0; w < warp; ++w) base += wsum[w];
  (void)nwarps;
  uint32_t below = base + inc - sum;
  if (below < r && r <= below + sum) {
    for (int j = 0; j < 4; ++j) {
      if (r <= below + v[j]) {
        *out_bin = threadIdx.x * 4 + j;
        *out_below = below;
        *out_cnt = v[j];
        break;
      }
      below += v[j];
    }
  }
  __syncthreads();
}

// Gather the (low coordinate bits, id) keys of every record in its segment's
// median bucket, at the segment's own range of the candidate array.
__device__ void level_collect(const LvParams &P, int64_t b) {
  __shared__ unsigned cnt[2];
  __shared__ unsigned long long basev[2];
  __shared__ int s_bin[2];
  __shared__ uint32_t s_below[2], s_cnt[2];
  const LvTree &T = tree_by_tile(P, b);
  TileSegs g = tile_segs(P, T, b);
  if (threadIdx.x < 2) cnt[threadIdx.x] = 0;
  // the bucket holding each segment's median (rank ceil(m/2)), from the
  // segment's histogram; the block whose tile holds the segment's first
  // record records it for the select
  for (int w = 0; w < (g.sz1 ? 2 : 1); ++w) {
    const int64_t gs = T.seg_off + g.idx0 + w;
    const int64_t sz = w ? g.sz1 : g.sz0;
    hist_rank_bin(P.hist + gs * kHistBins, (uint32_t)((sz + 1) >> 1), &s_bin[w], &s_below[w], &s_cnt[w]);
    const int64_t st = w ? g.st1 : g.st0;
    if (threadIdx.x == 0 && st >= g.p0) {
      SegState &S = P.seg[gs];
      S.bucket = s_bin[w];
      S.nbucket = (int32_t)s_cnt[w];
      S.rank = (int64_t)(((sz + 1) >> 1) - s_below[w]);
    }
  }
  __syncthreads();
  int32_t bk0 = s_bin[0], bk1 = g.sz1 ? s_bin[1] : -1;
  const int32_t *x = P.src + T.c * P.S + T.base;
  const int32_t *xi = P.src + P.dim * P.S + T.base;
  uint64_t key[kItems];
  unsigned slot[kItems];
  int nk = 0;
  // the tile's split coordinates, eight consecutive ones per thread
  // (kCoopThreads * kItems = tile)
  const int64_t pb = g.p0 + (int64_t)threadIdx.x * kItems;
  int32_t cv[kItems];
  load8(x, pb, g.p1, cv);
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const int64_t p = pb + j;
    const int32_t c = cv[j];
    const int w = p >= g.st1;
    if (p < g.p1 && (c >> kHistShift) == (w ? bk1 : bk0)) {
      key[nk] = ((uint64_t)(c & ((1 << kHistShift) - 1)) << 31) | (uint32_t)xi[p];
      slot[nk] = (atomicAdd(&cnt[w], 1u) << 1) | (unsigned)w;
      nk++;
    }
  }
  __syncthreads();
  if (threadIdx.x < 2 && (threadIdx.x == 0 || g.sz1) && cnt[threadIdx.x])
    basev[threadIdx.x] = atomicAdd(&P.seg[T.seg_off + g.idx0 + threadIdx.x].cand_n,
                                   (unsigned long long)cnt[threadIdx.x]);
  __syncthreads();
  for (int i = 0; i < nk; ++i) {
    int w = slot[i] & 1;
    int64_t st = w ? g.st1 : g.st0;
    P.cand[T.base + st + basev[w] + (slot[i] >> 1)] = key[i];
  }
}

// One CTA per segment: exact select of the median among its bucket's keys
// (8-bit digits over the 40-bit candidate key), then the node is written.
__device__ void level_select(const LvParams &P, int64_t gs, uint64_t *keys) {
  __shared__ uint32_t hist[256];
  __shared__ uint64_t s_pre;
  __shared__ int64_t s_rank;
  __shared__ uint32_t s_cnt;
  __shared__ uint64_t s_found;
  __shared__ uint32_t s_wsum[32];
  const LvTree &T = tree_by_seg(P, gs);
  int64_t idx = gs - T.seg_off;
  int64_t st, sz;
  seg_range(T.s, T.t, idx, st, sz);
  SegState &S = P.seg[gs];
  int64_t n = (int64_t)S.cand_n;
  const uint64_t *cand = P.cand + T.base + st;
  bool in_smem = n <= 2048;
  if (in_smem)
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) keys[i] = cand[i];
  if (threadIdx.x == 0) { s_pre = 0; s_rank = S.rank; s_cnt = (uint32_t)n; s_found = ~0ull; }
  __syncthreads();
  const int kbits = 31 + kHistShift;   // 40
  int shift = kbits;
  while (true) {
    if (s_cnt == 1) {
      // the unique key with this prefix
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        uint64_t k = in_smem ? keys[i] : cand[i];
        if ((k >> shift) == (s_pre >> shift)) s_found = k;
      }
      __syncthreads();
      break;
    }
    if (shift == 0) {
      if (threadIdx.x == 0) s_found = s_pre;
      __syncthreads();
      break;
    }
    int ns = max(0, shift - 8);
    int ww = shift - ns;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      uint64_t k = in_smem ? keys[i] : cand[i];
      if ((k >> shift) == (s_pre >> shift)) atomicAdd(&hist[(k >> ns) & ((1u << ww) - 1)], 1u);
    }
    __syncthreads();
    {
      // block scan of the 256 bins (one per thread) to find the rank's bucket
      const int j = threadIdx.x;
      const uint32_t v = j < (1 << ww) ? hist[j] : 0;
      uint32_t inc = v;
      const int lane = j & 31, warp = j >> 5;
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      if (lane == 31) s_wsum[warp] = inc;
      __syncthreads();
      uint32_t base = 0;
      for (int w = 0; w < warp; ++w) base += s_wsum[w];
      inc += base;
      const int64_t rank = s_rank;
      __syncthreads();
      if ((int64_t)inc >= rank && (int64_t)(inc - v) < rank) {
        s_pre |= (uint64_t)j << ns;
        s_rank = rank - (inc - v);
        s_cnt = v;
      }
    }
    shift = ns;
    __syncthreads();
  }
  // the segment's histogram is done with: cleared for the level after next
  for (int i = threadIdx.x; i < kHistBins / 4; i += blockDim.x)
    reinterpret_cast<uint4 *>(P.hist + gs * kHistBins)[i] = make_uint4(0, 0, 0, 0);
  if (threadIdx.x == 0) {
    uint64_t k40 = s_found;
    uint32_t coord = ((uint32_t)S.bucket << kHistShift) | (uint32_t)(k40 >> 31);
    uint64_t med = comp_key((int32_t)coord, (int32_t)(k40 & 0x7fffffffu));
    S.median = med;
    const NodeOut &o = T.out;
    int l = T.h + 1;
    int64_t v = veb_slot(l, T.t, idx);
    o.node[v] = Node{med, (int32_t)veb_slot(l, T.t + 1, 2 * idx), (int32_t)veb_slot(l, T.t + 1, 2 * idx + 1)};
  }
}


// K2: partition every tile's records around their segment's median into the
// other staging buffer.  Left records of a segment go to [st, st+ceil(m/2)),
// right ones after; each CTA reserves its ranges with one atomic per class.
// hnext: shared memory for the next level's histograms of the tile's (up to
// four) child segments, 16-bit counts packed in pairs (a tile has at most
// 4096 records).
__device__ void level_partition(const LvParams &P, int64_t b, int32_t *stage, uint32_t *hnext) {
  __shared__ unsigned long long wsum[32];
  __shared__ unsigned long long cbase[4];
  __shared__ int64_t gdst[4];              // global start of each class's run
  __shared__ int coff[5];                  // start of each class's run in `stage`
  __shared__ int cok[4];
  const LvTree &T = tree_by_tile(P, b);
  TileSegs g = tile_segs(P, T, b);
  const int64_t nxt = T.next_seg;
  const int cn = (T.t + 1) % P.dim;
  if (nxt >= 0)   // cleared before the block barriers below, filled after them
    for (int i = threadIdx.x; i < 4 * kHistBins / 8; i += blockDim.x)
      reinterpret_cast<uint4 *>(hnext)[i] = make_uint4(0, 0, 0, 0);
  const SegState *s0 = &P.seg[T.seg_off + g.idx0];
  uint64_t med0 = s0[0].median, med1 = g.sz1 ? s0[1].median : 0;
  const int32_t *xc = P.src + T.c * P.S + T.base;
  const int32_t *xi = P.src + P.dim * P.S + T.base;
  int64_t pb = g.p0 + (int64_t)threadIdx.x * kItems;
  int cls[kItems];
  int32_t cv[kItems], iv[kItems];
  load8(xc, pb, g.p1, cv);
  load8(xi, pb, g.p1, iv);
  unsigned long long mine = 0;   // 4 x 16-bit class counts
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    int64_t p = pb + j;
    cls[j] = -1;
    if (p < g.p1) {
      int w = p >= g.st1;
      uint64_t k = comp_key(cv[j], iv[j]);
      int c = 2 * w + (k > (w ? med1 : med0));
      cls[j] = c;
      mine += 1ull << (16 * c);
    }
  }
  // block exclusive scan of the packed counts
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long inc = mine;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long acc = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { unsigned long long v = wsum[w]; wsum[w] = acc; acc += v; }
    coff[0] = 0;
    for (int c = 0; c < 4; ++c) {
      unsigned long long tot = (acc >> (16 * c)) & 0xffff;
      cbase[c] = 0;
      if (tot) {
        const SegState &S = P.seg[T.seg_off + g.idx0 + (c >> 1)];
        unsigned long long *cur = (c & 1) ? (unsigned long long *)&S.rcur : (unsigned long long *)&S.lcur;
        cbase[c] = atomicAdd(cur, tot);
      }
      const int64_t st = (c >> 1) ? g.st1 : g.st0;
      const int64_t sz = (c >> 1) ? g.sz1 : g.sz0;
      const int64_t off = (c & 1) ? ((sz + 1) >> 1) : 0;
      const int64_t lim = (c & 1) ? sz - ((sz + 1) >> 1) : ((sz + 1) >> 1);
      gdst[c] = st + off + (int64_t)cbase[c];
      cok[c] = (int64_t)(cbase[c] + tot) <= lim;   // else the median did not halve the segment
      if (!cok[c]) atomicOr(T.err, kErrPartition);
      coff[c + 1] = coff[c] + (int)tot;
    }
  }
  __syncthreads();
  const unsigned long long ex = inc - mine + wsum[warp];
  int spos[kItems];                 // position of each item in the tile's output order
  int run[4] = {0, 0, 0, 0};
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const int c = cls[j];
    spos[j] = -1;
    if (c < 0) continue;
    spos[j] = coff[c] + (int)((ex >> (16 * c)) & 0xffff) + run[c];
    run[c]++;
  }
  // each array: scatter into shared memory, then write every class's run
  // with consecutive threads on consecutive addresses; the next level's
  // split coordinate also goes into its child segment's histogram.  The
  // next array's items are loaded as soon as this one's are scattered, so
  // that their loads overlap the barrier and the stores.
  const int ntile = coff[4];
  int32_t v[kItems];
  load8(P.src + T.base, pb, g.p1, v);
  for (int c = 0; c <= P.dim; ++c) {
#pragma unroll
    for (int j = 0; j < kItems; ++j)
      if (spos[j] >= 0) {
        stage[spos[j]] = v[j];
        if (c == cn && nxt >= 0) {
          const int bin = v[j] >> kHistShift;
          atomicAdd(&hnext[cls[j] * (kHistBins / 2) + (bin >> 1)], 1u << (16 * (bin & 1)));
        }
      }
    if (c < P.dim) load8(P.src + (c + 1) * P.S + T.base, pb, g.p1, v);
    __syncthreads();
    int32_t *y = P.dst + c * P.S + T.base;
    for (int i = threadIdx.x; i < ntile; i += blockDim.x) {
      const int k = (i >= coff[1]) + (i >= coff[2]) + (i >= coff[3]);
      if (cok[k]) y[gdst[k] + (i - coff[k])] = stage[i];
    }
    __syncthreads();
  }
  if (nxt >= 0)   // child (segment w, side) of level index idx0 + w is 2 (idx0 + w) + side
    for (int i = threadIdx.x; i < 4 * kHistBins / 2; i += blockDim.x) {
      const int k = i / (kHistBins / 2), wd = i % (kHistBins / 2);
      if ((k >> 1) && !g.sz1) continue;
      const uint32_t x = hnext[i];
      if (!x) continue;
      uint32_t *h = P.hist_next + (nxt + 2 * (g.idx0 + (k >> 1)) + (k & 1)) * kHistBins + 2 * wd;
      if (x & 0xffffu) atomicAdd(h, x & 0xffffu);
      if (x >> 16) atomicAdd(h + 1, x >> 16);
    }
}

// ---------------------------------------------------------------------------
// The gather and every global level of a build in one cooperative launch:
// each phase is a grid-stride loop over its work items (cleared-record
// blocks, pool entries, tiles, segments), and a grid barrier separates the
// phases, instead of one launch per phase and level.
// ---------------------------------------------------------------------------

constexpr int kCoopThreads = 512;   // = tile / kItems for 4096-record tiles

struct LevelWork {                  // one global level, in device memory
  LvParams P;
  int64_t ntile, nseg;
};

struct LevelsParams {
  GatherParams G;
  int64_t cl_blocks;                // cleared sources, in blocks of kCoopThreads records
  int64_t pool_total;               // pool entries
  const LevelWork *lv;              // [nlev]
  int nlev;
  unsigned *bar;                    // grid barrier state (2 words, zeroed)
  unsigned long long *err;          // where a barrier that gave up is recorded
};

__global__ void __launch_bounds__(kCoopThreads, 2) k_build_levels(const LevelsParams B) {
  // shared buffers for the phases' big arrays (histograms, candidate keys,
  // the partition's staging; the next level's histograms), 16 KB each
  __shared__ __align__(16) uint32_t s_big[2 * kHistBins];
  __shared__ __align__(16) uint32_t s_next[2 * kHistBins];
  for (int64_t b = blockIdx.x; b < B.cl_blocks; b += gridDim.x) {
    gather_cleared(B.G, b);
    __syncthreads();
  }
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < B.pool_total;
       k += (int64_t)gridDim.x * blockDim.x)
    gather_pool(B.G, k);
  if (B.nlev == 0) return;
  // the first level's histograms; every later level's come from the
  // partition of the level before
  grid_barrier(B.bar, B.err);
  for (int64_t b = blockIdx.x; b < B.lv[0].ntile; b += gridDim.x) {
    level_hist(B.lv[0].P, b, reinterpret_cast<uint32_t (*)[kHistBins]>(s_big));
    __syncthreads();
  }
  for (int it = 0; it < B.nlev; ++it) {
    const LevelWork &W = B.lv[it];
    const LvParams &P = W.P;
    grid_barrier(B.bar, B.err);
    for (int64_t b = blockIdx.x; b < W.ntile; b += gridDim.x) {
      level_collect(P, b);
      __syncthreads();
    }
    grid_barrier(B.bar, B.err);
    for (int64_t gs = blockIdx.x; gs < W.nseg; gs += gridDim.x) {
      level_select(P, gs, reinterpret_cast<uint64_t *>(s_big));
      __syncthreads();
    }
    grid_barrier(B.bar, B.err);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.nseg_next;
         i += (int64_t)gridDim.x * blockDim.x) {
      P.seg_next[i].cand_n = 0;
      P.seg_next[i].lcur = 0;
      P.seg_next[i].rcur = 0;
    }
    for (int64_t b = blockIdx.x; b < W.ntile; b += gridDim.x) {
      level_partition(P, b, reinterpret_cast<int32_t *>(s_big), s_next);
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// K1-K4 on chip: one CTA builds a whole subtree of <= cap records
// ---------------------------------------------------------------------------

struct SubParams {
  int ntrees, dim, cap;
  int64_t S;
  const int32_t *stg[2];
  const DTree *tree;
  const int64_t *sub_blk;      // [ntrees + 1] prefix of 2^g subtrees per tree, in launch order
  const int32_t *sub_ord;      // [ntrees] the trees in launch order (largest subtrees first)
};

// An asynchronous 4-byte copy from global to shared memory (completed by
// cp.async.wait_all).
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}

// Ascending bitonic sort of one 64-bit word per lane across a warp.
__device__ __forceinline__ uint64_t warp_sort32(uint64_t x, int lane) {
#pragma unroll
  for (int size = 2; size <= 32; size <<= 1)
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      const uint64_t y = __shfl_xor_sync(0xffffffffu, x, stride);
      const bool keep_min = ((lane & stride) == 0) == ((lane & size) == 0);
      x = keep_min ? min(x, y) : max(x, y);
    }
  return x;
}

// Ascending bitonic sort of 64 words across a warp, lane l holding elements
// 2l (x0) and 2l + 1 (x1).
__device__ __forceinline__ void warp_sort64(uint64_t &x0, uint64_t &x1, int lane) {
  const int e = 2 * lane;
#pragma unroll
  for (int size = 2; size <= 64; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 1; stride >>= 1) {
      const uint64_t y0 = __shfl_xor_sync(0xffffffffu, x0, stride >> 1);
      const uint64_t y1 = __shfl_xor_sync(0xffffffffu, x1, stride >> 1);
      const bool keep_min = ((e & stride) == 0) == ((e & size) == 0);
      x0 = keep_min ? min(x0, y0) : max(x0, y0);
      x1 = keep_min ? min(x1, y1) : max(x1, y1);
    }
    const uint64_t lo = min(x0, x1), hi = max(x0, x1);   // stride 1: inside the lane
    const bool up = (e & size) == 0;
    x0 = up ? lo : hi;
    x1 = up ? hi : lo;
  }
}

__device__ __forceinline__ uint64_t skey(const int32_t *sc, const int32_t *sid, int cap, int c,
                                         int it) {
  return comp_key(sc[c * cap + it], sid[it]);
}

// seg_range for a subtree (m < 2^31 points).
__device__ __forceinline__ void seg_range32(int m, int u, int idx, int &start, int &size) {
  start = 0;
  size = m;
  for (int j = u - 1; j >= 0; --j) {
    const int l = (size + 1) >> 1;
    if ((idx >> j) & 1) {
      start += l;
      size -= l;
    } else {
      size = l;
    }
  }
}

// Key bits a segment's median search still has to decide, given that every
// coordinate of the segment (in the split dimension) lies in [lo, hi]: the
// coordinate bits below their common prefix, and the 31 id bits.
__device__ __forceinline__ int open_key_bits(int32_t lo, int32_t hi) {
  if (lo > hi) return kKeyBits;
  return 31 + (lo == hi ? 0 : 32 - __clz(lo ^ hi));
}

// TH threads per CTA (1024, or 256 for subtrees of fewer than 2048 records):
// 2 * TH histogram bins per pass, TH / 8 segments per radix level at most.
template <int TH>
__global__ void __launch_bounds__(TH, TH == kSubThreads ? 1 : 3) k_subtree(const SubParams P) {
  constexpr int HB = 2 * TH;                   // bins of a level's histogram (all its segments)
  constexpr int LB = TH == 1024 ? 11 : TH == 256 ? 9 : -1;   // log2(HB)
  static_assert(LB > 0, "k_subtree: 1024 or 256 threads");
  constexpr int MS = TH / 8;                   // segments of a radix level (cap / 64 <= 8 TH / 64)
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ uint64_t s_pre[MS], s_res[MS];
  __shared__ int32_t s_st[MS], s_sz[MS], s_rank[MS],
      s_cnt2[MS], s_lb[MS], s_dig[MS],
      s_bel[MS], s_wq[MS];
  __shared__ unsigned char s_done[MS];
  __shared__ uint32_t s_w[32], s_base[8];
  __shared__ int s_ncand;
  // key bits still open per segment (the digits below them are the next to
  // decide): this level's, and the next level's set by the partition
  __shared__ int32_t s_sh[MS], s_shn[MS];

  const int cap = P.cap, dim = P.dim;
  int b = blockIdx.x;
  const int jj = find_le(P.sub_blk, P.ntrees, b);
  const int tj = P.sub_ord[jj];
  const DTree &T = P.tree[tj];
  const NodeOut o = T.out;
  const int t0 = T.g;
  int64_t i0 = b - P.sub_blk[jj];
  int64_t start0, m64;
  seg_range(T.s, t0, i0, start0, m64);
  const int m0 = (int)m64;
  const int l = T.h + 1;

  int32_t *sc = (int32_t *)sm;                          // [dim][cap]
  int32_t *sid = sc + (size_t)dim * cap;                // [cap]
  uint32_t *hist = (uint32_t *)(sid + cap);             // [HB]
  // [HB] a record that the pass counted in the bin: the only one where the
  // bin's count is 1
  uint16_t *wit = (uint16_t *)(hist + HB);
  uint16_t *perm0 = wit + HB;                           // [cap]
  uint16_t *perm1 = perm0 + cap;                        // [cap]
  uint16_t *binq = perm1 + cap;                         // [cap] first digit of each position's key
  unsigned char *segid = (unsigned char *)(binq + cap);   // [cap] segment of each position
  unsigned char *segid_n = segid + cap;                   // [cap] the same for the next level
  // per-segment coordinate bounds [lo, hi] in every dimension, of this
  // level's segments and of the next level's: [MS][dim][2] each
  int32_t *bcur = (int32_t *)(segid_n + cap);
  int32_t *bnxt = bcur + MS * dim * 2;

  const int32_t *src = P.stg[T.sel];
  if (threadIdx.x < dim) {
    bcur[2 * threadIdx.x] = INT32_MAX;
    bcur[2 * threadIdx.x + 1] = INT32_MIN;
  }
  for (int i = threadIdx.x; i < HB; i += blockDim.x) hist[i] = 0;   // bins start at zero
  // the records' planes, copied asynchronously (all of a thread's copies in
  // flight at once)
  const int32_t *rec0 = src + T.base + start0;
  for (int q = threadIdx.x; q < m0; q += blockDim.x) {
    for (int c = 0; c < dim; ++c) cp_async4(&sc[c * cap + q], rec0 + c * P.S + q);
    cp_async4(&sid[q], rec0 + dim * P.S + q);
    perm0[q] = (uint16_t)q;
    perm1[q] = (uint16_t)q;   // any slot a level leaves unwritten still names a record
    segid[q] = 0;
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  // the subtree's bounding box: the root segment's bounds
  for (int c = 0; c < dim; ++c) {
    int32_t lo = INT32_MAX, hi = INT32_MIN;
    for (int q = threadIdx.x; q < m0; q += blockDim.x) {
      const int32_t x = sc[c * cap + q];
      lo = min(lo, x);
      hi = max(hi, x);
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&bcur[2 * c], lo);
      atomicMax(&bcur[2 * c + 1], hi);
    }
  }
  __syncthreads();

  const int U = T.h - t0;
  const int nleaf = 1 << U;
  // [2 * nleaf] vEB slots by heap index, once computed after the radix
  // levels (with the warps' 64 results it may run on into `wit`)
  int32_t *nslot = (int32_t *)hist;
  bool slots_ready = false;
  bool hist_ready = false;   // `hist` holds this level's first-pass histogram already
  uint16_t *cur = perm0, *nxt = perm1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;

  for (int u = 0; u < U; ++u) {
    const int t = t0 + u;
    const int c = t % dim;
    const int nseg = 1 << u;
    int64_t st_, sz_;
    seg_range(m0, u, 0, st_, sz_);
    const int mmax = (int)sz_;
    if (mmax > kWarpMode) {
      // ---------------- radix mode: all segments of the level together ----
      const int w = LB - u;      // nseg << w == HB bins
      for (int s = threadIdx.x; s < nseg; s += blockDim.x) {
        int64_t a, z;
        seg_range(m0, u, s, a, z);
        s_st[s] = (int)a;
        s_sz[s] = (int)z;
        // the key bits above the open ones are the bounds' common prefix,
        // the same for every record of the segment
        const int32_t lo = bcur[(s * dim + c) * 2], hi = bcur[(s * dim + c) * 2 + 1];
        const int sh = open_key_bits(lo, hi);
        s_sh[s] = sh;
        s_pre[s] = sh >= kKeyBits ? 0 : ((uint64_t)lo >> (sh - 31)) << sh;
        s_rank[s] = (int)((z + 1) >> 1);
        s_cnt2[s] = 0;
        if (s == 0) s_ncand = 0;
        s_done[s] = 0;
      }
      __syncthreads();
      // Every pass decides the next w open bits of each segment's median
      // key (the digit below its s_sh open bits) from a histogram of the
      // records that still match the segment's prefix.  Pass 0 counts every
      // record; its histogram was filled by the previous level's partition,
      // except at the subtree's first level, and each position's digit is
      // kept in `binq`.  Pass 1 lists the records whose digit is their
      // segment's chosen one (in `nxt`, free until this level's partition)
      // and counts them; later passes read only that list.  A bucket that
      // holds one record ends its segment's search: the bin's witness is
      // the median.  The bins are zero at the start of every pass that
      // counts (each pass's bucket search clears them).
      uint16_t *cand = nxt;
      const int nbin = 1 << w, per = (nbin + 31) >> 5;   // bins per segment, per lane
      for (int pass = 0;; ++pass) {
        if (pass == 0) {
          if (!hist_ready) {
            for (int q = threadIdx.x; q < m0; q += blockDim.x) {
              const int s = segid[q], it = cur[q];
              const uint64_t k = skey(sc, sid, cap, c, it);
              const int sh = s_sh[s], ns = max(0, sh - w);
              const int dg = (int)((k >> ns) & ((1u << (sh - ns)) - 1));
              binq[q] = (uint16_t)dg;
              wit[(s << w) + dg] = (uint16_t)it;
              atomicAdd(&hist[(s << w) + dg], 1u);
            }
            __syncthreads();
          }
        } else if (pass == 1) {
          for (int q = threadIdx.x; q < m0; q += blockDim.x) {
            const int s = segid[q];
            if (s_done[s] || binq[q] != s_dig[s]) continue;
            cand[atomicAdd(&s_ncand, 1)] = (uint16_t)q;
            const int it = cur[q];
            const uint64_t k = skey(sc, sid, cap, c, it);
            const int sh = s_sh[s], ns = max(0, sh - w);
            const int dg = (int)((k >> ns) & ((1u << (sh - ns)) - 1));
            wit[(s << w) + dg] = (uint16_t)it;
            atomicAdd(&hist[(s << w) + dg], 1u);
          }
          __syncthreads();
        } else {
          const int nq = s_ncand;
          for (int i = threadIdx.x; i < nq; i += blockDim.x) {
            const int q = cand[i];
            const int s = segid[q];
            if (s_done[s]) continue;
            const int it = cur[q];
            const uint64_t k = skey(sc, sid, cap, c, it);
            const int sh = s_sh[s], ns = max(0, sh - w);
            if ((k >> sh) != (s_pre[s] >> sh)) continue;
            const int dg = (int)((k >> ns) & ((1u << (sh - ns)) - 1));
            wit[(s << w) + dg] = (uint16_t)it;
            atomicAdd(&hist[(s << w) + dg], 1u);
          }
          __syncthreads();
        }
        // the bucket holding each segment's rank-th candidate; the segment's
        // prefix, rank and open bits move into it and the bins are cleared
        int pending = 0;
        if (nseg < 8) {
          // few segments: an exclusive scan of all the bins (2 per thread)
          const int i2 = 2 * threadIdx.x;
          const uint32_t a0 = hist[i2], a1 = hist[i2 + 1];
          const uint32_t v = a0 + a1;
          uint32_t inc = v;
          for (int o2 = 1; o2 < 32; o2 <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o2);
            if (lane >= o2) inc += y;
          }
          if (lane == 31) s_w[warp] = inc;
          __syncthreads();
          if (warp == 0) {
            const uint32_t x = lane < nwarps ? s_w[lane] : 0;
            uint32_t xi = x;
            for (int o2 = 1; o2 < 32; o2 <<= 1) {
              const uint32_t y = __shfl_up_sync(0xffffffffu, xi, o2);
              if (lane >= o2) xi += y;
            }
            if (lane < nwarps) s_w[lane] = xi - x;
          }
          __syncthreads();
          const uint32_t e = inc - v + s_w[warp];
          if ((i2 & (nbin - 1)) == 0) s_base[i2 >> w] = e;   // the segment's first bin
          __syncthreads();
          hist[i2] = 0;
          hist[i2 + 1] = 0;
#pragma unroll
          for (int h2 = 0; h2 < 2; ++h2) {
            const int j = i2 + h2, s = j >> w;
            const uint32_t cj = h2 ? a1 : a0;
            if (s_done[s]) continue;
            // record the bucket only: s_rank is read by the other bins of this
            // segment in this same phase and is updated after the barrier
            const uint32_t below = (h2 ? e + a0 : e) - s_base[s], r = (uint32_t)s_rank[s];
            if (below < r && r <= below + cj) {
              s_dig[s] = j & (nbin - 1);
              s_bel[s] = (int)below;
              s_cnt2[s] = (int)cj;
              s_wq[s] = wit[j];
            }
          }
          __syncthreads();
          for (int s = threadIdx.x; s < nseg; s += blockDim.x) {
            if (s_done[s]) continue;
            const int cnt = s_cnt2[s];
            s_cnt2[s] = 0;
            const int ns = max(0, s_sh[s] - w);
            s_pre[s] |= (uint64_t)s_dig[s] << ns;
            s_rank[s] -= s_bel[s];
            s_sh[s] = ns;
            if (cnt == 1) {
              s_res[s] = skey(sc, sid, cap, c, s_wq[s]);
              s_done[s] = 1;
            } else if (cnt == 0) {   // counts inconsistent with the rank
              atomicOr(T.err, kErrPartition);
              s_done[s] = 1;
            } else if (ns == 0) {
              s_res[s] = s_pre[s];
              s_done[s] = 1;
            } else {
              pending = 1;
            }
          }
        } else {
          // one warp per segment: a scan of the segment's bins across the lanes
          for (int s = warp; s < nseg; s += nwarps) {
            if (s_done[s]) continue;
            uint32_t *h = hist + (s << w) + lane * per;
            const int nb = max(0, min(per, nbin - lane * per));
            uint32_t sum = 0;
            for (int i = 0; i < nb; ++i) sum += h[i];
            uint32_t inc = sum;
            for (int o2 = 1; o2 < 32; o2 <<= 1) {
              const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o2);
              if (lane >= o2) inc += y;
            }
            const uint32_t r = (uint32_t)s_rank[s];
            const bool mine = inc - sum < r && r <= inc;
            if (mine) {
              uint32_t below = inc - sum, cj = h[0];
              int i = 0;
              while (below + cj < r) {   // ends inside this lane's bins (r <= inc)
                below += cj;
                cj = h[++i];
              }
              const int ns = max(0, s_sh[s] - w), dg = lane * per + i;
              s_dig[s] = dg;
              s_pre[s] |= (uint64_t)dg << ns;
              s_rank[s] = (int)(r - below);
              s_sh[s] = ns;
              if (cj == 1) {
                s_res[s] = skey(sc, sid, cap, c, wit[(s << w) + dg]);
                s_done[s] = 1;
              } else if (ns == 0) {
                s_res[s] = s_pre[s];
                s_done[s] = 1;
              } else {
                pending = 1;
              }
            }
            if (!__any_sync(0xffffffffu, mine) && lane == 0) {   // counts inconsistent with the rank
              atomicOr(T.err, kErrPartition);
              s_done[s] = 1;
            }
            for (int i = 0; i < nb; ++i) h[i] = 0;
          }
        }
        if (!__syncthreads_or(pending)) break;
      }
      hist_ready = false;
      // node keys
      for (int s = threadIdx.x; s < nseg; s += blockDim.x) {
        int64_t bfs = (i0 << u) + s;
        int64_t v = veb_slot(l, t, bfs);
        o.node[v] = Node{s_res[s], (int32_t)veb_slot(l, t + 1, 2 * bfs), (int32_t)veb_slot(l, t + 1, 2 * bfs + 1)};
      }
      // stable partition by a block scan of the left flags (positions blocked
      // per thread); when the next level also selects by radix, its first
      // pass's histogram (the top bits of the next split coordinate, per
      // child segment) is counted on the way
      int64_t nst_, nsz_;
      seg_range(m0, u + 1, 0, nst_, nsz_);
      const bool next_radix = u + 1 < U && nsz_ > kWarpMode;
      const int wn = LB - 1 - u;             // the next level's digit width, LB - (u + 1)
      const int cn = (t + 1) % dim;
      if (next_radix) {
        // the children's bounds: the parent's, cut at the median's
        // coordinate in the split dimension (left: coordinates <= v, right:
        // >= v); and their open key bits in the next split dimension
        for (int s = threadIdx.x; s < nseg; s += blockDim.x) {
          const int32_t v = (int32_t)(s_res[s] >> 31);
          for (int cc = 0; cc < dim; ++cc) {
            const int32_t lo = bcur[(s * dim + cc) * 2], hi = bcur[(s * dim + cc) * 2 + 1];
            bnxt[(2 * s * dim + cc) * 2] = lo;
            bnxt[(2 * s * dim + cc) * 2 + 1] = cc == c ? v : hi;
            bnxt[((2 * s + 1) * dim + cc) * 2] = cc == c ? v : lo;
            bnxt[((2 * s + 1) * dim + cc) * 2 + 1] = hi;
          }
          for (int ch = 2 * s; ch <= 2 * s + 1; ++ch)
            s_shn[ch] = open_key_bits(bnxt[(ch * dim + cn) * 2], bnxt[(ch * dim + cn) * 2 + 1]);
        }
      }
      const int ipt = (cap + blockDim.x - 1) / blockDim.x;   // 2, 4 or 8 (cap <= 8 TH)
      const int q0 = threadIdx.x * ipt;
      // this thread's positions' records and segments, read once (one vector
      // load each where the positions fill one: no bank conflicts between
      // the lanes' neighbouring positions)
      uint32_t cq[4], sq[2];   // 16-bit record indices, 8-bit segments, packed
      if (ipt == 8) {
        const uint4 cv = *reinterpret_cast<const uint4 *>(cur + q0);
        const uint2 sv = *reinterpret_cast<const uint2 *>(segid + q0);
        cq[0] = cv.x; cq[1] = cv.y; cq[2] = cv.z; cq[3] = cv.w;
        sq[0] = sv.x; sq[1] = sv.y;
      } else {
        cq[0] = cq[1] = cq[2] = cq[3] = 0;
        sq[0] = sq[1] = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (j < ipt) {
            cq[j >> 1] |= (uint32_t)cur[q0 + j] << (16 * (j & 1));
            sq[j >> 2] |= (uint32_t)segid[q0 + j] << (8 * (j & 3));
          }
        }
      }
#define CQ(j) ((int)((cq[(j) >> 1] >> (16 * ((j) & 1))) & 0xffffu))
#define SQ(j) ((int)((sq[(j) >> 2] >> (8 * ((j) & 3))) & 0xffu))
      uint32_t flags = 0;
      int cnt = 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int q = q0 + j;
        if (j < ipt && q < m0) {
          const bool left = skey(sc, sid, cap, c, CQ(j)) <= s_res[SQ(j)];
          flags |= (uint32_t)left << j;
          cnt += left;
        }
      }
      uint32_t inc = cnt;
      for (int o2 = 1; o2 < 32; o2 <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o2);
        if (lane >= o2) inc += y;
      }
      __syncthreads();
      if (lane == 31) s_w[warp] = inc;
      __syncthreads();
      if (warp == 0) {
        uint32_t x = lane < nwarps ? s_w[lane] : 0, xi = x;
        for (int o2 = 1; o2 < 32; o2 <<= 1) {
          uint32_t y = __shfl_up_sync(0xffffffffu, xi, o2);
          if (lane >= o2) xi += y;
        }
        if (lane < nwarps) s_w[lane] = xi - x;
      }
      __syncthreads();
      uint32_t e = inc - cnt + s_w[warp];
      {
        uint32_t run = e;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int q = q0 + j;
          if (j < ipt && q < m0) {
            const int s = SQ(j);
            if (q == s_st[s]) s_lb[s] = (int)run;
            run += (flags >> j) & 1;
          }
        }
      }
      __syncthreads();
      {
        uint32_t run = e;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int q = q0 + j;
          if (j < ipt && q < m0) {
            const int s = SQ(j);
            int lrank = (int)run - s_lb[s];
            int half = (s_sz[s] + 1) >> 1;
            int rrank = (q - s_st[s]) - lrank;
            bool left = (flags >> j) & 1;
            int dst = left ? s_st[s] + lrank : s_st[s] + half + rrank;
            if (left ? (lrank < 0 || lrank >= half) : (rrank < 0 || rrank >= s_sz[s] - half)) {
              atomicOr(T.err, kErrPartition);
            } else {
              nxt[dst] = (uint16_t)CQ(j);
              segid_n[dst] = (unsigned char)(2 * s + (left ? 0 : 1));   // child segment
              if (next_radix) {   // the child's first digit, below its open key bits
                const int ch = 2 * s + (left ? 0 : 1), sh = s_shn[ch], ns = max(0, sh - wn);
                const uint64_t kn = skey(sc, sid, cap, cn, CQ(j));
                const int dg = (int)((kn >> ns) & ((1u << (sh - ns)) - 1));
                binq[dst] = (uint16_t)dg;
                wit[(ch << wn) + dg] = (uint16_t)CQ(j);
                atomicAdd(&hist[(ch << wn) + dg], 1u);
              }
            }
            run += (flags >> j) & 1;
          }
        }
      }
#undef CQ
#undef SQ
      __syncthreads();
      hist_ready = next_radix;
      unsigned char *ts = segid; segid = segid_n; segid_n = ts;
      int32_t *tb = bcur; bcur = bnxt; bnxt = tb;
    } else {
      // ---------------- warp mode: one warp splits each segment ------------
      // A segment of z <= 64 records.  Above the last level, two per lane
      // (positions a + lane and a + 32 + lane): the median key (rank
      // ceil(z/2) - 1; the keys are distinct) is found bit by bit from the
      // highest bit where the segment's keys differ (a ballot counts the
      // candidates with a 0 there, and the candidates keep the side that
      // holds the rank, until one is left), and the records with keys up to
      // the median take the segment's first ceil(z/2) positions (ballot
      // prefix counts).  At the last level a bitonic network across the warp
      // sorts words (key << 13 | position), distinct and ordered like the
      // keys (positions < cap <= 8192), so that every leaf holds its records
      // in key order.  At the first such level every node's vEB slot is
      // computed once, in heap order (node (u, s) at (1 << u) + s), in the
      // histogram space (free from here on); the leaves use them too.
      if (!slots_ready && nleaf <= (int)blockDim.x) {
        for (int x = threadIdx.x + 1; x < 2 * nleaf; x += blockDim.x) {
          const int ux = 31 - __clz(x);
          nslot[x] = (int32_t)veb_slot(l, t0 + ux, (i0 << ux) + (x - (1 << ux)));
        }
        slots_ready = true;
        __syncthreads();
      }
      const unsigned lt_mask = (1u << lane) - 1;   // lanes before this one
      for (int s = warp; s < nseg; s += nwarps) {
        int a, z;
        seg_range32(m0, u, s, a, z);
        if (z > 64) { if (lane == 0) atomicOr(T.err, kErrPartition); continue; }
        uint64_t med = 0;
        if (u == U - 1) {
          const int mr = ((z + 1) >> 1) - 1;
          if (z <= 32) {
            uint64_t x = lane < z ? (skey(sc, sid, cap, c, cur[a + lane]) << 13) | cur[a + lane] : ~0ull;
            x = warp_sort32(x, lane);
            if (lane < z) nxt[a + lane] = (uint16_t)(x & 8191u);
            med = __shfl_sync(0xffffffffu, x, mr) >> 13;
          } else {
            const int e0 = 2 * lane, e1 = 2 * lane + 1;
            uint64_t x0 = e0 < z ? (skey(sc, sid, cap, c, cur[a + e0]) << 13) | cur[a + e0] : ~0ull;
            uint64_t x1 = e1 < z ? (skey(sc, sid, cap, c, cur[a + e1]) << 13) | cur[a + e1] : ~0ull;
            warp_sort64(x0, x1, lane);
            if (e0 < z) nxt[a + e0] = (uint16_t)(x0 & 8191u);
            if (e1 < z) nxt[a + e1] = (uint16_t)(x1 & 8191u);
            med = __shfl_sync(0xffffffffu, (mr & 1) ? x1 : x0, mr >> 1) >> 13;
          }
        } else {
          const bool v0 = lane < z, v1 = 32 + lane < z;
          const int ra = v0 ? cur[a + lane] : 0, rb = v1 ? cur[a + 32 + lane] : 0;
          const uint64_t k0 = v0 ? skey(sc, sid, cap, c, ra) : 0, k1 = v1 ? skey(sc, sid, cap, c, rb) : 0;
          // the bits where the keys differ: OR and AND over the records
          const uint64_t ko = (v0 ? k0 : 0) | (v1 ? k1 : 0), ka = (v0 ? k0 : ~0ull) & (v1 ? k1 : ~0ull);
          const uint64_t all_or = ((uint64_t)__reduce_or_sync(0xffffffffu, (unsigned)(ko >> 32)) << 32) |
                                  __reduce_or_sync(0xffffffffu, (unsigned)ko);
          const uint64_t all_and = ((uint64_t)__reduce_and_sync(0xffffffffu, (unsigned)(ka >> 32)) << 32) |
                                   __reduce_and_sync(0xffffffffu, (unsigned)ka);
          const uint64_t diff = all_or ^ all_and;
          bool c0 = v0, c1 = v1;   // still candidates for the median
          int r = ((z + 1) >> 1) - 1, n = z;
          for (int bit = diff ? 63 - __clzll(diff) : -1; bit >= 0 && n > 1; --bit) {
            const bool b0 = (k0 >> bit) & 1, b1 = (k1 >> bit) & 1;
            const int cz = __popc(__ballot_sync(0xffffffffu, c0 && !b0)) + __popc(__ballot_sync(0xffffffffu, c1 && !b1));
            if (r < cz) {
              c0 = c0 && !b0;
              c1 = c1 && !b1;
              n = cz;
            } else {
              c0 = c0 && b0;
              c1 = c1 && b1;
              r -= cz;
              n -= cz;
            }
          }
          const unsigned m0b = __ballot_sync(0xffffffffu, c0), m1b = __ballot_sync(0xffffffffu, c1);
          med = __shfl_sync(0xffffffffu, m0b ? k0 : k1, __ffs(m0b ? m0b : m1b) - 1);
          // the split: left records first, each side in position order
          const bool l0 = v0 && k0 <= med, l1 = v1 && k1 <= med;
          const unsigned L0 = __ballot_sync(0xffffffffu, l0), L1 = __ballot_sync(0xffffffffu, l1);
          const unsigned R0 = __ballot_sync(0xffffffffu, v0 && !l0), R1 = __ballot_sync(0xffffffffu, v1 && !l1);
          const int nl = __popc(L0) + __popc(L1);
          if (v0) nxt[a + (l0 ? __popc(L0 & lt_mask) : nl + __popc(R0 & lt_mask))] = (uint16_t)ra;
          if (v1) nxt[a + (l1 ? __popc(L0) + __popc(L1 & lt_mask) : nl + __popc(R0) + __popc(R1 & lt_mask))] = (uint16_t)rb;
          if (lane == 0 && (n != 1 || __popc(m0b) + __popc(m1b) != 1 || nl != (z + 1) >> 1))
            atomicOr(T.err, kErrPartition);
        }
        if (slots_ready) {
          const int x = (1 << u) + s;
          if (lane == 0) o.node[nslot[x]] = Node{med, nslot[2 * x], nslot[2 * x + 1]};
        } else {
          // the node's vEB slot and its children's, three lanes at once
          const int64_t bfs = (i0 << u) + s;
          const int64_t sl = lane < 3 ? veb_slot(l, lane ? t + 1 : t, lane ? 2 * bfs + lane - 1 : bfs) : 0;
          const int64_t vl = __shfl_sync(0xffffffffu, sl, 1), vr = __shfl_sync(0xffffffffu, sl, 2);
          if (lane == 0) o.node[sl] = Node{med, (int32_t)vl, (int32_t)vr};
        }
      }
      __syncthreads();
    }
    uint16_t *tmp = cur; cur = nxt; nxt = tmp;
  }

  // leaves: slot, leaf range, box, live count; then the subtree's internal
  // nodes bottom-up
  const int64_t nleaves_tree = (int64_t)1 << T.h;
  if (nleaf <= (int)blockDim.x) {
    // Every node's vEB slot once, in heap order in shared memory (node (u, s)
    // at (1 << u) + s; the histogram space is free now), then per channel --
    // the live counts, then each coordinate's low and high bounds -- a value
    // per leaf in a thread, pairs combined by warp shuffles up to the warp's
    // subtree, the warps' results by warp 0: no barrier and no read-back of
    // global memory per level.
    int32_t *wlo = nslot + 2 * nleaf, *whi = wlo + 32; // [32] each: the warps' results
    if (!slots_ready) {
      for (int x = threadIdx.x + 1; x < 2 * nleaf; x += blockDim.x) {
        const int u = 31 - __clz(x);
        nslot[x] = (int32_t)veb_slot(l, t0 + u, (i0 << u) + (x - (1 << u)));
      }
      __syncthreads();
    }
    const int lf = threadIdx.x;
    const bool has = lf < nleaf;
    int a = 0, z = 0;
    if (has) {
      int64_t a64, z64;
      seg_range(m0, U, lf, a64, z64);
      a = (int)a64;
      z = (int)z64;
      const int64_t leaf = (i0 << U) + lf;
      o.node[nslot[nleaf + lf]] = Node{0, (int32_t)(-1 - leaf), 0};
      o.leaf_off[leaf] = (int32_t)(start0 + a);
      if (leaf == nleaves_tree - 1) o.leaf_off[nleaves_tree] = (int32_t)T.s;
    }
    const int kw = U < 5 ? U : 5;        // levels combined inside a warp
    for (int ch = -1; ch < dim; ++ch) {  // ch = -1: live counts
      int32_t lo = ch < 0 ? 0 : INT32_MAX, hi = INT32_MIN;
      if (has) {
        if (ch < 0) {
          lo = z;
        } else {
          for (int q = a; q < a + z; ++q) {
            const int32_t x = sc[ch * cap + cur[q]];
            lo = min(lo, x);
            hi = max(hi, x);
          }
        }
      }
      auto put = [&](int x, int32_t vlo, int32_t vhi) {   // node at heap index x
        const int64_t v = nslot[x];
        if (ch < 0) {
          o.live[v] = vlo;
        } else {
          o.box[v * 2 * dim + ch] = vlo;
          o.box[v * 2 * dim + dim + ch] = vhi;
        }
      };
      if (has) put(nleaf + lf, lo, hi);
      for (int k = 1; k <= kw; ++k) {
        const int32_t plo = __shfl_xor_sync(0xffffffffu, lo, 1 << (k - 1));
        const int32_t phi = __shfl_xor_sync(0xffffffffu, hi, 1 << (k - 1));
        lo = ch < 0 ? lo + plo : min(lo, plo);
        hi = max(hi, phi);
        const int idx = lf >> k;         // parent's index at level U - k
        if ((lane & ((1 << k) - 1)) == 0 && idx < (nleaf >> k)) put((1 << (U - k)) + idx, lo, hi);
      }
      if (U > 5) {                       // the warps' subtrees: combined by warp 0
        if (lane == 0) {
          wlo[warp] = lo;
          whi[warp] = hi;
        }
        __syncthreads();
        if (warp == 0) {
          const int nw = nleaf >> 5;     // <= 32
          lo = lane < nw ? wlo[lane] : (ch < 0 ? 0 : INT32_MAX);
          hi = lane < nw ? whi[lane] : INT32_MIN;
          for (int k = 1; k <= U - 5; ++k) {
            const int32_t plo = __shfl_xor_sync(0xffffffffu, lo, 1 << (k - 1));
            const int32_t phi = __shfl_xor_sync(0xffffffffu, hi, 1 << (k - 1));
            lo = ch < 0 ? lo + plo : min(lo, plo);
            hi = max(hi, phi);
            const int idx = lane >> k;
            if ((lane & ((1 << k) - 1)) == 0 && idx < (nw >> k)) put((1 << (U - 5 - k)) + idx, lo, hi);
          }
        }
        __syncthreads();
      }
    }
  } else {
    // more leaves than threads: leaves first, then each level from its
    // children in global memory
    for (int lf = threadIdx.x; lf < nleaf; lf += blockDim.x) {
      int64_t a64, z64;
      seg_range(m0, U, lf, a64, z64);
      int a = (int)a64, z = (int)z64;
      int64_t leaf = (i0 << U) + lf;
      int64_t v = veb_slot(l, T.h, leaf);
      o.node[v] = Node{0, (int32_t)(-1 - leaf), 0};
      o.live[v] = z;
      o.leaf_off[leaf] = (int32_t)(start0 + a);
      if (leaf == nleaves_tree - 1) o.leaf_off[nleaves_tree] = (int32_t)T.s;
      for (int cc = 0; cc < dim; ++cc) {
        int32_t lo = INT32_MAX, hi = INT32_MIN;
        for (int q = a; q < a + z; ++q) {
          int32_t x = sc[cc * cap + cur[q]];
          lo = min(lo, x);
          hi = max(hi, x);
        }
        o.box[v * 2 * dim + cc] = lo;
        o.box[v * 2 * dim + dim + cc] = hi;
      }
    }
    // internal nodes of the subtree, bottom-up (children are in global memory)
    for (int u = U - 1; u >= 0; --u) {
      __syncthreads();
      for (int s = threadIdx.x; s < (1 << u); s += blockDim.x) {
        int64_t bfs = (i0 << u) + s;
        int t = t0 + u;
        int64_t v = veb_slot(l, t, bfs);
        int64_t vl = veb_slot(l, t + 1, 2 * bfs), vr = veb_slot(l, t + 1, 2 * bfs + 1);
        o.live[v] = o.live[vl] + o.live[vr];
        for (int cc = 0; cc < dim; ++cc) {
          o.box[v * 2 * dim + cc] = min(o.box[vl * 2 * dim + cc], o.box[vr * 2 * dim + cc]);
          o.box[v * 2 * dim + dim + cc] =
              max(o.box[vl * 2 * dim + dim + cc], o.box[vr * 2 * dim + dim + cc]);
        }
      }
    }
  }
  // point records in leaf order (16-byte stores: a record is rs ints, a
  // multiple of 4)
  const int rs = rec_ints(dim);
  for (int q = threadIdx.x; q < m0; q += blockDim.x) {
    const int it = cur[q];
    int4 *dst = reinterpret_cast<int4 *>(o.pts + (start0 + q) * rs);
    for (int c4 = 0; c4 < rs; c4 += 4) {
      int32_t v[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int cc = c4 + e;
        v[e] = cc < dim ? sc[cc * cap + it] : cc == dim ? sid[it] : 0;
      }
      dst[c4 >> 2] = make_int4(v[0], v[1], v[2], v[3]);
    }
  }
}

// ---------------------------------------------------------------------------
// K4: boxes and live counts of the global-level nodes, deepest level first,
// in one cooperative launch (a grid barrier between depths)
// ---------------------------------------------------------------------------

struct BoxWork {               // the nodes of one depth t of the trees with global levels below t
  int nact, t;
  const int32_t *act;          // [nact] trees
  const int64_t *node;         // [nact + 1] prefix of 2^t nodes per tree
  int64_t total;
};

struct FinishParams {
  int dim, nlev;
  const DTree *tree;
  const BoxWork *bw;           // [nlev], by depth
  unsigned *bar;
  unsigned long long *err;
};

__device__ void box_up(const FinishParams &F, const BoxWork &W, int64_t g) {
  const int j = find_le(W.node, W.nact, g);
  const DTree &D = F.tree[W.act[j]];
  const NodeOut o = D.out;
  const int l = D.h + 1, t = W.t, dim = F.dim;
  const int64_t i = g - W.node[j];
  const int64_t v = veb_slot(l, t, i), vl = veb_slot(l, t + 1, 2 * i), vr = veb_slot(l, t + 1, 2 * i + 1);
  o.live[v] = o.live[vl] + o.live[vr];
  for (int c = 0; c < dim; ++c) {
    o.box[v * 2 * dim + c] = min(o.box[vl * 2 * dim + c], o.box[vr * 2 * dim + c]);
    o.box[v * 2 * dim + dim + c] = max(o.box[vl * 2 * dim + dim + c], o.box[vr * 2 * dim + dim + c]);
  }
}

__global__ void __launch_bounds__(256) k_build_finish(const FinishParams F) {
  for (int t = F.nlev - 1; t >= 0; --t) {
    const BoxWork &W = F.bw[t];
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < W.total;
         g += (int64_t)gridDim.x * blockDim.x)
      box_up(F, W, g);
    if (t > 0) grid_barrier(F.bar, F.err);
  }
}

// ---------------------------------------------------------------------------
// buffer helpers
// ---------------------------------------------------------------------------

// One CTA per list: bitonic sort of its n <= 16384 ids (np2 = n rounded up to
// a power of two, padded with INT32_MAX).
__global__ void k_sort_small_many(const SortList *lists) {
  extern __shared__ int32_t a[];
  const SortList L = lists[blockIdx.x];
  int32_t *ids = L.ids;
  const int n = L.n, np2 = L.np2;
  for (int i = threadIdx.x; i < np2; i += blockDim.x) a[i] = i < n ? ids[i] : INT32_MAX;
  __syncthreads();
  for (int k = 2; k <= np2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < np2; i += blockDim.x) {
        int p = i ^ j;
        if (p > i) {
          bool up = (i & k) == 0;
          int32_t x = a[i], y = a[p];
          if ((x > y) == up) { a[i] = y; a[p] = x; }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) ids[i] = a[i];
}

constexpr size_t kSubtreeSmemMax = 212 * 1024;   // dynamic part; static part ~6 KB

// Blocks of a cooperative launch of `fn` with `threads` threads: every block
// that fits on the device at once (SMs x resident blocks per SM), cached per
// kernel and device.
int coop_grid(const void *fn, int threads, int *out) {
  static std::mutex mu;
  static std::vector<std::pair<std::pair<const void *, int>, int>> cache;
  int dev = 0;
  int st = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (st) return st;
  std::lock_guard<std::mutex> lk(mu);
  for (auto &c : cache)
    if (c.first.first == fn && c.first.second == dev) {
      *out = c.second;
      return BDL_OK;
    }
  int sms = 0, per = 0;
  st = cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
  if (!st) st = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, 0), "occupancy");
  if (st) return st;
  if (per < 1) return set_error(BDL_EINTERNAL, "cooperative kernel does not fit on an SM");
  *out = sms * per;
  cache.push_back({{fn, dev}, *out});
  return BDL_OK;
}

// Dynamic shared memory of a k_subtree CTA of `th` threads for subtrees of
// at most `cap` records.
size_t subtree_smem_bytes(int dim, int cap, int th = kSubThreads) {
  return (size_t)cap * (4 * dim + 4) + (size_t)(2 * th) * (4 + 2) + (size_t)cap * 2 * 3 + 2 * (size_t)cap +
         2 * (size_t)(th / 8) * dim * 2 * 4;
}

NodeOut node_out(Tree *t) {
  NodeOut o;
  o.pts = t->pts;
  o.box = t->box;
  o.live = t->live_nodes;
  o.leaf_off = t->leaf_off;
  o.node = t->node;
  return o;
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Relative time of an on-chip subtree of n records with U levels below its
// root: per level, a fixed part (block barriers, bin scans) and a part that
// grows with the records (a CTA of 8,192 records: 0.3 + 0.7 per level).
double subtree_cost(int64_t n, int U) { return (double)std::max(U, 1) * (0.3 + 0.7 * (double)n / 8192.0); }

// Finish time of `cost` (any order; run largest first) on `slots` CTA slots
// that each take the next subtree when free (the block scheduler's order).
double schedule_makespan(std::vector<double> cost, int slots) {
  std::sort(cost.begin(), cost.end(), std::greater<double>());
  std::priority_queue<double, std::vector<double>, std::greater<double>> q;
  for (int i = 0; i < slots; ++i) q.push(0.0);
  double ms = 0;
  for (double c : cost) {
    const double t = q.top() + c;
    q.pop();
    q.push(t);
    ms = std::max(ms, t);
  }
  return ms;
}

// Global levels of a tree with `e` extra ones, bounded by gmax and by the
// global kernels' tiles: a level may split only segments of at least `tile`
// records (so that a tile meets at most two segments).
int deepened_g(const BuildTree &b, int gmax, int e, int tile) {
  int g = b.g;
  while (e > 0 && g < gmax && (b.s >> g) >= tile) {
    ++g;
    --e;
  }
  return g;
}

// Extra global levels for the trees with fewer than the deepest one's: the
// global kernel runs gmax levels anyway, so splitting such a tree further
// costs only its records' passes, and its smaller subtrees can fill the last
// wave of the subtree launch (one CTA per SM, often a few left over).  Of
// 0, 1, 2 or as many extra levels as allowed (the same for every such tree),
// the one with the shortest schedule under subtree_cost is applied.
void balance_subtrees(std::vector<BuildTree> &bt, int gmax, int slots, int tile) {
  if (gmax == 0) return;
  double best = 0;
  int best_e = 0;
  for (int e : {0, 1, 2, 64}) {
    std::vector<double> c;
    for (const auto &b : bt) {
      const int g = deepened_g(b, gmax, e, tile);
      const double x = subtree_cost(ceil_div(b.s, (int64_t)1 << g), b.h - g);
      c.insert(c.end(), (size_t)1 << g, x);
    }
    const double ms = schedule_makespan(std::move(c), slots);
    if (e == 0 || ms < best * 0.99) {
      best = ms;
      best_e = e;
    }
  }
  for (auto &b : bt) b.g = deepened_g(b, gmax, best_e, tile);
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Host image of a build plan: every per-tree, per-level and per-source array
// the kernels read, serialized into one buffer that is uploaded with a single
// copy.
struct PlanImage {
  std::vector<unsigned char> bytes;
  template <class T>
  size_t put(const std::vector<T> &v) {
    size_t off = align256(bytes.size());
    bytes.resize(off + std::max<size_t>(v.size() * sizeof(T), 8));
    if (!v.empty()) memcpy(bytes.data() + off, v.data(), v.size() * sizeof(T));
    return off;
  }
};

}  // namespace

int smem_subtree_capacity(int dim) {
  for (int cap = 8192; cap >= 2048; cap >>= 1)
    if (subtree_smem_bytes(dim, cap) <= kSubtreeSmemMax) return cap;
  return 2048;
}

int build_trees(bdl_forest *af, int dim, std::vector<BuildTree> &bt, const std::vector<ClearedSrc> &cl,
                cudaStream_t s) {
  if (af->cfg.split_rule == BDL_SPLIT_SPATIAL) return build_trees_spatial(af, dim, bt, cl, s);
  return build_trees_object(af, dim, bt, cl, s);
}

int build_trees_object(bdl_forest *af, int dim, std::vector<BuildTree> &bt,
                const std::vector<ClearedSrc> &cl, cudaStream_t s) {
  if (bt.empty()) return BDL_OK;
  const int ntree = (int)bt.size();
  const int cap = smem_subtree_capacity(dim);
  const int tile = std::min(4096, cap);

  // ---- layout: staging bases and global levels per tree ----
  int64_t S = 0;
  int gmax = 0;
  for (auto &b : bt) {
    b.base = S;
    S += (b.s + 7) / 8 * 8;
    int g = 0;
    while (g < b.h && ceil_div(b.s, (int64_t)1 << g) > cap) g++;
    b.g = g;
    gmax = std::max(gmax, g);
  }
  S = std::max<int64_t>(S, 8);
  int sms = 0;
  {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 1;
    if (const char *e = getenv("BDL_BUILD_SLOTS")) {   // slots of the schedule model
      const int v = atoi(e);
      if (v > 0) sms = v;
    }
    balance_subtrees(bt, gmax, std::max(sms, 1), tile);   // one subtree CTA per SM (its shared memory)
  }

  // ---- plan arrays ----
  std::vector<DTree> dt(ntree);
  std::vector<int64_t> pool_off(ntree + 1, 0);
  std::vector<int32_t> sub_ord(ntree);
  for (int j = 0; j < ntree; ++j) {
    const BuildTree &b = bt[j];
    DTree &d = dt[j];
    memset(&d, 0, sizeof(d));
    d.base = b.base;
    d.s = b.s;
    d.h = b.h;
    d.g = b.g;
    d.sel = b.g & 1;
    d.out = node_out(b.tree);
    d.from_cleared = b.from_cleared;
    d.pool_lo = b.pool_lo;
    d.pbuf = b.pool.buf;
    d.pnbuf = b.pool.nbuf;
    d.parr = b.pool.arr;
    d.pfirst = b.pool.first;
    d.idtab = b.idtab;
    d.err = b.err;
    pool_off[j + 1] = pool_off[j] + (b.s - b.from_cleared);
  }
  // the subtree launch runs the trees with the costliest subtrees first
  for (int j = 0; j < ntree; ++j) sub_ord[j] = j;
  auto cost_of = [&](int j) { return subtree_cost(ceil_div(bt[j].s, (int64_t)1 << bt[j].g), bt[j].h - bt[j].g); };
  std::stable_sort(sub_ord.begin(), sub_ord.end(), [&](int a, int b) { return cost_of(a) > cost_of(b); });
  // trees whose subtrees hold fewer than kSmallSub records (buffer trees,
  // the smallest trees) go to the 256-thread instance, in a launch of their
  // own after the 1,024-thread one, when there are enough of them to fill
  // the SMs (a batched build over many forests); a few stay in the large
  // launch, whose last wave they fill.  Each launch has its own order and
  // prefix.
  auto small = [&](int j) { return ceil_div(bt[j].s, (int64_t)1 << bt[j].g) < kSmallSub; };
  int64_t nsmall_sub = 0;
  for (int j = 0; j < ntree; ++j)
    if (small(j)) nsmall_sub += (int64_t)1 << bt[j].g;
  const bool split_small = nsmall_sub >= std::max(sms, 1);
  const int nbig = split_small ? (int)(std::stable_partition(sub_ord.begin(), sub_ord.end(),
                                                             [&](int j) { return !small(j); }) -
                                       sub_ord.begin())
                               : ntree;
  std::vector<int64_t> sub_blk(nbig + 1, 0), sub_blk_s(ntree - nbig + 1, 0);
  for (int j = 0; j < nbig; ++j) sub_blk[j + 1] = sub_blk[j] + ((int64_t)1 << bt[sub_ord[j]].g);
  for (int j = nbig; j < ntree; ++j)
    sub_blk_s[j - nbig + 1] = sub_blk_s[j - nbig] + ((int64_t)1 << bt[sub_ord[j]].g);
  const int TB = kCoopThreads;   // cleared records per gather work item
  std::vector<DCleared> dc(cl.size());
  std::vector<int64_t> cl_blk(cl.size() + 1, 0);
  for (size_t i = 0; i < cl.size(); ++i) {
    dc[i].pts = cl[i].pts;
    dc[i].size = cl[i].size;
    dc[i].dst = cl[i].dst;
    dc[i].pad_ = 0;
    cl_blk[i + 1] = cl_blk[i] + ceil_div(cl[i].size, TB);
  }
  // per global level: the trees still above the on-chip size, with segment
  // and tile prefixes; the same trees get their global nodes boxed bottom-up
  struct LevelHost { int nact; size_t act, seg, tile, node, lt; int64_t nseg, ntile, recs; };
  std::vector<LevelHost> lv(gmax);
  std::vector<int32_t> act_all;
  std::vector<LvTree> lt_all;
  std::vector<int64_t> pre_all;
  std::vector<std::pair<size_t, size_t>> act_pos(gmax), seg_pos(gmax), tile_pos(gmax), node_pos(gmax);
  int64_t nseg_max = 0;
  // each tree's first segment at each global level (for the histograms the
  // partition of the level before accumulates)
  std::vector<std::vector<int64_t>> segoff(gmax + 1, std::vector<int64_t>(ntree, -1));
  for (int it = 0; it < gmax; ++it) {
    int64_t segs = 0;
    for (int j = 0; j < ntree; ++j)
      if (bt[j].g > it) {
        segoff[it][j] = segs;
        segs += (int64_t)1 << it;
      }
  }
  for (int it = 0; it < gmax; ++it) {
    LevelHost &L = lv[it];
    L.act = act_all.size();
    L.lt = lt_all.size();
    int64_t segs = 0, tiles = 0;
    L.recs = 0;
    std::vector<int64_t> sp{0}, tp{0}, np{0};
    for (int j = 0; j < ntree; ++j) {
      if (bt[j].g <= it) continue;
      act_all.push_back(j);
      L.recs += bt[j].s;
      LvTree T;
      T.base = bt[j].base;
      T.s = bt[j].s;
      T.h = bt[j].h;
      T.t = it;
      T.c = it % dim;
      T.seg_off = segs;
      T.next_seg = segoff[it + 1][j];
      T.tile_off = tiles;
      T.out = dt[j].out;
      T.err = dt[j].err;
      lt_all.push_back(T);
      segs += (int64_t)1 << it;
      tiles += ceil_div(bt[j].s, tile);
      sp.push_back(segs);
      tp.push_back(tiles);
      np.push_back(segs);      // 2^it nodes per tree at depth it, same prefix as segments
    }
    L.nact = (int)(act_all.size() - L.act);
    L.nseg = segs;
    L.ntile = tiles;
    L.seg = pre_all.size(); pre_all.insert(pre_all.end(), sp.begin(), sp.end());
    L.tile = pre_all.size(); pre_all.insert(pre_all.end(), tp.begin(), tp.end());
    L.node = pre_all.size(); pre_all.insert(pre_all.end(), np.begin(), np.end());
    nseg_max = std::max(nseg_max, segs);
  }
  PlanImage img;
  const size_t o_dt = img.put(dt), o_dc = img.put(dc), o_clb = img.put(cl_blk),
               o_pool = img.put(pool_off), o_sub = img.put(sub_blk), o_subs = img.put(sub_blk_s),
               o_ord = img.put(sub_ord),
               o_act = img.put(act_all),
               o_pre = img.put(pre_all), o_lt = img.put(lt_all);
  std::vector<TreeSeg> pk_segs;
  std::vector<int64_t> pk_pre;
  {
    std::vector<Tree *> trees;
    for (auto &b : bt) trees.push_back(b.tree);
    pack_nodes_entries(trees, dim, pk_segs, pk_pre);
  }
  const size_t o_pk = img.put(pk_segs), o_pkpre = img.put(pk_pre);
  // per-level descriptors of the fused kernels: placeholders here, filled in
  // once the device addresses they hold are known
  const size_t o_lw = img.put(std::vector<LevelWork>(gmax)), o_bw = img.put(std::vector<BoxWork>(gmax));

  // ---- one device block: scratch + plan ----
  const size_t stg_bytes = align256((size_t)(dim + 1) * S * 4);
  const size_t cand_bytes = gmax ? align256((size_t)S * 8) : 0;
  // histograms and segment states alternate between two halves: a level
  // fills the next level's half while it reads its own
  const size_t hist_half = align256((size_t)nseg_max * kHistBins * 4), hist_bytes = 2 * hist_half;
  const size_t seg_half = align256((size_t)nseg_max * sizeof(SegState)), seg_bytes = 2 * seg_half;
  // per-tree gather cursors, then (at the next 256-byte boundary) the two
  // fused kernels' grid-barrier words
  const size_t cursor_bytes = align256((size_t)ntree * 8) + 256;
  const size_t plan_bytes = align256(img.bytes.size());
  const size_t total = 2 * stg_bytes + cand_bytes + hist_bytes + seg_bytes + cursor_bytes + plan_bytes;
  void *block = nullptr;
  int st = dev_alloc(af, &block, total, s);
  if (st) return st;
  unsigned char *p = (unsigned char *)block;
  int32_t *stg[2];
  stg[0] = (int32_t *)p; p += stg_bytes;
  stg[1] = (int32_t *)p; p += stg_bytes;
  uint64_t *cand = (uint64_t *)p; p += cand_bytes;
  SegState *seg = (SegState *)p; p += seg_bytes;     // zeroed here, then each level clears
  uint32_t *hist = (uint32_t *)p; p += hist_bytes;   // the next one's states and its own
  unsigned long long *cursor = (unsigned long long *)p; p += cursor_bytes;   // histograms
  unsigned char *plan = p;
  unsigned *bar = (unsigned *)((unsigned char *)cursor + align256((size_t)ntree * 8));   // [0..1] levels, [2..3] boxes
  const DTree *d_tree = (const DTree *)(plan + o_dt);
  const int32_t *d_act = (const int32_t *)(plan + o_act);
  const int64_t *d_pre = (const int64_t *)(plan + o_pre);

  // ---- the fused kernels' per-level descriptors, with device addresses ----
  GatherParams G;
  G.nsrc = (int)cl.size();
  G.ntrees = ntree;
  G.dim = dim;
  G.S = S;
  G.stg = stg[0];
  G.cursor = cursor;
  G.tree = d_tree;
  G.cl = (const DCleared *)(plan + o_dc);
  G.cl_blk = (const int64_t *)(plan + o_clb);
  G.pool_off = (const int64_t *)(plan + o_pool);
  double lv_bytes = 0;
  {
    LevelWork *lw = (LevelWork *)(img.bytes.data() + o_lw);
    BoxWork *bw = (BoxWork *)(img.bytes.data() + o_bw);
    for (int it = 0; it < gmax; ++it) {
      const LevelHost &L = lv[it];
      LevelWork W;
      memset(&W, 0, sizeof(W));
      LvParams &P = W.P;
      P.nact = L.nact;
      P.dim = dim;
      P.tile = tile;
      P.it = it;
      P.S = S;
      P.src = stg[it & 1];
      P.dst = stg[(it & 1) ^ 1];
      P.hist = (uint32_t *)((unsigned char *)hist + (it & 1) * hist_half);
      P.seg = (SegState *)((unsigned char *)seg + (it & 1) * seg_half);
      P.hist_next = (uint32_t *)((unsigned char *)hist + ((it + 1) & 1) * hist_half);
      P.seg_next = (SegState *)((unsigned char *)seg + ((it + 1) & 1) * seg_half);
      P.nseg_next = it + 1 < gmax ? lv[it + 1].nseg : 0;
      P.cand = cand;
      P.one = lt_all[L.lt];
      P.lt = (const LvTree *)(plan + o_lt) + L.lt;
      P.act_seg = d_pre + L.seg;
      P.act_tile = d_pre + L.tile;
      W.ntile = L.ntile;
      W.nseg = L.nseg;
      memcpy(lw + it, &W, sizeof(W));
      BoxWork B{L.nact, it, d_act + L.act, d_pre + L.node, L.nseg};
      memcpy(bw + it, &B, sizeof(B));
      // algorithmic bytes per record of the level: the split coordinate (4)
      // for the histogram and for the candidate gather, the record (d + 1
      // words) read and written by the partition
      lv_bytes += (double)L.recs * (8.0 + 8.0 * (dim + 1));
    }
  }
  st = h2d(plan, img.bytes.data(), img.bytes.size(), s);
  // segment states, histograms and cursors (contiguous) start at zero
  if (!st) st = small_zero(seg, seg_bytes + hist_bytes + cursor_bytes, s);
  if (st) {
    dev_free(af, block, total, s);
    return st;
  }
  auto coop = [&](const void *fn, int threads, void **args, int kid, double bytes) {
    int g = 0;
    int e = coop_grid(fn, threads, &g);
    if (e) return e;
    KScope ks_(kid, s, bytes);
    return cuda_check(cudaLaunchCooperativeKernel(fn, dim3((unsigned)g), dim3((unsigned)threads), args, 0, s),
                      "cooperative build kernel");
  };

  // ---- gather (K5) and the global levels (K1/K2), one cooperative launch ----
  if (cl_blk.back() || pool_off.back() || gmax) {
    // algorithmic bytes of the gather: every cleared record read, every live
    // one written to staging (d + 1 words); a pool entry's coordinates
    // gathered from the id table and written
    double cl_read = 0, cl_live = 0;
    for (auto &c : cl) cl_read += (double)c.size;
    for (auto &b : bt) cl_live += (double)b.from_cleared;
    const double rin = 4.0 * rec_ints(dim), rst = 4.0 * (dim + 1);
    const double gbytes = cl_read * rin + cl_live * rst + (double)pool_off.back() * (4.0 * dim + rst);
    LevelsParams B;
    B.G = G;
    B.cl_blocks = cl_blk.back();
    B.pool_total = pool_off.back();
    B.lv = (const LevelWork *)(plan + o_lw);
    B.nlev = gmax;
    B.bar = bar;
    B.err = bt[0].err;
    void *args[] = {(void *)&B};
    st = coop((const void *)k_build_levels, kCoopThreads, args, kK_build_levels, gbytes + lv_bytes);
  }

  // ---- subtrees on chip: the 1,024-thread launch, then the 256-thread one ----
  for (int part = 0; part < 2 && !st; ++part) {
    const int j0 = part ? nbig : 0, j1 = part ? ntree : nbig;
    if (j0 == j1) continue;
    SubParams P;
    P.ntrees = j1 - j0;
    P.dim = dim;
    P.cap = part ? kSmallSub : cap;
    P.S = S;
    P.stg[0] = stg[0];
    P.stg[1] = stg[1];
    P.tree = d_tree;
    P.sub_blk = (const int64_t *)(plan + (part ? o_subs : o_sub));
    P.sub_ord = (const int32_t *)(plan + o_ord) + j0;
    const int th = part ? kSmallSubThreads : kSubThreads;
    const size_t smem = subtree_smem_bytes(dim, P.cap, th);
    const void *fn = part ? (const void *)k_subtree<kSmallSubThreads> : (const void *)k_subtree<kSubThreads>;
    st = cuda_check(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                    "cudaFuncSetAttribute(k_subtree)");
    if (st) break;
    // algorithmic bytes: every record read from staging (d + 1 words) and
    // written in leaf order (rec_ints words); every node below the global
    // levels written (16-byte node, box, live count); the leaf offsets
    double sub_bytes = 0;
    for (int j = j0; j < j1; ++j) {
      const BuildTree &b = bt[sub_ord[j]];
      sub_bytes += (double)b.s * 4.0 * ((dim + 1) + rec_ints(dim)) +
                   (double)(((int64_t)2 << b.h) - ((int64_t)1 << b.g)) * (16.0 + 8.0 * dim + 4.0) +
                   4.0 * (double)(((int64_t)1 << b.h) + 1);
    }
    const unsigned grid = (unsigned)(part ? sub_blk_s.back() : sub_blk.back());
    KScope ks_(kK_subtree, s, sub_bytes);
    if (part) k_subtree<kSmallSubThreads><<<grid, kSmallSubThreads, smem, s>>>(P);
    else k_subtree<kSubThreads><<<grid, kSubThreads, smem, s>>>(P);
    st = cuda_check(cudaGetLastError(), "k_subtree");
  }

  // ---- boxes and live counts of the global-level nodes, deepest first ----
  if (!st && gmax) {
    FinishParams F;
    F.dim = dim;
    F.nlev = gmax;
    F.tree = d_tree;
    F.bw = (const BoxWork *)(plan + o_bw);
    F.bar = bar + 2;
    F.err = bt[0].err;
    void *args[] = {(void *)&F};
    st = coop((const void *)k_build_finish, 256, args, kK_build_finish, 0);
  }
  if (!st)
    launch_pack_nodes((const TreeSeg *)(plan + o_pk), (const int64_t *)(plan + o_pkpre), (int)pk_segs.size(),
                      pk_pre.back(), s);
  int err = st ? st : cuda_check(cudaGetLastError(), "build kernels");
  dev_free(af, block, total, s);
  return err;
}

size_t sort_small_table_bytes(size_t nlists) { return align256(std::max<size_t>(nlists, 1) * sizeof(SortList)); }

int launch_sort_small_many(const std::vector<SortList> &lists, void *table, cudaStream_t s) {
  int np2max = 0;
  for (const auto &L : lists) np2max = std::max(np2max, L.np2);
  if (lists.empty() || np2max <= 1) return BDL_OK;
  int st = h2d(table, lists.data(), lists.size() * sizeof(SortList), s);
  if (st) return st;
  cudaFuncSetAttribute(k_sort_small_many, cudaFuncAttributeMaxDynamicSharedMemorySize, 16384 * 4);
  KScope ks_(kK_sort_small, s);
  k_sort_small_many<<<(unsigned)lists.size(), 1024, (size_t)np2max * 4, s>>>((const SortList *)table);
  return cuda_check(cudaGetLastError(), "sort kernel");
}

}  // namespace bdl
