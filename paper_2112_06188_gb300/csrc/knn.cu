// knn.cu -- kNN_L (Alg. 5): exact k nearest neighbours of a batch of queries
// over every static tree (largest first, Sec. V-B) and the buffer.
//
// GPU design:
//  * One thread per query walks the trees one after another with its own
//    depth-first stack (nearer child first) and keeps its k best candidates
//    sorted by (squared distance, id) in shared memory, the current k-th in
//    registers -- the role of the paper's 2k-entry kNN buffer (Sec. IV-A3).
//  * Leaf points are first tested with a float distance that can only
//    overstate what the exact int64 test accepts; the exact distance is
//    computed for the few that pass.
//  * A subtree is skipped when its bounding box is farther than the current
//    k-th distance (strictly) or when it holds no live point (the NULL
//    subtree of Alg. 2).
//  * The walk reads packed records, each holding the codes, live counts and
//    boxes of the four descendants two levels below its node: one visit
//    orders four subtrees by their box distance and halves the chain of
//    dependent reads from root to leaf.  The records of a tree follow the
//    vEB order of the 4-ary tree they form.
//  * A counting instance of the kernel walks the binary nodes instead and
//    counts visited nodes and examined leaf points (measurement runs).
//  * Large query batches are first put in spatial order (counting sort on a
//    Morton prefix) so that a warp's threads walk neighbouring paths.
#include "bdl_internal.cuh"

#include <mutex>

namespace bdl {

namespace {

constexpr int kStack = 2 * kMaxLevel + 4;
constexpr uint64_t kNone = ~0ull;

// k-NN blocks: the default shape (128 threads, 32 queries per warp) runs an
// instance compiled for exactly that launch; every other shape (KnnShape:
// 64, 128 or 256 threads, 32, 64 or 128 queries per warp) runs the general
// instance, compiled for blocks of up to 256 threads with the same register
// budget (256 x 6 = 128 x 12 threads per SM).
constexpr int kKnnThreads = 128;
constexpr int kKnnMaxThreads = 256;

// The k best candidates of one query, sorted by (d2, id), live in shared
// memory with a warp's 32 lanes in consecutive words, so that its accesses
// hit 32 different banks: [slot][thread] (slot stride S = the block size)
// in the default-shape instance, [warp][slot][lane] (S = 32) in the general
// one, whose block size is a launch parameter.  Only the current k-th pair
// stays in registers for the pruning tests.
// The smallest float >= 1 / (1 - 2^-18): 1 + 2^-18 + 2^-23.  Float squared
// distances (box gaps or leaf points) are compared with the k-th distance
// scaled up by it (see box_dist_f).
constexpr float kBoundUp = 1.00000393390655517578125f;

template <int S>
struct TopK {
  uint64_t *d;     // d[j * S]
  int32_t *id;
  int n;           // entries held (<= k)
  uint64_t kd;     // current k-th distance (kNone while fewer than k held)
  int32_t kid;

  float kdf;       // pruning bound: kd rounded up to float, times kBoundUp rounded up

  __device__ __forceinline__ void init(uint64_t *sd, int32_t *sid, int k) {
    const int at = S == 32 ? (threadIdx.x >> 5) * k * 32 + (threadIdx.x & 31) : threadIdx.x;
    d = sd + at;
    id = sid + at;
    n = 0;
    kd = kNone;
    kid = INT32_MAX;
    kdf = __int_as_float(0x7f800000);   // +inf
  }
  __device__ __forceinline__ bool prune(float lb) const { return lb > kdf; }
  __device__ __forceinline__ bool better(uint64_t x, int32_t i) const {
    return x < kd || (x == kd && i < kid);
  }
  __device__ __forceinline__ void insert(uint64_t x, int32_t i, int k) {
    int j = n < k ? n : k - 1;
    while (j > 0) {
      uint64_t pd = d[(j - 1) * S];
      int32_t pi = id[(j - 1) * S];
      if (!(x < pd || (x == pd && i < pi))) break;
      d[j * S] = pd;
      id[j * S] = pi;
      --j;
    }
    d[j * S] = x;
    id[j * S] = i;
    if (n < k) n++;
    if (n == k) {
      kd = d[(k - 1) * S];
      kid = id[(k - 1) * S];
      kdf = __fmul_ru(__ull2float_ru(kd), kBoundUp);
    }
  }
};

// Squared distance from q to the box lo[dim], hi[dim] in float.  Each gap is
// exact in float and the d <= 16 rounded squares and sums are within
// (d + 1) * 2^-24 < 2^-18 relative of the exact value s*, so s * (1 - 2^-18)
// <= s*.  A subtree is pruned only when s exceeds the k-th distance kd
// rounded up and scaled up by kBoundUp >= 1 / (1 - 2^-18) (TopK::kdf): then
// s* >= s (1 - 2^-18) > kd, i.e. never when the exact rule (prune iff
// mindist^2 > kth) would keep it.  Leaf points take the same float test.
template <int D>
__device__ __forceinline__ float box_dist_f(const int32_t *q, const int32_t *box, int dim) {
  const int dd = D ? D : dim;
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < (D ? D : kMaxDim); ++c) {
    if (c < dd) {
      const int32_t x = q[c];
      // at most one of the two gaps is positive (lo <= hi)
      const float g = (float)max(max(box[c] - x, x - box[dd + c]), 0);
      s = fmaf(g, g, s);
    }
  }
  return s;
}

// A traversal stack entry: the node code and the lower bound of its box
// distance, in one 64-bit word (one local-memory access per push and pop).
__device__ __forceinline__ uint64_t stack_entry(float lb, int code) {
  return ((uint64_t)__float_as_uint(lb) << 32) | (uint32_t)code;
}

// Largest j in [0, n) with pre[j] <= x (pre[0] = 0 <= x < pre[n]).
__device__ __forceinline__ int knn_find(const int64_t *pre, int n, int64_t x) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// (a, ca), (b, cb) in ascending order of the bound.
__device__ __forceinline__ void cmp_swap(float &a, int &ca, float &b, int &cb) {
  if (b < a) {
    const float tf = a;
    a = b;
    b = tf;
    const int ti = ca;
    ca = cb;
    cb = ti;
  }
}

// The exact test of the points [pa, pz) of tree T's leaf order against the
// query: a float filter first (the rounded sum of squares exceeds the scaled
// k-th distance TopK::kdf only for a point whose exact distance exceeds the
// k-th, as for box_dist_f), then the exact int64 distance for the points that
// pass.  Erased points (negative ids) are skipped.
template <int D, bool STATS, class TK>
__device__ __forceinline__ void scan_leaf(const TreeView &T, int pa, int pz, const int32_t *q, int dim,
                                          int rs, int k, TK &best, unsigned long long &npts) {
  for (int j = pa; j < pz; ++j) {
    const int32_t *src = T.pts + (int64_t)j * rs;
    int32_t id;
    uint64_t s = 0;
    if (D) {
      int32_t p[D ? rec_ints(D) : 4];
#pragma unroll
      for (int c4 = 0; c4 < (D ? rec_ints(D) : 4); c4 += 4) {
        int4 v = *reinterpret_cast<const int4 *>(src + c4);
        p[c4] = v.x;
        p[c4 + 1] = v.y;
        p[c4 + 2] = v.z;
        p[c4 + 3] = v.w;
      }
      id = p[D ? D : 0];
      if (STATS) npts += id >= 0;
      float sf = 0.f;
#pragma unroll
      for (int c = 0; c < (D ? D : 1); ++c) {
        const float g = (float)(q[c] - p[c]);
        sf = fmaf(g, g, sf);
      }
      if (sf > best.kdf) continue;
#pragma unroll
      for (int c = 0; c < (D ? D : 1); ++c) {
        int32_t g = q[c] - p[c];
        s += (uint64_t)((int64_t)g * g);
      }
    } else {
      id = src[dim];
      if (STATS) npts += id >= 0;
      for (int c = 0; c < dim; ++c) {
        int32_t g = q[c] - src[c];
        s += (uint64_t)((int64_t)g * g);
      }
    }
    if (id < 0) continue;   // erased
    if (best.better(s, id)) best.insert(s, id, k);
  }
}

// Alg. 5 on tree T over the packed records, for whole warps in lockstep: each
// lane walks its own depth-first order (nearest entry first, the next entry
// to visit held in a register, the rest on a stack), and the leaves that come
// due wait until half of the working lanes have one, so that the warp
// scans them together.  A record gives the bounds of four entries at once.
template <int D, class TK>
__device__ __forceinline__ void walk_packed(const KnnJob &J, const TreeView &T, bool active,
                                            const int32_t *q, int dim, int k, TK &best,
                                            uint64_t *stk) {
  const int rec = packed_node_ints(dim);
  const int rs = rec_ints(dim);
  const float kInf = __int_as_float(0x7f800000);
  unsigned long long unused = 0;
  int sp = 0;
  uint64_t cur = 0;   // the next entry to visit (code >= 0: record; < 0: leaf -1-code)
  bool hc = false;
  if (active) {
    cur = stack_entry(box_dist_f<D>(q, T.box, dim), T.h > 0 ? 0 : -1);
    hc = true;
  }
  const int32_t nleaf = (int32_t)((int64_t)1 << T.h);
  const int32_t nrec = (int32_t)packed_nrec(T.h);
  int pa = 0, pz = 0;
  bool pending = false;   // a leaf [pa, pz) is due but not scanned yet
  while (true) {
    const unsigned wm = __ballot_sync(0xffffffffu, pending || hc || sp > 0);
    if (!wm) break;
    const unsigned pm = __ballot_sync(0xffffffffu, pending);
    if (2 * __popc(pm) >= __popc(wm)) {
      // half of the working lanes have a leaf due: scan them together
      if (pending) scan_leaf<D, false>(T, pa, pz, q, dim, rs, k, best, unused);
      pending = false;
      continue;
    }
    // otherwise every lane without a due leaf takes one traversal step
    if (pending || (!hc && sp == 0)) continue;
    uint64_t e;
    if (hc) {
      e = cur;
      hc = false;
    } else {
      --sp;
      e = stk[sp];
    }
    const int code = (int)(uint32_t)e;
    if (best.prune(__uint_as_float((uint32_t)(e >> 32)))) continue;
    int leaf = -1;
    if (code < 0) {
      leaf = -1 - code;
    } else if (code >= nrec || sp + 3 > kStack) {
      atomicOr(J.err, code >= nrec ? kErrChild : kErrStack);
    } else {
      const int32_t *r = T.pk + (int64_t)code * rec;
      const int4 cd = *reinterpret_cast<const int4 *>(r);
      const int4 lv = *reinterpret_cast<const int4 *>(r + 4);
      float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;   // box distances (see box_dist_f)
#pragma unroll
      for (int c = 0; c < (D ? D : kMaxDim); ++c) {
        if (c < dim) {
          const int4 lo = *reinterpret_cast<const int4 *>(r + 8 + 8 * c);
          const int4 hi = *reinterpret_cast<const int4 *>(r + 12 + 8 * c);
          const int32_t x = q[c];
          // the gap to [lo, hi] (lo <= hi): at most one difference is positive
          const float g0 = (float)max(max(lo.x - x, x - hi.x), 0);
          const float g1 = (float)max(max(lo.y - x, x - hi.y), 0);
          const float g2 = (float)max(max(lo.z - x, x - hi.z), 0);
          const float g3 = (float)max(max(lo.w - x, x - hi.w), 0);
          s0 = fmaf(g0, g0, s0);
          s1 = fmaf(g1, g1, s1);
          s2 = fmaf(g2, g2, s2);
          s3 = fmaf(g3, g3, s3);
        }
      }
      // entries without live points (and the two unused ones of an odd
      // tree's root) are never visited
      float b0 = lv.x > 0 ? s0 : kInf, b1 = lv.y > 0 ? s1 : kInf;
      float b2 = lv.z > 0 ? s2 : kInf, b3 = lv.w > 0 ? s3 : kInf;
      int c0 = cd.x, c1 = cd.y, c2 = cd.z, c3 = cd.w;
      // ascending by bound: five compare-exchanges
      cmp_swap(b0, c0, b1, c1);
      cmp_swap(b2, c2, b3, c3);
      cmp_swap(b0, c0, b2, c2);
      cmp_swap(b1, c1, b3, c3);
      cmp_swap(b1, c1, b2, c2);
      if (b3 != kInf && !best.prune(b3)) stk[sp++] = stack_entry(b3, c3);
      if (b2 != kInf && !best.prune(b2)) stk[sp++] = stack_entry(b2, c2);
      if (b1 != kInf && !best.prune(b1)) stk[sp++] = stack_entry(b1, c1);
      if (b0 != kInf && !best.prune(b0)) {
        if (c0 < 0) {
          leaf = -1 - c0;   // nearest entry is a leaf: due now
        } else {
          cur = stack_entry(b0, c0);
          hc = true;
        }
      }
    }
    if (leaf >= 0) {
      if (leaf >= nleaf) {
        atomicOr(J.err, kErrChild);
      } else {
        pa = T.leaf_off[leaf];
        pz = T.leaf_off[leaf + 1];
        if (pa < 0 || pz > T.size || pa > pz) atomicOr(J.err, kErrLeaf);
        else pending = true;
      }
    }
  }
}

// Alg. 5 on tree T as the binary tree it is, one lane on its own: the node
// arrays (children, boxes, live counts) instead of the packed records, the
// nearer child first, a leaf scanned as soon as it is reached.  It decides
// every prune exactly as walk_packed would at the binary nodes, and counts
// the nodes it visits (a node or leaf taken from the stack and not pruned, or
// a nearer child that is a leaf) and the live leaf points it examines: the
// counting instance of the kernel, for measurement runs.
template <int D, class TK>
__device__ __forceinline__ void walk_nodes(const KnnJob &J, const TreeView &T, const int32_t *q,
                                           int dim, int k, TK &best, uint64_t *stk,
                                           unsigned long long &nvisit, unsigned long long &npts) {
  const int rs = rec_ints(dim);
  const float kInf = __int_as_float(0x7f800000);
  const int32_t nleaf = (int32_t)((int64_t)1 << T.h);
  int sp = 0;
  stk[sp++] = stack_entry(box_dist_f<D>(q, T.box, dim), 0);   // code: node slot
  while (sp > 0) {
    const uint64_t e = stk[--sp];
    const int v = (int)(uint32_t)e;
    if (best.prune(__uint_as_float((uint32_t)(e >> 32)))) continue;
    nvisit++;
    if (v < 0 || v >= T.nnodes) {
      atomicOr(J.err, kErrChild);
      continue;
    }
    const Node nd = T.node[v];
    int leaf = -1;
    if (nd.l < 0) {
      leaf = -1 - nd.l;
    } else if (nd.l >= T.nnodes || nd.r < 0 || nd.r >= T.nnodes || sp + 2 > kStack) {
      atomicOr(J.err, sp + 2 > kStack ? kErrStack : kErrChild);
    } else {
      const float ml = T.live[nd.l] > 0 ? box_dist_f<D>(q, T.box + (int64_t)nd.l * 2 * dim, dim) : kInf;
      const float mr = T.live[nd.r] > 0 ? box_dist_f<D>(q, T.box + (int64_t)nd.r * 2 * dim, dim) : kInf;
      const bool lfirst = ml <= mr;
      const int vn = lfirst ? nd.l : nd.r, vf = lfirst ? nd.r : nd.l;
      const float mn = lfirst ? ml : mr, mf = lfirst ? mr : ml;
      if (mf != kInf && !best.prune(mf)) stk[sp++] = stack_entry(mf, vf);
      if (mn != kInf && !best.prune(mn)) {
        const int nl = T.node[vn].l;
        if (nl < 0) {   // nearer child is a leaf: scanned now
          nvisit++;
          leaf = -1 - nl;
        } else {
          stk[sp++] = stack_entry(mn, vn);
        }
      }
    }
    if (leaf >= 0) {
      if (leaf >= nleaf) {
        atomicOr(J.err, kErrChild);
      } else {
        const int pa = T.leaf_off[leaf], pz = T.leaf_off[leaf + 1];
        if (pa < 0 || pz > T.size || pa > pz) atomicOr(J.err, kErrLeaf);
        else scan_leaf<D, true>(T, pa, pz, q, dim, rs, k, best, npts);
      }
    }
  }
}

// Query t of job J (one forest's batch) against the trees trees[0 ..
// J.ntrees), then the buffer.  The timed instance (STATS false) is called by
// whole warps of one job, which stay resident and converged until each of
// their lanes is done; the counting instance walks each lane on its own.
template <int D, bool STATS, int S, bool TREES_SMEM = false>
__device__ __forceinline__ void knn_query(const KnnJob &J, const TreeView *trees, int64_t t, int k,
                                          unsigned long long *stats) {
  // k (d2, id) slots per thread (TopK<S>'s layout)
  extern __shared__ __align__(8) unsigned char knn_sm[];
  uint64_t *s_d = reinterpret_cast<uint64_t *>(knn_sm);
  int32_t *s_id = reinterpret_cast<int32_t *>(s_d + (size_t)k * blockDim.x);
  const int64_t m = J.m;
  const int32_t *qs = J.q, *perm = J.perm;
  int32_t *out_ids = J.oi;
  int64_t *out_d2 = J.od;
  const bool active = t < m;
  if (STATS && !active) return;
  const int64_t qi = active ? (perm ? perm[t] : t) : 0;
  const int dim = D ? D : J.dim;
  int32_t q[D ? D : kMaxDim];
#pragma unroll
  for (int c = 0; c < (D ? D : kMaxDim); ++c)
    if (c < dim) q[c] = active ? qs[qi * dim + c] : 0;
  TopK<S> best;
  best.init(s_d, s_id, k);
  unsigned long long nvisit = 0, npts = 0;
  uint64_t stk[kStack];   // (distance bits << 32) | code

  const int ntrees = J.ntrees;
  for (int ti = 0; ti < ntrees; ++ti) {
    // from a job table in global memory (TREES_SMEM), each tree's view is
    // copied into a shared slot of the warp, read where used during the walk
    // (kernel-parameter views are read through the constant cache instead)
    const TreeView *tp = &trees[ti];
    if (TREES_SMEM) {
      __shared__ TreeView s_tree[kKnnMaxThreads / 32];
      TreeView &slot = s_tree[threadIdx.x >> 5];
      __syncwarp();   // the warp is done with the previous tree's view
      if ((threadIdx.x & 31) == 0) slot = trees[ti];
      __syncwarp();
      tp = &slot;
    }
    const TreeView &T = *tp;
    if (T.live[0] <= 0) continue;
    if (STATS) walk_nodes<D>(J, T, q, dim, k, best, stk, nvisit, npts);
    else walk_packed<D>(J, T, active, q, dim, k, best, stk);
  }
  if (!active) return;
  // the buffer tree: exact scan of its points
  for (int64_t j = 0; j < J.nbuf; ++j) {
    const int32_t id = J.buf[j];
    const int32_t *p = J.idtab + (int64_t)id * dim;
    uint64_t s = 0;
#pragma unroll
    for (int c = 0; c < (D ? D : kMaxDim); ++c) {
      if (c < dim) {
        int32_t g = q[c] - p[c];
        s += (uint64_t)((int64_t)g * g);
      }
    }
    if (best.better(s, id)) best.insert(s, id, k);
  }
  int32_t *oi = out_ids + qi * k;
  int64_t *od = out_d2 + qi * k;
  for (int j = 0; j < k; ++j) {
    const bool ok = j < best.n;
    oi[j] = ok ? best.id[j * S] : -1;
    od[j] = ok ? (int64_t)best.d[j * S] : INT64_MAX;
  }
  if (STATS) {
    atomicAdd(&stats[0], nvisit);
    atomicAdd(&stats[1], npts);
    atomicAdd(&stats[2], 1ull);
  }
}

// Many forests: every warp finds its job in the table (jobs are warp-aligned:
// job j owns ceil(m_j / qpw) warps).  A warp answers qpw consecutive queries
// of its job (in the job's processing order), 32 at a time; every round ends
// with the warp converged.  GEN false: the default shape (qpw = 32).
template <int D, bool STATS, bool GEN>
__global__ void __launch_bounds__(GEN ? kKnnMaxThreads : kKnnThreads, GEN ? 6 : 12)
    k_knn(const KnnJob *jobs, const int64_t *job_warp, int njobs, int k, int qpw, unsigned long long *stats) {
  // the warp's job, copied into shared memory: its fields are read where
  // used instead of held in registers through the walk
  __shared__ KnnJob s_job[kKnnMaxThreads / 32];
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= job_warp[njobs]) return;   // (whole warps)
  const int jb = knn_find(job_warp, njobs, w);
  KnnJob &J = s_job[threadIdx.x >> 5];
  if ((threadIdx.x & 31) == 0) J = jobs[jb];
  __syncwarp();
  const int64_t t0 = w - job_warp[jb];
  if (!GEN) {
    knn_query<D, STATS, kKnnThreads, !STATS>(J, J.trees, t0 * 32 + (threadIdx.x & 31), k, stats);
  } else {
    for (int r = 0; r < qpw && t0 * qpw + r < J.m; r += 32) {   // warp-uniform bounds
      knn_query<D, STATS, 32, !STATS>(J, J.trees, t0 * qpw + r + (threadIdx.x & 31), k, stats);
      __syncwarp();
    }
  }
}

// One forest: its job and tree views travel as kernel parameters, read
// through the constant cache (the per-tree fields are warp-uniform).
struct KnnOne {
  KnnJob job;
  TreeView trees[kMaxLevel];
};

template <int D, bool STATS, bool GEN>
__global__ void __launch_bounds__(GEN ? kKnnMaxThreads : kKnnThreads, GEN ? 6 : 12)
    k_knn_one(const __grid_constant__ KnnOne P, int k, int qpw, unsigned long long *stats) {
  if (!GEN) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if ((t & ~(int64_t)31) >= P.job.m) return;     // whole warp past the end
    knn_query<D, STATS, kKnnThreads>(P.job, P.trees, t, k, stats);
  } else {
    const int64_t t0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * qpw;
    for (int r = 0; r < qpw && t0 + r < P.job.m; r += 32) {   // warp-uniform bounds
      knn_query<D, STATS, 32>(P.job, P.trees, t0 + r + (threadIdx.x & 31), k, stats);
      __syncwarp();
    }
  }
}

// The block size actually launched for shape sh and k: the requested one,
// halved while k slots per thread would pass 48 KB of shared memory.
int knn_block_for(const KnnShape &sh, int k) {
  int b = sh.block;
  while (b > 32 && (size_t)k * b * 12 > 48 * 1024) b >>= 1;
  return b;
}

template <int D>
void launch_d(const KnnJob *jobs, const int64_t *job_warp, int njobs, int64_t warps, int k,
              const KnnShape &sh, unsigned long long *stats, cudaStream_t s) {
  const int bt = knn_block_for(sh, k);
  const size_t smem = (size_t)k * bt * 12;   // <= 48 KB
  const unsigned grid = (unsigned)((warps * 32 + bt - 1) / bt);
  const bool gen = bt != kKnnThreads || sh.qpw != 32;
  void (*fn)(const KnnJob *, const int64_t *, int, int, int, unsigned long long *) =
      stats ? (gen ? k_knn<D, true, true> : k_knn<D, true, false>)
            : (gen ? k_knn<D, false, true> : k_knn<D, false, false>);
  // the kernel's own shared memory (the warps' job and tree slots) comes on
  // top of the top-k slots: past the default 48 KB per block (k = 32 at 128
  // threads) the launch needs the opt-in
  if (smem > 40 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  KScope ks_(stats ? kK_knn_count : kK_knn, s);
  fn<<<grid, bt, smem, s>>>(jobs, job_warp, njobs, k, sh.qpw, stats);
}

template <int D>
void launch_one(const KnnOne &P, int k, const KnnShape &sh, unsigned long long *stats, cudaStream_t s) {
  const int bt = knn_block_for(sh, k);
  const size_t smem = (size_t)k * bt * 12;
  KScope ks_(stats ? kK_knn_count : kK_knn, s);
  const int64_t warps = (P.job.m + sh.qpw - 1) / sh.qpw;
  const unsigned grid = (unsigned)((warps * 32 + bt - 1) / bt);
  const bool gen = bt != kKnnThreads || sh.qpw != 32;
  if (stats && gen)
    k_knn_one<D, true, true><<<grid, bt, smem, s>>>(P, k, sh.qpw, stats);
  else if (stats)
    k_knn_one<D, true, false><<<grid, bt, smem, s>>>(P, k, sh.qpw, stats);
  else if (gen)
    k_knn_one<D, false, true><<<grid, bt, smem, s>>>(P, k, sh.qpw, stats);
  else
    k_knn_one<D, false, false><<<grid, bt, smem, s>>>(P, k, sh.qpw, stats);
}

// ---------------------------------------------------------------------------
// packed node records (packed_node_ints): one per record node, built from the
// trees' node boxes and live counts
// ---------------------------------------------------------------------------

// One thread per record of many trees (table entry j owns the work items
// pre[j] .. pre[j+1]-1, one per record of tree j, in level order).
__global__ void k_pack_nodes(const TreeSeg *segs, const int64_t *pre, int nseg) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= pre[nseg]) return;
  const int j = knn_find(pre, nseg, x);
  const TreeSeg &T = segs[j];
  const int32_t *box = T.box, *live = T.live;
  const int h = T.h, dim = T.dim;
  int t;
  int64_t i;
  packed_record_of(h, x - pre[j], t, i);
  const int e = packed_step(h, t);
  int32_t *r = T.pk + packed_slot(h, t, i) * packed_node_ints(dim);
  for (int a = 0; a < 4; ++a) {
    int code = 0, lv = 0;
    const int32_t *bx = nullptr;
    if (a < (1 << e)) {   // entry a: descendant (t + e, i * 2^e + a)
      const int tc = t + e;
      const int64_t ci = (i << e) + a;
      code = tc == h ? (int)(-1 - ci) : (int)packed_slot(h, tc, ci);
      const int64_t v = veb_slot(h + 1, tc, ci);
      lv = live[v];
      bx = box + v * 2 * dim;
    }
    r[a] = code;
    r[4 + a] = lv;
    for (int c = 0; c < dim; ++c) {
      r[8 + 8 * c + a] = bx ? bx[c] : INT32_MAX;
      r[12 + 8 * c + a] = bx ? bx[dim + c] : INT32_MIN;
    }
  }
}

// ---------------------------------------------------------------------------
// spatial order of the queries: counting sort on a Morton prefix
// ---------------------------------------------------------------------------

constexpr int kScanPer = 4096;   // entries per scan block (1024 threads x 4)

__host__ __device__ inline int morton_bits_per_dim(int dim) {
  int b = 20 / dim;
  return b > 10 ? 10 : b;
}

__device__ __forceinline__ uint32_t morton_key(const int32_t *q, int dim, int B) {
  uint32_t key = 0;
  for (int b = B - 1; b >= 0; --b)
    for (int c = 0; c < dim; ++c) {
      int32_t x = min(max(q[c], 0), (1 << kCoordBits) - 1);
      key = (key << 1) | ((x >> (kCoordBits - B + b)) & 1);
    }
  return key;
}

// Point i's coordinates: row i of `coords`, or row ids[i] when ids is given.
__device__ __forceinline__ const int32_t *point_row(const int32_t *coords, const int32_t *ids,
                                                    int64_t i, int dim) {
  return coords + (ids ? (int64_t)ids[i] : i) * dim;
}

__global__ void k_qkey_hist(const int32_t *coords, const int32_t *ids, int64_t m,
                            const int64_t *m_dev, int dim, int B, uint32_t *hist) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m_dev && i >= *m_dev) return;
  if (i < m) atomicAdd(&hist[morton_key(point_row(coords, ids, i, dim), dim, B)], 1u);
}

__device__ uint32_t block_scan_u32(uint32_t v, uint32_t *total) {
  __shared__ uint32_t ws[33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = v;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  __syncthreads();
  if (lane == 31) ws[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    uint32_t x = lane < nw ? ws[lane] : 0, xi = x;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, xi, o);
      if (lane >= o) xi += y;
    }
    if (lane < nw) ws[lane] = xi - x;
    if (lane == nw - 1) ws[32] = xi;
  }
  __syncthreads();
  *total = ws[32];
  return inc - v + ws[warp];
}

// per block of kScanPer entries: exclusive scan in place, block total to bsum
__global__ void k_scan_local(uint32_t *a, int64_t n, uint32_t *bsum) {
  const int64_t base = (int64_t)blockIdx.x * kScanPer + threadIdx.x * 4;
  uint32_t v[4], s = 0;
  for (int j = 0; j < 4; ++j) {
    v[j] = base + j < n ? a[base + j] : 0;
    s += v[j];
  }
  uint32_t tot;
  uint32_t e = block_scan_u32(s, &tot);
  for (int j = 0; j < 4; ++j) {
    if (base + j < n) a[base + j] = e;
    e += v[j];
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// single block: exclusive scan of the (<= 1024 * 4) block totals
__global__ void k_scan_top(uint32_t *bsum, int64_t nb) {
  const int64_t base = threadIdx.x * 4;
  uint32_t v[4], s = 0;
  for (int j = 0; j < 4; ++j) {
    v[j] = base + j < nb ? bsum[base + j] : 0;
    s += v[j];
  }
  uint32_t tot;
  uint32_t e = block_scan_u32(s, &tot);
  for (int j = 0; j < 4; ++j) {
    if (base + j < nb) bsum[base + j] = e;
    e += v[j];
  }
}

// out[pos] = i (query order) or ids[i] (the ids themselves, reordered)
__global__ void k_qscatter(const int32_t *coords, const int32_t *ids, int64_t m,
                           const int64_t *m_dev, int dim, int B, uint32_t *offs,
                           const uint32_t *bsum, int32_t *out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m || (m_dev && i >= *m_dev)) return;
  uint32_t key = morton_key(point_row(coords, ids, i, dim), dim, B);
  uint32_t pos = bsum[key / kScanPer] + atomicAdd(&offs[key], 1u);
  if (pos < m) out[pos] = ids ? ids[i] : (int32_t)i;
}

// Many small query batches (one per job of a batched call) in one counting
// sort: the key is the job's rank, then a Morton prefix of B bits per
// coordinate, so that each job's queries come out together and in spatial
// order.  perm[off_j + t] = the t-th query of job j, as an index into job j's
// queries.
struct BatchSortJobs {
  const int32_t *const *q;   // [njobs] query arrays
  const int64_t *pre;        // [njobs + 1] query prefix
  int njobs, dim, B;
};

__device__ __forceinline__ uint32_t batch_key(const BatchSortJobs &S, int64_t x, int32_t &local) {
  const int j = knn_find(S.pre, S.njobs, x);
  local = (int32_t)(x - S.pre[j]);
  return ((uint32_t)j << (S.B * S.dim)) | morton_key(S.q[j] + (int64_t)local * S.dim, S.dim, S.B);
}

__global__ void k_bkey_hist(const BatchSortJobs S, uint32_t *hist) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= S.pre[S.njobs]) return;
  int32_t local;
  atomicAdd(&hist[batch_key(S, x, local)], 1u);
}

__global__ void k_bkey_scatter(const BatchSortJobs S, uint32_t *offs, const uint32_t *bsum, int32_t *perm) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t M = S.pre[S.njobs];
  if (x >= M) return;
  int32_t local;
  const uint32_t key = batch_key(S, x, local);
  const uint32_t pos = bsum[key / kScanPer] + atomicAdd(&offs[key], 1u);
  if (pos < M) perm[pos] = local;
}

}  // namespace

int batch_query_sort(std::vector<KnnCall> &calls, void *scratch, size_t bytes, cudaStream_t s) {
  const int n = (int)calls.size();
  if (n < 2) return BDL_OK;
  const int dim = calls[0].fv->dim;
  // bits per coordinate: the most with n * 2^(B*dim) <= 2^22 bins, at most 10
  int B = 0;
  while (B < 10 && ((int64_t)n << ((B + 1) * dim)) <= ((int64_t)1 << 22)) ++B;
  if (B == 0) return BDL_OK;
  const int64_t nbins = (int64_t)n << (B * dim);
  const int64_t nb = (nbins + kScanPer - 1) / kScanPer;
  int64_t M = 0;
  for (auto &c : calls) M += c.m;
  if (bytes < batch_query_sort_bytes(calls)) return set_error(BDL_EINTERNAL, "batch sort scratch too small");
  // scratch: perm [M], hist [nbins], block sums [nb], job table (q pointers, prefix)
  char *p = (char *)scratch;
  int32_t *perm = (int32_t *)p; p += ((size_t)M * 4 + 255) / 256 * 256;
  uint32_t *hist = (uint32_t *)p; p += ((size_t)nbins * 4 + 255) / 256 * 256;
  uint32_t *bsum = (uint32_t *)p; p += ((size_t)nb * 4 + 255) / 256 * 256;
  std::vector<unsigned char> img(((size_t)n * 8 + 255) / 256 * 256 + (size_t)(n + 1) * 8);
  const int32_t **qv = (const int32_t **)img.data();
  int64_t *pre = (int64_t *)(img.data() + ((size_t)n * 8 + 255) / 256 * 256);
  pre[0] = 0;
  for (int j = 0; j < n; ++j) {
    qv[j] = calls[j].q;
    pre[j + 1] = pre[j] + calls[j].m;
  }
  int st = h2d(p, img.data(), img.size(), s);
  if (st) return st;
  BatchSortJobs S;
  S.q = (const int32_t *const *)p;
  S.pre = (const int64_t *)(p + ((size_t)n * 8 + 255) / 256 * 256);
  S.njobs = n;
  S.dim = dim;
  S.B = B;
  st = small_zero(hist, (size_t)nbins * 4, s);
  if (st) return st;
  const unsigned g = (unsigned)((M + 255) / 256);
  { KScope ks_(kK_qsort, s); k_bkey_hist<<<g, 256, 0, s>>>(S, hist); }
  { KScope ks_(kK_qsort, s); k_scan_local<<<(unsigned)nb, 1024, 0, s>>>(hist, nbins, bsum); }
  { KScope ks_(kK_qsort, s); k_scan_top<<<1, 1024, 0, s>>>(bsum, nb); }
  { KScope ks_(kK_qsort, s); k_bkey_scatter<<<g, 256, 0, s>>>(S, hist, bsum, perm); }
  for (int j = 0; j < n; ++j) calls[j].perm = perm + pre[j];
  return cuda_check(cudaGetLastError(), "batch query sort");
}

size_t batch_query_sort_bytes(const std::vector<KnnCall> &calls) {
  const int n = (int)calls.size();
  if (n < 2) return 0;
  const int dim = calls[0].fv->dim;
  int B = 0;
  while (B < 10 && ((int64_t)n << ((B + 1) * dim)) <= ((int64_t)1 << 22)) ++B;
  const int64_t nbins = (int64_t)n << (B * dim);
  const int64_t nb = (nbins + kScanPer - 1) / kScanPer;
  int64_t M = 0;
  for (auto &c : calls) M += c.m;
  return ((size_t)M * 4 + 255) / 256 * 256 + ((size_t)nbins * 4 + 255) / 256 * 256 +
         ((size_t)nb * 4 + 255) / 256 * 256 + ((size_t)n * 8 + 255) / 256 * 256 + (size_t)(n + 1) * 8 + 256;
}

size_t knn_table_bytes(const std::vector<KnnCall> &calls) {
  if (calls.size() == 1) return 0;   // one forest: no table (kernel parameters)
  return knn_table_bytes_always(calls);
}

size_t knn_table_bytes_always(const std::vector<KnnCall> &calls) {
  size_t n = calls.size(), views = 0;
  for (const auto &c : calls) views += (size_t)c.fv->ntrees;
  return n * sizeof(KnnJob) + (n + 1) * 8 + views * sizeof(TreeView) + 64;
}

int upload_knn_table(const std::vector<KnnCall> &calls, void *table, int64_t *warps, int qpw,
                     cudaStream_t s) {
  const size_t n = calls.size();
  std::vector<unsigned char> img(knn_table_bytes_always(calls));
  KnnJob *jobs = (KnnJob *)img.data();
  int64_t *warp = (int64_t *)(img.data() + n * sizeof(KnnJob));
  const size_t views_off = n * sizeof(KnnJob) + (n + 1) * 8;
  TreeView *views = (TreeView *)(img.data() + views_off);
  size_t v = 0;
  warp[0] = 0;
  for (size_t j = 0; j < n; ++j) {
    const KnnCall &c = calls[j];
    KnnJob &J = jobs[j];
    memset(&J, 0, sizeof(J));
    J.trees = (const TreeView *)((char *)table + views_off) + v;
    J.ntrees = c.fv->ntrees;
    J.dim = c.fv->dim;
    J.idtab = c.fv->idtab;
    J.buf = c.fv->buf;
    J.nbuf = c.fv->nbuf;
    J.err = c.fv->err;
    J.q = c.q;
    J.perm = c.perm;
    J.m = c.m;
    J.oi = c.oi;
    J.od = c.od;
    for (int t = 0; t < c.fv->ntrees; ++t) views[v++] = c.fv->tree[t];
    warp[j + 1] = warp[j] + (c.m + qpw - 1) / qpw;
  }
  *warps = warp[n];
  if (warp[n] == 0) return BDL_OK;
  return h2d(table, img.data(), img.size(), s);
}

int launch_knn_table(const void *table, int njobs, int64_t warps, int dim, int k, const KnnShape &sh,
                     unsigned long long *stats, cudaStream_t s) {
  if (warps == 0) return BDL_OK;
  const KnnJob *dj = (const KnnJob *)table;
  const int64_t *dw = (const int64_t *)((const char *)table + njobs * sizeof(KnnJob));
  switch (dim) {
    case 2: launch_d<2>(dj, dw, njobs, warps, k, sh, stats, s); break;
    case 3: launch_d<3>(dj, dw, njobs, warps, k, sh, stats, s); break;
    case 5: launch_d<5>(dj, dw, njobs, warps, k, sh, stats, s); break;
    case 7: launch_d<7>(dj, dw, njobs, warps, k, sh, stats, s); break;
    default: launch_d<0>(dj, dw, njobs, warps, k, sh, stats, s); break;
  }
  return cuda_check(cudaGetLastError(), "knn kernel");
}

int launch_knn_jobs(const std::vector<KnnCall> &calls, int dim, int k, const KnnShape &sh, void *table,
                    unsigned long long *stats, cudaStream_t s) {
  const size_t n = calls.size();
  if (n == 1) {
    const KnnCall &c = calls[0];
    if (c.m == 0) return BDL_OK;
    KnnOne P;
    memset(&P, 0, sizeof(P));
    P.job.ntrees = c.fv->ntrees;
    P.job.dim = c.fv->dim;
    P.job.idtab = c.fv->idtab;
    P.job.buf = c.fv->buf;
    P.job.nbuf = c.fv->nbuf;
    P.job.err = c.fv->err;
    P.job.q = c.q;
    P.job.perm = c.perm;
    P.job.m = c.m;
    P.job.oi = c.oi;
    P.job.od = c.od;
    for (int t = 0; t < c.fv->ntrees; ++t) P.trees[t] = c.fv->tree[t];
    switch (dim) {
      case 2: launch_one<2>(P, k, sh, stats, s); break;
      case 3: launch_one<3>(P, k, sh, stats, s); break;
      case 5: launch_one<5>(P, k, sh, stats, s); break;
      case 7: launch_one<7>(P, k, sh, stats, s); break;
      default: launch_one<0>(P, k, sh, stats, s); break;
    }
    return cuda_check(cudaGetLastError(), "knn kernel");
  }
  int64_t warps = 0;
  int st = upload_knn_table(calls, table, &warps, sh.qpw, s);
  if (st) return st;
  return launch_knn_table(table, (int)n, warps, dim, k, sh, stats, s);
}

void pack_nodes_entries(const std::vector<Tree *> &trees, int dim, std::vector<TreeSeg> &segs,
                        std::vector<int64_t> &pre) {
  pre.assign(1, 0);
  for (const Tree *t : trees) {
    TreeSeg g;
    memset(&g, 0, sizeof(g));
    g.dim = dim;
    g.h = t->h;
    g.node = t->node;
    g.box = t->box;
    g.live = t->live_nodes;
    g.pk = t->pk;
    segs.push_back(g);
    pre.push_back(pre.back() + packed_nrec(t->h));
  }
}

void launch_pack_nodes(const TreeSeg *segs, const int64_t *pre, int nseg, int64_t total, cudaStream_t s) {
  if (total <= 0) return;
  KScope ks_(kK_pack_nodes, s);
  k_pack_nodes<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(segs, pre, nseg);
}

size_t query_sort_bytes(int64_t m, int dim) {
  int64_t nbins = (int64_t)1 << (morton_bits_per_dim(dim) * dim);
  int64_t nb = (nbins + kScanPer - 1) / kScanPer;
  return ((size_t)m * 4 + 255) / 256 * 256 + (size_t)nbins * 4 + 256 + (size_t)nb * 4 + 256;
}

void launch_point_sort(const int32_t *coords, const int32_t *ids, int64_t m, int dim,
                       void *scratch, int32_t *out, cudaStream_t s, const int64_t *m_dev) {
  const int B = morton_bits_per_dim(dim);
  const int64_t nbins = (int64_t)1 << (B * dim);
  const int64_t nb = (nbins + kScanPer - 1) / kScanPer;   // <= 256
  uint32_t *hist = (uint32_t *)scratch;
  uint32_t *bsum = (uint32_t *)((char *)scratch + ((size_t)nbins * 4 + 255) / 256 * 256);
  small_zero(hist, (size_t)nbins * 4, s);
  const unsigned g = (unsigned)((m + 255) / 256);
  { KScope ks_(kK_qsort, s); k_qkey_hist<<<g, 256, 0, s>>>(coords, ids, m, m_dev, dim, B, hist); }
  { KScope ks_(kK_qsort, s); k_scan_local<<<(unsigned)nb, 1024, 0, s>>>(hist, nbins, bsum); }
  { KScope ks_(kK_qsort, s); k_scan_top<<<1, 1024, 0, s>>>(bsum, nb); }
  { KScope ks_(kK_qsort, s); k_qscatter<<<g, 256, 0, s>>>(coords, ids, m, m_dev, dim, B, hist, bsum, out); }
}

void launch_query_sort(const int32_t *q, int64_t m, int dim, void *scratch, int32_t *perm,
                       cudaStream_t s) {
  launch_point_sort(q, nullptr, m, dim, scratch, perm, s);
}

}  // namespace bdl

// ---------------------------------------------------------------------------
// k-NN without device allocation
// ---------------------------------------------------------------------------
//
// bdl_knn takes scratch for the query ordering from the library's memory
// pool.  Some callers cannot let a query allocate: a process whose device
// memory is already fully reserved by another allocator (a framework's
// caching allocator holding the free memory, say) would see the allocation
// fail, and a latency-bound request path may not wait on the pool.  For them
// bdl_knn_noalloc keeps that scratch in the fixed array below instead.  The
// array exists on every GPU that loads the library, from load until exit.

namespace bdl {
namespace {

constexpr int64_t kNoAllocMaxQueries = 1 << 20;
constexpr size_t kNoAllocPermBytes = (size_t)kNoAllocMaxQueries * 4;   // query order
constexpr size_t kNoAllocScratchBytes = kNoAllocPermBytes + ((size_t)4 << 20) + 4096;

// query order [m], then the Morton histogram (<= 2^20 bins) and its block sums
static __device__ __align__(256) unsigned char g_knn_scratch[kNoAllocScratchBytes];

std::mutex g_knn_scratch_mu;
void *g_knn_scratch_addr[128];   // device address of g_knn_scratch, per device

// Device address of the array on the current device (looked up on first use;
// in host code the array's name is only a stand-in, not a device address).
int knn_scratch_address(int dev, void **out) {
  std::lock_guard<std::mutex> lk(g_knn_scratch_mu);
  if (dev < 0 || dev >= 128) return set_error(BDL_EINVAL, "device index out of range");
  if (!g_knn_scratch_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_knn_scratch);
    if (e != cudaSuccess) return cuda_check(e, "cudaGetSymbolAddress(k-NN scratch)");
    g_knn_scratch_addr[dev] = p;
  }
  *out = g_knn_scratch_addr[dev];
  return BDL_OK;
}

}  // namespace
}  // namespace bdl

extern "C" int bdl_knn_noalloc(bdl_forest *f, const int32_t *q, int64_t m, int k, int32_t *out_ids,
                               int64_t *out_d2, bdl_stream_t stream) {
  using namespace bdl;
  if (!f) return set_error(BDL_EINVAL, "forest is NULL");
  if (k < 1 || k > kMaxK) return set_error(BDL_EINVAL, "k must be in 1..32");
  if (m < 0) return set_error(BDL_EINVAL, "m < 0");
  if (m > kNoAllocMaxQueries)
    return set_error(BDL_EINVAL, "bdl_knn_noalloc takes at most 1,048,576 queries per call");
  if (m == 0) return BDL_OK;
  if (!q || !out_ids || !out_d2) return set_error(BDL_EINVAL, "NULL pointer");
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != f->device) cudaSetDevice(f->device);
  cudaStream_t s = (cudaStream_t)stream;
  void *scratch = nullptr;
  int st = knn_scratch_address(f->device, &scratch);
  if (!st) {
    ForestView fv = knn_view(f, false, s);   // never rebuilds (no allocation)
    int32_t *perm = nullptr;
    if (m >= kSortMinQueries) {
      perm = (int32_t *)scratch;
      launch_query_sort(q, m, f->dim, (char *)scratch + kNoAllocPermBytes, perm, s);
    }
    // a single forest's job goes by kernel parameters: no table to place
    std::vector<KnnCall> calls{KnnCall{&fv, q, perm, m, out_ids, out_d2}};
    st = finish_call(f, s, launch_knn_jobs(calls, f->dim, k, f->knn_shape, nullptr, f->knn_stats, s));
  }
  if (prev >= 0 && prev != f->device) cudaSetDevice(prev);
  return st;
}

