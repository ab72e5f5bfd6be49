// knn.cu -- kNN_L (Alg. 5): exact k nearest neighbours of a batch of queries
// over every static tree (largest first, Sec. V-B) and the buffer.
//
// GPU design: one thread per query walks the trees one after another with
// its own depth-first stack (nearer child first) and keeps its k best
// candidates sorted by (squared distance, id) in registers -- the role of the
// paper's 2k-entry kNN buffer (Sec. IV-A3).  A subtree is skipped when its
// bounding box is farther than the current k-th distance (strictly) or when
// it holds no live point (the NULL subtree of Alg. 2).
#include "bdl_internal.cuh"

namespace bdl {

namespace {

constexpr int kStack = 2 * kMaxLevel + 4;
constexpr uint64_t kNone = ~0ull;

template <int KMAX>
struct TopK {
  uint64_t d[KMAX];
  int32_t id[KMAX];
  uint64_t kd;     // current k-th distance (kNone while fewer than k held)
  int32_t kid;

  __device__ __forceinline__ void init() {
#pragma unroll
    for (int j = 0; j < KMAX; ++j) { d[j] = kNone; id[j] = INT32_MAX; }
    kd = kNone;
    kid = INT32_MAX;
  }
  __device__ __forceinline__ bool better(uint64_t x, int32_t i) const {
    return x < kd || (x == kd && i < kid);
  }
  __device__ __forceinline__ void insert(uint64_t x, int32_t i, int k) {
    bool placed = false;
#pragma unroll
    for (int j = KMAX - 1; j >= 1; --j) {
      if (j < k && !placed) {
        if (x < d[j - 1] || (x == d[j - 1] && i < id[j - 1])) {
          d[j] = d[j - 1];
          id[j] = id[j - 1];
        } else {
          d[j] = x;
          id[j] = i;
          placed = true;
        }
      }
    }
    if (!placed) { d[0] = x; id[0] = i; }
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
      if (j == k - 1) { kd = d[j]; kid = id[j]; }
  }
};

template <int D>
__device__ __forceinline__ uint64_t box_mindist(const int32_t *q, const int32_t *box, int dim) {
  const int dd = D ? D : dim;
  uint64_t s = 0;
#pragma unroll
  for (int c = 0; c < (D ? D : kMaxDim); ++c) {
    if (c < dd) {
      int64_t lo = box[c], hi = box[dd + c], x = q[c];
      int64_t g = x < lo ? lo - x : (x > hi ? x - hi : 0);
      s += (uint64_t)(g * g);
    }
  }
  return s;
}

template <int D, int KMAX>
__global__ void __launch_bounds__(128) k_knn(const ForestView F, const int32_t *qs, int64_t m, int k,
                                             int32_t *out_ids, int64_t *out_d2,
                                             unsigned long long *stats) {
  int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (qi >= m) return;
  const int dim = D ? D : F.dim;
  int32_t q[D ? D : kMaxDim];
#pragma unroll
  for (int c = 0; c < (D ? D : kMaxDim); ++c)
    if (c < dim) q[c] = qs[qi * dim + c];
  TopK<KMAX> best;
  best.init();
  unsigned long long nvisit = 0, npts = 0;
  int32_t sv[kStack];
  uint64_t smd[kStack];

  for (int ti = 0; ti < F.ntrees; ++ti) {
    const TreeView &T = F.tree[ti];
    const int2 *child = T.child;
    const int32_t *box = T.box;
    const int32_t *live = T.live;
    int sp = 0;
    if (live[0] > 0) {
      sv[0] = 0;
      smd[0] = box_mindist<D>(q, box, dim);
      sp = 1;
    }
    while (sp > 0) {
      --sp;
      int v = sv[sp];
      uint64_t md = smd[sp];
      if (md > best.kd) continue;
      nvisit++;
      int2 ch = child[v];
      if (ch.x < 0) {
        int leaf = -1 - ch.x;
        if (leaf >= ((int64_t)1 << T.h)) { atomicOr(F.err, kErrChild); continue; }
        int a = T.leaf_off[leaf], z = T.leaf_off[leaf + 1];
        if (a < 0 || z > T.size || a > z) { atomicOr(F.err, kErrLeaf); continue; }
        for (int j = a; j < z; ++j) {
          int32_t id = T.ids[j];
          if (id < 0) continue;
          npts++;
          uint64_t s = 0;
#pragma unroll
          for (int c = 0; c < (D ? D : kMaxDim); ++c) {
            if (c < dim) {
              int64_t g = (int64_t)q[c] - T.pts[(int64_t)c * T.size + j];
              s += (uint64_t)(g * g);
            }
          }
          if (best.better(s, id)) best.insert(s, id, k);
        }
      } else {
        int l = ch.x, r = ch.y;
        if (l >= T.nnodes || r < 0 || r >= T.nnodes) { atomicOr(F.err, kErrChild); continue; }
        if (sp + 2 > kStack) { atomicOr(F.err, kErrStack); continue; }
        uint64_t ml = live[l] > 0 ? box_mindist<D>(q, box + (int64_t)l * 2 * dim, dim) : kNone;
        uint64_t mr = live[r] > 0 ? box_mindist<D>(q, box + (int64_t)r * 2 * dim, dim) : kNone;
        bool lfirst = ml <= mr;
        int vn = lfirst ? l : r, vf = lfirst ? r : l;
        uint64_t mn = lfirst ? ml : mr, mf = lfirst ? mr : ml;
        if (mf != kNone && mf <= best.kd) { sv[sp] = vf; smd[sp] = mf; sp++; }
        if (mn != kNone && mn <= best.kd) { sv[sp] = vn; smd[sp] = mn; sp++; }
      }
    }
  }
  // the buffer tree: exact scan of its points
  for (int64_t j = 0; j < F.nbuf; ++j) {
    int32_t id = F.buf[j];
    const int32_t *p = F.idtab + (int64_t)id * dim;
    uint64_t s = 0;
#pragma unroll
    for (int c = 0; c < (D ? D : kMaxDim); ++c) {
      if (c < dim) {
        int64_t g = (int64_t)q[c] - p[c];
        s += (uint64_t)(g * g);
      }
    }
    if (best.better(s, id)) best.insert(s, id, k);
  }
  int32_t *oi = out_ids + qi * k;
  int64_t *od = out_d2 + qi * k;
#pragma unroll
  for (int j = 0; j < KMAX; ++j) {
    if (j < k) {
      bool ok = best.id[j] != INT32_MAX;
      oi[j] = ok ? best.id[j] : -1;
      od[j] = ok ? (int64_t)best.d[j] : INT64_MAX;
    }
  }
  if (stats) {
    atomicAdd(&stats[0], nvisit);
    atomicAdd(&stats[1], npts);
    atomicAdd(&stats[2], 1ull);
  }
}

template <int D, int KMAX>
void launch_dk(const ForestView &fv, const int32_t *q, int64_t m, int k, int32_t *oi, int64_t *od,
               unsigned long long *stats, cudaStream_t s) {
  { KScope ks_(kK_knn, s);
  k_knn<D, KMAX><<<(unsigned)((m + 127) / 128), 128, 0, s>>>(fv, q, m, k, oi, od, stats); }
}

template <int D>
void launch_d(const ForestView &fv, const int32_t *q, int64_t m, int k, int32_t *oi, int64_t *od,
              unsigned long long *stats, cudaStream_t s) {
  if (k <= 8) launch_dk<D, 8>(fv, q, m, k, oi, od, stats, s);
  else if (k <= 16) launch_dk<D, 16>(fv, q, m, k, oi, od, stats, s);
  else launch_dk<D, 32>(fv, q, m, k, oi, od, stats, s);
}

}  // namespace

int launch_knn(const ForestView &fv, const int32_t *q, int64_t m, int k, int32_t *out_ids,
               int64_t *out_d2, unsigned long long *stats, cudaStream_t s) {
  if (m <= 0) return BDL_OK;
  switch (fv.dim) {
    case 2: launch_d<2>(fv, q, m, k, out_ids, out_d2, stats, s); break;
    case 3: launch_d<3>(fv, q, m, k, out_ids, out_d2, stats, s); break;
    case 5: launch_d<5>(fv, q, m, k, out_ids, out_d2, stats, s); break;
    case 7: launch_d<7>(fv, q, m, k, out_ids, out_d2, stats, s); break;
    default: launch_d<0>(fv, q, m, k, out_ids, out_d2, stats, s); break;
  }
  return cuda_check(cudaGetLastError(), "knn kernel");
}

}  // namespace bdl
