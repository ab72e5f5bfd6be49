// knn.cu -- kNN_L (Alg. 5): exact k nearest neighbours of a batch of queries
// over every static tree (largest first, Sec. V-B) and the buffer.
//
// GPU design:
//  * One thread per query walks the trees one after another with its own
//    depth-first stack (nearer child first) and keeps its k best candidates
//    sorted by (squared distance, id) in registers -- the role of the paper's
//    2k-entry kNN buffer (Sec. IV-A3).
//  * A subtree is skipped when its bounding box is farther than the current
//    k-th distance (strictly) or when it holds no live point (the NULL
//    subtree of Alg. 2).
//  * Each internal node has a packed record holding both children's codes,
//    live counts and boxes, so one visit is one 32-byte-aligned read; the
//    records of a tree follow the vEB order of its internal levels.
//  * Large query batches are first put in spatial order (counting sort on a
//    Morton prefix) so that a warp's threads walk neighbouring paths.
#include "bdl_internal.cuh"

#include <mutex>

namespace bdl {

namespace {

constexpr int kStack = 2 * kMaxLevel + 4;
constexpr uint64_t kNone = ~0ull;

constexpr int kKnnThreads = 128;

// The k best candidates of one query, sorted by (d2, id), live in shared
// memory ([slot][thread], so a warp's accesses hit 32 different banks); only
// the current k-th pair stays in registers for the pruning tests.
struct TopK {
  uint64_t *d;     // d[j * kKnnThreads]
  int32_t *id;
  int n;           // entries held (<= k)
  uint64_t kd;     // current k-th distance (kNone while fewer than k held)
  int32_t kid;

  float kdf;       // kd rounded up to float (pruning bound)

  __device__ __forceinline__ void init(uint64_t *sd, int32_t *sid) {
    d = sd + threadIdx.x;
    id = sid + threadIdx.x;
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
      uint64_t pd = d[(j - 1) * kKnnThreads];
      int32_t pi = id[(j - 1) * kKnnThreads];
      if (!(x < pd || (x == pd && i < pi))) break;
      d[j * kKnnThreads] = pd;
      id[j * kKnnThreads] = pi;
      --j;
    }
    d[j * kKnnThreads] = x;
    id[j * kKnnThreads] = i;
    if (n < k) n++;
    if (n == k) {
      kd = d[(k - 1) * kKnnThreads];
      kid = id[(k - 1) * kKnnThreads];
      kdf = __ull2float_ru(kd);
    }
  }
};

// Squared distance from q to the box lo[dim], hi[dim] in float, scaled down
// by (1 - 2^-18): each gap is exact in float and the d <= 16 rounded squares
// and sums are within (d + 1) * 2^-24 relative of the exact value, so the
// result never exceeds the exact squared distance.  A subtree is pruned only
// when this lower bound exceeds the k-th distance rounded up, i.e. never when
// the exact rule (prune iff mindist^2 > kth) would keep it.
template <int D>
__device__ __forceinline__ float box_mindist_lb(const int32_t *q, const int32_t *box, int dim) {
  const int dd = D ? D : dim;
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < (D ? D : kMaxDim); ++c) {
    if (c < dd) {
      const int32_t x = q[c];
      // at most one of the two gaps is positive
      const float g = (float)(max(box[c] - x, 0) + max(x - box[dd + c], 0));
      s = fmaf(g, g, s);
    }
  }
  return s * (1.0f - 3.814697265625e-06f);   // 1 - 2^-18
}

template <int D, bool STATS>
__global__ void __launch_bounds__(kKnnThreads, 12) k_knn(const ForestView F, const int32_t *qs,
                                                         const int32_t *perm, int64_t m, int k,
                                                         int32_t *out_ids, int64_t *out_d2,
                                                         unsigned long long *stats) {
  // k (d2, id) slots per thread: [slot][thread]
  extern __shared__ __align__(8) unsigned char knn_sm[];
  uint64_t *s_d = reinterpret_cast<uint64_t *>(knn_sm);
  int32_t *s_id = reinterpret_cast<int32_t *>(s_d + (size_t)k * kKnnThreads);
  // whole warps stay resident (and converged) until every lane is done
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if ((t & ~(int64_t)31) >= m) return;
  const bool active = t < m;
  const int64_t qi = active ? (perm ? perm[t] : t) : 0;
  const int dim = D ? D : F.dim;
  const int rec = packed_node_ints(dim);
  const int rs = rec_ints(dim);
  int32_t q[D ? D : kMaxDim];
#pragma unroll
  for (int c = 0; c < (D ? D : kMaxDim); ++c)
    if (c < dim) q[c] = active ? qs[qi * dim + c] : 0;
  TopK best;
  best.init(s_d, s_id);
  unsigned long long nvisit = 0, npts = 0;
  int32_t sv[kStack];
  float smd[kStack];
  const float kInf = __int_as_float(0x7f800000);

  for (int ti = 0; ti < F.ntrees; ++ti) {
    const TreeView &T = F.tree[ti];
    if (T.live[0] <= 0) continue;
    // code >= 0: internal node record; code < 0: leaf -1-code
    int sp = 0;
    if (active) {
      sv[0] = T.h > 0 ? 0 : -1;
      smd[0] = box_mindist_lb<D>(q, T.box, dim);
      sp = 1;
    }
    const int32_t ninternal = (int32_t)(((int64_t)1 << T.h) - 1);
    int pa = 0, pz = 0;
    bool pending = false;   // a leaf [pa, pz) is due but not scanned yet
    while (true) {
      const unsigned wm = __ballot_sync(0xffffffffu, pending || sp > 0);
      if (!wm) break;
      const unsigned pm = __ballot_sync(0xffffffffu, pending);
      if (2 * __popc(pm) >= __popc(wm)) {
        // at least half of the working lanes have a leaf due: scan them together
        if (pending) {
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
#pragma unroll
              for (int c = 0; c < (D ? D : 1); ++c) {
                int32_t g = q[c] - p[c];
                s += (uint64_t)((int64_t)g * g);
              }
            } else {
              id = src[dim];
              for (int c = 0; c < dim; ++c) {
                int32_t g = q[c] - src[c];
                s += (uint64_t)((int64_t)g * g);
              }
            }
            if (id < 0) continue;
            if (STATS) npts++;
            if (best.better(s, id)) best.insert(s, id, k);
          }
          pending = false;
        }
        continue;
      }
      // otherwise every lane without a due leaf takes one traversal step
      if (pending || sp == 0) continue;
      --sp;
      const int code = sv[sp];
      if (best.prune(smd[sp])) continue;
      if (STATS) nvisit++;
      int leaf = -1;
      if (code < 0) {
        leaf = -1 - code;
      } else if (code >= ninternal || sp + 2 > kStack) {
        atomicOr(F.err, code >= ninternal ? kErrChild : kErrStack);
      } else {
        const int32_t *r = T.pk + (int64_t)code * rec;
        int4 hdr;
        float ml, mr;
        if (D) {
          // the whole 32-byte-aligned record in 16-byte loads
          int32_t rr[D ? packed_node_ints(D) : 4];
#pragma unroll
          for (int c4 = 0; c4 < (D ? packed_node_ints(D) : 4); c4 += 4) {
            const int4 v = *reinterpret_cast<const int4 *>(r + c4);
            rr[c4] = v.x;
            rr[c4 + 1] = v.y;
            rr[c4 + 2] = v.z;
            rr[c4 + 3] = v.w;
          }
          hdr = make_int4(rr[0], rr[1], rr[2], rr[3]);
          ml = hdr.z > 0 ? box_mindist_lb<D>(q, rr + 4, dim) : kInf;
          mr = hdr.w > 0 ? box_mindist_lb<D>(q, rr + 4 + 2 * (D ? D : 1), dim) : kInf;
        } else {
          hdr = *reinterpret_cast<const int4 *>(r);
          ml = hdr.z > 0 ? box_mindist_lb<D>(q, r + 4, dim) : kInf;
          mr = hdr.w > 0 ? box_mindist_lb<D>(q, r + 4 + 2 * dim, dim) : kInf;
        }
        const bool lfirst = ml <= mr;
        const int vn = lfirst ? hdr.x : hdr.y, vf = lfirst ? hdr.y : hdr.x;
        const float mn = lfirst ? ml : mr, mf = lfirst ? mr : ml;
        if (mf != kInf && !best.prune(mf)) { sv[sp] = vf; smd[sp] = mf; sp++; }
        if (mn != kInf && !best.prune(mn)) {
          if (vn < 0) {          // nearer child is a leaf: due now
            if (STATS) nvisit++;
            leaf = -1 - vn;
          } else {
            sv[sp] = vn;
            smd[sp] = mn;
            sp++;
          }
        }
      }
      if (leaf >= 0) {
        if (leaf > ninternal) {
          atomicOr(F.err, kErrChild);
        } else {
          pa = T.leaf_off[leaf];
          pz = T.leaf_off[leaf + 1];
          if (pa < 0 || pz > T.size || pa > pz) atomicOr(F.err, kErrLeaf);
          else pending = true;
        }
      }
    }
  }
  if (!active) return;
  // the buffer tree: exact scan of its points
  for (int64_t j = 0; j < F.nbuf; ++j) {
    const int32_t id = F.buf[j];
    const int32_t *p = F.idtab + (int64_t)id * dim;
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
    oi[j] = ok ? best.id[j * kKnnThreads] : -1;
    od[j] = ok ? (int64_t)best.d[j * kKnnThreads] : INT64_MAX;
  }
  if (STATS) {
    atomicAdd(&stats[0], nvisit);
    atomicAdd(&stats[1], npts);
    atomicAdd(&stats[2], 1ull);
  }
}

template <int D>
void launch_d(const ForestView &fv, const int32_t *q, const int32_t *perm, int64_t m, int k,
              int32_t *oi, int64_t *od, unsigned long long *stats, cudaStream_t s) {
  const size_t smem = (size_t)k * kKnnThreads * 12;   // <= 48 KB for k <= 32
  KScope ks_(kK_knn, s);
  const unsigned grid = (unsigned)((m + kKnnThreads - 1) / kKnnThreads);
  if (stats)
    k_knn<D, true><<<grid, kKnnThreads, smem, s>>>(fv, q, perm, m, k, oi, od, stats);
  else
    k_knn<D, false><<<grid, kKnnThreads, smem, s>>>(fv, q, perm, m, k, oi, od, stats);
}

// ---------------------------------------------------------------------------
// packed node records: one per internal node, in the vEB order of the tree's
// h internal levels (a complete tree of its own)
// ---------------------------------------------------------------------------

__global__ void k_pack_nodes(const Node *node, const int32_t *box, const int32_t *live, int h,
                             int dim, int32_t *pk) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nint = ((int64_t)1 << h) - 1;
  if (g >= nint) return;
  const int t = 63 - __clzll(g + 1);          // depth of the g-th internal node (BFS order)
  const int64_t i = g + 1 - ((int64_t)1 << t);
  const int64_t v = veb_slot(h + 1, t, i);    // slot among all nodes
  const int64_t p = veb_slot(h, t, i);        // slot among internal nodes
  const int rec = packed_node_ints(dim);
  const int rs = rec_ints(dim);
  int32_t *r = pk + p * rec;
  const Node nd = node[v];
  const int2 ch = make_int2(nd.l, nd.r);
  int code[2];
  if (t + 1 < h) {
    code[0] = (int)veb_slot(h, t + 1, 2 * i);
    code[1] = (int)veb_slot(h, t + 1, 2 * i + 1);
  } else {
    code[0] = (int)(-1 - 2 * i);
    code[1] = (int)(-2 - 2 * i);
  }
  r[0] = code[0];
  r[1] = code[1];
  r[2] = live[ch.x];
  r[3] = live[ch.y];
  for (int c = 0; c < 2 * dim; ++c) {
    r[4 + c] = box[(int64_t)ch.x * 2 * dim + c];
    r[4 + 2 * dim + c] = box[(int64_t)ch.y * 2 * dim + c];
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

__global__ void k_qkey_hist(const int32_t *coords, const int32_t *ids, int64_t m, int dim, int B,
                            uint32_t *hist) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
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
__global__ void k_qscatter(const int32_t *coords, const int32_t *ids, int64_t m, int dim, int B,
                           uint32_t *offs, const uint32_t *bsum, int32_t *out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  uint32_t key = morton_key(point_row(coords, ids, i, dim), dim, B);
  uint32_t pos = bsum[key / kScanPer] + atomicAdd(&offs[key], 1u);
  if (pos < m) out[pos] = ids ? ids[i] : (int32_t)i;
}

}  // namespace

int launch_knn(const ForestView &fv, const int32_t *q, const int32_t *perm, int64_t m, int k,
               int32_t *out_ids, int64_t *out_d2, unsigned long long *stats, cudaStream_t s) {
  if (m <= 0) return BDL_OK;
  switch (fv.dim) {
    case 2: launch_d<2>(fv, q, perm, m, k, out_ids, out_d2, stats, s); break;
    case 3: launch_d<3>(fv, q, perm, m, k, out_ids, out_d2, stats, s); break;
    case 5: launch_d<5>(fv, q, perm, m, k, out_ids, out_d2, stats, s); break;
    case 7: launch_d<7>(fv, q, perm, m, k, out_ids, out_d2, stats, s); break;
    default: launch_d<0>(fv, q, perm, m, k, out_ids, out_d2, stats, s); break;
  }
  return cuda_check(cudaGetLastError(), "knn kernel");
}

void launch_pack_nodes(const Tree *t, int dim, cudaStream_t s) {
  int64_t nint = ((int64_t)1 << t->h) - 1;
  if (nint <= 0) return;
  KScope ks_(kK_pack_nodes, s);
  k_pack_nodes<<<(unsigned)((nint + 255) / 256), 256, 0, s>>>(t->node, t->box, t->live_nodes, t->h,
                                                               dim, t->pk);
}

// After an erase only the live counts of the packed records change.
__global__ void k_pack_lives(const Node *node, const int32_t *live, int h, int dim, int32_t *pk) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nint = ((int64_t)1 << h) - 1;
  if (g >= nint) return;
  const int t = 63 - __clzll(g + 1);
  const int64_t i = g + 1 - ((int64_t)1 << t);
  const Node nd = node[veb_slot(h + 1, t, i)];
  int2 lv = make_int2(live[nd.l], live[nd.r]);
  *reinterpret_cast<int2 *>(pk + veb_slot(h, t, i) * packed_node_ints(dim) + 2) = lv;
}

void launch_pack_lives(const Tree *t, int dim, cudaStream_t s) {
  int64_t nint = ((int64_t)1 << t->h) - 1;
  if (nint <= 0) return;
  KScope ks_(kK_pack_nodes, s);
  k_pack_lives<<<(unsigned)((nint + 255) / 256), 256, 0, s>>>(t->node, t->live_nodes, t->h, dim, t->pk);
}

size_t query_sort_bytes(int64_t m, int dim) {
  int64_t nbins = (int64_t)1 << (morton_bits_per_dim(dim) * dim);
  int64_t nb = (nbins + kScanPer - 1) / kScanPer;
  return ((size_t)m * 4 + 255) / 256 * 256 + (size_t)nbins * 4 + 256 + (size_t)nb * 4 + 256;
}

void launch_point_sort(const int32_t *coords, const int32_t *ids, int64_t m, int dim,
                       void *scratch, int32_t *out, cudaStream_t s) {
  const int B = morton_bits_per_dim(dim);
  const int64_t nbins = (int64_t)1 << (B * dim);
  const int64_t nb = (nbins + kScanPer - 1) / kScanPer;   // <= 256
  uint32_t *hist = (uint32_t *)scratch;
  uint32_t *bsum = (uint32_t *)((char *)scratch + ((size_t)nbins * 4 + 255) / 256 * 256);
  cudaMemsetAsync(hist, 0, (size_t)nbins * 4, s);
  const unsigned g = (unsigned)((m + 255) / 256);
  { KScope ks_(kK_qsort, s); k_qkey_hist<<<g, 256, 0, s>>>(coords, ids, m, dim, B, hist); }
  { KScope ks_(kK_qsort, s); k_scan_local<<<(unsigned)nb, 1024, 0, s>>>(hist, nbins, bsum); }
  { KScope ks_(kK_qsort, s); k_scan_top<<<1, 1024, 0, s>>>(bsum, nb); }
  { KScope ks_(kK_qsort, s); k_qscatter<<<g, 256, 0, s>>>(coords, ids, m, dim, B, hist, bsum, out); }
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
    st = finish_call(f, s, launch_knn(fv, q, perm, m, k, out_ids, out_d2, f->knn_stats, s));
  }
  if (prev >= 0 && prev != f->device) cudaSetDevice(prev);
  return st;
}

