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

__global__ void k_append_validate(const int32_t *pts, int64_t n, int32_t *dst, int64_t *flag) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool bad = false;
  if (i < n) {
    int32_t v = pts[i];
    bad = v < 0 || v >= (1 << kCoordBits);
    dst[i] = v;
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr((unsigned long long *)flag, 1ull);
}

__global__ void k_set_alive(uint32_t *alive, int64_t first, int64_t n) {
  int64_t w = (first >> 5) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t last = first + n;  // exclusive
  if ((w << 5) >= last) return;
  uint32_t m = 0xffffffffu;
  if ((w << 5) < first) m &= 0xffffffffu << (first & 31);
  if (((w + 1) << 5) > last) m &= 0xffffffffu >> (32 - (last & 31));
  atomicOr(&alive[w], m);
}

__global__ void k_iota(int32_t *out, int64_t first, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (int32_t)(first + i);
}

// Clear the alive bit of every live id in the batch; the thread that clears
// it owns the erase of that id (repeats and dead ids drop out here).
__global__ void k_erase_mark(uint32_t *alive, int64_t next_id, const int32_t *ids, int64_t n,
                             int32_t *list, int64_t *count) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool own = false;
  int32_t id = -1;
  if (i < n) {
    id = ids[i];
    if (id >= 0 && id < next_id) {
      uint32_t bit = 1u << (id & 31);
      own = (atomicAnd(&alive[id >> 5], ~bit) & bit) != 0;
    }
  }
  unsigned m = __ballot_sync(0xffffffffu, own);
  if (!m) return;
  int lane = threadIdx.x & 31;
  unsigned long long base = 0;
  if (lane == __ffs(m) - 1) base = atomicAdd((unsigned long long *)count, (unsigned long long)__popc(m));
  base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
  if (own) list[base + __popc(m & ((1u << lane) - 1))] = id;
}

// K6a: split-block bloom filter over the live ids of one tree.
__global__ void k_bloom_build(const int32_t *pts, int64_t size, int dim, uint32_t *bloom,
                              int64_t blocks, uint64_t seed) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= size) return;
  int32_t id = pts[j * rec_ints(dim) + dim];
  if (id < 0) return;
  int64_t blk;
  uint64_t bits;
  bloom_hash(seed, blocks, id, blk, bits);
  for (int w = 0; w < 8; ++w) atomicOr(&bloom[blk * 8 + w], bloom_word_bit(bits, w));
}

// K6b + K7: for each erased id and each tree (largest first) probe the bloom
// filter (one 32-byte sector); on a hit descend by the composite key to the
// unique leaf, find the id, tombstone it and decrement the live counts along
// the path.  A live id that no tree holds is in the buffer.
__global__ void k_erase_locate(const ForestView F, uint64_t seed, const int32_t *list, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  bool pending = i < n;
  int32_t id = pending ? list[i] : 0;
  const int32_t *xq = F.idtab + (int64_t)id * F.dim;
  int32_t path[kMaxLevel + 2];
  // all bloom probes first: independent 32-byte loads, one per tree
  uint64_t maybe_mask = 0;
  if (pending) {
    for (int ti = 0; ti < F.ntrees; ++ti) {
      const TreeView &T = F.tree[ti];
      bool maybe = true;
      if (T.bloom) {
        int64_t blk;
        uint64_t bits;
        bloom_hash(seed, T.bloom_blocks, id, blk, bits);
        const uint4 *bw = reinterpret_cast<const uint4 *>(T.bloom + blk * 8);
        uint4 a = bw[0], b = bw[1];
        uint32_t wv[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
        for (int w = 0; w < 8; ++w) maybe = maybe && (wv[w] & bloom_word_bit(bits, w));
      }
      maybe_mask |= (uint64_t)maybe << ti;
    }
  }
  for (int ti = 0; ti < F.ntrees; ++ti) {
    const TreeView &T = F.tree[ti];
    bool found = false;
    if (pending) {
      if ((maybe_mask >> ti) & 1) {
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
        int leaf = -1 - nd.l;
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
      }
    }
    unsigned fm = __ballot_sync(0xffffffffu, found);
    if (found) {
      for (int d = 0; d <= T.h; ++d) {
        int v = path[d];
        unsigned peers = __match_any_sync(fm, v);
        if (lane == __ffs(peers) - 1) atomicSub(&T.live[v], __popc(peers));
      }
      pending = false;
    }
  }
}

// Keep the buffer ids that are still alive, in order (one CTA).
__global__ void k_buffer_compact(int32_t *buf, int64_t nbuf, const uint32_t *alive, int64_t *out_n) {
  __shared__ int wsum[32];
  __shared__ int base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t a = 0; a < nbuf; a += blockDim.x) {
    int64_t j = a + threadIdx.x;
    int32_t id = j < nbuf ? buf[j] : -1;
    bool keep = j < nbuf && ((alive[id >> 5] >> (id & 31)) & 1);
    unsigned m = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) wsum[warp] = __popc(m);
    __syncthreads();
    int pre = 0, tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      if (w < warp) pre += wsum[w];
      tot += wsum[w];
    }
    int dst = base + pre + __popc(m & ((1u << lane) - 1));
    __syncthreads();   // every read of buf[a..] is done before anyone writes
    if (keep) buf[dst] = id;
    __syncthreads();
    if (threadIdx.x == 0) base += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *out_n = base;
}

__global__ void k_gather_roots(const ForestView F, int64_t *out) {
  int t = threadIdx.x;
  if (t < F.ntrees) out[t] = F.tree[t].live[0];
}

// Ordered gather: mark the live ids of the given trees in a bitmap, then emit
// them in increasing order through a prefix sum of per-word popcounts.
__global__ void k_mark_ids(const int32_t *pts, int64_t size, int dim, uint32_t *bm) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= size) return;
  int32_t id = pts[j * rec_ints(dim) + dim];
  if (id >= 0) atomicOr(&bm[id >> 5], 1u << (id & 31));
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

__global__ void k_popc_blocks(const uint32_t *bm, int64_t nwords, int64_t *bsum) {
  int64_t w0 = ((int64_t)blockIdx.x * kScanBlock + threadIdx.x) * kScanWords;
  int c = 0;
  for (int k = 0; k < kScanWords; ++k)
    if (w0 + k < nwords) c += __popc(bm[w0 + k]);
  int tot;
  block_excl_scan(c, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_bsum(int64_t *bsum, int64_t nb) {
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t a = 0; a < nb; a += blockDim.x) {
    int64_t j = a + threadIdx.x;
    int v = j < nb ? (int)bsum[j] : 0;
    int tot;
    int e = block_excl_scan(v, &tot);
    if (j < nb) bsum[j] = carry + e;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
}

__global__ void k_emit_ids(const uint32_t *bm, int64_t nwords, const int64_t *bsum, int32_t *out,
                           int64_t nout, unsigned long long *err) {
  int64_t w0 = ((int64_t)blockIdx.x * kScanBlock + threadIdx.x) * kScanWords;
  uint32_t wv[kScanWords];
  int c = 0;
  for (int k = 0; k < kScanWords; ++k) {
    wv[k] = w0 + k < nwords ? bm[w0 + k] : 0u;
    c += __popc(wv[k]);
  }
  int tot;
  int64_t pos = bsum[blockIdx.x] + block_excl_scan(c, &tot);
  for (int k = 0; k < kScanWords; ++k) {
    uint32_t x = wv[k];
    while (x) {
      int b = __ffs(x) - 1;
      if (pos < nout) out[pos] = (int32_t)(((w0 + k) << 5) + b);
      else atomicOr(err, kErrGather);
      pos++;
      x &= x - 1;
    }
  }
}

}  // namespace

void launch_append_validate(const int32_t *pts, int64_t n, int dim, int32_t *idtab_dst,
                            int64_t *flag, cudaStream_t s) {
  int64_t tot = n * dim;
  if (tot <= 0) return;
  { KScope ks_(kK_append_validate, s);
  k_append_validate<<<(unsigned)cdiv(tot, 256), 256, 0, s>>>(pts, tot, idtab_dst, flag); }
}

void launch_set_alive(uint32_t *alive, int64_t first, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  int64_t words = ((first + n - 1) >> 5) - (first >> 5) + 1;
  { KScope ks_(kK_set_alive, s);
  k_set_alive<<<(unsigned)cdiv(words, 256), 256, 0, s>>>(alive, first, n); }
}

void launch_iota(int32_t *out, int64_t first, int64_t n, cudaStream_t s) {
  if (n <= 0 || !out) return;
  { KScope ks_(kK_iota, s);
  k_iota<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(out, first, n); }
}

void launch_erase_mark(uint32_t *alive, int64_t next_id, const int32_t *ids, int64_t n,
                       int32_t *list, int64_t *count, cudaStream_t s) {
  if (n <= 0) return;
  { KScope ks_(kK_erase_mark, s);
  k_erase_mark<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(alive, next_id, ids, n, list, count); }
}

void launch_bloom_build(const Tree *t, int f_dim, uint64_t seed, cudaStream_t s) {
  if (t->size <= 0) return;
  { KScope ks_(kK_bloom_build, s);
  k_bloom_build<<<(unsigned)cdiv(t->size, 256), 256, 0, s>>>(t->pts, t->size, f_dim, t->bloom,
                                                              t->bloom_blocks, seed); }
}

void launch_erase_locate(const ForestView &fv, uint64_t seed, const int32_t *list, int64_t n,
                         cudaStream_t s) {
  if (n <= 0 || fv.ntrees == 0) return;
  { KScope ks_(kK_erase_locate, s);
  k_erase_locate<<<(unsigned)cdiv(n, 128), 128, 0, s>>>(fv, seed, list, n); }
}

void launch_buffer_compact(int32_t *buf, int64_t nbuf, const uint32_t *alive, int64_t *out_n,
                           cudaStream_t s) {
  { KScope ks_(kK_buffer_compact, s);
  k_buffer_compact<<<1, 1024, 0, s>>>(buf, nbuf, alive, out_n); }
}

void launch_gather_roots(const ForestView &fv, int64_t *out, cudaStream_t s) {
  if (fv.ntrees == 0) return;
  { KScope ks_(kK_gather_roots, s);
  k_gather_roots<<<1, 64, 0, s>>>(fv, out); }
}

int collect_sorted_live(bdl_forest *f, const std::vector<Tree *> &from, int64_t n, int32_t *out,
                        cudaStream_t s) {
  if (n <= 0) return BDL_OK;
  int64_t nwords = (f->next_id + 31) >> 5;
  int64_t per_block = (int64_t)kScanBlock * kScanWords;
  int64_t nb = cdiv(nwords, per_block);
  size_t bytes = (size_t)nwords * 4 + 256 + (size_t)nb * 8;
  void *blk = nullptr;
  int st = dev_alloc(f, &blk, bytes, s);
  if (st) return st;
  uint32_t *bm = (uint32_t *)blk;
  int64_t *bsum = (int64_t *)((char *)blk + ((size_t)nwords * 4 + 255) / 256 * 256);
  cudaMemsetAsync(bm, 0, (size_t)nwords * 4, s);
  for (Tree *t : from) {
    { KScope ks_(kK_mark_ids, s);
    k_mark_ids<<<(unsigned)cdiv(t->size, 256), 256, 0, s>>>(t->pts, t->size, f->dim, bm); }
  }
  { KScope ks_(kK_popc_blocks, s);
  k_popc_blocks<<<(unsigned)nb, kScanBlock, 0, s>>>(bm, nwords, bsum); }
  { KScope ks_(kK_scan_bsum, s);
  k_scan_bsum<<<1, 1024, 0, s>>>(bsum, nb); }
  { KScope ks_(kK_emit_ids, s);
  k_emit_ids<<<(unsigned)nb, kScanBlock, 0, s>>>(bm, nwords, bsum, out, n, f->err); }
  int err = cuda_check(cudaGetLastError(), "collect_sorted_live");
  dev_free(f, blk, bytes, s);
  return err;
}

}  // namespace bdl
