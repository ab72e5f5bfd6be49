// Host-side check of the library's layout arithmetic (bdl_internal.cuh):
// the binary vEB slots, the segments of a level, the tree height, the bloom
// hash's SplitMix64 mixer, and the packed k-NN records' level order, slots
// and entries.  Prints the number of violations; exit status 0 when there are none.
#include <cstdio>
#include <vector>

#include "../paper_2112_06188_gb300/csrc/bdl_internal.cuh"

using namespace bdl;

int main() {
  long bad = 0;
  // vEB worked example (Sec. IV-A1, Fig. 3): a tree of 4 levels puts the
  // roots of its four bottom subtrees at slots 3, 6, 9 and 12
  for (int j = 0; j < 4; ++j)
    if (veb_slot(4, 2, j) != 3 + 3 * j) ++bad;
  // veb_slot(l, ., .) is a bijection onto [0, 2^l - 1)
  for (int l = 1; l <= 16; ++l) {
    const int64_t n = ((int64_t)1 << l) - 1;
    std::vector<char> seen(n, 0);
    for (int t = 0; t < l; ++t)
      for (int64_t i = 0; i < ((int64_t)1 << t); ++i) {
        const int64_t v = veb_slot(l, t, i);
        if (v < 0 || v >= n || seen[v]) ++bad;
        else seen[v] = 1;
      }
  }
  // segments of a tree over s points (reading G3: the left child of a
  // segment of m points holds ceil(m / 2) of them): seg_range and seg_of agree,
  // segments tile [0, s), and children split their parent that way
  for (int64_t sz : {1, 2, 3, 7, 16, 17, 100, 1000, 4097}) {
    for (int t = 0; t <= 8; ++t) {
      int64_t next = 0;
      for (int64_t i = 0; i < ((int64_t)1 << t); ++i) {
        int64_t st, m;
        seg_range(sz, t, i, st, m);
        if (st != next || m < 0) ++bad;
        next = st + m;
        int64_t l0, lm, r0, rm;
        seg_range(sz, t + 1, 2 * i, l0, lm);
        seg_range(sz, t + 1, 2 * i + 1, r0, rm);
        if (l0 != st || lm != (m + 1) / 2 || r0 != st + lm || rm != m - lm) ++bad;
        for (int64_t p = st; p < st + m; ++p) {
          int64_t a2, m2;
          if (seg_of(sz, t, p, a2, m2) != i || a2 != st || m2 != m) ++bad;
        }
      }
      if (next != sz) ++bad;
    }
  }
  // split levels h = ceil(log2(ceil(s / L)))
  for (int64_t sz = 1; sz <= 5000; sz += 37)
    for (int L : {2, 8, 16, 24, 32}) {
      const int h = tree_height(sz, L);
      const int64_t leaves = (sz + L - 1) / L;
      if (((int64_t)1 << h) < leaves || (h > 0 && ((int64_t)1 << (h - 1)) >= leaves)) ++bad;
    }
  // the bloom hash's mixer: SplitMix64's published first output for seed 0
  if (splitmix64(0) != 0xe220a8397b1dcdafull) ++bad;
  // packed records of a tree with h internal levels
  for (int h = 0; h <= 20; ++h) {
    const int64_t n = packed_nrec(h);
    std::vector<char> seen(n, 0);
    int64_t expect = 0;   // records: the root (h > 0) and every node at a depth t > 0 with h - t even
    for (int t = 0; t < h; ++t)
      if (t == 0 || (h - t) % 2 == 0) expect += (int64_t)1 << t;
    if (n != expect) ++bad;
    for (int64_t g = 0; g < n; ++g) {
      int t;
      int64_t i;
      packed_record_of(h, g, t, i);
      if (t < 0 || t >= h || i < 0 || i >= ((int64_t)1 << t) || !(t == 0 || (h - t) % 2 == 0)) {
        ++bad;
        continue;
      }
      const int64_t sl = packed_slot(h, t, i);
      if (sl < 0 || sl >= n || seen[sl]) ++bad;
      else seen[sl] = 1;
      // entries: two levels down (one for the root of an odd h), records or leaves
      const int e = packed_step(h, t);
      if (e != ((h % 2 == 1 && t == 0) ? 1 : 2)) ++bad;
      for (int a = 0; a < (1 << e); ++a) {
        const int tc = t + e;
        const int64_t ci = (i << e) + a;
        if (tc > h) ++bad;
        else if (tc < h) {
          const int64_t c = packed_slot(h, tc, ci);
          if (c < 0 || c >= n || (h - tc) % 2 != 0) ++bad;
        }
      }
    }
  }
  std::printf("%ld\n", bad);
  return bad != 0;
}
