// Host-side check of the library's layout arithmetic (bdl_internal.cuh):
// the binary vEB slots, and the packed k-NN records' level order, slots and
// entries.  Prints the number of violations; exit status 0 when there are none.
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
