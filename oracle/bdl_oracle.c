/*
 * bdl_oracle.c -- plain, serial CPU BDL-tree (arXiv 2112.06188).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline / reference legs of bench.py load this library.  It shares no
 * code, header, table or constant generator with the CUDA library, and the
 * CUDA library never calls it.
 *
 * What it computes, in the paper's order:
 *   Sec. III-D   logarithmic method: static trees of capacity X*2^i + a buffer
 *   Alg. 1       BuildvEB_S: recursive top/bottom construction in vEB order
 *   Alg. 2       Erase_S: partition the erase batch around each split
 *   Sec. IV-A    kNN_S with the 2k-entry kNN buffer
 *   Alg. 3       Insert_L: F_new = F + |P|/X, merge cleared trees into new ones
 *   Alg. 4       Erase_L: erase from every tree, reinsert trees below half
 *   Alg. 5       kNN_L: one tree at a time, largest first (Sec. V-B)
 *   Sec. V-A     per-tree bloom filter, built lazily before the first erase
 *   Sec. V-D     leaves hold up to L points
 *   Sec. V-C     the spatial-median splitting rule, as an alternative to the
 *                object median (orc_forest_set_split)
 * plus brute-force exact k-NN (the closed-form definition of the result).
 *
 * Readings where the paper is silent, ambiguous or garbled are stated at the
 * function that implements them (search for "Reading").
 *
 * Parity pins: the vEB worked example of Sec. IV-A1 (subtree offsets
 * 3,6,9,12), the insert example of Sec. IV-B1 / Fig. 4 (tree masks
 * 1->2->3->4), brute-force k-NN, and the invariants of Sec. IV (half splits,
 * binary counter of the live count, no tree below half after Erase_L).
 * Which pool points stay in the buffer (reading G5 below) and the bloom hash
 * family are "parity unpinned" beyond those invariants.
 *
 * Integers only: coordinates on a 2^20 grid, squared distances in int64,
 * ties broken by point id.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXDIM 16
#define OR_MAXLEVEL 48
#define OR_D2_NONE INT64_MAX

/* ------------------------------------------------------------------ */
/* data                                                                */
/* ------------------------------------------------------------------ */

typedef struct {
    int is_leaf;
    int depth;
    int64_t bfs;            /* index among the nodes of its depth, 0..2^depth-1 */
    int64_t key;            /* split key (internal nodes) */
    int64_t lo, mid, hi;    /* point range; [lo,mid) left child, [mid,hi) right */
    int64_t live;
    int32_t box[2 * OR_MAXDIM];   /* lo[0..d), hi[0..d) over the node's points */
} onode;

typedef struct {
    int level;
    int64_t size;           /* points stored (live + erased) */
    int64_t live;
    int h;                  /* split levels; leaves at depth h */
    int64_t nnodes;         /* 2^(h+1) - 1 */
    onode *nodes;           /* vEB order */
    int64_t *bfs2veb;       /* [2^t - 1 + i] -> vEB slot */
    int32_t *ids;           /* [size] in leaf order */
    unsigned char *dead;    /* [size] erased flags */
    uint32_t *bloom;        /* NULL until built (Sec. V-A: lazily) */
    int64_t bloom_blocks;
} otree;

typedef struct {
    int dim, L, X, bpk;
    int split;              /* 0: object median (default), 1: spatial median */
    uint64_t seed;
    int32_t *coord;         /* id table: [id][dim] */
    unsigned char *alive;   /* [id] */
    int64_t n_ids, cap_ids;
    int32_t *buf;           /* buffer ids, ascending */
    int64_t nbuf;
    otree *tree[OR_MAXLEVEL];
    uint64_t F;             /* bit i set <=> static tree i is full (Alg. 3) */
} oforest;

static void *xmalloc(size_t n) { void *p = malloc(n ? n : 1); if (!p) abort(); return p; }
static void *xcalloc(size_t n, size_t s) { void *p = calloc(n ? n : 1, s ? s : 1); if (!p) abort(); return p; }

/* composite split key in dimension c (reading G3): coordinate, ties by id */
static int64_t okey(const oforest *f, int32_t id, int c)
{
    return ((int64_t)f->coord[(int64_t)id * f->dim + c] << 31) | (int64_t)id;
}

static int64_t sqdist(const oforest *f, const int32_t *q, int32_t id)
{
    int64_t s = 0;
    for (int c = 0; c < f->dim; c++) {
        int64_t diff = (int64_t)q[c] - (int64_t)f->coord[(int64_t)id * f->dim + c];
        s += diff * diff;
    }
    return s;
}

/* ------------------------------------------------------------------ */
/* Alg. 1: BuildvEB_S                                                  */
/* ------------------------------------------------------------------ */

typedef struct { int64_t key; int32_t id; } kv;

static int kv_cmp(const void *a, const void *b)
{
    int64_t x = ((const kv *)a)->key, y = ((const kv *)b)->key;
    return (x > y) - (x < y);
}

/* Reading G1: the bottom part gets l_b = hyperceil(l/2) levels (smallest power
 * of two >= l/2).  The printed (l+1)/2 gives l_b = l for l = 2 and l = 4 and
 * would never terminate; the worked example (l = 4 -> l_b = l_t = 2) fixes l/2.
 * For odd l both forms agree. */
static int veb_bottom_levels(int l)
{
    int lb = 1;
    while (2 * lb < l) lb *= 2;       /* smallest power of two >= l/2 */
    return lb;
}

typedef struct {
    oforest *f;
    otree *t;
    int32_t *ids;   /* the tree's id array being arranged */
    kv *tmp;
} obuild;

/* BuildvEBRecursive(Q = ids[lo,hi), idx, c, l, top).
 * Reading G2: the node at depth t splits dimension t mod d, i.e. the bottom
 * subtrees start at (c + l_t) mod d; the base case is l = 1. */
static void build_rec(obuild *b, int64_t lo, int64_t hi, int64_t idx, int c, int l,
                      int top, int depth, int64_t bfs)
{
    oforest *f = b->f;
    otree *t = b->t;
    if (l == 1) {
        onode *nd = &t->nodes[idx];
        memset(nd, 0, sizeof(*nd));
        nd->depth = depth;
        nd->bfs = bfs;
        nd->lo = lo;
        nd->hi = hi;
        t->bfs2veb[((int64_t)1 << depth) - 1 + bfs] = idx;
        if (top && f->split == 1) {
            /* Spatial median (Sec. V-C): the splitting value is the average of
             * the smallest and largest coordinate c among the node's points,
             * and the points are partitioned around it.
             * Reading G12: on the integer grid the average is rounded down,
             * v = floor((min + max) / 2); points with coordinate <= v go left.
             * The stored key is (v << 31) | (2^31 - 1), so that a point's
             * composite key is <= it exactly when its coordinate is <= v and
             * descents by key stay as for the object median.  The tree keeps
             * the shape of reading G2 (h split levels), so children may hold
             * any number of points, none included; an empty node's v is 0. */
            int64_t m = hi - lo;
            int32_t mn = INT32_MAX, mx = INT32_MIN;
            for (int64_t i = lo; i < hi; i++) {
                int32_t x = f->coord[(int64_t)b->ids[i] * f->dim + c];
                if (x < mn) mn = x;
                if (x > mx) mx = x;
            }
            int64_t v = m > 0 ? ((int64_t)mn + (int64_t)mx) / 2 : 0;
            int64_t nl = 0;
            for (int64_t i = lo; i < hi; i++)      /* left part first, stable */
                if (f->coord[(int64_t)b->ids[i] * f->dim + c] <= v) b->tmp[nl++].id = b->ids[i];
            int64_t nr = nl;
            for (int64_t i = lo; i < hi; i++)
                if (f->coord[(int64_t)b->ids[i] * f->dim + c] > v) b->tmp[nr++].id = b->ids[i];
            for (int64_t i = 0; i < m; i++) b->ids[lo + i] = b->tmp[i].id;
            nd->is_leaf = 0;
            nd->key = (v << 31) | (int64_t)0x7FFFFFFF;
            nd->mid = lo + nl;
        } else if (top) {
            /* median partition in dimension c (Sec. V-C: by sorting).
             * Reading G3: the left child takes the ceil(m/2) smallest composite
             * keys; the node stores the largest key of the left child. */
            int64_t m = hi - lo;
            if (m < 1) abort();
            for (int64_t i = 0; i < m; i++) {
                b->tmp[i].id = b->ids[lo + i];
                b->tmp[i].key = okey(f, b->ids[lo + i], c);
            }
            qsort(b->tmp, (size_t)m, sizeof(kv), kv_cmp);
            for (int64_t i = 0; i < m; i++) b->ids[lo + i] = b->tmp[i].id;
            int64_t ml = (m + 1) / 2;
            nd->is_leaf = 0;
            nd->key = b->tmp[ml - 1].key;
            nd->mid = lo + ml;
        } else {
            nd->is_leaf = 1;
            nd->mid = hi;
        }
        return;
    }
    int lb = veb_bottom_levels(l);
    int lt = l - lb;
    build_rec(b, lo, hi, idx, c, lt, 1, depth, bfs);           /* top half */
    int64_t idxb = idx + ((int64_t)1 << lt) - 1;                 /* offset of bottoms */
    int64_t nb = (int64_t)1 << lt;
    int64_t bsize = ((int64_t)1 << lb) - 1;
    for (int64_t i = 0; i < nb; i++) {
        /* Q_i: the half of the points held by the top tree's parent node */
        int pd = depth + lt - 1;
        int64_t pbfs = (bfs << (lt - 1)) + (i >> 1);
        const onode *par = &t->nodes[t->bfs2veb[((int64_t)1 << pd) - 1 + pbfs]];
        int64_t qlo = (i & 1) ? par->mid : par->lo;
        int64_t qhi = (i & 1) ? par->hi : par->mid;
        build_rec(b, qlo, qhi, idxb + i * bsize, (c + lt) % f->dim, lb, top,
                  depth + lt, (bfs << lt) + i);
    }
}

static void node_box_live(const oforest *f, otree *t, onode *nd)
{
    int d = f->dim;
    for (int c = 0; c < d; c++) { nd->box[c] = INT32_MAX; nd->box[d + c] = INT32_MIN; }
    if (nd->is_leaf) {
        nd->live = 0;
        for (int64_t j = nd->lo; j < nd->hi; j++) {
            if (!t->dead[j]) nd->live++;
            for (int c = 0; c < d; c++) {
                int32_t x = f->coord[(int64_t)t->ids[j] * d + c];
                if (x < nd->box[c]) nd->box[c] = x;
                if (x > nd->box[d + c]) nd->box[d + c] = x;
            }
        }
    } else {
        const onode *a = &t->nodes[t->bfs2veb[((int64_t)1 << (nd->depth + 1)) - 1 + 2 * nd->bfs]];
        const onode *z = &t->nodes[t->bfs2veb[((int64_t)1 << (nd->depth + 1)) - 1 + 2 * nd->bfs + 1]];
        nd->live = a->live + z->live;
        for (int c = 0; c < d; c++) {
            nd->box[c] = a->box[c] < z->box[c] ? a->box[c] : z->box[c];
            nd->box[d + c] = a->box[d + c] > z->box[d + c] ? a->box[d + c] : z->box[d + c];
        }
    }
}

/* Reading G2: a complete tree with h = ceil(log2(ceil(s/L))) split levels and
 * 2^h leaves, i.e. l = h + 1 levels of nodes and 2^(h+1) - 1 nodes. */
static int tree_height(int64_t s, int L)
{
    int64_t nl = (s + L - 1) / L;
    int h = 0;
    while (((int64_t)1 << h) < nl) h++;
    return h;
}

static otree *build_tree(oforest *f, int level, const int32_t *ids, int64_t s)
{
    otree *t = (otree *)xcalloc(1, sizeof(otree));
    t->level = level;
    t->size = s;
    t->live = s;
    t->h = tree_height(s, f->L);
    t->nnodes = ((int64_t)2 << t->h) - 1;
    t->nodes = (onode *)xcalloc((size_t)t->nnodes, sizeof(onode));
    t->bfs2veb = (int64_t *)xmalloc((size_t)t->nnodes * sizeof(int64_t));
    t->ids = (int32_t *)xmalloc((size_t)s * sizeof(int32_t));
    t->dead = (unsigned char *)xcalloc((size_t)s, 1);
    memcpy(t->ids, ids, (size_t)s * sizeof(int32_t));
    obuild b = { f, t, t->ids, (kv *)xmalloc((size_t)s * sizeof(kv)) };
    build_rec(&b, 0, s, 0, 0, t->h + 1, 0, 0, 0);
    free(b.tmp);
    for (int dep = t->h; dep >= 0; dep--)
        for (int64_t i = 0; i < ((int64_t)1 << dep); i++)
            node_box_live(f, t, &t->nodes[t->bfs2veb[((int64_t)1 << dep) - 1 + i]]);
    return t;
}

static void free_tree(otree *t)
{
    if (!t) return;
    free(t->nodes); free(t->bfs2veb); free(t->ids); free(t->dead); free(t->bloom);
    free(t);
}

static onode *child(otree *t, const onode *nd, int right)
{
    return &t->nodes[t->bfs2veb[((int64_t)1 << (nd->depth + 1)) - 1 + 2 * nd->bfs + right]];
}

/* ------------------------------------------------------------------ */
/* Sec. V-A: bloom filter                                              */
/* ------------------------------------------------------------------ */
/* Reading G7: the paper gives neither hashes nor sizes.  This is a split-block
 * bloom filter keyed on the point id: 256-bit blocks of eight 32-bit words, one
 * block per key, one bit per word; blocks = smallest power of two >= ceil(size *
 * bits_per_key / 256).  Hash: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014),
 * h1 = SM(seed ^ id), h2 = SM(h1); block = h1 mod blocks, bit of word w =
 * bits [5w, 5w+5) of h2. */
static uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void bloom_positions(const oforest *f, int64_t blocks, int32_t id, int64_t *blk, uint32_t bit[8])
{
    uint64_t h1 = splitmix64(f->seed ^ (uint64_t)(uint32_t)id);
    uint64_t h2 = splitmix64(h1);
    *blk = (int64_t)(h1 & (uint64_t)(blocks - 1));
    for (int w = 0; w < 8; w++) bit[w] = (uint32_t)((h2 >> (5 * w)) & 31u);
}

static void bloom_build(const oforest *f, otree *t)
{
    int64_t need = (t->size * f->bpk + 255) / 256;
    int64_t blocks = 1;
    while (blocks < need) blocks *= 2;
    t->bloom_blocks = blocks;
    t->bloom = (uint32_t *)xcalloc((size_t)blocks * 8, sizeof(uint32_t));
    for (int64_t j = 0; j < t->size; j++) {
        if (t->dead[j]) continue;
        int64_t blk; uint32_t bit[8];
        bloom_positions(f, blocks, t->ids[j], &blk, bit);
        for (int w = 0; w < 8; w++) t->bloom[blk * 8 + w] |= 1u << bit[w];
    }
}

static int bloom_maybe(const oforest *f, const otree *t, int32_t id)
{
    int64_t blk; uint32_t bit[8];
    bloom_positions(f, t->bloom_blocks, id, &blk, bit);
    for (int w = 0; w < 8; w++)
        if (!(t->bloom[blk * 8 + w] & (1u << bit[w]))) return 0;
    return 1;
}

/* ------------------------------------------------------------------ */
/* Alg. 2: Erase_S                                                     */
/* ------------------------------------------------------------------ */
/* Deletion is by id (reading G7); the point's coordinates come from the id
 * table.  The collapse of Alg. 2 (an emptied subtree returns NULL, a node with
 * one empty child is replaced by the other) is kept as per-node live counts:
 * live == 0 is the NULL subtree, and queries skip it. */
static int64_t erase_rec(oforest *f, otree *t, onode *nd, int32_t *Q, int64_t nq)
{
    if (nq == 0) return nd->live;
    if (nd->is_leaf) {
        for (int64_t j = nd->lo; j < nd->hi; j++) {
            if (t->dead[j]) continue;
            for (int64_t e = 0; e < nq; e++)
                if (Q[e] == t->ids[j]) { t->dead[j] = 1; break; }
        }
        nd->live = 0;
        for (int64_t j = nd->lo; j < nd->hi; j++) nd->live += !t->dead[j];
        return nd->live;
    }
    /* partition Q around the node's split: composite key <= split goes left */
    int c = nd->depth % f->dim;
    int64_t nl = 0;
    for (int64_t e = 0; e < nq; e++) {
        if (okey(f, Q[e], c) <= nd->key) {
            int32_t tmp = Q[nl]; Q[nl] = Q[e]; Q[e] = tmp; nl++;
        }
    }
    int64_t a = erase_rec(f, t, child(t, nd, 0), Q, nl);
    int64_t z = erase_rec(f, t, child(t, nd, 1), Q + nl, nq - nl);
    nd->live = a + z;
    return nd->live;
}

/* ------------------------------------------------------------------ */
/* Alg. 3: Insert_L                                                    */
/* ------------------------------------------------------------------ */

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static void tree_live_ids(const otree *t, int32_t *out, int64_t *n)
{
    for (int64_t j = 0; j < t->size; j++)
        if (!t->dead[j]) out[(*n)++] = t->ids[j];
}

/* Insert the points with ids P[0..n) (their coordinates are in the id table).
 *
 * Reading G5 (buffer overflow, Sec. IV-B1): the pool is the buffer's ids in
 * ascending order followed by P; the last (b + n) mod X pool entries become the
 * new buffer and the first q*X feed the new trees, q = floor((b + n) / X).
 *
 * Reading G4 (which points go where when q sets several bits): every cleared
 * tree i (in F, not in F_new) is merged into the smallest new tree j > i (in
 * F_new, not in F); new tree j then takes cap_j - sum(cap_i of its cleared
 * trees) pool points, the new trees taking their pool chunks in increasing j. */
static void insert_ids(oforest *f, const int32_t *P, int64_t n)
{
    if (n == 0) return;
    int64_t X = f->X;
    int64_t t = f->nbuf + n;
    int32_t *pool = (int32_t *)xmalloc((size_t)t * sizeof(int32_t));
    memcpy(pool, f->buf, (size_t)f->nbuf * sizeof(int32_t));
    memcpy(pool + f->nbuf, P, (size_t)n * sizeof(int32_t));
    int64_t q = t / X, rem = t % X;

    uint64_t Fnew = f->F + (uint64_t)q;
    uint64_t newt = Fnew & ~f->F, cleared = f->F & ~Fnew;
    int64_t pos = 0;
    int prev_new = -1;
    otree *built[OR_MAXLEVEL] = { 0 };
    for (int j = 0; j < OR_MAXLEVEL; j++) {
        if (!((newt >> j) & 1)) continue;
        int64_t capj = X << j, from_cleared_cap = 0, from_cleared_live = 0;
        for (int i = prev_new + 1; i < j; i++)
            if ((cleared >> i) & 1) {
                from_cleared_cap += X << i;
                from_cleared_live += f->tree[i]->live;
            }
        int64_t shortfall = capj - from_cleared_cap;
        int64_t s = from_cleared_live + shortfall;
        int32_t *ids = (int32_t *)xmalloc((size_t)s * sizeof(int32_t));
        int64_t k = 0;
        for (int i = prev_new + 1; i < j; i++)
            if ((cleared >> i) & 1) tree_live_ids(f->tree[i], ids, &k);
        memcpy(ids + k, pool + pos, (size_t)shortfall * sizeof(int32_t));
        pos += shortfall;
        built[j] = build_tree(f, j, ids, s);
        free(ids);
        prev_new = j;
    }
    if (pos != q * X) abort();
    for (int i = 0; i < OR_MAXLEVEL; i++)
        if ((cleared >> i) & 1) { free_tree(f->tree[i]); f->tree[i] = NULL; }
    for (int j = 0; j < OR_MAXLEVEL; j++)
        if (built[j]) f->tree[j] = built[j];
    f->F = Fnew;
    /* new buffer: the last rem pool entries, kept in ascending id order */
    memcpy(f->buf, pool + (t - rem), (size_t)rem * sizeof(int32_t));
    f->nbuf = rem;
    qsort(f->buf, (size_t)rem, sizeof(int32_t), cmp_i32);
    free(pool);
}

/* ------------------------------------------------------------------ */
/* Alg. 4: Erase_L                                                     */
/* ------------------------------------------------------------------ */
/* Reading G6: after the whole batch, every static tree with live < cap/2
 * (cap = X*2^i, strict) is emptied; its live points R are reinserted by
 * Insert_L keeping their ids (R in ascending id order).  Ids that are not live
 * (never inserted, already erased, repeated in the batch) are ignored. */
static int64_t erase_ids(oforest *f, const int32_t *ids, int64_t n)
{
    int32_t *E = (int32_t *)xmalloc((size_t)(n ? n : 1) * sizeof(int32_t));
    int64_t ne = 0;
    for (int64_t e = 0; e < n; e++) {
        int32_t id = ids[e];
        if (id < 0 || id >= f->n_ids || !f->alive[id]) continue;
        f->alive[id] = 0;
        E[ne++] = id;
    }
    if (ne == 0) { free(E); return 0; }
    /* the buffer tree */
    int64_t nb = 0;
    for (int64_t j = 0; j < f->nbuf; j++)
        if (f->alive[f->buf[j]]) f->buf[nb++] = f->buf[j];
    f->nbuf = nb;
    /* line 2: every nonempty static tree, each batch filtered by its bloom */
    int32_t *Q = (int32_t *)xmalloc((size_t)ne * sizeof(int32_t));
    for (int i = 0; i < OR_MAXLEVEL; i++) {
        otree *t = f->tree[i];
        if (!t || t->live == 0) continue;
        if (!t->bloom) bloom_build(f, t);
        int64_t nq = 0;
        for (int64_t e = 0; e < ne; e++)
            if (bloom_maybe(f, t, E[e])) Q[nq++] = E[e];
        t->live = erase_rec(f, t, &t->nodes[0], Q, nq);
    }
    free(Q);
    /* line 3: gather the trees below half capacity */
    int64_t nr = 0;
    for (int i = 0; i < OR_MAXLEVEL; i++)
        if (f->tree[i]) nr += f->tree[i]->live;
    int32_t *R = (int32_t *)xmalloc((size_t)(nr ? nr : 1) * sizeof(int32_t));
    nr = 0;
    for (int i = 0; i < OR_MAXLEVEL; i++) {
        otree *t = f->tree[i];
        if (!t) continue;
        int64_t cap = (int64_t)f->X << i;
        if (2 * t->live < cap) {
            tree_live_ids(t, R, &nr);
            free_tree(t);
            f->tree[i] = NULL;
            f->F &= ~((uint64_t)1 << i);
        }
    }
    /* line 4: reinsert */
    qsort(R, (size_t)nr, sizeof(int32_t), cmp_i32);
    insert_ids(f, R, nr);
    free(R);
    free(E);
    return ne;
}

/* ------------------------------------------------------------------ */
/* kNN buffer (Sec. IV-A3) and kNN_S / kNN_L (Alg. 5)                  */
/* ------------------------------------------------------------------ */

typedef struct { int64_t d2; int32_t id; } cand;

static int cand_cmp(const void *a, const void *b)
{
    const cand *x = (const cand *)a, *y = (const cand *)b;
    if (x->d2 != y->d2) return (x->d2 > y->d2) - (x->d2 < y->d2);
    return (x->id > y->id) - (x->id < y->id);
}

/* 2k entries; appends, and when full keeps the k best (order (d2, id)). */
typedef struct { cand *a; int64_t n; int k; cand *tmp; } kbuf;

static void kb_add(kbuf *b, int64_t d2, int32_t id)
{
    b->a[b->n].d2 = d2;
    b->a[b->n].id = id;
    b->n++;
    if (b->n == 2 * (int64_t)b->k) {
        qsort(b->a, (size_t)b->n, sizeof(cand), cand_cmp);   /* selection by sorting */
        b->n = b->k;
    }
}

/* the k-th smallest squared distance held; only called when n >= k */
static int64_t kb_kth(kbuf *b)
{
    memcpy(b->tmp, b->a, (size_t)b->n * sizeof(cand));
    qsort(b->tmp, (size_t)b->n, sizeof(cand), cand_cmp);
    return b->tmp[b->k - 1].d2;
}

static int64_t box_mindist(const oforest *f, const int32_t *q, const int32_t *box)
{
    int64_t s = 0;
    for (int c = 0; c < f->dim; c++) {
        int64_t x = q[c], lo = box[c], hi = box[f->dim + c], g = 0;
        if (x < lo) g = lo - x; else if (x > hi) g = x - hi;
        s += g * g;
    }
    return s;
}

static int64_t box_maxdist(const oforest *f, const int32_t *q, const int32_t *box)
{
    int64_t s = 0;
    for (int c = 0; c < f->dim; c++) {
        int64_t x = q[c], a = x - box[c], z = box[f->dim + c] - x;
        if (a < 0) a = -a;
        if (z < 0) z = -z;
        int64_t g = a > z ? a : z;
        s += g * g;
    }
    return s;
}

typedef struct { int64_t nodes, points; } kstats;

static void add_all(const oforest *f, otree *t, const onode *nd, const int32_t *q, kbuf *b, kstats *st)
{
    st->nodes++;
    for (int64_t j = nd->lo; j < nd->hi; j++) {
        if (t->dead[j]) continue;
        st->points++;
        kb_add(b, sqdist(f, q, t->ids[j]), t->ids[j]);
    }
}

/* kNN_S: descend to the query's leaf, then while unwinding either fill the
 * buffer with the sibling (fewer than k held) or use the k-th distance:
 * sibling box within it -> add all its points, disjoint -> prune, else recurse.
 * Reading G8: "disjoint" is mindist^2 > kth (strict), "within" is
 * maxdist^2 <= kth; an empty (live == 0) subtree is the NULL of Alg. 2. */
static void knn_rec(const oforest *f, otree *t, const onode *nd, const int32_t *q, kbuf *b, kstats *st)
{
    if (nd->live == 0) return;
    st->nodes++;
    if (nd->is_leaf) {
        for (int64_t j = nd->lo; j < nd->hi; j++) {
            if (t->dead[j]) continue;
            st->points++;
            kb_add(b, sqdist(f, q, t->ids[j]), t->ids[j]);
        }
        return;
    }
    int c = nd->depth % f->dim;
    int64_t split_coord = nd->key >> 31;
    int go_right = (int64_t)q[c] > split_coord;
    const onode *near = child(t, nd, go_right), *far = child(t, nd, !go_right);
    knn_rec(f, t, near, q, b, st);
    if (far->live == 0) return;
    if (b->n < b->k) {
        add_all(f, t, far, q, b, st);
    } else {
        int64_t kth = kb_kth(b);
        if (box_maxdist(f, q, far->box) <= kth) add_all(f, t, far, q, b, st);
        else if (box_mindist(f, q, far->box) > kth) { /* pruned */ }
        else knn_rec(f, t, far, q, b, st);
    }
}

static void knn_one(oforest *f, const int32_t *q, int k, int32_t *out_ids, int64_t *out_d2, kstats *st)
{
    kbuf b;
    b.k = k;
    b.n = 0;
    b.a = (cand *)xmalloc((size_t)(2 * k) * sizeof(cand));
    b.tmp = (cand *)xmalloc((size_t)(2 * k) * sizeof(cand));
    /* Sec. V-B: the trees one after another, largest first, sharing one buffer */
    for (int i = OR_MAXLEVEL - 1; i >= 0; i--)
        if (f->tree[i]) knn_rec(f, f->tree[i], &f->tree[i]->nodes[0], q, &b, st);
    /* the buffer tree (Build_S): exact scan of its points */
    for (int64_t j = 0; j < f->nbuf; j++) kb_add(&b, sqdist(f, q, f->buf[j]), f->buf[j]);
    qsort(b.a, (size_t)b.n, sizeof(cand), cand_cmp);
    for (int j = 0; j < k; j++) {
        if (j < b.n) { out_ids[j] = b.a[j].id; out_d2[j] = b.a[j].d2; }
        else { out_ids[j] = -1; out_d2[j] = OR_D2_NONE; }
    }
    free(b.a);
    free(b.tmp);
}

/* ------------------------------------------------------------------ */
/* exported API (ctypes)                                               */
/* ------------------------------------------------------------------ */

void *orc_forest_new(int dim, int leaf_size, int buffer_size, int bloom_bits_per_key, uint64_t seed)
{
    if (dim < 1 || dim > OR_MAXDIM || leaf_size < 1 || buffer_size < 1 || bloom_bits_per_key < 1)
        return NULL;
    oforest *f = (oforest *)xcalloc(1, sizeof(oforest));
    f->dim = dim;
    f->L = leaf_size;
    f->X = buffer_size;
    f->bpk = bloom_bits_per_key;
    f->seed = seed;
    f->cap_ids = 1024;
    f->coord = (int32_t *)xmalloc((size_t)f->cap_ids * dim * sizeof(int32_t));
    f->alive = (unsigned char *)xcalloc((size_t)f->cap_ids, 1);
    f->buf = (int32_t *)xmalloc((size_t)buffer_size * sizeof(int32_t));
    return f;
}

/* Splitting rule of the trees built from now on: 0 object median, 1 spatial
 * median (Sec. V-C).  Returns 0, or -1 for an unknown rule. */
int orc_forest_set_split(void *h, int split)
{
    if (split != 0 && split != 1) return -1;
    ((oforest *)h)->split = split;
    return 0;
}

void orc_forest_free(void *h)
{
    oforest *f = (oforest *)h;
    if (!f) return;
    for (int i = 0; i < OR_MAXLEVEL; i++) free_tree(f->tree[i]);
    free(f->coord); free(f->alive); free(f->buf);
    free(f);
}

/* Insert n points [n][dim]; ids n_ids .. n_ids+n-1 in input order.
 * Returns the first id, or -1 if a coordinate is outside [0, 2^20). */
int64_t orc_insert(void *h, const int32_t *pts, int64_t n)
{
    oforest *f = (oforest *)h;
    for (int64_t i = 0; i < n * f->dim; i++)
        if (pts[i] < 0 || pts[i] >= (1 << 20)) return -1;
    if (f->n_ids + n > INT32_MAX) return -1;
    while (f->n_ids + n > f->cap_ids) {
        int64_t nc = 2 * f->cap_ids;
        f->coord = (int32_t *)realloc(f->coord, (size_t)nc * f->dim * sizeof(int32_t));
        f->alive = (unsigned char *)realloc(f->alive, (size_t)nc);
        if (!f->coord || !f->alive) abort();
        memset(f->alive + f->cap_ids, 0, (size_t)(nc - f->cap_ids));
        f->cap_ids = nc;
    }
    int64_t first = f->n_ids;
    memcpy(f->coord + first * f->dim, pts, (size_t)(n * f->dim) * sizeof(int32_t));
    int32_t *P = (int32_t *)xmalloc((size_t)(n ? n : 1) * sizeof(int32_t));
    for (int64_t i = 0; i < n; i++) { P[i] = (int32_t)(first + i); f->alive[first + i] = 1; }
    f->n_ids += n;
    insert_ids(f, P, n);
    free(P);
    return first;
}

int64_t orc_erase(void *h, const int32_t *ids, int64_t n) { return erase_ids((oforest *)h, ids, n); }

/* k-NN for m queries; rows sorted by (d2, id), padded with id -1 / INT64_MAX.
 * stats (optional, 2 entries): nodes visited, live points examined. */
void orc_knn(void *h, const int32_t *q, int64_t m, int k, int32_t *out_ids, int64_t *out_d2, int64_t *stats)
{
    oforest *f = (oforest *)h;
    kstats st = { 0, 0 };
    for (int64_t i = 0; i < m; i++)
        knn_one(f, q + i * f->dim, k, out_ids + i * k, out_d2 + i * k, &st);
    if (stats) { stats[0] = st.nodes; stats[1] = st.points; }
}

int64_t orc_live_count(void *h)
{
    oforest *f = (oforest *)h;
    int64_t s = f->nbuf;
    for (int i = 0; i < OR_MAXLEVEL; i++) if (f->tree[i]) s += f->tree[i]->live;
    return s;
}

uint64_t orc_tree_mask(void *h) { return ((oforest *)h)->F; }

int64_t orc_buffer(void *h, int32_t *out, int64_t cap)
{
    oforest *f = (oforest *)h;
    for (int64_t j = 0; j < f->nbuf && j < cap; j++) out[j] = f->buf[j];
    return f->nbuf;
}

/* info[0..5] = size, live, h, nnodes, bloom_blocks (0 = not built), level.
 * Returns 0, or -1 if tree `level` is empty. */
int orc_tree_info(void *h, int level, int64_t *info)
{
    oforest *f = (oforest *)h;
    if (level < 0 || level >= OR_MAXLEVEL || !f->tree[level]) return -1;
    otree *t = f->tree[level];
    info[0] = t->size; info[1] = t->live; info[2] = t->h; info[3] = t->nnodes;
    info[4] = t->bloom ? t->bloom_blocks : 0; info[5] = t->level;
    return 0;
}

/* Node arrays in vEB order.  child[2v], child[2v+1]: vEB slots of the
 * children, or (-1 - leaf, 0) for a leaf (leaf = its index at depth h).
 * Any output pointer may be NULL. */
int orc_tree_nodes(void *h, int level, int64_t *key, int32_t *child2, int32_t *box,
                   int64_t *live, int32_t *depth, int64_t *bfs)
{
    oforest *f = (oforest *)h;
    if (level < 0 || level >= OR_MAXLEVEL || !f->tree[level]) return -1;
    otree *t = f->tree[level];
    int d = f->dim;
    for (int64_t v = 0; v < t->nnodes; v++) {
        const onode *nd = &t->nodes[v];
        if (key) key[v] = nd->is_leaf ? 0 : nd->key;
        if (child2) {
            if (nd->is_leaf) { child2[2 * v] = (int32_t)(-1 - nd->bfs); child2[2 * v + 1] = 0; }
            else {
                child2[2 * v] = (int32_t)t->bfs2veb[((int64_t)1 << (nd->depth + 1)) - 1 + 2 * nd->bfs];
                child2[2 * v + 1] = (int32_t)t->bfs2veb[((int64_t)1 << (nd->depth + 1)) - 1 + 2 * nd->bfs + 1];
            }
        }
        if (box) for (int c = 0; c < 2 * d; c++) box[v * 2 * d + c] = nd->box[c];
        if (live) live[v] = nd->live;
        if (depth) depth[v] = nd->depth;
        if (bfs) bfs[v] = nd->bfs;
    }
    return 0;
}

/* Leaves: leaf_off[0..2^h] (point ranges by leaf index), ids and erased flags
 * of the points in leaf order. */
int orc_tree_leaves(void *h, int level, int64_t *leaf_off, int32_t *ids, unsigned char *dead)
{
    oforest *f = (oforest *)h;
    if (level < 0 || level >= OR_MAXLEVEL || !f->tree[level]) return -1;
    otree *t = f->tree[level];
    int64_t nl = (int64_t)1 << t->h;
    for (int64_t i = 0; i < nl; i++) leaf_off[i] = t->nodes[t->bfs2veb[nl - 1 + i]].lo;
    leaf_off[nl] = t->size;
    if (ids) memcpy(ids, t->ids, (size_t)t->size * sizeof(int32_t));
    if (dead) memcpy(dead, t->dead, (size_t)t->size);
    return 0;
}

int orc_tree_bloom(void *h, int level, uint32_t *words)
{
    oforest *f = (oforest *)h;
    if (level < 0 || level >= OR_MAXLEVEL || !f->tree[level] || !f->tree[level]->bloom) return -1;
    otree *t = f->tree[level];
    memcpy(words, t->bloom, (size_t)t->bloom_blocks * 8 * sizeof(uint32_t));
    return 0;
}

/* Membership answer of tree `level`'s bloom filter for one id (1 = maybe). */
int orc_bloom_maybe(void *h, int level, int32_t id)
{
    oforest *f = (oforest *)h;
    if (level < 0 || level >= OR_MAXLEVEL || !f->tree[level] || !f->tree[level]->bloom) return -1;
    return bloom_maybe(f, f->tree[level], id);
}

uint64_t orc_splitmix64(uint64_t x) { return splitmix64(x); }

/* Exact k-NN by definition: for every query the k smallest (d2, id) pairs over
 * the n given points, sorted, padded with id -1 / INT64_MAX. */
void orc_bruteforce_knn(int dim, const int32_t *pts, const int32_t *ids, int64_t n,
                        const int32_t *q, int64_t m, int k, int32_t *out_ids, int64_t *out_d2)
{
    cand *best = (cand *)xmalloc((size_t)k * sizeof(cand));
    for (int64_t i = 0; i < m; i++) {
        int64_t nb = 0;
        for (int64_t p = 0; p < n; p++) {
            int64_t s = 0;
            for (int c = 0; c < dim; c++) {
                int64_t diff = (int64_t)q[i * dim + c] - (int64_t)pts[p * dim + c];
                s += diff * diff;
            }
            cand x = { s, ids[p] };
            if (nb == k && cand_cmp(&x, &best[k - 1]) >= 0) continue;
            int64_t j = nb < k ? nb++ : k - 1;   /* insertion into the sorted best list */
            while (j > 0 && cand_cmp(&x, &best[j - 1]) < 0) { best[j] = best[j - 1]; j--; }
            best[j] = x;
        }
        for (int j = 0; j < k; j++) {
            out_ids[i * k + j] = j < nb ? best[j].id : -1;
            out_d2[i * k + j] = j < nb ? best[j].d2 : OR_D2_NONE;
        }
    }
    free(best);
}
