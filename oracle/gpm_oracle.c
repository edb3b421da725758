/*
 * gpm_oracle.c -- CPU ORACLE: TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, single-threaded restatement of what the paper's enumeration
 * computes, used to check the CUDA path.  Only the tests, the smoke check and
 * the benchmark's CPU-baseline leg may load it; the library never does, and
 * this file shares no code, header or table with the CUDA sources.
 *
 * What it implements.  The first routes below follow the paper's steps in
 * the paper's order; the later ones are faster restatements of the same
 * definitions, each pinned against the first ones and against closed forms
 * (tests/test_oracle_pins.py), and used only where the paper-order routes
 * cannot finish a full-size stored value:
 *
 *  - Eq. 1 (enumeration function E(G,tr,k)): a traversal tr grows by one
 *    vertex from its extensions while |tr| < k and is handed to the output
 *    function A when |tr| = k.
 *  - Algorithm 4, clique counting: extend from tr[0] only (range [0,1)),
 *    filter "lower" (keep extensions ordered after the last vertex of tr),
 *    compact, filter "is_clique" (keep extensions adjacent to every vertex of
 *    tr), and at |tr| = k-1 add the number of valid extensions
 *    (aggregate_counter, Section 4.3.4).
 *  - Algorithm 4, motif counting: extend from every vertex of tr (range
 *    [0,|tr|)), which yields the neighbourhood N(tr) of Definition 1; filter
 *    "canonical" with the incremental canonical-candidate test of Arabesque
 *    that the paper cites (Section 4.4); at |tr| = k-1 hand every tr+e to
 *    aggregate_pattern, which maps the induced k-vertex graph to its
 *    canonical representative (Section 4.3.4).
 *  - The canonical representative of a k-vertex graph is defined here as the
 *    smallest "full code" over all k! relabelings (the plain definition of
 *    the isomorphism class of Definition 3).  Full code: bit i(i-1)/2 + j is
 *    set iff vertices j < i are adjacent.
 *  - Brute force over all k-subsets for tiny graphs (n <= 40), classifying
 *    every induced subgraph, disconnected ones included.
 *  - Instrumentation of the clique search tree (nodes per clique size and
 *    the bytes a sorted-list merge would move, B_alg), on the (degree, id)
 *    orientation with sorted-list merges.
 *  - Motif counts by Wernicke's ESU enumeration (exclusive extension, every
 *    connected k-set once from its smallest vertex), classified by the same
 *    canonical code.
 *  - Clique counts of every size on bitsets over each root's
 *    out-neighbourhood (the same orientation; candidates as bitsets instead
 *    of sorted lists).
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *  - filter polarity: Algorithm 3 writes "if P then invalidate" while the
 *    text of Section 4.3.2 says extensions that do NOT satisfy P are
 *    invalidated; the text is followed (keep iff P holds).
 *  - aggregate_counter counts the valid (non-invalidated) extensions.
 *  - "lower" keeps extensions ordered after the last traversal vertex; the
 *    order is vertex id (ORC_ORDER_ID) or, optionally, (degree, id)
 *    (ORC_ORDER_DEGREE) so that per-root counts can be compared with a
 *    degree-ordered enumerator; totals do not depend on the order.
 *  - clique k = 1 counts vertices; motif counting only counts connected
 *    traversals (Section 4.3.4 handles only connected traversals).
 *
 * Counts are accumulated in unsigned __int128 and returned as (lo, hi)
 * 64-bit halves, so a caller can tell a true count >= 2^64 from a wrapped one.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

#define ORC_MAXK 16
#define ORC_ORDER_ID 0
#define ORC_ORDER_DEGREE 1

/* ------------------------------------------------------------ graph access */

typedef struct {
    int32_t n;
    const int32_t *indptr;
    const int32_t *indices;
} graph_t;

static int32_t deg(const graph_t *g, int32_t v) { return g->indptr[v + 1] - g->indptr[v]; }

/* (a, b) in E(G): binary search of b in the sorted list N(a). */
static int adjacent(const graph_t *g, int32_t a, int32_t b) {
    int64_t lo = g->indptr[a], hi = (int64_t)g->indptr[a + 1] - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        int32_t x = g->indices[mid];
        if (x == b) return 1;
        if (x < b) lo = mid + 1; else hi = mid - 1;
    }
    return 0;
}

/* ------------------------------------------------ canonical representative */

static int C2(int k) { return k * (k - 1) / 2; }
static int pair_bit(int j, int i) { /* j < i */ return i * (i - 1) / 2 + j; }

typedef struct {
    int k;
    int nperm;
    uint8_t *bitmap;   /* nperm x C(k,2): image bit index of each bit under each relabeling */
    /* memo: open addressing, full code -> canonical code */
    uint64_t *keys;
    uint64_t *vals;
    uint64_t cap;
    uint64_t used;
} canon_t;

static int next_perm(int *a, int k) {
    int i = k - 2;
    while (i >= 0 && a[i] > a[i + 1]) i--;
    if (i < 0) return 0;
    int j = k - 1;
    while (a[j] < a[i]) j--;
    int t = a[i]; a[i] = a[j]; a[j] = t;
    for (int l = i + 1, r = k - 1; l < r; l++, r--) { t = a[l]; a[l] = a[r]; a[r] = t; }
    return 1;
}

static int canon_init(canon_t *c, int k) {
    memset(c, 0, sizeof(*c));
    c->k = k;
    int nperm = 1;
    for (int i = 2; i <= k; i++) nperm *= i;
    c->nperm = nperm;
    int nb = C2(k);
    c->bitmap = (uint8_t *)malloc((size_t)nperm * (nb ? nb : 1));
    if (!c->bitmap) return -1;
    int p[ORC_MAXK];
    for (int i = 0; i < k; i++) p[i] = i;
    for (int t = 0; t < nperm; t++) {
        for (int i = 1; i < k; i++)
            for (int j = 0; j < i; j++) {
                int a = p[j], b = p[i];
                int lo = a < b ? a : b, hi = a < b ? b : a;
                c->bitmap[(size_t)t * nb + pair_bit(j, i)] = (uint8_t)pair_bit(lo, hi);
            }
        next_perm(p, k);
    }
    c->cap = 1u << 16;
    c->keys = (uint64_t *)malloc(c->cap * sizeof(uint64_t));
    c->vals = (uint64_t *)malloc(c->cap * sizeof(uint64_t));
    if (!c->keys || !c->vals) return -1;
    memset(c->keys, 0xff, c->cap * sizeof(uint64_t));
    return 0;
}

static void canon_free(canon_t *c) {
    free(c->bitmap); free(c->keys); free(c->vals);
    memset(c, 0, sizeof(*c));
}

static uint64_t hash64(uint64_t x) {
    x ^= x >> 33; x *= 0xff51afd7ed558ccdULL; x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ULL; x ^= x >> 33;
    return x;
}

/* Smallest full code over all k! relabelings: the definition, no pruning. */
static uint64_t canon_compute(const canon_t *c, uint64_t code) {
    int nb = C2(c->k);
    uint64_t best = ~0ULL;
    for (int t = 0; t < c->nperm; t++) {
        const uint8_t *img = c->bitmap + (size_t)t * nb;
        uint64_t r = 0;
        for (int b = 0; b < nb; b++)
            if ((code >> b) & 1) r |= 1ULL << img[b];
        if (r < best) best = r;
    }
    return best;
}

static int canon_grow(canon_t *c) {
    uint64_t ncap = c->cap * 2;
    uint64_t *nk = (uint64_t *)malloc(ncap * sizeof(uint64_t));
    uint64_t *nv = (uint64_t *)malloc(ncap * sizeof(uint64_t));
    if (!nk || !nv) { free(nk); free(nv); return -1; }
    memset(nk, 0xff, ncap * sizeof(uint64_t));
    for (uint64_t i = 0; i < c->cap; i++) {
        if (c->keys[i] == ~0ULL) continue;
        uint64_t h = hash64(c->keys[i]) & (ncap - 1);
        while (nk[h] != ~0ULL) h = (h + 1) & (ncap - 1);
        nk[h] = c->keys[i]; nv[h] = c->vals[i];
    }
    free(c->keys); free(c->vals);
    c->keys = nk; c->vals = nv; c->cap = ncap;
    return 0;
}

static uint64_t canon_get(canon_t *c, uint64_t code) {
    uint64_t h = hash64(code) & (c->cap - 1);
    while (c->keys[h] != ~0ULL) {
        if (c->keys[h] == code) return c->vals[h];
        h = (h + 1) & (c->cap - 1);
    }
    uint64_t v = canon_compute(c, code);
    if ((c->used + 1) * 2 > c->cap) {
        if (canon_grow(c) != 0) return v;
        h = hash64(code) & (c->cap - 1);
        while (c->keys[h] != ~0ULL) h = (h + 1) & (c->cap - 1);
    }
    c->keys[h] = code; c->vals[h] = v; c->used++;
    return v;
}

/* connectivity of a k-vertex graph given by its full code */
static int code_connected(int k, uint64_t code) {
    if (k <= 1) return 1;
    uint32_t seen = 1, frontier = 1;
    while (frontier) {
        uint32_t nxt = 0;
        for (int a = 0; a < k; a++) {
            if (!((frontier >> a) & 1)) continue;
            for (int b = 0; b < k; b++) {
                if (a == b) continue;
                int lo = a < b ? a : b, hi = a < b ? b : a;
                if ((code >> pair_bit(lo, hi)) & 1) nxt |= 1u << b;
            }
        }
        frontier = nxt & ~seen;
        seen |= nxt;
    }
    return seen == ((1u << k) - 1);
}

/* ------------------------------------------------- pattern-count histogram */

typedef struct {
    uint64_t *keys;
    u128 *vals;
    uint64_t cap, used;
} hist_t;

static int hist_init(hist_t *h) {
    h->cap = 1024; h->used = 0;
    h->keys = (uint64_t *)malloc(h->cap * sizeof(uint64_t));
    h->vals = (u128 *)calloc(h->cap, sizeof(u128));
    if (!h->keys || !h->vals) return -1;
    memset(h->keys, 0xff, h->cap * sizeof(uint64_t));
    return 0;
}
static void hist_free(hist_t *h) { free(h->keys); free(h->vals); }

static int hist_add(hist_t *h, uint64_t key, u128 inc) {
    uint64_t i = hash64(key) & (h->cap - 1);
    while (h->keys[i] != ~0ULL && h->keys[i] != key) i = (i + 1) & (h->cap - 1);
    if (h->keys[i] == key) { h->vals[i] += inc; return 0; }
    if ((h->used + 1) * 2 > h->cap) {
        uint64_t ncap = h->cap * 2;
        uint64_t *nk = (uint64_t *)malloc(ncap * sizeof(uint64_t));
        u128 *nv = (u128 *)calloc(ncap, sizeof(u128));
        if (!nk || !nv) { free(nk); free(nv); return -1; }
        memset(nk, 0xff, ncap * sizeof(uint64_t));
        for (uint64_t j = 0; j < h->cap; j++) {
            if (h->keys[j] == ~0ULL) continue;
            uint64_t p = hash64(h->keys[j]) & (ncap - 1);
            while (nk[p] != ~0ULL) p = (p + 1) & (ncap - 1);
            nk[p] = h->keys[j]; nv[p] = h->vals[j];
        }
        free(h->keys); free(h->vals);
        h->keys = nk; h->vals = nv; h->cap = ncap;
        i = hash64(key) & (h->cap - 1);
        while (h->keys[i] != ~0ULL) i = (i + 1) & (h->cap - 1);
    }
    h->keys[i] = key; h->vals[i] = inc; h->used++;
    return 0;
}

/* write the histogram sorted by key into (codes, lo, hi); returns entries */
static int64_t hist_export(const hist_t *h, int64_t cap, uint64_t *codes, uint64_t *lo, uint64_t *hi) {
    int64_t m = 0;
    for (uint64_t i = 0; i < h->cap; i++) {
        if (h->keys[i] == ~0ULL) continue;
        if (m < cap) {
            /* insertion into the sorted prefix */
            int64_t p = m;
            while (p > 0 && codes[p - 1] > h->keys[i]) {
                codes[p] = codes[p - 1]; lo[p] = lo[p - 1]; hi[p] = hi[p - 1]; p--;
            }
            codes[p] = h->keys[i];
            lo[p] = (uint64_t)h->vals[i];
            hi[p] = (uint64_t)(h->vals[i] >> 64);
        }
        m++;
    }
    return m;
}

/* ------------------------------------------------------ clique counting */

typedef struct {
    const graph_t *g;
    int k;
    int order;
    int32_t tr[ORC_MAXK];
    int32_t *ext[ORC_MAXK];    /* TE[i].ext: extension array of depth i */
    u128 count;
} clique_ctx;

static int before(const clique_ctx *c, int32_t a, int32_t b) {
    /* a ordered before b under the "lower" order */
    if (c->order == ORC_ORDER_DEGREE) {
        int32_t da = deg(c->g, a), db = deg(c->g, b);
        if (da != db) return da < db;
    }
    return a < b;
}

/* One level of Algorithm 4 (left) with |tr| = len. */
static void clique_level(clique_ctx *c, int len) {
    const graph_t *g = c->g;
    int32_t *ext = c->ext[len];
    int32_t first = c->tr[0];
    int64_t ne = 0;
    /* extend(TE, 0, 1): adjacency of tr[0], minus vertices already in tr */
    for (int32_t p = g->indptr[first]; p < g->indptr[first + 1]; p++) {
        int32_t e = g->indices[p];
        int in_tr = 0;
        for (int i = 0; i < len; i++) in_tr |= (c->tr[i] == e);
        ext[ne++] = in_tr ? -1 : e;
    }
    /* filter(lower, [u]), u = last vertex of tr: keep extensions after u */
    int32_t u = c->tr[len - 1];
    for (int64_t i = 0; i < ne; i++)
        if (ext[i] >= 0 && !before(c, u, ext[i])) ext[i] = -1;
    /* compact */
    int64_t w = 0;
    for (int64_t i = 0; i < ne; i++) if (ext[i] >= 0) ext[w++] = ext[i];
    ne = w;
    /* filter(is_clique): keep extensions adjacent to every vertex of tr */
    for (int64_t i = 0; i < ne; i++) {
        for (int j = 0; j < len && ext[i] >= 0; j++)
            if (!adjacent(g, c->tr[j], ext[i])) ext[i] = -1;
    }
    if (len == c->k - 1) {
        /* aggregate_counter: number of valid extensions */
        for (int64_t i = 0; i < ne; i++) c->count += (ext[i] >= 0);
        return;
    }
    /* move: push each valid extension in turn */
    for (int64_t i = 0; i < ne; i++) {
        if (ext[i] < 0) continue;
        c->tr[len] = ext[i];
        clique_level(c, len + 1);
    }
}

/*
 * Number of k-cliques whose first vertex (under the "lower" order) is a given
 * root, summed over the roots listed (all vertices when roots == NULL).
 * total[0..1] = (lo, hi) of the 128-bit sum; per_root (nullable) receives
 * each root's count, saturated at 2^64-1.  Returns 0, or -1 on bad input.
 */
int orc_clique_count(int32_t n, const int32_t *indptr, const int32_t *indices, int k, int order,
                     const int32_t *roots, int64_t n_roots, uint64_t *total, uint64_t *per_root) {
    if (n < 0 || k < 1 || k > ORC_MAXK || !total) return -1;
    graph_t g = {n, indptr, indices};
    clique_ctx c;
    memset(&c, 0, sizeof(c));
    c.g = &g; c.k = k; c.order = order;
    int32_t maxd = 0;
    for (int32_t v = 0; v < n; v++) if (deg(&g, v) > maxd) maxd = deg(&g, v);
    for (int i = 0; i < k; i++) {
        c.ext[i] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(maxd + 1));
        if (!c.ext[i]) { for (int j = 0; j < i; j++) free(c.ext[j]); return -1; }
    }
    int64_t nr = roots ? n_roots : n;
    u128 sum = 0;
    for (int64_t r = 0; r < nr; r++) {
        int32_t v = roots ? roots[r] : (int32_t)r;
        if (v < 0 || v >= n) { sum = 0; nr = -1; break; }
        c.count = 0;
        c.tr[0] = v;                       /* initial traversal [v] from the global queue */
        if (k == 1) c.count = 1;           /* |tr| = k: A(tr) */
        else clique_level(&c, 1);
        sum += c.count;
        if (per_root) per_root[r] = (c.count >> 64) ? ~0ULL : (uint64_t)c.count;
    }
    for (int i = 0; i < k; i++) free(c.ext[i]);
    if (nr < 0) return -1;
    total[0] = (uint64_t)sum;
    total[1] = (uint64_t)(sum >> 64);
    return 0;
}

/* ------------------------------------ clique search-tree instrumentation */

/*
 * The search tree of the degree-oriented clique enumeration, measured: a node
 * is a clique S whose candidates C(S) are the common out-neighbours of S
 * (orientation: u -> v iff (d(u), u) < (d(v), v)).  Expanding a child v of S
 * intersects two sorted lists, C(S) and N+(v); as a sorted-list merge reads
 * both, that step moves 4 (|C(S)| + d+(v)) bytes.  B_alg is that sum over
 * every child of every node of size 1 .. k-2 (the children of (k-2)-cliques
 * give the (k-1)-cliques whose candidate counts are the k-cliques: the
 * counted last level).  nodes[s] counts the s-cliques reached, s = 1 .. k.
 * The paper gauges the extension step by the global load transactions it
 * issues (its profiling table); B_alg is the analogous byte count of a
 * sorted-list enumerator, the yardstick the GPU path's memory traffic is
 * compared with.
 */
typedef struct {
    const graph_t *g;
    int k;
    const int32_t *off;       /* oriented out-lists, id order */
    const int32_t *out;
    int32_t *cand[ORC_MAXK + 1];
    u128 nodes[ORC_MAXK + 1];
    u128 bytes;
} instr_ctx;

static void instr_node(instr_ctx *c, int s, const int32_t *C, int64_t nc) {
    if (s == c->k - 1) {                 /* children are the k-cliques: counted, not expanded */
        c->nodes[c->k] += (u128)nc;
        return;
    }
    int32_t *next = c->cand[s + 1];
    for (int64_t i = 0; i < nc; i++) {
        int32_t v = C[i];
        const int32_t *nv = c->out + c->off[v];
        int64_t dv = c->off[v + 1] - c->off[v];
        c->bytes += (u128)4 * (u128)(nc + dv);
        int64_t a = 0, b = 0, m = 0;    /* merge of two id-sorted lists */
        while (a < nc && b < dv) {
            if (C[a] < nv[b]) a++;
            else if (C[a] > nv[b]) b++;
            else { next[m++] = C[a]; a++; b++; }
        }
        c->nodes[s + 1] += 1;
        instr_node(c, s + 1, next, m);
    }
}

/*
 * nodes_out[2*s], nodes_out[2*s+1] = (lo, hi) of the number of s-cliques
 * rooted at the listed roots (all vertices when roots == NULL; a clique's root
 * is its first vertex in the orientation), s = 1 .. k; bytes_out[0..1] = (lo,
 * hi) of B_alg.  Returns 0, -1 on bad input, -2 on allocation failure.
 */
int orc_clique_instrument(int32_t n, const int32_t *indptr, const int32_t *indices, int k,
                          const int32_t *roots, int64_t n_roots, uint64_t *nodes_out, uint64_t *bytes_out) {
    if (n < 0 || k < 1 || k > ORC_MAXK || !nodes_out || !bytes_out) return -1;
    graph_t g = {n, indptr, indices};
    int32_t *off = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t *out = (int32_t *)malloc(sizeof(int32_t) * ((size_t)(n ? indptr[n] : 0) + 1));
    if (!off || !out) { free(off); free(out); return -2; }
    int32_t maxd = 0;
    off[0] = 0;
    for (int32_t v = 0; v < n; v++) {
        int32_t dv = deg(&g, v), m = 0;
        for (int32_t p = indptr[v]; p < indptr[v + 1]; p++) {
            int32_t x = indices[p], dx = deg(&g, x);
            if (dv < dx || (dv == dx && v < x)) out[off[v] + m++] = x;
        }
        off[v + 1] = off[v] + m;
        if (m > maxd) maxd = m;
    }
    instr_ctx c;
    memset(&c, 0, sizeof(c));
    c.g = &g; c.k = k; c.off = off; c.out = out;
    int ok = 1;
    for (int i = 0; i <= k; i++) {
        c.cand[i] = (int32_t *)malloc(sizeof(int32_t) * ((size_t)maxd + 1));
        if (!c.cand[i]) ok = 0;
    }
    int64_t nr = roots ? n_roots : n;
    for (int64_t r = 0; ok && r < nr; r++) {
        int32_t v = roots ? roots[r] : (int32_t)r;
        if (v < 0 || v >= n) { ok = -1; break; }
        c.nodes[1] += 1;
        if (k >= 2) instr_node(&c, 1, out + off[v], off[v + 1] - off[v]);
    }
    for (int i = 0; i <= k; i++) free(c.cand[i]);
    free(off); free(out);
    if (ok != 1) return ok == 0 ? -2 : -1;
    for (int s = 0; s <= k; s++) {
        nodes_out[2 * s] = (uint64_t)c.nodes[s];
        nodes_out[2 * s + 1] = (uint64_t)(c.nodes[s] >> 64);
    }
    bytes_out[0] = (uint64_t)c.bytes;
    bytes_out[1] = (uint64_t)(c.bytes >> 64);
    return 0;
}

/* ------------------------------- clique counting on neighbourhood bitsets */

/*
 * A third clique route, for full-size stored values that the list routes
 * above cannot finish: the same degree-oriented search, with each node's
 * candidate set held as a bitset over the root's out-neighbourhood instead
 * of a sorted list.  For a root r with out-neighbours u_0 < .. < u_{d-1}
 * (ids ascending), bit j of row i is set iff j > i and u_i, u_j are
 * adjacent; the s-cliques whose lowest vertex (in the orientation) is r are
 * r plus an (s-1)-clique of G[N+(r)], each reached once along increasing
 * local indices.  A node of size s with candidates C has popc(C) children,
 * all (s+1)-cliques; the child through i has candidates C & row_i.  Nothing
 * here orders N+(r) by degree or trims rows: rows are full width.
 */
typedef struct {
    int k;
    int w;                    /* 64-bit words per row */
    uint64_t *rows;           /* d x w */
    uint64_t *cand;           /* (k + 1) x w scratch, one set per size */
    u128 nodes[ORC_MAXK + 1]; /* s-cliques of the current root */
} bits_ctx;

static int popc64(uint64_t x) { return __builtin_popcountll(x); }

static void bits_node(bits_ctx *c, int s, const uint64_t *C) {
    u128 nc = 0;
    for (int q = 0; q < c->w; q++) nc += (u128)popc64(C[q]);
    c->nodes[s + 1] += nc;                   /* every candidate is an (s+1)-clique */
    if (s + 1 >= c->k || nc == 0) return;
    uint64_t *next = c->cand + (size_t)(s + 1) * c->w;
    if (s + 2 == c->k) {
        /* the children are (k-1)-cliques: add their candidate counts (the
         * k-cliques) without descending */
        u128 leaves = 0;
        for (int q = 0; q < c->w; q++) {
            uint64_t word = C[q];
            while (word) {
                int i = 64 * q + __builtin_ctzll(word);
                word &= word - 1;
                const uint64_t *row = c->rows + (size_t)i * c->w;
                for (int z = 0; z < c->w; z++) leaves += (u128)popc64(C[z] & row[z]);
            }
        }
        c->nodes[s + 2] += leaves;
        return;
    }
    for (int q = 0; q < c->w; q++) {
        uint64_t word = C[q];
        while (word) {
            int i = 64 * q + __builtin_ctzll(word);
            word &= word - 1;
            const uint64_t *row = c->rows + (size_t)i * c->w;
            for (int z = 0; z < c->w; z++) next[z] = C[z] & row[z];
            bits_node(c, s + 1, next);
        }
    }
}

/*
 * counts_out[2*s], counts_out[2*s+1] = (lo, hi) of the number of s-cliques
 * (s = 1 .. k) whose root is listed (all vertices when roots == NULL; the
 * root of a clique is its first vertex in the (degree, id) orientation).
 * per_root (nullable): n_roots x (k + 1) uint64, entry [r][s] = root r's
 * s-cliques, saturated at 2^64-1.  Returns 0, -1 on bad input, -2 on
 * allocation failure.
 */
int orc_clique_count_bits(int32_t n, const int32_t *indptr, const int32_t *indices, int k,
                          const int32_t *roots, int64_t n_roots, uint64_t *counts_out, uint64_t *per_root) {
    if (n < 0 || k < 1 || k > ORC_MAXK || !counts_out) return -1;
    graph_t g = {n, indptr, indices};
    int32_t *off = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t *out = (int32_t *)malloc(sizeof(int32_t) * ((size_t)(n ? indptr[n] : 0) + 1));
    int32_t *local = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    if (!off || !out || !local) { free(off); free(out); free(local); return -2; }
    int32_t maxd = 0;
    off[0] = 0;
    for (int32_t v = 0; v < n; v++) {
        int32_t dv = deg(&g, v), m = 0;
        for (int32_t p = indptr[v]; p < indptr[v + 1]; p++) {
            int32_t x = indices[p], dx = deg(&g, x);
            if (dv < dx || (dv == dx && v < x)) out[off[v] + m++] = x;
        }
        off[v + 1] = off[v] + m;
        if (m > maxd) maxd = m;
        local[v] = -1;
    }
    bits_ctx c;
    memset(&c, 0, sizeof(c));
    c.k = k;
    int wmax = (maxd + 63) / 64;
    if (wmax < 1) wmax = 1;
    c.rows = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)maxd + 1) * wmax);
    c.cand = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)k + 2) * wmax);
    int ok = (c.rows && c.cand) ? 1 : 0;
    u128 total[ORC_MAXK + 1];
    memset(total, 0, sizeof(total));
    int64_t nr = roots ? n_roots : n;
    for (int64_t t = 0; ok == 1 && t < nr; t++) {
        int32_t r = roots ? roots[t] : (int32_t)t;
        if (r < 0 || r >= n) { ok = -1; break; }
        const int32_t *nb = out + off[r];
        int32_t d = off[r + 1] - off[r];
        int w = (d + 63) / 64;
        if (w < 1) w = 1;
        c.w = w;
        memset(c.nodes, 0, sizeof(c.nodes));
        c.nodes[1] = 1;
        for (int32_t i = 0; i < d; i++) local[nb[i]] = i;
        memset(c.rows, 0, sizeof(uint64_t) * (size_t)d * w);
        /* every edge inside N+(r) is an out-edge of exactly one endpoint */
        for (int32_t i = 0; i < d; i++) {
            int32_t u = nb[i];
            for (int32_t p = off[u]; p < off[u + 1]; p++) {
                int32_t j = local[out[p]];
                if (j < 0) continue;
                int32_t a = i < j ? i : j, b = i < j ? j : i;
                c.rows[(size_t)a * w + b / 64] |= 1ULL << (b % 64);
            }
        }
        if (k >= 2) {
            uint64_t *C = c.cand + (size_t)1 * w;
            for (int q = 0; q < w; q++) {
                int lo = 64 * q, hi = d - lo;
                C[q] = hi >= 64 ? ~0ULL : (hi <= 0 ? 0ULL : ((1ULL << hi) - 1));
            }
            bits_node(&c, 1, C);
        }
        for (int32_t i = 0; i < d; i++) local[nb[i]] = -1;
        for (int s = 1; s <= k; s++) {
            total[s] += c.nodes[s];
            if (per_root)
                per_root[(size_t)t * (k + 1) + s] = (c.nodes[s] >> 64) ? ~0ULL : (uint64_t)c.nodes[s];
        }
        if (per_root) per_root[(size_t)t * (k + 1)] = 0;
    }
    free(c.rows); free(c.cand); free(off); free(out); free(local);
    if (ok != 1) return ok == 0 ? -2 : -1;
    for (int s = 0; s <= k; s++) {
        counts_out[2 * s] = (uint64_t)total[s];
        counts_out[2 * s + 1] = (uint64_t)(total[s] >> 64);
    }
    return 0;
}

/* ------------------------------------------------------- motif counting */

typedef struct {
    const graph_t *g;
    int k;
    int32_t tr[ORC_MAXK];
    int32_t *ext[ORC_MAXK];
    int32_t *stamp;          /* per-vertex marker for duplicate removal in extend */
    int32_t stamp_id;
    canon_t canon;
    hist_t hist;
    u128 count;
    int err;
} motif_ctx;

/* Arabesque's incremental canonical-candidate test for appending e to tr:
 * e must come after tr[0], and after every vertex of tr that follows the
 * first traversal vertex adjacent to e. */
static int is_canonical(const motif_ctx *c, int len, int32_t e) {
    if (!(e > c->tr[0])) return 0;
    int f = -1;
    for (int i = 0; i < len; i++)
        if (adjacent(c->g, c->tr[i], e)) { f = i; break; }
    if (f < 0) return 0;
    for (int i = f + 1; i < len; i++)
        if (!(e > c->tr[i])) return 0;
    return 1;
}

/* aggregate_pattern on tr[0..k-1]: canonical representative of the induced graph */
static void aggregate_pattern(motif_ctx *c) {
    int k = c->k;
    uint64_t code = 0;
    for (int i = 1; i < k; i++)
        for (int j = 0; j < i; j++)
            if (adjacent(c->g, c->tr[j], c->tr[i])) code |= 1ULL << pair_bit(j, i);
    uint64_t rep = canon_get(&c->canon, code);
    if (hist_add(&c->hist, rep, 1) != 0) c->err = 1;
    c->count += 1;
}

static void motif_level(motif_ctx *c, int len) {
    const graph_t *g = c->g;
    int32_t *ext = c->ext[len];
    int64_t ne = 0;
    /* extend(TE, 0, len): N(tr), each vertex once, none of tr */
    c->stamp_id++;
    for (int i = 0; i < len; i++) c->stamp[c->tr[i]] = c->stamp_id;
    for (int i = 0; i < len; i++) {
        int32_t t = c->tr[i];
        for (int32_t p = g->indptr[t]; p < g->indptr[t + 1]; p++) {
            int32_t e = g->indices[p];
            if (c->stamp[e] == c->stamp_id) continue;
            c->stamp[e] = c->stamp_id;
            ext[ne++] = e;
        }
    }
    /* filter(canonical) */
    for (int64_t i = 0; i < ne; i++)
        if (!is_canonical(c, len, ext[i])) ext[i] = -1;
    /* compact */
    int64_t w = 0;
    for (int64_t i = 0; i < ne; i++) if (ext[i] >= 0) ext[w++] = ext[i];
    ne = w;
    for (int64_t i = 0; i < ne; i++) {
        c->tr[len] = ext[i];
        if (len == c->k - 1) aggregate_pattern(c);    /* |tr| = k */
        else motif_level(c, len + 1);                 /* move forward */
    }
}

/*
 * Induced connected k-vertex subgraphs whose smallest vertex id is one of the
 * listed roots (all when roots == NULL), aggregated by canonical code.
 * Writes up to cap entries (code ascending) into codes/lo/hi, the number of
 * distinct codes into *n_out, and per root (nullable) the number of sets,
 * saturated at 2^64-1.  total[0..1] = 128-bit number of sets.
 * Returns 0, -1 on bad input, -2 on allocation failure.
 */
int orc_motif_count(int32_t n, const int32_t *indptr, const int32_t *indices, int k,
                    const int32_t *roots, int64_t n_roots, int64_t cap,
                    uint64_t *codes, uint64_t *lo, uint64_t *hi, int64_t *n_out,
                    uint64_t *total, uint64_t *per_root) {
    if (n < 0 || k < 1 || k > 8 || !n_out || !total) return -1;
    graph_t g = {n, indptr, indices};
    motif_ctx c;
    memset(&c, 0, sizeof(c));
    c.g = &g; c.k = k;
    int64_t maxd = 0;
    for (int32_t v = 0; v < n; v++) if (deg(&g, v) > maxd) maxd = deg(&g, v);
    int rc = 0;
    if (canon_init(&c.canon, k) != 0 || hist_init(&c.hist) != 0) rc = -2;
    c.stamp = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    if (!c.stamp) rc = -2;
    for (int i = 0; i < k && rc == 0; i++) {
        c.ext[i] = (int32_t *)malloc(sizeof(int32_t) * (size_t)((int64_t)(i + 1) * maxd + 1));
        if (!c.ext[i]) rc = -2;
    }
    int64_t nr = roots ? n_roots : n;
    u128 sum = 0;
    for (int64_t r = 0; r < nr && rc == 0; r++) {
        int32_t v = roots ? roots[r] : (int32_t)r;
        if (v < 0 || v >= n) { rc = -1; break; }
        c.count = 0;
        c.tr[0] = v;
        if (k == 1) aggregate_pattern(&c);    /* |tr| = k */
        else motif_level(&c, 1);
        sum += c.count;
        if (per_root) per_root[r] = (c.count >> 64) ? ~0ULL : (uint64_t)c.count;
    }
    if (c.err) rc = -2;
    if (rc == 0) {
        *n_out = hist_export(&c.hist, cap, codes, lo, hi);
        total[0] = (uint64_t)sum;
        total[1] = (uint64_t)(sum >> 64);
    }
    for (int i = 0; i < k; i++) free(c.ext[i]);
    free(c.stamp);
    canon_free(&c.canon);
    hist_free(&c.hist);
    return rc;
}

/* ------------------------------------------------ motif counting by ESU */

/*
 * The same counts by Wernicke's ESU (exclusive-neighbourhood subgraph
 * enumeration), the reading of the canonicality filter that the GPU path
 * follows (Section 4.4 leaves the choice of filter to a standard method).
 * From root v the extension set is {u in N(v) : u > v};
 * moving w from the extension set into the subgraph adds the neighbours u of
 * w with u > v that are neither in the subgraph nor adjacent to it.  Every
 * connected k-set is reached exactly once, from its smallest vertex.  Each
 * set is classified as in aggregate_pattern (memoised canonical code of the
 * induced graph).  Written for the full-size checks the Arabesque route above
 * is too slow for; the two are compared with each other and with brute force.
 */
typedef struct {
    const graph_t *g;
    int k;
    int32_t root;
    int32_t sub[ORC_MAXK];
    uint64_t code[ORC_MAXK + 1];   /* full code of sub[0..len-1] */
    int32_t *ext[ORC_MAXK + 1];    /* extension set of depth len */
    uint16_t *adj;                 /* per vertex: bit j = adjacent to sub[j]; bit 15 = in sub */
    u128 *raw;                     /* k <= 7: count per full code, classified at the end */
    canon_t canon;
    hist_t hist;
    u128 count;
    int err;
} esu_ctx;

static void esu_classify(esu_ctx *c, uint64_t code) {
    c->count += 1;
    if (c->raw) { c->raw[code] += 1; return; }
    uint64_t rep = canon_get(&c->canon, code);
    if (hist_add(&c->hist, rep, 1) != 0) c->err = 1;
}

/* enter w as sub[pos] (on) or take it out (off): its own flag and its
 * neighbours' adjacency bit pos */
static void esu_mark(esu_ctx *c, int32_t w, int pos, int on) {
    const graph_t *g = c->g;
    const uint16_t bit = (uint16_t)(1u << pos);
    if (on) {
        c->adj[w] |= 0x8000;
        for (int32_t p = g->indptr[w]; p < g->indptr[w + 1]; p++) c->adj[g->indices[p]] |= bit;
    } else {
        c->adj[w] &= 0x7fff;
        for (int32_t p = g->indptr[w]; p < g->indptr[w + 1]; p++) c->adj[g->indices[p]] &= (uint16_t)~bit;
    }
}

/* subgraph sub[0..len-1]; extension set ext[len][0..n) */
static void esu_extend(esu_ctx *c, int len, int64_t n) {
    const graph_t *g = c->g;
    int32_t *ext = c->ext[len];
    while (n > 0) {
        int32_t w = ext[--n];
        /* w's edges to sub[0..len-1] are bits 0..len-1 of its adjacency mask */
        const uint64_t code = c->code[len] | ((uint64_t)(c->adj[w] & ((1u << len) - 1)) << pair_bit(0, len));
        if (len + 1 == c->k) { esu_classify(c, code); continue; }
        /* extension of sub + w: the rest of ext, then w's exclusive neighbours */
        int32_t *nx = c->ext[len + 1];
        int64_t m = 0;
        for (int64_t i = 0; i < n; i++) nx[m++] = ext[i];
        for (int32_t p = g->indptr[w]; p < g->indptr[w + 1]; p++) {
            int32_t u = g->indices[p];
            if (u > c->root && c->adj[u] == 0) nx[m++] = u;   /* not in sub, not adjacent to it */
        }
        c->sub[len] = w;
        c->code[len + 1] = code;
        esu_mark(c, w, len, 1);
        esu_extend(c, len + 1, m);
        esu_mark(c, w, len, 0);
    }
}

/* Same interface and results as orc_motif_count. */
int orc_motif_count_esu(int32_t n, const int32_t *indptr, const int32_t *indices, int k,
                        const int32_t *roots, int64_t n_roots, int64_t cap,
                        uint64_t *codes, uint64_t *lo, uint64_t *hi, int64_t *n_out,
                        uint64_t *total, uint64_t *per_root) {
    if (n < 0 || k < 1 || k > 8 || !n_out || !total) return -1;
    graph_t g = {n, indptr, indices};
    esu_ctx c;
    memset(&c, 0, sizeof(c));
    c.g = &g; c.k = k;
    int64_t maxd = 0;
    for (int32_t v = 0; v < n; v++) if (deg(&g, v) > maxd) maxd = deg(&g, v);
    int rc = 0;
    if (canon_init(&c.canon, k) != 0 || hist_init(&c.hist) != 0) rc = -2;
    c.adj = (uint16_t *)calloc((size_t)n + 1, sizeof(uint16_t));
    if (!c.adj) rc = -2;
    const uint64_t ncodes = k <= 7 ? (1ULL << C2(k)) : 0;
    if (ncodes) {
        c.raw = (u128 *)calloc((size_t)ncodes, sizeof(u128));
        if (!c.raw) rc = -2;
    }
    for (int i = 0; i <= k && rc == 0; i++) {
        c.ext[i] = (int32_t *)malloc(sizeof(int32_t) * (size_t)((int64_t)(i + 1) * maxd + 1));
        if (!c.ext[i]) rc = -2;
    }
    int64_t nr = roots ? n_roots : n;
    u128 sum = 0;
    for (int64_t r = 0; r < nr && rc == 0; r++) {
        int32_t v = roots ? roots[r] : (int32_t)r;
        if (v < 0 || v >= n) { rc = -1; break; }
        c.count = 0;
        c.root = v;
        c.sub[0] = v;
        c.code[1] = 0;
        if (k == 1) esu_classify(&c, 0);
        else {
            int64_t m = 0;
            for (int32_t p = indptr[v]; p < indptr[v + 1]; p++)
                if (indices[p] > v) c.ext[1][m++] = indices[p];
            esu_mark(&c, v, 0, 1);
            esu_extend(&c, 1, m);
            esu_mark(&c, v, 0, 0);
        }
        sum += c.count;
        if (per_root) per_root[r] = (c.count >> 64) ? ~0ULL : (uint64_t)c.count;
    }
    /* classify the full codes that occurred: one canonical lookup per code */
    for (uint64_t x = 0; rc == 0 && x < ncodes; x++)
        if (c.raw[x] && hist_add(&c.hist, canon_get(&c.canon, x), c.raw[x]) != 0) c.err = 1;
    if (c.err) rc = -2;
    if (rc == 0) {
        *n_out = hist_export(&c.hist, cap, codes, lo, hi);
        total[0] = (uint64_t)sum;
        total[1] = (uint64_t)(sum >> 64);
    }
    for (int i = 0; i <= k; i++) free(c.ext[i]);
    free(c.raw);
    free(c.adj);
    canon_free(&c.canon);
    hist_free(&c.hist);
    return rc;
}

/* --------------------------------------------------------- brute force */

/*
 * Every k-subset of V (n <= 40): the canonical code of each induced subgraph,
 * connected or not.  Writes up to cap entries (code ascending) into codes /
 * lo / hi / connected and the number of distinct codes into *n_out.
 */
int orc_brute_force(int32_t n, const int32_t *indptr, const int32_t *indices, int k, int64_t cap,
                    uint64_t *codes, uint64_t *lo, uint64_t *hi, uint8_t *connected, int64_t *n_out) {
    if (n < 0 || n > 40 || k < 1 || k > 8 || k > n || !n_out) return -1;
    graph_t g = {n, indptr, indices};
    canon_t cn;
    hist_t h;
    if (canon_init(&cn, k) != 0) return -2;
    if (hist_init(&h) != 0) { canon_free(&cn); return -2; }
    int s[ORC_MAXK];
    for (int i = 0; i < k; i++) s[i] = i;
    int rc = 0;
    for (;;) {
        uint64_t code = 0;
        for (int i = 1; i < k; i++)
            for (int j = 0; j < i; j++)
                if (adjacent(&g, s[j], s[i])) code |= 1ULL << pair_bit(j, i);
        if (hist_add(&h, canon_get(&cn, code), 1) != 0) { rc = -2; break; }
        int i = k - 1;
        while (i >= 0 && s[i] == n - k + i) i--;
        if (i < 0) break;
        s[i]++;
        for (int j = i + 1; j < k; j++) s[j] = s[j - 1] + 1;
    }
    if (rc == 0) {
        *n_out = hist_export(&h, cap, codes, lo, hi);
        if (connected)
            for (int64_t i = 0; i < *n_out && i < cap; i++) connected[i] = (uint8_t)code_connected(k, codes[i]);
    }
    canon_free(&cn);
    hist_free(&h);
    return rc;
}

/* ------------------------------------------------ canonical-code utilities */

/* canonical code (smallest full code over all relabelings) of one k-graph */
uint64_t orc_canon(int k, uint64_t code) {
    if (k < 1 || k > 8) return ~0ULL;
    canon_t c;
    if (canon_init(&c, k) != 0) return ~0ULL;
    uint64_t r = canon_compute(&c, code);
    canon_free(&c);
    return r;
}

/* canonical codes of many k-graphs at once (shares one relabeling table) */
int orc_canon_many(int k, const uint64_t *in, int64_t count, uint64_t *out) {
    if (k < 1 || k > 8) return -1;
    canon_t c;
    if (canon_init(&c, k) != 0) return -2;
    for (int64_t i = 0; i < count; i++) out[i] = canon_get(&c, in[i]);
    canon_free(&c);
    return 0;
}

int orc_code_connected(int k, uint64_t code) { return code_connected(k, code); }

/*
 * Distinct canonical codes over all 2^C(k,2) labelled k-graphs (k <= 6),
 * ascending; connected_only keeps the connected classes.
 */
int orc_classes(int k, int connected_only, int64_t cap, uint64_t *out, int64_t *n_out) {
    if (k < 1 || k > 6 || !n_out) return -1;
    canon_t c;
    hist_t h;
    if (canon_init(&c, k) != 0) return -2;
    if (hist_init(&h) != 0) { canon_free(&c); return -2; }
    uint64_t total = 1ULL << C2(k);
    for (uint64_t code = 0; code < total; code++) {
        if (connected_only && !code_connected(k, code)) continue;
        hist_add(&h, canon_get(&c, code), 1);
    }
    uint64_t *lo = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(cap > 0 ? cap : 1));
    uint64_t *hi = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(cap > 0 ? cap : 1));
    *n_out = hist_export(&h, cap, out, lo, hi);
    free(lo); free(hi);
    canon_free(&c);
    hist_free(&h);
    return 0;
}
