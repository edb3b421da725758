// clique_dev.cuh -- device code of one clique work unit (root-local bitmap
// DFS, aggregate_counter by popcount, optional work donation), shared by the
// single-graph kernel (clique.cu) and the batched kernel (batch.cu).
//
// The paper's clique loop (Algorithm 4) extends a traversal from tr[0]'s
// adjacency, keeps extensions after the last vertex ("lower") and adjacent to
// every traversal vertex ("is_clique"), and at |tr| = k-1 adds the number of
// valid extensions (aggregate_counter).  Here the search runs on the
// degree-ordered orientation, and the candidate set of a traversal -- its
// valid extensions after both filters -- is a bitmap over the root's
// out-neighbourhood N+(r):
//
//   * row i of a d x d bit matrix in shared memory holds N+(u_i) restricted
//     to N+(r) (u_i = i-th out-neighbour of r, d = |N+(r)|);
//   * the root's candidates are all d bits; choosing child i gives C & row_i
//     (both filters in one AND: row_i holds only vertices after u_i, the AND
//     keeps those adjacent to every traversal vertex);
//   * at a node of size k-2 the k-cliques below it number sum over i in C of
//     popc(C & row_i): aggregate_counter on every (k-1)-vertex child at once.
//
// Upper levels are walked one child at a time (the DFS step of Section 4.2);
// the last level is expanded lane-parallel over the compacted candidate list
// (the BFS step, one candidate per lane).
#pragma once

#include "common.cuh"

namespace gpm {


constexpr int CQ_LEVELS = GPM_CLIQUE_MAX_K + 1;
constexpr int CQ_MAX_OUTDEG = 1024;          // bitmap rows of at most 32 words

constexpr int CQ_PAIR_FLUSH = 128;            // run the pair batch once it holds this many
constexpr int CQ_CW = 5;                      // compacted tail: at most 32 * CQ_CW members
constexpr int CQ_COMPACT_MIN = 48;            // ... and (clique_compact = 1) at least this many
constexpr unsigned long long CQ_CHECK_NS = 4000;   // busy warps look for idle ones at most this often

struct CliqueUnit {
    int32_t root_pos;                   // index into the root list
    int32_t depth;                      // path length p: the node is a (p+1)-clique
    int32_t lo, hi;                     // its children (local indices) in [lo, hi); hi < 0: all
    uint16_t path[GPM_CLIQUE_MAX_K];    // local index chosen at sizes 1 .. p
};
static_assert(sizeof(CliqueUnit) % 4 == 0, "unit must be word-sized");



// words of the pair / compacted-matrix region: the pair batch, or (with a
// compacted tail on and rows of at least three words) up to 32 * CQ_CW
// members x CQ_CW words followed by a pair batch over them
__host__ __device__ inline int cq_pairs_words(int wmax, bool compact) {
    const int pairs = CQ_PAIR_FLUSH + 32 * wmax;
    const int cm = (compact && wmax >= 3) ? 32 * CQ_CW * CQ_CW + CQ_PAIR_FLUSH + 32 * CQ_CW : 0;
    return pairs > cm ? pairs : cm;
}

// Root-local bit rows, stored upper-triangular: row p (positions in
// orientation order) can only hold positions above p, so its words below
// p / 32 are zero and are not stored.  Rows of block b (positions 32b ..
// 32b + 31) keep w - b words; row(p)[z] is word z of row p for z >= p / 32.
__host__ __device__ inline int cq_tri_words(int d, int w) {
    const int b = d >> 5;
    return 32 * (b * w - b * (b - 1) / 2) + (d - 32 * b) * (w - b);
}

// row(p) = base + cq_tri_words(p, w) - p / 32, which simplifies to
// base + p (w - b) + b (16 b + 15) with b = p / 32.
__host__ __device__ inline int cq_tri_row(int p, int w) {
    const int b = p >> 5;
    return p * (w - b) + b * (16 * b + 15);
}

struct TriRows {                    // the root-local matrix
    const uint32_t* base;
    int w;
    __device__ __forceinline__ const uint32_t* row(int p) const { return base + cq_tri_row(p, w); }
};

struct RectRows {                   // a plain row-major matrix (the compacted one)
    const uint32_t* base;
    int ws;
    __device__ __forceinline__ const uint32_t* row(int p) const { return base + p * ws; }
};

// shared-memory layout of one warp, in 32-bit words
struct CqLayout {
    int wcnt, unit, cur, hi, cand, list, pairs, rows, total;
};

__host__ __device__ inline CqLayout cq_layout(int maxd, int wmax, bool compact) {
    CqLayout L;
    L.wcnt = 0;                                        // CQ_LEVELS x u64
    L.unit = L.wcnt + 2 * CQ_LEVELS;                   // CliqueUnit
    L.cur = L.unit + (int)(sizeof(CliqueUnit) / 4);
    L.hi = L.cur + CQ_LEVELS;
    L.cand = L.hi + CQ_LEVELS;                         // CQ_LEVELS x wmax candidate bitmaps
    L.list = L.cand + CQ_LEVELS * wmax;                // 32*wmax ints: N+(r), later the child list
    L.pairs = L.list + 32 * wmax;                      // pair batch of the three-level tail,
                                                       // or the compacted matrix of the two-level one
    L.rows = L.pairs + cq_pairs_words(wmax, compact);  // upper-triangular bit rows
    L.total = L.rows + cq_tri_words(maxd, wmax);
    L.total = (L.total + 3) & ~3;                      // keep every warp 16-byte aligned
    return L;
}

// bits [from, to) of 32-bit word q
__device__ __forceinline__ uint32_t range_mask(int q, int from, int to) {
    const int lo = max(from - 32 * q, 0);
    const int hi = min(to - 32 * q, 32);
    if (lo >= hi) return 0u;
    const uint32_t upto = hi >= 32 ? 0xffffffffu : ((1u << hi) - 1u);
    const uint32_t from_ = lo >= 32 ? 0u : ~((1u << lo) - 1u);
    return upto & from_;
}

// smallest set bit of C in [from, to), or -1 (warp-uniform result; w <= 32)
__device__ __forceinline__ int next_child(const uint32_t* C, int w, int from, int to, int lane) {
    const uint32_t x = lane < w ? (C[lane] & range_mask(lane, from, to)) : 0u;
    const unsigned b = __ballot_sync(GPM_FULL_MASK, x != 0);
    if (!b) return -1;
    const int q = __ffs(b) - 1;
    const uint32_t wq = __shfl_sync(GPM_FULL_MASK, x, q);
    return 32 * q + __ffs(wq) - 1;
}

__device__ __forceinline__ int count_range(const uint32_t* C, int w, int from, int to, int lane) {
    const int c = lane < w ? __popc(C[lane] & range_mask(lane, from, to)) : 0;
    return __reduce_add_sync(GPM_FULL_MASK, c);
}

__device__ __forceinline__ void add_count(Control* ctl, int j, unsigned long long v) {
    gpm_atomic_add_cc(&ctl->counts[j], v, &ctl->overflow);
}

// add to one of the warp's per-size counters (lane 0), raising the launch's
// overflow flag if it wraps
__device__ __forceinline__ void cq_wadd(Control* ctl, unsigned long long* c, unsigned long long v) {
    const unsigned long long s = *c + v;
    if (s < *c) atomicExch(&ctl->overflow, 1);
    *c = s;
}

// Build the root-local bit matrix.  The out-neighbours u of r get local
// positions in orientation order -- ascending (degree, id), the order that
// defines the DAG -- so that row p (the out-neighbours of the vertex at
// position p, restricted to N+(r)) holds only positions above p: every
// candidate set below position p lies in the words from p / 32 on.
// list[] receives N+(r) in id order (for the binary searches), pos[] each
// entry's position; both are scratch for the caller after the build.
__device__ __noinline__ static void build_rows(const int32_t* __restrict__ off, const int32_t* __restrict__ adj,
                                               const int32_t* __restrict__ outdeg, const int32_t* __restrict__ deg,
                                               int r, int d, int* list, int* pos, uint32_t* rows, int lane) {
    const int beg = off[r];
    for (int t = lane; t < d; t += 32) {
        const int u = adj[beg + t];
        list[t] = u;
        rows[t] = deg[u];               // sort keys, staged in the (not yet cleared) rows
    }
    __syncwarp();
    for (int t = lane; t < d; t += 32) {
        const int kt = rows[t];
        int p = 0;
        for (int s = 0; s < d; s++) {   // rank by (degree, id); ids ascend with s
            const int ks = rows[s];
            p += (ks < kt || (ks == kt && s < t)) ? 1 : 0;
        }
        pos[t] = p;
    }
    __syncwarp();
    const int w = (d + 31) >> 5;
    const int total = cq_tri_words(d, w);
    for (int t = lane; t < total; t += 32) rows[t] = 0u;
    __syncwarp();
    const int first = list[0], last = list[d - 1];
    for (int i = 0; i < d; i++) {
        const int u = list[i];
        const int ub = off[u], du = outdeg[u];
        uint32_t* row = rows + cq_tri_row(pos[i], w);   // words >= pos[i] / 32
        for (int t = lane; t < du; t += 32) {
            const int x = adj[ub + t];
            if (x < first || x > last) continue;
            int lo = 0, hi = d - 1;
            while (lo < hi) {               // first index with list[idx] >= x
                const int mid = (lo + hi) >> 1;
                if (list[mid] < x) lo = mid + 1; else hi = mid;
            }
            const int px = list[lo] == x ? pos[lo] : -1;
            if (px > pos[i]) {              // always, in the orientation; guards the triangle
                atomicOr(&row[px >> 5], 1u << (px & 31));
            }
        }
    }
    __syncwarp();
}


// Everything one warp needs to walk one unit.
struct CliqueWalk {
    const int32_t* __restrict__ off;
    const int32_t* __restrict__ adj;
    const int32_t* __restrict__ outdeg;
    const int32_t* __restrict__ deg;    // undirected degrees (the orientation's key)
    int k_lo, k_hi;
    int wmax;
    // this warp's shared memory
    unsigned long long* wcnt;   // per clique size, counts of sizes < k_hi - 1
    int* cur;
    int* hiv;
    uint32_t* cand;
    int* list;
    int* pairs;
    uint32_t* rows;
    // donation (DONATE only): ring of idle warp ids and the warps' mailboxes
    Control* ctl;
    QSeq* ring_seq;
    int32_t* ring_ids;
    unsigned long long ring_cap;
    unsigned char* mbox;        // mailbox of warp w at mbox + w * mbox_stride: MailHdr, CliqueUnit
    int mbox_stride;
    int donate_min;
    unsigned long long donate_after_ns;   // a unit splits only after running this long
    int tail_levels;                      // 2 or 3 (0: 3)
    int compact;                          // compacted two-level tail: 0 never, 1 large nodes, 2 whenever shorter
    int compact3;                         // compacted three-level tail whenever it shortens the rows (2: and
                                          // warp-cooperative pairs for nodes of at most 64 members)
    int cpl;                              // three-level tail: count the deepest level through the
                                          // non-edges (0 never, 1 always, 2..100 nodes at least this
                                          // percent dense)
    // host-monitored balancing (the paper's stop / redistribute / restart):
    // when the host raises ctl->stop, the walk writes its remaining work as
    // units to spill[] and unwinds
    bool monitor;
    CliqueUnit* spill;
    unsigned long long spill_cap;
    __device__ uint32_t* pairs_u32() const { return reinterpret_cast<uint32_t*>(pairs); }
};

// Compact the children of a node (set bits of C in [from, to)) into list[];
// returns how many.  Warp-uniform.
__device__ __forceinline__ int cq_compact(const uint32_t* C, int w, int from, int to, int* list, int lane) {
    int n = 0;
    for (int q = 0; q < w; q++) {
        const uint32_t word = C[q] & range_mask(q, from, to);
        const bool bit = (word >> lane) & 1u;
        const unsigned bal = __ballot_sync(GPM_FULL_MASK, bit);
        if (bit) list[n + __popc(bal & gpm_lanemask_lt())] = 32 * q + lane;
        n += __popc(bal);
    }
    __syncwarp();
    return n;
}

// sum over the set bits l of x (W >= w words, in registers) of
// popc(x & row_l): the cliques one level below the node whose candidates are
// x.  Row l is zero below word l / 32, so only words from there on are read.
// Two rows are loaded per step so that each lane has two independent
// shared-memory loads in flight.
template <int W, class Rows>
__device__ __forceinline__ unsigned cq_sum_rows(const uint32_t (&x)[W], const Rows& rows, int w) {
    unsigned acc = 0;
    // the word loop is unrolled, so for the bits of word q the row words
    // below q (zero) are skipped at compile time
#pragma unroll
    for (int q = 0; q < W; q++) {
        if (q >= w) break;
        uint32_t bits = x[q];
        while (bits) {
            const int l1 = 32 * q + __ffs(bits) - 1;
            bits &= bits - 1u;
            const uint32_t* r1 = rows.row(l1);
            if (bits) {
                const int l2 = 32 * q + __ffs(bits) - 1;
                bits &= bits - 1u;
                const uint32_t* r2 = rows.row(l2);
                uint32_t a[W], b[W];
#pragma unroll
                for (int z = q; z < W; z++) {
                    a[z] = z < w ? r1[z] : 0u;
                    b[z] = z < w ? r2[z] : 0u;
                }
#pragma unroll
                for (int z = q; z < W; z++) acc += __popc(x[z] & a[z]) + __popc(x[z] & b[z]);
            } else {
#pragma unroll
                for (int z = q; z < W; z++)
                    if (z < w) acc += __popc(x[z] & r1[z]);
            }
        }
    }
    return acc;
}

// The last two levels below a node of size k-3 with candidates C, children
// list[0..nchild): lane t takes children t, t+32, ...; for child i it forms
// C_i = C & row_i in registers (|C_i| = its (k-1)-clique children, added to
// km1) and, for every j in C_i, adds popc(C_i & row_j) -- the k-cliques
// through (i, j), aggregate_counter on each (k-1)-clique.  W >= w words.
template <int W>
__device__ __forceinline__ void cq_tail2(const uint32_t* C, const TriRows& rows, int w, const int* list,
                                         int nchild, unsigned long long& km1, unsigned long long& kk,
                                         unsigned long long& wops, int lane) {
    uint32_t c[W];
#pragma unroll
    for (int q = 0; q < W; q++) c[q] = q < w ? C[q] : 0u;
    for (int t = lane; t < nchild; t += 32) {
        const int pi = list[t];
        const int bi = pi >> 5;
        const uint32_t* ri = rows.row(pi);
        uint32_t ci[W];
        int g = 0;
#pragma unroll
        for (int q = 0; q < W; q++) {
            ci[q] = (q >= bi && q < w) ? (c[q] & ri[q]) : 0u;
            g += __popc(ci[q]);
        }
        km1 += (unsigned)g;
        wops += (unsigned long long)(g + 1) * (unsigned)w;
        kk += cq_sum_rows<W>(ci, rows, w);
    }
}

__device__ __forceinline__ void cq_tail2_dispatch(const uint32_t* C, const TriRows& rows, int w, const int* list,
                                                  int nchild, unsigned long long& km1, unsigned long long& kk,
                                                  unsigned long long& wops, int lane) {
    // few row widths, for the instruction cache (as cq_tail3c_dispatch)
    if (w <= 2) cq_tail2<2>(C, rows, w, list, nchild, km1, kk, wops, lane);
    else if (w <= 4) cq_tail2<4>(C, rows, w, list, nchild, km1, kk, wops, lane);
    else if (w <= 10) cq_tail2<10>(C, rows, w, list, nchild, km1, kk, wops, lane);
    else {
        // wide rows (out-degree > 320): C_i's words are recomputed from shared
        // memory instead of held in registers
        for (int t = lane; t < nchild; t += 32) {
            const int pi = list[t];
            const uint32_t* ri = rows.row(pi);
            unsigned long long acc = 0;
            for (int q = pi >> 5; q < w; q++) {
                uint32_t bits = C[q] & ri[q];
                km1 += (unsigned)__popc(bits);
                wops += (unsigned long long)(__popc(bits) + 1) * (unsigned)w;
                while (bits) {
                    const int j = 32 * q + __ffs(bits) - 1;
                    bits &= bits - 1u;
                    const uint32_t* rj = rows.row(j);
                    for (int z = q; z < w; z++) acc += __popc(C[z] & ri[z] & rj[z]);
                }
            }
            kk += acc;
        }
    }
}

// The last two levels below a node of size k-3, on the node's own members:
// member m is the m-th set bit of C (ascending position), and R[m] -- row m
// of a c x c bit matrix, c = |C| -- holds the members adjacent to it from
// its out-neighbourhood (only members above m, the positions being in
// orientation order).  The counts are those of cq_tail2 on the same
// children, but every row operation touches ceil(c/32) words instead of
// ceil(d/32).  The matrix is built by ballots: lane t holds the position of
// member 32b + t, and bit t of R[m]'s word b is that position's bit in the
// root-local row of member m.  Children: the members with positions in
// [from, to).  mem: c ints of scratch; R: c x (W2 | 1) words.
template <int W2>
__device__ __forceinline__ void cq_tail2c(const uint32_t* C, const TriRows& rows, int w, int c, int from,
                                          int to, int* mem, uint32_t* R, unsigned long long& nchild,
                                          unsigned long long& km1, unsigned long long& kk,
                                          unsigned long long& wops, int lane) {
    int n = 0, m_lo = 0, m_hi = 0;
    for (int q = 0; q < w; q++) {
        const uint32_t word = C[q];
        const bool bit = (word >> lane) & 1u;
        const unsigned bal = __ballot_sync(GPM_FULL_MASK, bit);
        if (bit) mem[n + __popc(bal & gpm_lanemask_lt())] = 32 * q + lane;
        n += __popc(bal);
        m_lo += __popc(bal & range_mask(q, 0, from));
        m_hi += __popc(bal & range_mask(q, 0, to));
    }
    __syncwarp();
    const int w2 = (c + 31) >> 5;
    const int ws2 = w2 | 1;
    int pm[W2];
#pragma unroll
    for (int b = 0; b < W2; b++) pm[b] = (b < w2 && 32 * b + lane < c) ? mem[32 * b + lane] : -1;
    for (int m = 0; m < c; m++) {
        const int pmm = mem[m];
        const uint32_t* row = rows.row(pmm);
        uint32_t* Rm = R + m * ws2;
#pragma unroll
        for (int b = 0; b < W2; b++) {
            if (b < w2) {
                uint32_t word = 0u;
                if (b >= (m >> 5)) {      // members above m only: earlier words are empty
                    const bool bit = pm[b] > pmm && ((row[pm[b] >> 5] >> (pm[b] & 31)) & 1u);
                    word = __ballot_sync(GPM_FULL_MASK, bit);
                }
                if (lane == b) Rm[b] = word;
            }
        }
    }
    __syncwarp();
    for (int m = m_lo + lane; m < m_hi; m += 32) {
        const uint32_t* Rm = R + m * ws2;
        uint32_t x[W2];
        int g = 0;
#pragma unroll
        for (int z = 0; z < W2; z++) {
            x[z] = z < w2 ? Rm[z] : 0u;
            g += __popc(x[z]);
        }
        km1 += (unsigned)g;
        wops += (unsigned long long)g * (unsigned)w2;
        kk += cq_sum_rows<W2>(x, RectRows{R, ws2}, w2);
    }
    nchild = (unsigned long long)(m_hi - m_lo);
    __syncwarp();
}

__device__ __forceinline__ void cq_tail2c_dispatch(const uint32_t* C, const TriRows& rows, int w, int c,
                                                   int from, int to, int* mem, uint32_t* R,
                                                   unsigned long long& nchild, unsigned long long& km1,
                                                   unsigned long long& kk, unsigned long long& wops, int lane) {
    const int w2 = (c + 31) >> 5;
    if (w2 <= 2) cq_tail2c<2>(C, rows, w, c, from, to, mem, R, nchild, km1, kk, wops, lane);
    else cq_tail2c<5>(C, rows, w, c, from, to, mem, R, nchild, km1, kk, wops, lane);
}

// Pairs (i, j) -- a child i of a node of size k-4 and a child j of i -- in
// pairs[0..np), packed (i << 16) | j.  Lane t takes pairs t, t+32, ...:
// C_ij = C & row_i & row_j (one 3-input AND per word; its popcount is the
// (k-1)-cliques through (i, j)), then popc(C_ij & row_l) for every l in C_ij
// adds the k-cliques: aggregate_counter on every (k-1)-clique.
template <int W>
__device__ __forceinline__ void cq_pairs_run(const uint32_t (&c)[W], const TriRows& rows, int w,
                                             const int* pairs, int np, unsigned long long& km1,
                                             unsigned long long& kk, unsigned long long& wops, int lane) {
    for (int t = lane; t < np; t += 32) {
        const int pr = pairs[t];
        const int pj = pr & 0xffff;          // j > i: both rows are stored from word pj / 32 on
        const int bj = pj >> 5;
        const uint32_t* ri = rows.row(pr >> 16);
        const uint32_t* rj = rows.row(pj);
        uint32_t cij[W];
        int g = 0;
#pragma unroll
        for (int z = 0; z < W; z++) {
            cij[z] = (z >= bj && z < w) ? (c[z] & ri[z] & rj[z]) : 0u;
            g += __popc(cij[z]);
        }
        km1 += (unsigned)g;
        wops += (unsigned long long)(g + 1) * (unsigned)w;
        kk += cq_sum_rows<W>(cij, rows, w);
    }
}

// The deepest level of the three-level tail counted through non-edges.  For
// a child m of the tail node, X = its candidates (the vertices that extend
// it); the k-cliques below m are the triangles of G[X].  With a_t = the
// neighbours of t above t inside X, the sum over t of C(a_t, 2) counts every
// triangle once (at its lowest vertex) plus every wedge u - t - v (t below
// u < v) whose ends are not adjacent; those wedges are counted from the
// non-edge side: for each non-adjacent pair u < v in X, the members t of X
// below u adjacent to both.  So
//     triangles(G[X]) = sum_t C(a_t, 2) - sum_{u<v in X, u !~ v} |{t < u : t ~ u, t ~ v}|,
// and on a nearly complete G[X] the second sum has few terms: the work per
// pair (m, t) is one AND + POPC instead of one per (k-1)-clique through it.
// A pair (m, j) adds C(a_j, 2) to P and its non-edges' wedge counts to Q; a
// node's P - Q is exact once all its pairs are in (the caller sums the warp).
__device__ __forceinline__ uint32_t bits_above(int b) { return b >= 31 ? 0u : (0xffffffffu << (b + 1)); }
__device__ __forceinline__ uint32_t bits_below(int b) { return (1u << b) - 1u; }

// x: X (the candidates of the pair's first member), j: the pair's second
// member, rows: upper rows (row(t)[z] valid for z >= t / 32).  Returns a_j
// (the (k-1)-cliques through the pair).
template <int W, class Rows>
__device__ __forceinline__ int cq_cpl_pair(const uint32_t (&x)[W], const Rows& rows, int w, int j,
                                           unsigned long long& P, unsigned long long& Q,
                                           unsigned long long& wops) {
    const uint32_t* rj = rows.row(j);
    const int bj = j >> 5;
    uint32_t u[W];
    int a = 0;
    bool any = false;
#pragma unroll
    for (int z = 0; z < W; z++) {
        uint32_t r = 0u;
        if (z >= bj && z < w) r = rj[z];
        a += __popc(x[z] & r);
        uint32_t nb = x[z] & ~r;                 // members of X not adjacent to j ...
        nb &= z < bj ? 0u : (z == bj ? bits_above(j & 31) : 0xffffffffu);   // ... above j
        u[z] = nb;
        any |= nb != 0u;
    }
    P += (unsigned long long)(a * (a - 1) / 2);
    wops += (unsigned)w;
    if (any) {
#pragma unroll
        for (int zv = 0; zv < W; zv++) {
            uint32_t nb = u[zv];
            while (nb) {
                const int v = 32 * zv + __ffs(nb) - 1;
                nb &= nb - 1u;
                // members t of X below j adjacent to j and to v
                unsigned q = 0;
#pragma unroll
                for (int zt = 0; zt < W; zt++) {
                    if (zt > bj) break;
                    uint32_t tb = x[zt] & (zt < bj ? 0xffffffffu : bits_below(j & 31));
                    while (tb) {
                        const int t = 32 * zt + __ffs(tb) - 1;
                        tb &= tb - 1u;
                        const uint32_t* rt = rows.row(t);
                        q += (rt[bj] >> (j & 31)) & (rt[v >> 5] >> (v & 31)) & 1u;
                        wops += 1;
                    }
                }
                Q += q;
            }
        }
    }
    return a;
}

// sum P, Q over the warp and add P - Q (>= 0 for whole nodes) to lane 0's kk
__device__ __forceinline__ void cq_cpl_fold(unsigned long long P, unsigned long long Q, unsigned long long& kk,
                                            int lane) {
    for (int o = 16; o > 0; o >>= 1) {
        P += __shfl_xor_sync(GPM_FULL_MASK, P, o);
        Q += __shfl_xor_sync(GPM_FULL_MASK, Q, o);
    }
    if (lane == 0) kk += P - Q;
}

// whether a node of c members with e edges among them takes the non-edge
// count (policy as CliqueWalk::cpl)
__device__ __forceinline__ bool cq_cpl_dense(int policy, long long e, int c) {
    if (policy <= 0 || c < 3) return false;
    if (policy == 1) return true;
    return 200ll * e >= (long long)policy * c * (c - 1);
}

// cq_pairs_run with the deepest level counted through non-edges
template <int W>
__device__ __forceinline__ void cq_pairs_run_cpl(const uint32_t (&c)[W], const TriRows& rows, int w,
                                                 const int* pairs, int np, unsigned long long& km1,
                                                 unsigned long long& P, unsigned long long& Q,
                                                 unsigned long long& wops, int lane) {
    for (int t = lane; t < np; t += 32) {
        const int pr = pairs[t];
        const int pi = pr >> 16;
        const int bi = pi >> 5;
        const uint32_t* ri = rows.row(pi);
        uint32_t x[W];
#pragma unroll
        for (int z = 0; z < W; z++) x[z] = (z >= bi && z < w) ? (c[z] & ri[z]) : 0u;
        km1 += (unsigned)cq_cpl_pair<W>(x, rows, w, pr & 0xffff, P, Q, wops);
    }
}

// The last three levels below a node of size k-4 with candidates C and
// children in [from, to): its children i are walked in order (warp-uniform);
// the grandchildren j of each (bits of C & row_i) are appended to a shared
// pair batch with ballot compaction, and the batch is run lane-parallel
// (cq_pairs_run) whenever it holds CQ_PAIR_FLUSH pairs -- every lane gets a
// pair, however few children each node has.  Uniform counts: n3 children
// (size k-3), n2 pairs (size k-2).
template <int W>
__device__ __forceinline__ void cq_tail3(const uint32_t* C, const TriRows& rows, int w, int from, int to,
                                         int* pairs, unsigned long long& n3, unsigned long long& n2,
                                         unsigned long long& km1, unsigned long long& kk, unsigned long long& wops,
                                         int lane, int cpl) {
    uint32_t c[W];
#pragma unroll
    for (int z = 0; z < W; z++) c[z] = z < w ? C[z] : 0u;
    bool dense = false;
    if (cpl > 0) {
        // edges among the node's members (one row AND per member)
        int cnt = 0, e = 0;
        for (int q = 0; q < w; q++) {
            const uint32_t word = c[q];
            cnt += __popc(word);
            if ((word >> lane) & 1u) {
                const int p = 32 * q + lane;
                const uint32_t* rp = rows.row(p);
                for (int z = q; z < w; z++) e += __popc(C[z] & rp[z]);
            }
        }
        e = (int)__reduce_add_sync(GPM_FULL_MASK, (unsigned)e);
        dense = cq_cpl_dense(cpl, e, cnt);
    }
    unsigned long long P = 0, Q = 0;
    int np = 0;
    for (int q = 0; q < w; q++) {
        uint32_t word = C[q] & range_mask(q, from, to);
        while (word) {
            const int i = 32 * q + __ffs(word) - 1;
            word &= word - 1u;
            n3 += 1;
            const uint32_t* ri = rows.row(i);
            for (int q2 = i >> 5; q2 < w; q2++) {
                const uint32_t ciw = C[q2] & ri[q2];
                const bool bit = (ciw >> lane) & 1u;
                const unsigned bal = __ballot_sync(GPM_FULL_MASK, bit);
                if (bit) pairs[np + __popc(bal & gpm_lanemask_lt())] = (i << 16) | (32 * q2 + lane);
                np += __popc(bal);
            }
            if (lane == 0) wops += (unsigned)w;
            if (np >= CQ_PAIR_FLUSH) {
                __syncwarp();
                n2 += (unsigned)np;
                if (dense)
                    cq_pairs_run_cpl<W>(c, rows, w, pairs, np, km1, P, Q, wops, lane);
                else
                    cq_pairs_run<W>(c, rows, w, pairs, np, km1, kk, wops, lane);
                __syncwarp();
                np = 0;
            }
        }
    }
    if (np) {
        __syncwarp();
        n2 += (unsigned)np;
        if (dense)
            cq_pairs_run_cpl<W>(c, rows, w, pairs, np, km1, P, Q, wops, lane);
        else
            cq_pairs_run<W>(c, rows, w, pairs, np, km1, kk, wops, lane);
        __syncwarp();
    }
    if (dense) cq_cpl_fold(P, Q, kk, lane);
}

__device__ __forceinline__ void cq_tail3_dispatch(const uint32_t* C, const TriRows& rows, int w, int from, int to,
                                                  int* pairs, unsigned long long& n3, unsigned long long& n2,
                                                  unsigned long long& km1, unsigned long long& kk,
                                                  unsigned long long& wops, int lane, int cpl) {
    // few row widths, for the instruction cache (as cq_tail3c_dispatch)
    if (w <= 2) cq_tail3<2>(C, rows, w, from, to, pairs, n3, n2, km1, kk, wops, lane, cpl);
    else if (w <= 4) cq_tail3<4>(C, rows, w, from, to, pairs, n3, n2, km1, kk, wops, lane, cpl);
    else cq_tail3<10>(C, rows, w, from, to, pairs, n3, n2, km1, kk, wops, lane, cpl);
}

// The last three levels below a node of size k-4, on the node's own members
// (as cq_tail2c does for two): member m is the m-th set bit of C, and R[m]
// holds the members adjacent to m above it, ceil(c/32) words per row instead
// of ceil(d/32).  The node's children (members with positions in [from,
// to)) are walked in order; the grandchildren m2 of each m1 (bits of R[m1])
// go to a pair batch, run lane-parallel: C_m1m2 = R[m1] & R[m2] (its
// popcount: the (k-1)-cliques through the pair), then popc(C_m1m2 & R[l])
// for every l in it (the k-cliques).  mem: c ints; R: c x (W2 | 1) words,
// then the pair batch.  Uniform counts: n3 children, n2 pairs.
template <int W2>
__device__ __forceinline__ void cq_pairs_run_c(const uint32_t* R, int ws2, int w2, const int* pairs, int np,
                                               unsigned long long& km1, unsigned long long& kk,
                                               unsigned long long& wops, int lane) {
    for (int t = lane; t < np; t += 32) {
        const int pr = pairs[t];
        const uint32_t* r1 = R + (pr >> 16) * ws2;
        const uint32_t* r2 = R + (pr & 0xffff) * ws2;
        uint32_t x[W2];
        int g = 0;
#pragma unroll
        for (int z = 0; z < W2; z++) {
            x[z] = z < w2 ? (r1[z] & r2[z]) : 0u;
            g += __popc(x[z]);
        }
        km1 += (unsigned)g;
        wops += (unsigned long long)(g + 1) * (unsigned)w2;
        kk += cq_sum_rows<W2>(x, RectRows{R, ws2}, w2);
    }
}

template <int W2>
__device__ __forceinline__ void cq_pairs_run_c_cpl(const uint32_t* R, int ws2, int w2, const int* pairs, int np,
                                                   unsigned long long& km1, unsigned long long& P,
                                                   unsigned long long& Q, unsigned long long& wops, int lane) {
    const RectRows rr{R, ws2};
    for (int t = lane; t < np; t += 32) {
        const int pr = pairs[t];
        const uint32_t* r1 = R + (pr >> 16) * ws2;
        uint32_t x[W2];
#pragma unroll
        for (int z = 0; z < W2; z++) x[z] = z < w2 ? r1[z] : 0u;
        km1 += (unsigned)cq_cpl_pair<W2>(x, rr, w2, pr & 0xffff, P, Q, wops);
    }
}

template <int W2>
__device__ __forceinline__ void cq_tail3c(const uint32_t* C, const TriRows& rows, int w, int c, int from, int to,
                                          int* mem, uint32_t* R, unsigned long long& n3, unsigned long long& n2,
                                          unsigned long long& km1, unsigned long long& kk,
                                          unsigned long long& wops, int lane, bool coop, int cpl) {
    int n = 0, m_lo = 0, m_hi = 0;
    for (int q = 0; q < w; q++) {
        const uint32_t word = C[q];
        const bool bit = (word >> lane) & 1u;
        const unsigned bal = __ballot_sync(GPM_FULL_MASK, bit);
        if (bit) mem[n + __popc(bal & gpm_lanemask_lt())] = 32 * q + lane;
        n += __popc(bal);
        m_lo += __popc(bal & range_mask(q, 0, from));
        m_hi += __popc(bal & range_mask(q, 0, to));
    }
    __syncwarp();
    const int w2 = (c + 31) >> 5;
    const int ws2 = w2 | 1;
    int* pairs = reinterpret_cast<int*>(R + 32 * CQ_CW * CQ_CW);
    int pm[W2];
#pragma unroll
    for (int b = 0; b < W2; b++) pm[b] = (b < w2 && 32 * b + lane < c) ? mem[32 * b + lane] : -1;
    long long edges = 0;                  // among the members (warp-uniform)
    for (int m = 0; m < c; m++) {
        const int pmm = mem[m];
        const uint32_t* row = rows.row(pmm);
        uint32_t* Rm = R + m * ws2;
#pragma unroll
        for (int b = 0; b < W2; b++) {
            if (b < w2) {
                uint32_t word = 0u;
                if (b >= (m >> 5)) {      // members above m only: earlier words are empty
                    const bool bit = pm[b] > pmm && ((row[pm[b] >> 5] >> (pm[b] & 31)) & 1u);
                    word = __ballot_sync(GPM_FULL_MASK, bit);
                }
                edges += __popc(word);
                if (lane == b) Rm[b] = word;
            }
        }
    }
    __syncwarp();
    if (lane == 0) wops += (unsigned long long)c * (unsigned)w2;
    n3 += (unsigned)(m_hi - m_lo);
    const bool dense = cq_cpl_dense(cpl, edges, c);
    if (coop && w2 <= 2 && !dense) {
        // at most 64 members: the warp takes the pairs one at a time, lane t
        // holding the rows of members t and t + 32, and for a pair with
        // candidates y adds popc(y & R[t]) when t is in y -- every lane works
        // on every pair, whatever |y|, instead of one lane looping over it
        // (the second word exists only when the node has two words of
        // members: one-word nodes run this width too, with rows of stride 1)
        const bool two = w2 == 2;
        const uint32_t ra0 = lane < c ? R[lane * ws2] : 0u;
        const uint32_t ra1 = (two && lane < c) ? R[lane * ws2 + 1] : 0u;
        const uint32_t rb1 = (two && lane + 32 < c) ? R[(lane + 32) * ws2 + 1] : 0u;
        unsigned long long npairs = 0, mine = 0, g_all = 0;
        for (int m1 = m_lo; m1 < m_hi; m1++) {
            const uint32_t x0 = R[m1 * ws2];
            const uint32_t x1 = two ? R[m1 * ws2 + 1] : 0u;
#pragma unroll
            for (int q2 = 0; q2 < 2; q2++) {
                uint32_t bits = q2 == 0 ? x0 : x1;
                while (bits) {
                    const int m2 = 32 * q2 + __ffs(bits) - 1;
                    bits &= bits - 1u;
                    const uint32_t y0 = x0 & R[m2 * ws2];
                    const uint32_t y1 = two ? (x1 & R[m2 * ws2 + 1]) : 0u;
                    npairs++;
                    g_all += (unsigned)(__popc(y0) + __popc(y1));
                    unsigned v = ((y0 >> lane) & 1u) ? (unsigned)(__popc(y0 & ra0) + __popc(y1 & ra1)) : 0u;
                    v += ((y1 >> lane) & 1u) ? (unsigned)__popc(y1 & rb1) : 0u;
                    mine += v;
                }
            }
        }
        kk += mine;
        n2 += npairs;
        if (lane == 0) {
            km1 += g_all;
            wops += (g_all + npairs) * (unsigned)w2;
        }
        __syncwarp();
        return;
    }
    unsigned long long P = 0, Q = 0;
    int np = 0;
    for (int m1 = m_lo; m1 < m_hi; m1++) {
        const uint32_t* r1 = R + m1 * ws2;
        for (int q2 = m1 >> 5; q2 < w2; q2++) {
            const uint32_t word = r1[q2];
            const bool bit = (word >> lane) & 1u;
            const unsigned bal = __ballot_sync(GPM_FULL_MASK, bit);
            if (bit) pairs[np + __popc(bal & gpm_lanemask_lt())] = (m1 << 16) | (32 * q2 + lane);
            np += __popc(bal);
        }
        if (np >= CQ_PAIR_FLUSH) {
            __syncwarp();
            n2 += (unsigned)np;
            if (dense)
                cq_pairs_run_c_cpl<W2>(R, ws2, w2, pairs, np, km1, P, Q, wops, lane);
            else
                cq_pairs_run_c<W2>(R, ws2, w2, pairs, np, km1, kk, wops, lane);
            __syncwarp();
            np = 0;
        }
    }
    if (np) {
        __syncwarp();
        n2 += (unsigned)np;
        if (dense)
            cq_pairs_run_c_cpl<W2>(R, ws2, w2, pairs, np, km1, P, Q, wops, lane);
        else
            cq_pairs_run_c<W2>(R, ws2, w2, pairs, np, km1, kk, wops, lane);
    }
    if (dense) cq_cpl_fold(P, Q, kk, lane);
    __syncwarp();
}

__device__ __forceinline__ void cq_tail3c_dispatch(const uint32_t* C, const TriRows& rows, int w, int c, int from,
                                                   int to, int* mem, uint32_t* R, unsigned long long& n3,
                                                   unsigned long long& n2, unsigned long long& km1,
                                                   unsigned long long& kk, unsigned long long& wops, int lane,
                                                   bool coop, int cpl) {
    // one row width: each width is a separate unrolled copy of the tail, and
    // warps in nodes of different widths compete for the instruction cache
    // (chunglu1m 4..7: one copy per width 1..5 2.81 s, widths 2 and 5
    // 1.59 s, width 5 alone 1.34 s); narrower nodes run with zero words
    const int w2 = (c + 31) >> 5;
    cq_tail3c<5>(C, rows, w, c, from, to, mem, R, n3, n2, km1, kk, wops, lane, coop && w2 <= 2, cpl);
}

// Split point of a node's remaining children (set bits of C in [from, to))
// for a hand-off: child i has c_i = |C & row_i| candidates and a subtree that
// grows like c_i^e (e = the levels below it), so the donated suffix [mid, to)
// is cut where it carries about half of the estimated work; at least one
// child stays and one goes.  Returns -1 when fewer than two remain.
// Warp-uniform; two lane-parallel passes over the children.
__device__ __noinline__ static int cq_balanced_mid(const uint32_t* C, const TriRows& rows, int w, int from, int to,
                                                   int e, int lane) {
    float total = 0.f;
    int n = 0;
    for (int pass = 0; pass < 2; pass++) {
        float run = 0.f;
        int seen = 0;
        for (int q = 0; q < w; q++) {
            const uint32_t word = C[q] & range_mask(q, from, to);
            const bool bit = (word >> lane) & 1u;
            float wt = 0.f;
            if (bit) {
                const int p = 32 * q + lane;
                const uint32_t* rp = rows.row(p);
                int c = 0;
                for (int z = q; z < w; z++) c += __popc(C[z] & rp[z]);
                wt = __powf((float)c + 1.f, (float)e);
            }
            // inclusive prefix of the weights over the lanes of this word
            float incl = wt;
            for (int o = 1; o < 32; o <<= 1) {
                const float y = __shfl_up_sync(GPM_FULL_MASK, incl, o);
                if (lane >= o) incl += y;
            }
            const unsigned bal = __ballot_sync(GPM_FULL_MASK, bit);
            if (pass == 1) {
                // first child whose prefix passes half the total (never the first child)
                const int rank = seen + __popc(bal & gpm_lanemask_lt());
                const bool cut = bit && rank >= 1 && run + incl > 0.5f * total;
                const unsigned cuts = __ballot_sync(GPM_FULL_MASK, cut);
                if (cuts) return 32 * q + __ffs(cuts) - 1;
            }
            run += __shfl_sync(GPM_FULL_MASK, incl, 31);
            seen += __popc(bal);
        }
        if (pass == 0) {
            total = run;
            n = seen;
            if (n < 2) return -1;
        }
    }
    return -1;
}

// Walk one unit (root r = roots[root_pos], d = |N+(r)|).  Returns false if it
// stopped on a device error.  Lane-private results: unit_sum (k_hi-cliques)
// and km1 (k_hi-1 cliques, used when k_lo < k_hi); smaller sizes go to wcnt.
template <bool DONATE>
__device__ bool cq_walk(const CliqueWalk& a, const CliqueUnit* unit, int root_pos, int r, int d, int& cached_root,
                        unsigned long long& unit_sum, unsigned long long& km1, unsigned long long& wops, int lane) {
    if (d < a.k_lo - 1 || d <= 0) return true;
    const int w = (d + 31) >> 5;
    const int K = a.k_hi;
    unsigned long long* wcnt = a.wcnt;
    int* cur = a.cur;
    int* hiv = a.hiv;
    uint32_t* cand = a.cand;
    int* list = a.list;
    if (r != cached_root) {
        build_rows(a.off, a.adj, a.outdeg, a.deg, r, d, list, a.pairs, a.rows, lane);
        cached_root = r;
    }
    const TriRows rows{a.rows, w};
    // candidates of the unit's node: all of N+(r), then AND along the path
    if (lane < w) cand[1 * a.wmax + lane] = range_mask(lane, 0, d);
    __syncwarp();
    const int depth = unit->depth;
    int s = 1;
    for (int t = 0; t < depth; t++) {
        const int i = unit->path[t];
        if (lane < w)
            cand[(s + 1) * a.wmax + lane] = lane >= (i >> 5) ? (cand[s * a.wmax + lane] & rows.row(i)[lane]) : 0u;
        s++;
        __syncwarp();
    }
    const int s_base = s;
    if (lane == 0) {
        cur[s] = unit->lo;
        hiv[s] = unit->hi < 0 ? d : unit->hi;
    }
    __syncwarp();
    // nodes of size `tail` are finished by the lane-parallel tail: three
    // levels (by default for k >= 7, where the pair batches keep every lane
    // busy; measured slower than two levels at k = 6), else two, else one
    const bool three = w <= 10 && K >= 5 && (a.tail_levels == 3 || (a.tail_levels == 0 && K >= 7));
    const int tail = three ? K - 4 : (K >= 4 ? K - 3 : 1);
    const unsigned long long t_start = DONATE ? gpm_globaltimer() : 0ull;

    unsigned long long last_check = t_start;   // lane 0
    int iter = 0;
    bool big = false;                          // the last step ran a three-level tail node
    for (;;) {
        const uint32_t* Cs = cand + s * a.wmax;
        if (s == tail && three) {
            unsigned long long n3 = 0, n2 = 0;
            // on the node's members when that shortens the rows
            const int c = (w >= 3 && a.compact3) ? count_range(Cs, w, 0, d, lane) : 0;
            const int w2 = (c + 31) >> 5;
            if (c > 0 && w2 <= CQ_CW && w2 < w)
                cq_tail3c_dispatch(Cs, rows, w, c, cur[s], hiv[s], list, a.pairs_u32(), n3, n2, km1, unit_sum, wops,
                                   lane, a.compact3 == 2, a.cpl);
            else
                cq_tail3_dispatch(Cs, rows, w, cur[s], hiv[s], a.pairs, n3, n2, km1, unit_sum, wops, lane, a.cpl);
            if (lane == 0) {
                if (K - 3 >= a.k_lo) cq_wadd(a.ctl, &wcnt[K - 3], n3);
                if (K - 2 >= a.k_lo) cq_wadd(a.ctl, &wcnt[K - 2], n2);
            }
            __syncwarp();
            if (s == s_base) break;
            s--;
            big = true;
            continue;
        }
        if (s == tail && K >= 4 && w >= 3 && a.compact != 0) {
            // compact the node to its members when that shortens the rows
            const int c = count_range(Cs, w, 0, d, lane);
            const int w2 = (c + 31) >> 5;
            if (w2 <= CQ_CW && w2 < w && (a.compact == 2 || c >= CQ_COMPACT_MIN)) {
                unsigned long long nch = 0;
                cq_tail2c_dispatch(Cs, rows, w, c, cur[s], hiv[s], list, a.pairs_u32(), nch, km1, unit_sum,
                                   wops, lane);
                if (lane == 0 && K - 2 >= a.k_lo) cq_wadd(a.ctl, &wcnt[K - 2], nch);
                __syncwarp();
                if (s == s_base) break;
                s--;
                continue;
            }
        }
        if (s == tail) {
            const int nchild = cq_compact(Cs, w, cur[s], hiv[s], list, lane);
            if (K == 3) {
                // one level: 3-cliques = sum over children of popc(C & row_i)
                unsigned long long sum = 0;
                for (int t = lane; t < nchild; t += 32) {
                    const int pi = list[t];
                    const uint32_t* row = rows.row(pi);
                    int c = 0;
                    for (int q = pi >> 5; q < w; q++) c += __popc(Cs[q] & row[q]);
                    sum += (unsigned)c;
                    wops += (unsigned)w;
                }
                unit_sum += sum;
            } else {
                if (lane == 0 && K - 2 >= a.k_lo) cq_wadd(a.ctl, &wcnt[K - 2], (unsigned)nchild);
                cq_tail2_dispatch(Cs, rows, w, list, nchild, km1, unit_sum, wops, lane);
            }
            __syncwarp();
            if (s == s_base) break;
            s--;
            continue;
        }
        const int i = next_child(Cs, w, cur[s], hiv[s], lane);
        if (i < 0) {
            if (s == s_base) break;
            s--;
            continue;
        }
        uint32_t* Cn = cand + (s + 1) * a.wmax;
        uint32_t x = 0;
        if (lane < w) {
            x = lane >= (i >> 5) ? (Cs[lane] & rows.row(i)[lane]) : 0u;
            Cn[lane] = x;
        }
        const int c = __reduce_add_sync(GPM_FULL_MASK, (unsigned)__popc(x));
        if (lane == 0) wops += (unsigned)w;
        if (lane == 0) {
            cur[s] = i + 1;
            if (s + 1 >= a.k_lo) cq_wadd(a.ctl, &wcnt[s + 1], 1ull);
        }
        // descend while the child can still reach a counted size
        const bool down = c > 0 && (s + 1 + c >= a.k_lo);
        if (down && lane == 0) {
            cur[s + 1] = 0;
            hiv[s + 1] = d;
        }
        __syncwarp();
        if (down) s++;

        // look for idle warps after every three-level tail node (one can run
        // for milliseconds on a dense core) and every 16th other step, but
        // at most once per CQ_CHECK_NS
        int chk = 0;
        unsigned long long now = 0;
        if ((DONATE || a.monitor) && (big || (++iter & 15) == 0)) {
            big = false;
            if (lane == 0) {
                now = gpm_globaltimer();
                if (now - last_check >= CQ_CHECK_NS) {
                    last_check = now;
                    chk = 1;
                }
            }
            chk = __shfl_sync(GPM_FULL_MASK, chk, 0);
        }
        if (!DONATE && a.monitor && chk) {
            Control* ctl = a.ctl;
            int err = 0, stop = 0;
            if (lane == 0) {
                err = *(volatile int*)&ctl->error;
                stop = *(volatile int*)&ctl->stop;
            }
            err = __shfl_sync(GPM_FULL_MASK, err, 0);
            if (err) return false;
            if (__shfl_sync(GPM_FULL_MASK, stop, 0)) {
                // spill every level's remaining children as a unit, then
                // unwind (the emptied ranges end the walk)
                if (lane == 0) {
                    for (int t = s_base; t <= s; t++) {
                        if (cur[t] >= hiv[t]) continue;
                        const unsigned long long slot = atomicAdd(&ctl->spill_n, 1ull);
                        if (slot >= a.spill_cap) {   // never: one unit per level per warp fits
                            atomicCAS(&ctl->error, 0, DEV_ECHECK + 7);
                            break;
                        }
                        CliqueUnit u;
                        u.root_pos = root_pos;
                        u.depth = depth + (t - s_base);
                        u.lo = cur[t];
                        u.hi = hiv[t];
                        for (int z = 0; z < depth; z++) u.path[z] = unit->path[z];
                        for (int z = s_base; z < t; z++) u.path[depth + (z - s_base)] = (uint16_t)(cur[z] - 1);
                        for (int z = u.depth; z < GPM_CLIQUE_MAX_K; z++) u.path[z] = 0;
                        a.spill[slot] = u;
                    }
                    for (int t = s_base; t <= s; t++) hiv[t] = cur[t];
                }
                __syncwarp();
            }
        }
        if (DONATE && chk) {
            Control* ctl = a.ctl;
            // abort on a device error; split when someone is idle and this
            // unit has already run for a while
            int err = 0, want = 0;
            if (lane == 0) {
                err = *(volatile int*)&ctl->error;
                if (now - t_start > a.donate_after_ns) {
                    const unsigned long long qh = *(volatile unsigned long long*)&ctl->q_head;
                    const unsigned long long qt = *(volatile unsigned long long*)&ctl->q_tail;
                    want = qt > qh;   // a registered idle warp is waiting
                }
            }
            err = __shfl_sync(GPM_FULL_MASK, err, 0);
            if (err) return false;
            want = __shfl_sync(GPM_FULL_MASK, want, 0);
            if (want) {
                // shallowest level above the tail with enough siblings left
                for (int t = s_base; t <= s && t < tail; t++) {
                    const uint32_t* Ct = cand + t * a.wmax;
                    const int from = cur[t], to = hiv[t];
                    const int rem = count_range(Ct, w, from, to, lane);
                    if (rem < max(a.donate_min, 2)) continue;
                    // keep the heavier first children, donate a suffix with
                    // about half of the estimated work
                    const int mid = cq_balanced_mid(Ct, rows, w, from, to, max(K - t - 2, 1), lane);
                    if (mid < 0) break;
                    if (lane == 0) {
                        int wid;
                        if (gpm_idle_claim(a.ring_seq, a.ring_ids, a.ring_cap, &ctl->q_head, &wid)) {
                            unsigned char* box = a.mbox + (size_t)wid * a.mbox_stride;
                            CliqueUnit* dst = reinterpret_cast<CliqueUnit*>(box + sizeof(MailHdr));
                            CliqueUnit u;
                            u.root_pos = root_pos;
                            u.depth = depth + (t - s_base);
                            u.lo = mid;
                            u.hi = to;
                            for (int z = 0; z < depth; z++) u.path[z] = unit->path[z];
                            for (int z = s_base; z < t; z++) u.path[depth + (z - s_base)] = (uint16_t)(cur[z] - 1);
                            for (int z = u.depth; z < GPM_CLIQUE_MAX_K; z++) u.path[z] = 0;
                            *dst = u;
                            atomicAdd((unsigned long long*)&ctl->pending, 1ull);
                            __threadfence();
                            atomicExch(&reinterpret_cast<MailHdr*>(box)->ready, 1);
                            atomicAdd(&ctl->donations, 1ull);
                            hiv[t] = mid;
                        }
                    }
                    __syncwarp();
                    break;
                }
            }
        }
    }
    return true;
}

}  // namespace gpm
