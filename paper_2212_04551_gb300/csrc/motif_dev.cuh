// motif_dev.cuh -- device code of one motif work unit (ESU-style extension,
// pattern-table aggregation, optional work donation), shared by the
// single-graph kernel (motif.cu) and the batched kernel (batch.cu).
//
// Algorithm 4 (motif counting) extends a traversal from the adjacency of all
// its vertices, keeps canonical candidates only, and at |tr| = k-1 maps every
// traversal + extension to its pattern with the edge-bitmap dictionary of
// Section 4.3.4.  The walk below reaches the same connected induced k-sets,
// each exactly once, with ESU's exclusive extension (Wernicke 2006):
//
//   * the root r is the smallest vertex of the set; ext_1 = {u in N(r): u > r};
//   * choosing w = ext_l[i] gives ext_{l+1} = ext_l[i+1:] followed by the
//     exclusive neighbours of w: u in N(w), u > r, u neither in the
//     traversal nor adjacent to it.
//
// A byte per vertex ("mark") records the traversal positions the vertex is
// adjacent to (bit j <=> adjacent to tr[j]) and whether it is in the
// traversal (bit 7): pushing w marks N(w) once, popping it unmarks N(w).  The
// exclusivity test and the traversal edge bitmap (the paper's induce step)
// are then one byte load per candidate.
//
// Traversal code (the paper's layout): the v0-v1 edge is implicit; v_i's
// edges to v_0..v_{i-1} sit at bit offset i(i-1)/2 - 1.  At |tr| = k-1 no
// extension array is built: the k-vertex leaves are (a) the remaining entries
// of the parent's array, whose code bits come from the marks, and (b) the
// exclusive neighbours of the newest vertex, which all share one code.
#pragma once

#include "common.cuh"
#include "list_ring.cuh"

namespace gpm {

constexpr int MT_MAXK = GPM_MOTIF_MAX_K;
constexpr int MT_MAXPAT = 853;                 // connected 7-vertex patterns: per-block shared counters
constexpr int MT_MAXPAT8 = 11117;              // connected 8-vertex patterns: counted in global memory
constexpr unsigned long long MT_CHECK_NS = 4000;  // busy warps look for idle ones at most this often
constexpr float MT_MIN_DONATE_WORK = 2048.f;    // estimated leaves a handed-over range must carry
constexpr int MT_AGG_UNROLL = 4;                 // adjacency entries per lane per round (mt_tail_agg)

// A work unit: the children at positions [lo, hi) of the extension array of
// the node tr = (sub[0], .., sub[depth-1]) (hi < 0: all of them).  The node's
// array is rebuilt by the receiving warp by replaying the path: tr[j] is the
// entry at position pos[j] of ext_j (1 <= j < depth), and ESU's arrays are a
// deterministic function of those choices -- so a unit is a few dozen bytes
// whatever the length of its array.
struct MotifUnit {
    int32_t root_pos;
    int32_t depth;
    int32_t lo, hi;
    int32_t sub[MT_MAXK];
    int32_t pos[MT_MAXK];
};
static_assert(sizeof(MotifUnit) % 4 == 0, "unit must be word-sized");

struct MtWarp {                 // per-warp shared state
    int sub[MT_MAXK + 1];
    int code[MT_MAXK + 1];      // traversal code of tr[0..l-1]
    int cur[MT_MAXK + 1];
    int hi[MT_MAXK + 1];
    int len[MT_MAXK + 1];
    unsigned long long qpos;    // claimed queue position of a donated unit
    MotifUnit unit;
};

// Everything one warp needs to walk one unit.
struct MotifWalk {
    const int32_t* __restrict__ indptr;
    const int32_t* __restrict__ indices;
    const uint16_t* __restrict__ lut;
    int k;
    unsigned char* mk;          // marks, indexed mk[v - mbase]
    int mbase;
    int32_t* slab;              // this warp's extension arrays
    const long long* lvl_off;   // start of ext_l inside the slab (k-1 entries used)
    // donation (DONATE only): ring of idle warp ids and the warps' mailboxes
    // (mailbox of warp w at mbox + w * mbox_stride: MailHdr, then MotifUnit)
    Control* ctl;
    QSeq* ring_seq;
    int32_t* ring_ids;
    unsigned long long ring_cap;
    unsigned char* mbox;
    int mbox_stride;
    int donate_min;
    unsigned long long donate_after_ns;   // a unit splits only after running this long
    int* err;                   // device error flag
    // aggregated last two levels (mt_tail_agg): this warp's class counters
    // (mt_agg_words(k) words of shared memory), used when a node one level
    // above the leaves has at least agg_min entries left (agg == nullptr or
    // agg_min <= 0: never)
    uint32_t* agg;
    int agg_min;
    // host-monitored balancing (the paper's stop / redistribute / restart):
    // when the host raises ctl->stop, the walk writes its remaining work as
    // units to spill[] and unwinds
    bool monitor;
    MotifUnit* spill;
    unsigned long long spill_cap;
};

// 32-bit words of one warp's class counters for size k: HA, HB, E (one per
// class) and the adjacent-pair table P (classes x classes), classes = 2^(k-2)
__host__ __device__ constexpr int mt_agg_words(int k) {
    return k < 3 ? 0 : 3 * (1 << (k - 2)) + (1 << (k - 2)) * (1 << (k - 2));
}

__device__ __forceinline__ int mt_code_off(int i) { return i * (i - 1) / 2 - 1; }   // bits of v_i, i >= 2

// Shared counters of one block (single-graph kernel); ovf: the launch's
// overflow flag, raised if a counter wraps.
struct BlockSink {
    static constexpr bool kList = false;
    unsigned long long* c;
    int* ovf;
    __device__ __forceinline__ void add(int pid, unsigned long long v) { gpm_atomic_add_cc(&c[pid], v, ovf); }
};

// The launch's global counters (k = 8: 11,117 patterns do not fit a block's
// shared memory).
struct GlobalSink {
    static constexpr bool kList = false;
    unsigned long long* c;
    int* ovf;
    __device__ __forceinline__ void add(int pid, unsigned long long v) { gpm_atomic_add_cc(&c[pid], v, ovf); }
};

// Per-warp counters of the current unit (batched kernel), flushed per unit.
struct WarpSink {
    static constexpr bool kList = false;
    unsigned long long* c;
    int* ovf;
    __device__ __forceinline__ void add(int pid, unsigned long long v) { gpm_atomic_add_cc(&c[pid], v, ovf); }
};

// Listing (aggregate_store): every leaf becomes a record in the host ring
// (list_ring.cuh) instead of a count.  The class-counted tail is off when
// listing; add() is never reached and flags a consistency error if it is.
struct ListSink {
    static constexpr bool kList = true;
    ListRing ring;
    unsigned long long tail_seen;   // lane 0
    int* err;
    __device__ __forceinline__ void add(int, unsigned long long) { atomicCAS(err, 0, DEV_ECHECK + 9); }
};

// one leaf per active lane under pattern pid: one add per distinct pattern
template <class Sink>
__device__ __forceinline__ void mt_count_leaves(Sink& sink, bool active, int pid, int* err) {
    const int key = active ? pid : -1;
    const unsigned grp = __match_any_sync(GPM_FULL_MASK, key);
    const int lane = threadIdx.x & 31;
    if (active && lane == __ffs(grp) - 1) {
        if (pid == 0xffff) atomicExch(err, DEV_EINVAL);
        else sink.add(pid, (unsigned long long)__popc(grp));
    }
}

// First position in the sorted N(v) holding a vertex above `root`.  Sets
// rooted at `root` hold no smaller vertex, so neither their marks nor their
// extensions ever look below it: every adjacency scan starts here.  Found by
// the whole warp (every lane must call): 32 evenly spaced probes narrow the
// range 32-fold per round, so a list of up to 1,024 entries needs two rounds
// of independent loads instead of a chain of ten dependent ones.
__device__ __forceinline__ int mt_above(const int32_t* __restrict__ indptr, const int32_t* __restrict__ indices,
                                        int v, int root, int lane) {
    int lo = indptr[v], hi = indptr[v + 1];
    while (hi - lo > 32) {
        const int step = (hi - lo + 31) >> 5;
        const int p = lo + lane * step;
        const int c = __popc(__ballot_sync(GPM_FULL_MASK, p < hi && indices[p] <= root));
        if (c == 0) return lo;                  // indices[lo] > root
        const int nlo = lo + (c - 1) * step + 1;  // indices[nlo - 1] <= root
        hi = min(hi, lo + c * step);              // indices[hi] > root, or hi is the end
        lo = nlo;
    }
    const int p = lo + lane;
    return lo + __popc(__ballot_sync(GPM_FULL_MASK, p < hi && indices[p] <= root));
}

// Marks and traversal codes of a unit's prefix tr[0..pdepth-1] (W->sub).
// Vertices below the root are never marked (see mt_above); tr[j] itself is
// above the root for j >= 1, and the root's own mark is never read.
__device__ __forceinline__ void mt_setup_prefix(const MotifWalk& a, MtWarp* W, int pdepth, int lane) {
    const int root = W->sub[0];
    for (int j = 0; j < pdepth; j++) {
        const int v = W->sub[j];
        for (int t = mt_above(a.indptr, a.indices, v, root, lane) + lane; t < a.indptr[v + 1]; t += 32)
            a.mk[a.indices[t] - a.mbase] |= (unsigned char)(1u << j);
        __syncwarp();
    }
    if (lane < pdepth) a.mk[W->sub[lane] - a.mbase] |= 0x80;
    __syncwarp();
    if (lane == 0) {
        W->code[1] = 0;
        W->code[2] = 0;
        for (int i = 2; i < pdepth; i++)
            W->code[i + 1] = W->code[i] | ((a.mk[W->sub[i] - a.mbase] & ((1 << i) - 1)) << mt_code_off(i));
    }
    __syncwarp();
}

// Zero the prefix marks (deeper marks were undone by the pops).
__device__ __forceinline__ void mt_clear_prefix(const MotifWalk& a, MtWarp* W, int pdepth, int lane) {
    const int root = W->sub[0];
    for (int j = 0; j < pdepth; j++) {
        const int v = W->sub[j];
        for (int t = mt_above(a.indptr, a.indices, v, root, lane) + lane; t < a.indptr[v + 1]; t += 32)
            a.mk[a.indices[t] - a.mbase] = 0;
        __syncwarp();
    }
    if (lane < pdepth) a.mk[W->sub[lane] - a.mbase] = 0;
    __syncwarp();
}

// First extension set of root r: the suffix of the sorted N(r) above r
// (warp-wide, like mt_above).
__device__ __forceinline__ int mt_root_ext_begin(const int32_t* __restrict__ indptr, const int32_t* __restrict__ indices,
                                                 int r, int lane) {
    return mt_above(indptr, indices, r, r, lane);
}

// Traversal code of tr + w for a child w at depth l (its bits against
// tr[0..l-1] come from the marks).
__device__ __forceinline__ int mt_child_code(const MotifWalk& a, const MtWarp* W, int l, int w) {
    const int sigw = a.mk[w - a.mbase] & ((1 << l) - 1);
    return l >= 2 ? (W->code[l] | (sigw << mt_code_off(l))) : 0;
}

// Push child w = ext[c] of depth l: ext_{l+1} = ext[c+1 .. len) followed by
// the exclusive neighbours of w (above the root, unmarked by tr[0..l-1] and
// not in tr), and N(w) is marked with bit l.  wb..we: N(w) above the root.
__device__ __forceinline__ bool mt_push(const MotifWalk& a, MtWarp* W, int l, int c, const int32_t* ext, int w,
                                        int wb, int we, int codew, int lane) {
    int32_t* nxt = a.slab + a.lvl_off[l + 1];
    const int len = W->len[l];
    const int inh = len - (c + 1);
    if ((long long)inh + (we - wb) > a.lvl_off[l + 2] - a.lvl_off[l + 1]) {   // never, by the level sizes
        if (lane == 0) atomicCAS(a.err, 0, DEV_ECHECK + 5);
        return false;
    }
    for (int t = lane; t < inh; t += 32) nxt[t] = ext[c + 1 + t];
    const unsigned char low = (unsigned char)(0x80 | ((1u << l) - 1));
    int n_new = inh;
    for (int t0 = wb; t0 < we; t0 += 32) {
        const int t = t0 + lane;
        bool ex = false;
        int x = 0;
        if (t < we) {
            x = a.indices[t];
            const unsigned char m = a.mk[x - a.mbase];
            ex = (m & low) == 0;
            a.mk[x - a.mbase] = m | (unsigned char)(1u << l);
        }
        const unsigned bal = __ballot_sync(GPM_FULL_MASK, ex);
        if (ex) nxt[n_new + __popc(bal & gpm_lanemask_lt())] = x;
        n_new += __popc(bal);
    }
    __syncwarp();
    if (lane == 0) {
        a.mk[w - a.mbase] |= 0x80;
        W->sub[l] = w;
        W->code[l + 1] = codew;
        W->len[l + 1] = n_new;
        W->cur[l + 1] = 0;
        W->hi[l + 1] = n_new;
    }
    __syncwarp();
    return true;
}

// Set up unit u (in W->unit): marks and array of the root, then the path
// replayed push by push; levels above the unit's own are left exhausted
// (cur = hi = the chosen position + 1).  Returns the array of the unit's
// node, or nullptr if the path does not match the graph (device error).
__device__ __forceinline__ const int32_t* mt_replay(const MotifWalk& a, MtWarp* W, int lane) {
    const int root = W->unit.sub[0];
    const int depth = W->unit.depth;
    if (depth < 1 || depth > max(a.k - 2, 1)) {
        if (lane == 0) atomicCAS(a.err, 0, DEV_ECHECK + 3);
        return nullptr;
    }
    if (lane == 0) W->sub[0] = root;
    __syncwarp();
    mt_setup_prefix(a, W, 1, lane);
    const int b = mt_root_ext_begin(a.indptr, a.indices, root, lane);
    const int32_t* ext = a.indices + b;
    if (lane == 0) W->len[1] = a.indptr[root + 1] - b;
    __syncwarp();
    for (int l = 1; l < depth; l++) {
        const int c = W->unit.pos[l];
        if (c < 0 || c >= W->len[l]) {
            if (lane == 0) atomicCAS(a.err, 0, DEV_ECHECK + 1);
            return nullptr;
        }
        const int w = ext[c];
        if (w != W->unit.sub[l]) {
            if (lane == 0) atomicCAS(a.err, 0, DEV_ECHECK + 2);
            return nullptr;
        }
        const int codew = mt_child_code(a, W, l, w);
        const int wb = mt_above(a.indptr, a.indices, w, root, lane), we = a.indptr[w + 1];
        if (!mt_push(a, W, l, c, ext, w, wb, we, codew, lane)) return nullptr;
        if (lane == 0) {
            W->cur[l] = c + 1;
            W->hi[l] = c + 1;
        }
        ext = a.slab + a.lvl_off[l + 1];
    }
    if (W->unit.lo < 0 || W->unit.lo > W->len[depth]) {
        if (lane == 0) atomicCAS(a.err, 0, DEV_ECHECK + 6);
        return nullptr;
    }
    if (lane == 0) {
        W->cur[depth] = W->unit.lo;
        W->hi[depth] = W->unit.hi < 0 ? W->len[depth] : min(W->unit.hi, W->len[depth]);
    }
    __syncwarp();
    return ext;
}

// Split point of children [from, to) of a node whose array has len entries:
// a child's subtree grows about like (len - c)^e (e = levels below it), so
// [from, mid) and [mid, to) carry about the same work when
// (len - mid)^(e+1) is the mean of (len - from)^(e+1) and (len - to)^(e+1).
__device__ __forceinline__ int mt_split(int from, int to, int len, int e) {
    const float A = (float)(len - from), B = (float)(len - to);
    const float q = (float)(e + 1);
    const float m = __powf(0.5f * (__powf(A, q) + __powf(fmaxf(B, 1.0f), q)), 1.0f / q);
    const int mid = len - (int)ceilf(m);
    return max(from + 1, min(mid, to - 1));
}

// Hand the later children of the shallowest splittable level to a
// registered idle warp (lane 0 only; a cold path, kept out of line).  The
// split balances estimated work; the unit carries the path, not the array.
__device__ __noinline__ static void mt_donate(Control* ctl, QSeq* ring_seq, int32_t* ring_ids,
                                              unsigned long long ring_cap, unsigned char* mbox, int mbox_stride,
                                              int donate_min, int k, MtWarp* W, int pdepth, int l, int root_pos) {
    for (int t = pdepth; t <= l; t++) {
        const int from = W->cur[t], to = W->hi[t];
        if (to - from < max(donate_min, 2)) continue;
        const int len = W->len[t];
        const int mid = mt_split(from, to, len, k - 1 - t);
        // estimated work of the later part: sum of (len - c)^e, e = levels below
        const float q = (float)(k - t);
        const float est = (__powf((float)(len - mid), q) - __powf(fmaxf((float)(len - to), 1.0f), q)) / q;
        if (est < MT_MIN_DONATE_WORK) continue;
        int wid;
        if (!gpm_idle_claim(ring_seq, ring_ids, ring_cap, &ctl->q_head, &wid)) return;
        if (wid < 0 || (unsigned long long)wid >= ring_cap) {   // never: ids are registered warps
            atomicCAS(&ctl->error, 0, DEV_ECHECK + 4);
            return;
        }
        unsigned char* box = mbox + (size_t)wid * mbox_stride;
        MotifUnit* u = reinterpret_cast<MotifUnit*>(box + sizeof(MailHdr));
        u->root_pos = root_pos;
        u->depth = t;
        u->lo = mid;
        u->hi = to;
        for (int z = 0; z < MT_MAXK; z++) {
            u->sub[z] = z < t ? W->sub[z] : -1;
            u->pos[z] = (z >= 1 && z < t) ? W->cur[z] - 1 : -1;
        }
        W->hi[t] = mid;
        atomicAdd((unsigned long long*)&ctl->pending, 1ull);
        __threadfence();
        atomicExch(&reinterpret_cast<MailHdr*>(box)->ready, 1);
        atomicAdd(&ctl->donations, 1ull);
        return;
    }
}

// The last two levels below a node tr of size k-2 (level l = k-2, array ext
// of length L), counted by class instead of leaf by leaf.  Its children are
// w = ext[c], c in A = [cur, hi); child w is the (k-1)-set tr+w, and its
// k-vertex leaves are tr+w+x for every later entry x = ext[c'] (c' > c) and
// for every exclusive neighbour x of w (above the root, neither in tr nor
// adjacent to it).  The induced graph of a leaf is fixed by code(tr), the
// class of w and of x -- an entry's class is its adjacency to tr, mark bits
// 0 .. k-3 -- and whether w and x are adjacent.  So:
//
//   * pairs {w, x} of entries: with HA / HB the class histograms of A and of
//     B = [hi, L), the pairs of classes {s1, s2} number C(HA[s],2) (s1 = s2)
//     or HA[s1] HA[s2] within A, plus HA[s1] HB[s2] (+ HA[s2] HB[s1]) across;
//     of these, the adjacent ones are found by scanning N(w) for every w in A
//     (an entry x of A counted from its smaller endpoint only, an entry of B
//     always), and the rest are non-adjacent;
//   * exclusive neighbours: counted per class of w during the same scans.
//
// One scan of N(w) per child replaces the per-leaf walk over the later
// entries (quadratic in L).  Mark bits 6 and 5 flag the entries of A u B and
// of B during the call (free at this level: tr uses bits 0 .. k-3 and 7).
// The adjacency lists of 32 children at a time are scanned as one flattened
// range, so every lane has an entry whatever the degrees.
template <class Sink>
__device__ __noinline__ void mt_tail_agg(const MotifWalk& a, MtWarp* W, int l, const int32_t* ext, int root,
                                         Sink& sink, unsigned long long& leaves, unsigned long long& scanned,
                                         int lane) {
    const int C = 1 << l;                        // classes: adjacency to tr[0 .. l-1]
    const unsigned lowtr = (unsigned)C - 1u;
    const int a0 = W->cur[l], a1 = W->hi[l], L = W->len[l];
    uint32_t* HA = a.agg;
    uint32_t* HB = HA + C;
    uint32_t* E = HB + C;
    uint32_t* P = E + C;                         // P[s1 * C + s2], s1 <= s2
    for (int i = lane; i < 3 * C + C * C; i += 32) HA[i] = 0u;
    __syncwarp();
    // classes of A and B, and their range marks
    for (int j0 = a0; j0 < L; j0 += 32) {
        const int j = j0 + lane;
        int key = -1;
        if (j < L) {
            const int x = ext[j];
            const unsigned char m = a.mk[x - a.mbase];
            a.mk[x - a.mbase] = m | (unsigned char)(j < a1 ? 0x40 : 0x60);
            key = (int)(m & lowtr) + (j < a1 ? 0 : C);
        }
        const unsigned grp = __match_any_sync(GPM_FULL_MASK, key);
        if (key >= 0 && lane == __ffs(grp) - 1) HA[key] += (uint32_t)__popc(grp);
    }
    __syncwarp();
    // scan N(w) for the children, 32 at a time
    for (int c0 = a0; c0 < a1; c0 += 32) {
        const int c = c0 + lane;
        int w = 0, sw = 0, b = 0, e = 0;
        if (c < a1) {
            w = ext[c];
            sw = a.mk[w - a.mbase] & lowtr;
            int lo = a.indptr[w], hi = a.indptr[w + 1];
            e = hi;
            while (lo < hi) {                    // first neighbour above the root
                const int mid = (lo + hi) >> 1;
                if (a.indices[mid] <= root) lo = mid + 1; else hi = mid;
            }
            b = lo;
        }
        const int len = e - b;
        int incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(GPM_FULL_MASK, incl, o);
            if (lane >= o) incl += y;
        }
        const int pre = incl - len;
        const int total = __shfl_sync(GPM_FULL_MASK, incl, 31);
        if (lane == 0) scanned += (unsigned)total;
        // MT_AGG_UNROLL entries per lane per round, their loads issued
        // together (the mark loads are random and latency-bound)
        for (int f0 = 0; f0 < total; f0 += 32 * MT_AGG_UNROLL) {
            int xs[MT_AGG_UNROLL], wts[MT_AGG_UNROLL], sts[MT_AGG_UNROLL];
#pragma unroll
            for (int u = 0; u < MT_AGG_UNROLL; u++) {
                const int f = f0 + 32 * u + lane;
                int t = 0;                       // owner: the last lane with pre <= f
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int pc = __shfl_sync(GPM_FULL_MASK, pre, t + step);
                    if (pc <= f) t += step;
                }
                wts[u] = __shfl_sync(GPM_FULL_MASK, w, t);
                sts[u] = __shfl_sync(GPM_FULL_MASK, sw, t);
                const int bt = __shfl_sync(GPM_FULL_MASK, b, t);
                const int pt = __shfl_sync(GPM_FULL_MASK, pre, t);
                xs[u] = f < total ? a.indices[bt + (f - pt)] : -1;
            }
            unsigned char ms[MT_AGG_UNROLL];
#pragma unroll
            for (int u = 0; u < MT_AGG_UNROLL; u++) ms[u] = xs[u] >= 0 ? a.mk[xs[u] - a.mbase] : (unsigned char)0;
#pragma unroll
            for (int u = 0; u < MT_AGG_UNROLL; u++) {
                bool ex = false;
                if (xs[u] >= 0) {
                    const unsigned m = ms[u];
                    if ((m & (lowtr | 0x80u)) == 0) {
                        ex = true;                   // exclusive neighbour of w
                    } else if ((m & 0x40u) && ((m & 0x20u) || xs[u] > wts[u])) {
                        const int s2 = (int)(m & lowtr);   // adjacent pair of entries (rare)
                        atomicAdd(&P[min(sts[u], s2) * C + max(sts[u], s2)], 1u);
                    }
                }
                // exclusive neighbours per child: the lanes of one child are
                // contiguous, so the first lane of each child's run adds the
                // run's count (children of one class may share a counter)
                const unsigned exm = __ballot_sync(GPM_FULL_MASK, ex);
                const int wprev = __shfl_up_sync(GPM_FULL_MASK, wts[u], 1);
                const bool head = xs[u] >= 0 && (lane == 0 || wprev != wts[u]);
                const unsigned heads = __ballot_sync(GPM_FULL_MASK, head);
                if (head) {
                    const unsigned later = heads & ~((2u << lane) - 1u);   // heads above this lane
                    const unsigned run = (later ? ((1u << (__ffs(later) - 1)) - 1u) : 0xffffffffu) & ~((1u << lane) - 1u);
                    const unsigned cnt = (unsigned)__popc(exm & run);
                    if (cnt) atomicAdd(&E[sts[u]], cnt);
                }
            }
        }
    }
    __syncwarp();
    // patterns: w = v_l (bits at mt_code_off(l), none for l = 1), x = v_{l+1}
    const int codetr = l >= 2 ? W->code[l] : 0;
    const int offx = mt_code_off(l + 1);
    unsigned long long mine = 0;
    for (int idx = lane; idx < C * C; idx += 32) {
        const int s1 = idx >> l, s2 = idx & (C - 1);
        if (s1 > s2) continue;
        const unsigned long long ha1 = HA[s1], ha2 = HA[s2], hb1 = HB[s1], hb2 = HB[s2];
        const unsigned long long within = s1 == s2 ? ha1 * (ha1 - (ha1 ? 1 : 0)) / 2 : ha1 * ha2;
        const unsigned long long across = ha1 * hb2 + (s1 != s2 ? ha2 * hb1 : 0ull);
        const unsigned long long adj = P[idx];
        const unsigned long long non = within + across - adj;
        const int cw = codetr | (l >= 2 ? (s1 << mt_code_off(l)) : 0);
        if (non) {
            const int pid = a.lut[cw | (s2 << offx)];
            if (pid == 0xffff) atomicExch(a.err, DEV_EINVAL);
            else sink.add(pid, non);
            mine += non;
        }
        if (adj) {
            const int pid = a.lut[cw | ((s2 | C) << offx)];
            if (pid == 0xffff) atomicExch(a.err, DEV_EINVAL);
            else sink.add(pid, adj);
            mine += adj;
        }
    }
    for (int s1 = lane; s1 < C; s1 += 32) {
        if (!E[s1]) continue;
        const int cw = codetr | (l >= 2 ? (s1 << mt_code_off(l)) : 0);
        const int pid = a.lut[cw | (C << offx)];
        if (pid == 0xffff) atomicExch(a.err, DEV_EINVAL);
        else sink.add(pid, (unsigned long long)E[s1]);
        mine += E[s1];
    }
    leaves += mine;
    // drop the range marks
    for (int j = a0 + lane; j < L; j += 32) a.mk[ext[j] - a.mbase] &= (unsigned char)0x9f;
    __syncwarp();
    if (lane == 0) W->cur[l] = a1;
    __syncwarp();
}

// The leaves below the (l+1)-set tr + w (tr = W->sub[0 .. l-1]) as records
// (tr, w, x; pattern id): first the exclusive neighbours x of w (adjacent to
// w alone among the set: one pattern), marking every neighbour of w on the
// way, then the remaining entries x of ext_l, whose adjacency to the set is
// read from the marks.  The same leaves, in the same classes, as the
// counting path above.
template <class Sink>
__device__ __forceinline__ void mt_list_leaves(const MotifWalk& a, MtWarp* W, int l, int c, const int32_t* ext,
                                               int w, int wb, int we, int codew, Sink& sink,
                                               unsigned long long& unit_leaves, int lane) {
    const int offk = mt_code_off(l + 1);
    const unsigned char low = (unsigned char)(0x80 | ((1u << l) - 1));
    const int pid_x = a.lut[codew | ((1 << l) << offk)];
    if (pid_x == 0xffff && lane == 0) atomicExch(a.err, DEV_EINVAL);
    for (int t0 = wb; t0 < we; t0 += 32) {
        const int t = t0 + lane;
        bool act = false;
        int x = 0;
        if (t < we) {
            x = a.indices[t];
            const unsigned char m = a.mk[x - a.mbase];
            act = (m & low) == 0;
            a.mk[x - a.mbase] = m | (unsigned char)(1u << l);
        }
        unit_leaves += act ? 1u : 0u;
        lr_emit(sink.ring, sink.tail_seen, W->sub, l, w, x, pid_x, act, lane);
    }
    __syncwarp();
    const int len = W->len[l];
    const unsigned lowk = (1u << (l + 1)) - 1u;
    for (int j0 = c + 1; j0 < len; j0 += 32) {
        const int j = j0 + lane;
        const bool act = j < len;
        int pid = 0, x = 0;
        if (act) {
            x = ext[j];
            const int sig = a.mk[x - a.mbase] & lowk;
            pid = a.lut[codew | (sig << offk)];
            if (pid == 0xffff) atomicExch(a.err, DEV_EINVAL);
            unit_leaves++;
        }
        lr_emit(sink.ring, sink.tail_seen, W->sub, l, w, x, pid, act, lane);
    }
    __syncwarp();
    for (int t = wb + lane; t < we; t += 32) a.mk[a.indices[t] - a.mbase] &= (unsigned char)~(1u << l);
    __syncwarp();
}

// Walk the unit whose node is at depth pdepth (W->cur/hi/len[pdepth] set,
// unit_ext = its extension array).  Returns false if it stopped on a device
// error (marks are then left dirty).  unit_leaves: lane-private leaf count.
template <bool DONATE, class Sink>
__device__ __forceinline__ bool mt_walk(const MotifWalk& a, MtWarp* W, int pdepth, int root, int root_pos, const int32_t* unit_ext,
                        Sink& sink, unsigned long long& unit_leaves, unsigned long long& scanned, int lane) {
    const int k = a.k;
    int l = pdepth;
    const unsigned long long t_start = DONATE ? gpm_globaltimer() : 0ull;
    unsigned long long last_check = t_start;   // lane 0
    for (;;) {
        const int c = W->cur[l];
        if (c >= W->hi[l]) {
            if (l == pdepth) break;
            // pop tr[l-1] (pushed at depth l-1)
            const int w = W->sub[l - 1];
            const int wb = mt_above(a.indptr, a.indices, w, root, lane), we = a.indptr[w + 1];
            if (lane == 0) scanned += (unsigned)(we - wb);
            for (int t = wb + lane; t < we; t += 32)
                a.mk[a.indices[t] - a.mbase] &= (unsigned char)~(1u << (l - 1));
            __syncwarp();
            if (lane == 0) a.mk[w - a.mbase] &= 0x7f;
            __syncwarp();
            l--;
            continue;
        }
        const int32_t* ext = l == pdepth ? unit_ext : a.slab + a.lvl_off[l];
        if (l + 2 == k && a.agg_min > 0 && W->len[l] - c >= a.agg_min) {
            // one level above the leaves with many entries left: count the
            // remaining children's leaves by class (then pop)
            __syncwarp();
            mt_tail_agg(a, W, l, ext, root, sink, unit_leaves, scanned, lane);
            continue;
        }
        const int w = ext[c];
        __syncwarp();                       // every lane has read cur[l] before it moves on
        if (lane == 0) W->cur[l] = c + 1;
        const int codew = mt_child_code(a, W, l, w);
        const int wb = mt_above(a.indptr, a.indices, w, root, lane), we = a.indptr[w + 1];
        if (lane == 0 && l + 1 != k - 1) scanned += (unsigned)(we - wb);
        const unsigned char low = (unsigned char)(0x80 | ((1u << l) - 1));
        if (l + 1 == k - 1) {
            if constexpr (Sink::kList) {
                // ---- last level, listing: a record per leaf of tr + w
                mt_list_leaves(a, W, l, c, ext, w, wb, we, codew, sink, unit_leaves, lane);
            } else {
                // ---- last level: leaves of the (k-1)-set tr + w
                const int offk = mt_code_off(l + 1);
                if (lane == 0) scanned += 2ull * (unsigned)(we - wb);
                int excl = 0;
                for (int t = wb + lane; t < we; t += 32) {
                    const int x = a.indices[t];
                    const unsigned char m = a.mk[x - a.mbase];
                    excl += (m & low) == 0 ? 1 : 0;
                    a.mk[x - a.mbase] = m | (unsigned char)(1u << l);
                }
                excl = __reduce_add_sync(GPM_FULL_MASK, (unsigned)excl);
                __syncwarp();
                if (excl && lane == 0) {
                    const int pid = a.lut[codew | ((1 << l) << offk)];
                    if (pid == 0xffff) atomicExch(a.err, DEV_EINVAL);
                    else sink.add(pid, (unsigned long long)excl);
                    unit_leaves += (unsigned)excl;
                }
                const int len = W->len[l];
                const unsigned lowk = (1u << (l + 1)) - 1u;
                for (int j0 = c + 1; j0 < len; j0 += 32) {
                    const int j = j0 + lane;
                    const bool act = j < len;
                    int pid = 0;
                    if (act) {
                        const int x = ext[j];
                        const int sig = a.mk[x - a.mbase] & lowk;
                        pid = a.lut[codew | (sig << offk)];
                        unit_leaves++;
                    }
                    mt_count_leaves(sink, act, pid, a.err);
                }
                __syncwarp();
                for (int t = wb + lane; t < we; t += 32) a.mk[a.indices[t] - a.mbase] &= (unsigned char)~(1u << l);
                __syncwarp();
            }
        } else {
            // ---- push w: ext_{l+1} = ext_l[c+1:] ++ exclusive neighbours of w
            if (!mt_push(a, W, l, c, ext, w, wb, we, codew, lane)) return false;
            l++;
        }

        if (!DONATE && a.monitor) {
            Control* ctl = a.ctl;
            int err = 0, stop = 0;
            const unsigned long long now = gpm_globaltimer();
            if (lane == 0 && now - last_check >= MT_CHECK_NS) {
                last_check = now;
                err = *(volatile int*)&ctl->error;
                stop = atomicAdd(&ctl->stop, 0);
            }
            err = __shfl_sync(GPM_FULL_MASK, err, 0);
            if (err) return false;
            if (__shfl_sync(GPM_FULL_MASK, stop, 0)) {
                // spill every level's remaining children as a unit (the path,
                // as a hand-off carries it), then unwind through the emptied
                // ranges, popping the marks on the way
                if (lane == 0) {
                    for (int t = pdepth; t <= l; t++) {
                        if (W->cur[t] >= W->hi[t]) continue;
                        const unsigned long long slot = atomicAdd(&ctl->spill_n, 1ull);
                        if (slot >= a.spill_cap) {   // never: one unit per level per warp fits
                            atomicCAS(&ctl->error, 0, DEV_ECHECK + 7);
                            break;
                        }
                        MotifUnit* u = a.spill + slot;
                        u->root_pos = root_pos;
                        u->depth = t;
                        u->lo = W->cur[t];
                        u->hi = W->hi[t];
                        for (int z = 0; z < MT_MAXK; z++) {
                            u->sub[z] = z < t ? W->sub[z] : -1;
                            u->pos[z] = (z >= 1 && z < t) ? W->cur[z] - 1 : -1;
                        }
                    }
                    for (int t = pdepth; t <= l; t++) W->hi[t] = W->cur[t];
                }
                __syncwarp();
            }
        }
        // donation check: after every step, but at most once per
        // MT_CHECK_NS (the lines it reads are shared by every warp)
        if (DONATE) {
            Control* ctl = a.ctl;
            int err = 0, want = 0;
            const unsigned long long now = gpm_globaltimer();
            if (lane == 0 && now - last_check >= MT_CHECK_NS) {
                last_check = now;
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
            if (want && lane == 0)
                mt_donate(ctl, a.ring_seq, a.ring_ids, a.ring_cap, a.mbox, a.mbox_stride, a.donate_min, k, W, pdepth,
                          l, root_pos);
            __syncwarp();
        }
    }
    return true;
}

}  // namespace gpm
