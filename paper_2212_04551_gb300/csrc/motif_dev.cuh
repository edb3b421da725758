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

namespace gpm {

constexpr int MT_MAXK = GPM_MOTIF_MAX_K;
constexpr int MT_LIST = 1024;                  // entries carried by one donated unit
constexpr int MT_MAXPAT = 853;                 // connected 7-vertex patterns
constexpr int MT_PAYLOAD_OFF = 64;             // payload offset inside a mailbox (after MailHdr + MotifUnit)

struct MotifUnit {
    int32_t root_pos;
    int32_t depth;              // |tr| of the donated node
    int32_t len;                // entries in its list (the node's extension-array suffix)
    int32_t child_hi;           // children to expand: list positions [0, child_hi)
    int32_t sub[MT_MAXK];
    int32_t list_off;           // >= 0: the list is indices[list_off ..] (a root's own
                                // extension set); < 0: it is the queue slot's payload
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
    // (mailbox of warp w at mbox + w * mbox_stride: MailHdr, MotifUnit, then
    // MT_LIST payload ints at MT_PAYLOAD_OFF)
    Control* ctl;
    QSeq* ring_seq;
    int32_t* ring_ids;
    unsigned long long ring_cap;
    unsigned char* mbox;
    int mbox_stride;
    int donate_min;
    unsigned long long donate_after_ns;   // a unit splits only after running this long
    int* err;                   // device error flag
};

__device__ __forceinline__ int mt_code_off(int i) { return i * (i - 1) / 2 - 1; }   // bits of v_i, i >= 2

// Shared counters of one block (single-graph kernel).
struct BlockSink {
    unsigned long long* c;
    __device__ __forceinline__ void add(int pid, unsigned long long v) { atomicAdd(&c[pid], v); }
};

// Per-warp counters of the current unit (batched kernel), flushed per unit.
struct WarpSink {
    unsigned long long* c;
    __device__ __forceinline__ void add(int pid, unsigned long long v) { atomicAdd(&c[pid], v); }
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
// extensions ever look below it: every adjacency scan starts here.  Short
// lists are scanned whole (a search would cost more than it skips).
__device__ __forceinline__ int mt_above(const int32_t* __restrict__ indptr, const int32_t* __restrict__ indices,
                                        int v, int root) {
    int lo = indptr[v], hi = indptr[v + 1];
    if (hi - lo <= 64) return lo;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (indices[mid] <= root) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Marks and traversal codes of a unit's prefix tr[0..pdepth-1] (W->sub).
// Vertices below the root are never marked (see mt_above); tr[j] itself is
// above the root for j >= 1, and the root's own mark is never read.
__device__ __forceinline__ void mt_setup_prefix(const MotifWalk& a, MtWarp* W, int pdepth, int lane) {
    const int root = W->sub[0];
    for (int j = 0; j < pdepth; j++) {
        const int v = W->sub[j];
        for (int t = mt_above(a.indptr, a.indices, v, root) + lane; t < a.indptr[v + 1]; t += 32)
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
        for (int t = mt_above(a.indptr, a.indices, v, root) + lane; t < a.indptr[v + 1]; t += 32)
            a.mk[a.indices[t] - a.mbase] = 0;
        __syncwarp();
    }
    if (lane < pdepth) a.mk[W->sub[lane] - a.mbase] = 0;
    __syncwarp();
}

// First extension set of root r: the suffix of the sorted N(r) above r.
__device__ __forceinline__ int mt_root_ext_begin(const int32_t* __restrict__ indptr, const int32_t* __restrict__ indices,
                                                 int r) {
    int lo = indptr[r], hi = indptr[r + 1];
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (indices[mid] <= r) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Walk the unit whose node is at depth pdepth (W->cur/hi/len[pdepth] set,
// unit_ext = its extension array).  Returns false if it stopped on a device
// error (marks are then left dirty).  unit_leaves: lane-private leaf count.
template <bool DONATE, class Sink>
__device__ bool mt_walk(const MotifWalk& a, MtWarp* W, int pdepth, int root, int root_pos, const int32_t* unit_ext,
                        Sink& sink, unsigned long long& unit_leaves, int lane) {
    const int k = a.k;
    int l = pdepth;
    int iter = 0;
    const unsigned long long t_start = DONATE ? gpm_globaltimer() : 0ull;
    for (;;) {
        const int c = W->cur[l];
        if (c >= W->hi[l]) {
            if (l == pdepth) break;
            // pop tr[l-1] (pushed at depth l-1)
            const int w = W->sub[l - 1];
            for (int t = mt_above(a.indptr, a.indices, w, root) + lane; t < a.indptr[w + 1]; t += 32)
                a.mk[a.indices[t] - a.mbase] &= (unsigned char)~(1u << (l - 1));
            __syncwarp();
            if (lane == 0) a.mk[w - a.mbase] &= 0x7f;
            __syncwarp();
            l--;
            continue;
        }
        const int32_t* ext = l == pdepth ? unit_ext : a.slab + a.lvl_off[l];
        const int w = ext[c];
        if (lane == 0) W->cur[l] = c + 1;
        const int sigw = a.mk[w - a.mbase] & ((1 << l) - 1);
        const int codew = l >= 2 ? (W->code[l] | (sigw << mt_code_off(l))) : 0;
        const int wb = mt_above(a.indptr, a.indices, w, root), we = a.indptr[w + 1];
        const unsigned char low = (unsigned char)(0x80 | ((1u << l) - 1));
        if (l + 1 == k - 1) {
            // ---- last level: leaves of the (k-1)-set tr + w
            const int offk = mt_code_off(l + 1);
            int excl = 0;
            for (int t = wb + lane; t < we; t += 32) {
                const int x = a.indices[t];
                const unsigned char m = a.mk[x - a.mbase];
                excl += (x > root && (m & low) == 0) ? 1 : 0;
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
        } else {
            // ---- push w: ext_{l+1} = ext_l[c+1:] ++ exclusive neighbours of w
            int32_t* nxt = a.slab + a.lvl_off[l + 1];
            const int len = W->len[l];
            const int inh = len - (c + 1);
            for (int t = lane; t < inh; t += 32) nxt[t] = ext[c + 1 + t];
            int n_new = inh;
            for (int t0 = wb; t0 < we; t0 += 32) {
                const int t = t0 + lane;
                bool ex = false;
                int x = 0;
                if (t < we) {
                    x = a.indices[t];
                    const unsigned char m = a.mk[x - a.mbase];
                    ex = x > root && (m & low) == 0;
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
            l++;
        }

        if (DONATE && (++iter & 7) == 0) {
            Control* ctl = a.ctl;
            int err = 0, want = 0;
            if (lane == 0) {
                err = *(volatile int*)&ctl->error;
                if (gpm_globaltimer() - t_start > a.donate_after_ns) {
                    const unsigned long long qh = *(volatile unsigned long long*)&ctl->q_head;
                    const unsigned long long qt = *(volatile unsigned long long*)&ctl->q_tail;
                    want = qt > qh;   // a registered idle warp is waiting
                }
            }
            err = __shfl_sync(GPM_FULL_MASK, err, 0);
            if (err) return false;
            want = __shfl_sync(GPM_FULL_MASK, want, 0);
            if (want) {
                // shallowest level with enough unexpanded children: give away the
                // upper half (its list suffix travels in the receiver's mailbox)
                for (int t = pdepth; t <= l; t++) {
                    const int from = W->cur[t], to = W->hi[t], len = W->len[t];
                    const int rem = to - from;
                    if (rem < max(a.donate_min, 2)) continue;
                    int start = from + (rem - rem / 2);
                    start = max(start, len - MT_LIST);
                    if (start >= to) continue;
                    int wid = -1;
                    if (lane == 0 && !gpm_idle_claim(a.ring_seq, a.ring_ids, a.ring_cap, &ctl->q_head, &wid)) wid = -1;
                    wid = __shfl_sync(GPM_FULL_MASK, wid, 0);
                    if (wid < 0) break;
                    unsigned char* box = a.mbox + (size_t)wid * a.mbox_stride;
                    int32_t* dst = reinterpret_cast<int32_t*>(box + MT_PAYLOAD_OFF);
                    const int32_t* src = t == pdepth ? unit_ext : a.slab + a.lvl_off[t];
                    for (int z = start + lane; z < len; z += 32) dst[z - start] = src[z];
                    if (lane == 0) {
                        MotifUnit u;
                        u.root_pos = root_pos;
                        u.depth = t;
                        u.len = len - start;
                        u.child_hi = to - start;
                        for (int z = 0; z < MT_MAXK; z++) u.sub[z] = z < t ? W->sub[z] : -1;
                        u.list_off = -1;
                        *reinterpret_cast<MotifUnit*>(box + sizeof(MailHdr)) = u;
                        W->hi[t] = start;
                        atomicAdd((unsigned long long*)&ctl->pending, 1ull);
                    }
                    __threadfence();
                    __syncwarp();
                    if (lane == 0) {
                        atomicExch(&reinterpret_cast<MailHdr*>(box)->ready, 1);
                        atomicAdd(&ctl->donations, 1ull);
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
