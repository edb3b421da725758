// motif.cu -- induced k-motif counting on the device (Algorithm 4, motif
// counting; aggregate_pattern of Section 4.3.4).
//
// Hot-path rows A2, A5 (extension step), A6 (pattern aggregation), A7 (per-
// warp DFS stack in HBM), A8 (work donation) and A9 (counter reduction).
//
// The paper extends a traversal from the adjacency of all its vertices
// (extend(TE, 0, TE.len)), keeps canonical candidates only (filter
// "canonical", an Arabesque-style test), and at |tr| = k-1 maps every
// traversal + extension to its pattern through the edge-bitmap dictionary.
// This kernel reaches the same set of connected induced subgraphs -- each
// exactly once -- with the exclusive-neighbourhood extension of ESU
// (Wernicke 2006) instead of re-filtering N(tr) at every level:
//
//   * root r = the smallest vertex of the subgraph; ext_1 = {u in N(r): u > r};
//   * choosing w = ext_l[i] gives ext_{l+1} = ext_l[i+1:] followed by the
//     exclusive neighbours of w: u in N(w), u > r, u not in the traversal and
//     not adjacent to any traversal vertex.
//
// Per warp, a byte per vertex ("mark", in HBM) records which traversal
// positions each vertex is adjacent to (bit j <=> adjacent to tr[j]) and
// whether it is in the traversal (bit 7).  Marks make the exclusivity test
// and the traversal edge bitmap (the paper's induce step) O(1) per
// candidate: pushing w marks N(w) once, popping it unmarks N(w).
//
// The traversal code is the paper's layout (Section 4.3.4): the v0-v1 edge is
// implicit, then v_i's edges to v_0..v_{i-1} at bit offset i(i-1)/2 - 1.
// At |tr| = k-1 -- the last level -- no extension array is built: the k-vertex
// leaves are (a) the remaining entries of the parent's extension array, whose
// code bits are read from the marks, and (b) the exclusive neighbours of the
// newest vertex, whose code is the same for all of them.  Each leaf is looked
// up in the pattern table and counted in per-block shared counters with one
// shared atomic per distinct pattern per warp step (__match_any_sync).
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "common.cuh"

namespace gpm {

constexpr int MT_MAXK = GPM_MOTIF_MAX_K;
constexpr int MT_LIST = 1024;                  // entries carried by one donated unit
constexpr unsigned long long MT_QUEUE_CAP = 4096;
constexpr int MT_MAXPAT = 853;                 // connected 7-vertex patterns

struct MotifUnit {
    int32_t root_pos;
    int32_t depth;              // |tr| of the donated node
    int32_t len;                // entries in the payload list (its extension array suffix)
    int32_t child_hi;           // children to expand: list positions [0, child_hi)
    int32_t sub[MT_MAXK];
    int32_t list_off;           // >= 0: the list is indices[list_off ..] (a root's own
                                // extension set); < 0: it is the slot's payload
};
static_assert(sizeof(MotifUnit) % 4 == 0, "unit must be word-sized");

struct MotifParams {
    const int32_t* __restrict__ indptr;
    const int32_t* __restrict__ indices;
    const int32_t* __restrict__ roots;
    long long n_roots;
    int n;
    int k;
    int npat;
    const uint16_t* __restrict__ lut;
    Control* ctl;
    QSeq* qseq;
    MotifUnit* qunits;
    int32_t* qpayload;          // MT_LIST ints per slot
    unsigned long long qcap;
    unsigned long long* per_root;
    unsigned char* marks;       // n bytes per warp
    int32_t* slab;              // slab_ints per warp
    long long slab_ints;
    long long lvl_off[MT_MAXK + 1];   // start of ext_l inside a warp's slab
    int donate, donate_min;
    unsigned long long max_idle_ns;
    unsigned long long* counts; // npat global counters
};

struct MtWarp {                 // per-warp shared state
    int sub[MT_MAXK + 1];
    int code[MT_MAXK + 1];      // traversal code of tr[0..l-1]
    int cur[MT_MAXK + 1];
    int hi[MT_MAXK + 1];
    int len[MT_MAXK + 1];
    unsigned long long qpos;    // claimed queue position of a donated unit
    MotifUnit unit;
};

__device__ __forceinline__ int code_off(int i) { return i * (i - 1) / 2 - 1; }   // bits of v_i, i >= 2

// count one leaf per active lane under pattern pid (warp-aggregated shared atomics)
__device__ __forceinline__ void count_leaves(unsigned long long* bcnt, bool active, int pid, int* err_flag) {
    const int key = active ? pid : -1;
    const unsigned grp = __match_any_sync(GPM_FULL_MASK, key);
    const int lane = threadIdx.x & 31;
    if (active && lane == __ffs(grp) - 1) {
        if (pid == 0xffff) atomicExch(err_flag, DEV_EINVAL);
        else atomicAdd(&bcnt[pid], (unsigned long long)__popc(grp));
    }
}

__device__ __forceinline__ void mark_or(unsigned char* mk, const int32_t* __restrict__ indices, int beg, int end,
                                        unsigned char bit, int lane) {
    for (int t = beg + lane; t < end; t += 32) mk[indices[t]] |= bit;
}
__device__ __forceinline__ void mark_andnot(unsigned char* mk, const int32_t* __restrict__ indices, int beg,
                                            int end, unsigned char bit, int lane) {
    for (int t = beg + lane; t < end; t += 32) mk[indices[t]] &= (unsigned char)~bit;
}

__global__ void __launch_bounds__(512) k_motif(MotifParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    unsigned long long* bcnt = reinterpret_cast<unsigned long long*>(smem_raw);
    MtWarp* W = reinterpret_cast<MtWarp*>(smem_raw + sizeof(unsigned long long) * MT_MAXPAT) + wib;
    for (int j = threadIdx.x; j < p.npat; j += blockDim.x) bcnt[j] = 0ull;
    __syncthreads();

    const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + wib;
    unsigned char* mk = p.marks + gw * (long long)p.n;
    int32_t* slab = p.slab + gw * p.slab_ints;
    Control* ctl = p.ctl;
    const int k = p.k;
    const int32_t* __restrict__ indptr = p.indptr;
    const int32_t* __restrict__ indices = p.indices;

    bool idle = false;
    unsigned long long polls = 0;
    int spin = 0;
    long long last_pending = -1;
    unsigned long long idle_since = 0;
    bool aborted = false;

    while (!aborted) {
        int kind = 0;
        if (lane == 0) {
            unsigned long long pos;
            if (p.donate && gpm_q_claim(p.qseq, p.qcap, &ctl->q_head, &pos)) {
                gpm_load_cg(&W->unit, &p.qunits[pos % p.qcap]);
                kind = 2;
                W->qpos = pos;
            } else {
                unsigned long long r = *(volatile unsigned long long*)&ctl->next_root;
                if (r < (unsigned long long)p.n_roots) r = atomicAdd(&ctl->next_root, 1ull);
                if (r < (unsigned long long)p.n_roots) {
                    W->unit.root_pos = (int32_t)r;
                    W->unit.depth = 1;
                    W->unit.sub[0] = p.roots[r];
                    kind = 1;
                }
            }
        }
        kind = __shfl_sync(GPM_FULL_MASK, kind, 0);
        __syncwarp();

        if (!kind) {
            if (!idle) {
                if (lane == 0) atomicAdd(&ctl->idle, 1);
                idle = true;
                last_pending = -1;
                idle_since = gpm_globaltimer();
            }
            long long pend = 0;
            int err = 0;
            if (lane == 0) {
                pend = *(volatile long long*)&ctl->pending;
                err = *(volatile int*)&ctl->error;
            }
            pend = __shfl_sync(GPM_FULL_MASK, pend, 0);
            err = __shfl_sync(GPM_FULL_MASK, err, 0);
            if (pend <= 0 || err) break;
            const unsigned long long now = gpm_globaltimer();
            if (pend != last_pending) {
                last_pending = pend;
                idle_since = now;
            } else if (now - idle_since > p.max_idle_ns) {
                if (lane == 0) atomicCAS(&ctl->error, 0, DEV_ETIMEOUT);
                break;
            }
            polls++;
            __nanosleep(++spin < 32 ? 256 : 2048);   // short backoff first, then longer
            continue;
        }
        if (idle) {
            if (lane == 0) atomicSub(&ctl->idle, 1);
            idle = false;
        }
        spin = 0;

        // ---------------------------------------------------- set up the unit
        const int root_pos = W->unit.root_pos;
        const int pdepth = W->unit.depth;
        const int root = W->unit.sub[0];
        if (lane == 0)
            for (int j = 0; j < pdepth; j++) W->sub[j] = W->unit.sub[j];
        __syncwarp();
        // marks of the prefix: bit j on N(tr[j]), bit 7 on tr itself
        for (int j = 0; j < pdepth; j++) {
            const int v = W->sub[j];
            mark_or(mk, indices, indptr[v], indptr[v + 1], (unsigned char)(1u << j), lane);
            __syncwarp();
        }
        if (lane < pdepth) mk[W->sub[lane]] |= 0x80;
        __syncwarp();
        if (lane == 0) {
            W->code[1] = 0;
            W->code[2] = 0;
            for (int i = 2; i < pdepth; i++)
                W->code[i + 1] = W->code[i] | ((mk[W->sub[i]] & ((1 << i) - 1)) << code_off(i));
        }
        // extension array of the unit's node: for a root, the suffix of N(r)
        // above r (lists are sorted); for a donated unit, its payload list
        const int32_t* unit_ext;
        if (kind == 1) {
            const int b = indptr[root], e = indptr[root + 1];
            int lo = b, hi = e;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (indices[mid] <= root) lo = mid + 1; else hi = mid;
            }
            unit_ext = indices + lo;
            if (lane == 0) {
                W->len[1] = e - lo;
                W->cur[1] = 0;
                W->hi[1] = e - lo;
            }
        } else if (W->unit.list_off >= 0) {
            // pre-split seed: the list is a suffix of the root's adjacency
            unit_ext = indices + W->unit.list_off;
            if (lane == 0) {
                gpm_q_release(p.qseq, p.qcap, W->qpos);
                W->len[pdepth] = W->unit.len;
                W->cur[pdepth] = 0;
                W->hi[pdepth] = W->unit.child_hi;
            }
        } else {
            int32_t* dst = slab + p.lvl_off[pdepth];
            const long long slot = (long long)(W->qpos % p.qcap);
            const int32_t* src = p.qpayload + slot * MT_LIST;
            const int len = W->unit.len;
            for (int t = lane; t < len; t += 32) dst[t] = __ldcg(src + t);
            __threadfence();
            __syncwarp();
            if (lane == 0) {
                gpm_q_release(p.qseq, p.qcap, W->qpos);
                W->len[pdepth] = len;
                W->cur[pdepth] = 0;
                W->hi[pdepth] = W->unit.child_hi;
            }
            unit_ext = dst;
        }
        __syncwarp();

        // ---------------------------------------------------------- DFS
        unsigned long long unit_leaves = 0;   // lane-private
        int l = pdepth;
        int iter = 0;
        for (;;) {
            const int c = W->cur[l];
            if (c >= W->hi[l]) {
                if (l == pdepth) break;
                // pop tr[l-1] (pushed at depth l-1)
                const int w = W->sub[l - 1];
                mark_andnot(mk, indices, indptr[w], indptr[w + 1], (unsigned char)(1u << (l - 1)), lane);
                __syncwarp();
                if (lane == 0) mk[w] &= 0x7f;
                __syncwarp();
                l--;
                continue;
            }
            const int32_t* ext = l == pdepth ? unit_ext : slab + p.lvl_off[l];
            const int w = ext[c];
            if (lane == 0) W->cur[l] = c + 1;
            const int sigw = mk[w] & ((1 << l) - 1);
            const int codew = l >= 2 ? (W->code[l] | (sigw << code_off(l))) : 0;
            const int wb = indptr[w], we = indptr[w + 1];
            const unsigned char low = (unsigned char)(0x80 | ((1u << l) - 1));
            if (l + 1 == k - 1) {
                // ---- last level: leaves of the (k-1)-set tr + w
                const int offk = code_off(l + 1);
                int excl = 0;
                for (int t = wb + lane; t < we; t += 32) {
                    const int x = indices[t];
                    const unsigned char m = mk[x];
                    excl += (x > root && (m & low) == 0) ? 1 : 0;
                    mk[x] = m | (unsigned char)(1u << l);
                }
                excl = __reduce_add_sync(GPM_FULL_MASK, (unsigned)excl);
                __syncwarp();
                if (excl) {
                    const int pid = p.lut[codew | ((1 << l) << offk)];
                    if (lane == 0) {
                        if (pid == 0xffff) atomicExch(&ctl->error, DEV_EINVAL);
                        else atomicAdd(&bcnt[pid], (unsigned long long)excl);
                    }
                    if (lane == 0) unit_leaves += (unsigned)excl;
                }
                const int len = W->len[l];
                const unsigned lowk = (1u << (l + 1)) - 1u;
                for (int j0 = c + 1; j0 < len; j0 += 32) {
                    const int j = j0 + lane;
                    const bool act = j < len;
                    int pid = 0;
                    if (act) {
                        const int x = ext[j];
                        const int sig = mk[x] & lowk;
                        pid = p.lut[codew | (sig << offk)];
                        unit_leaves++;
                    }
                    count_leaves(bcnt, act, pid, &ctl->error);
                }
                __syncwarp();
                mark_andnot(mk, indices, wb, we, (unsigned char)(1u << l), lane);
                __syncwarp();
            } else {
                // ---- push w: ext_{l+1} = ext_l[c+1:] ++ exclusive neighbours of w
                int32_t* nxt = slab + p.lvl_off[l + 1];
                const int len = W->len[l];
                const int inh = len - (c + 1);
                for (int t = lane; t < inh; t += 32) nxt[t] = ext[c + 1 + t];
                int n_new = inh;
                for (int t0 = wb; t0 < we; t0 += 32) {
                    const int t = t0 + lane;
                    bool ex = false;
                    int x = 0;
                    if (t < we) {
                        x = indices[t];
                        const unsigned char m = mk[x];
                        ex = x > root && (m & low) == 0;
                        mk[x] = m | (unsigned char)(1u << l);
                    }
                    const unsigned bal = __ballot_sync(GPM_FULL_MASK, ex);
                    if (ex) nxt[n_new + __popc(bal & gpm_lanemask_lt())] = x;
                    n_new += __popc(bal);
                }
                __syncwarp();
                if (lane == 0) {
                    mk[w] |= 0x80;
                    W->sub[l] = w;
                    W->code[l + 1] = codew;
                    W->len[l + 1] = n_new;
                    W->cur[l + 1] = 0;
                    W->hi[l + 1] = n_new;
                }
                __syncwarp();
                l++;
            }

            if ((++iter & 7) == 0) {
                int err = 0, want = 0;
                if (lane == 0) {
                    err = *(volatile int*)&ctl->error;
                    if (p.donate) {
                        const int idl = *(volatile int*)&ctl->idle;
                        const unsigned long long qh = *(volatile unsigned long long*)&ctl->q_head;
                        const unsigned long long qt = *(volatile unsigned long long*)&ctl->q_tail;
                        want = idl > 0 && (long long)(qt - qh) < (long long)idl;
                    }
                }
                err = __shfl_sync(GPM_FULL_MASK, err, 0);
                if (err) { aborted = true; break; }
                want = __shfl_sync(GPM_FULL_MASK, want, 0);
                if (want) {
                    for (int t = pdepth; t <= l; t++) {
                        const int from = W->cur[t], to = W->hi[t], len = W->len[t];
                        const int rem = to - from;
                        if (rem < max(p.donate_min, 2)) continue;
                        int start = from + (rem - rem / 2);
                        start = max(start, len - MT_LIST);
                        if (start >= to) continue;
                        unsigned long long pos = 0;
                        int ok = 0;
                        if (lane == 0) ok = gpm_q_reserve(p.qseq, p.qcap, &ctl->q_tail, &pos) ? 1 : 0;
                        ok = __shfl_sync(GPM_FULL_MASK, ok, 0);
                        if (!ok) break;
                        pos = __shfl_sync(GPM_FULL_MASK, pos, 0);
                        const long long slot = (long long)(pos % p.qcap);
                        int32_t* dst = p.qpayload + slot * MT_LIST;
                        const int32_t* src = t == pdepth ? unit_ext : slab + p.lvl_off[t];
                        for (int z = start + lane; z < len; z += 32) dst[z - start] = src[z];
                        if (lane == 0) {
                            MotifUnit u;
                            u.root_pos = root_pos;
                            u.depth = t;
                            u.len = len - start;
                            u.child_hi = to - start;
                            for (int z = 0; z < MT_MAXK; z++) u.sub[z] = z < t ? W->sub[z] : -1;
                            u.list_off = -1;
                            p.qunits[slot] = u;
                            W->hi[t] = start;
                            atomicAdd((unsigned long long*)&ctl->pending, 1ull);
                        }
                        __threadfence();
                        __syncwarp();
                        if (lane == 0) {
                            gpm_q_publish(p.qseq, p.qcap, pos);
                            atomicAdd(&ctl->donations, 1ull);
                        }
                        __syncwarp();
                        break;
                    }
                }
            }
        }
        if (aborted) break;   // marks are left dirty: the host re-clears them after an error

        // clear the prefix marks (deeper marks were undone by the pops)
        for (int j = 0; j < pdepth; j++) {
            const int v = W->sub[j];
            for (int t = indptr[v] + lane; t < indptr[v + 1]; t += 32) mk[indices[t]] = 0;
            __syncwarp();
        }
        if (lane < pdepth) mk[W->sub[lane]] = 0;
        __syncwarp();

        if (p.per_root) {
            const unsigned long long tot = gpm_warp_sum(unit_leaves);
            if (lane == 0 && tot) atomicAdd(&p.per_root[root_pos], tot);
        }
        if (lane == 0) {
            atomicAdd(&ctl->units_done, 1ull);
            atomicAdd((unsigned long long*)&ctl->pending, (unsigned long long)-1ll);
        }
    }

    if (lane == 0 && polls) atomicAdd(&ctl->idle_polls, polls);
    __syncthreads();
    for (int j = threadIdx.x; j < p.npat; j += blockDim.x) {
        const unsigned long long v = bcnt[j];
        if (v) {
            const unsigned long long old = atomicAdd(&p.counts[j], v);
            if (old + v < old) atomicExch(&ctl->overflow, 1);
        }
    }
}

// Pre-split seeds: root j of [n_counter, n_counter + n_split) is cut into
// `chunks` units over equal index ranges of its first extension set
// ({u in N(r): u > r}, a suffix of N(r)); each unit's list is that suffix from
// its first child on, by reference into the adjacency array.
__global__ void k_motif_seed(const int32_t* __restrict__ roots, long long n_counter, int n_split, int chunks,
                             const int32_t* __restrict__ indptr, const int32_t* __restrict__ indices,
                             QSeq* qseq, MotifUnit* qunits) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_split) return;
    const long long pos = n_counter + j;
    const int r = roots[pos];
    const int b = indptr[r], e = indptr[r + 1];
    int lo = b, hi = e;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (indices[mid] <= r) lo = mid + 1; else hi = mid;
    }
    const int L = e - lo;
    for (int c = 0; c < chunks; c++) {
        const long long slot = (long long)j * chunks + c;
        const int a = (int)((long long)L * c / chunks), z = (int)((long long)L * (c + 1) / chunks);
        MotifUnit u;
        u.root_pos = (int32_t)pos;
        u.depth = 1;
        u.len = L - a;
        u.child_hi = z - a;
        for (int q = 0; q < MT_MAXK; q++) u.sub[q] = q == 0 ? r : -1;
        u.list_off = lo + a;
        qunits[slot] = u;
        qseq[slot].seq = (unsigned long long)slot + 1;
    }
}

void run_motif(gpm_graph* g, int k, const int32_t* d_roots, int64_t n_roots,
               unsigned long long* d_per_root, uint64_t* counts_out, int64_t n_counter, int split_chunks) {
    if (k < 1 || k > MT_MAXK) fail(GPM_ENOTIMPL, "motif size k=" + std::to_string(k) + " not built");
    const PatternTable& tab = pattern_table(k);
    const int npat = (int)tab.num_patterns;
    cudaStream_t s = g->stream;
    if (!d_roots) {
        d_roots = ensure_root_order(g, GPM_APP_MOTIF);
        n_roots = g->n;
        n_counter = -1;
    }
    if (n_counter < 0 || n_counter > n_roots) n_counter = n_roots;
    const int n_split = (int)(n_roots - n_counter);
    if (n_split > 0 && (split_chunks < 1 || (unsigned long long)n_split * split_chunks > MT_QUEUE_CAP / 2))
        fail(GPM_EINVAL, "pre-split schedule does not fit the work queue");
    const unsigned long long n_seed = n_split > 0 ? (unsigned long long)n_split * split_chunks : 0ull;
    gpm_stats st{};
    std::vector<unsigned long long> host(npat, 0);

    if (k <= 2) {
        // k = 1: every root; k = 2: every edge from its smaller endpoint
        if (n_roots > 0) {
            std::vector<int32_t> r(n_roots);
            std::vector<int32_t> ip(g->n + 1);
            GPM_CUDA(cudaMemcpyAsync(r.data(), d_roots, sizeof(int32_t) * n_roots, cudaMemcpyDeviceToHost, s));
            GPM_CUDA(cudaMemcpyAsync(ip.data(), g->indptr.ptr, sizeof(int32_t) * (g->n + 1), cudaMemcpyDeviceToHost, s));
            std::vector<int32_t> ind((size_t)std::max<int64_t>(g->nnz, 1));
            if (k == 2 && g->nnz)
                GPM_CUDA(cudaMemcpyAsync(ind.data(), g->indices.ptr, sizeof(int32_t) * g->nnz, cudaMemcpyDeviceToHost, s));
            GPM_CUDA(cudaStreamSynchronize(s));
            std::vector<unsigned long long> pr(n_roots, 0);
            for (int64_t t = 0; t < n_roots; t++) {
                const int v = r[t];
                if (k == 1) pr[t] = 1;
                else {
                    // neighbours above v form a suffix of the sorted list
                    int c = 0;
                    for (int q = ip[v]; q < ip[v + 1]; q++) c += ind[q] > v;
                    pr[t] = c;
                }
                host[0] += pr[t];
            }
            if (d_per_root)
                GPM_CUDA(cudaMemcpyAsync(d_per_root, pr.data(), sizeof(unsigned long long) * n_roots,
                                         cudaMemcpyHostToDevice, s));
            GPM_CUDA(cudaStreamSynchronize(s));
        }
        g->stats = st;
        for (int j = 0; j < npat; j++) counts_out[j] = host[j];
        return;
    }

    const uint16_t* lut = device_lut(k);
    const int wpb = g->cfg.warps_per_block > 0 ? g->cfg.warps_per_block : 8;
    const size_t smem = sizeof(unsigned long long) * MT_MAXPAT + sizeof(MtWarp) * wpb;
    GPM_CUDA(cudaFuncSetAttribute(k_motif, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    Grid gr = plan_grid(g, (const void*)k_motif, wpb, smem);
    const long long nw = gr.total_warps();

    MotifParams p{};
    p.indptr = g->indptr.as<int32_t>();
    p.indices = g->indices.as<int32_t>();
    p.roots = d_roots;
    p.n_roots = n_counter;
    p.n = g->n;
    p.k = k;
    p.npat = npat;
    p.lut = lut;
    // extension arrays ext_1 .. ext_{k-2}; |ext_l| <= l * max degree
    long long off = 0;
    const long long D = std::max(g->max_deg, 1);
    for (int l = 0; l <= MT_MAXK; l++) {
        p.lvl_off[l] = off;
        if (l >= 1 && l <= k - 2) off += (long long)l * D + 4;
        off = (off + 3) & ~3ll;
    }
    p.slab_ints = std::max(off, 4ll);
    g->scratch_slab.ensure(sizeof(int32_t) * p.slab_ints * nw);
    const size_t mark_bytes = (size_t)g->n * nw;
    if (g->scratch_mark.bytes < mark_bytes || !g->scratch_mark.ptr) {
        g->scratch_mark.ensure(mark_bytes);
        g->mark_bytes_cleared = 0;
    }
    if (g->mark_bytes_cleared < mark_bytes) {
        GPM_CUDA(cudaMemsetAsync(g->scratch_mark.ptr, 0, g->scratch_mark.bytes, s));
        g->mark_bytes_cleared = g->scratch_mark.bytes;
    }
    p.marks = g->scratch_mark.as<unsigned char>();
    p.slab = g->scratch_slab.as<int32_t>();

    g->scratch_small.ensure(sizeof(Control) + sizeof(unsigned long long) * MT_MAXPAT);
    Control* ctl = g->scratch_small.as<Control>();
    p.counts = reinterpret_cast<unsigned long long*>(ctl + 1);
    Control h{};
    h.pending = n_counter + (long long)n_seed;
    h.q_tail = n_seed;
    GPM_CUDA(cudaMemcpyAsync(ctl, &h, sizeof(Control), cudaMemcpyHostToDevice, s));
    GPM_CUDA(cudaMemsetAsync(p.counts, 0, sizeof(unsigned long long) * MT_MAXPAT, s));
    if (d_per_root && n_roots > 0)
        GPM_CUDA(cudaMemsetAsync(d_per_root, 0, sizeof(unsigned long long) * n_roots, s));

    const size_t qbytes = (sizeof(QSeq) + sizeof(MotifUnit) + sizeof(int32_t) * MT_LIST) * MT_QUEUE_CAP;
    g->scratch_queue.ensure(qbytes);
    p.qseq = g->scratch_queue.as<QSeq>();
    p.qunits = reinterpret_cast<MotifUnit*>(p.qseq + MT_QUEUE_CAP);
    p.qpayload = reinterpret_cast<int32_t*>(p.qunits + MT_QUEUE_CAP);
    p.qcap = MT_QUEUE_CAP;
    k_queue_init<<<16, 256, 0, s>>>(p.qseq, MT_QUEUE_CAP);
    if (n_split > 0)
        k_motif_seed<<<(n_split + 127) / 128, 128, 0, s>>>(d_roots, n_counter, n_split, split_chunks, p.indptr,
                                                          p.indices, p.qseq, p.qunits);
    p.ctl = ctl;
    p.per_root = d_per_root;
    p.donate = g->cfg.donate;
    p.donate_min = std::max(2, g->cfg.donate_min);
    p.max_idle_ns = (unsigned long long)std::max(1, g->cfg.max_idle_ms) * 1000000ull;

    if (n_roots > 0) {
        GPM_CUDA(cudaEventRecord(g->ev0, s));
        k_motif<<<gr.blocks, wpb * 32, smem, s>>>(p);
        GPM_CUDA(cudaGetLastError());
        GPM_CUDA(cudaEventRecord(g->ev1, s));
        st.grid_blocks = gr.blocks;
        st.warps_per_block = wpb;
    }
    GPM_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(Control), cudaMemcpyDeviceToHost, s));
    GPM_CUDA(cudaMemcpyAsync(host.data(), p.counts, sizeof(unsigned long long) * npat, cudaMemcpyDeviceToHost, s));
    GPM_CUDA(cudaStreamSynchronize(s));
    if (st.grid_blocks) {
        float ms = 0.f;
        GPM_CUDA(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
        st.kernel_ms = ms;
    }
    st.units_done = h.units_done;
    st.donations = h.donations;
    st.idle_polls = h.idle_polls;
    g->stats = st;
    if (h.error) g->mark_bytes_cleared = 0;   // an aborted walk leaves marks behind
    if (h.error == DEV_ETIMEOUT) fail(GPM_ETIMEOUT, "an idle warp waited longer than max_idle_ms without progress");
    if (h.error == DEV_EINVAL) fail(GPM_ECUDA, "pattern table lookup hit an invalid traversal code");
    if (h.error) fail(GPM_ECUDA, "device error " + std::to_string(h.error));
    if (h.overflow) fail(GPM_EOVERFLOW, "a pattern count exceeds 2^64-1");
    for (int j = 0; j < npat; j++) counts_out[j] = host[j];
}

}  // namespace gpm
