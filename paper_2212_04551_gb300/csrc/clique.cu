// clique.cu -- k-clique counting on the device (Algorithm 4, clique counting).
//
// Hot-path rows A2 (root units), A3 (extension step), A4 (aggregate), A7
// (per-warp DFS stack), A8 (work donation) and A9 (counter reduction).
//
// The paper's clique loop extends a traversal from tr[0]'s adjacency, keeps
// extensions after the last vertex ("lower"), keeps those adjacent to every
// traversal vertex ("is_clique"), and at |tr| = k-1 adds the number of valid
// extensions (aggregate_counter).  Here the same search runs on the
// degree-ordered orientation (graph.cu), and the candidate set of a
// traversal -- the valid extensions after both filters -- is kept as a
// bitmap over the root's out-neighbourhood N+(r):
//
//   * per root r (d = |N+(r)|), row i of a d x d bit matrix in shared memory
//     holds N+(u_i) restricted to N+(r) (u_i = i-th out-neighbour of r);
//   * the root node's candidates are all d bits; choosing child i gives the
//     child's candidates C & row_i (the "lower" and "is_clique" filters in
//     one AND: row_i only holds vertices after u_i, and the AND keeps those
//     adjacent to every traversal vertex);
//   * at a node of size k-2 the number of k-cliques below it is
//     sum over i in C of popc(C & row_i) -- aggregate_counter applied to every
//     (k-1)-vertex child at once, without materialising the children.
//
// One warp owns one work unit (a root, or a donated range of children of a
// node deep in a root's tree).  Upper levels are walked one child at a time
// (the DFS step, Section 4.2); the last level is expanded lane-parallel over
// the compacted candidate list (the BFS step of DFS-wide, one candidate per
// lane).  Idle warps publish themselves in a counter; a busy warp that sees
// one splits the remaining children of its shallowest splittable level and
// pushes the upper half to a bounded device queue (replacing the paper's
// CPU stop/redistribute/restart balancing, Section 4.3.5).  Every wait is
// bounded by a no-progress timeout that raises GPM_ETIMEOUT.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "common.cuh"

namespace gpm {

constexpr int CQ_LEVELS = GPM_CLIQUE_MAX_K + 1;
constexpr int CQ_MAX_OUTDEG = 1024;          // bitmap rows of at most 32 words
constexpr unsigned long long CQ_QUEUE_CAP = 8192;

struct CliqueUnit {
    int32_t root_pos;                   // index into the root list
    int32_t depth;                      // path length p: the node is a (p+1)-clique
    int32_t lo, hi;                     // its children (local indices) in [lo, hi); hi < 0: all
    uint16_t path[GPM_CLIQUE_MAX_K];    // local index chosen at sizes 1 .. p
};
static_assert(sizeof(CliqueUnit) % 4 == 0, "unit must be word-sized");

struct CliqueParams {
    const int32_t* __restrict__ off;
    const int32_t* __restrict__ adj;
    const int32_t* __restrict__ outdeg;
    const int32_t* __restrict__ roots;
    long long n_roots;
    int k_lo, k_hi;
    int wmax;            // 32-bit words per bitmap row at the largest out-degree
    int ws;              // row stride in words (odd: lanes reading different rows hit different banks)
    int maxd;
    int stride_words;    // shared-memory words per warp
    Control* ctl;
    QSeq* qseq;
    CliqueUnit* qunits;
    unsigned long long qcap;
    unsigned long long* per_root;   // nullable
    int donate, donate_min;
    unsigned long long max_idle_ns;
};

// shared-memory layout of one warp, in 32-bit words
struct CqLayout {
    int wcnt, unit, cur, hi, cand, list, rows, total;
};

__host__ __device__ inline CqLayout cq_layout(int maxd, int wmax, int ws) {
    CqLayout L;
    L.wcnt = 0;                                        // CQ_LEVELS x u64
    L.unit = L.wcnt + 2 * CQ_LEVELS;                   // CliqueUnit
    L.cur = L.unit + (int)(sizeof(CliqueUnit) / 4);
    L.hi = L.cur + CQ_LEVELS;
    L.cand = L.hi + CQ_LEVELS;                         // CQ_LEVELS x wmax candidate bitmaps
    L.list = L.cand + CQ_LEVELS * wmax;                // 32*wmax ints: N+(r), later the child list
    L.rows = L.list + 32 * wmax;                       // maxd x ws bit rows
    L.total = L.rows + maxd * ws;
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
    if (!v) return;
    const unsigned long long old = atomicAdd(&ctl->counts[j], v);
    if (old + v < old) atomicExch(&ctl->overflow, 1);
}

// Build the root-local bit matrix: row i = N+(u_i) restricted to N+(r).
__device__ void build_rows(const CliqueParams& p, int r, int d, int ws, int* list, uint32_t* rows,
                           int lane) {
    const int beg = p.off[r];
    for (int t = lane; t < d; t += 32) list[t] = p.adj[beg + t];
    for (int t = lane; t < d * ws; t += 32) rows[t] = 0u;
    __syncwarp();
    const int first = list[0], last = list[d - 1];
    for (int i = 0; i < d; i++) {
        const int u = list[i];
        const int ub = p.off[u], du = p.outdeg[u];
        for (int t = lane; t < du; t += 32) {
            const int x = p.adj[ub + t];
            if (x < first || x > last) continue;
            int lo = 0, hi = d - 1;
            while (lo < hi) {               // first index with list[idx] >= x
                const int mid = (lo + hi) >> 1;
                if (list[mid] < x) lo = mid + 1; else hi = mid;
            }
            if (list[lo] == x) atomicOr(&rows[i * ws + (lo >> 5)], 1u << (lo & 31));
        }
    }
    __syncwarp();
}

__global__ void __launch_bounds__(512) k_clique(CliqueParams p) {
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const CqLayout L = cq_layout(p.maxd, p.wmax, p.ws);
    uint32_t* base = smem + (size_t)wib * p.stride_words;
    unsigned long long* wcnt = reinterpret_cast<unsigned long long*>(base + L.wcnt);
    CliqueUnit* unit = reinterpret_cast<CliqueUnit*>(base + L.unit);
    int* cur = reinterpret_cast<int*>(base + L.cur);
    int* hiv = reinterpret_cast<int*>(base + L.hi);
    uint32_t* cand = base + L.cand;
    int* list = reinterpret_cast<int*>(base + L.list);
    uint32_t* rows = base + L.rows;
    Control* ctl = p.ctl;

    for (int j = lane; j < CQ_LEVELS; j += 32) wcnt[j] = 0ull;
    __syncwarp();

    unsigned long long top_sum = 0;   // lane-private k_hi-clique count
    int cached_root = -1;
    bool idle = false;
    unsigned long long polls = 0;
    int spin = 0;
    long long last_pending = -1;
    unsigned long long idle_since = 0;
    bool aborted = false;

    while (!aborted) {
        // ---- acquire a unit: donated work first, then the next root
        int kind = 0;
        if (lane == 0) {
            unsigned long long pos;
            if (p.donate && gpm_q_claim(p.qseq, p.qcap, &ctl->q_head, &pos)) {
                gpm_load_cg(unit, &p.qunits[pos % p.qcap]);
                __threadfence();
                gpm_q_release(p.qseq, p.qcap, pos);
                kind = 2;
            } else {
                unsigned long long r = *(volatile unsigned long long*)&ctl->next_root;
                if (r < (unsigned long long)p.n_roots) r = atomicAdd(&ctl->next_root, 1ull);
                if (r < (unsigned long long)p.n_roots) {
                    unit->root_pos = (int32_t)r;
                    unit->depth = 0;
                    unit->lo = 0;
                    unit->hi = -1;
                    kind = 1;
                }
            }
        }
        kind = __shfl_sync(GPM_FULL_MASK, kind, 0);
        __syncwarp();

        if (!kind) {
            // ---- idle: wait (bounded) for donated work or global completion
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

        // ---- process the unit
        const int root_pos = unit->root_pos;
        const int r = p.roots[root_pos];
        const int d = p.outdeg[r];
        const int w = (d + 31) >> 5;
        const int ws = w | 1;
        unsigned long long unit_sum = 0;   // lane-private k_hi-cliques of this unit
        if (d >= p.k_lo - 1 && d > 0) {
            if (r != cached_root) {
                build_rows(p, r, d, ws, list, rows, lane);
                cached_root = r;
            }
            // candidates of the unit's node: all of N+(r), then AND along the path
            if (lane < w) cand[1 * p.wmax + lane] = range_mask(lane, 0, d);
            __syncwarp();
            const int depth = unit->depth;
            int s = 1;
            for (int t = 0; t < depth; t++) {
                const int i = unit->path[t];
                if (lane < w) cand[(s + 1) * p.wmax + lane] = cand[s * p.wmax + lane] & rows[i * ws + lane];
                s++;
                __syncwarp();
            }
            const int s_base = s;
            if (lane == 0) {
                cur[s] = unit->lo;
                hiv[s] = unit->hi < 0 ? d : unit->hi;
            }
            __syncwarp();

            int iter = 0;
            for (;;) {
                const uint32_t* Cs = cand + s * p.wmax;
                if (s == p.k_hi - 2) {
                    // last level: children of this node, lane-parallel
                    const int from = cur[s], to = hiv[s];
                    int nchild = 0;
                    for (int q = 0; q < w; q++) {
                        const uint32_t word = Cs[q] & range_mask(q, from, to);
                        const bool bit = (word >> lane) & 1u;
                        const unsigned bal = __ballot_sync(GPM_FULL_MASK, bit);
                        if (bit) list[nchild + __popc(bal & gpm_lanemask_lt())] = 32 * q + lane;
                        nchild += __popc(bal);
                    }
                    __syncwarp();
                    unsigned long long sum = 0;
                    for (int t = lane; t < nchild; t += 32) {
                        const uint32_t* row = rows + list[t] * ws;
                        int c = 0;
                        for (int q = 0; q < w; q++) c += __popc(Cs[q] & row[q]);
                        sum += (unsigned)c;
                    }
                    unit_sum += sum;
                    if (lane == 0 && s + 1 >= p.k_lo) wcnt[s + 1] += (unsigned)nchild;
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
                uint32_t* Cn = cand + (s + 1) * p.wmax;
                uint32_t x = 0;
                if (lane < w) {
                    x = Cs[lane] & rows[i * ws + lane];
                    Cn[lane] = x;
                }
                const int c = __reduce_add_sync(GPM_FULL_MASK, (unsigned)__popc(x));
                if (lane == 0) {
                    cur[s] = i + 1;
                    if (s + 1 >= p.k_lo) wcnt[s + 1] += 1ull;
                }
                // descend while the child can still reach a counted size
                const bool down = (s + 1 <= p.k_hi - 2) && c > 0 && (s + 1 + c >= p.k_lo);
                if (down && lane == 0) {
                    cur[s + 1] = 0;
                    hiv[s + 1] = d;
                }
                __syncwarp();
                if (down) s++;

                if ((++iter & 15) == 0) {
                    // abort on a device error; donate when someone is idle
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
                        // shallowest level (up to the current one) with enough siblings left
                        for (int t = s_base; t <= s && t <= p.k_hi - 3; t++) {
                            const uint32_t* Ct = cand + t * p.wmax;
                            const int from = cur[t], to = hiv[t];
                            const int rem = count_range(Ct, w, from, to, lane);
                            if (rem < max(p.donate_min, 2)) continue;
                            // keep the first rem - rem/2 remaining children, donate the rest
                            const int keep = rem - rem / 2;
                            int seen = 0, mid = -1;
                            for (int q = 0; q < w && mid < 0; q++) {
                                const uint32_t word = Ct[q] & range_mask(q, from, to);
                                const int pc = __popc(word);
                                if (seen + pc > keep) {
                                    uint32_t wv = word;
                                    for (int z = 0; z < keep - seen; z++) wv &= wv - 1u;
                                    mid = 32 * q + __ffs(wv) - 1;
                                }
                                seen += pc;
                            }
                            if (mid < 0) break;
                            int ok = 0;
                            if (lane == 0) {
                                unsigned long long pos;
                                if (gpm_q_reserve(p.qseq, p.qcap, &ctl->q_tail, &pos)) {
                                    CliqueUnit* dst = &p.qunits[pos % p.qcap];
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
                                    gpm_q_publish(p.qseq, p.qcap, pos);
                                    atomicAdd(&ctl->donations, 1ull);
                                    hiv[t] = mid;
                                    ok = 1;
                                }
                            }
                            ok = __shfl_sync(GPM_FULL_MASK, ok, 0);
                            __syncwarp();
                            break;
                        }
                    }
                }
            }
        }
        top_sum += unit_sum;
        if (p.per_root) {
            const unsigned long long tot = gpm_warp_sum(unit_sum);
            if (lane == 0 && tot) atomicAdd(&p.per_root[root_pos], tot);
        }
        __syncwarp();
        if (lane == 0) {
            atomicAdd(&ctl->units_done, 1ull);
            atomicAdd((unsigned long long*)&ctl->pending, (unsigned long long)-1ll);
        }
    }

    const unsigned long long tot = gpm_warp_sum(top_sum);
    __syncwarp();
    if (lane == 0) {
        if (polls) atomicAdd(&ctl->idle_polls, polls);
        add_count(ctl, p.k_hi, tot);
        for (int j = p.k_lo; j < p.k_hi; j++) add_count(ctl, j, wcnt[j]);
    }
}

// Pre-split seeds: split root j (entries [n_counter, n_counter + n_split) of
// the root list) into `chunks` units over equal index ranges of its children,
// placed in queue slots [j*chunks, (j+1)*chunks) and published.
__global__ void k_clique_seed(const int32_t* __restrict__ roots, long long n_counter, int n_split, int chunks,
                              const int32_t* __restrict__ outdeg, QSeq* qseq, CliqueUnit* qunits) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_split) return;
    const long long pos = n_counter + j;
    const int d = outdeg[roots[pos]];
    for (int c = 0; c < chunks; c++) {
        const long long slot = (long long)j * chunks + c;
        CliqueUnit u;
        u.root_pos = (int32_t)pos;
        u.depth = 0;
        u.lo = (int)((long long)d * c / chunks);
        u.hi = (int)((long long)d * (c + 1) / chunks);
        for (int z = 0; z < GPM_CLIQUE_MAX_K; z++) u.path[z] = 0;
        qunits[slot] = u;
        qseq[slot].seq = (unsigned long long)slot + 1;
    }
}

// k <= 2 per root: 1 (k = 1) or the out-degree (k = 2)
__global__ void k_clique_small(const int32_t* __restrict__ outdeg, const int32_t* __restrict__ roots,
                               long long n_roots, int k, unsigned long long* __restrict__ per_root,
                               Control* ctl) {
    unsigned long long local = 0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n_roots;
         t += (long long)gridDim.x * blockDim.x) {
        const unsigned long long v = k == 1 ? 1ull : (unsigned long long)outdeg[roots[t]];
        local += v;
        if (per_root) per_root[t] = v;
    }
    local = gpm_warp_sum(local);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(&ctl->counts[k], local);
}

void run_clique(gpm_graph* g, int k_lo, int k_hi, const int32_t* d_roots, int64_t n_roots,
                unsigned long long* d_per_root, uint64_t* counts_out, int64_t n_counter, int split_chunks) {
    if (k_lo < 1 || k_hi > GPM_CLIQUE_MAX_K || k_lo > k_hi) fail(GPM_EINVAL, "bad clique size range");
    ensure_dag(g);
    cudaStream_t s = g->stream;
    if (!d_roots) {
        d_roots = ensure_root_order(g, GPM_APP_CLIQUE);
        n_roots = g->n;
        n_counter = -1;
    }
    if (n_counter < 0 || n_counter > n_roots) n_counter = n_roots;
    const int n_split = (int)(n_roots - n_counter);
    if (n_split > 0 && (split_chunks < 1 || (unsigned long long)n_split * split_chunks > CQ_QUEUE_CAP / 2))
        fail(GPM_EINVAL, "pre-split schedule does not fit the work queue");
    const unsigned long long n_seed = n_split > 0 ? (unsigned long long)n_split * split_chunks : 0ull;
    g->scratch_small.ensure(sizeof(Control));
    Control* ctl = g->scratch_small.as<Control>();
    Control h{};
    h.pending = n_counter + (long long)n_seed;
    h.q_tail = n_seed;
    GPM_CUDA(cudaMemcpyAsync(ctl, &h, sizeof(Control), cudaMemcpyHostToDevice, s));
    if (d_per_root && n_roots > 0)
        GPM_CUDA(cudaMemsetAsync(d_per_root, 0, sizeof(unsigned long long) * n_roots, s));

    gpm_stats st{};
    if (k_hi <= 2) {
        // k = 1: one per root; k = 2: its out-degree (single sizes only)
        if (k_lo != k_hi) fail(GPM_EINVAL, "range counting needs k_lo >= 3");
        if (n_roots > 0) {
            k_clique_small<<<std::max(1, std::min<int>((int)((n_roots + 255) / 256), g->num_sms * 8)), 256, 0, s>>>(
                g->dag_outdeg.as<int32_t>(), d_roots, n_roots, k_hi, d_per_root, ctl);
            GPM_CUDA(cudaGetLastError());
        }
    } else if (n_roots > 0) {
        if (g->max_outdeg > CQ_MAX_OUTDEG)
            fail(GPM_ENOTIMPL, "oriented out-degree " + std::to_string(g->max_outdeg) +
                                   " exceeds the bitmap limit of " + std::to_string(CQ_MAX_OUTDEG));
        CliqueParams p{};
        p.off = g->dag_off.as<int32_t>();
        p.adj = g->dag_adj.as<int32_t>();
        p.outdeg = g->dag_outdeg.as<int32_t>();
        p.roots = d_roots;
        p.n_roots = n_counter;
        p.k_lo = std::max(k_lo, 3);
        p.k_hi = k_hi;
        p.maxd = std::max(g->max_outdeg, 1);
        p.wmax = (p.maxd + 31) / 32;
        p.ws = p.wmax | 1;
        const CqLayout L = cq_layout(p.maxd, p.wmax, p.ws);
        p.stride_words = L.total;
        int wpb = g->cfg.warps_per_block > 0 ? g->cfg.warps_per_block : 8;
        size_t smem = (size_t)wpb * L.total * 4;
        while (smem > 227 * 1024 && wpb > 1) {
            wpb /= 2;
            smem = (size_t)wpb * L.total * 4;
        }
        if (smem > 227 * 1024) fail(GPM_ENOTIMPL, "clique bitmap does not fit in shared memory");
        GPM_CUDA(cudaFuncSetAttribute(k_clique, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        Grid gr = plan_grid(g, (const void*)k_clique, wpb, smem);
        g->scratch_queue.ensure((sizeof(QSeq) + sizeof(CliqueUnit)) * CQ_QUEUE_CAP);
        p.qseq = g->scratch_queue.as<QSeq>();
        p.qunits = reinterpret_cast<CliqueUnit*>(p.qseq + CQ_QUEUE_CAP);
        p.qcap = CQ_QUEUE_CAP;
        k_queue_init<<<16, 256, 0, s>>>(p.qseq, CQ_QUEUE_CAP);
        if (n_split > 0)
            k_clique_seed<<<(n_split + 127) / 128, 128, 0, s>>>(d_roots, n_counter, n_split, split_chunks,
                                                               p.outdeg, p.qseq, p.qunits);
        p.ctl = ctl;
        p.per_root = d_per_root;
        p.donate = g->cfg.donate;
        p.donate_min = std::max(2, g->cfg.donate_min);
        p.max_idle_ns = (unsigned long long)std::max(1, g->cfg.max_idle_ms) * 1000000ull;
        GPM_CUDA(cudaEventRecord(g->ev0, s));
        k_clique<<<gr.blocks, wpb * 32, smem, s>>>(p);
        GPM_CUDA(cudaGetLastError());
        GPM_CUDA(cudaEventRecord(g->ev1, s));
        st.grid_blocks = gr.blocks;
        st.warps_per_block = wpb;
    }
    GPM_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(Control), cudaMemcpyDeviceToHost, s));
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
    if (h.error == DEV_ETIMEOUT) fail(GPM_ETIMEOUT, "an idle warp waited longer than max_idle_ms without progress");
    if (h.error) fail(GPM_ECUDA, "device error " + std::to_string(h.error));
    if (h.overflow) fail(GPM_EOVERFLOW, "clique count exceeds 2^64-1");
    for (int j = k_lo; j <= k_hi; j++) counts_out[j - k_lo] = h.counts[j];
}

}  // namespace gpm
