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
#include "clique_dev.cuh"
#include "monitor.cuh"

namespace gpm {

constexpr unsigned long long CQ_MAX_SEEDS = 65536;   // pre-split units per launch

struct CliqueParams {
    const int32_t* __restrict__ off;
    const int32_t* __restrict__ adj;
    const int32_t* __restrict__ outdeg;
    const int32_t* __restrict__ deg;
    const int32_t* __restrict__ roots;
    long long n_roots;
    int k_lo, k_hi;
    int wmax;            // 32-bit words per bitmap row at the largest out-degree
    int maxd;
    int stride_words;    // shared-memory words per warp
    Control* ctl;
    QSeq* ring_seq;             // idle-warp ring
    int32_t* ring_ids;
    unsigned long long ring_cap;
    unsigned char* mbox;        // per-warp mailboxes
    int mbox_stride;
    const CliqueUnit* seeds;    // pre-split seed units
    long long n_seeds;
    unsigned long long* per_root;   // nullable
    int donate, donate_min;
    unsigned long long donate_after_ns;
    unsigned long long max_idle_ns;
    int tail_levels;
    int compact;
    int compact3;
    int cpl;                    // three-level tail: deepest level through non-edges (policy of gpm_config)
    int monitor;                // host-monitored balancing (no donation): count active warps, obey stop
    CliqueUnit* spill;
    unsigned long long spill_cap;
};

__global__ void __maxnreg__(96) k_clique(CliqueParams p) {
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const CqLayout L = cq_layout(p.maxd, p.wmax, p.compact != 0 || p.compact3 != 0);
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
    CliqueWalk walk{};
    walk.off = p.off;
    walk.adj = p.adj;
    walk.outdeg = p.outdeg;
    walk.deg = p.deg;
    walk.k_lo = p.k_lo;
    walk.k_hi = p.k_hi;
    walk.wmax = p.wmax;
    walk.wcnt = wcnt;
    walk.cur = cur;
    walk.hiv = hiv;
    walk.cand = cand;
    walk.list = list;
    walk.pairs = reinterpret_cast<int*>(base + L.pairs);
    walk.rows = rows;
    walk.ctl = ctl;
    walk.ring_seq = p.ring_seq;
    walk.ring_ids = p.ring_ids;
    walk.ring_cap = p.ring_cap;
    walk.mbox = p.mbox;
    walk.mbox_stride = p.mbox_stride;
    walk.donate_min = p.donate_min;
    walk.donate_after_ns = p.donate_after_ns;
    walk.tail_levels = p.tail_levels;
    walk.compact = p.compact;
    walk.compact3 = p.compact3;
    walk.cpl = p.cpl;
    walk.monitor = p.monitor != 0;
    walk.spill = p.spill;
    walk.spill_cap = p.spill_cap;

    int ovf = 0;                      // a carry-checked sum wrapped (lane-private)
    unsigned long long top_sum = 0;   // lane-private k_hi-clique count
    unsigned long long top_km1 = 0;   // lane-private (k_hi-1)-clique count
    unsigned long long wops = 0;      // lane-private candidate-word operations
    int cached_root = -1;
    bool idle = false;
    unsigned long long polls = 0;
    int spin = 0;
    long long last_pending = -1;
    unsigned long long idle_since = 0;
    unsigned long long busy = 0;      // time spent inside work units (%globaltimer ns)
    bool aborted = false;
    bool exhausted = false;           // lane 0: no seeds or roots left

    const int gw = blockIdx.x * (blockDim.x >> 5) + wib;   // this warp's global id
    MailHdr* my_box = reinterpret_cast<MailHdr*>(p.mbox + (size_t)gw * p.mbox_stride);
    const CliqueUnit* my_unit = reinterpret_cast<const CliqueUnit*>(p.mbox + (size_t)gw * p.mbox_stride + sizeof(MailHdr));
    bool registered = false;

    while (!aborted) {
        // ---- acquire a unit: pre-split seeds, then roots, then donated work
        int kind = 0;
        if (lane == 0 && p.monitor && *(volatile int*)&ctl->stop) exhausted = true;   // the host redistributes
        if (lane == 0) {
            // seeds and roots only run out once: after that, look at the mailbox alone
            unsigned long long sd = exhausted ? ~0ull : *(volatile unsigned long long*)&ctl->next_seed;
            if (sd < (unsigned long long)p.n_seeds) sd = atomicAdd(&ctl->next_seed, 1ull);
            if (sd < (unsigned long long)p.n_seeds) {
                *unit = p.seeds[sd];
                kind = 3;
            } else {
                unsigned long long r = exhausted ? ~0ull : *(volatile unsigned long long*)&ctl->next_root;
                if (r < (unsigned long long)p.n_roots) r = atomicAdd(&ctl->next_root, 1ull);
                if (r >= (unsigned long long)p.n_roots) exhausted = true;
                if (r < (unsigned long long)p.n_roots) {
                    unit->root_pos = (int32_t)r;
                    unit->depth = 0;
                    unit->lo = 0;
                    unit->hi = -1;
                    kind = 1;
                } else if (registered && *(volatile int*)&my_box->ready) {
                    __threadfence();
                    gpm_load_cg(unit, my_unit);
                    *(volatile int*)&my_box->ready = 0;
                    kind = 2;
                }
            }
        }
        kind = __shfl_sync(GPM_FULL_MASK, kind, 0);
        __syncwarp();
        if (kind == 2) registered = false;

        if (!kind) {
            // without donation nothing can arrive once the roots and seeds
            // are gone: leave instead of waiting for the others to finish
            if (!p.donate) break;
            // ---- idle: register once for a hand-off, then wait (bounded) on
            // this warp's own mailbox or global completion
            if (!idle) {
                idle = true;
                last_pending = -1;
                idle_since = gpm_globaltimer();
            }
            if (p.donate && !registered) {
                int ok = 0;
                if (lane == 0) ok = gpm_idle_register(p.ring_seq, p.ring_ids, p.ring_cap, &ctl->q_tail, gw) ? 1 : 0;
                registered = __shfl_sync(GPM_FULL_MASK, ok, 0) != 0;
            }
            // the termination state is shared by every idle warp: look at it
            // every 16th spin only (the own mailbox is checked every spin)
            if ((polls & 15) == 0) {
                long long pend = 0;
                int err = 0;
                if (lane == 0) {
                    pend = *(volatile long long*)&ctl->pending;
                    err = *(volatile int*)&ctl->error;
                }
                pend = __shfl_sync(GPM_FULL_MASK, pend, 0);
                err = __shfl_sync(GPM_FULL_MASK, err, 0);
                if (pend <= 0 || err) break;
                if (pend != last_pending) {
                    last_pending = pend;
                    idle_since = gpm_globaltimer();
                }
            }
            const unsigned long long now = gpm_globaltimer();
            if (now - idle_since > p.max_idle_ns) {
                if (lane == 0) atomicCAS(&ctl->error, 0, DEV_ETIMEOUT);
                break;
            }
            polls++;
            __nanosleep(++spin < 32 ? 128 : 1024);   // short backoff first, then longer
            continue;
        }
        idle = false;
        spin = 0;
        const unsigned long long t_unit = gpm_globaltimer();
        if (p.monitor && lane == 0) atomicAdd(&ctl->active, 1);

        // ---- process the unit
        const int root_pos = unit->root_pos;
        const int r = p.roots[root_pos];
        const int d = p.outdeg[r];
        unsigned long long unit_sum = 0;   // lane-private k_hi-cliques of this unit
        // a root above the bitmap limit (and its seeds) is the list path's
        const bool ok = d > p.maxd ? true
                        : p.donate ? cq_walk<true>(walk, unit, root_pos, r, d, cached_root, unit_sum, top_km1, wops, lane)
                                   : cq_walk<false>(walk, unit, root_pos, r, d, cached_root, unit_sum, top_km1, wops, lane);
        if (!ok) aborted = true;
        top_sum = gpm_add_cc(top_sum, unit_sum, ovf);
        if (p.per_root) {
            const unsigned long long tot = gpm_warp_sum_cc(unit_sum, ovf);
            if (lane == 0) gpm_atomic_add_cc(&p.per_root[root_pos], tot, &ctl->overflow);
        }
        __syncwarp();
        if (lane == 0) {
            atomicAdd(&ctl->units_done, 1ull);
            atomicAdd((unsigned long long*)&ctl->pending, (unsigned long long)-1ll);
            if (p.monitor) atomicSub(&ctl->active, 1);
        }
        busy += gpm_globaltimer() - t_unit;
    }

    const unsigned long long tot = gpm_warp_sum_cc(top_sum, ovf);
    const unsigned long long km1 = gpm_warp_sum_cc(top_km1, ovf);
    const unsigned long long wsum = gpm_warp_sum(wops);
    __syncwarp();
    if (lane == 0) {
        if (ovf) atomicExch(&ctl->overflow, 1);
        atomicAdd(&ctl->word_ops, wsum);
        if (polls) atomicAdd(&ctl->idle_polls, polls);
        atomicAdd(&ctl->busy_ns, busy);
        add_count(ctl, p.k_hi, tot);
        if (p.k_hi >= 4 && p.k_hi - 1 >= p.k_lo) add_count(ctl, p.k_hi - 1, km1);
        for (int j = p.k_lo; j < p.k_hi - 1; j++) add_count(ctl, j, wcnt[j]);
    }
}

// Pre-split seeds: split root j (entries [n_counter, n_counter + n_split) of
// the root list) becomes its units of the plan (chunk_off, else `chunks`
// each) over ranges of its children cut by gpm_balanced_cut.
__global__ void k_clique_seed(const int32_t* __restrict__ roots, long long n_counter, int n_split, int chunks,
                              const int32_t* __restrict__ chunk_off, int k, const int32_t* __restrict__ outdeg,
                              CliqueUnit* seeds) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_split) return;
    const long long pos = n_counter + j;
    const int d = outdeg[roots[pos]];
    const long long base = chunk_off ? chunk_off[j] : (long long)j * chunks;
    const int ch = chunk_off ? chunk_off[j + 1] - chunk_off[j] : chunks;
    for (int c = 0; c < ch; c++) {
        const long long slot = base + c;
        CliqueUnit u;
        u.root_pos = (int32_t)pos;
        u.depth = 0;
        u.lo = gpm_balanced_cut(d, c, ch, k);
        u.hi = gpm_balanced_cut(d, c + 1, ch, k);
        for (int z = 0; z < GPM_CLIQUE_MAX_K; z++) u.path[z] = 0;
        seeds[slot] = u;
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

// Launch geometry, shared-memory layout and work-queue buffers of one
// k_clique launch over n_counter counter roots and n_seed seed units (room
// for extra_units more units beside the seeds: the monitored form's spill
// buffers).  Fills every field of p except ctl, per_root and the modes.
struct CliqueLaunch {
    CliqueParams p{};
    Grid gr;
    int wpb = 0;
    size_t smem = 0;
    CliqueUnit* seeds = nullptr;
    CliqueUnit* extra = nullptr;
};

static CliqueLaunch plan_clique_launch(gpm_graph* g, int k_lo, int k_hi, const int32_t* d_roots, int64_t n_counter,
                                       unsigned long long n_seed, unsigned long long extra_units) {
    CliqueLaunch c;
    CliqueParams& p = c.p;
    cudaStream_t s = g->stream;
    p.off = g->dag_off.as<int32_t>();
    p.adj = g->dag_adj.as<int32_t>();
    p.outdeg = g->dag_outdeg.as<int32_t>();
    p.deg = g->degree.as<int32_t>();
    p.roots = d_roots;
    p.n_roots = n_counter;
    p.k_lo = std::max(k_lo, 3);
    p.k_hi = k_hi;
    // roots above the bitmap limit are left to the list path (clique_list.cu)
    p.maxd = std::min(std::max(g->max_outdeg, 1), CQ_MAX_OUTDEG);
    p.wmax = (p.maxd + 31) / 32;
    p.compact = g->cfg.clique_compact;   // before the layout: it sizes the compaction region
    // the compacted three-level tail runs where the three-level tail does
    const bool three = k_hi >= 5 && (g->cfg.clique_tail == 3 || (g->cfg.clique_tail == 0 && k_hi >= 7));
    p.compact3 = three ? g->cfg.clique_compact3 : 0;
    const CqLayout L = cq_layout(p.maxd, p.wmax, p.compact != 0 || p.compact3 != 0);
    p.stride_words = L.total;
    int wpb = g->cfg.warps_per_block > 0 ? g->cfg.warps_per_block
                                          : best_warps_per_block((const void*)k_clique, (size_t)L.total * 4, 0);
    size_t smem = (size_t)wpb * L.total * 4;
    while (smem > 227 * 1024 && wpb > 1) {
        wpb /= 2;
        smem = (size_t)wpb * L.total * 4;
    }
    if (smem > 227 * 1024) fail(GPM_ENOTIMPL, "clique bitmap does not fit in shared memory");
    GPM_CUDA(cudaFuncSetAttribute(k_clique, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    c.gr = plan_grid(g, (const void*)k_clique, wpb, smem);
    c.wpb = wpb;
    c.smem = smem;
    // idle ring (capacity: a power of two >= every warp), mailboxes, seeds
    unsigned long long cap = 1;
    while (cap < (unsigned long long)c.gr.total_warps()) cap <<= 1;
    const size_t stride = (sizeof(MailHdr) + sizeof(CliqueUnit) + 127) & ~size_t(127);
    const size_t ring_bytes = (sizeof(QSeq) + sizeof(int32_t)) * cap;
    const size_t mbox_bytes = stride * (size_t)c.gr.total_warps();
    const size_t seed_bytes = sizeof(CliqueUnit) * std::max<unsigned long long>(n_seed, 1);
    const size_t extra_bytes = sizeof(CliqueUnit) * extra_units;
    g->scratch_queue.ensure(ring_bytes + mbox_bytes + seed_bytes + extra_bytes + 256);
    unsigned char* qb = g->scratch_queue.as<unsigned char>();
    p.ring_seq = reinterpret_cast<QSeq*>(qb);
    p.ring_ids = reinterpret_cast<int32_t*>(qb + sizeof(QSeq) * cap);
    p.ring_cap = cap;
    p.mbox = qb + ((ring_bytes + 127) & ~size_t(127));
    p.mbox_stride = (int)stride;
    c.seeds = reinterpret_cast<CliqueUnit*>(p.mbox + mbox_bytes);
    c.extra = extra_units ? c.seeds + std::max<unsigned long long>(n_seed, 1) : nullptr;
    p.seeds = c.seeds;
    p.n_seeds = (long long)n_seed;
    k_queue_init<<<16, 256, 0, s>>>(p.ring_seq, cap);
    GPM_CUDA(cudaMemsetAsync(p.mbox, 0, mbox_bytes, s));
    p.donate = g->cfg.donate;
    p.donate_min = std::max(2, g->cfg.donate_min);
    p.donate_after_ns = (unsigned long long)std::max(0, g->cfg.donate_after_us) * 1000ull;
    p.tail_levels = g->cfg.clique_tail;
    p.cpl = g->cfg.clique_cpl;
    p.max_idle_ns = (unsigned long long)std::max(1, g->cfg.max_idle_ms) * 1000000ull;
    return c;
}

void run_clique(gpm_graph* g, int k_lo, int k_hi, const int32_t* d_roots, int64_t n_roots,
                unsigned long long* d_per_root, uint64_t* counts_out, int64_t n_counter, const SplitPlan* plan) {
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
    const int split_chunks = plan ? plan->chunks : 0;
    const int32_t* chunk_off = plan ? plan->d_chunk_off : nullptr;
    const unsigned long long n_seed =
        n_split <= 0 ? 0ull : (chunk_off ? (unsigned long long)plan->n_seeds : (unsigned long long)n_split * split_chunks);
    if (n_split > 0 && ((!chunk_off && split_chunks < 1) || n_seed > CQ_MAX_SEEDS))
        fail(GPM_EINVAL, "pre-split schedule has too many units");
    g->scratch_small.ensure(sizeof(Control));
    Control* ctl = g->scratch_small.as<Control>();
    Control h{};
    h.pending = n_counter + (long long)n_seed;
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
        CliqueLaunch L = plan_clique_launch(g, k_lo, k_hi, d_roots, n_counter, n_seed, 0);
        CliqueParams& p = L.p;
        if (n_split > 0)
            k_clique_seed<<<(n_split + 127) / 128, 128, 0, s>>>(d_roots, n_counter, n_split, split_chunks,
                                                               chunk_off, k_hi, p.outdeg, L.seeds);
        p.ctl = ctl;
        p.per_root = d_per_root;
        GPM_CUDA(cudaEventRecord(g->ev0, s));
        k_clique<<<L.gr.blocks, L.wpb * 32, L.smem, s>>>(p);
        GPM_CUDA(cudaGetLastError());
        run_clique_list(g, k_lo, k_hi, d_roots, n_roots, d_per_root, ctl, CQ_MAX_OUTDEG);
        GPM_CUDA(cudaEventRecord(g->ev1, s));
        st.grid_blocks = L.gr.blocks;
        st.warps_per_block = L.wpb;
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
    st.word_ops = h.word_ops;
    st.busy_warp_ns = h.busy_ns;
    st.kernel_launches = st.grid_blocks ? (n_split > 0 ? 3 : 2) : (k_hi <= 2 && n_roots > 0 ? 1 : 0);
    if (st.grid_blocks && g->max_outdeg > CQ_MAX_OUTDEG) st.kernel_launches += 2;   // the list path
    g->stats = st;
    if (h.error == DEV_ETIMEOUT) fail(GPM_ETIMEOUT, "an idle warp waited longer than max_idle_ms without progress");
    if (h.error) fail(GPM_ECUDA, "device error " + std::to_string(h.error));
    if (h.overflow) fail(GPM_EOVERFLOW, "clique count exceeds 2^64-1");
    for (int j = k_lo; j <= k_hi; j++) counts_out[j - k_lo] = h.counts[j];
}

// The paper's load balancing (Section 4.3.5), for comparison with the
// in-kernel hand-off: see monitor.cuh.  Counts add up over the launches.
void run_clique_monitored(gpm_graph* g, int k, double threshold, uint64_t* count_out, MonitorStats* ms_out) {
    if (k < 3 || k > GPM_CLIQUE_MAX_K) fail(GPM_EINVAL, "monitored clique counting needs 3 <= k <= 16");
    ensure_dag(g);
    cudaStream_t s = g->stream;
    const int32_t* d_roots = ensure_root_order(g, GPM_APP_CLIQUE);
    const int64_t n_roots = g->n;
    g->scratch_small.ensure(sizeof(Control));
    Control* ctl = g->scratch_small.as<Control>();
    MonitorStats ms{};
    unsigned __int128 total = 0;
    gpm_stats st{};
    if (n_roots > 0) {
        // spill capacity: one unit per level per warp; two buffers used in
        // turn (the last launch's spill is the next launch's seeds)
        const Grid probe = plan_clique_launch(g, k, k, d_roots, n_roots, 0, 0).gr;
        const unsigned long long cap = (unsigned long long)probe.total_warps() * CQ_LEVELS;
        CliqueLaunch L = plan_clique_launch(g, k, k, d_roots, n_roots, cap, cap);
        CliqueUnit* bufs[2] = {L.seeds, L.extra};
        auto launch = [&](long long counter_roots, unsigned long long n_seeds, int turn) {
            CliqueParams p = L.p;
            p.ctl = ctl;
            p.per_root = nullptr;
            p.donate = 0;
            p.monitor = 1;
            p.n_roots = counter_roots;
            p.seeds = bufs[turn];
            p.n_seeds = (long long)n_seeds;
            p.spill = bufs[turn ^ 1];
            p.spill_cap = cap;
            GPM_CUDA(cudaEventRecord(g->ev0, s));
            k_clique<<<L.gr.blocks, L.wpb * 32, L.smem, s>>>(p);
            GPM_CUDA(cudaGetLastError());
            GPM_CUDA(cudaEventRecord(g->ev1, s));
        };
        auto after = [&](const Control& h) {
            total += h.counts[k];
            st.word_ops += h.word_ops;
            st.units_done += h.units_done;
        };
        ms = monitored_loop(g, ctl, L.gr.total_warps(), n_roots, threshold, cap, launch, after);
        if (g->max_outdeg > CQ_MAX_OUTDEG) {
            // roots above the bitmap limit: the list path, in one more launch
            Control h{};
            GPM_CUDA(cudaMemcpyAsync(ctl, &h, sizeof(Control), cudaMemcpyHostToDevice, s));
            GPM_CUDA(cudaEventRecord(g->ev0, s));
            run_clique_list(g, k, k, d_roots, n_roots, nullptr, ctl, CQ_MAX_OUTDEG);
            GPM_CUDA(cudaEventRecord(g->ev1, s));
            GPM_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(Control), cudaMemcpyDeviceToHost, s));
            GPM_CUDA(cudaStreamSynchronize(s));
            float lms = 0.f;
            GPM_CUDA(cudaEventElapsedTime(&lms, g->ev0, g->ev1));
            if (h.overflow) fail(GPM_EOVERFLOW, "clique count exceeds 2^64-1");
            total += h.counts[k];
            ms.kernel_ms += lms;
            ms.launches += 2;
        }
        st.grid_blocks = L.gr.blocks;
        st.warps_per_block = L.wpb;
        st.kernel_ms = ms.kernel_ms;
        st.kernel_launches = ms.launches;
    }
    g->stats = st;
    if (total >> 64) fail(GPM_EOVERFLOW, "clique count exceeds 2^64-1");
    *count_out = (uint64_t)total;
    if (ms_out) *ms_out = ms;
}

}  // namespace gpm

// ---------------------------------------------------------------------------
// The paper's DM_DFS baseline (Section 4.2 and Table optimizations-
// performance), for comparison only: one THREAD per root walks the root's
// whole search depth-first, with the candidate lists of every level held as
// sorted id lists in a per-thread stack in global memory, each child's list
// the merge-intersection of its parent's candidates with the child's
// out-neighbours in the degree orientation, and the last level counted by
// list length (aggregate_counter).  No warp cooperation, no bitmaps, no load balancing:
// threads take roots from a global counter, heaviest first.
namespace gpm {

__global__ void k_clique_dfs(const int32_t* __restrict__ off, const int32_t* __restrict__ adj,
                             const int32_t* __restrict__ outdeg, const int32_t* __restrict__ roots, long long n_roots,
                             int k, int maxd, int32_t* __restrict__ stack, Control* ctl) {
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    int32_t* st = stack + tid * (long long)(k - 1) * maxd;   // level s (2 .. k-1) list at st + (s - 2) * maxd
    int pos[GPM_CLIQUE_MAX_K + 1], len[GPM_CLIQUE_MAX_K + 1];
    const int32_t* lst[GPM_CLIQUE_MAX_K + 1];
    unsigned long long count = 0;
    int ovf = 0;
    for (;;) {
        const unsigned long long ri = atomicAdd(&ctl->next_root, 1ull);
        if (ri >= (unsigned long long)n_roots) break;
        const int r = roots[ri];
        // level 1: the root's out-neighbours
        lst[1] = adj + off[r];
        len[1] = outdeg[r];
        pos[1] = 0;
        if (k == 2) {
            count = gpm_add_cc(count, (unsigned long long)len[1], ovf);
            continue;
        }
        int s = 1;
        while (s >= 1) {
            if (s == k - 1) {   // aggregate_counter: every candidate completes a k-clique
                count = gpm_add_cc(count, (unsigned long long)len[s], ovf);
                s--;
                continue;
            }
            if (pos[s] >= len[s]) {
                s--;
                continue;
            }
            const int v = lst[s][pos[s]++];
            // the candidates that are also out-neighbours of v (sorted merge;
            // the orientation alone orders each clique's vertices)
            const int32_t* a = lst[s];
            const int na = len[s];
            const int32_t* b = adj + off[v];
            const int nb = outdeg[v];
            int32_t* out = st + (long long)(s - 1) * maxd;
            int i = 0, j = 0, m = 0;
            while (i < na && j < nb) {
                const int x = a[i], y = b[j];
                if (x < y) i++;
                else if (x > y) j++;
                else {
                    out[m++] = x;
                    i++;
                    j++;
                }
            }
            if (m == 0 && s + 1 < k - 1) continue;
            lst[s + 1] = out;
            len[s + 1] = m;
            pos[s + 1] = 0;
            s++;
        }
    }
    const unsigned long long tot = gpm_warp_sum_cc(count, ovf);
    if ((threadIdx.x & 31) == 0) {
        if (ovf) atomicExch(&ctl->overflow, 1);
        add_count(ctl, k, tot);
    }
}

void run_clique_dfs(gpm_graph* g, int k, uint64_t* count_out) {
    if (k < 2 || k > GPM_CLIQUE_MAX_K) fail(GPM_EINVAL, "k out of range [2, 16]");
    ensure_dag(g);
    cudaStream_t s = g->stream;
    const int32_t* d_roots = ensure_root_order(g, GPM_APP_CLIQUE);
    const int maxd = std::max(g->max_outdeg, 1);
    const int threads = 256;
    const int blocks = g->num_sms * 8;
    const long long nthreads = (long long)blocks * threads;
    g->scratch_slab.ensure(sizeof(int32_t) * (size_t)nthreads * (size_t)(k - 1) * (size_t)maxd);
    g->scratch_small.ensure(sizeof(Control));
    Control* ctl = g->scratch_small.as<Control>();
    Control h{};
    GPM_CUDA(cudaMemcpyAsync(ctl, &h, sizeof(Control), cudaMemcpyHostToDevice, s));
    GPM_CUDA(cudaEventRecord(g->ev0, s));
    if (g->n > 0)
        k_clique_dfs<<<blocks, threads, 0, s>>>(g->dag_off.as<int32_t>(), g->dag_adj.as<int32_t>(),
                                                g->dag_outdeg.as<int32_t>(), d_roots, g->n, k, maxd,
                                                g->scratch_slab.as<int32_t>(), ctl);
    GPM_CUDA(cudaGetLastError());
    GPM_CUDA(cudaEventRecord(g->ev1, s));
    GPM_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(Control), cudaMemcpyDeviceToHost, s));
    GPM_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    GPM_CUDA(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
    gpm_stats st{};
    st.kernel_ms = ms;
    st.grid_blocks = blocks;
    st.warps_per_block = threads / 32;
    st.kernel_launches = g->n > 0 ? 1 : 0;
    g->stats = st;
    if (h.overflow) fail(GPM_EOVERFLOW, "clique count exceeds 2^64-1");
    *count_out = h.counts[k];
}

}  // namespace gpm
