// motif.cu -- induced k-motif counting over one graph (Algorithm 4, motif
// counting; aggregate_pattern of Section 4.3.4).  Hot-path rows A2, A5, A6,
// A7, A8 and A9; the per-unit walk is in motif_dev.cuh.
//
// One persistent launch: each warp takes work units -- a root from a global
// counter over the root order, or a donated unit from the queue -- and walks
// it.  Leaves are counted in per-block shared counters and added to the
// global uint64 counters once per block.  The per-warp marks and extension
// arrays live in HBM, or in shared memory when the graph is small enough
// (n bytes of marks plus the arrays per warp).
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <type_traits>

#include "common.cuh"
#include "monitor.cuh"
#include "motif_dev.cuh"
#include "list_ring.cuh"

namespace gpm {

constexpr unsigned long long MT_MAX_SEEDS = 65536;   // pre-split units per launch

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
    QSeq* ring_seq;             // idle-warp ring
    int32_t* ring_ids;
    unsigned long long ring_cap;
    unsigned char* mbox;        // per-warp mailboxes
    int mbox_stride;
    const MotifUnit* seeds;     // pre-split seed units
    long long n_seeds;
    unsigned long long* per_root;
    unsigned char* marks;       // n bytes per warp (HBM variant)
    int32_t* slab;              // slab_ints per warp (HBM variant)
    long long slab_ints;
    long long lvl_off[MT_MAXK + 1];   // start of ext_l inside a warp's slab
    int mark_stride;            // shared variant: bytes of marks per warp (16-aligned)
    int smem_warp_bytes;        // shared variant: marks + slab per warp
    int donate, donate_min;
    unsigned long long donate_after_ns;
    unsigned long long max_idle_ns;
    unsigned long long* counts; // npat global counters
    int agg_min;                // aggregated last two levels from this many entries (0: never)
    int agg_words;              // shared words of class counters per warp (mt_agg_words(k))
    int monitor;                // host-monitored balancing (no donation): count active warps, obey stop
    MotifUnit* spill;
    unsigned long long spill_cap;
    ListRing list;              // LIST: the host ring the leaves go to
};

// GCOUNT: count patterns straight into the global counters (k = 8) instead
// of per-block shared ones.  LIST: hand every leaf to the host ring as a
// record instead of counting it (listing; donation on, class-counted tail off).
template <bool SMEM_STATE, bool GCOUNT, bool LIST = false>
__global__ void __launch_bounds__(512, 2) k_motif(MotifParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int nwb = blockDim.x >> 5;
    unsigned long long* bcnt = reinterpret_cast<unsigned long long*>(smem_raw);
    MtWarp* W = reinterpret_cast<MtWarp*>(smem_raw + sizeof(unsigned long long) * MT_MAXPAT) + wib;
    uint32_t* agg = reinterpret_cast<uint32_t*>(smem_raw + sizeof(unsigned long long) * MT_MAXPAT + sizeof(MtWarp) * nwb) +
                    (size_t)wib * p.agg_words;
    if (!GCOUNT && !LIST)
        for (int j = threadIdx.x; j < p.npat; j += blockDim.x) bcnt[j] = 0ull;

    const long long gw = (long long)blockIdx.x * nwb + wib;
    Control* ctl = p.ctl;
    MotifWalk a{};
    a.indptr = p.indptr;
    a.indices = p.indices;
    a.lut = p.lut;
    a.k = p.k;
    a.mbase = 0;
    a.lvl_off = p.lvl_off;
    a.ctl = ctl;
    a.ring_seq = p.ring_seq;
    a.ring_ids = p.ring_ids;
    a.ring_cap = p.ring_cap;
    a.mbox = p.mbox;
    a.mbox_stride = p.mbox_stride;
    a.donate_min = p.donate_min;
    a.donate_after_ns = p.donate_after_ns;
    a.err = &ctl->error;
    a.agg = p.agg_words > 0 ? agg : nullptr;
    a.agg_min = p.agg_words > 0 ? p.agg_min : 0;
    a.monitor = p.monitor != 0;
    a.spill = p.spill;
    a.spill_cap = p.spill_cap;
    if (SMEM_STATE) {
        unsigned char* tail = smem_raw + sizeof(unsigned long long) * MT_MAXPAT + sizeof(MtWarp) * nwb +
                              sizeof(uint32_t) * (size_t)p.agg_words * nwb;
        tail = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tail) + 15) & ~uintptr_t(15));
        a.mk = tail + (size_t)wib * p.smem_warp_bytes;
        a.slab = reinterpret_cast<int32_t*>(a.mk + p.mark_stride);
        for (int v = lane; v < p.mark_stride; v += 32) a.mk[v] = 0;
    } else {
        a.mk = p.marks + gw * (long long)p.n;
        a.slab = p.slab + gw * p.slab_ints;
    }
    __syncthreads();
    using CountSink = typename std::conditional<GCOUNT, GlobalSink, BlockSink>::type;
    using Sink = typename std::conditional<LIST, ListSink, CountSink>::type;
    Sink sink{};
    if constexpr (LIST) {
        sink.ring = p.list;
        sink.tail_seen = 0;
        sink.err = &ctl->error;
    } else {
        sink.c = GCOUNT ? p.counts : bcnt;
        sink.ovf = &ctl->overflow;
    }
    const int32_t* __restrict__ indptr = p.indptr;
    const int32_t* __restrict__ indices = p.indices;

    bool idle = false;
    unsigned long long polls = 0;
    unsigned long long scanned = 0;   // adjacency entries scanned by this warp (lane 0)
    int spin = 0;
    long long last_pending = -1;
    unsigned long long idle_since = 0;
    unsigned long long busy = 0;      // time spent inside work units (%globaltimer ns)
    bool aborted = false;
    bool exhausted = false;           // lane 0: no seeds or roots left

    unsigned char* my_box = p.mbox ? p.mbox + (size_t)gw * p.mbox_stride : nullptr;
    bool registered = false;

    while (!aborted) {
        // ---- acquire a unit: pre-split seeds, then roots, then donated work
        int kind = 0;
        if (lane == 0 && p.monitor && atomicAdd(&ctl->stop, 0)) exhausted = true;   // the host redistributes
        if (lane == 0) {
            // seeds and roots only run out once: after that, look at the mailbox alone
            unsigned long long sd = exhausted ? ~0ull : *(volatile unsigned long long*)&ctl->next_seed;
            if (sd < (unsigned long long)p.n_seeds) sd = atomicAdd(&ctl->next_seed, 1ull);
            if (sd < (unsigned long long)p.n_seeds) {
                W->unit = p.seeds[sd];
                kind = 3;
            } else {
                unsigned long long r = exhausted ? ~0ull : *(volatile unsigned long long*)&ctl->next_root;
                if (r < (unsigned long long)p.n_roots) r = atomicAdd(&ctl->next_root, 1ull);
                if (r >= (unsigned long long)p.n_roots) exhausted = true;
                if (r < (unsigned long long)p.n_roots) {
                    W->unit.root_pos = (int32_t)r;
                    W->unit.depth = 1;
                    W->unit.lo = 0;
                    W->unit.hi = -1;
                    W->unit.sub[0] = p.roots[r];
                    kind = 1;
                } else if (registered && *(volatile int*)&reinterpret_cast<MailHdr*>(my_box)->ready) {
                    __threadfence();
                    gpm_load_cg(&W->unit, reinterpret_cast<const MotifUnit*>(my_box + sizeof(MailHdr)));
                    *(volatile int*)&reinterpret_cast<MailHdr*>(my_box)->ready = 0;
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
                if (lane == 0) ok = gpm_idle_register(p.ring_seq, p.ring_ids, p.ring_cap, &ctl->q_tail, (int)gw) ? 1 : 0;
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
        const unsigned long long t_unit = gpm_globaltimer();
        spin = 0;
        if (p.monitor && lane == 0) atomicAdd(&ctl->active, 1);

        // ---------------------------------------------------- set up the unit
        // (a root, a pre-split range of a root's children, or a donated
        // range below a replayed path)
        const int root_pos = W->unit.root_pos;
        const int pdepth = W->unit.depth;
        const int root = W->unit.sub[0];
        const int32_t* unit_ext = mt_replay(a, W, lane);
        if (!unit_ext) {
            if (lane == 0) atomicCAS(&ctl->error, 0, DEV_EINVAL);
            aborted = true;
            break;
        }

        unsigned long long unit_leaves = 0;   // lane-private
        const bool ok = p.donate ? mt_walk<true>(a, W, pdepth, root, root_pos, unit_ext, sink, unit_leaves, scanned, lane)
                                 : mt_walk<false>(a, W, pdepth, root, root_pos, unit_ext, sink, unit_leaves, scanned, lane);
        if (!ok) {
            aborted = true;   // HBM marks are left dirty: the host re-clears them after an error
            break;
        }
        mt_clear_prefix(a, W, pdepth, lane);

        if (p.per_root) {
            int ovf = 0;
            const unsigned long long tot = gpm_warp_sum_cc(unit_leaves, ovf);
            if (lane == 0) {
                if (ovf) atomicExch(&ctl->overflow, 1);
                gpm_atomic_add_cc(&p.per_root[root_pos], tot, &ctl->overflow);
            }
        }
        if (lane == 0) {
            atomicAdd(&ctl->units_done, 1ull);
            atomicAdd((unsigned long long*)&ctl->pending, (unsigned long long)-1ll);
            if (p.monitor) atomicSub(&ctl->active, 1);
        }
        busy += gpm_globaltimer() - t_unit;
    }

    if (lane == 0 && polls) atomicAdd(&ctl->idle_polls, polls);
    if (lane == 0) atomicAdd(&ctl->busy_ns, busy);
    if (lane == 0 && scanned) atomicAdd(&ctl->word_ops, scanned);
    __syncthreads();
    if (!GCOUNT && !LIST)
        for (int j = threadIdx.x; j < p.npat; j += blockDim.x) gpm_atomic_add_cc(&p.counts[j], bcnt[j], &ctl->overflow);
}

// Pre-split seeds: root j of [n_counter, n_counter + n_split) becomes its
// units of the plan (chunk_off, else `chunks` each) over ranges of its first
// extension set ({u in N(r): u > r}, a suffix of N(r)) cut by
// gpm_balanced_cut.
__global__ void k_motif_seed(const int32_t* __restrict__ roots, long long n_counter, int n_split, int chunks,
                             const int32_t* __restrict__ chunk_off, int k, const int32_t* __restrict__ indptr,
                             const int32_t* __restrict__ indices, MotifUnit* seeds) {
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
    const long long base = chunk_off ? chunk_off[j] : (long long)j * chunks;
    const int ch = chunk_off ? chunk_off[j + 1] - chunk_off[j] : chunks;
    for (int c = 0; c < ch; c++) {
        const long long slot = base + c;
        MotifUnit u;
        u.root_pos = (int32_t)pos;
        u.depth = 1;
        u.lo = gpm_balanced_cut(L, c, ch, k);
        u.hi = gpm_balanced_cut(L, c + 1, ch, k);
        for (int q = 0; q < MT_MAXK; q++) {
            u.sub[q] = q == 0 ? r : -1;
            u.pos[q] = -1;
        }
        seeds[slot] = u;
    }
}

void run_motif(gpm_graph* g, int k, const int32_t* d_roots, int64_t n_roots,
               unsigned long long* d_per_root, uint64_t* counts_out, int64_t n_counter, const SplitPlan* plan,
               double monitor_threshold, MonitorStats* monitor_stats, ListJob* list) {
    const bool monitored = monitor_threshold >= 0.0;
    if (list && (monitored || k < 3 || d_roots || plan || d_per_root))
        fail(GPM_EINVAL, "listing runs over every root, k >= 3, without schedules");
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
    const int split_chunks = plan ? plan->chunks : 0;
    const int32_t* chunk_off = plan ? plan->d_chunk_off : nullptr;
    const unsigned long long n_seed =
        n_split <= 0 ? 0ull : (chunk_off ? (unsigned long long)plan->n_seeds : (unsigned long long)n_split * split_chunks);
    if (n_split > 0 && ((!chunk_off && split_chunks < 1) || n_seed > MT_MAX_SEEDS))
        fail(GPM_EINVAL, "pre-split schedule has too many units");
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

    // per-warp state in shared memory when it is small (marks + arrays)
    p.mark_stride = (int)((g->n + 15) & ~15);
    const long long warp_state = (long long)p.mark_stride + 4 * p.slab_ints;
    p.smem_warp_bytes = (int)((warp_state + 15) & ~15ll);
    const size_t fixed_smem = sizeof(unsigned long long) * MT_MAXPAT + 16;
    // the class-counted tail needs two free mark bits at level k-2: k <= 7
    const bool gcount = npat > MT_MAXPAT;
    p.agg_min = k <= 7 && !list ? g->cfg.motif_agg_min : 0;
    p.agg_words = p.agg_min > 0 ? mt_agg_words(k) : 0;
    const size_t agg_bytes = sizeof(uint32_t) * (size_t)p.agg_words;
    const bool smem_state =
        warp_state <= 12 * 1024 && fixed_smem + 8 * (sizeof(MtWarp) + agg_bytes + warp_state) <= 200 * 1024;
    const size_t per_warp = sizeof(MtWarp) + agg_bytes + (smem_state ? (size_t)p.smem_warp_bytes : 0);
    // Marks in HBM (large graphs): every warp owns n mark bytes that the
    // class-counted last levels read at random.  Those loads are
    // latency-bound, so more warps help, until the marks spill from L2 to
    // DRAM: the grid holds about 256 MB of marks (never fewer than 8 warps
    // per SM).  Measured on rmat16 (n = 65,536): 1,216 / 2,432 / 3,648 /
    // 4,864 warps: 4-motifs 252 / 188 / 175 / 216 ms, 5-motifs of root 132
    // 541 / 385 / 332 / 354 ms.
    int wpb = g->cfg.warps_per_block > 0
                  ? g->cfg.warps_per_block
                  : best_warps_per_block(smem_state ? (const void*)k_motif<true, false> : (const void*)k_motif<false, false>,
                                         per_warp, fixed_smem);
    int max_per_sm = 0;
    // Marks in shared memory (small graphs): four warps per block share the
    // block's pattern counters instead of sixteen (sbm2000 motif k = 6:
    // 17.9 s at 4 warps per block, 21.5 s at 16).
    if (smem_state && g->cfg.warps_per_block <= 0) wpb = std::min(wpb, 4);
    if (!smem_state && g->cfg.warps_per_block <= 0 && g->cfg.blocks_per_sm <= 0) {
        const long long mark_warps = (256ll << 20) / std::max<long long>(g->n, 1);
        const long long per_sm_warps = std::max<long long>(8, mark_warps / std::max(g->num_sms, 1));
        wpb = 4;
        max_per_sm = (int)std::max<long long>(2, per_sm_warps / wpb);
    }
    const size_t base_smem = sizeof(unsigned long long) * MT_MAXPAT + (sizeof(MtWarp) + agg_bytes) * wpb + 16;
    const size_t smem = base_smem + (smem_state ? (size_t)wpb * p.smem_warp_bytes : 0);
    const void* kfun = list ? (smem_state ? (const void*)k_motif<true, true, true> : (const void*)k_motif<false, true, true>)
                       : smem_state ? (gcount ? (const void*)k_motif<true, true> : (const void*)k_motif<true, false>)
                                    : (gcount ? (const void*)k_motif<false, true> : (const void*)k_motif<false, false>);
    GPM_CUDA(cudaFuncSetAttribute(kfun, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    Grid gr = plan_grid(g, kfun, wpb, smem, max_per_sm);
    const long long nw = gr.total_warps();
    if (!smem_state) {
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
    }

    g->scratch_small.ensure(sizeof(Control) + sizeof(unsigned long long) * MT_MAXPAT8);
    Control* ctl = g->scratch_small.as<Control>();
    p.counts = reinterpret_cast<unsigned long long*>(ctl + 1);
    Control h{};
    h.pending = n_counter + (long long)n_seed;
    GPM_CUDA(cudaMemcpyAsync(ctl, &h, sizeof(Control), cudaMemcpyHostToDevice, s));
    GPM_CUDA(cudaMemsetAsync(p.counts, 0, sizeof(unsigned long long) * npat, s));
    if (d_per_root && n_roots > 0)
        GPM_CUDA(cudaMemsetAsync(d_per_root, 0, sizeof(unsigned long long) * n_roots, s));

    // idle ring (capacity: a power of two >= every warp), mailboxes, seeds
    // (monitored: two spill buffers of one unit per level per warp instead)
    // (listing: always with hand-offs, whose checks also notice a stop)
    p.donate = monitored ? 0 : (list ? 1 : g->cfg.donate);
    unsigned long long cap = 1;
    while (cap < (unsigned long long)nw) cap <<= 1;
    const unsigned long long spill_cap = monitored ? (unsigned long long)nw * (MT_MAXK + 1) : 0ull;
    const size_t stride = (sizeof(MailHdr) + sizeof(MotifUnit) + 127) & ~size_t(127);
    const size_t ring_bytes = (sizeof(QSeq) + sizeof(int32_t)) * cap;
    const size_t mbox_bytes = p.donate ? stride * (size_t)nw : 0;
    const size_t seed_bytes = sizeof(MotifUnit) * std::max<unsigned long long>(std::max(n_seed, spill_cap), 1);
    g->scratch_queue.ensure(ring_bytes + mbox_bytes + seed_bytes * (monitored ? 2 : 1) + 256);
    unsigned char* qb = g->scratch_queue.as<unsigned char>();
    p.ring_seq = reinterpret_cast<QSeq*>(qb);
    p.ring_ids = reinterpret_cast<int32_t*>(qb + sizeof(QSeq) * cap);
    p.ring_cap = cap;
    p.mbox = p.donate ? qb + ((ring_bytes + 127) & ~size_t(127)) : nullptr;
    p.mbox_stride = (int)stride;
    MotifUnit* seeds = reinterpret_cast<MotifUnit*>(qb + ((ring_bytes + 127) & ~size_t(127)) + mbox_bytes);
    p.seeds = seeds;
    p.n_seeds = (long long)n_seed;
    k_queue_init<<<16, 256, 0, s>>>(p.ring_seq, cap);
    if (mbox_bytes) GPM_CUDA(cudaMemsetAsync(p.mbox, 0, mbox_bytes, s));
    if (n_split > 0)
        k_motif_seed<<<(n_split + 127) / 128, 128, 0, s>>>(d_roots, n_counter, n_split, split_chunks, chunk_off, k,
                                                          p.indptr, p.indices, seeds);
    p.ctl = ctl;
    p.per_root = d_per_root;
    p.donate_min = std::max(2, g->cfg.donate_min);
    p.donate_after_ns = (unsigned long long)std::max(0, g->cfg.donate_after_us) * 1000ull;
    p.max_idle_ns = (unsigned long long)std::max(1, g->cfg.max_idle_ms) * 1000000ull;

    if (list) p.list = list_ring_of(list, ctl);
    auto launch_kernel = [&](const MotifParams& q) {
        GPM_CUDA(cudaEventRecord(g->ev0, s));
        if (list) {
            if (smem_state) k_motif<true, true, true><<<gr.blocks, wpb * 32, smem, s>>>(q);
            else k_motif<false, true, true><<<gr.blocks, wpb * 32, smem, s>>>(q);
        } else if (smem_state) {
            if (gcount) k_motif<true, true><<<gr.blocks, wpb * 32, smem, s>>>(q);
            else k_motif<true, false><<<gr.blocks, wpb * 32, smem, s>>>(q);
        } else {
            if (gcount) k_motif<false, true><<<gr.blocks, wpb * 32, smem, s>>>(q);
            else k_motif<false, false><<<gr.blocks, wpb * 32, smem, s>>>(q);
        }
        GPM_CUDA(cudaGetLastError());
        GPM_CUDA(cudaEventRecord(g->ev1, s));
    };
    if (monitored && n_roots > 0) {
        // stop / redistribute / restart (monitor.cuh); the pattern counters
        // add up over the launches
        MotifUnit* bufs[2] = {seeds, seeds + std::max<unsigned long long>(std::max(n_seed, spill_cap), 1)};
        auto launch = [&](long long counter_roots, unsigned long long n_seeds, int turn) {
            MotifParams q = p;
            q.monitor = 1;
            q.n_roots = counter_roots;
            q.seeds = bufs[turn];
            q.n_seeds = (long long)n_seeds;
            q.spill = bufs[turn ^ 1];
            q.spill_cap = spill_cap;
            launch_kernel(q);
        };
        unsigned long long wops = 0, units = 0;
        auto after = [&](const Control& hc) {
            wops += hc.word_ops;
            units += hc.units_done;
        };
        const MonitorStats ms = monitored_loop(g, ctl, (int)nw, n_counter, monitor_threshold, spill_cap, launch, after);
        if (monitor_stats) *monitor_stats = ms;
        GPM_CUDA(cudaMemcpyAsync(host.data(), p.counts, sizeof(unsigned long long) * npat, cudaMemcpyDeviceToHost, s));
        GPM_CUDA(cudaStreamSynchronize(s));
        st.grid_blocks = gr.blocks;
        st.warps_per_block = wpb;
        st.kernel_ms = ms.kernel_ms;
        st.kernel_launches = ms.launches;
        st.word_ops = wops;
        st.units_done = units;
        g->stats = st;
        for (int j = 0; j < npat; j++) counts_out[j] = host[j];
        return;
    }
    if (n_roots > 0) {
        launch_kernel(p);
        st.grid_blocks = gr.blocks;
        st.warps_per_block = wpb;
        if (list) list_drain(list, g, ctl);
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
    st.word_ops = h.word_ops;
    st.busy_warp_ns = h.busy_ns;
    st.kernel_launches = st.grid_blocks ? (n_split > 0 ? 3 : 2) : 0;
    g->stats = st;
    if (h.error) g->mark_bytes_cleared = 0;   // an aborted walk leaves marks behind
    if (list && h.error == DEV_STOPPED) return;   // the consumer asked to stop
    if (list && h.error == DEV_ETIMEOUT)
        fail(GPM_ETIMEOUT, "the listing ring stayed full (or an idle warp waited) for longer than max_idle_ms (" +
                               list_where(list, h) + ")");
    if (h.error == DEV_ETIMEOUT) fail(GPM_ETIMEOUT, "an idle warp waited longer than max_idle_ms without progress");
    if (h.error == DEV_EINVAL) fail(GPM_ECUDA, "pattern table lookup hit an invalid traversal code");
    if (h.error >= DEV_ECHECK) fail(GPM_ECUDA, "device consistency check " + std::to_string(h.error - DEV_ECHECK) + " failed");
    if (h.error) fail(GPM_ECUDA, "device error " + std::to_string(h.error));
    if (h.overflow) fail(GPM_EOVERFLOW, "a pattern count exceeds 2^64-1");
    for (int j = 0; j < npat; j++) counts_out[j] = host[j];
}

void run_motif_monitored(gpm_graph* g, int k, double threshold, uint64_t* counts_out, MonitorStats* ms) {
    if (k < 3 || k > MT_MAXK) fail(GPM_EINVAL, "monitored motif counting needs 3 <= k <= 8");
    run_motif(g, k, nullptr, 0, nullptr, counts_out, -1, nullptr, threshold, ms);
}

}  // namespace gpm

// ---------------------------------------------------------------------------
// Allocation-free motif counting (gpm_motif_count_noalloc).
//
// For callers that may not allocate device memory at all -- code that runs
// inside a host application owning every device byte through its own pool,
// or real-time and embedded hosts with a fixed device-memory budget where a
// cudaMalloc at call time is not allowed.  The same shared-memory-state
// motif kernel runs with donation off; everything it needs beyond the
// caller's graph and result buffers -- control block, pattern counters,
// validation flags, root list, pattern table -- sits in one file-scope
// device array of fixed size, resident on every device that loads the
// library until the process exits.
// ---------------------------------------------------------------------------
namespace gpm {

constexpr int NA_MAX_N = 8192;                                 // vertices
constexpr size_t NA_CTL_OFF = 0;                               // Control
constexpr size_t NA_CNT_OFF = 1024;                            // MT_MAXPAT uint64 counters
constexpr size_t NA_FLAG_OFF = NA_CNT_OFF + 8192;              // validation flags, max degree
constexpr size_t NA_ROOT_OFF = NA_FLAG_OFF + 256;              // NA_MAX_N int32 roots
constexpr size_t NA_LUT_OFF = NA_ROOT_OFF + 4 * (size_t)NA_MAX_N;
constexpr size_t NA_LUT_BYTES = (size_t)2 << 20;               // 2^20 uint16: pattern table up to k = 7
constexpr size_t NA_SCRATCH_BYTES = NA_LUT_OFF + NA_LUT_BYTES;  // 2,139,392 bytes
static_assert(sizeof(Control) <= NA_CNT_OFF, "control block must fit its slot");
static_assert(sizeof(unsigned long long) * MT_MAXPAT <= 8192, "counters must fit their slot");
static_assert(NA_LUT_OFF % 256 == 0, "aligned table");

}  // namespace gpm

// The scratch.  Host code never uses this name as an address: it asks the
// runtime for the device address (gpm_noalloc_scratch_ptr) once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[gpm::NA_SCRATCH_BYTES];

namespace gpm {

__global__ void k_na_prepare(const int32_t* __restrict__ indptr, int32_t n, int32_t* __restrict__ roots,
                             int* __restrict__ maxdeg) {
    int local = 0;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        roots[v] = (int32_t)v;
        local = max(local, indptr[v + 1] - indptr[v]);
    }
    for (int o = 16; o > 0; o >>= 1) local = max(local, __shfl_xor_sync(GPM_FULL_MASK, local, o));
    if ((threadIdx.x & 31) == 0) atomicMax(maxdeg, local);
}

// Device address of the scratch on the current device; looked up on the
// first call per device (with that device current) and remembered.
static unsigned char* noalloc_scratch_ptr() {
    static std::mutex mu;
    static unsigned char* ptrs[256] = {nullptr};
    int dev = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= 256) fail(GPM_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(mu);
    if (!ptrs[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            fail(GPM_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        }
        ptrs[dev] = static_cast<unsigned char*>(p);
    }
    return ptrs[dev];
}

static void motif_count_noalloc(const int32_t* indptr, const int32_t* indices, int32_t n, int k, uint64_t* counts,
                                int64_t counts_len, cudaStream_t s) {
    if (k < 3 || k > 7) fail(GPM_EINVAL, "k out of range [3, 7] for the allocation-free path");
    if (n < 0 || n > NA_MAX_N)
        fail(GPM_EINVAL, "n = " + std::to_string(n) + " exceeds the allocation-free limit of " +
                             std::to_string(NA_MAX_N) + " vertices");
    if (!indptr || !counts) fail(GPM_EINVAL, "NULL pointer");
    const PatternTable& tab = pattern_table(k);
    const int npat = (int)tab.num_patterns;
    if (counts_len < npat) fail(GPM_EINVAL, "counts_len smaller than the number of patterns");
    if (tab.lut.size() * sizeof(uint16_t) > NA_LUT_BYTES) fail(GPM_EINVAL, "pattern table larger than its slot");
    unsigned char* base = noalloc_scratch_ptr();
    Control* ctl = reinterpret_cast<Control*>(base + NA_CTL_OFF);
    unsigned long long* dcounts = reinterpret_cast<unsigned long long*>(base + NA_CNT_OFF);
    int* flags = reinterpret_cast<int*>(base + NA_FLAG_OFF);   // [0] CSR errors, [1] max degree
    int32_t* roots = reinterpret_cast<int32_t*>(base + NA_ROOT_OFF);
    uint16_t* lut = reinterpret_cast<uint16_t*>(base + NA_LUT_OFF);

    int dev = 0, sms = 0;
    GPM_CUDA(cudaGetDevice(&dev));
    GPM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));

    // CSR checks and the maximum degree (every call: the scratch is shared)
    int32_t ends[2] = {0, 0};
    GPM_CUDA(cudaMemcpyAsync(&ends[0], indptr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GPM_CUDA(cudaMemcpyAsync(&ends[1], indptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GPM_CUDA(cudaStreamSynchronize(s));
    if (ends[0] != 0 || ends[1] < 0 || (ends[1] & 1)) fail(GPM_EINVAL, "invalid indptr");
    if (ends[1] > 0 && !indices) fail(GPM_EINVAL, "indices is NULL");
    GPM_CUDA(cudaMemsetAsync(flags, 0, 2 * sizeof(int), s));
    const int blocks = std::max(1, std::min(sms * 4, (n + 255) / 256));
    if (n > 0) {
        k_indptr_monotone<<<blocks, 256, 0, s>>>(indptr, n, flags);
        k_na_prepare<<<blocks, 256, 0, s>>>(indptr, n, roots, flags + 1);
        GPM_CUDA(cudaGetLastError());
    }
    int hf[2] = {0, 0};
    GPM_CUDA(cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, s));
    GPM_CUDA(cudaStreamSynchronize(s));
    if (hf[0]) fail(GPM_EINVAL, "indptr is not non-decreasing");
    if (n > 0 && ends[1] > 0) {
        k_validate<<<std::max(1, std::min(sms * 8, (n * 32 + 255) / 256)), 256, 0, s>>>(indptr, indices, n, ends[1],
                                                                                      flags);
        GPM_CUDA(cudaGetLastError());
        GPM_CUDA(cudaMemcpyAsync(hf, flags, sizeof(int), cudaMemcpyDeviceToHost, s));
        GPM_CUDA(cudaStreamSynchronize(s));
        if (hf[0]) fail(GPM_EINVAL, "invalid CSR (ids, self-loops, order, duplicates or symmetry)");
    }
    const int maxdeg = hf[1];

    // the kernel's per-warp state must fit in shared memory
    const int wpb = 8;
    MotifParams p{};
    long long off = 0;
    const long long D = std::max(maxdeg, 1);
    for (int l = 0; l <= MT_MAXK; l++) {
        p.lvl_off[l] = off;
        if (l >= 1 && l <= k - 2) off += (long long)l * D + 4;
        off = (off + 3) & ~3ll;
    }
    p.slab_ints = std::max(off, 4ll);
    p.mark_stride = (int)((n + 15) & ~15);
    const long long warp_state = (long long)p.mark_stride + 4 * p.slab_ints;
    const size_t base_smem = sizeof(unsigned long long) * MT_MAXPAT + sizeof(MtWarp) * wpb + 16;
    p.agg_min = 0;    // per-leaf counting only: no class counters in this launch's shared memory
    p.agg_words = 0;
    p.smem_warp_bytes = (int)((warp_state + 15) & ~15ll);
    const size_t smem = base_smem + (size_t)wpb * p.smem_warp_bytes;
    if (warp_state > 12 * 1024 || smem > 200 * 1024)
        fail(GPM_EINVAL, "graph too large for the allocation-free path (vertices + extension arrays must fit in "
                         "12 KB of shared memory per warp)");

    GPM_CUDA(cudaMemcpyAsync(lut, tab.lut.data(), tab.lut.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, s));
    GPM_CUDA(cudaMemsetAsync(base, 0, NA_CNT_OFF + sizeof(unsigned long long) * MT_MAXPAT, s));
    Control h{};
    h.pending = n;
    GPM_CUDA(cudaMemcpyAsync(ctl, &h, sizeof(Control), cudaMemcpyHostToDevice, s));

    p.indptr = indptr;
    p.indices = indices;
    p.roots = roots;
    p.n_roots = n;
    p.n = n;
    p.k = k;
    p.npat = npat;
    p.lut = lut;
    p.ctl = ctl;
    p.counts = dcounts;
    p.donate = 0;
    p.donate_min = 2;
    p.max_idle_ns = 120000000000ull;
    GPM_CUDA(cudaFuncSetAttribute(k_motif<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    GPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_motif<true, false>, wpb * 32, smem));
    if (per_sm <= 0) fail(GPM_EINVAL, "kernel cannot be resident");
    if (n > 0) {
        const int grid = std::max(1, std::min(per_sm * sms, (n + wpb - 1) / wpb));
        k_motif<true, false><<<grid, wpb * 32, smem, s>>>(p);
        GPM_CUDA(cudaGetLastError());
    }
    unsigned long long host[MT_MAXPAT];
    GPM_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(Control), cudaMemcpyDeviceToHost, s));
    GPM_CUDA(cudaMemcpyAsync(host, dcounts, sizeof(unsigned long long) * npat, cudaMemcpyDeviceToHost, s));
    GPM_CUDA(cudaStreamSynchronize(s));
    if (h.error == DEV_ETIMEOUT) fail(GPM_ETIMEOUT, "a bounded device wait ran out");
    if (h.error == DEV_EINVAL) fail(GPM_ECUDA, "pattern table lookup hit an invalid traversal code");
    if (h.error >= DEV_ECHECK) fail(GPM_ECUDA, "device consistency check " + std::to_string(h.error - DEV_ECHECK) + " failed");
    if (h.error) fail(GPM_ECUDA, "device error " + std::to_string(h.error));
    if (h.overflow) fail(GPM_EOVERFLOW, "a pattern count exceeds 2^64-1");
    for (int j = 0; j < npat; j++) counts[j] = host[j];
}

}  // namespace gpm

extern "C" gpm_status gpm_motif_count_noalloc(const int32_t* indptr, const int32_t* indices, int32_t n, int k,
                                              uint64_t* counts, int64_t counts_len, void* stream) {
    try {
        gpm::clear_error();
        gpm::motif_count_noalloc(indptr, indices, n, k, counts, counts_len, reinterpret_cast<cudaStream_t>(stream));
        return GPM_OK;
    } catch (const gpm::Error& e) {
        gpm::set_error(e.msg);
        return e.status;
    } catch (...) {
        gpm::set_error("unexpected internal error");
        return GPM_ECUDA;
    }
}
