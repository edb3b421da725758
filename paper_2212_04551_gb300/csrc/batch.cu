// batch.cu -- batched persistent launch (hot-path row A11; not in the paper).
//
// Thousands of small graphs, packed as one disjoint union (global vertex ids,
// graph_off[g] .. graph_off[g+1]-1 for graph g), are counted by ONE persistent
// kernel over units (task, root): clique units walk a root's bitmap search
// (clique_dev.cuh), motif units walk a root's ESU search (motif_dev.cuh).
// Every clique and every connected set lies inside one graph, so each unit's
// result is added to its root's graph: clique_out[g] and motif_out[g][pattern].
//
// Small graphs keep the whole per-warp motif state in shared memory: marks are
// indexed by the vertex's offset inside its graph (mbase = graph_off[g]), so
// a warp needs only (largest graph) bytes of marks.  Units are split only
// statically: the heaviest roots can be cut into several child ranges before
// the launch (batch_split); warps simply leave when the unit counter runs out
// -- no waiting at all.
//
// The launch (counter resets, kernel, read-back) is captured once into a CUDA
// graph per (clique k, motif k, launch shape) and replayed on every call.  An
// autotuner times the replay over warps per block, resident blocks per SM,
// the unit order, the class-counting threshold of the motif tail and the
// split of heavy roots, and keeps the fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "clique_dev.cuh"
#include "common.cuh"
#include "motif_dev.cuh"

namespace gpm {
gpm_graph* create_graph(const int32_t* indptr, const int32_t* indices, int32_t n, uint32_t flags, void* stream);
void destroy_graph(gpm_graph* g);
}  // namespace gpm

struct gpm_batch {
    gpm_graph* g = nullptr;          // the packed union
    int32_t n_graphs = 0;
    int32_t max_graph_n = 0;
    gpm::DevBuf goff, vgraph;        // graph offsets; vertex -> graph
    cudaStream_t stream = nullptr;   // capturable stream (owned when the caller gave none)
    bool own_stream = false;
    gpm_config cfg{};
    int32_t order_mode = 0;          // 0: motif units first, 1: interleaved by weight
    gpm_stats stats{};
    struct Captured {
        cudaGraphExec_t exec = nullptr;
        gpm::DevBuf units, uranges;  // this launch's unit list (baked into the graph)
        gpm::DevBuf dev_out;         // [G] clique + [G*npat] motif + Control
        unsigned long long* host_out = nullptr;   // pinned
        size_t words = 0;
        int blocks = 0, wpb = 0;
    };
    // (kc, km, wpb, bps, order, motif_agg_min, batch_split)
    std::map<std::tuple<int, int, int, int, int, int, int>, Captured> graphs;
};

namespace gpm {

struct BatchParams {
    const int32_t* __restrict__ indptr;
    const int32_t* __restrict__ indices;
    const int32_t* __restrict__ off;      // DAG
    const int32_t* __restrict__ adj;
    const int32_t* __restrict__ outdeg;
    const int32_t* __restrict__ deg;
    const int32_t* __restrict__ goff;
    const int32_t* __restrict__ vgraph;
    const int32_t* __restrict__ units;    // (task << 31) | root
    const int32_t* __restrict__ uranges;  // (piece << 16) | pieces: the unit's share of the root's children
    long long n_units;
    int kc, km;                           // clique / motif sizes (0: task absent)
    int npat;
    const uint16_t* __restrict__ lut;
    // shared-memory layout (bytes per warp)
    int cq_maxd, cq_wmax, cq_words;
    int mark_stride;
    long long lvl_off[MT_MAXK + 1];
    int slab_ints;
    int agg_min, agg_words;               // aggregated motif tail (mt_tail_agg)
    int warp_bytes;
    unsigned long long* clique_out;       // [G]
    unsigned long long* motif_out;        // [G][npat]
    Control* ctl;
};

__global__ void __launch_bounds__(512) k_batch(BatchParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    unsigned char* base = smem_raw + (size_t)wib * p.warp_bytes;
    // clique part
    uint32_t* cq = reinterpret_cast<uint32_t*>(base);
    const CqLayout L = cq_layout(p.cq_maxd, p.cq_wmax, false);
    CliqueUnit* unit = reinterpret_cast<CliqueUnit*>(cq + L.unit);
    CliqueWalk cw{};
    cw.off = p.off;
    cw.adj = p.adj;
    cw.outdeg = p.outdeg;
    cw.deg = p.deg;
    cw.k_lo = p.kc;
    cw.k_hi = p.kc;
    cw.wmax = p.cq_wmax;
    cw.wcnt = reinterpret_cast<unsigned long long*>(cq + L.wcnt);
    cw.cur = reinterpret_cast<int*>(cq + L.cur);
    cw.hiv = reinterpret_cast<int*>(cq + L.hi);
    cw.cand = cq + L.cand;
    cw.list = reinterpret_cast<int*>(cq + L.list);
    cw.pairs = reinterpret_cast<int*>(cq + L.pairs);
    cw.rows = cq + L.rows;
    cw.ctl = p.ctl;
    cw.ring_seq = nullptr;
    cw.ring_ids = nullptr;
    cw.ring_cap = 0;
    cw.mbox = nullptr;
    cw.mbox_stride = 0;
    cw.donate_min = 0;
    cw.donate_after_ns = 0;
    cw.tail_levels = 0;
    cw.compact = 0;
    cw.compact3 = 0;
    cw.cpl = 0;
    cw.monitor = false;
    cw.spill = nullptr;
    cw.spill_cap = 0;
    // motif part
    unsigned char* mt = base + (size_t)p.cq_words * 4;
    MtWarp* W = reinterpret_cast<MtWarp*>(mt);
    unsigned long long* wc = reinterpret_cast<unsigned long long*>(mt + ((sizeof(MtWarp) + 15) & ~size_t(15)));
    uint32_t* agg = reinterpret_cast<uint32_t*>(wc + ((p.npat + 1) & ~1));
    unsigned char* marks = reinterpret_cast<unsigned char*>(agg + ((p.agg_words + 3) & ~3));
    int32_t* slab = reinterpret_cast<int32_t*>(marks + p.mark_stride);
    MotifWalk mw{};
    mw.indptr = p.indptr;
    mw.indices = p.indices;
    mw.lut = p.lut;
    mw.k = p.km;
    mw.mk = marks;
    mw.mbase = 0;
    mw.slab = slab;
    mw.lvl_off = p.lvl_off;
    mw.ctl = p.ctl;
    mw.ring_seq = nullptr;
    mw.ring_ids = nullptr;
    mw.ring_cap = 0;
    mw.mbox = nullptr;
    mw.mbox_stride = 0;
    mw.donate_min = 0;
    mw.donate_after_ns = 0;
    mw.err = &p.ctl->error;
    mw.agg = p.agg_words > 0 ? agg : nullptr;
    mw.agg_min = p.agg_words > 0 ? p.agg_min : 0;
    mw.monitor = false;
    mw.spill = nullptr;
    mw.spill_cap = 0;
    for (int v = lane; v < p.mark_stride; v += 32) marks[v] = 0;
    for (int j = lane; j < p.npat; j += 32) wc[j] = 0ull;
    __syncwarp();
    WarpSink sink{wc, &p.ctl->overflow};
    int cached_root = -1;
    Control* ctl = p.ctl;
    unsigned long long busy = 0;      // time spent inside work units (%globaltimer ns)

    for (;;) {
        const unsigned long long t_unit = gpm_globaltimer();
        unsigned long long u = 0;
        if (lane == 0) {
            u = *(volatile unsigned long long*)&ctl->next_root;
            if (u < (unsigned long long)p.n_units) u = atomicAdd(&ctl->next_root, 1ull);
        }
        u = __shfl_sync(GPM_FULL_MASK, u, 0);
        if (u >= (unsigned long long)p.n_units) break;
        const int code = p.units[u];
        const int task = (int)(((unsigned)code) >> 31);
        const int r = code & 0x7fffffff;
        const int gidx = p.vgraph[r];
        const int piece = p.uranges[u] >> 16, pieces = max(p.uranges[u] & 0xffff, 1);
        if (task == 0) {
            // ---- clique unit
            const int d = p.outdeg[r];
            unsigned long long sum = 0;
            if (lane == 0) {
                unit->root_pos = 0;
                unit->depth = 0;
                unit->lo = (int)((long long)d * piece / pieces);
                unit->hi = pieces > 1 ? (int)((long long)d * (piece + 1) / pieces) : -1;
            }
            __syncwarp();
            unsigned long long km1 = 0, wops = 0;
            cq_walk<false>(cw, unit, 0, r, d, cached_root, sum, km1, wops, lane);
            int ovf = 0;
            sum = gpm_warp_sum_cc(sum, ovf);
            if (lane == 0) {
                if (ovf) atomicExch(&ctl->overflow, 1);
                gpm_atomic_add_cc(&p.clique_out[gidx], sum, &ctl->overflow);
            }
        } else {
            // ---- motif unit
            mw.mbase = p.goff[gidx];
            if (lane == 0) W->sub[0] = r;
            __syncwarp();
            mt_setup_prefix(mw, W, 1, lane);
            const int lo = mt_root_ext_begin(p.indptr, p.indices, r, lane);
            if (lane == 0) {
                const int len = p.indptr[r + 1] - lo;
                W->len[1] = len;
                W->cur[1] = (int)((long long)len * piece / pieces);
                W->hi[1] = (int)((long long)len * (piece + 1) / pieces);
            }
            __syncwarp();
            unsigned long long leaves = 0, scanned = 0;
            mt_walk<false>(mw, W, 1, r, 0, p.indices + lo, sink, leaves, scanned, lane);
            mt_clear_prefix(mw, W, 1, lane);
            __syncwarp();
            for (int j = lane; j < p.npat; j += 32) {
                const unsigned long long v = wc[j];
                if (v) {
                    const unsigned long long old = atomicAdd(&p.motif_out[(long long)gidx * p.npat + j], v);
                    if (old + v < old) atomicExch(&ctl->overflow, 1);
                    wc[j] = 0ull;
                }
            }
            __syncwarp();
        }
        if (lane == 0) atomicAdd(&ctl->units_done, 1ull);
        busy += gpm_globaltimer() - t_unit;
    }
    if (lane == 0) atomicAdd(&ctl->busy_ns, busy);
}

// units: (task << 31) | root.  Mode 0: every motif root (heaviest degree
// first), then every clique root (heaviest out-degree first).  Mode 1: both
// tasks merged into one heaviest-first list (weights: degree for motif units,
// out-degree for clique units, scaled to a common range).
static long long build_units(gpm_batch* b, int kc, int km, int mode, int split, gpm::DevBuf& out,
                             gpm::DevBuf& out_ranges) {
    gpm_graph* g = b->g;
    const int n = g->n;
    std::vector<int32_t> deg(n), od(n);
    if (n > 0) {
        GPM_CUDA(cudaMemcpyAsync(deg.data(), g->degree.ptr, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, b->stream));
        if (kc > 0)
            GPM_CUDA(cudaMemcpyAsync(od.data(), g->dag_outdeg.ptr, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, b->stream));
    }
    GPM_CUDA(cudaStreamSynchronize(b->stream));
    std::vector<std::pair<double, int32_t>> items;
    if (km > 0)
        for (int v = 0; v < n; v++) items.push_back({(double)deg[v] * deg[v], (int32_t)v | (int32_t)0x80000000});
    if (kc > 0)
        for (int v = 0; v < n; v++)
            if (od[v] >= kc - 1) items.push_back({(double)od[v] * od[v] * (mode == 1 ? 4.0 : 1.0), v});
    if (mode == 0) {
        auto mid = std::stable_partition(items.begin(), items.end(), [](const auto& x) { return x.second < 0; });
        std::stable_sort(items.begin(), mid, [](const auto& x, const auto& y) { return x.first > y.first; });
        std::stable_sort(mid, items.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
    } else {
        std::stable_sort(items.begin(), items.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
    }
    // split: units heavier than 1/4096 of the total weight become `split`
    // units over equal ranges of the root's children (kept in place: the
    // order stays heaviest first)
    double total = 0.0;
    for (const auto& it : items) total += it.first;
    const int pieces = std::max(1, std::min(split, 64));
    std::vector<int32_t> codes, ranges;
    codes.reserve(items.size());
    ranges.reserve(items.size());
    for (const auto& it : items) {
        const int np = (pieces > 1 && it.first > total / 4096.0) ? pieces : 1;
        for (int q = 0; q < np; q++) {
            codes.push_back(it.second);
            ranges.push_back((q << 16) | np);
        }
    }
    out.ensure(sizeof(int32_t) * std::max<size_t>(codes.size(), 1));
    out_ranges.ensure(sizeof(int32_t) * std::max<size_t>(ranges.size(), 1));
    if (!codes.empty()) {
        GPM_CUDA(cudaMemcpyAsync(out.ptr, codes.data(), sizeof(int32_t) * codes.size(), cudaMemcpyHostToDevice,
                                 b->stream));
        GPM_CUDA(cudaMemcpyAsync(out_ranges.ptr, ranges.data(), sizeof(int32_t) * ranges.size(),
                                 cudaMemcpyHostToDevice, b->stream));
    }
    GPM_CUDA(cudaStreamSynchronize(b->stream));
    return (long long)codes.size();
}

static gpm_batch::Captured& capture(gpm_batch* b, int kc, int km) {
    gpm_graph* g = b->g;
    const int wpb = b->cfg.warps_per_block > 0 ? b->cfg.warps_per_block : 8;
    const int bps = b->cfg.blocks_per_sm;
    const int split = std::max(1, b->cfg.batch_split);
    const auto key = std::make_tuple(kc, km, wpb, bps, b->order_mode, b->cfg.motif_agg_min, split);
    auto it = b->graphs.find(key);
    if (it != b->graphs.end()) return it->second;

    if (kc > 0) ensure_dag(g);
    DevBuf units, uranges;
    const long long n_units = build_units(b, kc, km, b->order_mode, split, units, uranges);
    const int npat = km > 0 ? (int)pattern_table(km).num_patterns : 0;

    BatchParams p{};
    p.indptr = g->indptr.as<int32_t>();
    p.indices = g->indices.as<int32_t>();
    p.off = kc > 0 ? g->dag_off.as<int32_t>() : nullptr;
    p.adj = kc > 0 ? g->dag_adj.as<int32_t>() : nullptr;
    p.outdeg = kc > 0 ? g->dag_outdeg.as<int32_t>() : nullptr;
    p.deg = kc > 0 ? g->degree.as<int32_t>() : nullptr;
    p.goff = b->goff.as<int32_t>();
    p.vgraph = b->vgraph.as<int32_t>();
    p.units = units.as<int32_t>();
    p.uranges = uranges.as<int32_t>();
    p.n_units = n_units;
    p.kc = kc;
    p.km = km;
    p.npat = npat;
    p.lut = km > 0 ? device_lut(km) : nullptr;
    if (kc > 0 && g->max_outdeg > 1024) fail(GPM_ENOTIMPL, "batched clique counting needs out-degrees <= 1024");
    p.cq_maxd = std::max(kc > 0 ? g->max_outdeg : 1, 1);
    p.cq_wmax = (p.cq_maxd + 31) / 32;
    p.cq_words = cq_layout(p.cq_maxd, p.cq_wmax, false).total;
    p.mark_stride = (b->max_graph_n + 15) & ~15;
    long long off = 0;
    const long long D = std::max(g->max_deg, 1);
    for (int l = 0; l <= MT_MAXK; l++) {
        p.lvl_off[l] = off;
        if (km > 0 && l >= 1 && l <= km - 2) off += (long long)l * D + 4;
        off = (off + 3) & ~3ll;
    }
    p.slab_ints = (int)std::max(off, 4ll);
    p.agg_min = b->cfg.motif_agg_min;
    p.agg_words = (km > 0 && p.agg_min > 0) ? mt_agg_words(km) : 0;
    const size_t mt_bytes = ((sizeof(MtWarp) + 15) & ~size_t(15)) + sizeof(unsigned long long) * ((npat + 1) & ~1) +
                            4 * (size_t)((p.agg_words + 3) & ~3) + p.mark_stride + 4 * (size_t)p.slab_ints;
    p.warp_bytes = (int)((p.cq_words * 4 + mt_bytes + 15) & ~size_t(15));
    const size_t smem = (size_t)wpb * p.warp_bytes;
    if (smem > 227 * 1024) fail(GPM_ENOTIMPL, "batched state does not fit in shared memory (graphs too large)");
    GPM_CUDA(cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = resident_blocks((const void*)k_batch, wpb * 32, smem);
    if (per_sm <= 0) fail(GPM_EINVAL, "batched kernel cannot be resident with this configuration");
    if (bps > 0) per_sm = std::min(per_sm, bps);
    const int blocks = per_sm * g->num_sms;

    gpm_batch::Captured& c = b->graphs[key];
    c.units = std::move(units);
    c.uranges = std::move(uranges);
    const size_t G = (size_t)b->n_graphs;
    const size_t ctl_words = (sizeof(Control) + 7) / 8;
    c.words = G + G * npat + ctl_words;
    try {
        c.dev_out.ensure(sizeof(unsigned long long) * c.words);
        GPM_CUDA(cudaMallocHost(&c.host_out, sizeof(unsigned long long) * c.words));
    } catch (...) {
        b->graphs.erase(key);
        throw;
    }
    p.clique_out = c.dev_out.as<unsigned long long>();
    p.motif_out = p.clique_out + G;
    p.ctl = reinterpret_cast<Control*>(p.motif_out + G * npat);
    c.blocks = blocks;
    c.wpb = wpb;

    cudaGraph_t graph = nullptr;
    GPM_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e1 = cudaMemsetAsync(c.dev_out.ptr, 0, sizeof(unsigned long long) * c.words, b->stream);
    if (e1 == cudaSuccess && p.n_units > 0) {
        k_batch<<<blocks, wpb * 32, smem, b->stream>>>(p);
        e1 = cudaGetLastError();
    }
    if (e1 == cudaSuccess)
        e1 = cudaMemcpyAsync(c.host_out, c.dev_out.ptr, sizeof(unsigned long long) * c.words, cudaMemcpyDeviceToHost,
                             b->stream);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaFreeHost(c.host_out);
        b->graphs.erase(key);
        check_cuda(e1 != cudaSuccess ? e1 : e2, "CUDA graph capture of the batched launch");
    }
    cudaError_t e3 = cudaGraphInstantiate(&c.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e3 != cudaSuccess) {
        cudaFreeHost(c.host_out);
        b->graphs.erase(key);
        check_cuda(e3, "cudaGraphInstantiate");
    }
    return c;
}

// One replay; results in cap.host_out.  Returns the device time (ms).
static float replay(gpm_batch* b, gpm_batch::Captured& cap) {
    GPM_CUDA(cudaEventRecord(b->g->ev0, b->stream));
    GPM_CUDA(cudaGraphLaunch(cap.exec, b->stream));
    GPM_CUDA(cudaEventRecord(b->g->ev1, b->stream));
    GPM_CUDA(cudaStreamSynchronize(b->stream));
    float ms = 0.f;
    GPM_CUDA(cudaEventElapsedTime(&ms, b->g->ev0, b->g->ev1));
    return ms;
}

__global__ void k_vertex_graph(const int32_t* __restrict__ goff, int32_t n_graphs, int32_t* __restrict__ vgraph,
                               int* __restrict__ bad) {
    for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < n_graphs;
         gi += (long long)gridDim.x * blockDim.x) {
        const int a = goff[gi], z = goff[gi + 1];
        if (z < a) {
            atomicOr(bad, 1);
            continue;
        }
        for (int v = a; v < z; v++) vgraph[v] = (int32_t)gi;
    }
}

// every edge stays inside its graph
__global__ void k_edges_inside(const int32_t* __restrict__ indptr, const int32_t* __restrict__ indices,
                               const int32_t* __restrict__ vgraph, int32_t n, int* __restrict__ bad) {
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
        for (int t = indptr[v]; t < indptr[v + 1]; t++)
            if (vgraph[indices[t]] != vgraph[v]) atomicOr(bad, 2);
}

gpm_batch* create_batch(const int32_t* graph_off, const int32_t* indptr, const int32_t* indices, int32_t n_graphs,
                        uint32_t flags, void* stream) {
    if (n_graphs < 0 || !graph_off) fail(GPM_EINVAL, "bad graph offsets");
    const bool dev = (flags & GPM_DEVICE_PTRS) != 0;
    std::vector<int32_t> goff(n_graphs + 1);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (dev) {
        GPM_CUDA(cudaMemcpyAsync(goff.data(), graph_off, sizeof(int32_t) * (n_graphs + 1), cudaMemcpyDeviceToHost, s));
        GPM_CUDA(cudaStreamSynchronize(s));
    } else {
        std::copy(graph_off, graph_off + n_graphs + 1, goff.begin());
    }
    if (goff[0] != 0) fail(GPM_EINVAL, "graph_off[0] != 0");
    int32_t maxn = 0;
    for (int32_t i = 0; i < n_graphs; i++) {
        if (goff[i + 1] < goff[i]) fail(GPM_EINVAL, "graph_off is not non-decreasing");
        maxn = std::max(maxn, goff[i + 1] - goff[i]);
    }
    gpm_batch* b = new gpm_batch();
    try {
        b->g = create_graph(indptr, indices, goff[n_graphs], flags, stream);
        b->n_graphs = n_graphs;
        b->max_graph_n = maxn;
        b->cfg = default_config();
        if (s) {
            b->stream = s;
        } else {
            GPM_CUDA(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
            b->own_stream = true;
        }
        b->g->stream = b->stream;
        b->goff.ensure(sizeof(int32_t) * (n_graphs + 1));
        GPM_CUDA(cudaMemcpyAsync(b->goff.ptr, goff.data(), sizeof(int32_t) * (n_graphs + 1), cudaMemcpyHostToDevice,
                                 b->stream));
        const int32_t n = b->g->n;
        b->vgraph.ensure(sizeof(int32_t) * std::max(n, 1));
        DevBuf flag;
        flag.ensure(sizeof(int));
        GPM_CUDA(cudaMemsetAsync(flag.ptr, 0, sizeof(int), b->stream));
        if (n_graphs > 0)
            k_vertex_graph<<<std::max(1, std::min((n_graphs + 255) / 256, 4096)), 256, 0, b->stream>>>(
                b->goff.as<int32_t>(), n_graphs, b->vgraph.as<int32_t>(), flag.as<int>());
        if (n > 0 && !(flags & GPM_SKIP_VALIDATE))
            k_edges_inside<<<std::max(1, std::min((n + 255) / 256, 4096)), 256, 0, b->stream>>>(
                b->g->indptr.as<int32_t>(), b->g->indices.as<int32_t>(), b->vgraph.as<int32_t>(), n, flag.as<int>());
        GPM_CUDA(cudaGetLastError());
        int hb = 0;
        GPM_CUDA(cudaMemcpyAsync(&hb, flag.ptr, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
        GPM_CUDA(cudaStreamSynchronize(b->stream));
        if (hb) fail(GPM_EINVAL, "an edge joins two different graphs of the batch");
    } catch (...) {
        if (b->g) destroy_graph(b->g);
        if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
        delete b;
        throw;
    }
    return b;
}

void destroy_batch(gpm_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (auto& kv : b->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.host_out) cudaFreeHost(kv.second.host_out);
    }
    b->graphs.clear();
    b->g->stream = nullptr;
    destroy_graph(b->g);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

void batch_count(gpm_batch* b, int kc, int km, uint64_t* clique_counts, uint64_t* motif_counts) {
    if (kc < 0 || kc > GPM_CLIQUE_MAX_K) fail(GPM_EINVAL, "clique k out of range [0, 16]");
    if (km < 0 || km > 7) fail(GPM_EINVAL, "batched motif k out of range [0, 7] (k = 8 needs global counters)");
    if (kc > 0 && kc < 3) fail(GPM_EINVAL, "batched clique counting needs k >= 3");
    if (km > 0 && km < 3) fail(GPM_EINVAL, "batched motif counting needs k >= 3");
    if (kc > 0 && !clique_counts) fail(GPM_EINVAL, "clique_counts is NULL");
    if (km > 0 && !motif_counts) fail(GPM_EINVAL, "motif_counts is NULL");
    gpm_batch::Captured& cap = capture(b, kc, km);
    const float ms = replay(b, cap);
    const size_t G = (size_t)b->n_graphs;
    const int npat = km > 0 ? (int)pattern_table(km).num_patterns : 0;
    const Control* h = reinterpret_cast<const Control*>(cap.host_out + G + G * npat);
    gpm_stats st{};
    st.kernel_ms = ms;
    st.units_done = h->units_done;
    st.busy_warp_ns = h->busy_ns;
    st.kernel_launches = 1;
    st.grid_blocks = cap.blocks;
    st.warps_per_block = cap.wpb;
    b->stats = st;
    if (h->error == DEV_EINVAL) fail(GPM_ECUDA, "pattern table lookup hit an invalid traversal code");
    if (h->error >= DEV_ECHECK) fail(GPM_ECUDA, "device consistency check " + std::to_string(h->error - DEV_ECHECK) + " failed");
    if (h->error) fail(GPM_ECUDA, "device error " + std::to_string(h->error));
    if (h->overflow) fail(GPM_EOVERFLOW, "a per-graph count exceeds 2^64-1");
    if (kc > 0) std::copy(cap.host_out, cap.host_out + G, clique_counts);
    if (km > 0) std::copy(cap.host_out + G, cap.host_out + G + G * npat, motif_counts);
}

// Time every candidate launch shape (median of reps replays) and keep the best.
gpm_config batch_autotune(gpm_batch* b, int kc, int km, int reps, double* best_ms) {
    static std::map<std::tuple<int, long long, long long, int, int>, std::pair<gpm_config, int>> cache;
    int dev = 0;
    GPM_CUDA(cudaGetDevice(&dev));
    const auto sig = std::make_tuple(dev, (long long)b->g->n, (long long)b->g->nnz, kc, km);
    auto hit = cache.find(sig);
    if (hit != cache.end()) {
        b->cfg = hit->second.first;
        b->order_mode = hit->second.second;
        if (best_ms) *best_ms = -1.0;
        return b->cfg;
    }
    gpm_config best = b->cfg;
    int best_mode = b->order_mode;
    double best_t = 1e300;
    const gpm_config saved = b->cfg;
    auto trial = [&](const gpm_config& c, int mode) {
        b->cfg = c;
        b->order_mode = mode;
        std::vector<float> t;
        try {
            gpm_batch::Captured& cap = capture(b, kc, km);
            replay(b, cap);   // warm
            for (int r = 0; r < std::max(1, reps); r++) t.push_back(replay(b, cap));
        } catch (const Error&) {
            return;           // shape not launchable (shared memory): skip it
        }
        std::sort(t.begin(), t.end());
        const double med = t[t.size() / 2];
        if (med < best_t) {
            best_t = med;
            best = c;
            best_mode = mode;
        }
    };
    // stage 1: launch shape and unit order
    for (int mode = 0; mode < 2; mode++)
        for (int wpb : {2, 4, 8, 16})
            for (int bps : {0, 1, 2}) {
                gpm_config c = saved;
                c.warps_per_block = wpb;
                c.blocks_per_sm = bps;
                trial(c, mode);
            }
    // stage 2: class-counting threshold of the motif tail (0: leaf by leaf)
    if (km > 0) {
        const gpm_config base = best;
        const int mode = best_mode;
        for (int agg : {0, 4, 16, 64}) {
            if (agg == base.motif_agg_min) continue;
            gpm_config c = base;
            c.motif_agg_min = agg;
            trial(c, mode);
        }
    }
    // stage 3: split of the heaviest roots into child ranges
    {
        const gpm_config base = best;
        const int mode = best_mode;
        for (int split : {1, 4, 16}) {
            if (split == std::max(1, base.batch_split)) continue;
            gpm_config c = base;
            c.batch_split = split;
            trial(c, mode);
        }
    }
    b->cfg = best;
    b->order_mode = best_mode;
    cache[sig] = {best, best_mode};
    if (best_ms) *best_ms = best_t;
    return best;
}

void batch_set_config(gpm_batch* b, const gpm_config& c) {
    if (c.warps_per_block < 0 || c.warps_per_block > 16 || (c.warps_per_block & (c.warps_per_block - 1)))
        fail(GPM_EINVAL, "warps_per_block must be a power of two in [1, 16]");
    if (c.blocks_per_sm < 0) fail(GPM_EINVAL, "blocks_per_sm < 0");
    if (c.motif_agg_min < 0) fail(GPM_EINVAL, "motif_agg_min < 0");
    if (c.batch_split < 0 || c.batch_split > 64) fail(GPM_EINVAL, "batch_split must be in [0, 64]");
    b->cfg = c;
}

gpm_stats batch_stats(const gpm_batch* b) { return b->stats; }

}  // namespace gpm
