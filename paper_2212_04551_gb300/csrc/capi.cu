// capi.cu -- the extern "C" boundary of libgpm (declared in include/gpm.h).
//
// Every entry point validates its arguments, runs the work on the graph's
// stream, synchronises before handing host results back, and maps internal
// failures to a gpm_status plus a thread-local message.  No exception, abort
// or trap crosses this boundary.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"

namespace gpm {
gpm_batch* create_batch(const int32_t* graph_off, const int32_t* indptr, const int32_t* indices, int32_t n_graphs,
                        uint32_t flags, void* stream);
void destroy_batch(gpm_batch* b);
void batch_count(gpm_batch* b, int kc, int km, uint64_t* clique_counts, uint64_t* motif_counts);
gpm_config batch_autotune(gpm_batch* b, int kc, int km, int reps, double* best_ms);
void batch_set_config(gpm_batch* b, const gpm_config& c);
gpm_stats batch_stats(const gpm_batch* b);
gpm_graph* create_graph(const int32_t* indptr, const int32_t* indices, int32_t n, uint32_t flags, void* stream);
void destroy_graph(gpm_graph* g);
const char* last_error_cstr();
}  // namespace gpm

using namespace gpm;

template <class F>
static gpm_status guarded(F&& f) {
    try {
        clear_error();
        f();
        return GPM_OK;
    } catch (const Error& e) {
        set_error(e.msg);
        return e.status;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return GPM_ENOMEM;
    } catch (...) {
        set_error("unexpected internal error");
        return GPM_ECUDA;
    }
}

// Copy a host root list to the device (validated), or pass NULL through.
static const int32_t* upload_roots(gpm_graph* g, const int32_t* roots, int64_t n_roots) {
    if (!roots) return nullptr;
    if (n_roots < 0) fail(GPM_EINVAL, "n_roots < 0");
    for (int64_t i = 0; i < n_roots; i++)
        if (roots[i] < 0 || roots[i] >= g->n) fail(GPM_EINVAL, "root id out of range");
    g->roots_tmp.ensure(sizeof(int32_t) * std::max<int64_t>(n_roots, 1));
    if (n_roots > 0)
        GPM_CUDA(cudaMemcpyAsync(g->roots_tmp.ptr, roots, sizeof(int32_t) * n_roots, cudaMemcpyHostToDevice,
                                 g->stream));
    return g->roots_tmp.as<int32_t>();
}

static void check_graph(const gpm_graph* g) {
    if (!g) fail(GPM_EINVAL, "graph is NULL");
}

static const int32_t* custom_or_null(gpm_graph* g, int64_t* n_roots) {
    if (g->cfg.order == GPM_ORDER_CUSTOM) {
        if (g->order_custom_len <= 0) fail(GPM_EINVAL, "GPM_ORDER_CUSTOM is selected but no root order was set");
        *n_roots = g->order_custom_len;
        return g->order_custom.as<int32_t>();
    }
    if (g->cfg.order == GPM_ORDER_ID) {
        *n_roots = g->n;
        return ensure_id_order(g);
    }
    return nullptr;   // heaviest-first order, chosen per application
}

// The schedule of app over a root list: roots ordered by score descending
// (the plain order when scores is NULL), then the roots chosen by
// `chunks_of` (score-ordered position, score -> units; 1 = not split) moved to
// the kernel list's end with their unit counts.
template <class ChunksOf>
static void build_schedule(gpm_graph* g, int app, const float* scores, const int32_t* roots, int64_t n_roots,
                           ChunksOf chunks_of, bool uniform, int32_t uniform_chunks) {
    if (app != GPM_APP_CLIQUE && app != GPM_APP_MOTIF) fail(GPM_EINVAL, "unknown app");
    const int64_t nr = roots ? n_roots : g->n;
    if (nr < 0) fail(GPM_EINVAL, "n_roots < 0");
    // the caller's list (validated: ids in range, each once)
    std::vector<int32_t> list(nr);
    if (roots) {
        std::vector<uint8_t> seen(g->n, 0);
        for (int64_t i = 0; i < nr; i++) {
            const int32_t r = roots[i];
            if (r < 0 || r >= g->n) fail(GPM_EINVAL, "root id out of range");
            if (seen[r]) fail(GPM_EINVAL, "root listed twice");
            seen[r] = 1;
            list[i] = r;
        }
    } else {
        for (int64_t i = 0; i < nr; i++) list[i] = (int32_t)i;
    }
    DevBuf d_list, d_key;
    d_list.ensure(sizeof(int32_t) * std::max<int64_t>(nr, 1));
    if (nr > 0)
        GPM_CUDA(cudaMemcpyAsync(d_list.ptr, list.data(), sizeof(int32_t) * nr, cudaMemcpyHostToDevice, g->stream));
    const float* key = scores;
    if (!key) {
        // plain order: degree (motif) or oriented out-degree (clique) as the score
        if (app == GPM_APP_CLIQUE) ensure_dag(g);
        std::vector<int32_t> dh(g->n);
        const DevBuf& src = app == GPM_APP_CLIQUE ? g->dag_outdeg : g->degree;
        if (g->n > 0)
            GPM_CUDA(cudaMemcpyAsync(dh.data(), src.ptr, sizeof(int32_t) * g->n, cudaMemcpyDeviceToHost, g->stream));
        GPM_CUDA(cudaStreamSynchronize(g->stream));
        std::vector<float> fh(g->n);
        for (int32_t v = 0; v < g->n; v++) fh[v] = (float)dh[v];
        d_key.ensure(sizeof(float) * std::max(g->n, 1));
        if (g->n > 0)
            GPM_CUDA(cudaMemcpyAsync(d_key.ptr, fh.data(), sizeof(float) * g->n, cudaMemcpyHostToDevice, g->stream));
        key = d_key.as<float>();
    }
    auto& S = g->sched[app];
    S.ready = false;
    order_by_score(g, key, d_list.as<int32_t>(), nr, S.roots);
    std::vector<int32_t> ord(nr);
    if (nr > 0)
        GPM_CUDA(cudaMemcpyAsync(ord.data(), S.roots.ptr, sizeof(int32_t) * nr, cudaMemcpyDeviceToHost, g->stream));
    std::vector<float> sc;
    if (scores && g->n > 0) {
        sc.resize(g->n);
        GPM_CUDA(cudaMemcpyAsync(sc.data(), scores, sizeof(float) * g->n, cudaMemcpyDeviceToHost, g->stream));
    }
    GPM_CUDA(cudaStreamSynchronize(g->stream));
    // the kernel takes the split roots from the END of its list (their
    // relative order kept)
    std::vector<int32_t> kern, split;
    std::vector<int32_t> off(1, 0);
    kern.reserve(nr);
    for (int64_t i = 0; i < nr; i++) {
        const int32_t ch = chunks_of(i, sc.empty() ? 0.f : sc[ord[i]]);
        if (ch > 1) {
            split.push_back(ord[i]);
            off.push_back(off.back() + ch);
        } else {
            kern.push_back(ord[i]);
        }
    }
    const int64_t ns = (int64_t)split.size();
    kern.insert(kern.end(), split.begin(), split.end());
    std::vector<int64_t> where(g->n, -1);
    for (int64_t i = 0; i < nr; i++) where[list[i]] = i;
    S.caller_index.assign(nr, 0);
    for (int64_t i = 0; i < nr; i++) S.caller_index[i] = where[kern[i]];
    if (nr > 0)
        GPM_CUDA(cudaMemcpyAsync(S.roots.ptr, kern.data(), sizeof(int32_t) * nr, cudaMemcpyHostToDevice, g->stream));
    S.n = nr;
    S.n_counter = nr - ns;
    S.n_seeds = off.back();
    S.chunks = uniform && ns > 0 ? uniform_chunks : 0;
    S.chunk_off.release();
    if (!uniform && ns > 0) {
        S.chunk_off.ensure(sizeof(int32_t) * off.size());
        GPM_CUDA(cudaMemcpyAsync(S.chunk_off.ptr, off.data(), sizeof(int32_t) * off.size(), cudaMemcpyHostToDevice,
                                 g->stream));
    }
    GPM_CUDA(cudaStreamSynchronize(g->stream));
    S.ready = true;
}

extern "C" {

gpm_status gpm_graph_create(const int32_t* indptr, const int32_t* indices, int32_t n, uint32_t flags,
                            void* stream, gpm_graph** out) {
    return guarded([&] {
        if (!out) fail(GPM_EINVAL, "out is NULL");
        *out = nullptr;
        *out = create_graph(indptr, indices, n, flags, stream);
    });
}

void gpm_graph_destroy(gpm_graph* g) {
    try {
        destroy_graph(g);
    } catch (...) {
    }
}

gpm_status gpm_graph_info(const gpm_graph* g, int32_t* n, int64_t* m, int32_t* max_degree) {
    return guarded([&] {
        check_graph(g);
        if (n) *n = g->n;
        if (m) *m = g->nnz / 2;
        if (max_degree) *max_degree = g->max_deg;
    });
}

gpm_status gpm_clique_count(gpm_graph* g, int k, uint64_t* out_count) {
    return guarded([&] {
        check_graph(g);
        if (!out_count) fail(GPM_EINVAL, "out_count is NULL");
        if (k < 1 || k > GPM_CLIQUE_MAX_K) fail(GPM_EINVAL, "k out of range [1, 16]");
        int64_t nr = 0;
        const int32_t* roots = custom_or_null(g, &nr);
        uint64_t c = 0;
        run_clique(g, k, k, roots, nr, nullptr, &c);
        *out_count = c;
    });
}

gpm_status gpm_clique_count_range(gpm_graph* g, int k_lo, int k_hi, uint64_t* counts) {
    return guarded([&] {
        check_graph(g);
        if (!counts) fail(GPM_EINVAL, "counts is NULL");
        if (k_lo < 3 || k_hi > GPM_CLIQUE_MAX_K || k_lo > k_hi) fail(GPM_EINVAL, "need 3 <= k_lo <= k_hi <= 16");
        int64_t nr = 0;
        const int32_t* roots = custom_or_null(g, &nr);
        std::vector<uint64_t> c(k_hi - k_lo + 1, 0);
        run_clique(g, k_lo, k_hi, roots, nr, nullptr, c.data());
        std::memcpy(counts, c.data(), sizeof(uint64_t) * c.size());
    });
}

gpm_status gpm_motif_count(gpm_graph* g, int k, uint64_t* counts, int64_t counts_len) {
    return guarded([&] {
        check_graph(g);
        if (!counts) fail(GPM_EINVAL, "counts is NULL");
        if (k < 1 || k > GPM_MOTIF_MAX_K) fail(GPM_EINVAL, "k out of range [1, 8]");
        const PatternTable& t = pattern_table(k);
        if (counts_len < t.num_patterns) fail(GPM_EINVAL, "counts_len smaller than the number of patterns");
        int64_t nr = 0;
        const int32_t* roots = custom_or_null(g, &nr);
        std::vector<uint64_t> c(t.num_patterns, 0);
        run_motif(g, k, roots, nr, nullptr, c.data());
        std::memcpy(counts, c.data(), sizeof(uint64_t) * c.size());
    });
}

gpm_status gpm_motif_num_patterns(int k, int64_t* out) {
    return guarded([&] {
        if (!out) fail(GPM_EINVAL, "out is NULL");
        if (k < 1 || k > GPM_MOTIF_MAX_K) fail(GPM_EINVAL, "k out of range [1, 8]");
        *out = pattern_table(k).num_patterns;
    });
}

gpm_status gpm_motif_pattern(int k, int64_t id, uint64_t* adj_code) {
    return guarded([&] {
        if (!adj_code) fail(GPM_EINVAL, "adj_code is NULL");
        if (k < 1 || k > GPM_MOTIF_MAX_K) fail(GPM_EINVAL, "k out of range [1, 8]");
        const PatternTable& t = pattern_table(k);
        if (id < 0 || id >= t.num_patterns) fail(GPM_EINVAL, "pattern id out of range");
        *adj_code = t.pattern_code[(size_t)id];
    });
}

gpm_status gpm_count_roots(gpm_graph* g, int app, int k, const int32_t* roots, int64_t n_roots,
                           uint64_t* counts, int64_t counts_len, uint64_t* per_root) {
    return guarded([&] {
        check_graph(g);
        if (!counts) fail(GPM_EINVAL, "counts is NULL");
        if (app != GPM_APP_CLIQUE && app != GPM_APP_MOTIF) fail(GPM_EINVAL, "unknown app");
        const int64_t nr = roots ? n_roots : g->n;
        const int32_t* d_roots = upload_roots(g, roots, n_roots);
        if (!d_roots) {
            // all vertices in id order
            std::vector<int32_t> all(g->n);
            for (int32_t v = 0; v < g->n; v++) all[v] = v;
            d_roots = upload_roots(g, all.data(), g->n);
        }
        unsigned long long* d_pr = nullptr;
        if (per_root) {
            g->per_root_tmp.ensure(sizeof(unsigned long long) * std::max<int64_t>(nr, 1));
            d_pr = g->per_root_tmp.as<unsigned long long>();
        }
        std::vector<uint64_t> c;
        if (app == GPM_APP_CLIQUE) {
            if (k < 1 || k > GPM_CLIQUE_MAX_K) fail(GPM_EINVAL, "k out of range [1, 16]");
            if (counts_len < 1) fail(GPM_EINVAL, "counts_len < 1");
            c.assign(1, 0);
            run_clique(g, k, k, d_roots, nr, d_pr, c.data());
        } else {
            if (k < 1 || k > GPM_MOTIF_MAX_K) fail(GPM_EINVAL, "k out of range [1, 8]");
            const PatternTable& t = pattern_table(k);
            if (counts_len < t.num_patterns) fail(GPM_EINVAL, "counts_len smaller than the number of patterns");
            c.assign(t.num_patterns, 0);
            run_motif(g, k, d_roots, nr, d_pr, c.data());
        }
        if (per_root && nr > 0) {
            GPM_CUDA(cudaMemcpyAsync(per_root, d_pr, sizeof(uint64_t) * nr, cudaMemcpyDeviceToHost, g->stream));
            GPM_CUDA(cudaStreamSynchronize(g->stream));
        }
        std::memcpy(counts, c.data(), sizeof(uint64_t) * c.size());
    });
}

gpm_status gpm_clique_count_dfs(gpm_graph* g, int k, uint64_t* out_count) {
    return guarded([&] {
        check_graph(g);
        if (!out_count) fail(GPM_EINVAL, "out_count is NULL");
        uint64_t c = 0;
        run_clique_dfs(g, k, &c);
        *out_count = c;
    });
}

gpm_status gpm_list(gpm_graph* g, int app, int k, int32_t pattern, int64_t ring_records, gpm_list_consumer consumer,
                    void* user, uint64_t* delivered) {
    if (delivered) *delivered = 0;
    return guarded([&] {
        check_graph(g);
        run_list(g, app, k, pattern, ring_records, consumer, user, delivered);
    });
}

gpm_status gpm_count_monitored(gpm_graph* g, int app, int k, double threshold, uint64_t* counts, int64_t counts_len,
                               gpm_monitor_stats* stats) {
    return guarded([&] {
        check_graph(g);
        if (!counts) fail(GPM_EINVAL, "counts is NULL");
        if (!(threshold >= 0.0 && threshold <= 1.0)) fail(GPM_EINVAL, "threshold must be in [0, 1]");
        MonitorStats ms{};
        std::vector<uint64_t> c;
        if (app == GPM_APP_CLIQUE) {
            if (counts_len < 1) fail(GPM_EINVAL, "counts_len < 1");
            c.assign(1, 0);
            run_clique_monitored(g, k, threshold, c.data(), &ms);
        } else if (app == GPM_APP_MOTIF) {
            if (k < 3 || k > GPM_MOTIF_MAX_K) fail(GPM_EINVAL, "k out of range [3, 8]");
            const PatternTable& t = pattern_table(k);
            if (counts_len < t.num_patterns) fail(GPM_EINVAL, "counts_len smaller than the number of patterns");
            c.assign(t.num_patterns, 0);
            run_motif_monitored(g, k, threshold, c.data(), &ms);
        } else {
            fail(GPM_EINVAL, "unknown app");
        }
        std::memcpy(counts, c.data(), sizeof(uint64_t) * c.size());
        if (stats) {
            stats->launches = ms.launches;
            stats->pad = 0;
            stats->spilled_units = ms.spilled_units;
            stats->kernel_ms = ms.kernel_ms;
            stats->wall_ms = ms.wall_ms;
        }
    });
}

gpm_status gpm_get_config(const gpm_graph* g, gpm_config* out) {
    return guarded([&] {
        check_graph(g);
        if (!out) fail(GPM_EINVAL, "out is NULL");
        *out = g->cfg;
    });
}

gpm_status gpm_set_config(gpm_graph* g, const gpm_config* cfg) {
    return guarded([&] {
        check_graph(g);
        if (!cfg) fail(GPM_EINVAL, "cfg is NULL");
        gpm_config c = *cfg;
        if (c.warps_per_block != 0 && c.warps_per_block != 1 && c.warps_per_block != 2 && c.warps_per_block != 4 &&
            c.warps_per_block != 8 && c.warps_per_block != 16)
            fail(GPM_EINVAL, "warps_per_block must be a power of two in [1, 16]");
        if (c.blocks_per_sm < 0) fail(GPM_EINVAL, "blocks_per_sm < 0");
        if (c.donate_min < 0) fail(GPM_EINVAL, "donate_min < 0");
        if (c.order < GPM_ORDER_ID || c.order > GPM_ORDER_CUSTOM) fail(GPM_EINVAL, "unknown order");
        if (c.max_idle_ms <= 0) fail(GPM_EINVAL, "max_idle_ms must be positive");
        if (c.donate_after_us < 0) fail(GPM_EINVAL, "donate_after_us < 0");
        if (c.clique_tail != 0 && c.clique_tail != 2 && c.clique_tail != 3) fail(GPM_EINVAL, "clique_tail must be 0, 2 or 3");
        if (c.clique_compact < 0 || c.clique_compact > 2) fail(GPM_EINVAL, "clique_compact must be 0, 1 or 2");
        if (c.motif_agg_min < 0) fail(GPM_EINVAL, "motif_agg_min < 0");
        if (c.clique_compact3 < 0 || c.clique_compact3 > 2) fail(GPM_EINVAL, "clique_compact3 must be 0, 1 or 2");
        if (c.batch_split < 0 || c.batch_split > 64) fail(GPM_EINVAL, "batch_split must be in [0, 64]");
        if (c.clique_cpl < 0 || c.clique_cpl > 100) fail(GPM_EINVAL, "clique_cpl must be in [0, 100]");
        g->cfg = c;
    });
}

gpm_status gpm_get_stats(const gpm_graph* g, gpm_stats* out) {
    return guarded([&] {
        check_graph(g);
        if (!out) fail(GPM_EINVAL, "out is NULL");
        *out = g->stats;
    });
}

gpm_status gpm_root_features(gpm_graph* g, int k, float* out, uint32_t flags) {
    return guarded([&] {
        check_graph(g);
        if (!out) fail(GPM_EINVAL, "out is NULL");
        if (k < 1 || k > GPM_CLIQUE_MAX_K) fail(GPM_EINVAL, "k out of range [1, 16]");
        if (flags & GPM_DEVICE_PTRS) {
            root_features(g, k, out);
        } else {
            DevBuf tmp;
            tmp.ensure(sizeof(float) * 8 * std::max(g->n, 1));
            root_features(g, k, tmp.as<float>());
            GPM_CUDA(cudaMemcpyAsync(out, tmp.ptr, sizeof(float) * 8 * g->n, cudaMemcpyDeviceToHost, g->stream));
            GPM_CUDA(cudaStreamSynchronize(g->stream));
        }
    });
}

gpm_status gpm_mlp_forward(const uint16_t* w_bf16, const float* x, int64_t n, float* y, void* stream) {
    return guarded([&] {
        if (n < 0) fail(GPM_EINVAL, "n < 0");
        if (n > 0 && (!w_bf16 || !x || !y)) fail(GPM_EINVAL, "NULL pointer");
        mlp_forward(w_bf16, x, n, y, reinterpret_cast<cudaStream_t>(stream));
    });
}

gpm_status gpm_mlp_grad(const uint16_t* w_bf16, const float* x, const float* t, int64_t n, float* grad,
                        float* loss, void* stream) {
    return guarded([&] {
        if (n < 0) fail(GPM_EINVAL, "n < 0");
        if (!w_bf16 || !grad || !loss || (n > 0 && (!x || !t))) fail(GPM_EINVAL, "NULL pointer");
        mlp_grad(w_bf16, x, t, n, grad, loss, reinterpret_cast<cudaStream_t>(stream));
    });
}

gpm_status gpm_mlp_adam(float* master, float* m, float* v, const float* grad, int32_t step, float lr,
                        uint16_t* w_bf16, void* stream) {
    return guarded([&] {
        if (!master || !m || !v || !grad || !w_bf16) fail(GPM_EINVAL, "NULL pointer");
        if (step < 1) fail(GPM_EINVAL, "step must be >= 1");
        mlp_adam(master, m, v, grad, step, lr, w_bf16, reinterpret_cast<cudaStream_t>(stream));
    });
}

gpm_status gpm_sched_from_scores(gpm_graph* g, int app, const float* scores, const int32_t* roots,
                                 int64_t n_roots, int32_t split_roots, int32_t split_chunks) {
    return guarded([&] {
        check_graph(g);
        if (split_roots < 0 || split_chunks < 0) fail(GPM_EINVAL, "negative split");
        const bool on = split_chunks > 1;
        build_schedule(g, app, scores, roots, n_roots,
                       [&](int64_t i, float) { return (on && i < split_roots) ? split_chunks : 1; }, true,
                       split_chunks);
    });
}

gpm_status gpm_sched_balanced(gpm_graph* g, int app, const float* scores, const int32_t* roots, int64_t n_roots,
                              int64_t target_units, int32_t max_chunks) {
    return guarded([&] {
        check_graph(g);
        if (!scores) fail(GPM_EINVAL, "scores is NULL");
        if (target_units < 1 || max_chunks < 1 || max_chunks > 4096) fail(GPM_EINVAL, "bad target_units or max_chunks");
        // predicted sizes of the listed roots (scores are log1p of a size)
        const int64_t nr = roots ? n_roots : g->n;
        std::vector<float> sc(g->n);
        if (g->n > 0)
            GPM_CUDA(cudaMemcpyAsync(sc.data(), scores, sizeof(float) * g->n, cudaMemcpyDeviceToHost, g->stream));
        GPM_CUDA(cudaStreamSynchronize(g->stream));
        auto size_of = [](float s) { return std::expm1(std::min(std::max((double)s, 0.0), 80.0)); };
        double total = 0.0;
        for (int64_t i = 0; i < nr; i++) {
            const int32_t r = roots ? roots[i] : (int32_t)i;
            if (r >= 0 && r < g->n) total += size_of(sc[r]);
        }
        const double share = total / (double)target_units;
        // at most 65,536 units in all (the seed list's capacity)
        int64_t budget = 65536;
        build_schedule(g, app, scores, roots, n_roots,
                       [&](int64_t, float s) {
                           if (share <= 0.0) return 1;
                           int32_t ch = (int32_t)std::min<double>(std::ceil(size_of(s) / share), (double)max_chunks);
                           ch = (int32_t)std::min<int64_t>(std::max(ch, 1), budget);
                           if (ch > 1) budget -= ch;
                           return ch;
                       },
                       false, 0);
    });
}

gpm_status gpm_count_scheduled(gpm_graph* g, int app, int k, uint64_t* counts, int64_t counts_len,
                               uint64_t* per_root) {
    return guarded([&] {
        check_graph(g);
        if (!counts) fail(GPM_EINVAL, "counts is NULL");
        if (app != GPM_APP_CLIQUE && app != GPM_APP_MOTIF) fail(GPM_EINVAL, "unknown app");
        auto& S = g->sched[app];
        if (!S.ready) fail(GPM_EINVAL, "no schedule set for this app (gpm_sched_from_scores / gpm_sched_balanced)");
        SplitPlan plan;
        plan.chunks = S.chunks;
        plan.d_chunk_off = S.chunk_off.ptr ? S.chunk_off.as<int32_t>() : nullptr;
        plan.n_seeds = S.n_seeds;
        unsigned long long* d_pr = nullptr;
        if (per_root) {
            g->per_root_tmp.ensure(sizeof(unsigned long long) * std::max<int64_t>(S.n, 1));
            d_pr = g->per_root_tmp.as<unsigned long long>();
        }
        std::vector<uint64_t> c;
        if (app == GPM_APP_CLIQUE) {
            if (k < 1 || k > GPM_CLIQUE_MAX_K) fail(GPM_EINVAL, "k out of range [1, 16]");
            if (counts_len < 1) fail(GPM_EINVAL, "counts_len < 1");
            c.assign(1, 0);
            run_clique(g, k, k, S.roots.as<int32_t>(), S.n, d_pr, c.data(), S.n_counter, &plan);
        } else {
            if (k < 1 || k > GPM_MOTIF_MAX_K) fail(GPM_EINVAL, "k out of range [1, 8]");
            const PatternTable& t = pattern_table(k);
            if (counts_len < t.num_patterns) fail(GPM_EINVAL, "counts_len smaller than the number of patterns");
            c.assign(t.num_patterns, 0);
            run_motif(g, k, S.roots.as<int32_t>(), S.n, d_pr, c.data(), S.n_counter, &plan);
        }
        if (per_root && S.n > 0) {
            std::vector<uint64_t> tmp(S.n);
            GPM_CUDA(cudaMemcpyAsync(tmp.data(), d_pr, sizeof(uint64_t) * S.n, cudaMemcpyDeviceToHost, g->stream));
            GPM_CUDA(cudaStreamSynchronize(g->stream));
            for (int64_t i = 0; i < S.n; i++) per_root[S.caller_index[i]] = tmp[i];
        }
        std::memcpy(counts, c.data(), sizeof(uint64_t) * c.size());
    });
}

gpm_status gpm_batch_create(const int32_t* graph_off, const int32_t* indptr, const int32_t* indices,
                            int32_t n_graphs, uint32_t flags, void* stream, gpm_batch** out) {
    return guarded([&] {
        if (!out) fail(GPM_EINVAL, "out is NULL");
        *out = nullptr;
        *out = create_batch(graph_off, indptr, indices, n_graphs, flags, stream);
    });
}

void gpm_batch_destroy(gpm_batch* b) {
    try {
        destroy_batch(b);
    } catch (...) {
    }
}

gpm_status gpm_batch_count(gpm_batch* b, int clique_k, int motif_k, uint64_t* clique_counts, uint64_t* motif_counts) {
    return guarded([&] {
        if (!b) fail(GPM_EINVAL, "batch is NULL");
        batch_count(b, clique_k, motif_k, clique_counts, motif_counts);
    });
}

gpm_status gpm_batch_autotune(gpm_batch* b, int clique_k, int motif_k, int reps, gpm_config* best,
                              double* best_ms) {
    return guarded([&] {
        if (!b) fail(GPM_EINVAL, "batch is NULL");
        if (reps < 1) fail(GPM_EINVAL, "reps < 1");
        double ms = 0;
        const gpm_config c = batch_autotune(b, clique_k, motif_k, reps, &ms);
        if (best) *best = c;
        if (best_ms) *best_ms = ms;
    });
}

gpm_status gpm_batch_set_config(gpm_batch* b, const gpm_config* cfg) {
    return guarded([&] {
        if (!b || !cfg) fail(GPM_EINVAL, "NULL argument");
        batch_set_config(b, *cfg);
    });
}

gpm_status gpm_batch_get_stats(const gpm_batch* b, gpm_stats* out) {
    return guarded([&] {
        if (!b || !out) fail(GPM_EINVAL, "NULL argument");
        *out = batch_stats(b);
    });
}

const char* gpm_last_error(void) { return last_error_cstr(); }

}  // extern "C"
