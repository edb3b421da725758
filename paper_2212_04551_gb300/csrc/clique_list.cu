// clique_list.cu -- k-clique counting for roots whose out-degree exceeds the
// bitmap limit (hot-path row A3, the list form of the extension step).
//
// The paper keeps a traversal's extensions as an array that each step
// filters ("lower", "is_clique") and compacts (Section 4.3, Algorithm 4);
// the bitmap kernel replaces that array by a bit row over N+(r), which needs
// d+(r) <= 1024 to fit in shared memory.  A root above that limit is counted
// here with the array form itself, on the degree orientation:
//
//   * the candidate list of a traversal is the sorted id list of the
//     vertices adjacent to all of it and after it in the orientation (the
//     common out-neighbours); choosing child w gives C & N+(w);
//   * a warp intersects two sorted lists by probing every entry of the
//     shorter one in the longer one (binary search, one entry per lane) and
//     compacting the hits with a ballot, so the child list stays sorted;
//   * at a traversal of size k-2 the k-cliques below it are
//     sum over w in C of |C & N+(w)| (the edges inside C, each counted at its
//     lower end), without writing the (k-1)-vertex children's lists.
//
// Work units are (heavy root, range of its children), the ranges cut by the
// same (L - c)^(k-1) work model as the pre-split seeds, taken from a counter
// in chunk-major order so that every heavy root's heaviest range goes first.
// A warp's lists live in a per-warp stack in global memory, one slot of
// max-out-degree ids per level.  No waits: a warp leaves when the units run
// out.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "common.cuh"
#include "list_ring.cuh"

namespace gpm {

constexpr int CL_WARPS = 4;       // warps per block
constexpr int CL_CHUNKS = 64;     // children ranges per heavy root

struct ListParams {
    const int32_t* __restrict__ off;      // orientation (padded offsets)
    const int32_t* __restrict__ adj;      // out-neighbours sorted by id
    const int32_t* __restrict__ outdeg;
    const int32_t* __restrict__ roots;    // the launch's root list
    const int32_t* __restrict__ heavy;    // positions in roots of the heavy roots
    int k_lo, k_hi;
    int maxd;                             // ids per stack slot
    int32_t* stack;                       // per warp: (k_hi - 3) slots
    Control* ctl;
    unsigned long long* per_root;         // nullable, indexed by root position
};

// Positions (in the root list) of the roots above the bitmap limit.
__global__ void k_clique_heavy(const int32_t* __restrict__ roots, long long n_roots,
                               const int32_t* __restrict__ outdeg, int limit, int32_t* heavy, Control* ctl) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n_roots;
         t += (long long)gridDim.x * blockDim.x)
        if (outdeg[roots[t]] > limit) heavy[atomicAdd(&ctl->n_heavy, 1)] = (int32_t)t;
}

// |a & b| for two sorted id lists; the common ids go, in order, to out when
// it is not null.  Lanes probe 32 consecutive entries of the shorter list at
// a time; the probes of one batch only move right in the longer list, so the
// next batch searches from the last lane's position.
__device__ int cl_intersect(const int32_t* a, int na, const int32_t* b, int nb, int32_t* out, int lane) {
    if (na > nb) {
        const int32_t* t = a;
        a = b;
        b = t;
        const int tn = na;
        na = nb;
        nb = tn;
    }
    int m = 0, from = 0;
    for (int base = 0; base < na; base += 32) {
        const int i = base + lane;
        int x = 0, pos = nb;
        bool hit = false;
        if (i < na) {
            x = a[i];
            int lo = from, hi = nb;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (b[mid] < x) lo = mid + 1;
                else hi = mid;
            }
            pos = lo;
            hit = lo < nb && b[lo] == x;
        }
        const unsigned bal = __ballot_sync(GPM_FULL_MASK, hit);
        if (hit && out) out[m + __popc(bal & gpm_lanemask_lt())] = x;
        m += __popc(bal);
        from = __shfl_sync(GPM_FULL_MASK, pos, 31);
    }
    __syncwarp();   // the list written above is read by every lane next
    return m;
}

// sum over w in C of |C & N+(w)|: the edges inside C
__device__ unsigned long long cl_edges_in(const ListParams& p, const int32_t* C, int c, int lane) {
    unsigned long long e = 0;
    if (c < 2) return 0;
    for (int i = 0; i < c; i++) {
        const int w = C[i];
        e += (unsigned long long)cl_intersect(C, c, p.adj + p.off[w], p.outdeg[w], nullptr, lane);
    }
    return e;
}

// lane 0 adds v to the warp's counter of clique size j (carry-checked)
__device__ __forceinline__ void cl_add(const ListParams& p, unsigned long long* wc, int j, unsigned long long v,
                                       int lane) {
    if (lane != 0 || j < p.k_lo || j > p.k_hi || !v) return;
    const unsigned long long s = wc[j] + v;
    if (s < wc[j]) atomicExch(&p.ctl->overflow, 1);
    wc[j] = s;
}

__global__ void __launch_bounds__(CL_WARPS * 32) k_clique_list(ListParams p) {
    __shared__ unsigned long long wcnt[CL_WARPS][GPM_CLIQUE_MAX_K + 1];
    __shared__ int s_pos[CL_WARPS][GPM_CLIQUE_MAX_K + 1];
    __shared__ int s_len[CL_WARPS][GPM_CLIQUE_MAX_K + 1];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    unsigned long long* wc = wcnt[wib];
    int* pos = s_pos[wib];
    int* len = s_len[wib];
    for (int j = lane; j <= GPM_CLIQUE_MAX_K; j += 32) wc[j] = 0ull;
    __syncwarp();
    const long long gw = blockIdx.x * (long long)CL_WARPS + wib;
    // slot of the list of a traversal of size s (2 <= s <= k_hi - 2)
    int32_t* const st = p.stack + gw * (long long)max(p.k_hi - 3, 1) * p.maxd;
    const int H = *(volatile int*)&p.ctl->n_heavy;
    const unsigned long long n_units = (unsigned long long)H * CL_CHUNKS;
    Control* ctl = p.ctl;
    int ovf = 0;
    for (;;) {
        unsigned long long u = 0;
        if (lane == 0) u = atomicAdd(&ctl->heavy_next, 1ull);
        u = __shfl_sync(GPM_FULL_MASK, u, 0);
        if (u >= n_units) break;
        const int h = (int)(u % (unsigned long long)H);
        const int chunk = (int)(u / (unsigned long long)H);
        const int t = p.heavy[h];
        const int r = p.roots[t];
        const int d = p.outdeg[r];
        const int lo = gpm_balanced_cut(d, chunk, CL_CHUNKS, p.k_hi);
        const int hi = gpm_balanced_cut(d, chunk + 1, CL_CHUNKS, p.k_hi);
        const int32_t* Nr = p.adj + p.off[r];
        unsigned long long top = 0;   // k_hi-cliques of this unit (lane-uniform)
        for (int i = lo; i < hi; i++) {
            // the traversal (r, v): its candidates are N+(r) & N+(v)
            const int v = Nr[i];
            const int32_t* Nv = p.adj + p.off[v];
            if (p.k_hi == 3) {
                const int c = cl_intersect(Nr, d, Nv, p.outdeg[v], nullptr, lane);
                top = gpm_add_cc(top, (unsigned long long)c, ovf);
                continue;
            }
            const int c2 = cl_intersect(Nr, d, Nv, p.outdeg[v], st, lane);
            cl_add(p, wc, 3, (unsigned long long)c2, lane);
            if (p.k_hi == 4) {
                top = gpm_add_cc(top, cl_edges_in(p, st, c2, lane), ovf);
                continue;
            }
            if (c2 == 0) continue;
            // depth first below (r, v) over the traversals of sizes 2 .. k_hi - 3
            // (their children's lists count cliques of sizes 4 .. k_hi - 1, and
            // at size k_hi - 3 the children's edges count the k_hi-cliques);
            // the traversal of size s has its list in slot s - 2
            int s = 2;
            if (lane == 0) {
                pos[2] = 0;
                len[2] = c2;
            }
            __syncwarp();
            while (s >= 2) {
                const int ps = pos[s], ls = len[s];
                if (ps >= ls) {
                    s--;
                    continue;
                }
                const int32_t* C = st + (long long)(s - 2) * p.maxd;
                const int w = C[ps];
                __syncwarp();
                if (lane == 0) pos[s] = ps + 1;
                // child (size s + 1): candidates C & N+(w); each completes an (s + 2)-clique
                int32_t* Cw = st + (long long)(s - 1) * p.maxd;
                const int cw = cl_intersect(C, ls, p.adj + p.off[w], p.outdeg[w], Cw, lane);
                cl_add(p, wc, s + 2, (unsigned long long)cw, lane);
                if (s + 3 == p.k_hi) {
                    top = gpm_add_cc(top, cl_edges_in(p, Cw, cw, lane), ovf);
                    continue;
                }
                if (cw == 0) continue;
                s++;
                if (lane == 0) {
                    pos[s] = 0;
                    len[s] = cw;
                }
                __syncwarp();
            }
        }
        if (lane == 0) {
            const unsigned long long old = wc[p.k_hi];
            wc[p.k_hi] = old + top;
            if (wc[p.k_hi] < old) ovf = 1;
            if (p.per_root) gpm_atomic_add_cc(&p.per_root[t], top, &ctl->overflow);
        }
        __syncwarp();
    }
    __syncwarp();
    if (lane == 0) {
        if (ovf) atomicExch(&ctl->overflow, 1);
        for (int j = p.k_lo; j <= p.k_hi; j++) gpm_atomic_add_cc(&ctl->counts[j], wc[j], &ctl->overflow);
    }
}

void run_clique_list(gpm_graph* g, int k_lo, int k_hi, const int32_t* d_roots, int64_t n_roots,
                     unsigned long long* d_per_root, Control* ctl, int bitmap_limit) {
    if (k_hi < 3 || n_roots <= 0 || g->max_outdeg <= bitmap_limit) return;
    cudaStream_t s = g->stream;
    const int maxd = g->max_outdeg;
    const size_t per_warp = sizeof(int32_t) * (size_t)std::max(k_hi - 3, 1) * (size_t)maxd;
    // at most 1 GiB of stacks; at least one block
    const size_t budget = size_t(1) << 30;
    long long blocks = (long long)g->num_sms * 8;
    blocks = std::min<long long>(blocks, std::max<long long>(1, (long long)(budget / (per_warp * CL_WARPS))));
    const size_t heavy_bytes = (sizeof(int32_t) * (size_t)n_roots + 255) & ~size_t(255);
    g->scratch_slab.ensure(heavy_bytes + per_warp * CL_WARPS * (size_t)blocks);
    int32_t* heavy = g->scratch_slab.as<int32_t>();
    ListParams p{};
    p.off = g->dag_off.as<int32_t>();
    p.adj = g->dag_adj.as<int32_t>();
    p.outdeg = g->dag_outdeg.as<int32_t>();
    p.roots = d_roots;
    p.heavy = heavy;
    p.k_lo = std::max(k_lo, 3);
    p.k_hi = k_hi;
    p.maxd = maxd;
    p.stack = reinterpret_cast<int32_t*>(g->scratch_slab.as<unsigned char>() + heavy_bytes);
    p.ctl = ctl;
    p.per_root = d_per_root;
    const int cblocks = (int)std::min<long long>((n_roots + 255) / 256, (long long)g->num_sms * 8);
    k_clique_heavy<<<cblocks, 256, 0, s>>>(d_roots, n_roots, p.outdeg, bitmap_limit, heavy, ctl);
    GPM_CUDA(cudaGetLastError());
    k_clique_list<<<(int)blocks, CL_WARPS * 32, 0, s>>>(p);
    GPM_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Listing (aggregate_store): every k-clique as a record of its k vertex ids
// in orientation order (root first), appended to the host ring
// (list_ring.cuh).  The same list-form search over every root: a traversal
// of size k-1 hands each of its candidates to the ring instead of counting
// them.  Units are (root, quarter of its children by the work model).

constexpr int CS_CHUNKS = 4;

struct StoreParams {
    const int32_t* __restrict__ off;
    const int32_t* __restrict__ adj;
    const int32_t* __restrict__ outdeg;
    const int32_t* __restrict__ roots;
    long long n_roots;
    int k;
    int maxd;
    int32_t* stack;        // per warp: k - 2 slots of maxd ids
    Control* ctl;
    ListRing ring;
};

// append the candidates C[0 .. c-1] of the traversal tr[0 .. np-1]
__device__ __forceinline__ bool cs_emit_all(const StoreParams& p, unsigned long long& tail_seen, const int* tr, int np,
                                            const int32_t* C, int c, int lane) {
    for (int base = 0; base < c; base += 32) {
        const bool act = base + lane < c;
        const int x = act ? C[base + lane] : 0;
        if (!lr_emit(p.ring, tail_seen, tr, np, -1, x, -1, act, lane)) return false;
    }
    return true;
}

__global__ void __launch_bounds__(CL_WARPS * 32) k_clique_store(StoreParams p) {
    __shared__ int s_tr[CL_WARPS][GPM_CLIQUE_MAX_K + 1];
    __shared__ int s_pos[CL_WARPS][GPM_CLIQUE_MAX_K + 1];
    __shared__ int s_len[CL_WARPS][GPM_CLIQUE_MAX_K + 1];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    int* tr = s_tr[wib];
    int* pos = s_pos[wib];
    int* len = s_len[wib];
    const long long gw = blockIdx.x * (long long)CL_WARPS + wib;
    int32_t* const st = p.stack + gw * (long long)max(p.k - 2, 1) * p.maxd;
    const unsigned long long n_units = (unsigned long long)p.n_roots * CS_CHUNKS;
    Control* ctl = p.ctl;
    unsigned long long tail_seen = 0;   // lane 0
    bool live = true;
    while (live) {
        unsigned long long u = 0;
        int err = 0;
        if (lane == 0) {
            u = atomicAdd(&ctl->next_root, 1ull);
            err = *(volatile int*)&ctl->error;
        }
        u = __shfl_sync(GPM_FULL_MASK, u, 0);
        if (__shfl_sync(GPM_FULL_MASK, err, 0) || u >= n_units) break;
        const long long t = (long long)(u / CS_CHUNKS);
        const int chunk = (int)(u % CS_CHUNKS);
        const int r = p.roots[t];
        const int d = p.outdeg[r];
        const int lo = gpm_balanced_cut(d, chunk, CS_CHUNKS, p.k);
        const int hi = gpm_balanced_cut(d, chunk + 1, CS_CHUNKS, p.k);
        const int32_t* Nr = p.adj + p.off[r];
        for (int i = lo; i < hi && live; i++) {
            const int v = Nr[i];
            __syncwarp();
            if (lane == 0) {
                tr[0] = r;
                tr[1] = v;
            }
            const int c2 = cl_intersect(Nr, d, p.adj + p.off[v], p.outdeg[v], st, lane);   // syncs the warp
            if (p.k == 3) {
                live = cs_emit_all(p, tail_seen, tr, 2, st, c2, lane);
                continue;
            }
            if (c2 == 0) continue;
            // depth first: the traversal of size s has its list in slot s - 2
            int s = 2;
            if (lane == 0) {
                pos[2] = 0;
                len[2] = c2;
            }
            __syncwarp();
            while (s >= 2 && live) {
                const int ps = pos[s], ls = len[s];
                if (ps >= ls) {
                    s--;
                    continue;
                }
                const int32_t* C = st + (long long)(s - 2) * p.maxd;
                const int w = C[ps];
                __syncwarp();
                if (lane == 0) {
                    pos[s] = ps + 1;
                    tr[s] = w;
                }
                int32_t* Cw = st + (long long)(s - 1) * p.maxd;
                const int cw = cl_intersect(C, ls, p.adj + p.off[w], p.outdeg[w], Cw, lane);
                if (s + 2 == p.k) {   // tr[0 .. s] is a (k-1)-clique: each candidate completes one
                    live = cs_emit_all(p, tail_seen, tr, s + 1, Cw, cw, lane);
                    continue;
                }
                if (cw == 0) continue;
                s++;
                if (lane == 0) {
                    pos[s] = 0;
                    len[s] = cw;
                }
                __syncwarp();
            }
        }
    }
}

void launch_clique_store(gpm_graph* g, int k, const ListRing& ring, Control* ctl) {
    ensure_dag(g);
    cudaStream_t s = g->stream;
    const int32_t* d_roots = ensure_root_order(g, GPM_APP_CLIQUE);
    const int maxd = std::max(g->max_outdeg, 1);
    const size_t per_warp = sizeof(int32_t) * (size_t)std::max(k - 2, 1) * (size_t)maxd;
    const size_t budget = size_t(1) << 30;
    long long blocks = (long long)g->num_sms * 8;
    blocks = std::min<long long>(blocks, std::max<long long>(1, (long long)(budget / (per_warp * CL_WARPS))));
    g->scratch_slab.ensure(per_warp * CL_WARPS * (size_t)blocks);
    StoreParams p{};
    p.off = g->dag_off.as<int32_t>();
    p.adj = g->dag_adj.as<int32_t>();
    p.outdeg = g->dag_outdeg.as<int32_t>();
    p.roots = d_roots;
    p.n_roots = g->n;
    p.k = k;
    p.maxd = maxd;
    p.stack = g->scratch_slab.as<int32_t>();
    p.ctl = ctl;
    p.ring = ring;
    GPM_CUDA(cudaEventRecord(g->ev0, s));
    if (g->n > 0) k_clique_store<<<(int)blocks, CL_WARPS * 32, 0, s>>>(p);
    GPM_CUDA(cudaGetLastError());
    GPM_CUDA(cudaEventRecord(g->ev1, s));
    g->stats = gpm_stats{};
    g->stats.grid_blocks = (int)blocks;
    g->stats.warps_per_block = CL_WARPS;
    g->stats.kernel_launches = g->n > 0 ? 1 : 0;
}

}  // namespace gpm
