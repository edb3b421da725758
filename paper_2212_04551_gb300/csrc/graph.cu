// graph.cu -- graph ingest and preprocessing on the device (hot-path row A1).
//
//  * CSR validation (Section 2: undirected, simple graphs; the adjacency of
//    every vertex contiguous and sorted, Section 4.3.1);
//  * vertex degrees;
//  * the degree-ordered orientation used by clique counting: u -> v iff
//    (d(u), u) < (d(v), v).  Every clique is then reached exactly once, from
//    its lowest vertex in that order -- the same role as the paper's "lower"
//    filter on vertex ids (Algorithm 4, clique counting), with out-lists
//    bounded by sqrt(2m) instead of the maximum degree.  Out-lists keep the
//    id order and are padded to a multiple of four entries (16-byte aligned
//    starts for vector loads), padding = INT32_MAX;
//  * root orders for the plain scheduler (heaviest first), by counting sort.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace gpm {

// ------------------------------------------------------------------ errors

static thread_local std::string t_last_error;

void set_error(const std::string& msg) { t_last_error = msg; }
void clear_error() { t_last_error.clear(); }
const char* last_error_cstr() { return t_last_error.c_str(); }

[[noreturn]] void fail(gpm_status s, const std::string& msg) { throw Error{s, msg}; }

void check_cuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return;
    gpm_status s = (e == cudaErrorMemoryAllocation) ? GPM_ENOMEM : GPM_ECUDA;
    fail(s, std::string(what) + ": " + cudaGetErrorString(e));
}

// --------------------------------------------------------------- buffers

DevBuf::~DevBuf() { release(); }

void DevBuf::release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}

void DevBuf::ensure(size_t need) {
    if (need <= bytes && ptr) return;
    release();
    size_t want = std::max<size_t>(need, 256);
    cudaError_t e = cudaMalloc(&ptr, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ptr = nullptr;
        fail(GPM_ENOMEM, "cudaMalloc of " + std::to_string(want) + " bytes failed: " +
                             cudaGetErrorString(e));
    }
    bytes = want;
}

// --------------------------------------------------------------- kernels

// Warp per vertex: ids in range, no self-loop, strictly ascending, and the
// reverse edge present (binary search of v in N(x)).
__global__ void k_validate(const int32_t* __restrict__ indptr, const int32_t* __restrict__ indices,
                           int32_t n, int64_t nnz, int* __restrict__ bad) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < n; v += nwarps) {
        const int64_t s = indptr[v], e = indptr[v + 1];
        if (s < 0 || e < s || e > nnz) {
            if (lane == 0) atomicOr(bad, 1);
            continue;
        }
        for (int64_t p = s + lane; p < e; p += 32) {
            const int32_t x = indices[p];
            int b = 0;
            if (x < 0 || x >= n) b |= 2;
            else {
                if (x == v) b |= 4;
                if (p > s && indices[p - 1] >= x) b |= 8;
                int64_t lo = indptr[x], hi = indptr[x + 1] - 1;
                bool found = false;
                if (lo >= 0 && hi < nnz) {
                    while (lo <= hi) {
                        const int64_t mid = (lo + hi) >> 1;
                        const int32_t y = indices[mid];
                        if (y == (int32_t)v) { found = true; break; }
                        if (y < (int32_t)v) lo = mid + 1; else hi = mid - 1;
                    }
                }
                if (!found) b |= 16;
            }
            if (b) atomicOr(bad, b);
        }
    }
}

__global__ void k_indptr_monotone(const int32_t* __restrict__ indptr, int32_t n, int* __restrict__ bad) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        if (indptr[v + 1] < indptr[v]) atomicOr(bad, 1);
}

__global__ void k_degree(const int32_t* __restrict__ indptr, int32_t n, int32_t* __restrict__ deg,
                         int* __restrict__ maxdeg) {
    int local = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int d = indptr[v + 1] - indptr[v];
        deg[v] = d;
        local = max(local, d);
    }
    for (int o = 16; o > 0; o >>= 1) local = max(local, __shfl_xor_sync(GPM_FULL_MASK, local, o));
    if ((threadIdx.x & 31) == 0) atomicMax(maxdeg, local);
}

__device__ __forceinline__ bool dag_before(int32_t du, int32_t u, int32_t dv, int32_t v) {
    return du < dv || (du == dv && u < v);
}

// out-degree in the degree orientation, and its padded length
__global__ void k_outdeg(const int32_t* __restrict__ indptr, const int32_t* __restrict__ indices,
                         const int32_t* __restrict__ deg, int32_t n, int32_t* __restrict__ outdeg,
                         int32_t* __restrict__ padded, int* __restrict__ maxout) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < n; v += nwarps) {
        const int32_t dv = deg[v];
        int c = 0;
        for (int64_t p = indptr[v] + lane; p < indptr[v + 1]; p += 32) {
            const int32_t x = indices[p];
            c += dag_before(dv, (int32_t)v, deg[x], x) ? 1 : 0;
        }
        c = gpm_warp_sum(c);
        if (lane == 0) {
            outdeg[v] = c;
            padded[v] = (c + 3) & ~3;
            atomicMax(maxout, c);
        }
    }
}

__global__ void k_dag_fill(const int32_t* __restrict__ indptr, const int32_t* __restrict__ indices,
                           const int32_t* __restrict__ deg, int32_t n, const int32_t* __restrict__ off,
                           int32_t* __restrict__ adj) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < n; v += nwarps) {
        const int32_t dv = deg[v];
        int64_t base = off[v];
        const int64_t end = off[v + 1];
        for (int64_t p0 = indptr[v]; p0 < indptr[v + 1]; p0 += 32) {
            const int64_t p = p0 + lane;
            bool keep = false;
            int32_t x = 0;
            if (p < indptr[v + 1]) {
                x = indices[p];
                keep = dag_before(dv, (int32_t)v, deg[x], x);
            }
            const unsigned bal = __ballot_sync(GPM_FULL_MASK, keep);
            if (keep) adj[base + __popc(bal & gpm_lanemask_lt())] = x;
            base += __popc(bal);
        }
        for (int64_t p = base + lane; p < end; p += 32) adj[p] = INT32_MAX;
    }
}

__global__ void k_queue_init(QSeq* q, unsigned long long cap) {
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < cap;
         i += (unsigned long long)gridDim.x * blockDim.x)
        q[i].seq = i;
}

// ------------------------------------------------------------------ scan

// Exclusive scan of int32 values in chunks of 1024 (block-local), then the
// chunk sums, then the add-back; totals are carried in int64.
static constexpr int SCAN_CHUNK = 1024;

__device__ __forceinline__ long long block_exclusive_scan_1024(long long x, long long* sh, long long* total) {
    // 1024 threads, one value each
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long v = x;
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(GPM_FULL_MASK, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) sh[wid] = v;
    __syncthreads();
    if (wid == 0) {
        long long w = sh[lane];
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(GPM_FULL_MASK, w, o);
            if (lane >= o) w += y;
        }
        sh[lane] = w;
    }
    __syncthreads();
    const long long before = (wid ? sh[wid - 1] : 0) + v - x;
    if (total) *total = sh[31];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(1024) k_scan_chunks(const int32_t* __restrict__ in, int64_t n,
                                                      long long* __restrict__ sums) {
    __shared__ long long sh[32];
    const int64_t i = blockIdx.x * (int64_t)SCAN_CHUNK + threadIdx.x;
    long long tot;
    block_exclusive_scan_1024(i < n ? in[i] : 0, sh, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_sums(long long* __restrict__ sums, int64_t nb,
                                                    long long* __restrict__ grand) {
    __shared__ long long sh[32];
    long long carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += SCAN_CHUNK) {
        const int64_t b = b0 + threadIdx.x;
        long long tot;
        const long long ex = block_exclusive_scan_1024(b < nb ? sums[b] : 0, sh, &tot);
        if (b < nb) sums[b] = carry + ex;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *grand = carry;
}

__global__ void __launch_bounds__(1024) k_scan_apply(const int32_t* __restrict__ in, int64_t n,
                                                     const long long* __restrict__ sums,
                                                     int32_t* __restrict__ out, const long long* grand) {
    __shared__ long long sh[32];
    const int64_t i = blockIdx.x * (int64_t)SCAN_CHUNK + threadIdx.x;
    const long long ex = block_exclusive_scan_1024(i < n ? in[i] : 0, sh, nullptr);
    if (i < n) out[i] = (int32_t)(sums[blockIdx.x] + ex);
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = (int32_t)min(*grand, (long long)INT32_MAX);
}

void exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, int64_t* total, cudaStream_t s,
                        DevBuf& tmp) {
    const int64_t nb = std::max<int64_t>(1, (n + SCAN_CHUNK - 1) / SCAN_CHUNK);
    tmp.ensure(sizeof(long long) * (nb + 1));
    long long* sums = tmp.as<long long>();
    long long* grand = sums + nb;
    k_scan_chunks<<<(unsigned)nb, SCAN_CHUNK, 0, s>>>(in, n, sums);
    k_scan_sums<<<1, SCAN_CHUNK, 0, s>>>(sums, nb, grand);
    k_scan_apply<<<(unsigned)nb, SCAN_CHUNK, 0, s>>>(in, n, sums, out, grand);
    GPM_CUDA(cudaGetLastError());
    long long h = 0;
    GPM_CUDA(cudaMemcpyAsync(&h, grand, sizeof(h), cudaMemcpyDeviceToHost, s));
    GPM_CUDA(cudaStreamSynchronize(s));
    *total = h;
}

// ---------------------------------------------------------- counting sort

__global__ void k_key_hist(const int32_t* __restrict__ key, int32_t n, int32_t maxkey,
                           int32_t* __restrict__ hist) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&hist[maxkey - min(key[v], maxkey)], 1);
}

__global__ void k_key_scatter(const int32_t* __restrict__ key, int32_t n, int32_t maxkey,
                              int32_t* __restrict__ cursor, int32_t* __restrict__ order) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int pos = atomicAdd(&cursor[maxkey - min(key[v], maxkey)], 1);
        order[pos] = (int32_t)v;
    }
}

static int grid_for(int64_t work, int threads, int sms) {
    int64_t b = (work + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)sms * 32));
}

// vertices sorted by key descending (ties in no particular order)
static void order_by_key_desc(gpm_graph* g, const int32_t* key, int32_t maxkey, DevBuf& out) {
    cudaStream_t s = g->stream;
    const int32_t n = g->n;
    out.ensure(sizeof(int32_t) * std::max(n, 1));
    DevBuf hist, cur, tmp;
    hist.ensure(sizeof(int32_t) * (maxkey + 2));
    cur.ensure(sizeof(int32_t) * (maxkey + 2));
    GPM_CUDA(cudaMemsetAsync(hist.ptr, 0, sizeof(int32_t) * (maxkey + 2), s));
    if (n > 0) {
        k_key_hist<<<grid_for(n, 256, g->num_sms), 256, 0, s>>>(key, n, maxkey, hist.as<int32_t>());
        int64_t total = 0;
        exclusive_scan_i32(hist.as<int32_t>(), cur.as<int32_t>(), maxkey + 1, &total, s, tmp);
        k_key_scatter<<<grid_for(n, 256, g->num_sms), 256, 0, s>>>(key, n, maxkey, cur.as<int32_t>(),
                                                                   out.as<int32_t>());
        GPM_CUDA(cudaGetLastError());
        GPM_CUDA(cudaStreamSynchronize(s));
    }
}

void ensure_dag(gpm_graph* g) {
    if (g->dag_ready) return;
    cudaStream_t s = g->stream;
    const int32_t n = g->n;
    g->dag_outdeg.ensure(sizeof(int32_t) * std::max(n, 1));
    DevBuf padded, tmp, dmax;
    padded.ensure(sizeof(int32_t) * std::max(n, 1));
    dmax.ensure(sizeof(int));
    GPM_CUDA(cudaMemsetAsync(dmax.ptr, 0, sizeof(int), s));
    g->dag_off.ensure(sizeof(int32_t) * (n + 1));
    if (n > 0) {
        k_outdeg<<<grid_for((int64_t)n * 32, 256, g->num_sms), 256, 0, s>>>(
            g->indptr.as<int32_t>(), g->indices.as<int32_t>(), g->degree.as<int32_t>(), n,
            g->dag_outdeg.as<int32_t>(), padded.as<int32_t>(), dmax.as<int>());
        GPM_CUDA(cudaGetLastError());
    }
    int64_t total = 0;
    if (n > 0) exclusive_scan_i32(padded.as<int32_t>(), g->dag_off.as<int32_t>(), n, &total, s, tmp);
    else GPM_CUDA(cudaMemsetAsync(g->dag_off.ptr, 0, sizeof(int32_t), s));
    if (total >= INT32_MAX) fail(GPM_EINVAL, "oriented graph too large for int32 offsets");
    g->dag_adj.ensure(sizeof(int32_t) * std::max<int64_t>(total, 4));
    if (n > 0) {
        k_dag_fill<<<grid_for((int64_t)n * 32, 256, g->num_sms), 256, 0, s>>>(
            g->indptr.as<int32_t>(), g->indices.as<int32_t>(), g->degree.as<int32_t>(), n,
            g->dag_off.as<int32_t>(), g->dag_adj.as<int32_t>());
        GPM_CUDA(cudaGetLastError());
    }
    int hmax = 0;
    GPM_CUDA(cudaMemcpyAsync(&hmax, dmax.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    GPM_CUDA(cudaStreamSynchronize(s));
    g->max_outdeg = hmax;
    g->dag_ready = true;
}

const int32_t* ensure_root_order(gpm_graph* g, int app) {
    if (app == GPM_APP_CLIQUE) {
        ensure_dag(g);
        if (!g->order_clique_ready) {
            order_by_key_desc(g, g->dag_outdeg.as<int32_t>(), std::max(g->max_outdeg, 0), g->order_clique);
            g->order_clique_ready = true;
        }
        return g->order_clique.as<int32_t>();
    }
    if (!g->order_motif_ready) {
        order_by_key_desc(g, g->degree.as<int32_t>(), std::max(g->max_deg, 0), g->order_motif);
        g->order_motif_ready = true;
    }
    return g->order_motif.as<int32_t>();
}

__global__ void k_iota(int32_t* out, int32_t n) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        out[v] = (int32_t)v;
}

const int32_t* ensure_id_order(gpm_graph* g) {
    if (!g->order_id_ready) {
        g->order_id.ensure(sizeof(int32_t) * std::max(g->n, 1));
        if (g->n > 0) {
            k_iota<<<grid_for(g->n, 256, g->num_sms), 256, 0, g->stream>>>(g->order_id.as<int32_t>(), g->n);
            GPM_CUDA(cudaGetLastError());
        }
        g->order_id_ready = true;
    }
    return g->order_id.as<int32_t>();
}

// ------------------------------------------------------------ create / destroy

gpm_config default_config() {
    gpm_config c;
    c.warps_per_block = 0;   // automatic: the most resident warps per SM
    c.blocks_per_sm = 0;
    c.donate_min = 4;
    c.order = GPM_ORDER_DEGREE_DESC;
    c.max_idle_ms = 120000;
    c.donate = 1;
    c.donate_after_us = 50;
    c.clique_tail = 0;
    c.clique_compact = 0;
    c.motif_agg_min = 16;
    c.clique_compact3 = 1;
    c.batch_split = 1;
    c.clique_cpl = 85;
    return c;
}

gpm_graph* create_graph(const int32_t* indptr, const int32_t* indices, int32_t n, uint32_t flags,
                        void* stream) {
    if (n < 0) fail(GPM_EINVAL, "n < 0");
    if (!indptr) fail(GPM_EINVAL, "indptr is NULL");
    const bool dev = (flags & GPM_DEVICE_PTRS) != 0;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    int32_t first = 0, last = 0;
    if (dev) {
        GPM_CUDA(cudaMemcpyAsync(&first, indptr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        GPM_CUDA(cudaMemcpyAsync(&last, indptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        GPM_CUDA(cudaStreamSynchronize(s));
    } else {
        first = indptr[0];
        last = indptr[n];
    }
    if (first != 0) fail(GPM_EINVAL, "indptr[0] != 0");
    if (last < 0) fail(GPM_EINVAL, "indptr[n] < 0");
    if (last > 0 && !indices) fail(GPM_EINVAL, "indices is NULL");
    if (last % 2) fail(GPM_EINVAL, "indptr[n] is odd: an undirected CSR stores every edge twice");

    gpm_graph* g = new gpm_graph();
    try {
        GPM_CUDA(cudaGetDevice(&g->device));
        GPM_CUDA(cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device));
        g->stream = s;
        g->n = n;
        g->nnz = last;
        g->cfg = default_config();
        g->indptr.ensure(sizeof(int32_t) * (n + 1));
        g->indices.ensure(sizeof(int32_t) * std::max<int64_t>(last, 1));
        g->degree.ensure(sizeof(int32_t) * std::max(n, 1));
        const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        GPM_CUDA(cudaMemcpyAsync(g->indptr.ptr, indptr, sizeof(int32_t) * (n + 1), kind, s));
        if (last > 0)
            GPM_CUDA(cudaMemcpyAsync(g->indices.ptr, indices, sizeof(int32_t) * (size_t)last, kind, s));
        DevBuf flag;
        flag.ensure(2 * sizeof(int));
        GPM_CUDA(cudaMemsetAsync(flag.ptr, 0, 2 * sizeof(int), s));
        int* bad = flag.as<int>();
        if (n > 0) {
            k_indptr_monotone<<<grid_for(n, 256, g->num_sms), 256, 0, s>>>(g->indptr.as<int32_t>(), n, bad);
            k_degree<<<grid_for(n, 256, g->num_sms), 256, 0, s>>>(g->indptr.as<int32_t>(), n,
                                                                 g->degree.as<int32_t>(), bad + 1);
            GPM_CUDA(cudaGetLastError());
        }
        int hb[2] = {0, 0};
        GPM_CUDA(cudaMemcpyAsync(hb, flag.ptr, sizeof(hb), cudaMemcpyDeviceToHost, s));
        GPM_CUDA(cudaStreamSynchronize(s));
        if (hb[0]) fail(GPM_EINVAL, "indptr is not non-decreasing");
        g->max_deg = hb[1];
        if (!(flags & GPM_SKIP_VALIDATE) && n > 0 && last > 0) {
            GPM_CUDA(cudaMemsetAsync(flag.ptr, 0, sizeof(int), s));
            k_validate<<<grid_for((int64_t)n * 32, 256, g->num_sms), 256, 0, s>>>(
                g->indptr.as<int32_t>(), g->indices.as<int32_t>(), n, last, bad);
            GPM_CUDA(cudaGetLastError());
            int v = 0;
            GPM_CUDA(cudaMemcpyAsync(&v, flag.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
            GPM_CUDA(cudaStreamSynchronize(s));
            if (v) {
                std::string why;
                if (v & 1) why += " bad indptr;";
                if (v & 2) why += " neighbour id out of range;";
                if (v & 4) why += " self-loop;";
                if (v & 8) why += " adjacency list not strictly ascending (unsorted or duplicate);";
                if (v & 16) why += " not symmetric;";
                fail(GPM_EINVAL, "invalid CSR:" + why);
            }
        }
        GPM_CUDA(cudaEventCreate(&g->ev0));
        GPM_CUDA(cudaEventCreate(&g->ev1));
    } catch (...) {
        if (g->ev0) cudaEventDestroy(g->ev0);
        if (g->ev1) cudaEventDestroy(g->ev1);
        delete g;
        throw;
    }
    return g;
}

void destroy_graph(gpm_graph* g) {
    if (!g) return;
    if (g->stream) cudaStreamSynchronize(g->stream);
    else cudaDeviceSynchronize();
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    delete g;
}

int resident_blocks(const void* kernel, int threads, size_t smem) {
    int nb = 0;
    check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem),
               "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    return nb;
}

int best_warps_per_block(const void* kernel, size_t smem_per_warp, size_t smem_fixed) {
    int best = 8, best_warps = -1;
    for (int wpb : {16, 8, 4, 2, 1}) {
        const size_t smem = smem_fixed + smem_per_warp * wpb;
        if (smem > 227 * 1024) continue;
        if (smem > 48 * 1024)
            check_cuda(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                       "cudaFuncSetAttribute");
        const int per_sm = resident_blocks(kernel, wpb * 32, smem);
        if (per_sm * wpb > best_warps) {
            best_warps = per_sm * wpb;
            best = wpb;
        }
    }
    return best;
}

Grid plan_grid(gpm_graph* g, const void* kernel, int warps_per_block, size_t smem_per_block, int max_per_sm) {
    Grid gr;
    gr.warps_per_block = warps_per_block;
    int per_sm = resident_blocks(kernel, warps_per_block * 32, smem_per_block);
    if (per_sm <= 0) fail(GPM_EINVAL, "kernel cannot be resident with this configuration (shared memory "
                                      + std::to_string(smem_per_block) + " B)");
    if (g->cfg.blocks_per_sm > 0) per_sm = std::min(per_sm, g->cfg.blocks_per_sm);
    else if (max_per_sm > 0) per_sm = std::min(per_sm, max_per_sm);
    gr.blocks = per_sm * g->num_sms;
    return gr;
}

}  // namespace gpm
