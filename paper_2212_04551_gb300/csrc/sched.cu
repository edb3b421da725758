// sched.cu -- the learned scheduler (hot-path row A10).
//
// Not part of the paper: a small MLP predicts each root's enumeration-subtree
// size from 8 per-root features; its predictions order the roots heaviest
// first and pre-split the heaviest ones into several work units before the
// enumeration starts, so that fewer splits are left to the in-kernel donation
// layer.  The network only changes which warp runs which part of the search,
// never what is counted.
//
//   features (FP32, per vertex v, for subgraph size k):
//     f0 log1p d(v)            f1 log1p d+(v) (degree-ordered out-degree)
//     f2 log1p |{u in N(v): u > v}|       (motif root's first extension set)
//     f3 log1p sum_{u in N(v)} d(u)       f4 log1p sum_{u in N(v), u > v} d(u)
//     f5 log1p triangles whose lowest (degree, id) vertex is v
//     f6 log1p core number of v           f7 k / 8 (one network serves several k)
//   network: 8 -> 64 -> 64 -> 1, ReLU, BF16 weights, FP32 activations and
//   accumulation; trained with MSE on log-sizes and Adam on FP32 master weights.
//
// The MLP is ~5k parameters and runs over at most a few hundred thousand
// roots (~0.3 GFLOP): microseconds against seconds of enumeration, so it is
// plain FP32 SIMT code with the weights broadcast from shared memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"

namespace gpm {

constexpr int MLP_IN = 8, MLP_H = 64;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + MLP_H * MLP_IN, OFF_W2 = OFF_B1 + MLP_H,
              OFF_B2 = OFF_W2 + MLP_H * MLP_H, OFF_W3 = OFF_B2 + MLP_H, OFF_B3 = OFF_W3 + MLP_H,
              MLP_NPARAM = OFF_B3 + 1;
static_assert(MLP_NPARAM == GPM_MLP_PARAMS, "parameter count");

// ------------------------------------------------------------- features

// triangles rooted at v in the degree orientation: sum over u in N+(v) of
// |N+(v) & N+(u)| (binary search of N+(u)'s entries in N+(v)); warp per v
__global__ void k_tri_root(const int32_t* __restrict__ off, const int32_t* __restrict__ adj,
                           const int32_t* __restrict__ outdeg, int32_t n, float* __restrict__ tri) {
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long v = warp; v < n; v += nw) {
        const int b = off[v], d = outdeg[v];
        long long c = 0;
        for (int i = 0; i < d; i++) {
            const int u = adj[b + i];
            const int ub = off[u], du = outdeg[u];
            for (int t = lane; t < du; t += 32) {
                const int x = adj[ub + t];
                int lo = 0, hi = d - 1;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (adj[b + mid] < x) lo = mid + 1; else hi = mid;
                }
                c += (d > 0 && adj[b + lo] == x) ? 1 : 0;
            }
        }
        c = gpm_warp_sum(c);
        if (lane == 0) tri[v] = (float)c;
    }
}

// Core numbers by peeling (the k-core decomposition): at level c every
// remaining vertex whose remaining degree is <= c gets core number c and is
// removed, which lowers its remaining neighbours' degrees; a level is
// repeated until it removes nothing, then c moves to the smallest remaining
// degree.  One pass of one level: flags[0] = 1 if it removed a vertex,
// flags[1] = the smallest remaining degree among the vertices it kept.
__global__ void k_core_init(const int32_t* __restrict__ deg, int32_t n, int32_t* __restrict__ rem,
                            int32_t* __restrict__ core) {
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        rem[v] = deg[v];
        core[v] = -1;
    }
}

__global__ void k_core_peel(const int32_t* __restrict__ indptr, const int32_t* __restrict__ indices, int32_t n,
                            int32_t c, int32_t* __restrict__ rem, int32_t* __restrict__ core, int* __restrict__ flags) {
    int removed = 0, keep_min = INT32_MAX;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        if (core[v] >= 0) continue;
        const int r = atomicAdd(&rem[v], 0);
        if (r <= c) {
            core[v] = c;
            removed = 1;
            for (int t = indptr[v]; t < indptr[v + 1]; t++) {
                const int u = indices[t];
                if (atomicAdd(&core[u], 0) < 0) atomicSub(&rem[u], 1);
            }
        } else {
            keep_min = min(keep_min, r);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        removed |= __shfl_xor_sync(GPM_FULL_MASK, removed, o);
        keep_min = min(keep_min, __shfl_xor_sync(GPM_FULL_MASK, keep_min, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (removed) atomicOr(&flags[0], 1);
        if (keep_min != INT32_MAX) atomicMin(&flags[1], keep_min);
    }
}

__global__ void k_features(const int32_t* __restrict__ indptr, const int32_t* __restrict__ indices,
                           const int32_t* __restrict__ deg, const int32_t* __restrict__ outdeg,
                           const float* __restrict__ tri, const int32_t* __restrict__ core, int32_t n, int k,
                           float* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long v = warp; v < n; v += nw) {
        const int b = indptr[v], e = indptr[v + 1];
        double s_all = 0, s_up = 0;
        int c_up = 0;
        for (int t = b + lane; t < e; t += 32) {
            const int u = indices[t];
            const int du = deg[u];
            s_all += du;
            if (u > v) {
                s_up += du;
                c_up++;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            s_all += __shfl_xor_sync(GPM_FULL_MASK, s_all, o);
            s_up += __shfl_xor_sync(GPM_FULL_MASK, s_up, o);
            c_up += __shfl_xor_sync(GPM_FULL_MASK, c_up, o);
        }
        if (lane == 0) {
            float* f = out + v * MLP_IN;
            f[0] = log1pf((float)(e - b));
            f[1] = log1pf((float)outdeg[v]);
            f[2] = log1pf((float)c_up);
            f[3] = (float)log1p(s_all);
            f[4] = (float)log1p(s_up);
            f[5] = log1pf(tri[v]);
            f[6] = log1pf((float)core[v]);
            f[7] = (float)k / 8.f;
        }
    }
}

static int blocks_for(int64_t items_x32, int threads, int sms) {
    int64_t b = (items_x32 + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)sms * 32));
}

// core numbers of every vertex into d_core (host-driven peeling passes)
static void core_numbers(gpm_graph* g, int32_t* d_core, DevBuf& tmp) {
    cudaStream_t s = g->stream;
    const int32_t n = g->n;
    tmp.ensure(sizeof(int32_t) * ((size_t)n + 8));
    int32_t* rem = tmp.as<int32_t>();
    int* flags = reinterpret_cast<int*>(rem + n);
    const int blocks = blocks_for((int64_t)n, 256, g->num_sms);
    k_core_init<<<blocks, 256, 0, s>>>(g->degree.as<int32_t>(), n, rem, d_core);
    GPM_CUDA(cudaGetLastError());
    int c = 0;
    for (long long pass = 0;; pass++) {
        if (pass > 4ll * n + 16) fail(GPM_ECUDA, "core decomposition did not converge");
        const int init[2] = {0, INT32_MAX};
        GPM_CUDA(cudaMemcpyAsync(flags, init, sizeof(init), cudaMemcpyHostToDevice, s));
        k_core_peel<<<blocks, 256, 0, s>>>(g->indptr.as<int32_t>(), g->indices.as<int32_t>(), n, c, rem, d_core,
                                           flags);
        GPM_CUDA(cudaGetLastError());
        int h[2];
        GPM_CUDA(cudaMemcpyAsync(h, flags, sizeof(h), cudaMemcpyDeviceToHost, s));
        GPM_CUDA(cudaStreamSynchronize(s));
        if (h[0]) continue;              // level c removed something: run it again
        if (h[1] == INT32_MAX) break;    // nothing left
        c = std::max(c + 1, h[1]);
    }
}

void root_features(gpm_graph* g, int k, float* d_out) {
    ensure_dag(g);
    cudaStream_t s = g->stream;
    DevBuf tri, core, tmp;
    tri.ensure(sizeof(float) * std::max(g->n, 1));
    core.ensure(sizeof(int32_t) * std::max(g->n, 1));
    if (g->n > 0) {
        core_numbers(g, core.as<int32_t>(), tmp);
        k_tri_root<<<blocks_for((int64_t)g->n * 32, 256, g->num_sms), 256, 0, s>>>(
            g->dag_off.as<int32_t>(), g->dag_adj.as<int32_t>(), g->dag_outdeg.as<int32_t>(), g->n, tri.as<float>());
        k_features<<<blocks_for((int64_t)g->n * 32, 256, g->num_sms), 256, 0, s>>>(
            g->indptr.as<int32_t>(), g->indices.as<int32_t>(), g->degree.as<int32_t>(), g->dag_outdeg.as<int32_t>(),
            tri.as<float>(), core.as<int32_t>(), g->n, k, d_out);
        GPM_CUDA(cudaGetLastError());
    }
    GPM_CUDA(cudaStreamSynchronize(s));
}

// ------------------------------------------------------------------ MLP

__device__ __forceinline__ void load_weights(const uint16_t* __restrict__ w, float* W) {
    for (int i = threadIdx.x; i < MLP_NPARAM; i += blockDim.x) {
        __nv_bfloat16_raw r;
        r.x = w[i];
        W[i] = __bfloat162float(__nv_bfloat16(r));
    }
    __syncthreads();
}

// thread per sample; y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3
__global__ void __launch_bounds__(256) k_mlp_forward(const uint16_t* __restrict__ w, const float* __restrict__ x,
                                                     long long n, float* __restrict__ y) {
    __shared__ float W[MLP_NPARAM];
    load_weights(w, W);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float xi[MLP_IN];
#pragma unroll
        for (int q = 0; q < MLP_IN; q++) xi[q] = x[i * MLP_IN + q];
        float h1[MLP_H];
#pragma unroll
        for (int j = 0; j < MLP_H; j++) {
            float s = W[OFF_B1 + j];
#pragma unroll
            for (int q = 0; q < MLP_IN; q++) s = fmaf(W[OFF_W1 + j * MLP_IN + q], xi[q], s);
            h1[j] = fmaxf(s, 0.f);
        }
        float out = W[OFF_B3];
        for (int j = 0; j < MLP_H; j++) {
            float s = W[OFF_B2 + j];
#pragma unroll
            for (int q = 0; q < MLP_H; q++) s = fmaf(W[OFF_W2 + j * MLP_H + q], h1[q], s);
            out = fmaf(W[OFF_W3 + j], fmaxf(s, 0.f), out);
        }
        y[i] = out;
    }
}

// Gradients of mean_i (y_i - t_i)^2 over a minibatch of n samples.  A block
// handles 64 samples at a time: one thread per sample computes the forward
// and the per-sample deltas into shared memory, then the block forms the
// weight gradients as sums over its samples and adds them to grad (FP32
// atomics).  grad and loss must be zero on entry.
constexpr int BW_TILE = 64;
__global__ void __launch_bounds__(BW_TILE) k_mlp_backward(const uint16_t* __restrict__ w, const float* __restrict__ x,
                                                          const float* __restrict__ t, long long n,
                                                          float* __restrict__ grad, float* __restrict__ loss) {
    extern __shared__ float sh[];
    float* W = sh;                                   // MLP_NPARAM
    float* X = W + MLP_NPARAM + 3;                   // BW_TILE x 8
    float* H1 = X + BW_TILE * MLP_IN;                // BW_TILE x 65
    float* H2 = H1 + BW_TILE * (MLP_H + 1);
    float* D2 = H2 + BW_TILE * (MLP_H + 1);          // dL/dz2
    float* D1 = D2 + BW_TILE * (MLP_H + 1);          // dL/dz1
    float* DY = D1 + BW_TILE * (MLP_H + 1);          // dL/dy
    load_weights(w, W);
    const int tid = threadIdx.x;
    const float inv_n = 1.0f / (float)n;
    float lsum = 0.f;
    // per-thread accumulators for the entries this thread owns
    float gW2[MLP_H];                                // row tid of dW2 (64 entries)
    float gW1[MLP_IN];                               // row tid of dW1
    float gb1 = 0.f, gb2 = 0.f, gw3 = 0.f, gb3 = 0.f;
#pragma unroll
    for (int q = 0; q < MLP_H; q++) gW2[q] = 0.f;
#pragma unroll
    for (int q = 0; q < MLP_IN; q++) gW1[q] = 0.f;

    for (long long base = (long long)blockIdx.x * BW_TILE; base < n; base += (long long)gridDim.x * BW_TILE) {
        const long long i = base + tid;
        const bool act = i < n;
        float xi[MLP_IN];
#pragma unroll
        for (int q = 0; q < MLP_IN; q++) {
            xi[q] = act ? x[i * MLP_IN + q] : 0.f;
            X[tid * MLP_IN + q] = xi[q];
        }
        for (int j = 0; j < MLP_H; j++) {
            float s = W[OFF_B1 + j];
#pragma unroll
            for (int q = 0; q < MLP_IN; q++) s = fmaf(W[OFF_W1 + j * MLP_IN + q], xi[q], s);
            H1[tid * (MLP_H + 1) + j] = s;           // z1 for now
        }
        float yv = W[OFF_B3];
        for (int j = 0; j < MLP_H; j++) {
            float s = W[OFF_B2 + j];
            for (int q = 0; q < MLP_H; q++) s = fmaf(W[OFF_W2 + j * MLP_H + q], fmaxf(H1[tid * (MLP_H + 1) + q], 0.f), s);
            H2[tid * (MLP_H + 1) + j] = s;           // z2 for now
            yv = fmaf(W[OFF_W3 + j], fmaxf(s, 0.f), yv);
        }
        const float diff = act ? (yv - t[i]) : 0.f;
        lsum += diff * diff;
        const float dy = 2.f * diff * inv_n;
        DY[tid] = dy;
        for (int j = 0; j < MLP_H; j++) {
            const float z2 = H2[tid * (MLP_H + 1) + j];
            D2[tid * (MLP_H + 1) + j] = z2 > 0.f ? dy * W[OFF_W3 + j] : 0.f;
        }
        for (int q = 0; q < MLP_H; q++) {
            float s = 0.f;
            for (int j = 0; j < MLP_H; j++) s = fmaf(D2[tid * (MLP_H + 1) + j], W[OFF_W2 + j * MLP_H + q], s);
            const float z1 = H1[tid * (MLP_H + 1) + q];
            D1[tid * (MLP_H + 1) + q] = z1 > 0.f ? s : 0.f;
        }
        __syncthreads();
        // thread tid owns row j = tid of dW2, dW1 and entry j of b1, b2, w3
        const int j = tid;
        for (int sidx = 0; sidx < BW_TILE; sidx++) {
            const float d2 = D2[sidx * (MLP_H + 1) + j];
            const float d1 = D1[sidx * (MLP_H + 1) + j];
#pragma unroll
            for (int q = 0; q < MLP_H; q++) gW2[q] = fmaf(d2, fmaxf(H1[sidx * (MLP_H + 1) + q], 0.f), gW2[q]);
#pragma unroll
            for (int q = 0; q < MLP_IN; q++) gW1[q] = fmaf(d1, X[sidx * MLP_IN + q], gW1[q]);
            gb1 += d1;
            gb2 += d2;
            gw3 = fmaf(DY[sidx], fmaxf(H2[sidx * (MLP_H + 1) + j], 0.f), gw3);
            if (j == 0) gb3 += DY[sidx];
        }
        __syncthreads();
    }
    const int j = tid;
    for (int q = 0; q < MLP_H; q++) atomicAdd(&grad[OFF_W2 + j * MLP_H + q], gW2[q]);
    for (int q = 0; q < MLP_IN; q++) atomicAdd(&grad[OFF_W1 + j * MLP_IN + q], gW1[q]);
    atomicAdd(&grad[OFF_B1 + j], gb1);
    atomicAdd(&grad[OFF_B2 + j], gb2);
    atomicAdd(&grad[OFF_W3 + j], gw3);
    if (j == 0) atomicAdd(&grad[OFF_B3], gb3);
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(GPM_FULL_MASK, lsum, o);
    if ((tid & 31) == 0) atomicAdd(loss, lsum * inv_n);
}

// Adam (Kingma & Ba 2015), bias-corrected; master weights FP32, BF16 copy out
__global__ void k_mlp_adam(float* __restrict__ master, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ grad, int step, float lr, float beta1, float beta2, float eps,
                           uint16_t* __restrict__ w) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= MLP_NPARAM) return;
    const float g = grad[i];
    const float mi = beta1 * m[i] + (1.f - beta1) * g;
    const float vi = beta2 * v[i] + (1.f - beta2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.f - powf(beta1, (float)step));
    const float vh = vi / (1.f - powf(beta2, (float)step));
    const float p = master[i] - lr * mh / (sqrtf(vh) + eps);
    master[i] = p;
    __nv_bfloat16 b = __float2bfloat16_rn(p);
    w[i] = __nv_bfloat16_raw(b).x;
}

void mlp_forward(const uint16_t* w, const float* x, int64_t n, float* y, cudaStream_t s) {
    if (n <= 0) return;
    int dev = 0, sms = 0;
    GPM_CUDA(cudaGetDevice(&dev));
    GPM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
    k_mlp_forward<<<blocks, 256, 0, s>>>(w, x, n, y);
    GPM_CUDA(cudaGetLastError());
}

void mlp_grad(const uint16_t* w, const float* x, const float* t, int64_t n, float* grad, float* loss, cudaStream_t s) {
    GPM_CUDA(cudaMemsetAsync(grad, 0, sizeof(float) * MLP_NPARAM, s));
    GPM_CUDA(cudaMemsetAsync(loss, 0, sizeof(float), s));
    if (n <= 0) return;
    int dev = 0, sms = 0;
    GPM_CUDA(cudaGetDevice(&dev));
    GPM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = sizeof(float) * (MLP_NPARAM + 3 + BW_TILE * MLP_IN + 4 * BW_TILE * (MLP_H + 1) + BW_TILE);
    GPM_CUDA(cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int blocks = (int)std::min<int64_t>((n + BW_TILE - 1) / BW_TILE, (int64_t)sms * 4);
    k_mlp_backward<<<blocks, BW_TILE, smem, s>>>(w, x, t, n, grad, loss);
    GPM_CUDA(cudaGetLastError());
}

void mlp_adam(float* master, float* m, float* v, const float* grad, int step, float lr, uint16_t* w, cudaStream_t s) {
    k_mlp_adam<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(master, m, v, grad, step, lr, 0.9f, 0.999f, 1e-8f, w);
    GPM_CUDA(cudaGetLastError());
}

// ------------------------------------------------------------ schedule

// monotone 16-bit key of a float score, descending order -> ascending key
__device__ __forceinline__ uint32_t score_key(float f) {
    uint32_t u = __float_as_uint(f);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);   // order-preserving map to uint32
    return 0xffffu - (u >> 16);
}

__global__ void k_score_hist(const float* __restrict__ score, const int32_t* __restrict__ roots, long long n,
                             int32_t* __restrict__ hist) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        atomicAdd(&hist[score_key(score[roots ? roots[i] : i])], 1);
}

__global__ void k_score_scatter(const float* __restrict__ score, const int32_t* __restrict__ roots, long long n,
                                int32_t* __restrict__ cursor, int32_t* __restrict__ order) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int v = roots ? roots[i] : (int)i;
        order[atomicAdd(&cursor[score_key(score[v])], 1)] = v;
    }
}

// roots (or all vertices) ordered by score descending (bucketed by the top 16
// bits of the float; ties in no particular order)
void order_by_score(gpm_graph* g, const float* d_score, const int32_t* d_roots, int64_t n_roots, DevBuf& out) {
    cudaStream_t s = g->stream;
    out.ensure(sizeof(int32_t) * std::max<int64_t>(n_roots, 1));
    DevBuf hist, cur, tmp;
    hist.ensure(sizeof(int32_t) * 65537);
    cur.ensure(sizeof(int32_t) * 65537);
    GPM_CUDA(cudaMemsetAsync(hist.ptr, 0, sizeof(int32_t) * 65537, s));
    if (n_roots > 0) {
        const int blocks = std::max(1, (int)std::min<int64_t>((n_roots + 255) / 256, (int64_t)g->num_sms * 16));
        k_score_hist<<<blocks, 256, 0, s>>>(d_score, d_roots, n_roots, hist.as<int32_t>());
        int64_t total = 0;
        exclusive_scan_i32(hist.as<int32_t>(), cur.as<int32_t>(), 65536, &total, s, tmp);
        k_score_scatter<<<blocks, 256, 0, s>>>(d_score, d_roots, n_roots, cur.as<int32_t>(), out.as<int32_t>());
        GPM_CUDA(cudaGetLastError());
    }
    GPM_CUDA(cudaStreamSynchronize(s));
}

}  // namespace gpm
