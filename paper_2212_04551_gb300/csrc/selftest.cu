// selftest.cu -- gpm_selftest_sum: the counting kernels' carry-checked
// reduction path (lane-private adds, warp sums, per-block shared counters,
// global counters), run over caller values, so that the overflow contract --
// a true count >= 2^64 gives GPM_EOVERFLOW, never a wrapped value -- can be
// exercised without a graph whose counts exceed 2^64 (which no test could
// enumerate).  It uses the same helpers as k_clique, k_motif and k_batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace gpm {

__global__ void k_selftest_sum(const unsigned long long* __restrict__ v, long long n, unsigned long long* out,
                               int* flag) {
    __shared__ unsigned long long block_total;
    if (threadIdx.x == 0) block_total = 0ull;
    __syncthreads();
    int ovf = 0;
    unsigned long long mine = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        mine = gpm_add_cc(mine, v[i], ovf);                 // lane-private, as a unit's count
    const unsigned long long w = gpm_warp_sum_cc(mine, ovf);   // warp
    if ((threadIdx.x & 31) == 0) {
        if (ovf) atomicExch(flag, 1);
        gpm_atomic_add_cc(&block_total, w, flag);            // block (shared counter)
    }
    __syncthreads();
    if (threadIdx.x == 0) gpm_atomic_add_cc(out, block_total, flag);   // global
}

void selftest_sum(const uint64_t* values, int64_t n, int blocks, int threads, uint64_t* out) {
    if (n < 0 || (n > 0 && !values) || !out) fail(GPM_EINVAL, "bad arguments");
    if (blocks < 1 || blocks > 65535 || threads < 32 || threads > 1024 || threads % 32)
        fail(GPM_EINVAL, "blocks in [1, 65535], threads a multiple of 32 in [32, 1024]");
    DevBuf buf;
    buf.ensure(sizeof(unsigned long long) * (size_t)(n + 2));
    unsigned long long* d = buf.as<unsigned long long>();
    unsigned long long* d_out = d + n;
    int* d_flag = reinterpret_cast<int*>(d + n + 1);
    if (n) GPM_CUDA(cudaMemcpy(d, values, sizeof(uint64_t) * n, cudaMemcpyHostToDevice));
    GPM_CUDA(cudaMemset(d_out, 0, 2 * sizeof(unsigned long long)));
    k_selftest_sum<<<blocks, threads>>>(d, n, d_out, d_flag);
    GPM_CUDA(cudaGetLastError());
    unsigned long long h[2] = {0, 0};
    GPM_CUDA(cudaMemcpy(h, d_out, sizeof(h), cudaMemcpyDeviceToHost));
    if (static_cast<int>(h[1] & 0xffffffffu)) fail(GPM_EOVERFLOW, "sum exceeds 2^64-1");
    *out = h[0];
}

}  // namespace gpm

extern "C" gpm_status gpm_selftest_sum(const uint64_t* values, int64_t n, int32_t blocks, int32_t threads,
                                       uint64_t* out) {
    try {
        gpm::clear_error();
        gpm::selftest_sum(values, n, blocks, threads, out);
        return GPM_OK;
    } catch (const gpm::Error& e) {
        gpm::set_error(e.msg);
        return e.status;
    } catch (...) {
        gpm::set_error("unexpected internal error");
        return GPM_ECUDA;
    }
}
