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

// ---------------------------------------------------------------------------
// L2 read bandwidth, measured: the denominator of the motif kernel's
// roofline, whose adjacency lists and per-warp marks are L2-resident.  A
// buffer of `bytes` (well below the 126 MB L2) is read `reps` times by a
// full grid after one warm pass; mode 0 streams it with coalesced 16-byte
// loads (bytes moved / time), mode 1 loads one 4-byte word from a
// pseudo-random 32-byte sector per lane (sectors x 32 B / time) -- the
// access shape of the marks.
namespace gpm {

__global__ void k_l2_stream(const uint4* __restrict__ buf, long long n16, int reps, unsigned* sink) {
    unsigned acc = 0;
    for (int r = 0; r < reps; r++)
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n16; i += (long long)gridDim.x * blockDim.x) {
            const uint4 v = __ldcg(buf + i);
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    if (acc == 0x9e3779b9u) atomicAdd(sink, 1u);   // keeps the loads; practically never true
}

__global__ void k_l2_sectors(const unsigned* __restrict__ buf, long long nsec, long long per_thread, unsigned* sink) {
    unsigned acc = 0;
    unsigned long long x = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) * 0x9e3779b97f4a7c15ull + 1ull;
    for (long long i = 0; i < per_thread; i++) {
        x ^= x << 13;
        x ^= x >> 7;
        x ^= x << 17;                              // xorshift64
        acc += __ldcg(buf + (x % (unsigned long long)nsec) * 8);
    }
    if (acc == 0x9e3779b9u) atomicAdd(sink, 1u);
}

double measure_l2(int64_t bytes, int mode, int reps) {
    if (bytes < (1 << 20) || bytes > (int64_t)(96ll << 20) || reps < 1 || (mode != 0 && mode != 1))
        fail(GPM_EINVAL, "bytes in [1 MB, 96 MB], reps >= 1, mode 0 or 1");
    int dev = 0, sms = 0;
    GPM_CUDA(cudaGetDevice(&dev));
    GPM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    DevBuf buf;
    buf.ensure((size_t)bytes + 256);
    GPM_CUDA(cudaMemset(buf.ptr, 1, (size_t)bytes));
    unsigned* sink = reinterpret_cast<unsigned*>(buf.as<unsigned char>() + bytes);
    cudaEvent_t e0, e1;
    GPM_CUDA(cudaEventCreate(&e0));
    GPM_CUDA(cudaEventCreate(&e1));
    const int blocks = sms * 8, threads = 256;
    double moved = 0.0;
    float ms = 0.f;
    if (mode == 0) {
        const long long n16 = bytes / 16;
        k_l2_stream<<<blocks, threads>>>(buf.as<uint4>(), n16, 1, sink);   // warm: bring it into L2
        GPM_CUDA(cudaEventRecord(e0));
        k_l2_stream<<<blocks, threads>>>(buf.as<uint4>(), n16, reps, sink);
        GPM_CUDA(cudaEventRecord(e1));
        moved = (double)n16 * 16.0 * reps;
    } else {
        const long long nsec = bytes / 32;
        const long long per_thread = std::max<long long>(1, nsec * reps / ((long long)blocks * threads));
        k_l2_stream<<<blocks, threads>>>(buf.as<uint4>(), bytes / 16, 1, sink);
        GPM_CUDA(cudaEventRecord(e0));
        k_l2_sectors<<<blocks, threads>>>(buf.as<unsigned>(), nsec, per_thread, sink);
        GPM_CUDA(cudaEventRecord(e1));
        moved = (double)per_thread * blocks * threads * 32.0;
    }
    GPM_CUDA(cudaGetLastError());
    GPM_CUDA(cudaEventSynchronize(e1));
    GPM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return moved / (ms * 1e-3) / 1e9;
}

}  // namespace gpm

extern "C" gpm_status gpm_measure_l2(int64_t bytes, int32_t mode, int32_t reps, double* gbs) {
    try {
        gpm::clear_error();
        if (!gbs) gpm::fail(GPM_EINVAL, "gbs is NULL");
        *gbs = gpm::measure_l2(bytes, mode, reps);
        return GPM_OK;
    } catch (const gpm::Error& e) {
        gpm::set_error(e.msg);
        return e.status;
    } catch (...) {
        gpm::set_error("unexpected internal error");
        return GPM_ECUDA;
    }
}
