// monitor.cuh -- host loop of the paper's load balancing (Section 4.3.5):
// stop, redistribute, restart, for comparison with the in-kernel hand-off.
//
// The kernel runs without donation; warps count themselves in ctl->active
// while they hold a unit.  The host polls the control block on a second
// stream while the launch runs; once every root and seed unit has been handed
// out and fewer than threshold x warps still hold work, it raises ctl->stop.
// Busy warps then write their remaining work to a spill buffer (one unit per
// level with children left) and leave, and the host launches the kernel again
// over the spilled units, until a launch spills nothing.
#pragma once

#include <chrono>
#include <thread>

#include "common.cuh"

namespace gpm {

// launch(counter_roots, n_seeds, turn): start one launch on g->stream taking
// `counter_roots` roots from the counter and `n_seeds` seed units from
// buffer `turn`, spilling into buffer `turn ^ 1`, between g->ev0 and g->ev1.
// after(h): called with the control block of every finished launch (errors
// are checked before).  Returns the statistics.
template <class Launch, class After>
MonitorStats monitored_loop(gpm_graph* g, Control* ctl, int warps, long long n_roots, double threshold,
                            unsigned long long spill_cap, Launch launch, After after) {
    cudaStream_t s = g->stream;
    MonitorStats ms{};
    cudaStream_t mon = nullptr;
    GPM_CUDA(cudaStreamCreateWithFlags(&mon, cudaStreamNonBlocking));
    Control* snap = nullptr;
    if (cudaMallocHost(&snap, sizeof(Control)) != cudaSuccess) {
        cudaGetLastError();
        cudaStreamDestroy(mon);
        fail(GPM_ENOMEM, "pinned host buffer for the monitor");
    }
    struct Cleanup {
        cudaStream_t m;
        Control* h;
        ~Cleanup() {
            cudaFreeHost(h);
            cudaStreamDestroy(m);
        }
    } cleanup{mon, snap};
    long long counter_roots = n_roots;
    unsigned long long n_seeds = 0;
    int turn = 0;
    const auto t_wall = std::chrono::steady_clock::now();
    for (;;) {
        Control h{};
        h.pending = counter_roots + (long long)n_seeds;
        GPM_CUDA(cudaMemcpyAsync(ctl, &h, sizeof(Control), cudaMemcpyHostToDevice, s));
        launch(counter_roots, n_seeds, turn);
        bool stopped = false;
        for (;;) {
            const cudaError_t q = cudaEventQuery(g->ev1);
            if (q == cudaSuccess) break;
            if (q != cudaErrorNotReady) check_cuda(q, "cudaEventQuery");
            if (!stopped) {
                GPM_CUDA(cudaMemcpyAsync(snap, ctl, sizeof(Control), cudaMemcpyDeviceToHost, mon));
                GPM_CUDA(cudaStreamSynchronize(mon));
                const bool handed_out =
                    snap->next_root >= (unsigned long long)counter_roots && snap->next_seed >= n_seeds;
                if (handed_out && snap->active < threshold * warps) {
                    const int one = 1;
                    GPM_CUDA(cudaMemcpyAsync(&ctl->stop, &one, sizeof(int), cudaMemcpyHostToDevice, mon));
                    GPM_CUDA(cudaStreamSynchronize(mon));
                    stopped = true;
                }
            }
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
        GPM_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(Control), cudaMemcpyDeviceToHost, s));
        GPM_CUDA(cudaStreamSynchronize(s));
        float kms = 0.f;
        GPM_CUDA(cudaEventElapsedTime(&kms, g->ev0, g->ev1));
        ms.kernel_ms += kms;
        ms.launches++;
        if (h.error == DEV_EINVAL) fail(GPM_ECUDA, "pattern table lookup hit an invalid traversal code");
        if (h.error >= DEV_ECHECK)
            fail(GPM_ECUDA, "device consistency check " + std::to_string(h.error - DEV_ECHECK) + " failed");
        if (h.error) fail(GPM_ECUDA, "device error " + std::to_string(h.error));
        if (h.overflow) fail(GPM_EOVERFLOW, "a count exceeds 2^64-1");
        after(h);
        if (h.spill_n == 0) break;
        if (h.spill_n > spill_cap) fail(GPM_ECUDA, "spill buffer overflow");
        ms.spilled_units += (long long)h.spill_n;
        counter_roots = 0;
        n_seeds = h.spill_n;
        turn ^= 1;
    }
    ms.wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_wall).count();
    return ms;
}

}  // namespace gpm
