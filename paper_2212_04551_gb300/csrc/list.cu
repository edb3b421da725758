// list.cu -- subgraph listing with an asynchronous host consumer
// (aggregate_store, Section 4.3.4), host side.
//
// The ring of records lives in mapped pinned host memory: the kernel writes
// records straight into it and this thread takes them, in order, while the
// kernel runs (list_ring.cuh has the record format and the device side).
// The consumer sees each batch once; the slots are given back to the device
// before the consumer runs, so production and consumption overlap.
//
// While the kernel runs, this thread talks to it only through mapped host
// words (the count of records taken, the stop request), never through a
// copy or any other operation on a stream: the runtime may place a second
// stream on the same hardware queue as the kernel's, and a copy queued there
// would wait for the kernel, which waits for the copy.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "list_ring.cuh"

namespace gpm {

struct ListJob {
    int k = 0;
    int stride = 0;                        // words per record: sequence + k ids + tag
    unsigned long long cap = 0;            // records
    int32_t* host_rec = nullptr;           // mapped pinned ring
    int32_t* dev_rec = nullptr;
    unsigned long long* host_flags = nullptr;  // mapped pinned: [0] records taken, [1] stop request
    unsigned long long* dev_flags = nullptr;   // the same words, device address
    DevBuf head;                           // device: records reserved
    int tag_filter = -1;
    unsigned long long max_wait_ns = 0;
    gpm_list_consumer consumer = nullptr;
    void* user = nullptr;
    uint64_t delivered = 0;
    bool stopped = false;
    std::string where;                     // the ring's state when a listing ended early
    cudaStream_t stream = nullptr;         // the launch's stream
    bool launched = false;

    ~ListJob() {
        // the kernel may still run after an error on the host side: its waits
        // are bounded, so wait for it before the ring goes away
        if (launched) cudaStreamSynchronize(stream);
        if (host_rec) cudaFreeHost(host_rec);
        if (host_flags) cudaFreeHost(host_flags);
    }
};

ListRing list_ring_of(const ListJob* j, Control* ctl) {
    ListRing r{};
    r.rec = j->dev_rec;
    r.cap = j->cap;
    r.stride = j->stride;
    r.head = j->head.as<unsigned long long>();
    r.tail = j->dev_flags;
    r.stop = j->dev_flags + 1;
    r.ctl = ctl;
    r.max_wait_ns = j->max_wait_ns;
    r.tag_filter = j->tag_filter;
    return r;
}

std::string list_where(const ListJob* j, const Control& h) {
    std::string s = j->where;
    if (h.error == DEV_ETIMEOUT && h.list_diag[1])
        s += "; the wait that ran out: records " + std::to_string(h.list_diag[0]) + " .. " +
             std::to_string(h.list_diag[0] + h.list_diag[1] - 1) + " with " + std::to_string(h.list_diag[2]) +
             " seen consumed";
    return s;
}

// Take the records of the launch that ends at g->ev1, in order, until it has
// ended and everything it reserved is taken (or the listing stopped / failed).
void list_drain(ListJob* j, gpm_graph* g, Control* ctl) {
    const int words = j->stride - 1;
    const unsigned long long batch = std::min<unsigned long long>(j->cap, 65536);
    std::vector<int32_t> staging((size_t)batch * words);
    unsigned long long tail = 0;
    bool ended = false;
    unsigned long long head_end = 0;
    int idle_polls = 0;
    for (;;) {
        unsigned long long n = 0;
        if (!j->stopped) {
            while (n < batch) {
                const unsigned long long q = tail + n;
                const int32_t* rec = j->host_rec + (size_t)(q % j->cap) * j->stride;
                const uint32_t seq = __atomic_load_n(reinterpret_cast<const uint32_t*>(rec), __ATOMIC_ACQUIRE);
                if (seq != (uint32_t)(q + 1)) break;
                std::memcpy(staging.data() + (size_t)n * words, rec + 1, sizeof(int32_t) * words);
                n++;
            }
        }
        if (n) {
            idle_polls = 0;
            tail += n;
            // the slots are free again (release: after the reads above)
            __atomic_store_n(&j->host_flags[0], tail, __ATOMIC_RELEASE);
            j->delivered += n;
            if (j->consumer(staging.data(), (int64_t)n, (int32_t)words, j->user) != 0 && !j->stopped) {
                // the warps that wait for ring space see the request and end
                // the listing (ctl->error = DEV_STOPPED); the records after
                // this batch are not taken
                j->stopped = true;
                __atomic_store_n(&j->host_flags[1], 1ull, __ATOMIC_RELEASE);
            }
            continue;
        }
        if (ended) {
            if (tail < head_end)
                fail(GPM_ECUDA, "listing ended with " + std::to_string(head_end - tail) + " records unwritten");
            break;
        }
        const cudaError_t q = cudaEventQuery(g->ev1);
        if (q == cudaSuccess) {
            // the kernel has ended: plain copies are safe now
            int err = 0;
            GPM_CUDA(cudaMemcpy(&head_end, j->head.ptr, sizeof(head_end), cudaMemcpyDeviceToHost));
            GPM_CUDA(cudaMemcpy(&err, &ctl->error, sizeof(int), cudaMemcpyDeviceToHost));
            if (j->stopped || err) {         // an aborted launch leaves reserved records unwritten
                const int32_t* rec = j->host_rec + (size_t)(tail % j->cap) * j->stride;
                j->where = "host took " + std::to_string(tail) + " of " + std::to_string(head_end) +
                           " reserved records; the next slot holds sequence " +
                           std::to_string(__atomic_load_n(reinterpret_cast<const uint32_t*>(rec), __ATOMIC_ACQUIRE));
                break;
            }
            ended = true;                   // everything reserved is written: take the rest
            continue;
        }
        if (q != cudaErrorNotReady) check_cuda(q, "cudaEventQuery");
        // nothing ready: spin briefly, then back off
        if (++idle_polls > 64) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

void run_list(gpm_graph* g, int app, int k, int32_t pattern, int64_t ring_records, gpm_list_consumer consumer,
              void* user, uint64_t* delivered) {
    if (delivered) *delivered = 0;
    if (!consumer) fail(GPM_EINVAL, "consumer is NULL");
    if (app == GPM_APP_CLIQUE) {
        if (k < 3 || k > GPM_CLIQUE_MAX_K) fail(GPM_EINVAL, "clique listing needs 3 <= k <= 16");
        if (pattern != -1) fail(GPM_EINVAL, "clique listing takes pattern -1");
    } else if (app == GPM_APP_MOTIF) {
        if (k < 3 || k > GPM_MOTIF_MAX_K) fail(GPM_EINVAL, "motif listing needs 3 <= k <= 8");
        if (pattern < -1 || pattern >= pattern_table(k).num_patterns) fail(GPM_EINVAL, "pattern id out of range");
    } else {
        fail(GPM_EINVAL, "unknown app");
    }
    if (ring_records == 0) ring_records = 65536;
    if (ring_records < 64 || ring_records > (int64_t(1) << 30)) fail(GPM_EINVAL, "ring_records out of range [64, 2^30]");
    ListJob j;
    // the count delivered so far is reported on every way out, errors included
    struct Report {
        const ListJob& j;
        uint64_t* out;
        ~Report() {
            if (out) *out = j.delivered;
        }
    } report{j, delivered};
    j.stream = g->stream;
    j.k = k;
    j.stride = k + 2;
    j.cap = (unsigned long long)ring_records;
    j.tag_filter = pattern;
    j.max_wait_ns = (unsigned long long)std::max(1, g->cfg.max_idle_ms) * 1000000ull;
    j.consumer = consumer;
    j.user = user;
    const size_t ring_bytes = sizeof(int32_t) * (size_t)j.cap * j.stride;
    if (cudaHostAlloc(reinterpret_cast<void**>(&j.host_rec), ring_bytes, cudaHostAllocMapped) != cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void**>(&j.host_flags), 64, cudaHostAllocMapped) != cudaSuccess) {
        cudaGetLastError();
        fail(GPM_ENOMEM, "mapped host ring of " + std::to_string(ring_bytes) + " bytes");
    }
    std::memset(j.host_rec, 0, ring_bytes);
    std::memset(j.host_flags, 0, 64);
    GPM_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void**>(&j.dev_rec), j.host_rec, 0));
    GPM_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void**>(&j.dev_flags), j.host_flags, 0));
    j.head.ensure(sizeof(unsigned long long));
    cudaStream_t s = g->stream;
    GPM_CUDA(cudaMemsetAsync(j.head.ptr, 0, sizeof(unsigned long long), s));
    j.launched = true;

    if (app == GPM_APP_MOTIF) {
        std::vector<uint64_t> unused((size_t)pattern_table(k).num_patterns, 0);
        run_motif(g, k, nullptr, 0, nullptr, unused.data(), -1, nullptr, -1.0, nullptr, &j);
    } else {
        g->scratch_small.ensure(sizeof(Control));
        Control* ctl = g->scratch_small.as<Control>();
        Control h{};
        GPM_CUDA(cudaMemcpyAsync(ctl, &h, sizeof(Control), cudaMemcpyHostToDevice, s));
        launch_clique_store(g, k, list_ring_of(&j, ctl), ctl);
        list_drain(&j, g, ctl);
        GPM_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(Control), cudaMemcpyDeviceToHost, s));
        GPM_CUDA(cudaStreamSynchronize(s));
        float ms = 0.f;
        GPM_CUDA(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
        g->stats.kernel_ms = ms;
        if (h.error == DEV_ETIMEOUT)
            fail(GPM_ETIMEOUT, "the ring stayed full for longer than max_idle_ms (" + list_where(&j, h) + ")");
        if (h.error && h.error != DEV_STOPPED) fail(GPM_ECUDA, "device error " + std::to_string(h.error));
    }
}

}  // namespace gpm
