// common.cuh -- internal declarations shared by the libgpm CUDA sources.
//
// Nothing here is part of the public ABI (include/gpm.h).  The library is
// single-GPU: every device buffer of a gpm_graph lives on the device that was
// current when the graph was created, and every kernel runs on the graph's
// stream.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "gpm.h"

namespace gpm {

// ------------------------------------------------------------------ errors

// Thread-local message of the last failure (gpm_last_error()).
void set_error(const std::string& msg);
void clear_error();

struct Error {
    gpm_status status;
    std::string msg;
};

// Throwing is internal only: every extern "C" entry point catches and maps
// to a status, so no exception crosses the ABI.
[[noreturn]] void fail(gpm_status s, const std::string& msg);
void check_cuda(cudaError_t e, const char* what);
#define GPM_CUDA(call) ::gpm::check_cuda((call), #call)

// --------------------------------------------------------- device buffers

// Grow-only device allocation owned by a graph.
struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : ptr(o.ptr), bytes(o.bytes) {
        o.ptr = nullptr;
        o.bytes = 0;
    }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) {
            release();
            ptr = o.ptr;
            bytes = o.bytes;
            o.ptr = nullptr;
            o.bytes = 0;
        }
        return *this;
    }
    ~DevBuf();
    void ensure(size_t need);   // may reallocate (contents lost)
    void release();
    template <class T> T* as() const { return static_cast<T*>(ptr); }
};

// -------------------------------------------------------------- the graph

struct DagView {
    const int32_t* off = nullptr;    // n+1 offsets, every list padded to a multiple of 4
    const int32_t* adj = nullptr;    // out-neighbours (higher (degree, id)), sorted by id
    const int32_t* outdeg = nullptr; // n exact out-degrees
    int32_t max_outdeg = 0;
};

}  // namespace gpm

struct gpm_graph {
    int device = 0;
    cudaStream_t stream = nullptr;
    int32_t n = 0;
    int64_t nnz = 0;            // indptr[n] = 2m
    int32_t max_deg = 0;
    int num_sms = 0;

    gpm::DevBuf indptr, indices, degree;

    // degree-ordered DAG (built on the first clique call)
    bool dag_ready = false;
    gpm::DevBuf dag_off, dag_adj, dag_outdeg;
    int32_t max_outdeg = 0;

    // root orders of the plain scheduler (built lazily)
    bool order_motif_ready = false, order_clique_ready = false;
    gpm::DevBuf order_motif, order_clique;
    bool order_id_ready = false;
    gpm::DevBuf order_id;
    // custom root order (learned scheduler or caller)
    gpm::DevBuf order_custom;
    int64_t order_custom_len = 0;

    // per-call scratch, grown on demand
    gpm::DevBuf scratch_small;     // counters, flags, queue control
    gpm::DevBuf scratch_queue;     // donation ring
    gpm::DevBuf scratch_slab;      // per-warp DFS stacks (extension arrays)
    gpm::DevBuf scratch_mark;      // per-warp vertex marks (motif)
    size_t mark_bytes_cleared = 0;
    gpm::DevBuf roots_tmp;         // caller root lists
    gpm::DevBuf per_root_tmp;

    // schedules built by gpm_sched_from_scores, per application
    struct Sched {
        bool ready = false;
        gpm::DevBuf roots;                 // kernel order: counter roots, then split roots
        int64_t n = 0, n_counter = 0;
        int32_t chunks = 0;                // units per split root (uniform plan)
        gpm::DevBuf chunk_off;             // per split root unit offsets (balanced plan), else empty
        int64_t n_seeds = 0;               // units of the split roots in all
        std::vector<int64_t> caller_index; // kernel position -> index in the caller's list
    } sched[2];

    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    gpm_config cfg{};
    gpm_stats stats{};
};

namespace gpm {

// --------------------------------------------------------- shared control

// Control block of one persistent enumeration launch (device memory).  The
// words that different groups of warps hammer sit on separate 128-byte
// lines: unit counters (warps taking work), termination state (polled by
// idle warps), the idle-ring positions (read by busy warps deciding to
// split), statistics, and the final counts.
struct alignas(128) Control {
    unsigned long long next_root;     // next index into the root list
    unsigned long long next_seed;     // next pre-split seed unit
    alignas(128) long long pending;   // roots + donated units not yet finished
    int error;                        // GPM_* status raised on the device
    int stop;                         // host-monitored balancing: spill the remaining work and leave
    alignas(128) int active;          // host-monitored balancing: warps holding a unit
    int pad_active;
    unsigned long long spill_n;       // host-monitored balancing: units spilled so far
    alignas(128) unsigned long long q_head;   // (alignas binds per declarator: one per line)
    unsigned long long q_tail;
    alignas(128) unsigned long long donations;
    unsigned long long units_done, idle_polls;
    unsigned long long word_ops;      // clique: 32-bit candidate-word AND+POPC operations
    unsigned long long busy_ns;       // sum over warps of time spent inside work units
    int overflow;
    int pad;
    alignas(128) unsigned long long counts[GPM_CLIQUE_MAX_K + 1];  // per clique size (clique kernel)
    alignas(128) unsigned long long heavy_next;   // clique list path: next (heavy root, chunk) unit
    int n_heavy;                                  // clique list path: roots above the bitmap limit
    int pad_heavy;
    unsigned long long list_diag[3];              // listing: the first wait that ran out (position, count, tail seen)
};

// Device-side status values (mirrors gpm_status).
enum : int { DEV_OK = 0, DEV_ETIMEOUT = GPM_ETIMEOUT, DEV_EOVERFLOW = GPM_EOVERFLOW,
             DEV_EINVAL = GPM_EINVAL,
             DEV_ECHECK = 64 };   // + n: internal consistency check n failed (the access was skipped)

// Launch geometry for a persistent kernel.
struct Grid {
    int blocks = 0;
    int warps_per_block = 0;
    int total_warps() const { return blocks * warps_per_block; }
};

// graph.cu
void ensure_dag(gpm_graph* g);
const int32_t* ensure_root_order(gpm_graph* g, int app);  // plain scheduler order
const int32_t* ensure_id_order(gpm_graph* g);             // 0, 1, ..., n-1
void exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, int64_t* total,
                        cudaStream_t s, DevBuf& tmp);

// lut.cpp (host pattern dictionary)
struct PatternTable {
    int k = 0;
    int64_t num_patterns = 0;
    std::vector<uint64_t> pattern_code;   // canonical full code of each pattern id
    std::vector<uint16_t> lut;            // traversal code -> pattern id (0xFFFF invalid)
};
const PatternTable& pattern_table(int k);  // built once per k, cached
const uint16_t* device_lut(int k);         // uploaded once per (device, k)

// Pre-split of a schedule's split roots (positions n_counter .. n_roots-1 of
// the root list): root j becomes units d_chunk_off[j] .. d_chunk_off[j+1]-1
// (device prefix sums), or `chunks` units each when d_chunk_off is null.
// The cuts between a root's units balance estimated work (see
// gpm_balanced_cut).
struct SplitPlan {
    int chunks = 0;
    const int32_t* d_chunk_off = nullptr;
    int64_t n_seeds = 0;
};

// Host-monitored balancing (the paper's stop / redistribute / restart)
struct MonitorStats {
    int32_t launches = 0;
    int64_t spilled_units = 0;
    double kernel_ms = 0.0;   // sum over the launches
    double wall_ms = 0.0;     // the whole loop, host monitor included
};
void run_clique_monitored(gpm_graph* g, int k, double threshold, uint64_t* count_out, MonitorStats* ms);
void run_clique_dfs(gpm_graph* g, int k, uint64_t* count_out);   // the paper's DM_DFS baseline
// clique_list.cu: roots whose out-degree exceeds the bitmap limit, counted
// by list intersection after the bitmap launch (same Control, same counters)
void run_clique_list(gpm_graph* g, int k_lo, int k_hi, const int32_t* d_roots, int64_t n_roots,
                     unsigned long long* d_per_root, Control* ctl, int bitmap_limit);
void run_motif_monitored(gpm_graph* g, int k, double threshold, uint64_t* counts_out, MonitorStats* ms);

// clique.cu / motif.cu
// d_roots[0 .. n_roots): the roots; the first n_counter are handed out one by
// one, the rest are pre-split as `plan` says (n_counter < 0: no pre-split).
// d_roots == NULL: every vertex, heaviest first.
void run_clique(gpm_graph* g, int k_lo, int k_hi, const int32_t* d_roots, int64_t n_roots,
                unsigned long long* d_per_root, uint64_t* counts_out, int64_t n_counter = -1,
                const SplitPlan* plan = nullptr);
struct ListJob;
void run_motif(gpm_graph* g, int k, const int32_t* d_roots, int64_t n_roots,
               unsigned long long* d_per_root, uint64_t* counts_out, int64_t n_counter = -1,
               const SplitPlan* plan = nullptr, double monitor_threshold = -1.0,
               MonitorStats* monitor_stats = nullptr, ListJob* list = nullptr);

// Listing (aggregate_store; list.cu, list_ring.cuh).  list_drain runs the
// host consumer until the launch recorded before g->ev1 has ended and its
// records are taken; list_ring_of is the device view of the job's ring.
struct ListRing;
ListRing list_ring_of(const ListJob* job, Control* ctl);
void list_drain(ListJob* job, gpm_graph* g, Control* ctl);
std::string list_where(const ListJob* job, const Control& h);
void launch_clique_store(gpm_graph* g, int k, const ListRing& ring, Control* ctl);
void run_list(gpm_graph* g, int app, int k, int32_t pattern, int64_t ring_records, gpm_list_consumer consumer,
              void* user, uint64_t* delivered);

// sched.cu
void root_features(gpm_graph* g, int k, float* d_out);
void mlp_forward(const uint16_t* w, const float* x, int64_t n, float* y, cudaStream_t s);
void mlp_grad(const uint16_t* w, const float* x, const float* t, int64_t n, float* grad, float* loss, cudaStream_t s);
void mlp_adam(float* master, float* m, float* v, const float* grad, int step, float lr, uint16_t* w, cudaStream_t s);
void order_by_score(gpm_graph* g, const float* d_score, const int32_t* d_roots, int64_t n_roots, DevBuf& out);

// helpers
int resident_blocks(const void* kernel, int threads, size_t smem);
// max_per_sm > 0 caps the resident blocks per SM unless the configuration sets blocks_per_sm
Grid plan_grid(gpm_graph* g, const void* kernel, int warps_per_block, size_t smem_per_block, int max_per_sm = 0);
// warps per block (16, 8, 4, 2 or 1) that keeps the most warps resident per SM
int best_warps_per_block(const void* kernel, size_t smem_per_warp, size_t smem_fixed);
gpm_config default_config();

}  // namespace gpm

#ifdef __CUDACC__
// ----------------------------------------------------------- device helpers

#define GPM_FULL_MASK 0xffffffffu

__device__ __forceinline__ unsigned long long gpm_globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Cut q of `ch` over the L children of a root, 0 = c_0 <= c_1 .. <= c_ch = L,
// so that the units [c_q, c_{q+1}) carry about equal estimated work: a root's
// child at position c (ESU array position, or orientation position for
// cliques) has about (L - c) candidates after it, and its subtree grows like
// (L - c)^(k-2), so the work after c is about (L - c)^(k-1).
__device__ __forceinline__ int gpm_balanced_cut(int L, int q, int ch, int k) {
    if (q <= 0) return 0;
    if (q >= ch) return L;
    const float r = powf(1.0f - (float)q / (float)ch, 1.0f / (float)max(k - 1, 1));
    const int c = L - (int)ceilf((float)L * r);
    return min(max(c, 0), L);
}

__device__ __forceinline__ unsigned gpm_lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <class T>
__device__ __forceinline__ T gpm_warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(GPM_FULL_MASK, v, o);
    return v;
}

// Carry-checked counting.  Counts are non-negative, so a partial sum that
// wraps means the true total is >= 2^64: the helpers below raise a flag
// instead of letting a wrapped value through (the GPM_EOVERFLOW contract).
// Inner-loop lane accumulators are not checked: each of their adds is below
// 2^16 and they are reset per work unit, so one would have to run for years
// to wrap; every add from a unit upwards goes through these helpers.
__device__ __forceinline__ unsigned long long gpm_add_cc(unsigned long long a, unsigned long long b, int& ovf) {
    const unsigned long long s = a + b;
    ovf |= s < a ? 1 : 0;
    return s;
}

// Sum over the warp (every lane gets it); ovf is raised in every lane when
// any partial sum wrapped.
__device__ __forceinline__ unsigned long long gpm_warp_sum_cc(unsigned long long v, int& ovf) {
    for (int o = 16; o > 0; o >>= 1) v = gpm_add_cc(v, __shfl_xor_sync(GPM_FULL_MASK, v, o), ovf);
    ovf = __any_sync(GPM_FULL_MASK, ovf) ? 1 : 0;
    return v;
}

// Atomic add into a (shared or global) counter; *flag = 1 if it wrapped.
__device__ __forceinline__ void gpm_atomic_add_cc(unsigned long long* c, unsigned long long v, int* flag) {
    if (!v) return;
    const unsigned long long old = atomicAdd(c, v);
    if (old + v < old) atomicExch(flag, 1);
}

// ------------------------------------------------- donation queue (device)
//
// Bounded multi-producer multi-consumer ring of sequence-numbered slots
// (after D. Vyukov's bounded MPMC queue).  Slot i starts with seq = i.  A
// producer reserves position p (seq == p), writes the unit -- and any payload
// kept beside the ring at index p % cap -- and publishes seq = p + 1.  A
// consumer claims p (seq == p + 1), reads, and releases with seq = p + cap.
// Every loop is bounded: a full, empty or contended queue reports failure
// and the caller keeps (or goes on looking for) work.  Reads of published
// data go through L2 (ld.global.cg): L1 is not coherent across SMs.
struct QSeq {
    unsigned long long seq;
};

namespace gpm {
__global__ void k_queue_init(QSeq* q, unsigned long long cap);
// CSR checks (graph.cu): bits of *bad: 1 indptr, 2 id range, 4 self-loop,
// 8 order/duplicates, 16 symmetry
__global__ void k_validate(const int32_t* __restrict__ indptr, const int32_t* __restrict__ indices, int32_t n,
                           int64_t nnz, int* __restrict__ bad);
__global__ void k_indptr_monotone(const int32_t* __restrict__ indptr, int32_t n, int* __restrict__ bad);
}

__device__ __forceinline__ bool gpm_q_reserve(QSeq* q, unsigned long long cap, unsigned long long* tail,
                                              unsigned long long* out_pos) {
    unsigned long long pos = *(volatile unsigned long long*)tail;
    for (int tries = 0; tries < 256; tries++) {
        const unsigned long long seq = *(volatile unsigned long long*)&q[pos % cap].seq;
        const long long dif = (long long)(seq - pos);
        if (dif == 0) {
            const unsigned long long prev = atomicCAS(tail, pos, pos + 1);
            if (prev == pos) {
                *out_pos = pos;
                return true;
            }
            pos = prev;
        } else if (dif < 0) {
            return false;  // full
        } else {
            pos = *(volatile unsigned long long*)tail;
        }
    }
    return false;
}

// call after every writer of the slot's data has executed __threadfence()
__device__ __forceinline__ void gpm_q_publish(QSeq* q, unsigned long long cap, unsigned long long pos) {
    atomicExch(&q[pos % cap].seq, pos + 1);
}

__device__ __forceinline__ bool gpm_q_claim(QSeq* q, unsigned long long cap, unsigned long long* head,
                                            unsigned long long* out_pos) {
    unsigned long long pos = *(volatile unsigned long long*)head;
    for (int tries = 0; tries < 256; tries++) {
        const unsigned long long seq = *(volatile unsigned long long*)&q[pos % cap].seq;
        const long long dif = (long long)(seq - (pos + 1));
        if (dif == 0) {
            const unsigned long long prev = atomicCAS(head, pos, pos + 1);
            if (prev == pos) {
                __threadfence();
                *out_pos = pos;
                return true;
            }
            pos = prev;
        } else if (dif < 0) {
            return false;  // empty
        } else {
            pos = *(volatile unsigned long long*)head;
        }
    }
    return false;
}

// call after every reader of the slot's data is done (and fenced)
__device__ __forceinline__ void gpm_q_release(QSeq* q, unsigned long long cap, unsigned long long pos) {
    atomicExch(&q[pos % cap].seq, pos + cap);
}

// ------------------------------------------ direct hand-off of donated work
//
// An idle warp registers its global warp id in a ring (the sequence-numbered
// ring above, holding ints, capacity >= every warp of the launch) and then
// watches only its OWN mailbox flag -- no shared word is polled.  A busy warp
// that splits its work claims one registered id from the ring, writes the
// unit (and payload) into that warp's mailbox, fences, and raises the flag.
// Only the few donors contend on the ring, never the many idle warps.
struct MailHdr {
    int ready;                 // 1: a unit is waiting in this mailbox
    int pad[3];
};

__device__ __forceinline__ bool gpm_idle_register(QSeq* seq, int32_t* ids, unsigned long long cap,
                                                  unsigned long long* tail, int wid) {
    unsigned long long pos;
    if (!gpm_q_reserve(seq, cap, tail, &pos)) return false;
    ids[pos % cap] = wid;
    __threadfence();
    gpm_q_publish(seq, cap, pos);
    return true;
}

__device__ __forceinline__ bool gpm_idle_claim(QSeq* seq, int32_t* ids, unsigned long long cap,
                                               unsigned long long* head, int* wid) {
    unsigned long long pos;
    if (!gpm_q_claim(seq, cap, head, &pos)) return false;
    *wid = __ldcg(ids + pos % cap);
    __threadfence();
    gpm_q_release(seq, cap, pos);
    return true;
}

// word-wise L2 copy of a published POD record
template <class U>
__device__ __forceinline__ void gpm_load_cg(U* dst, const U* src) {
    static_assert(sizeof(U) % 4 == 0, "record size must be a multiple of 4 bytes");
    const unsigned* s = reinterpret_cast<const unsigned*>(src);
    unsigned* d = reinterpret_cast<unsigned*>(dst);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(U) / 4); i++) d[i] = __ldcg(s + i);
}

#endif  // __CUDACC__
