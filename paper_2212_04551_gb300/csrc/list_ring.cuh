// list_ring.cuh -- the device side of subgraph listing (aggregate_store,
// Section 4.3.4): found k-vertex subgraphs are appended to a ring of records
// in mapped host memory that the host consumes while the kernel runs (the
// paper's producer-consumer buffer with an asynchronous CPU consumer).
//
// Record q (q = 0, 1, ...) sits in slot q mod cap; it is `stride` 32-bit
// words: a sequence word, the k vertex ids, and a tag (the pattern id of a
// motif, -1 for a clique).  A warp reserves up to 32 consecutive records on
// a device counter, waits (bounded) until the host has consumed far enough
// for them to be free, writes them, and then stores q + 1 in each record's
// sequence word (a system-scope release): the host takes records in order
// once their sequence word matches, and publishes the count it has taken in
// a mapped host word (beside it, a stop request).  The record a
// host waits for is never behind a wait of its own writer (a reservation of
// n <= 32 <= cap records at the host's position always fits), so the two
// sides cannot block each other.  A stop (the consumer asked for it), an
// error or a wait that runs out raises ctl->error; every later reservation
// then fails at once and the walks unwind at their next error check.
#pragma once

#include "common.cuh"

namespace gpm {

enum : int { DEV_STOPPED = 32 };   // the consumer asked to stop (not an error)

struct ListRing {
    int32_t* rec;                               // cap records (mapped host memory)
    unsigned long long cap;                     // records (>= 32)
    int stride;                                 // words per record: 1 + k + 1
    unsigned long long* head;                   // device: records reserved
    const unsigned long long* tail;             // mapped host word: records consumed
    const unsigned long long* stop;             // mapped host word: nonzero once the consumer asked to stop
    Control* ctl;
    unsigned long long max_wait_ns;             // a wait without host progress longer than this fails
    int tag_filter;                             // >= 0: only records with this tag
};

// The host's words (count of consumed records, stop request) in mapped host
// memory: system-scope acquire loads (the slots the count frees are written
// after it is read).  The release of a record's sequence word: after the
// record, at system scope (the host thread reads it from host memory).
__device__ __forceinline__ unsigned long long lr_load_sys(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void lr_publish(int32_t* p, int32_t v) {
    asm volatile("st.release.sys.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Lane 0: reserve n records; their first position, or ~0 when the listing
// is over (stop, error, or no host progress for max_wait_ns).
__device__ __forceinline__ unsigned long long lr_reserve(const ListRing& r, int n, unsigned long long& tail_seen) {
    if (*(volatile int*)&r.ctl->error) return ~0ull;
    const unsigned long long pos = atomicAdd(r.head, (unsigned long long)n);
    if (pos + n <= tail_seen + r.cap) return pos;
    unsigned long long t = lr_load_sys(r.tail);
    unsigned long long last = t, since = gpm_globaltimer();
    while (pos + n > t + r.cap) {
        if (*(volatile int*)&r.ctl->error) return ~0ull;
        if (lr_load_sys(r.stop)) {          // the consumer asked to stop: end the listing
            atomicCAS(&r.ctl->error, 0, DEV_STOPPED);
            return ~0ull;
        }
        const unsigned long long now = gpm_globaltimer();
        if (t != last) {
            last = t;
            since = now;
        } else if (now - since > r.max_wait_ns) {
            if (atomicCAS(&r.ctl->error, 0, DEV_ETIMEOUT) == 0) {
                r.ctl->list_diag[0] = pos;
                r.ctl->list_diag[1] = (unsigned long long)n;
                r.ctl->list_diag[2] = t;
            }
            return ~0ull;
        }
        __nanosleep(512);
        t = lr_load_sys(r.tail);
    }
    tail_seen = t;
    return pos;
}

// Warp-collective: every lane with `act` appends the record
// (pre[0 .. np-1], mid (if >= 0), x; tag).  pre is warp-shared.  Returns
// false once the listing is over.
__device__ __forceinline__ bool lr_emit(const ListRing& r, unsigned long long& tail_seen, const int* pre, int np,
                                        int mid, int x, int tag, bool act, int lane) {
    act = act && (r.tag_filter < 0 || tag == r.tag_filter);
    const unsigned bal = __ballot_sync(GPM_FULL_MASK, act);
    if (!bal) return true;
    unsigned long long pos = 0;
    if (lane == 0) pos = lr_reserve(r, __popc(bal), tail_seen);
    pos = __shfl_sync(GPM_FULL_MASK, pos, 0);
    if (pos == ~0ull) return false;
    if (act) {
        const unsigned long long q = pos + (unsigned)__popc(bal & gpm_lanemask_lt());
        int32_t* rec = r.rec + (size_t)(q % r.cap) * r.stride;
        int o = 1;
        for (int i = 0; i < np; i++) rec[o++] = pre[i];
        if (mid >= 0) rec[o++] = mid;
        rec[o++] = x;
        rec[o] = tag;
        lr_publish(rec, (int32_t)(uint32_t)(q + 1));
    }
    return true;
}

}  // namespace gpm
