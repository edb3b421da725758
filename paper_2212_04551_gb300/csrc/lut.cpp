// lut.cpp -- the canonical-relabelling dictionary (hot-path row A12), host side.
//
// Section 4.3.4 (Fig. 4) maps the edge bitmap of a k-vertex traversal to a
// canonical representative in two steps: traversal code -> (non-contiguous)
// representative -> contiguous pattern id.  The paper ships that dictionary as
// an input file; here it is built in-process, once per k, by an orbit sweep:
//
//   1. scan every full code f of a labelled k-vertex graph in increasing
//      order (bit i(i-1)/2 + j <=> edge {j, i}, j < i);
//   2. an f not yet assigned is the smallest member of its isomorphism
//      class: give it a new class and stamp every relabelling of f with it;
//   3. keep the connected classes (only connected traversals exist), and
//      number them by (edge count, smallest code) -- the contiguous ids;
//   4. traversal code t (the paper's C(k,2)-1 bit layout, v0-v1 implicit,
//      then v2's edges to v0..v1, v3's edges to v0..v2, ...) equals full
//      code (t << 1) | 1; LUT[t] = id of that code's class, or 0xFFFF when
//      some v_i (i >= 2) has no earlier neighbour (not a traversal).
//
// Cost: (#classes) x k! relabellings -- 1044 x 5040 for k = 7, 12,346 x
// 40,320 for k = 8 (about ten seconds, once per process; the class of every
// one of the 2^28 full codes is held as 16 bits: 512 MB while it runs, and
// the k = 8 table itself is 2^27 uint16 = 256 MB).
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "common.cuh"

namespace gpm {

static int pairs(int k) { return k * (k - 1) / 2; }
static int bit_of(int j, int i) { return i * (i - 1) / 2 + j; }  // j < i

static bool connected_code(int k, uint64_t f) {
    if (k <= 1) return true;
    uint32_t reach = 1;
    for (int round = 0; round < k; round++) {
        uint32_t next = reach;
        for (int i = 1; i < k; i++)
            for (int j = 0; j < i; j++)
                if ((f >> bit_of(j, i)) & 1) {
                    if ((reach >> i) & 1) next |= 1u << j;
                    if ((reach >> j) & 1) next |= 1u << i;
                }
        if (next == reach) break;
        reach = next;
    }
    return reach == (1u << k) - 1;
}

static std::unique_ptr<PatternTable> build_table(int k) {
    auto t = std::make_unique<PatternTable>();
    t->k = k;
    const int nb = pairs(k);
    if (k == 1) {
        t->num_patterns = 1;
        t->pattern_code = {0};
        t->lut = {0};
        return t;
    }
    const uint64_t nfull = 1ull << nb;
    // image bit of each bit under each relabelling
    std::vector<int> perm(k);
    std::iota(perm.begin(), perm.end(), 0);
    std::vector<std::vector<uint8_t>> images;
    do {
        std::vector<uint8_t> img(nb);
        for (int i = 1; i < k; i++)
            for (int j = 0; j < i; j++) {
                int a = perm[j], b = perm[i];
                img[bit_of(j, i)] = (uint8_t)bit_of(std::min(a, b), std::max(a, b));
            }
        images.push_back(std::move(img));
    } while (std::next_permutation(perm.begin(), perm.end()));

    // class ids fit in 16 bits: at most 12,346 classes for k <= 8
    const uint16_t UNSET = 0xffffu;
    std::vector<uint16_t> cls(nfull, UNSET);
    std::vector<uint64_t> cls_code;
    for (uint64_t f = 0; f < nfull; f++) {
        if (cls[f] != UNSET) continue;
        const uint16_t id = (uint16_t)cls_code.size();
        cls_code.push_back(f);
        for (const auto& img : images) {
            uint64_t r = 0;
            for (uint64_t b = f; b; b &= b - 1) r |= 1ull << img[__builtin_ctzll(b)];
            cls[r] = id;
        }
    }
    // connected classes, ordered by (edges, smallest code)
    std::vector<uint32_t> conn;
    for (uint32_t c = 0; c < cls_code.size(); c++)
        if (connected_code(k, cls_code[c])) conn.push_back(c);
    std::sort(conn.begin(), conn.end(), [&](uint32_t a, uint32_t b) {
        int ea = __builtin_popcountll(cls_code[a]), eb = __builtin_popcountll(cls_code[b]);
        if (ea != eb) return ea < eb;
        return cls_code[a] < cls_code[b];
    });
    std::vector<uint32_t> cls_to_pid(cls_code.size(), 0xffffu);
    t->pattern_code.resize(conn.size());
    for (size_t p = 0; p < conn.size(); p++) {
        cls_to_pid[conn[p]] = (uint32_t)p;
        t->pattern_code[p] = cls_code[conn[p]];
    }
    t->num_patterns = (int64_t)conn.size();

    const uint64_t ntrav = 1ull << (nb - 1);
    t->lut.assign(ntrav, 0xffffu);
    for (uint64_t tc = 0; tc < ntrav; tc++) {
        // every v_i (i >= 2) needs an earlier neighbour; v1 ~ v0 is implicit
        bool ok = true;
        for (int i = 2; i < k && ok; i++) {
            const int off = i * (i - 1) / 2 - 1;
            if (((tc >> off) & ((1ull << i) - 1)) == 0) ok = false;
        }
        if (!ok) continue;
        const uint64_t f = (tc << 1) | 1ull;
        t->lut[tc] = (uint16_t)cls_to_pid[cls[f]];
    }
    return t;
}

static std::mutex g_table_mu;
static std::map<int, std::unique_ptr<PatternTable>> g_tables;

const PatternTable& pattern_table(int k) {
    std::lock_guard<std::mutex> lock(g_table_mu);
    auto it = g_tables.find(k);
    if (it != g_tables.end()) return *it->second;
    if (k < 1 || k > GPM_MOTIF_MAX_K) fail(GPM_ENOTIMPL, "motif size k=" + std::to_string(k) + " not built");
    auto t = build_table(k);
    const PatternTable& ref = *t;
    g_tables[k] = std::move(t);
    return ref;
}

static std::mutex g_dlut_mu;
static std::map<std::pair<int, int>, uint16_t*> g_dluts;  // (device, k) -> device table (process lifetime)

const uint16_t* device_lut(int k) {
    const PatternTable& t = pattern_table(k);
    int dev = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    std::lock_guard<std::mutex> lock(g_dlut_mu);
    auto key = std::make_pair(dev, k);
    auto it = g_dluts.find(key);
    if (it != g_dluts.end()) return it->second;
    uint16_t* d = nullptr;
    const size_t bytes = t.lut.size() * sizeof(uint16_t);
    cudaError_t e = cudaMalloc(&d, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(GPM_ENOMEM, "cudaMalloc for the pattern table failed");
    }
    check_cuda(cudaMemcpy(d, t.lut.data(), bytes, cudaMemcpyHostToDevice), "cudaMemcpy(pattern table)");
    g_dluts[key] = d;
    return d;
}

}  // namespace gpm
