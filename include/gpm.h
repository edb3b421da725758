/*
 * gpm.h -- C ABI of libgpm: exact subgraph enumeration on one GB300 (sm_103a).
 *
 * The library counts k-vertex subgraphs of an undirected graph by repeated
 * subgraph extension, the enumeration function E(G, tr, k) of the paper
 * (Eq. 1): a traversal tr grows by one vertex of its neighbourhood
 * N(tr) (Definition 1) until |tr| = k, and the output function A aggregates
 * it.  Two applications are exported (Section 4.4, Algorithm 4):
 *
 *   - k-clique counting: A counts traversals whose vertices are pairwise
 *     adjacent; aggregate_counter adds the number of valid last-level
 *     extensions (Section 4.3.4);
 *   - induced k-motif counting: A maps every connected induced k-vertex
 *     subgraph to its canonical representative (pattern) and counts it per
 *     pattern (aggregate_pattern, canonical relabelling by dictionary,
 *     Section 4.3.4, Fig. 4).
 *
 * Conventions shared by every call:
 *   - Graphs are undirected int32 CSR: indptr[n+1] (indptr[0] = 0,
 *     non-decreasing), indices[indptr[n]]; each adjacency list sorted strictly
 *     ascending, symmetric, no self-loops, no duplicates, ids in [0, n).
 *   - Counts are exact uint64.  A true count >= 2^64 makes the call return
 *     GPM_EOVERFLOW (never a wrapped value).
 *   - Results are written only when the call returns GPM_OK.
 *   - Host-result calls synchronise the graph's stream before returning.
 *   - The library owns every device buffer it allocates; caller buffers are
 *     only read (inputs) or written (outputs) during the call.
 *   - No call aborts, traps or exits the process; failures are status codes
 *     with a message from gpm_last_error().
 *   - Calls on one gpm_graph must not run concurrently from several host
 *     threads (the graph caches per-call device buffers).
 */
#ifndef GPM_H
#define GPM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GPM_OK = 0,
    GPM_EINVAL = 1,     /* bad argument or malformed graph                    */
    GPM_ENOMEM = 2,     /* host or device allocation failed                   */
    GPM_ECUDA = 3,      /* a CUDA runtime call failed                         */
    GPM_ETIMEOUT = 4,   /* a bounded device wait ran out (work donation)      */
    GPM_EOVERFLOW = 5,  /* a count does not fit in uint64                     */
    GPM_ENOTIMPL = 6    /* the requested k or mode is not built               */
} gpm_status;

typedef struct gpm_graph gpm_graph; /* opaque, library-owned */

/* gpm_graph_create flags */
#define GPM_DEVICE_PTRS   1u  /* indptr/indices are device pointers (e.g. torch CUDA tensors) */
#define GPM_SKIP_VALIDATE 2u  /* trust the caller: skip the CSR checks                      */

/* applications (gpm_count_roots, gpm_sched_*) */
#define GPM_APP_CLIQUE 0
#define GPM_APP_MOTIF  1

/* limits */
#define GPM_CLIQUE_MAX_K 16
#define GPM_MOTIF_MAX_K  8

/*
 * Copy an undirected CSR graph (Section 2; adjacency lists contiguous, as in
 * Section 4.3.1) onto the device of the current CUDA context.
 *   indptr  : n+1 int32 offsets; indices: indptr[n] int32 neighbour ids.
 *             Host pointers unless flags has GPM_DEVICE_PTRS.  Both arrays
 *             are COPIED; the caller keeps ownership and may free them when
 *             the call returns.
 *   n       : number of vertices, 0 <= n < 2^31.
 *   stream  : cudaStream_t every later call on this graph runs on (NULL =
 *             the legacy default stream).
 *   out     : receives the new graph.
 * Unless GPM_SKIP_VALIDATE, the CSR is checked on the device (sorted strictly
 * ascending, ids in range, no self-loop, symmetric); a violation returns
 * GPM_EINVAL.  Errors: GPM_EINVAL, GPM_ENOMEM, GPM_ECUDA.
 */
gpm_status gpm_graph_create(const int32_t* indptr, const int32_t* indices, int32_t n,
                            uint32_t flags, void* stream, gpm_graph** out);

/* Free a graph and every device buffer it owns.  NULL is allowed. */
void gpm_graph_destroy(gpm_graph* g);

/* n and the number of undirected edges m (= indptr[n] / 2). */
gpm_status gpm_graph_info(const gpm_graph* g, int32_t* n, int64_t* m, int32_t* max_degree);

/*
 * Number of k-cliques (Algorithm 4, clique counting; Section 4.4), 1 <= k <=
 * GPM_CLIQUE_MAX_K.  k = 1 gives n and k = 2 gives m.  The enumeration runs on
 * the degree-ordered orientation of G (each clique is reached once, from its
 * lowest-(degree, id) vertex), which plays the role of the paper's "lower"
 * filter.  Roots with at most 1,024 out-neighbours are counted on bitmaps of
 * their out-neighbourhood in shared memory; roots above that, in the same
 * call, by sorted-list intersection (the paper's extension arrays) with
 * per-warp lists in device memory.  out_count: host pointer to one uint64.
 * Errors: GPM_EINVAL, GPM_ENOMEM, GPM_ECUDA, GPM_ETIMEOUT, GPM_EOVERFLOW.
 */
gpm_status gpm_clique_count(gpm_graph* g, int k, uint64_t* out_count);

/*
 * Numbers of j-cliques for every j in [k_lo, k_hi] from ONE enumeration to
 * depth k_hi (every level of the search is itself a clique of that size).
 * counts: host array of k_hi - k_lo + 1 uint64.  3 <= k_lo <= k_hi <=
 * GPM_CLIQUE_MAX_K.  Errors as gpm_clique_count.
 */
gpm_status gpm_clique_count_range(gpm_graph* g, int k_lo, int k_hi, uint64_t* counts);

/*
 * Per-pattern counts of connected induced k-vertex subgraphs (Algorithm 4,
 * motif counting; aggregate_pattern, Section 4.3.4), 1 <= k <=
 * GPM_MOTIF_MAX_K.  counts: host array of counts_len uint64, counts_len >=
 * gpm_motif_num_patterns(k); entry p is the number of subgraphs whose
 * canonical representative is pattern id p (see gpm_motif_pattern).  For
 * k <= 7 the last two levels are counted by entry class (motif_agg_min);
 * k = 8 counts leaf by leaf into global pattern counters.
 * Errors: GPM_EINVAL (also counts_len too small), GPM_ENOMEM, GPM_ECUDA,
 * GPM_ETIMEOUT, GPM_EOVERFLOW.
 */
gpm_status gpm_motif_count(gpm_graph* g, int k, uint64_t* counts, int64_t counts_len);

/*
 * Number of connected k-vertex patterns (pattern ids are 0 .. *out - 1):
 * 1, 1, 2, 6, 21, 112, 853, 11117 for k = 1 .. 8.  The k = 8 dictionary is
 * built on first use (about ten seconds of host time, 512 MB of host memory
 * while it runs; the table is 256 MB, on the host and on each device).
 */
gpm_status gpm_motif_num_patterns(int k, int64_t* out);

/*
 * Full adjacency code of pattern `id` at size k: bit i(i-1)/2 + j is set iff
 * vertices j < i of the pattern are adjacent, and the code is the smallest
 * over all relabellings (the canonical representative, Section 3).  Pattern
 * ids are ordered by (number of edges, canonical code), ascending -- the
 * contiguous identifiers of Section 4.3.4 ("(b) -> (c)" in Fig. 4).
 */
gpm_status gpm_motif_pattern(int k, int64_t id, uint64_t* adj_code);

/*
 * Exact partial counts over a set of roots: only the subgraphs whose root is
 * listed.  The root of a clique is its lowest-(degree, id) vertex; the root
 * of a connected motif subgraph is its smallest vertex id.  Disjoint root
 * sets add up to the full count.
 *   app      : GPM_APP_CLIQUE or GPM_APP_MOTIF.
 *   roots    : host array of n_roots distinct vertex ids (NULL: all
 *              vertices, n_roots ignored).
 *   counts   : host array of counts_len uint64 (1 for cliques, the number
 *              of patterns for motifs).
 *   per_root : nullable host array of n_roots uint64: each root's total
 *              (for motifs, summed over patterns).
 * Errors as gpm_clique_count / gpm_motif_count.
 */
gpm_status gpm_count_roots(gpm_graph* g, int app, int k, const int32_t* roots, int64_t n_roots,
                           uint64_t* counts, int64_t counts_len, uint64_t* per_root);

/*
 * Scheduling knobs.  None of them can change a count; they change only how
 * work is split and ordered (Section 4.3.5 replaced by in-kernel donation).
 */
typedef struct {
    int32_t warps_per_block;   /* 1, 2, 4, 8 or 16 (0 = automatic: the most resident   */
                               /* warps per SM for cliques; 4 for motifs, whose grid, */
                               /* when the marks live in HBM, is sized so that every  */
                               /* warp's marks fit in L2)                              */
    int32_t blocks_per_sm;     /* resident blocks per SM (0 = automatic)               */
    int32_t donate_min;        /* split a level only if >= this many siblings remain  */
    int32_t order;             /* GPM_ORDER_* root order of the plain scheduler         */
    int32_t max_idle_ms;       /* bounded wait: an idle warp gives up after this long  */
                               /* without any progress anywhere (GPM_ETIMEOUT)         */
    int32_t donate;            /* 0 disables work donation                             */
    int32_t donate_after_us;   /* a unit is split only after it has run this long      */
    int32_t clique_tail;       /* clique levels finished lane-parallel: 2 or 3 (0: 3 for k >= 7, else 2) */
    int32_t clique_compact;    /* two-level clique tail on the node's members (rows of ceil(|C|/32)   */
                               /* words instead of ceil(d/32)): 0 never, 1 when |C| >= 48 and the    */
                               /* rows get shorter, 2 whenever they get shorter                     */
    int32_t motif_agg_min;     /* motif: a node one level above the leaves whose extension array     */
                               /* has at least this many entries left counts its last two levels by  */
                               /* entry class instead of leaf by leaf (0: never)                     */
    int32_t clique_compact3;   /* three-level clique tail on the node's members whenever that        */
                               /* shortens the rows: 0 never, 1 (default), 2 also with the pairs of  */
                               /* nodes of at most 64 members taken one at a time by the whole warp  */
    int32_t batch_split;       /* batched launch: roots heavier than 1/4096 of the total estimated   */
                               /* work are cut into this many units over ranges of their children    */
                               /* before the launch (0 or 1: none; at most 64)                       */
    int32_t clique_cpl;        /* three-level clique tail (k >= 7): the k-cliques below each child of */
                               /* a tail node are counted as the triangles of its candidate graph,    */
                               /* sum_t C(a_t, 2) minus the open wedges found from the non-edges,     */
                               /* instead of one AND + POPC per (k-1)-clique: 0 never, 1 always,      */
                               /* 2..100 for tail nodes whose members are at least this percent       */
                               /* pairwise adjacent (default 85)                                      */
} gpm_config;

#define GPM_ORDER_ID          0  /* roots in id order                               */
#define GPM_ORDER_DEGREE_DESC 1  /* heaviest (largest out-/degree) roots first       */
#define GPM_ORDER_CUSTOM      2  /* order set by gpm_sched_set_order                 */

gpm_status gpm_get_config(const gpm_graph* g, gpm_config* out);
gpm_status gpm_set_config(gpm_graph* g, const gpm_config* cfg);

/* Statistics of the last counting call on g (device-measured). */
typedef struct {
    double   kernel_ms;        /* enumeration kernel time (CUDA events)          */
    uint64_t units_done;       /* work units (roots + donated units) finished     */
    uint64_t donations;        /* units handed to idle warps (work donation)      */
    uint64_t idle_polls;       /* spins of idle warps waiting for a hand-off      */
    int32_t  grid_blocks;      /* persistent grid size                            */
    int32_t  warps_per_block;
    uint64_t word_ops;         /* clique: 32-bit candidate-word AND+POPC operations; */
                               /* motif: adjacency entries scanned                   */
    int32_t  kernel_launches;  /* kernels the call launched (enumeration path)    */
    uint64_t busy_warp_ns;     /* sum over the grid's warps of the time spent      */
                               /* inside work units (%globaltimer); 1 - busy /     */
                               /* (warps x kernel time) is the idle warp fraction  */
} gpm_stats;

gpm_status gpm_get_stats(const gpm_graph* g, gpm_stats* out);

/*
 * The paper's load balancing, for comparison with the in-kernel hand-off
 * (Section 4.3.5: the CPU watches the share of active warps, stops the
 * kernel when it falls below a threshold -- 40 % for cliques and 10 % for
 * motifs in the paper's experiments -- redistributes the unfinished work and
 * relaunches).  Here: the kernel runs without donation over every root; the
 * host polls the number of warps holding work; once every root has been
 * handed out and fewer than threshold x warps still hold work, it raises a
 * stop flag, every busy warp writes its remaining work (one unit per level
 * with children left) to a spill buffer and leaves, and the host relaunches
 * over the spilled units, until a launch spills nothing.
 *   app, k    : GPM_APP_CLIQUE (3 <= k <= 16) or GPM_APP_MOTIF (3 <= k <= 8).
 *   threshold : 0 <= threshold <= 1 (0: never stop, the plain launch without
 *               donation).
 *   counts    : as gpm_count_roots over every root.
 *   stats     : nullable; launches, units spilled, summed kernel time and the
 *               whole loop's host time.
 * Same counts as gpm_clique_count / gpm_motif_count.  Errors as those.
 */
/*
 * The paper's DM_DFS baseline (Section 4.2; Table optimizations-performance),
 * for comparison only: k-cliques (2 <= k <= 16) counted by one thread per
 * root, depth first, with sorted candidate lists intersected by merges in a
 * per-thread stack in device memory -- no warp cooperation, no bitmaps, no
 * load balancing.  Same count as gpm_clique_count; its kernel time is in
 * gpm_get_stats.  The stack takes (k-1) x (largest out-degree) ints per
 * thread for 152 x 8 x 256 threads.  Errors as gpm_clique_count.
 */
gpm_status gpm_clique_count_dfs(gpm_graph* g, int k, uint64_t* out_count);

/*
 * Subgraph listing with an asynchronous host consumer (aggregate_store,
 * Section 4.3.4: found k-vertex subgraphs go to a buffer that the CPU
 * consumes while the GPU keeps producing).  The kernel appends one record
 * per subgraph to a ring in mapped (pinned) host memory; the calling thread
 * takes the records in order while the kernel runs and hands them to
 * `consumer` in batches.
 *   app, k       : GPM_APP_CLIQUE, 3 <= k <= 16: every k-clique; or
 *                  GPM_APP_MOTIF, 3 <= k <= 8: every connected induced
 *                  k-vertex subgraph.
 *   pattern      : -1 for every subgraph; for motifs, a pattern id (see
 *                  gpm_motif_pattern) to list only that pattern's subgraphs
 *                  (subgraph querying).  Cliques take -1 only.
 *   ring_records : ring capacity in records, >= 64 (0: 65,536).
 *   consumer     : called on the calling thread with `count` records of
 *                  `record_words` = k + 1 int32 each: the k vertex ids
 *                  (cliques: in (degree, id) order from the clique's first
 *                  vertex; motifs: in traversal order from the smallest id),
 *                  then the pattern id (motifs) or -1 (cliques).  The array
 *                  is valid during the call only.  Return 0 to go on, any
 *                  other value to stop the listing (the call then returns
 *                  GPM_OK with fewer records than exist).
 *   user         : passed through to consumer.
 *   delivered    : nullable; records handed to consumer.
 * Every subgraph is listed exactly once (the same sets gpm_clique_count /
 * gpm_motif_count count), in no particular order.  Kernel time is in
 * gpm_get_stats.  If the ring stays full for longer than max_idle_ms
 * (the consumer does not keep up), the device gives up: GPM_ETIMEOUT, with
 * the records delivered so far.  The consumer runs while the kernel runs
 * and the kernel waits for it, so the consumer must not wait for the
 * device: a call that synchronises with it (cudaFree, cudaDeviceSynchronize,
 * a synchronous copy, gpm_graph_destroy, a count on the same stream) blocks
 * until the listing kernel ends, which happens only when its wait for ring
 * space runs out (GPM_ETIMEOUT after max_idle_ms).
 * Errors: GPM_EINVAL, GPM_ENOMEM, GPM_ECUDA, GPM_ETIMEOUT.
 */
typedef int32_t (*gpm_list_consumer)(const int32_t* records, int64_t count, int32_t record_words, void* user);
gpm_status gpm_list(gpm_graph* g, int app, int k, int32_t pattern, int64_t ring_records, gpm_list_consumer consumer,
                    void* user, uint64_t* delivered);

typedef struct {
    int32_t launches;
    int32_t pad;
    int64_t spilled_units;
    double kernel_ms;
    double wall_ms;
} gpm_monitor_stats;

gpm_status gpm_count_monitored(gpm_graph* g, int app, int k, double threshold, uint64_t* counts, int64_t counts_len,
                               gpm_monitor_stats* stats);

/* ------------------------------------------------------------------------
 * Learned scheduler (not in the paper; changes only the order and splitting
 * of work, never a count).  A small MLP (8 -> 64 -> 64 -> 1, ReLU, BF16
 * weights, FP32 accumulation) predicts each root's enumeration-subtree size
 * from 8 per-root features; roots are then run heaviest-predicted first and
 * the heaviest are pre-split into several work units.
 * ---------------------------------------------------------------------- */

#define GPM_MLP_PARAMS 4801   /* W1 64x8, b1 64, W2 64x64, b2 64, w3 64, b3 1 (row-major, this order) */

/*
 * Per-vertex features for subgraph size k, FP32 [n][8]: log1p of degree, of
 * oriented out-degree, of the number of higher-id neighbours, of the
 * neighbour-degree sum (2-hop degree sum), of the higher-id neighbour-degree
 * sum, of the triangles rooted at v (lowest (degree, id) vertex), of the core
 * number of v (k-core decomposition); and k / 8, so that one network can
 * predict sizes for several k.  1 <= k <= GPM_CLIQUE_MAX_K.
 * out: n*8 floats, a device pointer if flags has GPM_DEVICE_PTRS, else host.
 */
gpm_status gpm_root_features(gpm_graph* g, int k, float* out, uint32_t flags);

/*
 * y[i] = MLP(x[i]) for i < n.  w_bf16: GPM_MLP_PARAMS BF16 values (as
 * uint16); x: n*8 FP32; y: n FP32.  All device pointers; stream: cudaStream_t
 * (NULL = legacy default).  Asynchronous on the stream.
 */
gpm_status gpm_mlp_forward(const uint16_t* w_bf16, const float* x, int64_t n, float* y, void* stream);

/*
 * grad[GPM_MLP_PARAMS] = gradient of mean_i (MLP(x[i]) - t[i])^2 with respect
 * to the (BF16) parameters, and loss[0] = that mean.  Device pointers,
 * overwritten; asynchronous on the stream.
 */
gpm_status gpm_mlp_grad(const uint16_t* w_bf16, const float* x, const float* t, int64_t n, float* grad,
                        float* loss, void* stream);

/*
 * One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected; step >= 1)
 * on FP32 master weights with FP32 moments m, v, then w_bf16 = BF16(master)
 * rounded to nearest-even.  Device pointers; asynchronous on the stream.
 */
gpm_status gpm_mlp_adam(float* master, float* m, float* v, const float* grad, int32_t step, float lr,
                        uint16_t* w_bf16, void* stream);

/*
 * Build the schedule of app over a root set: roots (host, n_roots distinct
 * vertex ids; NULL = every vertex) are ordered by score descending (scores:
 * device pointer to one FP32 per VERTEX; NULL = the plain order: degree for
 * motifs, oriented out-degree for cliques), and the first split_roots of that
 * order are each pre-split into split_chunks units over ranges of their
 * children cut to balance estimated work (a root's child at position c of L
 * has about L - c candidates after it, so the work from c on is taken to
 * grow like (L - c)^(k-1)).  Replaces any earlier schedule of that app.
 */
gpm_status gpm_sched_from_scores(gpm_graph* g, int app, const float* scores, const int32_t* roots,
                                 int64_t n_roots, int32_t split_roots, int32_t split_chunks);

/*
 * As gpm_sched_from_scores, with each root pre-split in proportion to its
 * predicted size: scores (required) are read as log1p of each root's
 * subtree size, the fair share is (sum of the listed roots' sizes) /
 * target_units, and a root becomes ceil(size / share) units (1 .. max_chunks,
 * at most 65,536 units in all), cut as above.  target_units is typically a
 * few times the warps of the launch.
 */
gpm_status gpm_sched_balanced(gpm_graph* g, int app, const float* scores, const int32_t* roots, int64_t n_roots,
                              int64_t target_units, int32_t max_chunks);

/*
 * Exact counts over the scheduled root set of app (as gpm_count_roots, but
 * run in the schedule's order and splitting).  per_root (nullable) is indexed
 * like the roots array given to gpm_sched_from_scores.
 */
gpm_status gpm_count_scheduled(gpm_graph* g, int app, int k, uint64_t* counts, int64_t counts_len,
                               uint64_t* per_root);

/* ------------------------------------------------------------------------
 * Batched persistent launch (not in the paper).  Many small graphs packed as
 * one disjoint union are counted by ONE persistent kernel over (task, root)
 * units, captured once in a CUDA graph and replayed on every call; results
 * are per graph.
 * ---------------------------------------------------------------------- */

typedef struct gpm_batch gpm_batch; /* opaque, library-owned */

/*
 * graph_off: n_graphs+1 vertex offsets (graph g owns vertices graph_off[g] ..
 * graph_off[g+1]-1); indptr / indices: the packed CSR over all
 * graph_off[n_graphs] vertices with GLOBAL vertex ids (the conventions of
 * gpm_graph_create; no edge may join two graphs -- checked unless
 * GPM_SKIP_VALIDATE).  Host pointers unless flags has GPM_DEVICE_PTRS; all
 * arrays are copied.  stream: cudaStream_t to run on (NULL: the library
 * creates a private stream, because the legacy default stream cannot be
 * captured).  Errors: GPM_EINVAL, GPM_ENOMEM, GPM_ECUDA.
 */
gpm_status gpm_batch_create(const int32_t* graph_off, const int32_t* indptr, const int32_t* indices,
                            int32_t n_graphs, uint32_t flags, void* stream, gpm_batch** out);

/* Free a batch, its captured launches and device buffers.  NULL is allowed. */
void gpm_batch_destroy(gpm_batch* b);

/*
 * Per-graph counts in one launch: clique_counts[g] = number of clique_k-
 * cliques of graph g, motif_counts[g * P + p] = count of pattern p of size
 * motif_k in graph g (P = gpm_motif_num_patterns(motif_k)).  A k of 0 skips
 * that task (its array may then be NULL); otherwise 3 <= clique_k <= 16,
 * 3 <= motif_k <= 7.  The first call with a given (clique_k, motif_k) and
 * launch shape captures a CUDA graph; later calls replay it.
 * Errors: GPM_EINVAL, GPM_ENOMEM, GPM_ECUDA, GPM_EOVERFLOW, GPM_ENOTIMPL (a
 * graph too large for the shared-memory state, or, with clique_k > 0, an
 * oriented out-degree above 1,024: the batched kernel has no list path).
 */
gpm_status gpm_batch_count(gpm_batch* b, int clique_k, int motif_k, uint64_t* clique_counts, uint64_t* motif_counts);

/*
 * Autotune the launch for (clique_k, motif_k), each candidate timed as the
 * median of `reps` replays, in three stages: (1) warps per block {2, 4, 8,
 * 16} x resident blocks per SM {max, 1, 2} x unit order {tasks grouped,
 * merged}; (2) with the best of those, the motif tail's class-counting
 * threshold motif_agg_min {0, 4, 16, 64}; (3) the split of heavy roots
 * batch_split {1, 4, 16}.  The per-warp stack is not a knob: its size is
 * fixed by the largest degree (a smaller one could not hold the extension
 * arrays).  The fastest is kept for this batch (and cached in-process for
 * batches of the same shape).  best (nullable) receives it; best_ms
 * (nullable) its median time, or -1 when it came from the cache.
 */
gpm_status gpm_batch_autotune(gpm_batch* b, int clique_k, int motif_k, int reps, gpm_config* best,
                              double* best_ms);

gpm_status gpm_batch_set_config(gpm_batch* b, const gpm_config* cfg);
gpm_status gpm_batch_get_stats(const gpm_batch* b, gpm_stats* out);

/*
 * Allocation-free motif counting.  The paper has no counterpart: this entry
 * point exists for callers that cannot let a library allocate device memory
 * -- host applications that own every device byte through their own pool or
 * allocator, and real-time or embedded hosts with a fixed device-memory
 * budget where a cudaMalloc during a call is not allowed.
 *
 * Same result as gpm_motif_count on the same graph (counts[p] = number of
 * connected induced k-vertex subgraphs of pattern id p), computed by the same
 * motif kernel with work donation off.  The call allocates nothing: it calls
 * no cudaMalloc or cudaFree and no allocating library routine; its scratch
 * (control block, counters, validation flags, root list, pattern table) is
 * one file-scope device array of 2,139,392 bytes that every device loading
 * the library holds until the process exits.
 *
 *   indptr, indices : DEVICE pointers to the undirected CSR (conventions of
 *                     gpm_graph_create; checked on the device); not copied.
 *   n               : 0 <= n <= 8192 vertices; the graph must also fit the
 *                     kernel's shared-memory state (n bytes of marks plus
 *                     sum over l <= k-2 of l * max_degree ints, at most 12 KB
 *                     per warp).  Larger graphs are rejected with GPM_EINVAL
 *                     and a message naming the limit.
 *   k               : 3 <= k <= 7.
 *   counts          : HOST array of counts_len uint64 (>= number of patterns).
 *   stream          : cudaStream_t to run on (NULL = legacy default stream);
 *                     the call synchronises it before returning.
 *
 * The first call on a device looks up the device address of the scratch
 * array (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  The address is kept for the life of the
 * process: after cudaDeviceReset (or any reset of the device's primary
 * context) this entry point must not be called again in that process.  The host-side pattern table of each k is
 * built once per process in host memory.  Every call on a device shares the
 * one scratch array, which keeps the last call's contents (each call clears
 * what must start at zero): calls that overlap on the GPU -- on different
 * streams or from different host threads -- race and must not be made.
 * Errors: GPM_EINVAL, GPM_ECUDA, GPM_EOVERFLOW.
 */
gpm_status gpm_motif_count_noalloc(const int32_t* indptr, const int32_t* indices, int32_t n, int k,
                                   uint64_t* counts, int64_t counts_len, void* stream);

/*
 * Self-test of the overflow contract (the paper is silent on overflow; the
 * library's reading is that a true count >= 2^64 is an error, never a
 * wrapped value).  Sums n uint64 values (host array) on the device through
 * the counting kernels' own carry-checked reduction path -- lane-private
 * adds over a grid-stride loop, warp sums, a per-block shared counter and a
 * global counter -- with `blocks` x `threads` threads (threads a multiple of
 * 32), so a caller can place large values in one lane, one warp, one block
 * or several blocks.  *out = the exact sum when it fits; otherwise the call
 * returns GPM_EOVERFLOW.  Allocates a temporary device buffer.
 * Errors: GPM_EINVAL, GPM_ENOMEM, GPM_ECUDA, GPM_EOVERFLOW.
 */
gpm_status gpm_selftest_sum(const uint64_t* values, int64_t n, int32_t blocks, int32_t threads, uint64_t* out);

/*
 * L2 read bandwidth of the current device in GB/s (not in the paper: the
 * denominator of the motif kernel's roofline, whose adjacency lists and
 * per-warp marks live in L2).  A buffer of `bytes` (1 MB .. 96 MB, inside
 * L2) is read `reps` times after a warm pass: mode 0 with coalesced 16-byte
 * loads (bytes / time), mode 1 with one 4-byte load per pseudo-random
 * 32-byte sector (sectors x 32 B / time, the access shape of the marks).
 * Allocates a temporary buffer.  Errors: GPM_EINVAL, GPM_ENOMEM, GPM_ECUDA.
 */
gpm_status gpm_measure_l2(int64_t bytes, int32_t mode, int32_t reps, double* gbs);

/* Message of the last failed call on this host thread ("" if none). */
const char* gpm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GPM_H */
