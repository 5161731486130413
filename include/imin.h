/*
 * imin.h -- C ABI of the GB300 library for influence minimization by vertex blocking
 * (arXiv 2302.13529): the sampled-dominator-tree estimator (Alg. 2) and the greedy drivers
 * AdvancedGreedy (Alg. 3) and GreedyReplace (Alg. 4), computed by sm_103a CUDA kernels.
 *
 * Conventions shared by every entry point
 *   - Return value: IMIN_OK (0) on success, a negative IMIN_ERR_* code otherwise. On failure
 *     imin_last_error() returns a message for the calling thread. No exception crosses the ABI.
 *   - Pointers: every array argument may be host memory or device memory of the current CUDA
 *     device; the library detects which (cudaPointerGetAttributes). The caller owns and frees
 *     its arrays; the library copies what it keeps.
 *   - Streams: `stream` is a cudaStream_t (NULL = legacy default stream). Work is enqueued on
 *     it. Calls that return host-visible results (host output buffers, counts) synchronize the
 *     stream before returning; calls whose outputs are all device buffers may return before
 *     the kernels finish.
 *   - Graph: directed, CSR by source. Vertex ids are 0..n-1; edge e of vertex u lies in
 *     [row_ptr[u], row_ptr[u+1]). Each edge carries a uint32 threshold thr[e] that encodes its
 *     independent-cascade probability p(u,v) (Sec. 3.1) as thr = ceil(p * 2^32) - 1: edge e is
 *     live in a sample when the sample's 32-bit uniform word for e is <= thr[e], so it is live
 *     with probability (thr+1)/2^32; thr = 0xFFFFFFFF means p = 1. Edges with p = 0 must be
 *     left out. Multi-edges and self-loops are accepted (self-loops never matter).
 *   - Random stream (Def. 4 sampled graphs): the word for edge e in sample j of call `round`
 *     under the 64-bit key K is word (e & 3) of Philox4x32-10 (Salmon et al., SC'11) with
 *     counter (e >> 2, j, round, 0) and key (K mod 2^32, K >> 32). Results therefore depend
 *     only on (graph, seed set, blocked set, theta, key, round) -- never on launch shape,
 *     stream, batching or device.
 *   - Seeds (Sec. 4, multiple seeds merged into one super-seed): seeds must be distinct; edges
 *     into seeds are ignored; seeds have no counter and are never chosen as blockers.
 *   - Blockers (Def. 2): every in-edge of a blocked vertex has probability 0.
 *   - Counters: the decrease counter of vertex u is the exact integer sum over the theta
 *     samples of the size of u's dominator subtree (Alg. 2 without its division by theta;
 *     Thm. 6). Dividing by theta gives the paper's estimate of the expected-spread decrease.
 */
#ifndef IMIN_H
#define IMIN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IMIN_OK 0
#define IMIN_ERR_INVALID (-1)   /* an argument violates the contract above */
#define IMIN_ERR_CUDA (-2)      /* a CUDA runtime call failed */
#define IMIN_ERR_NOMEM (-3)     /* device memory could not be allocated */
#define IMIN_ERR_CAPACITY (-4)  /* a sampled cascade exceeded the largest kernel tier */
#define IMIN_ERR_INTERNAL (-5)  /* a kernel reported an internal consistency failure */
#define IMIN_ERR_TIMEOUT (-6)   /* imin_server_wait: the request is not finished yet */

/* Opaque handle: a directed graph resident in device memory. */
typedef struct imin_graph imin_graph;

/* Load a graph (Sec. 3: G = (V, E) with probabilities p(u,v)) into device memory.
 *   n        number of vertices, 0 < n < 2^31
 *   m        number of edges, 0 <= m < 2^31; m == row_ptr[n]
 *   row_ptr  int32[n+1], non-decreasing, row_ptr[0] == 0
 *   col      int32[m], targets in [0, n)
 *   thr      uint32[m], thresholds as described above
 *   stream   stream for the uploads (synchronized before return)
 *   out      receives the handle; free it with imin_free_graph
 * Errors: IMIN_ERR_INVALID for a malformed CSR, IMIN_ERR_NOMEM, IMIN_ERR_CUDA. */
int imin_load_graph(int32_t n, int64_t m, const int32_t* row_ptr, const int32_t* col,
                    const uint32_t* thr, void* stream, imin_graph** out);

/* Load a graph under the linear-threshold model, the standard triggering model (Sec. 4.5: every
 * vertex v draws a triggering set of in-neighbours, and only edges from that set stay). In the
 * LT model the set holds at most one in-neighbour: in-edge (u, v) with probability b(u, v), none
 * with probability 1 - sum_u b(u, v).
 *   weight   uint32[m]: weight[e] + 1 is edge e's share b(u, v) * 2^32 (the same fixed point as
 *            the IC thresholds, so weight = 0xFFFFFFFF is b = 1). The in-edges of each vertex v,
 *            in ascending edge id, take consecutive intervals [lo_e, lo_e + weight[e]] of
 *            [0, 2^32); sample j of call `round` under key K keeps edge e = (u, v) iff v's word --
 *            word (v & 3) of Philox4x32-10 with counter (v >> 2, j, round, 0x80000000) and the
 *            key of the IC stream -- lies in e's interval. The shares of one vertex's in-edges
 *            must sum to at most 2^32.
 *   Other arguments as for imin_load_graph. Every entry point below accepts the handle and
 *   computes the same quantities (Alg. 2 counters, AdvancedGreedy, GreedyReplace, batches,
 *   serving, spread) on the LT sampled graphs.
 * Errors: as imin_load_graph; IMIN_ERR_INVALID also when some vertex's shares exceed 2^32. */
int imin_load_graph_lt(int32_t n, int64_t m, const int32_t* row_ptr, const int32_t* col,
                       const uint32_t* weight, void* stream, imin_graph** out);

/* The propagation model of a loaded graph: 0 = independent cascade, 1 = linear threshold. */
int imin_graph_model(const imin_graph* g);

/* Release a graph handle and its device memory (after all work using it has finished).
 * NULL is accepted. */
int imin_free_graph(imin_graph* g);

/* Number of vertices and edges of a loaded graph (either pointer may be NULL). */
int imin_graph_info(const imin_graph* g, int32_t* n, int64_t* m);

/* DecreaseESComputation (Alg. 2) on G[V \ B].
 *   seeds, n_seeds      S: int32[n_seeds], distinct, 1 <= n_seeds <= n
 *   blocked, n_blocked  B: int32[n_blocked], distinct, disjoint from S (NULL if n_blocked == 0)
 *   theta               number of sampled graphs, >= 1
 *   key, round          select the random stream (see above); `round` is the 0-based index of
 *                       this call within a greedy run
 *   out_delta           uint64[n]: out_delta[u] = sum over the theta samples of the size of u's
 *                       subtree in the sample's dominator tree rooted at the super-seed
 *                       (Thm. 6: the number of reached vertices whose every path from S passes
 *                       through u); 0 for seeds, blocked and unreached vertices.
 * Errors: IMIN_ERR_INVALID, IMIN_ERR_NOMEM, IMIN_ERR_CUDA, IMIN_ERR_CAPACITY. */
int imin_estimate_decrease(const imin_graph* g, const int32_t* seeds, int32_t n_seeds,
                           const int32_t* blocked, int32_t n_blocked, uint32_t theta,
                           uint64_t key, uint32_t round, uint64_t* out_delta, void* stream);

/* Expected spread E(S, G[V \ B]) by simulation (Def. 3; the paper evaluates the spread of every
 * blocker set it reports this way): out_sum = the sum over theta sampled graphs (sample j of call
 * `round` under `key`, the same stream as Alg. 2) of the number of vertices reachable from S,
 * seeds included. The estimate is out_sum / theta. Blocked vertices are never reached.
 *   seeds, blocked, theta, key, round   as for imin_estimate_decrease
 *   out_sum   host uint64: the sum
 * Synchronizes `stream`. Errors: IMIN_ERR_INVALID, IMIN_ERR_NOMEM, IMIN_ERR_CUDA,
 * IMIN_ERR_CAPACITY (a cascade of more than 2^18 vertices on a graph with n > 2^18). */
int imin_estimate_spread(const imin_graph* g, const int32_t* seeds, int32_t n_seeds,
                         const int32_t* blocked, int32_t n_blocked, uint32_t theta, uint64_t key,
                         uint32_t round, uint64_t* out_sum, void* stream);

/* AdvancedGreedy (Alg. 3): b rounds; round i (0-based) runs Alg. 2 with round index i on
 * G[V \ B] and appends the candidate of V \ (S u B) with the largest counter (strict '>' in
 * ascending vertex id, so the smallest id wins ties). Stops early only when V \ (S u B) is
 * empty.
 *   b             budget, >= 0
 *   out_blockers  int32[b]: the blockers in selection order
 *   out_count     host int32: number of blockers written (min(b, n - n_seeds))
 * Synchronizes `stream`. Errors as for imin_estimate_decrease. */
int imin_advanced_greedy(const imin_graph* g, const int32_t* seeds, int32_t n_seeds,
                         int32_t b, uint32_t theta, uint64_t key, int32_t* out_blockers,
                         int32_t* out_count, void* stream);

/* GreedyReplace (Alg. 4).
 *   Phase 1: CB = out-neighbours of S that are not seeds; k = min(|CB|, b) rounds (round
 *            indices 0..k-1) each run Alg. 2 on G[V \ B] and move the best remaining CB vertex
 *            into B (appended).
 *   Phase 2: for positions i = k-1 down to 0 (reverse insertion order), with round indices
 *            continuing from k: u = B[i] is unblocked, Alg. 2 runs on G[V \ (B \ {u})], the
 *            best vertex x of V \ (S u B \ {u}) (u included) takes position i, and the phase
 *            ends as soon as x == u.
 *   out_blockers  int32[b]: B in list order; out_count: k.
 * Synchronizes `stream`. Errors as for imin_estimate_decrease. */
int imin_greedy_replace(const imin_graph* g, const int32_t* seeds, int32_t n_seeds, int32_t b,
                        uint32_t theta, uint64_t key, int32_t* out_blockers, int32_t* out_count,
                        void* stream);

/* ---- comparison algorithms of the evaluation (Sec. 5) ------------------------------------
 * The paper compares AdvancedGreedy and GreedyReplace with BaselineGreedy (Alg. 1, the earlier
 * greedy that scores every candidate by Monte-Carlo simulation), Exact (every blocker set of
 * size b scored by simulation), OutDegree and Rand. The simulated scores use the sampled graphs
 * of the stream above: every set scored in one call sees the same samples (common random
 * numbers), so a result depends only on its arguments. */

/* Simulated spread (Def. 3) of many blocker sets at once:
 *   out_sums[i] = sum over samples j in [0, theta) of call `round` of |R_j| (seeds included),
 *   with `blocked` and the set_size vertices sets[i * set_size .. (i+1) * set_size - 1] blocked.
 *   sets       int32[n_sets * set_size] (host or device): each set's vertices distinct, neither
 *              seeds nor in `blocked`; 0 <= set_size <= 64
 *   out_sums   uint64[n_sets] (host or device)
 * Synchronizes `stream`. Errors: as imin_estimate_spread. */
int imin_estimate_spread_sets(const imin_graph* g, const int32_t* seeds, int32_t n_seeds,
                              const int32_t* blocked, int32_t n_blocked, const int32_t* sets,
                              int32_t n_sets, int32_t set_size, uint32_t theta, uint64_t key,
                              uint32_t round, uint64_t* out_sums, void* stream);

/* BaselineGreedy (Alg. 1) with simulations of r sampled graphs: b rounds; in round i (0-based)
 * every candidate u of V \ (S u B) is scored by its simulated spread decrease
 * sum_j |R_j(B)| - |R_j(B u {u})| over samples j in [0, r) of call i, and the candidate with the
 * largest decrease is appended (strict '>' in ascending id). Each round simulates r sampled
 * graphs per candidate (O(n r m) work per round, as the paper states for Alg. 1). Stops early
 * only when no candidate is left. Outputs as imin_advanced_greedy. Synchronizes `stream`. */
int imin_baseline_greedy(const imin_graph* g, const int32_t* seeds, int32_t n_seeds, int32_t b,
                         uint32_t r, uint64_t key, int32_t* out_blockers, int32_t* out_count,
                         void* stream);

/* Exact (Sec. 5, "Algorithms"): every k-subset of V \ S (k = min(b, n - n_seeds)) scored by its
 * simulated spread over samples [0, r) of call 0; the first subset in lexicographic order with
 * the smallest spread is returned in ascending ids (out_count = k). At most 10^8 subsets
 * (IMIN_ERR_INVALID beyond). Synchronizes `stream`. */
int imin_exact_blockers(const imin_graph* g, const int32_t* seeds, int32_t n_seeds, int32_t b,
                        uint32_t r, uint64_t key, int32_t* out_blockers, int32_t* out_count,
                        void* stream);

/* OutDegree (Sec. 5): the min(b, n - n_seeds) non-seed vertices of largest out-degree, in that
 * order (the smaller id first among equal degrees). out_blockers: host int32[b]. */
int imin_out_degree_blockers(const imin_graph* g, const int32_t* seeds, int32_t n_seeds, int32_t b,
                             int32_t* out_blockers, int32_t* out_count);

/* Rand (Sec. 5): min(b, c) distinct non-seed vertices (c of them), by a partial Fisher-Yates
 * shuffle of the non-seeds in ascending id: draw t swaps position t with position
 * t + floor(w_t (c - t) / 2^32), w_t = word 0 of Philox4x32-10 at counter (t, 0, 0, 0xC0000000)
 * under `key`. out_blockers: host int32[b]. */
int imin_random_blockers(const imin_graph* g, const int32_t* seeds, int32_t n_seeds, int32_t b,
                         uint64_t key, int32_t* out_blockers, int32_t* out_count);

/* imin_estimate_decrease for callers that cannot allocate memory at call time (the paper has
 * no counterpart; this is a deployment variant).
 * Some callers must not allocate device memory when they call in: code whose device memory
 * belongs to another allocator with a fixed budget (a framework's caching allocator, a serving
 * process that sizes all of its memory at start-up), and latency-critical paths that cannot
 * afford cudaMalloc/cudaFree, which may synchronize the whole device. This entry point computes
 * exactly what imin_estimate_decrease computes (same arguments, same results) but calls no
 * cudaMalloc, cudaFree or other allocating routine: besides the caller's inputs and output, all
 * working memory comes from one static device array of 64 MiB inside the library, which every
 * GPU that loads the library holds until the process exits.
 * Limits (from that size): n <= 65,536 vertices and theta <= 131,072 samples per call; larger
 * requests fail with IMIN_ERR_INVALID. A sampled cascade that would need the library's
 * whole-graph fallback kernel (more non-tree live edges or BFS levels than the block-per-sample
 * kernel holds) fails the call with IMIN_ERR_CAPACITY. After any non-OK return the contents of
 * out_delta are undefined (a device out_delta may hold partial counters).
 * out_delta may be host memory or device memory of the graph's device (device memory of another
 * GPU is rejected with IMIN_ERR_INVALID).
 * The static array is shared by all calls on a device and keeps the last call's contents (each
 * call clears what must start at zero); calls that overlap on the GPU race on it, so order them
 * (one stream, or events). The first call on each device resolves the array's device address,
 * and the first call for each graph size plans the kernel launch.
 * The call is synchronous: it synchronizes `stream` before its kernel (to check the seed and
 * blocked ids) and after it (to read the kernel's status). */
int imin_estimate_decrease_noalloc(const imin_graph* g, const int32_t* seeds, int32_t n_seeds,
                                   const int32_t* blocked, int32_t n_blocked, uint32_t theta,
                                   uint64_t key, uint32_t round, uint64_t* out_delta,
                                   void* stream);

/* ---- batched drivers ----------------------------------------------------------------------
 * Many independent queries -- each with its own loaded graph, seed set, budget, theta and key --
 * advanced together: every greedy round is one launch over the sampled graphs of all queries
 * still active, load-balanced over the whole GPU, followed by one selection launch with a block
 * per query. Each query's result (blockers and count) is identical to what
 * imin_advanced_greedy / imin_greedy_replace return for it alone (same random streams, same
 * round numbering, same tie rule). Graphs must all live on the current device. Queries are
 * grouped by graph size so that each group's launch reserves only the memory its largest graph
 * needs. Each query takes the warp/block cutoff imin_autotune picks for its graph and seed-set
 * size class (tuned on `stream` on first use and cached, as for the single-query calls). */
typedef struct imin_query {
    const imin_graph* graph;  /* in: loaded graph */
    const int32_t* seeds;     /* in: n_seeds distinct vertex ids (host or device) */
    int32_t n_seeds;
    int32_t b;                /* in: budget */
    uint32_t theta;           /* in: sampled graphs per round */
    uint64_t key;             /* in: random-stream key */
    int32_t* out_blockers;    /* out: int32[b] (host or device), blockers in the driver's order */
    int32_t out_count;        /* out: number of blockers written */
} imin_query;

/* Alg. 3 for every query of `queries` (n_queries >= 0). Synchronizes `stream`. Errors as for
 * imin_advanced_greedy; on error no out_count is meaningful. */
int imin_batch_advanced_greedy(imin_query* queries, int32_t n_queries, void* stream);

/* Alg. 4 for every query of `queries`; GreedyReplace's phase-2 early stop is per query. */
int imin_batch_greedy_replace(imin_query* queries, int32_t n_queries, void* stream);

/* Pick the queue granularity of a batch (samples of one query per work item of a step; the
 * paper has no counterpart) and keep it for the life of the process under a fingerprint of the
 * batch (per query: its graph's fingerprint, seed-set size, budget and theta; and the driver).
 * After a warm-up call, times the first 3 steps of the batch for each candidate {4, 8, 16, 32,
 * 64}, twice, and keeps the fastest; later imin_batch_* calls on the same batch use it (others use
 * min(16, theta-dependent default)). The granularity never changes a result. The tuning calls
 * write into scratch buffers: the queries' outputs are not touched.
 *   driver     0 = AdvancedGreedy, 1 = GreedyReplace
 *   out_chunk  receives the chosen granularity
 * Synchronizes `stream`. Errors as for imin_batch_advanced_greedy. */
int imin_autotune_batch(imin_query* queries, int32_t n_queries, int32_t driver, void* stream,
                        int32_t* out_chunk);

/* ---- serving: continuous batching of queries --------------------------------------------
 * A server owns a worker thread and a CUDA stream on the current device. Requests (an
 * AdvancedGreedy or GreedyReplace query on a loaded graph) are admitted in arrival order (a
 * request waiting at its class's cap may be passed by requests that fit, at most 4 of its own
 * class) whenever a batch slot is free, their device state (about 8n + n/4 bytes plus seeds and
 * blockers) fits the memory budget and their graph-size class is under its per-step sample cap (more requests of one class per step add little throughput once their samples fill
 * the GPU, and every one of them would finish later). Each step advances the admitted requests of one graph-size
 * class (n <= 2^16, 2^17, 2^18, larger) by one greedy round in shared launches (one Alg. 2 launch
 * over the sampled graphs of those requests, then one selection launch). The class a step
 * serves is the busy class that has had the least GPU time, so requests on small graphs advance
 * at their own pace next to requests on large ones. A request runs its own rounds 0, 1, ... on
 * the steps that serve its class, so its random stream and result are exactly those of
 * imin_advanced_greedy / imin_greedy_replace called alone. Finished requests leave between
 * steps and free their slot and memory. Graphs must stay loaded until their requests finish.
 * At admission each request takes its graph's tuned warp/block cutoff (tuned on the server's
 * stream the first time a graph and seed-set size class is seen). */
typedef struct imin_server imin_server;

typedef struct imin_server_config {
    uint64_t memory_budget;  /* bytes of request state the server may hold (0: 1/4 of free memory) */
    int32_t max_active;      /* batch slots (0: 256) */
    int32_t max_class_samples;  /* sampled graphs per step that one size class may batch across its
                                   requests (0: 200,000). A pending request waits while its class
                                   is at the cap (it runs alone when it exceeds the cap by itself);
                                   requests of other classes are admitted past it, and so are at
                                   most 4 later requests of its own class that fit. */
} imin_server_config;

typedef struct imin_server_stats {
    uint64_t submitted, admitted, completed;
    uint64_t steps;          /* batched steps run */
    uint64_t samples;        /* sampled graphs processed */
    uint64_t memory_in_use;  /* bytes of admitted request state */
    uint64_t pending;        /* requests waiting for admission */
} imin_server_stats;

int imin_server_create(const imin_server_config* cfg, imin_server** out);

/* Queue a request. driver: 0 = AdvancedGreedy (Alg. 3), 1 = GreedyReplace (Alg. 4). seeds (host or
 * device) are copied. Never waits for the GPU. *ticket identifies the request for
 * imin_server_wait. Errors: IMIN_ERR_INVALID, IMIN_ERR_NOMEM (state larger than the whole
 * budget), or the server's fatal error after a failed step. Thread-safe. */
int imin_server_submit(imin_server* srv, int32_t driver, const imin_graph* g, const int32_t* seeds,
                       int32_t n_seeds, int32_t b, uint32_t theta, uint64_t key, uint64_t* ticket);

/* Wait up to timeout_ms (negative: forever) for a request; on success copies its blockers
 * (host int32[capacity]) and count, reports the latency from submission to completion in
 * milliseconds, and releases the ticket. IMIN_ERR_TIMEOUT leaves the ticket valid. */
int imin_server_wait(imin_server* srv, uint64_t ticket, int64_t timeout_ms, int32_t* out_blockers,
                     int32_t capacity, int32_t* out_count, double* latency_ms);

int imin_server_get_stats(imin_server* srv, imin_server_stats* out);

/* Finish all submitted requests, stop the worker and release the server. */
int imin_server_destroy(imin_server* srv);

/* Work counters of one Alg. 2 call, for throughput accounting (not part of the method). */
typedef struct imin_stats {
    uint64_t samples;        /* sampled graphs processed (theta) */
    uint64_t reached;        /* sum over samples of |R|, seeds included */
    uint64_t examined_edges; /* sum over samples of the out-edges of reached vertices */
    uint64_t live_edges;     /* sum over samples of live edges into reached non-seed vertices */
    uint64_t nontree_edges;  /* live edges that were not BFS discovery edges */
    uint64_t dom_passes;     /* dominator fixed-point passes */
    /* per kernel tier, counting the samples each tier finished: 0 = warp per sample with a
       shared-memory hash, 1 = warp per sample with global scratch for up to 16K reached
       vertices, 2 = warp per sample with whole-graph scratch (final fallback), 3 = block per
       sample with a shared-memory visited bitmap (graphs with n <= 2^18) */
    uint64_t tier_samples[4];
    uint64_t tier_reached[4];
    uint64_t tier_examined_edges[4];
    uint64_t tier_live_edges[4];
} imin_stats;

/* imin_estimate_decrease plus the work counters of the call. Synchronizes `stream`. */
int imin_estimate_decrease_stats(const imin_graph* g, const int32_t* seeds, int32_t n_seeds,
                                 const int32_t* blocked, int32_t n_blocked, uint32_t theta,
                                 uint64_t key, uint32_t round, uint64_t* out_delta,
                                 imin_stats* stats, void* stream);

/* ---- autotuning (launch configuration only; the paper has no counterpart) ---------------- */

/* Choose the warp/block cutoff for this graph and seed-set size and cache it in the graph handle.
 * Samples of Alg. 2 whose cascade (non-seed reached vertices) stays within the cutoff are
 * finished by the warp-per-sample tier; larger ones are re-run by the block-per-sample tier.
 * After untimed warm-up calls that estimate the time per sample, the tuner times three Alg. 2
 * calls (round 0 of `key`, no blockers; each sized to take about 2 ms, at most 24 samples per
 * resident block of the block tier and at most 65,536) for each candidate cutoff
 * {0, 64, 96, 128, 192} (0 = block tier only), interleaved, and keeps the candidate with the
 * smallest minimum time. When fewer than 4 samples per block fit in 2 ms (huge cascades), it does
 * not time the candidates: it keeps 96 if the warm-up's warp tier finished at least a tenth of
 * its samples, and 0 otherwise. The first warm-up call samples at most 1,024 graphs (at most the caller's
 * theta for the lazy tuning).
 * The cutoff never changes any result of this library, only which kernel computes a sample.
 * The estimate and greedy calls tune lazily on first use for each graph and seed-set size class
 * (ceil(log2 n_seeds)) unless IMIN_AUTOTUNE=0 (fixed cutoff 96) or IMIN_TIER0_VERTICES=<c>
 * (forced cutoff c); a call on a stream under capture uses 96. Results are also kept for the
 * life of the process under a fingerprint of the graph (its sizes and sampled CSR entries), so a
 * new handle of the same graph does not tune again. This entry point re-tunes unconditionally.
 *   seeds     int32[n_seeds], host or device, distinct ids in [0, n).
 *   key       Philox key of the timed calls.
 *   stream    CUDA stream (NULL: legacy default); synchronized.
 *   out_cutoff  receives the chosen cutoff.
 * Errors: IMIN_ERR_INVALID (bad handle, seeds or NULL output), IMIN_ERR_CUDA, IMIN_ERR_NOMEM. */
int imin_autotune(const imin_graph* g, const int32_t* seeds, int32_t n_seeds, uint64_t key,
                  void* stream, int32_t* out_cutoff);

/* ---- measurement hooks (throughput accounting; the paper has no counterpart) ------------- */

/* Work counters of the last successful estimate / greedy call on the calling thread, summed
 * over all of that call's Alg. 2 rounds. */
int imin_last_stats(imin_stats* out);

/* Number of CUDA kernels this library has launched in the process so far. */
uint64_t imin_launch_count(void);

/* Per-kind kernel timing. When enabled, every kernel launch of the entry points above is
 * bracketed by CUDA events recorded on the stream it is launched on -- inside the CUDA graph of
 * a greedy or batched driver as event-record nodes, so the captured production path is what is
 * timed; the elapsed times are added up when the entry point synchronizes. Kinds: 0-3 = sample
 * tiers 0-3, 4 = blocker selection, 5 = other small kernels (only launches of kind 5 made by the
 * greedy drivers are timed). Timing adds event records between launches. */
typedef struct imin_profile {
    uint64_t launches[6];
    double ms[6];
} imin_profile;
int imin_profile_enable(int on);
int imin_profile_read(imin_profile* out, int reset);

/* Message describing the last failure on the calling thread ("" if none). */
const char* imin_last_error(void);

/* ABI version of this header (IMIN_ABI_VERSION). */
#define IMIN_ABI_VERSION 1
int imin_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* IMIN_H */
