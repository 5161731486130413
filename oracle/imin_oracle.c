/*
 * imin_oracle.c -- CPU oracle for the sampled-dominator-tree estimator and the two greedy
 * drivers of "Minimizing the Influence of Misinformation via Vertex Blocking" (arXiv
 * 2302.13529).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain, obviously-correct statement of what
 * the GPU path must compute. Only the test suite, the smoke check and the benchmark's CPU
 * baseline may load it. It shares no code, header or table with the CUDA library; the two
 * are written independently from the same definitions.
 *
 * What it computes, step by step in the paper's order:
 *   - Random sampled graph g (Def. 4, Sec. 4.2.2): every edge e = (u,v) is kept
 *     independently with probability p(u,v). Edge e is kept in sample j of call `round`
 *     iff  W(key, round, j, e) <= thr[e],  where W is one 32-bit word of Philox4x32-10
 *     (below) and thr = ceil(p * 2^32) - 1 (keep probability (thr+1)/2^32).
 *   - Multiple seeds are merged into one super-seed s' (Sec. 4, "From Multiple Seeds to One
 *     Seed"): s' -> s for every seed s. Edges that enter a seed are dropped (a seed is active
 *     from time 0; the merged graph has no edge into s'). Each original seed edge keeps its
 *     own draw: the merged edge s' -> u is live iff one of them is, which has exactly the
 *     probability 1 - prod(1 - p_i) the paper assigns to it.
 *   - Blockers (Def. 2): every in-edge of a blocked vertex has probability 0, i.e. blocked
 *     vertices are never reached.
 *   - Only the part of g reachable from s' matters for dominators from s' (Defs. 5-6 speak
 *     of paths from s'), so the sample is built by a breadth-first search from the seeds that
 *     decides each out-edge of a reached vertex exactly once; the recorded live edges among
 *     reached vertices are the reachable part of g.
 *   - Dominator tree by Lengauer-Tarjan (Sec. 4.2.3, Lemma 3): DFS numbering from s',
 *     semidominators with path-compressed EVAL/LINK, implicit idom via Lemma 3, then the
 *     final fix-up pass in DFS order.
 *   - c[u] = size of u's dominator subtree (Alg. 2; Thm. 6: c[u] = sigma^{->u}(s', g)).
 *   - Delta[u] += c[u] for every reached non-seed u (Alg. 2). The paper's division by theta is
 *     left out: counts are kept as exact uint64 sums, and the argmax is unchanged by the
 *     common positive factor 1/theta.
 *   - AdvancedGreedy (Alg. 3) and GreedyReplace (Alg. 4), argmax with strict '>' scanning
 *     candidates in ascending vertex id (so the smallest id wins ties).
 *   - The expected spread E(S, G[V \ B]) (Def. 3) by simulation: the sum of |R| (seeds
 *     included) over sampled graphs of the same stream.
 *   - Every entry point also runs under the linear-threshold model, the standard triggering
 *     model (Sec. 4.5), selected by its last argument (0: IC, 1: LT); only the live-edge
 *     decision changes (see the LT section below).
 *
 * Philox4x32-10 is written from J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw,
 * "Parallel Random Numbers: As Easy as 1, 2, 3", SC'11, Sec. 3.3 (Philox): 4 x 32-bit counter,
 * 2 x 32-bit key, 10 rounds; each round multiplies counter words 0 and 2 by the two round
 * multipliers (full 64-bit products), and builds the new counter from the high halves xor'd
 * with the other two words and the round key, and the low halves; the key is bumped by the
 * two Weyl constants between rounds.
 *
 * Stream layout: for edge id e in sample j of call `round` under 64-bit key K,
 *   counter = ( (e >> 2) & 0xffffffff, j, round, (e >> 2) >> 32 ),  key = ( K & 0xffffffff, K >> 32 )
 *   word    = output[e & 3]
 * so one Philox evaluation serves the four edge ids 4q .. 4q+3.
 *
 * `round` numbers the calls of DecreaseESComputation within one query from 0: AdvancedGreedy
 * uses round i-1 in its i-th iteration; GreedyReplace numbers its phase-1 calls first and
 * continues the count through phase 2.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------------------------------
 * Philox4x32-10
 * ---------------------------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

ORACLE_API void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* The 32-bit uniform word that decides edge e in sample j of call `round`. */
ORACLE_API uint32_t oracle_edge_word(uint64_t key, uint32_t round, uint32_t sample, int64_t e)
{
    uint64_t q = (uint64_t)e >> 2;
    uint32_t ctr[4] = {(uint32_t)q, sample, round, (uint32_t)(q >> 32)};
    uint32_t k[2] = {(uint32_t)key, (uint32_t)(key >> 32)};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, k, out);
    return out[e & 3];
}

/* Def. 4: edge e is present in the sampled graph iff its word is <= its threshold. */
static int edge_live(uint64_t key, uint32_t round, uint32_t sample, int64_t e, uint32_t thr)
{
    return oracle_edge_word(key, round, sample, e) <= thr;
}

/* ------------------------------------------------------------------------------------------
 * Linear-threshold model, the best-known triggering model (Sec. 4.5: every vertex v draws a
 * triggering set from a distribution over subsets of its in-neighbours, and only edges from that
 * set stay). In the LT model the set holds at most one in-neighbour: edge (u, v) with probability
 * b(u, v), none with probability 1 - sum_u b(u, v). Encoding: thr[e] + 1 is edge e's share of
 * 2^32 (the same fixed point as the IC thresholds), the in-edges of v in ascending edge id take
 * consecutive intervals [lo_e, lo_e + thr[e]] of [0, 2^32), and sample j keeps edge e = (u, v)
 * iff v's word of that sample lies in e's interval. v's word is one 32-bit word of the same
 * Philox stream, counter (v >> 2, j, round, 0x80000000), word v & 3 -- the last counter word
 * keeps vertex words apart from edge words, whose last counter word is e >> 34 < 2^29.
 * ---------------------------------------------------------------------------------------- */
ORACLE_API uint32_t oracle_vertex_word(uint64_t key, uint32_t round, uint32_t sample, int32_t v)
{
    uint32_t ctr[4] = {(uint32_t)v >> 2, sample, round, 0x80000000u};
    uint32_t k[2] = {(uint32_t)key, (uint32_t)(key >> 32)};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, k, out);
    return out[v & 3];
}

/* ------------------------------------------------------------------------------------------
 * growable int32 array
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    int32_t *a;
    int64_t n, cap;
} ivec;

static int iv_push(ivec *v, int32_t x)
{
    if (v->n == v->cap) {
        int64_t nc = v->cap ? v->cap * 2 : 64;
        int32_t *na = (int32_t *)realloc(v->a, (size_t)nc * sizeof(int32_t));
        if (!na) return -1;
        v->a = na;
        v->cap = nc;
    }
    v->a[v->n++] = x;
    return 0;
}

static int iv_resize(ivec *v, int64_t n)
{
    if (n > v->cap) {
        int32_t *na = (int32_t *)realloc(v->a, (size_t)n * sizeof(int32_t));
        if (!na) return -1;
        v->a = na;
        v->cap = n;
    }
    v->n = n;
    return 0;
}

static void iv_free(ivec *v)
{
    free(v->a);
    v->a = NULL;
    v->n = v->cap = 0;
}

/* ------------------------------------------------------------------------------------------
 * graph view and per-query state
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    int32_t n;
    int64_t m;
    const int32_t *row_ptr;
    const int32_t *col;
    const uint32_t *thr;  /* IC: live threshold; LT: interval width - 1 */
    const uint32_t *lo;   /* LT: start of each edge's interval; NULL for the IC model */
} graph_t;

/* Whether edge e = (u, v) is live in sample j of call `round` (Def. 4 for IC; the triggering
 * set draw above for LT). */
static int live(const graph_t *g, uint64_t key, uint32_t round, uint32_t sample, int64_t e, int32_t v)
{
    if (!g->lo) return edge_live(key, round, sample, e, g->thr[e]);
    return oracle_vertex_word(key, round, sample, v) - g->lo[e] <= g->thr[e];
}

/* LT: lo[e] for every edge; fails when the shares of some vertex's in-edges exceed 2^32. */
static int lt_offsets(const graph_t *g, uint32_t *lo)
{
    uint64_t *acc = (uint64_t *)calloc((size_t)g->n + 1, sizeof(uint64_t));
    if (!acc) return -1;
    int rc = 0;
    for (int64_t e = 0; e < g->m && !rc; e++) {
        int32_t v = g->col[e];
        if (v < 0 || v >= g->n) {
            rc = -1;
            break;
        }
        lo[e] = (uint32_t)acc[v];
        acc[v] += (uint64_t)g->thr[e] + 1;
        if (acc[v] > (1ull << 32)) rc = -1;
    }
    free(acc);
    return rc;
}

/* model 0: IC (Def. 4); model 1: LT. For LT, *lo receives the interval starts (free it). */
static int graph_model(graph_t *g, int32_t model, uint32_t **lo)
{
    *lo = NULL;
    g->lo = NULL;
    if (model == 0) return 0;
    if (model != 1) return -1;
    *lo = (uint32_t *)malloc(((size_t)g->m + 1) * sizeof(uint32_t));
    if (!*lo || lt_offsets(g, *lo)) {
        free(*lo);
        *lo = NULL;
        return -1;
    }
    g->lo = *lo;
    return 0;
}

typedef struct {
    /* size n */
    int32_t *local;      /* global id -> local id (1..R) in the current sample, 0 if unreached */
    uint8_t *is_seed;
    uint8_t *is_blocked;
    /* per-sample local graph (node 0 = super-seed s') */
    ivec gid;            /* local -> global (gid[0] = -1) */
    ivec esrc, edst;     /* live edges among reached vertices, local ids */
    ivec succ_ptr, succ, pred_ptr, pred;
    /* Lengauer-Tarjan arrays (local ids) */
    ivec dfn, vertex, parent, semi, idom, ancestor, label, bucket_head, bucket_next, stack,
        stack_it, cstack;
    ivec csize;
} state_t;

static int state_init(state_t *s, int32_t n)
{
    memset(s, 0, sizeof(*s));
    s->local = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    s->is_seed = (uint8_t *)calloc((size_t)n + 1, 1);
    s->is_blocked = (uint8_t *)calloc((size_t)n + 1, 1);
    if (!s->local || !s->is_seed || !s->is_blocked) return -1;
    return 0;
}

static void state_free(state_t *s)
{
    free(s->local);
    free(s->is_seed);
    free(s->is_blocked);
    ivec *all[] = {&s->gid, &s->esrc, &s->edst, &s->succ_ptr, &s->succ, &s->pred_ptr, &s->pred,
                   &s->dfn, &s->vertex, &s->parent, &s->semi, &s->idom, &s->ancestor,
                   &s->label, &s->bucket_head, &s->bucket_next, &s->stack, &s->stack_it,
                   &s->cstack, &s->csize};
    for (size_t i = 0; i < sizeof(all) / sizeof(all[0]); i++) iv_free(all[i]);
}

/* Checks shared by every entry point: CSR shape, vertex ranges, seed uniqueness. */
static int validate(const graph_t *g, const int32_t *seeds, int32_t ns, const int32_t *blocked,
                    int32_t nb, state_t *s)
{
    if (g->n < 0 || g->m < 0 || !g->row_ptr) return -1;
    if (g->row_ptr[0] != 0 || g->row_ptr[g->n] != g->m) return -1;
    for (int32_t u = 0; u < g->n; u++)
        if (g->row_ptr[u + 1] < g->row_ptr[u]) return -1;
    for (int64_t e = 0; e < g->m; e++)
        if (g->col[e] < 0 || g->col[e] >= g->n) return -1;
    for (int32_t i = 0; i < ns; i++) {
        if (seeds[i] < 0 || seeds[i] >= g->n || s->is_seed[seeds[i]]) return -1;
        s->is_seed[seeds[i]] = 1;
    }
    for (int32_t i = 0; i < nb; i++) {
        if (blocked[i] < 0 || blocked[i] >= g->n || s->is_seed[blocked[i]] ||
            s->is_blocked[blocked[i]])
            return -1;
        s->is_blocked[blocked[i]] = 1;
    }
    return 0;
}

/* Build successor and predecessor lists of the local sampled graph (counting sort). */
static int build_adjacency(state_t *s, int32_t N)
{
    int64_t E = s->esrc.n;
    if (iv_resize(&s->succ_ptr, N + 1) || iv_resize(&s->pred_ptr, N + 1) ||
        iv_resize(&s->succ, E) || iv_resize(&s->pred, E))
        return -1;
    memset(s->succ_ptr.a, 0, (size_t)(N + 1) * sizeof(int32_t));
    memset(s->pred_ptr.a, 0, (size_t)(N + 1) * sizeof(int32_t));
    for (int64_t k = 0; k < E; k++) {
        s->succ_ptr.a[s->esrc.a[k] + 1]++;
        s->pred_ptr.a[s->edst.a[k] + 1]++;
    }
    for (int32_t i = 0; i < N; i++) {
        s->succ_ptr.a[i + 1] += s->succ_ptr.a[i];
        s->pred_ptr.a[i + 1] += s->pred_ptr.a[i];
    }
    ivec fill_s = {0}, fill_p = {0};
    if (iv_resize(&fill_s, N) || iv_resize(&fill_p, N)) {
        iv_free(&fill_s);
        iv_free(&fill_p);
        return -1;
    }
    memcpy(fill_s.a, s->succ_ptr.a, (size_t)N * sizeof(int32_t));
    memcpy(fill_p.a, s->pred_ptr.a, (size_t)N * sizeof(int32_t));
    for (int64_t k = 0; k < E; k++) {
        s->succ.a[fill_s.a[s->esrc.a[k]]++] = s->edst.a[k];
        s->pred.a[fill_p.a[s->edst.a[k]]++] = s->esrc.a[k];
    }
    iv_free(&fill_s);
    iv_free(&fill_p);
    return 0;
}

/* ------------------------------------------------------------------------------------------
 * Lengauer-Tarjan on the local graph with N nodes, root 0. Writes idom (local ids) with
 * idom[0] = 0, and the DFS preorder in `vertex` (vertex[i] = node with DFS number i).
 * ---------------------------------------------------------------------------------------- */

/* EVAL's path compression, done with an explicit stack instead of recursion: the nodes on
 * the ancestor path are compressed from the top down, each taking the smaller-semi label of
 * its ancestor and then skipping over it. */
static void lt_compress(state_t *s, int32_t v)
{
    int32_t *anc = s->ancestor.a, *lab = s->label.a, *semi = s->semi.a;
    s->cstack.n = 0;
    int32_t x = v;
    while (anc[anc[x]] != -1) {
        iv_push(&s->cstack, x);
        x = anc[x];
    }
    for (int64_t i = s->cstack.n - 1; i >= 0; i--) {
        x = s->cstack.a[i];
        int32_t a = anc[x];
        if (semi[lab[a]] < semi[lab[x]]) lab[x] = lab[a];
        anc[x] = anc[a];
    }
}

static int32_t lt_eval(state_t *s, int32_t v)
{
    if (s->ancestor.a[v] == -1) return v;
    lt_compress(s, v);
    return s->label.a[v];
}

static int lengauer_tarjan(state_t *s, int32_t N)
{
    if (iv_resize(&s->dfn, N) || iv_resize(&s->vertex, N) || iv_resize(&s->parent, N) ||
        iv_resize(&s->semi, N) || iv_resize(&s->idom, N) || iv_resize(&s->ancestor, N) ||
        iv_resize(&s->label, N) || iv_resize(&s->bucket_head, N) ||
        iv_resize(&s->bucket_next, N) || iv_resize(&s->stack, N) || iv_resize(&s->stack_it, N))
        return -1;
    int32_t *dfn = s->dfn.a, *vertex = s->vertex.a, *parent = s->parent.a, *semi = s->semi.a,
            *idom = s->idom.a, *anc = s->ancestor.a, *lab = s->label.a, *bh = s->bucket_head.a,
            *bn = s->bucket_next.a;
    for (int32_t i = 0; i < N; i++) {
        dfn[i] = -1;
        anc[i] = -1;
        lab[i] = i;
        bh[i] = -1;
        idom[i] = -1;
    }
    /* Step 1: depth-first search from the root, numbering nodes in preorder. */
    int32_t cnt = 0, top = 0;
    int32_t *stk = s->stack.a, *it = s->stack_it.a;
    dfn[0] = cnt;
    vertex[cnt++] = 0;
    parent[0] = -1;
    stk[top] = 0;
    it[top] = s->succ_ptr.a[0];
    top++;
    while (top > 0) {
        int32_t v = stk[top - 1];
        if (it[top - 1] < s->succ_ptr.a[v + 1]) {
            int32_t w = s->succ.a[it[top - 1]++];
            if (dfn[w] == -1) {
                dfn[w] = cnt;
                vertex[cnt++] = w;
                parent[w] = v;
                stk[top] = w;
                it[top] = s->succ_ptr.a[w];
                top++;
            }
        } else {
            top--;
        }
    }
    if (cnt != N) return -2; /* every local node is reachable by construction */
    for (int32_t i = 0; i < N; i++) semi[i] = dfn[i];

    /* Steps 2-3: semidominators in reverse preorder; implicit idoms through buckets. */
    for (int32_t i = N - 1; i >= 1; i--) {
        int32_t w = vertex[i];
        for (int32_t k = s->pred_ptr.a[w]; k < s->pred_ptr.a[w + 1]; k++) {
            int32_t v = s->pred.a[k];
            int32_t u = lt_eval(s, v);
            if (semi[u] < semi[w]) semi[w] = semi[u];
        }
        int32_t sd = vertex[semi[w]];
        bn[w] = bh[sd];
        bh[sd] = w;
        int32_t p = parent[w];
        anc[w] = p; /* LINK(parent(w), w) */
        for (int32_t v = bh[p]; v != -1; v = bn[v]) {
            int32_t u = lt_eval(s, v);
            idom[v] = (semi[u] < semi[v]) ? u : p;
        }
        bh[p] = -1;
    }
    /* Step 4: explicit idoms in preorder. */
    for (int32_t i = 1; i < N; i++) {
        int32_t w = vertex[i];
        if (idom[w] != vertex[semi[w]]) idom[w] = idom[idom[w]];
    }
    idom[0] = 0;
    return 0;
}

/* ------------------------------------------------------------------------------------------
 * One sampled graph: BFS from the seeds over live edges, dominator tree, subtree sizes.
 * On return the local graph occupies s->gid (N = s->gid.n nodes incl. the root), s->idom and
 * s->csize; s->local maps reached global ids to local ids (caller must reset via
 * clear_sample()).
 * ---------------------------------------------------------------------------------------- */
static int run_sample(const graph_t *g, const int32_t *seeds, int32_t ns, uint64_t key,
                      uint32_t round, uint32_t sample, state_t *s)
{
    s->gid.n = 0;
    s->esrc.n = 0;
    s->edst.n = 0;
    if (iv_push(&s->gid, -1)) return -1; /* local 0: super-seed s' */
    for (int32_t i = 0; i < ns; i++) {
        int32_t v = seeds[i];
        s->local[v] = (int32_t)s->gid.n;
        if (iv_push(&s->gid, v) || iv_push(&s->esrc, 0) || iv_push(&s->edst, s->local[v]))
            return -1;
    }
    /* breadth-first search; the gid array doubles as the queue */
    for (int64_t qi = 1; qi < s->gid.n; qi++) {
        int32_t u = s->gid.a[qi];
        for (int64_t e = g->row_ptr[u]; e < g->row_ptr[u + 1]; e++) {
            int32_t v = g->col[e];
            if (s->is_seed[v] || s->is_blocked[v]) continue;
            if (!live(g, key, round, sample, e, v)) continue;
            if (s->local[v] == 0) {
                s->local[v] = (int32_t)s->gid.n;
                if (iv_push(&s->gid, v)) return -1;
            }
            if (iv_push(&s->esrc, (int32_t)qi) || iv_push(&s->edst, s->local[v])) return -1;
        }
    }
    int32_t N = (int32_t)s->gid.n;
    if (build_adjacency(s, N)) return -1;
    int rc = lengauer_tarjan(s, N);
    if (rc) return rc;
    /* subtree sizes: idom(w) precedes w in DFS preorder, so a reverse preorder sweep adds
       every finished subtree into its parent */
    if (iv_resize(&s->csize, N)) return -1;
    for (int32_t i = 0; i < N; i++) s->csize.a[i] = 1;
    for (int32_t i = N - 1; i >= 1; i--) {
        int32_t w = s->vertex.a[i];
        s->csize.a[s->idom.a[w]] += s->csize.a[w];
    }
    return 0;
}

static void clear_sample(state_t *s)
{
    for (int64_t i = 1; i < s->gid.n; i++) s->local[s->gid.a[i]] = 0;
}

/* ------------------------------------------------------------------------------------------
 * Public entry points (all return 0 on success, negative on invalid input / failure)
 * ---------------------------------------------------------------------------------------- */

/* Per-sample detail for tests: c_out[v] = subtree size of v (0 if v unreached, seeds
 * included), idom_out[v] = global id of v's immediate dominator (-1 if the super-seed or v
 * unreached), *n_reached = |R| including seeds, *n_live = number of live edges among R. */
ORACLE_API int oracle_sample(int32_t n, int64_t m, const int32_t *row_ptr, const int32_t *col,
                             const uint32_t *thr, const int32_t *seeds, int32_t ns,
                             const int32_t *blocked, int32_t nb, uint64_t key, uint32_t round,
                             uint32_t sample, uint32_t *c_out, int32_t *idom_out,
                             int64_t *n_reached, int64_t *n_live, int32_t model)
{
    graph_t g = {n, m, row_ptr, col, thr, NULL};
    uint32_t *lo = NULL;
    if (graph_model(&g, model, &lo)) return -1;
    state_t s;
    if (state_init(&s, n)) {
        free(lo);
        return -1;
    }
    int rc = validate(&g, seeds, ns, blocked, nb, &s);
    if (!rc) rc = run_sample(&g, seeds, ns, key, round, sample, &s);
    if (!rc) {
        for (int32_t v = 0; v < n; v++) {
            c_out[v] = 0;
            idom_out[v] = -1;
        }
        for (int64_t i = 1; i < s.gid.n; i++) {
            int32_t v = s.gid.a[i];
            c_out[v] = (uint32_t)s.csize.a[i];
            idom_out[v] = s.gid.a[s.idom.a[i]];
        }
        *n_reached = s.gid.n - 1;
        *n_live = s.esrc.n - ns;
    }
    state_free(&s);
    free(lo);
    return rc;
}

/* Alg. 2 over samples j in [j0, j1): delta[v] += c[v] for every reached non-seed v.
 * delta is accumulated into (not cleared). */
static int decrease_range(const graph_t *g, const int32_t *seeds, int32_t ns, uint64_t key,
                          uint32_t round, uint32_t j0, uint32_t j1, uint64_t *delta,
                          state_t *s)
{
    for (uint32_t j = j0; j < j1; j++) {
        int rc = run_sample(g, seeds, ns, key, round, j, s);
        if (rc) {
            clear_sample(s);
            return rc;
        }
        for (int64_t i = 1 + ns; i < s->gid.n; i++)
            delta[s->gid.a[i]] += (uint64_t)s->csize.a[i];
        clear_sample(s);
    }
    return 0;
}

/* ------------------------------------------------------------------------------------------
 * Optional parallelism over samples. Alg. 2's counters and the simulated spread are sums over
 * independent samples, so splitting [j0, j1) into blocks handled by worker threads, each with
 * its own state and its own partial sums, and adding the partial sums gives exactly the result
 * of the sequential loop (integer addition is associative). The default is one thread: the
 * plain sequential loop.
 * ---------------------------------------------------------------------------------------- */
static int g_threads = 1;

ORACLE_API void oracle_set_threads(int32_t threads) { g_threads = threads < 1 ? 1 : threads; }
ORACLE_API int32_t oracle_get_threads(void) { return g_threads; }

enum { SAMPLE_BLOCK = 16 };

typedef struct {
    const graph_t *g;
    const int32_t *seeds;
    int32_t ns;
    uint64_t key;
    uint32_t round, j1;
    const state_t *parent;     /* seed / blocked marks to copy */
    int spread;                /* 0: Alg. 2 counters; 1: sum of |R| */
    uint32_t *next;            /* next unclaimed sample (shared) */
    pthread_mutex_t *mu;
    uint64_t *delta;           /* this worker's partial counters [n] (Alg. 2) */
    uint64_t sum;              /* this worker's partial sum of |R| (spread) */
    int rc;
} worker_t;

static int reach_count(const graph_t *g, const int32_t *seeds, int32_t ns, uint64_t key,
                       uint32_t round, uint32_t sample, state_t *s, int64_t *count);

static void *worker_main(void *arg)
{
    worker_t *w = (worker_t *)arg;
    const int32_t n = w->g->n;
    state_t s;
    if (state_init(&s, n)) {
        w->rc = -1;
        return NULL;
    }
    memcpy(s.is_seed, w->parent->is_seed, (size_t)n);
    memcpy(s.is_blocked, w->parent->is_blocked, (size_t)n);
    for (;;) {
        pthread_mutex_lock(w->mu);
        const uint32_t a = *w->next;
        const uint32_t b = (w->j1 - a > SAMPLE_BLOCK) ? a + SAMPLE_BLOCK : w->j1;
        *w->next = b;
        pthread_mutex_unlock(w->mu);
        if (a >= w->j1 || w->rc) break;
        if (!w->spread) {
            w->rc = decrease_range(w->g, w->seeds, w->ns, w->key, w->round, a, b, w->delta, &s);
        } else {
            for (uint32_t j = a; j < b && !w->rc; j++) {
                int64_t c = 0;
                w->rc = reach_count(w->g, w->seeds, w->ns, w->key, w->round, j, &s, &c);
                w->sum += (uint64_t)c;
                clear_sample(&s);
            }
        }
    }
    state_free(&s);
    return NULL;
}

/* Samples [j0, j1) on g_threads threads: adds Alg. 2's counters into delta (spread = 0) or the
 * sum of |R| into *sum (spread = 1). s holds the query's seed / blocked marks. */
static int run_parallel(const graph_t *g, const int32_t *seeds, int32_t ns, uint64_t key,
                        uint32_t round, uint32_t j0, uint32_t j1, const state_t *s, int spread,
                        uint64_t *delta, uint64_t *sum)
{
    int T = g_threads;
    if ((int64_t)(j1 - j0) < (int64_t)T * SAMPLE_BLOCK) T = (int)((j1 - j0) / SAMPLE_BLOCK) + 1;
    worker_t *w = (worker_t *)calloc((size_t)T, sizeof(worker_t));
    pthread_t *th = (pthread_t *)calloc((size_t)T, sizeof(pthread_t));
    uint8_t *started = (uint8_t *)calloc((size_t)T, 1);
    if (!w || !th || !started) {
        free(w);
        free(th);
        free(started);
        return -1;
    }
    pthread_mutex_t mu = PTHREAD_MUTEX_INITIALIZER;
    uint32_t next = j0;
    int rc = 0;
    for (int t = 0; t < T; t++) {
        w[t] = (worker_t){g, seeds, ns, key, round, j1, s, spread, &next, &mu, NULL, 0, 0};
        if (!spread) {
            w[t].delta = (uint64_t *)calloc((size_t)g->n + 1, sizeof(uint64_t));
            if (!w[t].delta) rc = -1;
        }
    }
    for (int t = 0; t < T && !rc; t++) {
        if (pthread_create(&th[t], NULL, worker_main, &w[t]) != 0) rc = -1;
        else started[t] = 1;
    }
    if (rc) {  /* stop the workers that started: claim every remaining sample */
        pthread_mutex_lock(&mu);
        next = j1;
        pthread_mutex_unlock(&mu);
    }
    for (int t = 0; t < T; t++) {
        if (started[t]) pthread_join(th[t], NULL);
        if (!rc && w[t].rc) rc = w[t].rc;
    }
    for (int t = 0; t < T; t++) {
        if (!rc) {
            if (spread) *sum += w[t].sum;
            else
                for (int32_t v = 0; v < g->n; v++) delta[v] += w[t].delta[v];
        }
        free(w[t].delta);
    }
    free(w);
    free(th);
    free(started);
    return rc;
}

/* Alg. 2 over samples [j0, j1), adding into delta: the sequential loop, or run_parallel. */
static int alg2(const graph_t *g, const int32_t *seeds, int32_t ns, uint64_t key, uint32_t round,
                uint32_t j0, uint32_t j1, uint64_t *delta, state_t *s)
{
    if (g_threads <= 1 || j1 - j0 < 2 * SAMPLE_BLOCK)
        return decrease_range(g, seeds, ns, key, round, j0, j1, delta, s);
    return run_parallel(g, seeds, ns, key, round, j0, j1, s, 0, delta, NULL);
}

ORACLE_API int oracle_decrease_range(int32_t n, int64_t m, const int32_t *row_ptr,
                                     const int32_t *col, const uint32_t *thr,
                                     const int32_t *seeds, int32_t ns, const int32_t *blocked,
                                     int32_t nb, uint64_t key, uint32_t round, uint32_t j0,
                                     uint32_t j1, uint64_t *delta, int32_t model)
{
    graph_t g = {n, m, row_ptr, col, thr, NULL};
    uint32_t *lo = NULL;
    if (graph_model(&g, model, &lo)) return -1;
    state_t s;
    if (state_init(&s, n)) {
        free(lo);
        return -1;
    }
    int rc = validate(&g, seeds, ns, blocked, nb, &s);
    if (!rc) {
        memset(delta, 0, (size_t)n * sizeof(uint64_t));
        rc = alg2(&g, seeds, ns, key, round, j0, j1, delta, &s);
    }
    state_free(&s);
    free(lo);
    return rc;
}

/* Alg. 2 (DecreaseESComputation) on G[V \ B]: delta[v] = sum over theta samples of c[v]. */
ORACLE_API int oracle_decrease(int32_t n, int64_t m, const int32_t *row_ptr, const int32_t *col,
                               const uint32_t *thr, const int32_t *seeds, int32_t ns,
                               const int32_t *blocked, int32_t nb, uint32_t theta, uint64_t key,
                               uint32_t round, uint64_t *delta, int32_t model)
{
    return oracle_decrease_range(n, m, row_ptr, col, thr, seeds, ns, blocked, nb, key, round, 0,
                                 theta, delta, model);
}

/* ------------------------------------------------------------------------------------------
 * Expected spread by simulation (Def. 3: E(S, G) = expected number of active vertices, seeds
 * included; the paper evaluates every blocker set it reports by simulating cascades). Sample j
 * of call `round` is the live-edge graph of Def. 4 on the same word stream as Alg. 2; its
 * cascade is the set of vertices reachable from the seeds over live edges without entering a
 * blocked vertex.
 * ---------------------------------------------------------------------------------------- */

/* |R| of one sample (seeds included), by breadth-first search; s->gid is the queue. */
static int reach_count(const graph_t *g, const int32_t *seeds, int32_t ns, uint64_t key,
                       uint32_t round, uint32_t sample, state_t *s, int64_t *count)
{
    s->gid.n = 0;
    if (iv_push(&s->gid, -1)) return -1; /* keeps local ids >= 1, as in run_sample */
    for (int32_t i = 0; i < ns; i++) {
        s->local[seeds[i]] = (int32_t)s->gid.n;
        if (iv_push(&s->gid, seeds[i])) return -1;
    }
    for (int64_t qi = 1; qi < s->gid.n; qi++) {
        int32_t u = s->gid.a[qi];
        for (int64_t e = g->row_ptr[u]; e < g->row_ptr[u + 1]; e++) {
            int32_t v = g->col[e];
            if (s->local[v] != 0 || s->is_blocked[v]) continue;
            if (!live(g, key, round, sample, e, v)) continue;
            s->local[v] = (int32_t)s->gid.n;
            if (iv_push(&s->gid, v)) return -1;
        }
    }
    *count = s->gid.n - 1;
    return 0;
}

/* *total += sum over samples j in [j0, j1) of |R_j| (seeds included), blocked vertices as marked
 * in s: the sequential loop, or run_parallel. */
static int spread_sum(const graph_t *g, const int32_t *seeds, int32_t ns, uint64_t key, uint32_t round,
                      uint32_t j0, uint32_t j1, state_t *s, uint64_t *total)
{
    if (g_threads > 1 && j1 - j0 >= 2 * SAMPLE_BLOCK)
        return run_parallel(g, seeds, ns, key, round, j0, j1, s, 1, NULL, total);
    for (uint32_t j = j0; j < j1; j++) {
        int64_t c = 0;
        int rc = reach_count(g, seeds, ns, key, round, j, s, &c);
        clear_sample(s);
        if (rc) return rc;
        *total += (uint64_t)c;
    }
    return 0;
}

/* *out_sum = sum over samples j in [j0, j1) of |R_j| (seeds included). */
ORACLE_API int oracle_spread_range(int32_t n, int64_t m, const int32_t *row_ptr, const int32_t *col,
                                   const uint32_t *thr, const int32_t *seeds, int32_t ns,
                                   const int32_t *blocked, int32_t nb, uint64_t key, uint32_t round,
                                   uint32_t j0, uint32_t j1, uint64_t *out_sum, int32_t model)
{
    graph_t g = {n, m, row_ptr, col, thr, NULL};
    uint32_t *lo = NULL;
    if (graph_model(&g, model, &lo)) return -1;
    state_t s;
    if (state_init(&s, n)) {
        free(lo);
        return -1;
    }
    int rc = validate(&g, seeds, ns, blocked, nb, &s);
    uint64_t total = 0;
    if (!rc) rc = spread_sum(&g, seeds, ns, key, round, j0, j1, &s, &total);
    if (!rc) *out_sum = total;
    state_free(&s);
    free(lo);
    return rc;
}

/* Number of Alg. 2 calls the last AdvancedGreedy / GreedyReplace call of this process made
 * (GreedyReplace: its phase-1 calls plus the phase-2 calls up to and including the one that
 * stopped the walk). */
static int32_t g_last_calls = 0;

ORACLE_API int32_t oracle_last_calls(void) { return g_last_calls; }

/* strict-'>' argmax over candidate vertices in ascending id; -1 if there is none */
static int32_t argmax_mask(const uint64_t *delta, int32_t n, const uint8_t *is_cand)
{
    int32_t x = -1;
    for (int32_t u = 0; u < n; u++)
        if (is_cand[u] && (x == -1 || delta[u] > delta[x])) x = u;
    return x;
}

/* Alg. 3 AdvancedGreedy: b rounds of Alg. 2 on G[V \ B] followed by the argmax over
 * V \ (S u B). Stops early only when no candidate is left. */
ORACLE_API int oracle_advanced_greedy(int32_t n, int64_t m, const int32_t *row_ptr,
                                      const int32_t *col, const uint32_t *thr,
                                      const int32_t *seeds, int32_t ns, int32_t b,
                                      uint32_t theta, uint64_t key, int32_t *out_blockers,
                                      int32_t *out_count, int32_t model)
{
    graph_t g = {n, m, row_ptr, col, thr, NULL};
    uint32_t *lo = NULL;
    if (graph_model(&g, model, &lo)) return -1;
    state_t s;
    if (b < 0 || theta == 0) {
        free(lo);
        return -1;
    }
    if (state_init(&s, n)) {
        free(lo);
        return -1;
    }
    int rc = validate(&g, seeds, ns, NULL, 0, &s);
    uint64_t *delta = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    uint8_t *cand = (uint8_t *)calloc((size_t)n + 1, 1);
    if (!delta || !cand) rc = -1;
    int32_t count = 0;
    g_last_calls = 0;
    if (!rc) {
        int32_t left = 0;
        for (int32_t u = 0; u < n; u++) {
            cand[u] = !s.is_seed[u];
            left += cand[u];
        }
        for (int32_t i = 0; i < b && left > 0; i++, left--) {
            memset(delta, 0, (size_t)n * sizeof(uint64_t));
            rc = alg2(&g, seeds, ns, key, (uint32_t)i, 0, theta, delta, &s);
            g_last_calls = i + 1;
            if (rc) break;
            int32_t x = argmax_mask(delta, n, cand);
            out_blockers[count++] = x;
            cand[x] = 0;
            s.is_blocked[x] = 1;
        }
    }
    *out_count = count;
    free(delta);
    free(cand);
    state_free(&s);
    free(lo);
    return rc;
}

/* Alg. 4 GreedyReplace.
 * Phase 1: CB = N_out(S) \ S; min(|CB|, b) rounds of Alg. 2 on G[V \ B] with the argmax over
 *          the remaining CB; the winner leaves CB and is appended to B.
 * Phase 2: for positions i = |B|-1 down to 0 (reverse insertion order): u = B[i] is unblocked,
 *          Alg. 2 runs on G[V \ (B \ {u})], the argmax x is taken over V \ (S u B \ {u}) (u
 *          itself is a candidate again), x takes position i, and the phase stops when x = u.
 * out_blockers receives B in list order. */
ORACLE_API int oracle_greedy_replace(int32_t n, int64_t m, const int32_t *row_ptr,
                                     const int32_t *col, const uint32_t *thr,
                                     const int32_t *seeds, int32_t ns, int32_t b,
                                     uint32_t theta, uint64_t key, int32_t *out_blockers,
                                     int32_t *out_count, int32_t model)
{
    graph_t g = {n, m, row_ptr, col, thr, NULL};
    uint32_t *lo = NULL;
    if (graph_model(&g, model, &lo)) return -1;
    state_t s;
    if (b < 0 || theta == 0) {
        free(lo);
        return -1;
    }
    if (state_init(&s, n)) {
        free(lo);
        return -1;
    }
    int rc = validate(&g, seeds, ns, NULL, 0, &s);
    uint64_t *delta = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    uint8_t *cand = (uint8_t *)calloc((size_t)n + 1, 1);
    if (!delta || !cand) rc = -1;
    int32_t count = 0;
    uint32_t round = 0;
    g_last_calls = 0;
    if (!rc) {
        /* CB: out-neighbours of the seeds that are not seeds themselves */
        for (int32_t i = 0; i < ns; i++) {
            int32_t u = seeds[i];
            for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; e++)
                if (!s.is_seed[col[e]]) cand[col[e]] = 1;
        }
        int32_t ncb = 0;
        for (int32_t u = 0; u < n; u++) ncb += cand[u];
        int32_t rounds = ncb < b ? ncb : b;
        for (int32_t i = 0; i < rounds && !rc; i++) {
            memset(delta, 0, (size_t)n * sizeof(uint64_t));
            rc = alg2(&g, seeds, ns, key, round++, 0, theta, delta, &s);
            if (rc) break;
            int32_t x = argmax_mask(delta, n, cand);
            cand[x] = 0;
            out_blockers[count++] = x;
            s.is_blocked[x] = 1;
        }
        /* phase 2: candidates are every vertex that is neither a seed nor blocked */
        for (int32_t u = 0; u < n; u++) cand[u] = !s.is_seed[u] && !s.is_blocked[u];
        for (int32_t i = count - 1; i >= 0 && !rc; i--) {
            int32_t u = out_blockers[i];
            s.is_blocked[u] = 0;
            cand[u] = 1;
            memset(delta, 0, (size_t)n * sizeof(uint64_t));
            rc = alg2(&g, seeds, ns, key, round++, 0, theta, delta, &s);
            if (rc) break;
            int32_t x = argmax_mask(delta, n, cand);
            out_blockers[i] = x;
            s.is_blocked[x] = 1;
            cand[x] = 0;
            if (x == u) break;
        }
    }
    *out_count = count;
    if (round > 0) g_last_calls = (int32_t)round;
    free(delta);
    free(cand);
    state_free(&s);
    free(lo);
    return rc;
}


/* ------------------------------------------------------------------------------------------
 * The comparison algorithms of Sec. 5, all evaluated by simulation (Def. 3) on the sampled
 * graphs of the same stream:
 *   - spread of many blocker sets: every set sees the same samples j in [0, theta) of call
 *     `round` (common random numbers);
 *   - BaselineGreedy (Alg. 1): b rounds; in round i every candidate u of V \ (S u B) is scored
 *     by its simulated spread decrease sum_j |R_j(B)| - |R_j(B u {u})| over samples j in
 *     [0, r) of call i, and the largest decrease wins (strict '>' in ascending id);
 *   - Exact: every min(b, |V \ S|)-subset of V \ S, in lexicographic order, scored by its
 *     simulated spread over samples [0, r) of call 0; the first subset with the smallest spread
 *     wins;
 *   - OutDegree: the b non-seed vertices of largest out-degree (ties: smaller id first);
 *   - Rand: b distinct non-seed vertices chosen uniformly by a partial Fisher-Yates shuffle of
 *     the non-seeds in ascending id, draw t taking index t + floor(w_t * (c - t) / 2^32) with
 *     w_t = word 0 of Philox4x32-10 at counter (t, 0, 0, 0xC0000000) under the key (c = number of
 *     non-seeds).
 * ---------------------------------------------------------------------------------------- */

/* Simulated spread of blocked-set s: marks set members blocked, sums, unmarks. */
static int spread_of_set(const graph_t *g, const int32_t *seeds, int32_t ns, const int32_t *set, int32_t k,
                         uint64_t key, uint32_t round, uint32_t theta, state_t *s, uint64_t *out)
{
    int rc = 0;
    int32_t marked = 0;
    for (; marked < k; marked++) {
        const int32_t v = set[marked];
        if (v < 0 || v >= g->n || s->is_seed[v] || s->is_blocked[v]) {
            rc = -1;
            break;
        }
        s->is_blocked[v] = 1;
    }
    uint64_t total = 0;
    if (!rc) rc = spread_sum(g, seeds, ns, key, round, 0, theta, s, &total);
    for (int32_t i = 0; i < marked; i++) s->is_blocked[set[i]] = 0;
    if (!rc) *out = total;
    return rc;
}

ORACLE_API int oracle_spread_sets(int32_t n, int64_t m, const int32_t *row_ptr, const int32_t *col,
                                  const uint32_t *thr, const int32_t *seeds, int32_t ns,
                                  const int32_t *blocked, int32_t nb, const int32_t *sets, int32_t nsets,
                                  int32_t k, uint64_t key, uint32_t round, uint32_t theta,
                                  uint64_t *out_sums, int32_t model)
{
    graph_t g = {n, m, row_ptr, col, thr, NULL};
    uint32_t *lo = NULL;
    if (nsets < 0 || k < 0 || graph_model(&g, model, &lo)) return -1;
    state_t s;
    if (state_init(&s, n)) {
        free(lo);
        return -1;
    }
    int rc = validate(&g, seeds, ns, blocked, nb, &s);
    for (int32_t i = 0; i < nsets && !rc; i++)
        rc = spread_of_set(&g, seeds, ns, sets + (int64_t)i * k, k, key, round, theta, &s, out_sums + i);
    state_free(&s);
    free(lo);
    return rc;
}

ORACLE_API int oracle_baseline_greedy(int32_t n, int64_t m, const int32_t *row_ptr, const int32_t *col,
                                      const uint32_t *thr, const int32_t *seeds, int32_t ns, int32_t b,
                                      uint32_t r, uint64_t key, int32_t *out_blockers, int32_t *out_count,
                                      int32_t model)
{
    graph_t g = {n, m, row_ptr, col, thr, NULL};
    uint32_t *lo = NULL;
    if (b < 0 || r == 0 || graph_model(&g, model, &lo)) return -1;
    state_t s;
    if (state_init(&s, n)) {
        free(lo);
        return -1;
    }
    int rc = validate(&g, seeds, ns, NULL, 0, &s);
    int32_t count = 0;
    for (int32_t i = 0; i < b && !rc; i++) {
        uint64_t base = 0;
        rc = spread_sum(&g, seeds, ns, key, (uint32_t)i, 0, r, &s, &base);
        int32_t x = -1;
        uint64_t best = 0;
        for (int32_t u = 0; u < n && !rc; u++) {
            if (s.is_seed[u] || s.is_blocked[u]) continue;
            uint64_t su = 0;
            rc = spread_of_set(&g, seeds, ns, &u, 1, key, (uint32_t)i, r, &s, &su);
            const uint64_t dec = base - su;  /* blocking u never adds reached vertices */
            if (!rc && (x == -1 || dec > best)) {
                x = u;
                best = dec;
            }
        }
        if (rc || x == -1) break;
        out_blockers[count++] = x;
        s.is_blocked[x] = 1;
    }
    *out_count = count;
    state_free(&s);
    free(lo);
    return rc;
}

ORACLE_API int oracle_exact(int32_t n, int64_t m, const int32_t *row_ptr, const int32_t *col,
                            const uint32_t *thr, const int32_t *seeds, int32_t ns, int32_t b, uint32_t r,
                            uint64_t key, int32_t *out_blockers, int32_t *out_count, int32_t model)
{
    graph_t g = {n, m, row_ptr, col, thr, NULL};
    uint32_t *lo = NULL;
    if (b < 0 || r == 0 || graph_model(&g, model, &lo)) return -1;
    state_t s;
    if (state_init(&s, n)) {
        free(lo);
        return -1;
    }
    int rc = validate(&g, seeds, ns, NULL, 0, &s);
    int32_t *cand = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t *idx = (int32_t *)malloc(sizeof(int32_t) * ((size_t)b + 1));
    int32_t *set = (int32_t *)malloc(sizeof(int32_t) * ((size_t)b + 1));
    if (!cand || !idx || !set) rc = -1;
    int32_t c = 0, k = 0;
    if (!rc) {
        for (int32_t u = 0; u < n; u++)
            if (!s.is_seed[u]) cand[c++] = u;
        k = b < c ? b : c;
        for (int32_t i = 0; i < k; i++) idx[i] = i;
        uint64_t best = 0;
        int have = 0;
        for (;;) {  /* k-subsets of cand in lexicographic order of their index vectors */
            for (int32_t i = 0; i < k; i++) set[i] = cand[idx[i]];
            uint64_t sp = 0;
            rc = spread_of_set(&g, seeds, ns, set, k, key, 0, r, &s, &sp);
            if (rc) break;
            if (!have || sp < best) {
                have = 1;
                best = sp;
                for (int32_t i = 0; i < k; i++) out_blockers[i] = set[i];
            }
            int32_t i = k - 1;
            while (i >= 0 && idx[i] == c - k + i) i--;
            if (i < 0) break;
            idx[i]++;
            for (int32_t t = i + 1; t < k; t++) idx[t] = idx[t - 1] + 1;
        }
    }
    *out_count = rc ? 0 : k;
    free(cand);
    free(idx);
    free(set);
    state_free(&s);
    free(lo);
    return rc;
}

ORACLE_API int oracle_out_degree(int32_t n, const int32_t *row_ptr, const int32_t *seeds, int32_t ns,
                                 int32_t b, int32_t *out_blockers, int32_t *out_count)
{
    if (n <= 0 || b < 0 || ns < 0) return -1;
    uint8_t *taken = (uint8_t *)calloc((size_t)n, 1);
    if (!taken) return -1;
    for (int32_t i = 0; i < ns; i++) {
        if (seeds[i] < 0 || seeds[i] >= n || taken[seeds[i]]) {
            free(taken);
            return -1;
        }
        taken[seeds[i]] = 1;
    }
    int32_t count = 0;
    for (; count < b; count++) {  /* b selection passes: the largest remaining out-degree */
        int32_t x = -1;
        for (int32_t u = 0; u < n; u++)
            if (!taken[u] && (x == -1 || row_ptr[u + 1] - row_ptr[u] > row_ptr[x + 1] - row_ptr[x])) x = u;
        if (x == -1) break;
        out_blockers[count] = x;
        taken[x] = 1;
    }
    *out_count = count;
    free(taken);
    return 0;
}

ORACLE_API int oracle_random_blockers(int32_t n, const int32_t *seeds, int32_t ns, int32_t b, uint64_t key,
                                      int32_t *out_blockers, int32_t *out_count)
{
    if (n <= 0 || b < 0 || ns < 0) return -1;
    uint8_t *is_seed = (uint8_t *)calloc((size_t)n, 1);
    int32_t *cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!is_seed || !cand) {
        free(is_seed);
        free(cand);
        return -1;
    }
    int rc = 0;
    for (int32_t i = 0; i < ns && !rc; i++) {
        if (seeds[i] < 0 || seeds[i] >= n || is_seed[seeds[i]]) rc = -1;
        else is_seed[seeds[i]] = 1;
    }
    int32_t c = 0;
    for (int32_t u = 0; u < n && !rc; u++)
        if (!is_seed[u]) cand[c++] = u;
    const int32_t k = rc ? 0 : (b < c ? b : c);
    const uint32_t kk[2] = {(uint32_t)key, (uint32_t)(key >> 32)};
    for (int32_t t = 0; t < k; t++) {
        const uint32_t ctr[4] = {(uint32_t)t, 0, 0, 0xC0000000u};
        uint32_t w[4];
        oracle_philox4x32_10(ctr, kk, w);
        const int32_t pick = t + (int32_t)(((uint64_t)w[0] * (uint64_t)(c - t)) >> 32);
        const int32_t tmp = cand[t];
        cand[t] = cand[pick];
        cand[pick] = tmp;
        out_blockers[t] = cand[t];
    }
    *out_count = k;
    free(is_seed);
    free(cand);
    return rc;
}
