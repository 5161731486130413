/*
 * graphgen.c -- seeded synthetic directed graphs (input generation only; none of the method's
 * arithmetic lives here). Used through paper_2302_13529_gb300/workloads.py.
 *
 *   imin_gen_chung_lu: directed Chung-Lu graph with power-law expected degrees
 *   imin_gen_rmat:     R-MAT graph with quadrant probabilities (a, b, c, d)
 *
 * Both draw (source, target) pairs, reject self-loops and duplicates until exactly m distinct
 * edges exist (the first m distinct pairs in draw order), and return a CSR sorted by
 * (source, target).
 *
 * Random numbers: xoshiro256** (D. Blackman, S. Vigna, "Scrambled linear pseudorandom number
 * generators", ACM TOMS 2021) seeded through splitmix64 (G. L. Steele, D. Lea, C. H. Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014). Weighted sampling: Vose's
 * alias method (M. D. Vose, "A linear algorithm for generating random numbers with a given
 * distribution", IEEE TSE 1991).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GEN_API __attribute__((visibility("default")))

typedef struct {
    uint64_t s[4];
} rng_t;

static uint64_t splitmix64(uint64_t *x)
{
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void rng_seed(rng_t *r, uint64_t seed)
{
    uint64_t x = seed;
    for (int i = 0; i < 4; i++) r->s[i] = splitmix64(&x);
}

static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t rng_next(rng_t *r)
{
    const uint64_t out = rotl(r->s[1] * 5, 7) * 9;
    const uint64_t t = r->s[1] << 17;
    r->s[2] ^= r->s[0];
    r->s[3] ^= r->s[1];
    r->s[1] ^= r->s[2];
    r->s[0] ^= r->s[3];
    r->s[2] ^= t;
    r->s[3] = rotl(r->s[3], 45);
    return out;
}

static inline double rng_uniform(rng_t *r) { return (double)(rng_next(r) >> 11) * 0x1.0p-53; }

/* uniform integer in [0, n) by the multiply-shift reduction of a 32-bit word */
static inline uint32_t rng_below(uint32_t word, uint32_t n) { return (uint32_t)(((uint64_t)word * n) >> 32); }

/* ---- Vose alias table ------------------------------------------------------------------- */
typedef struct {
    int32_t n;
    double *prob;
    int32_t *alias;
} alias_t;

static int alias_build(alias_t *a, const double *w, int32_t n)
{
    a->n = n;
    a->prob = (double *)malloc(sizeof(double) * n);
    a->alias = (int32_t *)malloc(sizeof(int32_t) * n);
    double *p = (double *)malloc(sizeof(double) * n);
    int32_t *small = (int32_t *)malloc(sizeof(int32_t) * n);
    int32_t *large = (int32_t *)malloc(sizeof(int32_t) * n);
    if (!a->prob || !a->alias || !p || !small || !large) return -1;
    double sum = 0;
    for (int32_t i = 0; i < n; i++) sum += w[i];
    int32_t ns = 0, nl = 0;
    for (int32_t i = 0; i < n; i++) {
        p[i] = w[i] * n / sum;
        if (p[i] < 1.0) small[ns++] = i;
        else large[nl++] = i;
    }
    while (ns > 0 && nl > 0) {
        const int32_t l = small[--ns], g = large[--nl];
        a->prob[l] = p[l];
        a->alias[l] = g;
        p[g] = (p[g] + p[l]) - 1.0;
        if (p[g] < 1.0) small[ns++] = g;
        else large[nl++] = g;
    }
    while (nl > 0) {
        const int32_t g = large[--nl];
        a->prob[g] = 1.0;
        a->alias[g] = g;
    }
    while (ns > 0) {
        const int32_t l = small[--ns];
        a->prob[l] = 1.0;
        a->alias[l] = l;
    }
    free(p);
    free(small);
    free(large);
    return 0;
}

static inline int32_t alias_draw(const alias_t *a, rng_t *r)
{
    const uint64_t x = rng_next(r);
    const int32_t i = (int32_t)rng_below((uint32_t)(x >> 32), (uint32_t)a->n);
    const double u = (double)(x & 0xFFFFFFFFull) * 0x1.0p-32;
    return u < a->prob[i] ? i : a->alias[i];
}

static void alias_free(alias_t *a)
{
    free(a->prob);
    free(a->alias);
}

/* ---- distinct edge set ------------------------------------------------------------------ */
typedef struct {
    uint64_t *slot;
    uint64_t mask;
    int shift;
} hset_t;

static int hset_init(hset_t *h, int64_t m)
{
    uint64_t cap = 1;
    int bits = 0;
    while (cap < (uint64_t)(2 * m + 16)) {
        cap <<= 1;
        bits++;
    }
    h->slot = (uint64_t *)malloc(sizeof(uint64_t) * cap);
    if (!h->slot) return -1;
    memset(h->slot, 0xFF, sizeof(uint64_t) * cap);
    h->mask = cap - 1;
    h->shift = 64 - bits;
    return 0;
}

/* 1 if key was new */
static inline int hset_insert(hset_t *h, uint64_t key)
{
    uint64_t i = (key * 0x9E3779B97F4A7C15ull) >> h->shift;
    for (;;) {
        const uint64_t k = h->slot[i];
        if (k == key) return 0;
        if (k == UINT64_MAX) {
            h->slot[i] = key;
            return 1;
        }
        i = (i + 1) & h->mask;
    }
}

/* ---- keys (src * n + dst) -> CSR ------------------------------------------------------- */
static int keys_to_csr(uint64_t *keys, int64_t m, int32_t n, int32_t *row_ptr, int32_t *col)
{
    /* LSD radix sort, 16 bits per pass, over the bits a key can use */
    uint64_t maxkey = (uint64_t)n * (uint64_t)n;
    int passes = 0;
    while (passes < 4 && (maxkey >> (16 * passes)) != 0) passes++;
    uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * (m > 0 ? m : 1));
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * 65536);
    if (!tmp || !cnt) return -1;
    uint64_t *src = keys, *dst = tmp;
    for (int p = 0; p < passes; p++) {
        const int sh = 16 * p;
        memset(cnt, 0, sizeof(int64_t) * 65536);
        for (int64_t i = 0; i < m; i++) cnt[(src[i] >> sh) & 0xFFFF]++;
        int64_t run = 0;
        for (int b = 0; b < 65536; b++) {
            const int64_t c = cnt[b];
            cnt[b] = run;
            run += c;
        }
        for (int64_t i = 0; i < m; i++) dst[cnt[(src[i] >> sh) & 0xFFFF]++] = src[i];
        uint64_t *t = src;
        src = dst;
        dst = t;
    }
    memset(row_ptr, 0, sizeof(int32_t) * ((size_t)n + 1));
    for (int64_t i = 0; i < m; i++) {
        row_ptr[src[i] / (uint64_t)n + 1]++;
        col[i] = (int32_t)(src[i] % (uint64_t)n);
    }
    for (int32_t u = 0; u < n; u++) row_ptr[u + 1] += row_ptr[u];
    free(tmp);
    free(cnt);
    return 0;
}

static void permutation(int32_t *perm, int32_t n, rng_t *r)
{
    for (int32_t i = 0; i < n; i++) perm[i] = i;
    for (int32_t i = n - 1; i > 0; i--) {
        const int32_t j = (int32_t)rng_below((uint32_t)(rng_next(r) >> 32), (uint32_t)i + 1);
        const int32_t t = perm[i];
        perm[i] = perm[j];
        perm[j] = t;
    }
}

/* sum_{i=0}^{n-1} (i + x)^(-alpha): the first 4096 terms exactly, the smooth tail by its
 * midpoint integral (relative error far below what the offset needs). */
static double weight_sum(int32_t n, double x, double alpha)
{
    const int32_t head = n < 4096 ? n : 4096;
    double sum = 0;
    for (int32_t i = 0; i < head; i++) sum += pow(i + x, -alpha);
    if (head < n) {
        const double a = head - 0.5 + x, b = n - 0.5 + x;
        sum += (pow(b, 1.0 - alpha) - pow(a, 1.0 - alpha)) / (1.0 - alpha);
    }
    return sum;
}

/* Offset i0 of w_i = (i + i0)^(-1/(gamma-1)) such that the heaviest vertex expects about
 * dmax_frac * n edge endpoints (bisection on a log scale). */
static double chung_lu_offset(int32_t n, int64_t m, double gamma, double dmax_frac)
{
    const double alpha = 1.0 / (gamma - 1.0);
    double target = dmax_frac * n;
    if (target < (double)m / n) target = (double)m / n;
    double lo = 1e-3, hi = (double)n;
    for (int it = 0; it < 60; it++) {
        const double mid = sqrt(lo * hi);
        const double sum = weight_sum(n, mid, alpha);
        const double top = m * pow(mid, -alpha) / sum;
        if (top > target) lo = mid;
        else hi = mid;
    }
    return hi;
}

/* Directed Chung-Lu: out- and in-weights w_i = (i + i0)^(-1/(gamma-1)) assigned to vertices
 * by two independent random permutations; sources drawn proportionally to out-weights, targets
 * to in-weights. Returns 0, or -1 (out of memory / too dense). */
GEN_API int imin_gen_chung_lu(int32_t n, int64_t m, double gamma, double dmax_frac, uint64_t seed,
                              int32_t *row_ptr, int32_t *col)
{
    if (n < 2 || m < 0 || (double)m > 0.5 * (double)n * (double)(n - 1)) return -1;
    rng_t r;
    rng_seed(&r, seed);
    const double i0 = chung_lu_offset(n, m, gamma, dmax_frac);
    double *base = (double *)malloc(sizeof(double) * n);
    double *w = (double *)malloc(sizeof(double) * n);
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * n);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (m > 0 ? m : 1));
    hset_t h;
    alias_t aout, ain;
    if (!base || !w || !perm || !keys || hset_init(&h, m)) return -1;
    for (int32_t i = 0; i < n; i++) base[i] = pow(i + i0, -1.0 / (gamma - 1.0));
    permutation(perm, n, &r);
    for (int32_t i = 0; i < n; i++) w[perm[i]] = base[i];
    if (alias_build(&aout, w, n)) return -1;
    permutation(perm, n, &r);
    for (int32_t i = 0; i < n; i++) w[perm[i]] = base[i];
    if (alias_build(&ain, w, n)) return -1;
    int64_t got = 0, draws = 0;
    const int64_t max_draws = 64 * (m + 1024);
    while (got < m && draws < max_draws) {
        const int32_t s = alias_draw(&aout, &r), t = alias_draw(&ain, &r);
        draws++;
        if (s == t) continue;
        const uint64_t key = (uint64_t)s * (uint64_t)n + (uint64_t)t;
        if (hset_insert(&h, key)) keys[got++] = key;
    }
    int rc = got == m ? keys_to_csr(keys, m, n, row_ptr, col) : -1;
    free(base);
    free(w);
    free(perm);
    free(keys);
    free(h.slot);
    alias_free(&aout);
    alias_free(&ain);
    return rc;
}

/* R-MAT on n = 2^scale vertices: each edge descends `scale` levels, picking quadrant a / b / c /
 * d with the given probabilities (source bit set for c, d; target bit set for b, d); vertex ids
 * are then relabelled by a random permutation (raw R-MAT puts the hubs at low ids). */
GEN_API int imin_gen_rmat(int32_t scale, int64_t m, double a, double b, double c, uint64_t seed,
                          int32_t *row_ptr, int32_t *col)
{
    if (scale < 1 || scale > 30 || m < 0) return -1;
    const int32_t n = (int32_t)1 << scale;
    if ((double)m > 0.5 * (double)n * (double)(n - 1)) return -1;
    rng_t r;
    rng_seed(&r, seed);
    /* quadrant thresholds on a 32-bit uniform word: two levels per 64-bit draw */
    const uint64_t t1 = (uint64_t)(a * 4294967296.0), t2 = (uint64_t)((a + b) * 4294967296.0),
                   t3 = (uint64_t)((a + b + c) * 4294967296.0);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (m > 0 ? m : 1));
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * n);
    hset_t h;
    if (!keys || !perm || hset_init(&h, m)) return -1;
    int64_t got = 0, draws = 0;
    const int64_t max_draws = 64 * (m + 1024);
    while (got < m && draws < max_draws) {
        uint32_t s = 0, t = 0;
        uint64_t word = 0;
        for (int l = 0; l < scale; l++) {
            if ((l & 1) == 0) word = rng_next(&r);
            const uint64_t u = (l & 1) ? (word >> 32) : (word & 0xFFFFFFFFull);
            const uint32_t sb = u >= t2;
            const uint32_t tb = (u >= t1 && u < t2) || u >= t3;
            s = (s << 1) | sb;
            t = (t << 1) | tb;
        }
        draws++;
        if (s == t) continue;
        const uint64_t key = (uint64_t)s * (uint64_t)n + (uint64_t)t;
        if (hset_insert(&h, key)) keys[got++] = key;
    }
    int rc = -1;
    if (got == m) {
        permutation(perm, n, &r);
        for (int64_t i = 0; i < m; i++) {
            const uint64_t s = keys[i] / (uint64_t)n, t = keys[i] % (uint64_t)n;
            keys[i] = (uint64_t)perm[s] * (uint64_t)n + (uint64_t)perm[t];
        }
        rc = keys_to_csr(keys, m, n, row_ptr, col);
    }
    free(keys);
    free(perm);
    free(h.slot);
    return rc;
}
