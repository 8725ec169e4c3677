/*
 * rmat_oracle.c -- scalar CPU oracle for the alias-path R-MAT generator
 * (Huebschle-Schneider & Sanders, arXiv 1905.03525).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the product path.  It is written to
 * be read against the paper, not to be fast: one edge at a time, one level at
 * a time, FP64 for probabilities and exact integers everywhere else.
 *
 * Readings of the paper that the code follows (the paper is silent or
 * garbled on these points; the CUDA library makes the same choices):
 *   R1  stop rule of the table-construction fragment: expand while
 *       |Q| + 3 < bound (this reproduces the table sizes of Fig. 1:
 *       bound 2^12 -> 4093 entries).
 *   R2  ties in deleteMax: larger p first, then the lexicographically
 *       smaller symbol string.
 *   R3  entries whose path already has min(k, 32) levels are not expanded.
 *   R4  canonical entry order = lexicographic order of the symbol strings;
 *       the table is padded with zero-probability entries to N = 2^b.
 *   R5  p -> u32 weights w with sum 2^32: floor(p 2^32), remainder to the
 *       largest fractional parts (ties to the lower index).
 *   R6  integer Vose alias table with FIFO small/large lists.
 *   R7  one 32-bit Philox word per draw: top b bits = column, low 32-b bits
 *       compared with the column threshold.
 *   R8  bits left over after k levels are dropped (the sampling-loop fragment
 *       carries them to the next edge; keying the stream per edge makes every
 *       edge independent of the others instead).
 *   R9  the four parameters are divided by their sum before use.
 */
#include "rmat_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11).  Round: two 32x32->64 products of the even     */
/* counter words with the round multipliers; the new words are the high     */
/* halves xored with the odd words and the round key, and the low halves.   */
/* The key is bumped by the Weyl constants between rounds.                  */
/* ------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

uint32_t orc_word(uint64_t seed, uint64_t e, uint64_t n)
{
    uint64_t q = n / 4;
    uint32_t ctr[4] = {(uint32_t)q, (uint32_t)(q >> 32), (uint32_t)e, (uint32_t)(e >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[n % 4];
}

/* ------------------------------------------------------------------ */
/* Tables                                                              */
/* ------------------------------------------------------------------ */
struct orc_table {
    int entries;    /* |Q| */
    int bits;       /* b, N = 2^b */
    int max_len;
    uint64_t *sym;  /* N symbol strings, first level in bits 63..62 */
    uint8_t *len;   /* N path lengths (levels) */
    double *p;      /* N path probabilities */
    uint64_t *w;    /* N quantised weights, sum 2^32 */
    uint32_t *thr;  /* N alias thresholds */
    uint32_t *alias;/* N alias targets */
};

static int symbol_at(uint64_t sym, int t) { return (int)((sym >> (62 - 2 * t)) & 3u); }

static int normalise(const double in[4], double out[4])
{
    for (int i = 0; i < 4; ++i)
        if (!(in[i] >= 0.0) || !isfinite(in[i])) return -1;
    double s = ((in[0] + in[1]) + in[2]) + in[3];
    if (!(fabs(s - 1.0) <= 1e-9)) return -1;
    for (int i = 0; i < 4; ++i) out[i] = in[i] / s;
    return 0;
}

/* Entry of Q while the table-construction fragment runs. */
typedef struct { double p; uint64_t sym; int len; } qentry;

/* Is x to be expanded before y?  Larger p first; equal p: lexicographically
 * smaller symbol string first (reading R2).  Entries of Q never are prefixes
 * of each other, so comparing the left-aligned strings is lexicographic. */
static int q_before(const qentry *x, const qentry *y)
{
    if (x->p != y->p) return x->p > y->p;
    return x->sym < y->sym;
}

/* Binary max-heap on q_before. */
typedef struct { qentry *v; size_t n, cap; } qheap;

static int heap_push(qheap *h, qentry e)
{
    if (h->n == h->cap) {
        size_t nc = h->cap ? 2 * h->cap : 64;
        qentry *nv = (qentry *)realloc(h->v, nc * sizeof(qentry));
        if (!nv) return -1;
        h->v = nv; h->cap = nc;
    }
    size_t i = h->n++;
    h->v[i] = e;
    while (i > 0) {
        size_t parent = (i - 1) / 2;
        if (!q_before(&h->v[i], &h->v[parent])) break;
        qentry tmp = h->v[i]; h->v[i] = h->v[parent]; h->v[parent] = tmp;
        i = parent;
    }
    return 0;
}

static qentry heap_pop(qheap *h)
{
    qentry top = h->v[0];
    h->v[0] = h->v[--h->n];
    size_t i = 0;
    for (;;) {
        size_t l = 2 * i + 1, r = l + 1, best = i;
        if (l < h->n && q_before(&h->v[l], &h->v[best])) best = l;
        if (r < h->n && q_before(&h->v[r], &h->v[best])) best = r;
        if (best == i) break;
        qentry tmp = h->v[i]; h->v[i] = h->v[best]; h->v[best] = tmp;
        i = best;
    }
    return top;
}

static int cmp_sym(const void *x, const void *y)
{
    const qentry *a = (const qentry *)x, *b = (const qentry *)y;
    return (a->sym > b->sym) - (a->sym < b->sym);
}

/* Sort key for the largest-remainder step: fractional part desc, index asc. */
typedef struct { double frac; int idx; } fracidx;

static int cmp_frac(const void *x, const void *y)
{
    const fracidx *a = (const fracidx *)x, *b = (const fracidx *)y;
    if (a->frac != b->frac) return (a->frac < b->frac) - (a->frac > b->frac);
    return (a->idx > b->idx) - (a->idx < b->idx);
}

static orc_table *table_alloc(int entries)
{
    int bits = 0;
    while ((1LL << bits) < entries) ++bits;
    if (bits < 1) bits = 1;
    size_t N = (size_t)1 << bits;
    orc_table *t = (orc_table *)calloc(1, sizeof(orc_table));
    if (!t) return NULL;
    t->entries = entries;
    t->bits = bits;
    t->sym = (uint64_t *)calloc(N, sizeof(uint64_t));
    t->len = (uint8_t *)calloc(N, sizeof(uint8_t));
    t->p = (double *)calloc(N, sizeof(double));
    t->w = (uint64_t *)calloc(N, sizeof(uint64_t));
    t->thr = (uint32_t *)calloc(N, sizeof(uint32_t));
    t->alias = (uint32_t *)calloc(N, sizeof(uint32_t));
    if (!t->sym || !t->len || !t->p || !t->w || !t->thr || !t->alias) {
        orc_table_free(t);
        return NULL;
    }
    return t;
}

/* Quantisation (reading R5) and integer Vose alias construction (R6,
 * Walker's alias method as used in Sec. 2). */
static int quantise_and_alias(orc_table *t)
{
    int N = 1 << t->bits;
    uint64_t C = (uint64_t)1 << (32 - t->bits);
    const uint64_t total = (uint64_t)1 << 32;

    /* w_i = floor(p_i 2^32); the scaling by 2^32 is exact in FP64. */
    uint64_t sum = 0;
    fracidx *fr = (fracidx *)malloc((size_t)N * sizeof(fracidx));
    if (!fr) return -1;
    for (int i = 0; i < N; ++i) {
        double x = ldexp(t->p[i], 32);
        double fl = floor(x);
        t->w[i] = (uint64_t)fl;
        fr[i].frac = x - fl;
        fr[i].idx = i;
        sum += t->w[i];
    }
    if (sum > total) { free(fr); return -1; }
    uint64_t delta = total - sum;
    if (delta > (uint64_t)N) { free(fr); return -1; }
    qsort(fr, (size_t)N, sizeof(fracidx), cmp_frac);
    for (uint64_t r = 0; r < delta; ++r) t->w[fr[r].idx] += 1;
    free(fr);

    /* Vose: small = {i : w_i < C}, large = {i : w_i >= C}, both FIFO in
     * ascending index order. */
    uint64_t *rest = (uint64_t *)malloc((size_t)N * sizeof(uint64_t));
    int *small = (int *)malloc((size_t)N * sizeof(int));
    int *large = (int *)malloc((size_t)N * sizeof(int));
    if (!rest || !small || !large) { free(rest); free(small); free(large); return -1; }
    int s_head = 0, s_tail = 0, l_head = 0, l_tail = 0;
    for (int i = 0; i < N; ++i) {
        rest[i] = t->w[i];
        if (rest[i] < C) small[s_tail++] = i;
        else large[l_tail++] = i;
    }
    while (s_head < s_tail && l_head < l_tail) {
        int s = small[s_head++];
        int l = large[l_head];
        t->thr[s] = (uint32_t)rest[s];
        t->alias[s] = (uint32_t)l;
        rest[l] -= C - rest[s];
        if (rest[l] < C) {
            l_head++;
            small[s_tail++] = l;   /* each index enters small at most once */
        }
    }
    int ok = (s_head == s_tail);
    while (l_head < l_tail) {
        int l = large[l_head++];
        t->thr[l] = (uint32_t)(C - 1);
        t->alias[l] = (uint32_t)l;
    }
    free(rest); free(small); free(large);
    return ok ? 0 : -1;
}

orc_table *orc_table_variable(double a, double b, double c, double d, int k, uint64_t bound)
{
    double in[4] = {a, b, c, d}, P[4];
    if (normalise(in, P) != 0) return NULL;
    if (k < 1 || k > 64 || bound < 5 || bound > ((uint64_t)1 << 24)) return NULL;
    int cap = k < 32 ? k : 32;

    /* Q starts as the empty path with probability 1.  Entries that reached
     * the depth cap leave the heap for `done` (reading R3). */
    qheap heap = {0};
    qentry *done = (qentry *)malloc((size_t)bound * sizeof(qentry));
    if (!done) return NULL;
    size_t ndone = 0;
    qentry root = {1.0, 0, 0};
    if (heap_push(&heap, root) != 0) { free(done); return NULL; }
    /* Reading R1: expand while |Q| + 3 < bound. */
    while (heap.n > 0 && heap.n + ndone + 3 < bound) {
        qentry e = heap_pop(&heap);
        for (int s = 0; s < 4; ++s) {
            qentry child;
            child.p = e.p * P[s];
            child.len = e.len + 1;
            child.sym = e.sym | ((uint64_t)s << (62 - 2 * e.len));
            if (child.len >= cap) done[ndone++] = child;
            else if (heap_push(&heap, child) != 0) { free(heap.v); free(done); return NULL; }
        }
    }
    int entries = (int)(heap.n + ndone);
    qentry *all = (qentry *)malloc((size_t)entries * sizeof(qentry));
    if (!all) { free(heap.v); free(done); return NULL; }
    memcpy(all, done, ndone * sizeof(qentry));
    memcpy(all + ndone, heap.v, heap.n * sizeof(qentry));
    free(heap.v); free(done);

    /* Reading R4: lexicographic order of the symbol strings. */
    qsort(all, (size_t)entries, sizeof(qentry), cmp_sym);

    orc_table *t = table_alloc(entries);
    if (!t) { free(all); return NULL; }
    for (int i = 0; i < entries; ++i) {
        t->sym[i] = all[i].sym;
        t->len[i] = (uint8_t)all[i].len;
        t->p[i] = all[i].p;
        if (all[i].len > t->max_len) t->max_len = all[i].len;
    }
    free(all);
    if (quantise_and_alias(t) != 0) { orc_table_free(t); return NULL; }
    return t;
}

orc_table *orc_table_fixed(const double *Pin, int ell)
{
    if (ell < 1 || ell > 12) return NULL;
    double *P = (double *)malloc((size_t)ell * 4 * sizeof(double));
    if (!P) return NULL;
    for (int t = 0; t < ell; ++t)
        if (normalise(Pin + 4 * t, P + 4 * t) != 0) { free(P); return NULL; }
    int entries = 1 << (2 * ell);
    orc_table *t = table_alloc(entries);
    if (!t) { free(P); return NULL; }
    t->max_len = ell;
    /* Entry i is the path whose symbols are the base-4 digits of i, first
     * level = most significant digit; p is the product of the level
     * parameters taken from the top level down. */
    for (int i = 0; i < entries; ++i) {
        uint64_t sym = 0;
        double p = 1.0;
        for (int lvl = 0; lvl < ell; ++lvl) {
            int s = (i >> (2 * (ell - 1 - lvl))) & 3;
            sym |= (uint64_t)s << (62 - 2 * lvl);
            p = p * P[4 * lvl + s];
        }
        t->sym[i] = sym;
        t->len[i] = (uint8_t)ell;
        t->p[i] = p;
    }
    free(P);
    if (quantise_and_alias(t) != 0) { orc_table_free(t); return NULL; }
    return t;
}

void orc_table_free(orc_table *t)
{
    if (!t) return;
    free(t->sym); free(t->len); free(t->p); free(t->w); free(t->thr); free(t->alias);
    free(t);
}

int orc_table_entries(const orc_table *t) { return t->entries; }
int orc_table_bits(const orc_table *t) { return t->bits; }
int orc_table_max_len(const orc_table *t) { return t->max_len; }

void orc_table_get(const orc_table *t, uint64_t *sym, uint8_t *len, double *p,
                   uint64_t *w, uint32_t *thr, uint32_t *alias)
{
    size_t N = (size_t)1 << t->bits;
    if (sym) memcpy(sym, t->sym, N * sizeof(uint64_t));
    if (len) memcpy(len, t->len, N * sizeof(uint8_t));
    if (p) memcpy(p, t->p, N * sizeof(double));
    if (w) memcpy(w, t->w, N * sizeof(uint64_t));
    if (thr) memcpy(thr, t->thr, N * sizeof(uint32_t));
    if (alias) memcpy(alias, t->alias, N * sizeof(uint32_t));
}

/* Reading R7: column j = top b bits of the word, residual r = the other bits;
 * the column's own entry if r < thr[j], else its alias. */
uint32_t orc_draw(const orc_table *t, uint32_t u)
{
    uint32_t j = t->bits == 32 ? u : (u >> (32 - t->bits));
    uint32_t r = u & (uint32_t)((((uint64_t)1) << (32 - t->bits)) - 1);
    return r < t->thr[j] ? j : t->alias[j];
}

/* ------------------------------------------------------------------ */
/* Sampling loop (Sec. 2 sampling-loop fragment, with reading R8)      */
/* ------------------------------------------------------------------ */
static uint64_t splitmix64_next(uint64_t *state)
{
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void orc_scramble_constants(uint64_t scramble_seed, int k, uint64_t out[6])
{
    uint64_t mask = k >= 64 ? ~0ull : ((1ull << k) - 1);
    uint64_t st = scramble_seed;
    for (int i = 0; i < 3; ++i) {
        out[2 * i] = (splitmix64_next(&st) | 1ull) & mask;
        out[2 * i + 1] = splitmix64_next(&st) & mask;
    }
}

uint64_t orc_scramble(uint64_t x, int k, const uint64_t c[6])
{
    uint64_t mask = k >= 64 ? ~0ull : ((1ull << k) - 1);
    int h = (k + 1) / 2;
    for (int i = 0; i < 3; ++i) {
        x ^= x >> h;
        x = (x * c[2 * i] + c[2 * i + 1]) & mask;
    }
    return x;
}

/* The sampling loop.  The edge starts with pre_len levels already fixed
 * (row and column prefixes pre_r, pre_c: the tile of a partitioned graph;
 * pre_len = 0 for a whole graph) and draws the remaining levels. */
static int gen_core(const orc_table *const *tables, int ngroups, int k, int undirected,
                    const uint64_t *consts, uint64_t seed, uint64_t e0, uint64_t count,
                    uint64_t pre_r, uint64_t pre_c, int pre_len, uint64_t *row, uint64_t *col)
{
    if (ngroups < 1 || k < 1 || k > 64 || pre_len < 0 || pre_len > k) return -1;
    if (ngroups > 1) {
        int sum = 0;
        for (int g = 0; g < ngroups; ++g) sum += tables[g]->max_len;
        if (sum != k || pre_len != 0) return -1;
    }
    for (uint64_t i = 0; i < count; ++i) {
        uint64_t e = e0 + i;
        uint64_t r = pre_r, c = pre_c;
        int filled = pre_len;
        uint64_t n = 0;
        while (filled < k) {
            const orc_table *t = tables[ngroups > 1 ? n : 0];
            uint32_t u = orc_word(seed, e, n);
            n++;
            uint32_t sel = orc_draw(t, u);
            int L = t->len[sel];
            int take = L < k - filled ? L : k - filled;
            for (int lvl = 0; lvl < take; ++lvl) {
                int s = symbol_at(t->sym[sel], lvl);
                r = (r << 1) | (uint64_t)(s >> 1);
                c = (c << 1) | (uint64_t)(s & 1);
            }
            filled += take;
        }
        if (consts) {
            r = orc_scramble(r, k, consts);
            c = orc_scramble(c, k, consts);
        }
        if (undirected && r > c) { uint64_t tmp = r; r = c; c = tmp; }
        row[i] = r;
        col[i] = c;
    }
    return 0;
}

int orc_generate_scrambled(const orc_table *const *tables, int ngroups, int k, int undirected,
                           const uint64_t *consts, uint64_t seed, uint64_t e0, uint64_t count,
                           uint64_t *row, uint64_t *col)
{
    return gen_core(tables, ngroups, k, undirected, consts, seed, e0, count, 0, 0, 0, row, col);
}

int orc_generate(const orc_table *const *tables, int ngroups, int k, int undirected,
                 uint64_t seed, uint64_t e0, uint64_t count, uint64_t *row, uint64_t *col)
{
    return orc_generate_scrambled(tables, ngroups, k, undirected, NULL, seed, e0, count, row, col);
}

/* ------------------------------------------------------------------ */
/* Stochastic Kronecker graphs with an n0 x n0 initiator (Sec. 3: a    */
/* larger matrix instead of the 2 x 2 one in the recursion).  Symbol   */
/* s = n0 * i + j selects initiator cell (i, j), i.e. row digit i and  */
/* column digit j of the level; a path is a sequence of symbols.       */
/* ------------------------------------------------------------------ */
#define KRON_MAX_DEPTH 40

struct orc_ktable {
    int n0, cap;
    orc_table *base;   /* len, p, w, thr, alias, entries, bits, max_len */
    uint8_t *sym;      /* N x KRON_MAX_DEPTH symbols, first level first */
};

typedef struct { double p; int len; uint8_t sym[KRON_MAX_DEPTH]; } kentry;

/* Larger p first; equal p: lexicographically smaller symbol sequence first
 * (readings R2 and R16). */
static int k_before(const kentry *x, const kentry *y)
{
    if (x->p != y->p) return x->p > y->p;
    int n = x->len < y->len ? x->len : y->len;
    for (int i = 0; i < n; ++i)
        if (x->sym[i] != y->sym[i]) return x->sym[i] < y->sym[i];
    return x->len < y->len;
}

static int cmp_ksym(const void *a, const void *b)
{
    const kentry *x = (const kentry *)a, *y = (const kentry *)b;
    int n = x->len < y->len ? x->len : y->len;
    for (int i = 0; i < n; ++i)
        if (x->sym[i] != y->sym[i]) return x->sym[i] < y->sym[i] ? -1 : 1;
    return (x->len > y->len) - (x->len < y->len);
}

/* Plain array heap on k_before (sift up / sift down). */
typedef struct { kentry *v; size_t n, cap; } kheap;

static int kheap_push(kheap *h, const kentry *e)
{
    if (h->n == h->cap) {
        size_t nc = h->cap ? 2 * h->cap : 64;
        kentry *nv = (kentry *)realloc(h->v, nc * sizeof(kentry));
        if (!nv) return -1;
        h->v = nv; h->cap = nc;
    }
    size_t i = h->n++;
    h->v[i] = *e;
    while (i > 0) {
        size_t parent = (i - 1) / 2;
        if (!k_before(&h->v[i], &h->v[parent])) break;
        kentry tmp = h->v[i]; h->v[i] = h->v[parent]; h->v[parent] = tmp;
        i = parent;
    }
    return 0;
}

static kentry kheap_pop(kheap *h)
{
    kentry top = h->v[0];
    h->v[0] = h->v[--h->n];
    size_t i = 0;
    for (;;) {
        size_t l = 2 * i + 1, r = l + 1, best = i;
        if (l < h->n && k_before(&h->v[l], &h->v[best])) best = l;
        if (r < h->n && k_before(&h->v[r], &h->v[best])) best = r;
        if (best == i) break;
        kentry tmp = h->v[i]; h->v[i] = h->v[best]; h->v[best] = tmp;
        i = best;
    }
    return top;
}

/* Depth cap: the longest path whose row (or column) digits stay below 2^32,
 * i.e. the largest L with n0^L <= 2^32 (32 for n0 = 2), and at most k. */
static int kron_cap(int n0, int k)
{
    int L = 0;
    double v = 1.0;
    while (v * n0 <= 4294967296.0) { v *= n0; ++L; }
    return k < L ? k : L;
}

static int kron_normalise(const double *theta, int n0, double *out)
{
    int S = n0 * n0;
    double s = 0.0;
    for (int i = 0; i < S; ++i) {
        if (!(theta[i] >= 0.0) || !isfinite(theta[i])) return -1;
        s = s + theta[i];
    }
    if (!(fabs(s - 1.0) <= 1e-9)) return -1;
    for (int i = 0; i < S; ++i) out[i] = theta[i] / s;
    return 0;
}

/* Largest k with n0^k <= 2^64. */
static int kron_max_k(int n0)
{
    int k = 0;
    double v = 1.0;
    while (v * n0 <= 18446744073709551616.0) { v *= n0; ++k; }
    return k;
}

static orc_ktable *ktable_from(kentry *all, int entries, int n0, int cap)
{
    orc_ktable *t = (orc_ktable *)calloc(1, sizeof(orc_ktable));
    if (!t) return NULL;
    t->n0 = n0;
    t->cap = cap;
    t->base = table_alloc(entries);
    if (!t->base) { free(t); return NULL; }
    size_t N = (size_t)1 << t->base->bits;
    t->sym = (uint8_t *)calloc(N * KRON_MAX_DEPTH, 1);
    if (!t->sym) { orc_table_free(t->base); free(t); return NULL; }
    for (int i = 0; i < entries; ++i) {
        t->base->len[i] = (uint8_t)all[i].len;
        t->base->p[i] = all[i].p;
        memcpy(t->sym + (size_t)i * KRON_MAX_DEPTH, all[i].sym, (size_t)all[i].len);
        if (all[i].len > t->base->max_len) t->base->max_len = all[i].len;
    }
    if (quantise_and_alias(t->base) != 0) { orc_kron_table_free(t); return NULL; }
    return t;
}

orc_ktable *orc_kron_table_variable(const double *theta, int n0, int k, uint64_t bound)
{
    if (n0 < 2 || n0 > 16) return NULL;
    const int S = n0 * n0;
    if (k < 1 || k > kron_max_k(n0) || bound < (uint64_t)S + 1 || bound > ((uint64_t)1 << 24)) return NULL;
    double P[256];
    if (kron_normalise(theta, n0, P) != 0) return NULL;
    const int cap = kron_cap(n0, k);

    kheap heap = {0};
    kentry *done = (kentry *)malloc((size_t)bound * sizeof(kentry));
    if (!done) return NULL;
    size_t ndone = 0;
    kentry root;
    memset(&root, 0, sizeof root);
    root.p = 1.0;
    if (kheap_push(&heap, &root) != 0) { free(done); return NULL; }
    /* Reading R16: expand while |Q| + n0^2 - 1 < bound (R1 for n0 = 2). */
    while (heap.n > 0 && heap.n + ndone + (size_t)(S - 1) < bound) {
        kentry e = kheap_pop(&heap);
        for (int s = 0; s < S; ++s) {
            kentry child = e;
            child.p = e.p * P[s];
            child.sym[e.len] = (uint8_t)s;
            child.len = e.len + 1;
            if (child.len >= cap) done[ndone++] = child;
            else if (kheap_push(&heap, &child) != 0) { free(heap.v); free(done); return NULL; }
        }
    }
    int entries = (int)(heap.n + ndone);
    kentry *all = (kentry *)malloc((size_t)entries * sizeof(kentry));
    if (!all) { free(heap.v); free(done); return NULL; }
    memcpy(all, done, ndone * sizeof(kentry));
    memcpy(all + ndone, heap.v, heap.n * sizeof(kentry));
    free(heap.v); free(done);
    qsort(all, (size_t)entries, sizeof(kentry), cmp_ksym);   /* reading R4 */
    orc_ktable *t = ktable_from(all, entries, n0, cap);
    free(all);
    return t;
}

orc_ktable *orc_kron_table_fixed(const double *theta, int n0, int ell)
{
    if (n0 < 2 || n0 > 16 || ell < 1) return NULL;
    const int S = n0 * n0;
    double entries_d = 1.0;
    for (int i = 0; i < ell; ++i) entries_d *= S;
    if (entries_d > (double)(1 << 24) || ell > kron_cap(n0, 64)) return NULL;
    double P[256];
    if (kron_normalise(theta, n0, P) != 0) return NULL;
    int entries = (int)entries_d;
    kentry *all = (kentry *)calloc((size_t)entries, sizeof(kentry));
    if (!all) return NULL;
    /* Entry i: symbols = the base-n0^2 digits of i, most significant first. */
    for (int i = 0; i < entries; ++i) {
        int x = i;
        for (int lvl = ell - 1; lvl >= 0; --lvl) { all[i].sym[lvl] = (uint8_t)(x % S); x /= S; }
        double p = 1.0;
        for (int lvl = 0; lvl < ell; ++lvl) p = p * P[all[i].sym[lvl]];
        all[i].p = p;
        all[i].len = ell;
    }
    orc_ktable *t = ktable_from(all, entries, n0, ell);
    free(all);
    return t;
}

void orc_kron_table_free(orc_ktable *t)
{
    if (!t) return;
    orc_table_free(t->base);
    free(t->sym);
    free(t);
}

int orc_kron_table_entries(const orc_ktable *t) { return t->base->entries; }
int orc_kron_table_bits(const orc_ktable *t) { return t->base->bits; }
int orc_kron_table_max_len(const orc_ktable *t) { return t->base->max_len; }

void orc_kron_table_get(const orc_ktable *t, uint8_t *sym, uint8_t *len, double *p,
                        uint64_t *w, uint32_t *thr, uint32_t *alias)
{
    size_t N = (size_t)1 << t->base->bits;
    int L = t->base->max_len;
    for (size_t i = 0; i < N; ++i)
        if (sym) memcpy(sym + i * (size_t)L, t->sym + i * KRON_MAX_DEPTH, (size_t)L);
    orc_table_get(t->base, NULL, len, p, w, thr, alias);
}

uint32_t orc_kron_draw(const orc_ktable *t, uint32_t u) { return orc_draw(t->base, u); }

int orc_kron_generate(const orc_ktable *t, int k, uint64_t seed, uint64_t e0, uint64_t count,
                      uint64_t *row, uint64_t *col)
{
    if (!t || k < 1 || k > kron_max_k(t->n0)) return -1;
    const uint64_t n0 = (uint64_t)t->n0;
    for (uint64_t i = 0; i < count; ++i) {
        uint64_t e = e0 + i, r = 0, c = 0, n = 0;
        int filled = 0;
        while (filled < k) {
            uint32_t sel = orc_draw(t->base, orc_word(seed, e, n));
            n++;
            int L = t->base->len[sel];
            int take = L < k - filled ? L : k - filled;
            for (int lvl = 0; lvl < take; ++lvl) {
                int s = t->sym[(size_t)sel * KRON_MAX_DEPTH + lvl];
                r = r * n0 + (uint64_t)(s / t->n0);
                c = c * n0 + (uint64_t)(s % t->n0);
            }
            filled += take;
        }
        row[i] = r;
        col[i] = c;
    }
    return 0;
}

static void kdist_rec(const orc_ktable *t, int k, int quantised, int filled, uint64_t r, uint64_t c,
                      double prob, uint64_t nv, double *out)
{
    if (filled >= k) { out[r * nv + c] += prob; return; }
    int N = 1 << t->base->bits;
    for (int j = 0; j < N; ++j) {
        double pj = quantised ? ldexp((double)t->base->w[j], -32) : t->base->p[j];
        if (pj == 0.0) continue;
        int L = t->base->len[j];
        int take = L < k - filled ? L : k - filled;
        uint64_t rr = r, cc = c;
        for (int lvl = 0; lvl < take; ++lvl) {
            int s = t->sym[(size_t)j * KRON_MAX_DEPTH + lvl];
            rr = rr * (uint64_t)t->n0 + (uint64_t)(s / t->n0);
            cc = cc * (uint64_t)t->n0 + (uint64_t)(s % t->n0);
        }
        kdist_rec(t, k, quantised, filled + take, rr, cc, prob * pj, nv, out);
    }
}

int orc_kron_edge_distribution(const orc_ktable *t, int k, int quantised, double *out)
{
    if (!t || k < 1) return -1;
    uint64_t nv = 1;
    for (int i = 0; i < k; ++i) nv *= (uint64_t)t->n0;
    if (nv > 4096) return -1;
    memset(out, 0, (size_t)(nv * nv) * sizeof(double));
    kdist_rec(t, k, quantised, 0, 0, 0, 1.0, nv, out);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Partitioned graphs (Sec. 3, communication-free generation of       */
/* partitioned graphs): a divide-and-conquer pass gives the number of */
/* edges in each of the 2^t x 2^t tiles of the adjacency matrix, then */
/* the sampling loop fills each tile's lower k - t levels.             */
/* ------------------------------------------------------------------ */

/* Word n of the stream of binomial j (0, 1, 2) at recursion node `node`
 * (= R * 2^depth + C) of depth `depth`.  Counter word 1 has its top bit set:
 * an edge's stream has the high half of its block index there, which is 0. */
uint32_t orc_partition_word(uint64_t seed, int depth, uint64_t node, int j, uint64_t n)
{
    uint32_t ctr[4] = {(uint32_t)(n / 4), 0x80000000u | ((uint32_t)j << 8) | (uint32_t)depth,
                       (uint32_t)node, (uint32_t)(node >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[n % 4];
}

typedef struct {
    uint64_t seed, node, n;
    int depth, j;
} ustream;

/* Uniform in (0, 1) from two words: x = 26 + 26 high bits, (x + 1/2) / 2^52
 * (exact in FP64). */
static double next_uniform(ustream *s)
{
    uint32_t w0 = orc_partition_word(s->seed, s->depth, s->node, s->j, s->n++);
    uint32_t w1 = orc_partition_word(s->seed, s->depth, s->node, s->j, s->n++);
    double x = (double)(w0 >> 6) * 67108864.0 + (double)(w1 >> 6);
    return (x + 0.5) * 0x1p-52;
}

/* Inversion by sequential search (n p < 10, p <= 1/2): walk the pmf from 0,
 * f(x) = f(x-1) * ((n+1) s / x - s) with s = p/q; a uniform that outruns the
 * rounded pmf restarts with a fresh uniform. */
static uint64_t binomial_inversion(uint64_t n, double p, ustream *s)
{
    const double q = 1.0 - p, sr = p / q, a = ((double)n + 1.0) * sr, f0 = pow(q, (double)n);
    for (;;) {
        double u = next_uniform(s), f = f0;
        uint64_t x = 0;
        while (u > f) {
            u -= f;
            x++;
            if (x > n) break;
            f *= a / (double)x - sr;
        }
        if (x <= n) return x;
    }
}

/* BTRS, transformed rejection with squeeze (W. Hoermann, "The generation of
 * binomial random variates", J. Statist. Comput. Simul. 46, 1993), for
 * n p >= 10, p <= 1/2.  The final test compares with the exact log pmf. */
static uint64_t binomial_btrs(uint64_t n, double p, ustream *s)
{
    const double q = 1.0 - p, nd = (double)n;
    const double spq = sqrt(nd * p * q);
    const double b = 1.15 + 2.53 * spq;
    const double a = -0.0873 + 0.0248 * b + 0.01 * p;
    const double c = nd * p + 0.5;
    const double vr = 0.92 - 4.2 / b;
    const double alpha = (2.83 + 5.1 / b) * spq;
    const double lpq = log(p / q);
    const double m = floor((nd + 1.0) * p);
    const double h = lgamma(m + 1.0) + lgamma(nd - m + 1.0);
    for (;;) {
        const double u = next_uniform(s) - 0.5;
        double v = next_uniform(s);
        const double us = 0.5 - fabs(u);
        const double x = floor((2.0 * a / us + b) * u + c);
        if (x < 0.0 || x > nd) continue;
        if (us >= 0.07 && v <= vr) return (uint64_t)x;
        v = log(v * alpha / (a / (us * us) + b));
        if (v <= h - lgamma(x + 1.0) - lgamma(nd - x + 1.0) + (x - m) * lpq) return (uint64_t)x;
    }
}

uint64_t orc_binomial(uint64_t n, double p, uint64_t seed, int depth, uint64_t node, int j)
{
    ustream s = {seed, node, 0, depth, j};
    if (n == 0 || !(p > 0.0)) return 0;
    if (p >= 1.0) return n;
    const int flip = p > 0.5;
    const double pp = flip ? 1.0 - p : p;
    const uint64_t x = (double)n * pp < 10.0 ? binomial_inversion(n, pp, &s) : binomial_btrs(n, pp, &s);
    return flip ? n - x : x;
}

typedef struct {
    double P[4];
    int t;
    uint64_t seed, r0, r1, next, n, cap;
    uint64_t *tr, *tc, *cnt, *first;
} part_ctx;

/* Node (depth, R, C) holds `count` edges.  Nodes outside the tile rows
 * [r0, r1) are not split; their edges only advance the edge numbering. */
static void part_rec(part_ctx *x, int depth, uint64_t R, uint64_t C, uint64_t count)
{
    if (count == 0) return;
    const int below = x->t - depth;
    const uint64_t lo = R << below, hi = (R + 1) << below;
    if (hi <= x->r0 || lo >= x->r1) {
        x->next += count;
        return;
    }
    if (below == 0) {
        if (x->n < x->cap) {
            x->tr[x->n] = R;
            x->tc[x->n] = C;
            x->cnt[x->n] = count;
            x->first[x->n] = x->next;
        }
        x->n++;
        x->next += count;
        return;
    }
    const uint64_t node = (R << depth) | C;
    const double *P = x->P;
    const double den_b = (P[1] + P[2]) + P[3], den_c = P[2] + P[3];
    const uint64_t na = orc_binomial(count, P[0], x->seed, depth, node, 0);
    const uint64_t nb = orc_binomial(count - na, den_b > 0.0 ? P[1] / den_b : 0.0, x->seed, depth, node, 1);
    const uint64_t nc = orc_binomial(count - na - nb, den_c > 0.0 ? P[2] / den_c : 0.0, x->seed, depth, node, 2);
    const uint64_t nd = count - na - nb - nc;
    part_rec(x, depth + 1, 2 * R, 2 * C, na);          /* a: upper left  */
    part_rec(x, depth + 1, 2 * R, 2 * C + 1, nb);      /* b: upper right */
    part_rec(x, depth + 1, 2 * R + 1, 2 * C, nc);      /* c: lower left  */
    part_rec(x, depth + 1, 2 * R + 1, 2 * C + 1, nd);  /* d: lower right */
}

int64_t orc_partition(double a, double b, double c, double d, int t, uint64_t m, uint64_t seed,
                      uint64_t row_tile_begin, uint64_t row_tile_end, uint64_t cap,
                      uint64_t *tile_row, uint64_t *tile_col, uint64_t *count, uint64_t *first)
{
    part_ctx x;
    const double in[4] = {a, b, c, d};
    if (t < 0 || t > 30 || normalise(in, x.P) != 0) return -1;
    if (row_tile_begin > row_tile_end || row_tile_end > ((uint64_t)1 << t)) return -1;
    if (cap && (!tile_row || !tile_col || !count || !first)) return -1;
    x.t = t;
    x.seed = seed;
    x.r0 = row_tile_begin;
    x.r1 = row_tile_end;
    x.next = 0;
    x.n = 0;
    x.cap = cap;
    x.tr = tile_row;
    x.tc = tile_col;
    x.cnt = count;
    x.first = first;
    part_rec(&x, 0, 0, 0, m);
    return (int64_t)x.n;
}

int orc_generate_tile(const orc_table *table, int k, int t, uint64_t tile_row, uint64_t tile_col,
                      uint64_t seed, uint64_t first, uint64_t count, uint64_t *row, uint64_t *col)
{
    if (t < 0 || t > k || (t < 64 && (tile_row >> t || tile_col >> t))) return -1;
    return gen_core(&table, 1, k, 0, NULL, seed, first, count, tile_row, tile_col, t, row, col);
}

/* Threshold round(x 2^32), saturated to 2^32 - 1. */
static uint32_t naive_threshold(double x)
{
    double v = floor(ldexp(x, 32) + 0.5);
    if (v >= 4294967295.0) return 0xFFFFFFFFu;
    if (v <= 0.0) return 0;
    return (uint32_t)v;
}

int orc_generate_naive(const double *Pin, int k, int undirected, uint64_t seed,
                       uint64_t e0, uint64_t count, uint64_t *row, uint64_t *col)
{
    if (k < 1 || k > 64) return -1;
    uint32_t *T = (uint32_t *)malloc((size_t)k * 3 * sizeof(uint32_t));
    if (!T) return -1;
    for (int lvl = 0; lvl < k; ++lvl) {
        double P[4];
        if (normalise(Pin + 4 * lvl, P) != 0) { free(T); return -1; }
        T[3 * lvl + 0] = naive_threshold(P[0]);
        T[3 * lvl + 1] = naive_threshold(P[0] + P[1]);
        T[3 * lvl + 2] = naive_threshold((P[0] + P[1]) + P[2]);
    }
    for (uint64_t i = 0; i < count; ++i) {
        uint64_t e = e0 + i;
        uint64_t r = 0, c = 0;
        for (int lvl = 0; lvl < k; ++lvl) {
            uint32_t u = orc_word(seed, e, (uint64_t)lvl);
            int s = (u >= T[3 * lvl]) + (u >= T[3 * lvl + 1]) + (u >= T[3 * lvl + 2]);
            r = (r << 1) | (uint64_t)(s >> 1);
            c = (c << 1) | (uint64_t)(s & 1);
        }
        if (undirected && r > c) { uint64_t tmp = r; r = c; c = tmp; }
        row[i] = r;
        col[i] = c;
    }
    free(T);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Exact edge distribution by enumeration of draw sequences            */
/* ------------------------------------------------------------------ */
static void dist_rec(const orc_table *const *tables, int ngroups, int k, int quantised,
                     int draw, int filled, uint64_t r, uint64_t c, double prob, double *out)
{
    if (filled >= k) {
        out[(r << k) | c] += prob;
        return;
    }
    const orc_table *t = tables[ngroups > 1 ? draw : 0];
    int N = 1 << t->bits;
    for (int i = 0; i < N; ++i) {
        double pi = quantised ? ldexp((double)t->w[i], -32) : t->p[i];
        if (pi == 0.0) continue;
        int L = t->len[i];
        int take = L < k - filled ? L : k - filled;
        uint64_t rr = r, cc = c;
        for (int lvl = 0; lvl < take; ++lvl) {
            int s = symbol_at(t->sym[i], lvl);
            rr = (rr << 1) | (uint64_t)(s >> 1);
            cc = (cc << 1) | (uint64_t)(s & 1);
        }
        dist_rec(tables, ngroups, k, quantised, draw + 1, filled + take, rr, cc, prob * pi, out);
    }
}

int orc_edge_distribution(const orc_table *const *tables, int ngroups, int k,
                          int quantised, double *out)
{
    if (k < 1 || k > 12 || ngroups < 1) return -1;
    memset(out, 0, sizeof(double) * ((size_t)1 << (2 * k)));
    dist_rec(tables, ngroups, k, quantised, 0, 0, 0, 0, 1.0, out);
    return 0;
}
