/*
 * rmat_oracle.h -- plain, slow, scalar CPU oracle for the alias-path R-MAT
 * generator of Huebschle-Schneider & Sanders, "Linear Work Generation of R-MAT
 * Graphs" (arXiv 1905.03525).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code: only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code with the CUDA library.
 *
 * What it computes (paper section in brackets):
 *   - path probabilities of the R-MAT recursion, FP64 products      [Sec. 1, Sec. 2]
 *   - the variable-length table of similar-probability paths        [Sec. 2, table-construction fragment]
 *   - the fixed-length table of all 4^l paths                       [Sec. 2]
 *   - u32 quantisation + integer Walker/Vose alias table            [Sec. 2, Walker's alias method]
 *   - Philox4x32-10 word stream keyed by (seed, edge index)         [Salmon et al., SC'11]
 *   - the sampling loop: draw, concatenate path bits, cut at k      [Sec. 2, sampling-loop fragment]
 *   - undirected mirroring (min, max)                               [Sec. 3]
 *   - the naive per-bit R-MAT process (k quadrant draws per edge)   [Sec. 1]
 *   - exact edge distribution implied by a table, by enumeration    [Sec. 1 definition, for pins]
 *   - scrambling: seeded bijective relabelling of vertex IDs        [Sec. 3]
 *   - Kronecker initiators of size n0 x n0 (tables, generation)     [Sec. 3]
 *   - partitioned graphs: divide-and-conquer tile edge counts by    [Sec. 3]
 *     binomial splits (inversion; BTRS, Hoermann 1993), then the
 *     sampling loop inside each tile
 *
 * Conventions: symbol s = 2*rowbit + colbit, a->0, b->1, c->2, d->3 (Sec. 1:
 * a = upper-left, b = upper-right, c = lower-left, d = lower-right; the
 * table-construction fragment appends (0,0),(0,1),(1,0),(1,1) for a,b,c,d).
 * Level 0 is the top recursion level = most significant bit of row/column.
 */
#ifndef RMAT_ORACLE_H
#define RMAT_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_table orc_table;

/* Philox4x32-10 block function (Salmon, Moraes, Dror, Shaw, SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Word n (n = 0, 1, 2, ...) of the random stream of edge e under `seed`:
 * key = (seed lo, seed hi), counter = (q lo, q hi, e lo, e hi), q = n / 4,
 * and the word is output word n % 4 of that block. */
uint32_t orc_word(uint64_t seed, uint64_t e, uint64_t n);

/* Variable-length table (Sec. 2 table-construction fragment): repeated
 * expansion of the maximum-probability entry while |Q| + 3 < bound.
 * Depth cap min(k, 32).  NULL on invalid arguments. */
orc_table *orc_table_variable(double a, double b, double c, double d, int k, uint64_t bound);

/* Fixed-length table: all 4^ell paths of length ell, level t of a path using
 * the parameters P[4*t .. 4*t+3].  NULL on invalid arguments. */
orc_table *orc_table_fixed(const double *P, int ell);

void orc_table_free(orc_table *t);

int orc_table_entries(const orc_table *t); /* |Q| before padding */
int orc_table_bits(const orc_table *t);    /* b: padded size N = 2^b */
int orc_table_max_len(const orc_table *t);

/* Copy out the table, each array of length N = 2^b (padding entries at the
 * end have p = 0, len = 0).  sym: symbol string, 2 bits per level, first level
 * in the top bits of the 64-bit word.  Any pointer may be NULL. */
void orc_table_get(const orc_table *t, uint64_t *sym, uint8_t *len, double *p,
                   uint64_t *w, uint32_t *thr, uint32_t *alias);

/* One alias draw from 32-bit word u: index of the selected entry. */
uint32_t orc_draw(const orc_table *t, uint32_t u);

/* Generate edges e0 .. e0+count-1.  With ngroups == 1 every draw uses
 * tables[0]; with ngroups > 1 draw g uses tables[g] and the groups' lengths
 * must add up to k.  Returns 0, or -1 on invalid arguments. */
int orc_generate(const orc_table *const *tables, int ngroups, int k, int undirected,
                 uint64_t seed, uint64_t e0, uint64_t count, uint64_t *row, uint64_t *col);

/* Scrambling (Sec. 3: Graph 500 hides the structure by relabelling vertex IDs;
 * a constant-time post-processing).  pi is a bijection of [0, 2^k): three
 * rounds of x ^= x >> ceil(k/2); x = (x * m_i + a_i) mod 2^k, with odd m_i.
 * The constants come from the scramble seed through SplitMix64 (Steele, Lea,
 * Flood 2014): m_0, a_0, m_1, a_1, m_2, a_2 are its first six outputs, each
 * reduced mod 2^k, the m_i with their low bit set. */
void orc_scramble_constants(uint64_t scramble_seed, int k, uint64_t out[6]);
uint64_t orc_scramble(uint64_t x, int k, const uint64_t consts[6]);

/* orc_generate with optional scrambling (consts != NULL): both endpoints are
 * relabelled by pi before undirected mirroring. */
int orc_generate_scrambled(const orc_table *const *tables, int ngroups, int k, int undirected,
                           const uint64_t *consts, uint64_t seed, uint64_t e0, uint64_t count,
                           uint64_t *row, uint64_t *col);

/* Stochastic Kronecker graphs with an n0 x n0 initiator theta (Sec. 3: a
 * k x k matrix instead of the 2 x 2 one; n0 = 2..16, row-major theta summing
 * to 1).  Symbol s = n0 * i + j picks cell (i, j): row digit i, column digit
 * j of the level, in base n0.  Tables as for R-MAT with n0^2 children per
 * expansion: variable-length (expand while |Q| + n0^2 - 1 < bound, depth cap
 * min(k, largest L with n0^L <= 2^32)) or all (n0^2)^ell paths.  Generation
 * is the R-MAT sampling loop with base-n0 digits; n0^k <= 2^64. */
typedef struct orc_ktable orc_ktable;
orc_ktable *orc_kron_table_variable(const double *theta, int n0, int k, uint64_t bound);
orc_ktable *orc_kron_table_fixed(const double *theta, int n0, int ell);
void orc_kron_table_free(orc_ktable *t);
int orc_kron_table_entries(const orc_ktable *t);
int orc_kron_table_bits(const orc_ktable *t);
int orc_kron_table_max_len(const orc_ktable *t);
/* sym: N x max_len symbols (first level first); other arrays as orc_table_get. */
void orc_kron_table_get(const orc_ktable *t, uint8_t *sym, uint8_t *len, double *p,
                        uint64_t *w, uint32_t *thr, uint32_t *alias);
uint32_t orc_kron_draw(const orc_ktable *t, uint32_t u);
int orc_kron_generate(const orc_ktable *t, int k, uint64_t seed, uint64_t e0, uint64_t count,
                      uint64_t *row, uint64_t *col);
/* Exact P(row, col) over the n0^k x n0^k matrix (n0^k <= 4096). */
int orc_kron_edge_distribution(const orc_ktable *t, int k, int quantised, double *out);

/* Partitioned graphs (Sec. 3).  The 2^k x 2^k adjacency matrix is cut into
 * 2^t x 2^t tiles.  From the root (depth 0, m edges) every node (depth, R, C)
 * splits its edges among its quadrants a, b, c, d by three binomials:
 * n_a ~ Bin(n, a), n_b ~ Bin(n - n_a, b/(b+c+d)), n_c ~ Bin(n - n_a - n_b,
 * c/(c+d)), n_d = the rest; binomial j draws from the stream
 * orc_partition_word(seed, depth, R * 2^depth + C, j, .).  Tiles (depth t)
 * are listed in quadtree order (a, b, c, d at every level); the edges of a
 * tile are numbered consecutively from the count of all edges before it in
 * that order, and edge e of tile (R, C) is the sampling loop of edge e
 * started with the t levels (R, C) already fixed.  Only nodes that meet the
 * tile rows [row_tile_begin, row_tile_end) are split. */
uint32_t orc_partition_word(uint64_t seed, int depth, uint64_t node, int j, uint64_t n);
/* Binomial(n, p): inversion for n min(p, 1-p) < 10, else BTRS (Hoermann 1993);
 * p > 1/2 draws n - Bin(n, 1 - p). */
uint64_t orc_binomial(uint64_t n, double p, uint64_t seed, int depth, uint64_t node, int j);
/* Non-empty tiles meeting the rows, at most `cap` written; returns how many
 * there are (or -1 on invalid arguments). */
int64_t orc_partition(double a, double b, double c, double d, int t, uint64_t m, uint64_t seed,
                      uint64_t row_tile_begin, uint64_t row_tile_end, uint64_t cap,
                      uint64_t *tile_row, uint64_t *tile_col, uint64_t *count, uint64_t *first);
/* Edges first .. first+count-1 of tile (tile_row, tile_col) of a depth-t
 * partition (single table). */
int orc_generate_tile(const orc_table *table, int k, int t, uint64_t tile_row, uint64_t tile_col,
                      uint64_t seed, uint64_t first, uint64_t count, uint64_t *row, uint64_t *col);

/* Naive per-bit R-MAT (Sec. 1): level t draws one quadrant from word t with
 * thresholds round(a 2^32), round((a+b) 2^32), round((a+b+c) 2^32) of the
 * level's normalised parameters P[4t..4t+3]. */
int orc_generate_naive(const double *P, int k, int undirected, uint64_t seed,
                       uint64_t e0, uint64_t count, uint64_t *row, uint64_t *col);

/* Exact probability of every edge (row, col), out[row * 2^k + col], implied by
 * drawing from the tables as orc_generate does.  quantised = 0 uses the FP64
 * path probabilities p, quantised = 1 uses w / 2^32.  Intended for k <= 8. */
int orc_edge_distribution(const orc_table *const *tables, int ngroups, int k,
                          int quantised, double *out);

#ifdef __cplusplus
}
#endif
#endif
