/*
 * rmat.h -- C ABI of librmat, a GB300 (sm_103a) generator of R-MAT graphs with
 * constant work per edge, after Huebschle-Schneider & Sanders, "Linear Work
 * Generation of R-MAT Graphs" (arXiv 1905.03525).
 *
 * The R-MAT model (Sec. 1): a directed multigraph on n = 2^k nodes with m
 * edges; each edge descends k times into one of the four quadrants of the
 * adjacency matrix, upper-left with probability a, upper-right b, lower-left c,
 * lower-right d (a + b + c + d = 1), emitting one row bit and one column bit
 * per level.  The generator samples whole paths of that recursion at once from
 * an alias table (Sec. 2) and concatenates their bits until k levels are
 * filled.
 *
 * Conventions shared by every call:
 *   - Every call returns an rmat_status; nothing aborts.  On failure
 *     rmat_last_error() returns a message (thread-local, valid until the
 *     thread's next librmat call).  Arguments are checked on the host before
 *     anything is launched.
 *   - "device pointer" means memory of the current CUDA device (cudaMalloc,
 *     torch.cuda, ...).  Output buffers are owned by the caller.
 *   - Edge layout: an array of (row, col) pairs, row first.  Tables with
 *     k <= 32 write uint32 pairs (8 bytes per edge), tables with k > 32 write
 *     uint64 pairs (16 bytes per edge).
 *   - Determinism: edge i of a call is edge number edge_offset + i of the
 *     graph (table, seed), and its bytes depend only on (table, seed,
 *     edge_offset + i): never on how a graph is split into calls, on the
 *     launch shape, on batching or on serving.
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11) with key = seed
 *     and counter = (block q, edge index e); edge e consumes words 0, 1, 2,
 *     ... of its own stream, one 32-bit word per alias draw.
 *   - Sizes: one call generates at most RMAT_MAX_EDGES edges (per graph of a
 *     batch, per request of a server, per partitioned graph); larger counts
 *     return RMAT_ERR_INVALID_ARGUMENT.  edge_offset + count must also fit
 *     64 bits.
 */
#ifndef RMAT_H
#define RMAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *rmat_stream_t; /* same type as cudaStream_t; NULL = legacy default stream */

typedef enum {
    RMAT_OK = 0,
    RMAT_ERR_INVALID_ARGUMENT = 1, /* a parameter is out of range; nothing was launched */
    RMAT_ERR_OUT_OF_MEMORY = 2,    /* a device or host allocation failed */
    RMAT_ERR_CUDA = 3,             /* a CUDA runtime call failed (message has the CUDA error) */
    RMAT_ERR_TIMEOUT = 4,          /* a bounded wait ran out (device flag or host deadline) */
    RMAT_ERR_UNSUPPORTED = 5       /* no device, wrong architecture, or a table too large */
} rmat_status;

typedef struct rmat_table rmat_table; /* opaque; owned by the library */

/* Largest edge count of one call (2^56: 2^60 bytes of u64 output). */
#define RMAT_MAX_EDGES (1ull << 56)

/* Table flags. */
#define RMAT_UNDIRECTED 1u /* emit (min(r,c), max(r,c)): mirror the lower-left triangle (Sec. 3) */

/*
 * rmat_build_table -- variable-length table of similar-probability paths
 * (Sec. 2, table-construction fragment).
 *
 * Starting from the empty path, the most probable entry is repeatedly replaced
 * by its four children (probabilities ap, bp, cp, dp; bits (0,0), (0,1),
 * (1,0), (1,1) appended to (row, col)) while |Q| + 3 < table_bound, which
 * gives the largest table of 1 + 3t entries below the bound (Fig. 1 sizes:
 * bound 2^12 -> 4093).  Ties go to the lexicographically smaller path; paths
 * stop growing at min(k, 32) levels.  Path probabilities are FP64 products,
 * quantised to u32 weights that sum to 2^32 (floor, then +1 to the largest
 * fractional parts) and turned into an integer Vose alias table.
 *
 * a, b, c, d : quadrant probabilities, each >= 0, |a+b+c+d - 1| <= 1e-9; they
 *              are divided by their sum before use.
 * k          : levels = log2(nodes), 1 <= k <= 64.
 * table_bound: 5 <= table_bound <= 2^24.
 * out        : receives the new table (host memory; device copy made lazily).
 */
rmat_status rmat_build_table(double a, double b, double c, double d, int k,
                             uint64_t table_bound, rmat_table **out);

/*
 * rmat_build_table_fixed -- all 4^ell paths of length ell (Sec. 2, "paths of a
 * fixed length"), 1 <= ell <= 12.  Entry i is the path whose symbols are the
 * base-4 digits of i (most significant digit = top level).  Same
 * quantisation and alias construction as rmat_build_table.
 */
rmat_status rmat_build_table_fixed(double a, double b, double c, double d, int k, int ell,
                                   rmat_table **out);

/*
 * rmat_build_table_levels -- per-level parameters, one fixed-length table per
 * group of ell consecutive levels (Sec. 3, smoothing by perturbed parameters,
 * in its exact form for noise shared by all edges).
 *
 * abcd : k x 4 doubles, row t = (a, b, c, d) of level t (level 0 = top = most
 *        significant bit).  Each row is checked and normalised like above.
 * ell  : group length, 1 <= ell <= 12; group g covers levels g*ell ..
 *        min(k, (g+1)*ell) - 1 and is sampled with word g of the edge's stream.
 * flags: RMAT_UNDIRECTED or 0.
 * At most 64 groups.
 */
rmat_status rmat_build_table_levels(const double *abcd, int k, int ell, unsigned flags,
                                    rmat_table **out);

/* Set or clear flags (RMAT_UNDIRECTED) on an existing table. */
rmat_status rmat_table_set_flags(rmat_table *t, unsigned flags);

/*
 * rmat_table_set_scramble -- relabel vertex IDs by a seeded bijection pi of
 * [0, 2^k) (Sec. 3: scrambling is a constant-time post-processing that hides
 * the graph's structure, as Graph 500 does).  Each edge (r, c) becomes
 * (pi(r), pi(c)), before undirected mirroring.  pi: three rounds of
 *   x ^= x >> ceil(k/2);  x = (x * m_i + a_i) mod 2^k      (m_i odd),
 * each round a bijection; m_0, a_0, m_1, a_1, m_2, a_2 are the first six
 * outputs of SplitMix64 seeded with scramble_seed, reduced mod 2^k (the m_i
 * with their low bit set).  enable = 0 turns it off.
 */
rmat_status rmat_table_set_scramble(rmat_table *t, int enable, uint64_t scramble_seed);

typedef struct {
    int k;              /* levels */
    int groups;         /* 1, or the number of level groups */
    int entries;        /* |Q| of group 0 (before padding) */
    int bits;           /* b of group 0: padded size 2^b */
    int max_len;        /* longest path of any group, in levels */
    int index_bytes;    /* 4 (vertex IDs < 2^32: k <= 32, or n0^k <= 2^32) or 8 */
    unsigned flags;
    uint64_t device_image_bytes; /* size of the device copy of all groups */
    int n0;             /* initiator size: 2 for R-MAT, n0 for rmat_build_table_kron */
} rmat_table_info_t;

rmat_status rmat_table_info(const rmat_table *t, rmat_table_info_t *info);

/* Entries and padded size of one group. */
rmat_status rmat_table_group_info(const rmat_table *t, int group, int *entries, int *bits,
                                  int *max_len);

/*
 * rmat_build_table_gpu -- the table of rmat_build_table(a, b, c, d, k,
 * table_bound), built on the current GPU (Sec. 3, parallelization: expand
 * every path above a probability threshold level by level, then build the
 * alias table).  The result is identical to rmat_build_table's -- entries,
 * order, probabilities, weights, alias pairs and device image -- and its
 * device copy on this GPU is the image the build produced.  One launch of a
 * single 1024-thread CTA on `stream`; the call returns when the table is
 * ready (synchronous).  Needs a, b, c, d >= 1e-9 (else RMAT_ERR_UNSUPPORTED; use
 * rmat_build_table); device scratch about 30 bytes per expanded node (~4x
 * the bound) plus the table, allocated and freed by the call.
 */
rmat_status rmat_build_table_gpu(double a, double b, double c, double d, int k,
                                 uint64_t table_bound, rmat_stream_t stream, rmat_table **out);

/*
 * Stochastic Kronecker graphs (Sec. 3: an n0 x n0 matrix instead of the 2 x 2
 * one in the recursion).  theta: n0 x n0 initiator, row-major, entries >= 0
 * summing to 1 (within 1e-9; divided by their sum); 2 <= n0 <= 16.  The
 * graph has n0^k vertices (n0^k <= 2^64); level t of an edge picks initiator
 * cell (i, j) with probability theta[i][j], i being digit t (from the most
 * significant) of the row in base n0 and j that of the column.  Symbol
 * s = n0 * i + j.  Tables generalise the R-MAT ones: a variable-length table
 * expands an entry into its n0^2 children while |Q| + n0^2 - 1 < bound
 * (largest tie-break and canonical order as for R-MAT; paths stop at min(k,
 * L) levels, L the largest with n0^L <= 2^32); a fixed table holds all
 * (n0^2)^ell paths.  rmat_generate and rmat_generate_host accept the table;
 * each edge draws whole paths as for R-MAT (one Philox word per draw) and
 * appends their base-n0 digits until k levels are filled, the last path cut
 * to its top digits.  Output: (row, col) u32 pairs when n0^k <= 2^32, else
 * u64 (index_bytes of rmat_table_info).  n0 = 2 builds the R-MAT table of
 * (a, b, c, d) = (theta[0][0], theta[0][1], theta[1][0], theta[1][1]).  For
 * n0 > 2 the table must fit in shared memory (24 bytes per column, about
 * 9000 columns), and flags, scrambling, batches and partitions are refused
 * (RMAT_ERR_UNSUPPORTED).
 */
rmat_status rmat_build_table_kron(const double *theta, int n0, int k, uint64_t table_bound,
                                  rmat_table **out);
rmat_status rmat_build_table_kron_fixed(const double *theta, int n0, int k, int ell,
                                        rmat_table **out);

/*
 * rmat_table_export -- copy out group `group` in canonical order (paths in
 * lexicographic order, zero-probability padding at the end), arrays of length
 * 2^bits.  sym: the path, 2 bits per level (2*rowbit + colbit), top level in
 * bits 63..62 (Kronecker tables: the symbols as base-n0^2 digits, first level
 * most significant, left-aligned in L digits, L the depth cap of n0); len:
 * levels; p: FP64 probability; w: u32 weight (held in a
 * uint64); thr/alias: the alias table (draw: column j = top `bits` bits of a
 * word, residual r = the rest; entry j if r < thr[j], else alias[j]).
 * Any pointer may be NULL.  Host memory.
 */
rmat_status rmat_table_export(const rmat_table *t, int group, uint64_t *sym, uint8_t *len,
                              double *p, uint64_t *w, uint32_t *thr, uint32_t *alias);

/* Upload the device copy now for the current device (otherwise the first
 * rmat_generate on a device does it, synchronously).  Do this before
 * capturing rmat_generate into a CUDA graph. */
rmat_status rmat_table_upload(rmat_table *t);

void rmat_free_table(rmat_table *t);

/*
 * rmat_generate -- edges edge_offset .. edge_offset+count-1 of the graph
 * (table, seed) into `out` (device pointer, 8-byte aligned; 16-byte aligned
 * lets the kernel use bulk (TMA) stores), count * 8 or 16 bytes.
 * Asynchronous on `stream`; the caller synchronises.  count == 0 is a no-op.
 * Sampling loop of Sec. 2: per edge, draw a path from the alias table with one
 * Philox word, append its row/column bits, repeat until k levels are filled;
 * the surplus levels of the last path are dropped (each edge has its own
 * random stream, so no bits carry over between edges).
 */
rmat_status rmat_generate(const rmat_table *t, uint64_t seed, uint64_t edge_offset,
                          uint64_t count, void *out, rmat_stream_t stream);

/*
 * rmat_generate_host -- as rmat_generate, but `host_out` is host memory
 * (pinned memory gives full copy bandwidth).  Generates in device chunks and
 * overlaps each chunk's device-to-host copy with the next chunk's
 * generation.  Blocking: returns when all edges are in host_out.  Uses a
 * library-owned device staging area (allocated on first use, kept).
 */
rmat_status rmat_generate_host(const rmat_table *t, uint64_t seed, uint64_t edge_offset,
                               uint64_t count, void *host_out, rmat_stream_t stream);

/*
 * rmat_generate_naive -- the plain R-MAT process of Sec. 1: k quadrant draws
 * per edge, level t using word t of the same Philox stream and the
 * thresholds round(a 2^32), round((a+b) 2^32), round((a+b+c) 2^32) of level
 * t's normalised parameters abcd[4t..4t+3].  Baseline only: same distribution
 * as rmat_generate, not the same bits.  Output layout as rmat_generate.
 */
rmat_status rmat_generate_naive(const double *abcd, int k, unsigned flags, uint64_t seed,
                                uint64_t edge_offset, uint64_t count, void *out,
                                rmat_stream_t stream);

/*
 * Launch shape.  rmat_generate uses the autotuned shape for (table, device)
 * when one was recorded with rmat_set_launch_config, else a default.
 * threads: 128..1024, multiple of 32; ctas_per_sm: 1..8; tile_edges: edges
 * per warp tile, multiple of 32, 32..1024.  Results never depend on it.
 */
typedef struct {
    int threads;
    int ctas_per_sm;
    int tile_edges;
} rmat_launch_config_t;

rmat_status rmat_set_launch_config(rmat_table *t, const rmat_launch_config_t *cfg);
rmat_status rmat_get_launch_config(const rmat_table *t, rmat_launch_config_t *cfg);

/* ---------------------------------------------------------------------- */
/* Batched generation: many graphs, one persistent launch.                 */
/* ---------------------------------------------------------------------- */
typedef struct rmat_batch rmat_batch; /* opaque */

/* Create an empty batch. */
rmat_status rmat_batch_create(rmat_batch **out);

/* Add edges edge_offset .. edge_offset+count-1 of graph (t, seed) written to
 * `out` (device, 8-byte aligned).  The table must outlive the batch. */
rmat_status rmat_batch_add(rmat_batch *b, const rmat_table *t, uint64_t seed,
                           uint64_t edge_offset, uint64_t count, void *out);

/* Add a tile of a partitioned graph (Sec. 3): edges edge_offset ..
 * edge_offset+count-1, each started with its top tile_levels levels fixed to
 * (tile_row, tile_col) -- the tile's rows [tile_row * 2^(k-tile_levels), ...)
 * and columns likewise -- and the remaining k - tile_levels levels drawn from
 * the edge's stream as in rmat_generate.  tile_levels = 0 is rmat_batch_add.
 * The table must have one group (rmat_build_table or rmat_build_table_fixed)
 * without RMAT_UNDIRECTED or scrambling (either would move edges out of the
 * tile); tile_levels <= min(k, 30); coordinates < 2^tile_levels. */
rmat_status rmat_batch_add_tile(rmat_batch *b, const rmat_table *t, uint64_t seed,
                                uint64_t edge_offset, uint64_t count, int tile_levels,
                                uint64_t tile_row, uint64_t tile_col, void *out);

/* Pack table images and work list into device memory (synchronous; done
 * automatically by the first launch).  Call before graph capture.  cfg may be
 * NULL (default shape: 1024 threads, one CTA per SM, 512-edge tiles -- 256
 * for k > 32 -- halved while the largest table would not fit in shared memory
 * beside them).
 * Adding graphs after preparing discards the device state (and with it any
 * CUDA graph that captured rmat_batch_launch). */
rmat_status rmat_batch_prepare(rmat_batch *b, const rmat_launch_config_t *cfg);

/* One persistent launch that generates every added graph.  Capturable in a
 * CUDA graph after rmat_batch_prepare. */
rmat_status rmat_batch_launch(rmat_batch *b, rmat_stream_t stream);

/* Number of graphs / total edges in the batch. */
rmat_status rmat_batch_size(const rmat_batch *b, uint64_t *graphs, uint64_t *edges);

void rmat_batch_free(rmat_batch *b);

/* ---------------------------------------------------------------------- */
/* Partitioned graphs (Sec. 3: communication-free generation of partitioned */
/* graphs, each PE holding all edges of some rows)                          */
/* ---------------------------------------------------------------------- */
/* The 2^k x 2^k adjacency matrix is cut into 2^t x 2^t square tiles
 * (t = tile_levels).  Tile counts come from a divide-and-conquer pass over the
 * quadtree: node (depth, R, C) holding n edges gives
 *   n_a ~ Bin(n, a), n_b ~ Bin(n - n_a, b/(b+c+d)), n_c ~ Bin(n - n_a - n_b, c/(c+d)),
 *   n_d = n - n_a - n_b - n_c
 * to its children (2R, 2C), (2R, 2C+1), (2R+1, 2C), (2R+1, 2C+1), with (a, b,
 * c, d) the table's normalised parameters.  Binomial j in {0, 1, 2} of node
 * (depth, R, C) uses the Philox4x32-10 stream with key = seed and counter
 * (n / 4, 2^31 | j << 8 | depth, node lo, node hi), node = R * 2^depth + C,
 * word n % 4; a uniform is (x + 1/2) 2^-52 with x = (w0 >> 6) 2^26 + (w1 >> 6)
 * of two consecutive words.  Bin(n, p) for p > 1/2 is n - Bin(n, 1 - p); for
 * n p < 10 it is inversion by sequential search (restarting with a new
 * uniform if the rounded pmf runs out), else BTRS (Hoermann 1993).
 * Tiles are taken in quadtree order (a, b, c, d at every level) and the edges
 * numbered consecutively in that order: a tile's edges are edge_offset =
 * first .. first+count-1 of rmat_batch_add_tile.  A PE that owns tile rows
 * [row_tile_begin, row_tile_end) splits only the nodes meeting them and gets
 * exactly those tiles of the global partition (no communication). */
typedef struct rmat_partition rmat_partition; /* opaque */

/* Compute the tiles of this PE (host only, no device work).  The table (one
 * group; not undirected, not scrambled) must outlive the partition.  Empty
 * tiles are left out.  Errors: RMAT_ERR_INVALID_ARGUMENT (table kind,
 * tile_levels outside [0, min(k, 30)], row range outside [0, 2^tile_levels]). */
rmat_status rmat_partition_create(const rmat_table *t, int tile_levels, uint64_t m, uint64_t seed,
                                  uint64_t row_tile_begin, uint64_t row_tile_end,
                                  rmat_partition **out);

/* Number of (non-empty) tiles of this PE and their total edges. */
rmat_status rmat_partition_info(const rmat_partition *p, uint64_t *tiles, uint64_t *edges);

/* Copy the tiles out, in quadtree order; each array (any may be NULL) holds
 * `tiles` entries: tile row and column, edge count, first edge number. */
rmat_status rmat_partition_tiles(const rmat_partition *p, uint64_t *tile_row, uint64_t *tile_col,
                                 uint64_t *count, uint64_t *first_edge);

/* Generate this PE's edges into `out` (device, 8-byte aligned, `edges`
 * pairs of u32 for k <= 32, else u64), tile after tile in quadtree order, in
 * one persistent launch (asynchronous on `stream`): a dedicated kernel for
 * u32 compact tables held in shared memory, the batched kernel otherwise.
 * The first call (on a device, or for a given `out` on the batched path)
 * prepares the launch (a synchronous upload of the tile list); calls on one
 * partition must not run concurrently, on the host or the device. */
rmat_status rmat_generate_partition(rmat_partition *p, void *out, rmat_stream_t stream);

void rmat_free_partition(rmat_partition *p);

/* Remove repeated edges (Sec. 3: in a partitioned graph equal edges share a
 * tile, so each PE removes its duplicates alone).  `edges`: device array of
 * `count` (row, col) u32 pairs of a graph with k <= 31 levels (for instance
 * the output of rmat_generate_partition); the first occurrence of every
 * (row, col) in array order is kept and the survivors are compacted to the
 * front in that order; *unique receives their number.  Synchronous on
 * `stream`; count <= 2^31.  Device scratch of about 24 bytes per edge is
 * allocated by the first call on a device and kept for later calls there
 * (grown when a call needs more; rmat_dedup_release frees it); calls on one
 * device take turns on it under a lock.  A hash bucket of more than 3072
 * edges (possible only when few keys repeat many times) is done in a device
 * table of 16-byte slots, a power of two at least twice that bucket, that the
 * call allocates and frees.  Errors: RMAT_ERR_INVALID_ARGUMENT (k, count,
 * alignment), RMAT_ERR_OUT_OF_MEMORY, RMAT_ERR_UNSUPPORTED (no current
 * device), RMAT_ERR_CUDA. */
rmat_status rmat_dedup_edges(void *edges, uint64_t count, int k, uint64_t *unique, rmat_stream_t stream);

/* Free the scratch that rmat_dedup_edges keeps on the current device (no-op
 * when it holds none, or when there is no device).  Not to be called while a
 * rmat_dedup_edges call on that device is running in another thread: it
 * waits for that call's lock.  Errors: RMAT_ERR_CUDA. */
rmat_status rmat_dedup_release(void);

/* ---------------------------------------------------------------------- */
/* Serving: continuous batching of generation requests                     */
/* ---------------------------------------------------------------------- */
/* A server owns one device-memory arena (hbm_budget_bytes) and one worker
 * thread.  Requests queue in FIFO order and are admitted when a slot is free
 * and their table plus one chunk buffer fit the arena.  Each step generates
 * the next chunk of admitted requests in one persistent batched launch --
 * requests that finish with this chunk first, then the others round-robin, up
 * to step_edges edges -- and consumes the chunks: a checksum kernel adds
 * mix(e, row, col) of every edge into the request's checksum (see
 * rmat_request_status_t), and an optional callback sees each chunk on the
 * device.  A finished request frees its memory and slot before the next step,
 * so queued requests join while others are still running.  Each request's
 * edges (and checksum) are identical to rmat_generate of the same table and
 * seed, alone or in any mix.  Arrival, admission and completion times are on
 * the server's clock (seconds since create). */
typedef struct rmat_server rmat_server; /* opaque */

typedef struct {
    uint64_t hbm_budget_bytes; /* device memory for tables and chunk buffers (allocated at create) */
    uint64_t chunk_edges;      /* largest chunk of one request per step (e.g. 2^28) */
    uint64_t step_edges;       /* edges per step over all requests (>= chunk_edges) */
    int max_active;            /* requests generated concurrently, 1..4096 */
    double wait_timeout_s;     /* host-side bound on one step; beyond it the step's requests fail */
    uint64_t gpu_build_min_bound; /* requests with an explicit table_bound >= this have their table built on
                                     the GPU (rmat_build_table_gpu) by the server's builder thread, off the
                                     submitting thread; 0 = every table on the submitting thread */
} rmat_server_config_t;

typedef struct {
    double a, b, c, d;    /* as rmat_build_table */
    int k;
    uint64_t m;           /* edges 0..m-1 of the graph, m >= 1 */
    uint64_t seed;
    uint64_t table_bound; /* variable-length table bound; 0 = the largest power of two <= 8192
                             whose table the batched kernel can keep in shared memory */
    unsigned flags;       /* RMAT_UNDIRECTED or 0 */
    int scramble;         /* nonzero: relabel vertices as rmat_table_set_scramble(t, 1, scramble_seed) */
    uint64_t scramble_seed;
} rmat_request_t;

enum { RMAT_REQ_QUEUED = 0, RMAT_REQ_RUNNING = 1, RMAT_REQ_DONE = 2, RMAT_REQ_FAILED = 3 };

typedef struct {
    uint64_t id;
    int state;            /* RMAT_REQ_* */
    uint64_t edges_done;
    /* sum mod 2^64 over the request's edges e of mix(x), with
     *   x = e*0x9E3779B97F4A7C15 + row*0xC2B2AE3D27D4EB4F + col*0x165667B19E3779F9
     * and mix the splitmix64 finaliser (x ^= x>>30; x *= 0xBF58476D1CE4E5B9;
     * x ^= x>>27; x *= 0x94D049BB133111EB; x ^= x>>31), all mod 2^64 */
    uint64_t checksum;
    double submit_s, admit_s, done_s;
    rmat_status error;    /* why the request failed, if it did */
    uint64_t table_bound; /* the bound the request's table was built with */
} rmat_request_status_t;

typedef struct {
    uint64_t steps, edges, queued, active, memory_used;
    double clock_s;
} rmat_server_stats_t;

/* Called on the worker thread after each chunk is generated and checksummed;
 * device_edges (on the server's device) is valid only during the call. */
typedef void (*rmat_chunk_fn)(void *user, uint64_t request_id, uint64_t edge_offset, uint64_t count,
                              const void *device_edges);

/* Create a server on the current device; allocates the arena and starts the
 * worker. */
rmat_status rmat_server_create(const rmat_server_config_t *cfg, rmat_server **out);
rmat_status rmat_server_set_chunk_callback(rmat_server *s, rmat_chunk_fn fn, void *user);
/* Build the request's table on the calling thread (or, for an explicit
 * table_bound >= gpu_build_min_bound, hand it to the server's builder thread,
 * which builds it on the GPU; the request is admitted once it is ready) and
 * queue the request.  Thread-safe.
 * RMAT_ERR_OUT_OF_MEMORY if the request could never fit the budget. */
rmat_status rmat_server_submit(rmat_server *s, const rmat_request_t *req, uint64_t *id);
rmat_status rmat_server_status(rmat_server *s, uint64_t id, rmat_request_status_t *st);
/* Block until the request is done or failed, or timeout_s passes
 * (RMAT_ERR_TIMEOUT; the request keeps running). */
rmat_status rmat_server_wait(rmat_server *s, uint64_t id, double timeout_s, rmat_request_status_t *st);
/* Block until every submitted request is done or failed. */
rmat_status rmat_server_drain(rmat_server *s, double timeout_s);
rmat_status rmat_server_stats(rmat_server *s, rmat_server_stats_t *out);
/* Fail the requests still queued, finish the running ones, free everything. */
void rmat_server_destroy(rmat_server *s);

/* ---------------------------------------------------------------------- */
/* Generation without device allocation                                    */
/* ---------------------------------------------------------------------- */
/* The paper has no counterpart to this call; it serves callers that cannot
 * allocate device memory -- a process whose device memory is already
 * reserved by another framework's caching allocator, a latency-critical path
 * that must not take the driver's allocation locks (cudaMalloc/cudaFree can
 * synchronise the device), or a deployment with a fixed memory budget.
 *
 * rmat_generate_batch_noalloc -- the batched generation of rmat_batch_launch
 * for n graphs (tables[i], seeds[i]): edges edge_offsets[i] ..
 * edge_offsets[i]+counts[i]-1 into outs[i] (device, 8-byte aligned).  It
 * calls no cudaMalloc/cudaFree and allocates no host memory: the work
 * counter, job list, unit map and copies of the table blobs live in one
 * library-owned device array of RMAT_NOALLOC_SCRATCH_BYTES, which every GPU
 * that loads the library keeps until the process exits.
 *   - n <= RMAT_NOALLOC_MAX_GRAPHS; all tables of one call have the same
 *     output width (all k <= 32 or all k > 32); their blobs, the job list and
 *     one 4-byte entry per work unit (262144 edges; 131072 for k > 32 or
 *     when a table is too large for the default tile) must fit the scratch.
 *     Anything larger returns RMAT_ERR_INVALID_ARGUMENT and launches nothing.
 *   - Set-up: the first call on a device looks up the scratch's device
 *     address (once per device, with that device current) and loads the
 *     batched kernel there.  The runtime may defer placing the scratch (and
 *     the kernel code) in device memory until this first use, so that first
 *     call can take device memory.  A call with n = 0 does exactly this set-up
 *     and launches nothing (the argument arrays may then be NULL): make it on
 *     each device before reserving the rest of the device's memory, and before
 *     any stream capture; later calls then take no device memory at all.
 *   - Asynchronous on `stream`.  Every call shares the one scratch array and
 *     overwrites it (the work counter is cleared each call): calls whose work
 *     overlaps on the GPU -- on different streams, or from threads that race
 *     -- corrupt each other.  Order them on one stream or synchronise.
 * Output bytes are identical to rmat_generate / rmat_batch_launch for the same
 * (table, seed, edge index). */
#define RMAT_NOALLOC_SCRATCH_BYTES (4u << 20)
#define RMAT_NOALLOC_MAX_GRAPHS 64u
rmat_status rmat_generate_batch_noalloc(const rmat_table *const *tables, const uint64_t *seeds,
                                        const uint64_t *edge_offsets, const uint64_t *counts,
                                        void *const *outs, uint32_t n, rmat_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Device error flag                                                       */
/* ---------------------------------------------------------------------- */
/* Read and clear the device-side error flag (non-zero when a kernel's
 * bounded wait gave up).  Synchronises the device.  RMAT_ERR_TIMEOUT if set. */
rmat_status rmat_check_device_errors(void);

/* Failure-path self-test: launches one warp that waits, through the bounded
 * wait the generation kernels use on their table copies, on an mbarrier phase
 * that nothing completes; after `limit` polls (1..2^22, ~0.1 us each after
 * the first 16) it gives up and records the error in the device error word
 * like a production kernel would, and exits.  The call synchronises the
 * device and returns what rmat_check_device_errors then returns:
 * RMAT_ERR_TIMEOUT, with the word cleared and the context usable. */
rmat_status rmat_selftest_bounded_wait(uint32_t limit);

/* Library version string and the compiled GPU architecture. */
const char *rmat_version(void);

const char *rmat_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
