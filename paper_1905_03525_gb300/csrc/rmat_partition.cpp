// rmat_partition.cpp -- partitioned graphs (Sec. 3, communication-free
// generation of partitioned graphs).
//
// The 2^k x 2^k adjacency matrix is cut into 2^t x 2^t square tiles.  A
// divide-and-conquer pass over the quadtree gives the number of edges of
// every tile: node (depth, R, C) holding n edges hands them to its quadrants
// a, b, c, d by three conditional binomials, each drawn from its own
// counter-based stream, so a PE that owns some rows of tiles splits only the
// nodes that meet its rows and still agrees with every other PE.  Each tile
// is then generated by the sampling kernel with the tile's t levels fixed
// (a batched job per tile), which keeps every edge of a PE's rows on that PE.
//
// Host side only; the per-tile generation runs in k_part_fast when the table
// takes the contract-case kernel (u32 compact tables in shared memory), else
// in k_batch (rmat_kernels.cu).
#include <cuda_runtime.h>

#include <cmath>
#include <new>
#include <vector>

#include "rmat_internal.h"
#include "rmat_kernels.h"

struct rmat_partition {
    const rmat_table *t = nullptr;
    int levels = 0;
    uint64_t m = 0, seed = 0, r0 = 0, r1 = 0;
    std::vector<uint64_t> row, col, count, first;
    uint64_t edges = 0;
    rmat_batch *batch = nullptr;  // prepared for `batch_out`
    void *batch_out = nullptr;
    rmat::PartTile *dtiles = nullptr;  // the contract-case kernel's tile list, on device `dtiles_dev`
    int dtiles_dev = -1, dtile = 0;    // ... for warp tiles of `dtile` edges
    uint32_t ntiles = 0;
    uint64_t nwt = 0;
};

namespace rmat {
namespace {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) on the host.
void philox_block(const uint32_t ctr_in[4], uint32_t k0, uint32_t k1, uint32_t out[4]) {
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    for (int round = 0; round < 10; ++round) {
        const uint64_t p0 = uint64_t(0xD2511F53u) * c[0];
        const uint64_t p1 = uint64_t(0xCD9E8D57u) * c[2];
        const uint32_t n0 = uint32_t(p1 >> 32) ^ c[1] ^ k0;
        const uint32_t n2 = uint32_t(p0 >> 32) ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = uint32_t(p1);
        c[2] = n2;
        c[3] = uint32_t(p0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    for (int i = 0; i < 4; ++i) out[i] = c[i];
}

// The stream of binomial j of recursion node `node` (R * 2^depth + C) at
// `depth`: word n is word n % 4 of the block with counter
// (n / 4, 2^31 | j << 8 | depth, node lo, node hi) under key = seed.  Edge
// streams have the high half of their block index in counter word 1 (0), so
// the two never share a block.
class SplitStream {
   public:
    SplitStream(uint64_t seed, int depth, uint64_t node, int j)
        : k0_(uint32_t(seed)), k1_(uint32_t(seed >> 32)) {
        ctr_[1] = 0x80000000u | (uint32_t(j) << 8) | uint32_t(depth);
        ctr_[2] = uint32_t(node);
        ctr_[3] = uint32_t(node >> 32);
    }
    uint32_t word() {
        if (n_ % 4 == 0) {
            ctr_[0] = uint32_t(n_ / 4);
            philox_block(ctr_, k0_, k1_, block_);
        }
        return block_[n_++ % 4];
    }
    // (x + 1/2) / 2^52 with x the top 26 bits of two words: in (0, 1), exact.
    double uniform() {
        const uint32_t hi = word() >> 6;
        const uint32_t lo = word() >> 6;
        return (double(hi) * 67108864.0 + double(lo) + 0.5) * 0x1p-52;
    }

   private:
    uint32_t k0_, k1_;
    uint32_t ctr_[4] = {0, 0, 0, 0};
    uint32_t block_[4] = {0, 0, 0, 0};
    uint64_t n_ = 0;
};

// Sequential-search inversion for n p < 10 (p <= 1/2): pmf(x) =
// pmf(x - 1) * ((n + 1) p/q / x - p/q); a uniform beyond the rounded total
// starts over.
uint64_t binomial_by_inversion(uint64_t n, double p, SplitStream &s) {
    const double q = 1.0 - p;
    const double ratio = p / q;
    const double scale = (double(n) + 1.0) * ratio;
    const double pmf0 = std::pow(q, double(n));
    for (;;) {
        double u = s.uniform();
        double pmf = pmf0;
        uint64_t x = 0;
        bool overrun = false;
        while (u > pmf) {
            u -= pmf;
            if (++x > n) {
                overrun = true;
                break;
            }
            pmf *= scale / double(x) - ratio;
        }
        if (!overrun) return x;
    }
}

// BTRS, transformed rejection with squeeze (W. Hoermann, "The generation of
// binomial random variates", J. Statist. Comput. Simul. 46, 1993), for
// n p >= 10 and p <= 1/2.
uint64_t binomial_by_btrs(uint64_t n, double p, SplitStream &s) {
    const double q = 1.0 - p;
    const double N = double(n);
    const double spq = std::sqrt(N * p * q);
    const double b = 1.15 + 2.53 * spq;
    const double a = -0.0873 + 0.0248 * b + 0.01 * p;
    const double c = N * p + 0.5;
    const double v_r = 0.92 - 4.2 / b;
    const double alpha = (2.83 + 5.1 / b) * spq;
    const double log_pq = std::log(p / q);
    const double mode = std::floor((N + 1.0) * p);
    const double h = std::lgamma(mode + 1.0) + std::lgamma(N - mode + 1.0);
    for (;;) {
        const double u = s.uniform() - 0.5;
        double v = s.uniform();
        const double us = 0.5 - std::fabs(u);
        const double x = std::floor((2.0 * a / us + b) * u + c);
        if (x < 0.0 || x > N) continue;
        if (us >= 0.07 && v <= v_r) return uint64_t(x);
        v = std::log(v * alpha / (a / (us * us) + b));
        if (v <= h - std::lgamma(x + 1.0) - std::lgamma(N - x + 1.0) + (x - mode) * log_pq) return uint64_t(x);
    }
}

uint64_t binomial(uint64_t n, double p, uint64_t seed, int depth, uint64_t node, int j) {
    if (n == 0 || !(p > 0.0)) return 0;
    if (p >= 1.0) return n;
    SplitStream s(seed, depth, node, j);
    const bool flip = p > 0.5;
    const double pp = flip ? 1.0 - p : p;
    const uint64_t x = double(n) * pp < 10.0 ? binomial_by_inversion(n, pp, s) : binomial_by_btrs(n, pp, s);
    return flip ? n - x : x;
}

// Depth-first over the quadtree in a, b, c, d order; `next` numbers the
// edges of every tile passed, on this PE or not.
struct Splitter {
    rmat_partition *p;
    double P[4];
    uint64_t next = 0;

    void visit(int depth, uint64_t R, uint64_t C, uint64_t n) {
        if (n == 0) return;
        const int below = p->levels - depth;
        const uint64_t lo = R << below, hi = (R + 1) << below;
        if (hi <= p->r0 || lo >= p->r1) {  // no row of this PE: skip, keep numbering
            next += n;
            return;
        }
        if (below == 0) {
            p->row.push_back(R);
            p->col.push_back(C);
            p->count.push_back(n);
            p->first.push_back(next);
            p->edges += n;
            next += n;
            return;
        }
        const uint64_t node = (R << depth) | C;
        const double bcd = (P[1] + P[2]) + P[3];
        const double cd = P[2] + P[3];
        const uint64_t na = binomial(n, P[0], p->seed, depth, node, 0);
        const uint64_t nb = binomial(n - na, bcd > 0.0 ? P[1] / bcd : 0.0, p->seed, depth, node, 1);
        const uint64_t nc = binomial(n - na - nb, cd > 0.0 ? P[2] / cd : 0.0, p->seed, depth, node, 2);
        const uint64_t nd = n - na - nb - nc;
        visit(depth + 1, 2 * R, 2 * C, na);
        visit(depth + 1, 2 * R, 2 * C + 1, nb);
        visit(depth + 1, 2 * R + 1, 2 * C, nc);
        visit(depth + 1, 2 * R + 1, 2 * C + 1, nd);
    }
};

}  // namespace
}  // namespace rmat

using namespace rmat;

extern "C" {

rmat_status rmat_partition_create(const rmat_table *t, int tile_levels, uint64_t m, uint64_t seed,
                                  uint64_t row_tile_begin, uint64_t row_tile_end, rmat_partition **out) {
    clear_error();
    if (!out) return fail(RMAT_ERR_INVALID_ARGUMENT, "out is NULL");
    *out = nullptr;
    if (!t) return fail(RMAT_ERR_INVALID_ARGUMENT, "table is NULL");
    if (!t->has_params || t->per_level || t->groups.size() != 1)
        return fail(RMAT_ERR_INVALID_ARGUMENT, "partitions take a table of one (a, b, c, d) (variable or fixed)");
    if (t->flags & RMAT_UNDIRECTED || t->scramble)
        return fail(RMAT_ERR_INVALID_ARGUMENT, "a partition keeps edges in their tiles: no undirected, no scrambling");
    if (tile_levels < 0 || tile_levels > t->k || tile_levels > 30)
        return fail(RMAT_ERR_INVALID_ARGUMENT, "tile_levels must be in [0, min(k, 30)]");
    if (row_tile_begin > row_tile_end || row_tile_end > (uint64_t(1) << tile_levels))
        return fail(RMAT_ERR_INVALID_ARGUMENT, "tile rows must satisfy begin <= end <= 2^tile_levels");
    if (m > RMAT_MAX_EDGES) return fail(RMAT_ERR_INVALID_ARGUMENT, "m above RMAT_MAX_EDGES");
    rmat_partition *p = new (std::nothrow) rmat_partition;
    if (!p) return fail(RMAT_ERR_OUT_OF_MEMORY, "host allocation failed");
    p->t = t;
    p->levels = tile_levels;
    p->m = m;
    p->seed = seed;
    p->r0 = row_tile_begin;
    p->r1 = row_tile_end;
    try {
        Splitter sp{p, {t->params[0], t->params[1], t->params[2], t->params[3]}};
        sp.visit(0, 0, 0, m);
    } catch (const std::bad_alloc &) {
        delete p;
        return fail(RMAT_ERR_OUT_OF_MEMORY, "host allocation failed");
    }
    *out = p;
    return RMAT_OK;
}

rmat_status rmat_partition_info(const rmat_partition *p, uint64_t *tiles, uint64_t *edges) {
    clear_error();
    if (!p) return fail(RMAT_ERR_INVALID_ARGUMENT, "partition is NULL");
    if (tiles) *tiles = p->row.size();
    if (edges) *edges = p->edges;
    return RMAT_OK;
}

rmat_status rmat_partition_tiles(const rmat_partition *p, uint64_t *tile_row, uint64_t *tile_col, uint64_t *count,
                                 uint64_t *first_edge) {
    clear_error();
    if (!p) return fail(RMAT_ERR_INVALID_ARGUMENT, "partition is NULL");
    for (size_t i = 0; i < p->row.size(); ++i) {
        if (tile_row) tile_row[i] = p->row[i];
        if (tile_col) tile_col[i] = p->col[i];
        if (count) count[i] = p->count[i];
        if (first_edge) first_edge[i] = p->first[i];
    }
    return RMAT_OK;
}

rmat_status rmat_generate_partition(rmat_partition *p, void *out, rmat_stream_t stream) {
    clear_error();
    if (!p) return fail(RMAT_ERR_INVALID_ARGUMENT, "partition is NULL");
    if (p->edges == 0) return RMAT_OK;
    if (!out) return fail(RMAT_ERR_INVALID_ARGUMENT, "output pointer is NULL");
    if (reinterpret_cast<uintptr_t>(out) & 7u) return fail(RMAT_ERR_INVALID_ARGUMENT, "output must be 8-byte aligned");
    AliasPlan plan;
    const uint32_t *img = nullptr;
    if (rmat_status st = plan_and_image(p->t, plan, &img)) return st;
    if (plan.fast_kernel && plan.fmt == kCompact && !plan.u64 && !plan.levels && !p->t->flags && !p->t->scramble) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return fail(RMAT_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        if (!p->dtiles || p->dtiles_dev != dev || p->dtile != plan.tile) {
            if (p->dtiles) cudaFree(p->dtiles);
            p->dtiles = nullptr;
            std::vector<PartTile> v;
            uint64_t at = 0, wt = 0;
            for (size_t i = 0; i < p->row.size(); ++i) {
                if (p->count[i]) {
                    Job J{};
                    set_tile_prefix(J, p->t, p->levels, p->row[i], p->col[i]);
                    PartTile P{};
                    P.e0 = p->first[i];
                    P.out = at;
                    P.count = p->count[i];
                    P.wt0 = wt;
                    P.pre_row = uint32_t(J.pre_row);
                    P.pre_col = uint32_t(J.pre_col);
                    P.pre_len = J.pre_len;
                    v.push_back(P);
                    wt += (p->count[i] + uint64_t(plan.tile) - 1) / uint64_t(plan.tile);
                }
                at += p->count[i];
            }
            e = cudaMalloc(&p->dtiles, v.size() * sizeof(PartTile));
            if (e == cudaSuccess) e = cudaMemcpy(p->dtiles, v.data(), v.size() * sizeof(PartTile), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                if (p->dtiles) cudaFree(p->dtiles);
                p->dtiles = nullptr;
                cudaGetLastError();
                return fail(e == cudaErrorMemoryAllocation ? RMAT_ERR_OUT_OF_MEMORY : RMAT_ERR_CUDA,
                            std::string("partition tile list: ") + cudaGetErrorString(e));
            }
            p->dtiles_dev = dev;
            p->dtile = plan.tile;
            p->ntiles = uint32_t(v.size());
            p->nwt = wt;
        }
        return launch_partition_fast(p->t, img, plan, p->seed, p->dtiles, p->ntiles, p->nwt, out,
                                     reinterpret_cast<cudaStream_t>(stream));
    }
    if (!p->batch || p->batch_out != out) {
        rmat_batch_free(p->batch);
        p->batch = nullptr;
        p->batch_out = nullptr;
        rmat_batch *b = nullptr;
        if (rmat_status st = rmat_batch_create(&b)) return st;
        const uint64_t eb = p->t->k > 32 ? 16 : 8;
        uint64_t at = 0;
        for (size_t i = 0; i < p->row.size(); ++i) {
            void *dst = static_cast<unsigned char *>(out) + at * eb;
            if (rmat_status st = rmat_batch_add_tile(b, p->t, p->seed, p->first[i], p->count[i], p->levels,
                                                     p->row[i], p->col[i], dst)) {
                rmat_batch_free(b);
                return st;
            }
            at += p->count[i];
        }
        if (rmat_status st = rmat_batch_prepare(b, nullptr)) {
            rmat_batch_free(b);
            return st;
        }
        p->batch = b;
        p->batch_out = out;
    }
    return rmat_batch_launch(p->batch, stream);
}

void rmat_free_partition(rmat_partition *p) {
    if (!p) return;
    rmat_batch_free(p->batch);
    if (p->dtiles) cudaFree(p->dtiles);
    delete p;
}

}  // extern "C"
