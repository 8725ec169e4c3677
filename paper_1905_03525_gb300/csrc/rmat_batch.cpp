// rmat_batch.cpp -- batched generation: many graphs (or ranges of graphs) in
// one persistent launch.  The batch packs every distinct table blob into one
// device arena, lists one Job per graph and cuts each job into work units of
// unit_edges edges; the persistent kernel's CTAs pop units from an atomic
// counter, restage the table into shared memory when the job changes, and
// generate the unit one warp tile at a time.  Generalises the paper's
// independent edge blocks (Sec. 4, blocks of 2^16 edges per thread) from one
// graph to many.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <new>
#include <vector>

#include "rmat_internal.h"
#include "rmat_kernels.h"

namespace {

struct Side {
    bool u64 = false;
    void *arena = nullptr;
    rmat::Job *jobs = nullptr;
    rmat::Scramble *scr = nullptr;
    uint32_t *unit_job = nullptr;
    unsigned long long *counter = nullptr;
    uint64_t units = 0;
    uint64_t njobs = 0;
    rmat::BatchArgs args{};
    int grid = 0, threads = 0;
    size_t smem = 0;
};

void free_side(Side &s) {
    if (s.arena) cudaFree(s.arena);
    if (s.jobs) cudaFree(s.jobs);
    if (s.scr) cudaFree(s.scr);
    if (s.unit_job) cudaFree(s.unit_job);
    if (s.counter) cudaFree(s.counter);
    s = Side{};
}

}  // namespace

struct rmat_batch {
    struct Entry {
        const rmat_table *t;
        uint64_t seed, e0, count;
        void *out;
        int tile_levels;  // > 0: a tile of a partitioned graph
        uint64_t tile_row, tile_col;
    };
    std::vector<Entry> entries;
    bool prepared = false;
    int device = -1;
    Side side[3];  // u32 jobs for k_batch_fast, other u32 jobs, u64 jobs
    rmat_launch_config_t cfg{1024, 1, 512};
    bool cfg_set = false;  // else the tile adapts to the tables (prepare_side)
    uint64_t edges = 0;
};

namespace rmat {
namespace {

rmat_status cuda_err(const char *what, cudaError_t e) {
    return fail(RMAT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <class T>
rmat_status dev_alloc(T **p, size_t bytes) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(RMAT_ERR_OUT_OF_MEMORY, "batch device allocation failed");
    }
    return RMAT_OK;
}

// Whether a u32 entry runs in k_batch_fast: a whole graph (no tile prefix),
// compact paths, one table for all levels, plain epilogue, and a table that
// fits in shared memory beside the warps' tiles of the batch's shape.
bool fast_entry(const rmat_batch *b, const rmat_batch::Entry &en, const DeviceProps &props) {
    const rmat_table *t = en.t;
    if (t->k > 32 || en.tile_levels || t->format != kCompact || t->per_level || t->flags || t->scramble) return false;
    const int threads = std::max(128, std::min(1024, b->cfg.threads / 32 * 32));
    const int tile = std::max(32, std::min(1024, b->cfg.tile_edges / 32 * 32));
    return kBatchHeaderBytes + size_t(threads / 32) * warp_bytes(false, false, tile) + t->image.size() * 4 <=
           size_t(props.max_smem);
}

// kind 0: the u32 entries that take k_batch_fast; 1: the other u32 entries;
// 2: the u64 entries.  Each kind is one launch.
rmat_status prepare_side(rmat_batch *b, int kind, const DeviceProps &props, Side &s) {
    const bool u64 = kind == 2;
    s.u64 = u64;
    std::vector<const rmat_batch::Entry *> mine;
    for (const auto &en : b->entries)
        if ((en.t->k > 32) == u64 && en.count && (u64 || fast_entry(b, en, props) == (kind == 0)))
            mine.push_back(&en);
    if (mine.empty()) return RMAT_OK;

    int threads = std::max(128, std::min(1024, b->cfg.threads / 32 * 32));
    int tile = std::max(32, std::min(1024, b->cfg.tile_edges / 32 * 32));
    size_t largest_blob = 0;
    for (const auto *en : mine) largest_blob = std::max(largest_blob, en->t->image.size() * 4);
    if (!b->cfg_set) {
        // Default shape: 512-edge tiles (256 for u64) fill phase 2's batches
        // best; halve the tile while the largest table would not fit in
        // shared memory beside the warps' tiles.
        tile = u64 ? 256 : 512;
        while (tile > (u64 ? 128 : 256) &&
               kBatchHeaderBytes + size_t(threads / 32) * warp_bytes(u64, false, tile) + largest_blob > size_t(props.max_smem))
            tile /= 2;
    }
    const size_t per_warp = warp_bytes(u64, false, tile);
    while (kBatchHeaderBytes + size_t(threads / 32) * per_warp > size_t(props.max_smem) && threads > 128) threads /= 2;
    const size_t warps_bytes = size_t(threads / 32) * per_warp;
    const size_t budget = size_t(props.max_smem) - kBatchHeaderBytes - warps_bytes;

    // arena of distinct blobs
    std::map<const rmat_table *, size_t> offset;
    size_t arena_bytes = 0;
    uint32_t max_blob = 0;
    for (const auto *en : mine) {
        if (offset.count(en->t)) continue;
        offset[en->t] = arena_bytes;
        const size_t bytes = en->t->image.size() * 4;
        arena_bytes += (bytes + 255) & ~size_t(255);
        if (bytes <= budget) max_blob = std::max<uint32_t>(max_blob, uint32_t(bytes));
    }
    if (rmat_status st = dev_alloc(&s.arena, arena_bytes)) return st;
    for (const auto &kv : offset) {
        cudaError_t e = cudaMemcpy(static_cast<unsigned char *>(s.arena) + kv.second, kv.first->image.data(),
                                   kv.first->image.size() * 4, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_err("batch arena upload", e);
    }

    // 16 tiles per warp per unit: the CTA waits for its slowest warp once per
    // unit, and 2^30 edges still make ~27 units per CTA for the final wave.
    const uint64_t unit_edges = uint64_t(threads / 32) * tile * 16;
    std::vector<Job> jobs;
    std::vector<Scramble> scrs;
    jobs.reserve(mine.size());
    scrs.reserve(mine.size());
    uint64_t units = 0;
    for (const auto *en : mine) {
        const uint32_t *blob =
            reinterpret_cast<const uint32_t *>(static_cast<unsigned char *>(s.arena) + offset[en->t]);
        const bool smem = en->t->image.size() * 4 <= budget;
        Job J = make_job(en->t, blob, smem, en->seed, en->e0, en->count, en->out);
        if (en->tile_levels) set_tile_prefix(J, en->t, en->tile_levels, en->tile_row, en->tile_col);
        J.unit_begin = units;
        units += (en->count + unit_edges - 1) / unit_edges;
        jobs.push_back(J);
        scrs.push_back(make_scramble(en->t));
    }
    if (units >= (uint64_t(1) << 40)) return fail(RMAT_ERR_INVALID_ARGUMENT, "batch too large");
    std::vector<uint32_t> unit_job(units);
    for (size_t j = 0; j < jobs.size(); ++j) {
        const uint64_t end = j + 1 < jobs.size() ? jobs[j + 1].unit_begin : units;
        std::fill(unit_job.begin() + jobs[j].unit_begin, unit_job.begin() + end, uint32_t(j));
    }
    if (rmat_status st = dev_alloc(&s.jobs, jobs.size() * sizeof(Job))) return st;
    if (rmat_status st = dev_alloc(&s.scr, scrs.size() * sizeof(Scramble))) return st;
    if (rmat_status st = dev_alloc(&s.unit_job, unit_job.size() * sizeof(uint32_t))) return st;
    if (rmat_status st = dev_alloc(&s.counter, sizeof(unsigned long long))) return st;
    cudaError_t e = cudaMemcpy(s.jobs, jobs.data(), jobs.size() * sizeof(Job), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_err("batch job upload", e);
    e = cudaMemcpy(s.scr, scrs.data(), scrs.size() * sizeof(Scramble), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_err("batch scramble upload", e);
    e = cudaMemcpy(s.unit_job, unit_job.data(), unit_job.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_err("batch unit upload", e);

    s.smem = batch_smem_bytes(u64, threads, tile, max_blob);
    int per_sm = 0;
    if (rmat_status st = batch_occupancy(u64, threads, s.smem, per_sm)) return st;
    if (per_sm < 1) return fail(RMAT_ERR_UNSUPPORTED, "batch launch shape does not fit on an SM");
    per_sm = std::min(per_sm, std::max(1, b->cfg.ctas_per_sm));
    s.threads = threads;
    s.units = units;
    s.njobs = jobs.size();
    s.grid = int(std::min<uint64_t>(uint64_t(props.sms) * per_sm, units));
    s.args.jobs = s.jobs;
    s.args.scr = s.scr;
    s.args.unit_job = s.unit_job;
    s.args.units = units;
    s.args.unit_edges = unit_edges;
    s.args.counter = s.counter;
    s.args.max_blob_bytes = max_blob;
    s.args.tile = tile;
    s.args.err = props.err;
    for (const Job &J : jobs) s.args.general |= (J.pre_len || (J.flags & kScrambleFlag)) ? 1 : 0;
    // whole graphs with u32 IDs, compact tables in shared memory and the plain
    // epilogue take the lean kernel (k_batch_fast)
    bool fast = kind == 0;
    for (const Job &J : jobs) fast = fast && J.smem && J.draws1 >= 1 && J.draws1 <= 4;
    s.args.fast = fast ? 1 : 0;
    return RMAT_OK;
}

}  // namespace
}  // namespace rmat

using namespace rmat;

extern "C" {

rmat_status rmat_batch_create(rmat_batch **out) {
    clear_error();
    if (!out) return fail(RMAT_ERR_INVALID_ARGUMENT, "out is NULL");
    *out = new (std::nothrow) rmat_batch;
    if (!*out) return fail(RMAT_ERR_OUT_OF_MEMORY, "host allocation failed");
    return RMAT_OK;
}

rmat_status rmat_batch_add(rmat_batch *b, const rmat_table *t, uint64_t seed, uint64_t edge_offset, uint64_t count,
                           void *out) {
    clear_error();
    if (!b || !t) return fail(RMAT_ERR_INVALID_ARGUMENT, "NULL batch or table");
    if (t->n0 > 2) return fail(RMAT_ERR_UNSUPPORTED, "Kronecker tables (n0 > 2) are generated by rmat_generate only");
    if (count && !out) return fail(RMAT_ERR_INVALID_ARGUMENT, "output pointer is NULL");
    if (reinterpret_cast<uintptr_t>(out) & 7u) return fail(RMAT_ERR_INVALID_ARGUMENT, "output must be 8-byte aligned");
    if (count > RMAT_MAX_EDGES) return fail(RMAT_ERR_INVALID_ARGUMENT, "count above RMAT_MAX_EDGES");
    if (count > ~uint64_t(0) - edge_offset)
        return fail(RMAT_ERR_INVALID_ARGUMENT, "edge_offset + count overflows 64 bits");
    if (b->entries.size() >= 0xFFFFFFFFu) return fail(RMAT_ERR_INVALID_ARGUMENT, "too many graphs");
    b->entries.push_back({t, seed, edge_offset, count, out, 0, 0, 0});
    b->edges += count;
    if (b->prepared) {
        for (Side &s : b->side) free_side(s);
        b->prepared = false;
    }
    return RMAT_OK;
}

rmat_status rmat_batch_add_tile(rmat_batch *b, const rmat_table *t, uint64_t seed, uint64_t edge_offset,
                                uint64_t count, int tile_levels, uint64_t tile_row, uint64_t tile_col, void *out) {
    clear_error();
    if (!b || !t) return fail(RMAT_ERR_INVALID_ARGUMENT, "NULL batch or table");
    if (t->per_level || t->groups.size() != 1)
        return fail(RMAT_ERR_INVALID_ARGUMENT, "tiles take a single-group (variable or fixed) table");
    if (t->flags & RMAT_UNDIRECTED || t->scramble)
        return fail(RMAT_ERR_INVALID_ARGUMENT, "a tile keeps its edges: no undirected mirroring, no scrambling");
    if (tile_levels < 0 || tile_levels > t->k || tile_levels > 30)
        return fail(RMAT_ERR_INVALID_ARGUMENT, "tile_levels must be in [0, min(k, 30)]");
    if ((tile_row >> tile_levels) || (tile_col >> tile_levels))
        return fail(RMAT_ERR_INVALID_ARGUMENT, "tile coordinates must be < 2^tile_levels");
    if (rmat_status st = rmat_batch_add(b, t, seed, edge_offset, count, out)) return st;
    auto &en = b->entries.back();
    en.tile_levels = tile_levels;
    en.tile_row = tile_row;
    en.tile_col = tile_col;
    return RMAT_OK;
}

rmat_status rmat_batch_prepare(rmat_batch *b, const rmat_launch_config_t *cfg) {
    clear_error();
    if (!b) return fail(RMAT_ERR_INVALID_ARGUMENT, "batch is NULL");
    if (cfg) {
        if (cfg->threads < 128 || cfg->threads > 1024 || cfg->threads % 32 || cfg->ctas_per_sm < 1 ||
            cfg->ctas_per_sm > 8 || cfg->tile_edges < 32 || cfg->tile_edges > 1024 || cfg->tile_edges % 32)
            return fail(RMAT_ERR_INVALID_ARGUMENT, "bad batch launch config");
        b->cfg = *cfg;
        b->cfg_set = true;
    }
    DeviceProps props;
    if (rmat_status st = device_props(props)) return st;
    for (Side &s : b->side) free_side(s);
    b->prepared = false;
    for (int u = 0; u < 3; ++u)
        if (rmat_status st = prepare_side(b, u, props, b->side[u])) {
            for (Side &s : b->side) free_side(s);
            return st;
        }
    cudaGetDevice(&b->device);
    b->prepared = true;
    return RMAT_OK;
}

rmat_status rmat_batch_launch(rmat_batch *b, rmat_stream_t stream) {
    clear_error();
    if (!b) return fail(RMAT_ERR_INVALID_ARGUMENT, "batch is NULL");
    if (!b->prepared)
        if (rmat_status st = rmat_batch_prepare(b, nullptr)) return st;
    for (Side &s : b->side) {
        if (!s.units) continue;
        if (rmat_status st = launch_batch(s.u64, s.args, s.grid, s.threads, s.smem,
                                          reinterpret_cast<cudaStream_t>(stream)))
            return st;
    }
    return RMAT_OK;
}

rmat_status rmat_batch_size(const rmat_batch *b, uint64_t *graphs, uint64_t *edges) {
    clear_error();
    if (!b) return fail(RMAT_ERR_INVALID_ARGUMENT, "batch is NULL");
    if (graphs) *graphs = b->entries.size();
    if (edges) *edges = b->edges;
    return RMAT_OK;
}

void rmat_batch_free(rmat_batch *b) {
    if (!b) return;
    for (Side &s : b->side) free_side(s);
    delete b;
}

}  // extern "C"
