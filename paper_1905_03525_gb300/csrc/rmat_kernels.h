// rmat_kernels.h -- host-side interface of the kernel translation unit.
#pragma once

#include <cuda_runtime.h>

#include "rmat_internal.h"

namespace rmat {

struct DeviceProps {
    bool valid = false;
    int sms = 0;
    int max_smem = 0;  // opt-in dynamic shared memory per block
    int cc = 0;
    unsigned *err = nullptr;  // device error flag
};

// One generation job: edges e0 .. e0+count-1 of the graph (table blob, seed),
// written to `out`.  Passed by value to k_alias, read from device memory by
// k_batch.
struct Job {
    const uint32_t *blob;  // device table blob (header + groups)
    uint32_t blob_bytes;
    int k;
    int draws1;            // draws in phase 1 (<= 4)
    int ngroups;
    unsigned flags;
    uint32_t ks[20];       // Philox round keys: seed + r * (Weyl constants), r = 0..9
    uint64_t e0, count;
    void *out;
    uint32_t fmt;          // image format
    uint32_t smem;         // blob staged in shared memory
    uint32_t levels;       // draw g uses group g
    uint32_t a0, bs0, ba0; // group 0: word offsets of A, Bs, Ba in the blob
    uint32_t bits0;        // group 0: b
    uint32_t one;          // 1 (a multiplier the compiler cannot fold: see dev::Acc32::append)
    uint64_t unit_begin;   // first work unit of this job (batches)
    // Batched jobs only: levels fixed before the first draw (the tile of a
    // partitioned graph), left-aligned in the accumulator word.
    uint64_t pre_row, pre_col;
    uint32_t pre_len;
};

// One tile of a partitioned graph for the contract-case partition kernel:
// its edges e0 .. e0 + count - 1 go to output slots out .. out + count - 1
// (edges from the start of the PE's output), in warp tiles wt0, wt0 + 1, ...
// of the launch; pre_* are the tile's levels, left-aligned in 32 bits.
struct PartTile {
    uint64_t e0, out, count, wt0;
    uint32_t pre_row, pre_col, pre_len, pad;
};

// Vertex relabelling constants of a job (used when flags & kScrambleFlag),
// in the form the kernels apply them: to an identifier held left-aligned in a
// W-bit word (W = 32 for k <= 32, else 64), s = W - k.  m[i] is the round's
// odd multiplier, a[i] its addend times 2^s (mod 2^W), mask = the top k bits.
// Kept out of Job so that the batched kernel's register copy of a job stays
// small.
struct Scramble {
    uint64_t m[3], a[3], mask;
};

// Job flag (beside RMAT_UNDIRECTED): relabel vertex IDs with Job::scr.
constexpr unsigned kScrambleFlag = 0x100u;

// Shared memory of the batched kernel ahead of the staged table: its mbarrier
// (8 bytes), the current work unit (8) and the job's Philox round keys (80).
constexpr size_t kBatchHeaderBytes = 96;

struct BatchArgs {
    const Job *jobs;
    const Scramble *scr;       // one per job
    const uint32_t *unit_job;  // job of every work unit
    uint64_t units;
    uint64_t unit_edges;
    unsigned long long *counter;
    uint32_t max_blob_bytes;   // shared bytes reserved for a staged blob
    int tile;
    unsigned *err;
    int general;               // some job is a partition tile (pre_len > 0) or relabels IDs
    int fast;                  // every job takes k_batch_fast (u32 compact shared-memory tables, plain epilogue)
};

// One launch of the Kronecker kernel (n0 > 2): edges e0 .. e0+count-1.
constexpr int kMaxKronK = 40;  // n0 >= 3: n0^k <= 2^64
struct KronJob {
    const uint32_t *blob;  // device image (header, AA, P, then the packed arrays when present)
    uint32_t blob_bytes;     // bytes the general kernel stages (header, AA, P)
    uint32_t aa_off, p_off;  // byte offsets of AA and P in the image
    uint32_t mulb;           // 2^b: column j = umulhi(u, 2^b)
    uint32_t c_off, c_bytes; // packed arrays (A32, P32, powers): byte offset and size; c_bytes = 0 if absent
    uint32_t c_shift;        // bits per coordinate in a packed path
    uint32_t bits;           // b
    int k;
    uint32_t ks[20];         // Philox round keys of the seed
    uint64_t e0, count;
    void *out;
    uint64_t pw[kMaxKronK + 1];  // n0^j
    uint64_t mg[33];             // floor(2^64 / n0^d) + 1: floor(x / n0^d) = umul64hi(x, mg[d]) for x < 2^32
};

rmat_status device_props(DeviceProps &out);
// One warp waiting on a never-completed mbarrier phase, bounded to `limit` polls.
rmat_status launch_wait_selftest(uint32_t limit, cudaStream_t stream);
rmat_launch_config_t default_launch_config(const rmat_table *t);
rmat_status plan_alias_launch(const rmat_table *t, const rmat_launch_config_t &want, AliasPlan &plan);
Job make_job(const rmat_table *t, const uint32_t *dblob, bool smem, uint64_t seed, uint64_t e0, uint64_t count,
             void *out);
Scramble make_scramble(const rmat_table *t);
// Start every edge of a batched job inside tile (R, C) of a depth-`levels`
// partition: the tile's levels are fixed, the draws fill the other k - levels.
void set_tile_prefix(Job &J, const rmat_table *t, int levels, uint64_t R, uint64_t C);
// Every tile of a partition (u32 compact tables that take k_alias_fast) in one
// launch of k_part_fast; `tiles` (device, ntiles entries, non-empty tiles in
// output order) cover nwt warp tiles of plan.tile edges.
rmat_status launch_partition_fast(const rmat_table *t, const uint32_t *dblob, const AliasPlan &plan, uint64_t seed,
                                  const PartTile *tiles, uint32_t ntiles, uint64_t nwt, void *out,
                                  cudaStream_t stream);
rmat_status launch_alias(const rmat_table *t, const uint32_t *dblob, const AliasPlan &plan, uint64_t seed,
                         uint64_t e0, uint64_t count, void *out, cudaStream_t stream);
size_t warp_bytes(bool u64, bool levels, int tile);
size_t batch_smem_bytes(bool u64, int threads, int tile, uint32_t max_blob_bytes);
rmat_status batch_occupancy(bool u64, int threads, size_t smem, int &per_sm);
rmat_status launch_batch(bool u64, const BatchArgs &args, int grid, int threads, size_t smem, cudaStream_t stream);
// Load every variant of the batched kernel on the current device now (code
// and attributes), so that no later launch has module loading to do.
rmat_status load_batch_kernels();
rmat_status launch_checksum(bool u64, const BatchArgs &args, unsigned long long *sums, int grid,
                            cudaStream_t stream);
rmat_status launch_naive(const uint32_t *thr3, int k, unsigned flags, uint64_t seed, uint64_t e0,
                         uint64_t count, void *out, cudaStream_t stream);
rmat_status read_and_clear_device_error(unsigned &value);

}  // namespace rmat
