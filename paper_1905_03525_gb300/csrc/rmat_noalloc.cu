// rmat_noalloc.cu -- batched generation for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc: processes whose device memory is
// entirely reserved up front by another framework's caching allocator, code
// on a latency-critical path that must not take the driver's allocation locks
// (cudaMalloc/cudaFree can synchronise the device), and environments with a
// fixed, audited memory budget.  rmat_generate_batch_noalloc serves them: it
// runs the batched persistent kernel with all of its scratch -- work counter,
// job list, unit-to-job map and the packed table blobs -- in one file-scope
// device array of fixed size, so it allocates nothing.  The caller still
// passes the tables (host objects) and the output buffers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "rmat_internal.h"
#include "rmat_kernels.h"

namespace rmat {
namespace {

// Scratch of the no-allocation entry point.  Every GPU that loads the library
// holds it until the process exits.  In host code the name is only a
// host-side stand-in: the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[RMAT_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_scratch_ptr[kMaxDevices] = {};  // device address of the scratch, per device
bool g_kernels_loaded[kMaxDevices] = {};           // batched kernel loaded on the device

// Host staging of one call's scratch image (static: the call allocates
// nothing; the mutex serialises calls on the host).
unsigned char g_host_image[RMAT_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch on device `dev` (current), looked up once per
// device; the first lookup also loads the batched kernel there.  Called with
// g_mu held.
rmat_status scratch_address(int dev, unsigned char **out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(RMAT_ERR_UNSUPPORTED, "device ordinal out of range");
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return fail(RMAT_ERR_CUDA, std::string("cudaGetSymbolAddress(no-alloc scratch): ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_ptr[dev];
    if (!g_kernels_loaded[dev]) {
        if (rmat_status st = load_batch_kernels()) return st;
        g_kernels_loaded[dev] = true;
    }
    return RMAT_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace rmat

using namespace rmat;

extern "C" rmat_status rmat_generate_batch_noalloc(const rmat_table *const *tables, const uint64_t *seeds,
                                                   const uint64_t *edge_offsets, const uint64_t *counts,
                                                   void *const *outs, uint32_t n, rmat_stream_t stream_) {
    clear_error();
    if (n == 0) {
        // Set-up only: the scratch's device address (loading its module) and
        // the batched kernel's code on this device, so that later calls find
        // everything resident -- nothing is launched.
        int dev = 0;
        const cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return fail(RMAT_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        DeviceProps props;
        if (rmat_status st = device_props(props)) return st;
        std::lock_guard<std::mutex> lk(g_mu);
        unsigned char *scratch = nullptr;
        return scratch_address(dev, &scratch);
    }
    if (!tables || !seeds || !edge_offsets || !counts || !outs)
        return fail(RMAT_ERR_INVALID_ARGUMENT, "NULL argument array");
    if (n > RMAT_NOALLOC_MAX_GRAPHS)
        return fail(RMAT_ERR_INVALID_ARGUMENT, "more graphs than RMAT_NOALLOC_MAX_GRAPHS in one no-alloc call");
    bool u64 = false;
    for (uint32_t i = 0; i < n; ++i) {
        if (!tables[i]) return fail(RMAT_ERR_INVALID_ARGUMENT, "NULL table");
        if (tables[i]->n0 > 2)
            return fail(RMAT_ERR_UNSUPPORTED, "Kronecker tables (n0 > 2) are generated by rmat_generate only");
        if (counts[i] && !outs[i]) return fail(RMAT_ERR_INVALID_ARGUMENT, "NULL output pointer");
        if (reinterpret_cast<uintptr_t>(outs[i]) & 7u)
            return fail(RMAT_ERR_INVALID_ARGUMENT, "output must be 8-byte aligned");
        if (counts[i] > RMAT_MAX_EDGES) return fail(RMAT_ERR_INVALID_ARGUMENT, "count above RMAT_MAX_EDGES");
        if (counts[i] > ~uint64_t(0) - edge_offsets[i])
            return fail(RMAT_ERR_INVALID_ARGUMENT, "edge_offset + count overflows 64 bits");
        if (i == 0) u64 = tables[0]->k > 32;
        if ((tables[i]->k > 32) != u64)
            return fail(RMAT_ERR_INVALID_ARGUMENT, "one no-alloc call takes tables of one output width (all k <= 32 or all k > 32)");
    }

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(RMAT_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    DeviceProps props;
    if (rmat_status st = device_props(props)) return st;

    std::lock_guard<std::mutex> lk(g_mu);
    unsigned char *scratch = nullptr;
    if (rmat_status st = scratch_address(dev, &scratch)) return st;

    // Launch shape of the batched kernel (as rmat_batch_prepare's default):
    // 512-edge tiles (256 for u64), halved while the largest table would not
    // fit in shared memory beside them.
    int threads = 1024;
    size_t largest_blob = 0;
    for (uint32_t i = 0; i < n; ++i) largest_blob = std::max(largest_blob, tables[i]->image.size() * 4);
    int tile = u64 ? 256 : 512;
    while (tile > (u64 ? 128 : 256) &&
           kBatchHeaderBytes + size_t(threads / 32) * warp_bytes(u64, false, tile) + largest_blob > size_t(props.max_smem))
        tile /= 2;
    const size_t per_warp = warp_bytes(u64, false, tile);
    while (kBatchHeaderBytes + size_t(threads / 32) * per_warp > size_t(props.max_smem) && threads > 128) threads /= 2;
    const size_t budget = size_t(props.max_smem) - kBatchHeaderBytes - size_t(threads / 32) * per_warp;
    const uint64_t unit_edges = uint64_t(threads / 32) * tile * 16;  // as rmat_batch_prepare

    // Scratch layout: [counter][jobs][relabelling constants][unit -> job][table blobs].
    uint64_t units = 0;
    for (uint32_t i = 0; i < n; ++i) units += (counts[i] + unit_edges - 1) / unit_edges;
    const size_t off_jobs = 256;
    const size_t off_scr = align256(off_jobs + sizeof(Job) * n);
    const size_t off_units = align256(off_scr + sizeof(Scramble) * n);
    size_t off_blobs = align256(off_units + sizeof(uint32_t) * units);
    if (units > RMAT_NOALLOC_SCRATCH_BYTES / 4 || off_blobs > RMAT_NOALLOC_SCRATCH_BYTES)
        return fail(RMAT_ERR_INVALID_ARGUMENT, "too many edges for the no-alloc scratch");
    size_t blob_off[RMAT_NOALLOC_MAX_GRAPHS];
    size_t end = off_blobs;
    uint32_t max_blob = 0;
    for (uint32_t i = 0; i < n; ++i) {
        blob_off[i] = end;
        for (uint32_t j = 0; j < i; ++j)
            if (tables[j] == tables[i]) blob_off[i] = blob_off[j];
        if (blob_off[i] != end) continue;
        const size_t bytes = tables[i]->image.size() * 4;
        end = align256(end + bytes);
        if (end > RMAT_NOALLOC_SCRATCH_BYTES)
            return fail(RMAT_ERR_INVALID_ARGUMENT, "tables exceed the no-alloc scratch (RMAT_NOALLOC_SCRATCH_BYTES)");
        if (bytes <= budget) max_blob = std::max<uint32_t>(max_blob, uint32_t(bytes));
    }

    // Build the image on the host, then one copy into the scratch.  The
    // counter starts at zero (the launch below also clears it on the stream).
    std::memset(g_host_image, 0, off_blobs);
    Job *jobs = reinterpret_cast<Job *>(g_host_image + off_jobs);
    Scramble *scrs = reinterpret_cast<Scramble *>(g_host_image + off_scr);
    uint32_t *unit_job = reinterpret_cast<uint32_t *>(g_host_image + off_units);
    uint64_t u = 0;
    for (uint32_t i = 0; i < n; ++i) {
        const rmat_table *t = tables[i];
        const uint32_t *dblob = reinterpret_cast<const uint32_t *>(scratch + blob_off[i]);
        const bool smem = t->image.size() * 4 <= budget;
        jobs[i] = make_job(t, dblob, smem, seeds[i], edge_offsets[i], counts[i], outs[i]);
        jobs[i].unit_begin = u;
        scrs[i] = make_scramble(t);
        const uint64_t nu = (counts[i] + unit_edges - 1) / unit_edges;
        for (uint64_t k = 0; k < nu; ++k) unit_job[u + k] = i;
        u += nu;
        std::memcpy(g_host_image + blob_off[i], t->image.data(), t->image.size() * 4);
    }
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    // Pageable source: for a host-to-device copy from pageable memory the
    // runtime copies the source into its own staging memory before
    // cudaMemcpyAsync returns (CUDA Runtime API, "API synchronization
    // behavior"), so the next call may rewrite the static host image while
    // this copy is still queued on the stream.
    e = cudaMemcpyAsync(scratch, g_host_image, end, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return fail(RMAT_ERR_CUDA, std::string("scratch upload: ") + cudaGetErrorString(e));
    if (units == 0) return RMAT_OK;

    const size_t smem = batch_smem_bytes(u64, threads, tile, max_blob);
    int per_sm = 0;
    if (rmat_status st = batch_occupancy(u64, threads, smem, per_sm)) return st;
    if (per_sm < 1) return fail(RMAT_ERR_UNSUPPORTED, "launch shape does not fit on an SM");
    BatchArgs args{};
    args.jobs = reinterpret_cast<const Job *>(scratch + off_jobs);
    args.scr = reinterpret_cast<const Scramble *>(scratch + off_scr);
    args.unit_job = reinterpret_cast<const uint32_t *>(scratch + off_units);
    args.units = units;
    args.unit_edges = unit_edges;
    args.counter = reinterpret_cast<unsigned long long *>(scratch);
    args.max_blob_bytes = max_blob;
    args.tile = tile;
    args.err = props.err;
    for (uint32_t i = 0; i < n; ++i) args.general |= tables[i]->scramble ? 1 : 0;
    const int grid = int(std::min<uint64_t>(uint64_t(props.sms) * per_sm, units));
    return launch_batch(u64, args, grid, threads, smem, stream);
}
