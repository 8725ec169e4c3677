// rmat_dedup.cu -- removal of repeated edges (Sec. 3: generating partitioned
// graphs makes duplicate elimination a local operation, since two equal edges
// fall into the same tile and so onto the same PE).
//
// The first occurrence of every (row, col), in the order of the input, stays;
// the survivors are compacted to the front in that order, so the result is a
// pure function of the input array.  Three passes over the edges:
//   1. insert key = row * 2^k + col into an open-addressing hash table of
//      16-byte slots {key, first index} (linear probing): one 128-bit CAS
//      claims a free slot with the edge's key and index; an edge that finds
//      its key already there lowers the slot's first index with atomicMin
//      when its own index is smaller; each edge remembers its slot;
//   2. an edge survives iff it holds its slot's first index: one flag byte
//      per edge and per-chunk counts;
//   3. exclusive scan of the chunk counts, then an ordered chunk-local
//      compaction driven by the flags (sequential reads) into a second
//      buffer, copied back.
// The table has at least twice as many slots as edges; every probe loop is
// bounded by the table size and reports an error instead of spinning.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "rmat_internal.h"
#include "rmat_kernels.h"

namespace rmat {
namespace {

constexpr uint64_t kEmpty = ~uint64_t(0);
constexpr int kBlock = 1024;
constexpr int kPerThread = 4;                      // edges per thread in the compaction
static_assert(kPerThread == 4, "k_dedup_count stores a thread's flags as one 4-byte word");
constexpr uint64_t kChunk = uint64_t(kBlock) * kPerThread;

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    // splitmix64 finaliser (Steele, Lea, Flood 2014) as the hash
    x ^= x >> 30;
    x *= 0xBF58476D1CE4E5B9ull;
    x ^= x >> 27;
    x *= 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__device__ __forceinline__ uint64_t edge_key(const uint2 *e, uint64_t i, int k) {
    const uint2 v = e[i];
    return (uint64_t(v.x) << k) | v.y;
}

// 128-bit compare-and-swap (PTX atom.cas.b128, sm_90 and later) on the
// 16-byte-aligned pair {lo at addr, hi at addr + 8}; returns the old pair.
__device__ __forceinline__ void cas128(unsigned long long *addr, uint64_t cmp_lo, uint64_t cmp_hi, uint64_t new_lo,
                                       uint64_t new_hi, uint64_t &old_lo, uint64_t &old_hi) {
    asm volatile(
        "{\n\t.reg .b128 c, n, o;\n\t"
        "mov.b128 c, {%2, %3};\n\t"
        "mov.b128 n, {%4, %5};\n\t"
        "atom.global.cas.b128 o, [%6], c, n;\n\t"
        "mov.b128 {%0, %1}, o;\n\t}"
        : "=l"(old_lo), "=l"(old_hi)
        : "l"(cmp_lo), "l"(cmp_hi), "l"(new_lo), "l"(new_hi), "l"(addr)
        : "memory");
}

// Slot h of the table: tab[2h] = key (kEmpty when free), tab[2h + 1] = the
// smallest index of an edge with that key (all ones while free).  A slot
// leaves the free state once, by the CAS that writes both words; after that
// only its index word changes, by atomicMin.
__global__ void k_dedup_insert(const uint2 *edges, uint64_t n, int k, unsigned long long *tab, uint64_t mask,
                               uint32_t *slot_of, unsigned *err) {
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t key = edge_key(edges, i, k);
        uint64_t h = mix64(key) & mask;
        bool placed = false;
        for (uint64_t probe = 0; probe <= mask; ++probe) {  // at most one pass over the table
            uint64_t old_key, old_first;
            cas128(tab + 2 * h, kEmpty, kEmpty, key, i, old_key, old_first);
            if (old_key == kEmpty || old_key == key) {
                if (old_key == key && i < old_first) atomicMin(tab + 2 * h + 1, (unsigned long long)i);
                slot_of[i] = uint32_t(h);
                placed = true;
                break;
            }
            h = (h + 1) & mask;
        }
        if (!placed) atomicOr(err, 2u);
    }
}

// Survivor flags of chunk `c` (kChunk edges, thread t holds edges
// c*kChunk + t*kPerThread + j; one byte per edge) and the chunk's count.
__global__ void __launch_bounds__(kBlock) k_dedup_count(uint64_t n, const uint32_t *slot_of,
                                                        const unsigned long long *tab, uint8_t *flag,
                                                        uint32_t *chunk_count) {
    __shared__ uint32_t warp_sum[kBlock / 32];
    const uint64_t base = blockIdx.x * kChunk + uint64_t(threadIdx.x) * kPerThread;
    uint32_t c = 0, bits = 0;
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) {
        const uint64_t i = base + j;
        if (i < n && tab[2 * uint64_t(slot_of[i]) + 1] == i) {
            ++c;
            bits |= 1u << (8 * j);
        }
    }
    if (base + kPerThread <= n) {
        *reinterpret_cast<uint32_t *>(flag + base) = bits;  // kPerThread == 4 flag bytes
    } else {
#pragma unroll
        for (int j = 0; j < kPerThread; ++j)
            if (base + j < n) flag[base + j] = uint8_t(bits >> (8 * j));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kBlock / 32; ++w) t += warp_sum[w];
        chunk_count[blockIdx.x] = t;
    }
}

// Exclusive scan of the chunk counts in place (one block; chunks up to ~2^22).
__global__ void __launch_bounds__(kBlock) k_dedup_scan(uint32_t *counts, uint64_t chunks, unsigned long long *total) {
    __shared__ uint32_t sm[kBlock / 32];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint64_t b0 = 0; b0 < chunks; b0 += kBlock) {
        const uint64_t b = b0 + threadIdx.x;
        const uint32_t v = b < chunks ? counts[b] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) sm[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t y = sm[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t z = __shfl_up_sync(0xffffffffu, y, o);
                if (lane >= o) y += z;
            }
            sm[lane] = y;
        }
        __syncthreads();
        const uint64_t excl = carry + (x - v) + (warp ? sm[warp - 1] : 0u);
        if (b < chunks) counts[b] = uint32_t(excl);  // offsets within one call stay below 2^32 edges
        __syncthreads();
        if (threadIdx.x == 0) carry += sm[kBlock / 32 - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

// Ordered compaction of chunk `c` to dst starting at offsets[c].
__global__ void __launch_bounds__(kBlock) k_dedup_compact(const uint2 *edges, uint64_t n, const uint8_t *flag,
                                                          const uint32_t *offsets, uint2 *dst) {
    __shared__ uint32_t warp_base[kBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t base = blockIdx.x * kChunk + uint64_t(threadIdx.x) * kPerThread;
    uint32_t keep = 0, c = 0;
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) {
        const uint64_t i = base + j;
        if (i < n && flag[i]) {
            keep |= 1u << j;
            ++c;
        }
    }
    uint32_t x = c;  // inclusive scan over the warp, then over the warps
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_base[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t y = warp_base[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t z = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += z;
        }
        warp_base[lane] = y;
    }
    __syncthreads();
    uint64_t out = uint64_t(offsets[blockIdx.x]) + (x - c) + (warp ? warp_base[warp - 1] : 0u);
#pragma unroll
    for (int j = 0; j < kPerThread; ++j)
        if (keep & (1u << j)) dst[out++] = edges[base + j];
}

}  // namespace
}  // namespace rmat

using namespace rmat;

extern "C" rmat_status rmat_dedup_edges(void *edges, uint64_t count, int k, uint64_t *unique,
                                        rmat_stream_t stream_) {
    clear_error();
    if (!unique) return fail(RMAT_ERR_INVALID_ARGUMENT, "unique is NULL");
    *unique = 0;
    if (k < 1 || k > 31) return fail(RMAT_ERR_INVALID_ARGUMENT, "duplicate removal takes k in [1, 31]");
    if (count == 0) return RMAT_OK;
    if (!edges) return fail(RMAT_ERR_INVALID_ARGUMENT, "edges is NULL");
    if (reinterpret_cast<uintptr_t>(edges) & 7u) return fail(RMAT_ERR_INVALID_ARGUMENT, "edges must be 8-byte aligned");
    if (count > (uint64_t(1) << 31)) return fail(RMAT_ERR_INVALID_ARGUMENT, "at most 2^31 edges per call");
    DeviceProps props;
    if (rmat_status st = device_props(props)) return st;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);

    uint64_t slots = 1;
    while (slots < 2 * count) slots <<= 1;
    const uint64_t chunks = (count + kChunk - 1) / kChunk;
    // scratch: the table (key, first index) per slot, slot per edge, flag
    // byte per edge, chunk counts, the compacted copy, the total and an error
    // word
    const size_t off_slot = slots * 16;
    const size_t off_flag = off_slot + ((count * 4 + 255) & ~size_t(255));
    const size_t off_cnt = off_flag + ((count + 255) & ~size_t(255));
    const size_t off_dst = off_cnt + ((chunks * 4 + 255) & ~size_t(255));
    const size_t off_tot = off_dst + count * 8;
    const size_t bytes = off_tot + 16;
    unsigned char *scratch = nullptr;
    if (cudaMalloc(&scratch, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(RMAT_ERR_OUT_OF_MEMORY, "device scratch for duplicate removal");
    }
    auto *tab = reinterpret_cast<unsigned long long *>(scratch);
    auto *slot_of = reinterpret_cast<uint32_t *>(scratch + off_slot);
    auto *flag = reinterpret_cast<uint8_t *>(scratch + off_flag);
    auto *cnt = reinterpret_cast<uint32_t *>(scratch + off_cnt);
    auto *dst = reinterpret_cast<uint2 *>(scratch + off_dst);
    auto *total = reinterpret_cast<unsigned long long *>(scratch + off_tot);
    auto *err = reinterpret_cast<unsigned *>(scratch + off_tot + 8);
    const uint2 *src = static_cast<const uint2 *>(edges);
    const int grid = props.sms * 8;
    cudaError_t e = cudaMemsetAsync(tab, 0xFF, slots * 16, stream);  // kEmpty keys, first = max
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, 4, stream);
    if (e == cudaSuccess) {
        k_dedup_insert<<<grid, 256, 0, stream>>>(src, count, k, tab, slots - 1, slot_of, err);
        k_dedup_count<<<unsigned(chunks), kBlock, 0, stream>>>(count, slot_of, tab, flag, cnt);
        k_dedup_scan<<<1, kBlock, 0, stream>>>(cnt, chunks, total);
        k_dedup_compact<<<unsigned(chunks), kBlock, 0, stream>>>(src, count, flag, cnt, dst);
        e = cudaGetLastError();
    }
    unsigned long long host_total = 0;
    unsigned host_err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host_total, total, 8, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host_err, err, 4, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e == cudaSuccess && !host_err && host_total)
        e = cudaMemcpyAsync(edges, dst, host_total * 8, cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    cudaFree(scratch);
    if (e != cudaSuccess) return fail(RMAT_ERR_CUDA, std::string("duplicate removal: ") + cudaGetErrorString(e));
    if (host_err) return fail(RMAT_ERR_CUDA, "duplicate removal: hash table full (internal error)");
    *unique = host_total;
    return RMAT_OK;
}
