// rmat_dedup.cu -- removal of repeated edges (Sec. 3: generating partitioned
// graphs makes duplicate elimination a local operation, since two equal edges
// fall into the same tile and so onto the same PE).
//
// The first occurrence of every (row, col), in the order of the input, stays;
// the survivors are compacted to the front in that order, so the result is a
// pure function of the input array.  Two radix passes on a hash of the key
// cut the edges into buckets small enough for one CTA's shared memory, and
// every bucket is deduplicated there; nothing random touches device memory
// but one bit per repeated edge:
//   1. histogram of the level-1 digit, the top B1 bits of h = mix64(key),
//      key = row * 2^k + col, and its exclusive scan on the device;
//   2. scatter of {h, index} into the level-1 buckets, a tile at a time,
//      staged in shared memory so that every run is written in one burst
//      (mix64 is a bijection, so equal hashes mean equal edges and later
//      passes need neither the key nor the hash function);
//   3. when the edges need more than 2^B1 buckets, one CTA per level-1 bucket
//      counts the next B2 bits of h, scans them and scatters its edges into
//      its sub-buckets (a second buffer, staged the same way), for
//      2^(B1+B2) buckets of at most ~2048 edges on average;
//   4. one CTA per bucket: the bucket's hashes staged in shared memory and an
//      open-addressing table there (a 32-bit CAS claims a slot for the entry
//      that first brings a key, a 32-bit atomicMin keeps the smallest edge
//      index of that key); every edge that is not its key's smallest index
//      clears its bit in a survivor bitmap that starts all ones.  A bucket
//      too large for shared memory (many copies of few keys) is listed and
//      done afterwards in a device-memory table, one bucket after another;
//   5. per-chunk survivor counts, one-block scan, ordered chunk-local
//      compaction into a spare buffer, copied back.
// The scratch (about 24 bytes per edge) is kept between calls.  Every probe
// loop is bounded by its table's size and reports an error instead of
// spinning.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "rmat_device.cuh"
#include "rmat_internal.h"
#include "rmat_kernels.h"

namespace rmat {
namespace {

constexpr uint64_t kFree = ~uint64_t(0);           // fill of the overflow table: bucket number 0xFFFFFFFF
constexpr int kBlock = 1024;
constexpr int kPerThread = 4;                      // edges per thread in the compaction
constexpr uint64_t kChunk = uint64_t(kBlock) * kPerThread;
constexpr int kL1MaxBits = 10;                     // level-1 buckets: at most 1024
constexpr int kMaxBits = 20;                       // buckets in all: at most 2^20
constexpr int kL2MaxBits = kMaxBits - kL1MaxBits;  // sub-buckets per level-1 bucket: at most 1024
constexpr uint64_t kLocalTarget = 2048;            // mean edges per bucket, at most
constexpr uint32_t kLocalMax = 3072;               // largest bucket done in shared memory
constexpr uint32_t kLocalSlots = 4096;             // its table: load <= 0.75
constexpr int kLocalThreads = 512;
constexpr int kLocalCtas = 4;                      // per SM (56 KB of shared memory each)
constexpr int kLocalPer = 2;                       // edges per thread and batch
constexpr size_t kLocalSmem = size_t(kLocalMax) * 8 + size_t(kLocalSlots) * 8;  // hashes; owners, smallest indices

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    // splitmix64 finaliser (Steele, Lea, Flood 2014) as the hash; a bijection
    // of 64-bit words
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

// The top `bits` bits of a hash (0 when bits = 0).
__device__ __forceinline__ uint32_t top_bits(uint64_t h, int bits) { return bits ? uint32_t(h >> (64 - bits)) : 0u; }

// Exclusive prefix sum over a block of NT threads (a multiple of 32, at most
// 1024), one value each; `ws` holds 32 words.  Every thread of the block
// calls it.
template <int NT>
__device__ __forceinline__ uint32_t block_exclusive(uint32_t v, uint32_t *ws) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t y = lane < NT / 32 ? ws[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t z = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += z;
        }
        ws[lane] = y;
    }
    __syncthreads();
    return x - v + (warp ? ws[warp - 1] : 0u);
}

// 1. Level-1 bucket sizes: a block histogram in shared memory, added to `counts`.
__global__ void __launch_bounds__(kBlock) k_dd_hist(const uint2 *edges, uint64_t n, int k, int bits,
                                                    uint32_t *counts) {
    __shared__ uint32_t h[1u << kL1MaxBits];
    const uint32_t nb = 1u << bits;
    for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) h[b] = 0;
    __syncthreads();
    // four edges per thread in flight
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i0 = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i0 < n; i0 += 4 * stride) {
        uint64_t key[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint64_t i = i0 + u * stride;
            key[u] = i < n ? edge_key(edges, i, k) : 0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (i0 + u * stride < n) atomicAdd(&h[top_bits(mix64(key[u]), bits)], 1u);
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x)
        if (h[b]) atomicAdd(&counts[b], h[b]);
}

// 2. Level-1 scatter, one tile of kScatterTile edges at a time (persistent
// blocks): every edge's bucket and rank within the tile come from
// shared-memory counters; one atomic per bucket and tile reserves a run from
// the bucket cursors; the tile is staged in shared memory sorted by bucket,
// and written out so that consecutive threads write consecutive entries of a
// run (a run is written in one burst, so L2 merges the partial lines at its
// ends with the neighbouring runs instead of evicting them half written).
// When `edges` is 16-byte aligned, the next tile is fetched into shared
// memory by a bulk copy while this one is ranked, staged and written (an
// odd last edge of a tile is read directly).
constexpr int kScatterTile = 8192;
constexpr int kScatterPer = kScatterTile / kBlock;
constexpr size_t kScatterIn = 16;                                   // after the mbarrier
constexpr size_t kScatterKey = kScatterIn + size_t(kScatterTile) * 8;
constexpr size_t kScatterPos = kScatterKey + size_t(kScatterTile) * 8;
constexpr size_t kScatterDig = kScatterPos + size_t(kScatterTile) * 2;
constexpr size_t kScatterCnt = kScatterDig + size_t(kScatterTile) * 2;
constexpr size_t kScatterSmem = kScatterCnt + 3 * 4 * (size_t(1) << kL1MaxBits);
constexpr uint32_t kWaitLimit = 1u << 22;                           // polls of a bounded mbarrier wait
static_assert((1 << kL1MaxBits) <= kBlock, "one bucket counter per thread of the scatter");
__global__ void __launch_bounds__(kBlock, 1) k_dd_scatter(const uint2 *edges, uint64_t n, int k, int bits,
                                                          uint32_t *cursor, uint64_t *bhash, uint32_t *bidx,
                                                          unsigned *err) {
    extern __shared__ __align__(16) unsigned char dsm[];
    auto *mbar = reinterpret_cast<uint64_t *>(dsm);
    auto *in = reinterpret_cast<uint2 *>(dsm + kScatterIn);
    auto *skey = reinterpret_cast<uint64_t *>(dsm + kScatterKey);
    auto *spos = reinterpret_cast<uint16_t *>(dsm + kScatterPos);
    auto *sdig = reinterpret_cast<uint16_t *>(dsm + kScatterDig);
    auto *cnt = reinterpret_cast<uint32_t *>(dsm + kScatterCnt);
    uint32_t *off = cnt + (1u << kL1MaxBits);
    uint32_t *gbase = off + (1u << kL1MaxBits);
    __shared__ uint32_t ws[32];
    const uint32_t t = threadIdx.x;
    const uint64_t tiles = (n + kScatterTile - 1) / kScatterTile;
    const bool tma = (reinterpret_cast<uintptr_t>(edges) & 15u) == 0;
    // edges of tile `tile` that the bulk copy brings (an even number)
    auto copied = [&](uint64_t tile) -> uint32_t {
        if (!tma || tile >= tiles) return 0u;
        const uint64_t t0 = tile * kScatterTile;
        return uint32_t(min(uint64_t(kScatterTile), n - t0)) & ~1u;
    };
    auto issue = [&](uint64_t tile) {  // thread 0
        const uint32_t c = copied(tile);
        if (!c) return;
        dev::fence_proxy_async_smem();
        dev::mbar_arrive_expect_tx(mbar, c * 8u);
        const unsigned char *src = reinterpret_cast<const unsigned char *>(edges + tile * kScatterTile);
        for (uint32_t o = 0; o < c * 8u; o += 32768u)
            dev::bulk_g2s(reinterpret_cast<unsigned char *>(in) + o, src + o, min(32768u, c * 8u - o), mbar);
    };
    if (t == 0) {
        dev::mbar_init(mbar, 1);
        dev::fence_mbar_init();
    }
    cnt[t] = 0;
    __syncthreads();
    if (t == 0) issue(blockIdx.x);
    uint32_t parity = 0;
    for (uint64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const uint64_t t0 = tile * kScatterTile;
        const uint32_t tn = uint32_t(min(uint64_t(kScatterTile), n - t0));
        const uint32_t nc = copied(tile);
        if (nc) {
            const bool ok = __syncthreads_and(dev::mbar_wait_bounded(mbar, parity, kWaitLimit)) != 0;
            parity ^= 1u;
            if (!ok) {  // never expected: give the copy one more bounded wait, then stop
                if (t == 0) atomicOr(err, 16u);
                dev::mbar_wait_bounded(mbar, parity ^ 1u, kWaitLimit);
                return;
            }
        }
        uint64_t h[kScatterPer];
        uint32_t dig[kScatterPer], rank[kScatterPer];
#pragma unroll
        for (int u = 0; u < kScatterPer; ++u) {
            const uint32_t i = u * kBlock + t;
            uint2 v = make_uint2(0, 0);
            if (i < nc) v = in[i];
            else if (i < tn) v = edges[t0 + i];
            h[u] = (uint64_t(v.x) << k) | v.y;
        }
        __syncthreads();  // the copy buffer is free
        if (t == 0) issue(tile + gridDim.x);
#pragma unroll
        for (int u = 0; u < kScatterPer; ++u) {
            h[u] = mix64(h[u]);
            dig[u] = top_bits(h[u], bits);
            rank[u] = u * kBlock + t < tn ? atomicAdd(&cnt[dig[u]], 1u) : 0u;
        }
        __syncthreads();
        const uint32_t c = cnt[t];  // 0 past the last bucket
        const uint32_t ex = block_exclusive<kBlock>(c, ws);
        off[t] = ex;
        const uint32_t gb = c ? atomicAdd(&cursor[t], c) : 0u;  // used after the staging
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kScatterPer; ++u) {
            const uint32_t i = u * kBlock + t;
            if (i >= tn) continue;
            const uint32_t p = off[dig[u]] + rank[u];
            skey[p] = h[u];
            spos[p] = uint16_t(i);
            sdig[p] = uint16_t(dig[u]);
        }
        gbase[t] = gb;
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kScatterPer; ++u) {
            const uint32_t p = u * kBlock + t;
            if (p >= tn) continue;
            const uint32_t d = sdig[p];
            const uint32_t g = gbase[d] + (p - off[d]);
            bhash[g] = skey[p];
            bidx[g] = uint32_t(t0) + spos[p];
        }
        cnt[t] = 0;
        __syncthreads();
    }
}

// 3. Level-2 split of level-1 bucket b = blockIdx.x, entries [lo1[b], hi1[b])
// of (akey, aidx): counts of the digit (h >> (64 - B)) mod 2^B2 (the bits
// below the level-1 digit) over the bucket, their scan, the start of every
// sub-bucket in sub_start[b * 2^B2 + d]; then the bucket a tile of
// kSplitTile entries at a time, staged in shared memory sorted by sub-bucket
// as in the level-1 scatter, into (bkey, bidx).  The block owns its bucket, so
// the sub-bucket cursors live in shared memory.  The next tile comes into
// shared memory by two bulk copies (hashes and indices, widened to 16-byte
// boundaries) while this one is ranked, staged and written.  One block per
// SM; each thread owns kSplitDpt sub-bucket counters.
constexpr int kSplitThreads = 1024;
constexpr int kSplitTile = 8192;
constexpr int kSplitPer = kSplitTile / kSplitThreads;
constexpr uint32_t kSplitDigits = 1u << kL2MaxBits;
constexpr int kSplitDpt = int(kSplitDigits) / kSplitThreads;
static_assert(kSplitDpt * kSplitThreads == int(kSplitDigits), "whole sub-bucket counters per thread of the split");
constexpr size_t kSplitInH = 16;                                     // after the mbarrier
constexpr size_t kSplitInI = kSplitInH + size_t(kSplitTile + 8) * 8;
constexpr size_t kSplitKey = kSplitInI + size_t(kSplitTile + 8) * 4;
constexpr size_t kSplitIdx = kSplitKey + size_t(kSplitTile) * 8;
constexpr size_t kSplitCnt = kSplitIdx + size_t(kSplitTile) * 4;
constexpr size_t kSplitSmem = kSplitCnt + 4 * 4 * size_t(kSplitDigits);
__global__ void __launch_bounds__(kSplitThreads, 1) k_dd_split(const uint64_t *akey, const uint32_t *aidx,
                                                               const uint32_t *lo1, const uint32_t *hi1, int B,
                                                               int B2, uint64_t *bkey, uint32_t *bidx,
                                                               uint32_t *sub_start, unsigned *err) {
    extern __shared__ __align__(16) unsigned char dsm[];
    auto *mbar = reinterpret_cast<uint64_t *>(dsm);
    auto *inh = reinterpret_cast<uint64_t *>(dsm + kSplitInH);
    auto *ini = reinterpret_cast<uint32_t *>(dsm + kSplitInI);
    auto *skey = reinterpret_cast<uint64_t *>(dsm + kSplitKey);
    auto *sidx = reinterpret_cast<uint32_t *>(dsm + kSplitIdx);
    auto *cnt = reinterpret_cast<uint32_t *>(dsm + kSplitCnt);
    uint32_t *off = cnt + kSplitDigits;
    uint32_t *base = off + kSplitDigits;
    uint32_t *cur = base + kSplitDigits;
    __shared__ uint32_t ws[32];
    const uint32_t t = threadIdx.x, d0 = kSplitDpt * t;  // this thread's counters: d0 .. d0 + kSplitDpt - 1
    const uint32_t b = blockIdx.x, lo = lo1[b], hi = hi1[b];
    const uint32_t nd = 1u << B2, dmask = nd - 1;
    const int sh = 64 - B;
    auto digit = [&](uint64_t h) { return uint32_t(h >> sh) & dmask; };
    if (t == 0) {
        dev::mbar_init(mbar, 1);
        dev::fence_mbar_init();
    }
#pragma unroll
    for (int q = 0; q < kSplitDpt; ++q) cnt[d0 + q] = 0;
    __syncthreads();
    for (uint32_t j0 = lo + t; j0 < hi; j0 += 8 * kSplitThreads) {
        uint64_t key[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const uint32_t j = j0 + u * kSplitThreads;
            key[u] = j < hi ? akey[j] : 0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (j0 + u * kSplitThreads < hi) atomicAdd(&cnt[digit(key[u])], 1u);
    }
    __syncthreads();
    {
        uint32_t v[kSplitDpt], sum = 0;  // 0 past the last sub-bucket
#pragma unroll
        for (int q = 0; q < kSplitDpt; ++q) sum += (v[q] = cnt[d0 + q]);
        uint32_t e = lo + block_exclusive<kSplitThreads>(sum, ws);
#pragma unroll
        for (int q = 0; q < kSplitDpt; ++q) {
            if (d0 + q < nd) sub_start[(b << B2) + d0 + q] = e;
            cur[d0 + q] = e;
            cnt[d0 + q] = 0;
            e += v[q];
        }
    }
    __syncthreads();
    // the tile at j0: hashes [j0 & ~1, even end), indices [j0 & ~3, end rounded
    // up to 4), so that both copies start and end on 16-byte boundaries (the
    // widening reads at most three entries past the bucket, still inside the
    // scratch)
    auto issue = [&](uint32_t j0) {  // thread 0
        const uint32_t tn = min(uint32_t(kSplitTile), hi - j0);
        const uint32_t ah = j0 & ~1u, eh = (j0 + tn + 1) & ~1u;
        const uint32_t ai = j0 & ~3u, ei = (j0 + tn + 3) & ~3u;
        dev::fence_proxy_async_smem();
        dev::mbar_arrive_expect_tx(mbar, (eh - ah) * 8u + (ei - ai) * 4u);
        auto copy = [&](void *dst, const void *src, uint32_t bytes) {  // pieces of at most 32 KB
            for (uint32_t o = 0; o < bytes; o += 32768u)
                dev::bulk_g2s(static_cast<unsigned char *>(dst) + o, static_cast<const unsigned char *>(src) + o,
                              min(32768u, bytes - o), mbar);
        };
        copy(inh, akey + ah, (eh - ah) * 8u);
        copy(ini, aidx + ai, (ei - ai) * 4u);
    };
    if (t == 0 && lo < hi) issue(lo);
    uint32_t parity = 0;
    for (uint32_t j0 = lo; j0 < hi; j0 += kSplitTile) {
        const uint32_t tn = min(uint32_t(kSplitTile), hi - j0);
        const bool ok = __syncthreads_and(dev::mbar_wait_bounded(mbar, parity, kWaitLimit)) != 0;
        parity ^= 1u;
        if (!ok) {  // never expected: give the copy one more bounded wait, then stop
            if (t == 0) atomicOr(err, 32u);
            dev::mbar_wait_bounded(mbar, parity ^ 1u, kWaitLimit);
            return;
        }
        uint64_t key[kSplitPer];
        uint32_t idx[kSplitPer];
        const uint32_t dh = j0 & 1u, di = j0 & 3u;
#pragma unroll
        for (int u = 0; u < kSplitPer; ++u) {
            const uint32_t i = u * kSplitThreads + t;
            key[u] = i < tn ? inh[dh + i] : 0;
            idx[u] = i < tn ? ini[di + i] : 0;
        }
        __syncthreads();  // the copy buffers are free
        if (t == 0 && j0 + kSplitTile < hi) issue(j0 + kSplitTile);
        uint32_t dig[kSplitPer], rank[kSplitPer];
#pragma unroll
        for (int u = 0; u < kSplitPer; ++u) {
            dig[u] = digit(key[u]);
            rank[u] = u * kSplitThreads + t < tn ? atomicAdd(&cnt[dig[u]], 1u) : 0u;
        }
        __syncthreads();
        {
            uint32_t c[kSplitDpt], sum = 0;
#pragma unroll
            for (int q = 0; q < kSplitDpt; ++q) sum += (c[q] = cnt[d0 + q]);
            uint32_t o = block_exclusive<kSplitThreads>(sum, ws);
#pragma unroll
            for (int q = 0; q < kSplitDpt; ++q) {
                off[d0 + q] = o;
                base[d0 + q] = cur[d0 + q];
                cur[d0 + q] += c[q];
                o += c[q];
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kSplitPer; ++u) {
            if (u * kSplitThreads + t >= tn) continue;
            const uint32_t p = off[dig[u]] + rank[u];
            skey[p] = key[u];
            sidx[p] = idx[u];
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kSplitPer; ++u) {
            const uint32_t p = u * kSplitThreads + t;
            if (p >= tn) continue;
            const uint64_t hv = skey[p];
            const uint32_t d = digit(hv);
            bkey[base[d] + (p - off[d])] = hv;
            bidx[base[d] + (p - off[d])] = sidx[p];
        }
#pragma unroll
        for (int q = 0; q < kSplitDpt; ++q) cnt[d0 + q] = 0;
        __syncthreads();
    }
}

// 4. Bucket s = blockIdx.x, entries [starts[s], starts[s + 1]) (n for the
// last), deduplicated in shared memory.  The bucket's hashes are staged in
// shared memory (entry r at sh[r]; equal hashes, equal edges), and a table of
// T slots, a power of two at least twice the bucket (at most kLocalSlots, so a
// bucket of at most kLocalMax edges always finds a free slot within T probes),
// holds in own[slot] 1 + the entry that claimed it (0 = free; claimed by a
// 32-bit CAS) and in low[slot] the smallest edge index of that entry's key.
// A slot's owner never changes once set, and every copy of a key probes the
// same sequence, so all copies meet in one slot; each lowers low[] to its own
// index, and after the barrier every copy that does not hold the minimum
// clears its survivor bit.  A thread keeps its edges' indices and slots in
// registers (at most kLocalBatches x kLocalPer edges).  A larger bucket goes
// to the overflow list (ovf[0] = how many, ovf[1 + i] = bucket).
constexpr int kLocalBatches = int(kLocalMax / (kLocalPer * kLocalThreads));
static_assert(kLocalBatches * kLocalPer * kLocalThreads == int(kLocalMax), "whole batches per thread");
__global__ void __launch_bounds__(kLocalThreads, kLocalCtas) k_dd_local(const uint64_t *hash, const uint32_t *idx,
                                                               const uint32_t *starts, uint32_t nsub, uint32_t n,
                                                               uint32_t *bitmap, uint32_t *ovf, unsigned *err) {
    extern __shared__ __align__(16) unsigned char dsm[];
    auto *sh = reinterpret_cast<uint64_t *>(dsm);
    auto *own = reinterpret_cast<uint32_t *>(dsm + size_t(kLocalMax) * 8);
    auto *low = own + kLocalSlots;
    const uint32_t s = blockIdx.x;
    const uint32_t lo = starts[s], hi = s + 1 < nsub ? starts[s + 1] : n;
    const uint32_t cnt = hi - lo;
    if (cnt <= 1) return;  // a lone edge is a first occurrence
    if (cnt > kLocalMax) {
        if (threadIdx.x == 0) ovf[1 + atomicAdd(ovf, 1u)] = s;
        return;
    }
    uint32_t T = 64;
    while (T < 2 * cnt && T < kLocalSlots) T <<= 1;
    const uint32_t tmask = T - 1;
    const int batches = int((cnt + kLocalPer * kLocalThreads - 1) / (kLocalPer * kLocalThreads));
    uint32_t id[kLocalPer * kLocalBatches], sl[kLocalPer * kLocalBatches];
#pragma unroll
    for (int bt = 0; bt < kLocalBatches; ++bt) {
        if (bt >= batches) break;
        uint64_t hv[kLocalPer];
#pragma unroll
        for (int u = 0; u < kLocalPer; ++u) {
            const uint32_t r = threadIdx.x + (bt * kLocalPer + u) * kLocalThreads;
            hv[u] = r < cnt ? hash[lo + r] : 0;
            id[bt * kLocalPer + u] = r < cnt ? idx[lo + r] : 0;
        }
#pragma unroll
        for (int u = 0; u < kLocalPer; ++u) {
            const uint32_t r = threadIdx.x + (bt * kLocalPer + u) * kLocalThreads;
            if (r < cnt) sh[r] = hv[u];
        }
    }
    for (uint32_t i = threadIdx.x; i < T; i += kLocalThreads) {
        own[i] = 0;
        low[i] = ~0u;
    }
    __syncthreads();
    volatile uint32_t *vown = own;
    bool lost = false;
#pragma unroll
    for (int bt = 0; bt < kLocalBatches; ++bt) {
        if (bt >= batches) break;
#pragma unroll
        for (int u = 0; u < kLocalPer; ++u) {
            const int e = bt * kLocalPer + u;
            const uint32_t r = threadIdx.x + e * kLocalThreads;
            sl[e] = 0;
            if (r >= cnt) continue;
            const uint64_t hv = sh[r];
            uint32_t h = uint32_t(hv) & tmask;
            bool placed = false;
            for (uint32_t probe = 0; probe < T; ++probe) {
                uint32_t o = vown[h];
                if (o == 0) o = atomicCAS(&own[h], 0u, r + 1);
                if (o == 0 || sh[o - 1] == hv) {
                    placed = true;
                    break;
                }
                h = (h + 1) & tmask;
            }
            if (!placed) {  // never expected: T exceeds the bucket's size
                lost = true;
                h = 0;
            }
            atomicMin(&low[h], id[e]);
            sl[e] = h;
        }
    }
    if (lost) atomicOr(err, 8u);
    __syncthreads();
#pragma unroll
    for (int bt = 0; bt < kLocalBatches; ++bt) {
        if (bt >= batches) break;
#pragma unroll
        for (int u = 0; u < kLocalPer; ++u) {
            const int e = bt * kLocalPer + u;
            if (threadIdx.x + e * kLocalThreads >= cnt) continue;
            if (low[sl[e]] != id[e]) atomicAnd(bitmap + (id[e] >> 5), ~(1u << (id[e] & 31)));
        }
    }
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

// 4'. A bucket too large for shared memory, entries [begin, begin + count):
// insert into a device-memory table of 16-byte slots {hash, (bucket << 32) |
// smallest index}; a slot is told free by its second word only.  The table is shared by the overflow buckets, one after
// another: a slot holding another bucket's number counts as free.  A CAS only
// ever succeeds on a slot that does not carry this bucket's number, and
// atomicMin only ever targets slots that do, so no successful CAS overlaps a
// minimum on the same slot.  Every decision rests on a CAS's 16-byte
// snapshot, except that a plain read showing this bucket and this key is
// final (such a slot's key never changes within the launch).
__global__ void __launch_bounds__(256) k_dd_insert(const uint64_t *bkey, const uint32_t *bidx, uint64_t begin,
                                                   uint32_t count, unsigned long long *tab, uint64_t mask,
                                                   uint32_t bucket, unsigned *err) {
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < count; j += gridDim.x * blockDim.x) {
        const uint64_t key = bkey[begin + j];
        const uint64_t mine = (uint64_t(bucket) << 32) | bidx[begin + j];
        uint64_t h = key & mask;  // `key` is the edge's hash
        bool placed = false, lost = false;
        for (uint64_t probe = 0; probe <= mask && !placed && !lost; ++probe) {
            unsigned long long *slot = tab + 2 * h;
            uint64_t ek = slot[0], ew = slot[1];  // a guess; the CAS returns the truth
            bool next = false;
            for (int tries = 0; tries < 64 && !placed && !next; ++tries) {
                uint64_t gk, gw;
                if ((ew >> 32) == bucket) {
                    if (ek == key) {
                        if (mine < ew) atomicMin(slot + 1, (unsigned long long)mine);
                        placed = true;
                        break;
                    }
                    // another key of this bucket: confirm with a CAS that cannot
                    // succeed on a slot of this bucket
                    cas128(slot, kFree, kFree, key, mine, gk, gw);
                    if (gk == kFree && gw == kFree) placed = true;
                    else if (gk == ek && gw == ew) next = true;
                } else {
                    cas128(slot, ek, ew, key, mine, gk, gw);
                    if (gk == ek && gw == ew) placed = true;
                }
                ek = gk;
                ew = gw;
            }
            if (!placed && !next) lost = true;  // the slot kept changing (never expected)
            h = (h + 1) & mask;
        }
        if (!placed) atomicOr(err, 2u);
    }
}

// 4''. After k_dd_insert of the same bucket: every edge whose index is not its
// key's smallest clears its survivor bit.
__global__ void __launch_bounds__(256) k_dd_clear(const uint64_t *bkey, const uint32_t *bidx, uint64_t begin,
                                                  uint32_t count, const unsigned long long *tab, uint64_t mask,
                                                  uint32_t bucket, uint32_t *bitmap, unsigned *err) {
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < count; j += gridDim.x * blockDim.x) {
        const uint64_t key = bkey[begin + j];
        const uint32_t idx = bidx[begin + j];
        uint64_t h = key & mask;
        bool found = false;
        for (uint64_t probe = 0; probe <= mask; ++probe) {
            const uint64_t k0 = tab[2 * h], w = tab[2 * h + 1];
            if ((w >> 32) == bucket && k0 == key) {
                if (uint32_t(w) != idx) atomicAnd(bitmap + (idx >> 5), ~(1u << (idx & 31)));
                found = true;
                break;
            }
            h = (h + 1) & mask;
        }
        if (!found) atomicOr(err, 4u);
    }
}

// 5a. Survivors of chunk `c` (kChunk edges: one bitmap word per thread; bits
// at or past n are masked off).
constexpr int kCountThreads = int(kChunk / 32);
__global__ void __launch_bounds__(kCountThreads) k_dd_count(uint64_t n, const uint32_t *bitmap,
                                                            uint32_t *chunk_count) {
    __shared__ uint32_t warp_sum[kCountThreads / 32];
    const uint64_t first = blockIdx.x * kChunk + uint64_t(threadIdx.x) * 32;
    uint32_t c = 0;
    if (first < n) {
        uint32_t w = bitmap[first >> 5];
        if (n - first < 32) w &= (1u << (n - first)) - 1u;
        c = __popc(w);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kCountThreads / 32; ++w) t += warp_sum[w];
        chunk_count[blockIdx.x] = t;
    }
}

// Exclusive scan of `counts` in place (one block; up to ~2^22 entries); the
// sum goes to *total.
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

// 5c. Ordered compaction of chunk `c` to dst starting at offsets[c]: thread
// t keeps the survivors among edges c * kChunk + 4t .. + 3 (one nibble of the
// bitmap, bits at or past n masked off), ranked by a block prefix sum.
__global__ void __launch_bounds__(kBlock) k_dd_compact(const uint2 *edges, uint64_t n, const uint32_t *bitmap,
                                                       const uint32_t *offsets, uint2 *dst) {
    static_assert(kPerThread == 4, "a thread takes one nibble of a bitmap word");
    __shared__ uint32_t ws[32];
    const uint64_t base = blockIdx.x * kChunk + uint64_t(threadIdx.x) * kPerThread;
    uint32_t keep = 0;
    if (base < n) {
        keep = (bitmap[base >> 5] >> (base & 31)) & 0xFu;
        if (n - base < 4) keep &= (1u << (n - base)) - 1u;
    }
    const uint32_t c = __popc(keep);
    uint64_t out = uint64_t(offsets[blockIdx.x]) + block_exclusive<kBlock>(c, ws);
#pragma unroll
    for (int j = 0; j < kPerThread; ++j)
        if (keep & (1u << j)) dst[out++] = edges[base + j];
}

// Scratch kept between calls, per device; the mutex also serialises calls on
// one device (they share the buffer).
constexpr int kMaxDevices = 64;
struct Scratch {
    std::mutex mu;
    unsigned char *ptr = nullptr;
    size_t bytes = 0;
};
Scratch g_scratch[kMaxDevices];

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
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return fail(RMAT_ERR_UNSUPPORTED, "duplicate removal: no usable current device");
    }
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    auto cuda_fail = [](const char *what, cudaError_t e) {
        return fail(RMAT_ERR_CUDA, std::string("duplicate removal, ") + what + ": " + cudaGetErrorString(e));
    };

    // B bits of buckets (mean size at most kLocalTarget), B1 of them at level 1
    int B = 0;
    while (B < kMaxBits && (count >> B) > kLocalTarget) ++B;
    const int B1 = std::min(B, kL1MaxBits), B2 = B - B1;
    const uint32_t nb1 = 1u << B1, nsub = 1u << B;
    const uint32_t n = uint32_t(count);
    const uint64_t chunks = (count + kChunk - 1) / kChunk;
    const uint64_t words = (count + 31) / 32;
    // scratch: level-1 starts and cursors, sub-bucket starts, the overflow
    // list, two {key, index} buffers, the survivor bitmap, chunk counts, the
    // total and an error word
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t off_cursor = up(4 * size_t(nb1));
    const size_t off_sub = off_cursor + up(4 * size_t(nb1));
    const size_t off_ovf = off_sub + up(4 * size_t(nsub));
    const size_t off_akey = off_ovf + up(4 * (size_t(nsub) + 1));
    const size_t off_bkey = off_akey + up(8 * count + 256);  // 256 bytes of slack after each array: the
    const size_t off_aidx = off_bkey + up(8 * count + 256);  // split's widened copies read a few entries
    const size_t off_bidx = off_aidx + up(4 * count + 256);  // past a bucket
    const size_t off_bits = off_bidx + up(4 * count + 256);
    const size_t off_cnt = off_bits + up(4 * words);
    const size_t off_tot = off_cnt + up(4 * chunks);
    const size_t bytes = off_tot + 256;

    Scratch &sc = g_scratch[dev];
    std::lock_guard<std::mutex> lock(sc.mu);
    if (sc.bytes < bytes) {
        if (sc.ptr) cudaFree(sc.ptr);
        sc.ptr = nullptr;
        sc.bytes = 0;
        if (cudaMalloc(&sc.ptr, bytes) != cudaSuccess) {
            cudaGetLastError();
            sc.ptr = nullptr;
            return fail(RMAT_ERR_OUT_OF_MEMORY, "device scratch for duplicate removal");
        }
        sc.bytes = bytes;
    }
    unsigned char *scratch = sc.ptr;
    unsigned long long *tab = nullptr;  // overflow table, only when some bucket needs it
    auto done = [&](rmat_status st) {
        cudaStreamSynchronize(stream);
        if (tab) cudaFree(tab);
        return st;
    };
    auto *start1 = reinterpret_cast<uint32_t *>(scratch);
    auto *cursor = reinterpret_cast<uint32_t *>(scratch + off_cursor);
    auto *sub = reinterpret_cast<uint32_t *>(scratch + off_sub);
    auto *ovf = reinterpret_cast<uint32_t *>(scratch + off_ovf);
    auto *akey = reinterpret_cast<uint64_t *>(scratch + off_akey);
    auto *bkey = reinterpret_cast<uint64_t *>(scratch + off_bkey);
    auto *aidx = reinterpret_cast<uint32_t *>(scratch + off_aidx);
    auto *bidx = reinterpret_cast<uint32_t *>(scratch + off_bidx);
    auto *bitmap = reinterpret_cast<uint32_t *>(scratch + off_bits);
    auto *cnt = reinterpret_cast<uint32_t *>(scratch + off_cnt);
    auto *total = reinterpret_cast<unsigned long long *>(scratch + off_tot);
    auto *err = reinterpret_cast<unsigned *>(scratch + off_tot + 8);
    const uint2 *src = static_cast<const uint2 *>(edges);

    // 1-2. level-1 sizes, starts (scan on the device), scatter
    cudaError_t e = cudaMemsetAsync(start1, 0, 4 * size_t(nb1), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, 4, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ovf, 0, 4, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(bitmap, 0xFF, 4 * words, stream);  // every edge survives until cleared
    if (e == cudaSuccess) {
        k_dd_hist<<<props.sms * 2, kBlock, 0, stream>>>(src, count, k, B1, start1);
        k_dedup_scan<<<1, kBlock, 0, stream>>>(start1, nb1, total);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(cursor, start1, 4 * size_t(nb1), cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_dd_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kScatterSmem));
    if (e == cudaSuccess) {
        const uint64_t tiles = (count + kScatterTile - 1) / kScatterTile;
        const unsigned sgrid = unsigned(std::min<uint64_t>(tiles, uint64_t(props.sms)));
        k_dd_scatter<<<sgrid, kBlock, kScatterSmem, stream>>>(src, count, k, B1, cursor, akey, aidx, err);
        e = cudaGetLastError();
    }
    // 3. level-2 split (cursor[b] now ends level-1 bucket b)
    const uint64_t *lkey = akey;
    const uint32_t *lidx = aidx, *starts = start1;
    uint2 *dst = reinterpret_cast<uint2 *>(bkey);
    if (e == cudaSuccess && B2 > 0)
        e = cudaFuncSetAttribute(k_dd_split, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSplitSmem));
    if (e == cudaSuccess && B2 > 0) {
        k_dd_split<<<nb1, kSplitThreads, kSplitSmem, stream>>>(akey, aidx, start1, cursor, B, B2, bkey, bidx, sub, err);
        e = cudaGetLastError();
        lkey = bkey;
        lidx = bidx;
        starts = sub;
        dst = reinterpret_cast<uint2 *>(akey);
    }
    // 4. buckets in shared memory
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_dd_local, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kLocalSmem));
    if (e == cudaSuccess) {
        k_dd_local<<<nsub, kLocalThreads, kLocalSmem, stream>>>(lkey, lidx, starts, nsub, n, bitmap, ovf, err);
        e = cudaGetLastError();
    }
    uint32_t novf = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&novf, ovf, 4, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return done(cuda_fail("partition", e));
    // 4'. buckets too large for shared memory, one after another in one table
    if (novf) {
        std::vector<uint32_t> list(novf), hs(nsub);
        e = cudaMemcpyAsync(list.data(), ovf + 1, 4 * size_t(novf), cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), starts, 4 * size_t(nsub), cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return done(cuda_fail("overflow list", e));
        std::sort(list.begin(), list.end());
        auto size_of = [&](uint32_t s) { return (s + 1 < nsub ? hs[s + 1] : n) - hs[s]; };
        uint64_t largest = 1;
        for (uint32_t s : list) largest = std::max<uint64_t>(largest, size_of(s));
        uint64_t slots = 1;
        while (slots < 2 * largest) slots <<= 1;
        if (cudaMalloc(&tab, slots * 16) != cudaSuccess) {
            cudaGetLastError();
            tab = nullptr;
            return done(fail(RMAT_ERR_OUT_OF_MEMORY, "device hash table for duplicate removal"));
        }
        e = cudaMemsetAsync(tab, 0xFF, slots * 16, stream);  // no slot belongs to a bucket
        for (uint32_t s : list) {
            if (e != cudaSuccess) break;
            const uint32_t c = size_of(s);
            const unsigned g = unsigned(std::min<uint64_t>((c + 255) / 256, uint64_t(props.sms) * 8));
            k_dd_insert<<<g, 256, 0, stream>>>(lkey, lidx, hs[s], c, tab, slots - 1, s, err);
            k_dd_clear<<<g, 256, 0, stream>>>(lkey, lidx, hs[s], c, tab, slots - 1, s, bitmap, err);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) return done(cuda_fail("overflow buckets", e));
    }
    // 5. ordered compaction from the bitmap
    if (e == cudaSuccess) {
        k_dd_count<<<unsigned(chunks), kCountThreads, 0, stream>>>(count, bitmap, cnt);
        k_dedup_scan<<<1, kBlock, 0, stream>>>(cnt, chunks, total);
        k_dd_compact<<<unsigned(chunks), kBlock, 0, stream>>>(src, count, bitmap, cnt, dst);
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
    if (e != cudaSuccess) return done(cuda_fail("kernels", e));
    if (host_err) return done(fail(RMAT_ERR_CUDA, "duplicate removal: hash table full (internal error)"));
    *unique = host_total;
    return done(RMAT_OK);
}

extern "C" rmat_status rmat_dedup_release(void) {
    clear_error();
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return RMAT_OK;  // no device, nothing held
    }
    Scratch &sc = g_scratch[dev];
    std::lock_guard<std::mutex> lock(sc.mu);
    if (sc.ptr) {
        const cudaError_t e = cudaFree(sc.ptr);
        sc.ptr = nullptr;
        sc.bytes = 0;
        if (e != cudaSuccess)
            return fail(RMAT_ERR_CUDA, std::string("cudaFree(dedup scratch): ") + cudaGetErrorString(e));
    }
    return RMAT_OK;
}
