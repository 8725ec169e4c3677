// rmat_device.cuh -- device building blocks of the sampling kernels (sm_103a):
// Philox4x32-10, the alias draw, path concatenation, and the TMA / mbarrier
// primitives (inline PTX) used to stage tables and store edge tiles.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rmat {
namespace dev {

// --------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Counter (c0..c3) =
// (block q lo, q hi, edge lo, edge hi), key = (seed lo, seed hi).  Each round
// multiplies the even counter words by the round constants (one 32x32->64
// multiply each), xors the high halves with the odd words and the round key,
// and keeps the low halves; the key advances by the Weyl constants.
// --------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t m0 = uint64_t(0xD2511F53u) * c0;
        const uint64_t m1 = uint64_t(0xCD9E8D57u) * c2;
        const uint32_t n0 = uint32_t(m1 >> 32) ^ c1 ^ k0;
        const uint32_t n2 = uint32_t(m0 >> 32) ^ c3 ^ k1;
        c1 = uint32_t(m1);
        c3 = uint32_t(m0);
        c0 = n0;
        c2 = n2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(c0, c1, c2, c3);
}

// The same block function with the ten round keys precomputed (ks[2r],
// ks[2r+1] = key of round r).  When `ks` lives in a kernel parameter the xors
// read the round keys straight from the constant bank instead of adding the
// Weyl constants in registers.
__device__ __forceinline__ uint4 philox_ks(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                           const uint32_t (&ks)[20]) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t m0 = uint64_t(0xD2511F53u) * c0;
        const uint64_t m1 = uint64_t(0xCD9E8D57u) * c2;
        const uint32_t n0 = uint32_t(m1 >> 32) ^ c1 ^ ks[2 * round];
        const uint32_t n2 = uint32_t(m0 >> 32) ^ c3 ^ ks[2 * round + 1];
        c1 = uint32_t(m1);
        c3 = uint32_t(m0);
        c0 = n0;
        c2 = n2;
    }
    return make_uint4(c0, c1, c2, c3);
}

// x >> n with n >= 32 giving 0 (one funnel shift).
__device__ __forceinline__ uint32_t shr_clamp(uint32_t x, uint32_t n) {
    return __funnelshift_rc(x, 0u, n);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t lds32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

__device__ __forceinline__ uint32_t lds8(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u8 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

__device__ __forceinline__ uint32_t lds16(uint32_t addr) {
    unsigned short v;
    asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(addr));
    return v;
}

__device__ __forceinline__ uint2 lds64(uint32_t addr) {
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(addr));
    return v;
}

__device__ __forceinline__ ulonglong2 lds128u64(uint32_t addr) {
    ulonglong2 v;
    asm volatile("ld.shared.v2.u64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "r"(addr));
    return v;
}

__device__ __forceinline__ void sts8(uint32_t addr, uint32_t v) {
    asm volatile("st.shared.u8 [%0], %1;" ::"r"(addr), "h"((unsigned short)v) : "memory");
}

__device__ __forceinline__ void sts16(uint32_t addr, uint32_t v) {
    asm volatile("st.shared.u16 [%0], %1;" ::"r"(addr), "h"((unsigned short)v) : "memory");
}

__device__ __forceinline__ void sts64(uint32_t addr, uint32_t a, uint32_t b) {
    asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(addr), "r"(a), "r"(b) : "memory");
}

__device__ __forceinline__ void sts128u64(uint32_t addr, uint64_t a, uint64_t b) {
    asm volatile("st.shared.v2.u64 [%0], {%1, %2};" ::"r"(addr), "l"(a), "l"(b) : "memory");
}

__device__ __forceinline__ uint4 lds128(uint32_t addr) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(addr));
    return v;
}

// Philox4x32-10 with the round keys in shared memory at `sks` (20 words, the
// layout of philox_ks's `ks`): one broadcast 16-byte load per two rounds.
__device__ __forceinline__ uint4 philox_sks(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t sks) {
#pragma unroll
    for (int pair = 0; pair < 5; ++pair) {
        const uint4 kk = lds128(sks + 16u * uint32_t(pair));
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint64_t m0 = uint64_t(0xD2511F53u) * c0;
            const uint64_t m1 = uint64_t(0xCD9E8D57u) * c2;
            const uint32_t n0 = uint32_t(m1 >> 32) ^ c1 ^ (h ? kk.z : kk.x);
            const uint32_t n2 = uint32_t(m0 >> 32) ^ c3 ^ (h ? kk.w : kk.y);
            c1 = uint32_t(m1);
            c3 = uint32_t(m0);
            c0 = n0;
            c2 = n2;
        }
    }
    return make_uint4(c0, c1, c2, c3);
}

// Where one table (group) lives and how to split a word for it.  Every table
// has b >= 2 (at least four entries), so the column shift is 2..30.
template <bool SMEM>
struct Group {
    uint32_t sA, sBs, sBa;            // shared byte addresses (SMEM)
    const uint32_t *gA, *gBs, *gBa;   // global addresses (!SMEM)
    uint32_t shb;                     // 32 - b: column j = u >> (32 - b)
    uint32_t one;                     // 1, known only at run time (see Acc32::append)
};

// Blob header word `w` (group descriptors), from shared or global memory.
template <bool SMEM>
__device__ __forceinline__ uint32_t blob_word(uint32_t sbase, const uint32_t *gblob, uint32_t w) {
    if constexpr (SMEM) return lds32(sbase + 4u * w);
    else return __ldg(gblob + w);
}

template <bool SMEM>
__device__ __forceinline__ Group<SMEM> group(uint32_t sbase, const uint32_t *gblob, uint32_t g) {
    Group<SMEM> G;
    const uint32_t aoff = blob_word<SMEM>(sbase, gblob, g);
    const uint32_t bsoff = blob_word<SMEM>(sbase, gblob, 64u + g);
    const uint32_t baoff = blob_word<SMEM>(sbase, gblob, 128u + g);
    const uint32_t bits = blob_word<SMEM>(sbase, gblob, 192u + g);
    G.sA = sbase + 4u * aoff;
    G.sBs = sbase + 4u * bsoff;
    G.sBa = sbase + 4u * baoff;
    G.gA = gblob + aoff;
    G.gBs = gblob + bsoff;
    G.gBa = gblob + baoff;
    G.shb = 32u - bits;
    G.one = 1u;
    return G;
}

// Left-aligned accumulators.  Appending a path ORs its bits in below the
// `filled` levels already present; bits that fall below the accumulator are
// the surplus of the last path and are dropped.
struct Acc32 {
    uint32_t row, col, filled;
    __device__ __forceinline__ void clear() { row = col = filled = 0; }
    // The first path of an edge: nothing to shift.
    __device__ __forceinline__ void set(uint32_t r, uint32_t c, uint32_t L) {
        row = r;
        col = c;
        filled = L;
    }
    // Any number of levels may be appended: shifts of 32 or more give 0.  The
    // path's bits land below the `filled` levels already present, so OR-ing
    // them in is an add; written as a multiply-add by a run-time 1 it issues
    // on the FMA pipe, leaving the ALU pipe (shifts, compares, selects of the
    // draw) less loaded -- the ALU pipe is the one that bounds the kernel.
    __device__ __forceinline__ void append(uint32_t r, uint32_t c, uint32_t L, uint32_t one) {
        row = shr_clamp(r, filled) * one + row;
        col = shr_clamp(c, filled) * one + col;
        filled += L;
    }
    __device__ __forceinline__ uint64_t out_row(int k) const { return row >> (32 - k); }
    __device__ __forceinline__ uint64_t out_col(int k) const { return col >> (32 - k); }
};

struct Acc64 {
    uint64_t row, col;
    uint32_t filled;
    __device__ __forceinline__ void clear() { row = col = 0; filled = 0; }
    __device__ __forceinline__ void set(uint32_t r, uint32_t c, uint32_t L) {
        row = uint64_t(r) << 32;
        col = uint64_t(c) << 32;
        filled = L;
    }
    // Only called while filled < k <= 64.
    __device__ __forceinline__ void append(uint32_t r, uint32_t c, uint32_t L, uint32_t /*one*/) {
        row |= (uint64_t(r) << 32) >> filled;
        col |= (uint64_t(c) << 32) >> filled;
        filled += L;
    }
    __device__ __forceinline__ uint64_t out_row(int k) const { return row >> (64 - k); }
    __device__ __forceinline__ uint64_t out_col(int k) const { return col >> (64 - k); }
};

// One alias draw from word u: column j = top b bits of u; the draw keeps j
// iff u < A[j] = (j << (32-b)) + thr[j], i.e. iff the residual (low 32-b
// bits) < thr[j], and then takes path Bs[j], else path Ba[j] (the alias's).
// Compact path entry x: row bits in 31..19, length in 18..13, column bits in
// 12..0 (both left-aligned in their 13-bit fields); wide entry: {row, col,
// length, 0}.  `first` sets the accumulators (an edge's first path needs no
// shift), otherwise the path is appended.
template <int FMT, bool SMEM, bool FIRST = false, class Acc>
__device__ __forceinline__ void draw(const Group<SMEM> &G, uint32_t u, Acc &acc) {
    const uint32_t j = u >> G.shb;
    uint32_t r, c, L;
    if constexpr (SMEM) {
        const uint32_t off = 4u * j;
        const bool keep = u < lds32(G.sA + off);
        if constexpr (FMT == 0) {
            const uint32_t x = lds32((keep ? G.sBs : G.sBa) + off);
            r = x & 0xFFF80000u;
            c = x << 19;
            L = (x >> 13) & 63u;
        } else {
            const uint4 v = lds128((keep ? G.sBs : G.sBa) + 4u * off);
            r = v.x;
            c = v.y;
            L = v.z;
        }
    } else {
        const bool keep = u < __ldg(G.gA + j);
        if constexpr (FMT == 0) {
            const uint32_t x = __ldg((keep ? G.gBs : G.gBa) + j);
            r = x & 0xFFF80000u;
            c = x << 19;
            L = (x >> 13) & 63u;
        } else {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(keep ? G.gBs : G.gBa) + j);
            r = v.x;
            c = v.y;
            L = v.z;
        }
    }
    if constexpr (FIRST) acc.set(r, c, L);
    else acc.append(r, c, L, G.one);
}

// The same draw from a table of fixed-length paths (every entry has exactly
// L levels, 1 <= L <= 12: the per-level tables), returning the path's row and
// column bits right-aligned in r and c.
template <int FMT, bool SMEM>
__device__ __forceinline__ void draw_fixed(const Group<SMEM> &G, uint32_t u, uint32_t L, uint32_t &r,
                                           uint32_t &c) {
    const uint32_t j = u >> G.shb;
    const uint32_t s = 32u - L;
    if constexpr (SMEM) {
        const uint32_t off = 4u * j;
        const bool keep = u < lds32(G.sA + off);
        if constexpr (FMT == 0) {
            const uint32_t x = lds32((keep ? G.sBs : G.sBa) + off);
            r = x >> s;
            c = (x << 19) >> s;
        } else {
            const uint4 v = lds128((keep ? G.sBs : G.sBa) + 4u * off);
            r = v.x >> s;
            c = v.y >> s;
        }
    } else {
        const bool keep = u < __ldg(G.gA + j);
        if constexpr (FMT == 0) {
            const uint32_t x = __ldg((keep ? G.gBs : G.gBa) + j);
            r = x >> s;
            c = (x << 19) >> s;
        } else {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(keep ? G.gBs : G.gBa) + j);
            r = v.x >> s;
            c = v.y >> s;
        }
    }
}

// --------------------------------------------------------------------------
// PTX helpers: mbarrier, TMA bulk copies (global <-> shared), proxy fences.
// --------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase: gives up after `limit` polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t limit) {
    for (uint32_t it = 0; it < limit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it > 16) __nanosleep(128);
    }
    return false;
}

// global -> shared bulk copy completing on an mbarrier (16-byte aligned
// addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void *dst_smem, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst_smem)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// shared -> global bulk copy in the thread's bulk async-group.
__device__ __forceinline__ void bulk_s2g(void *dst, const void *src_smem, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                 "r"(smem_u32(src_smem)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_s2g_addr(void *dst, uint32_t src_smem, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src_smem), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Wait until every committed group has finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read_0() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

__device__ __forceinline__ void bulk_wait_all() {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Order this thread's generic-proxy shared-memory accesses before later
// async-proxy (TMA) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ uint32_t lane_mask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace dev
}  // namespace rmat
