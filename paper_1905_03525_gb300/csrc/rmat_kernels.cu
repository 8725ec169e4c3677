// rmat_kernels.cu -- the sampling kernels of librmat (sm_103a) and their
// launch logic.
//
// gen_tile: the per-edge sampling loop of arXiv 1905.03525, Sec. 2 (sampling-
// loop fragment) for one warp tile of consecutive edges, several per lane:
//   phase 1  one Philox4x32-10 block (4 words) per edge, up to 4 alias draws,
//            path bits OR-ed into left-aligned row/column registers;
//   phase 2  edges that still lack levels after 4 words are queued per warp
//            tile (one warp prefix sum over the lanes' bit masks) and finished
//            32 at a time with further Philox blocks, so that the rare long
//            edges do not make every lane of a warp pay for a second block.
//   Edges are written into a per-warp shared tile that leaves with one TMA
//   bulk store (asynchronous: it overlaps the sampling of the next tile).
// Per-level tables (Sec. 3, one table per level group) take exactly one draw
// per group, with no phase 2.
//
// k_alias: one job (a graph, or a range of one); table blob staged once per
//          CTA into shared memory by a TMA bulk copy on an mbarrier.
// k_batch: many jobs in one persistent launch; CTAs pop work units from an
//          atomic counter and restage the table when the job changes.
// k_alias_fast: the contract case of k_alias (compact u32 tables in shared
//          memory, four phase-1 draws, plain or relabelling epilogue), whole
//          tiles only.
// k_kron / k_kron_fast: n0 x n0 initiators (Sec. 3); the fast kernel takes
//          packed tables in k_alias_fast's shape.
// k_naive: the plain R-MAT process (Sec. 1), one quadrant draw per level.
#include <algorithm>
#include <cstdio>
#include <mutex>
#include <type_traits>
#include <vector>

#include "rmat_device.cuh"
#include "rmat_internal.h"
#include "rmat_kernels.h"

namespace rmat {

__device__ unsigned int g_device_error;

namespace {

constexpr uint32_t kWaitLimit = 1u << 22;

// Bytes of one warp's shared region: the output tile, the level count of
// every unfinished edge (1 byte per edge) and the queue of unfinished edges
// (2 bytes per edge).  One tile buffer is enough: the bulk store of a tile
// has read its few KB out of shared memory long before the warp has sampled
// the next tile, and the memory saved buys larger tiles (fuller phase-2
// batches).
__host__ __device__ constexpr uint32_t warp_region_bytes(bool u64, bool levels, int tile) {
    return uint32_t(tile) * (u64 ? 16u : 8u) + (levels ? 0u : 3u * uint32_t(tile));
}

template <bool U64>
struct AccT;
template <>
struct AccT<false> { using type = dev::Acc32; using word = uint32_t; };
template <>
struct AccT<true> { using type = dev::Acc64; using word = uint64_t; };

// Where a warp keeps its tile and queue (shared address).
struct WarpState {
    uint32_t region;
    int tile;
    bool issued;  // a bulk store is (or may be) in flight
    int lane;
};

// Group 0 of the job's table from the job's own fields (kernel parameters:
// uniform values, no shared-memory loads).
template <bool SMEM>
__device__ __forceinline__ dev::Group<SMEM> group0(const Job &J, uint32_t sblob) {
    dev::Group<SMEM> G;
    G.sA = sblob + 4u * J.a0;
    G.sBs = sblob + 4u * J.bs0;
    G.sBa = sblob + 4u * J.ba0;
    G.gA = J.blob + J.a0;
    G.gBs = J.blob + J.bs0;
    G.gBa = J.blob + J.ba0;
    G.shb = 32u - J.bits0;
    G.one = J.one;
    return G;
}

// Where a tile's Philox round keys come from: the job's schedule in a kernel
// parameter (uint32_t[20]: constant-bank operands of the xors; k_alias) or
// the schedule staged in shared memory (SharedKeys: five broadcast loads per
// block; k_batch, whose job is a register copy).
struct SharedKeys {
    uint32_t addr;
};
template <class K>
constexpr bool kConstKeys = !std::is_same<K, SharedKeys>::value;

// Philox block q of edge e under the job's key.
template <class K>
__device__ __forceinline__ uint4 edge_block(const K &ks, uint32_t q, uint64_t e) {
    if constexpr (std::is_same<K, SharedKeys>::value)
        return dev::philox_sks(q, 0u, uint32_t(e), uint32_t(e >> 32), ks.addr);
    else
        return dev::philox_ks(q, 0u, uint32_t(e), uint32_t(e >> 32), ks);
}

// Write edge `idx` of the tile at shared address `stage`.
template <bool U64>
__device__ __forceinline__ void put_pair(uint32_t stage, uint32_t idx, uint64_t r, uint64_t c) {
    if constexpr (U64)
        dev::sts128u64(stage + 16u * idx, r, c);
    else
        dev::sts64(stage + 8u * idx, uint32_t(r), uint32_t(c));
}

// Vertex relabelling pi (three rounds of x ^= x >> ceil(k/2); x = x*m + a,
// all mod 2^k), a bijection of [0, 2^k), applied to the accumulator word X
// that holds x in its top k bits (W-bit word, s = W - k; the bits below may
// hold levels drawn past k).  With X = x * 2^s: X*m + a*2^s = (x*m + a) * 2^s
// mod 2^W, and (X >> h) with its bits below 2^s cleared is (x >> h) * 2^s, so
// the rounds need no reduction mod 2^k.  Returns pi(x), right-aligned.
template <bool U64>
__device__ __forceinline__ uint64_t scramble_id(typename AccT<U64>::word X, const Job &J, const Scramble &S) {
    const uint32_t h = uint32_t(J.k + 1) >> 1;
    using Word = typename AccT<U64>::word;
    constexpr uint32_t W = U64 ? 64 : 32;
    const Word M = Word(S.mask);
    X &= M;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        X ^= (X >> h) & M;
        X = X * Word(S.m[i]) + Word(S.a[i]);
    }
    return uint64_t(X >> (W - uint32_t(J.k)));
}

// w * 2^L + bits for 1 <= L <= 12 (a per-level group); the 64-bit form
// shifts its two halves with one funnel shift, the amount being known to be
// below 32.
__device__ __forceinline__ uint32_t append_fixed(uint32_t w, uint32_t bits, uint32_t L) { return (w << L) | bits; }
__device__ __forceinline__ uint64_t append_fixed(uint64_t w, uint32_t bits, uint32_t L) {
    const uint32_t lo = uint32_t(w), hi = uint32_t(w >> 32);
    return (uint64_t(__funnelshift_l(lo, hi, L)) << 32) | ((lo << L) | bits);
}

// Store-epilogue variants (template argument EPI): bit 0 mirrors the edge to
// (min, max); bit 1 relabels every edge; bit 2 relabels when the job's flags
// ask for it (a batched launch mixes jobs with and without relabelling).
constexpr int kEpiUndir = 1, kEpiScr = 2, kEpiScrFlag = 4;

template <int EPI>
__device__ __forceinline__ bool relabel(const Job &J) {
    return (EPI & kEpiScr) || ((EPI & kEpiScrFlag) && (J.flags & kScrambleFlag));
}

template <bool U64, int EPI>
__device__ __forceinline__ void put_final(uint32_t stage, uint32_t idx, const typename AccT<U64>::type &acc,
                                          const Job &J, const Scramble &S) {
    uint64_t r, c;
    if (relabel<EPI>(J)) {
        r = scramble_id<U64>(acc.row, J, S);
        c = scramble_id<U64>(acc.col, J, S);
    } else {
        r = acc.out_row(J.k);
        c = acc.out_col(J.k);
    }
    if ((EPI & kEpiUndir) && r > c) {
        const uint64_t t = r;
        r = c;
        c = t;
    }
    put_pair<U64>(stage, idx, r, c);
}

// The same for IDs already right-aligned (row, col < 2^k): relabelling takes
// them left-aligned, the plain store as they are.
template <bool U64, int EPI>
__device__ __forceinline__ void put_final_right(uint32_t stage, uint32_t idx, typename AccT<U64>::word row,
                                                typename AccT<U64>::word col, const Job &J, const Scramble &S) {
    using Word = typename AccT<U64>::word;
    constexpr uint32_t W = U64 ? 64u : 32u;
    uint64_t r = row, c = col;
    if (relabel<EPI>(J)) {
        r = scramble_id<U64>(Word(row << (W - uint32_t(J.k))), J, S);
        c = scramble_id<U64>(Word(col << (W - uint32_t(J.k))), J, S);
    }
    if ((EPI & kEpiUndir) && r > c) {
        const uint64_t t = r;
        r = c;
        c = t;
    }
    put_pair<U64>(stage, idx, r, c);
}

// Phase 1 over a tile: one Philox block and up to `draws1` draws per edge,
// several edges per lane in flight (D = 4: draws1 is known to be 4, and the
// four draws are straight-line code; D = 0: draws1 read from the job).  Finished
// edges go to their output slot; unfinished ones leave their raw accumulators
// in the same slot, their level count in p_fill, and a bit in the lane's mask
// (bit i = edge i*32 + lane).
template <int FMT, bool U64, bool SMEM, int EPI, bool FULL, bool PRE, int D, class K>
__device__ __forceinline__ uint32_t phase1(const Job &J, const K &ks, const Scramble &S,
                                           const dev::Group<SMEM> &G0, uint64_t ebase, uint32_t n, uint32_t stage,
                                           uint32_t p_fill, int lane) {
    using Acc = typename AccT<U64>::type;
    const uint32_t uk = uint32_t(J.k);
    uint32_t pm = 0;
    const uint32_t iters = (n + 31) / 32;
    // U32 accumulators tolerate draws past k (clamped shifts); U64 ones are
    // extended only while short of k.
    auto step = [&](Acc &acc, uint32_t u) {
        if (!U64 || acc.filled < uk) dev::draw<FMT, SMEM>(G0, u, acc);
    };
    using Word = typename AccT<U64>::word;
    constexpr uint32_t W = U64 ? 64u : 32u;
    const uint32_t sh = W - uk;
    auto settle = [&](const Acc &acc, uint32_t it) {
        const uint32_t idx = it * 32 + lane;
        if (!FULL && idx >= n) return;
        const bool done = acc.filled >= uk;
        Word r = done ? Word(acc.row >> sh) : acc.row;
        Word c = done ? Word(acc.col >> sh) : acc.col;
        if (relabel<EPI>(J) && done) {
            r = scramble_id<U64>(acc.row, J, S);
            c = scramble_id<U64>(acc.col, J, S);
        }
        if ((EPI & kEpiUndir) && done && r > c) {
            const Word t = r;
            r = c;
            c = t;
        }
        put_pair<U64>(stage, idx, r, c);
        dev::sts8(p_fill + idx, acc.filled);
        pm |= uint32_t(!done) << it;
    };
    // E edges per lane in flight (edges it*32 + lane, (it+1)*32 + lane, ...):
    // their independent Philox chains and table loads overlap.  Four pays off
    // in the single-graph kernel for compact entries and u32 IDs (plain or
    // relabelled); elsewhere two (more would spill, or measured slower in the
    // batched kernel).
    constexpr int E = (kConstKeys<K> && FMT == 0 && !U64 && !(EPI & kEpiScrFlag)) ? 4 : 2;
    for (uint32_t it = 0; it < iters; it += E) {
        uint4 w[E];
        Acc a[E];
#pragma unroll
        for (int q = 0; q < E; ++q) w[q] = edge_block(ks, 0u, ebase + (it + q) * 32 + lane);
        if constexpr (PRE) {
            // batched jobs may start below the top level (a partition tile)
#pragma unroll
            for (int q = 0; q < E; ++q) {
                a[q].row = Word(J.pre_row);
                a[q].col = Word(J.pre_col);
                a[q].filled = J.pre_len;
                step(a[q], w[q].x);
            }
        } else {
#pragma unroll
            for (int q = 0; q < E; ++q) dev::draw<FMT, SMEM, true>(G0, w[q].x, a[q]);
        }
        if (D >= 2 || J.draws1 > 1) {
#pragma unroll
            for (int q = 0; q < E; ++q) step(a[q], w[q].y);
        }
        if (D >= 3 || J.draws1 > 2) {
#pragma unroll
            for (int q = 0; q < E; ++q) step(a[q], w[q].z);
        }
        if (D >= 4 || J.draws1 > 3) {
#pragma unroll
            for (int q = 0; q < E; ++q) step(a[q], w[q].w);
        }
#pragma unroll
        for (int q = 0; q < E; ++q)  // a tile of FULL edges holds whole groups; others may end inside one
            if (FULL || q == 0 || it + q < iters) settle(a[q], it + q);
    }
    return pm;
}

// sgroups: shared address of precomputed group descriptors (uint4 {A, Bs, Ba,
// 32 - b} per group) for per-level tables staged in shared memory, or 0 to read
// them from the blob header at every draw.
// ks: where the Philox round keys come from (see edge_block).  PRE: edges
// start with the job's prefix levels (batched jobs).  D: phase 1's draw count
// when known at compile time (4), else 0.  FULL: the tile is known to hold
// W.tile edges (otherwise chosen at run time from n).
template <int FMT, bool U64, bool SMEM, bool LEVELS, int EPI, bool PRE, int D, bool FULL, class K>
__device__ __forceinline__ void gen_tile(const Job &J, const K &ks, const Scramble &S, uint32_t sblob,
                                         const uint32_t *gblob, const dev::Group<SMEM> &G0, uint64_t first,
                                         uint32_t n, WarpState &W, uint32_t sgroups = 0) {
    using Acc = typename AccT<U64>::type;
    constexpr uint32_t EB = U64 ? 16 : 8;
    const int lane = W.lane;
    const uint32_t uk = uint32_t(J.k);
    const uint32_t stage = W.region;
    const uint32_t p_fill = W.region + uint32_t(W.tile) * EB;        // 1 byte per edge
    const uint32_t p_q = p_fill + uint32_t(W.tile);                  // 2 bytes per edge
    const uint64_t ebase = J.e0 + first;

    // The bulk store of the previous tile must have read the buffer.
    if (lane == 0 && W.issued) dev::bulk_wait_read_0();
    __syncwarp();

    if constexpr (LEVELS) {
        // Per-level tables hold fixed-length paths: every path of group g has
        // L_g = b_g / 2 levels (4^L_g columns) and the groups' lengths add up
        // to k.  So a draw appends its bits right-aligned, row = row * 2^L_g +
        // bits, with a shift the whole warp shares, and the words leave as
        // they are (left-aligned only for relabelling).
        // EL edges per lane (idx, idx + 32, ...) share each group's descriptor;
        // two in the single-graph kernel, one in the batched kernel, whose
        // register copy of the job leaves no room for a second.
        constexpr int EL = kConstKeys<K> ? 2 : 1;
        using Word = typename AccT<U64>::word;
        for (uint32_t base = 0; base < n; base += 32 * EL) {
            Word row[EL], col[EL];
#pragma unroll
            for (int q = 0; q < EL; ++q) row[q] = col[q] = 0;
            for (int q = 0; 4 * q < J.ngroups; ++q) {
                uint32_t ws[EL][4];
#pragma unroll
                for (int x = 0; x < EL; ++x) {
                    const uint4 w = edge_block(ks, uint32_t(q), ebase + base + 32 * x + lane);
                    ws[x][0] = w.x;
                    ws[x][1] = w.y;
                    ws[x][2] = w.z;
                    ws[x][3] = w.w;
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int g = 4 * q + i;
                    if (g < J.ngroups) {
                        dev::Group<SMEM> Gg;
                        if (SMEM && sgroups) {
                            const uint4 gd = dev::lds128(sgroups + 16u * uint32_t(g));
                            Gg.sA = gd.x;
                            Gg.sBs = gd.y;
                            Gg.sBa = gd.z;
                            Gg.shb = gd.w;
                        } else {
                            Gg = dev::group<SMEM>(sblob, gblob, uint32_t(g));
                        }
                        const uint32_t L = (32u - Gg.shb) >> 1;  // 4^L columns
#pragma unroll
                        for (int x = 0; x < EL; ++x) {
                            uint32_t r, c;
                            dev::draw_fixed<FMT, SMEM>(Gg, ws[x][i], L, r, c);
                            row[x] = append_fixed(row[x], r, L);
                            col[x] = append_fixed(col[x], c, L);
                        }
                    }
                }
            }
#pragma unroll
            for (int x = 0; x < EL; ++x) {
                const uint32_t idx = base + 32 * x + lane;
                if (idx < n) put_final_right<U64, EPI>(stage, idx, row[x], col[x], J, S);
            }
        }
    } else {
        // whole groups of E edges per lane (E <= 4): phase 1 without edge guards
        const uint32_t pm = (FULL || (n == uint32_t(W.tile) && n % 128u == 0))
                                ? phase1<FMT, U64, SMEM, EPI, true, PRE, D>(J, ks, S, G0, ebase, n, stage, p_fill, lane)
                                : phase1<FMT, U64, SMEM, EPI, false, PRE, D>(J, ks, S, G0, ebase, n, stage, p_fill, lane);
        // Phase 2: queue the unfinished edges of the whole tile (warp prefix
        // sum of the lanes' counts), then finish them 32 at a time.
        const uint32_t cnt = __popc(pm);
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        if (total) {
            uint32_t pos = incl - cnt;
            for (uint32_t m = pm; m; m &= m - 1) dev::sts16(p_q + 2u * pos++, (__ffs(m) - 1) * 32 + lane);
            __syncwarp();
            for (uint32_t pb = 0; pb < total; pb += 32) {
                const bool has = pb + lane < total;
                Acc acc;
                acc.clear();
                acc.filled = uk;
                uint32_t idx = 0;
                if (has) {
                    idx = dev::lds16(p_q + 2u * (pb + lane));
                    if constexpr (U64) {
                        const ulonglong2 v = dev::lds128u64(stage + 16u * idx);
                        acc.row = v.x;
                        acc.col = v.y;
                    } else {
                        const uint2 v = dev::lds64(stage + 8u * idx);
                        acc.row = v.x;
                        acc.col = v.y;
                    }
                    acc.filled = dev::lds8(p_fill + idx);
                }
                const uint64_t e = ebase + idx;
                // every draw adds >= 1 level, so k <= 64 levels need <= 16 more
                // blocks; the loop leaves as soon as no lane of the warp needs
                // another draw (a warp-uniform branch)
                for (uint32_t q = 1; q <= 17; ++q) {
                    if (!__any_sync(0xffffffffu, acc.filled < uk)) break;
                    const uint4 w = edge_block(ks, q, e);
                    if (U64) {
                        if (acc.filled < uk) dev::draw<FMT, SMEM>(G0, w.x, acc);
                    } else {
                        dev::draw<FMT, SMEM>(G0, w.x, acc);
                    }
                    if (!__any_sync(0xffffffffu, acc.filled < uk)) break;
                    if (!U64 || acc.filled < uk) dev::draw<FMT, SMEM>(G0, w.y, acc);
                    if (!__any_sync(0xffffffffu, acc.filled < uk)) break;
                    if (!U64 || acc.filled < uk) dev::draw<FMT, SMEM>(G0, w.z, acc);
                    if (!__any_sync(0xffffffffu, acc.filled < uk)) break;
                    if (!U64 || acc.filled < uk) dev::draw<FMT, SMEM>(G0, w.w, acc);
                }
                if (has) put_final<U64, EPI>(stage, idx, acc, J, S);
            }
        }
    }

    // Store the tile: one TMA bulk copy when aligned, else plain stores.
    unsigned char *gdst = reinterpret_cast<unsigned char *>(J.out) + first * EB;
    const uint32_t bytes = n * EB;
    if (((reinterpret_cast<uintptr_t>(gdst) | bytes) & 15u) == 0) {
        dev::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
            dev::bulk_s2g_addr(gdst, stage, bytes);
            dev::bulk_commit();
        }
        W.issued = true;
    } else {
        __syncwarp();
        uint2 *dst = reinterpret_cast<uint2 *>(gdst);
        for (uint32_t i = lane; i < bytes / 8; i += 32) dst[i] = dev::lds64(stage + 8u * i);
        __syncwarp();
    }
}

// Stage a blob into shared memory with one bulk copy (chunks of 32 KB) on
// `mbar`, phase `parity`; every thread returns whether it landed in time.
__device__ __forceinline__ bool stage_blob(unsigned char *dst, const uint32_t *src, uint32_t bytes, uint64_t *mbar,
                                           uint32_t parity) {
    if (threadIdx.x == 0) {
        dev::fence_proxy_async_smem();
        dev::mbar_arrive_expect_tx(mbar, bytes);
        const unsigned char *s = reinterpret_cast<const unsigned char *>(src);
        for (uint32_t off = 0; off < bytes; off += 32768u) {
            const uint32_t c = min(32768u, bytes - off);
            dev::bulk_g2s(dst + off, s + off, c, mbar);
        }
    }
    const bool ok = dev::mbar_wait_bounded(mbar, parity, kWaitLimit);
    return __syncthreads_and(ok) != 0;
}

template <int FMT, bool U64, bool SMEM, bool LEVELS, int EPI, int D>
__global__ void __launch_bounds__(1024, 1) k_alias(const __grid_constant__ Job J, const __grid_constant__ Scramble S,
                                                int tile, unsigned *err) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem);
    // per-level tables in shared memory get 1 KB of precomputed group descriptors
    constexpr uint32_t kGroupBytes = (LEVELS && SMEM) ? 16u * kMaxGroups : 0u;
    unsigned char *s_blob = smem + 16 + kGroupBytes;
    const uint32_t blob_bytes = SMEM ? J.blob_bytes : 0;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;

    if constexpr (SMEM) {
        if (threadIdx.x == 0) {
            dev::mbar_init(mbar, 1);
            dev::fence_mbar_init();
        }
        __syncthreads();
        if (!stage_blob(s_blob, J.blob, J.blob_bytes, mbar, 0)) {
            if (threadIdx.x == 0) {
                atomicOr(err, 1u);
                dev::mbar_wait_bounded(mbar, 0, kWaitLimit);  // let a late copy land before exit
            }
            return;
        }
    }
    const uint32_t sblob = dev::smem_u32(s_blob);
    const dev::Group<SMEM> G0 = group0<SMEM>(J, sblob);
    uint32_t sgroups = 0;
    if constexpr (LEVELS && SMEM) {
        sgroups = dev::smem_u32(smem + 16);
        for (int g = threadIdx.x; g < J.ngroups; g += blockDim.x) {
            const dev::Group<true> Gg = dev::group<true>(sblob, J.blob, uint32_t(g));
            uint4 *d = reinterpret_cast<uint4 *>(smem + 16) + g;
            *d = make_uint4(Gg.sA, Gg.sBs, Gg.sBa, Gg.shb);
        }
        __syncthreads();
    }

    WarpState W;
    W.region = dev::smem_u32(s_blob) + blob_bytes + uint32_t(warp) * warp_region_bytes(U64, LEVELS, tile);
    W.tile = tile;
    W.issued = false;
    W.lane = lane;
    // full tiles round-robin over the warps, then the ragged last tile (if
    // any) on the warp whose turn it is
    const uint64_t nfull = J.count / uint64_t(tile);
    const uint64_t stride = uint64_t(gridDim.x) * nwarps;
    uint64_t t = uint64_t(blockIdx.x) * nwarps + warp;
    if (tile % 128 == 0) {
        for (; t < nfull; t += stride)
            gen_tile<FMT, U64, SMEM, LEVELS, EPI, false, D, true>(J, J.ks, S, sblob, J.blob, G0, t * tile,
                                                                   uint32_t(tile), W, sgroups);
    } else {
        for (; t < nfull; t += stride)
            gen_tile<FMT, U64, SMEM, LEVELS, EPI, false, D, false>(J, J.ks, S, sblob, J.blob, G0, t * tile,
                                                                    uint32_t(tile), W, sgroups);
    }
    if (t == nfull && J.count % uint64_t(tile))
        gen_tile<FMT, U64, SMEM, LEVELS, EPI, false, D, false>(J, J.ks, S, sblob, J.blob, G0, t * tile,
                                                                uint32_t(J.count % uint64_t(tile)), W, sgroups);
    if (lane == 0 && W.issued) dev::bulk_wait_all();
}

// The contract case of the single-graph kernel and nothing else: compact
// entries, u32 IDs, the table in shared memory, one group, phase 1 known to
// take four draws, the plain epilogue, whole tiles only (the tile a multiple of
// 128 edges and the count a multiple of the tile) and a 16-byte-aligned
// output.  The arithmetic is gen_tile's; it is a kernel of its own because the
// compiler's split of the loop between the ALU and FMA pipes -- the two pipes
// that bound this kernel -- shifts with any other code in the kernel (the
// general kernel's ragged-tile and unaligned-store paths cost ~5 %).  The host
// sends everything else, and the ragged tail of a launch, to k_alias.
template <bool SCR>
__global__ void __launch_bounds__(1024, 1) k_alias_fast(const __grid_constant__ Job J,
                                                        const __grid_constant__ Scramble S, int tile) {
    extern __shared__ __align__(128) unsigned char smem[];
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(J.blob);
        uint4 *dst = reinterpret_cast<uint4 *>(smem);
        for (uint32_t i = threadIdx.x; i < J.blob_bytes / 16; i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const uint32_t sblob = dev::smem_u32(smem);
    const dev::Group<true> G = group0<true>(J, sblob);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint32_t stage = sblob + J.blob_bytes + uint32_t(warp) * warp_region_bytes(false, false, tile);
    const uint32_t p_fill = stage + 8u * uint32_t(tile), p_q = p_fill + uint32_t(tile);
    const uint32_t uk = uint32_t(J.k), sh = 32u - uk;
    const uint32_t iters = uint32_t(tile) / 32;
    const uint64_t ntiles = J.count / uint64_t(tile);
    bool issued = false;
    for (uint64_t t = uint64_t(blockIdx.x) * nwarps + warp; t < ntiles; t += uint64_t(gridDim.x) * nwarps) {
        const uint64_t first = t * uint64_t(tile);
        const uint64_t ebase = J.e0 + first;
        if (lane == 0 && issued) dev::bulk_wait_read_0();
        __syncwarp();
        // phase 1: one Philox block and four draws per edge, four edges per lane
        uint32_t pm = 0;
        for (uint32_t it = 0; it < iters; it += 4) {
            uint4 w[4];
            dev::Acc32 a[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint64_t e = ebase + (it + q) * 32 + lane;
                w[q] = dev::philox_ks(0u, 0u, uint32_t(e), uint32_t(e >> 32), J.ks);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) dev::draw<0, true, true>(G, w[q].x, a[q]);
#pragma unroll
            for (int q = 0; q < 4; ++q) dev::draw<0, true>(G, w[q].y, a[q]);
#pragma unroll
            for (int q = 0; q < 4; ++q) dev::draw<0, true>(G, w[q].z, a[q]);
#pragma unroll
            for (int q = 0; q < 4; ++q) dev::draw<0, true>(G, w[q].w, a[q]);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t idx = (it + q) * 32 + lane;
                const bool done = a[q].filled >= uk;
                uint32_t r = done ? a[q].row >> sh : a[q].row, c = done ? a[q].col >> sh : a[q].col;
                if (SCR && done) {  // relabelled IDs (Sec. 3 scrambling), fused into the store
                    r = uint32_t(scramble_id<false>(a[q].row, J, S));
                    c = uint32_t(scramble_id<false>(a[q].col, J, S));
                }
                dev::sts64(stage + 8u * idx, r, c);
                dev::sts8(p_fill + idx, a[q].filled);
                pm |= uint32_t(!done) << (it + q);
            }
        }
        // phase 2: the unfinished edges of the tile, 32 at a time
        const uint32_t cnt = __popc(pm);
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        if (total) {
            uint32_t pos = incl - cnt;
            for (uint32_t m = pm; m; m &= m - 1) dev::sts16(p_q + 2u * pos++, (__ffs(m) - 1) * 32 + lane);
            __syncwarp();
            for (uint32_t pb = 0; pb < total; pb += 32) {
                const bool has = pb + lane < total;
                dev::Acc32 acc;
                acc.row = acc.col = 0;
                acc.filled = uk;
                uint32_t idx = 0;
                if (has) {
                    idx = dev::lds16(p_q + 2u * (pb + lane));
                    const uint2 v = dev::lds64(stage + 8u * idx);
                    acc.row = v.x;
                    acc.col = v.y;
                    acc.filled = dev::lds8(p_fill + idx);
                }
                const uint64_t e = ebase + idx;
                for (uint32_t q = 1; q <= 17; ++q) {  // k <= 32 levels: at most 8 more blocks
                    if (!__any_sync(0xffffffffu, acc.filled < uk)) break;
                    const uint4 w = dev::philox_ks(q, 0u, uint32_t(e), uint32_t(e >> 32), J.ks);
                    dev::draw<0, true>(G, w.x, acc);
                    if (!__any_sync(0xffffffffu, acc.filled < uk)) break;
                    dev::draw<0, true>(G, w.y, acc);
                    if (!__any_sync(0xffffffffu, acc.filled < uk)) break;
                    dev::draw<0, true>(G, w.z, acc);
                    if (!__any_sync(0xffffffffu, acc.filled < uk)) break;
                    dev::draw<0, true>(G, w.w, acc);
                }
                if (has) {
                    if (SCR)
                        dev::sts64(stage + 8u * idx, uint32_t(scramble_id<false>(acc.row, J, S)),
                                   uint32_t(scramble_id<false>(acc.col, J, S)));
                    else
                        dev::sts64(stage + 8u * idx, acc.row >> sh, acc.col >> sh);
                }
            }
        }
        // the tile leaves by one bulk store
        dev::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
            dev::bulk_s2g_addr(reinterpret_cast<unsigned char *>(J.out) + first * 8u, stage, uint32_t(tile) * 8u);
            dev::bulk_commit();
        }
        issued = true;
    }
    if (lane == 0 && issued) dev::bulk_wait_all();
}

// The tiles of a partitioned graph (Sec. 3) in k_alias_fast's shape: one
// table and one seed for all of them, so the table is staged once and the
// round keys come from the kernel parameters.  A warp takes a contiguous share
// of the launch's warp tiles, finds the tile of its first by binary search and
// walks the tile list forward from there;
// the edges start from the tile's levels, then take four straight-line draws
// (u32 accumulators ignore draws past k) and the usual second phase.  A
// warp tile that ends its tile early runs guarded, and one whose output is
// not 16-byte aligned leaves by plain coalesced stores instead of a bulk
// store.
__global__ void __launch_bounds__(1024, 1) k_part_fast(const __grid_constant__ Job J, const PartTile *tiles,
                                                       uint32_t ntiles, uint64_t nwt, int tile) {
    extern __shared__ __align__(128) unsigned char smem[];
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(J.blob);
        uint4 *dst = reinterpret_cast<uint4 *>(smem);
        for (uint32_t i = threadIdx.x; i < J.blob_bytes / 16; i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const uint32_t sblob = dev::smem_u32(smem);
    const dev::Group<true> G = group0<true>(J, sblob);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint32_t stage = sblob + J.blob_bytes + uint32_t(warp) * warp_region_bytes(false, false, tile);
    const uint32_t p_fill = stage + 8u * uint32_t(tile), p_q = p_fill + uint32_t(tile);
    const uint32_t uk = uint32_t(J.k), sh = 32u - uk;
    // this warp's contiguous share of the warp tiles, and the tile holding the first
    const uint64_t gw = uint64_t(blockIdx.x) * nwarps + warp, all = uint64_t(gridDim.x) * nwarps;
    const uint64_t w_begin = gw * nwt / all, w_end = (gw + 1) * nwt / all;
    uint32_t j = 0;
    for (uint32_t lo = 0, hi = ntiles; hi - lo > 1;) {  // the last tile with wt0 <= w_begin
        const uint32_t mid = (lo + hi) / 2;
        if (tiles[mid].wt0 <= w_begin) lo = mid;
        else hi = mid;
        j = lo;
    }
    bool issued = false;
    for (uint64_t w = w_begin; w < w_end; ++w) {
        while (j + 1 < ntiles && tiles[j + 1].wt0 <= w) ++j;
        const PartTile &P = tiles[j];
        const uint64_t first = (w - P.wt0) * uint64_t(tile);
        const uint32_t n = uint32_t(min(uint64_t(tile), P.count - first));
        const uint64_t ebase = P.e0 + first;
        unsigned char *dst = reinterpret_cast<unsigned char *>(J.out) + (P.out + first) * 8u;
        const uint32_t pr = P.pre_row, pc = P.pre_col, pl = P.pre_len;
        if (lane == 0 && issued) dev::bulk_wait_read_0();
        __syncwarp();
        // phase 1: one Philox block and four draws per edge, four edges per lane
        uint32_t pm = 0;
        const uint32_t iters = (n + 31) / 32;
        for (uint32_t it = 0; it < iters; it += 4) {
            uint4 w4[4];
            dev::Acc32 a[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint64_t e = ebase + (it + q) * 32 + lane;
                w4[q] = dev::philox_ks(0u, 0u, uint32_t(e), uint32_t(e >> 32), J.ks);
                a[q].row = pr;
                a[q].col = pc;
                a[q].filled = pl;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) dev::draw<0, true>(G, w4[q].x, a[q]);
#pragma unroll
            for (int q = 0; q < 4; ++q) dev::draw<0, true>(G, w4[q].y, a[q]);
#pragma unroll
            for (int q = 0; q < 4; ++q) dev::draw<0, true>(G, w4[q].z, a[q]);
#pragma unroll
            for (int q = 0; q < 4; ++q) dev::draw<0, true>(G, w4[q].w, a[q]);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t idx = (it + q) * 32 + lane;
                if (idx >= n) continue;
                const bool done = a[q].filled >= uk;
                dev::sts64(stage + 8u * idx, done ? a[q].row >> sh : a[q].row, done ? a[q].col >> sh : a[q].col);
                dev::sts8(p_fill + idx, a[q].filled);
                pm |= uint32_t(!done) << (it + q);
            }
        }
        // phase 2: the unfinished edges of the warp tile, 32 at a time
        const uint32_t cnt = __popc(pm);
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        if (total) {
            uint32_t pos = incl - cnt;
            for (uint32_t m = pm; m; m &= m - 1) dev::sts16(p_q + 2u * pos++, (__ffs(m) - 1) * 32 + lane);
            __syncwarp();
            for (uint32_t pb = 0; pb < total; pb += 32) {
                const bool has = pb + lane < total;
                dev::Acc32 acc;
                acc.row = acc.col = 0;
                acc.filled = uk;
                uint32_t idx = 0;
                if (has) {
                    idx = dev::lds16(p_q + 2u * (pb + lane));
                    const uint2 v = dev::lds64(stage + 8u * idx);
                    acc.row = v.x;
                    acc.col = v.y;
                    acc.filled = dev::lds8(p_fill + idx);
                }
                const uint64_t e = ebase + idx;
                for (uint32_t q = 1; q <= 17; ++q) {  // k <= 32 levels: at most 8 more blocks
                    if (!__any_sync(0xffffffffu, acc.filled < uk)) break;
                    const uint4 w = dev::philox_ks(q, 0u, uint32_t(e), uint32_t(e >> 32), J.ks);
                    dev::draw<0, true>(G, w.x, acc);
                    if (!__any_sync(0xffffffffu, acc.filled < uk)) break;
                    dev::draw<0, true>(G, w.y, acc);
                    if (!__any_sync(0xffffffffu, acc.filled < uk)) break;
                    dev::draw<0, true>(G, w.z, acc);
                    if (!__any_sync(0xffffffffu, acc.filled < uk)) break;
                    dev::draw<0, true>(G, w.w, acc);
                }
                if (has) dev::sts64(stage + 8u * idx, acc.row >> sh, acc.col >> sh);
            }
        }
        if (n == uint32_t(tile) && (reinterpret_cast<uintptr_t>(dst) & 15u) == 0) {
            // a whole, aligned warp tile leaves by one bulk store
            dev::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                dev::bulk_s2g_addr(dst, stage, uint32_t(tile) * 8u);
                dev::bulk_commit();
            }
            issued = true;
        } else {
            __syncwarp();
            uint2 *o = reinterpret_cast<uint2 *>(dst);
            for (uint32_t i = lane; i < n; i += 32) o[i] = dev::lds64(stage + 8u * i);
            __syncwarp();
        }
    }
    if (lane == 0 && issued) dev::bulk_wait_all();
}

// One work unit of a batch: edges [u * unit_edges, ...) of job unit_job[u].
template <bool U64, int FMT, bool SMEM, bool LEVELS, int EPI, bool PRE>
__device__ __forceinline__ void batch_unit(const Job &J, const Scramble &S, SharedKeys ks, uint32_t sblob,
                                           uint64_t local_unit, uint64_t unit_edges, int nwarps, int warp,
                                           WarpState &W) {
    const dev::Group<SMEM> G0 = group0<SMEM>(J, sblob);
    const uint64_t f0 = local_unit * unit_edges;
    const uint64_t end = min(J.count, f0 + unit_edges);
    for (uint64_t first = f0 + uint64_t(warp) * W.tile; first < end; first += uint64_t(nwarps) * W.tile) {
        const uint64_t left = end - first;
        const uint32_t n = left < uint64_t(W.tile) ? uint32_t(left) : uint32_t(W.tile);
        gen_tile<FMT, U64, SMEM, LEVELS, EPI, PRE, 0, false>(J, ks, S, sblob, J.blob, G0, first, n, W);
    }
}

// GEN: some job starts below the top level (a partition tile) or relabels its
// IDs; the plain variant keeps the prefix and the relabelling test out of the
// registers, which lets compact u32 tables run four edges per lane.
template <bool U64, bool GEN>
__global__ void __launch_bounds__(1024) k_batch(BatchArgs B) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem);
    unsigned long long *s_unit = reinterpret_cast<unsigned long long *>(smem + 8);
    uint32_t *s_ks = reinterpret_cast<uint32_t *>(smem + 16);  // the job's Philox round keys
    unsigned char *s_blob = smem + kBatchHeaderBytes;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const uint32_t sblob = dev::smem_u32(s_blob);
    const SharedKeys ks{dev::smem_u32(s_ks)};

    if (threadIdx.x == 0) {
        dev::mbar_init(mbar, 1);
        dev::fence_mbar_init();
    }
    WarpState W;
    W.region = sblob + B.max_blob_bytes + uint32_t(warp) * warp_region_bytes(U64, false, B.tile);
    W.tile = B.tile;
    W.issued = false;
    W.lane = lane;

    const Job *staged = nullptr;
    uint32_t parity = 0;
    unsigned long long next = 0;
    if (threadIdx.x == 0) next = atomicAdd(B.counter, 1ull);
    for (;;) {
        if (threadIdx.x == 0) {
            *s_unit = next;
            if (next < B.units) next = atomicAdd(B.counter, 1ull);  // prefetch the following unit
        }
        __syncthreads();
        const unsigned long long unit = *s_unit;
        if (unit >= B.units) break;
        const uint32_t jid = B.unit_job[unit];
        const Job *jp = B.jobs + jid;
        const Job J = *jp;
        if (jp != staged) {
            // every warp is past the barrier above: nobody reads the old job's
            // round keys or table
            if (threadIdx.x < 20) s_ks[threadIdx.x] = jp->ks[threadIdx.x];
            if (J.smem) {
                if (!stage_blob(s_blob, J.blob, J.blob_bytes, mbar, parity)) {  // (its barrier publishes s_ks)
                    if (threadIdx.x == 0) {
                        atomicOr(B.err, 1u);
                        dev::mbar_wait_bounded(mbar, parity, kWaitLimit);
                    }
                    break;
                }
                parity ^= 1u;
            } else {
                __syncthreads();
            }
            staged = jp;
        }
        const uint64_t local = unit - J.unit_begin;
        const int sel = (J.fmt ? 8 : 0) | (J.smem ? 4 : 0) | (J.levels ? 2 : 0) | ((J.flags & RMAT_UNDIRECTED) ? 1 : 0);
        const Scramble &S = B.scr[jid];  // read (from global memory) only when relabelling
#define RMAT_UNIT(F, SM, L, U) \
    batch_unit<U64, F, SM, L, (U ? kEpiUndir : 0) | (GEN ? kEpiScrFlag : 0), GEN>(J, S, ks, sblob, local, \
                                                                                 B.unit_edges, nwarps, warp, W)
        switch (sel) {
            case 0: RMAT_UNIT(0, false, false, false); break;
            case 1: RMAT_UNIT(0, false, false, true); break;
            case 2: RMAT_UNIT(0, false, true, false); break;
            case 3: RMAT_UNIT(0, false, true, true); break;
            case 4: RMAT_UNIT(0, true, false, false); break;
            case 5: RMAT_UNIT(0, true, false, true); break;
            case 6: RMAT_UNIT(0, true, true, false); break;
            case 7: RMAT_UNIT(0, true, true, true); break;
            case 8: RMAT_UNIT(1, false, false, false); break;
            case 9: RMAT_UNIT(1, false, false, true); break;
            case 10: RMAT_UNIT(1, false, true, false); break;
            case 11: RMAT_UNIT(1, false, true, true); break;
            case 12: RMAT_UNIT(1, true, false, false); break;
            case 13: RMAT_UNIT(1, true, false, true); break;
            case 14: RMAT_UNIT(1, true, true, false); break;
            default: RMAT_UNIT(1, true, true, true); break;
        }
#undef RMAT_UNIT
        __syncthreads();  // s_unit and the staged table are reused next round
    }
    if (lane == 0 && W.issued) dev::bulk_wait_all();
}

// One warp tile of k_batch_fast: phase 1 takes one Philox block and D draws
// for four edges per lane (the job's draws1, known per job), the unfinished
// edges finish 32 at a time, and the tile leaves by a bulk store when its
// output is 16-byte aligned (by plain stores otherwise).  FULL: the tile holds
// W.tile edges, a multiple of 128.
template <int D, bool FULL>
__device__ __forceinline__ void fast_batch_tile(const Job &J, const dev::Group<true> &G, SharedKeys ks,
                                                uint64_t first, uint32_t n, WarpState &W) {
    const int lane = W.lane;
    const uint32_t uk = uint32_t(J.k), sh = 32u - uk;
    const uint32_t stage = W.region, p_fill = stage + 8u * uint32_t(W.tile), p_q = p_fill + uint32_t(W.tile);
    const uint64_t ebase = J.e0 + first;
    if (lane == 0 && W.issued) dev::bulk_wait_read_0();
    __syncwarp();
    uint32_t pm = 0;
    const uint32_t iters = (n + 31) / 32;
    for (uint32_t it = 0; it < iters; it += 4) {
        uint4 w[4];
        dev::Acc32 a[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) w[q] = edge_block(ks, 0u, ebase + (it + q) * 32 + lane);
#pragma unroll
        for (int q = 0; q < 4; ++q) dev::draw<0, true, true>(G, w[q].x, a[q]);
        if constexpr (D >= 2) {
#pragma unroll
            for (int q = 0; q < 4; ++q) dev::draw<0, true>(G, w[q].y, a[q]);
        }
        if constexpr (D >= 3) {
#pragma unroll
            for (int q = 0; q < 4; ++q) dev::draw<0, true>(G, w[q].z, a[q]);
        }
        if constexpr (D >= 4) {
#pragma unroll
            for (int q = 0; q < 4; ++q) dev::draw<0, true>(G, w[q].w, a[q]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t idx = (it + q) * 32 + lane;
            if (!FULL && idx >= n) continue;
            const bool done = a[q].filled >= uk;
            dev::sts64(stage + 8u * idx, done ? a[q].row >> sh : a[q].row, done ? a[q].col >> sh : a[q].col);
            dev::sts8(p_fill + idx, a[q].filled);
            pm |= uint32_t(!done) << (it + q);
        }
    }
    const uint32_t cnt = __popc(pm);
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    if (total) {
        uint32_t pos = incl - cnt;
        for (uint32_t m = pm; m; m &= m - 1) dev::sts16(p_q + 2u * pos++, (__ffs(m) - 1) * 32 + lane);
        __syncwarp();
        for (uint32_t pb = 0; pb < total; pb += 32) {
            const bool has = pb + lane < total;
            dev::Acc32 acc;
            acc.row = acc.col = 0;
            acc.filled = uk;
            uint32_t idx = 0;
            if (has) {
                idx = dev::lds16(p_q + 2u * (pb + lane));
                const uint2 v = dev::lds64(stage + 8u * idx);
                acc.row = v.x;
                acc.col = v.y;
                acc.filled = dev::lds8(p_fill + idx);
            }
            const uint64_t e = ebase + idx;
            // the remaining words of block 0, then blocks 1, 2, ...
            if constexpr (D < 4) {
                const uint4 w = edge_block(ks, 0u, e);
                if (D < 2 && __any_sync(0xffffffffu, acc.filled < uk)) dev::draw<0, true>(G, w.y, acc);
                if (D < 3 && __any_sync(0xffffffffu, acc.filled < uk)) dev::draw<0, true>(G, w.z, acc);
                if (__any_sync(0xffffffffu, acc.filled < uk)) dev::draw<0, true>(G, w.w, acc);
            }
            for (uint32_t q = 1; q <= 17; ++q) {  // k <= 32 levels: at most 8 more blocks
                if (!__any_sync(0xffffffffu, acc.filled < uk)) break;
                const uint4 w = edge_block(ks, q, e);
                dev::draw<0, true>(G, w.x, acc);
                if (!__any_sync(0xffffffffu, acc.filled < uk)) break;
                dev::draw<0, true>(G, w.y, acc);
                if (!__any_sync(0xffffffffu, acc.filled < uk)) break;
                dev::draw<0, true>(G, w.z, acc);
                if (!__any_sync(0xffffffffu, acc.filled < uk)) break;
                dev::draw<0, true>(G, w.w, acc);
            }
            if (has) dev::sts64(stage + 8u * idx, acc.row >> sh, acc.col >> sh);
        }
    }
    unsigned char *gdst = reinterpret_cast<unsigned char *>(J.out) + first * 8u;
    const uint32_t bytes = n * 8u;
    if (((reinterpret_cast<uintptr_t>(gdst) | bytes) & 15u) == 0) {
        dev::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
            dev::bulk_s2g_addr(gdst, stage, bytes);
            dev::bulk_commit();
        }
        W.issued = true;
    } else {
        __syncwarp();
        uint2 *dst = reinterpret_cast<uint2 *>(gdst);
        for (uint32_t i = lane; i < n; i += 32) dst[i] = dev::lds64(stage + 8u * i);
        __syncwarp();
    }
}

// Batches of whole graphs with u32 IDs, compact tables in shared memory and
// the plain epilogue (rmat_batch_prepare gathers such jobs into a launch of
// their own): k_batch's work units and table restaging, with k_alias_fast's
// sampling loop (four edges per lane; phase-1 draws specialised per job) and
// the round keys in shared memory.  Without k_batch's sixteen table variants
// the loop has the registers for four edges per lane.
__global__ void __launch_bounds__(1024, 1) k_batch_fast(BatchArgs B) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem);
    unsigned long long *s_unit = reinterpret_cast<unsigned long long *>(smem + 8);
    uint32_t *s_ks = reinterpret_cast<uint32_t *>(smem + 16);
    unsigned char *s_blob = smem + kBatchHeaderBytes;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const uint32_t sblob = dev::smem_u32(s_blob);
    const SharedKeys ks{dev::smem_u32(s_ks)};
    if (threadIdx.x == 0) {
        dev::mbar_init(mbar, 1);
        dev::fence_mbar_init();
    }
    WarpState W;
    W.region = sblob + B.max_blob_bytes + uint32_t(warp) * warp_region_bytes(false, false, B.tile);
    W.tile = B.tile;
    W.issued = false;
    W.lane = lane;
    const bool whole = B.tile % 128 == 0;
    const Job *staged = nullptr;
    uint32_t parity = 0;
    unsigned long long next = 0;
    if (threadIdx.x == 0) next = atomicAdd(B.counter, 1ull);
    for (;;) {
        if (threadIdx.x == 0) {
            *s_unit = next;
            if (next < B.units) next = atomicAdd(B.counter, 1ull);
        }
        __syncthreads();
        const unsigned long long unit = *s_unit;
        if (unit >= B.units) break;
        const Job *jp = B.jobs + B.unit_job[unit];
        if (jp != staged) {
            if (threadIdx.x < 20) s_ks[threadIdx.x] = jp->ks[threadIdx.x];
            if (!stage_blob(s_blob, jp->blob, jp->blob_bytes, mbar, parity)) {  // (its barrier publishes s_ks)
                if (threadIdx.x == 0) {
                    atomicOr(B.err, 1u);
                    dev::mbar_wait_bounded(mbar, parity, kWaitLimit);
                }
                break;
            }
            parity ^= 1u;
            staged = jp;
        }
        const Job &J = *jp;
        const dev::Group<true> G = group0<true>(J, sblob);
        const uint64_t f0 = (unit - J.unit_begin) * B.unit_edges;
        const uint64_t end = min(J.count, f0 + B.unit_edges);
        const int d = J.draws1;
        for (uint64_t first = f0 + uint64_t(warp) * W.tile; first < end; first += uint64_t(nwarps) * W.tile) {
            const uint32_t n = uint32_t(min(uint64_t(W.tile), end - first));
            const bool full = whole && n == uint32_t(W.tile);
#define RMAT_FAST_TILE(DD)                                          \
    if (full) fast_batch_tile<DD, true>(J, G, ks, first, n, W);     \
    else fast_batch_tile<DD, false>(J, G, ks, first, n, W);
            if (d >= 4) { RMAT_FAST_TILE(4) }
            else if (d == 3) { RMAT_FAST_TILE(3) }
            else if (d == 2) { RMAT_FAST_TILE(2) }
            else { RMAT_FAST_TILE(1) }
#undef RMAT_FAST_TILE
        }
        __syncthreads();  // s_unit and the staged table are reused next round
    }
    if (lane == 0 && W.issued) dev::bulk_wait_all();
}

// Stochastic Kronecker graphs with an n0 x n0 initiator, n0 > 2 (Sec. 3).
// One edge per thread over a persistent grid: the table (AA = {A, alias},
// P = {row digits, column digits, L, n0^L - 1}) is staged in shared memory,
// each draw picks column j = umulhi(u, 2^b), keeps it iff u < A[j] (else its
// alias), and appends the path's digits in base n0; the draw that would pass
// k levels keeps only the path's top k - filled digits (floor division by
// n0^d as a multiply-high).  Every draw adds >= 1 level (zero-weight columns
// always defer to their alias), so k <= 40 levels need <= 10 blocks.
template <bool U64>
__global__ void __launch_bounds__(1024, 1) k_kron(const __grid_constant__ KronJob J) {
    extern __shared__ __align__(128) unsigned char smem[];
    const uint4 *src = reinterpret_cast<const uint4 *>(J.blob);
    uint4 *dst = reinterpret_cast<uint4 *>(smem);
    for (uint32_t i = threadIdx.x; i < J.blob_bytes / 16; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    using Word = typename AccT<U64>::word;
    const uint32_t sAA = dev::smem_u32(smem) + J.aa_off;
    const uint32_t sP = dev::smem_u32(smem) + J.p_off;
    const uint32_t uk = uint32_t(J.k);
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < J.count; i += stride) {
        const uint64_t e = J.e0 + i;
        Word row = 0, col = 0;
        uint32_t filled = 0;
        auto draw = [&](uint32_t u) {
            const uint32_t j = __umulhi(u, J.mulb);
            const uint2 aa = dev::lds64(sAA + 8u * j);
            const uint4 p = dev::lds128(sP + 16u * (u < aa.x ? j : aa.y));
            if (filled + p.z <= uk) {
                row = row * Word(p.w) + row + Word(p.x);  // row * n0^L + digits
                col = col * Word(p.w) + col + Word(p.y);
                filled += p.z;
            } else {
                const uint32_t take = uk - filled, d = p.z - take;
                row = row * Word(J.pw[take]) + Word(__umul64hi(uint64_t(p.x), J.mg[d]));
                col = col * Word(J.pw[take]) + Word(__umul64hi(uint64_t(p.y), J.mg[d]));
                filled = uk;
            }
        };
        for (uint32_t q = 0; q < 16 && filled < uk; ++q) {
            const uint4 w = dev::philox_ks(q, 0u, uint32_t(e), uint32_t(e >> 32), J.ks);
            draw(w.x);
            if (filled >= uk) break;
            draw(w.y);
            if (filled >= uk) break;
            draw(w.z);
            if (filled >= uk) break;
            draw(w.w);
        }
        if constexpr (U64) {
            // outputs are only 8-byte aligned: two 8-byte stores
            uint64_t *o = reinterpret_cast<uint64_t *>(J.out) + 2 * i;
            o[0] = row;
            o[1] = col;
        } else {
            reinterpret_cast<uint2 *>(J.out)[i] = make_uint2(row, col);
        }
    }
}

// Contract case of the Kronecker kernel: u32 IDs and paths that pack into one
// word (P32 = r | c << S | L << 2S), with A32 = (thr << b) | alias as in the
// compact R-MAT image and n0^L from a 16-word power table, all in shared
// memory (8 bytes per column).  Phase 1 takes one Philox block and four draws
// for every edge of a warp's tile, four edges per lane; the edges still short
// of k levels continue, 32 at a time, on the next blocks; the tile leaves by
// one bulk store.  The draws, the words they use and the arithmetic are those
// of k_kron: keep column j iff u mod 2^(32-b) < thr[j] (the same test as
// u < A[j] there), append x * n0^L + digits, and on the draw that passes k
// levels keep the path's top k - filled digits (without a branch: every draw
// takes min(L, k - filled) digits, dividing by n0^d with a 32-bit magic
// multiplier, exact since digits x n0^d < 2^28).
__global__ void __launch_bounds__(1024, 1) k_kron_fast(const __grid_constant__ KronJob J, int tile) {
    extern __shared__ __align__(128) unsigned char smem[];
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(reinterpret_cast<const unsigned char *>(J.blob) + J.c_off);
        uint4 *dst = reinterpret_cast<uint4 *>(smem);
        for (uint32_t i = threadIdx.x; i < J.c_bytes / 16; i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const uint32_t b = J.bits, N = 1u << b, shb = 32u - b, lowmask = (1u << shb) - 1u;  // 1 <= b <= 31
    const uint32_t sA = dev::smem_u32(smem), sP = sA + 4u * ((N + 3u) & ~3u), sPW = sP + 4u * ((N + 3u) & ~3u);
    const uint32_t sMD = sPW + 64u;
    const uint32_t S = J.c_shift, rmask = (1u << S) - 1u, S2 = 2u * S;
    const uint32_t uk = uint32_t(J.k);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint32_t stage = sA + J.c_bytes + uint32_t(warp) * warp_region_bytes(false, false, tile);
    const uint32_t p_fill = stage + 8u * uint32_t(tile), p_q = p_fill + uint32_t(tile);
    const uint32_t iters = uint32_t(tile) / 32;
    const uint64_t ntiles = J.count / uint64_t(tile);
    auto draw = [&](uint32_t u, uint32_t &row, uint32_t &col, uint32_t &filled) {
        const uint32_t j = u >> shb;
        const uint32_t a = dev::lds32(sA + 4u * j);
        const uint32_t sel = (u & lowmask) < (a >> b) ? j : (a & (N - 1u));
        const uint32_t p = dev::lds32(sP + 4u * sel);
        const uint32_t r = p & rmask, c = (p >> S) & rmask, L = p >> S2;
        // the top `take` of the path's L digits: x div n0^(L - take), the
        // whole path while it fits, nothing once the edge is full
        const uint32_t take = min(L, uk - filled), d = L - take;
        const uint32_t m = dev::lds32(sPW + 4u * take), md = dev::lds32(sMD + 4u * d);
        row = row * m + (d ? __umulhi(r, md) : r);
        col = col * m + (d ? __umulhi(c, md) : c);
        filled += take;
    };
    bool issued = false;
    for (uint64_t t = uint64_t(blockIdx.x) * nwarps + warp; t < ntiles; t += uint64_t(gridDim.x) * nwarps) {
        const uint64_t first = t * uint64_t(tile);
        const uint64_t ebase = J.e0 + first;
        if (lane == 0 && issued) dev::bulk_wait_read_0();
        __syncwarp();
        // phase 1: one Philox block and four draws per edge, four edges per lane
        uint32_t pm = 0;
        for (uint32_t it = 0; it < iters; it += 4) {
            uint4 w[4];
            uint32_t row[4], col[4], filled[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint64_t e = ebase + (it + q) * 32 + lane;
                w[q] = dev::philox_ks(0u, 0u, uint32_t(e), uint32_t(e >> 32), J.ks);
                row[q] = col[q] = filled[q] = 0;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) draw(w[q].x, row[q], col[q], filled[q]);
#pragma unroll
            for (int q = 0; q < 4; ++q) draw(w[q].y, row[q], col[q], filled[q]);
#pragma unroll
            for (int q = 0; q < 4; ++q) draw(w[q].z, row[q], col[q], filled[q]);
#pragma unroll
            for (int q = 0; q < 4; ++q) draw(w[q].w, row[q], col[q], filled[q]);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t idx = (it + q) * 32 + lane;
                dev::sts64(stage + 8u * idx, row[q], col[q]);
                dev::sts8(p_fill + idx, filled[q]);
                pm |= uint32_t(filled[q] < uk) << (it + q);
            }
        }
        // phase 2: the unfinished edges of the tile, 32 at a time
        const uint32_t cnt = __popc(pm);
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        if (total) {
            uint32_t pos = incl - cnt;
            for (uint32_t m = pm; m; m &= m - 1) dev::sts16(p_q + 2u * pos++, (__ffs(m) - 1) * 32 + lane);
            __syncwarp();
            for (uint32_t pb = 0; pb < total; pb += 32) {
                const bool has = pb + lane < total;
                uint32_t row = 0, col = 0, filled = uk, idx = 0;
                if (has) {
                    idx = dev::lds16(p_q + 2u * (pb + lane));
                    const uint2 v = dev::lds64(stage + 8u * idx);
                    row = v.x;
                    col = v.y;
                    filled = dev::lds8(p_fill + idx);
                }
                const uint64_t e = ebase + idx;
                for (uint32_t q = 1; q <= 17; ++q) {  // k <= 32 levels, >= 1 level a draw: at most 8 more blocks
                    if (!__any_sync(0xffffffffu, filled < uk)) break;
                    const uint4 w = dev::philox_ks(q, 0u, uint32_t(e), uint32_t(e >> 32), J.ks);
                    draw(w.x, row, col, filled);
                    if (!__any_sync(0xffffffffu, filled < uk)) break;
                    draw(w.y, row, col, filled);
                    if (!__any_sync(0xffffffffu, filled < uk)) break;
                    draw(w.z, row, col, filled);
                    if (!__any_sync(0xffffffffu, filled < uk)) break;
                    draw(w.w, row, col, filled);
                }
                if (has) dev::sts64(stage + 8u * idx, row, col);
            }
        }
        // the tile leaves by one bulk store
        dev::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
            dev::bulk_s2g_addr(reinterpret_cast<unsigned char *>(J.out) + first * 8u, stage, uint32_t(tile) * 8u);
            dev::bulk_commit();
        }
        issued = true;
    }
    if (lane == 0 && issued) dev::bulk_wait_all();
}

// Order-independent checksum of the edges of every job of a step: the sum
// mod 2^64 of mix(e, row, col) over the job's edges, where
//   x = e * 0x9E3779B97F4A7C15 + row * 0xC2B2AE3D27D4EB4F + col * 0x165667B19E3779F9
//   mix = x ^ (x >> 30); * 0xBF58476D1CE4E5B9; ^ (>> 27); * 0x94D049BB133111EB; ^ (>> 31)
// (splitmix64's finaliser).  Chunk sums add up to the graph's sum however the
// graph is split.  sums[j] accumulates job j's sum.
template <bool U64>
__global__ void __launch_bounds__(256) k_checksum(BatchArgs B, unsigned long long *sums) {
    __shared__ unsigned long long part[8];
    for (uint64_t unit = blockIdx.x; unit < B.units; unit += gridDim.x) {
        const uint32_t jid = B.unit_job[unit];
        const Job &J = B.jobs[jid];
        const uint64_t f0 = (unit - J.unit_begin) * B.unit_edges;
        const uint64_t end = min(J.count, f0 + B.unit_edges);
        unsigned long long acc = 0;
        auto edge = [&](uint64_t i) {
            uint64_t r, c;
            if (U64) {
                const ulonglong2 v = reinterpret_cast<const ulonglong2 *>(J.out)[i];
                r = v.x;
                c = v.y;
            } else {
                const uint2 v = reinterpret_cast<const uint2 *>(J.out)[i];
                r = v.x;
                c = v.y;
            }
            return make_ulonglong2(r, c);
        };
        auto mix = [&](uint64_t i, ulonglong2 v) {
            uint64_t x = (J.e0 + i) * 0x9E3779B97F4A7C15ull + v.x * 0xC2B2AE3D27D4EB4Full + v.y * 0x165667B19E3779F9ull;
            x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
            x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
            return x ^ (x >> 31);
        };
        // four independent loads in flight per thread before the arithmetic
        const uint64_t bd = blockDim.x;
        uint64_t i = f0 + threadIdx.x;
        for (; i + 3 * bd < end; i += 4 * bd) {
            const ulonglong2 v0 = edge(i), v1 = edge(i + bd), v2 = edge(i + 2 * bd), v3 = edge(i + 3 * bd);
            acc += mix(i, v0) + mix(i + bd, v1) + mix(i + 2 * bd, v2) + mix(i + 3 * bd, v3);
        }
        for (; i < end; i += bd) acc += mix(i, edge(i));
        for (int o = 16; o; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long tot = 0;
            for (int w = 0; w < int(blockDim.x >> 5); ++w) tot += part[w];
            atomicAdd(sums + jid, tot);
        }
        __syncthreads();
    }
}

struct NaiveArgs {
    int k;
    unsigned flags;
    uint32_t key0, key1;
    uint64_t e0, count;
    void *out;
    uint32_t thr[64 * 3];
};

template <bool U64>
__global__ void __launch_bounds__(256) k_naive(NaiveArgs a) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < a.count; i += stride) {
        const uint64_t e = a.e0 + i;
        uint64_t row = 0, col = 0;
        for (int q = 0; 4 * q < a.k; ++q) {
            const uint4 w = dev::philox(uint32_t(q), 0u, uint32_t(e), uint32_t(e >> 32), a.key0, a.key1);
            const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int lvl = 4 * q + j;
                if (lvl < a.k) {
                    const uint32_t u = ws[j];
                    const uint32_t s = uint32_t(u >= a.thr[3 * lvl]) + uint32_t(u >= a.thr[3 * lvl + 1]) +
                                       uint32_t(u >= a.thr[3 * lvl + 2]);
                    row = (row << 1) | (s >> 1);
                    col = (col << 1) | (s & 1u);
                }
            }
        }
        if ((a.flags & RMAT_UNDIRECTED) && row > col) {
            const uint64_t t = row;
            row = col;
            col = t;
        }
        if (U64)
            reinterpret_cast<ulonglong2 *>(a.out)[i] = make_ulonglong2(row, col);
        else
            reinterpret_cast<uint2 *>(a.out)[i] = make_uint2(uint32_t(row), uint32_t(col));
    }
}

template <int FMT, bool U64, bool SMEM, bool LEVELS, int EPI, int D>
void *alias_kernel_ptr() {
    // per-level tables take one draw per group: the draw count never applies
    return reinterpret_cast<void *>(&k_alias<FMT, U64, SMEM, LEVELS, EPI, LEVELS ? 0 : D>);
}

using KernelFn = void *(*)();
#define RMAT_K2(D, F, U, S, L) \
    {alias_kernel_ptr<F, U, S, L, 0, D>, alias_kernel_ptr<F, U, S, L, 1, D>, alias_kernel_ptr<F, U, S, L, 2, D>, \
     alias_kernel_ptr<F, U, S, L, 3, D>}
#define RMAT_K4(D, F, U, S) {RMAT_K2(D, F, U, S, false), RMAT_K2(D, F, U, S, true)}
#define RMAT_K8(D, F, U) {RMAT_K4(D, F, U, false), RMAT_K4(D, F, U, true)}
#define RMAT_K16(D) {{RMAT_K8(D, 0, false), RMAT_K8(D, 0, true)}, {RMAT_K8(D, 1, false), RMAT_K8(D, 1, true)}}
// [phase-1 draws known to be 4][format][u64][shared table][per-level][epilogue: undirected | relabel << 1]
KernelFn alias_kernel_table[2][2][2][2][2][4] = {RMAT_K16(0), RMAT_K16(4)};
#undef RMAT_K16
#undef RMAT_K8
#undef RMAT_K4
#undef RMAT_K2

std::mutex g_props_mu;
std::vector<DeviceProps> g_props;

unsigned *device_error_ptr() {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_device_error) != cudaSuccess) return nullptr;
    return static_cast<unsigned *>(p);
}

// The dynamic shared-memory limit is an attribute of the kernel function, not
// of a launch: raise it once per kernel to the device maximum, so that any
// later launch of that kernel may use up to the maximum.  (Occupancy still
// follows each launch's actual size.)
std::mutex g_attr_mu;
std::vector<std::pair<void *, int>> g_attr_done;  // (kernel, device)

cudaError_t set_smem_attr(void *kernel, size_t /*bytes*/) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_attr_mu);
    for (const auto &kd : g_attr_done)
        if (kd.first == kernel && kd.second == dev) return cudaSuccess;
    int max_smem = 0;
    e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e == cudaSuccess) g_attr_done.emplace_back(kernel, dev);
    return e;
}

}  // namespace

rmat_status device_props(DeviceProps &out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(RMAT_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    std::lock_guard<std::mutex> lk(g_props_mu);
    if (int(g_props.size()) <= dev) g_props.resize(dev + 1);
    DeviceProps &p = g_props[dev];
    if (!p.valid) {
        cudaDeviceProp prop;
        e = cudaGetDeviceProperties(&prop, dev);
        if (e != cudaSuccess)
            return fail(RMAT_ERR_CUDA, std::string("cudaGetDeviceProperties: ") + cudaGetErrorString(e));
        if (prop.major < 10)
            return fail(RMAT_ERR_UNSUPPORTED, "librmat is built for sm_103a (GB300); this device is sm_" +
                                                  std::to_string(prop.major * 10 + prop.minor));
        p.sms = prop.multiProcessorCount;
        p.max_smem = int(prop.sharedMemPerBlockOptin);
        p.cc = prop.major * 10 + prop.minor;
        p.err = device_error_ptr();
        if (!p.err) return fail(RMAT_ERR_UNSUPPORTED, "kernel image not loadable on this device (built for sm_103a)");
        p.valid = true;
    }
    out = p;
    return RMAT_OK;
}

rmat_launch_config_t default_launch_config(const rmat_table *t) {
    rmat_launch_config_t c;
    c.threads = 1024;
    c.ctas_per_sm = 1;
    c.tile_edges = t->k > 32 ? 256 : 512;
    return c;
}

size_t warp_bytes(bool u64, bool levels, int tile) { return warp_region_bytes(u64, levels, tile); }

rmat_status plan_kron_launch(const rmat_table *t, const DeviceProps &props, AliasPlan &plan) {
    const bool u64 = wide_ids(t);
    plan.fmt = kKron;
    plan.u64 = u64;
    plan.levels = false;
    plan.smem_table = true;
    plan.threads = 1024;
    plan.tile = 0;
    const uint32_t packed_words = t->gdesc[0].ba_off_words;  // 0: no packed arrays
    plan.smem_bytes = size_t(packed_words ? packed_words : t->image.size()) * 4;
    if (plan.smem_bytes > size_t(props.max_smem))
        return fail(RMAT_ERR_UNSUPPORTED, "Kronecker table larger than shared memory (use a smaller bound)");
    plan.kernel = u64 ? reinterpret_cast<void *>(&k_kron<true>) : reinterpret_cast<void *>(&k_kron<false>);
    cudaError_t e = set_smem_attr(plan.kernel, plan.smem_bytes);
    if (e != cudaSuccess) return fail(RMAT_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    plan.fast_kernel = nullptr;
    if (packed_words && !u64) {
        const int tile = 512;
        const size_t fast = (t->image.size() - packed_words) * 4 + 32 * size_t(warp_region_bytes(false, false, tile));
        if (fast <= size_t(props.max_smem)) {
            e = set_smem_attr(reinterpret_cast<void *>(&k_kron_fast), fast);
            if (e != cudaSuccess)
                return fail(RMAT_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
            plan.fast_kernel = reinterpret_cast<void *>(&k_kron_fast);
            plan.fast_smem_bytes = fast;
            plan.tile = tile;
        }
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, plan.kernel, plan.threads, plan.smem_bytes);
    if (e != cudaSuccess) return fail(RMAT_ERR_CUDA, std::string("occupancy query: ") + cudaGetErrorString(e));
    if (per_sm < 1) return fail(RMAT_ERR_UNSUPPORTED, "launch shape does not fit on an SM");
    plan.ctas_per_sm = per_sm;
    plan.sms = props.sms;
    plan.err = props.err;
    return RMAT_OK;
}

rmat_status launch_kron(const rmat_table *t, const uint32_t *dblob, const AliasPlan &plan, uint64_t seed,
                        uint64_t e0, uint64_t count, void *out, cudaStream_t stream) {
    KronJob J{};
    J.blob = dblob;
    J.blob_bytes = uint32_t(plan.smem_bytes);
    J.aa_off = 4u * t->gdesc[0].a_off_words;
    J.p_off = 4u * t->gdesc[0].bs_off_words;
    J.mulb = 1u << t->gdesc[0].bits;
    J.c_off = 4u * t->gdesc[0].ba_off_words;
    J.c_bytes = J.c_off ? uint32_t(t->image.size() * 4) - J.c_off : 0u;
    J.c_shift = uint32_t(kron_packed_shift(t));
    J.bits = uint32_t(t->gdesc[0].bits);
    J.k = t->k;
    const uint32_t k0 = uint32_t(seed), k1 = uint32_t(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        J.ks[2 * r] = k0 + uint32_t(r) * 0x9E3779B9u;
        J.ks[2 * r + 1] = k1 + uint32_t(r) * 0xBB67AE85u;
    }
    J.e0 = e0;
    J.count = count;
    J.out = out;
    uint64_t v = 1;
    for (int j = 0; j <= kMaxKronK; ++j) {
        J.pw[j] = j <= t->k ? v : 0;  // n0^k may be 2^64 (wraps to 0; used only times 0)
        v *= uint64_t(t->n0);
    }
    const uint64_t two32 = uint64_t(1) << 32;
    uint64_t D = 1;  // n0^d while it is <= 2^32, then held above 2^32 (no wrap-around)
    for (int d = 0; d <= 32; ++d) {
        J.mg[d] = (d >= 1 && D <= two32) ? uint64_t(((unsigned __int128)1 << 64) / D) + 1 : 0;
        D = D <= two32 ? D * uint64_t(t->n0) : D;
    }
    // The whole tiles of an aligned output go to the contract-case kernel when
    // the table packs; the ragged tail (and every other case) to k_kron.
    int tile = plan.tile;
    if (plan.fast_kernel && count >= uint64_t(tile) && (reinterpret_cast<uintptr_t>(out) & 15u) == 0) {
        const uint64_t nfull = count / uint64_t(tile);
        KronJob F = J;
        F.count = nfull * uint64_t(tile);
        const uint64_t warps = plan.threads / 32;
        const unsigned fgrid = unsigned(std::max<uint64_t>(1, std::min<uint64_t>((nfull + warps - 1) / warps, plan.sms)));
        void *fparams[] = {&F, &tile};
        cudaError_t e = cudaLaunchKernel(plan.fast_kernel, dim3(fgrid), dim3(plan.threads), fparams,
                                         plan.fast_smem_bytes, stream);
        if (e != cudaSuccess) return fail(RMAT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
        if (count == F.count) return RMAT_OK;
        J.e0 += F.count;
        J.count = count - F.count;
        J.out = static_cast<unsigned char *>(out) + F.count * 8u;
        count = J.count;
    }
    const uint64_t blocks = (count + plan.threads - 1) / plan.threads;
    const unsigned grid = unsigned(std::max<uint64_t>(1, std::min<uint64_t>(blocks, uint64_t(plan.sms) * plan.ctas_per_sm)));
    void *params[] = {&J};
    cudaError_t e = cudaLaunchKernel(plan.kernel, dim3(grid), dim3(plan.threads), params, plan.smem_bytes, stream);
    if (e != cudaSuccess) return fail(RMAT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return RMAT_OK;
}

// Draws of phase 1 (one Philox block): as many as k levels can need, at most
// four -- ceil(k / shortest path with non-zero weight).
int phase1_draws(const rmat_table *t) {
    const int min_len = std::max(1, t->groups[0].min_len);
    return std::max(1, std::min(4, (t->k + min_len - 1) / min_len));
}

rmat_status plan_alias_launch(const rmat_table *t, const rmat_launch_config_t &want, AliasPlan &plan) {
    DeviceProps props;
    if (rmat_status st = device_props(props)) return st;
    if (t->n0 > 2) return plan_kron_launch(t, props, plan);
    const bool u64 = t->k > 32;
    const bool levels = t->per_level;
    const size_t img = t->image.size() * 4;

    int threads = std::max(128, std::min(1024, want.threads / 32 * 32));
    int tile = std::max(32, std::min(1024, want.tile_edges / 32 * 32));
    const int ctas = std::max(1, std::min(8, want.ctas_per_sm));
    auto need = [&](bool smem_table, int th, int tl) {
        return size_t(16) + (smem_table ? img + (levels ? 16 * kMaxGroups : 0) : 0) +
               size_t(th / 32) * warp_region_bytes(u64, levels, tl);
    };
    bool smem_table = true;
    // shrink the tile, then the CTA, until the table fits beside the warp tiles
    while (need(true, threads, tile) > size_t(props.max_smem)) {
        if (tile > 128) tile /= 2;
        else if (threads > 256) threads /= 2;
        else {
            smem_table = false;
            break;
        }
    }
    if (!smem_table) {
        threads = std::max(128, std::min(1024, want.threads / 32 * 32));
        tile = std::max(32, std::min(1024, want.tile_edges / 32 * 32));
        while (need(false, threads, tile) > size_t(props.max_smem)) {
            if (tile > 32) tile /= 2;
            else threads /= 2;
        }
    }
    plan.fmt = t->format;
    plan.u64 = u64;
    plan.levels = levels;
    plan.smem_table = smem_table;
    plan.threads = threads;
    plan.tile = tile;
    plan.smem_bytes = need(smem_table, threads, tile);
    const int d4 = phase1_draws(t) == 4 ? 1 : 0;
    const int epi = ((t->flags & RMAT_UNDIRECTED) ? kEpiUndir : 0) | (t->scramble ? kEpiScr : 0);
    plan.kernel = alias_kernel_table[d4][plan.fmt][u64][smem_table][levels][epi]();
    // the contract case: compact u32 tables in shared memory, four phase-1
    // draws, the plain epilogue or relabelling alone
    plan.fast_kernel = !(d4 && plan.fmt == kCompact && !u64 && smem_table && !levels) ? nullptr
                       : epi == 0        ? reinterpret_cast<void *>(&k_alias_fast<false>)
                       : epi == kEpiScr  ? reinterpret_cast<void *>(&k_alias_fast<true>)
                                         : nullptr;
    cudaError_t e = set_smem_attr(plan.kernel, plan.smem_bytes);
    if (e == cudaSuccess && plan.fast_kernel) e = set_smem_attr(plan.fast_kernel, plan.smem_bytes);
    if (e == cudaSuccess && plan.fast_kernel) e = set_smem_attr(reinterpret_cast<void *>(&k_part_fast), plan.smem_bytes);
    if (e != cudaSuccess) return fail(RMAT_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, plan.kernel, threads, plan.smem_bytes);
    if (e != cudaSuccess) return fail(RMAT_ERR_CUDA, std::string("occupancy query: ") + cudaGetErrorString(e));
    if (per_sm < 1) return fail(RMAT_ERR_UNSUPPORTED, "launch shape does not fit on an SM");
    plan.ctas_per_sm = std::min(per_sm, ctas);
    plan.sms = props.sms;
    plan.err = props.err;
    return RMAT_OK;
}

Job make_job(const rmat_table *t, const uint32_t *dblob, bool smem, uint64_t seed, uint64_t e0, uint64_t count,
             void *out) {
    Job J{};
    J.blob = dblob;
    J.blob_bytes = uint32_t(t->image.size() * 4);
    J.k = t->k;
    J.one = 1u;
    J.draws1 = phase1_draws(t);
    J.ngroups = int(t->groups.size());
    J.levels = t->per_level ? 1u : 0u;
    J.flags = t->flags;
    for (int r = 0; r < 10; ++r) {
        J.ks[2 * r] = uint32_t(seed) + uint32_t(r) * 0x9E3779B9u;
        J.ks[2 * r + 1] = uint32_t(seed >> 32) + uint32_t(r) * 0xBB67AE85u;
    }
    J.e0 = e0;
    J.count = count;
    J.out = out;
    J.fmt = uint32_t(t->format);
    J.smem = smem ? 1u : 0u;
    if (t->scramble) J.flags |= kScrambleFlag;
    J.a0 = t->gdesc[0].a_off_words;
    J.bs0 = t->gdesc[0].bs_off_words;
    J.ba0 = t->gdesc[0].ba_off_words;
    J.bits0 = uint32_t(t->gdesc[0].bits);
    J.unit_begin = 0;
    return J;
}

void set_tile_prefix(Job &J, const rmat_table *t, int levels, uint64_t R, uint64_t C) {
    const int W = t->k > 32 ? 64 : 32;
    J.pre_len = uint32_t(levels);
    J.pre_row = levels ? R << (W - levels) : 0;
    J.pre_col = levels ? C << (W - levels) : 0;
    const int min_len = std::max(1, t->groups[0].min_len);
    J.draws1 = std::max(1, std::min(4, (t->k - levels + min_len - 1) / min_len));
}

Scramble make_scramble(const rmat_table *t) {
    Scramble S{};
    if (!t->scramble) return S;
    const int W = t->k > 32 ? 64 : 32;
    const int s = W - t->k;
    const uint64_t wmask = W == 64 ? ~0ull : 0xFFFFFFFFull;
    for (int i = 0; i < 3; ++i) {
        S.m[i] = t->scr[2 * i];
        S.a[i] = (t->scr[2 * i + 1] << s) & wmask;
    }
    S.mask = (wmask << s) & wmask;
    return S;
}

rmat_status launch_partition_fast(const rmat_table *t, const uint32_t *dblob, const AliasPlan &plan, uint64_t seed,
                                  const PartTile *tiles, uint32_t ntiles, uint64_t nwt, void *out,
                                  cudaStream_t stream) {
    if (nwt == 0) return RMAT_OK;
    if (!plan.fast_kernel) return fail(RMAT_ERR_UNSUPPORTED, "table does not take the contract-case kernel");
    Job J = make_job(t, dblob, true, seed, 0, 0, out);
    int tile = plan.tile;
    const uint64_t warps = uint64_t(plan.threads / 32);
    const uint64_t max_ctas = uint64_t(plan.sms) * plan.ctas_per_sm;
    const unsigned grid = unsigned(std::max<uint64_t>(1, std::min((nwt + warps - 1) / warps, max_ctas)));
    void *params[] = {&J, &tiles, &ntiles, &nwt, &tile};
    cudaError_t e = cudaLaunchKernel(reinterpret_cast<void *>(&k_part_fast), dim3(grid), dim3(plan.threads), params,
                                     plan.smem_bytes, stream);
    if (e != cudaSuccess) return fail(RMAT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return RMAT_OK;
}

rmat_status launch_alias(const rmat_table *t, const uint32_t *dblob, const AliasPlan &plan, uint64_t seed,
                         uint64_t e0, uint64_t count, void *out, cudaStream_t stream) {
    if (count == 0) return RMAT_OK;
    if (plan.fmt == kKron) return launch_kron(t, dblob, plan, seed, e0, count, out, stream);
    Job J = make_job(t, dblob, plan.smem_table, seed, e0, count, out);
    Scramble S = make_scramble(t);
    unsigned *err = plan.err;
    const int warps = plan.threads / 32;
    // Small launches: smaller tiles (down to 64 edges) until every warp of a
    // full grid has a tile.  A smaller tile fits in the planned shared memory,
    // and the bytes written never depend on the tile size.
    int tile = plan.tile;
    const uint64_t grid_warps = uint64_t(plan.sms) * plan.ctas_per_sm * warps;
    while (tile > 64 && tile % 64 == 0 && (count + tile - 1) / tile < grid_warps) tile /= 2;
    const uint64_t max_ctas = uint64_t(plan.sms) * plan.ctas_per_sm;
    // The whole tiles of an aligned output go to the contract-case kernel when
    // the table allows it; the ragged tail (and every other case) to k_alias.
    if (plan.fast_kernel && tile % 128 == 0 && count >= uint64_t(tile) &&
        (reinterpret_cast<uintptr_t>(out) & 15u) == 0) {
        // a launch too small to give every warp of the GPU a tile takes
        // smaller tiles (down to 128 edges; the bytes do not depend on it)
        int ftile = tile;
        while (ftile > 128 && count / uint64_t(ftile) < max_ctas * uint64_t(warps)) ftile /= 2;
        const uint64_t nfull = count / uint64_t(ftile);
        Job F = J;
        F.count = nfull * uint64_t(ftile);
        const unsigned grid = unsigned(std::max<uint64_t>(1, std::min((nfull + warps - 1) / warps, max_ctas)));
        void *params[] = {&F, &S, &ftile};
        cudaError_t e =
            cudaLaunchKernel(plan.fast_kernel, dim3(grid), dim3(plan.threads), params, plan.smem_bytes, stream);
        if (e != cudaSuccess) return fail(RMAT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
        if (count == F.count) return RMAT_OK;
        J.e0 += F.count;
        J.count = count - F.count;
        J.out = static_cast<unsigned char *>(out) + F.count * 8u;
        count = J.count;
    }
    const uint64_t ntiles = (count + tile - 1) / tile;
    const uint64_t want_ctas = (ntiles + warps - 1) / warps;
    const unsigned grid = unsigned(std::max<uint64_t>(1, std::min(want_ctas, max_ctas)));
    void *params[] = {&J, &S, &tile, &err};
    cudaError_t e = cudaLaunchKernel(plan.kernel, dim3(grid), dim3(plan.threads), params, plan.smem_bytes, stream);
    if (e != cudaSuccess) return fail(RMAT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return RMAT_OK;
}

size_t batch_smem_bytes(bool u64, int threads, int tile, uint32_t max_blob_bytes) {
    return kBatchHeaderBytes + size_t(max_blob_bytes) + size_t(threads / 32) * warp_region_bytes(u64, false, tile);
}

void *batch_kernel(bool u64, bool general) {
    if (u64) return general ? reinterpret_cast<void *>(&k_batch<true, true>)
                            : reinterpret_cast<void *>(&k_batch<true, false>);
    return general ? reinterpret_cast<void *>(&k_batch<false, true>) : reinterpret_cast<void *>(&k_batch<false, false>);
}

rmat_status batch_occupancy(bool u64, int threads, size_t smem, int &per_sm) {
    for (bool pre : {false, true}) {
        const cudaError_t e = set_smem_attr(batch_kernel(u64, pre), smem);
        if (e != cudaSuccess)
            return fail(RMAT_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    }
    // the smaller occupancy of the two variants (same CTA shape)
    int per_sm_pre = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel(u64, false), threads, smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_pre, batch_kernel(u64, true), threads, smem);
    per_sm = std::min(per_sm, per_sm_pre);
    if (e != cudaSuccess) return fail(RMAT_ERR_CUDA, std::string("occupancy query: ") + cudaGetErrorString(e));
    return RMAT_OK;
}

rmat_status load_batch_kernels() {
    for (bool u64 : {false, true})
        for (bool general : {false, true}) {
            cudaFuncAttributes attr;
            cudaError_t e = cudaFuncGetAttributes(&attr, batch_kernel(u64, general));
            if (e == cudaSuccess) e = set_smem_attr(batch_kernel(u64, general), 0);
            if (e != cudaSuccess)
                return fail(RMAT_ERR_CUDA, std::string("loading the batched kernel: ") + cudaGetErrorString(e));
        }
    return RMAT_OK;
}

rmat_status launch_batch(bool u64, const BatchArgs &args, int grid, int threads, size_t smem, cudaStream_t stream) {
    void *fn = (!u64 && args.fast) ? reinterpret_cast<void *>(&k_batch_fast) : batch_kernel(u64, args.general != 0);
    if (!u64 && args.fast) {
        const cudaError_t ea = set_smem_attr(fn, smem);
        if (ea != cudaSuccess) return fail(RMAT_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(ea));
    }
    cudaError_t e = cudaMemsetAsync(args.counter, 0, sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return fail(RMAT_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    BatchArgs a = args;
    void *params[] = {&a};
    e = cudaLaunchKernel(fn, dim3(grid), dim3(threads), params, smem, stream);
    if (e != cudaSuccess) return fail(RMAT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return RMAT_OK;
}

rmat_status launch_checksum(bool u64, const BatchArgs &args, unsigned long long *sums, int grid,
                            cudaStream_t stream) {
    void *fn = u64 ? reinterpret_cast<void *>(&k_checksum<true>) : reinterpret_cast<void *>(&k_checksum<false>);
    BatchArgs a = args;
    void *params[] = {&a, &sums};
    const unsigned g = unsigned(std::max<uint64_t>(1, std::min<uint64_t>(uint64_t(grid), args.units)));
    cudaError_t e = cudaLaunchKernel(fn, dim3(g), dim3(256), params, 0, stream);
    if (e != cudaSuccess) return fail(RMAT_ERR_CUDA, std::string("checksum launch: ") + cudaGetErrorString(e));
    return RMAT_OK;
}

rmat_status launch_naive(const uint32_t *thr3, int k, unsigned flags, uint64_t seed, uint64_t e0, uint64_t count,
                         void *out, cudaStream_t stream) {
    if (count == 0) return RMAT_OK;
    DeviceProps props;
    if (rmat_status st = device_props(props)) return st;
    NaiveArgs a;
    a.k = k;
    a.flags = flags;
    a.key0 = uint32_t(seed);
    a.key1 = uint32_t(seed >> 32);
    a.e0 = e0;
    a.count = count;
    a.out = out;
    std::copy(thr3, thr3 + 3 * k, a.thr);
    const uint64_t blocks = (count + 255) / 256;
    const unsigned grid = unsigned(std::min<uint64_t>(blocks, uint64_t(props.sms) * 8));
    void *params[] = {&a};
    void *fn = k > 32 ? reinterpret_cast<void *>(&k_naive<true>) : reinterpret_cast<void *>(&k_naive<false>);
    cudaError_t e = cudaLaunchKernel(fn, dim3(grid), dim3(256), params, 0, stream);
    if (e != cudaSuccess) return fail(RMAT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return RMAT_OK;
}

rmat_status read_and_clear_device_error(unsigned &value) {
    DeviceProps props;
    if (rmat_status st = device_props(props)) return st;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail(RMAT_ERR_CUDA, std::string("cudaDeviceSynchronize: ") + cudaGetErrorString(e));
    e = cudaMemcpyFromSymbol(&value, g_device_error, sizeof(unsigned));
    if (e != cudaSuccess) return fail(RMAT_ERR_CUDA, std::string("cudaMemcpyFromSymbol: ") + cudaGetErrorString(e));
    const unsigned zero = 0;
    e = cudaMemcpyToSymbol(g_device_error, &zero, sizeof(unsigned));
    if (e != cudaSuccess) return fail(RMAT_ERR_CUDA, std::string("cudaMemcpyToSymbol: ") + cudaGetErrorString(e));
    return RMAT_OK;
}

}  // namespace rmat
