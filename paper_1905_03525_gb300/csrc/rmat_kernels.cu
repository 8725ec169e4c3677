// rmat_kernels.cu -- the sampling kernels of librmat (sm_103a) and their
// launch logic.
//
// k_alias: the per-edge sampling loop of arXiv 1905.03525, Sec. 2 (sampling-
// loop fragment), one edge per lane:
//   phase 1  one Philox4x32-10 block (4 words) per edge, up to 4 alias draws,
//            path bits OR-ed into left-aligned row/column registers;
//   phase 2  edges that still lack levels after 4 words are queued per warp
//            (ballot + popc compaction in shared memory) and finished 32 at a
//            time with further Philox blocks, so that the rare long edges do
//            not make every lane of a warp pay for a second block.
// The alias table is staged once per CTA into shared memory by a TMA bulk
// copy completing on an mbarrier.  Edges are written into a per-warp shared
// tile and leave with one TMA bulk store per tile (double-buffered, so the
// store of tile i overlaps the sampling of tile i+1).
// Per-level tables (Sec. 3, one table per level group) use exactly one draw
// per group, with no phase 2.
//
// k_naive: the plain R-MAT process (Sec. 1), one quadrant draw per level.
#include <algorithm>
#include <cstdio>
#include <mutex>
#include <vector>

#include "rmat_device.cuh"
#include "rmat_internal.h"
#include "rmat_kernels.h"

namespace rmat {

__device__ unsigned int g_device_error;

namespace {

constexpr int kPendCap = 64;           // per-warp queue of unfinished edges
constexpr uint32_t kWaitLimit = 1u << 22;
constexpr int kMaxGroups = 64;

struct AliasArgs {
    const uint32_t *image;  // device table image
    uint32_t image_bytes;   // bytes to stage (multiple of 16); 0 = table read from global
    uint32_t a_off, b_off;  // group-0 offsets (words)
    uint32_t bits;
    int k;
    int draws1;             // draws in phase 1 (<= 4)
    int ngroups;            // per-level: number of groups
    unsigned flags;
    uint32_t key0, key1;
    uint64_t e0;            // global index of the first edge
    uint64_t count;
    void *out;
    int tile;               // edges per warp tile
    unsigned *err;
};

struct LevelDesc {
    uint32_t a_off[kMaxGroups];
    uint32_t b_off[kMaxGroups];
    uint32_t bits[kMaxGroups];
};

template <bool U64>
struct AccT;
template <>
struct AccT<false> { using type = dev::Acc32; using word = uint32_t; };
template <>
struct AccT<true> { using type = dev::Acc64; using word = uint64_t; };

template <int FMT, bool U64, bool SMEM, bool LEVELS>
__global__ void __launch_bounds__(1024) k_alias(AliasArgs args, LevelDesc ld) {
    using Acc = typename AccT<U64>::type;
    using Word = typename AccT<U64>::word;
    constexpr uint32_t EB = U64 ? 16 : 8;
    constexpr uint32_t PB = LEVELS ? 0 : kPendCap * (8 + 2 * sizeof(Word));

    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem);
    uint32_t *s_lvl = reinterpret_cast<uint32_t *>(smem + 16);  // 3 x kMaxGroups words
    unsigned char *s_tab = smem + 16 + (LEVELS ? 3 * kMaxGroups * 4 : 0);
    const uint32_t tab_bytes = SMEM ? args.image_bytes : 0;
    unsigned char *s_warps = s_tab + tab_bytes;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int k = args.k;

    if (LEVELS) {
        for (int g = threadIdx.x; g < args.ngroups; g += blockDim.x) {
            s_lvl[g] = ld.a_off[g];
            s_lvl[kMaxGroups + g] = ld.b_off[g];
            s_lvl[2 * kMaxGroups + g] = ld.bits[g];
        }
    }

    const uint32_t *tab;
    if constexpr (SMEM) {
        if (threadIdx.x == 0) {
            dev::mbar_init(mbar, 1);
            dev::fence_mbar_init();
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            dev::mbar_arrive_expect_tx(mbar, args.image_bytes);
            const unsigned char *src = reinterpret_cast<const unsigned char *>(args.image);
            for (uint32_t off = 0; off < args.image_bytes; off += 32768u) {
                const uint32_t n = min(32768u, args.image_bytes - off);
                dev::bulk_g2s(s_tab + off, src + off, n, mbar);
            }
        }
        const bool ok = dev::mbar_wait_bounded(mbar, 0, kWaitLimit);
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) {
                atomicOr(args.err, 1u);
                // give the copy in flight a bounded chance to land before exit
                dev::mbar_wait_bounded(mbar, 0, kWaitLimit);
            }
            return;
        }
        tab = reinterpret_cast<const uint32_t *>(s_tab);
    } else {
        __syncthreads();
        tab = args.image;
    }

    const uint32_t bits0 = args.bits;
    const uint32_t mask0 = (1u << bits0) - 1u;
    const uint32_t *A0 = tab + args.a_off;
    const uint32_t *B0 = tab + args.b_off;
    const int tile = args.tile;

    unsigned char *wreg = s_warps + size_t(warp) * (2 * tile * EB + PB);
    uint32_t *p_idx = reinterpret_cast<uint32_t *>(wreg + 2 * tile * EB);
    uint32_t *p_fill = p_idx + kPendCap;
    Word *p_row = reinterpret_cast<Word *>(p_fill + kPendCap);
    Word *p_col = p_row + kPendCap;

    auto draw = [&](Acc &acc, uint32_t u) {
        const uint32_t sel = dev::alias_select<SMEM>(A0, u, bits0, mask0);
        uint32_t r, c, L;
        dev::fetch_path<FMT, SMEM>(B0, sel, r, c, L);
        acc.append(r, c, L);
    };
    // U32 accumulators tolerate draws past k (shifts clamp, surplus bits
    // fall off); U64 ones are only extended while short of k.
    auto draw_guarded = [&](Acc &acc, uint32_t u) {
        if (U64) {
            if (acc.filled < uint32_t(k)) draw(acc, u);
        } else {
            draw(acc, u);
        }
    };
    auto put = [&](unsigned char *stage, uint32_t idx, const Acc &acc) {
        uint64_t r = acc.out_row(k), c = acc.out_col(k);
        if ((args.flags & RMAT_UNDIRECTED) && r > c) {
            const uint64_t t = r;
            r = c;
            c = t;
        }
        if constexpr (U64)
            reinterpret_cast<ulonglong2 *>(stage)[idx] = make_ulonglong2(r, c);
        else
            reinterpret_cast<uint2 *>(stage)[idx] = make_uint2(uint32_t(r), uint32_t(c));
    };

    const uint64_t ntiles = (args.count + tile - 1) / tile;
    const uint64_t stride = uint64_t(gridDim.x) * nwarps;
    int buf = 0;
    bool issued = false;
    for (uint64_t t = uint64_t(blockIdx.x) * nwarps + warp; t < ntiles; t += stride, buf ^= 1) {
        const uint64_t first = t * tile;
        const uint64_t left = args.count - first;
        const uint32_t n = left < uint64_t(tile) ? uint32_t(left) : uint32_t(tile);
        const uint64_t ebase = args.e0 + first;
        unsigned char *stage = wreg + buf * tile * EB;

        // The bulk store issued two tiles ago read this buffer; wait for it.
        if (lane == 0 && issued) dev::bulk_wait_read_1();
        __syncwarp();

        if constexpr (LEVELS) {
            for (uint32_t base = 0; base < n; base += 32) {
                const uint32_t idx = base + lane;
                const uint64_t e = ebase + idx;
                Acc acc;
                acc.clear();
                for (int q = 0; 4 * q < args.ngroups; ++q) {
                    const uint4 w = dev::philox(uint32_t(q), 0u, uint32_t(e), uint32_t(e >> 32),
                                                args.key0, args.key1);
                    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int g = 4 * q + i;
                        if (g < args.ngroups) {
                            const uint32_t bg = s_lvl[2 * kMaxGroups + g];
                            const uint32_t mg = (1u << bg) - 1u;
                            const uint32_t sel = dev::alias_select<SMEM>(tab + s_lvl[g], ws[i], bg, mg);
                            uint32_t r, c, L;
                            dev::fetch_path<FMT, SMEM>(tab + s_lvl[kMaxGroups + g], sel, r, c, L);
                            acc.append(r, c, L);
                        }
                    }
                }
                if (idx < n) put(stage, idx, acc);
            }
        } else {
            uint32_t pcount = 0;  // warp-uniform
            auto finish = [&](uint32_t pbase, uint32_t nb) {
                // Lanes take queued edges pbase .. pbase+nb-1 and continue
                // their streams from block 1.
                const bool has = uint32_t(lane) < nb;
                Acc acc;
                acc.clear();
                acc.filled = uint32_t(k);
                uint32_t idx = 0;
                if (has) {
                    idx = p_idx[pbase + lane];
                    acc.row = p_row[pbase + lane];
                    acc.col = p_col[pbase + lane];
                    acc.filled = p_fill[pbase + lane];
                }
                const uint64_t e = ebase + idx;
                bool more = true;
                // each draw adds >= 1 level, so at most k draws are ever needed
                for (uint32_t q = 1; more && q <= 17; ++q) {
                    const uint4 w = dev::philox(q, 0u, uint32_t(e), uint32_t(e >> 32), args.key0,
                                                args.key1);
                    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        if (more && !__any_sync(0xffffffffu, acc.filled < uint32_t(k))) more = false;
                        if (more && acc.filled < uint32_t(k)) draw(acc, ws[i]);
                    }
                }
                if (has) put(stage, idx, acc);
            };

            for (uint32_t base = 0; base < uint32_t(tile); base += 32) {
                const uint32_t idx = base + lane;
                const bool valid = idx < n;
                const uint64_t e = ebase + idx;
                const uint4 w = dev::philox(0u, 0u, uint32_t(e), uint32_t(e >> 32), args.key0, args.key1);
                Acc acc;
                acc.clear();
                draw_guarded(acc, w.x);
                if (args.draws1 > 1) draw_guarded(acc, w.y);
                if (args.draws1 > 2) draw_guarded(acc, w.z);
                if (args.draws1 > 3) draw_guarded(acc, w.w);
                const bool done = acc.filled >= uint32_t(k);
                if (valid && done) put(stage, idx, acc);
                const bool pend = valid && !done;
                const uint32_t bal = __ballot_sync(0xffffffffu, pend);
                if (pend) {
                    const uint32_t pos = pcount + __popc(bal & dev::lane_mask_lt());
                    p_idx[pos] = idx;
                    p_row[pos] = acc.row;
                    p_col[pos] = acc.col;
                    p_fill[pos] = acc.filled;
                }
                pcount += __popc(bal);
                if (pcount >= 32) {
                    __syncwarp();
                    finish(pcount - 32, 32);
                    pcount -= 32;
                    __syncwarp();
                }
                if (base + 32 >= n) break;
            }
            if (pcount) {
                __syncwarp();
                finish(0, pcount);
                __syncwarp();
            }
        }

        // Store the tile: one TMA bulk copy when aligned, else plain stores.
        unsigned char *gdst = reinterpret_cast<unsigned char *>(args.out) + first * EB;
        const uint32_t bytes = n * EB;
        const bool bulk = ((reinterpret_cast<uintptr_t>(gdst) | bytes) & 15u) == 0;
        if (bulk) {
            dev::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                dev::bulk_s2g(gdst, stage, bytes);
                dev::bulk_commit();
            }
            issued = true;
        } else {
            __syncwarp();
            const uint64_t *src = reinterpret_cast<const uint64_t *>(stage);
            uint64_t *dst = reinterpret_cast<uint64_t *>(gdst);
            for (uint32_t i = lane; i < bytes / 8; i += 32) dst[i] = src[i];
            __syncwarp();
        }
    }
    if (lane == 0 && issued) dev::bulk_wait_all();
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

template <int FMT, bool U64, bool SMEM, bool LEVELS>
void *alias_kernel_ptr() {
    return reinterpret_cast<void *>(&k_alias<FMT, U64, SMEM, LEVELS>);
}

using KernelFn = void *(*)();
KernelFn alias_kernel_table[2][2][2][2] = {
    {{{alias_kernel_ptr<0, false, false, false>, alias_kernel_ptr<0, false, false, true>},
      {alias_kernel_ptr<0, false, true, false>, alias_kernel_ptr<0, false, true, true>}},
     {{alias_kernel_ptr<0, true, false, false>, alias_kernel_ptr<0, true, false, true>},
      {alias_kernel_ptr<0, true, true, false>, alias_kernel_ptr<0, true, true, true>}}},
    {{{alias_kernel_ptr<1, false, false, false>, alias_kernel_ptr<1, false, false, true>},
      {alias_kernel_ptr<1, false, true, false>, alias_kernel_ptr<1, false, true, true>}},
     {{alias_kernel_ptr<1, true, false, false>, alias_kernel_ptr<1, true, false, true>},
      {alias_kernel_ptr<1, true, true, false>, alias_kernel_ptr<1, true, true, true>}}}};

std::mutex g_props_mu;
std::vector<DeviceProps> g_props;

unsigned *device_error_ptr() {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_device_error) != cudaSuccess) return nullptr;
    return static_cast<unsigned *>(p);
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
    c.tile_edges = t->k > 32 ? 128 : 256;
    return c;
}

rmat_status plan_alias_launch(const rmat_table *t, const rmat_launch_config_t &want, AliasPlan &plan) {
    DeviceProps props;
    if (rmat_status st = device_props(props)) return st;
    const bool u64 = t->k > 32;
    const bool levels = t->per_level;
    const uint32_t EB = u64 ? 16 : 8;
    const uint32_t PB = levels ? 0 : kPendCap * (8 + 2 * (u64 ? 8 : 4));
    const uint32_t head = 16 + (levels ? 3 * kMaxGroups * 4 : 0);
    const uint32_t img = uint32_t(t->image.size() * 4);

    int threads = std::max(128, std::min(1024, want.threads / 32 * 32));
    int tile = std::max(32, std::min(1024, want.tile_edges / 32 * 32));
    int ctas = std::max(1, std::min(8, want.ctas_per_sm));
    auto need = [&](bool smem_table, int th, int tl) {
        return size_t(head) + (smem_table ? img : 0) + size_t(th / 32) * (2 * size_t(tl) * EB + PB);
    };
    bool smem_table = true;
    // shrink tile, then threads, until the table fits next to the warp tiles
    while (need(true, threads, tile) > size_t(props.max_smem)) {
        if (tile > 64) tile /= 2;
        else if (threads > 128) threads /= 2;
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
    plan.kernel = alias_kernel_table[plan.fmt][u64][smem_table][levels]();
    if (plan.smem_bytes > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(plan.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(plan.smem_bytes));
        if (e != cudaSuccess)
            return fail(RMAT_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, plan.kernel, threads,
                                                                  plan.smem_bytes);
    if (e != cudaSuccess)
        return fail(RMAT_ERR_CUDA, std::string("occupancy query: ") + cudaGetErrorString(e));
    if (per_sm < 1) return fail(RMAT_ERR_UNSUPPORTED, "launch shape does not fit on an SM");
    plan.ctas_per_sm = std::min(per_sm, ctas);
    plan.sms = props.sms;
    plan.err = props.err;
    return RMAT_OK;
}

rmat_status launch_alias(const rmat_table *t, const uint32_t *dimage, const AliasPlan &plan, uint64_t seed,
                         uint64_t e0, uint64_t count, void *out, cudaStream_t stream) {
    if (count == 0) return RMAT_OK;
    const PathTable &g0 = t->groups[0];
    AliasArgs a;
    a.image = dimage;
    a.image_bytes = plan.smem_table ? uint32_t(t->image.size() * 4) : 0;
    a.a_off = t->gdesc[0].a_off_words;
    a.b_off = t->gdesc[0].b_off_words;
    a.bits = uint32_t(g0.bits);
    a.k = t->k;
    const int need_draws = (t->k + g0.min_len - 1) / std::max(1, g0.min_len);
    a.draws1 = std::max(1, std::min(4, need_draws));
    a.ngroups = int(t->groups.size());
    a.flags = t->flags;
    a.key0 = uint32_t(seed);
    a.key1 = uint32_t(seed >> 32);
    a.e0 = e0;
    a.count = count;
    a.out = out;
    a.tile = plan.tile;
    a.err = plan.err;
    LevelDesc ld{};
    if (t->per_level) {
        for (size_t g = 0; g < t->gdesc.size(); ++g) {
            ld.a_off[g] = t->gdesc[g].a_off_words;
            ld.b_off[g] = t->gdesc[g].b_off_words;
            ld.bits[g] = uint32_t(t->gdesc[g].bits);
        }
    }
    const int warps = plan.threads / 32;
    const uint64_t ntiles = (count + plan.tile - 1) / plan.tile;
    const uint64_t want_ctas = (ntiles + warps - 1) / warps;
    const uint64_t max_ctas = uint64_t(plan.sms) * plan.ctas_per_sm;
    const unsigned grid = unsigned(std::max<uint64_t>(1, std::min(want_ctas, max_ctas)));
    void *params[] = {&a, &ld};
    cudaError_t e = cudaLaunchKernel(plan.kernel, dim3(grid), dim3(plan.threads), params, plan.smem_bytes, stream);
    if (e != cudaSuccess) return fail(RMAT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
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
