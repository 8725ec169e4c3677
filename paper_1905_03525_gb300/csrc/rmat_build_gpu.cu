// rmat_build_gpu.cu -- construction of the variable-length R-MAT table on the
// GPU (Sec. 3, parallelization: expand every entry above a probability
// threshold level by level, then build the alias table), giving exactly the
// table of the sequential construction (Sec. 2 table-construction fragment,
// readings R1-R6): same entries, order, probabilities, weights and alias
// pairs.
//
// Why the two agree.  The sequential loop pops the queue maximum under the
// order (p desc, symbols asc) and pushes its four children.  A child is never
// more probable than its parent (p * P[s] <= p in FP64) and its symbol string
// extends the parent's, so the order is monotone along every path and the
// popped nodes are exactly the first T nodes of that order among all nodes
// above the depth cap, T = floor((bound - 2) / 3) (fewer if the tree above the
// cap is smaller).  The table is the set of children of popped nodes that were
// not popped themselves, in lexicographic order.
//
// One CTA of 1024 threads runs the whole construction in one launch:
//   1. level-synchronous expansion of every node with p >= theta (theta from
//      the host, a safe lower bound on the T-th probability), children in
//      (parent, symbol) order so that each level is in lexicographic order;
//   2. the T-th node: radix select on the FP64 bits of p, then on the symbol
//      keys within the tie class at the cut;
//   3. leaf counts bottom-up and lexicographic ranks top-down (DFS offsets);
//   4. u32 quantisation with the largest-remainder rule (radix select on the
//      fractional parts, lower index first among ties);
//   5. integer Vose with FIFO queues (sequential, one thread, streaming its
//      queues of {index, value} pairs);
//   6. the device image (A, Bs, Ba as rmat_image.cpp lays them out).
// The node arrays live in a device scratch sized by the host; any overflow
// sets an error in the status and the kernel returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "rmat_internal.h"
#include "rmat_kernels.h"

namespace rmat {
namespace {

struct BuildStatus {
    uint32_t error;      // 0 ok, 1 node scratch overflow, 2 threshold too high, 3 quantisation, 4 alias
    uint32_t entries;    // |Q|
    uint32_t bits;
    uint32_t max_len;
    uint32_t min_len;
    uint32_t format;
    uint64_t nodes;      // nodes generated
    uint64_t expanded;   // T_eff
    uint64_t stamp[8];   // %globaltimer (ns) at the end of phases 1..6 (stamp[0]: start)
};

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct BuildArgs {
    double P[4];
    int cap;             // min(k, 32)
    uint64_t T;          // expansions of the sequential loop
    double theta;        // every node with p >= theta is a candidate
    int theta_all;       // theta = 0: the whole tree above the cap
    // node scratch
    double *np;
    uint64_t *nkey;
    uint8_t *ndepth;
    uint8_t *nflag;      // bit 0 candidate, bit 1 expanded, bit 2 in the table tree
    uint32_t *ncbase;    // first child of an expanded candidate
    uint32_t *nleaf;
    uint32_t *noff;
    uint64_t node_cap;
    uint32_t *level_lo;  // 34 entries
    // table (Nmax entries)
    uint64_t *sym;
    uint8_t *len;
    double *p;
    uint64_t *w;
    uint32_t *thr;
    uint32_t *alias;
    uint2 *small_q;      // FIFO of {index, weight or rest} (< C)
    uint2 *large_q;      // {index, weight} (>= C)
    uint32_t *image;
    uint64_t nmax;
    BuildStatus *st;
};

constexpr int kThreads = 1024;

// Exclusive block scan of one value per thread; `total` gets the sum.
__device__ uint32_t block_scan(uint32_t v, uint32_t &total, uint32_t *sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sm[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t y = lane < nw ? sm[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t z = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += z;
        }
        sm[lane] = y;
    }
    __syncthreads();
    const uint32_t excl = x - v + (warp ? sm[warp - 1] : 0u);
    total = sm[nw - 1];
    __syncthreads();
    return excl;
}

__device__ uint64_t block_sum64(uint64_t v, unsigned long long *sm) {
    if (threadIdx.x == 0) *sm = 0;
    __syncthreads();
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(sm, (unsigned long long)v);
    __syncthreads();
    const uint64_t r = *sm;
    __syncthreads();
    return r;
}

// Radix select over 64-bit keys of the elements i < n with pred(i): the key
// of rank `rank` (1-based) in descending (desc) or ascending order.
template <class KeyF, class PredF>
__device__ uint64_t block_select(uint64_t n, uint64_t rank, bool desc, KeyF key, PredF pred, uint32_t *hist,
                                 unsigned long long *sh) {
    uint64_t prefix = 0, mask = 0;
    for (int byte = 7; byte >= 0; --byte) {
        for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        for (uint64_t i = threadIdx.x; i < n; i += blockDim.x)
            if (pred(i)) {
                const uint64_t kv = key(i);
                if ((kv & mask) == prefix) atomicAdd(&hist[(kv >> (8 * byte)) & 255u], 1u);
            }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint64_t acc = 0;
            int sel = desc ? 0 : 255;
            for (int s = 0; s < 256; ++s) {
                const int b = desc ? 255 - s : s;
                if (acc + hist[b] >= rank) {
                    sel = b;
                    break;
                }
                acc += hist[b];
            }
            sh[0] = (unsigned long long)sel;
            sh[1] = (unsigned long long)(rank - acc);
        }
        __syncthreads();
        prefix |= uint64_t(sh[0]) << (8 * byte);
        mask |= uint64_t(0xFF) << (8 * byte);
        rank = sh[1];
        __syncthreads();
    }
    return prefix;
}

__device__ uint64_t dbits(double x) { return uint64_t(__double_as_longlong(x)); }

__global__ void __launch_bounds__(kThreads, 1) k_build_table(const __grid_constant__ BuildArgs A) {
    __shared__ uint32_t sm_scan[33];
    __shared__ uint32_t hist[256];
    __shared__ unsigned long long sh[4];
    __shared__ uint32_t s_flag;
    const uint32_t tid = threadIdx.x;
    BuildStatus *st = A.st;

    // 1. expansion, level by level
    if (tid == 0) {
        st->stamp[0] = gtimer();
        A.np[0] = 1.0;
        A.nkey[0] = 0;
        A.ndepth[0] = 0;
        A.nflag[0] = 0;
        A.level_lo[0] = 0;
        A.level_lo[1] = 1;
        s_flag = 0;
    }
    __syncthreads();
    int levels = 1;  // levels present: 0 .. levels-1
    for (int d = 0; d < A.cap; ++d) {
        const uint32_t lo = A.level_lo[d], hi = A.level_lo[d + 1];
        uint64_t next = hi;
        for (uint32_t base = lo; base < hi; base += blockDim.x) {
            const uint32_t i = base + tid;
            const bool cand = i < hi && (A.theta_all || A.np[i] >= A.theta);
            uint32_t total;
            const uint32_t ex = block_scan(cand ? 1u : 0u, total, sm_scan);
            if (next + 4ull * total > A.node_cap) {
                if (tid == 0) st->error = 1;
                return;
            }
            if (i < hi) A.nflag[i] = cand ? 1 : 0;
            if (cand) {
                const uint32_t c0 = uint32_t(next + 4ull * ex);
                A.ncbase[i] = c0;
                const double pi = A.np[i];
                const uint64_t ki = A.nkey[i];
                for (int s = 0; s < 4; ++s) {
                    A.np[c0 + s] = pi * A.P[s];
                    A.nkey[c0 + s] = ki | (uint64_t(s) << (62 - 2 * d));
                    A.ndepth[c0 + s] = uint8_t(d + 1);
                    A.nflag[c0 + s] = 0;
                }
            }
            next += 4ull * total;
        }
        if (tid == 0) A.level_lo[d + 2] = uint32_t(next);
        __syncthreads();
        levels = d + 2;
        if (next == hi) {
            levels = d + 1;
            break;
        }
    }
    const uint64_t nodes = A.level_lo[levels];
    if (tid == 0) st->stamp[1] = gtimer();

    // 2. the T-th candidate under (p desc, key asc)
    uint32_t cnt_local = 0;
    for (uint64_t i = tid; i < nodes; i += blockDim.x) cnt_local += A.nflag[i] & 1u;
    const uint64_t ncand = block_sum64(cnt_local, sh + 2);
    uint64_t T = A.T;
    if (ncand < T) {
        if (!A.theta_all) {  // the threshold cut off part of the first T nodes
            if (tid == 0) st->error = 2;
            return;
        }
        T = ncand;  // the whole tree above the cap is expanded
    }
    uint64_t pi_bits = 0, kappa = 0;
    if (T > 0) {
        auto is_cand = [&](uint64_t i) { return (A.nflag[i] & 1u) != 0; };
        pi_bits = block_select(nodes, T, true, [&](uint64_t i) { return dbits(A.np[i]); }, is_cand, hist, sh);
        uint32_t gt_local = 0;
        for (uint64_t i = tid; i < nodes; i += blockDim.x)
            gt_local += ((A.nflag[i] & 1u) && dbits(A.np[i]) > pi_bits) ? 1u : 0u;
        const uint64_t ngt = block_sum64(gt_local, sh + 2);
        kappa = block_select(nodes, T - ngt, false, [&](uint64_t i) { return A.nkey[i]; },
                             [&](uint64_t i) { return (A.nflag[i] & 1u) && dbits(A.np[i]) == pi_bits; }, hist, sh);
    }
    // expanded: candidate above the cut; the children of expanded nodes and
    // the root form the table tree
    for (uint64_t i = tid; i < nodes; i += blockDim.x) {
        const uint64_t pb = dbits(A.np[i]);
        const bool ex = T > 0 && (A.nflag[i] & 1u) && (pb > pi_bits || (pb == pi_bits && A.nkey[i] <= kappa));
        if (ex) A.nflag[i] |= 2u;
    }
    if (tid == 0) A.nflag[0] |= 4u;
    __syncthreads();
    for (uint64_t i = tid; i < nodes; i += blockDim.x)
        if (A.nflag[i] & 2u)
            for (int s = 0; s < 4; ++s) A.nflag[A.ncbase[i] + s] |= 4u;
    __syncthreads();

    if (tid == 0) st->stamp[2] = gtimer();

    // 3. leaf counts bottom-up, then lexicographic offsets top-down
    for (int d = levels - 1; d >= 0; --d) {
        for (uint32_t i = A.level_lo[d] + tid; i < A.level_lo[d + 1]; i += blockDim.x) {
            const uint8_t f = A.nflag[i];
            uint32_t c = 0;
            if (f & 2u) {
                const uint32_t b = A.ncbase[i];
                c = A.nleaf[b] + A.nleaf[b + 1] + A.nleaf[b + 2] + A.nleaf[b + 3];
            } else if (f & 4u) {
                c = 1;
            }
            A.nleaf[i] = c;
        }
        __syncthreads();
    }
    if (tid == 0) A.noff[0] = 0;
    __syncthreads();
    for (int d = 0; d < levels; ++d) {
        for (uint32_t i = A.level_lo[d] + tid; i < A.level_lo[d + 1]; i += blockDim.x)
            if (A.nflag[i] & 2u) {
                uint32_t o = A.noff[i];
                const uint32_t b = A.ncbase[i];
                for (int s = 0; s < 4; ++s) {
                    A.noff[b + s] = o;
                    o += A.nleaf[b + s];
                }
            }
        __syncthreads();
    }
    const uint32_t entries = A.nleaf[0];
    int bits = 1;
    while ((uint64_t(1) << bits) < entries) ++bits;
    const uint32_t N = 1u << bits;
    if (N > A.nmax) {
        if (tid == 0) st->error = 1;
        return;
    }
    for (uint32_t j = tid; j < N; j += blockDim.x) {
        A.sym[j] = 0;
        A.len[j] = 0;
        A.p[j] = 0.0;
    }
    __syncthreads();
    uint32_t ml_local = 0;
    for (uint64_t i = tid; i < nodes; i += blockDim.x) {
        const uint8_t f = A.nflag[i];
        if ((f & 4u) && !(f & 2u)) {
            const uint32_t r = A.noff[i];
            A.sym[r] = A.nkey[i];
            A.len[r] = A.ndepth[i];
            A.p[r] = A.np[i];
            ml_local = max(ml_local, uint32_t(A.ndepth[i]));
        }
    }
    __syncthreads();

    if (tid == 0) st->stamp[3] = gtimer();

    // 4. quantisation: w = floor(p 2^32), the missing units to the largest
    // fractional parts (lower index first among equal parts)
    uint64_t wsum_local = 0;
    for (uint32_t j = tid; j < N; j += blockDim.x) {
        const double x = A.p[j] * 4294967296.0;  // exact scaling
        const double fl = floor(x);
        A.w[j] = uint64_t(fl);
        wsum_local += uint64_t(fl);
    }
    const uint64_t wsum = block_sum64(wsum_local, sh + 2);
    const uint64_t two32 = uint64_t(1) << 32;
    if (wsum > two32 || two32 - wsum > N) {
        if (tid == 0) st->error = 3;
        return;
    }
    const uint64_t missing = two32 - wsum;
    auto frac_bits = [&](uint64_t j) {
        const double x = A.p[j] * 4294967296.0;
        return dbits(x - floor(x));
    };
    if (missing) {
        const uint64_t phi = block_select(N, missing, true, frac_bits, [](uint64_t) { return true; }, hist, sh);
        uint32_t gt_local = 0;
        for (uint32_t j = tid; j < N; j += blockDim.x) gt_local += frac_bits(j) > phi ? 1u : 0u;
        const uint64_t ngt = block_sum64(gt_local, sh + 2);
        const uint64_t r = missing - ngt;  // among parts equal to phi, the first r indices
        uint32_t carry = 0;
        for (uint32_t base = 0; base < N; base += blockDim.x) {
            const uint32_t j = base + tid;
            const uint64_t fb = j < N ? frac_bits(j) : 0;
            const bool tie = j < N && fb == phi;
            uint32_t total;
            const uint32_t ex = block_scan(tie ? 1u : 0u, total, sm_scan);
            if (j < N && (fb > phi || (tie && carry + ex < r))) A.w[j] += 1;
            carry += total;
        }
    }
    __syncthreads();

    if (tid == 0) st->stamp[4] = gtimer();

    // 5. integer Vose, FIFO queues in index order.  The queue X holds the
    // lights (index order) and, behind them, heavies as they turn light, each
    // with its deficit C - rest; D is the running sum of deficits along X.
    // Heavy h (excess e = w - C) takes the queue entries from the current
    // position until D first exceeds D(start) + e; it turns light with
    // deficit D - D(start) - e and joins the back of X.  Warp 0 runs this
    // heavy by heavy, holding 32 queue entries and their sums in registers:
    // one ballot finds where a heavy turns, and the lanes write the alias
    // pairs of all entries it took -- the sequential FIFO loop, step for step.
    const uint64_t C = two32 >> bits;
    uint32_t ns = 0, nl = 0;
    uint64_t def_local = 0;
    for (uint32_t base = 0; base < N; base += blockDim.x) {
        const uint32_t j = base + tid;
        const bool small = j < N && A.w[j] < C;
        const bool large = j < N && !small;
        uint32_t ts, tl;
        const uint32_t es = block_scan(small ? 1u : 0u, ts, sm_scan);
        const uint32_t el = block_scan(large ? 1u : 0u, tl, sm_scan);
        if (small) {
            A.small_q[ns + es] = make_uint2(j, uint32_t(C - A.w[j]));
            def_local += C - A.w[j];
        }
        if (large) A.large_q[nl + el] = make_uint2(j, uint32_t(A.w[j] - C));  // w < 2^32: >= 4 entries have p > 0
        ns += ts;
        nl += tl;
    }
    const uint64_t deficit = block_sum64(def_local, sh + 2);
    __shared__ uint32_t s_stop;
    if (tid < 32) {
        const unsigned FULL = 0xffffffffu;
        const uint32_t lane = tid;
        uint2 *X = A.small_q;
        const uint2 *H = A.large_q;
        uint32_t pos = 0, tail = ns;
        uint64_t Dpos = 0, Dtail = deficit;
        uint32_t cbase = 0, xi = 0, xd = 0;
        uint64_t xD = 0;
        auto load_chunk = [&]() {  // entries cbase + lane, sums from Dpos (cbase == pos)
            __syncwarp();  // lane 0's appends to X are visible to the other lanes
            const uint32_t t = cbase + lane;
            const bool v = t < tail;
            const uint2 e = v ? X[t] : make_uint2(0u, 0u);
            xi = e.x;
            xd = v ? e.y : 0u;
            uint64_t incl = xd;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t y = __shfl_up_sync(FULL, incl, o);
                if (lane >= uint32_t(o)) incl += y;
            }
            xD = Dpos + incl;
        };
        load_chunk();
        uint32_t hb = 0;
        uint2 hv = lane < nl ? H[lane] : make_uint2(0u, 0u);
        uint32_t j = 0, stop = nl;
        bool ok = true;
        for (; j < nl; ++j) {
            if (j >= hb + 32) {
                hb = j;
                hv = hb + lane < nl ? H[hb + lane] : make_uint2(0u, 0u);
            }
            const uint32_t hidx = __shfl_sync(FULL, hv.x, j - hb);
            const uint64_t F = Dpos + __shfl_sync(FULL, hv.y, j - hb);
            bool exhausted = false;
            for (;;) {  // each pass takes >= 1 entry, turns the heavy, or empties X
                if (pos >= cbase + 32) {
                    cbase = pos;
                    load_chunk();
                }
                const uint32_t t = cbase + lane;
                const bool valid = t >= pos && t < tail;
                const unsigned m = __ballot_sync(FULL, valid && xD > F);
                if (m) {
                    const uint32_t tc = cbase + uint32_t(__ffs(m)) - 1;
                    if (valid && t <= tc) {
                        A.thr[xi] = uint32_t(C) - xd;
                        A.alias[xi] = hidx;
                    }
                    const uint64_t Dt = __shfl_sync(FULL, xD, tc - cbase);
                    const uint32_t o = uint32_t(Dt - F);
                    if (lane == 0) X[tail] = make_uint2(hidx, o);
                    Dtail += o;
                    if (tail >= cbase && tail < cbase + 32 && lane == tail - cbase) {
                        xi = hidx;
                        xd = o;
                        xD = Dtail;
                    }
                    ++tail;
                    pos = tc + 1;
                    Dpos = Dt;
                    break;
                }
                if (valid) {  // the heavy takes every remaining entry of the window
                    A.thr[xi] = uint32_t(C) - xd;
                    A.alias[xi] = hidx;
                }
                if (cbase + 32 >= tail) {  // X is empty: this heavy and the rest stay heavy
                    pos = tail;
                    exhausted = true;
                    break;
                }
                Dpos = __shfl_sync(FULL, xD, 31);
                pos = cbase + 32;
            }
            if (exhausted) {
                stop = j;
                break;
            }
        }
        if (j == nl) ok = pos == tail;  // every heavy turned light: X must be empty
        if (lane == 0) {
            s_stop = stop;
            s_flag = ok ? 0u : 4u;
        }
    }
    __syncthreads();
    if (s_flag) {
        if (tid == 0) st->error = s_flag;
        return;
    }
    for (uint32_t x = s_stop + tid; x < nl; x += blockDim.x) {
        const uint32_t l = A.large_q[x].x;
        A.thr[l] = uint32_t(C - 1);
        A.alias[l] = l;
    }
    __syncthreads();
    if (tid == 0) st->stamp[5] = gtimer();
    uint32_t minl_local = 64;
    for (uint32_t j = tid; j < N; j += blockDim.x)
        if (A.w[j] > 0) minl_local = min(minl_local, uint32_t(A.len[j]));
    // reductions of max_len and min_len
    __shared__ uint32_t s_max, s_min;
    if (tid == 0) {
        s_max = 0;
        s_min = 64;
    }
    __syncthreads();
    atomicMax(&s_max, ml_local);
    atomicMin(&s_min, minl_local);
    __syncthreads();
    const uint32_t max_len = s_max;

    // 6. device image: header, then A, Bs, Ba (compact u32 or wide uint4)
    const bool compact = max_len <= 13;
    const uint32_t bw = compact ? 1u : 4u;
    const uint32_t a_off = uint32_t(kHeaderWords);
    const uint32_t bs_off = a_off + ((N + 3u) & ~3u);
    const uint32_t ba_off = bs_off + ((N * bw + 3u) & ~3u);
    for (uint32_t x = tid; x < kHeaderWords; x += blockDim.x) A.image[x] = 0;
    __syncthreads();
    if (tid == 0) {
        A.image[0] = a_off;
        A.image[kMaxGroups] = bs_off;
        A.image[2 * kMaxGroups] = ba_off;
        A.image[3 * kMaxGroups] = uint32_t(bits);
    }
    auto put = [&](uint32_t off, uint32_t slot, uint32_t i) {
        const int L = A.len[i];
        uint32_t r = 0, c = 0;
        const uint64_t sy = A.sym[i];
        for (int t = 0; t < L; ++t) {
            const uint32_t s = uint32_t(sy >> (62 - 2 * t)) & 3u;
            r = (r << 1) | (s >> 1);
            c = (c << 1) | (s & 1u);
        }
        if (compact) {
            const uint32_t r13 = L ? r << (13 - L) : 0u;
            const uint32_t c13 = L ? c << (13 - L) : 0u;
            A.image[off + slot] = (r13 << 19) | (uint32_t(L) << 13) | c13;
        } else {
            A.image[off + 4 * slot + 0] = L ? r << (32 - L) : 0u;
            A.image[off + 4 * slot + 1] = L ? c << (32 - L) : 0u;
            A.image[off + 4 * slot + 2] = uint32_t(L);
            A.image[off + 4 * slot + 3] = 0u;
        }
    };
    for (uint32_t j = tid; j < N; j += blockDim.x) {
        A.image[a_off + j] = j * uint32_t(C) + A.thr[j];
        put(bs_off, j, j);
        put(ba_off, j, A.alias[j]);
    }
    const uint32_t total_words = ba_off + ((N * bw + 3u) & ~3u);
    for (uint32_t x = bs_off - ((N + 3u) & ~3u) + N + tid; x < bs_off; x += blockDim.x) A.image[x] = 0;  // pad
    if (tid == 0) {
        st->entries = entries;
        st->bits = uint32_t(bits);
        st->max_len = max_len;
        st->min_len = s_min;
        st->format = compact ? 0u : 1u;
        st->nodes = nodes;
        st->expanded = T;
        st->stamp[6] = gtimer();
        st->error = 0;
        (void)total_words;
    }
}

// Host estimate of the cut: nodes above the cap grouped by their symbol
// counts (i, j, l, h), p = a^i b^j c^l d^h with multiplicity d!/(i!j!l!h!).
// Returns theta slightly below the T-th largest p (the FP64 path products
// differ from the exact ones by far less than the margin) and the number of
// nodes at or above it.
void estimate_cut(const double P[4], int cap, uint64_t T, double &theta, bool &all, double &count) {
    struct Comp {
        double lp, mult;
    };
    double lf[65];  // log n!
    lf[0] = 0.0;
    for (int n = 1; n <= 64; ++n) lf[n] = lf[n - 1] + std::log(double(n));
    double lP[4];
    for (int s = 0; s < 4; ++s) lP[s] = std::log(P[s]);
    std::vector<Comp> comps;
    comps.reserve(size_t(cap + 3) * (cap + 2) * (cap + 1) * cap / 24 + 1);
    double total = 0.0;
    for (int d = 0; d < cap; ++d)
        for (int i = 0; i <= d; ++i)
            for (int j = 0; i + j <= d; ++j)
                for (int l = 0; i + j + l <= d; ++l) {
                    const int h = d - i - j - l;
                    const double m = std::exp(lf[d] - lf[i] - lf[j] - lf[l] - lf[h]);
                    comps.push_back({i * lP[0] + j * lP[1] + l * lP[2] + h * lP[3], m});
                    total += m;
                }
    if (total < double(T)) {  // the whole tree above the cap is expanded
        all = true;
        theta = 0.0;
        count = total;
        return;
    }
    // weighted quickselect: the log-probability at which the multiplicities,
    // taken in decreasing order, reach T
    size_t lo = 0, hi = comps.size();
    double need = double(T), cut = 0.0;
    for (;;) {
        if (hi <= lo) {  // rounding in the sums: the last pivot passed is the cut
            break;
        }
        const double pivot = comps[lo + (hi - lo) / 2].lp;
        cut = pivot;
        auto mid1 = std::partition(comps.begin() + lo, comps.begin() + hi, [&](const Comp &c) { return c.lp > pivot; });
        auto mid2 = std::partition(mid1, comps.begin() + hi, [&](const Comp &c) { return c.lp == pivot; });
        double w_gt = 0.0, w_eq = 0.0;
        for (auto it = comps.begin() + lo; it != mid1; ++it) w_gt += it->mult;
        for (auto it = mid1; it != mid2; ++it) w_eq += it->mult;
        if (need <= w_gt) {
            hi = size_t(mid1 - comps.begin());
        } else if (need <= w_gt + w_eq) {
            cut = pivot;
            break;
        } else {
            need -= w_gt + w_eq;
            lo = size_t(mid2 - comps.begin());
        }
    }
    all = false;
    const double lcut = cut - 1e-9;
    theta = std::exp(lcut);
    count = 0.0;
    for (const Comp &c : comps)
        if (c.lp >= lcut - 1e-9) count += c.mult;
}

// Carves typed arrays out of one device allocation (256-byte aligned).
struct Carver {
    size_t bytes = 0;
    unsigned char *base = nullptr;
    template <class T>
    void take(T **p, size_t n) {
        bytes = (bytes + 255) & ~size_t(255);
        *p = reinterpret_cast<T *>(base + bytes);
        bytes += std::max<size_t>(n * sizeof(T), 16);
    }
};

void carve(BuildArgs &A, Carver &c, uint64_t node_cap, uint64_t nmax) {
    c.take(&A.np, node_cap);
    c.take(&A.nkey, node_cap);
    c.take(&A.ndepth, node_cap);
    c.take(&A.nflag, node_cap);
    c.take(&A.ncbase, node_cap);
    c.take(&A.nleaf, node_cap);
    c.take(&A.noff, node_cap);
    c.take(&A.level_lo, 40);
    c.take(&A.sym, nmax);
    c.take(&A.len, nmax);
    c.take(&A.p, nmax);
    c.take(&A.w, nmax);
    c.take(&A.thr, nmax);
    c.take(&A.alias, nmax);
    c.take(&A.st, 1);  // sym .. st: one contiguous span, copied back at once
    c.take(&A.small_q, nmax);
    c.take(&A.large_q, nmax);
}

// Per-device scratch and pinned staging, reused by every build on the device
// (grow-only; builds on one device are serialised).
struct BuildCache {
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    unsigned char *pinned = nullptr;
    size_t pinned_bytes = 0;
};
std::mutex g_build_mu;
std::map<int, BuildCache> g_build_cache;

rmat_status grow(BuildCache &c, size_t scratch_bytes, size_t pinned_bytes) {
    if (c.scratch_bytes < scratch_bytes) {
        if (c.scratch) cudaFree(c.scratch);
        c.scratch = nullptr;
        c.scratch_bytes = 0;
        if (cudaMalloc(&c.scratch, scratch_bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(RMAT_ERR_OUT_OF_MEMORY, "device scratch for the table build");
        }
        c.scratch_bytes = scratch_bytes;
    }
    if (c.pinned_bytes < pinned_bytes) {
        if (c.pinned) cudaFreeHost(c.pinned);
        c.pinned = nullptr;
        c.pinned_bytes = 0;
        if (cudaMallocHost(reinterpret_cast<void **>(&c.pinned), pinned_bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(RMAT_ERR_OUT_OF_MEMORY, "pinned staging for the table build");
        }
        c.pinned_bytes = pinned_bytes;
    }
    return RMAT_OK;
}

}  // namespace
}  // namespace rmat

using namespace rmat;

extern "C" rmat_status rmat_build_table_gpu(double a, double b, double c, double d, int k, uint64_t table_bound,
                                            rmat_stream_t stream_, rmat_table **out) {
    clear_error();
    if (!out) return fail(RMAT_ERR_INVALID_ARGUMENT, "out is NULL");
    *out = nullptr;
    if (k < 1 || k > 64) return fail(RMAT_ERR_INVALID_ARGUMENT, "k must be in [1, 64]");
    if (table_bound < 5 || table_bound > (uint64_t(1) << 24))
        return fail(RMAT_ERR_INVALID_ARGUMENT, "table_bound must be in [5, 2^24]");
    const double in[4] = {a, b, c, d};
    double P[4];
    if (rmat_status st = normalise_params(in, P)) return st;
    // every product of <= 32 parameters stays a normal FP64 number
    for (int s = 0; s < 4; ++s)
        if (!(P[s] >= 1e-9))
            return fail(RMAT_ERR_UNSUPPORTED, "the GPU build needs a, b, c, d >= 1e-9 (use rmat_build_table)");
    DeviceProps props;
    if (rmat_status st = device_props(props)) return st;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);

    BuildArgs A{};
    for (int s = 0; s < 4; ++s) A.P[s] = P[s];
    A.cap = std::min(k, 32);
    A.T = (table_bound - 2) / 3;
    double theta = 0.0, count = 0.0;
    bool all = false;
    estimate_cut(P, A.cap, A.T, theta, all, count);
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_build_mu);
    BuildCache &cache = g_build_cache[dev];
    void *image = nullptr;
    auto release = [&]() {
        if (image) cudaFree(image);
        image = nullptr;
    };
    rmat_status result = RMAT_ERR_UNSUPPORTED;
    // the estimate is exact up to rounding; a retry with a lower threshold
    // (and more scratch) covers a cut that still fell inside the first T nodes
    for (int attempt = 0; attempt < 3; ++attempt) {
        A.theta = theta;
        A.theta_all = all ? 1 : 0;
        const double cand = std::min(count * 1.05 + 4096.0, 1e10);
        const uint64_t node_cap = uint64_t(1) + 4 * uint64_t(cand);
        if (node_cap > (uint64_t(1) << 31)) return fail(RMAT_ERR_UNSUPPORTED, "table too large for the GPU build");
        int bits = 1;
        while ((uint64_t(1) << bits) < 1 + 3 * A.T) ++bits;
        const uint64_t nmax = uint64_t(1) << bits;
        A.node_cap = node_cap;
        A.nmax = nmax;
        Carver cv;
        carve(A, cv, node_cap, nmax);  // sizes only
        const size_t span_lo = reinterpret_cast<size_t>(A.sym), span_hi = reinterpret_cast<size_t>(A.st + 1);
        const size_t image_words_max = kHeaderWords + 9 * nmax + 16;
        if (rmat_status st = grow(cache, cv.bytes, std::max(span_hi - span_lo, image_words_max * 4))) return st;
        cv.bytes = 0;
        cv.base = static_cast<unsigned char *>(cache.scratch);
        carve(A, cv, node_cap, nmax);
        if (cudaMalloc(&image, image_words_max * 4) != cudaSuccess) {
            cudaGetLastError();
            return fail(RMAT_ERR_OUT_OF_MEMORY, "device allocation for the table image failed");
        }
        A.image = static_cast<uint32_t *>(image);
        cudaError_t e = cudaMemsetAsync(A.st, 0xFF, sizeof(BuildStatus), stream);
        void *params[] = {&A};
        if (e == cudaSuccess)
            e = cudaLaunchKernel(reinterpret_cast<void *>(&k_build_table), dim3(1), dim3(kThreads), params, 0, stream);
        const size_t span = reinterpret_cast<size_t>(A.st + 1) - reinterpret_cast<size_t>(A.sym);
        if (e == cudaSuccess) e = cudaMemcpyAsync(cache.pinned, A.sym, span, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) {
            release();
            return fail(RMAT_ERR_CUDA, std::string("table build kernel: ") + cudaGetErrorString(e));
        }
        auto host_of = [&](const void *dptr) {
            return cache.pinned + (reinterpret_cast<size_t>(dptr) - reinterpret_cast<size_t>(A.sym));
        };
        BuildStatus hs;
        std::memcpy(&hs, host_of(A.st), sizeof(hs));
        if (hs.error == 2 || hs.error == 1) {  // cut too high, or scratch too small: lower the cut
            release();
            theta *= 0.5;
            count = count * 4.0 + 4096.0;
            result = RMAT_ERR_UNSUPPORTED;
            continue;
        }
        if (hs.error) {
            release();
            return fail(RMAT_ERR_INVALID_ARGUMENT, "GPU table build: quantisation or alias construction failed");
        }
        rmat_table *t = new (std::nothrow) rmat_table;
        if (!t) {
            release();
            return fail(RMAT_ERR_OUT_OF_MEMORY, "host allocation failed");
        }
        t->k = k;
        t->has_params = true;
        std::copy(P, P + 4, t->params);
        t->groups.resize(1);
        PathTable &g = t->groups[0];
        const size_t N = size_t(1) << hs.bits;
        g.entries = int(hs.entries);
        g.bits = int(hs.bits);
        g.max_len = int(hs.max_len);
        g.min_len = int(hs.min_len);
        const size_t bw = hs.format == 0 ? 1 : 4;
        const size_t words = kHeaderWords + ((N + 3) & ~size_t(3)) + 2 * ((N * bw + 3) & ~size_t(3));
        try {
            g.sym.resize(N);
            g.len.resize(N);
            g.p.resize(N);
            g.w.resize(N);
            g.thr.resize(N);
            g.alias.resize(N);
            t->image.resize(words);
        } catch (const std::bad_alloc &) {
            delete t;
            release();
            return fail(RMAT_ERR_OUT_OF_MEMORY, "host allocation failed");
        }
        std::memcpy(g.sym.data(), host_of(A.sym), N * 8);
        std::memcpy(g.len.data(), host_of(A.len), N);
        std::memcpy(g.p.data(), host_of(A.p), N * 8);
        std::memcpy(g.w.data(), host_of(A.w), N * 8);
        std::memcpy(g.thr.data(), host_of(A.thr), N * 4);
        std::memcpy(g.alias.data(), host_of(A.alias), N * 4);
        e = cudaMemcpyAsync(cache.pinned, image, words * 4, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) {
            delete t;
            release();
            return fail(RMAT_ERR_CUDA, std::string("table copy-back: ") + cudaGetErrorString(e));
        }
        std::memcpy(t->image.data(), cache.pinned, words * 4);
        t->format = hs.format == 0 ? kCompact : kWide;
        GroupDesc gd;
        gd.a_off_words = t->image[0];
        gd.bs_off_words = t->image[kMaxGroups];
        gd.ba_off_words = t->image[2 * kMaxGroups];
        gd.bits = g.bits;
        gd.len = g.max_len;
        t->gdesc.assign(1, gd);
        // the device image stays on this device as the table's copy
        DeviceCopy dc;
        dc.ptr = image;
        dc.bytes = words * 4;
        t->dev[dev] = dc;
        *out = t;
        return RMAT_OK;
    }
    release();
    return fail(result, "GPU table build: could not bracket the table's probability cut");
}
