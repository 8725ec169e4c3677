// rmat_image.cpp -- packing of the alias tables into the device image that the
// sampling kernels stage into shared memory.
//
// Per table (group) of N = 2^b columns the image holds three arrays:
//   A[j]   u32  (j << (32-b)) + thr[j]: the draw with 32-bit word u keeps
//               column j = u >> (32-b) iff u < A[j]  (<=> residual < thr[j]);
//   Bs[j]       the path of entry j          (taken when u < A[j]);
//   Ba[j]       the path of entry alias[j]   (taken otherwise).
// Holding the alias's path beside the column makes a draw two independent-of-
// content loads: A[j], then Bs[j] or Ba[j] -- the same shared-memory traffic
// as looking up alias[j] and then its path, with fewer instructions (no alias
// index to extract, no second address from loaded data).
// Path entries, ready to be OR-ed into left-aligned row/column accumulators:
//     compact (paths <= 13 levels), u32:
//              bits 31..19 row bits, left-aligned in the 13-bit field
//              bits 18..13 path length L
//              bits 12..0  column bits, left-aligned in the 13-bit field
//     wide (paths <= 32 levels), uint4:
//              {row bits << (32-L), column bits << (32-L), L, 0}
// Two 4-byte random shared-memory loads per draw is the least traffic for a
// random column: each costs one bank access per lane.  The blob starts with a
// header of kHeaderWords words -- words g, 64+g, 128+g and 192+g hold the A,
// Bs and Ba offsets (in words from the blob start) and b of group g -- followed
// by the groups back to back, each array 16-byte aligned, so that one bulk
// copy stages descriptors and tables.
#include <algorithm>

#include "rmat_internal.h"

namespace rmat {

namespace {

void path_bits(uint64_t sym, int len, uint32_t &row, uint32_t &col) {
    row = col = 0;
    for (int t = 0; t < len; ++t) {
        const uint32_t s = uint32_t(sym >> (62 - 2 * t)) & 3u;
        row = (row << 1) | (s >> 1);
        col = (col << 1) | (s & 1u);
    }
}

size_t round16w(size_t words) { return (words + 3) & ~size_t(3); }

}  // namespace

// Kronecker tables (n0 > 2, one group): after the header,
//   AA[j] uint2 {A[j], alias[j]}   (A as above)
//   P[j]  uint4 {row digits, column digits, L, n0^L - 1}
// where the digits of the path's L levels are read as base-n0 numbers (both
// < n0^L <= 2^32); the kernel appends a path as x = x * n0^L + digits, i.e.
// x * (n0^L - 1) + x + digits, which keeps n0^L = 2^32 within 32 bits.
// When the IDs fit 32 bits and the longest path's digits fit S bits with
// 2S + 4 <= 32 (kron_packed_shift), packed arrays follow for the contract-case
// kernel:
//   A32[j] = (thr[j] << b) | alias[j]       (as in the compact R-MAT image)
//   P32[j] = r | c << S | L << 2S           (row digits, column digits, L)
//   PW[L]  = n0^L, L < 16
//   MD[d]  = ceil(2^32 / n0^d), 1 <= d < 16: floor(x / n0^d) = umulhi(x, MD[d])
//            for the digits x of a path of L >= d levels (x * n0^d < n0^2L <= 2^28)
// Header word g is the AA offset, 64 + g the P offset, 128 the packed
// arrays' offset (0 if absent), 192 + g = b.
int kron_packed_shift(const rmat_table *t) {
    const PathTable &g = t->groups[0];
    if (wide_ids(t) || g.max_len > 15) return 0;
    uint64_t v = 1;
    for (int l = 0; l < g.max_len; ++l) v *= uint64_t(t->n0);
    int S = 1;
    while ((uint64_t(1) << S) < v) ++S;  // digits < n0^max_len <= 2^S
    return 2 * S + 4 <= 32 ? S : 0;
}

rmat_status build_kron_image(rmat_table *t) {
    const PathTable &g = t->groups[0];
    const size_t N = size_t(1) << g.bits;
    GroupDesc d;
    d.a_off_words = uint32_t(kHeaderWords);
    d.bs_off_words = uint32_t(kHeaderWords + round16w(2 * N));
    d.ba_off_words = 0;
    d.bits = g.bits;
    d.len = g.max_len;
    const int S = kron_packed_shift(t);
    const size_t packed = round16w(d.bs_off_words + 4 * N);
    d.ba_off_words = S ? uint32_t(packed) : 0u;
    t->format = kKron;
    t->gdesc.assign(1, d);
    t->image.assign(S ? packed + round16w(N) * 2 + 32 : packed, 0u);
    t->image[0] = d.a_off_words;
    t->image[kMaxGroups] = d.bs_off_words;
    t->image[2 * kMaxGroups] = d.ba_off_words;
    t->image[3 * kMaxGroups] = uint32_t(g.bits);
    const uint32_t C = uint32_t((uint64_t(1) << 32) >> g.bits);
    const uint64_t n0 = uint64_t(t->n0);
    uint32_t *AA = t->image.data() + d.a_off_words;
    uint32_t *P = t->image.data() + d.bs_off_words;
    for (size_t j = 0; j < N; ++j) {
        AA[2 * j] = uint32_t(j) * C + g.thr[j];
        AA[2 * j + 1] = g.alias[j];
        const int L = g.len[j];
        uint64_t r = 0, c = 0, pw = 1;
        for (int lvl = 0; lvl < L; ++lvl) {
            const uint32_t s = kron_symbol(g.sym[j], t->n0, lvl);
            r = r * n0 + s / n0;
            c = c * n0 + s % n0;
            pw *= n0;
        }
        P[4 * j + 0] = uint32_t(r);
        P[4 * j + 1] = uint32_t(c);
        P[4 * j + 2] = uint32_t(L);
        P[4 * j + 3] = uint32_t(pw - 1);
        if (S) {
            uint32_t *A32 = t->image.data() + d.ba_off_words;
            uint32_t *P32 = A32 + round16w(N);
            A32[j] = (g.thr[j] << g.bits) | g.alias[j];
            P32[j] = uint32_t(r) | (uint32_t(c) << S) | (uint32_t(L) << (2 * S));
        }
    }
    if (S) {
        uint32_t *PW = t->image.data() + d.ba_off_words + 2 * round16w(N);
        uint32_t *MD = PW + 16;
        uint64_t v = 1;
        for (int l = 0; l < 16; ++l, v *= n0) {
            PW[l] = l <= g.max_len ? uint32_t(v) : 0u;
            MD[l] = (l >= 1 && l <= g.max_len) ? uint32_t(((uint64_t(1) << 32) + v - 1) / v) : 0u;
        }
    }
    return RMAT_OK;
}

rmat_status build_image(rmat_table *t) {
    if (t->n0 > 2) return build_kron_image(t);
    int max_len = 0;
    for (const PathTable &g : t->groups) max_len = std::max(max_len, g.max_len);
    if (max_len > 32) return fail(RMAT_ERR_UNSUPPORTED, "paths longer than 32 levels");
    t->format = max_len <= 13 ? kCompact : kWide;
    const size_t bwords = t->format == kCompact ? 1 : 4;

    size_t total = kHeaderWords;
    t->gdesc.clear();
    for (const PathTable &g : t->groups) {
        const size_t N = size_t(1) << g.bits;
        GroupDesc d;
        d.a_off_words = uint32_t(total);
        total += round16w(N);
        d.bs_off_words = uint32_t(total);
        total += round16w(N * bwords);
        d.ba_off_words = uint32_t(total);
        total += round16w(N * bwords);
        d.bits = g.bits;
        d.len = g.max_len;
        t->gdesc.push_back(d);
    }
    t->image.assign(total, 0u);
    for (size_t gi = 0; gi < t->groups.size(); ++gi) {
        const PathTable &g = t->groups[gi];
        const GroupDesc &d = t->gdesc[gi];
        t->image[gi] = d.a_off_words;
        t->image[kMaxGroups + gi] = d.bs_off_words;
        t->image[2 * kMaxGroups + gi] = d.ba_off_words;
        t->image[3 * kMaxGroups + gi] = uint32_t(g.bits);
        const size_t N = size_t(1) << g.bits;
        const uint32_t C = uint32_t((uint64_t(1) << 32) >> g.bits);
        uint32_t *A = t->image.data() + d.a_off_words;
        uint32_t *Bs = t->image.data() + d.bs_off_words;
        uint32_t *Ba = t->image.data() + d.ba_off_words;
        auto put_path = [&](uint32_t *B, size_t slot, size_t i) {
            const int L = g.len[i];
            uint32_t r, c;
            path_bits(g.sym[i], L, r, c);
            if (t->format == kCompact) {
                const uint32_t r13 = L ? r << (13 - L) : 0u;
                const uint32_t c13 = L ? c << (13 - L) : 0u;
                B[slot] = (r13 << 19) | (uint32_t(L) << 13) | c13;
            } else {
                B[4 * slot + 0] = L ? r << (32 - L) : 0u;
                B[4 * slot + 1] = L ? c << (32 - L) : 0u;
                B[4 * slot + 2] = uint32_t(L);
                B[4 * slot + 3] = 0u;
            }
        };
        for (size_t j = 0; j < N; ++j) {
            A[j] = uint32_t(j) * C + g.thr[j];  // thr < C, so no overflow
            put_path(Bs, j, j);
            put_path(Ba, j, g.alias[j]);
        }
    }
    return RMAT_OK;
}

}  // namespace rmat
