// rmat_image.cpp -- packing of the alias tables into the device image that the
// sampling kernels stage into shared memory.
//
// Per table (group) of N = 2^b columns the image holds two arrays:
//   A[j]  u32  (thr[j] << b) | alias[j]      -- one word decides a draw:
//              with the word u = (j << (32-b)) | r, the draw keeps column j iff
//              r < thr[j]  <=>  ((u << b) | (2^b - 1)) < A[j].
//   B[i]       the path of entry i, ready to be OR-ed into left-aligned
//              row/column accumulators:
//     compact (paths <= 13 levels), u32:
//              bits 31..19 row bits, left-aligned in the 13-bit field
//              bits 18..13 path length L
//              bits 12..0  column bits, left-aligned in the 13-bit field
//     wide (paths <= 32 levels), uint4:
//              {row bits << (32-L), column bits << (32-L), L, 0}
// Two 4-byte shared-memory loads per draw (A[j], then B[sel]) is the least
// shared-memory traffic for a random column: each costs one bank access per
// lane.  The blob starts with a header of kHeaderWords words -- word g, 64+g
// and 128+g hold the A offset, B offset and b of group g (offsets in words
// from the blob start) -- followed by the groups back to back, each array
// 16-byte aligned, so that one bulk copy stages descriptors and tables.
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

rmat_status build_image(rmat_table *t) {
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
        d.b_off_words = uint32_t(total);
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
        t->image[kMaxGroups + gi] = d.b_off_words;
        t->image[2 * kMaxGroups + gi] = uint32_t(g.bits);
        const size_t N = size_t(1) << g.bits;
        uint32_t *A = t->image.data() + d.a_off_words;
        uint32_t *B = t->image.data() + d.b_off_words;
        for (size_t j = 0; j < N; ++j) A[j] = (g.thr[j] << g.bits) | g.alias[j];
        for (size_t i = 0; i < N; ++i) {
            const int L = g.len[i];
            uint32_t r, c;
            path_bits(g.sym[i], L, r, c);
            if (t->format == kCompact) {
                const uint32_t r13 = L ? r << (13 - L) : 0u;
                const uint32_t c13 = L ? c << (13 - L) : 0u;
                B[i] = (r13 << 19) | (uint32_t(L) << 13) | c13;
            } else {
                B[4 * i + 0] = L ? r << (32 - L) : 0u;
                B[4 * i + 1] = L ? c << (32 - L) : 0u;
                B[4 * i + 2] = uint32_t(L);
                B[4 * i + 3] = 0u;
            }
        }
    }
    return RMAT_OK;
}

}  // namespace rmat
