// rmat_table.cpp -- host construction of the R-MAT path tables (arXiv
// 1905.03525, Sec. 2) and of their integer alias structures.
//
// Variable-length tables follow the table-construction fragment of Sec. 2: a
// max-priority queue of candidate entries, starting from the empty path,
// whose maximum is repeatedly replaced by its four children (probabilities
// a p, b p, c p, d p; symbols 0..3 = row/col bits 00, 01, 10, 11).  The loop
// runs while |Q| + 3 < bound, which reproduces the table sizes of Fig. 1
// (largest 1 + 3t below the bound).  Fixed-length tables enumerate all 4^l
// paths (Sec. 2, "paths of a fixed length").  Both are then quantised to u32
// weights summing to 2^32 and turned into an alias table (Walker's method,
// cited in Sec. 2) with Vose's integer construction.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <queue>

#include "rmat_internal.h"

namespace rmat {

namespace {

struct Candidate {
    double p;
    uint64_t path;  // symbols, top level in bits 63..62
    int depth;
};

// std::priority_queue pops the element that is "largest" under this order:
// higher probability first; equal probabilities pop the lexicographically
// smaller path first.  Live candidates are leaves of one expansion tree and
// never prefixes of each other, so comparing the left-aligned words is the
// lexicographic comparison.
struct PopOrder {
    bool operator()(const Candidate &x, const Candidate &y) const {
        if (x.p != y.p) return x.p < y.p;
        return x.path > y.path;
    }
};

int bits_for(size_t entries) {
    int b = 1;
    while ((size_t(1) << b) < entries) ++b;
    return b;
}

// Quantisation to weights with sum 2^32 and Vose's alias construction on
// integers; fills w, thr, alias of a table whose p/len/sym are set.
rmat_status quantise_alias(PathTable &t) {
    const size_t N = size_t(1) << t.bits;
    const uint64_t C = uint64_t(1) << (32 - t.bits);
    const uint64_t two32 = uint64_t(1) << 32;

    t.w.assign(N, 0);
    std::vector<double> frac(N);
    uint64_t total = 0;
    for (size_t i = 0; i < N; ++i) {
        const double scaled = std::ldexp(t.p[i], 32);  // exact
        const double whole = std::floor(scaled);
        t.w[i] = uint64_t(whole);
        frac[i] = scaled - whole;                      // exact
        total += t.w[i];
    }
    if (total > two32 || two32 - total > N)
        return fail(RMAT_ERR_INVALID_ARGUMENT, "path probabilities do not sum to 1");
    const uint64_t missing = two32 - total;
    if (missing) {
        std::vector<uint32_t> order(N);
        std::iota(order.begin(), order.end(), 0u);
        // largest fractional part first, lower index first among equals
        std::stable_sort(order.begin(), order.end(),
                         [&](uint32_t x, uint32_t y) { return frac[x] > frac[y]; });
        for (uint64_t i = 0; i < missing; ++i) t.w[order[i]] += 1;
    }

    t.thr.assign(N, 0);
    t.alias.assign(N, 0);
    std::vector<uint64_t> left(t.w);
    std::vector<uint32_t> small_q, large_q;
    small_q.reserve(N);
    large_q.reserve(N);
    for (size_t i = 0; i < N; ++i) (left[i] < C ? small_q : large_q).push_back(uint32_t(i));
    size_t si = 0, li = 0;
    while (si < small_q.size() && li < large_q.size()) {
        const uint32_t s = small_q[si++];
        const uint32_t l = large_q[li];
        t.thr[s] = uint32_t(left[s]);
        t.alias[s] = l;
        left[l] = left[l] + left[s] - C;
        if (left[l] < C) {
            ++li;
            small_q.push_back(l);
        }
    }
    if (si != small_q.size()) return fail(RMAT_ERR_INVALID_ARGUMENT, "alias construction left a deficit");
    for (; li < large_q.size(); ++li) {
        const uint32_t l = large_q[li];
        t.thr[l] = uint32_t(C - 1);
        t.alias[l] = l;
    }
    t.min_len = 64;
    for (size_t i = 0; i < N; ++i)
        if (t.w[i] > 0) t.min_len = std::min<int>(t.min_len, t.len[i]);
    return RMAT_OK;
}

}  // namespace

rmat_status normalise_params(const double in[4], double out[4]) {
    for (int i = 0; i < 4; ++i)
        if (!std::isfinite(in[i]) || in[i] < 0.0)
            return fail(RMAT_ERR_INVALID_ARGUMENT, "a, b, c, d must be finite and non-negative");
    const double s = ((in[0] + in[1]) + in[2]) + in[3];
    if (!(std::fabs(s - 1.0) <= 1e-9))
        return fail(RMAT_ERR_INVALID_ARGUMENT, "a + b + c + d must equal 1 (within 1e-9)");
    for (int i = 0; i < 4; ++i) out[i] = in[i] / s;
    return RMAT_OK;
}

rmat_status build_variable(const double P[4], int k, uint64_t bound, PathTable &t) {
    const int cap = std::min(k, 32);
    std::priority_queue<Candidate, std::vector<Candidate>, PopOrder> q;
    std::vector<Candidate> final_entries;
    q.push({1.0, 0, 0});
    while (!q.empty() && q.size() + final_entries.size() + 3 < bound) {
        const Candidate top = q.top();
        q.pop();
        const int shift = 62 - 2 * top.depth;
        for (uint64_t s = 0; s < 4; ++s) {
            Candidate ch{top.p * P[s], top.path | (s << shift), top.depth + 1};
            if (ch.depth >= cap)
                final_entries.push_back(ch);
            else
                q.push(ch);
        }
    }
    while (!q.empty()) {
        final_entries.push_back(q.top());
        q.pop();
    }
    std::sort(final_entries.begin(), final_entries.end(),
              [](const Candidate &x, const Candidate &y) { return x.path < y.path; });

    t.entries = int(final_entries.size());
    t.bits = bits_for(final_entries.size());
    const size_t N = size_t(1) << t.bits;
    t.sym.assign(N, 0);
    t.len.assign(N, 0);
    t.p.assign(N, 0.0);
    t.max_len = 0;
    for (size_t i = 0; i < final_entries.size(); ++i) {
        t.sym[i] = final_entries[i].path;
        t.len[i] = uint8_t(final_entries[i].depth);
        t.p[i] = final_entries[i].p;
        t.max_len = std::max(t.max_len, final_entries[i].depth);
    }
    return quantise_alias(t);
}

int kron_depth_cap(int n0) {
    int L = 0;
    double v = 1.0;
    while (v * n0 <= 4294967296.0) {
        v *= n0;
        ++L;
    }
    return L;
}

int kron_max_k(int n0) {
    int k = 0;
    double v = 1.0;
    while (v * n0 <= 18446744073709551616.0) {
        v *= n0;
        ++k;
    }
    return k;
}

bool wide_ids(const rmat_table *t) {
    if (t->n0 == 2) return t->k > 32;
    double v = 1.0;
    for (int i = 0; i < t->k; ++i) v *= t->n0;
    return v > 4294967296.0;
}

namespace {

// Place value of the symbol at `level` in a left-aligned key of
// kron_depth_cap(n0) base-S digits (S = n0^2): S^(D - 1 - level).  S^D =
// n0^(2D) <= 2^64, so every key fits 64 bits; for n0 = 2 this is the R-MAT
// layout (2 bits per level, top level in bits 63..62).
std::vector<uint64_t> kron_places(int n0) {
    const int D = kron_depth_cap(n0);
    const uint64_t S = uint64_t(n0) * uint64_t(n0);
    std::vector<uint64_t> place(D);
    uint64_t v = 1;
    for (int lvl = D - 1; lvl >= 0; --lvl) {
        place[lvl] = v;
        if (lvl) v *= S;
    }
    return place;
}

}  // namespace

uint32_t kron_symbol(uint64_t key, int n0, int level) {
    const uint64_t S = uint64_t(n0) * uint64_t(n0);
    return uint32_t((key / kron_places(n0)[level]) % S);
}

rmat_status normalise_theta(const double *in, int n0, std::vector<double> &out) {
    const int S = n0 * n0;
    double s = 0.0;
    for (int i = 0; i < S; ++i) {
        if (!std::isfinite(in[i]) || in[i] < 0.0)
            return fail(RMAT_ERR_INVALID_ARGUMENT, "initiator entries must be finite and non-negative");
        s = s + in[i];
    }
    if (!(std::fabs(s - 1.0) <= 1e-9)) return fail(RMAT_ERR_INVALID_ARGUMENT, "initiator must sum to 1 (within 1e-9)");
    out.resize(S);
    for (int i = 0; i < S; ++i) out[i] = in[i] / s;
    return RMAT_OK;
}

// Kronecker generalisation of build_variable (Sec. 3: an n0 x n0 initiator):
// an expansion adds the n0^2 children, the loop runs while |Q| + n0^2 - 1 <
// bound, and paths stop at min(k, kron_depth_cap(n0)) levels.
rmat_status build_kron_variable(const double *P, int n0, int k, uint64_t bound, PathTable &t) {
    const int S = n0 * n0;
    const int cap = std::min(k, kron_depth_cap(n0));
    const std::vector<uint64_t> place = kron_places(n0);
    std::priority_queue<Candidate, std::vector<Candidate>, PopOrder> q;
    std::vector<Candidate> final_entries;
    q.push({1.0, 0, 0});
    while (!q.empty() && q.size() + final_entries.size() + uint64_t(S - 1) < bound) {
        const Candidate top = q.top();
        q.pop();
        for (int s = 0; s < S; ++s) {
            Candidate ch{top.p * P[s], top.path + uint64_t(s) * place[top.depth], top.depth + 1};
            if (ch.depth >= cap)
                final_entries.push_back(ch);
            else
                q.push(ch);
        }
    }
    while (!q.empty()) {
        final_entries.push_back(q.top());
        q.pop();
    }
    std::sort(final_entries.begin(), final_entries.end(),
              [](const Candidate &x, const Candidate &y) { return x.path < y.path; });
    t.n0 = n0;
    t.entries = int(final_entries.size());
    t.bits = bits_for(final_entries.size());
    const size_t N = size_t(1) << t.bits;
    t.sym.assign(N, 0);
    t.len.assign(N, 0);
    t.p.assign(N, 0.0);
    t.max_len = 0;
    for (size_t i = 0; i < final_entries.size(); ++i) {
        t.sym[i] = final_entries[i].path;
        t.len[i] = uint8_t(final_entries[i].depth);
        t.p[i] = final_entries[i].p;
        t.max_len = std::max(t.max_len, final_entries[i].depth);
    }
    return quantise_alias(t);
}

// All (n0^2)^ell paths; entry i has the base-n0^2 digits of i as symbols.
rmat_status build_kron_fixed(const double *P, int n0, int ell, PathTable &t) {
    const size_t S = size_t(n0) * size_t(n0);
    const std::vector<uint64_t> place = kron_places(n0);
    std::vector<double> prob(1, 1.0), next;
    std::vector<uint64_t> path(1, 0), next_path;
    for (int lvl = 0; lvl < ell; ++lvl) {
        next.resize(prob.size() * S);
        next_path.resize(prob.size() * S);
        for (size_t i = 0; i < prob.size(); ++i)
            for (size_t s = 0; s < S; ++s) {
                next[S * i + s] = prob[i] * P[s];
                next_path[S * i + s] = path[i] + uint64_t(s) * place[lvl];
            }
        prob.swap(next);
        path.swap(next_path);
    }
    t.n0 = n0;
    t.entries = int(prob.size());
    t.bits = bits_for(prob.size());
    const size_t N = size_t(1) << t.bits;
    t.max_len = ell;
    t.sym.assign(N, 0);
    t.len.assign(N, 0);
    t.p.assign(N, 0.0);
    for (size_t i = 0; i < prob.size(); ++i) {
        t.p[i] = prob[i];
        t.sym[i] = path[i];
        t.len[i] = uint8_t(ell);
    }
    return quantise_alias(t);
}

rmat_status build_fixed(const double *P, int ell, PathTable &t) {
    const size_t N = size_t(1) << (2 * ell);
    t.entries = int(N);
    t.bits = 2 * ell;
    t.max_len = ell;
    t.sym.assign(N, 0);
    t.len.assign(N, uint8_t(ell));
    t.p.assign(N, 0.0);
    // Breadth-first product: level-t probabilities of all prefixes, each
    // prefix extended by its four children in digit order, so that entry i
    // has the base-4 digits of i as its symbols and p = ((P0 * P1) * ...).
    std::vector<double> prob(1, 1.0), next;
    std::vector<uint64_t> path(1, 0), next_path;
    for (int lvl = 0; lvl < ell; ++lvl) {
        next.resize(prob.size() * 4);
        next_path.resize(prob.size() * 4);
        for (size_t i = 0; i < prob.size(); ++i)
            for (uint64_t s = 0; s < 4; ++s) {
                next[4 * i + s] = prob[i] * P[4 * lvl + s];
                next_path[4 * i + s] = path[i] | (s << (62 - 2 * lvl));
            }
        prob.swap(next);
        path.swap(next_path);
    }
    for (size_t i = 0; i < N; ++i) {
        t.p[i] = prob[i];
        t.sym[i] = path[i];
    }
    return quantise_alias(t);
}

}  // namespace rmat
