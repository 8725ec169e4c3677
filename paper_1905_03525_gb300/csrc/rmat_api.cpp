// rmat_api.cpp -- the C ABI of librmat (declared in include/rmat.h): argument
// checking, table construction entry points, device copies of table images,
// and the single-graph generation calls.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "rmat_internal.h"
#include "rmat_kernels.h"

namespace rmat {

namespace {
thread_local std::string t_error;

rmat_status cuda_fail(const char *what, cudaError_t e) {
    return fail(RMAT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

rmat_status check_k(int k) {
    if (k < 1 || k > 64) return fail(RMAT_ERR_INVALID_ARGUMENT, "k must be in [1, 64]");
    return RMAT_OK;
}

rmat_status finish_table(rmat_table *t, rmat_table **out) {
    if (rmat_status st = build_image(t)) {
        delete t;
        return st;
    }
    *out = t;
    return RMAT_OK;
}

// Per-device staging area of rmat_generate_host.
struct HostStaging {
    void *buf[2] = {nullptr, nullptr};
    size_t bytes = 0;
    cudaStream_t copy = nullptr;
    cudaEvent_t produced[2] = {nullptr, nullptr};
    cudaEvent_t drained[2] = {nullptr, nullptr};
};
std::mutex g_staging_mu;
std::map<int, HostStaging> g_staging;
constexpr size_t kStagingBytes = size_t(256) << 20;

rmat_status get_staging(HostStaging *&out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail("cudaGetDevice", e);
    std::lock_guard<std::mutex> lk(g_staging_mu);
    HostStaging &s = g_staging[dev];
    if (!s.buf[0]) {
        for (int i = 0; i < 2; ++i) {
            e = cudaMalloc(&s.buf[i], kStagingBytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(RMAT_ERR_OUT_OF_MEMORY, "staging buffer allocation failed");
            }
            if ((e = cudaEventCreateWithFlags(&s.produced[i], cudaEventDisableTiming)) != cudaSuccess)
                return cuda_fail("cudaEventCreate", e);
            if ((e = cudaEventCreateWithFlags(&s.drained[i], cudaEventDisableTiming)) != cudaSuccess)
                return cuda_fail("cudaEventCreate", e);
        }
        if ((e = cudaStreamCreateWithFlags(&s.copy, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail("cudaStreamCreate", e);
        s.bytes = kStagingBytes;
    }
    out = &s;
    return RMAT_OK;
}

rmat_status check_generate_args(const rmat_table *t, uint64_t edge_offset, uint64_t count, const void *out) {
    if (!t) return fail(RMAT_ERR_INVALID_ARGUMENT, "table is NULL");
    if (count && !out) return fail(RMAT_ERR_INVALID_ARGUMENT, "output pointer is NULL");
    if (reinterpret_cast<uintptr_t>(out) & 7u) return fail(RMAT_ERR_INVALID_ARGUMENT, "output must be 8-byte aligned");
    if (count > RMAT_MAX_EDGES) return fail(RMAT_ERR_INVALID_ARGUMENT, "count above RMAT_MAX_EDGES");
    if (count > ~uint64_t(0) - edge_offset)
        return fail(RMAT_ERR_INVALID_ARGUMENT, "edge_offset + count overflows 64 bits");
    return RMAT_OK;
}

rmat_status get_plan(const rmat_table *tc, AliasPlan &plan) {
    rmat_table *t = const_cast<rmat_table *>(tc);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail("cudaGetDevice", e);
    {
        std::lock_guard<std::mutex> lk(t->mu);
        auto it = t->plans.find(dev);
        if (it != t->plans.end()) {
            plan = it->second;
            return RMAT_OK;
        }
    }
    rmat_launch_config_t cfg = t->cfg_set ? t->cfg : default_launch_config(t);
    if (rmat_status st = plan_alias_launch(t, cfg, plan)) return st;
    std::lock_guard<std::mutex> lk(t->mu);
    t->plans[dev] = plan;
    return RMAT_OK;
}

}  // namespace

rmat_status fail(rmat_status st, const std::string &msg) {
    t_error = msg;
    return st;
}

rmat_status plan_and_image(const rmat_table *t, AliasPlan &plan, const uint32_t **img) {
    if (rmat_status st = get_plan(t, plan)) return st;
    return ensure_device_copy(t, img);
}

void clear_error() { t_error.clear(); }

rmat_status ensure_device_copy(const rmat_table *tc, const uint32_t **dptr) {
    rmat_table *t = const_cast<rmat_table *>(tc);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail("cudaGetDevice", e);
    std::lock_guard<std::mutex> lk(t->mu);
    DeviceCopy &dc = t->dev[dev];
    if (!dc.ptr) {
        const size_t bytes = t->image.size() * 4;
        void *p = nullptr;
        e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(RMAT_ERR_OUT_OF_MEMORY, "table image allocation failed");
        }
        e = cudaMemcpy(p, t->image.data(), bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(p);
            return cuda_fail("table upload", e);
        }
        dc.ptr = p;
        dc.bytes = bytes;
    }
    *dptr = static_cast<const uint32_t *>(dc.ptr);
    return RMAT_OK;
}

}  // namespace rmat

using namespace rmat;

extern "C" {

const char *rmat_last_error(void) { return t_error.c_str(); }

const char *rmat_version(void) { return "librmat 0.1 (sm_103a)"; }

rmat_status rmat_build_table(double a, double b, double c, double d, int k, uint64_t table_bound,
                             rmat_table **out) {
    clear_error();
    if (!out) return fail(RMAT_ERR_INVALID_ARGUMENT, "out is NULL");
    *out = nullptr;
    if (rmat_status st = check_k(k)) return st;
    if (table_bound < 5 || table_bound > (uint64_t(1) << 24))
        return fail(RMAT_ERR_INVALID_ARGUMENT, "table_bound must be in [5, 2^24]");
    const double in[4] = {a, b, c, d};
    double P[4];
    if (rmat_status st = normalise_params(in, P)) return st;
    rmat_table *t = new (std::nothrow) rmat_table;
    if (!t) return fail(RMAT_ERR_OUT_OF_MEMORY, "host allocation failed");
    t->k = k;
    t->has_params = true;
    std::copy(P, P + 4, t->params);
    t->groups.resize(1);
    try {
        if (rmat_status st = build_variable(P, k, table_bound, t->groups[0])) {
            delete t;
            return st;
        }
    } catch (const std::bad_alloc &) {
        delete t;
        return fail(RMAT_ERR_OUT_OF_MEMORY, "host allocation failed");
    }
    return finish_table(t, out);
}

rmat_status rmat_build_table_fixed(double a, double b, double c, double d, int k, int ell, rmat_table **out) {
    clear_error();
    if (!out) return fail(RMAT_ERR_INVALID_ARGUMENT, "out is NULL");
    *out = nullptr;
    if (rmat_status st = check_k(k)) return st;
    if (ell < 1 || ell > 12) return fail(RMAT_ERR_INVALID_ARGUMENT, "ell must be in [1, 12]");
    const double in[4] = {a, b, c, d};
    double P[4];
    if (rmat_status st = normalise_params(in, P)) return st;
    std::vector<double> levels(size_t(4) * ell);
    for (int t = 0; t < ell; ++t) std::copy(P, P + 4, levels.begin() + 4 * t);
    rmat_table *t = new (std::nothrow) rmat_table;
    if (!t) return fail(RMAT_ERR_OUT_OF_MEMORY, "host allocation failed");
    t->k = k;
    t->has_params = true;
    std::copy(P, P + 4, t->params);
    t->groups.resize(1);
    try {
        if (rmat_status st = build_fixed(levels.data(), ell, t->groups[0])) {
            delete t;
            return st;
        }
    } catch (const std::bad_alloc &) {
        delete t;
        return fail(RMAT_ERR_OUT_OF_MEMORY, "host allocation failed");
    }
    return finish_table(t, out);
}

rmat_status rmat_build_table_kron(const double *theta, int n0, int k, uint64_t table_bound, rmat_table **out) {
    clear_error();
    if (!out) return fail(RMAT_ERR_INVALID_ARGUMENT, "out is NULL");
    *out = nullptr;
    if (!theta) return fail(RMAT_ERR_INVALID_ARGUMENT, "theta is NULL");
    if (n0 < 2 || n0 > 16) return fail(RMAT_ERR_INVALID_ARGUMENT, "n0 must be in [2, 16]");
    if (n0 == 2) return rmat_build_table(theta[0], theta[1], theta[2], theta[3], k, table_bound, out);
    if (k < 1 || k > kron_max_k(n0)) return fail(RMAT_ERR_INVALID_ARGUMENT, "k must satisfy 1 <= k and n0^k <= 2^64");
    if (table_bound < uint64_t(n0) * n0 + 1 || table_bound > (uint64_t(1) << 24))
        return fail(RMAT_ERR_INVALID_ARGUMENT, "table_bound must be in [n0^2 + 1, 2^24]");
    std::vector<double> P;
    if (rmat_status st = normalise_theta(theta, n0, P)) return st;
    rmat_table *t = new (std::nothrow) rmat_table;
    if (!t) return fail(RMAT_ERR_OUT_OF_MEMORY, "host allocation failed");
    t->k = k;
    t->n0 = n0;
    t->groups.resize(1);
    try {
        if (rmat_status st = build_kron_variable(P.data(), n0, k, table_bound, t->groups[0])) {
            delete t;
            return st;
        }
    } catch (const std::bad_alloc &) {
        delete t;
        return fail(RMAT_ERR_OUT_OF_MEMORY, "host allocation failed");
    }
    return finish_table(t, out);
}

rmat_status rmat_build_table_kron_fixed(const double *theta, int n0, int k, int ell, rmat_table **out) {
    clear_error();
    if (!out) return fail(RMAT_ERR_INVALID_ARGUMENT, "out is NULL");
    *out = nullptr;
    if (!theta) return fail(RMAT_ERR_INVALID_ARGUMENT, "theta is NULL");
    if (n0 < 2 || n0 > 16) return fail(RMAT_ERR_INVALID_ARGUMENT, "n0 must be in [2, 16]");
    if (n0 == 2) return rmat_build_table_fixed(theta[0], theta[1], theta[2], theta[3], k, ell, out);
    if (k < 1 || k > kron_max_k(n0)) return fail(RMAT_ERR_INVALID_ARGUMENT, "k must satisfy 1 <= k and n0^k <= 2^64");
    double entries = 1.0;
    for (int i = 0; i < ell; ++i) entries *= double(n0) * n0;
    if (ell < 1 || ell > kron_depth_cap(n0) || entries > double(1 << 24))
        return fail(RMAT_ERR_INVALID_ARGUMENT, "ell must be >= 1 with (n0^2)^ell <= 2^24");
    std::vector<double> P;
    if (rmat_status st = normalise_theta(theta, n0, P)) return st;
    rmat_table *t = new (std::nothrow) rmat_table;
    if (!t) return fail(RMAT_ERR_OUT_OF_MEMORY, "host allocation failed");
    t->k = k;
    t->n0 = n0;
    t->groups.resize(1);
    try {
        if (rmat_status st = build_kron_fixed(P.data(), n0, ell, t->groups[0])) {
            delete t;
            return st;
        }
    } catch (const std::bad_alloc &) {
        delete t;
        return fail(RMAT_ERR_OUT_OF_MEMORY, "host allocation failed");
    }
    return finish_table(t, out);
}

rmat_status rmat_build_table_levels(const double *abcd, int k, int ell, unsigned flags, rmat_table **out) {
    clear_error();
    if (!out) return fail(RMAT_ERR_INVALID_ARGUMENT, "out is NULL");
    *out = nullptr;
    if (!abcd) return fail(RMAT_ERR_INVALID_ARGUMENT, "abcd is NULL");
    if (rmat_status st = check_k(k)) return st;
    if (ell < 1 || ell > 12) return fail(RMAT_ERR_INVALID_ARGUMENT, "ell must be in [1, 12]");
    if ((k + ell - 1) / ell > 64) return fail(RMAT_ERR_INVALID_ARGUMENT, "more than 64 level groups");
    if (flags & ~RMAT_UNDIRECTED) return fail(RMAT_ERR_INVALID_ARGUMENT, "unknown flag");
    std::vector<double> P(size_t(4) * k);
    for (int t = 0; t < k; ++t)
        if (rmat_status st = normalise_params(abcd + 4 * t, P.data() + 4 * t)) return st;
    rmat_table *t = new (std::nothrow) rmat_table;
    if (!t) return fail(RMAT_ERR_OUT_OF_MEMORY, "host allocation failed");
    t->k = k;
    t->flags = flags;
    t->per_level = true;
    try {
        for (int g0 = 0; g0 < k; g0 += ell) {
            const int n = std::min(ell, k - g0);
            t->groups.emplace_back();
            if (rmat_status st = build_fixed(P.data() + 4 * g0, n, t->groups.back())) {
                delete t;
                return st;
            }
        }
    } catch (const std::bad_alloc &) {
        delete t;
        return fail(RMAT_ERR_OUT_OF_MEMORY, "host allocation failed");
    }
    return finish_table(t, out);
}

rmat_status rmat_table_set_flags(rmat_table *t, unsigned flags) {
    clear_error();
    if (!t) return fail(RMAT_ERR_INVALID_ARGUMENT, "table is NULL");
    if (flags & ~RMAT_UNDIRECTED) return fail(RMAT_ERR_INVALID_ARGUMENT, "unknown flag");
    if (flags && t->n0 > 2) return fail(RMAT_ERR_UNSUPPORTED, "Kronecker tables (n0 > 2) take no flags");
    t->flags = flags;
    return RMAT_OK;
}

rmat_status rmat_table_set_scramble(rmat_table *t, int enable, uint64_t scramble_seed) {
    clear_error();
    if (!t) return fail(RMAT_ERR_INVALID_ARGUMENT, "table is NULL");
    if (enable && t->n0 > 2) return fail(RMAT_ERR_UNSUPPORTED, "Kronecker tables (n0 > 2) are not scrambled");
    std::lock_guard<std::mutex> lk(t->mu);
    t->scramble = enable != 0;
    if (t->scramble) {
        // SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): add the golden-ratio
        // increment, then the two xor-shift-multiply steps of its finaliser.
        uint64_t state = scramble_seed;
        const uint64_t mask = t->k >= 64 ? ~uint64_t(0) : ((uint64_t(1) << t->k) - 1);
        for (int i = 0; i < 6; ++i) {
            state += 0x9E3779B97F4A7C15ull;
            uint64_t z = state;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            t->scr[i] = (i % 2 == 0 ? (z | 1u) : z) & mask;
        }
    }
    t->plans.clear();
    return RMAT_OK;
}

rmat_status rmat_table_info(const rmat_table *t, rmat_table_info_t *info) {
    clear_error();
    if (!t || !info) return fail(RMAT_ERR_INVALID_ARGUMENT, "NULL argument");
    info->k = t->k;
    info->groups = int(t->groups.size());
    info->entries = t->groups[0].entries;
    info->bits = t->groups[0].bits;
    int ml = 0;
    for (const PathTable &g : t->groups) ml = std::max(ml, g.max_len);
    info->max_len = ml;
    info->index_bytes = wide_ids(t) ? 8 : 4;
    info->n0 = t->n0;
    info->flags = t->flags;
    info->device_image_bytes = uint64_t(t->image.size()) * 4;
    return RMAT_OK;
}

rmat_status rmat_table_group_info(const rmat_table *t, int group, int *entries, int *bits, int *max_len) {
    clear_error();
    if (!t) return fail(RMAT_ERR_INVALID_ARGUMENT, "table is NULL");
    if (group < 0 || group >= int(t->groups.size())) return fail(RMAT_ERR_INVALID_ARGUMENT, "no such group");
    const PathTable &g = t->groups[group];
    if (entries) *entries = g.entries;
    if (bits) *bits = g.bits;
    if (max_len) *max_len = g.max_len;
    return RMAT_OK;
}

rmat_status rmat_table_export(const rmat_table *t, int group, uint64_t *sym, uint8_t *len, double *p, uint64_t *w,
                              uint32_t *thr, uint32_t *alias) {
    clear_error();
    if (!t) return fail(RMAT_ERR_INVALID_ARGUMENT, "table is NULL");
    if (group < 0 || group >= int(t->groups.size())) return fail(RMAT_ERR_INVALID_ARGUMENT, "no such group");
    const PathTable &g = t->groups[group];
    const size_t N = size_t(1) << g.bits;
    if (sym) std::memcpy(sym, g.sym.data(), N * sizeof(uint64_t));
    if (len) std::memcpy(len, g.len.data(), N);
    if (p) std::memcpy(p, g.p.data(), N * sizeof(double));
    if (w) std::memcpy(w, g.w.data(), N * sizeof(uint64_t));
    if (thr) std::memcpy(thr, g.thr.data(), N * sizeof(uint32_t));
    if (alias) std::memcpy(alias, g.alias.data(), N * sizeof(uint32_t));
    return RMAT_OK;
}

rmat_status rmat_table_upload(rmat_table *t) {
    clear_error();
    if (!t) return fail(RMAT_ERR_INVALID_ARGUMENT, "table is NULL");
    DeviceProps props;
    if (rmat_status st = device_props(props)) return st;
    const uint32_t *p = nullptr;
    return ensure_device_copy(t, &p);
}

void rmat_free_table(rmat_table *t) {
    if (!t) return;
    for (auto &kv : t->dev)
        if (kv.second.ptr) cudaFree(kv.second.ptr);
    delete t;
}

rmat_status rmat_set_launch_config(rmat_table *t, const rmat_launch_config_t *cfg) {
    clear_error();
    if (!t || !cfg) return fail(RMAT_ERR_INVALID_ARGUMENT, "NULL argument");
    if (cfg->threads < 128 || cfg->threads > 1024 || cfg->threads % 32)
        return fail(RMAT_ERR_INVALID_ARGUMENT, "threads must be a multiple of 32 in [128, 1024]");
    if (cfg->ctas_per_sm < 1 || cfg->ctas_per_sm > 8) return fail(RMAT_ERR_INVALID_ARGUMENT, "ctas_per_sm in [1, 8]");
    if (cfg->tile_edges < 32 || cfg->tile_edges > 1024 || cfg->tile_edges % 32)
        return fail(RMAT_ERR_INVALID_ARGUMENT, "tile_edges must be a multiple of 32 in [32, 1024]");
    std::lock_guard<std::mutex> lk(t->mu);
    t->cfg = *cfg;
    t->cfg_set = true;
    t->plans.clear();
    return RMAT_OK;
}

rmat_status rmat_get_launch_config(const rmat_table *t, rmat_launch_config_t *cfg) {
    clear_error();
    if (!t || !cfg) return fail(RMAT_ERR_INVALID_ARGUMENT, "NULL argument");
    *cfg = t->cfg_set ? t->cfg : default_launch_config(t);
    return RMAT_OK;
}

rmat_status rmat_generate(const rmat_table *t, uint64_t seed, uint64_t edge_offset, uint64_t count, void *out,
                          rmat_stream_t stream) {
    clear_error();
    if (rmat_status st = check_generate_args(t, edge_offset, count, out)) return st;
    if (count == 0) return RMAT_OK;
    const uint32_t *img = nullptr;
    AliasPlan plan;
    if (rmat_status st = get_plan(t, plan)) return st;
    if (rmat_status st = ensure_device_copy(t, &img)) return st;
    return launch_alias(t, img, plan, seed, edge_offset, count, out, reinterpret_cast<cudaStream_t>(stream));
}

rmat_status rmat_generate_host(const rmat_table *t, uint64_t seed, uint64_t edge_offset, uint64_t count,
                               void *host_out, rmat_stream_t stream_) {
    clear_error();
    if (rmat_status st = check_generate_args(t, edge_offset, count, host_out)) return st;
    if (count == 0) return RMAT_OK;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    const uint32_t *img = nullptr;
    AliasPlan plan;
    if (rmat_status st = get_plan(t, plan)) return st;
    if (rmat_status st = ensure_device_copy(t, &img)) return st;
    HostStaging *s = nullptr;
    if (rmat_status st = get_staging(s)) return st;
    const uint64_t eb = wide_ids(t) ? 16 : 8;
    const uint64_t chunk = s->bytes / eb;
    cudaError_t e;
    uint64_t done = 0;
    for (uint64_t i = 0; done < count; ++i) {
        const int b = int(i & 1);
        const uint64_t n = std::min(chunk, count - done);
        if (i >= 2 && (e = cudaStreamWaitEvent(stream, s->drained[b], 0)) != cudaSuccess)
            return cuda_fail("cudaStreamWaitEvent", e);
        if (rmat_status st = launch_alias(t, img, plan, seed, edge_offset + done, n, s->buf[b], stream)) return st;
        if ((e = cudaEventRecord(s->produced[b], stream)) != cudaSuccess) return cuda_fail("cudaEventRecord", e);
        if ((e = cudaStreamWaitEvent(s->copy, s->produced[b], 0)) != cudaSuccess)
            return cuda_fail("cudaStreamWaitEvent", e);
        if ((e = cudaMemcpyAsync(static_cast<unsigned char *>(host_out) + done * eb, s->buf[b], n * eb,
                                 cudaMemcpyDeviceToHost, s->copy)) != cudaSuccess)
            return cuda_fail("cudaMemcpyAsync", e);
        if ((e = cudaEventRecord(s->drained[b], s->copy)) != cudaSuccess) return cuda_fail("cudaEventRecord", e);
        done += n;
    }
    if ((e = cudaStreamSynchronize(s->copy)) != cudaSuccess) return cuda_fail("cudaStreamSynchronize", e);
    return RMAT_OK;
}

rmat_status rmat_generate_naive(const double *abcd, int k, unsigned flags, uint64_t seed, uint64_t edge_offset,
                                uint64_t count, void *out, rmat_stream_t stream) {
    clear_error();
    if (!abcd) return fail(RMAT_ERR_INVALID_ARGUMENT, "abcd is NULL");
    if (rmat_status st = check_k(k)) return st;
    if (flags & ~RMAT_UNDIRECTED) return fail(RMAT_ERR_INVALID_ARGUMENT, "unknown flag");
    if (count && !out) return fail(RMAT_ERR_INVALID_ARGUMENT, "output pointer is NULL");
    if (reinterpret_cast<uintptr_t>(out) & 7u) return fail(RMAT_ERR_INVALID_ARGUMENT, "output must be 8-byte aligned");
    if (count > RMAT_MAX_EDGES) return fail(RMAT_ERR_INVALID_ARGUMENT, "count above RMAT_MAX_EDGES");
    if (count > ~uint64_t(0) - edge_offset)
        return fail(RMAT_ERR_INVALID_ARGUMENT, "edge_offset + count overflows 64 bits");
    std::vector<uint32_t> thr(size_t(3) * k);
    auto threshold = [](double x) -> uint32_t {
        const double v = std::floor(std::ldexp(x, 32) + 0.5);
        if (v >= 4294967295.0) return 0xFFFFFFFFu;
        if (v <= 0.0) return 0u;
        return uint32_t(v);
    };
    for (int t = 0; t < k; ++t) {
        double P[4];
        if (rmat_status st = normalise_params(abcd + 4 * t, P)) return st;
        thr[3 * t + 0] = threshold(P[0]);
        thr[3 * t + 1] = threshold(P[0] + P[1]);
        thr[3 * t + 2] = threshold((P[0] + P[1]) + P[2]);
    }
    return launch_naive(thr.data(), k, flags, seed, edge_offset, count, out,
                        reinterpret_cast<cudaStream_t>(stream));
}

rmat_status rmat_selftest_bounded_wait(uint32_t limit) {
    clear_error();
    if (limit < 1 || limit > (1u << 22)) return fail(RMAT_ERR_INVALID_ARGUMENT, "limit must be in [1, 2^22]");
    if (rmat_status st = launch_wait_selftest(limit, nullptr)) return st;
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail(RMAT_ERR_CUDA, std::string("self-test: ") + cudaGetErrorString(e));
    return rmat_check_device_errors();
}

rmat_status rmat_check_device_errors(void) {
    clear_error();
    unsigned v = 0;
    if (rmat_status st = read_and_clear_device_error(v)) return st;
    if (v) return fail(RMAT_ERR_TIMEOUT, "a kernel's bounded wait on its table copy gave up");
    return RMAT_OK;
}

}  // extern "C"
