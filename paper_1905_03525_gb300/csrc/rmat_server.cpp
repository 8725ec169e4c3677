// rmat_server.cpp -- a generation server with continuous batching.
//
// Clients submit requests (a, b, c, d, k, m, seed) from any thread.  One worker
// thread owns the GPU work:
//   admission  requests leave the FIFO queue when a slot is free and their
//              table blob plus one chunk buffer fit the device-memory budget
//              (a first-fit sub-allocator over one arena of that size);
//   step       the next chunk (<= chunk_edges) of admitted requests -- those
//              that finish in this chunk first, then the others round-robin,
//              up to step_edges in all -- goes into ONE persistent batched
//              launch (the same kernel as rmat_batch_launch), followed by a
//              batched checksum kernel that consumes the chunks (and an
//              optional client callback that sees each chunk on the device);
//   completion a request whose last chunk is consumed releases its memory and
//              its slot at once, and queued requests are admitted before the
//              next step, so new work joins the GPU while other requests are
//              still being generated.
// Tables of requests with a large explicit bound (>= gpu_build_min_bound) are
// built on the GPU (Sec. 3 parallel construction, rmat_build_table_gpu) by a
// builder thread on its own stream: submit returns at once, and admission
// takes such a request once its table is ready (requests behind it in the
// queue are not held up).  Smaller tables are built on the submitting thread.
// Every edge's bytes depend only on (table, seed, edge index), so a request's
// output and checksum are the same alone and in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "rmat_internal.h"
#include "rmat_kernels.h"

namespace rmat {
namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over [0, size) with 256-byte granularity.
class Arena {
  public:
    explicit Arena(size_t size) { free_[0] = size; }
    bool alloc(size_t bytes, size_t &off) {
        bytes = (bytes + 255) & ~size_t(255);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                off = it->first;
                const size_t rest = it->second - bytes;
                free_.erase(it);
                if (rest) free_[off + bytes] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) & ~size_t(255);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }

  private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0;
};

struct Request {
    uint64_t id = 0;
    rmat_request_t desc{};
    rmat_table *table = nullptr;
    int state = RMAT_REQ_QUEUED;
    uint64_t next = 0;         // first edge of the next chunk
    uint64_t checksum = 0;
    size_t blob_off = 0, blob_bytes = 0, buf_off = 0, buf_bytes = 0;
    uint64_t buf_edges = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    rmat_status err = RMAT_OK;
    bool ready = true;         // table built (false while the builder thread works on it)
};

}  // namespace
}  // namespace rmat

struct rmat_server {
    rmat_server_config_t cfg{};
    int device = 0;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::thread worker;
    std::deque<rmat::Request *> queue;
    std::deque<rmat::Request *> to_build;  // requests whose table the builder thread makes
    std::condition_variable cv_build;
    std::thread builder;
    cudaStream_t build_stream = nullptr;
    std::vector<rmat::Request *> active;
    std::map<uint64_t, rmat::Request *> all;
    uint64_t next_id = 1;
    rmat_chunk_fn chunk_fn = nullptr;
    void *chunk_user = nullptr;
    // device state (worker thread only)
    cudaStream_t stream = nullptr;
    unsigned char *arena_dev = nullptr;
    rmat::Arena *arena = nullptr;
    rmat::Job *d_jobs = nullptr;
    rmat::Scramble *d_scr = nullptr;
    uint32_t *d_units = nullptr;
    unsigned long long *d_counter = nullptr, *d_sums = nullptr;
    rmat::Job *h_jobs = nullptr;       // pinned staging
    rmat::Scramble *h_scr = nullptr;
    uint32_t *h_units = nullptr;
    unsigned long long *h_sums = nullptr;
    uint64_t max_units = 0;
    rmat::DeviceProps props;
    uint64_t steps = 0, edges = 0;
};

namespace rmat {
namespace {

double now_s(const rmat_server *s) {
    return std::chrono::duration<double>(Clock::now() - s->t0).count();
}

constexpr int kThreads = 1024;
// The smallest warp tile a step uses (the automatic table bound keeps every
// table stageable beside tiles of this size), and the unit size it implies
// (units hold 16 tiles per warp, so larger tiles only make fewer units).
int tile_for(bool u64) { return u64 ? 128 : 256; }
uint64_t unit_edges_for(bool u64) { return uint64_t(kThreads / 32) * tile_for(u64) * 16; }

void release(rmat_server *s, Request *r) {
    if (r->blob_bytes) s->arena->release(r->blob_off, r->blob_bytes);
    if (r->buf_bytes) s->arena->release(r->buf_off, r->buf_bytes);
    r->blob_bytes = r->buf_bytes = 0;
}

void finish(rmat_server *s, Request *r, int state, rmat_status err) {
    release(s, r);
    r->state = state;
    r->err = err;
    r->t_done = now_s(s);
    if (r->table) {
        rmat_free_table(r->table);
        r->table = nullptr;
    }
}

// Admit queued requests in FIFO order while a slot is free and memory fits;
// requests whose table is still being built are passed over.
void admit(rmat_server *s) {
    for (auto it = s->queue.begin(); it != s->queue.end() && int(s->active.size()) < s->cfg.max_active;) {
        Request *r = *it;
        if (!r->ready) {
            ++it;
            continue;
        }
        const uint64_t eb = r->table->k > 32 ? 16 : 8;
        const size_t blob = r->table->image.size() * 4;
        const uint64_t edges = std::min<uint64_t>(r->desc.m, s->cfg.chunk_edges);
        size_t boff, coff;
        if (!s->arena->alloc(blob, boff)) break;
        if (!s->arena->alloc(edges * eb, coff)) {
            s->arena->release(boff, blob);
            break;
        }
        it = s->queue.erase(it);
        r->blob_off = boff;
        r->blob_bytes = blob;
        r->buf_off = coff;
        r->buf_bytes = edges * eb;
        r->buf_edges = edges;
        r->state = RMAT_REQ_RUNNING;
        r->t_admit = now_s(s);
        cudaError_t e = cudaMemcpyAsync(s->arena_dev + boff, r->table->image.data(), blob, cudaMemcpyHostToDevice,
                                        s->stream);
        if (e != cudaSuccess) {
            finish(s, r, RMAT_REQ_FAILED, RMAT_ERR_CUDA);
            s->cv_done.notify_all();
            continue;
        }
        s->active.push_back(r);
    }
}

// Wait for the stream with a host-side deadline.
rmat_status wait_stream(rmat_server *s) {
    const auto deadline = Clock::now() + std::chrono::duration<double>(s->cfg.wait_timeout_s);
    for (;;) {
        const cudaError_t e = cudaStreamQuery(s->stream);
        if (e == cudaSuccess) return RMAT_OK;
        if (e != cudaErrorNotReady) return fail(RMAT_ERR_CUDA, std::string("server step: ") + cudaGetErrorString(e));
        if (Clock::now() > deadline) return fail(RMAT_ERR_TIMEOUT, "server step exceeded wait_timeout_s");
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

// One step over the chosen jobs of one output width.
rmat_status run_step(rmat_server *s, const std::vector<Request *> &picked, const std::vector<uint64_t> &counts,
                     bool u64) {
    if (picked.empty()) return RMAT_OK;
    // 512-edge tiles (256 for u64) unless the step's largest table would not
    // fit in shared memory beside them (as rmat_batch_prepare's default)
    size_t largest = 0;
    for (const Request *r : picked) largest = std::max(largest, r->blob_bytes);
    int tile = u64 ? 256 : 512;
    while (tile > tile_for(u64) &&
           kBatchHeaderBytes + size_t(kThreads / 32) * warp_bytes(u64, false, tile) + largest > size_t(s->props.max_smem))
        tile /= 2;
    const uint64_t ue = uint64_t(kThreads / 32) * tile * 16;
    const size_t per_warp = warp_bytes(u64, false, tile);
    const size_t budget = size_t(s->props.max_smem) - kBatchHeaderBytes - size_t(kThreads / 32) * per_warp;
    uint64_t units = 0;
    uint32_t max_blob = 0;
    for (size_t j = 0; j < picked.size(); ++j) {
        Request *r = picked[j];
        const uint32_t *blob = reinterpret_cast<const uint32_t *>(s->arena_dev + r->blob_off);
        const bool smem = r->blob_bytes <= budget;
        if (smem) max_blob = std::max<uint32_t>(max_blob, uint32_t(r->blob_bytes));
        Job J = make_job(r->table, blob, smem, r->desc.seed, r->next, counts[j], s->arena_dev + r->buf_off);
        J.unit_begin = units;
        const uint64_t nu = (counts[j] + ue - 1) / ue;
        for (uint64_t k = 0; k < nu; ++k) s->h_units[units + k] = uint32_t(j);
        units += nu;
        s->h_jobs[j] = J;
        s->h_scr[j] = make_scramble(r->table);
    }
    cudaError_t e;
    if ((e = cudaMemcpyAsync(s->d_jobs, s->h_jobs, picked.size() * sizeof(Job), cudaMemcpyHostToDevice, s->stream)) ||
        (e = cudaMemcpyAsync(s->d_scr, s->h_scr, picked.size() * sizeof(Scramble), cudaMemcpyHostToDevice,
                             s->stream)) ||
        (e = cudaMemcpyAsync(s->d_units, s->h_units, units * sizeof(uint32_t), cudaMemcpyHostToDevice, s->stream)) ||
        (e = cudaMemsetAsync(s->d_sums, 0, picked.size() * sizeof(unsigned long long), s->stream)))
        return fail(RMAT_ERR_CUDA, std::string("server upload: ") + cudaGetErrorString(e));
    BatchArgs a{};
    a.jobs = s->d_jobs;
    a.scr = s->d_scr;
    a.unit_job = s->d_units;
    a.units = units;
    a.unit_edges = ue;
    a.counter = s->d_counter;
    a.max_blob_bytes = max_blob;
    a.tile = tile;
    a.err = s->props.err;
    for (const Request *r : picked) a.general |= r->table->scramble ? 1 : 0;
    const size_t smem = batch_smem_bytes(u64, kThreads, tile, max_blob);
    int per_sm = 0;
    if (rmat_status st = batch_occupancy(u64, kThreads, smem, per_sm)) return st;
    const int grid = int(std::min<uint64_t>(uint64_t(s->props.sms) * std::max(1, per_sm), units));
    if (rmat_status st = launch_batch(u64, a, grid, kThreads, smem, s->stream)) return st;
    if (rmat_status st = launch_checksum(u64, a, s->d_sums, s->props.sms * 8, s->stream)) return st;
    if ((e = cudaMemcpyAsync(s->h_sums, s->d_sums, picked.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                             s->stream)))
        return fail(RMAT_ERR_CUDA, std::string("server readback: ") + cudaGetErrorString(e));
    if (rmat_status st = wait_stream(s)) return st;
    for (size_t j = 0; j < picked.size(); ++j) {
        Request *r = picked[j];
        if (s->chunk_fn) s->chunk_fn(s->chunk_user, r->id, r->next, counts[j], s->arena_dev + r->buf_off);
        r->checksum += s->h_sums[j];
        r->next += counts[j];
        s->edges += counts[j];
    }
    ++s->steps;
    return RMAT_OK;
}

void worker_main(rmat_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    size_t rr = 0;  // round-robin cursor over requests that need several chunks
    for (;;) {
        admit(s);
        if (s->active.empty()) {
            if (s->stop && s->queue.empty() && s->to_build.empty()) break;
            s->cv_work.wait_for(lk, std::chrono::milliseconds(20));
            continue;
        }
        // Pick this step's chunks: requests that finish with this chunk first
        // (short jobs leave quickly), then the others round-robin.
        std::vector<Request *> finishing, longer;
        for (Request *r : s->active) (r->desc.m - r->next <= r->buf_edges ? finishing : longer).push_back(r);
        std::vector<Request *> order = finishing;
        for (size_t i = 0; i < longer.size(); ++i) order.push_back(longer[(rr + i) % longer.size()]);
        rr += 1;
        std::vector<Request *> pick[2];
        std::vector<uint64_t> cnt[2];
        uint64_t budget = s->cfg.step_edges;
        for (Request *r : order) {
            const uint64_t n = std::min<uint64_t>(r->buf_edges, r->desc.m - r->next);
            if (n > budget && !(pick[0].empty() && pick[1].empty())) continue;
            const int w = r->table->k > 32 ? 1 : 0;
            pick[w].push_back(r);
            cnt[w].push_back(n);
            budget = n >= budget ? 0 : budget - n;
            if (!budget) break;
        }
        lk.unlock();
        rmat_status st = RMAT_OK;
        for (int w = 0; w < 2 && st == RMAT_OK; ++w) st = run_step(s, pick[w], cnt[w], w == 1);
        lk.lock();
        if (st != RMAT_OK) {
            // A failed step fails the requests in it; the server keeps serving.
            // Their memory is released only once the device work is over.
            cudaStreamSynchronize(s->stream);
            for (int w = 0; w < 2; ++w)
                for (Request *r : pick[w]) {
                    finish(s, r, RMAT_REQ_FAILED, st);
                    s->active.erase(std::find(s->active.begin(), s->active.end(), r));
                }
            s->cv_done.notify_all();
            continue;
        }
        bool any_done = false;
        for (size_t i = 0; i < s->active.size();) {
            Request *r = s->active[i];
            if (r->next >= r->desc.m) {
                finish(s, r, RMAT_REQ_DONE, RMAT_OK);
                s->active.erase(s->active.begin() + long(i));
                any_done = true;
            } else {
                ++i;
            }
        }
        if (any_done) s->cv_done.notify_all();
    }
}

// Build the request's table (GPU construction, host construction when the
// parameters are outside the GPU build's range) with its flags and
// relabelling.
rmat_status build_request_table(rmat_server *s, const rmat_request_t &q, uint64_t bound, bool on_gpu,
                                rmat_table **out) {
    rmat_table *t = nullptr;
    rmat_status st = RMAT_ERR_UNSUPPORTED;
    if (on_gpu) st = rmat_build_table_gpu(q.a, q.b, q.c, q.d, q.k, bound, reinterpret_cast<rmat_stream_t>(s->build_stream), &t);
    if (st == RMAT_ERR_UNSUPPORTED) st = rmat_build_table(q.a, q.b, q.c, q.d, q.k, bound, &t);
    if (st == RMAT_OK) st = rmat_table_set_flags(t, q.flags);
    if (st == RMAT_OK) st = rmat_table_set_scramble(t, q.scramble, q.scramble_seed);
    if (st != RMAT_OK) {
        if (t) rmat_free_table(t);
        return st;
    }
    *out = t;
    return RMAT_OK;
}

void builder_main(rmat_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        while (s->to_build.empty() && !s->stop) s->cv_build.wait(lk);
        if (s->to_build.empty()) break;
        Request *r = s->to_build.front();
        s->to_build.pop_front();
        const rmat_request_t q = r->desc;
        lk.unlock();
        rmat_table *t = nullptr;
        const rmat_status st = build_request_table(s, q, q.table_bound, true, &t);
        lk.lock();
        if (st != RMAT_OK) {
            s->queue.erase(std::find(s->queue.begin(), s->queue.end(), r));
            finish(s, r, RMAT_REQ_FAILED, st);
            s->cv_done.notify_all();
            continue;
        }
        r->table = t;
        r->ready = true;
        s->cv_work.notify_one();
    }
}

template <class T>
rmat_status dev_alloc(T **p, size_t bytes) {
    if (cudaMalloc(reinterpret_cast<void **>(p), std::max<size_t>(bytes, 256)) != cudaSuccess) {
        cudaGetLastError();
        return fail(RMAT_ERR_OUT_OF_MEMORY, "server device allocation failed");
    }
    return RMAT_OK;
}

template <class T>
rmat_status host_alloc(T **p, size_t bytes) {
    if (cudaHostAlloc(reinterpret_cast<void **>(p), std::max<size_t>(bytes, 256), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return fail(RMAT_ERR_OUT_OF_MEMORY, "server pinned allocation failed");
    }
    return RMAT_OK;
}

void free_server(rmat_server *s) {
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->arena_dev) cudaFree(s->arena_dev);
    if (s->d_jobs) cudaFree(s->d_jobs);
    if (s->d_scr) cudaFree(s->d_scr);
    if (s->d_units) cudaFree(s->d_units);
    if (s->d_counter) cudaFree(s->d_counter);
    if (s->d_sums) cudaFree(s->d_sums);
    if (s->h_jobs) cudaFreeHost(s->h_jobs);
    if (s->h_scr) cudaFreeHost(s->h_scr);
    if (s->h_units) cudaFreeHost(s->h_units);
    if (s->h_sums) cudaFreeHost(s->h_sums);
    if (s->stream) cudaStreamDestroy(s->stream);
    if (s->build_stream) cudaStreamDestroy(s->build_stream);
    for (auto &kv : s->all) {
        if (kv.second->table) rmat_free_table(kv.second->table);
        delete kv.second;
    }
    delete s->arena;
    delete s;
}

void fill_status(const Request *r, rmat_request_status_t *st) {
    st->id = r->id;
    st->state = r->state;
    st->edges_done = r->next;
    st->checksum = r->checksum;
    st->submit_s = r->t_submit;
    st->admit_s = r->t_admit;
    st->done_s = r->t_done;
    st->error = r->err;
    st->table_bound = r->desc.table_bound;
}

}  // namespace
}  // namespace rmat

using namespace rmat;

extern "C" {

rmat_status rmat_server_create(const rmat_server_config_t *cfg, rmat_server **out) {
    clear_error();
    if (!cfg || !out) return fail(RMAT_ERR_INVALID_ARGUMENT, "NULL argument");
    *out = nullptr;
    if (cfg->hbm_budget_bytes < (uint64_t(1) << 20)) return fail(RMAT_ERR_INVALID_ARGUMENT, "budget below 1 MiB");
    if (cfg->chunk_edges < 1024 || cfg->step_edges < cfg->chunk_edges || cfg->max_active < 1 || cfg->max_active > 4096 ||
        !(cfg->wait_timeout_s > 0))
        return fail(RMAT_ERR_INVALID_ARGUMENT, "bad server configuration");
    rmat_server *s = new (std::nothrow) rmat_server;
    if (!s) return fail(RMAT_ERR_OUT_OF_MEMORY, "host allocation failed");
    s->cfg = *cfg;
    s->t0 = Clock::now();
    cudaGetDevice(&s->device);
    rmat_status st = device_props(s->props);
    if (st == RMAT_OK && (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
                          cudaStreamCreateWithFlags(&s->build_stream, cudaStreamNonBlocking) != cudaSuccess))
        st = fail(RMAT_ERR_CUDA, "stream creation failed");
    if (st == RMAT_OK) st = dev_alloc(&s->arena_dev, cfg->hbm_budget_bytes);
    // Work list of one step: at most max_active jobs and
    // step_edges / unit_edges + max_active units.
    s->max_units = cfg->step_edges / unit_edges_for(true) + uint64_t(cfg->max_active) + 1;
    if (st == RMAT_OK) st = dev_alloc(&s->d_jobs, sizeof(Job) * cfg->max_active);
    if (st == RMAT_OK) st = dev_alloc(&s->d_scr, sizeof(Scramble) * cfg->max_active);
    if (st == RMAT_OK) st = dev_alloc(&s->d_units, sizeof(uint32_t) * s->max_units);
    if (st == RMAT_OK) st = dev_alloc(&s->d_counter, sizeof(unsigned long long));
    if (st == RMAT_OK) st = dev_alloc(&s->d_sums, sizeof(unsigned long long) * cfg->max_active);
    if (st == RMAT_OK) st = host_alloc(&s->h_jobs, sizeof(Job) * cfg->max_active);
    if (st == RMAT_OK) st = host_alloc(&s->h_scr, sizeof(Scramble) * cfg->max_active);
    if (st == RMAT_OK) st = host_alloc(&s->h_units, sizeof(uint32_t) * s->max_units);
    if (st == RMAT_OK) st = host_alloc(&s->h_sums, sizeof(unsigned long long) * cfg->max_active);
    if (st != RMAT_OK) {
        const std::string msg = rmat_last_error();
        free_server(s);
        return fail(st, msg);
    }
    s->arena = new Arena(cfg->hbm_budget_bytes);
    s->worker = std::thread(worker_main, s);
    s->builder = std::thread(builder_main, s);
    *out = s;
    return RMAT_OK;
}

rmat_status rmat_server_set_chunk_callback(rmat_server *s, rmat_chunk_fn fn, void *user) {
    clear_error();
    if (!s) return fail(RMAT_ERR_INVALID_ARGUMENT, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    s->chunk_fn = fn;
    s->chunk_user = user;
    return RMAT_OK;
}

rmat_status rmat_server_submit(rmat_server *s, const rmat_request_t *req, uint64_t *id) {
    clear_error();
    if (!s || !req) return fail(RMAT_ERR_INVALID_ARGUMENT, "NULL argument");
    if (req->m == 0) return fail(RMAT_ERR_INVALID_ARGUMENT, "a request needs m >= 1 edges");
    if (req->m > RMAT_MAX_EDGES) return fail(RMAT_ERR_INVALID_ARGUMENT, "m above RMAT_MAX_EDGES");
    // table_bound 0: the largest power-of-two bound <= 8192 whose blob the
    // batched kernel can stage in shared memory (deep paths of skewed
    // parameters make wide, 36-byte columns); otherwise exactly the bound asked.
    const bool u64 = req->k > 32;
    const size_t smem_budget = size_t(s->props.max_smem) - kBatchHeaderBytes -
                               size_t(kThreads / 32) * warp_bytes(u64, false, tile_for(u64));
    uint64_t bound = req->table_bound ? req->table_bound : 8192;
    const uint64_t eb = req->k > 32 ? 16 : 8;
    const uint64_t chunk_bytes = (std::min<uint64_t>(req->m, s->cfg.chunk_edges) * eb + 255) & ~uint64_t(255);
    const bool on_gpu = req->table_bound && s->cfg.gpu_build_min_bound && req->table_bound >= s->cfg.gpu_build_min_bound;
    rmat_table *t = nullptr;
    if (on_gpu) {
        // checked now with the largest image a table of this bound can have
        // (wide entries: 36 bytes per column of the padded size)
        if (req->table_bound < 5 || req->table_bound > (uint64_t(1) << 24) || req->k < 1 || req->k > 64)
            return fail(RMAT_ERR_INVALID_ARGUMENT, "table_bound must be in [5, 2^24] and k in [1, 64]");
        const double in[4] = {req->a, req->b, req->c, req->d};
        double P[4];
        if (rmat_status st = normalise_params(in, P)) return st;
        uint64_t N = 1;
        while (N < req->table_bound) N <<= 1;
        const uint64_t image_max = ((4 * kHeaderWords + 36 * N + 64) + 255) & ~uint64_t(255);
        if (image_max + chunk_bytes > s->cfg.hbm_budget_bytes)
            return fail(RMAT_ERR_OUT_OF_MEMORY, "request needs more device memory than the server's whole budget");
    } else {
        for (;;) {
            if (rmat_status st = build_request_table(s, *req, bound, false, &t)) return st;
            if (req->table_bound || t->image.size() * 4 <= smem_budget || bound <= 64) break;
            rmat_free_table(t);
            t = nullptr;
            bound /= 2;
        }
        const uint64_t need = ((t->image.size() * 4 + 255) & ~uint64_t(255)) + chunk_bytes;
        if (need > s->cfg.hbm_budget_bytes) {
            rmat_free_table(t);
            return fail(RMAT_ERR_OUT_OF_MEMORY, "request needs more device memory than the server's whole budget");
        }
    }
    Request *r = new (std::nothrow) Request;
    if (!r) {
        rmat_free_table(t);
        return fail(RMAT_ERR_OUT_OF_MEMORY, "host allocation failed");
    }
    r->desc = *req;
    r->desc.table_bound = bound;
    r->table = t;
    r->ready = !on_gpu;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->id = s->next_id++;
        r->t_submit = now_s(s);
        s->all[r->id] = r;
        s->queue.push_back(r);
        if (on_gpu) s->to_build.push_back(r);
    }
    if (on_gpu) s->cv_build.notify_one();
    else s->cv_work.notify_one();
    if (id) *id = r->id;
    return RMAT_OK;
}

rmat_status rmat_server_status(rmat_server *s, uint64_t id, rmat_request_status_t *st) {
    clear_error();
    if (!s || !st) return fail(RMAT_ERR_INVALID_ARGUMENT, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return fail(RMAT_ERR_INVALID_ARGUMENT, "unknown request id");
    fill_status(it->second, st);
    return RMAT_OK;
}

rmat_status rmat_server_wait(rmat_server *s, uint64_t id, double timeout_s, rmat_request_status_t *st) {
    clear_error();
    if (!s) return fail(RMAT_ERR_INVALID_ARGUMENT, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return fail(RMAT_ERR_INVALID_ARGUMENT, "unknown request id");
    Request *r = it->second;
    const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s);
    while (r->state == RMAT_REQ_QUEUED || r->state == RMAT_REQ_RUNNING) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout &&
            (r->state == RMAT_REQ_QUEUED || r->state == RMAT_REQ_RUNNING)) {
            if (st) fill_status(r, st);
            return fail(RMAT_ERR_TIMEOUT, "request not finished within timeout");
        }
    }
    if (st) fill_status(r, st);
    if (r->state == RMAT_REQ_FAILED) return fail(r->err ? r->err : RMAT_ERR_CUDA, "request failed");
    return RMAT_OK;
}

rmat_status rmat_server_drain(rmat_server *s, double timeout_s) {
    clear_error();
    if (!s) return fail(RMAT_ERR_INVALID_ARGUMENT, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s);
    while (!s->queue.empty() || !s->active.empty()) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout &&
            (!s->queue.empty() || !s->active.empty()))
            return fail(RMAT_ERR_TIMEOUT, "server not drained within timeout");
    }
    return RMAT_OK;
}

rmat_status rmat_server_stats(rmat_server *s, rmat_server_stats_t *out) {
    clear_error();
    if (!s || !out) return fail(RMAT_ERR_INVALID_ARGUMENT, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    out->steps = s->steps;
    out->edges = s->edges;
    out->queued = s->queue.size();
    out->active = s->active.size();
    out->memory_used = s->arena->used();
    out->clock_s = now_s(s);
    return RMAT_OK;
}

void rmat_server_destroy(rmat_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->to_build.clear();
    }
    // the builder finishes the table it is making, then stops
    s->cv_build.notify_all();
    if (s->builder.joinable()) s->builder.join();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        // requests still queued are failed without running
        while (!s->queue.empty()) {
            finish(s, s->queue.front(), RMAT_REQ_FAILED, RMAT_ERR_INVALID_ARGUMENT);
            s->queue.pop_front();
        }
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    s->cv_done.notify_all();
    free_server(s);
}

}  // extern "C"
