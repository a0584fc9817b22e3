// hec_serve.cu -- the solve server of include/hecgpu.h: a request queue,
// admission by device memory, lanes (host threads with their own CUDA
// streams) that set up and solve requests concurrently, and a keyed cache of
// set-up systems.  Built on the library's own entry points; host C++ only.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <list>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/hecgpu.h"
#include "runtime.h"

using namespace hec;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0, tag = 0, key = 0;
    uint64_t pattern = 0; // hash of row_ptr and col (matrix requests)
    int n = 0, k = 0;
    bool has_matrix = true;
    std::vector<int32_t> rp, ci;
    std::vector<double> va, b;
    double t_submit = 0.0;
};

// A set-up system: the single-system handles, or a one-system batch.
struct Resident {
    hec_matrix_t A = nullptr;
    hec_precond_t M = nullptr;
    hec_batch_t B = nullptr;
    int64_t bytes = 0;
    int n = 0, k = 0;
    int64_t nnz = 0;
    uint64_t pattern = 0;
    int users = 0;
    std::list<uint64_t>::iterator lru;
    void destroy()
    {
        if (M)
            hec_precond_destroy(M);
        if (A)
            hec_matrix_destroy(A);
        if (B)
            hec_batch_destroy(B);
        A = nullptr;
        M = nullptr;
        B = nullptr;
    }
};

} // namespace

struct hec_server_s {
    hec_server_opts_t o{};
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_mem;
    std::deque<Request> pending;
    std::deque<hec_result_t> finished;            // not yet polled
    std::unordered_map<uint64_t, std::vector<double>> solutions;
    std::unordered_map<uint64_t, Resident> cache;  // by key
    std::list<uint64_t> lru;                        // idle cached keys, oldest first
    std::unordered_map<uint64_t, int> busy;         // keys being set up or solved
    std::vector<cudaStream_t> streams;              // one per lane, kept to the end
    int64_t reserved = 0;  // running requests' estimates + cached systems
    int running = 0;
    uint64_t next_ticket = 1;
    bool stopping = false;
    bool verbose = false;  // HEC_SERVER_VERBOSE set: failed requests are reported on stderr
    std::vector<std::thread> lanes;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

// Device bytes of a request before its setup: the HEC slab and tail, FP64
// and FP32 factor layouts (fill estimated from the level k) and the GMRES
// workspace.  Replaced by the handles' own count once set up.
int64_t estimate_bytes(const Request &q, int m)
{
    const int64_t nnz = (int64_t)q.ci.size(), n = q.n;
    const int64_t fill = q.k == 0 ? 1 : q.k == 1 ? 3 : 6;
    return nnz * 24 + fill * nnz * 24 + n * 8 * (int64_t)(m + 16);
}

int64_t resident_bytes(const Resident &R)
{
    int64_t t = 0;
    if (R.A) {
        hec_matrix_info_t mi;
        if (hec_matrix_info(R.A, &mi) == HEC_OK)
            t += mi.device_bytes;
    }
    if (R.M) {
        hec_precond_info_t pi;
        if (hec_precond_info(R.M, &pi) == HEC_OK)
            t += pi.device_bytes;
    }
    if (R.B) {
        hec_batch_info_t bi;
        if (hec_batch_info(R.B, &bi) == HEC_OK)
            t += bi.device_bytes;
    }
    return t;
}

// FNV-1a over the sparsity pattern: equal patterns let a keyed request with
// new values refactor its resident system instead of setting it up again.
uint64_t pattern_hash(const std::vector<int32_t> &rp, const std::vector<int32_t> &ci)
{
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](const std::vector<int32_t> &v) {
        for (int32_t x : v) {
            h ^= (uint32_t)x;
            h *= 1099511628211ull;
        }
    };
    mix(rp);
    mix(ci);
    return h;
}

int setup(hec_server_s *S, const Request &q, cudaStream_t st, Resident &R)
{
    R.n = q.n;
    R.k = q.k;
    R.nnz = (int64_t)q.ci.size();
    R.pattern = q.pattern;
    if (q.n <= S->o.small_rows) {
        const int64_t sp[2] = {0, q.n};
        std::vector<int64_t> rp(q.rp.begin(), q.rp.end());
        hec_batch_csr_t c{1, 0, sp, rp.data(), q.ci.data(), q.va.data()};
        hec_batch_config_t cfg{256, 0, 0, 0};  // fixed: results independent of the mix
        HEC_TRY(hec_build_batched(&c, &cfg, st, &R.B));
        return ilu_k_setup_batched(R.B, q.k);
    }
    hec_csr_t c{q.n, (int32_t)q.ci.size(), q.rp.data(), q.ci.data(), q.va.data(), 0};
    HEC_TRY(hec_build(&c, nullptr, st, &R.A));
    const int nb = std::max(1, std::min(64, (q.n + S->o.block_rows - 1) / S->o.block_rows));
    HEC_TRY(ilu_k_setup(R.A, q.k, nb, nb > 1 ? 1 : 0, st, &R.M));
    return level_schedule(R.M, st);
}

// Evicts idle cached systems, oldest first, until `need` more bytes fit.
// Called with the lock held.
void make_room(hec_server_s *S, int64_t need)
{
    while (S->reserved + need > S->o.device_budget && !S->lru.empty()) {
        const uint64_t key = S->lru.front();
        S->lru.pop_front();
        auto it = S->cache.find(key);
        S->reserved -= it->second.bytes;
        it->second.destroy();
        S->cache.erase(it);
    }
}

// The next request a lane may start, in arrival order, skipping requests
// whose key another lane holds (a set-up system serves one solve at a
// time).  -1: none startable.  With the lock held.
int pick(hec_server_s *S)
{
    for (size_t i = 0; i < S->pending.size(); ++i) {
        const uint64_t key = S->pending[i].key;
        if (key == 0 || S->busy.find(key) == S->busy.end())
            return (int)i;
    }
    return -1;
}

void lane_main(hec_server_s *S, int lane)
{
    cudaStream_t st = S->streams[lane];
    double *db = nullptr, *dx = nullptr;
    size_t cap = 0;
    const int m = S->o.restart;
    for (;;) {
        Request q;
        bool reuse = false;
        int64_t need = 0;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            // admission in arrival order: the first startable request waits
            // until its memory fits (evicting idle cached systems)
            int idx = -1;
            for (;;) {
                idx = pick(S);
                if (idx < 0) {
                    if (S->stopping && S->pending.empty())
                        break;
                    S->cv_work.wait(lk);
                    continue;
                }
                const Request &h = S->pending[idx];
                auto it = h.key ? S->cache.find(h.key) : S->cache.end();
                reuse = it != S->cache.end();
                need = reuse ? (int64_t)h.n * 8 * (m + 16) : estimate_bytes(h, m);
                if (reuse)
                    S->lru.erase(it->second.lru);  // pinned: not evictable while in use
                make_room(S, need);
                if (S->reserved + need <= S->o.device_budget || S->running == 0)
                    break;
                if (reuse)
                    it->second.lru = S->lru.insert(S->lru.end(), h.key);
                S->cv_mem.wait(lk);
            }
            if (idx < 0)
                break;
            q = std::move(S->pending[idx]);
            S->pending.erase(S->pending.begin() + idx);
            if (q.key)
                S->busy[q.key] = lane;
            if (reuse)
                S->cache[q.key].users = 1;
            S->reserved += need;
            ++S->running;
        }
        hec_result_t r{};
        r.ticket = q.ticket;
        r.tag = q.tag;
        r.t_submit = q.t_submit;
        r.lane = lane;
        r.reused = reuse ? 1 : 0;
        r.t_start = S->now();
        Resident local;
        Resident *R = &local;
        int rc = HEC_OK;
        bool broken = false;  // a cached system's refactor or new set-up failed part-way
        if (reuse) {
            {
                std::lock_guard<std::mutex> lk(S->mu);
                R = &S->cache[q.key];
            }
            if (R->n != q.n || R->k != q.k) {
                rc = fail(HEC_ERR_INVALID, "key %llu was set up for another matrix",
                          (unsigned long long)q.key);
            } else if (q.has_matrix && R->A && R->nnz == (int64_t)q.va.size() &&
                       R->pattern == q.pattern) {
                // same pattern, new values: refactor on the device (HEC values,
                // ILU(k) of every RAS block, triangular-solve layouts); the
                // entry count is compared as well, since the refactor reads
                // exactly the resident matrix's count of values
                rc = hec_refactor(R->A, R->M, q.va.data(), st);
                r.refactored = 1;
                broken = rc < 0;
            } else if (q.has_matrix) {
                // another pattern, or a one-CTA batched system: set it up again
                R->destroy();
                rc = abi_guard("hec_server set-up", [&]() { return setup(S, q, st, *R); });
                broken = rc < 0;
            }
        } else if (!q.has_matrix) {
            rc = fail(HEC_ERR_INVALID, "key %llu is not resident and the request has no matrix",
                      (unsigned long long)q.key);
        } else {
            rc = abi_guard("hec_server set-up", [&]() { return setup(S, q, st, local); });
        }
        r.t_setup = S->now();
        const size_t nb = (size_t)q.n * sizeof(double);
        if (rc == HEC_OK && nb > cap) {
            if (db)
                cudaFreeAsync(db, st);
            if (dx)
                cudaFreeAsync(dx, st);
            cap = nb;
            if (cudaMallocAsync((void **)&db, cap, st) != cudaSuccess ||
                cudaMallocAsync((void **)&dx, cap, st) != cudaSuccess) {
                cudaGetLastError();
                db = dx = nullptr;
                cap = 0;
                rc = HEC_ERR_OOM;
            }
        }
        if (rc == HEC_OK && cudaMemcpyAsync(db, q.b.data(), nb, cudaMemcpyHostToDevice, st) != cudaSuccess)
            rc = HEC_ERR_CUDA;
        hec_solve_info_t info{};
        if (rc == HEC_OK) {
            hec_solve_opts_t so{HEC_GMRES, HEC_X0_ZERO | (S->o.flags & HEC_MIXED_FP32), 0};
            rc = R->B ? krylov_solve_batched(R->B, db, dx, 1, S->o.tol, S->o.maxit, m, &so, st, &info,
                                             nullptr)
                      : krylov_solve(R->A, R->M, db, dx, S->o.tol, S->o.maxit, m, &so, st, &info);
        }
        std::vector<double> x;
        if (rc >= 0 && S->o.keep_solutions) {
            rc = abi_guard("hec_server solution copy", [&]() -> int {
                x.resize(q.n);
                if (cudaMemcpyAsync(x.data(), dx, nb, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                    cudaStreamSynchronize(st) != cudaSuccess)
                    return fail(HEC_ERR_CUDA, "solution copy of request %llu",
                                (unsigned long long)q.ticket);
                return rc;
            });
        }
        if (rc < 0 && S->verbose)
            fprintf(stderr, "hec_server: request %llu (n = %d) failed: %s\n",
                    (unsigned long long)q.ticket, q.n, last_error_text());
        r.status = rc;
        r.fp64_finish = info.fp64_finish ? 1 : 0;
        r.iters = info.iters;
        r.rel_resid = info.rel_resid;
        const int64_t used = resident_bytes(*R);
        r.device_bytes = used;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->reserved -= need;
            if (q.key)
                S->busy.erase(q.key);
            if (reuse && broken) {
                // its handles may hold part of the old and part of the new
                // system: drop the entry, so that the key must come back
                // with a matrix
                Resident &c = S->cache[q.key];
                S->reserved -= c.bytes;
                c.destroy();
                S->cache.erase(q.key);
            } else if (reuse) {
                Resident &c = S->cache[q.key];
                c.users = 0;
                S->reserved += used - c.bytes; // refactor maps or a new set-up
                c.bytes = used;
                c.lru = S->lru.insert(S->lru.end(), q.key);
            } else if (q.key && rc >= 0 && S->cache.find(q.key) == S->cache.end()) {
                local.bytes = used;
                local.users = 0;
                S->reserved += used;
                Resident &c = S->cache[q.key];
                c = local;
                c.lru = S->lru.insert(S->lru.end(), q.key);
                local = Resident();
            }
            --S->running;
            r.t_done = S->now();
            S->finished.push_back(r);
            if (S->o.keep_solutions && rc >= 0)
                S->solutions[q.ticket] = std::move(x);
        }
        local.destroy();
        S->cv_mem.notify_all();
        S->cv_work.notify_all();  // a request held back by this key may start
        S->cv_done.notify_all();
    }
    if (db)
        cudaFreeAsync(db, st);
    if (dx)
        cudaFreeAsync(dx, st);
    cudaStreamSynchronize(st);
}

} // namespace

int hec_server_create(const hec_server_opts_t *opts, hec_server_t *out)
{
    return abi_guard(__func__, [&]() -> int {
        if (!out)
            return fail(HEC_ERR_INVALID, "null argument");
        *out = nullptr;
        hec_server_opts_t o{};
        if (opts)
            o = *opts;
        if (o.lanes < 0 || o.lanes > 64 || o.restart < 0 || o.restart > 31 || o.maxit < 0 ||
            o.small_rows < 0 || o.block_rows < 0 || o.device_budget < 0 || !(o.tol >= 0.0))
            return fail(HEC_ERR_INVALID, "bad server options");
        if (o.lanes == 0)
            o.lanes = 8;
        if (o.restart == 0)
            o.restart = 30;
        if (o.maxit == 0)
            o.maxit = 20000;
        if (o.tol == 0.0)
            o.tol = 1e-8;
        if (o.small_rows == 0)
            o.small_rows = 32768;
        if (o.block_rows == 0)
            o.block_rows = 16384;
        if (o.device_budget == 0) {
            size_t fr = 0, tot = 0;
            if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
                cudaGetLastError();
                return fail(HEC_ERR_CUDA, "no CUDA device");
            }
            o.device_budget = (int64_t)(fr / 2);
        }
        auto S = new hec_server_s();
        S->o = o;
        S->t0 = Clock::now();
        S->verbose = std::getenv("HEC_SERVER_VERBOSE") != nullptr;
        for (int i = 0; i < o.lanes; ++i) {
            cudaStream_t st = nullptr;
            if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
                cudaGetLastError();
                for (cudaStream_t t : S->streams)
                    cudaStreamDestroy(t);
                delete S;
                return fail(HEC_ERR_CUDA, "cannot create a lane stream");
            }
            S->streams.push_back(st);
        }
        for (int i = 0; i < o.lanes; ++i)
            S->lanes.emplace_back(lane_main, S, i);
        *out = S;
        return HEC_OK;
    });
}

int hec_server_submit(hec_server_t S, const hec_request_t *req, uint64_t *ticket)
{
    return abi_guard(__func__, [&]() -> int {
        if (!S || !req || !req->b || req->A.on_device)
            return fail(HEC_ERR_INVALID, "invalid request (host arrays required)");
        const bool has = req->A.row_ptr != nullptr;
        if (!has && req->key == 0)
            return fail(HEC_ERR_INVALID, "a request without a matrix needs a key");
        if (has && (!req->A.col || !req->A.val))
            return fail(HEC_ERR_INVALID, "invalid request matrix");
        const int n = req->A.n;
        if (n < 1 || req->ilu_k < 0 ||
            (has && (req->A.nnz < 0 || req->A.row_ptr[0] != 0 || req->A.row_ptr[n] != req->A.nnz)))
            return fail(HEC_ERR_INVALID, "invalid request matrix");
        Request q;
        q.tag = req->tag;
        q.key = req->key;
        q.n = n;
        q.k = req->ilu_k;
        q.has_matrix = has;
        if (has) {
            q.rp.assign(req->A.row_ptr, req->A.row_ptr + n + 1);
            q.ci.assign(req->A.col, req->A.col + req->A.nnz);
            q.va.assign(req->A.val, req->A.val + req->A.nnz);
            q.pattern = pattern_hash(q.rp, q.ci);
        }
        q.b.assign(req->b, req->b + n);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            if (S->stopping)
                return fail(HEC_ERR_INVALID, "server is shutting down");
            q.ticket = S->next_ticket++;
            q.t_submit = S->now();
            if (ticket)
                *ticket = q.ticket;
            S->pending.push_back(std::move(q));
        }
        S->cv_work.notify_one();
        return HEC_OK;
    });
}

int hec_server_poll(hec_server_t S, hec_result_t *out, int32_t max, int32_t *count, int32_t wait_ms)
{
    return abi_guard(__func__, [&]() -> int {
        if (!S || !count || (max > 0 && !out))
            return fail(HEC_ERR_INVALID, "invalid argument");
        std::unique_lock<std::mutex> lk(S->mu);
        if (S->finished.empty() && wait_ms > 0)
            S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms),
                                [&]() { return !S->finished.empty(); });
        int c = 0;
        while (c < max && !S->finished.empty()) {
            out[c++] = S->finished.front();
            S->finished.pop_front();
        }
        *count = c;
        return HEC_OK;
    });
}

int hec_server_solution(hec_server_t S, uint64_t ticket, double *x, int32_t n)
{
    return abi_guard(__func__, [&]() -> int {
        if (!S || !x)
            return fail(HEC_ERR_INVALID, "invalid argument");
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->solutions.find(ticket);
        if (it == S->solutions.end())
            return fail(HEC_ERR_INVALID, "no stored solution for ticket %llu", (unsigned long long)ticket);
        if ((size_t)n != it->second.size())
            return fail(HEC_ERR_INVALID, "solution has %zu values, not %d", it->second.size(), n);
        std::memcpy(x, it->second.data(), sizeof(double) * it->second.size());
        S->solutions.erase(it);
        return HEC_OK;
    });
}

double hec_server_clock(hec_server_t S) { return S ? S->now() : 0.0; }

int hec_server_stats(hec_server_t S, int32_t *queued, int32_t *running, int32_t *finished,
                     int64_t *reserved_bytes)
{
    return abi_guard(__func__, [&]() -> int {
        if (!S)
            return fail(HEC_ERR_INVALID, "invalid argument");
        std::lock_guard<std::mutex> lk(S->mu);
        if (queued)
            *queued = (int32_t)S->pending.size();
        if (running)
            *running = S->running;
        if (finished)
            *finished = (int32_t)S->finished.size();
        if (reserved_bytes)
            *reserved_bytes = S->reserved;
        return HEC_OK;
    });
}

void hec_server_destroy(hec_server_t S)
{
    if (!S)
        return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
    }
    S->cv_work.notify_all();
    S->cv_mem.notify_all();
    for (auto &t : S->lanes)
        t.join();
    // cached systems free their memory on the lanes' streams: destroy them first
    for (auto &kv : S->cache)
        kv.second.destroy();
    for (cudaStream_t st : S->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    delete S;
}
