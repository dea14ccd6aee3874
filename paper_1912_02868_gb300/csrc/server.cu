// Solve server: continuous batching of requests over many gauge configurations
// on one GPU (the serving pattern layered on the method of Section 2).
//
// * A request is (key, operator description, right-hand sides, tolerance).  The
//   key names an operator; its hierarchy and coarse deflation space are built
//   on first use and kept resident (an LRU cache under an HBM byte budget).
// * Work is split into one item per right-hand side.  A pool of worker
//   threads takes items in arrival order; each runs on a solve context of the
//   item's hierarchy (own workspaces and CUDA stream), so items of different
//   requests and different lattice sizes overlap on the device, and a request
//   that arrives while others run is admitted as soon as a worker and, for a
//   new key, memory are free.
// * With a block precision (MG_MIXED_BF16 / MG_MIXED_FP16) a key runs one
//   lockstep block solve at a time on its hierarchy: the worker that takes an
//   item also takes every queued item of the same key and tolerance, up to
//   rhs_block, from any request, and solves them together (tensor-core block
//   products).  Items that arrive while a block runs join the next block.
// * The deflation space of a new key is built by GMRES-DR on a fixed seeded
//   right-hand side (not on a request's), so every later solve of that key -
//   alone or in any mix - runs the same arithmetic and gives the same result.
// * Nothing here waits on the device except through the library's own calls;
//   every wait on the host is a condition variable tied to a queue change.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "handle.cuh"

namespace mg {

namespace {

using clk = std::chrono::steady_clock;

struct Request {
    mg_request r{};
    unsigned long long ticket = 0;
    clk::time_point t_submit, t_done;
    int remaining = 0;
    std::vector<int> iters;
    std::vector<double> relres;
    mg_status status = MG_OK;
    std::string error;
    bool done = false;
};

struct Entry {
    unsigned long long key = 0;
    int Lx = 0, Lt = 0;
    mg_handle owner = nullptr;
    cudaStream_t ostream = nullptr;    // the owner's stream (contexts have their own)
    std::vector<mg_handle> free_ctx;   // idle solve contexts (the owner is one of them once ready)
    std::vector<mg_handle> all_ctx;    // contexts other than the owner
    size_t bytes = 0;
    bool ready = false;                // hierarchy and deflation space built
    bool building = false;
    bool failed = false;
    int active = 0;                    // items running on this entry
    unsigned long long last_use = 0;
};

struct Item {
    std::shared_ptr<Request> req;
    int rhs;
};

// device staging of a block gathered from several requests (one per worker)
struct Staging {
    double2* b = nullptr;
    double2* x = nullptr;
    size_t cap = 0;  // bytes of each buffer
};

}  // namespace

struct Server {
    mg_params p{};
    size_t budget = 0;
    int nworkers = 1;
    bool block = false;  // lockstep block solves (block precisions)
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Item> queue;
    std::map<unsigned long long, std::shared_ptr<Request>> reqs;
    std::map<unsigned long long, std::unique_ptr<Entry>> cache;
    std::vector<std::thread> workers;
    bool stop = false;
    unsigned long long next_ticket = 1, tick = 0;
    size_t bytes = 0;
    long long evictions = 0, completed = 0, cold_starts = 0, batches = 0;
    std::map<unsigned long long, size_t> demand;  // estimated bytes of every key ever requested
    int max_batch = 0;
    int device = 0;

    void worker_loop();
    bool pick(std::vector<Item>& batch, Entry*& e, mg_handle& ctx, bool& cold, bool& new_ctx);
    void take_more(std::vector<Item>& batch);
    void evict_for(size_t need);
    void finish_batch(const std::vector<Item>& batch, Entry* e, mg_handle ctx, const int* iters,
                      const double* relres, mg_status st, const std::string& err);
    mg_status solve_batch(const std::vector<Item>& batch, Entry* e, mg_handle ctx, Staging& stg, int* iters,
                          double* relres);
};

namespace {

// canonical right-hand side that builds the deflation space of a new key
void seeded_rhs(std::vector<double>& v, long ncomplex, unsigned long long key) {
    v.resize(2 * ncomplex);
    auto mix = [](unsigned long long z) {
        z += 0x9E3779B97F4A7C15ULL;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    };
    const unsigned long long k0 = mix(key ^ 0xD3F1A7ULL);
    for (long i = 0; i < ncomplex; ++i) {
        const double u1 = ((double)(mix(k0 ^ mix(2 * i)) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        const double u2 = ((double)(mix(k0 ^ mix(2 * i + 1)) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        const double rad = std::sqrt(-std::log(u1));
        v[2 * i] = rad * std::cos(6.283185307179586 * u2);
        v[2 * i + 1] = rad * std::sin(6.283185307179586 * u2);
    }
}

size_t estimate_bytes(const mg_params& p, int Lx, int Lt) {
    // hierarchy (FP64 + FP32 copies) + one set of workspaces, rounded up
    const double s0 = (double)Lx * Lt, s1 = s0 / 16, s2 = s0 / 256;
    const double hier = 24.0 * s0 * 2 + (5 * 576 * 24.0) * (s1 + s2) + 24.0 * 24 * 16 * (s1 + s2 * 12);
    double ws = 16.0 * 2 * s0 * (2 * p.fgmres_m + 12) + 16.0 * 24 * s1 * 12 + 16.0 * 24 * s2 * 4 * (p.dr_m + 1);
    if (p.precision == MG_MIXED_BF16 || p.precision == MG_MIXED_FP16) {
        // lockstep block workspaces for rhs_block right-hand sides (rounded up to 8):
        // FP64 FGMRES basis and vectors, FP32 V-cycle vectors, the coarse bases, and
        // the 16-bit operator copies of the two coarse grids
        const double nbp = 8.0 * ((p.rhs_block + 7) / 8);
        const double per = 16.0 * 2 * s0 * (2 * p.fgmres_m + 4) + 8.0 * 2 * s0 * 2 + 8.0 * 24 * s1 * (p.smooth_steps + 4) +
                           8.0 * 24 * s2 * (p.dr_m + 4);
        ws += nbp * per + 4.0 * 5 * 576 * (s1 + s2);
    }
    return (size_t)((hier + ws) * 1.15) + (8u << 20);
}

}  // namespace

void Server::evict_for(size_t need) {
    // least recently used idle entries first
    while (budget && bytes + need > budget) {
        Entry* victim = nullptr;
        for (auto& kv : cache) {
            Entry* e = kv.second.get();
            if (e->active || e->building || !e->ready) continue;
            if (e->free_ctx.size() != e->all_ctx.size() + 1) continue;
            if (!victim || e->last_use < victim->last_use) victim = e;
        }
        if (!victim) return;
        for (mg_handle c : victim->all_ctx) mg_destroy(c);
        mg_destroy(victim->owner);
        if (victim->ostream) cudaStreamDestroy(victim->ostream);
        bytes -= std::min(bytes, victim->bytes);
        ++evictions;
        cache.erase(victim->key);
    }
}

// Under the lock, block mode: append to `batch` the queued items of the same key
// and tolerance as batch[0], in arrival order, up to rhs_block items.
void Server::take_more(std::vector<Item>& batch) {
    const mg_request& r0 = batch[0].req->r;
    for (auto q = queue.begin(); q != queue.end() && (int)batch.size() < p.rhs_block;) {
        const mg_request& r = q->req->r;
        if (r.key == r0.key && r.tol == r0.tol) {
            batch.push_back(*q);
            q = queue.erase(q);
        } else {
            ++q;
        }
    }
}

// Under the lock: the first queued item that can run now (in block mode with
// the queued items that join it).  On success the items are removed from the
// queue and, unless `cold` or `new_ctx`, ctx is an idle context of e.
bool Server::pick(std::vector<Item>& batch, Entry*& e, mg_handle& ctx, bool& cold, bool& new_ctx) {
    for (auto q = queue.begin(); q != queue.end(); ++q) {
        const mg_request& r = q->req->r;
        auto f = cache.find(r.key);
        cold = new_ctx = false;
        ctx = nullptr;
        if (f == cache.end()) {
            const size_t need = estimate_bytes(p, r.L_x, r.L_t);
            if (budget && bytes + need > budget) evict_for(need);
            if (budget && bytes + need > budget && !cache.empty()) continue;  // wait for memory
            auto ne = std::make_unique<Entry>();
            ne->key = r.key;
            ne->Lx = r.L_x;
            ne->Lt = r.L_t;
            ne->building = true;
            ne->bytes = need;
            e = ne.get();
            bytes += need;
            cache[r.key] = std::move(ne);
            cold = true;
        } else {
            e = f->second.get();
            if (e->failed) {
                cold = false;
            } else if (e->building) {
                continue;
            } else if (!e->free_ctx.empty()) {
                ctx = e->free_ctx.back();
                e->free_ctx.pop_back();
            } else if (!block && (int)e->all_ctx.size() + 1 < nworkers) {
                const size_t need = estimate_bytes(p, e->Lx, e->Lt) / 4;
                if (budget && bytes + need > budget) evict_for(need);
                if (budget && bytes + need > budget) continue;
                new_ctx = true;
            } else {
                continue;
            }
        }
        batch.assign(1, *q);
        queue.erase(q);
        if (block && !cold && !e->failed) take_more(batch);
        e->active += 1;
        e->last_use = ++tick;
        return true;
    }
    return false;
}

void Server::finish_batch(const std::vector<Item>& batch, Entry* e, mg_handle ctx, const int* iters,
                          const double* relres, mg_status st, const std::string& err) {
    std::lock_guard<std::mutex> lk(mu);
    if (ctx) e->free_ctx.push_back(ctx);
    e->active -= 1;
    ++batches;
    max_batch = std::max(max_batch, (int)batch.size());
    if (block && e->owner) {  // the block workspaces are allocated by the first block solve
        const size_t now = handle_device_bytes(e->owner);
        if (now > e->bytes) {
            bytes += now - e->bytes;
            e->bytes = now;
        }
    }
    for (size_t i = 0; i < batch.size(); ++i) {
        const Item& it = batch[i];
        Request& R = *it.req;
        R.iters[it.rhs] = iters[i];
        R.relres[it.rhs] = relres[i];
        if (st != MG_OK && R.status == MG_OK) {
            R.status = st;
            R.error = err;
        }
        if (--R.remaining == 0) {
            R.t_done = clk::now();
            R.done = true;
            ++completed;
            cv_done.notify_all();
        }
    }
    cv_work.notify_all();
}

// Solve the items of `batch` (one key, one tolerance) on ctx.  Consecutive
// right-hand sides of one request are solved in place; a block gathered from
// several requests goes through the worker's device staging buffers.
mg_status Server::solve_batch(const std::vector<Item>& batch, Entry* e, mg_handle ctx, Staging& stg, int* iters,
                              double* relres) {
    const mg_request& r0 = batch[0].req->r;
    const long n0 = (long)r0.L_x * r0.L_t * 2;  // complex entries of one right-hand side
    const int nb = (int)batch.size();
    cudaStream_t cs = (ctx == e->owner) ? e->ostream : handle_stream(ctx);
    bool contiguous = true;
    for (int i = 1; i < nb; ++i)
        contiguous = contiguous && batch[i].req == batch[0].req && batch[i].rhs == batch[0].rhs + i;
    if (contiguous) {
        const double2* b = static_cast<const double2*>(r0.b) + (long)batch[0].rhs * n0;
        double2* x = static_cast<double2*>(r0.x) + (long)batch[0].rhs * n0;
        return mg_solve(ctx, b, x, nb, r0.tol, cs, iters, relres, nullptr);
    }
    const size_t need = (size_t)nb * n0 * sizeof(double2);
    if (stg.cap < need) {
        if (stg.b) cudaFree(stg.b);
        if (stg.x) cudaFree(stg.x);
        stg.b = stg.x = nullptr;
        {
            std::lock_guard<std::mutex> lk(mu);
            bytes -= std::min(bytes, 2 * stg.cap);
        }
        stg.cap = 0;
        if (cudaMalloc(&stg.b, need) != cudaSuccess || cudaMalloc(&stg.x, need) != cudaSuccess) {
            (void)cudaGetLastError();
            if (stg.b) cudaFree(stg.b);
            stg.b = nullptr;
            return set_error("out of device memory for a block of %d right-hand sides", nb), MG_ENOMEM;
        }
        stg.cap = need;
        std::lock_guard<std::mutex> lk(mu);
        bytes += 2 * need;
    }
    const size_t vb = (size_t)n0 * sizeof(double2);
    for (int i = 0; i < nb; ++i) {
        const mg_request& r = batch[i].req->r;
        MG_CUDA_TRY(cudaMemcpyAsync(stg.b + (long)i * n0, static_cast<const double2*>(r.b) + (long)batch[i].rhs * n0,
                                    vb, cudaMemcpyDefault, cs));
    }
    mg_status st = mg_solve(ctx, stg.b, stg.x, nb, r0.tol, cs, iters, relres, nullptr);
    if (st != MG_OK && st != MG_ENOTCONV) return st;
    for (int i = 0; i < nb; ++i) {
        const mg_request& r = batch[i].req->r;
        MG_CUDA_TRY(cudaMemcpyAsync(static_cast<double2*>(r.x) + (long)batch[i].rhs * n0, stg.x + (long)i * n0, vb,
                                    cudaMemcpyDefault, cs));
    }
    MG_CUDA_TRY(cudaStreamSynchronize(cs));
    return st;
}

void Server::worker_loop() {
    cudaSetDevice(device);
    Staging stg;
    while (true) {
        std::vector<Item> batch;
        Entry* e = nullptr;
        mg_handle ctx = nullptr;
        bool cold = false, new_ctx = false;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] { return stop || (!queue.empty() && pick(batch, e, ctx, cold, new_ctx)); });
            if (stop && batch.empty()) break;
        }
        const mg_request& r = batch[0].req->r;
        mg_status st = MG_OK;
        std::string err;
        if (cold) {
            // build the hierarchy and its deflation space (seeded right-hand side)
            mg_handle h = nullptr;
            mg_params pp = p;
            pp.parallel = 1;
            cudaStream_t os = nullptr;
            if (cudaStreamCreateWithFlags(&os, cudaStreamNonBlocking) != cudaSuccess) {
                (void)cudaGetLastError();
                os = nullptr;
                st = MG_ECUDA;
                err = "cudaStreamCreate failed";
            }
            if (st == MG_OK)
                st = mg_setup(r.gauge, r.L_x, r.L_t, r.m0, pp.nvec, pp.block, &pp, r.starts0, r.starts1, os, &h);
            if (st == MG_OK) {
                std::vector<double> bw;
                const long n0 = (long)r.L_x * r.L_t * 2;
                seeded_rhs(bw, n0, r.key);
                std::vector<double> xw(2 * n0);
                int itw = 0;
                double rrw = 0;
                st = mg_solve(h, bw.data(), xw.data(), 1, 1e-8, os, &itw, &rrw, nullptr);
                if (st == MG_ENOTCONV) st = MG_OK;
            }
            if (st != MG_OK && err.empty()) err = mg_last_error();
            std::lock_guard<std::mutex> lk(mu);
            e->building = false;
            ++cold_starts;
            if (st == MG_OK) {
                e->owner = h;
                e->ostream = os;
                e->ready = true;
                bytes -= std::min(bytes, e->bytes);
                e->bytes = handle_device_bytes(h);
                bytes += e->bytes;
                ctx = h;  // run this item on the owner
                if (block) take_more(batch);  // and the items of this key that queued meanwhile
            } else {
                if (h) mg_destroy(h);
                if (os) cudaStreamDestroy(os);
                e->failed = true;
            }
            cv_work.notify_all();
        } else if (new_ctx) {
            mg_handle c = nullptr;
            st = make_solve_context(e->owner, &c);
            if (st != MG_OK) err = mg_last_error();
            std::lock_guard<std::mutex> lk(mu);
            if (st == MG_OK) {
                e->all_ctx.push_back(c);
                const size_t cb = handle_device_bytes(c);
                e->bytes += cb;
                bytes += cb;
                ctx = c;
            }
        }
        std::vector<int> iters(batch.size(), 0);
        std::vector<double> relres(batch.size(), INFINITY);
        if (st == MG_OK && e->failed) {
            st = MG_ECUDA;
            err = "the hierarchy of this key could not be built";
        }
        if (st == MG_OK) {
            st = solve_batch(batch, e, ctx, stg, iters.data(), relres.data());
            if (st != MG_OK && st != MG_ENOTCONV) err = mg_last_error();
        }
        finish_batch(batch, e, ctx, iters.data(), relres.data(), st, err);
    }
    if (stg.b) cudaFree(stg.b);
    if (stg.x) cudaFree(stg.x);
    std::lock_guard<std::mutex> lk(mu);
    bytes -= std::min(bytes, 2 * stg.cap);
}

}  // namespace mg

using namespace mg;

struct mg_server_s {
    Server s;
};

extern "C" {

mg_status mg_server_create(const mg_params* p, unsigned long long hbm_budget_bytes, int workers, mg_server* out) {
    if (!out) return set_error("out is NULL"), MG_EINVAL;
    *out = nullptr;
    if (workers < 1 || workers > 256) return set_error("workers must be in [1, 256]"), MG_EINVAL;
    mg_server_s* sv = new (std::nothrow) mg_server_s();
    if (!sv) return set_error("out of host memory"), MG_ENOMEM;
    Server& S = sv->s;
    mg_default_params(&S.p);
    if (p) S.p = *p;
    S.budget = (size_t)hbm_budget_bytes;
    S.nworkers = workers;
    S.block = S.p.precision == MG_MIXED_BF16 || S.p.precision == MG_MIXED_FP16;
    if (cudaGetDevice(&S.device) != cudaSuccess) {
        delete sv;
        return set_error("no CUDA device"), MG_ECUDA;
    }
    for (int w = 0; w < workers; ++w) S.workers.emplace_back([&S] { S.worker_loop(); });
    *out = sv;
    return MG_OK;
}

mg_status mg_server_submit(mg_server sv, const mg_request* r, unsigned long long* ticket) {
    if (!sv || !r || !ticket) return set_error("NULL argument"), MG_EINVAL;
    if (!r->gauge || !r->b || !r->x || r->nrhs < 1) return set_error("request needs gauge, b, x, nrhs >= 1"), MG_EINVAL;
    if (r->L_x < 16 || r->L_t < 16 || r->L_x % 16 || r->L_t % 16)
        return set_error("lattice extents must be positive multiples of 16"), MG_EINVAL;
    if (!(r->tol > 0.0 && r->tol < 1.0)) return set_error("tol must be in (0, 1)"), MG_EINVAL;
    Server& S = sv->s;
    auto R = std::make_shared<Request>();
    R->r = *r;
    R->t_submit = clk::now();
    R->remaining = r->nrhs;
    R->iters.assign(r->nrhs, 0);
    R->relres.assign(r->nrhs, INFINITY);
    {
        std::lock_guard<std::mutex> lk(S.mu);
        if (S.stop) return set_error("server is shutting down"), MG_EINVAL;
        R->ticket = S.next_ticket++;
        S.reqs[R->ticket] = R;
        for (int i = 0; i < r->nrhs; ++i) S.queue.push_back(Item{R, i});
        S.demand[r->key] = estimate_bytes(S.p, r->L_x, r->L_t);
        *ticket = R->ticket;
    }
    S.cv_work.notify_all();
    return MG_OK;
}

mg_status mg_server_wait(mg_server sv, unsigned long long ticket, int* iters, double* relres, double* latency_s) {
    if (!sv) return set_error("server is NULL"), MG_EINVAL;
    Server& S = sv->s;
    std::shared_ptr<Request> R;
    {
        std::unique_lock<std::mutex> lk(S.mu);
        auto f = S.reqs.find(ticket);
        if (f == S.reqs.end()) return set_error("unknown ticket %llu", ticket), MG_EINVAL;
        R = f->second;
        S.cv_done.wait(lk, [&] { return R->done; });
        S.reqs.erase(ticket);
    }
    for (int i = 0; i < R->r.nrhs; ++i) {
        if (iters) iters[i] = R->iters[i];
        if (relres) relres[i] = R->relres[i];
    }
    if (latency_s) latency_s[0] = std::chrono::duration<double>(R->t_done - R->t_submit).count();
    if (R->status != MG_OK && R->status != MG_ENOTCONV) set_error("%s", R->error.c_str());
    if (R->status == MG_ENOTCONV) set_error("some right-hand side reached max_outer");
    return R->status;
}

mg_status mg_server_poll(mg_server sv, unsigned long long ticket, int* done, int* iters, double* relres,
                         double* latency_s) {
    if (!sv || !done) return set_error("server or done is NULL"), MG_EINVAL;
    Server& S = sv->s;
    {
        std::lock_guard<std::mutex> lk(S.mu);
        auto f = S.reqs.find(ticket);
        if (f == S.reqs.end()) return set_error("unknown ticket %llu", ticket), MG_EINVAL;
        if (!f->second->done) {
            *done = 0;
            return MG_OK;
        }
    }
    *done = 1;
    return mg_server_wait(sv, ticket, iters, relres, latency_s);
}

mg_status mg_server_stats(mg_server sv, mg_server_info* out) {
    if (!sv || !out) return set_error("NULL argument"), MG_EINVAL;
    Server& S = sv->s;
    std::lock_guard<std::mutex> lk(S.mu);
    out->resident_keys = (int)S.cache.size();
    out->device_bytes = (unsigned long long)S.bytes;
    out->evictions = S.evictions;
    out->cold_starts = S.cold_starts;
    out->completed = S.completed;
    out->queued_items = (long long)S.queue.size();
    out->batches = S.batches;
    unsigned long long d = 0;
    for (const auto& kv : S.demand) d += kv.second;
    out->demand_bytes = d;
    out->max_batch = S.max_batch;
    return MG_OK;
}

mg_status mg_server_destroy(mg_server sv) {
    if (!sv) return MG_OK;
    Server& S = sv->s;
    {
        std::lock_guard<std::mutex> lk(S.mu);
        S.stop = true;
        S.queue.clear();
    }
    S.cv_work.notify_all();
    for (auto& t : S.workers) t.join();
    for (auto& kv : S.cache) {
        for (mg_handle c : kv.second->all_ctx) mg_destroy(c);
        if (kv.second->owner) mg_destroy(kv.second->owner);
        if (kv.second->ostream) cudaStreamDestroy(kv.second->ostream);
    }
    {
        std::lock_guard<std::mutex> lk(S.mu);
        for (auto& kv : S.reqs) kv.second->done = true;
    }
    S.cv_done.notify_all();
    delete sv;
    return MG_OK;
}

}  // extern "C"
