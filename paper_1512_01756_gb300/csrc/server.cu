// Serving runtime: asynchronous Poisson / Helmholtz solve requests on one GPU.
//
// smpm_submit() queues a request (grid, order, k^2, f, g, tol, u) and returns a
// ticket at once; smpm_poll() reports whether it is done.  Worker threads, each
// with its own CUDA stream, take the oldest pending request together with the
// other pending requests on the same grid, order and tolerance (any k^2),
// build one multi-operator handle for their k^2 values and run all of them in
// one batched solve (every request keeps its own Krylov space and convergence
// test; the batch's kernel launches cover all of them).  Requests that arrive
// while batches are on the GPU wait in the queue and are taken by the next
// free worker, so their work overlaps with the batches already running (one
// stream per worker).  Admission: a batch starts only if its estimated device
// footprint (operators + Krylov bases + work vectors) fits the server's byte
// budget next to the batches in flight.
//
// Operator cache: a batch of a single k^2 keeps its handle (operators, Krylov
// basis, workspace) on the device after the solve, keyed by the grid options
// and k^2; a later batch with the same key reuses it without setup.  Cached
// handles are idle (bound to the legacy stream), least recently used first
// out when their bytes exceed a quarter of the budget.
//
// The server is layered on the public entry points (smpm_setup_multi,
// smpm_solve_multi, smpm_last_residuals, smpm_set_stream); all solver
// arithmetic is theirs.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/smpm.h"
#include "smpm_internal.h"

namespace smpm {
void set_last_error(const std::string& msg);
}

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    unsigned long long id = 0;
    smpm_grid grid{};
    double k2 = 0.0, tol = 1e-10;
    const double* f = nullptr;
    const double* g = nullptr;
    double* u = nullptr;
    double t_submit = 0.0, t_done = 0.0;
    bool done = false;
    smpm_stats st{};
    std::string err;   // the worker's error message of a failed request
};

bool same_problem(const Request& a, const Request& b) {
    const smpm_grid &x = a.grid, &y = b.grid;
    return x.mx == y.mx && x.mz == y.mz && x.order == y.order && x.lx == y.lx && x.lz == y.lz &&
           x.z_ratio == y.z_ratio && x.tau_scale == y.tau_scale && x.deflation_groups == y.deflation_groups &&
           x.restart == y.restart && x.max_iter == y.max_iter && x.precision == y.precision && x.krylov == y.krylov &&
           a.tol == b.tol;
}

// Device bytes of a batch: operators per k^2 (slot inverses, G, block-Jacobi
// inverses, the mirror-form halves of the interior ones and of the slots,
// coarse operator)
// plus, per right-hand side, the Krylov basis and the work vectors of the solve.
long long footprint(const smpm_grid& g, int nop, int R) {
    const long long n = g.order + 1, fz = n * g.mz, nfz = n * fz, mx = g.mx;
    const long long d = (long long)(mx - 1) * (g.deflation_groups ? g.mz : 1);
    const long long m = g.restart > 0 ? g.restart : 64;
    const long long ld = 2 * fz * mx + fz + 32, r = nfz * mx;
    const long long op = 3 * (3 * n * fz * fz) + 3 * 4 * fz * fz + 4 * 16 * fz * fz + 10 * fz * fz + d * d + 6 * 4 * fz;
    const long long per_rhs = (m + 1) * ld * (g.precision == 1 ? 2 : 1) + 12 * ld + 8 * r + 3 * (m + 2) * ((2 * fz * mx + 1023) / 1024);
    return 8 * (nop * op + (long long)R * per_rhs) + (64LL << 20);
}

struct CacheEntry {
    Request key;          // grid options, tol unused
    smpm_handle h = nullptr;
    long long bytes = 0;
};

bool same_operator(const Request& a, const Request& b) {
    Request x = a, y = b;
    x.tol = y.tol = 0.0;
    return same_problem(x, y) && a.k2 == b.k2;
}

struct Server {
    int device = 0;
    int max_batch = 16;
    long long budget = 0, inflight = 0;
    std::deque<CacheEntry> cache;          // front = most recently used
    long long cache_bytes = 0;
    long long cache_hits = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request*> pending;
    std::map<unsigned long long, std::unique_ptr<Request>> all;
    std::vector<std::thread> workers;
    std::atomic<unsigned long long> next_id{1};
    bool stop = false;

    void worker_loop() {
        cudaSetDevice(device);
        cudaStream_t stream = nullptr;
        cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
        double *fb = nullptr, *gb = nullptr, *ub = nullptr;
        size_t cap_f = 0, cap_g = 0;
        for (;;) {
            std::vector<Request*> batch;
            long long est = 0;
            {
                std::unique_lock<std::mutex> lk(mu);
                for (;;) {
                    if (stop && pending.empty()) goto out;
                    // the oldest request whose batch fits the budget leads a batch of
                    // the pending requests that share its grid options and tol
                    std::vector<const Request*> tried;
                    for (size_t lead = 0; lead < pending.size() && batch.empty(); ++lead) {
                        Request* r0 = pending[lead];
                        bool seen = false;
                        for (const Request* t : tried) seen = seen || same_problem(*t, *r0);
                        if (seen) continue;
                        tried.push_back(r0);
                        std::vector<size_t> take{lead};
                        for (size_t i = lead + 1; i < pending.size() && (int)take.size() < max_batch; ++i)
                            if (same_problem(*pending[i], *r0)) take.push_back(i);
                        std::vector<double> ks;
                        for (size_t i : take) ks.push_back(pending[i]->k2);
                        std::sort(ks.begin(), ks.end());
                        const int nop = (int)(std::unique(ks.begin(), ks.end()) - ks.begin());
                        est = footprint(r0->grid, nop, (int)take.size());
                        if (inflight == 0 || inflight + cache_bytes + est <= budget) {   // admission by device footprint
                            for (size_t q = take.size(); q-- > 0;) {
                                batch.insert(batch.begin(), pending[take[q]]);
                                pending.erase(pending.begin() + (long)take[q]);
                            }
                            inflight += est;
                        }
                    }
                    if (!batch.empty()) break;
                    cv.wait(lk);
                }
            }
            smpm::NvtxRange nvtx_range("smpm served batch");
            // order the batch by k^2 so that operator indices are non-decreasing
            std::stable_sort(batch.begin(), batch.end(), [](const Request* a, const Request* b) { return a->k2 < b->k2; });
            std::vector<double> k2s;
            std::vector<int> ops;
            for (Request* q : batch) {
                if (k2s.empty() || k2s.back() != q->k2) k2s.push_back(q->k2);
                ops.push_back((int)k2s.size() - 1);
            }
            const int R = (int)batch.size();
            const smpm_grid grid = batch[0]->grid;
            smpm_handle h = nullptr;
            bool hit = false;
            if (k2s.size() == 1) {
                std::lock_guard<std::mutex> lk(mu);
                for (auto it = cache.begin(); it != cache.end(); ++it)
                    if (same_operator(it->key, *batch[0])) {
                        h = it->h;
                        cache_bytes -= it->bytes;
                        cache.erase(it);
                        hit = true;
                        ++cache_hits;
                        break;
                    }
            }
            int rc = SMPM_OK;
            if (hit)
                rc = smpm_set_stream(h, stream);
            else
                rc = smpm_setup_multi(&grid, (int)k2s.size(), k2s.data(), stream, &h);
            long long r = 0, nb = 0, kk = 0;
            smpm_stats st{};
            std::vector<double> res(R, 0.0);
            if (rc == SMPM_OK) rc = smpm_sizes(h, &r, &nb, &kk);
            if (rc == SMPM_OK) {
                const bool any_g = std::any_of(batch.begin(), batch.end(), [](const Request* q) { return q->g; });
                const size_t need_f = (size_t)R * r, need_g = any_g ? (size_t)R * nb : 0;
                // staging buffers grow on the worker's stream (stream-ordered, no device-wide sync)
                if (need_f > cap_f) {
                    if (fb) cudaFreeAsync(fb, stream);
                    if (ub) cudaFreeAsync(ub, stream);
                    fb = ub = nullptr;
                    cap_f = 0;
                    if (cudaMallocAsync(&fb, need_f * 8, stream) != cudaSuccess ||
                        cudaMallocAsync(&ub, need_f * 8, stream) != cudaSuccess) {
                        cudaGetLastError();
                        rc = SMPM_ENOMEM;
                    } else {
                        cap_f = need_f;
                    }
                }
                if (rc == SMPM_OK && need_g > cap_g) {
                    if (gb) cudaFreeAsync(gb, stream);
                    gb = nullptr;
                    cap_g = 0;
                    if (cudaMallocAsync(&gb, need_g * 8, stream) != cudaSuccess) {
                        cudaGetLastError();
                        rc = SMPM_ENOMEM;
                    } else {
                        cap_g = need_g;
                    }
                }
                if (rc == SMPM_ENOMEM) smpm::set_last_error("serving: staging buffer allocation failed");
                if (rc == SMPM_OK) {
                    for (int i = 0; i < R; ++i) {
                        cudaMemcpyAsync(fb + (size_t)i * r, batch[i]->f, r * 8, cudaMemcpyDefault, stream);
                        if (any_g) {
                            if (batch[i]->g)
                                cudaMemcpyAsync(gb + (size_t)i * nb, batch[i]->g, nb * 8, cudaMemcpyDefault, stream);
                            else
                                cudaMemsetAsync(gb + (size_t)i * nb, 0, nb * 8, stream);
                        }
                    }
                    rc = smpm_solve_multi(h, R, ops.data(), fb, any_g ? gb : nullptr, batch[0]->tol, ub, &st);
                    if (rc == SMPM_OK || rc == SMPM_ENOCONV) {
                        smpm_last_residuals(h, R, res.data());
                        for (int i = 0; i < R; ++i)
                            cudaMemcpyAsync(batch[i]->u, ub + (size_t)i * r, r * 8, cudaMemcpyDefault, stream);
                        cudaStreamSynchronize(stream);
                    }
                }
            }
            const std::string err = (rc == SMPM_OK || rc == SMPM_ENOCONV) ? std::string() : std::string(smpm_last_error());
            if (h) {
                // keep a single-k^2 handle for later batches (idle, on the legacy stream)
                bool kept = false;
                if (k2s.size() == 1 && (rc == SMPM_OK || rc == SMPM_ENOCONV) && smpm_set_stream(h, nullptr) == SMPM_OK) {
                    CacheEntry e;
                    e.key = *batch[0];
                    e.h = h;
                    e.bytes = smpm_device_bytes(h);
                    std::vector<smpm_handle> evict;
                    {
                        std::lock_guard<std::mutex> lk(mu);
                        if (e.bytes <= budget / 4) {
                            cache.push_front(e);
                            cache_bytes += e.bytes;
                            kept = true;
                            while (cache_bytes > budget / 4 && !cache.empty()) {
                                cache_bytes -= cache.back().bytes;
                                evict.push_back(cache.back().h);
                                cache.pop_back();
                            }
                        }
                    }
                    for (smpm_handle x : evict) smpm_release(x);
                }
                if (!kept) smpm_release(h);
            }
            const double t = now_ms();
            {
                std::lock_guard<std::mutex> lk(mu);
                inflight -= est;
                for (int i = 0; i < R; ++i) {
                    Request* q = batch[i];
                    q->st = st;
                    if (hit) q->st.setup_ms = 0.0;     // operators taken from the cache
                    q->st.status = rc;
                    q->st.rel_resid_true = res[i];
                    q->st.solve_ms = t - q->t_submit;      // latency: completion - submission
                    q->st.restarts = R;                    // batch size the request ran in
                    q->t_done = t;
                    q->err = err;
                    q->done = true;
                }
            }
            cv.notify_all();
        }
    out:
        if (fb) cudaFreeAsync(fb, stream);
        if (gb) cudaFreeAsync(gb, stream);
        if (ub) cudaFreeAsync(ub, stream);
        cudaStreamSynchronize(stream);
        cudaStreamDestroy(stream);
    }
};

}  // namespace

extern "C" {

int smpm_server_create(int nworkers, long long device_budget_bytes, int max_batch, smpm_server_t* out) {
    if (!out || nworkers < 1 || nworkers > 64 || max_batch < 1) {
        smpm::set_last_error("smpm_server_create: need 1 <= nworkers <= 64, max_batch >= 1");
        return SMPM_EINVAL;
    }
    auto* s = new Server();
    cudaGetDevice(&s->device);
    s->max_batch = max_batch;
    if (device_budget_bytes <= 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        device_budget_bytes = (long long)(fr * 0.8);
    }
    s->budget = device_budget_bytes;
    // keep freed operator and Krylov memory in the device pool between batches
    // (up to the budget) instead of releasing it to the system at every sync
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess) {
        unsigned long long keep = (unsigned long long)device_budget_bytes;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    for (int i = 0; i < nworkers; ++i) s->workers.emplace_back([s] { s->worker_loop(); });
    *out = reinterpret_cast<smpm_server_t>(s);
    return SMPM_OK;
}

int smpm_submit(smpm_server_t srv, const smpm_grid* grid, double k2, const double* f, const double* g, double tol,
                double* u, unsigned long long* ticket) {
    auto* s = reinterpret_cast<Server*>(srv);
    if (!s || !grid || !f || !u || !ticket || !(tol > 0.0) || !(k2 >= 0.0)) {
        smpm::set_last_error("smpm_submit: bad argument");
        return SMPM_EINVAL;
    }
    if (grid->krylov != 0) {   // a batch joins unrelated requests: each keeps its own Krylov space
        smpm::set_last_error("smpm_submit: krylov must be 0 for served requests");
        return SMPM_EINVAL;
    }
    auto q = std::make_unique<Request>();
    q->id = s->next_id++;
    q->grid = *grid;
    q->k2 = k2; q->tol = tol; q->f = f; q->g = g; q->u = u;
    q->t_submit = now_ms();
    *ticket = q->id;
    // admission: a request whose footprint alone exceeds the budget can never
    // run; it is refused at once and reported by smpm_poll
    const long long est = footprint(*grid, 1, 1);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            smpm::set_last_error("smpm_submit: server is shutting down");
            return SMPM_EINVAL;
        }
        if (est > s->budget) {
            q->st.status = SMPM_ENOMEM;
            q->err = "serving: request footprint " + std::to_string(est) + " bytes exceeds the device budget of " +
                     std::to_string(s->budget) + " bytes";
            q->t_done = q->t_submit;
            q->done = true;
            s->all[q->id] = std::move(q);
            return SMPM_OK;
        }
        s->pending.push_back(q.get());
        s->all[q->id] = std::move(q);
    }
    s->cv.notify_all();
    return SMPM_OK;
}

int smpm_poll(smpm_server_t srv, unsigned long long ticket, smpm_stats* st) {
    auto* s = reinterpret_cast<Server*>(srv);
    if (!s) return SMPM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) {
        smpm::set_last_error("smpm_poll: unknown ticket");
        return SMPM_EINVAL;
    }
    if (!it->second->done) return SMPM_EBUSY;
    if (st) *st = it->second->st;
    const int rc = it->second->st.status;
    if (rc != SMPM_OK) smpm::set_last_error(it->second->err);
    s->all.erase(it);
    return rc;
}

int smpm_request_footprint(const smpm_grid* grid, int nop, int nrhs, long long* bytes) {
    if (!grid || !bytes || nop < 1 || nrhs < 1) {
        smpm::set_last_error("smpm_request_footprint: bad argument");
        return SMPM_EINVAL;
    }
    *bytes = footprint(*grid, nop, nrhs);
    return SMPM_OK;
}

int smpm_server_destroy(smpm_server_t srv) {
    auto* s = reinterpret_cast<Server*>(srv);
    if (!s) return SMPM_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    for (auto& t : s->workers) t.join();
    for (CacheEntry& e : s->cache) smpm_release(e.h);
    delete s;
    return SMPM_OK;
}

}  // extern "C"
