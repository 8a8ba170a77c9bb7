// serve.cpp -- a request loop for scattering solves (lfmm_server_* in include/lfmm.h).
// Each request is one solve of the paper's problem (Sec. 2, the system of Sec. 3.3 by
// GMRES with the preconditioner of Sec. 4.2); the loop itself has no counterpart in
// the paper, which solves one problem at a time.
//
// Requests (a layer stack, scatterer elements, an incidence angle, a tolerance,
// the precision, the operator: single layer or combined field) queue in arrival
// order.  `slots` worker threads each drive one CUDA stream; a worker takes the
// request at the head of the queue as soon as the estimated device footprints of
// the requests on the GPU plus this one fit the HBM budget, and builds it on its
// stream: medium, geometry (tree, tables, near field, preconditioner), right-hand
// side.  The solve itself joins the batch engine: one thread that advances every
// admitted solve by one GMRES step per round (lockstep solves, solver.cu), their FP64
// operator products in shared launches (one launch per stage for all of them) and one
// host synchronisation per round; a request joins at the next round after its set-up
// and leaves when it has converged or stopped.  The worker then copies the solution
// to host memory and releases the request.  Requests that arrive while others run
// are admitted as slots and memory free up; set-ups overlap the engine's rounds on
// the device.  A solve in a batch takes the same steps with the same bits as alone
// (solver.cu), so a result is the same alone and in the mix.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/lfmm.h"
#include "geometry.h"

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    int64_t ticket = 0;
    int32_t n_layers = 0;
    std::vector<double> yint, k, eta;
    int64_t n = 0;
    std::vector<double> pts, w, nrm;   // nrm: combined field only
    int32_t flags = 0;
    double angle = 0.0, tol = 1e-8;
    int32_t precision = 0, p = 20, leaf = 64, max_iter = 1000, precond = 1;
    int64_t footprint = 0;
    // results
    std::vector<double> x;   // 2n (re, im)
    lfmm_gmres_info info{};
    lfmm_status status = LFMM_OK;
    std::string err;
    double t_submit = 0, t_admit = 0, t_done = 0, setup_s = 0;
    bool done = false;
    // between set-up and finalisation
    lfmm_medium med = nullptr;
    lfmm_geometry geo = nullptr;
    void* db = nullptr;                  // right-hand side (device, input order)
    lfmm::BatchSolve* bs = nullptr;
    bool solved = false;                 // the engine is done with it (or it failed)
};

}  // namespace

struct lfmm_server_s {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> queue;
    std::unordered_map<int64_t, std::shared_ptr<Request>> tickets;
    int64_t next_ticket = 1;
    int64_t in_use = 0, budget = 0, peak_in_use = 0;
    int running = 0, peak_running = 0;
    bool stop = false;
    int device = 0;
    std::vector<std::thread> workers;
    // the batch engine: solves handed over by the workers, and those it is running
    std::thread engine;
    std::condition_variable cv_engine, cv_solved;
    std::vector<std::shared_ptr<Request>> pending;
    int workers_left = 0;
};

namespace {

// Device bytes one request holds while it runs: the Krylov basis (max_iter + 1
// vectors), the stored near field and preconditioner (~62 and ~50 complex entries
// per point at leaf size 64), the leaf expansion basis (p + 2 complex values per
// point), multipoles/locals and work vectors, and the reaction tables and set-up
// scratch (a fixed allowance).
int64_t footprint_estimate(int64_t n, int p, int leaf, int max_iter) {
    const double per_point = 16.0 * (max_iter + 1) + 16.0 * (1.0 + leaf / 64.0) * 120.0 + 16.0 * 24.0 +
                             16.0 * (p + 2.0);
    const double expansions = 16.0 * (2.0 * p + 1.0) * (double)n / 4.0;
    return (int64_t)(per_point * (double)n + expansions) + ((int64_t)256 << 20);
}

// set-up of a request on its worker's stream: medium, geometry, right-hand side, and the
// solve's state (preconditioner, sorted right-hand side); false on an error (recorded)
bool setup_request(Request& r, cudaStream_t s) {
    const double t0 = now_s();
    auto fail = [&](lfmm_status st) {
        r.status = st;
        r.err = lfmm_last_error();
        return false;
    };
    lfmm_status st = lfmm_medium_create(r.n_layers, r.yint.data(), r.k.data(), r.eta.data(), &r.med);
    if (st < 0) return fail(st);
    lfmm_params prm{r.p, r.leaf, r.flags, 0};
    st = lfmm_geometry_build(r.med, r.n, r.pts.data(), r.w.data(), r.nrm.empty() ? nullptr : r.nrm.data(), &prm,
                             &r.geo);
    if (st < 0) return fail(st);
    if (cudaMallocAsync(&r.db, 16 * (size_t)r.n, s) != cudaSuccess) {
        (void)cudaGetLastError();   // not this worker's next request's error
        r.db = nullptr;
        r.status = LFMM_ERR_OUT_OF_MEMORY;
        r.err = "cudaMallocAsync failed for the request's right-hand side";
        return false;
    }
    st = lfmm_rhs_plane_wave(r.geo, 1, &r.angle, r.db, LFMM_DEVICE_PTRS, s);
    if (st < 0) return fail(st);
    st = lfmm::guarded_call([&]() -> lfmm_status {
        r.bs = lfmm::batch_solve_create(r.geo, (const cd*)r.db, r.tol, r.max_iter, r.precond != 0, r.precision,
                                        s);
        return LFMM_OK;
    });
    if (st < 0) return fail(st);
    r.setup_s = now_s() - t0;
    return true;
}

// the solution to host memory and the release of everything the request holds
void finish_request(Request& r, cudaStream_t s) {
    if (r.bs && r.status >= 0) {
        void* dx = nullptr;
        if (cudaMallocAsync(&dx, 16 * (size_t)r.n, s) != cudaSuccess) {
            (void)cudaGetLastError();
            r.status = LFMM_ERR_OUT_OF_MEMORY;
            r.err = "cudaMallocAsync failed for the request's solution";
        } else {
            const lfmm_status st = lfmm::guarded_call([&]() -> lfmm_status {
                lfmm::batch_solve_finish(r.bs, (cd*)dx, &r.info, s);
                return LFMM_OK;
            });
            if (st < 0) {
                r.status = st;
                r.err = lfmm_last_error();
            } else {
                r.status = r.info.converged ? LFMM_OK : LFMM_NOT_CONVERGED;
                r.x.resize(2 * (size_t)r.n);
                if (cudaMemcpyAsync(r.x.data(), dx, 16 * (size_t)r.n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                    cudaStreamSynchronize(s) != cudaSuccess) {
                    (void)cudaGetLastError();
                    r.status = LFMM_ERR_CUDA;
                    r.err = "copy of the solution failed";
                }
            }
            cudaFreeAsync(dx, s);
        }
    }
    if (r.bs) lfmm::guarded_call([&]() -> lfmm_status { lfmm::batch_solve_destroy(r.bs, s); return LFMM_OK; });
    r.bs = nullptr;
    if (r.db) cudaFreeAsync(r.db, s);
    r.db = nullptr;
    cudaStreamSynchronize(s);
    if (r.geo) lfmm_geometry_destroy(r.geo);
    if (r.med) lfmm_medium_destroy(r.med);
    r.geo = nullptr;
    r.med = nullptr;
}

void worker_main(lfmm_server_s* S) {
    cudaSetDevice(S->device);
    cudaStream_t s = nullptr;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    for (;;) {
        std::shared_ptr<Request> r;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            // admission: the head of the queue, once its footprint fits beside the running ones
            S->cv_work.wait(lk, [&] {
                return (S->stop && S->queue.empty()) ||
                       (!S->queue.empty() && S->in_use + S->queue.front()->footprint <= S->budget);
            });
            if (S->queue.empty()) break;   // stopping, nothing left
            r = S->queue.front();
            S->queue.pop_front();
            S->in_use += r->footprint;
            S->peak_in_use = std::max(S->peak_in_use, S->in_use);
            S->running += 1;
            S->peak_running = std::max(S->peak_running, S->running);
            r->t_admit = now_s();
        }
        try {
            if (setup_request(*r, s)) {
                // hand the solve to the engine and wait for it
                std::unique_lock<std::mutex> lk(S->mu);
                S->pending.push_back(r);
                S->cv_engine.notify_all();
                S->cv_solved.wait(lk, [&] { return r->solved; });
            }
            finish_request(*r, s);
        } catch (const std::bad_alloc&) {   // the host copy of the solution
            r->status = LFMM_ERR_OUT_OF_MEMORY;
            r->err = "host allocation failed";
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            r->t_done = now_s();
            r->done = true;
            S->in_use -= r->footprint;
            S->running -= 1;
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
    if (s) cudaStreamDestroy(s);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->workers_left -= 1;
    }
    S->cv_engine.notify_all();
}

// The batch engine: every round takes the solves handed over since the last one, then
// advances all running solves by one GMRES step together.
void engine_main(lfmm_server_s* S) {
    cudaSetDevice(S->device);
    cudaStream_t s = nullptr;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    std::vector<std::shared_ptr<Request>> active;
    bool released = false;
    auto release = [&](const std::shared_ptr<Request>& r) {
        std::lock_guard<std::mutex> lk(S->mu);
        r->solved = true;
        released = true;
    };
    for (;;) {
        std::vector<std::shared_ptr<Request>> fresh;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_engine.wait(lk, [&] { return !S->pending.empty() || !active.empty() || S->workers_left == 0; });
            if (S->pending.empty() && active.empty()) break;   // every worker has stopped
            fresh.swap(S->pending);
        }
        for (auto& r : fresh) {
            const lfmm_status st = lfmm::guarded_call([&]() -> lfmm_status {
                lfmm::batch_solve_begin(r->bs, s);
                return LFMM_OK;
            });
            if (st < 0) {
                r->status = st;
                r->err = lfmm_last_error();
                release(r);
            } else {
                active.push_back(r);
            }
        }
        std::vector<lfmm::BatchSolve*> round;
        for (auto& r : active) round.push_back(r->bs);
        const lfmm_status st = lfmm::guarded_call([&]() -> lfmm_status {
            lfmm::batch_solve_round(round, s);
            return LFMM_OK;
        });
        std::vector<std::shared_ptr<Request>> keep;
        for (auto& r : active) {
            if (st < 0) {   // the round failed: every solve in it reports the error
                r->status = st;
                r->err = lfmm_last_error();
                release(r);
            } else if (lfmm::batch_solve_done(r->bs)) {
                release(r);
            } else {
                keep.push_back(r);
            }
        }
        if (released) S->cv_solved.notify_all();
        released = false;
        active.swap(keep);
    }
    if (s) cudaStreamDestroy(s);
}

}  // namespace

extern "C" lfmm_status lfmm_server_create(const lfmm_server_params* prm, lfmm_server* out) {
    if (!out || !prm) return LFMM_ERR_INVALID_ARG;
    *out = nullptr;
    if (prm->slots < 1 || prm->slots > 64 || prm->hbm_budget <= 0) return LFMM_ERR_INVALID_ARG;
    lfmm_server_s* S = new lfmm_server_s();
    S->budget = prm->hbm_budget;
    if (cudaGetDevice(&S->device) != cudaSuccess) { delete S; return LFMM_ERR_CUDA; }
    S->workers_left = prm->slots;
    for (int i = 0; i < prm->slots; ++i) S->workers.emplace_back(worker_main, S);
    S->engine = std::thread(engine_main, S);
    *out = S;
    return LFMM_OK;
}

static lfmm_status server_submit(lfmm_server S, const lfmm_request* q, int64_t* ticket);

extern "C" lfmm_status lfmm_server_submit(lfmm_server S, const lfmm_request* q, int64_t* ticket) {
    try {
        return server_submit(S, q, ticket);
    } catch (const std::bad_alloc&) {   // the request's copies of its inputs
        return LFMM_ERR_OUT_OF_MEMORY;
    }
}

static lfmm_status server_submit(lfmm_server S, const lfmm_request* q, int64_t* ticket) {
    if (!S || !q || !ticket) return LFMM_ERR_INVALID_ARG;
    if (q->n_layers < 1 || q->n < 1 || !q->points || !q->weights || !q->wavenumber || !q->density ||
        (q->n_layers > 1 && !q->interface_y) || !(q->tol > 0.0) || q->max_iter < 1 ||
        (q->precision != 0 && q->precision != 1) || (q->flags & ~LFMM_COMBINED_FIELD) != 0 ||
        ((q->flags & LFMM_COMBINED_FIELD) && !q->normals))
        return LFMM_ERR_INVALID_ARG;
    auto r = std::make_shared<Request>();
    r->n_layers = q->n_layers;
    r->yint.assign(q->interface_y, q->interface_y + (q->n_layers - 1));
    r->k.assign(q->wavenumber, q->wavenumber + 2 * q->n_layers);
    r->eta.assign(q->density, q->density + q->n_layers);
    r->n = q->n;
    r->pts.assign(q->points, q->points + 2 * q->n);
    r->w.assign(q->weights, q->weights + q->n);
    r->flags = q->flags;
    if (q->flags & LFMM_COMBINED_FIELD) r->nrm.assign(q->normals, q->normals + 2 * q->n);
    r->angle = q->angle_rad;
    r->tol = q->tol;
    r->precision = q->precision;
    r->p = q->p > 0 ? q->p : 20;
    r->leaf = q->leaf_size > 0 ? q->leaf_size : 64;
    r->max_iter = q->max_iter;
    r->precond = q->precond;
    r->footprint = footprint_estimate(r->n, r->p, r->leaf, r->max_iter);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) return LFMM_ERR_INVALID_ARG;
        if (r->footprint > S->budget) return LFMM_ERR_HBM_BUDGET;   // would never be admitted
        r->ticket = S->next_ticket++;
        r->t_submit = now_s();
        S->queue.push_back(r);
        S->tickets[r->ticket] = r;
        *ticket = r->ticket;
    }
    S->cv_work.notify_all();
    return LFMM_OK;
}

extern "C" lfmm_status lfmm_server_wait(lfmm_server S, int64_t ticket, void* x, lfmm_gmres_info* info,
                                        lfmm_request_times* times) {
    if (!S) return LFMM_ERR_INVALID_ARG;
    std::shared_ptr<Request> r;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        auto it = S->tickets.find(ticket);
        if (it == S->tickets.end()) return LFMM_ERR_INVALID_ARG;
        r = it->second;
        S->cv_done.wait(lk, [&] { return r->done; });
        S->tickets.erase(it);
    }
    if (info) *info = r->info;
    if (times) {
        times->queue_seconds = r->t_admit - r->t_submit;
        times->service_seconds = r->t_done - r->t_admit;
        times->latency_seconds = r->t_done - r->t_submit;
        times->setup_seconds = r->setup_s;
        times->footprint_bytes = r->footprint;
    }
    if (r->status < 0) return r->status;
    if (x) std::memcpy(x, r->x.data(), 16 * (size_t)r->n);
    return r->status;
}

extern "C" lfmm_status lfmm_server_stats(lfmm_server S, int64_t* peak_bytes, int32_t* peak_running) {
    if (!S) return LFMM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    if (peak_bytes) *peak_bytes = S->peak_in_use;
    if (peak_running) *peak_running = S->peak_running;
    return LFMM_OK;
}

extern "C" lfmm_status lfmm_server_destroy(lfmm_server S) {
    if (!S) return LFMM_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto& t : S->workers) t.join();
    S->cv_engine.notify_all();
    if (S->engine.joinable()) S->engine.join();
    delete S;
    return LFMM_OK;
}
