// Many independent pencils (wavenumber, shift and Mach sweeps) and the serving loop.
//
// Every pencil runs the full path (build, factor, Krylov-Schur) on a worker stream; workers are
// host threads that each own one non-blocking stream, so the pencils' kernels overlap on the
// device while each solve stays bit-for-bit the same as when it runs alone (all reductions use a
// fixed order and no result depends on timing).  Device memory comes from the stream-ordered pool.
#include <algorithm>
#include <cmath>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "factor.cuh"

namespace klst {

// Device bytes one solve holds at its peak (pencil tables, factors with the float64 inverse
// formed during factorisation, capacitance buffers, Krylov bases, refinement and extraction work).
int64_t solve_footprint(const klst_pencil_desc& d, int precision, const klst_eigs_opts& o) {
    const int64_t nx = d.nx, nxi = (int64_t)d.qx * d.qy, n = 2 * nx * nxi, r = 4 * nx;
    const int64_t m = o.ncv, nev = o.nev;
    int64_t b = 0;
    b += 2 * nxi * 8 * nx * 8 + 4 * nx * nx * 8 + 2 * nx * nxi * 8;               // pencil (+ build scratch)
    // K^{-1} in float64 while it is formed, plus the stored complex64 (MIXED) or df64 (DF64) copy
    b += nxi * nx * nx * 16 + (precision == KLST_MIXED ? nxi * nx * nx * 8 : precision == KLST_DF64 ? nxi * nx * nx * 16 : 0);
    if (precision == KLST_FP64 && tc_solve_supported((int)nx))                   // tensor-core slices of K^{-1}
        b += (int64_t)tc_kinv_bytes((int)nx, (int)nxi);
    if (ns_inverse_supported((int)nx))                                           // Newton-Schulz scratch
        b += (int64_t)ns_scratch_bytes((int)nx, (int)nxi);
    b += 11 * r * r * 16;                                                        // capacitance buffers
    b += 2 * n * (m + 1) * 16 + 3 * n * nev * 16;                                // Krylov bases + extraction
    b += (precision == KLST_MIXED ? 3 * n * nev * 16 + (int64_t)oz_dx_ws_bytes((int)nx, (int)nxi, (int)nev) : 0);  // refinement work
    b += (int64_t)oz_dx_bytes((int)nx);                                           // D_x slices
    if (o.arith == KLST_ARITH_DF64)                                              // df64 basis: w, v and partial dots
        b += 2 * n * 16 + ((n + 511) / 512) * (m + 2) * 16;
    b += 31 * m * m * 32 + 8 * m * m * 16;                                       // Schur work and rotation log
    if (o.arith != KLST_ARITH_DF64) b += 31 * m * m * 36 + 2048;                 // float64 step: sorted log + levels
    if (o.arith != KLST_ARITH_DF64 && basis_slices_supported((int)m))            // integer slices of the basis
        b += (int64_t)basis_slices_bytes(n) + n * (m + 1) * 8 + 256 * (m + 1) * 16;
    if (o.arith != KLST_ARITH_DF64 && 2 * m <= 256)                              // tensor-core rotation slices
        b += (int64_t)oz_workspace_bytes((int)n, 2 * (int)std::max<int64_t>(m, nev), (int)(2 * m));
    return b + (64 << 20);
}

// Request checks shared by the batch and serving entry points: the pencil sizes klst_build_pencil
// accepts, a known precision and klst_eigs's option rules, so that nothing is sized from a bad value.
static int validate_request(const klst_pencil_desc& d, int precision, const klst_eigs_opts& o) {
    if (d.nx < 4 || d.nx > 128 || d.qx < 1 || d.qx > 256 || d.qy < 1 || d.qy > 256) {
        set_error("invalid pencil sizes nx=%d qx=%d qy=%d", d.nx, d.qx, d.qy);
        return KLST_EINVAL;
    }
    if (precision != KLST_FP64 && precision != KLST_MIXED && precision != KLST_DF64) {
        set_error("invalid precision %d", precision);
        return KLST_EINVAL;
    }
    return validate_eigs_opts(&o, 2 * (int64_t)d.nx * d.qx * d.qy);
}

struct SolveResult {
    int status = KLST_OK;
    std::vector<double> evals, resid;
    klst_eigs_info info{};
};

// Full path for one pencil on stream s.
static void solve_one_impl(const klst_pencil_desc& d, double2 sigma, int precision, const klst_eigs_opts& o,
                           cudaStream_t s, SolveResult& out) {
    out.evals.assign(2 * o.nev, 0.0);
    out.resid.assign(o.nev, 0.0);
    memset(&out.info, 0, sizeof(out.info));
    klst_pencil p = nullptr;
    klst_factor f = nullptr;
    int rc = klst_build_pencil(&d, (klst_stream)s, &p);
    if (rc == KLST_OK) rc = klst_factor_shift(p, sigma.x, sigma.y, precision, (klst_stream)s, &f);
    if (rc == KLST_OK) rc = klst_eigs(f, &o, out.evals.data(), nullptr, out.resid.data(), &out.info, (klst_stream)s);
    if (f) klst_factor_destroy(f);
    if (p) klst_pencil_destroy(p);
    cudaStreamSynchronize(s);
    out.status = rc;
    if (rc != KLST_OK && rc != KLST_ENOCONV && rc != KLST_EREFINE)  // nothing computed: no pair may count
        for (auto& r : out.resid) r = INFINITY;
}

// A host exception (a failed host allocation) becomes the request's status instead of
// terminating the process with every other request in flight.
static void solve_one(const klst_pencil_desc& d, double2 sigma, int precision, const klst_eigs_opts& o,
                      cudaStream_t s, SolveResult& out) {
    try {
        solve_one_impl(d, sigma, precision, o, s, out);
    } catch (...) {
        cudaStreamSynchronize(s);
        out.status = KLST_ENOMEM;
        out.evals.assign(2 * std::max(o.nev, 0), 0.0);
        out.resid.assign(std::max(o.nev, 0), INFINITY);
        set_error("host exception during a solve (out of host memory?)");
    }
}

}  // namespace klst

using namespace klst;

extern "C" int klst_batch_eigs(int32_t npencils, const klst_pencil_desc* descs, const double* sigmas,
                               int32_t precision, const klst_eigs_opts* opts, int32_t nworkers, double* evals_host,
                               double* resid_host, int32_t* status_host, klst_eigs_info* infos) {
    if (npencils < 1 || !descs || !sigmas || !opts || !evals_host || !status_host) {
        set_error("invalid arguments to klst_batch_eigs");
        return KLST_EINVAL;
    }
    if (opts->v0) {
        set_error("klst_batch_eigs seeds every start vector (opts->v0 must be NULL; pencil i uses seed + i)");
        return KLST_EINVAL;
    }
    for (int i = 0; i < npencils; ++i)
        if (int vrc = validate_request(descs[i], precision, *opts)) return vrc;
    for (int i = 0; i < npencils; ++i) status_host[i] = KLST_ECUDA;  // until a worker runs it
    int dev = 0;
    KLST_CK(cudaGetDevice(&dev));
    const int W = std::max(1, std::min<int>(npencils, nworkers > 0 ? nworkers : 16));
    // largest pencils first, for balance
    std::vector<int> order(npencils);
    for (int i = 0; i < npencils; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (int64_t)descs[a].nx * descs[a].qx * descs[a].qy > (int64_t)descs[b].nx * descs[b].qx * descs[b].qy;
    });
    std::atomic<int> next(0);
    std::vector<std::thread> pool;
    for (int w = 0; w < W; ++w) {
        pool.emplace_back([&, w]() {
            cudaSetDevice(dev);
            cudaStream_t s;
            if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return;
            for (int t; (t = next.fetch_add(1)) < npencils;) {
                const int i = order[t];
                klst_eigs_opts o = *opts;
                o.seed = opts->seed + (uint64_t)i;
                o.est_out = nullptr;
                SolveResult res;
                solve_one(descs[i], mk(sigmas[2 * i], sigmas[2 * i + 1]), precision, o, s, res);
                memcpy(evals_host + (size_t)2 * o.nev * i, res.evals.data(), sizeof(double) * 2 * o.nev);
                if (resid_host) memcpy(resid_host + (size_t)o.nev * i, res.resid.data(), sizeof(double) * o.nev);
                status_host[i] = res.status;
                if (infos) infos[i] = res.info;
            }
            cudaStreamDestroy(s);
        });
    }
    for (auto& t : pool) t.join();
    int worst = KLST_OK;
    for (int i = 0; i < npencils; ++i)
        if (status_host[i] != KLST_OK && worst == KLST_OK) worst = status_host[i];
    if (worst != KLST_OK) set_error("one or more pencils failed; see status_host");
    return worst;
}

// ------------------------------------------------------------------ serving
struct klst_server_s {
    struct Req {
        uint64_t ticket;
        klst_pencil_desc desc;
        double2 sigma;
        int precision;
        klst_eigs_opts opts;
        int64_t footprint;
        std::chrono::steady_clock::time_point t_submit, t_start, t_done;
        bool done = false;
        bool claimed = false;   // a poll is collecting it: no other poll may touch it
        int passed = 0;         // times a later request was admitted ahead of it
        SolveResult res;
    };
    std::mutex mu;
    std::condition_variable cv, cv_done;
    std::deque<Req*> queue;                  // waiting, in arrival order
    std::map<uint64_t, Req*> all;            // every request not yet collected
    int64_t budget = 0, in_flight = 0;
    int slots = 0, running = 0;
    // Backfill is bounded: once the head request has been passed over kMaxPassed times, or has
    // waited kMaxWaitMs, nothing else is admitted until it fits, so a large request cannot starve
    // behind a stream of small ones.
    static constexpr int kMaxPassed = 8;
    static constexpr double kMaxWaitMs = 2000.0;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::vector<std::thread> workers;
    int dev = 0;
};

static void server_worker(klst_server S) {
    cudaSetDevice(S->dev);
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return;
    for (;;) {
        klst_server_s::Req* r = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            for (;;) {
                if (S->stop) break;
                // admit the oldest request that fits the remaining HBM budget; a later one may
                // backfill past a head request that has to wait for memory, until the head has
                // been passed over kMaxPassed times or has waited kMaxWaitMs
                if (!S->queue.empty()) {
                    klst_server_s::Req* head = S->queue.front();
                    const double waited = std::chrono::duration<double, std::milli>(
                        std::chrono::steady_clock::now() - head->t_submit).count();
                    const bool may_pass = head->passed < klst_server_s::kMaxPassed && waited < klst_server_s::kMaxWaitMs;
                    for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
                        if (it != S->queue.begin() && !may_pass) break;
                        if (S->in_flight + (*it)->footprint <= S->budget) {
                            r = *it;
                            if (it != S->queue.begin()) head->passed += 1;
                            S->queue.erase(it);
                            break;
                        }
                    }
                }
                if (r) break;
                // a waiting head re-evaluates its age periodically even when nothing finishes
                S->cv.wait_for(lk, std::chrono::milliseconds(50));
            }
            if (!r) break;
            S->in_flight += r->footprint;
            S->running += 1;
            r->t_start = std::chrono::steady_clock::now();
        }
        solve_one(r->desc, r->sigma, r->precision, r->opts, s, r->res);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            r->t_done = std::chrono::steady_clock::now();
            r->done = true;
            S->in_flight -= r->footprint;
            S->running -= 1;
        }
        S->cv.notify_all();
        S->cv_done.notify_all();
    }
    cudaStreamDestroy(s);
}

extern "C" int64_t klst_solve_footprint(const klst_pencil_desc* d, int32_t precision, const klst_eigs_opts* o) {
    if (!d || !o) { set_error("invalid arguments to klst_solve_footprint"); return KLST_EINVAL; }
    if (int vrc = validate_request(*d, precision, *o)) return vrc;
    return solve_footprint(*d, precision, *o);
}

extern "C" int klst_server_create(int64_t hbm_budget_bytes, int32_t max_slots, klst_server* out) {
    if (!out || max_slots < 1 || hbm_budget_bytes <= 0) { set_error("invalid server arguments"); return KLST_EINVAL; }
    klst_server S = new klst_server_s();
    S->budget = hbm_budget_bytes;
    S->slots = max_slots;
    cudaGetDevice(&S->dev);
    for (int i = 0; i < max_slots; ++i) S->workers.emplace_back(server_worker, S);
    *out = S;
    return KLST_OK;
}

extern "C" int klst_server_submit(klst_server S, const klst_pencil_desc* d, double sig_re, double sig_im,
                                  int32_t precision, const klst_eigs_opts* o, uint64_t* ticket) {
    if (!S || !d || !o || !ticket || o->v0) { set_error("invalid submit arguments (opts->v0 must be NULL)"); return KLST_EINVAL; }
    if (int vrc = validate_request(*d, precision, *o)) return vrc;
    auto* r = new klst_server_s::Req();
    r->desc = *d;
    r->sigma = mk(sig_re, sig_im);
    r->precision = precision;
    r->opts = *o;
    r->opts.est_out = nullptr;
    r->footprint = solve_footprint(*d, precision, *o);
    r->t_submit = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (r->footprint > S->budget) {
            delete r;
            set_error("request needs %lld bytes, more than the server's HBM budget", (long long)solve_footprint(*d, precision, *o));
            return KLST_ENOMEM;
        }
        r->ticket = S->next_ticket++;
        S->queue.push_back(r);
        S->all[r->ticket] = r;
        *ticket = r->ticket;
    }
    S->cv.notify_all();
    return KLST_OK;
}

extern "C" int klst_server_poll(klst_server S, uint64_t ticket, int32_t wait, int32_t* done, double* evals_host,
                                double* resid_host, klst_eigs_info* info, double* latency_ms) {
    if (!S || !done) { set_error("invalid poll arguments"); return KLST_EINVAL; }
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) { set_error("unknown or already collected ticket"); return KLST_EINVAL; }
    klst_server_s::Req* r = it->second;
    if (r->claimed) { set_error("ticket is being collected by another poll"); return KLST_EINVAL; }
    if (wait) {
        // claim the ticket so that a concurrent poll cannot collect (and free) it while this one sleeps
        r->claimed = true;
        S->cv_done.wait(lk, [&] { return r->done; });
    }
    *done = r->done ? 1 : 0;
    if (!r->done) return KLST_OK;
    const int nev = r->opts.nev;
    if (evals_host) memcpy(evals_host, r->res.evals.data(), sizeof(double) * 2 * nev);
    if (resid_host) memcpy(resid_host, r->res.resid.data(), sizeof(double) * nev);
    if (info) *info = r->res.info;
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    const int st = r->res.status;
    S->all.erase(it);
    delete r;
    return st;
}

extern "C" int klst_server_stats(klst_server S, int32_t* queued, int32_t* running, int64_t* bytes_in_flight) {
    if (!S) { set_error("server is NULL"); return KLST_EINVAL; }
    std::lock_guard<std::mutex> lk(S->mu);
    if (queued) *queued = (int32_t)S->queue.size();
    if (running) *running = S->running;
    if (bytes_in_flight) *bytes_in_flight = S->in_flight;
    return KLST_OK;
}

extern "C" void klst_server_destroy(klst_server S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    for (auto& t : S->workers) t.join();
    for (auto& kv : S->all) delete kv.second;
    delete S;
}
