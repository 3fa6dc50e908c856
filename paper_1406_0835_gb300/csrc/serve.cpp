// Serving loop for equation-of-state requests on one GPU (include/ofdft.h,
// ofdft_serve_*).
//
// Requests queue in arrival order.  A pool of worker threads (one per slot)
// admits the first queued request whose device footprint fits in what the
// memory budget has left as soon as a slot is free; a request that does not
// fit yet may be passed by at most max_bypass later ones, after which
// nothing is admitted ahead of it (so it cannot starve).  The admitted
// request gets its own context and stream and runs its MD steps there, so
// requests that arrive while others run overlap with them on the device.
// Contexts share nothing, which makes each result independent of the mix.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/ofdft.h"

namespace {

struct Pending {
    long long id;
    ofdft_request r;
    std::vector<double> ions, Z, vel;
    double footprint;
    double t_submit;
    int bypassed = 0;     // later requests admitted ahead of this one
    std::atomic<bool> cancel{false};   // set by ofdft_serve_cancel while it runs
};

}  // namespace

struct ofdft_server {
    ofdft_serve_params p{};
    double budget = 0.0;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Pending *> queue;
    std::map<long long, ofdft_result> done;
    std::map<long long, Pending *> active;   // admitted and running
    long long next_id = 1, submitted = 0, finished = 0;
    int running = 0, peak_running = 0;
    double used = 0.0, peak_used = 0.0;
    bool stopping = false;
    std::vector<std::thread> workers;

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

// Run one request to completion on its own context (or sleep in dry-run mode).
ofdft_result run_request(ofdft_server *s, Pending *q)
{
    ofdft_result res;
    std::memset(&res, 0, sizeof(res));
    res.id = q->id;
    res.footprint_bytes = q->footprint;
    res.t_submit = q->t_submit;
    const ofdft_request &r = q->r;
    if (s->p.dry_run) {
        // the initial minimisation and each step take an equal share
        const double part_ms = s->p.dry_run_ms / (r.md_steps + 1);
        res.status = OFDFT_OK;
        for (int k = 0; k <= r.md_steps; ++k) {
            if (k > 0 && q->cancel.load()) {
                res.status = OFDFT_ECANCELED;
                break;
            }
            std::this_thread::sleep_for(std::chrono::duration<double, std::milli>(part_ms));
            if (k > 0) res.steps_done = k;
        }
        return res;
    }
    ofdft_params pr;
    ofdft_default_params(&pr);
    pr.xc = r.xc;
    pr.rc = r.rc;
    pr.precision = r.precision;
    pr.device = s->p.device;
    pr.stream = nullptr;                      // the context's own stream
    ofdft_ctx *c = nullptr;
    ofdft_status st = ofdft_setup(r.cell, r.grid, r.nat, q->ions.data(), q->Z.data(), r.T_kelvin,
                                  r.functional, &pr, &c);
    if (st != OFDFT_OK) {
        res.status = st;
        return res;
    }
    ofdft_md_params mp;
    mp.dt_fs = r.dt_fs;
    mp.T_kelvin = r.T_kelvin;
    mp.tau_steps = 100.0;
    mp.gtol = r.gtol;
    mp.maxit = r.maxit;
    ofdft_energy E;
    ofdft_stats stats;
    std::memset(&E, 0, sizeof(E));
    // the initial minimisation and forces, then one call per step
    st = ofdft_md_step(c, &mp, 0, nullptr, q->vel.empty() ? nullptr : q->vel.data(), nullptr, &E, &stats);
    res.evaluations += stats.evaluations;
    double psum = 0.0;
    int done = 0;         // MD steps completed (0 when the initial minimisation failed)
    while (st == OFDFT_OK && done < r.md_steps) {
        if (q->cancel.load()) {
            st = OFDFT_ECANCELED;
            break;
        }
        st = ofdft_md_step(c, &mp, 1, nullptr, nullptr, nullptr, &E, &stats);
        res.evaluations += stats.evaluations;
        if (st == OFDFT_OK) {
            psum += E.P;
            ++done;
        }
    }
    res.status = st;
    res.E = E;
    res.steps_done = done;
    res.P_mean = r.md_steps > 0 ? (done > 0 ? psum / done : 0.0) : E.P;
    ofdft_destroy(c);
    return res;
}

// Queue position of the request to admit next, or -1: the first one that
// fits, unless an earlier one that does not fit has been passed max_bypass
// times already (with max_bypass 0 only the head is ever admitted).
long pick(const ofdft_server *s)
{
    for (size_t j = 0; j < s->queue.size(); ++j) {
        const Pending *q = s->queue[j];
        if (s->used + q->footprint <= s->budget) return (long)j;
        if (q->bypassed >= s->p.max_bypass) return -1;
    }
    return -1;
}

void worker(ofdft_server *s)
{
    if (!s->p.dry_run) cudaSetDevice(s->p.device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        long j = -1;
        s->cv.wait(lk, [s, &j] {
            if (s->queue.empty()) return s->stopping;
            j = pick(s);
            return j >= 0;
        });
        if (s->queue.empty()) break;          // stopping and nothing left
        Pending *q = s->queue[j];
        for (long i = 0; i < j; ++i) s->queue[i]->bypassed += 1;
        s->queue.erase(s->queue.begin() + j);
        s->used += q->footprint;
        s->running += 1;
        if (s->used > s->peak_used) s->peak_used = s->used;
        if (s->running > s->peak_running) s->peak_running = s->running;
        const double t_admit = s->now();
        s->active[q->id] = q;
        lk.unlock();
        ofdft_result res = run_request(s, q);
        res.t_admit = t_admit;
        lk.lock();
        s->active.erase(q->id);
        res.t_done = s->now();
        s->used -= q->footprint;
        s->running -= 1;
        s->done[q->id] = res;
        s->finished += 1;
        delete q;
        s->cv.notify_all();
    }
}

}  // namespace

extern "C" {

ofdft_status ofdft_serve_start(const ofdft_serve_params *p, ofdft_server **out)
{
    if (!p || !out || p->max_slots < 1 || p->max_bypass < 0) return OFDFT_EINVAL;
    *out = nullptr;
    ofdft_server *s = new (std::nothrow) ofdft_server();
    if (!s) return OFDFT_ENOMEM;
    s->p = *p;
    s->t0 = std::chrono::steady_clock::now();
    if (p->hbm_budget_bytes > 0.0) {
        s->budget = p->hbm_budget_bytes;
    } else if (p->dry_run) {
        delete s;
        return OFDFT_EINVAL;                   // a dry run needs an explicit budget
    } else {
        size_t fr = 0, tot = 0;
        if (cudaSetDevice(p->device) != cudaSuccess || cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            delete s;
            return OFDFT_EDEVICE;
        }
        s->budget = 0.9 * (double)fr;
    }
    for (int i = 0; i < p->max_slots; ++i) s->workers.emplace_back(worker, s);
    *out = s;
    return OFDFT_OK;
}

ofdft_status ofdft_serve_submit(ofdft_server *s, const ofdft_request *r, long long *id)
{
    if (!s || !r || !r->ions || !r->Z || r->nat <= 0 || r->md_steps < 0) return OFDFT_EINVAL;
    double fp = 0.0;
    ofdft_status st = ofdft_footprint(r->grid, r->nat, r->precision, &fp);
    if (st != OFDFT_OK) return st;
    if (fp > s->budget) return OFDFT_ENOMEM;
    Pending *q = new (std::nothrow) Pending();
    if (!q) return OFDFT_ENOMEM;
    q->r = *r;
    q->ions.assign(r->ions, r->ions + 3 * r->nat);
    q->Z.assign(r->Z, r->Z + r->nat);
    if (r->vel) q->vel.assign(r->vel, r->vel + 3 * r->nat);
    q->r.ions = q->r.Z = q->r.vel = nullptr;   // the copies above are what runs
    q->footprint = fp;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) {
        delete q;
        return OFDFT_EINVAL;
    }
    q->id = s->next_id++;
    q->t_submit = s->now();
    s->queue.push_back(q);
    s->submitted += 1;
    if (id) *id = q->id;
    s->cv.notify_all();
    return OFDFT_OK;
}

ofdft_status ofdft_serve_poll(ofdft_server *s, long long id, ofdft_result *res)
{
    if (!s) return OFDFT_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->done.find(id);
    if (it != s->done.end()) {
        if (res) *res = it->second;
        return OFDFT_OK;
    }
    return (id >= 1 && id < s->next_id) ? OFDFT_EBUSY : OFDFT_EINVAL;
}

ofdft_status ofdft_serve_cancel(ofdft_server *s, long long id)
{
    if (!s) return OFDFT_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
        Pending *q = *it;
        if (q->id != id) continue;
        s->queue.erase(it);
        ofdft_result res;
        std::memset(&res, 0, sizeof(res));
        res.id = id;
        res.status = OFDFT_ECANCELED;
        res.t_submit = q->t_submit;
        res.t_admit = -1.0;          // never admitted
        res.t_done = s->now();
        res.footprint_bytes = q->footprint;
        s->done[id] = res;
        s->finished += 1;
        delete q;
        s->cv.notify_all();          // a request behind it may fit now
        return OFDFT_OK;
    }
    auto a = s->active.find(id);
    if (a != s->active.end()) {
        a->second->cancel.store(true);
        return OFDFT_OK;
    }
    return s->done.count(id) ? OFDFT_OK : OFDFT_EINVAL;
}

ofdft_status ofdft_serve_drain(ofdft_server *s, double timeout_s)
{
    if (!s) return OFDFT_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto pred = [s] { return s->finished == s->submitted; };
    if (timeout_s <= 0.0) {
        s->cv.wait(lk, pred);
        return OFDFT_OK;
    }
    return s->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), pred) ? OFDFT_OK : OFDFT_ETIMEOUT;
}

double ofdft_serve_clock(ofdft_server *s) { return s ? s->now() : 0.0; }

ofdft_status ofdft_serve_peaks(ofdft_server *s, double *bytes, int *running)
{
    if (!s) return OFDFT_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (bytes) *bytes = s->peak_used;
    if (running) *running = s->peak_running;
    return OFDFT_OK;
}

ofdft_status ofdft_serve_stop(ofdft_server *s)
{
    if (!s) return OFDFT_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv.notify_all();
    for (std::thread &t : s->workers) t.join();
    delete s;
    return OFDFT_OK;
}

}  // extern "C"
