// Serving loop for forward solves (no counterpart in the paper): requests with their own source,
// frequency k, mesh size and receivers arrive at any time and share one resident velocity model.
//
// * Admission by HBM footprint: each request's peak device memory is estimated from its sizes
//   (beam state and its sorted copy, sort keys, decomposition temporaries, a capped record buffer);
//   requests start while the sum over running requests stays within the budget (a request is always
//   admitted when nothing runs, so an oversized one fails on its own).  Order: submission order, or
//   the least estimated work (beams x steps) first with an age bound that serves any request waiting
//   longer than the limit first (oldest first).
// * Cancellation: a queued request is dropped; a running one stops at its next window of steps.
// * Continuous batching on streams: each worker thread owns a non-blocking stream and runs one
//   admitted request at a time through the solve pipeline; requests on different workers share
//   the GPU, so the kernels of small requests fill the SMs together.  Workers keep the device and
//   pinned buffers of finished requests in a per-thread block cache, so steady-state serving makes
//   no cudaMalloc/cudaFree calls (which would synchronise every stream).
// * Latency: submit, start and end times (host steady clock; end after the request's stream has
//   drained) per request.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cmath>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fga_internal.cuh"

namespace fga {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t id = 0;
    fga_init_desc init{};
    fga_solve_desc sd{};
    std::vector<double> times;
    fga_lattice rxL{}, snL{};                  // copies of lattice descriptors (axes below)
    std::vector<double> rx_axes[3], sn_axes[3];
    void *seis_out = nullptr, *snap_out = nullptr;
    double bytes = 0.0;
    int64_t beams = 0;
    double work = 0.0;                         // estimated work: beams x steps
    std::atomic<int> cancel{0};
    // results
    bool done = false;
    fga_status status = FGA_OK;
    std::string error;
    int worker = -1;
    Clock::time_point t_submit, t_start, t_end;
};

int popcount4(unsigned m) { return (m & 1) + ((m >> 1) & 1) + ((m >> 2) & 1) + ((m >> 3) & 1); }

}  // namespace

// peak device bytes of one forward solve with a record buffer of at most rec_cap bytes
double estimate_solve_bytes(const fga_init_desc *d, double rec_cap) {
    const double rb = d->precision == FGA_PREC_FP64 ? 8.0 : 4.0;
    const double M = std::pow((double)d->nq, 3) * std::pow((double)d->np, 3);
    const double nb = M * popcount4(d->class_mask);
    const double cap = std::ceil(nb / 32.0) * 32.0;
    const double A = (double)d->nq * d->np;
    const double ny0 = d->ny[0], ny1 = d->ny[1], ny2 = d->ny[2];
    const double cbytes = 2.0 * rb;
    const double state = NFS * rb * cap, ints = 4.0 * 4.0 * cap, sort = 4.0 * 4.0 * cap;
    const double decomp = cbytes * (A * (ny0 + ny1 + ny2) + ny0 * ny1 * A * 3.0 + ny0 * A * A * 3.0 +
                                    A * A * A * 3.0 * (d->g ? 2.0 : 1.0));
    const double during_decomp = state + ints + decomp;
    const double during_solve = 2.0 * state + ints + sort + rec_cap;
    return std::max(during_decomp, during_solve) + 64.0 * 1024 * 1024;
}

}  // namespace fga

struct fga_server {
    const fga_model *model = nullptr;
    int n_workers = 0;
    double budget = 0.0, rec_cap = 0.0;
    int policy = FGA_SERVE_FIFO;
    double age_limit = 2.0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<fga::Request *> queue;   // submission order
    std::unordered_map<int64_t, fga::Request *> all;
    int64_t next_id = 1;
    double inflight_bytes = 0.0, peak_bytes = 0.0;
    int running = 0, peak_running = 0;
    int64_t completed = 0;
    bool stop = false;
    fga::Clock::time_point t0;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
    int device = 0;

    // the queued request to start next (caller holds mu; queue not empty): FIFO, or the least
    // estimated work unless the oldest request has waited longer than the age limit
    std::deque<fga::Request *>::iterator pick() {
        if (policy != FGA_SERVE_SHORTEST) return queue.begin();
        const auto now = fga::Clock::now();
        if (std::chrono::duration<double>(now - queue.front()->t_submit).count() > age_limit) return queue.begin();
        auto best = queue.begin();
        for (auto it = queue.begin(); it != queue.end(); ++it)
            if ((*it)->work < (*best)->work) best = it;
        return best;
    }

    void worker_main(int w) {
        cudaSetDevice(device);
        cudaStream_t s = streams[(size_t)w];
        fga::block_cache_enable(s);
        for (;;) {
            fga::Request *r = nullptr;
            {
                std::unique_lock<std::mutex> lk(mu);
                // wake up at least every 50 ms so that the age limit is honoured while requests wait
                for (;;) {
                    if (queue.empty()) {
                        if (stop) break;
                    } else {
                        const fga::Request *h = *pick();
                        if (running == 0 || inflight_bytes + h->bytes <= budget) break;
                    }
                    cv_work.wait_for(lk, std::chrono::milliseconds(50));
                }
                if (queue.empty()) break;  // stop requested and nothing left
                auto it = pick();
                r = *it;
                queue.erase(it);
                inflight_bytes += r->bytes;
                running++;
                peak_bytes = std::max(peak_bytes, inflight_bytes);
                peak_running = std::max(peak_running, running);
                r->worker = w;
                r->t_start = fga::Clock::now();
            }
            const fga_status st =
                fga::solve_impl(model, &r->init, &r->sd, r->seis_out, r->snap_out, s, rec_cap, &r->cancel);
            cudaStreamSynchronize(s);
            std::string err;
            if (st != FGA_OK) {
                char buf[512];
                fga_last_error(buf, sizeof buf);
                err = buf;
            }
            // keep the cache within this worker's share of the budget
            fga::block_cache_trim((size_t)(budget / std::max(1, n_workers)));
            {
                std::lock_guard<std::mutex> lk(mu);
                r->t_end = fga::Clock::now();
                r->status = st;
                r->error = err;
                r->done = true;
                inflight_bytes -= r->bytes;
                running--;
                completed++;
            }
            cv_done.notify_all();
            cv_work.notify_all();
        }
        fga::block_cache_disable();
    }
};

using namespace fga;

extern "C" {

fga_status fga_server_create(fga_server **out, const fga_model *m, const fga_server_desc *d) {
    FGA_CHECK(out && m && d, "fga_server_create: NULL argument");
    FGA_CHECK(d->n_workers >= 1 && d->n_workers <= 64, "fga_server_create: n_workers must be in 1..64");
    FGA_CHECK(m->dev.kind != FGA_MEDIUM_LAYERED, "fga_server_create: layered media are not served");
    std::unique_ptr<fga_server> owner(new fga_server());   // freed on every early return
    fga_server *sv = owner.get();
    sv->model = m;
    sv->n_workers = d->n_workers;
    FGA_CUDA(cudaGetDevice(&sv->device));
    size_t free_b = 0, total_b = 0;
    FGA_CUDA(cudaMemGetInfo(&free_b, &total_b));
    sv->budget = d->hbm_budget_bytes > 0 ? d->hbm_budget_bytes : 0.85 * (double)free_b;
    sv->rec_cap = d->record_cap_bytes > 0 ? d->record_cap_bytes : 2.0e9;
    FGA_CHECK(d->policy == FGA_SERVE_FIFO || d->policy == FGA_SERVE_SHORTEST, "fga_server_create: unknown policy");
    sv->policy = d->policy;
    sv->age_limit = d->age_limit_s > 0 ? d->age_limit_s : 2.0;
    sv->t0 = Clock::now();
    for (int w = 0; w < d->n_workers; w++) {
        cudaStream_t s = nullptr;
        const cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (cudaStream_t t : sv->streams) cudaStreamDestroy(t);
            return cuda_fail(e, "fga_server_create: cudaStreamCreateWithFlags");
        }
        sv->streams.push_back(s);
    }
    for (int w = 0; w < d->n_workers; w++) sv->workers.emplace_back([sv, w] { sv->worker_main(w); });
    *out = owner.release();
    return FGA_OK;
}

fga_status fga_server_submit(fga_server *sv, const fga_init_desc *init, const fga_solve_desc *sd, void *seis_out,
                             void *snap_out, int64_t *id) {
    FGA_CHECK(sv && init && sd && id, "fga_server_submit: NULL argument");
    FGA_CHECK(init->f && init->nq >= 1 && init->np >= 1, "fga_server_submit: bad init descriptor");
    FGA_CHECK(sd->n_times >= 0 && (sd->n_times == 0 || sd->times), "fga_server_submit: times missing");
    std::unique_ptr<Request> owner(new Request());   // freed on every early return until it is queued
    Request *r = owner.get();
    r->init = *init;
    r->sd = *sd;
    r->times.assign(sd->times, sd->times + sd->n_times);
    r->sd.times = r->times.data();
    // lattice descriptors are host data: keep copies with the request
    auto copy_lattice = [](const fga_lattice *src, fga_lattice &dst, std::vector<double> ax[3]) {
        dst = *src;
        for (int d = 0; d < 3; d++) {
            ax[d].assign(src->axis[d], src->axis[d] + std::max(src->n[d], 0));
            dst.axis[d] = ax[d].data();
        }
    };
    if (sd->rx_lattice) {
        FGA_CHECK(sd->rx_lattice->n[0] >= 1 && sd->rx_lattice->n[1] >= 1 && sd->rx_lattice->n[2] >= 1,
                  "fga_server_submit: bad receiver lattice");
        copy_lattice(sd->rx_lattice, r->rxL, r->rx_axes);
        r->sd.rx_lattice = &r->rxL;
    }
    if (sd->snap_lattice) {
        FGA_CHECK(sd->snap_lattice->n[0] >= 1 && sd->snap_lattice->n[1] >= 1 && sd->snap_lattice->n[2] >= 1,
                  "fga_server_submit: bad snapshot lattice");
        copy_lattice(sd->snap_lattice, r->snL, r->sn_axes);
        r->sd.snap_lattice = &r->snL;
    }
    r->seis_out = seis_out;
    r->snap_out = snap_out;
    r->bytes = estimate_solve_bytes(init, sv->rec_cap);
    r->beams = (int64_t)std::pow((double)init->nq, 3) * (int64_t)std::pow((double)init->np, 3) *
               popcount4(init->class_mask);
    r->work = (double)r->beams * std::max(sd->nsteps, 1);
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        FGA_CHECK(!sv->stop, "fga_server_submit: server is shutting down");
        r->id = sv->next_id++;
        r->t_submit = Clock::now();
        sv->all[r->id] = r;
        sv->queue.push_back(r);
        owner.release();
        *id = r->id;
    }
    sv->cv_work.notify_all();
    return FGA_OK;
}

fga_status fga_server_wait(fga_server *sv, int64_t id, double timeout_s, fga_request_info *info) {
    FGA_CHECK(sv, "fga_server_wait: NULL server");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->all.find(id);
    FGA_CHECK(it != sv->all.end(), "fga_server_wait: unknown or already collected request id");
    Request *r = it->second;
    auto ready = [&] { return r->done; };
    if (timeout_s > 0) {
        if (!sv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
            set_error("fga_server_wait: timed out");
            return FGA_ERR_TIMEOUT;
        }
    } else {
        sv->cv_done.wait(lk, ready);
    }
    if (info) {
        info->status = r->status;
        info->worker = r->worker;
        info->t_submit = std::chrono::duration<double>(r->t_submit - sv->t0).count();
        info->t_start = std::chrono::duration<double>(r->t_start - sv->t0).count();
        info->t_end = std::chrono::duration<double>(r->t_end - sv->t0).count();
        info->bytes = r->bytes;
        info->beams = r->beams;
    }
    const fga_status st = r->status;
    if (st != FGA_OK) set_error("request " + std::to_string(id) + ": " + r->error);
    sv->all.erase(it);
    delete r;
    return st;
}

fga_status fga_server_cancel(fga_server *sv, int64_t id) {
    FGA_CHECK(sv, "fga_server_cancel: NULL server");
    bool dropped = false;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->all.find(id);
        FGA_CHECK(it != sv->all.end(), "fga_server_cancel: unknown or already collected request id");
        Request *r = it->second;
        if (r->done) return FGA_OK;
        auto q = std::find(sv->queue.begin(), sv->queue.end(), r);
        if (q != sv->queue.end()) {   // not started: finished at once
            sv->queue.erase(q);
            r->t_start = r->t_end = Clock::now();
            r->status = FGA_ERR_CANCELLED;
            r->error = "the request was cancelled before it started";
            r->done = true;
            sv->completed++;
            dropped = true;
        } else {
            r->cancel.store(1);      // running: stops at its next window of steps
        }
    }
    if (dropped) sv->cv_done.notify_all();
    return FGA_OK;
}

fga_status fga_server_stats(fga_server *sv, fga_server_stats_t *out) {
    FGA_CHECK(sv && out, "fga_server_stats: NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    out->queued = (int64_t)sv->queue.size();
    out->running = sv->running;
    out->completed = sv->completed;
    out->peak_running = sv->peak_running;
    out->inflight_bytes = sv->inflight_bytes;
    out->peak_bytes = sv->peak_bytes;
    out->budget_bytes = sv->budget;
    return FGA_OK;
}

fga_status fga_server_destroy(fga_server *sv) {
    if (!sv) return FGA_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    for (auto &t : sv->workers) t.join();
    for (cudaStream_t s : sv->streams) cudaStreamDestroy(s);
    for (auto &kv : sv->all) delete kv.second;
    delete sv;
    return FGA_OK;
}

}  // extern "C"
