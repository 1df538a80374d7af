// Serving: continuous batching of many Davidson solves on one GPU.
//
// tbsci_submit copies a request into the queue. One scheduler thread owns a
// private context and, every round:
//   1. admits queued requests in arrival order while a slot is free and the
//      HBM budget holds the request's estimated footprint (strings, tables,
//      prepared space, Davidson vectors) and hands them to a set-up thread,
//      which builds their device objects with its own context and stream while
//      the scheduler keeps advancing the running solves; set-up requests join
//      the running ones as they become ready;
//   2. polls every admitted solve's Davidson engine without blocking, so the
//      host logic of whichever solves have finished a phase runs while the
//      device keeps working on the others (each solve has its own stream);
//   3. gathers the sigma work that solves are waiting for and issues the small
//      jobs as one batched launch per precision (every job computed exactly as a
//      launch of its own would: CTAs never mix jobs), ordered after each solve's
//      stream and before the solve continues; jobs above 2^20 determinant-vectors
//      get launches of their own on their solve's stream, so the small batch runs
//      beside them instead of waiting for them;
//   4. retires finished solves, releasing their memory for the next admissions.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

int64_t binom64(int n, int k) {
    if (k < 0 || k > n) return 0;
    unsigned __int128 v = 1;
    for (int i = 1; i <= k; ++i) v = v * (unsigned)(n - k + i) / (unsigned)i;
    return v > (unsigned __int128)INT64_MAX ? INT64_MAX : (int64_t)v;
}

struct Req {
    uint64_t ticket = 0;
    tbsci_request r{};
    std::vector<double> h, eri;
    std::vector<uint64_t> alpha, beta;
    bool full_a = false, full_b = false;
    double t_submit = 0, t_admit = -1, t_first = -1;
    size_t bytes = 0;
    int64_t la = 0, lb = 0;
    tbsci_strings *sa = nullptr, *sb = nullptr;
    tbsci_tables *ta = nullptr, *tb = nullptr;
    tbsci_ham *ham = nullptr;
    tbsci::Plan *plan = nullptr;
    tbsci::DavEngine *eng = nullptr;
    cudaEvent_t ready = nullptr;
    cudaStream_t stream = nullptr;  // the solve's stream (priority by size)
    bool waiting_sigma = false;

    void release() {
        if (eng) tbsci::engine_destroy(eng);
        eng = nullptr;
        if (stream) cudaStreamDestroy(stream);
        stream = nullptr;
        if (ready) cudaEventDestroy(ready);
        ready = nullptr;
        tbsci_hamiltonian_destroy(ham);
        tbsci_tables_destroy(ta);
        tbsci_tables_destroy(tb);
        tbsci_strings_destroy(sa);
        tbsci_strings_destroy(sb);
        ham = nullptr;
        ta = tb = nullptr;
        sa = sb = nullptr;
    }
};

// Device bytes one spin's link tables and prepared values take (upper estimate:
// the full-space link counts scaled by the selected fraction of strings).
size_t spin_bytes(int n, int N, int64_t l) {
    const int64_t full = std::max<int64_t>(1, binom64(n, N));
    const double frac = std::min(1.0, (double)l / (double)full);
    const double s1 = (double)N * (n - N) * frac, d2 = (double)binom64(N, 2) * binom64(n - N, 2) * frac;
    // singles: 8 B link + 8 B index + 12 B values; doubles: 12 B link + 4 B + 12 B values
    return (size_t)((double)l * (s1 * 28.0 + d2 * 28.0 + 64.0));
}

}  // namespace

struct tbsci_server {
    tbsci_server_opts opts{};
    tbsci_ctx *ctx = nullptr;   // the scheduler thread's context
    tbsci_ctx *sctx = nullptr;  // the set-up thread's context
    std::thread th, setup_th;
    // requests handed to the set-up thread (owned here) and their outcomes
    std::vector<std::unique_ptr<Req>> in_setup;
    std::mutex smu;
    std::condition_variable scv;
    std::deque<std::pair<Req *, bool>> setup_q;  // request, injected admission failure
    std::vector<std::pair<Req *, tbsci_status>> setup_done;
    bool setup_stop = false;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::unique_ptr<Req>> queue;
    std::vector<std::unique_ptr<Req>> active;
    std::unordered_map<uint64_t, tbsci_result> done;
    std::unordered_map<uint64_t, bool> live;  // submitted tickets not yet collected
    uint64_t next_ticket = 1;
    bool stop = false;
    size_t used = 0;
    int admissions = 0;
    int n_active_pub = 0;
    cudaStream_t sstream = nullptr;
    cudaEvent_t sig_done = nullptr;
    tbsci::BatchScratch scratch;
    Clock::time_point t0;
    int64_t big_job_det = 1 << 20;  // determinants x vectors above which a sigma is not batched
    int prio_low = 0, prio_high = 0;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

    void finish(std::unique_ptr<Req> &q, tbsci_status st) {
        tbsci_result res{};
        res.status = st;
        res.nroots = q->r.nroots;
        res.ndet = q->la * q->lb;
        res.t_submit = q->t_submit;
        res.t_admit = q->t_admit;
        res.t_first_sigma = q->t_first;
        if (q->eng) {
            tbsci_davidson_info info{};
            double e[8] = {0};
            tbsci_status rs = tbsci::engine_results(q->eng, e, nullptr, &info);
            if (st == TBSCI_OK) res.status = rs;
            for (int k = 0; k < q->r.nroots && k < 8; ++k) {
                res.energies[k] = e[k];
                res.residual[k] = info.residual[k];
            }
            res.iterations = info.iterations;
            res.nsigma = info.nsigma;
            res.nsigma_f32 = info.nsigma_f32;
        }
        q->release();
        if (q->t_admit >= 0) used -= std::min(used, q->bytes);
        res.t_done = now();
        std::lock_guard<std::mutex> lk(mu);
        done[q->ticket] = res;
        cv_done.notify_all();
    }

    // Builds a request's device objects (set-up thread, its own context).
    tbsci_status setup(Req &q) {
        tbsci_ctx *c = sctx;
        TB_TRY(tbsci_build_strings(c, q.r.norb, q.r.nalpha, q.full_a ? nullptr : q.alpha.data(),
                                   (int64_t)q.alpha.size(), &q.sa));
        TB_TRY(tbsci_build_strings(c, q.r.norb, q.r.nbeta, q.full_b ? nullptr : q.beta.data(), (int64_t)q.beta.size(),
                                   &q.sb));
        TB_TRY(tbsci_build_excitation_tables(c, q.sa, 0, &q.ta));
        TB_TRY(tbsci_build_excitation_tables(c, q.sb, 0, &q.tb));
        TB_TRY(tbsci_hamiltonian_create(c, q.r.norb, q.h.data(), q.eri.data(), q.r.ecore, &q.ham));
        TB_TRY(tbsci::plan_get(c, q.ham, q.ta, q.tb, &q.plan));
        // small solves get the highest stream priority: the block scheduler then
        // prefers their CTAs over the queued CTAs of large solves
        const bool small = (double)q.la * (double)q.lb * q.r.nroots <= (double)big_job_det;
        TB_CUDA(c, cudaStreamCreateWithPriority(&q.stream, cudaStreamNonBlocking, small ? prio_high : prio_low));
        tbsci_davidson_opts o{};
        o.mixed = q.r.mixed;
        o.tol_energy = q.r.tol_energy;
        o.tol_residual = q.r.tol_residual;
        o.max_iter = q.r.max_iter;
        o.stream = (tbsci_stream)q.stream;
        TB_TRY(tbsci::engine_create(c, q.ham, q.plan, q.r.nroots, &o, &q.eng));
        TB_CUDA(c, cudaEventCreateWithFlags(&q.ready, cudaEventDisableTiming));
        tbsci::engine_set_ctx(q.eng, ctx);  // polled and driven by the scheduler from here on
        return TBSCI_OK;
    }

    void setup_loop() {
        cudaSetDevice(opts.device);
        for (;;) {
            std::pair<Req *, bool> job;
            {
                std::unique_lock<std::mutex> lk(smu);
                scv.wait(lk, [&] { return setup_stop || !setup_q.empty(); });
                if (setup_q.empty()) break;  // stopping, nothing left
                job = setup_q.front();
                setup_q.pop_front();
            }
            const tbsci_status st = job.second ? TBSCI_ENOMEM : setup(*job.first);
            std::lock_guard<std::mutex> lk(smu);
            setup_done.push_back({job.first, st});
        }
    }

    // Moves requests whose set-up finished into the running set (or ends them).
    bool collect_setups() {
        std::vector<std::pair<Req *, tbsci_status>> done_now;
        {
            std::lock_guard<std::mutex> lk(smu);
            done_now.swap(setup_done);
        }
        for (auto &d : done_now) {
            auto it = std::find_if(in_setup.begin(), in_setup.end(),
                                   [&](const std::unique_ptr<Req> &x) { return x.get() == d.first; });
            std::unique_ptr<Req> q = std::move(*it);
            in_setup.erase(it);
            if (d.second != TBSCI_OK) finish(q, d.second);
            else active.push_back(std::move(q));
        }
        return !done_now.empty();
    }

    // Admission in arrival order while a slot and the budget allow.
    bool admit() {
        bool any = false;
        for (;;) {
            std::unique_ptr<Req> q;
            {
                std::lock_guard<std::mutex> lk(mu);
                if (queue.empty() || (int)(active.size() + in_setup.size()) >= opts.max_active) break;
                Req &f = *queue.front();
                if (f.bytes > opts.hbm_budget) {
                    q = std::move(queue.front());
                    queue.pop_front();
                } else if (used + f.bytes > opts.hbm_budget && !(active.empty() && in_setup.empty())) {
                    break;  // wait until running solves release memory
                } else {
                    q = std::move(queue.front());
                    queue.pop_front();
                }
            }
            any = true;
            if (q->bytes > opts.hbm_budget) {
                ctx->err = "request larger than the HBM budget";
                finish(q, TBSCI_ENOMEM);
                continue;
            }
            ++admissions;
            q->t_admit = now();
            used += q->bytes;
            const bool inject = opts.fail_admission_at > 0 && admissions == opts.fail_admission_at;
            Req *raw = q.get();
            in_setup.push_back(std::move(q));
            {
                std::lock_guard<std::mutex> lk(smu);
                setup_q.push_back({raw, inject});
            }
            scv.notify_one();
        }
        return any;
    }

    void round() {
        bool progressed = admit();
        progressed |= collect_setups();
        // host logic of every solve whose device phase has completed
        for (size_t i = 0; i < active.size(); ++i) {
            bool prog = false;
            tbsci_status st = tbsci::engine_poll(active[i]->eng, false, &prog);
            progressed |= prog;
            if (st != TBSCI_OK) {
                finish(active[i], st);
                active.erase(active.begin() + i);
                --i;
            }
        }
        // batched sigma for every solve waiting on one, grouped by sigma type
        std::vector<tbsci::SigmaJob> jobs[4];
        std::vector<Req *> waiting;
        for (auto &q : active) {
            const void *c;
            void *s;
            int k;
            tbsci_dtype dt;
            if (!tbsci::engine_wants_sigma(q->eng, &c, &s, &k, &dt)) continue;
            // large jobs get a launch of their own on their solve's stream, so the
            // batch of small jobs does not wait behind them (it runs beside them)
            const bool big = (double)q->la * (double)q->lb * k > (double)big_job_det;
            if (opts.fuse_sigma < 0 || big) {
                tbsci_status st = tbsci::sigma_launch(ctx, q->ham, q->plan, c, s, k, dt, tbsci::engine_stream(q->eng));
                if (st == TBSCI_OK) st = tbsci::engine_sigma_done(q->eng);
                if (q->t_first < 0) q->t_first = now();
                if (st != TBSCI_OK) q->waiting_sigma = true;  // marks the failure for the sweep below
                progressed = true;
                continue;
            }
            cudaEventRecord(q->ready, tbsci::engine_stream(q->eng));
            cudaStreamWaitEvent(sstream, q->ready, 0);
            jobs[(int)dt].push_back({q->ham, q->plan, c, s, k});
            waiting.push_back(q.get());
        }
        if (!waiting.empty()) {
            tbsci_status bst = TBSCI_OK;
            for (int d = 0; d < 4 && bst == TBSCI_OK; ++d)
                if (!jobs[d].empty())
                    bst = tbsci::sigma_launch_batch(ctx, jobs[d].data(), (int)jobs[d].size(), (tbsci_dtype)d,
                                                    sstream, &scratch);
            cudaEventRecord(sig_done, sstream);
            const double t = now();
            for (Req *q : waiting) {
                cudaStreamWaitEvent(tbsci::engine_stream(q->eng), sig_done, 0);
                tbsci_status st = bst == TBSCI_OK ? tbsci::engine_sigma_done(q->eng) : bst;
                if (st != TBSCI_OK) q->waiting_sigma = true;
                if (q->t_first < 0) q->t_first = t;
            }
            progressed = true;
        }
        // solves whose sigma could not be issued end with the error
        for (size_t i = 0; i < active.size(); ++i) {
            if (active[i]->waiting_sigma) {
                finish(active[i], TBSCI_ECUDA);
                active.erase(active.begin() + i);
                --i;
            }
        }
        // retire
        for (size_t i = 0; i < active.size(); ++i) {
            if (tbsci::engine_done(active[i]->eng)) {
                finish(active[i], TBSCI_OK);
                active.erase(active.begin() + i);
                --i;
                progressed = true;
            }
        }
        {
            std::lock_guard<std::mutex> lk(mu);
            n_active_pub = (int)active.size();
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }

    void loop() {
        cudaSetDevice(opts.device);
        for (;;) {
            {
                std::unique_lock<std::mutex> lk(mu);
                if (stop && active.empty() && in_setup.empty()) break;
                if (queue.empty() && active.empty() && in_setup.empty()) {
                    cv_work.wait_for(lk, std::chrono::milliseconds(20));
                    continue;
                }
            }
            round();
        }
    }
};

extern "C" {

tbsci_status tbsci_server_create(const tbsci_server_opts *o, tbsci_server **out) {
    if (!out) return TBSCI_EINVAL;
    *out = nullptr;
    auto srv = std::make_unique<tbsci_server>();
    if (o) srv->opts = *o;
    if (srv->opts.hbm_budget == 0) srv->opts.hbm_budget = (size_t)60 << 30;
    if (srv->opts.max_active <= 0) srv->opts.max_active = 64;
    if (srv->opts.max_queue <= 0) srv->opts.max_queue = 4096;
    tbsci_status st = tbsci_create(srv->opts.device, &srv->ctx);
    if (st != TBSCI_OK) return st;
    st = tbsci_create(srv->opts.device, &srv->sctx);
    if (st != TBSCI_OK) {
        tbsci_destroy(srv->ctx);
        return st;
    }
    if (srv->opts.tune_cache) {
        st = tbsci_tune_cache_load(srv->ctx, srv->opts.tune_cache);
        if (st == TBSCI_OK) st = tbsci_tune_cache_load(srv->sctx, srv->opts.tune_cache);
        if (st != TBSCI_OK) {
            tbsci_destroy(srv->sctx);
            tbsci_destroy(srv->ctx);
            return st;
        }
    }
    srv->opts.tune_cache = nullptr;  // the caller's string is not kept
    cudaDeviceGetStreamPriorityRange(&srv->prio_low, &srv->prio_high);
    if (cudaStreamCreateWithPriority(&srv->sstream, cudaStreamNonBlocking, srv->prio_high) != cudaSuccess ||
        cudaEventCreateWithFlags(&srv->sig_done, cudaEventDisableTiming) != cudaSuccess) {
        tbsci_destroy(srv->sctx);
        tbsci_destroy(srv->ctx);
        return TBSCI_ECUDA;
    }
    srv->t0 = Clock::now();
    tbsci_server *raw = srv.get();
    srv->setup_th = std::thread([raw] { raw->setup_loop(); });
    srv->th = std::thread([raw] { raw->loop(); });
    *out = srv.release();
    return TBSCI_OK;
}

tbsci_status tbsci_submit(tbsci_server *srv, const tbsci_request *req, uint64_t *ticket) {
    if (!srv || !req || !ticket) return TBSCI_EINVAL;
    const tbsci_request &r = *req;
    if (r.norb < 1 || r.norb > 64 || r.nalpha < 0 || r.nalpha > r.norb || r.nbeta < 0 || r.nbeta > r.norb ||
        r.nroots < 1 || r.nroots > 8 || !r.h || !r.eri || (r.alpha && r.n_alpha < 0) || (r.beta && r.n_beta < 0) ||
        r.mixed < 0 || r.mixed > 3)
        return TBSCI_EINVAL;
    auto q = std::make_unique<Req>();
    q->r = r;
    const size_t n2 = (size_t)r.norb * r.norb;
    q->h.assign(r.h, r.h + n2);
    q->eri.assign(r.eri, r.eri + n2 * n2);
    q->full_a = r.alpha == nullptr;
    q->full_b = r.beta == nullptr;
    if (r.alpha) q->alpha.assign(r.alpha, r.alpha + r.n_alpha);
    if (r.beta) q->beta.assign(r.beta, r.beta + r.n_beta);
    q->la = q->full_a ? binom64(r.norb, r.nalpha) : r.n_alpha;
    q->lb = q->full_b ? binom64(r.norb, r.nbeta) : r.n_beta;
    tbsci_davidson_opts o{};
    o.mixed = r.mixed;
    q->bytes = spin_bytes(r.norb, r.nalpha, q->la) + spin_bytes(r.norb, r.nbeta, q->lb) +
               tbsci::engine_device_bytes(q->la * q->lb, r.nroots, &o) + (size_t)r.norb * r.norb * 64 * (q->lb + 64);
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stop) return TBSCI_EBUSY;
    if ((int)srv->queue.size() >= srv->opts.max_queue) return TBSCI_EAGAIN;
    q->ticket = srv->next_ticket++;
    q->t_submit = srv->now();
    *ticket = q->ticket;
    srv->live[q->ticket] = true;
    srv->queue.push_back(std::move(q));
    srv->cv_work.notify_one();
    return TBSCI_OK;
}

tbsci_status tbsci_poll(tbsci_server *srv, uint64_t ticket, int timeout_ms, tbsci_result *out) {
    if (!srv || !out) return TBSCI_EINVAL;
    std::unique_lock<std::mutex> lk(srv->mu);
    if (!srv->live.count(ticket)) return TBSCI_EINVAL;
    auto ready = [&] { return srv->done.count(ticket) > 0; };
    if (!ready()) {
        if (timeout_ms == 0) return TBSCI_ETIMEOUT;
        if (timeout_ms < 0) srv->cv_done.wait(lk, ready);
        else if (!srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return TBSCI_ETIMEOUT;
    }
    *out = srv->done[ticket];
    srv->done.erase(ticket);
    srv->live.erase(ticket);
    return TBSCI_OK;
}

tbsci_status tbsci_server_load(tbsci_server *srv, int *queued, int *active) {
    if (!srv) return TBSCI_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (queued) *queued = (int)srv->queue.size();
    if (active) *active = srv->n_active_pub;
    return TBSCI_OK;
}

void tbsci_server_destroy(tbsci_server *srv) {
    if (!srv) return;
    std::deque<std::unique_ptr<Req>> dropped;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        dropped.swap(srv->queue);
        srv->cv_work.notify_all();
    }
    if (srv->th.joinable()) srv->th.join();
    {
        std::lock_guard<std::mutex> lk(srv->smu);
        srv->setup_stop = true;
    }
    srv->scv.notify_all();
    if (srv->setup_th.joinable()) srv->setup_th.join();
    for (auto &q : dropped) srv->finish(q, TBSCI_EBUSY);
    cudaSetDevice(srv->opts.device);
    if (srv->sig_done) cudaEventDestroy(srv->sig_done);
    if (srv->sstream) cudaStreamDestroy(srv->sstream);
    tbsci_ctx *ctx = srv->ctx, *sctx = srv->sctx;
    delete srv;
    tbsci_destroy(sctx);
    tbsci_destroy(ctx);
}

}  // extern "C"
