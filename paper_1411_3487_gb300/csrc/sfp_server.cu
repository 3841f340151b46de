// sfp_server.cu -- continuous-batching request loop over pools of slots.
//
// Jobs (chain length, step count, step size, shear rate, noise key) arrive at
// any time through sfp_server_submit.  A worker thread owns the GPU work:
//   admit   each waiting job takes a free slot of a pool with its (length,
//           step size); a new pool is created when none has room and the HBM
//           budget allows it, after evicting idle pools of other shapes if
//           needed.  Admitted slots start from the equilibrium sampler keyed
//           by (seed, job id) with their own step counter at 0.
//   step    every pool with active slots advances by one quantum of steps in
//           one sfp_step call (one fused launch on the tensor-core path); a
//           slot whose job ends inside the quantum stops at its last step
//           (per-slot stop step), so no job runs past its length.
//   retire  finished slots are read back, their results queued for
//           sfp_server_poll, and the slots reused by the next admissions.
//           A slot that has reached its stop step no longer changes, so the
//           jobs that finished in one round are read on a side stream of the
//           pool while the next round's quanta already run: each pool's
//           stream always has its next quantum queued.
// Jobs that arrive while others run join the next quantum of the same launch:
// their work overlaps on the device.  A job's noise is keyed by its own id
// and step counter, so its result does not depend on the slot it ran in or on
// the other jobs in the pool.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/sfp.h"
#include "sfp_internal.h"

namespace {

struct Pool;

struct Job {
    sfp_job desc{};
    uint64_t ticket = 0;
    double dtau = 0.0;
    double t_submit = 0.0, t_admit = -1.0, t_finish = -1.0;
    int32_t status = SFP_OK;
    Pool* pool = nullptr;
    int slot = -1;
    int64_t remaining = 0;          // steps still to run (host mirror of the slot)
    int64_t fin_round = -1;         // the round whose quantum ran the job's last step
    std::vector<double> modes;      // [3][M] after the run (kept if requested)
    double com_nm[3] = {0, 0, 0};
};

struct Pool {
    sfp_batch* b = nullptr;
    cudaStream_t stream = nullptr;  // the pool's own stream: pools of different shapes overlap
    cudaStream_t rs = nullptr;      // reads of finished slots, beside the next quanta
    cudaEvent_t ev[2] = {nullptr, nullptr};   // end of the pool's quantum of round r, in ev[r & 1]
    int M = 0;
    double dtau = 0.0;
    int cap = 0;
    std::vector<Job*> slot_job;     // nullptr = free slot
    int active = 0;                 // slots holding a job (running or waiting to be read)
    int running = 0;                // slots whose job still has steps to run
    size_t bytes = 0;
    // slots admitted in this round, started together
    std::vector<int32_t> st_slot;
    std::vector<uint32_t> st_job;
    std::vector<int64_t> st_stop;
    std::vector<double> st_shear;
};

}  // namespace

struct sfp_server {
    sfp_params params{};
    sfp_server_config cfg{};
    double c_ps = 0.0;
    int device = 0;
    std::chrono::steady_clock::time_point t0;

    // shared with submitting / polling threads, guarded by mu
    std::mutex mu;
    std::condition_variable cv;        // worker wake-up (submissions, stop)
    std::condition_variable cv_done;   // waiters for completions / idle
    std::deque<std::unique_ptr<Job>> jobs;   // every submitted job, index = ticket
    std::deque<Job*> incoming;         // submitted, not yet seen by the worker
    std::deque<Job*> done;             // finished, not yet polled
    std::vector<double> latencies;     // finish - submit of every finished job
    bool abort = false;
    int64_t n_pending = 0, n_active = 0, n_finished = 0;
    double bead_steps_done = 0.0;
    size_t held = 0;
    int32_t worker_error = SFP_OK;
    std::string worker_msg;

    // owned by the worker thread
    int64_t round = 0;                 // quanta issued so far
    std::deque<Job*> pending;
    std::vector<std::unique_ptr<Pool>> pools;
    std::thread worker;

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

thread_local std::string g_srv_err;

int srv_fail(int code, const std::string& msg)
{
    g_srv_err = msg;
    return code;
}

// Create a pool of cap slots for (M, dtau) within the remaining budget;
// SFP_ENOMEM when it does not fit.
int make_pool(sfp_server* s, int M, double dtau, int cap, std::unique_ptr<Pool>* out)
{
    std::vector<sfp_chain_desc> d(cap);
    for (int i = 0; i < cap; ++i) {
        d[i] = sfp_chain_desc{};
        d[i].n_beads = M;
        d[i].dtau = dtau;
        d[i].job_id = (uint64_t)i;
    }
    size_t left = 0;
    if (s->cfg.hbm_budget_bytes) {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->held >= s->cfg.hbm_budget_bytes) return SFP_ENOMEM;
        left = s->cfg.hbm_budget_bytes - s->held;
    }
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
        return srv_fail(SFP_ECUDA, "pool stream creation failed");
    sfp_batch* b = nullptr;
    int rc = sfp_create(&s->params, d.data(), cap, s->cfg.seed, s->cfg.precision, st, left, &b);
    if (rc) {
        cudaStreamDestroy(st);
        return rc;
    }
    if ((rc = sfp::internal_idle_all(b))) {
        sfp_destroy(b);
        cudaStreamDestroy(st);
        return rc;
    }
    std::unique_ptr<Pool> p(new Pool());
    p->stream = st;
    if (cudaStreamCreateWithFlags(&p->rs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev[1], cudaEventDisableTiming) != cudaSuccess) {
        if (p->rs) cudaStreamDestroy(p->rs);
        for (cudaEvent_t e : p->ev)
            if (e) cudaEventDestroy(e);
        sfp_destroy(b);
        cudaStreamDestroy(st);
        return srv_fail(SFP_ECUDA, "pool stream creation failed");
    }
    sfp::internal_shape(b, nullptr, nullptr, nullptr, &p->bytes);
    p->b = b;
    p->M = M;
    p->dtau = dtau;
    p->cap = cap;
    p->slot_job.assign(cap, nullptr);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->held += p->bytes;
    }
    *out = std::move(p);
    return SFP_OK;
}

void release_pool(Pool& p)
{
    sfp_destroy(p.b);
    cudaStreamDestroy(p.stream);
    cudaStreamDestroy(p.rs);
    for (cudaEvent_t e : p.ev) cudaEventDestroy(e);
}

void drop_pool(sfp_server* s, size_t i)
{
    release_pool(*s->pools[i]);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->held -= s->pools[i]->bytes;
    }
    s->pools.erase(s->pools.begin() + (long)i);
}

int find_free(const Pool& p)
{
    for (int k = 0; k < p.cap; ++k)
        if (!p.slot_job[k]) return k;
    return -1;
}

// Give waiting jobs free slots (FIFO; a job that cannot be placed does not
// block jobs of other shapes behind it), then start the new slots.
int admit(sfp_server* s)
{
    std::deque<Job*> still;
    bool budget_full = false;
    while (!s->pending.empty()) {
        Job* j = s->pending.front();
        s->pending.pop_front();
        Pool* pool = nullptr;
        int slot = -1;
        for (auto& p : s->pools)
            if (p->M == j->desc.n_beads && p->dtau == j->dtau && (slot = find_free(*p)) >= 0) {
                pool = p.get();
                break;
            }
        if (!pool && !budget_full) {
            std::unique_ptr<Pool> np;
            int cap = s->cfg.slots_per_pool;
            int rc = make_pool(s, j->desc.n_beads, j->dtau, cap, &np);
            while (rc == SFP_ENOMEM) {
                // evict an idle pool (no running and no just-admitted slots) and retry;
                // with none left, try a pool of half as many slots
                size_t victim = s->pools.size();
                for (size_t k = 0; k < s->pools.size(); ++k)
                    if (s->pools[k]->active == 0) {
                        victim = k;
                        break;
                    }
                if (victim < s->pools.size()) {
                    drop_pool(s, victim);
                } else if (cap > 1) {
                    cap = std::max(1, cap / 2);
                } else {
                    break;
                }
                rc = make_pool(s, j->desc.n_beads, j->dtau, cap, &np);
            }
            if (rc == SFP_OK) {
                s->pools.push_back(std::move(np));
                pool = s->pools.back().get();
                slot = 0;
            } else if (rc == SFP_ENOMEM) {
                bool running = false;
                for (auto& p : s->pools) running = running || p->active > 0;
                if (!running) {
                    // nothing will free memory: this job can never fit the budget
                    std::lock_guard<std::mutex> lk(s->mu);
                    j->status = SFP_ENOMEM;
                    j->t_admit = j->t_finish = s->now();
                    s->done.push_back(j);
                    s->latencies.push_back(j->t_finish - j->t_submit);
                    s->n_pending--;
                    s->n_finished++;
                    s->cv_done.notify_all();
                    continue;
                }
                budget_full = true;
            } else {
                return srv_fail(rc, std::string("pool creation failed: ") + sfp_last_error());
            }
        }
        if (!pool) {
            still.push_back(j);
            continue;
        }
        pool->slot_job[slot] = j;
        pool->active++;
        pool->running++;
        j->pool = pool;
        j->slot = slot;
        j->remaining = j->desc.n_steps;
        j->t_admit = s->now();
        pool->st_slot.push_back(slot);
        pool->st_job.push_back((uint32_t)j->desc.job_id);
        pool->st_stop.push_back(j->desc.n_steps);
        pool->st_shear.push_back(j->desc.shear_rate_per_s);
        std::lock_guard<std::mutex> lk(s->mu);
        s->n_pending--;
        s->n_active++;
    }
    s->pending.swap(still);
    for (auto& p : s->pools) {
        if (p->st_slot.empty()) continue;
        const int rc = sfp::internal_slots_start(p->b, p->st_slot.data(), p->st_job.data(), p->st_stop.data(),
                                                 p->st_shear.data(), (int32_t)p->st_slot.size());
        p->st_slot.clear();
        p->st_job.clear();
        p->st_stop.clear();
        p->st_shear.clear();
        if (rc) return srv_fail(rc, std::string("slot start failed: ") + sfp_last_error());
    }
    return SFP_OK;
}

// Read back and release the slots whose jobs have run all their steps.
// Read back and hand out the jobs that ran their last step in a round up to
// `upto`.  side: each pool reads on its side stream after the event of round
// upto (the next round's quanta may run meanwhile), else after everything
// queued on the pool's stream.
int retire(sfp_server* s, int64_t upto, bool side)
{
    for (auto& pp : s->pools) {
        Pool& p = *pp;
        std::vector<int32_t> fin;
        for (int c = 0; c < p.cap; ++c)
            if (p.slot_job[c] && p.slot_job[c]->fin_round >= 0 && p.slot_job[c]->fin_round <= upto) fin.push_back(c);
        if (fin.empty()) continue;
        const int n = (int)fin.size();
        std::vector<double> modes(s->cfg.keep_results ? (size_t)n * 3 * p.M : 0), com((size_t)n * 3);
        std::vector<int64_t> steps(n);
        const int rc = sfp::internal_slots_read(p.b, fin.data(), n, s->cfg.keep_results ? modes.data() : nullptr,
                                                com.data(), steps.data(), side ? p.rs : nullptr,
                                                side ? p.ev[upto & 1] : nullptr);
        const double t = s->now();
        std::lock_guard<std::mutex> lk(s->mu);
        for (int i = 0; i < n; ++i) {
            Job* j = p.slot_job[fin[i]];
            j->t_finish = t;
            j->status = rc ? rc : (steps[i] == j->desc.n_steps ? SFP_OK : SFP_ECUDA);
            std::memcpy(j->com_nm, &com[(size_t)3 * i], sizeof j->com_nm);
            if (s->cfg.keep_results)
                j->modes.assign(modes.begin() + (long)i * 3 * p.M, modes.begin() + (long)(i + 1) * 3 * p.M);
            j->pool = nullptr;
            j->slot = -1;
            p.slot_job[fin[i]] = nullptr;
            p.active--;
            s->done.push_back(j);
            s->latencies.push_back(j->t_finish - j->t_submit);
            s->bead_steps_done += (double)j->desc.n_beads * (double)j->desc.n_steps;
            s->n_active--;
            s->n_finished++;
        }
        s->cv_done.notify_all();
        if (rc) return srv_fail(rc, std::string("slot read failed: ") + sfp_last_error());
    }
    return SFP_OK;
}

void worker_main(sfp_server* s)
{
    cudaSetDevice(s->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->abort) break;
            if (s->pending.empty() && s->n_active == 0 && s->incoming.empty()) {
                s->cv_done.notify_all();
                s->cv.wait_for(lk, std::chrono::milliseconds(50));
                if (s->abort) break;
            }
            while (!s->incoming.empty()) {
                s->pending.push_back(s->incoming.front());
                s->incoming.pop_front();
            }
        }
        int rc = admit(s);
        if (!rc) {
            // one quantum of every pool with running slots, each on its own stream
            // (queued without waiting, so the shapes share the GPU), the pool
            // with the most work (running slots x M^2) first; an event marks the
            // end of each pool's quantum of this round
            const int64_t r = s->round;
            std::vector<Pool*> order;
            for (auto& p : s->pools)
                if (p->running > 0) order.push_back(p.get());
            std::stable_sort(order.begin(), order.end(), [](const Pool* x, const Pool* y) {
                return (double)x->running * x->M * x->M > (double)y->running * y->M * y->M;
            });
            for (Pool* p : order) {
                // the quantum covers the slots up to the highest running one
                int top = 0;
                for (int c = 0; c < p->cap; ++c)
                    if (p->slot_job[c] && p->slot_job[c]->fin_round < 0) top = c + 1;
                sfp::internal_set_active(p->b, top);
                rc = sfp_step(p->b, s->cfg.quantum_steps);
                if (!rc && cudaEventRecord(p->ev[r & 1], p->stream) != cudaSuccess) rc = SFP_ECUDA;
                if (rc) {
                    srv_fail(rc, std::string("step failed: ") + sfp_last_error());
                    break;
                }
                for (Job* j : p->slot_job)
                    if (j && j->fin_round < 0) {
                        j->remaining -= s->cfg.quantum_steps;
                        if (j->remaining <= 0) {
                            j->fin_round = r;
                            p->running--;
                        }
                    }
            }
            if (!rc) {
                // the jobs of the previous round are read while this round runs; with
                // nothing queued this round, every finished job at once
                rc = order.empty() ? retire(s, r, false) : retire(s, r - 1, true);
                s->round++;
            }
        }
        if (rc) {
            std::lock_guard<std::mutex> lk(s->mu);
            s->worker_error = rc;
            s->worker_msg = g_srv_err;
            s->cv_done.notify_all();
            break;
        }
    }
    for (auto& p : s->pools) release_pool(*p);
    s->pools.clear();
    std::lock_guard<std::mutex> lk(s->mu);
    s->held = 0;
    s->cv_done.notify_all();
}

double percentile(std::vector<double> v, double q)
{
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (double)(v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - (double)i;
    return i + 1 < v.size() ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
}

}  // namespace

extern "C" {

int sfp_server_config_default(sfp_server_config* c)
{
    if (!c) return srv_fail(SFP_EINVAL, "config is NULL");
    *c = sfp_server_config{};
    c->seed = 1;
    c->precision = SFP_FP32;
    c->hbm_budget_bytes = 0;
    c->slots_per_pool = 512;
    c->quantum_steps = 64;
    c->keep_results = 1;
    return SFP_OK;
}

int sfp_server_create(const sfp_params* params, const sfp_server_config* cfg, sfp_server** out)
{
    if (!out) return srv_fail(SFP_EINVAL, "out is NULL");
    *out = nullptr;
    if (!params || !cfg) return srv_fail(SFP_EINVAL, "params and config are required");
    if (cfg->slots_per_pool < 1 || cfg->quantum_steps < 1) return srv_fail(SFP_EINVAL, "slots_per_pool and quantum_steps must be >= 1");
    if (cfg->seed >> 32) return srv_fail(SFP_EINVAL, "seed must be < 2^32");
    double dv[8];
    int rc = sfp_derive(params, dv);
    if (rc) return srv_fail(rc, sfp_last_error());
    sfp_server* s = new sfp_server();
    s->params = *params;
    s->cfg = *cfg;
    s->c_ps = dv[2];
    s->t0 = std::chrono::steady_clock::now();
    const cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) {
        delete s;
        return srv_fail(SFP_ECUDA, std::string("server device: ") + cudaGetErrorString(e));
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return SFP_OK;
}

int sfp_server_submit(sfp_server* s, const sfp_job* job, uint64_t* ticket)
{
    if (!s || !job) return srv_fail(SFP_EINVAL, "NULL argument");
    if (job->n_beads < 3 || job->n_beads > 4096) return srv_fail(SFP_EINVAL, "n_beads outside 3..4096");
    if (job->n_steps < 0) return srv_fail(SFP_EINVAL, "n_steps < 0");
    if (job->job_id >> 32) return srv_fail(SFP_EINVAL, "job_id must be < 2^32");
    if (job->reserved != 0) return srv_fail(SFP_EINVAL, "reserved must be 0");
    const double dtau = job->dtau > 0.0 ? job->dtau : job->dt_ps / s->c_ps;
    if (!(dtau > 0.0) || !std::isfinite(dtau)) return srv_fail(SFP_EINVAL, "step must be > 0");
    if (!std::isfinite(job->shear_rate_per_s)) return srv_fail(SFP_EINVAL, "shear rate not finite");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->worker_error) return srv_fail(s->worker_error, "server stopped after an error: " + s->worker_msg);
    std::unique_ptr<Job> j(new Job());
    j->desc = *job;
    j->dtau = dtau;
    j->ticket = (uint64_t)s->jobs.size();
    j->t_submit = s->now();
    s->incoming.push_back(j.get());
    if (ticket) *ticket = j->ticket;
    s->jobs.push_back(std::move(j));
    s->n_pending++;
    s->cv.notify_one();
    return SFP_OK;
}

int sfp_server_poll(sfp_server* s, sfp_job_result* out, int32_t max_results, int32_t* n_out)
{
    if (!s || !n_out || (max_results > 0 && !out)) return srv_fail(SFP_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    int32_t n = 0;
    while (n < max_results && !s->done.empty()) {
        const Job& j = *s->done.front();
        s->done.pop_front();
        sfp_job_result& r = out[n++];
        r = sfp_job_result{};
        r.ticket = j.ticket;
        r.job_id = j.desc.job_id;
        r.n_beads = j.desc.n_beads;
        r.status = j.status;
        r.n_steps = j.desc.n_steps;
        r.submit_s = j.t_submit;
        r.admit_s = j.t_admit;
        r.finish_s = j.t_finish;
        std::memcpy(r.com_nm, j.com_nm, sizeof r.com_nm);
    }
    *n_out = n;
    return s->worker_error ? srv_fail(s->worker_error, s->worker_msg) : SFP_OK;
}

int sfp_server_result_modes(sfp_server* s, uint64_t ticket, double* host_modes, size_t n_doubles)
{
    if (!s || !host_modes) return srv_fail(SFP_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    if (ticket >= s->jobs.size()) return srv_fail(SFP_EINVAL, "unknown ticket");
    const Job& j = *s->jobs[ticket];
    if (j.t_finish < 0.0) return srv_fail(SFP_EINVAL, "job has not finished");
    if (j.modes.empty()) return srv_fail(SFP_EINVAL, "results are not kept (keep_results = 0)");
    if (n_doubles < j.modes.size()) return srv_fail(SFP_EINVAL, "buffer too small");
    std::memcpy(host_modes, j.modes.data(), j.modes.size() * sizeof(double));
    return SFP_OK;
}

int sfp_server_wait_idle(sfp_server* s, double timeout_s)
{
    if (!s) return srv_fail(SFP_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (s->n_pending > 0 || s->n_active > 0) {
        if (s->worker_error) return srv_fail(s->worker_error, s->worker_msg);
        if (s->cv_done.wait_until(lk, until) == std::cv_status::timeout) return srv_fail(SFP_ETIMEDOUT, "jobs still running");
    }
    return s->worker_error ? srv_fail(s->worker_error, s->worker_msg) : SFP_OK;
}

int sfp_server_stats(sfp_server* s, double out[10])
{
    if (!s || !out) return srv_fail(SFP_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    out[0] = (double)s->jobs.size();
    out[1] = (double)s->n_finished;
    out[2] = (double)s->n_pending;
    out[3] = (double)s->n_active;
    out[4] = (double)s->held;
    out[5] = percentile(s->latencies, 0.50);
    out[6] = percentile(s->latencies, 0.99);
    out[7] = s->latencies.empty() ? 0.0 : *std::max_element(s->latencies.begin(), s->latencies.end());
    out[8] = s->now();
    out[9] = s->bead_steps_done;
    return SFP_OK;
}

int sfp_server_destroy(sfp_server* s)
{
    if (!s) return SFP_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->abort = true;
        s->cv.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    delete s;
    return SFP_OK;
}

const char* sfp_server_last_error(void) { return g_srv_err.c_str(); }

}  // extern "C"
