// md_server.cu -- continuous-batching request loop over pools (host code).
//
// One pool per potential kind, each driven by its own host thread:
//   admit:   while the FIFO queue's head fits (md_batch_add succeeds: a free system slot
//            and free atom/cell ranges, i.e. the job's device footprint), admit it;
//   step:    md_run(chunk) -- every admitted job advances together, each stopping on
//            the device when its step budget runs out;
//   harvest: jobs that stopped are read back (final state into the job's buffers,
//            energies), removed, and timestamped; their slots admit the next jobs.
// Jobs are submitted from any thread; submission copies the inputs, so the caller's
// arrays may be reused at once.  The pools run on separate CUDA streams, so the two
// kinds' kernels overlap on the device.
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

#include <cuda_runtime.h>

#include "md.h"

namespace {

using Clock = std::chrono::steady_clock;
constexpr double kHeadWait = 0.5;   // seconds a job that does not fit lets later ones pass

struct Job {
    int64_t id = 0;
    int kind = 0, param_set = 0;
    double box[3] = {0, 0, 0};
    int pbc[3] = {0, 0, 0};
    int64_t n = 0, n_steps = 0;
    double damp = 0;
    std::vector<int32_t> types;
    std::vector<double> x, y, z, vx, vy, vz;
    double *x_out = nullptr, *v_out = nullptr;
    md_job_result res{};
    int slot = -1;
};

struct PoolRunner {
    int kind = 0;
    double dt = 1.0;
    int max_jobs = 0;
    md_ctx *ctx = nullptr;
    std::deque<std::shared_ptr<Job>> queue;          // guarded by the server mutex
    std::map<int, std::shared_ptr<Job>> running;     // slot -> job (runner thread only)
    std::thread th;
};

}  // namespace

struct md_server {
    md_server_options opt{};
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::map<int64_t, std::shared_ptr<Job>> jobs;
    int64_t next_id = 1;
    md_server_stats stats{};
    PoolRunner pools[2];   // 0: Tersoff, 1: SW
    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

void finish(md_server *srv, const std::shared_ptr<Job> &j, int status)
{
    std::lock_guard<std::mutex> lk(srv->mu);
    j->res.done = 1;
    j->res.status = status;
    j->res.t_done = srv->now();
    if (status == MD_OK) {
        srv->stats.completed += 1;
        srv->stats.atom_steps += (double)j->n * (double)j->n_steps;
    } else {
        srv->stats.failed += 1;
    }
    srv->cv_done.notify_all();
}

md_status admit(md_server *srv, PoolRunner &pr, const std::shared_ptr<Job> &j)
{
    md_system sd;
    std::memset(&sd, 0, sizeof(sd));
    for (int a = 0; a < 3; ++a) {
        sd.box[a] = j->box[a];
        sd.pbc[a] = j->pbc[a];
    }
    sd.n_atoms = j->n;
    sd.types = j->types.data();
    sd.param_set = j->param_set;
    sd.x = j->x.data(); sd.y = j->y.data(); sd.z = j->z.data();
    sd.vx = j->vx.data(); sd.vy = j->vy.data(); sd.vz = j->vz.data();
    sd.n_steps = j->n_steps;
    sd.damp = j->damp;
    int slot = -1;
    md_status s = md_batch_add(pr.ctx, &sd, &slot);
    if (s == MD_OK) {
        j->slot = slot;
        pr.running[slot] = j;
        std::lock_guard<std::mutex> lk(srv->mu);
        j->res.t_admit = srv->now();
        srv->stats.admitted += 1;
        // the inputs live on the device now
        std::vector<double>().swap(j->x); std::vector<double>().swap(j->y); std::vector<double>().swap(j->z);
        std::vector<double>().swap(j->vx); std::vector<double>().swap(j->vy); std::vector<double>().swap(j->vz);
    }
    return s;
}

void runner(md_server *srv, int which)
{
    PoolRunner &pr = srv->pools[which];
    cudaSetDevice(srv->opt.device);
    std::vector<int> active(pr.max_jobs);
    std::vector<int64_t> left(pr.max_jobs);
    std::vector<double> tot((size_t)pr.max_jobs * 13), kin(pr.max_jobs);
    std::vector<int> err(pr.max_jobs);
    const int chunk = srv->opt.chunk_steps > 0 ? srv->opt.chunk_steps : 8;
    double busy_since = -1.0;
    for (;;) {
        // admission: first fit over the queue in arrival order.  A job that does not fit
        // yet (no free slot, or no contiguous range for its atoms in the fragmented pool)
        // lets later jobs pass, unless it has waited longer than kHeadWait: then it
        // blocks the queue until it fits, so large jobs are not starved.
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            srv->cv_work.wait(lk, [&] { return srv->stop || !pr.queue.empty() || !pr.running.empty(); });
            if (srv->stop && pr.queue.empty() && pr.running.empty()) break;
            for (size_t qi = 0; qi < pr.queue.size();) {
                std::shared_ptr<Job> j = pr.queue[qi];
                lk.unlock();
                const double t_a = srv->now();
                const md_status s = admit(srv, pr, j);
                lk.lock();
                srv->stats.admit_seconds += srv->now() - t_a;
                if (s == MD_OK) {
                    pr.queue.erase(pr.queue.begin() + (long)qi);
                } else if (s == MD_ERR_OOM && !pr.running.empty()) {
                    if (srv->now() - j->res.t_submit > kHeadWait) break;   // it waits; so do the rest
                    ++qi;
                } else {
                    pr.queue.erase(pr.queue.begin() + (long)qi);   // can never fit, or invalid
                    lk.unlock();
                    finish(srv, j, s);
                    lk.lock();
                }
            }
        }
        if (pr.running.empty()) continue;
        if (busy_since < 0) busy_since = srv->now();
        const double t_run = srv->now();
        double resident = 0;
        for (auto &kv : pr.running) resident += (double)kv.second->n;
        md_status s = md_run(pr.ctx, chunk, pr.dt, nullptr);
        if (s == MD_OK) s = md_batch_status(pr.ctx, active.data(), left.data(), tot.data(), kin.data());
        bool any_stopped = false;
        for (auto &kv : pr.running) any_stopped |= active[kv.first] == 0;
        if (s == MD_OK && any_stopped) s = md_batch_errors(pr.ctx, err.data());   // why they stopped
        const double t_harvest = srv->now();
        if (s != MD_OK) {   // the pool itself failed (a CUDA error): fail every running job
            for (auto &kv : pr.running) {
                md_batch_remove(pr.ctx, kv.first);
                finish(srv, kv.second, s);
            }
            pr.running.clear();
            continue;
        }
        // a job that failed on the device (non-finite values, an overlong list, ...) was
        // stopped there alone: it fails with that status, the others go on
        std::vector<int> done;
        for (auto &kv : pr.running)
            if (active[kv.first] == 0) done.push_back(kv.first);
        for (int slot : done) {
            std::shared_ptr<Job> j = pr.running[slot];
            if (err[slot] != MD_OK) {
                md_batch_remove(pr.ctx, slot);
                pr.running.erase(slot);
                finish(srv, j, err[slot]);
                continue;
            }
            const md_status g = md_batch_get_state(pr.ctx, slot, j->x_out, j->v_out);
            j->res.U = tot[(size_t)slot * 13];
            j->res.K = kin[slot];
            md_batch_remove(pr.ctx, slot);
            pr.running.erase(slot);
            finish(srv, j, g);
        }
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            srv->stats.run_seconds += t_harvest - t_run;
            srv->stats.resident_atom_steps += resident * chunk;
            srv->stats.harvest_seconds += srv->now() - t_harvest;
            srv->stats.chunks += 1;
            if (pr.running.empty() && busy_since >= 0) {
                srv->stats.busy_seconds += srv->now() - busy_since;
                busy_since = -1.0;
            }
        }
    }
}

}  // namespace

extern "C" {

md_status md_server_create(md_server **out, const md_server_options *opt, const md_params *tersoff_sets,
                           const double *tersoff_masses, const md_params *sw_set, const double *sw_mass)
{
    if (!out || !opt) return MD_ERR_ARG;
    *out = nullptr;
    if (opt->max_jobs_per_pool < 1) return MD_ERR_ARG;
    if (opt->tersoff_atoms > 0 && (!tersoff_sets || !tersoff_masses || !(opt->tersoff_dt > 0))) return MD_ERR_ARG;
    if (opt->sw_atoms > 0 && (!sw_set || !sw_mass || !(opt->sw_dt > 0))) return MD_ERR_ARG;
    md_server *srv = new md_server();
    srv->opt = *opt;
    srv->t0 = Clock::now();
    md_options mo;
    md_default_options(&mo);
    mo.precision = opt->precision;
    mo.device = opt->device;
    for (int w = 0; w < 2; ++w) {
        PoolRunner &pr = srv->pools[w];
        pr.kind = w == 0 ? MD_TERSOFF : MD_SW;
        pr.max_jobs = opt->max_jobs_per_pool;
        const int64_t cap = w == 0 ? opt->tersoff_atoms : opt->sw_atoms;
        if (cap <= 0) continue;
        pr.dt = w == 0 ? opt->tersoff_dt : opt->sw_dt;
        const md_status s = w == 0 ? md_batch_create(&pr.ctx, cap, pr.max_jobs, 2, tersoff_sets, 2, tersoff_masses,
                                                     nullptr, &mo)
                                   : md_batch_create(&pr.ctx, cap, pr.max_jobs, 1, sw_set, 1, sw_mass, nullptr, &mo);
        if (s != MD_OK) {
            md_server_destroy(srv);
            return s;
        }
    }
    for (int w = 0; w < 2; ++w)
        if (srv->pools[w].ctx) srv->pools[w].th = std::thread(runner, srv, w);
    *out = srv;
    return MD_OK;
}

md_status md_server_submit(md_server *srv, const md_job *job, int64_t *job_id)
{
    if (!srv || !job || !job_id) return MD_ERR_ARG;
    const int w = job->kind == MD_TERSOFF ? 0 : (job->kind == MD_SW ? 1 : -1);
    if (w < 0 || !srv->pools[w].ctx) return MD_ERR_ARG;
    if (job->n_atoms < 1 || job->n_steps < 1 || !job->x || !job->y || !job->z || !job->types) return MD_ERR_ARG;
    auto j = std::make_shared<Job>();
    j->kind = job->kind;
    j->param_set = job->param_set;
    for (int a = 0; a < 3; ++a) {
        j->box[a] = job->box[a];
        j->pbc[a] = job->pbc[a];
    }
    j->n = job->n_atoms;
    j->n_steps = job->n_steps;
    j->damp = job->damp;
    const size_t n = (size_t)job->n_atoms;
    j->types.assign(job->types, job->types + n);
    j->x.assign(job->x, job->x + n);
    j->y.assign(job->y, job->y + n);
    j->z.assign(job->z, job->z + n);
    j->vx = job->vx ? std::vector<double>(job->vx, job->vx + n) : std::vector<double>(n, 0.0);
    j->vy = job->vy ? std::vector<double>(job->vy, job->vy + n) : std::vector<double>(n, 0.0);
    j->vz = job->vz ? std::vector<double>(job->vz, job->vz + n) : std::vector<double>(n, 0.0);
    j->x_out = job->x_out;
    j->v_out = job->v_out;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        j->id = srv->next_id++;
        j->res.t_submit = srv->now();
        srv->jobs[j->id] = j;
        srv->pools[w].queue.push_back(j);
        srv->stats.submitted += 1;
    }
    srv->cv_work.notify_all();
    *job_id = j->id;
    return MD_OK;
}

md_status md_server_poll(md_server *srv, int64_t job_id, md_job_result *out)
{
    if (!srv || !out) return MD_ERR_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(job_id);
    if (it == srv->jobs.end()) return MD_ERR_ARG;
    *out = it->second->res;
    return MD_OK;
}

md_status md_server_wait(md_server *srv, int64_t job_id, md_job_result *out)
{
    if (!srv) return MD_ERR_ARG;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(job_id);
    if (it == srv->jobs.end()) return MD_ERR_ARG;
    std::shared_ptr<Job> j = it->second;
    srv->cv_done.wait(lk, [&] { return j->res.done != 0; });
    if (out) *out = j->res;
    return MD_OK;
}

md_status md_server_wait_timeout(md_server *srv, int64_t job_id, double timeout_s, md_job_result *out)
{
    if (!srv || !(timeout_s >= 0)) return MD_ERR_ARG;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(job_id);
    if (it == srv->jobs.end()) return MD_ERR_ARG;
    std::shared_ptr<Job> j = it->second;
    const auto limit = std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    const bool done = srv->cv_done.wait_for(lk, limit, [&] { return j->res.done != 0; });
    if (out) *out = j->res;
    return done ? MD_OK : MD_ERR_TIMEOUT;
}

md_status md_server_drain(md_server *srv)
{
    if (!srv) return MD_ERR_ARG;
    std::unique_lock<std::mutex> lk(srv->mu);
    srv->cv_done.wait(lk, [&] { return srv->stats.completed + srv->stats.failed >= srv->stats.submitted; });
    return MD_OK;
}

md_status md_server_stats_get(md_server *srv, md_server_stats *out)
{
    if (!srv || !out) return MD_ERR_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    *out = srv->stats;
    return MD_OK;
}

double md_server_clock(const md_server *srv) { return srv ? srv->now() : 0.0; }

void md_server_destroy(md_server *srv)
{
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    for (auto &pr : srv->pools)
        if (pr.th.joinable()) pr.th.join();
    for (auto &pr : srv->pools)
        if (pr.ctx) md_destroy(pr.ctx);
    delete srv;
}

}  // extern "C"
