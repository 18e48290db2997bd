// Serving (declared in include/dilbm.h): continuous batching of DI-LBM jobs.
//
// Every admitted job is an ordinary context (dilbm_create) that stays
// resident on the device until it has run its steps; all running jobs of one
// storage type advance together as one batch (dilbm_batch_*), so that one
// sweep launch and one particle launch per step cover every lattice in the
// mix.  With per-job storage the batches of the storage types present run
// side by side (each on its own stream), by the same macro-steps.  The server only
// decides who runs: it admits queued jobs by free job slots and by a device
// memory budget, cuts the run into macro-steps no longer than the shortest
// remaining job, and re-forms the batch when jobs join or leave.  The method
// itself (Eqs. 13-19, 22-24, 28-29) is untouched, so every job's result is
// the one dilbm_step gives it alone.
#include "dilbm.h"
#include "dilbm_trace.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <memory>
#include <string>
#include <unordered_map>
#include <vector>

namespace dilbm {
int set_last_error(int code, const std::string &msg);
int check_problem(const dilbm_grid *g, dilbm_lattice lattice, double tau, double interface_width,
                  const dilbm_particle *particles, int np);
}  // namespace dilbm

namespace {

int sfail(int code, const std::string &msg) { return dilbm::set_last_error(code, msg); }

int scuda(cudaError_t e, const char *what) {
    return sfail(e == cudaErrorMemoryAllocation ? DILBM_ERR_OOM : DILBM_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

constexpr int MAX_JOBS = 1024;
constexpr int NSTORE = 3;             // FP32, FP16, BF16 deviations: one batch each

struct Job {
    long long id = 0;
    dilbm_grid grid{};
    double tau = 0.0, eps = 0.0;
    std::vector<dilbm_particle> parts;
    long long nsteps = 0, done = 0, window = 0;
    int state = DILBM_JOB_QUEUED;
    int error = DILBM_OK;
    double arrival = -1.0, admitted = -1.0, finished = -1.0;
    unsigned long long footprint = 0;
    double nodes = 0.0;
    dilbm_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;       // the job's own stream (set-up and read-back)
    std::vector<double> force, force_mean;   // np x 3 at DONE
    std::vector<dilbm_particle> final_state;
};

}  // namespace

struct dilbm_server {
    dilbm_server_config cfg{};
    unsigned long long budget = 0;
    unsigned long long in_use = 0;
    std::chrono::steady_clock::time_point t0;
    std::unordered_map<long long, std::unique_ptr<Job>> jobs;
    std::deque<Job *> queue;              // arrival (submit) order
    std::vector<Job *> running;           // admitted, not yet finished
    std::vector<Job *> members[NSTORE];   // the jobs of each storage type's batch, in member order
    dilbm_batch *batch[NSTORE] = {};
    bool dirty = false;                   // running set changed since the batch was formed
    long long next_id = 0;
    long long n_done = 0, n_failed = 0, macro = 0;
    double node_updates = 0.0, busy = 0.0, t_form = 0.0, t_admit = 0.0, t_wait = 0.0, t_retire = 0.0;
    long long launches_gone = 0;          // kernels of destroyed contexts and batches

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

// Free a job's device memory (its context and stream) and return its budget.
void release(dilbm_server *s, Job *j) {
    if (j->ctx) {
        s->launches_gone += dilbm_launch_count(j->ctx);
        dilbm_destroy(j->ctx);
        j->ctx = nullptr;
        s->in_use -= j->footprint;
    }
    if (j->stream) {
        cudaStreamDestroy(j->stream);
        j->stream = nullptr;
    }
}

void drop_batch(dilbm_server *s) {
    for (int c = 0; c < NSTORE; ++c)
        if (s->batch[c]) {
            s->launches_gone += dilbm_batch_launch_count(s->batch[c]);
            dilbm_batch_destroy(s->batch[c]);
            s->batch[c] = nullptr;
        }
}

bool has_batch(const dilbm_server *s) {
    for (int c = 0; c < NSTORE; ++c)
        if (s->batch[c]) return true;
    return false;
}

// Admit queued jobs while a slot is free and the budget allows.  A job that
// cannot be created for lack of device memory stays queued (the memory of
// running jobs returns as they finish) unless nothing else holds memory.
int admit(dilbm_server *s) {
    int added = 0;
    for (auto it = s->queue.begin(); it != s->queue.end();) {
        if ((int)s->running.size() >= s->cfg.max_jobs) break;
        Job *j = *it;
        if (s->in_use + j->footprint > s->budget) {
            if (s->cfg.policy == DILBM_ADMIT_FIFO) break;
            ++it;
            continue;
        }
        cudaError_t e = cudaStreamCreateWithFlags(&j->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return scuda(e, "cudaStreamCreateWithFlags");
        const int rc = dilbm_create(&j->grid, DILBM_D2Q9, j->tau, j->eps, j->parts.empty() ? nullptr : j->parts.data(),
                                    (int)j->parts.size(), j->stream, &j->ctx);
        if (rc == DILBM_ERR_OOM && (!s->running.empty() || s->in_use > 0)) {
            cudaStreamDestroy(j->stream);
            j->stream = nullptr;
            break;                                      // retry when memory returns
        }
        it = s->queue.erase(it);
        if (rc != DILBM_OK) {
            cudaStreamDestroy(j->stream);
            j->stream = nullptr;
            j->ctx = nullptr;
            j->state = DILBM_JOB_FAILED;
            j->error = rc;
            j->finished = s->now();
            ++s->n_failed;
            continue;
        }
        j->state = DILBM_JOB_RUNNING;
        j->admitted = s->now();
        s->in_use += j->footprint;
        s->running.push_back(j);
        s->dirty = true;
        ++added;
    }
    return added;
}

void fill_stats(const dilbm_server *s, dilbm_server_stats *st) {
    st->running = (int)s->running.size();
    st->queued = (int)s->queue.size();
    st->done = s->n_done;
    st->failed = s->n_failed;
    st->macro_steps = s->macro;
    st->node_updates = s->node_updates;
    st->busy_seconds = s->busy;
    st->form_seconds = s->t_form;
    st->admit_seconds = s->t_admit;
    st->wait_seconds = s->t_wait;
    st->retire_seconds = s->t_retire;
    st->memory_in_use = s->in_use;
    long long l = s->launches_gone;
    for (int c = 0; c < NSTORE; ++c) l += s->batch[c] ? dilbm_batch_launch_count(s->batch[c]) : 0;
    for (const Job *j : s->running) l += j->ctx ? dilbm_launch_count(j->ctx) : 0;
    st->launches = l;
}

}  // namespace

extern "C" {

int dilbm_server_create(const dilbm_server_config *cfg, void *cuda_stream, dilbm_server **out) {
    (void)cuda_stream;       // every job runs on a stream of its own
    if (!cfg || !out) return sfail(DILBM_ERR_INVALID_ARG, "config and out must not be NULL");
    *out = nullptr;
    if (cfg->storage != DILBM_STORAGE_PER_JOB && cfg->storage != DILBM_STORAGE_AUTO &&
        (cfg->storage < DILBM_FP32 || cfg->storage > DILBM_BF16_DEV))
        return sfail(DILBM_ERR_INVALID_ARG, "unknown storage");
    if (cfg->max_jobs < 1 || cfg->max_jobs > MAX_JOBS)
        return sfail(DILBM_ERR_INVALID_ARG, "max_jobs must be 1.." + std::to_string(MAX_JOBS));
    if (cfg->macro_steps < 1) return sfail(DILBM_ERR_INVALID_ARG, "macro_steps must be >= 1");
    if (cfg->policy != DILBM_ADMIT_FIFO && cfg->policy != DILBM_ADMIT_FIRST_FIT)
        return sfail(DILBM_ERR_INVALID_ARG, "unknown admission policy");
    unsigned long long budget = 0;
    if (cfg->memory_budget > 0.0) {
        budget = (unsigned long long)cfg->memory_budget;
    } else {
        size_t free_b = 0, total_b = 0;
        cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
        if (e != cudaSuccess) return scuda(e, "cudaMemGetInfo");
        budget = (unsigned long long)(0.9 * (double)free_b);
    }
    dilbm_server *s = new dilbm_server();
    s->cfg = *cfg;
    if (!(s->cfg.auto_tau_max > 0.0)) s->cfg.auto_tau_max = 0.6;
    if (!(s->cfg.auto_area_max > 0.0)) s->cfg.auto_area_max = 0.05;
    s->budget = budget;
    s->t0 = std::chrono::steady_clock::now();
    *out = s;
    return DILBM_OK;
}

int dilbm_server_submit(dilbm_server *s, const dilbm_job *job, long long *id) {
    if (!s || !job || !id) return sfail(DILBM_ERR_INVALID_ARG, "NULL argument");
    if (job->nsteps < 1) return sfail(DILBM_ERR_INVALID_ARG, "a job needs nsteps >= 1");
    if (job->mean_window < 0 || job->mean_window > job->nsteps)
        return sfail(DILBM_ERR_INVALID_ARG, "mean_window must be 0..nsteps");
    dilbm_grid g = job->grid;
    if (s->cfg.storage == DILBM_STORAGE_AUTO) {
        double area = 0.0;
        for (int k = 0; k < job->np && job->particles; ++k)
            area += 3.14159265358979323846 * job->particles[k].r * job->particles[k].r;
        const double frac = area / ((double)g.nx * (double)g.ny);
        g.storage = (job->tau > s->cfg.auto_tau_max || frac > s->cfg.auto_area_max) ? DILBM_FP32 : DILBM_FP16_DEV;
    } else if (s->cfg.storage != DILBM_STORAGE_PER_JOB) {
        g.storage = s->cfg.storage;
    }
    int rc = dilbm::check_problem(&g, DILBM_D2Q9, job->tau, job->interface_width, job->particles, job->np);
    if (rc) return rc;
    if (g.method != DILBM_METHOD_DI) return sfail(DILBM_ERR_INVALID_ARG, "the server runs DI-LBM jobs only");
    unsigned long long fp = 0;
    if ((rc = dilbm_footprint(&g, job->np, &fp))) return rc;
    if (fp > s->budget)
        return sfail(DILBM_ERR_INVALID_ARG, "job needs " + std::to_string(fp) + " bytes, more than the server's budget of " +
                                                std::to_string(s->budget));
    auto j = std::make_unique<Job>();
    j->id = s->next_id++;
    j->grid = g;
    j->tau = job->tau;
    j->eps = job->interface_width;
    j->parts.assign(job->particles, job->particles + job->np);
    j->nsteps = job->nsteps;
    j->window = job->mean_window;
    j->footprint = fp;
    j->nodes = (double)g.nx * (double)g.ny;
    j->arrival = job->arrival >= 0.0 ? job->arrival : s->now();
    s->queue.push_back(j.get());
    *id = j->id;
    s->jobs.emplace(j->id, std::move(j));
    return DILBM_OK;
}

int dilbm_server_progress(dilbm_server *s, dilbm_server_stats *stats) {
    const dilbm::TraceRange trace("dilbm_server_progress");
    if (!s) return sfail(DILBM_ERR_INVALID_ARG, "NULL server");
    const double t_in = s->now();
    int rc = DILBM_OK;
    if (s->running.empty()) {
        if ((rc = admit(s)) < 0) return rc;
        s->t_admit += s->now() - t_in;
    }
    if (!s->running.empty()) {
        double t = s->now();
        if (s->dirty || !has_batch(s)) {
            drop_batch(s);
            for (int c = 0; c < NSTORE; ++c) s->members[c].clear();
            for (Job *j : s->running) s->members[j->grid.storage].push_back(j);
            for (int c = 0; c < NSTORE; ++c) {
                if (s->members[c].empty()) continue;
                std::vector<dilbm_ctx *> m(s->members[c].size());
                for (size_t q = 0; q < m.size(); ++q) m[q] = s->members[c][q]->ctx;
                if ((rc = dilbm_batch_create(m.data(), (int)m.size(), nullptr, &s->batch[c]))) return rc;
            }
            s->dirty = false;
        }
        // the macro-step ends where the first job finishes or opens its
        // mean-force window
        long long k = s->cfg.macro_steps;
        for (int c = 0; c < NSTORE; ++c)
            for (Job *j : s->members[c]) {
                const long long left = j->nsteps - j->done;
                k = std::min(k, left > j->window ? left - j->window : left);
            }
        for (int c = 0; c < NSTORE; ++c)
            if (s->batch[c] && (rc = dilbm_batch_step(s->batch[c], k))) return rc;
        double t2 = s->now();
        s->t_form += t2 - t;
        // newcomers are set up on their own streams while the GPU steps
        if ((rc = admit(s)) < 0) return rc;
        t = s->now();
        s->t_admit += t - t2;
        std::vector<Job *> members;
        std::vector<int> codes;
        for (int c = 0; c < NSTORE; ++c) {
            if (!s->batch[c]) continue;
            std::vector<int> cc(s->members[c].size(), DILBM_OK);
            if ((rc = dilbm_batch_errors(s->batch[c], cc.data()))) return rc;
            members.insert(members.end(), s->members[c].begin(), s->members[c].end());
            codes.insert(codes.end(), cc.begin(), cc.end());
        }
        t2 = s->now();
        s->t_wait += t2 - t;
        ++s->macro;
        bool left = false;
        for (size_t q = 0; q < members.size(); ++q) {
            Job *j = members[q];
            if (codes[q] != DILBM_OK) {
                j->state = DILBM_JOB_FAILED;
                j->error = codes[q];
            } else {
                j->done += k;
                s->node_updates += j->nodes * (double)k;
                if (j->done < j->nsteps) {
                    if (j->window > 0 && j->nsteps - j->done == j->window &&
                        (rc = dilbm_force_mean_reset(j->ctx)))
                        return rc;
                    continue;
                }
                const size_t np = j->parts.size();
                const size_t n3 = 3 * (np > 0 ? np : 1);
                j->force.assign(n3, 0.0);
                j->force_mean.assign(n3, 0.0);
                j->final_state.assign(np > 0 ? np : 1, dilbm_particle{});
                int frc = dilbm_forces(j->ctx, j->force.data(), nullptr, j->final_state.data());
                long long nmean = 0;
                if (frc == DILBM_OK && j->window > 0) frc = dilbm_force_mean(j->ctx, j->force_mean.data(), &nmean);
                if (frc == DILBM_OK && j->window > 0 && nmean != j->window)
                    frc = sfail(DILBM_ERR_CUDA, "mean-force window of job " + std::to_string(j->id) + " covers " +
                                                    std::to_string(nmean) + " steps");
                j->state = frc == DILBM_OK ? DILBM_JOB_DONE : DILBM_JOB_FAILED;
                j->error = frc;
            }
            j->finished = s->now();
            if (j->state == DILBM_JOB_DONE) ++s->n_done;
            else ++s->n_failed;
            left = true;
        }
        if (left) {
            // contexts are freed before the next macro-step is launched
            // (cudaFree waits for the device)
            drop_batch(s);
            std::vector<Job *> still;
            still.reserve(s->running.size());
            for (Job *j : s->running) {
                if (j->state == DILBM_JOB_RUNNING) still.push_back(j);
                else release(s, j);
            }
            s->running.swap(still);
            for (int c = 0; c < NSTORE; ++c) s->members[c].clear();
            s->dirty = true;
        }
        s->t_retire += s->now() - t2;
    }
    s->busy += s->now() - t_in;
    if (stats) fill_stats(s, stats);
    return DILBM_OK;
}

int dilbm_server_status(const dilbm_server *s, long long id, dilbm_job_status *st) {
    if (!s || !st) return sfail(DILBM_ERR_INVALID_ARG, "NULL argument");
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) return sfail(DILBM_ERR_INVALID_ARG, "unknown job id " + std::to_string(id));
    const Job &j = *it->second;
    st->state = j.state;
    st->error = j.error;
    st->np = (int)j.parts.size();
    st->steps_done = j.done;
    st->arrival = j.arrival;
    st->admitted = j.admitted;
    st->finished = j.finished;
    st->footprint = j.footprint;
    st->storage = j.grid.storage;
    return DILBM_OK;
}

int dilbm_server_result(dilbm_server *s, long long id, double *force, double *force_mean, dilbm_particle *state) {
    if (!s) return sfail(DILBM_ERR_INVALID_ARG, "NULL server");
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) return sfail(DILBM_ERR_INVALID_ARG, "unknown job id " + std::to_string(id));
    Job &j = *it->second;
    if (j.state != DILBM_JOB_DONE) return sfail(DILBM_ERR_INVALID_ARG, "job " + std::to_string(id) + " is not done");
    const size_t np = j.parts.size();
    if (np > 0 && !force) return sfail(DILBM_ERR_INVALID_ARG, "force must not be NULL");
    if (np > 0) std::copy(j.force.begin(), j.force.begin() + 3 * np, force);
    if (force_mean && np > 0) std::copy(j.force_mean.begin(), j.force_mean.begin() + 3 * np, force_mean);
    if (state && np > 0) std::copy(j.final_state.begin(), j.final_state.begin() + np, state);
    s->jobs.erase(it);
    return DILBM_OK;
}

double dilbm_server_clock(const dilbm_server *s) { return s ? s->now() : -1.0; }

void dilbm_server_destroy(dilbm_server *s) {
    if (!s) return;
    drop_batch(s);
    for (auto &kv : s->jobs) release(s, kv.second.get());
    delete s;
}

}  // extern "C"
