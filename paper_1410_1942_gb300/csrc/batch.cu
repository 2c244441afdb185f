// batch.cu -- poisson_batch_submit / poisson_poll: many independent solves of uneven size
// driven together, FP64 refinement step by refinement step.
//
// Each outer (refinement) step of the batch is two CUDA graphs on the executor's stream:
//   R: x64 += d for every job (k_batch_update), r32 = b - A64 x64 and its norms
//      (k_batch_residual), scalars copied to the host;
//   S: the inner-solve controls copied to the device, z = D^-1 r for every job
//      (k_batch_init), ONE cooperative persistent PCG launch over all unfinished jobs
//      (k_pcg on the batch's work list), scalars copied back.
// Between them the host decides, per job, whether it has converged (then its solution is copied
// out and its ticket finishes) and sets the next inner tolerance.  Jobs submitted while a batch
// runs join it at the next outer step (continuous batching): the job table, the work list and
// the graphs are rebuilt then.  Finished jobs stay in the table, inactive, until the next
// rebuild.  Jobs that cannot run in the batch's persistent kernel are solved with poisson_solve:
// those whose solves launch only ordinary kernels (multigrid, FP64, column kernels) on worker
// threads, several at once, each on its handle's own stream, so that small solves overlap on
// the GPU; those that run a persistent cooperative launch of their own (periodic one-sweep,
// red-black) one by one when polled -- two grid-filling cooperative launches in flight at once
// could keep each other's CTAs from becoming resident, and their grid barriers would end by
// deadline.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "alloc.h"
#include "poisson.h"
#include "capi_internal.h"
#include "jobs.cuh"
#include "kernels.h"
#include "march.h"
#include "xfer.h"

using namespace pcg;

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Job {
    poisson_t* h = nullptr;
    const double* rhs = nullptr;
    double* p = nullptr;
    double tol = 0.0;
    uint64_t ticket = 0;
    bool batched = false;   // runs in the persistent batch (else poisson_solve)
    bool pooled = false;    // poisson_solve on a worker thread (else one by one at poll)
    cudaEvent_t ready = nullptr;  // pooled: the caller's work on the handle's stream at submit
    bool admitted = false;  // data staged on the device
    bool finished = false;
    int status = POISSON_PENDING;
    poisson_stats stats{};
    int outer = 0, inner = 0, stalls = 0;
    double prev = INFINITY, rel = INFINITY, t0 = 0.0;
};

constexpr int MAX_OUTER = 60;

struct Executor {
    bool bf16 = false;
    cudaStream_t st = nullptr;
    std::vector<Job*> table;  // jobs of the current job table (finished ones inactive)
    std::deque<Job*> waiting;
    // device state of the job table
    JobDev* d_jobs = nullptr;
    JobDev* h_jobs = nullptr;  // pinned
    Scalars* d_sc = nullptr;
    Scalars* h_sc = nullptr;  // pinned
    double* d_part = nullptr;
    MarchCtl* h_ctl = nullptr;  // pinned
    int cap = 0;                // jobs the buffers hold
    size_t part_cap = 0;
    int blocks = 0;
    MarchPlan plan{};
    cudaGraphExec_t gR = nullptr, gS = nullptr;
    bool dirty = true;
    // development trace (POISSON_TRACE): rebuilds and refinement steps, with their host time
    bool trace = getenv("POISSON_TRACE") != nullptr;
    long long n_rebuild = 0, n_step = 0;
    double t_rebuild = 0.0, t_step = 0.0;

    void report() const {
        if (trace && (n_rebuild || n_step))
            fprintf(stderr,
                    "[poisson batch] %lld rebuilds (%.2f ms each), %lld refinement steps "
                    "(%.2f ms each), graphs %s\n",
                    n_rebuild, n_rebuild ? 1e3 * t_rebuild / n_rebuild : 0.0, n_step,
                    n_step ? 1e3 * t_step / n_step : 0.0, gR ? "on" : "off");
    }

    ~Executor() {
        report();
        release();
    }

    void release_graphs() {
        if (gR) cudaGraphExecDestroy(gR);
        if (gS) cudaGraphExecDestroy(gS);
        gR = gS = nullptr;
    }
    void release() {
        release_graphs();
        march_plan_free(&plan);
        if (d_jobs) lib_free(d_jobs);
        if (d_sc) lib_free(d_sc);
        if (d_part) lib_free(d_part);
        if (h_jobs) lib_free_host(h_jobs);
        if (h_sc) lib_free_host(h_sc);
        if (h_ctl) lib_free_host(h_ctl);
        d_jobs = nullptr;
        d_sc = nullptr;
        d_part = nullptr;
        h_jobs = nullptr;
        h_sc = nullptr;
        h_ctl = nullptr;
        cap = 0;
        part_cap = 0;
    }

    bool has_work() const {
        if (!waiting.empty()) return true;
        for (Job* j : table)
            if (!j->finished) return true;
        return false;
    }

    int ensure_stream() {
        if (st) return POISSON_OK;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return POISSON_ECUDA;
        }
        return POISSON_OK;
    }

    // Stages a job's right side and start on the executor stream (b64 = -h^2 rhs, x64 = p).
    int stage(Job* j) {
        poisson_t* H = j->h;
        const size_t n = (size_t)H->d.n, bytes = n * sizeof(double);
        const bool drhs = is_device_ptr(j->rhs), dp = is_device_ptr(j->p);
        if (drhs) {
            launch_scale((long long)n, j->rhs, -(H->h * H->h), H->b64, st);
        } else {
            if (copy_user(H->b64, j->rhs, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
                return POISSON_ECUDA;
            launch_scale((long long)n, H->b64, -(H->h * H->h), H->b64, st);
        }
        if (copy_user(H->x64, j->p, bytes, dp ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            st) != cudaSuccess)
            return POISSON_ECUDA;
        if (cudaMemsetAsync(H->d32, 0, n * sizeof(float), st) != cudaSuccess ||
            cudaMemsetAsync(H->p32a, 0, n * sizeof(float), st) != cudaSuccess)
            return POISSON_ECUDA;
        j->admitted = true;
        j->t0 = now_s();
        return POISSON_OK;
    }

    int finish(Job* j, int status) {
        poisson_t* H = j->h;
        const size_t bytes = sizeof(double) * (size_t)H->d.n;
        const bool dp = is_device_ptr(j->p);
        if (copy_user(j->p, H->x64, bytes, dp ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            cudaGetLastError();
            status = POISSON_ECUDA;
        }
        j->finished = true;
        j->status = status;
        j->stats.outer_iters = j->outer;
        j->stats.inner_iters = j->inner;
        j->stats.rel_residual = j->rel;
        j->stats.seconds = now_s() - j->t0;
        return POISSON_OK;
    }

    // Rebuilds the job table (unfinished jobs plus admitted newcomers), the work list and the
    // graphs.
    int rebuild() {
        release_graphs();
        std::vector<Job*> keep;
        for (Job* j : table)
            if (!j->finished) keep.push_back(j);
        while (!waiting.empty()) {
            Job* j = waiting.front();
            waiting.pop_front();
            int rc = stage(j);
            if (rc) {
                j->finished = true;
                j->status = rc;
                continue;
            }
            keep.push_back(j);
        }
        table = keep;
        dirty = false;
        if (table.empty()) return POISSON_OK;
        const int nj = (int)table.size();
        // buffers
        size_t part = 0;
        std::vector<JobDev> jd(nj);
        int off = 0;
        for (int q = 0; q < nj; ++q) {
            poisson_t* H = table[q]->h;
            JobDev& J = jd[q];
            J = JobDev{};
            J.d = H->d;
            J.kc = H->kc;
            J.gx = (H->d.nx + TX - 1) / TX;
            J.gy = (H->d.ny + TY - 1) / TY;
            const int gz = (H->d.nz + H->kc - 1) / H->kc;
            J.blocks = J.gx * J.gy * gz;
            J.blk_off = off;
            off += J.blocks;
            J.bf16 = bf16 ? 1 : 0;
            J.bx = H->bx; J.by = H->by; J.bz = H->bz; J.diag = H->diag;
            J.b64 = H->b64; J.x64 = H->x64;
            J.d32 = H->d32; J.r32 = H->r32; J.z32 = H->z32; J.pa32 = H->p32a;
            J.sa32 = H->s32a; J.wa32 = H->w32a;
            J.eta32 = H->eta32; J.eta16 = H->eta16;
            part += 2 * (size_t)J.blocks;
            J.tol2 = 0.25;
            J.max_iter = 1;
            J.active = 1;
        }
        blocks = off;
        if (nj > cap || part > part_cap) {
            const int ncap = std::max(nj, 2 * cap);
            const size_t npart = std::max(part, 2 * part_cap);
            if (d_jobs) lib_free(d_jobs);
            if (d_sc) lib_free(d_sc);
            if (d_part) lib_free(d_part);
            if (h_jobs) lib_free_host(h_jobs);
            if (h_sc) lib_free_host(h_sc);
            d_jobs = nullptr; d_sc = nullptr; d_part = nullptr; h_jobs = nullptr; h_sc = nullptr;
            if (lib_malloc((void**)&d_jobs, sizeof(JobDev) * ncap) != cudaSuccess ||
                lib_malloc((void**)&d_sc, sizeof(Scalars) * ncap) != cudaSuccess ||
                lib_malloc((void**)&d_part, sizeof(double) * npart) != cudaSuccess ||
                lib_malloc_host((void**)&h_jobs, sizeof(JobDev) * ncap) != cudaSuccess ||
                lib_malloc_host((void**)&h_sc, sizeof(Scalars) * ncap) != cudaSuccess) {
                cudaGetLastError();
                return POISSON_ENOMEM;
            }
            cap = ncap;
            part_cap = npart;
        }
        if (!h_ctl && lib_malloc_host((void**)&h_ctl, sizeof(MarchCtl)) != cudaSuccess) {
            cudaGetLastError();
            h_ctl = nullptr;
            return POISSON_ENOMEM;
        }
        size_t poff = 0;
        for (int q = 0; q < nj; ++q) {
            jd[q].sc = d_sc + q;
            jd[q].partials = d_part + poff;
            poff += 2 * (size_t)jd[q].blocks;
            h_jobs[q] = jd[q];
        }
        if (cudaMemsetAsync(d_sc, 0, sizeof(Scalars) * nj, st) != cudaSuccess ||
            cudaMemcpyAsync(d_jobs, h_jobs, sizeof(JobDev) * nj, cudaMemcpyHostToDevice, st) !=
                cudaSuccess)
            return POISSON_ECUDA;
        // work list: every job of the table; variant: the one tuned for the largest job
        std::vector<MarchSolve> ms(nj);
        int big = 0;
        for (int q = 0; q < nj; ++q) {
            poisson_t* H = table[q]->h;
            ms[q] = MarchSolve{H->d, H->d32, H->r32, H->z32, H->p32a, H->p32b,
                               bf16 ? (const void*)H->eta16 : (const void*)H->eta32, d_sc + q,
                               H->s32a, H->s32b, H->w32a, H->w32b};
            if (H->d.n > table[big]->h->d.n) big = q;
        }
        const poisson_t* HB = table[big]->h;
        const int var = HB->march ? HB->plan.variant : 0;
        const int strat = HB->march ? HB->plan.strategy : MARCH_SPLIT_EQUAL;
        int nsm = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const int nctas = std::max(1, march_occupancy(var, bf16)) * std::max(1, nsm);
        int rc = march_plan_build(&plan, ms.data(), nj, var, bf16, nctas, strat, st);
        // a lockstep deal can spread one CTA over too many solves: fall back to the equal split
        if (rc == -1 && strat != MARCH_SPLIT_EQUAL)
            rc = march_plan_build(&plan, ms.data(), nj, var, bf16, nctas, MARCH_SPLIT_EQUAL, st);
        if (rc == -2) return POISSON_ENOMEM;
        if (rc != 0) return POISSON_EINVAL;
        return capture();
    }

    // Graph R (update, residual, scalars to host) and graph S (controls, init, persistent PCG,
    // scalars to host).  Without graphs the same sequence is launched directly.
    void seq_R() {
        launch_batch_update(d_jobs, (int)table.size(), blocks, st);
        launch_batch_residual(d_jobs, (int)table.size(), blocks, st);
        cudaMemcpyAsync(h_sc, d_sc, sizeof(Scalars) * table.size(), cudaMemcpyDeviceToHost, st);
    }
    int seq_S() {
        cudaMemcpyAsync(d_jobs, h_jobs, sizeof(JobDev) * table.size(), cudaMemcpyHostToDevice, st);
        launch_batch_init(d_jobs, (int)table.size(), blocks, st);
        cudaMemcpyAsync(plan.ctl, h_ctl, sizeof(MarchCtl), cudaMemcpyHostToDevice, st);
        const int rc = launch_march_pcg(plan, st);
        cudaMemcpyAsync(h_sc, d_sc, sizeof(Scalars) * table.size(), cudaMemcpyDeviceToHost, st);
        return rc;
    }
    int capture() {
        cudaGraph_t g = nullptr;
        bool ok = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            seq_R();
            ok = cudaStreamEndCapture(st, &g) == cudaSuccess && g;
            ok = ok && cudaGraphInstantiate(&gR, g, 0) == cudaSuccess;
            if (g) cudaGraphDestroy(g);
        }
        g = nullptr;
        if (ok) {
            ok = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                const int rc = seq_S();
                ok = cudaStreamEndCapture(st, &g) == cudaSuccess && g && rc == 0;
                ok = ok && cudaGraphInstantiate(&gS, g, 0) == cudaSuccess;
                if (g) cudaGraphDestroy(g);
            }
        }
        if (!ok) {  // run the sequences directly
            cudaGetLastError();
            release_graphs();
        }
        return POISSON_OK;
    }

    // One outer step of the whole batch.
    int step() {
        int rc = ensure_stream();
        if (rc) return rc;
        const double ts = now_s();
        if (dirty || !waiting.empty()) {
            rc = rebuild();
            ++n_rebuild;
            t_rebuild += now_s() - ts;
            if (trace && (n_rebuild % 64) == 1) report();
            if (rc) {
                for (Job* j : table)
                    if (!j->finished) { j->finished = true; j->status = rc; }
                table.clear();
                return rc;
            }
        }
        if (table.empty()) return POISSON_OK;
        const int nj = (int)table.size();
        if (gR) {
            if (cudaGraphLaunch(gR, st) != cudaSuccess) return POISSON_ECUDA;
        } else {
            seq_R();
        }
        if (cudaStreamSynchronize(st) != cudaSuccess) return POISSON_ECUDA;
        int running = 0;
        for (int q = 0; q < nj; ++q) {
            Job* j = table[q];
            JobDev& J = h_jobs[q];
            if (j->finished) {
                J.active = 0;
                continue;
            }
            const Scalars& s = h_sc[q];
            j->outer += 1;
            if (s.bb == 0.0) {
                cudaMemsetAsync(j->h->x64, 0, sizeof(double) * (size_t)j->h->d.n, st);
                j->rel = 0.0;
                finish(j, POISSON_OK);
                J.active = 0;
                continue;
            }
            const double rel = std::sqrt(s.rr / s.bb);
            j->rel = rel;
            int status = POISSON_PENDING;
            if (!std::isfinite(rel)) status = POISSON_EBREAKDOWN;
            else if (rel <= j->tol) status = POISSON_OK;
            else {
                if (rel > 0.5 * j->prev) ++j->stalls; else j->stalls = 0;
                if (j->inner >= j->h->opts.max_iters || j->stalls >= 3 || j->outer > MAX_OUTER)
                    status = POISSON_ENOTCONV;
            }
            if (status != POISSON_PENDING) {
                finish(j, status);
                J.active = 0;
                continue;
            }
            j->prev = rel;
            double target = std::max(j->h->opts.inner_tol, 0.3 * j->tol / rel);
            target = std::min(target, 0.5);
            J.tol2 = target * target;
            J.max_iter = std::max(1, j->h->opts.max_iters - j->inner);
            J.active = 1;
            ++running;
        }
        if (running == 0) {
            dirty = true;  // drop the finished jobs at the next rebuild
            ++n_step;
            t_step += now_s() - ts;
            if (waiting.empty()) report();  // the batch has drained
            return POISSON_OK;
        }
        *h_ctl = MarchCtl{0u, nj, 0, 0, 0ull};
        if (gS) {
            if (cudaGraphLaunch(gS, st) != cudaSuccess) return POISSON_ECUDA;
        } else if (seq_S() != 0) {
            return POISSON_ECUDA;
        }
        if (cudaStreamSynchronize(st) != cudaSuccess) return POISSON_ECUDA;
        for (int q = 0; q < nj; ++q) {
            Job* j = table[q];
            if (j->finished || !h_jobs[q].active) continue;
            const Scalars& s = h_sc[q];
            j->inner += s.iter;
            if (s.done == TIMEDOUT) {
                j->rel = INFINITY;
                finish(j, POISSON_ETIMEOUT);
            } else if (s.done == BREAKDOWN && s.iter == 0) {
                finish(j, POISSON_EBREAKDOWN);
            }
        }
        ++n_step;
        t_step += now_s() - ts;
        return POISSON_OK;
    }
};

std::mutex g_mu;
std::unordered_map<uint64_t, Job*> g_jobs;
std::deque<Job*> g_serial;  // jobs solved one by one at poll
Executor* g_exec[2] = {nullptr, nullptr};  // FP32 and BF16 coefficients
uint64_t g_next = 1;

bool batchable(const poisson_t* H) {
    // (periodic handles run their own padded one-sweep plans: solved one by one)
    return H->opts.precision != POISSON_FP64 && H->opts.precond == POISSON_JACOBI &&
           march_supported(H->d) && H->march && !H->periodic();
}

// A handle whose solve launches no persistent cooperative kernel (see the header comment).
bool poolable(const poisson_t* H) { return !H->march && !H->rb; }

// Worker threads for the pooled jobs, started with the first one.  Each takes a job, makes the
// handle's device current and runs poisson_solve on a non-blocking stream of its own (ordered
// after the caller's work on the handle's stream by an event recorded at submit; the handle's
// stream is restored afterwards), then publishes the result under g_mu.  Own streams let the
// jobs overlap on the GPU even when their handles run on the legacy default stream, and let the
// CG loop replay its chunk graph (a legacy stream cannot be captured).
constexpr int N_WORKERS = 8;

struct Pool {
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Job*> queue;
    std::vector<std::thread> threads;
    bool stop = false;

    void push(Job* j);
    ~Pool() {
        {
            std::lock_guard<std::mutex> lk(mu);
            stop = true;
        }
        cv.notify_all();
        for (auto& t : threads)
            if (t.joinable()) t.join();
    }
};
Pool g_pool;

void worker() {
    std::unordered_map<int, cudaStream_t> own;  // the worker's stream on each device
    for (;;) {
        Job* j = nullptr;
        {
            std::unique_lock<std::mutex> lk(g_pool.mu);
            g_pool.cv.wait(lk, [] { return g_pool.stop || !g_pool.queue.empty(); });
            if (g_pool.queue.empty()) {  // stopping
                for (auto& kv : own)
                    if (kv.second) {
                        cudaSetDevice(kv.first);
                        cudaStreamDestroy(kv.second);
                    }
                return;
            }
            j = g_pool.queue.front();
            g_pool.queue.pop_front();
        }
        const int dev = j->h->device;
        cudaSetDevice(dev);
        cudaStream_t& w = own[dev];
        if (!w && cudaStreamCreateWithFlags(&w, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            w = nullptr;
        }
        poisson_stats st{};
        int rc;
        if (w) {
            cudaStreamWaitEvent(w, j->ready, 0);
            const cudaStream_t hs = j->h->st;
            j->h->st = w;
            rc = poisson_solve(j->h, j->rhs, j->p, j->tol, &st);
            j->h->st = hs;
        } else {
            cudaEventSynchronize(j->ready);
            rc = poisson_solve(j->h, j->rhs, j->p, j->tol, &st);
        }
        cudaEventDestroy(j->ready);
        std::lock_guard<std::mutex> lk(g_mu);  // poll reads the job under g_mu
        j->stats = st;
        j->status = rc;
        j->finished = true;
    }
}

void Pool::push(Job* j) {
    {
        std::lock_guard<std::mutex> lk(mu);
        queue.push_back(j);
        if (threads.empty())
            for (int i = 0; i < N_WORKERS; ++i) threads.emplace_back(worker);
    }
    cv.notify_one();
}

}  // namespace

bool batch_handle_busy(const poisson_t* H) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& kv : g_jobs)
        if (kv.second->h == H) return true;
    return false;
}

extern "C" int poisson_batch_submit(poisson_t* const* handles, const double* const* rhs,
                                    double* const* p, const double* tol, int n,
                                    uint64_t* tickets) {
    if (!handles || !rhs || !p || !tol || !tickets || n <= 0) return POISSON_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    for (int i = 0; i < n; ++i) {
        if (!handles[i] || !rhs[i] || !p[i] || !(tol[i] > 0.0)) return POISSON_EINVAL;
        if (!handles[i]->ready) return POISSON_ENOTREADY;
        for (int j = 0; j < i; ++j)
            if (handles[j] == handles[i]) return POISSON_EINVAL;
        for (auto& kv : g_jobs)  // a handle may be in one unreported job at a time
            if (kv.second->h == handles[i] && !kv.second->finished) return POISSON_EINVAL;
    }
    for (int i = 0; i < n; ++i) {
        Job* j = new Job();
        j->h = handles[i];
        j->rhs = rhs[i];
        j->p = p[i];
        j->tol = tol[i];
        j->ticket = g_next++;
        j->batched = batchable(handles[i]);
        j->pooled = !j->batched && poolable(handles[i]);
        g_jobs[j->ticket] = j;
        if (j->batched) {
            const int e = handles[i]->opts.precision == POISSON_FP32_BF16COEF ? 1 : 0;
            if (!g_exec[e]) {
                g_exec[e] = new Executor();
                g_exec[e]->bf16 = (e == 1);
            }
            g_exec[e]->waiting.push_back(j);
        } else if (j->pooled) {
            if (cudaEventCreateWithFlags(&j->ready, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventRecord(j->ready, handles[i]->st) != cudaSuccess) {
                cudaGetLastError();
                if (j->ready) cudaEventDestroy(j->ready);
                j->ready = nullptr;
                j->pooled = false;  // solved at poll on the handle's stream
                g_serial.push_back(j);
            } else {
                g_pool.push(j);
            }
        } else {
            g_serial.push_back(j);
        }
        tickets[i] = j->ticket;
    }
    return POISSON_OK;
}

extern "C" int poisson_poll(uint64_t ticket, poisson_stats* stats) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_jobs.find(ticket);
    if (it == g_jobs.end()) return POISSON_ENOTICKET;
    Job* j = it->second;
    if (!j->finished) {
        if (j->batched) {
            Executor* e = g_exec[j->h->opts.precision == POISSON_FP32_BF16COEF ? 1 : 0];
            const int rc = e->step();
            if (rc != POISSON_OK && !j->finished) {
                j->finished = true;
                j->status = rc;
            }
        } else if (j->pooled) {
            // a worker publishes the result
        } else {
            // solve the serial jobs in submission order up to this one
            while (!g_serial.empty()) {
                Job* s = g_serial.front();
                g_serial.pop_front();
                s->status = poisson_solve(s->h, s->rhs, s->p, s->tol, &s->stats);
                s->finished = true;
                if (s == j) break;
            }
        }
    }
    if (!j->finished) return POISSON_PENDING;
    if (stats) *stats = j->stats;
    const int status = j->status;
    g_jobs.erase(it);
    // the executor may still list the job in its table: it is finished, and is dropped at
    // the next rebuild before any further access
    for (Executor* e : g_exec)
        if (e)
            for (Job*& t : e->table)
                if (t == j) t = nullptr;
    delete j;
    for (Executor* e : g_exec)
        if (e) {
            auto& tb = e->table;
            const size_t before = tb.size();
            tb.erase(std::remove(tb.begin(), tb.end(), nullptr), tb.end());
            if (tb.size() != before) e->dirty = true;
        }
    return status;
}
