// batch.cu -- poisson_batch_submit / poisson_poll.
#include <mutex>
#include <unordered_map>
#include <vector>

#include "poisson.h"
#include "capi_internal.h"

namespace {
struct Job {
    poisson_t* h;
    const double* rhs;
    double* p;
    double tol;
    int status;
    bool finished;
    poisson_stats stats;
};
std::mutex g_mu;
std::unordered_map<uint64_t, Job> g_jobs;
std::vector<uint64_t> g_queue;
uint64_t g_next = 1;
}  // namespace

extern "C" int poisson_batch_submit(poisson_t* const* handles, const double* const* rhs,
                                    double* const* p, const double* tol, int n,
                                    uint64_t* tickets) {
    if (!handles || !rhs || !p || !tol || !tickets || n <= 0) return POISSON_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (!handles[i] || !rhs[i] || !p[i] || !(tol[i] > 0.0)) return POISSON_EINVAL;
        if (!handles[i]->ready) return POISSON_ENOTREADY;
        for (int j = 0; j < i; ++j)
            if (handles[j] == handles[i]) return POISSON_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    for (int i = 0; i < n; ++i) {
        const uint64_t t = g_next++;
        g_jobs[t] = Job{handles[i], rhs[i], p[i], tol[i], POISSON_PENDING, false, {}};
        g_queue.push_back(t);
        tickets[i] = t;
    }
    return POISSON_OK;
}

extern "C" int poisson_poll(uint64_t ticket, poisson_stats* stats) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_jobs.find(ticket);
    if (it == g_jobs.end()) return POISSON_ENOTICKET;
    if (!it->second.finished) {
        // run queued solves in submission order up to and including this ticket
        while (!g_queue.empty()) {
            const uint64_t t = g_queue.front();
            g_queue.erase(g_queue.begin());
            Job& j = g_jobs[t];
            j.status = poisson_solve(j.h, j.rhs, j.p, j.tol, &j.stats);
            j.finished = true;
            if (t == ticket) break;
        }
    }
    Job j = it->second;
    if (!j.finished) return POISSON_PENDING;
    if (stats) *stats = j.stats;
    g_jobs.erase(it);
    return j.status;
}
