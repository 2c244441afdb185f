// capi.cu -- the C ABI of libpoisson (declared in include/poisson.h): handles, operator set-up,
// the single-solve drivers (plain FP64 PCG; FP32 inner PCG inside FP64 iterative refinement)
// and the operator / preconditioner entry points used to check the kernels one by one.
#include <algorithm>
#include <chrono>
#include <map>
#include <tuple>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "alloc.h"
#include "poisson.h"
#include "kernels.h"
#include "capi_internal.h"
#include "march.h"
#include "march_rb.h"
#include "xfer.h"

using namespace pcg;

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) {                                   \
            last_cuda_error() = e_;                                \
            return POISSON_ECUDA;                                  \
        }                                                          \
    } while (0)

// NVTX ranges around the phases of a solve (set-up, refinement steps, inner solves), for
// timeline tools; without a tool attached they cost a few instructions each.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

cudaError_t& last_cuda_error() {
    static thread_local cudaError_t e = cudaSuccess;
    return e;
}

static double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
static int dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) return POISSON_OK;
    if (lib_malloc((void**)p, sizeof(T) * count) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return POISSON_ENOMEM;
    }
    return POISSON_OK;
}

static void dfree(void* p) {
    if (p) lib_free(p);
}

extern "C" void poisson_default_opts(poisson_opts* o) {
    if (!o) return;
    o->precision = POISSON_FP32;
    o->precond = POISSON_JACOBI;
    o->omega = 1.0;
    o->max_iters = 20000;
    o->inner_tol = 1e-4;
    o->tile = 0;
    o->stream = nullptr;
    o->dirichlet_walls = 0;
    o->periodic_x = 0;
}

// z-chunk per thread: about 2048 blocks per launch, at least one plane and at most 64 per thread
// (on the 1024 x 512 x 256 wedge 64 planes beat whole 256-plane columns by 4 % in the MG solve).
static int choose_kc(const Dims& d) {
    const long long tiles = (long long)((d.nx + TX - 1) / TX) * ((d.ny + TY - 1) / TY);
    long long kc = (tiles * d.nz) / 2048;
    if (kc < 1) kc = 1;
    if (kc > 64) kc = 64;
    if (kc > d.nz) kc = d.nz;
    return (int)kc;
}

static void prof_add(poisson_t* H, int cls, cudaEvent_t a, cudaEvent_t b);

// ------------------------------------------------------------------ march kernel tuning
// Every variant is tried on the handle's own buffers (zeroed; the scalars reset before every
// launch) with a persistent grid of (resident CTAs per SM) x (SMs) CTAs, its phases A and B
// timed with events, and the fastest kept; the choice is cached per shape and coefficient type.
// Shapes are tuned per size class: each dimension rounded up to a power of two (at least 16).
struct TuneKey {
    int nx, ny, nz, bf16;
    bool operator<(const TuneKey& o) const {
        return std::tie(nx, ny, nz, bf16) < std::tie(o.nx, o.ny, o.nz, o.bf16);
    }
};
static int size_class(int v) {
    int c = 16;
    while (c < v) c <<= 1;
    return c;
}
static TuneKey tune_key(const Dims& d, bool bf16) {
    return TuneKey{size_class(d.nx), size_class(d.ny), size_class(d.nz), bf16 ? 1 : 0};
}
static std::mutex g_tune_mu;
static std::map<TuneKey, std::pair<int, int>> g_tuned;  // (variant, split strategy)

static int num_sms() {
    static const int n = [] {  // (initialised once, thread-safe)
        int dev = 0, m = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev);
        return m > 0 ? m : 1;
    }();
    return n;
}

static MarchSolve march_solve_of(poisson_t* H) {
    const bool bf16 = H->opts.precision == POISSON_FP32_BF16COEF;
    if (H->periodic())  // the one-sweep kernels on padded rows (u: pu, s^: ps, w^: pw)
        return MarchSolve{H->d, H->d32, H->r32, H->pu[0], H->p32a, H->pu[1],
                          bf16 ? (const void*)H->peta16 : (const void*)H->peta32, H->sc,
                          H->ps[0], H->ps[1], H->pw[0], H->pw[1]};
    return MarchSolve{H->d, H->d32, H->r32, H->z32, H->p32a, H->p32b,
                      bf16 ? (const void*)H->eta16 : (const void*)H->eta32, H->sc,
                      H->s32a, H->s32b, H->w32a, H->w32b};
}

static int build_plan(poisson_t* H, int var, int strategy) {
    const bool bf16 = H->opts.precision == POISSON_FP32_BF16COEF;
    const MarchSolve s = march_solve_of(H);
    const int nctas = march_occupancy(var, bf16) * num_sms();
    return march_plan_build(&H->plan, &s, 1, var, bf16, nctas, strategy, H->st);
}

// One FP32 inner PCG through the persistent kernel: init (z = D^{-1} r, scalars), p_in = 0,
// control words, cooperative launch, then wait.  r32 holds the right side, d32 the (zeroed)
// correction.  POISSON_ECUDA if the launch is refused.
static int march_run(poisson_t* H, bool bf16, double tol2, int max_iter, Scalars* result = nullptr) {
    cudaStream_t st = H->st;
    const Dims d = H->d;
    cudaMemsetAsync(H->d32, 0, sizeof(float) * (size_t)d.n, st);
    cudaMemsetAsync(H->p32a, 0, sizeof(float) * (size_t)d.n, st);
    if (march_variant(H->plan.variant).family == 1) {
        // the start-up sweep reads s^ and w^ (times alpha = beta = 0): they must be finite
        if (H->periodic()) {
            const size_t np = (size_t)(d.nx + 2 * PAD_V) * d.ny * d.nz;
            cudaMemsetAsync(H->ps[0], 0, sizeof(float) * np, st);
            cudaMemsetAsync(H->pw[0], 0, sizeof(float) * np, st);
        } else {
            cudaMemsetAsync(H->s32a, 0, sizeof(float) * (size_t)d.n, st);
            cudaMemsetAsync(H->w32a, 0, sizeof(float) * (size_t)d.n, st);
        }
    }
    if (bf16)
        launch_cg_init<float, CoefEta<__nv_bfloat16>>(d, H->kc, CoefEta<__nv_bfloat16>{H->eta16},
                                                      H->r32, H->z32, H->sc, H->partials, tol2, 0,
                                                      max_iter, st);
    else
        launch_cg_init<float, CoefEta<float>>(d, H->kc, CoefEta<float>{H->eta32}, H->r32, H->z32,
                                              H->sc, H->partials, tol2, 0, max_iter, st);
    if (H->periodic()) launch_pad_rows_f32(d, PAD_V, H->z32, H->pu[0], st);  // u = D^-1 r, padded
    *H->ctl_host = MarchCtl{0u, 1, 0, 0, 0ull};
    CK(cudaMemcpyAsync(H->plan.ctl, H->ctl_host, sizeof(MarchCtl), cudaMemcpyHostToDevice, st));
    const bool prof = H->prof_on && result;
    if (prof) CK(cudaEventRecord(H->prof_ev[PROF_PCG], st));
    if (launch_march_pcg(H->plan, st) != 0) return POISSON_ECUDA;
    if (prof) CK(cudaEventRecord(H->prof_ev[PROF_PCG + 1], st));
    CK(cudaStreamSynchronize(st));
    if (prof) prof_add(H, POISSON_K_PCG, H->prof_ev[PROF_PCG], H->prof_ev[PROF_PCG + 1]);
    if (result) CK(cudaMemcpy(result, H->sc, sizeof(Scalars), cudaMemcpyDeviceToHost));
    return POISSON_OK;
}

static int setup_march(poisson_t* H) {
    const bool bf16 = H->opts.precision == POISSON_FP32_BF16COEF;
    const Dims d = H->d;
    const int forced = H->opts.tile;
    int var = -1, strategy = MARCH_SPLIT_EQUAL;
    if (forced > 0) {
        var = march_variant_of_tile(forced);
        strategy = march_split_of_tile(forced);
        // periodic x runs on the one-sweep kernels only (others: the column kernels)
        if (H->periodic() && march_variant(var).family != 1) return POISSON_OK;
    } else {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(tune_key(d, bf16));
        if (it != g_tuned.end()) {
            var = it->second.first;
            strategy = it->second.second;
        }
    }
    if (var < 0 && forced <= 0) {
        // a constant-density model problem (rho = 1) with r = 1, TUNE_ITERS iterations per try
        constexpr int TUNE_ITERS = 16;
        const long long n = d.n;
        cudaStream_t st = H->st;
        if (bf16) launch_fill_bf16(n, H->eta16, 0.5f, st);
        else launch_fill_f32(n, H->eta32, 0.5f, st);
        if (H->periodic()) {  // the one-sweep kernels read rho/2 from padded rows
            if (H->peta32) launch_pad_rows_f32(d, 4, H->eta32, H->peta32, st);
            if (H->peta16) launch_pad_rows_bf16(d, 8, H->eta16, H->peta16, st);
        }
        launch_fill_f32(n, H->r32, 1.0f, st);
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best = 1e30f;
        // candidates: the 2 x 2-cells-per-thread variants of families 0 and 1 (64-wide tiles, 8
        // or 16 rows, with or without a producer warp, 3-, 4- or 6-stage rings); the 1 x 1
        // variant and family 2 (A p formed in the sweep, bound by its arithmetic) never won
        for (int cand = 0; cand < march_variant_count(); ++cand) {
            const MarchVariant mv = march_variant(cand);
            if (mv.cx != 2 || mv.family >= 2 || march_occupancy(cand, bf16) <= 0) continue;
            if (H->periodic() && mv.family != 1) continue;  // only the one-sweep kernels wrap
            for (int strat = 0; strat < MARCH_SPLITS; ++strat) {
                if (build_plan(H, cand, strat) != 0) continue;
                float t[2];
                bool good = true;
                for (int rep = 0; rep < 2 && good; ++rep) {
                    cudaEventRecord(e0, st);
                    good = march_run(H, bf16, 0.0, TUNE_ITERS) == POISSON_OK;
                    cudaEventRecord(e1, st);
                    cudaEventSynchronize(e1);
                    cudaEventElapsedTime(&t[rep], e0, e1);
                }
                if (!good || cudaGetLastError() != cudaSuccess) continue;
                const float tt = std::min(t[0], t[1]);
                if (tt < best) {
                    best = tt;
                    var = cand;
                    strategy = strat;
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaMemsetAsync(H->sc, 0, sizeof(Scalars), st);
        cudaStreamSynchronize(st);
        if (var >= 0) {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tuned[tune_key(d, bf16)] = {var, strategy};
        }
    }
    if (var < 0) return POISSON_OK;  // stay on the column kernels
    const int rc = build_plan(H, var, strategy);
    if (rc == -2) return POISSON_ENOMEM;
    H->march = (rc == 0);
    return POISSON_OK;
}

// ------------------------------------------------------------------ red-black SSOR marching
// The compressed black vectors of the red-black kernels, carved from the handle's FP32 inner
// vectors (each holds n floats, two black vectors of n/2; n is a multiple of 8, so both halves
// start on 16-byte boundaries as the tensor maps need).
struct RbBuffers {
    float *x, *p, *u0, *u1, *s0, *s1, *w0, *w1;
};
static RbBuffers rb_buffers(poisson_t* H) {
    const size_t nh = (size_t)H->d.n / 2;
    return RbBuffers{H->z32, H->z32 + nh, H->p32a, H->p32a + nh,
                     H->p32b, H->p32b + nh, H->s32a, H->s32a + nh};
}

static MarchSolve rb_solve_of(poisson_t* H) {
    const bool bf16 = H->opts.precision == POISSON_FP32_BF16COEF;
    const RbBuffers b = rb_buffers(H);
    return MarchSolve{H->d, b.x, H->r32, b.u0, b.p, b.u1,
                      bf16 ? (const void*)H->eta16 : (const void*)H->eta32, H->sc,
                      b.s0, b.s1, b.w0, b.w1};
}

// One FP32 inner solve A32 d = r32 by red-black SSOR PCG (omega = 1) as CG on the black Schur
// complement: start (red relaxation, reduced right side, scalars), the persistent launch, then
// d = (x_B, D_R^-1 (r_R + C x_B)) into d32.  POISSON_ECUDA if the launch is refused.
static int march_rb_run(poisson_t* H, bool bf16, double tol2, int max_iter,
                        Scalars* result = nullptr) {
    cudaStream_t st = H->st;
    const Dims d = H->d;
    const RbBuffers b = rb_buffers(H);
    if (bf16)
        launch_rb_init<__nv_bfloat16>(d, H->eta16, H->r32, b.u0, b.s0, b.w0, b.p, b.x, H->sc,
                                      H->partials, tol2, max_iter, st);
    else
        launch_rb_init<float>(d, H->eta32, H->r32, b.u0, b.s0, b.w0, b.p, b.x, H->sc, H->partials,
                              tol2, max_iter, st);
    *H->ctl_host = MarchCtl{0u, 1, 0, 0, 0ull};
    CK(cudaMemcpyAsync(H->plan.ctl, H->ctl_host, sizeof(MarchCtl), cudaMemcpyHostToDevice, st));
    const bool prof = H->prof_on && result;
    if (prof) CK(cudaEventRecord(H->prof_ev[PROF_PCG], st));
    if (launch_march_pcg(H->plan, st) != 0) return POISSON_ECUDA;
    if (prof) CK(cudaEventRecord(H->prof_ev[PROF_PCG + 1], st));
    if (bf16) launch_rb_finish<__nv_bfloat16>(d, H->eta16, H->r32, b.x, H->d32, st);
    else launch_rb_finish<float>(d, H->eta32, H->r32, b.x, H->d32, st);
    CK(cudaStreamSynchronize(st));
    if (prof) prof_add(H, POISSON_K_PCG, H->prof_ev[PROF_PCG], H->prof_ev[PROF_PCG + 1]);
    if (result) CK(cudaMemcpy(result, H->sc, sizeof(Scalars), cudaMemcpyDeviceToHost));
    return POISSON_OK;
}

static std::map<TuneKey, std::pair<int, int>> g_tuned_rb;  // (variant, split), under g_tune_mu

static int build_rb_plan(poisson_t* H, int var, int strategy) {
    const bool bf16 = H->opts.precision == POISSON_FP32_BF16COEF;
    const MarchSolve s = rb_solve_of(H);
    const int nctas = march_occupancy(var, bf16) * num_sms();
    if (nctas <= 0) return -1;
    return march_plan_build(&H->plan, &s, 1, var, bf16, nctas, strategy, H->st);
}

// Variant and split of the red-black kernels: a forced family-3 tile, else the fastest of every
// family-3 variant and split on a constant-density model problem (16 iterations per try, cached
// per size class like the Jacobi kernels).  A forced tile of another family keeps the column
// kernels.
static int setup_rb(poisson_t* H) {
    const bool bf16 = H->opts.precision == POISSON_FP32_BF16COEF;
    const Dims d = H->d;
    const int forced = H->opts.tile;
    int var = -1, strategy = MARCH_SPLIT_LOCKSTEP;
    if (forced > 0) {
        var = march_variant_of_tile(forced);
        strategy = march_split_of_tile(forced);
        if (var < 0 || march_variant(var).family != 3) return POISSON_OK;
    } else {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned_rb.find(tune_key(d, bf16));
        if (it != g_tuned_rb.end()) {
            var = it->second.first;
            strategy = it->second.second;
        }
    }
    if (var < 0) {
        constexpr int TUNE_ITERS = 16;
        cudaStream_t st = H->st;
        const long long n = d.n;
        if (bf16) launch_fill_bf16(n, H->eta16, 0.5f, st);
        else launch_fill_f32(n, H->eta32, 0.5f, st);
        launch_fill_f32(n, H->r32, 1.0f, st);
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best = 1e30f;
        for (int cand = 0; cand < march_variant_count(); ++cand) {
            if (march_variant(cand).family != 3 || march_occupancy(cand, bf16) <= 0) continue;
            for (int strat = 0; strat < MARCH_SPLITS; ++strat) {
                if (build_rb_plan(H, cand, strat) != 0) continue;
                float t[2];
                bool good = true;
                for (int rep = 0; rep < 2 && good; ++rep) {
                    cudaEventRecord(e0, st);
                    good = march_rb_run(H, bf16, 0.0, TUNE_ITERS) == POISSON_OK;
                    cudaEventRecord(e1, st);
                    cudaEventSynchronize(e1);
                    cudaEventElapsedTime(&t[rep], e0, e1);
                }
                if (!good || cudaGetLastError() != cudaSuccess) continue;
                const float tt = std::min(t[0], t[1]);
                if (tt < best) {
                    best = tt;
                    var = cand;
                    strategy = strat;
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaMemsetAsync(H->sc, 0, sizeof(Scalars), st);
        cudaStreamSynchronize(st);
        if (var >= 0) {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tuned_rb[tune_key(d, bf16)] = {var, strategy};
        }
    }
    if (var < 0) return POISSON_OK;  // stay on the column kernels
    const int rc = build_rb_plan(H, var, strategy);
    if (rc == -2) return POISSON_ENOMEM;
    H->rb = (rc == 0);
    return POISSON_OK;
}

static void drop_chunk_graph(poisson_t* H) {
    if (H->chunk_exec) cudaGraphExecDestroy(H->chunk_exec);
    if (H->chunk_graph) cudaGraphDestroy(H->chunk_graph);
    H->chunk_exec = nullptr;
    H->chunk_graph = nullptr;
    H->chunk_tag = nullptr;
    H->chunk_nodes = 0;
}

static void free_state(poisson_t* H) {
    drop_chunk_graph(H);
    void* ptrs[] = {H->bx, H->by, H->bz, H->diag, H->dinv, H->top64, H->rinv2, H->ax64, H->ay64,
                    H->az64, H->vol64, H->bx32, H->by32, H->bz32, H->diag32, H->pu[0], H->pu[1],
                    H->ps[0], H->ps[1], H->pw[0], H->pw[1], H->peta32, H->peta16, H->eta32, H->eta16, H->x64,
                    H->b64, H->r64, H->z64, H->p64a, H->p64b, H->d32, H->r32, H->z32,
                    H->p32a, H->p32b, H->s32a, H->s32b, H->w32a, H->w32b, H->sc,
                    H->partials, H->io_a, H->io_b, H->io_c, H->io_c32};
    for (void* p : ptrs) dfree(p);
    if (H->sc_host) lib_free_host(H->sc_host);
    if (H->ctl_host) lib_free_host(H->ctl_host);
    for (auto& e : H->ev) if (e) cudaEventDestroy(e);
    for (auto& e : H->prof_ev) if (e) cudaEventDestroy(e);
    if (H->plan.trace) {
        // development aid (POISSON_TRACE set): CTA 0's time per part of a PCG iteration
        unsigned long long t[TRACE_PARTS] = {};
        if (cudaMemcpy(t, H->plan.trace, sizeof(t), cudaMemcpyDeviceToHost) == cudaSuccess && t[TR_ITERS]) {
            const char* names[] = {"phaseA", "bar1", "alpha", "phaseB", "bar2", "beta", "iters",
                                   "wait_slowest", "release", "(sums_kcycles",
                                   "decide_kcycles)"};
            fprintf(stderr, "[poisson trace] %dx%dx%d %llu iterations, us/iteration:", H->d.nx,
                    H->d.ny, H->d.nz, t[TR_ITERS]);
            for (int q = 0; q < TRACE_PARTS; ++q)
                if (q != TR_ITERS)
                    fprintf(stderr, " %s=%.2f", names[q], 1e-3 * (double)t[q] / (double)t[TR_ITERS]);
            fprintf(stderr, "\n");
        }
        cudaGetLastError();
    }
    march_plan_free(&H->plan);
    mg_free(&H->mg);
}

// The options of a new handle (defaults for NULL) and its grid, checked; POISSON_EINVAL if any is
// out of range.
static int check_create(int nx, int ny, int nz, const poisson_opts* opts, poisson_opts* out,
                        Dims* out_dims) {
    if (nx <= 0 || ny <= 0 || nz <= 0) return POISSON_EINVAL;
    const long long n = (long long)nx * ny * nz;
    if (n >= (1LL << 31)) return POISSON_EINVAL;
    poisson_opts o;
    poisson_default_opts(&o);
    if (opts) o = *opts;
    if (o.precision < POISSON_FP64 || o.precision > POISSON_FP32_BF16COEF) return POISSON_EINVAL;
    if (o.precond != POISSON_JACOBI && o.precond != POISSON_RBSSOR && o.precond != POISSON_MG)
        return POISSON_EINVAL;
    if (!(o.omega > 0.0 && o.omega < 2.0)) return POISSON_EINVAL;
    if (o.max_iters <= 0 || !(o.inner_tol > 0.0 && o.inner_tol < 1.0)) return POISSON_EINVAL;
    if (o.tile < -1 || (o.tile > 0 && march_variant_of_tile(o.tile) < 0))
        return POISSON_EINVAL;
    // the red-black kernels (tile codes 3xxxxxxx) run only the red-black SSOR preconditioner
    if (o.tile > 0 && march_variant(march_variant_of_tile(o.tile)).family == 3 &&
        o.precond != POISSON_RBSSOR)
        return POISSON_EINVAL;
    if (o.dirichlet_walls < 0 || o.dirichlet_walls > POISSON_WALLS_ALL) return POISSON_EINVAL;
    if (o.periodic_x != 0 && o.periodic_x != 1) return POISSON_EINVAL;
    if (o.periodic_x && (o.dirichlet_walls & (POISSON_WALL_XM | POISSON_WALL_XP))) return POISSON_EINVAL;
    if (o.periodic_x && o.precond == POISSON_RBSSOR && nx % 2) return POISSON_EINVAL;

    const Dims dims{nx, ny, nz, nx * ny, (int)n,
                    o.dirichlet_walls | (o.periodic_x ? PERIODIC_X : 0)};
    if (o.precond == POISSON_MG) {
        // the V-cycle needs at least one coarser level
        MgHier probe;
        if (mg_plan(dims, &probe) < 2) return POISSON_EINVAL;
    }
    *out = o;
    *out_dims = dims;
    return POISSON_OK;
}

// Reduction partial slots of one column-kernel launch of the handle's grid.
static size_t column_blocks(const Dims& d, int kc) {
    const dim3 g((d.nx + TX - 1) / TX, (d.ny + TY - 1) / TY, (d.nz + kc - 1) / kc);
    return (size_t)g.x * g.y * g.z;
}

// Every device array a handle allocates at creation, in allocation order: f(&pointer, count,
// element size).  poisson_create allocates with this list and poisson_required_bytes counts it,
// so the two cannot drift apart.
template <typename F>
static void for_each_array(poisson_t* H, F&& f) {
    const Dims& d = H->d;
    const poisson_opts& o = H->opts;
    const size_t N = (size_t)d.n, D8 = sizeof(double), F4 = sizeof(float);
    f((void**)&H->bx, N, D8); f((void**)&H->by, N, D8); f((void**)&H->bz, N, D8);
    f((void**)&H->diag, N, D8);
    f((void**)&H->top64, (size_t)d.sxy, D8);
    if (o.periodic_x && o.precision != POISSON_FP64 && d.nx % 8 == 0) {
        // padded rows for the one-sweep marching kernels (ghost columns, PAD_V each side)
        const size_t np = (size_t)(d.nx + 2 * PAD_V) * d.ny * d.nz;
        for (int b = 0; b < 2; ++b) {
            f((void**)&H->pu[b], np, F4); f((void**)&H->ps[b], np, F4);
            f((void**)&H->pw[b], np, F4);
        }
        if (o.precision == POISSON_FP32)
            f((void**)&H->peta32, (size_t)(d.nx + 8) * d.ny * d.nz, F4);
        else
            f((void**)&H->peta16, (size_t)(d.nx + 16) * d.ny * d.nz, sizeof(__nv_bfloat16));
    }
    if (o.dirichlet_walls) f((void**)&H->rinv2, N, D8);  // (not needed for periodic x)
    f((void**)&H->eta32, N, F4); f((void**)&H->eta16, N, sizeof(__nv_bfloat16));
    f((void**)&H->x64, N, D8); f((void**)&H->b64, N, D8);
    if (o.precision == POISSON_FP64) {
        f((void**)&H->dinv, N, D8);
        f((void**)&H->r64, N, D8); f((void**)&H->z64, N, D8); f((void**)&H->p64a, N, D8);
        f((void**)&H->p64b, N, D8);
    } else {
        for (float** q : {&H->d32, &H->r32, &H->z32, &H->p32a, &H->p32b, &H->s32a, &H->s32b,
                          &H->w32a, &H->w32b})
            f((void**)q, N, F4);
    }
    f((void**)&H->sc, 1, sizeof(Scalars));
    f((void**)&H->partials, std::max<size_t>(2 * H->nblocks + 64, 4096), D8);
}

// Device bytes of the multigrid hierarchy of a planned MgHier (the fine pre-smoothed vector and
// seven arrays per coarse cell).
static size_t mg_bytes(const MgHier& m, bool dbl) {
    const size_t es = dbl ? sizeof(double) : sizeof(float);
    size_t b = es * (size_t)m.d[0].n;
    for (int l = 1; l < m.nlev; ++l) b += 7 * es * (size_t)m.d[l].n;
    return b;
}

// Upper bound on the persistent-launch plan of one handle (work list, tensor maps, partial
// sums, control words): MAXSEG segments per CTA, at most 8 resident CTAs per SM.
static size_t plan_bytes_max() {
    const size_t ctas = 8 * (size_t)num_sms();
    const size_t segs = ctas * MAXSEG;
    return sizeof(SolveDev) + segs * (sizeof(Seg) + 4 * sizeof(float2)) +
           (ctas + 1) * sizeof(int) + MAPS_PER_SOLVE * sizeof(CUtensorMap) + sizeof(MarchCtl) +
           4096;
}

extern "C" int poisson_create(int nx, int ny, int nz, double h, const poisson_opts* opts,
                              poisson_t** out) {
    if (!out || !(h > 0.0) || !std::isfinite(h)) return POISSON_EINVAL;
    poisson_opts o;
    Dims dims;
    const int cr = check_create(nx, ny, nz, opts, &o, &dims);
    if (cr != POISSON_OK) return cr;

    poisson_t* H = new (std::nothrow) poisson_t();
    if (!H) return POISSON_ENOMEM;
    H->d = dims;
    H->h = h;
    H->opts = o;
    H->st = (cudaStream_t)o.stream;
    H->kc = choose_kc(H->d);
    cudaGetDevice(&H->device);
    H->nblocks = column_blocks(H->d, H->kc);

    int rc = POISSON_OK;
    auto A = [&](int r) { if (rc == POISSON_OK) rc = r; };
    for_each_array(H, [&](void** p, size_t count, size_t es) {
        if (rc != POISSON_OK) return;
        *p = nullptr;
        if (count == 0) return;
        if (lib_malloc(p, es * count) != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            rc = POISSON_ENOMEM;
        }
    });
    if (o.precond == POISSON_MG && rc == POISSON_OK) {
        mg_plan(H->d, &H->mg);
        A(mg_alloc(&H->mg, o.precision == POISSON_FP64));
    }
    if (rc == POISSON_OK && lib_malloc_host((void**)&H->sc_host, 2 * sizeof(Scalars)) != cudaSuccess) {
        cudaGetLastError();
        H->sc_host = nullptr;
        rc = POISSON_ENOMEM;
    }
    if (rc == POISSON_OK && lib_malloc_host((void**)&H->ctl_host, sizeof(MarchCtl)) != cudaSuccess) {
        cudaGetLastError();
        H->ctl_host = nullptr;
        rc = POISSON_ENOMEM;
    }
    for (auto& e : H->ev)
        if (rc == POISSON_OK && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            rc = POISSON_ECUDA;
    if (rc == POISSON_OK && cudaMemsetAsync(H->sc, 0, sizeof(Scalars), H->st) != cudaSuccess)
        rc = POISSON_ECUDA;
    if (rc == POISSON_OK && o.precision != POISSON_FP64 && o.precond == POISSON_JACOBI &&
        o.tile != -1 && march_supported(H->d))
        A(setup_march(H));
    if (rc == POISSON_OK && o.precision != POISSON_FP64 && o.precond == POISSON_RBSSOR &&
        o.omega == 1.0 && o.tile != -1 && march_supported(H->d) && !o.periodic_x)
        A(setup_rb(H));
    if (rc != POISSON_OK) {
        free_state(H);
        delete H;
        return rc;
    }
    *out = H;
    return POISSON_OK;
}

extern "C" int poisson_destroy(poisson_t* H) {
    if (!H) return POISSON_OK;
    // a job of a batch (possibly running on a worker thread) still uses the handle
    if (batch_handle_busy(H)) return POISSON_EINVAL;
    cudaStreamSynchronize(H->st);
    free_state(H);
    delete H;
    return POISSON_OK;
}

extern "C" int poisson_required_bytes(int nx, int ny, int nz, const poisson_opts* opts,
                                      uint64_t budget, uint64_t* bytes) {
    if (!bytes) return POISSON_EINVAL;
    poisson_opts o;
    Dims dims;
    const int cr = check_create(nx, ny, nz, opts, &o, &dims);
    if (cr != POISSON_OK) return cr;
    poisson_t probe;
    probe.d = dims;
    probe.opts = o;
    probe.nblocks = column_blocks(dims, choose_kc(dims));
    size_t b = 0;
    for_each_array(&probe, [&](void**, size_t count, size_t es) { b += count * es; });
    if (o.precond == POISSON_MG) {
        MgHier m;
        mg_plan(dims, &m);
        b += mg_bytes(m, o.precision == POISSON_FP64);
    }
    if (o.precision != POISSON_FP64) b += plan_bytes_max();
    *bytes = (uint64_t)b;
    return (budget > 0 && b > budget) ? POISSON_ENOMEM_BUDGET : POISSON_OK;
}

extern "C" int poisson_handle_bytes(poisson_t* H, uint64_t* bytes) {
    if (!H || !bytes) return POISSON_EINVAL;
    size_t b = 0;
    poisson_t* Hc = H;
    for_each_array(Hc, [&](void** p, size_t count, size_t es) { b += (*p) ? count * es : 0; });
    if (H->mg.nlev >= 2) b += mg_bytes(H->mg, H->mg.dbl);
    const MarchPlan& pl = H->plan;
    b += pl.cap_solves + pl.cap_segs + pl.cap_cta + pl.cap_maps + pl.cap_pa + pl.cap_pb + pl.cap_ctl;
    const size_t n = (size_t)H->d.n, nu = (size_t)(H->d.nx + 1) * H->d.ny * H->d.nz,
                 nv = (size_t)H->d.nx * (H->d.ny + 1) * H->d.nz,
                 nw = (size_t)H->d.sxy * (H->d.nz + 1);
    if (H->ax64) b += sizeof(double) * (nu + nv + nw + n);  // cut-cell fractions
    if (H->bx32) b += 4 * sizeof(float) * n;                 // their FP32 faces and diagonal
    if (H->io_a) b += sizeof(double) * n;                    // staging of the checking calls
    if (H->io_b) b += sizeof(double) * n;
    if (H->io_c) b += sizeof(double) * n;
    if (H->io_c32) b += sizeof(float) * n;
    if (H->plan.trace) b += sizeof(unsigned long long) * TRACE_PARTS;
    *bytes = (uint64_t)b;
    return POISSON_OK;
}

extern "C" int poisson_set_density(poisson_t* H, const double* F, double rho_air,
                                   double rho_water, int mem) {
    if (!H || !F || !(rho_air > 0.0) || !(rho_water > 0.0)) return POISSON_EINVAL;
    NvtxRange range("poisson_set_density");
    if (mem != POISSON_MEM_HOST && mem != POISSON_MEM_DEVICE) return POISSON_EINVAL;
    const bool dev = is_device_ptr(F);
    if (dev != (mem == POISSON_MEM_DEVICE)) return POISSON_EINVAL;
    const size_t bytes = sizeof(double) * (size_t)H->d.n;
    const double* Fd = F;
    if (!dev) {
        // stage F through b64 (overwritten by every solve)
        CK(copy_user(H->b64, F, bytes, cudaMemcpyHostToDevice, H->st));
        Fd = H->b64;
    }
    // the density check's flag lives in the reduction partials (free between solves)
    unsigned* bad = reinterpret_cast<unsigned*>(H->partials);
    CK(cudaMemsetAsync(bad, 0, sizeof(unsigned), H->st));
    H->ready = false;
    launch_setup(H->d, Fd, rho_air, rho_water, H->bx, H->by, H->bz, H->diag, H->dinv, H->top64,
                 H->rinv2, H->eta32, H->eta16, H->apertures(), bad, H->st);
    unsigned bad_host = 0;
    CK(cudaMemcpyAsync(&bad_host, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, H->st));
    CK(cudaStreamSynchronize(H->st));
    if (bad_host) return POISSON_EINVAL;  // left not ready: solves give ENOTREADY
    if (H->periodic() && H->pu[0]) {
        // rho/2 in rows padded by its halo width (4 FP32 / 8 BF16 columns, 16 bytes)
        if (H->peta32) launch_pad_rows_f32(H->d, 4, H->eta32, H->peta32, H->st);
        if (H->peta16) launch_pad_rows_bf16(H->d, 8, H->eta16, H->peta16, H->st);
    }
    if (H->cut() && H->bx32) {
        const long long n = H->d.n;
        launch_narrow_f32(n, H->bx, H->bx32, H->st);
        launch_narrow_f32(n, H->by, H->by32, H->st);
        launch_narrow_f32(n, H->bz, H->bz32, H->st);
        launch_narrow_f32(n, H->diag, H->diag32, H->st);
    }
    if (H->opts.precond == POISSON_MG) mg_setup(&H->mg, H->bx, H->by, H->bz, H->diag, H->st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(H->st));
    H->ready = true;
    return POISSON_OK;
}

extern "C" int poisson_set_apertures(poisson_t* H, const double* ax, const double* ay,
                                     const double* az, const double* vol, int mem) {
    if (!H) return POISSON_EINVAL;
    drop_chunk_graph(H);  // the inner operator (and its arrays) may change
    const Dims d = H->d;
    const size_t nu = (size_t)(d.nx + 1) * d.ny * d.nz, nv = (size_t)d.nx * (d.ny + 1) * d.nz,
                 nw = (size_t)d.sxy * (d.nz + 1), n = (size_t)d.n;
    if (!ax && !ay && !az && !vol) {
        // back to the plain operator
        for (double** q : {&H->ax64, &H->ay64, &H->az64, &H->vol64}) {
            dfree(*q);
            *q = nullptr;
        }
        H->d.walls &= ~CUT_CELLS;
        // the plan built at create, if any
        H->march = H->plan.segs != nullptr && H->opts.precond == POISSON_JACOBI;
        H->rb = H->plan.segs != nullptr && H->opts.precond == POISSON_RBSSOR;
        H->ready = false;
        return POISSON_OK;
    }
    if (!ax || !ay || !az || !vol) return POISSON_EINVAL;
    if (mem != POISSON_MEM_HOST && mem != POISSON_MEM_DEVICE) return POISSON_EINVAL;
    for (const double* q : {ax, ay, az, vol})
        if (is_device_ptr(q) != (mem == POISSON_MEM_DEVICE)) return POISSON_EINVAL;
    int rc = POISSON_OK;
    auto A = [&](int r) { if (rc == POISSON_OK) rc = r; };
    if (!H->ax64) {
        A(dalloc(&H->ax64, nu)); A(dalloc(&H->ay64, nv)); A(dalloc(&H->az64, nw));
        A(dalloc(&H->vol64, n));
    }
    if (H->opts.precision != POISSON_FP64 && !H->bx32) {
        A(dalloc(&H->bx32, n)); A(dalloc(&H->by32, n)); A(dalloc(&H->bz32, n));
        A(dalloc(&H->diag32, n));
    }
    if (rc != POISSON_OK) return rc;
    const cudaMemcpyKind kind = mem == POISSON_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                                          : cudaMemcpyHostToDevice;
    CK(copy_user(H->ax64, ax, sizeof(double) * nu, kind, H->st));
    CK(copy_user(H->ay64, ay, sizeof(double) * nv, kind, H->st));
    CK(copy_user(H->az64, az, sizeof(double) * nw, kind, H->st));
    CK(copy_user(H->vol64, vol, sizeof(double) * n, kind, H->st));
    CK(cudaStreamSynchronize(H->st));
    H->d.walls |= CUT_CELLS;
    H->march = false;  // the marching kernels form faces from rho/2 and cannot carry fractions
    H->rb = false;
    H->ready = false;  // poisson_set_density builds the cut operator
    return POISSON_OK;
}

// ------------------------------------------------------------------ profiling events
// Event pairs around CG phase / residual kernels (poisson_profile).  Slot q of a chunk owns
// events [q * PROF_PER_CHUNK, (q + 1) * PROF_PER_CHUNK).
static int prof_events(poisson_t* H) {
    if (!H->prof_ev.empty()) return POISSON_OK;
    H->prof_ev.resize(PROF_EVENTS);
    for (auto& e : H->prof_ev) CK(cudaEventCreate(&e));
    return POISSON_OK;
}

static void prof_add(poisson_t* H, int cls, cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) == cudaSuccess) {
        H->prof.ms[cls] += ms;
        H->prof.launches[cls] += 1;
    } else {
        cudaGetLastError();
    }
}

// ------------------------------------------------------------------ inner CG loop
// Queues chunks of CG_CHUNK iterations; reads the scalars of chunk n while chunk n+1 runs.
// pass_a(p_in_is_a) and pass_b(p_is_a) launch one CG phase each on the handle's stream.
// A stream that can be captured into a graph (not the legacy or per-thread default stream).
static bool capturable(cudaStream_t st) {
    return st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread;
}

// Captures `passes` (the launches of one CG chunk) on the handle's stream as a graph for code
// path `tag`.  The passes' launch arguments (buffers, scalars, sizes) are the handle's own and do
// not change between chunks, and a chunk has an even number of iterations, so every chunk starts
// on the same p buffer and one graph serves them all.  false (nothing launched, no graph) when
// the capture fails; the caller then launches the passes directly.
template <typename F>
static bool capture_chunk(poisson_t* H, const void* tag, F&& passes) {
    drop_chunk_graph(H);
    if (cudaStreamBeginCapture(H->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    passes();
    cudaGraph_t g = nullptr;
    if (cudaStreamEndCapture(H->st, &g) != cudaSuccess || !g) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        return false;
    }
    size_t n = 0;
    cudaGraphGetNodes(g, nullptr, &n);
    g_kernel_launches.fetch_sub((unsigned long long)n, std::memory_order_relaxed);  // not run
    cudaGraphExec_t x = nullptr;
    if (cudaGraphInstantiate(&x, g, 0) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        return false;
    }
    H->chunk_graph = g;
    H->chunk_exec = x;
    H->chunk_tag = tag;
    H->chunk_nodes = n;
    return true;
}

template <typename V, typename Coef, typename PassA, typename PassB>
static int cg_loop(poisson_t* H, const Coef& coef, V* r, V* z, double tol2, int rel_to_b,
                   int max_iter, Scalars* result, PassA pass_a, PassB pass_b) {
    const int K = CG_CHUNK;
    cudaStream_t st = H->st;
    const bool prof = H->prof_on;
    if (H->opts.precond == POISSON_MG)
        mg_init<V, Coef>(&H->mg, H->d, H->kc, coef, r, z, H->sc, H->partials, tol2, rel_to_b,
                         max_iter, st);
    else if (H->opts.precond == POISSON_RBSSOR)
        launch_ssor_init<V, Coef>(H->d, H->kc, coef, r, z, H->opts.omega, H->sc, H->partials, tol2,
                                  rel_to_b, max_iter, st);
    else
        launch_cg_init<V, Coef>(H->d, H->kc, coef, r, z, H->sc, H->partials, tol2, rel_to_b,
                                max_iter, st);
    static_assert(CG_CHUNK % 2 == 0, "a chunk returns to the p buffer it started from");
    static const char tag = 0;  // this code path (one per instantiation of the loop)
    bool in_is_a = true;
    auto passes = [&] {
        bool a = true;
        for (int q = 0; q < K; ++q) {
            pass_a(a);
            pass_b(!a);
            a = !a;
        }
    };
    auto enqueue_chunk = [&](int slot) -> int {
        cudaEvent_t* ev = prof ? &H->prof_ev[slot * PROF_PER_CHUNK] : nullptr;
        // without per-phase events, on a capturable stream: one graph launch per chunk
        if (!prof && capturable(st) &&
            (H->chunk_tag == &tag || capture_chunk(H, &tag, passes))) {
            CK(cudaGraphLaunch(H->chunk_exec, st));
            g_kernel_launches.fetch_add((unsigned long long)H->chunk_nodes,
                                        std::memory_order_relaxed);
            CK(cudaMemcpyAsync(&H->sc_host[slot], H->sc, sizeof(Scalars), cudaMemcpyDeviceToHost,
                               st));
            CK(cudaEventRecord(H->ev[slot], st));
            return POISSON_OK;
        }
        for (int q = 0; q < K; ++q) {
            if (prof) CK(cudaEventRecord(ev[3 * q], st));
            pass_a(in_is_a);
            if (prof) CK(cudaEventRecord(ev[3 * q + 1], st));
            pass_b(!in_is_a);
            if (prof) CK(cudaEventRecord(ev[3 * q + 2], st));
            in_is_a = !in_is_a;
        }
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(&H->sc_host[slot], H->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, st));
        CK(cudaEventRecord(H->ev[slot], st));
        return POISSON_OK;
    };
    // Scalars copied back with a chunk tell how many of its iterations did work.
    int it_seen = 0;
    auto harvest = [&](int slot) {
        if (!prof) return;
        const int it_now = H->sc_host[slot].iter;
        // iterations of this chunk that did work (later ones returned at once)
        const int live = std::max(0, std::min(K, it_now - it_seen));
        cudaEvent_t* ev = &H->prof_ev[slot * PROF_PER_CHUNK];
        for (int q = 0; q < live; ++q) {
            prof_add(H, POISSON_K_CG_A, ev[3 * q], ev[3 * q + 1]);
            prof_add(H, POISSON_K_CG_B, ev[3 * q + 1], ev[3 * q + 2]);
        }
        it_seen = it_now;
    };
    int rc = enqueue_chunk(0);
    if (rc) return rc;
    int slot = 0;
    long long launched = K;
    for (;;) {
        const bool more = launched < (long long)max_iter + K;
        if (more) {
            rc = enqueue_chunk(slot ^ 1);
            if (rc) return rc;
            launched += K;
        }
        CK(cudaEventSynchronize(H->ev[slot]));
        const Scalars s = H->sc_host[slot];
        harvest(slot);
        if (s.done != RUNNING || !more) {
            CK(cudaStreamSynchronize(st));
            CK(cudaMemcpy(result, H->sc, sizeof(Scalars), cudaMemcpyDeviceToHost));
            return POISSON_OK;
        }
        slot ^= 1;
    }
}

// Column-kernel passes (any shape, any precision; Jacobi, red-black SSOR or the V-cycle).
template <typename V, typename Coef>
static int cg_loop_columns(poisson_t* H, const Coef& coef, V* x, V* r, V* z, V* pa, V* pb,
                           double tol2, int rel_to_b, int max_iter, Scalars* result) {
    const Dims d = H->d;
    const int kc = H->kc;
    cudaStream_t st = H->st;
    auto A = [=](bool in_a) {
        launch_cg_a<V, Coef>(d, kc, coef, z, in_a ? pa : pb, in_a ? pb : pa, H->sc, H->partials, st);
    };
    const bool ssor = H->opts.precond == POISSON_RBSSOR;
    const bool mg = H->opts.precond == POISSON_MG;
    const double omega = H->opts.omega;
    auto B = [=](bool p_a) {
        if (mg)
            mg_cg_b<V, Coef>(&H->mg, d, kc, coef, p_a ? pa : pb, x, r, z, H->sc, H->partials, st);
        else if (ssor)
            launch_cg_b_ssor<V, Coef>(d, kc, coef, p_a ? pa : pb, x, r, z, omega, H->sc,
                                      H->partials, st);
        else
            launch_cg_b<V, Coef>(d, kc, coef, p_a ? pa : pb, x, r, z, H->sc, H->partials, st);
    };
    return cg_loop<V, Coef>(H, coef, r, z, tol2, rel_to_b, max_iter, result, A, B);
}

// Reads the scalars after a residual kernel (and books its time when profiling).
static int read_scalars(poisson_t* H, Scalars* s) {
    CK(cudaMemcpyAsync(&H->sc_host[0], H->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, H->st));
    CK(cudaStreamSynchronize(H->st));
    *s = H->sc_host[0];
    if (H->prof_on)
        prof_add(H, POISSON_K_RESIDUAL, H->prof_ev[PROF_RES],
                 H->prof_ev[PROF_RES + 1]);
    return POISSON_OK;
}

// Plain FP64 PCG on A64 x = b; restarts from the recomputed residual if the recurrence drifts.
static int solve_fp64(poisson_t* H, double tol, int* outer, int* inner, double* rel_out) {
    const CoefFaces64 c{H->bx, H->by, H->bz, H->diag, H->dinv};
    const size_t bytes = sizeof(double) * (size_t)H->d.n;
    int total = 0, status = POISSON_ENOTCONV;
    double rel = INFINITY;
    int restarts = 0;
    for (;; ++restarts) {
        if (H->prof_on) CK(cudaEventRecord(H->prof_ev[PROF_RES], H->st));
        launch_residual64(H->d, H->kc, c, H->b64, H->x64, H->r64, H->sc, H->partials, H->st);
        if (H->prof_on) CK(cudaEventRecord(H->prof_ev[PROF_RES + 1], H->st));
        CK(cudaGetLastError());
        Scalars s;
        int rc = read_scalars(H, &s);
        if (rc) return rc;
        if (s.bb == 0.0) {
            CK(cudaMemsetAsync(H->x64, 0, bytes, H->st));
            rel = 0.0;
            status = POISSON_OK;
            break;
        }
        rel = std::sqrt(s.rr / s.bb);
        if (!std::isfinite(rel)) { status = POISSON_EBREAKDOWN; break; }
        if (rel <= tol) { status = POISSON_OK; break; }
        if (total >= H->opts.max_iters || restarts >= 8) { status = POISSON_ENOTCONV; break; }
        CK(cudaMemsetAsync(H->p64a, 0, bytes, H->st));
        Scalars res;
        rc = cg_loop_columns<double, CoefFaces64>(H, c, H->x64, H->r64, H->z64, H->p64a, H->p64b,
                                                  tol * tol, 1, H->opts.max_iters - total, &res);
        if (rc) return rc;
        total += res.iter;
        if (res.done == TIMEDOUT) { status = POISSON_ETIMEOUT; break; }
        if (res.done == BREAKDOWN && res.iter == 0) { status = POISSON_EBREAKDOWN; break; }
    }
    *outer = restarts + 1;
    *inner = total;
    *rel_out = rel;
    return status;
}

// FP32 inner PCG on the reduced-precision operator inside FP64 iterative refinement:
//   r = b - A64 x (FP64); stop when ||r||/||b|| <= tol; solve A32 d = r (FP32 PCG, relative
//   reduction inner_tol); x += d.
template <typename C32>
static int solve_mixed(poisson_t* H, const C32& c32, bool bf16, double tol, int* outer, int* inner,
                       double* rel_out) {
    const CoefFaces64 c64{H->bx, H->by, H->bz, H->diag, nullptr};
    const size_t bytes32 = sizeof(float) * (size_t)H->d.n;
    int total = 0, status = POISSON_ENOTCONV, k = 0;
    double rel = INFINITY, prev = INFINITY;
    int stalls = 0;
    for (k = 0;; ++k) {
        if (H->prof_on) CK(cudaEventRecord(H->prof_ev[PROF_RES], H->st));
        launch_residual64_f32(H->d, H->kc, c64, H->b64, H->x64, H->r32, H->sc, H->partials, H->st);
        if (H->prof_on) CK(cudaEventRecord(H->prof_ev[PROF_RES + 1], H->st));
        CK(cudaGetLastError());
        Scalars s;
        int rc = read_scalars(H, &s);
        if (rc) return rc;
        if (s.bb == 0.0) {
            CK(cudaMemsetAsync(H->x64, 0, sizeof(double) * (size_t)H->d.n, H->st));
            rel = 0.0;
            status = POISSON_OK;
            break;
        }
        rel = std::sqrt(s.rr / s.bb);
        if (!std::isfinite(rel)) { status = POISSON_EBREAKDOWN; break; }
        if (rel <= tol) { status = POISSON_OK; break; }
        if (rel > 0.5 * prev) ++stalls; else stalls = 0;
        if (total >= H->opts.max_iters || stalls >= 3 || k >= 60) { status = POISSON_ENOTCONV; break; }
        prev = rel;
        double target = std::max(H->opts.inner_tol, 0.3 * tol / rel);
        target = std::min(target, 0.5);
        CK(cudaMemsetAsync(H->d32, 0, bytes32, H->st));
        CK(cudaMemsetAsync(H->p32a, 0, bytes32, H->st));
        NvtxRange inner_range("inner solve");
        Scalars res;
        rc = POISSON_ECUDA;
        bool inner_done = false, rb_used = false;
        if (H->rb && H->opts.precond == POISSON_RBSSOR) {
            rb_used = true;
            rc = march_rb_run(H, bf16, target * target, H->opts.max_iters - total, &res);
            if (rc == POISSON_ECUDA) H->rb = false;  // launch refused: use the column kernels
            else inner_done = true;
        } else if (H->march && H->opts.precond == POISSON_JACOBI) {
            rc = march_run(H, bf16, target * target, H->opts.max_iters - total, &res);
            if (rc == POISSON_ECUDA) H->march = false;  // launch refused: use the column kernels
            else inner_done = true;
        }
        if (!inner_done)
            rc = cg_loop_columns<float, C32>(H, c32, H->d32, H->r32, H->z32, H->p32a,
                                                    H->p32b, target * target, 0,
                                                    H->opts.max_iters - total, &res);
        if (rc) return rc;
        total += res.iter;
        // (the red-black solve's correction holds its red relaxation even after 0 iterations)
        if (res.iter > 0 || (rb_used && inner_done && res.done != BREAKDOWN && res.done != TIMEDOUT))
            launch_update64(H->d.n, H->x64, H->d32, H->st);
        CK(cudaGetLastError());
        if (res.done == TIMEDOUT) { status = POISSON_ETIMEOUT; break; }
        if (res.done == BREAKDOWN && res.iter == 0) { status = POISSON_EBREAKDOWN; break; }
    }
    *outer = k + 1;
    *inner = total;
    *rel_out = rel;
    return status;
}

extern "C" int poisson_test_unreachable_barrier(poisson_t* H, int extra) {
    if (!H || extra < 0 || extra > 1024) return POISSON_EINVAL;
    if (!(H->march || H->rb) || H->cut()) return POISSON_EINVAL;
    H->plan.barrier_extra = extra;
    return POISSON_OK;
}

extern "C" int poisson_solve(poisson_t* H, const double* rhs, double* p, double tol,
                             poisson_stats* stats) {
    if (!H || !rhs || !p || !(tol > 0.0)) return POISSON_EINVAL;
    if (!H->ready) return POISSON_ENOTREADY;
    NvtxRange range("poisson_solve");
    const double t0 = now_s();
    const size_t n = (size_t)H->d.n, bytes = sizeof(double) * n;
    const bool drhs = is_device_ptr(rhs), dp = is_device_ptr(p);
    const double a = -(H->h * H->h);
    if (drhs) {
        launch_scale((long long)n, rhs, a, H->b64, H->st, H->vol64);
    } else {
        CK(copy_user(H->b64, rhs, bytes, cudaMemcpyHostToDevice, H->st));
        launch_scale((long long)n, H->b64, a, H->b64, H->st, H->vol64);
    }
    CK(cudaGetLastError());
    CK(copy_user(H->x64, p, bytes, dp ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       H->st));
    int outer = 0, inner = 0;
    double rel = 0.0;
    int status;
    switch (H->opts.precision) {
        case POISSON_FP64: status = solve_fp64(H, tol, &outer, &inner, &rel); break;
        default:
            if (H->cut())  // the open fractions live in the stored faces
                status = solve_mixed(H, CoefFaces32{H->bx32, H->by32, H->bz32, H->diag32}, false,
                                     tol, &outer, &inner, &rel);
            else if (H->opts.precision == POISSON_FP32)
                status = solve_mixed(H, CoefEta<float>{H->eta32}, false, tol, &outer, &inner, &rel);
            else
                status = solve_mixed(H, CoefEta<__nv_bfloat16>{H->eta16}, true, tol, &outer, &inner,
                                     &rel);
            break;
    }
    if (status == POISSON_ECUDA) return status;
    CK(copy_user(p, H->x64, bytes, dp ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       H->st));
    CK(cudaStreamSynchronize(H->st));
    if (stats) {
        stats->outer_iters = outer;
        stats->inner_iters = inner;
        stats->rel_residual = rel;
        stats->seconds = now_s() - t0;
    }
    return status;
}

// ------------------------------------------------------------------ checking entry points
static int io_buffers(poisson_t* H) {
    if (H->io_a) return POISSON_OK;
    int rc = dalloc(&H->io_a, (size_t)H->d.n);
    if (rc == POISSON_OK) rc = dalloc(&H->io_b, (size_t)H->d.n);
    return rc;
}

// Runs `fn(in_dev, out_dev)` on device copies of host arrays when needed.
template <typename Fn>
static int with_io(poisson_t* H, const double* in, double* out, Fn fn) {
    const size_t bytes = sizeof(double) * (size_t)H->d.n;
    const bool din = is_device_ptr(in), dout = is_device_ptr(out);
    if (!din || !dout) {
        int rc = io_buffers(H);
        if (rc) return rc;
    }
    const double* xi = in;
    double* yo = out;
    if (!din) {
        CK(copy_user(H->io_a, in, bytes, cudaMemcpyHostToDevice, H->st));
        xi = H->io_a;
    }
    if (!dout) yo = H->io_b;
    fn(xi, yo);
    CK(cudaGetLastError());
    if (!dout) CK(copy_user(out, yo, bytes, cudaMemcpyDeviceToHost, H->st));
    CK(cudaStreamSynchronize(H->st));
    return POISSON_OK;
}

extern "C" int poisson_apply(poisson_t* H, const double* x, double* y, int precision) {
    if (!H || !x || !y || x == y) return POISSON_EINVAL;
    if (!H->ready) return POISSON_ENOTREADY;
    const Dims d = H->d;
    const int kc = H->kc;
    cudaStream_t st = H->st;
    switch (precision) {
        case POISSON_FP64: {
            const CoefFaces64 c{H->bx, H->by, H->bz, H->diag, nullptr};
            return with_io(H, x, y, [&](const double* a, double* b) {
                launch_apply<double, CoefFaces64>(d, kc, c, a, b, st);
            });
        }
        case POISSON_FP32:
        case POISSON_FP32_BF16COEF:
            if (H->cut()) {
                const CoefFaces32 c{H->bx32, H->by32, H->bz32, H->diag32};
                return with_io(H, x, y, [&](const double* a, double* b) {
                    launch_apply<float, CoefFaces32>(d, kc, c, a, b, st);
                });
            }
            if (precision == POISSON_FP32_BF16COEF) {
                const CoefEta<__nv_bfloat16> c{H->eta16};
                return with_io(H, x, y, [&](const double* a, double* b) {
                    launch_apply<float, CoefEta<__nv_bfloat16>>(d, kc, c, a, b, st);
                });
            } else {
                const CoefEta<float> c{H->eta32};
                return with_io(H, x, y, [&](const double* a, double* b) {
                    launch_apply<float, CoefEta<float>>(d, kc, c, a, b, st);
                });
            }
        default: return POISSON_EINVAL;
    }
}

extern "C" int poisson_precond_apply(poisson_t* H, const double* r, double* z, int kind,
                                     int precision) {
    if (!H || !r || !z || r == z) return POISSON_EINVAL;
    if (!H->ready) return POISSON_ENOTREADY;
    if (kind != POISSON_JACOBI && kind != POISSON_RBSSOR && kind != POISSON_MG)
        return POISSON_EINVAL;
    if (precision < POISSON_FP64 || precision > POISSON_FP32_BF16COEF) return POISSON_EINVAL;
    const Dims d = H->d;
    const int kc = H->kc;
    cudaStream_t st = H->st;
    if (kind == POISSON_MG) {
        // the handle's own hierarchy, in the handle's own precision
        if (H->opts.precond != POISSON_MG || precision != H->opts.precision) return POISSON_EINVAL;
        if (precision == POISSON_FP64) {
            const CoefFaces64 c{H->bx, H->by, H->bz, H->diag, nullptr};
            return with_io(H, r, z, [&](const double* a, double* b) {
                mg_apply<double, CoefFaces64>(&H->mg, d, kc, c, a, b, st);
            });
        }
        // FP32 V-cycle on narrowed copies (r32 and d32 are rebuilt by every solve)
        return with_io(H, r, z, [&](const double* a, double* b) {
            launch_narrow_f32(d.n, a, H->r32, st);
            if (H->cut())
                mg_apply<float, CoefFaces32>(&H->mg, d, kc,
                                             CoefFaces32{H->bx32, H->by32, H->bz32, H->diag32},
                                             H->r32, H->d32, st);
            else if (precision == POISSON_FP32)
                mg_apply<float, CoefEta<float>>(&H->mg, d, kc, CoefEta<float>{H->eta32}, H->r32,
                                                H->d32, st);
            else
                mg_apply<float, CoefEta<__nv_bfloat16>>(
                    &H->mg, d, kc, CoefEta<__nv_bfloat16>{H->eta16}, H->r32, H->d32, st);
            launch_widen_f32(d.n, H->d32, b, st);
        });
    }
    const double om = H->opts.omega;
    if (kind == POISSON_RBSSOR) {
        // sweeps in the precision's arithmetic on a scratch vector of that type
        if (precision == POISSON_FP64) {
            if (!H->io_c) {
                int rc = dalloc(&H->io_c, (size_t)d.n);
                if (rc) return rc;
            }
        } else if (!H->io_c32) {
            int rc = dalloc(&H->io_c32, (size_t)d.n);
            if (rc) return rc;
        }
    }
    switch (precision) {
        case POISSON_FP64: {
            const CoefFaces64 c{H->bx, H->by, H->bz, H->diag, nullptr};
            return with_io(H, r, z, [&](const double* a, double* b) {
                if (kind == POISSON_RBSSOR)
                    launch_ssor_apply<double, CoefFaces64>(d, kc, c, a, H->io_c, om, b, st);
                else
                    launch_jacobi<double, CoefFaces64>(d, kc, c, a, b, st);
            });
        }
        case POISSON_FP32: {
            if (H->cut()) {
                const CoefFaces32 c{H->bx32, H->by32, H->bz32, H->diag32};
                return with_io(H, r, z, [&](const double* a, double* b) {
                    if (kind == POISSON_RBSSOR)
                        launch_ssor_apply<float, CoefFaces32>(d, kc, c, a, H->io_c32, om, b, st);
                    else
                        launch_jacobi<float, CoefFaces32>(d, kc, c, a, b, st);
                });
            }
            const CoefEta<float> c{H->eta32};
            return with_io(H, r, z, [&](const double* a, double* b) {
                if (kind == POISSON_RBSSOR)
                    launch_ssor_apply<float, CoefEta<float>>(d, kc, c, a, H->io_c32, om, b, st);
                else
                    launch_jacobi<float, CoefEta<float>>(d, kc, c, a, b, st);
            });
        }
        default: {
            const CoefEta<__nv_bfloat16> c{H->eta16};
            return with_io(H, r, z, [&](const double* a, double* b) {
                if (kind == POISSON_RBSSOR)
                    launch_ssor_apply<float, CoefEta<__nv_bfloat16>>(d, kc, c, a, H->io_c32, om, b,
                                                                    st);
                else
                    launch_jacobi<float, CoefEta<__nv_bfloat16>>(d, kc, c, a, b, st);
            });
        }
    }
}

extern "C" int poisson_get_operator(poisson_t* H, double* bx, double* by, double* bz,
                                    double* diag) {
    if (!H) return POISSON_EINVAL;
    if (!H->ready) return POISSON_ENOTREADY;
    const size_t bytes = sizeof(double) * (size_t)H->d.n;
    const double* src[4] = {H->bx, H->by, H->bz, H->diag};
    double* dst[4] = {bx, by, bz, diag};
    for (int q = 0; q < 4; ++q) {
        if (!dst[q]) continue;
        CK(copy_user(dst[q], src[q], bytes,
                           is_device_ptr(dst[q]) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           H->st));
    }
    CK(cudaStreamSynchronize(H->st));
    return POISSON_OK;
}

extern "C" uint64_t poisson_kernel_launches(void) {
    return (uint64_t)g_kernel_launches.load(std::memory_order_relaxed);
}

extern "C" int poisson_profile(poisson_t* H, int enable) {
    if (!H) return POISSON_EINVAL;
    if (enable) {
        int rc = prof_events(H);
        if (rc) return rc;
    }
    H->prof_on = enable != 0;
    H->prof = poisson_kernel_times{};
    return POISSON_OK;
}

extern "C" int poisson_profile_read(poisson_t* H, poisson_kernel_times* out) {
    if (!H || !out) return POISSON_EINVAL;
    *out = H->prof;
    return POISSON_OK;
}

extern "C" int poisson_describe(poisson_t* H, char* buf, int len) {
    if (!H || !buf || len <= 0) return POISSON_EINVAL;
    const char* prec = H->opts.precision == POISSON_FP64 ? "fp64"
                       : H->opts.precision == POISSON_FP32 ? "fp32" : "fp32/bf16-coef";
    if (H->march || H->rb) {
        const MarchVariant v = march_variant(H->plan.variant);
        snprintf(buf, (size_t)len,
                 "%s march tile=%d (%dx%d cells, %dx%d per thread%s, %d stages) persistent %s "
                 "ctas=%d segments=%d split=%s",
                 prec, march_tile_of(H->plan.variant) + 1000000 * H->plan.strategy, v.width,
                 v.height, v.cx, v.cy, v.ws ? ", producer warp" : "", v.ns,
                 v.family == 3   ? "one-sweep red-black SSOR (black Schur complement)"
                 : v.family == 2 ? "one-sweep (A p formed)"
                 : v.family == 1 ? "one-sweep"
                                 : "two-sweep",
                 H->plan.nctas, H->plan.nsegs,
                 H->plan.strategy == MARCH_SPLIT_BALANCED        ? "balanced"
                 : H->plan.strategy == MARCH_SPLIT_LOCKSTEP      ? "lockstep"
                 : H->plan.strategy == MARCH_SPLIT_LOCKSTEP_FILL ? "lockstep-fill"
                                                                 : "equal");
    } else {
        char mgs[48] = "";
        if (H->opts.precond == POISSON_MG) snprintf(mgs, sizeof mgs, " mg-vcycle levels=%d", H->mg.nlev);
        snprintf(buf, (size_t)len, "%s columns (%dx%d threads) zchunk=%d%s%s", prec, TX, TY, H->kc,
                 H->cut() ? " cut-cells" : "", mgs);
    }
    return POISSON_OK;
}

extern "C" const char* poisson_strerror(int s) {
    switch (s) {
        case POISSON_OK: return "ok";
        case POISSON_PENDING: return "pending";
        case POISSON_EINVAL: return "invalid argument";
        case POISSON_ENOMEM: return "out of memory";
        case POISSON_ENOTCONV: return "not converged (iteration cap)";
        case POISSON_EBREAKDOWN: return "CG breakdown (p.Ap <= 0 or non-finite)";
        case POISSON_ETIMEOUT: return "device wait timed out";
        case POISSON_ENOTREADY: return "density not set";
        case POISSON_ECUDA: return "CUDA runtime error";
        case POISSON_ENOMEM_BUDGET: return "over the device-memory budget";
        case POISSON_ENOTICKET: return "unknown ticket";
        case POISSON_ETOOLARGE: return "grid too large for the allocation-free entry point";
        default: return "unknown status";
    }
}

extern "C" const char* poisson_version(void) { return "libpoisson 0.1 (sm_103a)"; }
