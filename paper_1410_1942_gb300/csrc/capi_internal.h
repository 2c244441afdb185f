// capi_internal.h -- the handle behind the opaque poisson_t of include/poisson.h.
#pragma once

#include <vector>

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "poisson.h"
#include "internal.cuh"
#include "march.h"
#include "mg.h"

struct poisson_s {
    pcg::Dims d{};
    double h = 0.0;
    poisson_opts opts{};
    cudaStream_t st = nullptr;
    int kc = 1;          // z-planes per thread in the column kernels
    int device = 0;
    size_t nblocks = 0;  // blocks of one column-kernel launch (= reduction partials)
    bool ready = false;  // density set

    // FP64 operator: low-side face coefficients, diagonal, 1/diagonal (FP64 Jacobi only)
    double *bx = nullptr, *by = nullptr, *bz = nullptr, *diag = nullptr, *dinv = nullptr;
    // 2/rho_c of the top layer (nx*ny): the coefficient of the Dirichlet top face, for the
    // velocity correction of poisson_project
    double* top64 = nullptr;
    // 2/rho_c per cell, only when the handle has Dirichlet side/bottom walls (their faces in
    // poisson_project)
    double* rinv2 = nullptr;
    // free-slip cut cells (poisson_set_apertures): open fractions of the MAC faces, fluid
    // fractions of the cells, and the FP32 copies of the cut faces and diagonal for the inner
    // solve (all null without cut cells)
    double *ax64 = nullptr, *ay64 = nullptr, *az64 = nullptr, *vol64 = nullptr;
    float *bx32 = nullptr, *by32 = nullptr, *bz32 = nullptr, *diag32 = nullptr;
    pcg::Apertures apertures() const { return pcg::Apertures{ax64, ay64, az64, vol64}; }
    // periodic x on the one-sweep marching kernels: u, s^, w^ (both buffers) and rho/2 in rows
    // padded with ghost columns (PAD_V each side; rho/2 by its halo width)
    float *pu[2] = {nullptr, nullptr}, *ps[2] = {nullptr, nullptr}, *pw[2] = {nullptr, nullptr};
    float* peta32 = nullptr;
    __nv_bfloat16* peta16 = nullptr;
    bool periodic() const { return (d.walls & pcg::PERIODIC_X) != 0; }
    bool cut() const { return vol64 != nullptr; }
    // rho / 2 per cell for the reduced-precision inner operator
    float* eta32 = nullptr;
    __nv_bfloat16* eta16 = nullptr;
    // FP64 solution and right side (b = -h^2 s)
    double *x64 = nullptr, *b64 = nullptr;
    // plain FP64 PCG vectors
    double *r64 = nullptr, *z64 = nullptr, *p64a = nullptr, *p64b = nullptr;
    // FP32 inner PCG vectors (d = correction)
    float *d32 = nullptr, *r32 = nullptr, *z32 = nullptr, *p32a = nullptr, *p32b = nullptr;
    // the one-sweep kernels' s^ and w^ (both buffers); u is z32 / p32b, p is p32a
    float *s32a = nullptr, *s32b = nullptr, *w32a = nullptr, *w32b = nullptr;
    // device scalars, reduction partials, pinned host mirror (2 slots), chunk events
    pcg::Scalars* sc = nullptr;
    double* partials = nullptr;
    pcg::Scalars* sc_host = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    // staging for the checking entry points when given host arrays
    double *io_a = nullptr, *io_b = nullptr;
    double* io_c = nullptr;   // SSOR apply scratch (FP64)
    float* io_c32 = nullptr;  // SSOR apply scratch (FP32)
    // multigrid V-cycle hierarchy (POISSON_MG): Galerkin levels in the inner precision
    pcg::MgHier mg{};
    // TMA plane-marching kernels for the FP32 inner solve (when the shape allows them)
    bool march = false;
    // red-black SSOR (omega = 1) inner solve on the plane-marching kernels of march_rb.cu: CG on
    // the black Schur complement, compressed black vectors in the first and second halves of
    // z32 (x, p), p32a (u, both buffers), p32b (s^), s32a (w^); plan in `plan`
    bool rb = false;
    pcg::MarchPlan plan{};  // persistent work-list launch over this handle's grid
    pcg::MarchCtl* ctl_host = nullptr;  // pinned staging of plan.ctl
    // the column-kernel CG chunk (CG_CHUNK iterations of phases A and B) as a CUDA graph,
    // captured on the first chunk run on a capturable stream; chunk_tag names the code path it
    // was captured for, chunk_nodes its kernels
    cudaGraph_t chunk_graph = nullptr;
    cudaGraphExec_t chunk_exec = nullptr;
    const void* chunk_tag = nullptr;
    size_t chunk_nodes = 0;
    // poisson_profile: event pairs around the timed kernels, accumulated times
    bool prof_on = false;
    poisson_kernel_times prof{};
    std::vector<cudaEvent_t> prof_ev;
};

constexpr int CG_CHUNK = 8;                    // CG iterations queued per host check
constexpr int PROF_PER_CHUNK = 3 * CG_CHUNK;   // events per chunk slot when profiling
constexpr int PROF_RES = 2 * PROF_PER_CHUNK;   // event pair around a residual kernel
constexpr int PROF_PCG = PROF_RES + 2;         // event pair around a persistent PCG launch
constexpr int PROF_EVENTS = PROF_PCG + 2;

cudaError_t& last_cuda_error();
bool is_device_ptr(const void* p);
// Whether a handle is in a batch job not yet reported by poisson_poll (batch.cu).
bool batch_handle_busy(const poisson_t* H);
