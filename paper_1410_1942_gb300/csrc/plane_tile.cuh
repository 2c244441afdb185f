// plane_tile.cuh -- shared-memory x-y planes of the column kernels' TX x TY tiles with a one-cell
// halo, for the fine-level z-marching kernels of the rho/2 operator (k_cg_a_sm in kernels.cu,
// k_mg_cg_b_sm and k_mg_smooth_sm in mg.cu).
//
// Those kernels march a thread's cell column in z with planes k-1, k, k+1 in registers.  Their x
// and y neighbours come from a shared plane instead of from global memory: every thread stores
// its own value of plane k, the threads with a halo slot store the ring's values (loaded a plane
// ahead), and one barrier per plane (two buffers) publishes them.  A cell then issues two or
// three global loads per plane instead of a dozen.
#pragma once

#include "internal.cuh"
#include "kernels.h"

namespace pcg {

constexpr int PT_W = TX + 2, PT_H = TY + 2, PT_N = PT_W * PT_H;

// Halo slot of the block's thread t = threadIdx.x + TX threadIdx.y: the row below the tile
// (t < TX), the row above (TX <= t < 2 TX), the column to the left (next TY) and to the right
// (next TY); (hx, hy) relative to the tile's first cell.  false: the thread has no slot.
__device__ __forceinline__ bool pt_halo_slot(int t, int& hx, int& hy) {
    if (t < TX) { hx = t; hy = -1; return true; }
    if (t < 2 * TX) { hx = t - TX; hy = TY; return true; }
    if (t < 2 * TX + TY) { hx = -1; hy = t - 2 * TX; return true; }
    if (t < 2 * TX + 2 * TY) { hx = TX; hy = t - 2 * TX - TY; return true; }
    hx = hy = 0;
    return false;
}

// Index in the shared plane of the tile cell (x, y), x in [-1, TX], y in [-1, TY].
__device__ __forceinline__ int pt_index(int x, int y) { return (y + 1) * PT_W + x + 1; }

// Whether the staged kernels serve a grid: whole tiles along x (every x neighbour of an active
// cell is in its tile or its halo) and no periodic wrap.
inline bool plane_tiles_fit(const Dims& d) { return d.nx % TX == 0 && !(d.walls & PERIODIC_X); }

}  // namespace pcg
