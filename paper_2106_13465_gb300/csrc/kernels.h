// kernels.h -- device data layout and the launch interface between the
// C-ABI layer (hydro_abi.cu) and the kernel translation units.
//
// HBM layout of a context (one allocation per state buffer, two buffers that
// the sweeps ping-pong between: the first sweep of a step reads A and writes
// B, the second reads B and writes A, so a step always ends in A):
//   grid g occupies elements [off_g, off_g + 4 * plane_g) of a buffer;
//   plane q (rho, rho*u, rho*v, E) starts at off_g + q * plane_g;
//   cell (i, j) of a plane is at j * pitch_g + i, pitch_g = nx rounded up to
//   a multiple of 32 elements, plane_g = ny * pitch_g, off_g 256-B aligned.
// Interior cells only: the 2 ghost cells per side along the sweep axis are
// formed while a line is read (boundary conditions folded into the load).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "godunov.cuh"

namespace hydro {

enum { BC_REFLECT = 0, BC_TRANSMISSIVE = 1, BC_PERIODIC = 2 };
enum { DIR_X = 0, DIR_Y = 1 };
enum { STATUS_BAD_RHO = 1u, STATUS_BAD_E = 2u };

constexpr int kWarpLines = 32;      // lines per warp tile (one per lane)
constexpr int kSweepThreads = 128;  // threads per CTA of the sweep kernels

struct GridDesc {
    long long off;    // element offset of plane 0 in a state buffer
    long long plane;  // elements per plane (ny * pitch)
    int nx, ny, pitch;
    int bc[4];        // x low, x high, y low, y high
    double h;
};

// A warp tile: lines [line0, line0 + 32) of grid `grid`, cells
// [cell0, cell0 + ncell) along each line.
struct Tile {
    int grid, line0, cell0, ncell;
};

// Per-grid record of the time integration.
struct GridRun {
    double dt;                   // dt of the step in flight
    double t;                    // simulated time
    unsigned long long wmax[2];  // max wave speed (bits of a double >= 0) of the
                                 // state, double-buffered by step parity
};

// Context-wide device counters.
struct DevCounters {
    unsigned int acc;          // wmax slot holding the current state's speed
    unsigned int status;       // sticky STATUS_* flags
    unsigned int tile_ctr[2];  // work counters of the two sweeps of a step
    unsigned long long steps;
    unsigned long long riemann_fp64;
};

template <class T>
struct SweepArgs {
    const T* src;
    T* dst;
    const GridDesc* grids;
    const Tile* tiles;
    int ntiles;
    int which;       // 0: first sweep of the step, 1: second (folds in CFL max)
    GridRun* run;
    DevCounters* ctr;
    Consts<T> K;
    Consts<double> Kd;  // FP64 constants (the FP32 path's near-vacuum solves)
};

// Resident CTAs per SM of the sweep kernel (occupancy calculator).
template <class T>
int sweep_ctas_per_sm(int dir);

// ---- launchers (defined in the kernel translation units) ------------------
template <class T>
cudaError_t launch_sweep(int dir, const SweepArgs<T>& a, int nctas, cudaStream_t s);

cudaError_t launch_step_prologue(GridRun* run, const GridDesc* grids, int ngrids,
                                 DevCounters* ctr, const double* dt_override, double cfl,
                                 double* dt_log, cudaStream_t s);

template <class T>
cudaError_t launch_cfl_init(const T* state, const GridDesc* grids, int grid, const GridDesc& gd,
                            GridRun* run, DevCounters* ctr, Consts<T> K, cudaStream_t s);

template <class T>
cudaError_t launch_pack(const double* U, T* state, const GridDesc& gd, cudaStream_t s);

template <class T>
cudaError_t launch_unpack(const T* state, double* U, const GridDesc& gd, cudaStream_t s);

template <class T>
cudaError_t launch_conservation(const T* state, const GridDesc& gd, double* rows,
                                double* out4, cudaStream_t s);

}  // namespace hydro
