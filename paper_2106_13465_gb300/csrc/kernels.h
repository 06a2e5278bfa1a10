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
//
// Each grid and buffer also has three TMA tensor maps over this layout, a 3D
// tensor (x, y, q) of extents (nx, ny, 4) with byte strides
// (pitch * esz, plane * esz):
//   x-sweep map: box (64 cells, 1 row, 4 planes)    -- one row segment,
//                starting at x = -4 + 60 k
//   y-sweep map: box (32 columns, 4 rows, 4 planes) -- 32 columns x 4 cells
//   fused map:   box (64 cells, kFusedRows + 4 rows, 4 planes) -- the input
//                of a fused step tile (below)
// stored at maps[map_index(grid, buffer, kind)].
//
// Fused step (one kernel per step instead of two sweeps).  A tile is the
// 60 columns [60 k - 2, 60 k + 58) of one x segment times up to kFusedRows
// rows [y0, y0 + rows); its input box is the 64 columns of the segment times
// rows [y0 - 2, y0 + rows + 2), loaded by one TMA copy into shared memory.
// The first sweep of the step runs on the box in place (x first: every box
// row, i.e. the tile's rows and 2 halo rows on each side; y first: every box
// column), the second writes the tile's cells to the other state buffer.
// Stored as (grid, line0 = k, cell0 = y0, ncell = rows).
//
// Work lists.  Walks (y sweep; FP64 x sweep): a tile is 32 lines (one per
// lane: columns in y, rows in x) x ncell cells.  FP32 x sweep: a tile is a
// run of consecutive segments of one row, stored as (grid, line0 = row,
// cell0 = first segment index, ncell = segments).
//
// Adaptive walk tiles (FP64, both directions).  The cells of each line group
// (32 lines) are divided into cost blocks of walk_block(d) cells (1 row in y,
// 4 columns in x, so that x pieces keep their 32-byte alignment).  Every walk
// records, per block, the estimated work of the tile that covered it (the
// largest over the warp's lanes of the sum of solve_work over the lane's
// cells, spread evenly over the tile's blocks); before the next sweep in the
// same direction a small kernel splits each tile of a static tiling (the one
// the scheduling model picks for uniform cost, in whole blocks) into pieces
// whose recorded work stays below kYCostCap times the mean work of a static
// tile.  Uniform work keeps the static tiles; where the Riemann solver works
// harder the tiles get shorter, so no warp is left with a tile far above the
// average when the queue runs dry.  Long pieces are queued before the others
// (longest jobs first, the short ones fill the tail): those of at least
// kYBigJob times the mean and kYBigOfMax times the largest piece of the
// previous sweep.  Where a few lines hold hard Riemann problems (one-block
// pieces at several times the mean) only they count as long, so they start
// at once, spread over the SMs, and do not wait behind the ordinary tiles;
// where the work is spread evenly the ordinary tiles are the long jobs and
// the split-off remainders the short ones.  The work estimate depends only
// on the state, so the tiling of a run is reproducible.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "godunov.cuh"

namespace hydro {

enum { BC_REFLECT = 0, BC_TRANSMISSIVE = 1, BC_PERIODIC = 2 };
enum { DIR_X = 0, DIR_Y = 1, DIR_FUSED = 2 };  // also the kinds of tensor map and work list
enum { STATUS_BAD_RHO = 1u, STATUS_BAD_E = 2u, STATUS_TIMEOUT = 4u, STATUS_BAD_TILE = 8u };

// kernel variants: FP64; FP32 main pass (tiles with a near-vacuum interface
// are queued for a second pass); FP32 second pass (FP64 near vacuum)
enum { VAR_F64 = 0, VAR_F32_MAIN = 1, VAR_F32_REDO = 2 };

constexpr int kWarpLines = 32;      // lines per warp tile (one per lane)
constexpr int kYBlock = 1;          // rows per cost block of the adaptive y tiles
constexpr int kXBlock = 4;          // columns per cost block of the adaptive x tiles (FP64
                                    // x walks start and end on multiples of 4 columns)
constexpr double kYCostCap = 1.0;   // adaptive tile work cap / mean static tile work
constexpr double kYBigJob = 0.5;    // adaptive tiles queued first: work / mean static tile work
constexpr double kYBigOfMax = 0.5;  // ... and work / largest piece of the previous sweep
// cells per cost block of the adaptive tiles of walk direction d
__host__ __device__ constexpr int walk_block(int d) { return d == 0 ? kXBlock : kYBlock; }
constexpr int kSweepThreads = 128;  // threads per CTA of the sweep kernels
// polls of an mbarrier before a sweep warp gives up waiting for a TMA copy
// (the default of SweepArgs::wait_limit, and the bound of the wait for the
// copies still in flight after a timeout)
constexpr unsigned kWaitLimit = 1u << 22;
constexpr unsigned long long kWaitNs = 1000000000ull;  // ... and at most about a second

// TMA ring geometry per warp.  x sweep: one slot holds a 64-cell segment of
// one row, 4 planes; y sweep: one slot holds 4 rows x 32 columns, 4 planes.
constexpr int kXSegment = 64;  // cells per x segment (2 per lane)
constexpr int kXStride = 60;   // segments overlap by 4 cells; 60 results each
constexpr int kFusedRows = 32;                  // output rows of a fused tile
constexpr int kFusedBoxRows = kFusedRows + 4;   // rows of its input box
constexpr int kFusedThreads = 128;              // threads per CTA of the fused kernel
constexpr int kMapKinds = 3;                    // tensor maps per grid and buffer
__host__ __device__ constexpr size_t map_index(int grid, int buffer, int kind) {
    return ((size_t)grid * 2 + buffer) * kMapKinds + kind;
}
template <class T>
__host__ __device__ constexpr int fused_box_bytes() {
    return 4 * kFusedBoxRows * kXSegment * (int)sizeof(T);
}
template <class T>
__host__ __device__ constexpr int fused_smem_bytes() {
    return fused_box_bytes<T>() + 16;  // the box and its mbarrier
}
__host__ __device__ constexpr int ring_slots(int dir) { return 4; }
template <class T>
__host__ __device__ constexpr int slot_bytes(int dir) {
    return dir == DIR_X ? 4 * kXSegment * (int)sizeof(T) : 4 * 4 * 32 * (int)sizeof(T);
}
template <class T>
__host__ __device__ constexpr int sweep_smem_bytes(int dir) {
    return (kSweepThreads / 32) * ring_slots(dir) * (slot_bytes<T>(dir) + 8);
}
// The x walk (FP64): a ring of 2 chunk slots per warp (4 columns x 32 rows x
// 4 planes each, as the y walk's slots), then, 128-byte aligned, 2 output
// staging blocks of the same shape per warp, written to global memory by TMA.
constexpr int kXWalkSlots = 2;
template <class T>
__host__ __device__ constexpr int xwalk_stage_offset() {
    return ((kSweepThreads / 32) * kXWalkSlots * (slot_bytes<T>(DIR_Y) + 8) + 127) / 128 * 128;
}
template <class T>
__host__ __device__ constexpr int xwalk_smem_bytes() {
    return xwalk_stage_offset<T>() + (kSweepThreads / 32) * 2 * slot_bytes<T>(DIR_Y);
}

struct GridDesc {
    long long off;    // element offset of plane 0 in a state buffer
    long long plane;  // elements per plane (ny * pitch)
    int nx, ny, pitch;
    int bc[4];        // x low, x high, y low, y high
    double h;
    // adaptive walk tiles, per walk direction d (0 x, 1 y): the grid's first
    // cost block, its line groups of 32 (x: rows, y: columns) and the cost
    // blocks of walk_block(d) cells along a line group
    long long wblk[2];
    int wlg[2], wnb[2];
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
    unsigned int smax32;         // FP64 contexts: max FP32 estimate of the wave
                                 // speed of the step's new state (bits of a float)
};


// SM ids below this bound spread the long adaptive tiles (see claim_tile).
constexpr int kMaxSmIds = 256;

// Context-wide device counters.
struct DevCounters {
    unsigned int acc;            // wmax slot holding the current state's speed
    unsigned int status;         // sticky STATUS_* flags
    unsigned int tile_ctr[2];    // work counters of the two sweeps of a step
    unsigned int redo_count[2];  // tiles queued for the FP32 second pass
    unsigned int redo_claim[2];  // work counters of the second pass
    unsigned long long steps;
    unsigned long long riemann_fp64;
    unsigned int wtiles[2][2];            // adaptive tiles of walk direction d in the
                                          // current step: the list holds wtiles[d][0]
                                          // long jobs from its front and wtiles[d][1]
                                          // short ones from its back
    unsigned long long wcost_total[2][2]; // recorded work of direction d, by step parity
    unsigned int wcost_max[2][2];         // largest recorded tile work, by step parity
    unsigned int sm_slot[2][kMaxSmIds];   // per sweep of the step: warps started on each SM
    int wait_site;                        // the first wait that gave up: kernel (1 x, 2 y,
    int wait_tile;                        // 3 fused, 4 fused second pass) and its tile
};

template <class T>
struct SweepArgs {
    const T* src;
    T* dst;
    const GridDesc* grids;
    const Tile* tiles;
    const CUtensorMap* maps;
    int ntiles;
    int ngrids;
    const unsigned int* ntiles_dev;  // adaptive tiles: the two counts on the device
                                     // (ntiles is then the capacity of the list)
    unsigned long long* wclaim;      // adaptive tiles: step count at which each long
                                     // job was last claimed (each taken once per step)
    int nsm;                         // SMs of the device
    float* wcost;                    // FP64 walks: per-block work recorded here
    unsigned int* tile_smax;         // FP64 second sweep: max FP32 speed estimate per tile
    unsigned wait_limit;  // polls of a TMA completion before a warp gives up
    int which;       // 0: first sweep of the step, 1: second (folds in CFL max)
    int src_buf;     // buffer index of src (its tensor maps)
    int* redo_list;  // [2][redo_cap] tile indices for the FP32 second pass
    int redo_cap;
    GridRun* run;
    DevCounters* ctr;
    Consts<T> K;
    Consts<double> Kd;  // FP64 constants (the FP32 path's near-vacuum solves)
};

// Resident CTAs per SM of a sweep kernel variant (occupancy calculator,
// including its dynamic shared memory).
template <class T>
int sweep_ctas_per_sm(int dir, int var);

// ---- launchers (defined in the kernel translation units) ------------------
// FP64 contexts: the max wave speed of the state a step produced.  The
// second sweep keeps the max M of an FP32 estimate of every new cell's speed
// per grid (smax32) and per tile (tile_smax); this pass then visits the tiles
// of that sweep whose own max is not below M (1 - kCflScreen) (every tile if
// M is not finite), evaluates the exact FP64 speed of each of their cells
// whose estimate is not below that bound, and folds it into wmax[acc].  The
// estimate is within 2e-3 of the exact speed (relative), well inside
// kCflScreen / 2, so the cell of the exact maximum is always evaluated.
// tiles / ntiles / ntiles_dev / dir describe the second sweep's work list as
// in SweepArgs (dir DIR_FUSED: the fused step's tile list).
constexpr float kCflScreen = 1e-2f;
cudaError_t launch_cfl_fp64(const double* state, const GridDesc* grids, const Tile* tiles, int ntiles,
                            const unsigned int* ntiles_dev, int dir, const unsigned int* tile_smax,
                            GridRun* run, const DevCounters* ctr, const Consts<double>& K, int nctas,
                            cudaStream_t s);

// The max wave speed of one FP64 grid's state (an uploaded state): the same
// screen as launch_cfl_fp64 over every cell (max FP32 estimate M), then the
// exact FP64 speed of the cells within kCflScreen of M, into wmax[acc].  run's
// slots of the grid must be zero.
cudaError_t launch_cfl_screened_fp64(const double* state, const GridDesc& gd, int grid, GridRun* run,
                                     const DevCounters* ctr, const Consts<double>& K, cudaStream_t s);

template <class T>
cudaError_t launch_sweep(int dir, int var, const SweepArgs<T>& a, int nctas, cudaStream_t s);

// Fused step: both sweeps of a step in one launch over the fused tile list
// (a.tiles, a.ntiles); order 0 sweeps x then y, order 1 y then x.  a.src is
// the state at the start of the step, a.dst receives the new state; the
// CFL wave speed of the new state is folded in as by the second sweep.
template <class T>
cudaError_t launch_fused(int order, int var, const SweepArgs<T>& a, int nctas, cudaStream_t s);

// Resident CTAs per SM of the fused kernel (and raise its shared-memory limit).
template <class T>
int fused_ctas_per_sm(int var);

// Cut the adaptive tiles of walk direction dir from the recorded work: each
// of the nstat tiles of the static tiling `stat` (whole cost blocks) is
// split where its pieces' work would exceed cap_per_total times the total
// recorded work of the previous sweep in that direction; pieces of at least
// big_per_total times that total and big_of_max times the largest tile work
// it recorded are queued first, the rest last (list of cap_tiles slots).
cudaError_t launch_retile(int dir, const GridDesc* grids, const Tile* stat, int nstat, const float* wcost,
                          DevCounters* ctr, Tile* tiles, int cap_tiles, double cap_per_total,
                          double big_per_total, double big_of_max, cudaStream_t s);

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
