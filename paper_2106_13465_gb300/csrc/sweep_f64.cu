// sweep_f64.cu -- FP64 instantiations of the sweep kernels and of the fused
// step kernel, and the FP64 CFL passes.  FP64 additions, multiplications, fused multiply-adds and
// square roots are IEEE; divisions go through a refined FP32 reciprocal and
// the rarefaction power through a 7th root (gamma = 7/5) or exp2/log2, each
// within a few ulp (godunov.cuh: trcp, root7, pow_z).
#include "fused_tma.cuh"

namespace hydro {

template <>
cudaError_t launch_sweep<double>(int dir, int var, const SweepArgs<double>& a, int nctas, cudaStream_t s) {
    (void)var;
    if (nctas <= 0) return cudaSuccess;
    if (dir == DIR_X) return launch_one<double, DIR_X, VAR_F64>(a, nctas, s);
    return launch_one<double, DIR_Y, VAR_F64>(a, nctas, s);
}

// ---- CFL wave speed of the new state (FP64 contexts) ----------------------
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = (w > v) ? w : v;
    }
    return v;
}

// One warp per tile of the second sweep (a warp-strided loop over the list).
__global__ void __launch_bounds__(256) cfl_refine_kernel(const double* __restrict__ st,
                                                         const GridDesc* __restrict__ grids,
                                                         const Tile* __restrict__ tiles, int ntiles,
                                                         const unsigned int* ntiles_dev, int dir,
                                                         const unsigned int* __restrict__ tile_smax,
                                                         GridRun* run, const DevCounters* ctr, Consts<double> K) {
    const unsigned acc = ctr->acc;
    const int lane = threadIdx.x & 31;
    const unsigned nf = ntiles_dev ? ntiles_dev[0] : (unsigned)ntiles;
    const unsigned nb = ntiles_dev ? ntiles_dev[1] : 0u;
    const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
    for (unsigned i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nf + nb; i += nwarps) {
        const int t = (i < nf) ? (int)i : ntiles - 1 - (int)(i - nf);
        const Tile tile = tiles[t];
        const float M = __uint_as_float(run[tile.grid].smax32);
        const bool all = !isfinite(M);
        const float thr = all ? 0.0f : M * (1.0f - kCflScreen);
        if (!all && __uint_as_float(tile_smax[t]) < thr) continue;  // no cell near the max
        const GridDesc g = grids[tile.grid];
        unsigned long long m = 0ull;
        auto visit = [&](int i, int j) {
            const double* q = st + g.off + (long long)j * g.pitch + i;
            const double r = q[0], mn = q[g.plane], mt = q[2 * g.plane], E = q[3 * g.plane];
            if (!(cfl_estimate(K, r, mn, mt, E) < thr)) {
                const double w = cfl_speed(K, Cons<double>{r, mn, mt, E});
                const unsigned long long b = (unsigned long long)__double_as_longlong(w);
                m = (b > m) ? b : m;
            }
        };
        if (dir == DIR_X) {
            // FP64 walks the x lines: rows line0 .. line0 + 31, columns
            // cell0 .. cell0 + ncell - 1 (a lane per row)
            const int row = tile.line0 + lane;
            if (row < g.ny)
                for (int x = tile.cell0; x < tile.cell0 + tile.ncell; ++x) visit(x, row);
        } else if (dir == DIR_FUSED) {
            // columns [60 line0 - 2, 60 line0 + 58) of rows cell0 .. cell0 + ncell - 1
            const int x0 = max(0, kXStride * tile.line0 - 2);
            const int x1 = min(g.nx, kXStride * tile.line0 + kXStride - 2);
            for (int j = tile.cell0; j < tile.cell0 + tile.ncell; ++j)
                for (int x = x0 + lane; x < x1; x += 32) visit(x, j);
        } else {
            const int col = tile.line0 + lane;
            if (col < g.nx)
                for (int j = tile.cell0; j < tile.cell0 + tile.ncell; ++j) visit(col, j);
        }
        m = warp_max_u64(m);
        if (lane == 0 && m) atomicMax(&run[tile.grid].wmax[acc], m);
    }
}

cudaError_t launch_cfl_fp64(const double* state, const GridDesc* grids, const Tile* tiles, int ntiles,
                            const unsigned int* ntiles_dev, int dir, const unsigned int* tile_smax,
                            GridRun* run, const DevCounters* ctr, const Consts<double>& K, int nctas,
                            cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    cfl_refine_kernel<<<nctas, 256, 0, s>>>(state, grids, tiles, ntiles, ntiles_dev, dir, tile_smax, run, ctr, K);
    return cudaGetLastError();
}

// Whole-grid screen (PASS 0: max FP32 estimate into smax32) and exact pass
// (PASS 1: FP64 speed of the cells near that max into wmax[acc]).
template <int PASS>
__global__ void __launch_bounds__(256) cfl_grid_kernel(const double* __restrict__ st, GridDesc g, int grid,
                                                       GridRun* run, const DevCounters* ctr, Consts<double> K) {
    float thr = 0.0f;
    if (PASS == 1) {
        const float M = __uint_as_float(run[grid].smax32);
        thr = isfinite(M) ? M * (1.0f - kCflScreen) : 0.0f;
    }
    unsigned long long m = 0ull;
    const long long ncell = (long long)g.nx * g.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(c / g.nx), i = (int)(c - (long long)j * g.nx);
        const double* q = st + g.off + (long long)j * g.pitch + i;
        const double r = q[0], mn = q[g.plane], mt = q[2 * g.plane], E = q[3 * g.plane];
        const float e = cfl_estimate(K, r, mn, mt, E);
        if (PASS == 0) {
            const unsigned long long b = __float_as_uint(e);
            m = (b > m) ? b : m;
        } else if (!(e < thr)) {
            const unsigned long long b =
                (unsigned long long)__double_as_longlong(cfl_speed(K, Cons<double>{r, mn, mt, E}));
            m = (b > m) ? b : m;
        }
    }
    m = warp_max_u64(m);
    if ((threadIdx.x & 31) == 0 && m) {
        if (PASS == 0) atomicMax(&run[grid].smax32, (unsigned)m);
        else atomicMax(&run[grid].wmax[ctr->acc], m);
    }
}

cudaError_t launch_cfl_screened_fp64(const double* state, const GridDesc& gd, int grid, GridRun* run,
                                     const DevCounters* ctr, const Consts<double>& K, cudaStream_t s) {
    const long long ncell = (long long)gd.nx * gd.ny;
    long long nb = (ncell + 255) / 256;
    if (nb > 4096) nb = 4096;
    cfl_grid_kernel<0><<<(int)nb, 256, 0, s>>>(state, gd, grid, run, ctr, K);
    cfl_grid_kernel<1><<<(int)nb, 256, 0, s>>>(state, gd, grid, run, ctr, K);
    return cudaGetLastError();
}

template <>
cudaError_t launch_fused<double>(int order, int var, const SweepArgs<double>& a, int nctas, cudaStream_t s) {
    (void)var;
    if (nctas <= 0) return cudaSuccess;
    return launch_fused_var<double, VAR_F64>(order, a, nctas, s);
}

template <>
int fused_ctas_per_sm<double>(int var) {
    (void)var;
    return fused_occupancy<double, VAR_F64>();
}

template <>
int sweep_ctas_per_sm<double>(int dir, int var) {
    (void)var;
    return dir == DIR_X ? occupancy_one<double, DIR_X, VAR_F64>() : occupancy_one<double, DIR_Y, VAR_F64>();
}

}  // namespace hydro
