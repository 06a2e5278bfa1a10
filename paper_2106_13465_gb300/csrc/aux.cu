// aux.cu -- small kernels around the sweeps: the per-step dt prologue, the
// CFL wave-speed reduction of a freshly loaded state, FP64 <-> storage
// conversion, and the deterministic FP64 conservation sums.
#include "kernels.h"

namespace hydro {

// Per step, before its two sweeps: dt of every grid from the maximum wave
// speed of the state at the start of the step, dt = C h / w (FP64), or the
// caller's value; advance the grid's time; clear the speed slot the step's
// second sweep fills; reset the sweeps' work counters.
__global__ void step_prologue_kernel(GridRun* run, const GridDesc* grids, int ngrids,
                                     DevCounters* ctr, const double* dt_override, double cfl,
                                     double* dt_log) {
    const unsigned src = ctr->acc, dst = src ^ 1u;
    for (int g = threadIdx.x; g < ngrids; g += blockDim.x) {
        const double w = __longlong_as_double((long long)run[g].wmax[src]);
        const double dt = dt_override ? dt_override[g] : cfl * grids[g].h / w;
        run[g].dt = dt;
        run[g].t += dt;
        run[g].wmax[dst] = 0ull;
        if (dt_log) dt_log[g] = dt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ctr->acc = dst;
        ctr->tile_ctr[0] = 0u;
        ctr->tile_ctr[1] = 0u;
        ctr->redo_count[0] = 0u;
        ctr->redo_count[1] = 0u;
        ctr->redo_claim[0] = 0u;
        ctr->redo_claim[1] = 0u;
        ctr->steps += 1ull;
    }
}

cudaError_t launch_step_prologue(GridRun* run, const GridDesc* grids, int ngrids,
                                 DevCounters* ctr, const double* dt_override, double cfl,
                                 double* dt_log, cudaStream_t s) {
    const int nt = ngrids < 1024 ? ((ngrids + 31) / 32) * 32 : 1024;
    step_prologue_kernel<<<1, nt, 0, s>>>(run, grids, ngrids, ctr, dt_override, cfl, dt_log);
    return cudaGetLastError();
}

// ---- CFL speed of a loaded state ------------------------------------------
__global__ void cfl_zero_kernel(GridRun* run, int grid, const DevCounters* ctr) {
    run[grid].wmax[ctr->acc] = 0ull;
}

template <class T>
__global__ void cfl_reduce_kernel(const T* __restrict__ state, GridDesc g, int grid,
                                  GridRun* run, const DevCounters* ctr, Consts<T> K) {
    T smax = T(0);
    const long long ncell = (long long)g.nx * g.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(c / g.nx), i = (int)(c - (long long)j * g.nx);
        const T* p = state + g.off + (long long)j * g.pitch + i;
        const Cons<T> u = {p[0], p[g.plane], p[2 * g.plane], p[3 * g.plane]};
        const T s = cfl_speed(K, u);
        smax = (s <= smax) ? smax : s;
    }
    double m = (double)smax;
    for (int o = 16; o > 0; o >>= 1) {
        const double v = __shfl_xor_sync(0xffffffffu, m, o);
        m = (v <= m) ? m : v;
    }
    if ((threadIdx.x & 31) == 0)
        atomicMax(&run[grid].wmax[ctr->acc], (unsigned long long)__double_as_longlong(m));
}

template <class T>
cudaError_t launch_cfl_init(const T* state, const GridDesc* grids, int grid, const GridDesc& gd,
                            GridRun* run, DevCounters* ctr, Consts<T> K, cudaStream_t s) {
    (void)grids;
    cfl_zero_kernel<<<1, 1, 0, s>>>(run, grid, ctr);
    const long long ncell = (long long)gd.nx * gd.ny;
    long long nb = (ncell + 255) / 256;
    if (nb > 4096) nb = 4096;
    cfl_reduce_kernel<T><<<(int)nb, 256, 0, s>>>(state, gd, grid, run, ctr, K);
    return cudaGetLastError();
}

// ---- FP64 [4][ny][nx] <-> pitched storage ----------------------------------
template <class T>
__global__ void pack_kernel(const double* __restrict__ U, T* __restrict__ state, GridDesc g) {
    const long long n = 4ll * g.nx * g.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const long long q = c / ((long long)g.nx * g.ny);
        const long long r = c - q * g.nx * g.ny;
        const int j = (int)(r / g.nx), i = (int)(r - (long long)j * g.nx);
        state[g.off + q * g.plane + (long long)j * g.pitch + i] = (T)U[c];
    }
}

template <class T>
__global__ void unpack_kernel(const T* __restrict__ state, double* __restrict__ U, GridDesc g) {
    const long long n = 4ll * g.nx * g.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const long long q = c / ((long long)g.nx * g.ny);
        const long long r = c - q * g.nx * g.ny;
        const int j = (int)(r / g.nx), i = (int)(r - (long long)j * g.nx);
        U[c] = (double)state[g.off + q * g.plane + (long long)j * g.pitch + i];
    }
}

static int elementwise_blocks(long long n) {
    long long nb = (n + 255) / 256;
    return (int)(nb > 8192 ? 8192 : (nb < 1 ? 1 : nb));
}

template <class T>
cudaError_t launch_pack(const double* U, T* state, const GridDesc& gd, cudaStream_t s) {
    pack_kernel<T><<<elementwise_blocks(4ll * gd.nx * gd.ny), 256, 0, s>>>(U, state, gd);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_unpack(const T* state, double* U, const GridDesc& gd, cudaStream_t s) {
    unpack_kernel<T><<<elementwise_blocks(4ll * gd.nx * gd.ny), 256, 0, s>>>(state, U, gd);
    return cudaGetLastError();
}

// ---- deterministic FP64 conservation sums -----------------------------------
// Stage 1: one warp per (row, plane); lane l sums cells l, l+32, ... in order,
// then a fixed xor-shuffle tree.  Stage 2: one warp per plane over the row
// sums, same pattern, times h^2.  The order never depends on scheduling.
__device__ __forceinline__ double warp_sum_fixed(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <class T>
__global__ void row_sums_kernel(const T* __restrict__ state, GridDesc g, double* rows) {
    const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = blockIdx.x; j < g.ny; j += gridDim.x) {
        const T* p = state + g.off + q * g.plane + (long long)j * g.pitch;
        double s = 0.0;
        for (int i = lane; i < g.nx; i += 32) s += (double)p[i];
        s = warp_sum_fixed(s);
        if (lane == 0) rows[(long long)q * g.ny + j] = s;
    }
}

__global__ void final_sums_kernel(const double* rows, int ny, double h, double* out4) {
    const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double s = 0.0;
    for (int j = lane; j < ny; j += 32) s += rows[(long long)q * ny + j];
    s = warp_sum_fixed(s);
    if (lane == 0) out4[q] = s * h * h;
}

template <class T>
cudaError_t launch_conservation(const T* state, const GridDesc& gd, double* rows, double* out4,
                                cudaStream_t s) {
    const int nb = gd.ny < 8192 ? gd.ny : 8192;
    row_sums_kernel<T><<<nb, 128, 0, s>>>(state, gd, rows);
    final_sums_kernel<<<1, 128, 0, s>>>(rows, gd.ny, gd.h, out4);
    return cudaGetLastError();
}

template cudaError_t launch_cfl_init<double>(const double*, const GridDesc*, int, const GridDesc&,
                                             GridRun*, DevCounters*, Consts<double>, cudaStream_t);
template cudaError_t launch_cfl_init<float>(const float*, const GridDesc*, int, const GridDesc&,
                                            GridRun*, DevCounters*, Consts<float>, cudaStream_t);
template cudaError_t launch_pack<double>(const double*, double*, const GridDesc&, cudaStream_t);
template cudaError_t launch_pack<float>(const double*, float*, const GridDesc&, cudaStream_t);
template cudaError_t launch_unpack<double>(const double*, double*, const GridDesc&, cudaStream_t);
template cudaError_t launch_unpack<float>(const float*, double*, const GridDesc&, cudaStream_t);
template cudaError_t launch_conservation<double>(const double*, const GridDesc&, double*, double*,
                                                 cudaStream_t);
template cudaError_t launch_conservation<float>(const float*, const GridDesc&, double*, double*,
                                                cudaStream_t);

}  // namespace hydro
