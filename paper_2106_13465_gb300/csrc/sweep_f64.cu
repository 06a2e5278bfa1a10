// sweep_f64.cu -- FP64 instantiation of the fused sweep kernel (IEEE double
// division, square root and power throughout).
#include "sweep_tma.cuh"

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

// After the second sweep, which left M = the grid's max FP32 speed estimate
// in smax32: the exact FP64 speed of every cell whose estimate is not below
// M (1 - kCflScreen) (every cell if M is not finite), folded into wmax[acc]
// (bits of non-negative doubles order as unsigned integers).
__global__ void __launch_bounds__(256) cfl_refine_kernel(const double* __restrict__ st,
                                                         const GridDesc* __restrict__ grids,
                                                         const Strip* __restrict__ strips, int nstrips,
                                                         GridRun* run, const DevCounters* ctr, Consts<double> K) {
    const unsigned acc = ctr->acc;
    const int lane = threadIdx.x & 31;
    for (int si = blockIdx.x; si < nstrips; si += gridDim.x) {
        const Strip sp = strips[si];
        const GridDesc g = grids[sp.grid];
        const float M = __uint_as_float(run[sp.grid].smax32);
        const float thr = isfinite(M) ? M * (1.0f - kCflScreen) : 0.0f;
        unsigned long long m = 0ull;
        const int n = sp.nrows * g.nx;
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const int dj = k / g.nx, i = k - dj * g.nx;
            const double* q = st + g.off + (long long)(sp.row0 + dj) * g.pitch + i;
            const double r = q[0], mn = q[g.plane], mt = q[2 * g.plane], E = q[3 * g.plane];
            if (!(cfl_estimate(K, r, mn, mt, E) < thr)) {
                const double w = cfl_speed(K, Cons<double>{r, mn, mt, E});
                const unsigned long long b = (unsigned long long)__double_as_longlong(w);
                m = (b > m) ? b : m;
            }
        }
        m = warp_max_u64(m);
        if (lane == 0 && m) atomicMax(&run[sp.grid].wmax[acc], m);
    }
}

cudaError_t launch_cfl_fp64(const double* state, const GridDesc* grids, const Strip* strips, int nstrips,
                            GridRun* run, const DevCounters* ctr, const Consts<double>& K, int nctas,
                            cudaStream_t s) {
    if (nstrips <= 0) return cudaSuccess;
    const int blocks = nctas < nstrips ? nctas : nstrips;
    cfl_refine_kernel<<<blocks, 256, 0, s>>>(state, grids, strips, nstrips, run, ctr, K);
    return cudaGetLastError();
}

template <>
int sweep_ctas_per_sm<double>(int dir, int var) {
    (void)var;
    return dir == DIR_X ? occupancy_one<double, DIR_X, VAR_F64>() : occupancy_one<double, DIR_Y, VAR_F64>();
}

}  // namespace hydro
