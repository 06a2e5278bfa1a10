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
// FP32 estimate of cfl_speed for an FP64 state.  Its relative error is below
// 1e-3 for every finite state: the rounding of the inputs and of the FP32
// operations is a few 1e-7 relative, except where the pressure comes from
// cancellation (kinetic energy far above the internal energy); there the
// error of c is at most ~sqrt(eps32) of the speed, which the flow speed then
// dominates.  NaN inputs give NaN.
__device__ __forceinline__ float cfl_estimate(float gm1, float gam, float rfl, float cf2g, double r, double mn,
                                              double mt, double E) {
    float rho = (float)r;
    rho = (rho < rfl) ? rfl : rho;
    const float ir = 1.0f / rho;
    const float u = (float)mn * ir, v = (float)mt * ir;
    float p = gm1 * ((float)E - 0.5f * rho * (u * u + v * v));
    const float pm = rho * cf2g;
    p = (p < pm) ? pm : p;
    const float c = sqrtf(gam * p * ir);
    return fmaxf(fabsf(u), fabsf(v)) + c;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = (w > v) ? w : v;
    }
    return v;
}

// PASS 0: per-grid max of the FP32 estimate (bits of non-negative floats and
// NaN order as unsigned integers, NaN above +inf).  PASS 1: the exact FP64
// speed of every cell whose estimate is not below M (1 - kCflScreen), folded
// into wmax[acc] like the sweeps' fold it replaces.
template <int PASS>
__global__ void __launch_bounds__(256) cfl_fp64_kernel(const double* __restrict__ st,
                                                       const GridDesc* __restrict__ grids,
                                                       const Strip* __restrict__ strips, int nstrips,
                                                       GridRun* run, const DevCounters* ctr, Consts<double> K) {
    const float gm1 = (float)K.gm1, gam = (float)K.gamma, rfl = (float)K.rho_floor, cf2g = (float)K.cf2g;
    const unsigned acc = ctr->acc;
    const int lane = threadIdx.x & 31;
    for (int si = blockIdx.x; si < nstrips; si += gridDim.x) {
        const Strip sp = strips[si];
        const GridDesc g = grids[sp.grid];
        float thr = 0.0f;
        if (PASS == 1) {
            const float M = __uint_as_float(run[sp.grid].smax32);
            thr = isfinite(M) ? M * (1.0f - kCflScreen) : 0.0f;
        }
        unsigned long long m = 0ull;
        const int n = sp.nrows * g.nx;
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const int j = sp.row0 + k / g.nx, i = k - (k / g.nx) * g.nx;
            const double* q = st + g.off + (long long)j * g.pitch + i;
            const double r = q[0], mn = q[g.plane], mt = q[2 * g.plane], E = q[3 * g.plane];
            const float e = cfl_estimate(gm1, gam, rfl, cf2g, r, mn, mt, E);
            if (PASS == 0) {
                const unsigned long long b = __float_as_uint(e);
                m = (b > m) ? b : m;
            } else if (!(e < thr)) {
                const double w = cfl_speed(K, Cons<double>{r, mn, mt, E});
                const unsigned long long b = (unsigned long long)__double_as_longlong(w);
                m = (b > m) ? b : m;
            }
        }
        m = warp_max_u64(m);
        if (lane == 0 && m) {
            if (PASS == 0) atomicMax(&run[sp.grid].smax32, (unsigned)m);
            else atomicMax(&run[sp.grid].wmax[acc], m);
        }
    }
}

cudaError_t launch_cfl_fp64(const double* state, const GridDesc* grids, const Strip* strips, int nstrips,
                            GridRun* run, const DevCounters* ctr, const Consts<double>& K, int nctas,
                            cudaStream_t s) {
    if (nstrips <= 0) return cudaSuccess;
    const int blocks = nctas < nstrips ? nctas : nstrips;
    cfl_fp64_kernel<0><<<blocks, 256, 0, s>>>(state, grids, strips, nstrips, run, ctr, K);
    cfl_fp64_kernel<1><<<blocks, 256, 0, s>>>(state, grids, strips, nstrips, run, ctr, K);
    return cudaGetLastError();
}

template <>
int sweep_ctas_per_sm<double>(int dir, int var) {
    (void)var;
    return dir == DIR_X ? occupancy_one<double, DIR_X, VAR_F64>() : occupancy_one<double, DIR_Y, VAR_F64>();
}

}  // namespace hydro
