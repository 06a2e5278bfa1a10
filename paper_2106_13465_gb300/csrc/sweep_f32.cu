// sweep_f32.cu -- FP32 instantiations of the sweep kernels and of the fused
// step kernel: the main pass and the second pass over tiles holding a
// near-vacuum interface (solved again in FP64).  Built with fast single-precision division, square root and
// power; FP64 operations are IEEE.
#include "fused_tma.cuh"

namespace hydro {

__device__ __noinline__ Cons<double> flux_fp64_near_vacuum(const Consts<double>* Kd, Prim<double> L,
                                                           Prim<double> R) {
    return godunov_flux_exact<double, true>(*Kd, L, R, nullptr);  // the variants read at run time
}

template <>
cudaError_t launch_sweep<float>(int dir, int var, const SweepArgs<float>& a, int nctas, cudaStream_t s) {
    if (nctas <= 0) return cudaSuccess;
    if (var == VAR_F32_REDO)
        return dir == DIR_X ? launch_one<float, DIR_X, VAR_F32_REDO>(a, nctas, s)
                            : launch_one<float, DIR_Y, VAR_F32_REDO>(a, nctas, s);
    return dir == DIR_X ? launch_one<float, DIR_X, VAR_F32_MAIN>(a, nctas, s)
                        : launch_one<float, DIR_Y, VAR_F32_MAIN>(a, nctas, s);
}

template <>
cudaError_t launch_fused<float>(int order, int var, const SweepArgs<float>& a, int nctas, cudaStream_t s) {
    if (nctas <= 0) return cudaSuccess;
    if (var == VAR_F32_REDO) return launch_fused_var<float, VAR_F32_REDO>(order, a, nctas, s);
    return launch_fused_var<float, VAR_F32_MAIN>(order, a, nctas, s);
}

template <>
int fused_ctas_per_sm<float>(int var) {
    return var == VAR_F32_REDO ? fused_occupancy<float, VAR_F32_REDO>() : fused_occupancy<float, VAR_F32_MAIN>();
}

template <>
int sweep_ctas_per_sm<float>(int dir, int var) {
    if (var == VAR_F32_REDO)
        return dir == DIR_X ? occupancy_one<float, DIR_X, VAR_F32_REDO>() : occupancy_one<float, DIR_Y, VAR_F32_REDO>();
    return dir == DIR_X ? occupancy_one<float, DIR_X, VAR_F32_MAIN>() : occupancy_one<float, DIR_Y, VAR_F32_MAIN>();
}

}  // namespace hydro
