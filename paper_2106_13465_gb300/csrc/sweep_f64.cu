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

template <>
int sweep_ctas_per_sm<double>(int dir, int var) {
    (void)var;
    return dir == DIR_X ? occupancy_one<double, DIR_X, VAR_F64>() : occupancy_one<double, DIR_Y, VAR_F64>();
}

}  // namespace hydro
