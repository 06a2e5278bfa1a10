// sweep_f64.cu -- FP64 instantiation of the fused sweep kernel (IEEE double
// division, square root and power throughout).
#include "sweep_impl.cuh"

namespace hydro {

template <class T>
int sweep_ctas_per_sm(int dir) {
    int n = 0;
    if (dir == DIR_X)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_kernel<T, DIR_X>, kSweepThreads, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_kernel<T, DIR_Y>, kSweepThreads, 0);
    return n;
}

template cudaError_t launch_sweep<double>(int, const SweepArgs<double>&, int, cudaStream_t);
template int sweep_ctas_per_sm<double>(int);

}  // namespace hydro
