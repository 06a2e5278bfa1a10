// sweep_f32.cu -- FP32 instantiation of the fused sweep kernel.  Built with
// fast single-precision division, square root and power; FP64 operations are
// IEEE.  Near vacuum an interface is solved again in FP64.
#include "sweep_impl.cuh"

namespace hydro {

__device__ __noinline__ Cons<double> flux_fp64_near_vacuum(const Consts<double>* Kd,
                                                           Prim<double> L, Prim<double> R) {
    return godunov_flux_exact(*Kd, L, R, nullptr);
}

__device__ __forceinline__ Cons<float> FluxOp<float>::eval(const SweepArgs<float>& a,
                                                           const Prim<float>& L,
                                                           const Prim<float>& R, unsigned& nfb) {
    const Consts<float>& K = a.K;
    const float pmn = (L.p < R.p) ? L.p : R.p;
    const float pmx = (L.p < R.p) ? R.p : L.p;
    Star<float> s;
    Side<float> SL, SR;
    const bool near_vacuum_states = pmn < 1e-6f * pmx;
    if (!near_vacuum_states) {
        SL = make_side(K, L);
        SR = make_side(K, R);
        s = riemann_star(K, SL, SR);
    }
    if (near_vacuum_states || s.floored || s.p < 1e-3f * pmn) {
        ++nfb;
        const Prim<double> Ld = {L.r, L.u, L.v, L.p}, Rd = {R.r, R.u, R.v, R.p};
        const Cons<double> F = flux_fp64_near_vacuum(&a.Kd, Ld, Rd);
        return Cons<float>{(float)F.r, (float)F.mn, (float)F.mt, (float)F.E};
    }
    return physical_flux(K, sample0(K, SL, SR, s));
}

template <class T>
int sweep_ctas_per_sm(int dir) {
    int n = 0;
    if (dir == DIR_X)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_kernel<T, DIR_X>, kSweepThreads, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_kernel<T, DIR_Y>, kSweepThreads, 0);
    return n;
}

template cudaError_t launch_sweep<float>(int, const SweepArgs<float>&, int, cudaStream_t);
template int sweep_ctas_per_sm<float>(int);

}  // namespace hydro
