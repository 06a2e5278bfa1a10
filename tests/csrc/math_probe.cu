// Test helper: evaluates the sweep kernels' FP64 arithmetic helpers
// (godunov.cuh) elementwise on device arrays, so their error bounds can be
// checked against correctly rounded references.  Built by the test that
// uses it; not part of the library.
#include <cuda_runtime.h>
#include "godunov.cuh"

namespace {
__global__ void eval_kernel(int fn, const double* __restrict__ x, const double* __restrict__ y,
                            double* __restrict__ out, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double r;
    switch (fn) {
        case 0: r = hydro::trcp(x[i]); break;
        case 1: r = hydro::root7(x[i]); break;
        case 2: r = hydro::tdiv(x[i], y[i]); break;
        default: r = hydro::trsqrt(x[i]); break;
    }
    out[i] = r;
}
}  // namespace

// fn: 0 trcp(x), 1 root7(x), 2 tdiv(x, y), 3 trsqrt(x); device arrays of n
// doubles (y used by fn 2 only).  Returns 0, or the CUDA error code.
extern "C" int math_probe_eval(int fn, const double* x, const double* y, double* out, long long n) {
    if (n <= 0) return 0;
    const int tb = 256;
    const long long nb = (n + tb - 1) / tb;
    eval_kernel<<<(unsigned)nb, tb>>>(fn, x, y, out, n);
    const cudaError_t e = cudaDeviceSynchronize();
    return (int)e;
}
