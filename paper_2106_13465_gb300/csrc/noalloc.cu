// noalloc.cu -- hydro_conservation_noalloc: the domain totals of a state the
// caller already holds on the device, computed without allocating anything.
//
// Who needs this: callers that must not allocate device memory while they
// run -- code that records work into a CUDA graph or stream capture (where
// cudaMalloc/cudaFree are not allowed), host loops with hard latency limits
// (cudaMalloc and cudaFree can synchronise the whole device), and plugins
// that live inside a host framework owning all GPU memory through its own
// allocator.  Such callers cannot create a hydro_ctx (it owns its buffers), so
// this entry point works on caller-owned input and output pointers only.
//
// The two-stage reduction needs per-row partial sums.  They live in a
// file-scope __device__ array of fixed size (kNoallocMaxRows rows x 4
// planes of doubles, 1 MiB), which every GPU that loads the library keeps
// until the process exits.  Host code cannot use the array's name as a device
// address (in host code it names a host-side stand-in), so the first call on
// each device looks the address up with cudaGetSymbolAddress while that
// device is current, and later calls on the device reuse it.
#include <cuda_runtime.h>

#include <mutex>

#include "hydro.h"
#include "kernels.h"

#define HYDRO_NOALLOC_MAX_ROWS 32768

// row sums of the reduction: [4][HYDRO_NOALLOC_MAX_ROWS] doubles (1 MiB)
static __device__ __align__(256) double g_noalloc_rows[4 * HYDRO_NOALLOC_MAX_ROWS];

namespace {

constexpr int kNoallocMaxRows = HYDRO_NOALLOC_MAX_ROWS;
constexpr int kMaxDevices = 64;

std::mutex g_mu;
double* g_rows_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
hydro_status scratch_on_current_device(double** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HYDRO_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_rows_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_rows);
        if (e != cudaSuccess || !p) return HYDRO_ECUDA;
        g_rows_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_rows_ptr[dev];
    return HYDRO_OK;
}

}  // namespace

extern "C" {

hydro_status hydro_conservation_noalloc(const double* U, int nx, int ny, double h, double* sums,
                                        void* cuda_stream) {
    if (!U || !sums || nx < 1 || ny < 1 || !(h > 0.0)) return HYDRO_EINVAL;
    if (ny > kNoallocMaxRows) return HYDRO_EINVAL;  // beyond the fixed scratch array
    double* rows = nullptr;
    hydro_status st = scratch_on_current_device(&rows);
    if (st != HYDRO_OK) return st;
    // the caller's array: 4 planes of ny rows of nx cells, no padding
    hydro::GridDesc g{};
    g.off = 0;
    g.plane = (long long)nx * ny;
    g.nx = nx;
    g.ny = ny;
    g.pitch = nx;
    g.h = h;
    const cudaError_t e = hydro::launch_conservation<double>(U, g, rows, sums, (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? HYDRO_OK : HYDRO_ECUDA;
}

}  // extern "C"
