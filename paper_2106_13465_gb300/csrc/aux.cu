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
        run[g].smax32 = 0u;
        if (dt_log) dt_log[g] = dt;
    }
    for (int i = threadIdx.x; i < kMaxSmIds; i += blockDim.x) {
        ctr->sm_slot[0][i] = 0u;
        ctr->sm_slot[1][i] = 0u;
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
        ctr->wtiles[0][0] = 0u;
        ctr->wtiles[0][1] = 0u;
        ctr->wtiles[1][0] = 0u;
        ctr->wtiles[1][1] = 0u;
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

// ---- adaptive walk tiles (FP64 x and y) ------------------------------------
// One thread per tile of the static tiling (the tiling the scheduling model
// picks for uniform cost; every tile a whole number of cost blocks except at
// the end of a line).  The thread walks the tile's blocks in order and
// starts a new piece before block b when adding b would take the piece's
// recorded work above `cap` (a piece always gets at least one block), so
// uniform work reproduces the static tiling and the tiles where the solver
// works harder are split.  Pieces of at least `big` work are queued first
// (from the front of the list), the others last (from its back): the warps
// start on the long jobs and the short ones fill the tail of the sweep.
// Each warp reserves its threads' slots with one atomic per class.  The
// previous step's sweep in the same direction recorded the work and its
// total (in the slot of its step parity); this kernel clears the slot the
// coming sweep fills.  A piece starts on a cost block (of blk cells).
template <bool EMIT>
__device__ __forceinline__ void split_tile(const Tile& st, const float* __restrict__ cst, int blk, float cap,
                                           float big, Tile* __restrict__ out, int cap_tiles, unsigned& nf,
                                           unsigned& nb) {
    const int b0 = st.cell0 / blk, b1 = (st.cell0 + st.ncell + blk - 1) / blk;
    const int rend = st.cell0 + st.ncell;
    float acc = 0.0f;
    int start = b0;
    auto put = [&](int r0, int nrows, float work) {
        if (work >= big) {
            if (EMIT) out[nf] = Tile{st.grid, st.line0, r0, nrows};
            ++nf;
        } else {
            if (EMIT) out[cap_tiles - 1 - (int)nb] = Tile{st.grid, st.line0, r0, nrows};
            ++nb;
        }
    };
    for (int b = b0; b < b1; ++b) {
        const float c = cst[b];
        if (b > start && acc + c > cap) {
            put(start * blk, (b - start) * blk, acc);
            acc = 0.0f;
            start = b;
        }
        acc += c;
    }
    put(start * blk, rend - start * blk, acc);
}

__device__ __forceinline__ unsigned warp_exclusive_scan(unsigned v, int lane, unsigned& total) {
    unsigned incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    total = __shfl_sync(0xffffffffu, incl, 31);
    return incl - v;
}

__global__ void retile_kernel(int dir, const GridDesc* __restrict__ grids, const Tile* __restrict__ stat,
                              int nstat, const float* __restrict__ wcost, DevCounters* ctr,
                              Tile* __restrict__ tiles, int cap_tiles, double cap_per_total,
                              double big_per_total, double big_of_max) {
    const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int lane = threadIdx.x & 31;
    const unsigned par = (unsigned)(ctr->steps & 1ull);
    const double total = (double)ctr->wcost_total[dir][par ^ 1u];
    const double bmax = big_of_max * (double)ctr->wcost_max[dir][par ^ 1u];
    if (i == 0) {
        ctr->wcost_total[dir][par] = 0ull;
        ctr->wcost_max[dir][par] = 0u;
    }
    const float cap = (float)(total * cap_per_total);
    const float big = (float)fmax(total * big_per_total, bmax);
    Tile st{};
    const float* cst = nullptr;
    unsigned nf = 0, nb = 0;
    if (i < nstat) {
        st = stat[i];
        const GridDesc& g = grids[st.grid];
        cst = wcost + g.wblk[dir] + (long long)(st.line0 / kWarpLines) * g.wnb[dir];
        split_tile<false>(st, cst, walk_block(dir), cap, big, tiles, cap_tiles, nf, nb);
    }
    // warp-aggregated reservation of the pieces' slots, one atomic per class
    unsigned tf, tb;
    const unsigned of = warp_exclusive_scan(nf, lane, tf), ob = warp_exclusive_scan(nb, lane, tb);
    unsigned basef = 0, baseb = 0;
    if (lane == 0) {
        basef = atomicAdd(&ctr->wtiles[dir][0], tf);
        baseb = atomicAdd(&ctr->wtiles[dir][1], tb);
    }
    basef = __shfl_sync(0xffffffffu, basef, 0) + of;
    baseb = __shfl_sync(0xffffffffu, baseb, 0) + ob;
    if (i < nstat) split_tile<true>(st, cst, walk_block(dir), cap, big, tiles, cap_tiles, basef, baseb);
}

cudaError_t launch_retile(int dir, const GridDesc* grids, const Tile* stat, int nstat, const float* wcost,
                          DevCounters* ctr, Tile* tiles, int cap_tiles, double cap_per_total,
                          double big_per_total, double big_of_max, cudaStream_t s) {
    const int threads = 128;
    const int blocks = (nstat + threads - 1) / threads;
    retile_kernel<<<blocks, threads, 0, s>>>(dir, grids, stat, nstat, wcost, ctr, tiles, cap_tiles, cap_per_total,
                                             big_per_total, big_of_max);
    return cudaGetLastError();
}

// ---- CFL speed of a loaded state ------------------------------------------
__global__ void cfl_zero_kernel(GridRun* run, int grid, const DevCounters* ctr) {
    run[grid].wmax[ctr->acc] = 0ull;
    run[grid].smax32 = 0u;
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
    // FP64: an FP32 screen, then the exact speed near its maximum only
    if constexpr (sizeof(T) == 8) return launch_cfl_screened_fp64(state, gd, grid, run, ctr, K, s);
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
