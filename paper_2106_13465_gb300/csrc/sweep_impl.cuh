// sweep_impl.cuh -- the fused 1D Godunov sweep kernel (§1; Fig. 5 READ /
// COMPUTE / WRITE fused into one pass), included by the FP64 and FP32
// translation units.
//
// Work decomposition: a persistent grid of CTAs whose warps claim warp tiles
// (32 lines x ncell cells of one grid) from a work counter, so one launch
// covers any number of grids of any shapes.  Lane l of a warp owns line
// line0 + l and walks it from cell0 - 2 to cell0 + ncell + 1 keeping a
// 3-cell window of conserved and primitive states, the right face of the
// previous cell and the flux at the previous interface in registers: each
// input cell is read once, each interface solved once (plus one extra solve
// and two extra reads per tile end), each output cell written once.
// Boundary conditions are folded into the read: a ghost index outside
// [0, n) is mapped to its mirror (reflective: normal momentum negated;
// transmissive) or wrap-around (periodic) source cell.
#pragma once
#include "kernels.h"

namespace hydro {

template <class T>
struct FluxOp;

// FP64: the exact solver throughout.
template <>
struct FluxOp<double> {
    static __device__ __forceinline__ Cons<double> eval(const SweepArgs<double>& a,
                                                        const Prim<double>& L,
                                                        const Prim<double>& R, unsigned& nfb) {
        (void)nfb;
        return godunov_flux_exact(a.K, L, R, nullptr);
    }
};

// FP64 solve of one interface for the FP32 path near vacuum (kept out of
// line so the FP32 fast path does not carry its registers).
__device__ __noinline__ Cons<double> flux_fp64_near_vacuum(const Consts<double>* Kd,
                                                           Prim<double> L, Prim<double> R);

// FP32: Newton in FP32; the whole interface is solved again in FP64 when the
// problem is near vacuum: min(pL,pR) < 1e-6 max(pL,pR), the FP32 iterate hit
// the pressure floor, or p* < 1e-3 min(pL,pR) (strong double rarefaction).
template <>
struct FluxOp<float> {
    static __device__ __forceinline__ Cons<float> eval(const SweepArgs<float>& a,
                                                       const Prim<float>& L,
                                                       const Prim<float>& R, unsigned& nfb);
};

template <class T, int DIR>
__device__ __forceinline__ Cons<T> load_cell(const T* __restrict__ line_base, long long stride,
                                             long long plane, int k, int n, int bclo, int bchi) {
    constexpr int PN = (DIR == DIR_X) ? 1 : 2;  // plane of the normal momentum
    constexpr int PT = (DIR == DIR_X) ? 2 : 1;
    int kk = k;
    bool flip = false;
    if (k < 0) {
        if (bclo == BC_PERIODIC) kk = k + n;
        else { kk = -1 - k; flip = (bclo == BC_REFLECT); }
    } else if (k >= n) {
        if (bchi == BC_PERIODIC) kk = k - n;
        else { kk = 2 * n - 1 - k; flip = (bchi == BC_REFLECT); }
    }
    const T* p = line_base + (long long)kk * stride;
    Cons<T> u;
    u.r = __ldg(p);
    u.mn = __ldg(p + PN * plane);
    u.mt = __ldg(p + PT * plane);
    u.E = __ldg(p + 3 * plane);
    if (flip) u.mn = -u.mn;
    return u;
}

template <class T, int DIR>
__global__ void __launch_bounds__(kSweepThreads) sweep_kernel(const SweepArgs<T> a) {
    constexpr int PN = (DIR == DIR_X) ? 1 : 2;
    constexpr int PT = (DIR == DIR_X) ? 2 : 1;
    const int lane = threadIdx.x & 31;
    const unsigned acc = a.ctr->acc;
    const Consts<T>& K = a.K;
    unsigned nfb = 0, bad = 0;

    for (;;) {
        int t = 0;
        if (lane == 0) t = (int)atomicAdd(&a.ctr->tile_ctr[a.which], 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= a.ntiles) break;
        const Tile tile = a.tiles[t];
        const GridDesc g = a.grids[tile.grid];
        const double dt = a.run[tile.grid].dt;

        const int n = (DIR == DIR_X) ? g.nx : g.ny;
        const int nlines = (DIR == DIR_X) ? g.ny : g.nx;
        const int line = tile.line0 + lane;
        const bool valid = line < nlines;
        const int ls = valid ? line : nlines - 1;  // idle lanes re-read a real line
        const long long stride = (DIR == DIR_X) ? 1 : g.pitch;
        const long long lbase = g.off + ((DIR == DIR_X) ? (long long)ls * g.pitch : (long long)ls);
        const T* __restrict__ src = a.src + lbase;
        T* __restrict__ dst = a.dst + lbase;
        const int bclo = (DIR == DIR_X) ? g.bc[0] : g.bc[2];
        const int bchi = (DIR == DIR_X) ? g.bc[1] : g.bc[3];

        const T dtdx = T(dt / g.h);
        const T hdtdx = T(-0.5) * dtdx;
        const int s0 = tile.cell0, s1 = tile.cell0 + tile.ncell;

        // window at i = s0 - 2: u0 = U_i, u1 = U_{i+1}
        Cons<T> u0 = load_cell<T, DIR>(src, stride, g.plane, s0 - 2, n, bclo, bchi);
        Cons<T> u1 = load_cell<T, DIR>(src, stride, g.plane, s0 - 1, n, bclo, bchi);
        T ir1;
        Prim<T> w0 = cons_to_prim(K, u0), w1 = cons_to_prim(K, u1, ir1);
        Prim<T> wr0 = w0;          // right face of cell i (set from i = s0 - 1 on)
        Cons<T> flo = {T(0), T(0), T(0), T(0)};  // flux at i - 1/2
        T smax = T(0);

        for (int i = s0 - 2; i < s1; ++i) {
            const Cons<T> u2 = load_cell<T, DIR>(src, stride, g.plane, i + 2, n, bclo, bchi);
            T ir2;
            const Prim<T> w2 = cons_to_prim(K, u2, ir2);
            Prim<T> wl1, wr1;
            trace(K, hdtdx, w0, w1, ir1, w2, wl1, wr1);     // cell i + 1
            Cons<T> fhi = flo;
            if (i >= s0 - 1) fhi = FluxOp<T>::eval(a, wr0, wl1, nfb);  // interface i + 1/2
            if (i >= s0) {
                Cons<T> out;
                out.r = u0.r - dtdx * (fhi.r - flo.r);
                out.mn = u0.mn - dtdx * (fhi.mn - flo.mn);
                out.mt = u0.mt - dtdx * (fhi.mt - flo.mt);
                out.E = u0.E - dtdx * (fhi.E - flo.E);
                if (valid) {
                    T* d = dst + (long long)i * stride;
                    d[0] = out.r;
                    d[PN * g.plane] = out.mn;
                    d[PT * g.plane] = out.mt;
                    d[3 * g.plane] = out.E;
                    bad |= (out.r > T(0)) ? 0u : STATUS_BAD_RHO;
                    bad |= (out.E > T(0)) ? 0u : STATUS_BAD_E;
                    if (a.which == 1) {
                        // CFL wave speed of the new state (next step's dt)
                        T ir;
                        const Prim<T> w = cons_to_prim(K, out, ir);
                        const T au = tabs(w.u), av = tabs(w.v);
                        const T s = ((au > av) ? au : av) + tsqrt(K.gamma * w.p * ir);
                        smax = (s <= smax) ? smax : s;
                    }
                }
            }
            flo = fhi;
            u0 = u1; u1 = u2;
            w0 = w1; w1 = w2; ir1 = ir2;
            wr0 = wr1;
        }

        if (a.which == 1) {
            double m = (double)smax;
            for (int o = 16; o > 0; o >>= 1) {
                const double v = __shfl_xor_sync(0xffffffffu, m, o);
                m = (v <= m) ? m : v;
            }
            if (lane == 0)
                atomicMax(&a.run[tile.grid].wmax[acc], (unsigned long long)__double_as_longlong(m));
        }
    }

    // flush the per-lane counters once per warp
    for (int o = 16; o > 0; o >>= 1) {
        nfb += __shfl_xor_sync(0xffffffffu, nfb, o);
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if (lane == 0) {
        if (bad) atomicOr(&a.ctr->status, bad);
        if (nfb) atomicAdd(&a.ctr->riemann_fp64, (unsigned long long)nfb);
    }
}

template <class T>
cudaError_t launch_sweep(int dir, const SweepArgs<T>& a, int nctas, cudaStream_t s) {
    if (nctas <= 0) return cudaSuccess;
    if (dir == DIR_X) sweep_kernel<T, DIR_X><<<nctas, kSweepThreads, 0, s>>>(a);
    else sweep_kernel<T, DIR_Y><<<nctas, kSweepThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace hydro
