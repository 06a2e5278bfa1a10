// fused_tma.cuh -- one kernel per time step: both 1D sweeps of a step (§1;
// the READ, COMPUTE and WRITE steps of Fig. 5 for the x and the y lines of a
// tile) on a tile held in shared memory, so the state crosses HBM once per
// step instead of once per sweep.  Included by the FP64 and FP32
// translation units next to the split sweep kernels (sweep_tma.cuh), whose
// per-cell arithmetic it shares, so the results are bit-identical to theirs.
//
// Tile (kernels.h): the 60 columns [60 k - 2, 60 k + 58) of x segment k times
// up to kFusedRows rows [y0, y0 + rows).  Its input box -- the segment's 64
// columns [60 k - 4, 60 k + 60) times rows [y0 - 2, y0 + rows + 2), all four
// planes -- arrives by one TMA copy (one elected thread, one mbarrier, a
// bounded wait).  On a periodic axis the box cells just outside the grid are
// then filled with the wrap-around cells; on a reflective or transmissive
// axis a boundary position reads its mirror cell, which always lies in the
// box.  Order 0 (x then y):
//   1. every needed box row is swept along x (a warp per row, lane l on
//      cells 2l and 2l+1 as in the split x sweep) and its 60 results are
//      written back into the box row in place;
//   2. the tile's 60 columns are swept along y (a lane per column walking
//      the box column, as in the split y sweep) straight to the other state
//      buffer.
// Order 1 (y then x): every needed box column is swept along y in place
// (the two row halves of a column are walked by different warps, so each
// walker first reads the two positions before and after its own rows, which
// the neighbouring walker overwrites), then the tile's rows are swept along
// x to the other buffer.  A barrier separates the two sweeps.  The halo rows
// (order 0) or columns (order 1) are swept by every tile that holds them:
// the price of one HBM pass per step is that extra arithmetic (4 rows per
// 32, or 4 columns per 60).
//
// As in the split sweeps: the FP32 main pass queues a tile holding a
// near-vacuum interface for the second pass (which recomputes the whole tile
// with those interfaces in FP64); the CFL wave speed of the new state is
// folded in (FP32 exact, FP64 an FP32 estimate per tile for the exact pass
// over the tiles near the maximum); every wait is bounded.  The uniform-
// stencil shortcuts of the split FP64 sweeps are not taken here (they
// change no result, only the time on mostly uniform states).
#pragma once
#include "sweep_tma.cuh"

namespace hydro {

// Position k of a line of n cells -> the line position whose box cell holds
// its state, and whether its normal momentum flips.  Positions before -2 or
// after n+1 (they feed no result) take position -2 or n+1.  Reflective /
// transmissive: the mirror cell; periodic: the position itself (the box
// holds the wrap-around cell there, fill_periodic).
struct BoxPos {
    int k;
    bool flip;
};
__device__ __forceinline__ BoxPos box_pos(int k, int n, int bclo, int bchi) {
    k = k < -2 ? -2 : (k > n + 1 ? n + 1 : k);
    if (k < 0) return (bclo == BC_PERIODIC) ? BoxPos{k, false} : BoxPos{-1 - k, bclo == BC_REFLECT};
    if (k >= n) return (bchi == BC_PERIODIC) ? BoxPos{k, false} : BoxPos{2 * n - 1 - k, bchi == BC_REFLECT};
    return BoxPos{k, false};
}

constexpr int kBoxPlane = kFusedBoxRows * kXSegment;  // elements per plane of the box

// State of box cell (row r, column c) with the normal momentum of direction DIR.
template <class T, int DIR>
__device__ __forceinline__ Cons<T> box_get(const T* box, int r, int c) {
    constexpr int PN = (DIR == DIR_X) ? 1 : 2, PT = 3 - PN;
    const T* p = box + r * kXSegment + c;
    return Cons<T>{p[0], p[PN * kBoxPlane], p[PT * kBoxPlane], p[3 * kBoxPlane]};
}
template <class T, int DIR>
__device__ __forceinline__ void box_put(T* box, int r, int c, const Cons<T>& u) {
    constexpr int PN = (DIR == DIR_X) ? 1 : 2, PT = 3 - PN;
    T* p = box + r * kXSegment + c;
    p[0] = u.r;
    p[PN * kBoxPlane] = u.mn;
    p[PT * kBoxPlane] = u.mt;
    p[3 * kBoxPlane] = u.E;
}

// Periodic axes: the box cells whose grid position lies within two cells
// outside the grid along a periodic axis get the wrap-around cell from src
// (corners of two periodic axes wrap both coordinates; a corner outside a
// mirror axis is never read).  Tiles away from the grid's edges return at once.
template <class T>
__device__ __forceinline__ void fill_periodic(T* box, const T* __restrict__ src, const GridDesc& g, int bx, int by) {
    const bool px = g.bc[0] == BC_PERIODIC, py = g.bc[2] == BC_PERIODIC;
    const bool edge = bx < 0 || bx + kXSegment > g.nx || by < 0 || by + kFusedBoxRows > g.ny;
    if (!edge || (!px && !py)) return;
    for (int i = threadIdx.x; i < kBoxPlane; i += blockDim.x) {
        const int r = i / kXSegment, c = i - r * kXSegment;
        int x = bx + c, y = by + r;
        const bool ox = x < 0 || x >= g.nx, oy = y < 0 || y >= g.ny;
        if (!ox && !oy) continue;
        if (ox) {
            if (!px || x < -2 || x > g.nx + 1) continue;
            x = x < 0 ? x + g.nx : x - g.nx;
        }
        if (oy) {
            if (!py || y < -2 || y > g.ny + 1) continue;
            y = y < 0 ? y + g.ny : y - g.ny;
        }
        const T* s = src + g.off + (long long)y * g.pitch + x;
#pragma unroll
        for (int q = 0; q < 4; ++q) box[q * kBoxPlane + i] = s[q * g.plane];
    }
}

// Per-tile bookkeeping of a thread.
template <class T>
struct FusedAcc {
    unsigned tbad = 0;   // status bits of the tile's new cells
    bool redo = false;   // FP32 main pass: a near-vacuum interface met
    T smax = T(0);       // FP32: max CFL speed of the new state
    unsigned sbits = 0;  // FP64: max FP32 estimate of it (float bits)
};

// Sweep box row r (grid row y) along x, the lanes mapped on the segment as
// in the split x sweep (XMap).  OUT_GLOBAL: to the destination buffer (the
// second sweep, with the CFL speed), else in place into the box.
template <class T, int VAR, bool SV, bool OUT_GLOBAL>
__device__ __forceinline__ void fused_x_row(const SweepArgs<T>& a, T* box, int r, int y, const GridDesc& g, int bx,
                                            T dtdx, T hdtdx, int lane, FusedAcc<T>& acc, unsigned& nfb) {
    const int n = g.nx;
    const int P0 = XMap<T>::pos(lane, 0), P1 = XMap<T>::pos(lane, 1);
    Cons<T> uA, uB;
    if (bx >= 0 && bx + kXSegment <= n) {
        uA = box_get<T, DIR_X>(box, r, P0);
        uB = box_get<T, DIR_X>(box, r, P1);
    } else {
        const BoxPos pa = box_pos(bx + P0, n, g.bc[0], g.bc[1]), pb = box_pos(bx + P1, n, g.bc[0], g.bc[1]);
        uA = flip(box_get<T, DIR_X>(box, r, pa.k - bx), pa.flip);
        uB = flip(box_get<T, DIR_X>(box, r, pb.k - bx), pb.flip);
    }
    __syncwarp();  // every lane has read before any writes back in place
    bool r0 = false, r1 = false;
    Cons<T> nA, nB;
    segment_update<T, VAR, SV>(a, dtdx, hdtdx, lane, uA, uB, nA, nB, r0, r1, nfb);
    acc.redo |= segment_redo<T>(lane, bx, n, r0, r1);
    const bool v0 = seg_result(P0, bx, n), v1 = seg_result(P1, bx, n);
    if (OUT_GLOBAL) {
        store_seg<T>(a.dst + g.off + (long long)y * g.pitch, g.plane, lane, bx, v0, v1, nA, nB);
        if (v0) check_cell<T, 1>(a.K, nA, acc.tbad, acc.smax, acc.sbits);
        if (v1) check_cell<T, 1>(a.K, nB, acc.tbad, acc.smax, acc.sbits);
    } else {
        if (v0) {
            box_put<T, DIR_X>(box, r, P0, nA);
            check_cell<T, 0>(a.K, nA, acc.tbad, acc.smax, acc.sbits);
        }
        if (v1) {
            box_put<T, DIR_X>(box, r, P1, nB);
            check_cell<T, 0>(a.K, nB, acc.tbad, acc.smax, acc.sbits);
        }
    }
}

// Sweep box column c (grid column x) along y over the rows [s0, s1): a walk
// from position s0 - 2 to s1 + 1 with the window of the split y sweep.  The
// two positions before s0 and after s1 are read first, then the CTA-wide
// barrier (every thread calls this once per sweep), since the walker of the
// neighbouring rows may overwrite them in place.  `active`: the column is
// swept (else the thread only joins the barrier).
template <class T, int VAR, bool SV, bool OUT_GLOBAL>
__device__ __forceinline__ void fused_y_col(const SweepArgs<T>& a, T* box, int c, int x, const GridDesc& g, int by,
                                            int s0, int s1, bool active, T dtdx, T hdtdx, FusedAcc<T>& acc,
                                            unsigned& nfb) {
    const Consts<T>& K = a.K;
    const int n = g.ny, bclo = g.bc[2], bchi = g.bc[3];
    active = active && s0 < s1;
    auto cell = [&](int k) {
        const BoxPos p = box_pos(k, n, bclo, bchi);
        return flip(box_get<T, DIR_Y>(box, p.k - by, c), p.flip);
    };
    Cons<T> lead0{}, lead1{}, trail0{}, trail1{};
    if (active) {
        lead0 = cell(s0 - 2);
        lead1 = cell(s0 - 1);
        trail0 = cell(s1);
        trail1 = cell(s1 + 1);
    }
    __syncthreads();
    if (!active) return;
    YWalk<T> w = {};
    w.u0 = lead0;
    w.u1 = lead1;
    w.w1 = cons_to_prim(K, lead1, w.ir1);
    w.dl = pdiff(w.w1, cons_to_prim(K, lead0));
    T* __restrict__ q0 = a.dst + g.off + x;
    unsigned wk = 0;
#pragma unroll 1
    for (int k = s0; k <= s1 + 1; ++k) {
        const Cons<T> u = (k == s1) ? trail0 : ((k == s1 + 1) ? trail1 : cell(k));
        T ir2;
        const Prim<T> w2 = cons_to_prim(K, u, ir2);
        Prim<T> wl1, wr1;
        const Prim<T> dr = pdiff(w2, w.w1);
        trace<T, SV>(K, hdtdx, w.w1, w.ir1, w.dl, dr, wl1, wr1);  // cell k - 1
        if (k == s0) w.wr0 = wl1;  // the face left of cell s0-1 is not formed: a throw-away problem
        bool rd = false;
        const Cons<T> fhi = FluxOp<T, VAR, SV>::eval(a, w.wr0, wl1, rd, nfb, wk);  // (k-1) - 1/2
        if (k >= s0 + 1) acc.redo |= rd;
        if (k >= s0 + 2) {
            const Cons<T> out = update(w.u0, dtdx, fhi, w.flo);  // row k - 2
            if (OUT_GLOBAL) {
                const long long o = (long long)(k - 2) * g.pitch;
                q0[o] = out.r;
                q0[o + 2 * g.plane] = out.mn;
                q0[o + g.plane] = out.mt;
                q0[o + 3 * g.plane] = out.E;
                check_cell<T, 1>(K, out, acc.tbad, acc.smax, acc.sbits);
            } else {
                box_put<T, DIR_Y>(box, k - 2 - by, c, out);
                check_cell<T, 0>(K, out, acc.tbad, acc.smax, acc.sbits);
            }
        }
        w.flo = fhi;
        w.u0 = w.u1;
        w.dl = dr;
        w.wr0 = wr1;
        w.u1 = u;
        w.w1 = w2;
        w.ir1 = ir2;
    }
}

template <class T, int VAR>
struct FusedMinBlocks { static constexpr int value = 1; };
template <> struct FusedMinBlocks<float, VAR_F32_MAIN> { static constexpr int value = 5; };
template <> struct FusedMinBlocks<double, VAR_F64> { static constexpr int value = 3; };

template <class T, int VAR, int ORDER, bool SV>
__global__ void __launch_bounds__(kFusedThreads, (FusedMinBlocks<T, VAR>::value))
    fused_step_kernel(const SweepArgs<T> a) {
    constexpr int NW = kFusedThreads / 32;
    static_assert(NW == 4, "the y sweep of a tile is four walkers (two column groups x two row halves)");
    extern __shared__ __align__(128) unsigned char smem[];
    T* box = reinterpret_cast<T*>(smem);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + fused_box_bytes<T>());
    __shared__ int s_tile;
    __shared__ unsigned s_sbits;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();

    const unsigned accslot = a.ctr->acc;
    unsigned parity = 0, kbad = 0, nfb = 0;
    bool aborted = false;
    for (;;) {
        if (threadIdx.x == 0) {
            int t = -1;
            if (VAR == VAR_F32_REDO) {
                const unsigned i = atomicAdd(&a.ctr->redo_claim[0], 1u);
                if (i < a.ctr->redo_count[0]) t = a.redo_list[i];
            } else {
                const unsigned i = atomicAdd(&a.ctr->tile_ctr[0], 1u);
                if (i < (unsigned)a.ntiles) t = (int)i;
            }
            s_tile = t;
            s_sbits = 0u;
        }
        __syncthreads();
        const int t = s_tile;
        if (t < 0) break;
        const Tile tile = a.tiles[t];
        const GridDesc g = a.grids[tile.grid];
        const int y0 = tile.cell0, rows = tile.ncell;
        const int bx = kXStride * tile.line0 - 4, by = y0 - 2;
        bool bad = tile.grid < 0 || tile.grid >= a.ngrids || rows < 1 || rows > kFusedRows || y0 < 0 ||
                   y0 + rows > g.ny || tile.line0 < 0 || bx + 2 >= g.nx;
        if (bad) {  // never produced by the host
            kbad |= STATUS_BAD_TILE;
            __syncthreads();
            continue;
        }
        if (threadIdx.x == 0) {
            // the previous tile's in-place writes (generic proxy) come before
            // this copy (async proxy) into the same bytes
            fence_proxy_async_smem();
            mbar_expect_tx(bar, fused_box_bytes<T>());
            tma_load_3d(box, a.maps + map_index(tile.grid, a.src_buf, DIR_FUSED), bx, by, 0, bar);
        }
        const bool ok = mbar_wait_bounded(bar, parity, a.wait_limit);
        if (!__syncthreads_and(ok)) {
            aborted = true;
            if (threadIdx.x == 0) {
                record_wait_site(a.ctr, VAR == VAR_F32_REDO ? 4 : 3, t);
                mbar_wait_bounded(bar, parity);  // the copy still in flight
            }
            break;
        }
        parity ^= 1u;
        fill_periodic<T>(box, a.src, g, bx, by);
        __syncthreads();

        const double dt = a.run[tile.grid].dt;
        const T dtdx = T(dt / g.h);
        const T hdtdx = T(-0.5) * dtdx;
        FusedAcc<T> acc;
        // the y walkers: column group (warp & 1), row half (warp >> 1)
        const int half = (rows + 1) / 2;
        const int ys0 = y0 + (warp >> 1) * half, ys1 = (warp >> 1) ? y0 + rows : y0 + half;
        if (ORDER == 0) {
            // 1. x along the box rows the y sweep reads: in-grid rows, and the
            //    wrap-around rows of a periodic y axis
            for (int r = warp; r < rows + 4; r += NW) {
                const int y = by + r;
                const bool need = (y >= 0 && y < g.ny) || (g.bc[2] == BC_PERIODIC && y >= -2 && y <= g.ny + 1);
                if (need) fused_x_row<T, VAR, SV, false>(a, box, r, y, g, bx, dtdx, hdtdx, lane, acc, nfb);
            }
            __syncthreads();
            // 2. y along the tile's columns (box columns 2 .. 61), to dst
            const int c = 2 + 32 * (warp & 1) + lane;
            const int x = bx + c;
            fused_y_col<T, VAR, SV, true>(a, box, c, x, g, by, ys0, ys1, c < 62 && x >= 0 && x < g.nx, dtdx, hdtdx,
                                      acc, nfb);
        } else {
            // 1. y along the box columns the x sweep reads, in place
            const int c = 32 * (warp & 1) + lane;
            const int x = bx + c;
            const bool need = (x >= 0 && x < g.nx) || (g.bc[0] == BC_PERIODIC && x >= -2 && x <= g.nx + 1);
            fused_y_col<T, VAR, SV, false>(a, box, c, x, g, by, ys0, ys1, need, dtdx, hdtdx, acc, nfb);
            __syncthreads();
            // 2. x along the tile's rows (box rows 2 .. rows+1), to dst
            for (int r = 2 + warp; r < rows + 2; r += NW)
                fused_x_row<T, VAR, SV, true>(a, box, r, by + r, g, bx, dtdx, hdtdx, lane, acc, nfb);
        }

        // end of the tile (the barrier also keeps the box until every thread is done)
        const bool redo = (VAR == VAR_F32_MAIN) && __syncthreads_or(acc.redo);
        if (VAR != VAR_F32_MAIN) __syncthreads();
        if (redo) {
            if (threadIdx.x == 0) {
                const unsigned i = atomicAdd(&a.ctr->redo_count[0], 1u);
                a.redo_list[i] = t;
            }
            continue;
        }
        kbad |= acc.tbad;
        if constexpr (sizeof(T) == 8) {
            const unsigned m = __reduce_max_sync(0xffffffffu, acc.sbits);
            if (lane == 0 && m) atomicMax(&s_sbits, m);
            __syncthreads();
            if (threadIdx.x == 0) {
                a.tile_smax[t] = s_sbits;
                // (the maximum only grows: most tiles skip the atomic)
                if (s_sbits && s_sbits > __ldcg(&a.run[tile.grid].smax32)) atomicMax(&a.run[tile.grid].smax32, s_sbits);
            }
        } else {
            double m = (double)acc.smax;
            for (int o = 16; o > 0; o >>= 1) {
                const double v = __shfl_xor_sync(0xffffffffu, m, o);
                m = (v <= m) ? m : v;
            }
            const unsigned long long mb = (unsigned long long)__double_as_longlong(m);
            if (lane == 0 && mb > __ldcg(&a.run[tile.grid].wmax[accslot]))
                atomicMax(&a.run[tile.grid].wmax[accslot], mb);
        }
    }

    if (aborted && threadIdx.x == 0) atomicOr(&a.ctr->status, STATUS_TIMEOUT);
    for (int o = 16; o > 0; o >>= 1) {
        nfb += __shfl_xor_sync(0xffffffffu, nfb, o);
        kbad |= __shfl_xor_sync(0xffffffffu, kbad, o);
    }
    if (lane == 0) {
        if (kbad) atomicOr(&a.ctr->status, kbad);
        if (nfb) atomicAdd(&a.ctr->riemann_fp64, (unsigned long long)nfb);
    }
}

template <class T, int VAR>
cudaError_t launch_fused_var(int order, const SweepArgs<T>& a, int nctas, cudaStream_t s) {
    constexpr int smem = fused_smem_bytes<T>();
    const bool sv = scheme_variant(a.K);
    if (order == 0) {
        if (sv) fused_step_kernel<T, VAR, 0, true><<<nctas, kFusedThreads, smem, s>>>(a);
        else fused_step_kernel<T, VAR, 0, false><<<nctas, kFusedThreads, smem, s>>>(a);
    } else {
        if (sv) fused_step_kernel<T, VAR, 1, true><<<nctas, kFusedThreads, smem, s>>>(a);
        else fused_step_kernel<T, VAR, 1, false><<<nctas, kFusedThreads, smem, s>>>(a);
    }
    return cudaGetLastError();
}

template <class T, int VAR>
int fused_occupancy() {
    constexpr int smem = fused_smem_bytes<T>();
    int best = 1 << 30;
    for (auto fn : {fused_step_kernel<T, VAR, 0, false>, fused_step_kernel<T, VAR, 1, false>,
                    fused_step_kernel<T, VAR, 0, true>, fused_step_kernel<T, VAR, 1, true>}) {
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 0;
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kFusedThreads, smem) != cudaSuccess) return 0;
        best = nb < best ? nb : best;
    }
    return best;
}

}  // namespace hydro
