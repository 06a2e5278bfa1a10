// sweep_tma.cuh -- the fused 1D Godunov sweep kernel (§1; the READ, COMPUTE
// and WRITE steps of Fig. 5 fused into one pass over HBM), included by the
// FP64 and FP32 translation units.
//
// Work decomposition.  A persistent grid of CTAs whose warps claim tasks from
// a work counter, so one launch covers any number of grids of any shapes.
//   x sweep, FP32 (sweep_x_kernel): a task is a run of overlapping 64-cell
//            segments of one row (segment k starts at x = -4 + 60 k); lane l
//            holds cells 2l and 2l+1 of the segment and takes its
//            neighbours' primitives, faces and fluxes by warp shuffles;
//            lanes 1..30 hold the 60 results.
//   line walks (sweep_walk_kernel): a task (tile) is 32 lines x L cells;
//            lane l walks line line0 + l from cell0 - 2 to cell0 + L + 1 (the
//            5-point stencil of Figs. 1-2) with a window of the last two
//            conserved states, the last primitives and their one-sided
//            difference, the right face of the previous cell and the flux
//            at the previous interface in registers.  y sweep (both
//            precisions): the lines are columns.  x sweep (FP64): the lines
//            are rows.  FP64 tiles are cut every step from the work the
//            previous sweep in their direction recorded (adaptive tiles).
// In all, every interface is solved once per task and every cell written
// once.
//
// Data movement.  Each warp owns a ring of shared-memory slots fed by TMA
// (cp.async.bulk.tensor, one elected lane, completion on an mbarrier per
// slot).  x segments: a slot holds one segment (64 cells x 4 planes); lane l
// reads its two cells with one 8- or 16-byte load per plane, and the warp
// writes its 60 results as consecutive cells of each plane.  y walk: a slot
// holds 4 rows x 32 columns x 4 planes; lane l reads column l (consecutive
// words) and a warp writes 32 consecutive cells per plane.  x walk: a slot
// holds 4 columns x 32 rows x 4 planes; the warp collects its outputs in a
// staging block of the same shape and writes it by a TMA store.  The ring is
// refilled as slots are consumed, so several are in flight while the warp
// computes.
//
// Boundary conditions are folded into the read: a position k outside [0, n)
// of a line takes the mirror cell (reflective: normal momentum negated;
// transmissive) or the wrap-around cell (periodic).  Mirror cells come by
// shuffle from the same x segment, or from a walk's first chunk and its
// register window; wrap-around cells with a direct load.  TMA reads
// outside the grid are zero-filled and feed no result.
//
// Every wait on an mbarrier is bounded: after SweepArgs::wait_limit polls
// (kWaitLimit unless a caller lowered it to exercise this path) the warp
// records STATUS_TIMEOUT, waits -- bounded by kWaitLimit -- for its own copies
// still in flight and leaves the kernel.
#pragma once
#include "kernels.h"

namespace hydro {

// --------------------------------------------------------------- PTX ------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// At most `limit` polls and about kWaitNs nanoseconds (a poll may suspend
// the thread for a while), whichever comes first.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, unsigned limit = kWaitLimit) {
    if (limit && mbar_try_wait(bar, parity)) return true;  // the usual case: no timer read
    const unsigned long long t0 = global_ns();
    for (unsigned it = 0; it < limit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 63u && global_ns() - t0 > kWaitNs) return false;
    }
    return false;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, int x, int y, int z, const void* src) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(map),
                 "r"(x), "r"(y), "r"(z), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
template <int N>
__device__ __forceinline__ void bulk_wait() {
    asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// --------------------------------------------------------- interface flux --
// SV: the scheme variants of a.K are read (else the defaults are compiled in).
template <class T, int VAR, bool SV>
struct FluxOp;

template <bool SV>
struct FluxOp<double, VAR_F64, SV> {
    static __device__ __forceinline__ Cons<double> eval(const SweepArgs<double>& a, const Prim<double>& L,
                                                        const Prim<double>& R, bool& redo, unsigned& nfb,
                                                        unsigned& work) {
        (void)redo; (void)nfb;
        return godunov_flux_exact<double, SV>(a.K, L, R, nullptr, &work);
    }
};

// The FP32 criterion for an FP64 solve (near vacuum): min(pL,pR) < 1e-6
// max(pL,pR), the FP32 iterate reached the pressure floor, or
// p* < 1e-3 min(pL,pR) (strong double rarefaction).
__device__ __forceinline__ bool near_vacuum_f32(const Prim<float>& L, const Prim<float>& R,
                                                const Star<float>& s) {
    const float pmn = fminf(L.p, R.p), pmx = fmaxf(L.p, R.p);
    return pmn < 1e-6f * pmx || s.floored || s.p < 1e-3f * pmn;
}

// FP32 main pass: the FP32 solve; a near-vacuum interface marks its tile for
// the second pass (its provisional result is overwritten there).
template <bool SV>
struct FluxOp<float, VAR_F32_MAIN, SV> {
    static __device__ __forceinline__ Cons<float> eval(const SweepArgs<float>& a, const Prim<float>& L,
                                                       const Prim<float>& R, bool& redo, unsigned& nfb,
                                                       unsigned& work) {
        (void)nfb; (void)work;
        if (Shortcuts<float>::flux && same_bits(L, R)) return equal_state_flux(a.K, L);  // no solve, no FP64
        const Side<float> SL = make_side(a.K, L), SR = make_side(a.K, R);
        const Star<float> s = riemann_star<float, SV>(a.K, SL, SR);
        if (near_vacuum_f32(L, R, s)) redo = true;
        return physical_flux(a.K, sample0(a.K, SL, SR, s));
    }
};

__device__ __noinline__ Cons<double> flux_fp64_near_vacuum(const Consts<double>* Kd, Prim<double> L,
                                                           Prim<double> R);

// FP32 second pass: the same FP32 solve, and the FP64 solve where the
// near-vacuum criterion holds.
template <bool SV>
struct FluxOp<float, VAR_F32_REDO, SV> {
    static __device__ __forceinline__ Cons<float> eval(const SweepArgs<float>& a, const Prim<float>& L,
                                                       const Prim<float>& R, bool& redo, unsigned& nfb,
                                                       unsigned& work) {
        (void)redo; (void)work;
        if (Shortcuts<float>::flux && same_bits(L, R)) return equal_state_flux(a.K, L);
        const Side<float> SL = make_side(a.K, L), SR = make_side(a.K, R);
        const Star<float> s = riemann_star<float, SV>(a.K, SL, SR);
        if (near_vacuum_f32(L, R, s)) {
            ++nfb;
            const Prim<double> Ld = {L.r, L.u, L.v, L.p}, Rd = {R.r, R.u, R.v, R.p};
            const Cons<double> F = flux_fp64_near_vacuum(&a.Kd, Ld, Rd);
            return Cons<float>{(float)F.r, (float)F.mn, (float)F.mt, (float)F.E};
        }
        return physical_flux(a.K, sample0(a.K, SL, SR, s));
    }
};


// ------------------------------------------------------------ helpers -----
// Mirror image of a state about a reflective wall: the normal momentum is
// negated as 0 - m, which equals -m except that a zero momentum stays +0.  A
// gas at rest then mirrors to bitwise the same state, so the equal-state and
// uniform-stencil shortcuts hold across the wall (with -m the +-0 pair forces
// a full Riemann solve at every wall interface, whose result only differs in
// the sign of zeros).
__device__ __forceinline__ double neg0(double m) { return __dsub_rn(0.0, m); }
__device__ __forceinline__ float neg0(float m) { return __fsub_rn(0.0f, m); }
template <class T>
__device__ __forceinline__ Cons<T> flip(Cons<T> u, bool f) {
    if (f) u.mn = neg0(u.mn);
    return u;
}

// Cell k of a line straight from global memory (boundary cells, span halos).
template <class T, int DIR>
__device__ __forceinline__ Cons<T> global_cell(const T* __restrict__ base, const GridDesc& g, int line, int k) {
    constexpr int PN = (DIR == DIR_X) ? 1 : 2, PT = 3 - PN;
    const long long o = g.off + ((DIR == DIR_X) ? (long long)line * g.pitch + k : (long long)k * g.pitch + line);
    Cons<T> u;
    u.r = __ldg(base + o);
    u.mn = __ldg(base + o + PN * g.plane);
    u.mt = __ldg(base + o + PT * g.plane);
    u.E = __ldg(base + o + 3 * g.plane);
    return u;
}

// The state at position k of a line of n cells when k is outside [0, n):
// mirror image (reflective: normal momentum negated; transmissive) or
// wrap-around (periodic).
template <class T, int DIR>
__device__ __forceinline__ Cons<T> ghost_cell(const T* __restrict__ base, const GridDesc& g, int line, int k,
                                              int n, int bclo, int bchi) {
    const int bc = (k < 0) ? bclo : bchi;
    if (bc == BC_PERIODIC) return global_cell<T, DIR>(base, g, line, (k < 0) ? k + n : k - n);
    return flip(global_cell<T, DIR>(base, g, line, (k < 0) ? -1 - k : 2 * n - 1 - k), bc == BC_REFLECT);
}

// Per-warp ring of TMA slots with one mbarrier each.
template <int S, int SLOT>
struct WarpRing {
    unsigned char* base;
    uint64_t* bar;
    unsigned parity = 0;   // bit s: parity of the next completion of slot s
    unsigned pending = 0;  // bit s: a load into slot s is in flight (lane 0's view)

    __device__ __forceinline__ void init(unsigned char* smem, int warp, int nwarps, int lane) {
        base = smem + warp * S * SLOT;
        bar = reinterpret_cast<uint64_t*>(smem + nwarps * S * SLOT) + warp * S;
        if (lane == 0) {
            for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
            fence_mbar_init();
        }
        __syncwarp();
    }
    __device__ __forceinline__ unsigned char* slot(int s) const { return base + s * SLOT; }
    // lane 0: load box (x, y, 0) of `map` into slot s
    __device__ __forceinline__ void issue(int s, const CUtensorMap* map, int x, int y) {
        mbar_expect_tx(&bar[s], SLOT);
        tma_load_3d(base + s * SLOT, map, x, y, 0, &bar[s]);
        pending |= 1u << s;
    }
    // all lanes: wait for slot s, at most `limit` polls (the outcome is
    // warp-uniform)
    __device__ __forceinline__ bool wait(int s, int lane, unsigned limit) {
        const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bar[s], (parity >> s) & 1u, limit));
        if (ok) {
            parity ^= 1u << s;
            if (lane == 0) pending &= ~(1u << s);
        }
        return ok;
    }
    // lane 0, after a timeout: wait (at most kWaitLimit polls each) for this
    // warp's copies in flight
    __device__ __forceinline__ void drain() {
        for (int s = 0; s < S; ++s)
            if (pending & (1u << s)) mbar_wait_bounded(&bar[s], (parity >> s) & 1u);
    }
};

// ---- FP32 estimate of the CFL wave speed of an FP64 state ------------------
// FP64 -> FP32 by truncating the significand on the integer pipe (the FP64
// pipe, the sweep's bottleneck, stays free): relative error below 2^-23 for
// values in the FP32 normal range, +-0 below it, +-inf above it and for NaN.
__device__ __forceinline__ float f32_trunc(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32);
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
    if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
    if (e <= 0) return __uint_as_float(sign);
    return __uint_as_float(sign | ((unsigned)e << 23) | (unsigned)((b >> 29) & 0x7fffffu));
}

// FP32 estimate of cfl_speed of an FP64 state, used to find the few cells
// that need the exact FP64 speed.  Its relative error is below 2e-3 for every
// state whose values are finite in FP32: the inputs and the FP32 operations
// round to a few 1e-7, except where the pressure comes from cancellation
// (kinetic energy far above the internal energy); there the absolute error
// of c is at most sqrt(g (g - 1) k eps32) |u| (k ~ 5 roundings), under 1e-3
// of the speed, which the flow speed then dominates.  An infinite or NaN
// estimate (overflow, NaN input) sends every cell of the grid to the exact
// evaluation.
__device__ __forceinline__ float cfl_estimate(const Consts<double>& K, double r, double mn, double mt, double E) {
    const float rfl = K.f_rho_floor, gm1 = K.f_gm1, gam = K.f_gamma, cf2g = K.f_cf2g;
    float rho = f32_trunc(r);
    rho = (rho < rfl) ? rfl : rho;
    const float ir = 1.0f / rho;
    const float u = f32_trunc(mn) * ir, v = f32_trunc(mt) * ir;
    float p = gm1 * (f32_trunc(E) - 0.5f * rho * (u * u + v * v));
    const float pm = rho * cf2g;
    p = (p < pm) ? pm : p;
    const float c = sqrtf(gam * p * ir);
    return fmaxf(fabsf(u), fabsf(v)) + c;
}

// Record the first wait that gave up (kernel site, tile); one thread calls it.
__device__ __forceinline__ void record_wait_site(DevCounters* ctr, int site, int tile) {
    if (atomicCAS(&ctr->wait_site, 0, site) == 0) ctr->wait_tile = tile;
}

// Claim the next tile: the main pass takes the work list in order, the FP32
// second pass takes the tiles the main pass queued.  -1 when none is left.
//
// Adaptive walk tiles (FP64): long jobs from the front of the list, then
// short ones from its back.  The long jobs are the few rows of heavy Riemann
// problems of a sweep, and two of them in one SM sub-partition halve each
// other's FP64 rate, so a warp's first claim spreads them over the SMs: the
// s-th warp to start on SM m takes long job s * nsm + m, if nobody has.  Every long job also stays in the counter's
// order, and a job is taken by whoever first swaps the step count `ep` into
// its claim word, so each is taken exactly once however many warps an SM
// runs.
template <class T, int VAR>
__device__ __forceinline__ int claim_tile(const SweepArgs<T>& a, int lane, bool first = false,
                                          unsigned long long ep = 0) {
    int t = -1;
    if (lane == 0) {
        if (VAR == VAR_F32_REDO) {
            const unsigned i = atomicAdd(&a.ctr->redo_claim[a.which], 1u);
            t = (i < a.ctr->redo_count[a.which]) ? a.redo_list[a.which * a.redo_cap + i] : -1;
        } else if (a.ntiles_dev) {
            const unsigned nf = a.ntiles_dev[0], nb = a.ntiles_dev[1];
            if (first && a.wclaim) {
                unsigned sm;
                asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
                if (sm < (unsigned)kMaxSmIds) {
                    const unsigned long long j =
                        (unsigned long long)atomicAdd(&a.ctr->sm_slot[a.which][sm], 1u) * (unsigned)a.nsm + sm;
                    if (j < nf && atomicExch(&a.wclaim[j], ep) != ep) t = (int)j;
                }
            }
            while (t < 0) {
                const unsigned i = atomicAdd(&a.ctr->tile_ctr[a.which], 1u);
                if (i >= nf + nb) break;
                if (i >= nf) t = a.ntiles - 1 - (int)(i - nf);
                else if (!a.wclaim || atomicExch(&a.wclaim[i], ep) != ep) t = (int)i;
            }
        } else {
            const unsigned i = atomicAdd(&a.ctr->tile_ctr[a.which], 1u);
            t = (i < (unsigned)a.ntiles) ? (int)i : -1;
        }
    }
    return __shfl_sync(0xffffffffu, t, 0);
}

// End of a tile: an FP32 main-pass tile with a near-vacuum interface is queued
// for the second pass (its results there replace these); otherwise its status
// bits and, on the second sweep of a step, its wave-speed maximum are kept.
template <class T, int VAR, int WHICH>
__device__ __forceinline__ void finish_tile(const SweepArgs<T>& a, int t, int grid, unsigned acc, bool redo,
                                            unsigned tbad, T smax, unsigned sbits, unsigned& kbad, int lane) {
    if (VAR == VAR_F32_MAIN && __any_sync(0xffffffffu, redo)) {
        if (lane == 0) {
            const unsigned i = atomicAdd(&a.ctr->redo_count[a.which], 1u);
            a.redo_list[a.which * a.redo_cap + i] = t;
        }
        return;
    }
    kbad |= tbad;
    if (WHICH == 1 && sizeof(T) == 8) {
        // FP64: max of the FP32 speed estimates (bits order as unsigned), per
        // grid and per tile (the CFL pass visits only tiles near the max)
        const unsigned m = __reduce_max_sync(0xffffffffu, sbits);
        if (lane == 0) {
            a.tile_smax[t] = m;
            // (the maximum only grows: most tiles skip the atomic)
            if (m && m > __ldcg(&a.run[grid].smax32)) atomicMax(&a.run[grid].smax32, m);
        }
    }
    if (WHICH == 1 && sizeof(T) == 4) {
        double m = (double)smax;
        for (int o = 16; o > 0; o >>= 1) {
            const double v = __shfl_xor_sync(0xffffffffu, m, o);
            m = (v <= m) ? m : v;
        }
        const unsigned long long mb = (unsigned long long)__double_as_longlong(m);
        if (lane == 0 && mb > __ldcg(&a.run[grid].wmax[acc])) atomicMax(&a.run[grid].wmax[acc], mb);
    }
}

// Work (solve_work units) of a row whose 5-point stencil is uniform: no
// arithmetic at all, the cell is copied.
constexpr unsigned kUniformWork = 4u;

// Bitwise equality of two conserved states.
template <class T>
__device__ __forceinline__ auto diff_bits(const Cons<T>& a, const Cons<T>& b) {
    return diff_bits(a.r, b.r) | diff_bits(a.mn, b.mn) | diff_bits(a.mt, b.mt) | diff_bits(a.E, b.E);
}
template <class T>
__device__ __forceinline__ bool same_bits(const Cons<T>& a, const Cons<T>& b) {
    return diff_bits(a, b) == 0;
}

// Status bits and (second sweep) CFL wave speed of one new cell state.
template <class T, int WHICH>
__device__ __forceinline__ void check_cell(const Consts<T>& K, const Cons<T>& out, unsigned& tbad, T& smax,
                                           unsigned& sbits) {
    tbad |= positive(out.r) ? 0u : STATUS_BAD_RHO;
    tbad |= positive(out.E) ? 0u : STATUS_BAD_E;
    // FP32: the CFL wave speed of the new state (next step's dt) is folded
    // in here.  FP64: only an FP32 estimate here; after the sweep the cells
    // whose estimate is near the grid's maximum get the exact FP64 speed
    // (launch_cfl_fp64), so the FP64 pipe works on a few cells only
    if constexpr (WHICH == 1 && sizeof(T) == 8) {
        const unsigned b = __float_as_uint(cfl_estimate(K, out.r, out.mn, out.mt, out.E));
        sbits = (b > sbits) ? b : sbits;
    }
    if constexpr (WHICH == 1 && sizeof(T) == 4) {
        const T sp = cfl_speed(K, out);
        smax = (sp <= smax) ? smax : sp;
    }
}

template <class T>
__device__ __forceinline__ Cons<T> update(const Cons<T>& u, T dtdx, const Cons<T>& fhi, const Cons<T>& flo) {
    Cons<T> o;
    o.r = tfma(-dtdx, fhi.r - flo.r, u.r);
    o.mn = tfma(-dtdx, fhi.mn - flo.mn, u.mn);
    o.mt = tfma(-dtdx, fhi.mt - flo.mt, u.mt);
    o.E = tfma(-dtdx, fhi.E - flo.E, u.E);
    return o;
}

template <class T, int VAR, int DIR>
struct MinBlocks { static constexpr int value = 1; };
template <> struct MinBlocks<float, VAR_F32_MAIN, DIR_Y> { static constexpr int value = 5; };
template <> struct MinBlocks<float, VAR_F32_MAIN, DIR_X> { static constexpr int value = 7; };
template <> struct MinBlocks<double, VAR_F64, DIR_Y> { static constexpr int value = 3; };
template <> struct MinBlocks<double, VAR_F64, DIR_X> { static constexpr int value = 3; };

// ============================================================ line walker ===
// A lane per line: lane l walks line line0 + l along the cells [s0, s1) of a
// tile, with chunks of 4 cells of 32 lines (positions s0-2+4c .. s0+1+4c)
// arriving by TMA.  Chunk 0 holds the four warm-up positions s0-2 .. s0+1;
// every later chunk holds four positions that each complete one output cell.
// LD = DIR_Y: the lines are columns (the y sweep, both precisions; chunk box
// 32 columns x 4 rows).  LD = DIR_X: the lines are rows (the FP64 x sweep;
// chunk box 4 columns x 32 rows, its x start s0 - 2 + 4c even, as a TMA copy
// of FP64 needs: the tile start s0 is even).  The FP64 x sweep walks rather
// than taking segments (sweep_x_kernel, which FP32 keeps): no cell is
// computed twice (a segment computes 64 cells for 60 results) and each warp
// instruction of the solver serves one interface per lane.
template <class T>
struct YWalk {
    Cons<T> u0, u1;   // conserved states at k-2, k-1
    Prim<T> dl;       // primitives at k-1 minus those at k-2
    Prim<T> w1;       // primitives at k-1
    T ir1;            // 1/rho at k-1
    Prim<T> wr0;      // right face of cell k-2
    Cons<T> flo;      // flux at (k-2) - 1/2
};

// this lane's cell j (position kc + j) of a chunk in shared memory: y, the
// box [plane][4 rows][32 columns] (normal momentum plane 2); x, the box
// [plane][32 rows][4 columns] (normal momentum plane 1)
template <class T, int LD>
__device__ __forceinline__ Cons<T> chunk_cell(const T* sp, int j, int lane) {
    constexpr int C = 4;
    if constexpr (LD == DIR_Y)
        return Cons<T>{sp[(0 * C + j) * 32 + lane], sp[(2 * C + j) * 32 + lane], sp[(1 * C + j) * 32 + lane],
                       sp[(3 * C + j) * 32 + lane]};
    else
        return Cons<T>{sp[(0 * 32 + lane) * C + j], sp[(1 * 32 + lane) * C + j], sp[(2 * 32 + lane) * C + j],
                       sp[(3 * 32 + lane) * C + j]};
}

// Boundary cell at position k (k in {-2, -1, n, n+1}) of a walk.
// Reflective / transmissive: the mirror cells 1, 0 are in the first chunk
// (positions -2..1), the mirror cells n-1, n-2 are the walk's last two
// conserved states (n-2 is saved when position n is formed); periodic: the
// wrap-around cell from global memory.
template <class T, int LD>
__device__ __forceinline__ Cons<T> walk_ghost(const T* __restrict__ src, const GridDesc& g, int line, int k, int n,
                                              int bclo, int bchi, const T* sp, int kc, int lane,
                                              const YWalk<T>& w, Cons<T>& gsave) {
    const int bc = (k < 0) ? bclo : bchi;
    if (bc == BC_PERIODIC) return global_cell<T, LD>(src, g, line, (k < 0) ? k + n : k - n);
    const bool f = (bc == BC_REFLECT);
    if (k < 0) return flip(chunk_cell<T, LD>(sp, -1 - k - kc, lane), f);
    if (k == n) {
        gsave = flip(w.u0, f);
        return flip(w.u1, f);
    }
    return gsave;
}

template <class T, int VAR, int WHICH, bool SV, int LD>
__global__ void __launch_bounds__(kSweepThreads, (MinBlocks<T, VAR, LD>::value))
    sweep_walk_kernel(const SweepArgs<T> a) {
    constexpr int C = 4;
    // x: outputs staged in shared memory and stored by TMA (below)
    constexpr bool kStage = (LD == DIR_X);
    constexpr int S = kStage ? kXWalkSlots : ring_slots(DIR_Y);
    constexpr int SLOT = slot_bytes<T>(DIR_Y);
    constexpr int NWARPS = kSweepThreads / 32;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpRing<S, SLOT> ring;
    ring.init(smem, warp, NWARPS, lane);
    T* const stage = reinterpret_cast<T*>(smem + xwalk_stage_offset<T>() + warp * 2 * SLOT);

    const Consts<T>& K = a.K;
    const unsigned acc = a.ctr->acc;
    // FP64: every tile records its estimated work for the adaptive tiles
    constexpr bool kRecord = (VAR == VAR_F64);
    unsigned kbad = 0, nfb = 0;
    bool aborted = false;
    // step count of this sweep: the claim word of the adaptive tiles
    const unsigned long long ep = a.wclaim ? __ldcg(&a.ctr->steps) : 0ull;
    // recorded work of this warp's tiles (lane 0), added to the sweep's
    // totals once at the end (an atomic per tile on one address serialises)
    unsigned long long wsum = 0ull;
    unsigned wbig = 0u;
    bool first = true;

    for (;;) {
        const int t = claim_tile<T, VAR>(a, lane, first, ep);
        first = false;
        if (t < 0) break;
        unsigned tcost = 0;  // this lane's estimated work on the tile (solve_work units)
        const Tile tile = a.tiles[t];
        if (tile.grid < 0 || tile.grid >= a.ngrids) {
            kbad |= STATUS_BAD_TILE;
            continue;
        }
        const GridDesc g = a.grids[tile.grid];
        const double dt = a.run[tile.grid].dt;
        const int n = (LD == DIR_Y) ? g.ny : g.nx, nlines = (LD == DIR_Y) ? g.nx : g.ny;
        if (tile.cell0 < 0 || tile.ncell < 1 || tile.cell0 + tile.ncell > n || tile.line0 < 0 ||
            tile.line0 >= nlines || (tile.line0 & (kWarpLines - 1)) ||
            (kStage && ((tile.cell0 & 3) || ((tile.ncell & 3) && tile.cell0 + tile.ncell != n)))) {
            kbad |= STATUS_BAD_TILE;  // never produced by the host or the tiler
            continue;
        }
        const int line0 = tile.line0, line = line0 + lane;
        const bool valid = line < nlines;
        const int lsafe = valid ? line : nlines - 1;
        const int bclo = (LD == DIR_Y) ? g.bc[2] : g.bc[0], bchi = (LD == DIR_Y) ? g.bc[3] : g.bc[1];
        const int s0 = tile.cell0, s1 = tile.cell0 + tile.ncell;
        const int kfirst = s0 - 2, klast = s1 + 1;
        // chunk c holds positions kbase + 4c .. kbase + 4c + 3: y from
        // kfirst; x from s0 - 4 (whole 32-byte row pieces, s0 being a
        // multiple of 4), or from 0 at the grid's left end (the ghosts
        // mirror cells of that chunk or wrap around)
        const int kbase = kStage ? ((kfirst < 0) ? 0 : (kfirst & ~3)) : kfirst;
        const int nch = (klast - kbase) / C + 1;
        const CUtensorMap* msrc = a.maps + map_index(tile.grid, a.src_buf, LD);
        const CUtensorMap* mdst = a.maps + map_index(tile.grid, a.src_buf ^ 1, LD);
        auto issue = [&](int c) {
            if (LD == DIR_Y) ring.issue(c % S, msrc, line0, kbase + c * C);
            else ring.issue(c % S, msrc, kbase + c * C, line0);
        };
        if (lane == 0)
            for (int c = 0; c < S && c < nch; ++c) issue(c);

        const T dtdx = T(dt / g.h);
        const T hdtdx = T(-0.5) * dtdx;
        // this lane's line in the four output planes (normal momentum is
        // plane 2 for y, 1 for x), cell k at offset k * kstride; a plane
        // holds fewer than 2^31 elements (checked on the host)
        T* __restrict__ q0 = a.dst + g.off + ((LD == DIR_Y) ? (long long)lsafe : (long long)lsafe * g.pitch);
        T* __restrict__ qn = q0 + ((LD == DIR_Y) ? 2 : 1) * g.plane;
        T* __restrict__ qt = q0 + ((LD == DIR_Y) ? 1 : 2) * g.plane;
        T* __restrict__ qe = q0 + 3 * g.plane;
        const unsigned pitch = (LD == DIR_Y) ? (unsigned)g.pitch : 1u;
        // Output cell q (warp-uniform) of this lane's line.  y: stored at
        // once (a warp writes 32 consecutive cells).  x: a lane's cells are
        // a row apart, so the warp collects 4 consecutive cells of its 32
        // rows in a staging block (the layout of a chunk slot) and stores
        // the block by TMA when it is full or holds the row's last cell;
        // each block [s0 + 4b, s0 + 4b + 4) lies in the tile (or is clipped
        // at the grid's right end and its last row), and a block's buffer
        // is reused only after the store issued from it has read it.
        auto emit = [&](int q, const Cons<T>& out) {
            if constexpr (kStage) {
                const int b = (q - s0) >> 2, col = (q - s0) & 3;
                T* st = stage + (b & 1) * (SLOT / (int)sizeof(T));
                st[(0 * 32 + lane) * C + col] = out.r;
                st[(1 * 32 + lane) * C + col] = out.mn;
                st[(2 * 32 + lane) * C + col] = out.mt;
                st[(3 * 32 + lane) * C + col] = out.E;
                if (col == 3 || q == s1 - 1) {
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        tma_store_3d(mdst, s0 + 4 * b, line0, 0, st);
                        bulk_commit();
                        bulk_wait_read<1>();  // the other block's buffer is free again
                    }
                    __syncwarp();
                }
            } else if (valid) {
                const unsigned o = (unsigned)q * pitch;
                q0[o] = out.r;
                qn[o] = out.mn;
                qt[o] = out.mt;
                qe[o] = out.E;
            }
        };
        YWalk<T> w = {};
        Cons<T> gsave = {};  // mirror of row n-2, kept for position n+1
        int run = 1;         // positions ending at the current one with equal conserved bits
        bool copied = false; // the previous row was a copy (uniform stencil)
        T smax = T(0);
        unsigned sbits = 0;  // FP64: max FP32 speed estimate (float bits)
        unsigned tbad = 0;
        bool redo = false;

        for (int c = 0; c < nch; ++c) {
            const int sl = c % S;
            if (!ring.wait(sl, lane, a.wait_limit)) {
                aborted = true;
                if (lane == 0) record_wait_site(a.ctr, LD == DIR_Y ? 2 : 1, t);
                break;
            }
            const T* sp = reinterpret_cast<const T*>(ring.slot(sl));
            const int kc = kbase + c * C;
            int j0 = 0;
            if (c == 0) {
                // positions s0-2 and s0-1 only fill the window (both < n - 1;
                // below 0 they mirror cells of this chunk or wrap around);
                // jf = kfirst - kbase is 0 (y), 2 (x) or -2 (x, s0 = 0)
                const int jf = kStage ? kfirst - kbase : 0;
                Cons<T> u = (jf >= 0) ? chunk_cell<T, LD>(sp, jf, lane) : Cons<T>{};
                if (kfirst < 0) u = walk_ghost<T, LD>(a.src, g, lsafe, kfirst, n, bclo, bchi, sp, kc, lane, w, gsave);
                w.u0 = u;
                const Prim<T> w0 = cons_to_prim(K, u);
                u = (jf >= 0) ? chunk_cell<T, LD>(sp, jf + 1, lane) : Cons<T>{};
                if (kfirst + 1 < 0)
                    u = walk_ghost<T, LD>(a.src, g, lsafe, kfirst + 1, n, bclo, bchi, sp, kc, lane, w, gsave);
                w.u1 = u;
                w.w1 = cons_to_prim(K, u, w.ir1);
                w.dl = pdiff(w.w1, w0);
                run = (Shortcuts<T>::stencil && same_bits(w.u1, w.u0)) ? 2 : 1;
                j0 = jf + 2;
            } else if (Shortcuts<T>::stencil && kc + C - 1 <= klast && kc + C - 1 < n &&
                       __all_sync(0xffffffffu, !valid || copied)) {
                // the previous row was a copy, so the window is the fixed
                // point of a uniform column (u0 = u1, w0 = w1 = wr0, flux
                // flo): if the chunk's four cells equal u1 bit for bit, the
                // per-position steps below would copy u0 to rows kc-2 ..
                // kc+1, leave the window as it is and count no status or
                // speed -- do exactly that, for the whole warp at once
                unsigned long long dif = 0;
#pragma unroll
                for (int j = 0; j < C; ++j) dif |= (unsigned long long)diff_bits(chunk_cell<T, LD>(sp, j, lane), w.u1);
                if (__all_sync(0xffffffffu, !valid || dif == 0)) {
                    // (kc >= s0 + 3 here: a copy needs positions >= s0 + 2)
                    for (int j = 0; j < C; ++j) emit(kc + j - 2, w.u0);
                    run += C;
                    if (kRecord) tcost += C * kUniformWork;
                    j0 = C;
                }
            }
            // one copy of the per-cell arithmetic: position k completes the
            // trace of cell k-1, the flux at (k-1)-1/2 and (from k = s0+2 on)
            // the update of row k-2
            #pragma unroll 1
            for (int j = j0; j < C; ++j) {
                const int k = kc + j;
                if (k > klast) break;
                Cons<T> u = chunk_cell<T, LD>(sp, j, lane);
                if (k >= n) u = walk_ghost<T, LD>(a.src, g, lsafe, k, n, bclo, bchi, sp, kc, lane, w, gsave);
                const bool same = Shortcuts<T>::stencil && same_bits(u, w.u1);
                run = same ? run + 1 : 1;
                // rows k-4..k equal bit for bit: the traces of k-3..k-1 return
                // the cell, both interfaces of row k-2 are equal-state problems
                // of that one state, so their fluxes are equal (fhi = flo) and
                // the update returns row k-2 unchanged
                const bool uniform = run >= 5 && k >= s0 + 2;
                unsigned wk = kUniformWork;
                T ir2;
                Prim<T> w2, wr1, dr;
                Cons<T> fhi;
                if (!uniform) {
                    if (same) {  // the same conserved bits give the same primitives
                        w2 = w.w1;
                        ir2 = w.ir1;
                    } else {
                        w2 = cons_to_prim(K, u, ir2);
                    }
                    dr = pdiff(w2, w.w1);
                    Prim<T> wl1;
                    trace<T, SV>(K, hdtdx, w.w1, w.ir1, w.dl, dr, wl1, wr1);  // cell k - 1
                    // at k = s0 the face left of cell s0-1 is not formed: solve
                    // a trivial problem (equal states) whose flux is never used
                    if (k == s0) w.wr0 = wl1;
                    fhi = FluxOp<T, VAR, SV>::eval(a, w.wr0, wl1, redo, nfb, wk);
                }
                if (kRecord) tcost += wk;
                if (uniform) {  // the window rotates equal states (their
                                // difference is +0, as computed for finite states)
                    w2 = w.w1;
                    ir2 = w.ir1;
                    wr1 = w.w1;
                    dr = Prim<T>{T(0), T(0), T(0), T(0)};
                    fhi = w.flo;
                }
                if (k >= s0 + 2) {
                    Cons<T> out = w.u0;
                    if (!uniform) out = update(w.u0, dtdx, fhi, w.flo);
                    emit(k - 2, out);
                    // a copy equal to the previous row's copy has its status
                    // and wave speed already counted
                    if (valid && !(uniform && copied)) check_cell<T, WHICH>(K, out, tbad, smax, sbits);
                }
                copied = uniform;
                w.flo = fhi;
                w.u0 = w.u1;
                w.dl = dr;
                w.wr0 = wr1;
                w.u1 = u;
                w.w1 = w2;
                w.ir1 = ir2;
            }
            __syncwarp();
            if (lane == 0 && c + S < nch) {
                fence_proxy_async_smem();
                issue(c + S);
            }
        }
        if constexpr (kStage) {
            // the staging blocks are read before the next tile writes them
            if (lane == 0) bulk_wait_read<0>();
            __syncwarp();
        }
        if (aborted) break;
        // the tile's work is that of its busiest lane (one reduction per
        // tile: a reduction per row measured 13 % more FP64 instructions)
        if (kRecord) tcost = __reduce_max_sync(0xffffffffu, tcost);
        if (kRecord && a.wcost && lane == 0) {
            // the tile's work, spread evenly over its cost blocks (the tile
            // and grid fields are read again here rather than kept in
            // registers through the walk)
            const int4 tt = __ldcg(reinterpret_cast<const int4*>(a.tiles + t));  // grid, line0, cell0, ncell
            const long long wblk = __ldcg(&a.grids[tt.x].wblk[LD]);
            const int wnb = __ldcg(&a.grids[tt.x].wnb[LD]);
            constexpr int B = walk_block(LD);
            const int b0 = tt.z / B, b1 = (tt.z + tt.w - 1) / B;
            const float dens = (float)tcost / (float)(b1 - b0 + 1);
            float* cst = a.wcost + wblk + (long long)(tt.y / kWarpLines) * wnb;
            for (int b = b0; b <= b1; ++b) cst[b] = dens;
            wsum += tcost;
            wbig = tcost > wbig ? tcost : wbig;
        }
        finish_tile<T, VAR, WHICH>(a, t, tile.grid, acc, redo && valid, tbad, smax, sbits, kbad, lane);
    }

    if (aborted && lane == 0) {
        atomicOr(&a.ctr->status, STATUS_TIMEOUT);
        ring.drain();
    }
    if constexpr (kStage) {
        if (lane == 0) bulk_wait<0>();  // this warp's stores have completed
    }
    if (kRecord && a.wcost && lane == 0 && wsum) {
        const unsigned par = (unsigned)(__ldcg(&a.ctr->steps) & 1ull);
        atomicAdd(&a.ctr->wcost_total[LD][par], wsum);
        atomicMax(&a.ctr->wcost_max[LD][par], wbig);
    }
    for (int o = 16; o > 0; o >>= 1) {
        nfb += __shfl_xor_sync(0xffffffffu, nfb, o);
        kbad |= __shfl_xor_sync(0xffffffffu, kbad, o);
    }
    if (lane == 0) {
        if (kbad) atomicOr(&a.ctr->status, kbad);
        if (nfb) atomicAdd(&a.ctr->riemann_fp64, (unsigned long long)nfb);
    }
}

// =================================================================== x ===
// Lines are rows.  A row is covered by overlapping 64-cell segments that
// start at x = -4 + 60 k (TMA box 64 cells x 1 row x 4 planes; the start is
// 16-byte aligned for FP32 and FP64) and each produce the 60 cells
// [60 k - 2, 60 k + 58).  Lane l holds cells A = x + 2l and B = A + 1.  From
// lane l-1 it takes the primitives of A-1 and the right face of A-1, from
// lane l+1 the primitives of B+1 and the flux at B+1/2; it traces A and B,
// solves the interfaces A-1/2 and A+1/2 and updates A and B.  Lanes 1..30
// hold the 60 results (lanes 0 and 31 only feed their neighbours), so a
// segment needs nothing from the previous one and a warp writes 60
// consecutive cells per plane.  A warp task is a run of consecutive segments
// of one row: (grid, line0 = row, cell0 = first segment, ncell = segments).
template <class T>
__device__ __forceinline__ Prim<T> shfl_up1(const Prim<T>& v) {
    return Prim<T>{__shfl_up_sync(0xffffffffu, v.r, 1), __shfl_up_sync(0xffffffffu, v.u, 1),
                   __shfl_up_sync(0xffffffffu, v.v, 1), __shfl_up_sync(0xffffffffu, v.p, 1)};
}
template <class T>
__device__ __forceinline__ Prim<T> shfl_down1(const Prim<T>& v) {
    return Prim<T>{__shfl_down_sync(0xffffffffu, v.r, 1), __shfl_down_sync(0xffffffffu, v.u, 1),
                   __shfl_down_sync(0xffffffffu, v.v, 1), __shfl_down_sync(0xffffffffu, v.p, 1)};
}
template <class T>
__device__ __forceinline__ Cons<T> shfl_idx(const Cons<T>& v, int src) {
    return Cons<T>{__shfl_sync(0xffffffffu, v.r, src), __shfl_sync(0xffffffffu, v.mn, src),
                   __shfl_sync(0xffffffffu, v.mt, src), __shfl_sync(0xffffffffu, v.E, src)};
}
template <class T>
__device__ __forceinline__ Cons<T> shfl_down1(const Cons<T>& v) {
    return Cons<T>{__shfl_down_sync(0xffffffffu, v.r, 1), __shfl_down_sync(0xffffffffu, v.mn, 1),
                   __shfl_down_sync(0xffffffffu, v.mt, 1), __shfl_down_sync(0xffffffffu, v.E, 1)};
}

// two consecutive cells (j, j+1) of every plane of a ring slot (x layout [q][64])
template <class T>
__device__ __forceinline__ void read_pair(const unsigned char* slot, int j, Cons<T>& c0, Cons<T>& c1) {
    constexpr int PB = kXSegment * (int)sizeof(T);
    T v[4][2];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (sizeof(T) == 4) {
            const float2 f = *reinterpret_cast<const float2*>(slot + q * PB + j * sizeof(T));
            v[q][0] = (T)f.x; v[q][1] = (T)f.y;
        } else {
            const double2 f = *reinterpret_cast<const double2*>(slot + q * PB + j * sizeof(T));
            v[q][0] = (T)f.x; v[q][1] = (T)f.y;
        }
    }
    c0 = Cons<T>{v[0][0], v[1][0], v[2][0], v[3][0]};
    c1 = Cons<T>{v[0][1], v[1][1], v[2][1], v[3][1]};
}

template <class T>
__device__ __forceinline__ void store_pair(T* __restrict__ p, long long plane, const Cons<T>& a, const Cons<T>& b,
                                           bool lo, bool hi) {
    const T va[4] = {a.r, a.mn, a.mt, a.E}, vb[4] = {b.r, b.mn, b.mt, b.E};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        T* d = p + q * plane;
        if (lo && hi) {
            if (sizeof(T) == 4) *reinterpret_cast<float2*>(d) = make_float2((float)va[q], (float)vb[q]);
            else *reinterpret_cast<double2*>(d) = make_double2((double)va[q], (double)vb[q]);
        } else if (lo) {
            d[0] = va[q];
        }
    }
}

// Lane mapping of a 64-cell x segment: lane l holds the cells at segment
// positions pos(l, 0) = 2l and pos(l, 1) = 2l+1.  The results are the
// positions 2 .. 61 (the others only feed them); every interface is solved
// once.  (A mapping of lane l to positions l and l+32, which gives each
// Riemann solve of a warp 32 consecutive interfaces instead of every other
// one of 64, was measured 6-7 % slower in FP64 and is not used.)
template <class T>
struct XMap {
    static __device__ __forceinline__ int pos(int lane, int j) { return 2 * lane + j; }
    static __device__ __forceinline__ int lane_of(int p) { return p >> 1; }
    static __device__ __forceinline__ int cell_of(int p) { return p & 1; }
};

// The arithmetic of one segment: lane l holds the conserved states u0, u1 of
// its cells A = 2l and B = 2l+1 (ghosts already in place) and returns their
// updated states n0, n1 (meaningful at positions 2 .. 61) and the
// second-pass requests of its two Riemann problems A-1/2 (r0) and A+1/2
// (r1).  It takes the primitives of A-1 and the right face of A-1 from lane
// l-1, the primitives of B+1 and the flux at B+1/2 from lane l+1.  Lanes 0
// and 31 have no left / right neighbour in the segment and hold no result;
// they mirror their own cells so their throw-away Riemann problems stay
// mild and do not stretch the warp's Newton loop.
template <class T, int VAR, bool SV>
__device__ __forceinline__ void segment_update(const SweepArgs<T>& a, T dtdx, T hdtdx, int lane,
                                               const Cons<T>& u0, const Cons<T>& u1, Cons<T>& n0,
                                               Cons<T>& n1, bool& r0, bool& r1, unsigned& nfb) {
    const Consts<T>& K = a.K;
    unsigned wk = 0;  // scheduling work estimate, unused in x
    T ir0, ir1;
    const Prim<T> W0 = cons_to_prim(K, u0, ir0);
    const Prim<T> W1 = cons_to_prim(K, u1, ir1);
    Prim<T> Wm = shfl_up1(W1);    // cell A-1
    Prim<T> Wp = shfl_down1(W0);  // cell B+1
    if (lane == 0) Wm = W0;
    if (lane == 31) Wp = W1;
    Prim<T> WLA, WRA, WLB, WRB;
    const Prim<T> dAB = pdiff(W1, W0);  // right difference of A, left of B
    trace<T, SV>(K, hdtdx, W0, ir0, pdiff(W0, Wm), dAB, WLA, WRA);  // cell A
    trace<T, SV>(K, hdtdx, W1, ir1, dAB, pdiff(Wp, W1), WLB, WRB);  // cell B
    Prim<T> WRm = shfl_up1(WRB);  // right face of A-1
    if (lane == 0) WRm = WLA;
    const Cons<T> Fm = FluxOp<T, VAR, SV>::eval(a, WRm, WLA, r0, nfb, wk);  // A - 1/2
    const Cons<T> Fc = FluxOp<T, VAR, SV>::eval(a, WRA, WLB, r1, nfb, wk);  // A + 1/2
    const Cons<T> Fp = shfl_down1(Fm);                                 // B + 1/2
    n0 = update(u0, dtdx, Fc, Fm);
    n1 = update(u1, dtdx, Fp, Fc);
}

// A cell at segment position p of the segment starting at x is a result
// stored in a row of n cells.
__device__ __forceinline__ bool seg_result(int p, int x, int n) {
    return p >= 2 && p <= kXSegment - 3 && x + p >= 0 && x + p < n;
}

// Whether a lane's second-pass requests r0, r1 (segment_update) concern an
// interface next to a stored result (every lane calls it: it shuffles).
template <class T>
__device__ __forceinline__ bool segment_redo(int lane, int x, int n, bool r0, bool r1) {
    // A-1/2 and A+1/2 feed A and B; B+1/2 (lane l+1's r0) feeds B
    const bool lo = seg_result(2 * lane, x, n), hi = seg_result(2 * lane + 1, x, n);
    const bool r0n = __shfl_down_sync(0xffffffffu, r0, 1);
    return ((r0 || r1) && lo) || (r0n && lo && hi);
}

// The lane's two cells from a segment laid out [plane][64] (ring slot).
template <class T>
__device__ __forceinline__ void read_seg(const unsigned char* slot, int lane, Cons<T>& u0, Cons<T>& u1) {
    read_pair<T>(slot, 2 * lane, u0, u1);
}

// Store the lane's stored results (row pointer drow, segment start x).
template <class T>
__device__ __forceinline__ void store_seg(T* __restrict__ drow, long long plane, int lane, int x, bool v0, bool v1,
                                          const Cons<T>& n0, const Cons<T>& n1) {
    if (v0) store_pair<T>(drow + x + 2 * lane, plane, n0, n1, v0, v1);
}

template <class T, int VAR, int WHICH, bool SV>
__global__ void __launch_bounds__(kSweepThreads, (MinBlocks<T, VAR, DIR_X>::value))
    sweep_x_kernel(const SweepArgs<T> a) {
    constexpr int SEG = kXSegment, STEP = kXStride;
    constexpr int S = ring_slots(DIR_X);
    constexpr int SLOT = slot_bytes<T>(DIR_X);
    constexpr int NWARPS = kSweepThreads / 32;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpRing<S, SLOT> ring;
    ring.init(smem, warp, NWARPS, lane);

    const Consts<T>& K = a.K;
    const unsigned acc = a.ctr->acc;
    unsigned kbad = 0, nfb = 0;
    bool aborted = false;

    for (;;) {
        const int t = claim_tile<T, VAR>(a, lane);
        if (t < 0) break;
        const Tile tile = a.tiles[t];
        const GridDesc g = a.grids[tile.grid];
        const double dt = a.run[tile.grid].dt;
        const int n = g.nx, row = tile.line0;
        const int k0 = tile.cell0, nseg = tile.ncell;
        const int bclo = g.bc[0], bchi = g.bc[1];
        const CUtensorMap* msrc = a.maps + map_index(tile.grid, a.src_buf, DIR_X);
        if (lane == 0)
            for (int c = 0; c < S && c < nseg; ++c) ring.issue(c, msrc, -4 + STEP * (k0 + c), row);

        const T dtdx = T(dt / g.h);
        const T hdtdx = T(-0.5) * dtdx;
        T* __restrict__ drow = a.dst + g.off + (long long)row * g.pitch;
        T smax = T(0);
        unsigned sbits = 0;  // FP64: max FP32 speed estimate (float bits)
        unsigned tbad = 0;
        bool redo = false;

        for (int c = 0; c < nseg; ++c) {
            const int x = -4 + STEP * (k0 + c);
            const int sl = c % S;
            if (!ring.wait(sl, lane, a.wait_limit)) {
                aborted = true;
                if (lane == 0) record_wait_site(a.ctr, 1, t);
                break;
            }
            const int P0 = XMap<T>::pos(lane, 0), P1 = XMap<T>::pos(lane, 1);
            Cons<T> uA, uB;  // the cells at positions P0, P1
            read_seg<T>(ring.slot(sl), lane, uA, uB);
            __syncwarp();
            if (lane == 0 && c + S < nseg) {
                fence_proxy_async_smem();
                ring.issue(sl, msrc, -4 + STEP * (k0 + c + S), row);
            }
            if (x < 0 || x + SEG > n) {
                // positions -2, -1 and n, n+1 are boundary cells.  Reflective /
                // transmissive: the mirror cells 1, 0 or n-1, n-2 lie in this
                // segment, so they come by shuffle; periodic: the wrap-around
                // cells come from global memory.
                const int kA = x + P0, kB = x + P1;
                const bool gA = (kA >= -2 && kA < 0) || (kA >= n && kA <= n + 1);
                const bool gB = (kB >= -2 && kB < 0) || (kB >= n && kB <= n + 1);
                const int bcA = (kA < 0) ? bclo : bchi, bcB = (kB < 0) ? bclo : bchi;
                const bool mA = gA && bcA != BC_PERIODIC, mB = gB && bcB != BC_PERIODIC;
                const int sA = mA ? ((kA < 0) ? -1 - kA : 2 * n - 1 - kA) - x : P0;
                const int sB = mB ? ((kB < 0) ? -1 - kB : 2 * n - 1 - kB) - x : P1;
                const int lA = XMap<T>::lane_of(sA), lB = XMap<T>::lane_of(sB);
                const Cons<T> a0 = shfl_idx(uA, lA), a1 = shfl_idx(uB, lA);
                const Cons<T> b0 = shfl_idx(uA, lB), b1 = shfl_idx(uB, lB);
                if (mA) uA = flip(XMap<T>::cell_of(sA) ? a1 : a0, bcA == BC_REFLECT);
                else if (gA) uA = ghost_cell<T, DIR_X>(a.src, g, row, kA, n, bclo, bchi);
                if (mB) uB = flip(XMap<T>::cell_of(sB) ? b1 : b0, bcB == BC_REFLECT);
                else if (gB) uB = ghost_cell<T, DIR_X>(a.src, g, row, kB, n, bclo, bchi);
                // positions beyond the boundary cells (zero-filled) take a copy
                // of the nearest boundary cell: they feed no result, and equal
                // states keep their throw-away Riemann problems trivial
                const int lo2 = -2 - x, hi2 = n + 1 - x;  // segment positions of -2, n+1
                const int pl = (lo2 > 0) ? lo2 : 0, ph = (hi2 < SEG - 1) ? hi2 : SEG - 1;
                const Cons<T> cl0 = shfl_idx(uA, XMap<T>::lane_of(pl)), cl1 = shfl_idx(uB, XMap<T>::lane_of(pl));
                const Cons<T> ch0 = shfl_idx(uA, XMap<T>::lane_of(ph)), ch1 = shfl_idx(uB, XMap<T>::lane_of(ph));
                const Cons<T> cl = XMap<T>::cell_of(pl) ? cl1 : cl0, ch = XMap<T>::cell_of(ph) ? ch1 : ch0;
                if (kA < -2) uA = cl;
                if (kB < -2) uB = cl;
                if (kA > n + 1) uA = ch;
                if (kB > n + 1) uB = ch;
            }
            const bool v0 = seg_result(P0, x, n), v1 = seg_result(P1, x, n);
            if (Shortcuts<T>::stencil) {
                // all 64 cells of the segment equal bit for bit (ghosts and
                // fill included): every stencil is uniform, the traces return
                // the cells, all fluxes are equal and each result is its cell
                const Cons<T> ref = shfl_idx(uA, 0);
                if (__all_sync(0xffffffffu, (diff_bits(uA, ref) | diff_bits(uB, ref)) == 0)) {
                    // one status and wave-speed check stands for all the copies
                    const int first = __ffs(__ballot_sync(0xffffffffu, v0 || v1)) - 1;
                    store_seg<T>(drow, g.plane, lane, x, v0, v1, uA, uB);
                    if (lane == first) check_cell<T, WHICH>(K, uA, tbad, smax, sbits);
                    continue;
                }
            }
            bool r0 = false, r1 = false;
            Cons<T> nA, nB;
            segment_update<T, VAR, SV>(a, dtdx, hdtdx, lane, uA, uB, nA, nB, r0, r1, nfb);
            // a second-pass request counts only for interfaces feeding stored cells
            redo |= segment_redo<T>(lane, x, n, r0, r1);
            store_seg<T>(drow, g.plane, lane, x, v0, v1, nA, nB);
            if (v0) check_cell<T, WHICH>(K, nA, tbad, smax, sbits);
            if (v1) check_cell<T, WHICH>(K, nB, tbad, smax, sbits);
        }
        if (aborted) break;
        finish_tile<T, VAR, WHICH>(a, t, tile.grid, acc, redo, tbad, smax, sbits, kbad, lane);
    }

    if (aborted && lane == 0) {
        atomicOr(&a.ctr->status, STATUS_TIMEOUT);
        ring.drain();
    }
    for (int o = 16; o > 0; o >>= 1) {
        nfb += __shfl_xor_sync(0xffffffffu, nfb, o);
        kbad |= __shfl_xor_sync(0xffffffffu, kbad, o);
    }
    if (lane == 0) {
        if (kbad) atomicOr(&a.ctr->status, kbad);
        if (nfb) atomicAdd(&a.ctr->riemann_fp64, (unsigned long long)nfb);
    }
}

// ---------------------------------------------------------------- launch --
// The x sweep walks lines in FP64 and takes segments in FP32.
template <class T>
__host__ __device__ constexpr bool x_walks() { return sizeof(T) == 8; }

template <class T, int VAR, int WHICH, int DIR, bool SV>
struct KernelOf {
    static constexpr auto fn() {
        if constexpr (DIR == DIR_X && !x_walks<T>()) return sweep_x_kernel<T, VAR, WHICH, SV>;
        else return sweep_walk_kernel<T, VAR, WHICH, SV, DIR>;
    }
};

// Dynamic shared memory of a sweep launch (a walker's ring holds chunks).
template <class T, int DIR>
constexpr int launch_smem_bytes() {
    if constexpr (DIR == DIR_X) return x_walks<T>() ? xwalk_smem_bytes<T>() : sweep_smem_bytes<T>(DIR_X);
    return sweep_smem_bytes<T>(DIR_Y);
}

// Whether the constants select a scheme variant (the kernels compiled with
// SV = true read the variant flags; the others have the defaults built in).
template <class T>
bool scheme_variant(const Consts<T>& K) {
    return K.two_shock || K.slope != SLOPE_MINMOD || K.char_trace;
}

// Launch (the dynamic shared-memory limit was raised by occupancy_one, which
// the context calls for every variant it uses before the first launch).
template <class T, int DIR, int VAR>
cudaError_t launch_one(const SweepArgs<T>& a, int nctas, cudaStream_t s) {
    constexpr int smem = launch_smem_bytes<T, DIR>();
    const bool sv = scheme_variant(a.K);
    if (a.which == 0) {
        if (sv) KernelOf<T, VAR, 0, DIR, true>::fn()<<<nctas, kSweepThreads, smem, s>>>(a);
        else KernelOf<T, VAR, 0, DIR, false>::fn()<<<nctas, kSweepThreads, smem, s>>>(a);
    } else {
        if (sv) KernelOf<T, VAR, 1, DIR, true>::fn()<<<nctas, kSweepThreads, smem, s>>>(a);
        else KernelOf<T, VAR, 1, DIR, false>::fn()<<<nctas, kSweepThreads, smem, s>>>(a);
    }
    return cudaGetLastError();
}

// Raise the kernels' dynamic shared-memory limit and return their resident
// CTAs per SM (the smallest over the sweep-order and scheme instances).
template <class T, int DIR, int VAR>
int occupancy_one() {
    constexpr int smem = launch_smem_bytes<T, DIR>();
    int best = 1 << 30;
    for (auto fn : {KernelOf<T, VAR, 0, DIR, false>::fn(), KernelOf<T, VAR, 1, DIR, false>::fn(),
                    KernelOf<T, VAR, 0, DIR, true>::fn(), KernelOf<T, VAR, 1, DIR, true>::fn()}) {
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 0;
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kSweepThreads, smem) != cudaSuccess) return 0;
        best = nb < best ? nb : best;
    }
    return best;
}

}  // namespace hydro
