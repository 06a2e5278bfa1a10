// sweep_tma.cuh -- the fused 1D Godunov sweep kernel (§1; the READ, COMPUTE
// and WRITE steps of Fig. 5 fused into one pass over HBM), included by the
// FP64 and FP32 translation units.
//
// Work decomposition.  A persistent grid of CTAs whose warps claim warp tiles
// (32 lines x ncell cells of one grid) from a work counter, so one launch
// covers any number of grids of any shapes.  Lane l owns line line0 + l and
// walks it from cell cell0 - 2 to cell0 + ncell + 1 (the 5-point stencil of
// Figs. 1-2), keeping a 2-cell window of conserved and primitive states, the
// right face of the previous cell and the flux at the previous interface in
// registers: every interface is solved once, every cell is written once.
//
// Data movement.  Each warp owns a ring of shared-memory slots fed by TMA
// (cp.async.bulk.tensor, one elected lane, completion on an mbarrier per
// slot).  A slot holds one chunk: 32 lines x C cells x 4 planes.
//   x sweep: lines are rows; a chunk is 32 rows x 16 bytes of x per plane
//            (C = 4 FP32 / 2 FP64 cells), 16-byte rows in shared memory, so
//            lane r reads its cells with one 16-byte load per plane (rows r,
//            r+8, r+16, r+24 share banks: 4 wavefronts per 512 bytes, the
//            minimum).  Results are written back in place and the chunk is
//            stored with a TMA tile store: reads and writes both coalesced
//            with no global transpose.
//   y sweep: lines are columns; a chunk is 4 rows x 32 columns per plane;
//            lane l reads column l (consecutive words), and writes its results
//            straight to global memory (a warp writes 32 consecutive cells).
// The ring is refilled as chunks are consumed, so several chunks per warp are
// in flight while the warp computes.
//
// Boundary conditions are folded into the read: a position k outside [0, n)
// of a line takes the mirror cell (reflective: normal momentum negated;
// transmissive) or the wrap-around cell (periodic).  Mirror cells are read
// from the ring or from the register window; wrap-around cells with a direct
// load.  TMA reads outside the grid are zero-filled and never used.
//
// Every wait on an mbarrier is bounded: after kWaitLimit polls the warp
// records STATUS_TIMEOUT, waits (bounded again) for its own copies still in
// flight and leaves the kernel.
#pragma once
#include "kernels.h"

namespace hydro {

constexpr unsigned kWaitLimit = 1u << 22;

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
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
    for (unsigned it = 0; it < kWaitLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
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
template <class T, int VAR>
struct FluxOp;

template <>
struct FluxOp<double, VAR_F64> {
    static __device__ __forceinline__ Cons<double> eval(const SweepArgs<double>& a, const Prim<double>& L,
                                                        const Prim<double>& R, bool& redo, unsigned& nfb) {
        (void)redo; (void)nfb;
        return godunov_flux_exact(a.K, L, R, nullptr);
    }
};

// The FP32 criterion for an FP64 solve (near vacuum): min(pL,pR) < 1e-6
// max(pL,pR), the FP32 iterate reached the pressure floor, or
// p* < 1e-3 min(pL,pR) (strong double rarefaction).
__device__ __forceinline__ bool near_vacuum_f32(const Prim<float>& L, const Prim<float>& R,
                                                const Star<float>& s) {
    const float pmn = (L.p < R.p) ? L.p : R.p;
    const float pmx = (L.p < R.p) ? R.p : L.p;
    return pmn < 1e-6f * pmx || s.floored || s.p < 1e-3f * pmn;
}

// FP32 main pass: the FP32 solve; a near-vacuum interface marks its tile for
// the second pass (its provisional result is overwritten there).
template <>
struct FluxOp<float, VAR_F32_MAIN> {
    static __device__ __forceinline__ Cons<float> eval(const SweepArgs<float>& a, const Prim<float>& L,
                                                       const Prim<float>& R, bool& redo, unsigned& nfb) {
        (void)nfb;
        const Side<float> SL = make_side(a.K, L), SR = make_side(a.K, R);
        const Star<float> s = riemann_star(a.K, SL, SR);
        if (near_vacuum_f32(L, R, s)) redo = true;
        return physical_flux(a.K, sample0(a.K, SL, SR, s));
    }
};

__device__ __noinline__ Cons<double> flux_fp64_near_vacuum(const Consts<double>* Kd, Prim<double> L,
                                                           Prim<double> R);

// FP32 second pass: the same FP32 solve, and the FP64 solve where the
// near-vacuum criterion holds.
template <>
struct FluxOp<float, VAR_F32_REDO> {
    static __device__ __forceinline__ Cons<float> eval(const SweepArgs<float>& a, const Prim<float>& L,
                                                       const Prim<float>& R, bool& redo, unsigned& nfb) {
        (void)redo;
        const Side<float> SL = make_side(a.K, L), SR = make_side(a.K, R);
        const Star<float> s = riemann_star(a.K, SL, SR);
        if (near_vacuum_f32(L, R, s)) {
            ++nfb;
            const Prim<double> Ld = {L.r, L.u, L.v, L.p}, Rd = {R.r, R.u, R.v, R.p};
            const Cons<double> F = flux_fp64_near_vacuum(&a.Kd, Ld, Rd);
            return Cons<float>{(float)F.r, (float)F.mn, (float)F.mt, (float)F.E};
        }
        return physical_flux(a.K, sample0(a.K, SL, SR, s));
    }
};

template <class T, int VAR>
struct MinBlocks { static constexpr int value = 1; };
template <> struct MinBlocks<float, VAR_F32_MAIN> { static constexpr int value = 4; };
template <> struct MinBlocks<double, VAR_F64> { static constexpr int value = 2; };

// ------------------------------------------------------------ helpers -----
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

// this lane's cells of a chunk in shared memory (normal/tangential order)
template <class T, int DIR>
__device__ __forceinline__ void read_chunk(const unsigned char* slot, int lane, Cons<T> (&cell)[chunk_cells<T>(DIR)]) {
    constexpr int C = chunk_cells<T>(DIR);
    constexpr int PB = 32 * C * (int)sizeof(T);  // bytes per plane
    constexpr int PN = (DIR == DIR_X) ? 1 : 2, PT = 3 - PN;
    if (DIR == DIR_X) {
        // one 16-byte row per plane: C consecutive cells of this lane's row
        T v[4][C];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 raw = *reinterpret_cast<const float4*>(slot + q * PB + lane * 16);
            const T* e = reinterpret_cast<const T*>(&raw);
#pragma unroll
            for (int j = 0; j < C; ++j) v[q][j] = e[j];
        }
#pragma unroll
        for (int j = 0; j < C; ++j) cell[j] = Cons<T>{v[0][j], v[PN][j], v[PT][j], v[3][j]};
    } else {
        const T* s = reinterpret_cast<const T*>(slot);
#pragma unroll
        for (int j = 0; j < C; ++j)
            cell[j] = Cons<T>{s[(0 * C + j) * 32 + lane], s[(PN * C + j) * 32 + lane],
                              s[(PT * C + j) * 32 + lane], s[(3 * C + j) * 32 + lane]};
    }
}

// write this lane's result for cell j of a chunk (x sweep, in place)
template <class T>
__device__ __forceinline__ void write_slot_x(unsigned char* slot, int lane, int j, const Cons<T>& u) {
    constexpr int C = chunk_cells<T>(DIR_X);
    constexpr int PB = 32 * C * (int)sizeof(T);
    T* p = reinterpret_cast<T*>(slot + lane * 16) + j;
    *p = u.r;
    *reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(p) + 1 * PB) = u.mn;
    *reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(p) + 2 * PB) = u.mt;
    *reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(p) + 3 * PB) = u.E;
}

template <class T>
__device__ __forceinline__ Cons<T> flip(Cons<T> u, bool f) {
    if (f) u.mn = -u.mn;
    return u;
}

// --------------------------------------------------------------- kernel ---
template <class T, int DIR, int VAR>
__global__ void __launch_bounds__(kSweepThreads, (MinBlocks<T, VAR>::value))
    sweep_kernel(const SweepArgs<T> a) {
    constexpr int C = chunk_cells<T>(DIR);
    constexpr int S = ring_slots(DIR);
    constexpr int SLOT = slot_bytes<T>(DIR);
    constexpr int PN = (DIR == DIR_X) ? 1 : 2, PT = 3 - PN;
    constexpr int SKIP = (DIR == DIR_X && sizeof(T) == 4) ? 2 : 0;  // x FP32: 4-cell aligned halo
    constexpr int NWARPS = kSweepThreads / 32;

    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* ring = smem + warp * S * SLOT;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + NWARPS * S * SLOT) + warp * S;
    if (lane == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncwarp();

    const Consts<T>& K = a.K;
    const unsigned acc = a.ctr->acc;
    unsigned parity = 0;   // bit s: parity of the next completion of slot s
    unsigned pending = 0;  // bit s: a load into slot s is in flight (lane 0's view)
    unsigned kbad = 0, nfb = 0;
    bool aborted = false;

    for (;;) {
        // ---- claim a tile ------------------------------------------------
        int t = 0;
        if (lane == 0) {
            if (VAR == VAR_F32_REDO) {
                const unsigned i = atomicAdd(&a.ctr->redo_claim[a.which], 1u);
                t = (i < a.ctr->redo_count[a.which]) ? a.redo_list[a.which * a.redo_cap + i] : -1;
            } else {
                const unsigned i = atomicAdd(&a.ctr->tile_ctr[a.which], 1u);
                t = (i < (unsigned)a.ntiles) ? (int)i : -1;
            }
        }
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t < 0) break;

        const Tile tile = a.tiles[t];
        const GridDesc g = a.grids[tile.grid];
        const double dt = a.run[tile.grid].dt;
        const int n = (DIR == DIR_X) ? g.nx : g.ny;
        const int nlines = (DIR == DIR_X) ? g.ny : g.nx;
        const int line0 = tile.line0, line = line0 + lane;
        const bool valid = line < nlines;
        const int bclo = (DIR == DIR_X) ? g.bc[0] : g.bc[2];
        const int bchi = (DIR == DIR_X) ? g.bc[1] : g.bc[3];
        const int s0 = tile.cell0, s1 = tile.cell0 + tile.ncell;
        const int kfirst = s0 - 2 - SKIP;  // first position of chunk 0
        const int klast = s1 + 1;          // last position the walk needs
        const int nch = (klast - kfirst) / C + 1;
        const CUtensorMap* msrc = a.maps + ((size_t)tile.grid * 2 + a.src_buf) * 2 + DIR;
        const CUtensorMap* mdst = a.maps + ((size_t)tile.grid * 2 + (a.src_buf ^ 1)) * 2 + DIR;

        auto issue = [&](int c) {  // lane 0
            const int s = c % S;
            mbar_expect_tx(&bar[s], SLOT);
            if (DIR == DIR_X) tma_load_3d(ring + s * SLOT, msrc, kfirst + c * C, line0, 0, &bar[s]);
            else tma_load_3d(ring + s * SLOT, msrc, line0, kfirst + c * C, 0, &bar[s]);
            pending |= 1u << s;
        };
        if (lane == 0)
            for (int c = 0; c < S && c < nch; ++c) issue(c);

        // ---- ghosts at the low end of the line ------------------------------
        Cons<T> gl0 = {T(1), T(0), T(0), T(1)}, gl1 = gl0;  // positions -2, -1
        const int lsafe = valid ? line : nlines - 1;
        if (s0 == 0) {
            if (bclo == BC_PERIODIC) {
                gl0 = global_cell<T, DIR>(a.src, g, lsafe, n - 2);
                gl1 = global_cell<T, DIR>(a.src, g, lsafe, n - 1);
            } else {
                // mirror of cells 1 and 0, which sit in one chunk of the ring
                const int c0 = (0 - kfirst) / C, j0 = (0 - kfirst) % C;
                const int s = c0 % S;
                if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bar[s], (parity >> s) & 1u))) {
                    aborted = true;
                    break;
                }
                Cons<T> cell[C];
                read_chunk<T, DIR>(ring + s * SLOT, lane, cell);
                const bool f = (bclo == BC_REFLECT);
                gl1 = flip(cell[j0], f);
                gl0 = flip(cell[j0 + 1], f);
            }
        }

        // ---- walk ---------------------------------------------------------
        const T dtdx = T(dt / g.h);
        const T hdtdx = T(-0.5) * dtdx;
        const bool fhi_flip = (bchi == BC_REFLECT);
        Cons<T> u0 = gl0, u1 = gl0, grh = gl0;
        Prim<T> w0 = {T(1), T(0), T(0), T(1)}, w1 = w0, wr0 = w0;
        T ir1 = T(1);
        Cons<T> flo = {T(0), T(0), T(0), T(0)};
        T smax = T(0);
        unsigned tbad = 0;
        bool redo = false;

        for (int c = 0; c < nch; ++c) {
            const int s = c % S;
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bar[s], (parity >> s) & 1u))) {
                aborted = true;
                break;
            }
            parity ^= 1u << s;
            if (lane == 0) pending &= ~(1u << s);
            Cons<T> cell[C];
            read_chunk<T, DIR>(ring + s * SLOT, lane, cell);

#pragma unroll
            for (int j = 0; j < C; ++j) {
                const int k = kfirst + c * C + j;
                if (k < s0 - 2 || k > klast) continue;  // warp-uniform
                Cons<T> u = cell[j];
                if (k < 0) {
                    u = (k == -2) ? gl0 : gl1;
                } else if (k >= n) {
                    if (bchi == BC_PERIODIC) {
                        u = global_cell<T, DIR>(a.src, g, lsafe, k - n);
                    } else if (k == n) {
                        u = flip(u1, fhi_flip);      // mirror of cell n-1
                        grh = flip(u0, fhi_flip);    // mirror of cell n-2, for n+1
                    } else {
                        u = grh;
                    }
                }
                if (k == s0 - 2) {
                    u0 = u;
                    w0 = cons_to_prim(K, u);
                } else if (k == s0 - 1) {
                    u1 = u;
                    w1 = cons_to_prim(K, u, ir1);
                } else {
                    T ir2;
                    const Prim<T> w2 = cons_to_prim(K, u, ir2);
                    Prim<T> wl1, wr1;
                    trace(K, hdtdx, w0, w1, ir1, w2, wl1, wr1);  // cell k - 1
                    Cons<T> fhi = flo;
                    if (k >= s0 + 1) fhi = FluxOp<T, VAR>::eval(a, wr0, wl1, redo, nfb);  // k-2 | k-1
                    if (k >= s0 + 2) {
                        // conservative update of cell k - 2
                        Cons<T> out;
                        out.r = u0.r - dtdx * (fhi.r - flo.r);
                        out.mn = u0.mn - dtdx * (fhi.mn - flo.mn);
                        out.mt = u0.mt - dtdx * (fhi.mt - flo.mt);
                        out.E = u0.E - dtdx * (fhi.E - flo.E);
                        const int ko = k - 2;
                        if (DIR == DIR_X) {
                            const int co = (ko - kfirst) / C, jo = (ko - kfirst) % C;
                            write_slot_x<T>(ring + (co % S) * SLOT, lane, jo, out);
                        } else if (valid) {
                            T* d = a.dst + g.off + (long long)ko * g.pitch + line;
                            d[0] = out.r;
                            d[PN * g.plane] = out.mn;
                            d[PT * g.plane] = out.mt;
                            d[3 * g.plane] = out.E;
                        }
                        if (valid) {
                            tbad |= (out.r > T(0)) ? 0u : STATUS_BAD_RHO;
                            tbad |= (out.E > T(0)) ? 0u : STATUS_BAD_E;
                            if (a.which == 1) {
                                // CFL wave speed of the new state (next step's dt)
                                T ir;
                                const Prim<T> w = cons_to_prim(K, out, ir);
                                const T au = tabs(w.u), av = tabs(w.v);
                                const T sp = ((au > av) ? au : av) + tsqrt(K.gamma * w.p * ir);
                                smax = (sp <= smax) ? smax : sp;
                            }
                        }
                    }
                    flo = fhi;
                    u0 = u1; u1 = u;
                    w0 = w1; w1 = w2; ir1 = ir2;
                    wr0 = wr1;
                }
            }
            __syncwarp();

            if (DIR == DIR_X) {
                // chunk c-1 is complete: store it when it holds results
                if (c >= 1) {
                    const int ks = kfirst + (c - 1) * C;
                    if (ks >= s0 && ks < s1) {
                        fence_proxy_async_smem();
                        __syncwarp();
                        if (lane == 0) tma_store_3d(mdst, ks, line0, 0, ring + ((c - 1) % S) * SLOT);
                    }
                }
                if (lane == 0) {
                    bulk_commit();
                    // refill the slot of chunk c-2 once its store has read it
                    const int cr = c - 2 + S;
                    if (c >= 2 && cr < nch) {
                        bulk_wait_read<1>();
                        fence_proxy_async_smem();
                        issue(cr);
                    }
                }
            } else {
                if (lane == 0 && c + S < nch) {
                    fence_proxy_async_smem();
                    issue(c + S);
                }
            }
        }
        if (aborted) break;

        if (DIR == DIR_X) {
            // the last chunk when it holds results (ragged end of a line)
            const int ks = kfirst + (nch - 1) * C;
            if (ks >= s0 && ks < s1) {
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) tma_store_3d(mdst, ks, line0, 0, ring + ((nch - 1) % S) * SLOT);
            }
            if (lane == 0) {
                bulk_commit();
                bulk_wait_read<0>();  // every slot free before the next tile
            }
            __syncwarp();
        }

        // ---- tile epilogue: queue for the FP32 second pass, or publish ----
        if (VAR == VAR_F32_MAIN && __any_sync(0xffffffffu, redo && valid)) {
            if (lane == 0) {
                const unsigned i = atomicAdd(&a.ctr->redo_count[a.which], 1u);
                a.redo_list[a.which * a.redo_cap + i] = t;
            }
        } else {
            kbad |= tbad;
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
    }

    if (aborted) {
        // record the timeout and wait (bounded) for this warp's copies in flight
        if (lane == 0) {
            atomicOr(&a.ctr->status, STATUS_TIMEOUT);
            for (int s = 0; s < S; ++s)
                if (pending & (1u << s)) mbar_wait_bounded(&bar[s], (parity >> s) & 1u);
        }
    }
    if (DIR == DIR_X && lane == 0) bulk_wait<0>();  // results globally visible

    for (int o = 16; o > 0; o >>= 1) {
        nfb += __shfl_xor_sync(0xffffffffu, nfb, o);
        kbad |= __shfl_xor_sync(0xffffffffu, kbad, o);
    }
    if (lane == 0) {
        if (kbad) atomicOr(&a.ctr->status, kbad);
        if (nfb) atomicAdd(&a.ctr->riemann_fp64, (unsigned long long)nfb);
    }
}

// Launch (the dynamic shared-memory limit was raised by occupancy_one, which
// the context calls for every variant it uses before the first launch).
template <class T, int DIR, int VAR>
cudaError_t launch_one(const SweepArgs<T>& a, int nctas, cudaStream_t s) {
    constexpr int smem = sweep_smem_bytes<T>(DIR);
    sweep_kernel<T, DIR, VAR><<<nctas, kSweepThreads, smem, s>>>(a);
    return cudaGetLastError();
}

// Raise the kernel's dynamic shared-memory limit and return its resident
// CTAs per SM.
template <class T, int DIR, int VAR>
int occupancy_one() {
    constexpr int smem = sweep_smem_bytes<T>(DIR);
    if (cudaFuncSetAttribute(sweep_kernel<T, DIR, VAR>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
        cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<T, DIR, VAR>, kSweepThreads, smem) !=
        cudaSuccess)
        return 0;
    return nb;
}

}  // namespace hydro
