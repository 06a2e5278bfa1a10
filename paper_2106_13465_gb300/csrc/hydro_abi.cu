// hydro_abi.cu -- the C ABI of include/hydro.h: context and HBM layout, tile
// work-lists, the step driver (§1, Fig. 5: per step a dt, then a sweep along
// each direction, the order alternating), CUDA-graph capture of the step
// loop, state transfer and diagnostics.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <functional>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "hydro.h"
#include "kernels.h"

using namespace hydro;

namespace {

thread_local std::string g_init_error;

constexpr int kDefaultTileLen = 0;  // 0: chosen per direction by auto_tile_len
constexpr int kDefaultGraphSteps = 20;

long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

template <class T>
Consts<T> make_consts(const hydro_params& p, double tol) {
    const double g = p.gamma;
    Consts<T> K;
    K.gamma = (T)g;
    K.gm1 = (T)(g - 1.0);
    K.g_gm1 = (T)(g / (g - 1.0));
    K.z = (T)((g - 1.0) / (2.0 * g));
    K.zs = (T)((g + 1.0) / (2.0 * g));
    K.G3 = (T)(2.0 * g / (g - 1.0));
    K.G4 = (T)(2.0 / (g - 1.0));
    K.G5 = (T)(2.0 / (g + 1.0));
    K.G6 = (T)((g - 1.0) / (g + 1.0));
    K.G7 = (T)((g - 1.0) / 2.0);
    K.inv_g = (T)(1.0 / g);
    K.hgp1 = (T)((g + 1.0) / 2.0);
    K.sqg = (T)std::sqrt(g);
    K.rho_floor = (T)p.rho_floor;
    K.cf2g = (T)(p.c_floor * p.c_floor / g);
    K.pmin = (T)(p.rho_floor * (p.c_floor * p.c_floor / g));
    K.tol = (T)tol;
    K.niter = p.niter_riemann;
    K.g75 = (g == 1.4) ? 1 : 0;
    K.two_shock = p.riemann_solver == HYDRO_RIEMANN_TWO_SHOCK ? 1 : 0;
    K.slope = p.slope_type == HYDRO_SLOPE_MC ? SLOPE_MC : (p.slope_type == HYDRO_SLOPE_NONE ? SLOPE_NONE : SLOPE_MINMOD);
    K.char_trace = p.trace_type == HYDRO_TRACE_CHARACTERISTIC ? 1 : 0;
    double c = 1.0, z = (g - 1.0) / (2.0 * g);
    for (int k = 1; k <= kBinomTerms; ++k) {
        c *= (z - (k - 1)) / k;  // C(z, k)
        K.bz[k - 1] = (T)c;
    }
    // below it (p/p_K)^z came from exp2/log2 (the 7th root for g = 7/5 costs
    // no more than the series, so 0 there)
    K.pz_series = K.g75 ? (T)0 : (T)std::pow(1.0 - kBinomRadius, z);
    K.f_gamma = (float)g;
    K.f_gm1 = (float)(g - 1.0);
    K.f_rho_floor = (float)p.rho_floor;
    K.f_cf2g = (float)(p.c_floor * p.c_floor / g);
    return K;
}

}  // namespace

struct hydro_ctx {
    int prec = 64;
    size_t esz = 8;
    double cfl = 0.8;
    Consts<double> Kd{};
    Consts<float> Kf{};
    std::vector<hydro_grid> grids;
    std::vector<GridDesc> gd;
    int device = 0;
    int nsm = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t capture_stream = nullptr;
    void* buf[2] = {nullptr, nullptr};
    size_t buf_elems = 0;
    GridDesc* d_grids = nullptr;
    Tile* d_tiles[3] = {nullptr, nullptr, nullptr};  // work lists: x, y, fused step
    int ntiles[3] = {0, 0, 0};
    GridRun* d_run = nullptr;
    DevCounters* d_ctr = nullptr;
    double* d_stage = nullptr;  // FP64 [4][ny][nx] staging (FP32 contexts)
    double* d_rows = nullptr;   // conservation row sums [4][max ny]
    double* d_out4 = nullptr;
    double* d_dt_ovr = nullptr;
    size_t dt_ovr_cap = 0;
    double* d_dt_log = nullptr;
    size_t dt_log_cap = 0;
    CUtensorMap* d_maps = nullptr;  // [grid][buffer][dir]
    int* d_redo = nullptr;          // [2][redo_cap] FP32 second-pass tile lists
    // adaptive walk tiles (FP64), per walk direction d (0 x, 1 y)
    float* d_wcost[2] = {nullptr, nullptr};               // recorded cost per block
    unsigned long long* d_wclaim[2] = {nullptr, nullptr};  // claim words of the long jobs
    Tile* d_wstat[2] = {nullptr, nullptr};                 // static tiling the pieces split
    unsigned int* d_tile_smax = nullptr;  // FP64: max speed estimate per tile of a second sweep
    int tile_smax_cap = 0;
    int nwstat[2] = {0, 0};
    long long nwblocks[2] = {0, 0};         // cost blocks of all grids
    bool w_adaptive[2] = {false, false};    // tiles cut from recorded costs every step
    double w_cap[2] = {0.0, 0.0};           // cost cap / total recorded cost
    int redo_cap = 0;
    int ctas_redo[3] = {0, 0, 0};
    hydro_tuning tuning{kDefaultTileLen, 0, kDefaultGraphSteps, 0, 0};
    int ctas[3] = {0, 0, 0};    // CTAs per launch (x sweep, y sweep, fused step)
    int tile_len_used[2] = {0, 0};
    long long step = 0;         // steps since the last hydro_set_state
    long long launches = 0;     // kernels launched by the step calls since hydro_init
    unsigned wait_limit = kWaitLimit;  // polls of a TMA completion before a sweep warp gives up
    int cur = 0;                // state buffer holding the current state (a fused
                                // step moves it to the other buffer)
    cudaGraphExec_t gexec = nullptr;
    int gexec_steps = 0;
    int gexec_cur = 0;          // `cur` the graph was captured for
    std::string err;
};

namespace {

hydro_status fail(hydro_ctx* c, hydro_status st, const std::string& msg) {
    if (c) c->err = msg;
    else g_init_error = msg;
    return st;
}

hydro_status fail_cuda(hydro_ctx* c, const char* what, cudaError_t e) {
    return fail(c, HYDRO_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define HCK(ctx, call)                                                  \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return fail_cuda((ctx), #call, e_);      \
    } while (0)

bool valid_bc(const int bc[4]) {
    for (int k = 0; k < 4; ++k)
        if (bc[k] < HYDRO_BC_REFLECT || bc[k] > HYDRO_BC_PERIODIC) return false;
    if ((bc[0] == HYDRO_BC_PERIODIC) != (bc[1] == HYDRO_BC_PERIODIC)) return false;
    if ((bc[2] == HYDRO_BC_PERIODIC) != (bc[3] == HYDRO_BC_PERIODIC)) return false;
    return true;
}

hydro_status validate_params(const hydro_params* p) {
    if (!p) return fail(nullptr, HYDRO_EINVAL, "params is NULL");
    if (p->precision != HYDRO_PREC_FP32 && p->precision != HYDRO_PREC_FP64)
        return fail(nullptr, HYDRO_EINVAL, "precision must be 32 or 64");
    if (!(p->gamma > 1.0) || !std::isfinite(p->gamma))
        return fail(nullptr, HYDRO_EINVAL, "gamma must be finite and > 1");
    if (!(p->cfl > 0.0) || !std::isfinite(p->cfl))
        return fail(nullptr, HYDRO_EINVAL, "cfl must be finite and > 0");
    if (p->niter_riemann < 0 || p->niter_riemann > 1000)
        return fail(nullptr, HYDRO_EINVAL, "niter_riemann must be in [0, 1000]");
    if (!(p->rho_floor > 0.0) || !(p->c_floor > 0.0))
        return fail(nullptr, HYDRO_EINVAL, "rho_floor and c_floor must be > 0");
    if (p->riemann_solver != HYDRO_RIEMANN_EXACT && p->riemann_solver != HYDRO_RIEMANN_TWO_SHOCK)
        return fail(nullptr, HYDRO_EINVAL, "riemann_solver must be HYDRO_RIEMANN_EXACT or HYDRO_RIEMANN_TWO_SHOCK");
    if (p->slope_type < HYDRO_SLOPE_MINMOD || p->slope_type > HYDRO_SLOPE_NONE)
        return fail(nullptr, HYDRO_EINVAL, "slope_type must be HYDRO_SLOPE_MINMOD, _MC or _NONE");
    if (p->trace_type != HYDRO_TRACE_MUSCL_HANCOCK && p->trace_type != HYDRO_TRACE_CHARACTERISTIC)
        return fail(nullptr, HYDRO_EINVAL, "trace_type must be HYDRO_TRACE_MUSCL_HANCOCK or _CHARACTERISTIC");
    if (p->ngrids < 1 || !p->grids)
        return fail(nullptr, HYDRO_EINVAL, "need ngrids >= 1 and a grids array");
    for (int g = 0; g < p->ngrids; ++g) {
        const hydro_grid& G = p->grids[g];
        char buf[160];
        if (G.nx < 2 || G.ny < 2 || G.nx > (1 << 24) || G.ny > (1 << 24)) {
            snprintf(buf, sizeof buf, "grid %d: nx, ny must be in [2, 2^24] (got %d x %d)", g, G.nx, G.ny);
            return fail(nullptr, HYDRO_EINVAL, buf);
        }
        // the y sweep addresses a column of a plane with 32-bit offsets
        if ((long long)round_up(G.nx, 32) * G.ny >= (1LL << 31)) {
            snprintf(buf, sizeof buf, "grid %d: a plane (ny x nx rounded up to 32) must hold fewer than 2^31 cells", g);
            return fail(nullptr, HYDRO_EINVAL, buf);
        }
        if (!(G.h > 0.0) || !std::isfinite(G.h)) {
            snprintf(buf, sizeof buf, "grid %d: h must be finite and > 0", g);
            return fail(nullptr, HYDRO_EINVAL, buf);
        }
        if (!valid_bc(G.bc)) {
            snprintf(buf, sizeof buf, "grid %d: bad boundary conditions (periodic must pair)", g);
            return fail(nullptr, HYDRO_EINVAL, buf);
        }
    }
    return HYDRO_OK;
}

// x segments of a row of n cells: segment k covers results [60k-2, 60k+58).
int x_segments(int n) { return (n + 2 + kXStride - 1) / kXStride; }

// Tile work-lists.  y sweep: for each grid, columns in groups of 32 (one per
// lane), rows in runs of len.  x sweep, walking (FP64, xwalk): rows in
// groups of 32, columns in runs of len.  x sweep in segments (FP32): for each
// grid and row, runs of len consecutive segments (one warp task each).
void build_tiles(const std::vector<GridDesc>& gd, int dir, int len, std::vector<Tile>& out, bool xwalk = false) {
    out.clear();
    for (int g = 0; g < (int)gd.size(); ++g) {
        if (dir == DIR_X && xwalk) {
            for (int l0 = 0; l0 < gd[g].ny; l0 += kWarpLines)
                for (int c0 = 0; c0 < gd[g].nx; c0 += len)
                    out.push_back(Tile{g, l0, c0, std::min(len, gd[g].nx - c0)});
        } else if (dir == DIR_Y) {
            for (int l0 = 0; l0 < gd[g].nx; l0 += kWarpLines)
                for (int c0 = 0; c0 < gd[g].ny; c0 += len)
                    out.push_back(Tile{g, l0, c0, std::min(len, gd[g].ny - c0)});
        } else {
            const int ns = x_segments(gd[g].nx);
            for (int j = 0; j < gd[g].ny; ++j)
                for (int k0 = 0; k0 < ns; k0 += len)
                    out.push_back(Tile{g, j, k0, std::min(len, ns - k0)});
        }
    }
}

// Fused step tiles: for each grid, x segment k (columns [60k - 2, 60k + 58))
// times runs of kFusedRows rows.
void build_fused_tiles(const std::vector<GridDesc>& gd, std::vector<Tile>& out) {
    out.clear();
    for (int g = 0; g < (int)gd.size(); ++g) {
        const int ns = x_segments(gd[g].nx);
        for (int y0 = 0; y0 < gd[g].ny; y0 += kFusedRows)
            for (int k = 0; k < ns; ++k) out.push_back(Tile{g, k, y0, std::min(kFusedRows, gd[g].ny - y0)});
    }
}

// Cost of a tile in cell units for the scheduling model: a walk (y, or x
// walking), its cells plus its 4-cell halo; x segments, the 64 cells of
// each of its segments plus a start-up.
double tile_cost(const Tile& t, int dir, bool xwalk = false) {
    if (dir == DIR_Y || xwalk) return t.ncell + 4.0;
    return t.ncell * (double)kXSegment + 16.0;
}

// Makespan of the dynamic tile queue on `warps` resident warps (list
// scheduling in queue order).
double list_schedule_makespan(const std::vector<Tile>& tiles, int dir, int warps, bool xwalk = false) {
    std::vector<double> heap(std::max(1, warps), 0.0);  // min-heap of warp finish times
    std::make_heap(heap.begin(), heap.end(), std::greater<double>());
    double span = 0.0;
    for (const Tile& t : tiles) {
        std::pop_heap(heap.begin(), heap.end(), std::greater<double>());
        heap.back() += tile_cost(t, dir, xwalk);
        span = std::max(span, heap.back());
        std::push_heap(heap.begin(), heap.end(), std::greater<double>());
    }
    return span;
}

int auto_tile_len(const std::vector<GridDesc>& gd, int dir, int warps, bool xwalk = false) {
    std::vector<int> cand;
    if (xwalk) {
        // x walks at most 64 cells: on copy-dominated fields (the 10000^2
        // explosion) the x walk ran 7 % faster with 64-cell tiles than with
        // the model's 192, while the FP64-bound 8192^2 field lost 0.7 %
        for (int L = 4; L <= 64; L += 4) cand.push_back(L);
    } else if (dir == DIR_Y) {
        for (int L = 4; L <= 128; L += 4) cand.push_back(L);
        for (int L : {160, 192, 256, 384, 512}) cand.push_back(L);
    } else {
        for (int L : {1, 2, 3, 4, 5, 6, 8, 10, 12, 16, 24, 32, 48, 64, 128}) cand.push_back(L);
    }
    int best = cand[0];
    double best_span = 1e300;
    std::vector<Tile> t;
    for (int L : cand) {
        build_tiles(gd, dir, L, t, xwalk);
        if (t.size() > 4000000) continue;
        const double span = list_schedule_makespan(t, dir, warps, xwalk);
        if (span < best_span * 0.999) { best_span = span; best = L; }
    }
    return best;
}

// TMA tensor maps of every grid over both state buffers (see kernels.h).
hydro_status build_tensor_maps(hydro_ctx* c) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
        return fail(c, HYDRO_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    const size_t nmaps = c->gd.size() * 2 * kMapKinds;
    std::vector<CUtensorMap> maps(nmaps);
    const CUtensorMapDataType dtype = c->prec == 64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    for (size_t g = 0; g < c->gd.size(); ++g) {
        const GridDesc& d = c->gd[g];
        const cuuint64_t dims[3] = {(cuuint64_t)d.nx, (cuuint64_t)d.ny, 4};
        const cuuint64_t strides[2] = {(cuuint64_t)d.pitch * c->esz, (cuuint64_t)d.plane * c->esz};
        const cuuint32_t estr[3] = {1, 1, 1};
        for (int b = 0; b < 2; ++b) {
            void* base = (char*)c->buf[b] + (size_t)d.off * c->esz;
            for (int dir = 0; dir < kMapKinds; ++dir) {
                // x: a segment (FP32) or a chunk of 4 columns x 32 rows (FP64 walks)
                const bool xw = dir == DIR_X && c->prec == 64;
                const cuuint32_t box[3] = {dir == DIR_Y ? 32u : (xw ? 4u : (cuuint32_t)kXSegment),
                                           dir == DIR_X ? (xw ? 32u : 1u) : (dir == DIR_Y ? 4u : (cuuint32_t)kFusedBoxRows),
                                           4u};
                CUresult r = encode(&maps[map_index((int)g, b, dir)], dtype, 3, base, dims, strides, box, estr,
                                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
                if (r != CUDA_SUCCESS) {
                    char buf[160];
                    snprintf(buf, sizeof buf, "cuTensorMapEncodeTiled failed (%d) for grid %zu", (int)r, g);
                    return fail(c, HYDRO_ECUDA, buf);
                }
            }
        }
    }
    HCK(c, cudaMalloc(&c->d_maps, sizeof(CUtensorMap) * nmaps));
    HCK(c, cudaMemcpy(c->d_maps, maps.data(), sizeof(CUtensorMap) * nmaps, cudaMemcpyHostToDevice));
    return HYDRO_OK;
}

// Cost blocks before any sweep has run: the cells each block holds (a
// uniform cost per cell), and the same total in both parity slots.
hydro_status init_wcost(hydro_ctx* c) {
    for (int dir = 0; dir < 2; ++dir) {
        std::vector<float> cost((size_t)c->nwblocks[dir]);
        unsigned long long total = 0;
        const int B = walk_block(dir);
        for (int g = 0; g < (int)c->gd.size(); ++g) {
            const GridDesc& d = c->gd[g];
            const int n = dir == DIR_X ? d.nx : d.ny;
            for (int lg = 0; lg < d.wlg[dir]; ++lg) {
                for (int b = 0; b < d.wnb[dir]; ++b) {
                    const int cells = std::min(B, n - b * B);
                    cost[(size_t)(d.wblk[dir] + (long long)lg * d.wnb[dir] + b)] = (float)cells;
                    total += (unsigned long long)cells;
                }
            }
        }
        const unsigned long long tot2[2] = {total, total};
        HCK(c, cudaMemcpy(c->d_wcost[dir], cost.data(), sizeof(float) * cost.size(), cudaMemcpyHostToDevice));
        HCK(c, cudaMemcpy(&c->d_ctr->wcost_total[dir][0], tot2, sizeof tot2, cudaMemcpyHostToDevice));
    }
    return HYDRO_OK;
}

hydro_status upload_tiles(hydro_ctx* c) {
    for (int d = 0; d < 2; ++d) {
        const int var = c->prec == 64 ? VAR_F64 : VAR_F32_MAIN;
        int per_sm = c->tuning.ctas_per_sm;
        const int occ = c->prec == 64 ? sweep_ctas_per_sm<double>(d, var) : sweep_ctas_per_sm<float>(d, var);
        if (occ <= 0) return fail(c, HYDRO_ECUDA, "sweep kernel cannot be resident on an SM");
        if (per_sm <= 0 || per_sm > occ) per_sm = occ;
        const int warps_per_cta = kSweepThreads / 32;
        const int resident_warps = c->nsm * per_sm * warps_per_cta;
        const int chosen = d == DIR_X ? c->tuning.span_len / kXStride : c->tuning.tile_len;
        if (c->d_tiles[d]) cudaFree(c->d_tiles[d]);
        c->d_tiles[d] = nullptr;
        if (chosen == 0 && c->prec == 64) {
            // adaptive walk tiles (FP64, where the cost of a cell varies most
            // with the Riemann problems it meets): the list is cut on the
            // device every step; it never holds more tiles than there are
            // cost blocks.  The length cap is the model's static tile length;
            // the cost cap a multiple of the mean cost of such a tile.
            const bool xwalk = d == DIR_X;
            const int B = walk_block(d);
            const int L = auto_tile_len(c->gd, d, resident_warps, xwalk);
            const int lb = std::max(B, L / B * B);  // L is a multiple of 4
            std::vector<Tile> t;
            build_tiles(c->gd, d, lb, t, xwalk);
            if (c->d_wstat[d]) cudaFree(c->d_wstat[d]);
            c->d_wstat[d] = nullptr;
            HCK(c, cudaMalloc(&c->d_wstat[d], sizeof(Tile) * t.size()));
            HCK(c, cudaMemcpy(c->d_wstat[d], t.data(), sizeof(Tile) * t.size(), cudaMemcpyHostToDevice));
            c->nwstat[d] = (int)t.size();
            c->w_adaptive[d] = true;
            c->w_cap[d] = kYCostCap / (double)t.size();
            c->tile_len_used[d] = 0;
            HCK(c, cudaMalloc(&c->d_tiles[d], sizeof(Tile) * (size_t)c->nwblocks[d]));
            c->ntiles[d] = (int)std::min<long long>(c->nwblocks[d], 1LL << 30);
            // claim words start below every step count (steps count from 1)
            if (c->d_wclaim[d]) cudaFree(c->d_wclaim[d]);
            c->d_wclaim[d] = nullptr;
            HCK(c, cudaMalloc(&c->d_wclaim[d], sizeof(unsigned long long) * (size_t)c->nwblocks[d]));
            HCK(c, cudaMemset(c->d_wclaim[d], 0, sizeof(unsigned long long) * (size_t)c->nwblocks[d]));
        } else {
            c->w_adaptive[d] = false;
            // FP64 walks the x lines: span_len (a multiple of 60, so of 4) is
            // then the cells of a walk
            const bool xwalk = d == DIR_X && c->prec == 64;
            const int pick = xwalk ? c->tuning.span_len : chosen;
            const int L = pick > 0 ? pick : auto_tile_len(c->gd, d, resident_warps, xwalk);
            c->tile_len_used[d] = L;
            std::vector<Tile> t;
            build_tiles(c->gd, d, L, t, xwalk);
            HCK(c, cudaMalloc(&c->d_tiles[d], sizeof(Tile) * t.size()));
            HCK(c, cudaMemcpy(c->d_tiles[d], t.data(), sizeof(Tile) * t.size(), cudaMemcpyHostToDevice));
            c->ntiles[d] = (int)t.size();
        }
        const int need = (c->ntiles[d] + warps_per_cta - 1) / warps_per_cta;
        c->ctas[d] = std::max(1, std::min(need, c->nsm * per_sm));
        if (c->prec == 32) {
            const int occ2 = sweep_ctas_per_sm<float>(d, VAR_F32_REDO);
            if (occ2 <= 0) return fail(c, HYDRO_ECUDA, "second-pass kernel cannot be resident on an SM");
            c->ctas_redo[d] = std::max(1, std::min(need, c->nsm * occ2));
        }
    }
    {
        // fused step tiles (used when tuning.fused is set)
        std::vector<Tile> t;
        build_fused_tiles(c->gd, t);
        if (c->d_tiles[DIR_FUSED]) cudaFree(c->d_tiles[DIR_FUSED]);
        c->d_tiles[DIR_FUSED] = nullptr;
        HCK(c, cudaMalloc(&c->d_tiles[DIR_FUSED], sizeof(Tile) * t.size()));
        HCK(c, cudaMemcpy(c->d_tiles[DIR_FUSED], t.data(), sizeof(Tile) * t.size(), cudaMemcpyHostToDevice));
        c->ntiles[DIR_FUSED] = (int)t.size();
        const int var = c->prec == 64 ? VAR_F64 : VAR_F32_MAIN;
        const int occ = c->prec == 64 ? fused_ctas_per_sm<double>(var) : fused_ctas_per_sm<float>(var);
        if (occ <= 0) return fail(c, HYDRO_ECUDA, "fused step kernel cannot be resident on an SM");
        int per_sm = c->tuning.ctas_per_sm;
        if (per_sm <= 0 || per_sm > occ) per_sm = occ;
        c->ctas[DIR_FUSED] = std::max(1, std::min(c->ntiles[DIR_FUSED], c->nsm * per_sm));
        if (c->prec == 32) {
            const int occ2 = fused_ctas_per_sm<float>(VAR_F32_REDO);
            if (occ2 <= 0) return fail(c, HYDRO_ECUDA, "fused second-pass kernel cannot be resident on an SM");
            c->ctas_redo[DIR_FUSED] = std::max(1, std::min(c->ntiles[DIR_FUSED], c->nsm * occ2));
        }
    }
    const int max_tiles = std::max(c->ntiles[DIR_FUSED], std::max(c->ntiles[0], c->ntiles[1]));
    if (c->prec == 64) {
        const int cap = max_tiles;
        if (cap > c->tile_smax_cap) {
            cudaFree(c->d_tile_smax);
            c->d_tile_smax = nullptr;
            c->tile_smax_cap = 0;
            HCK(c, cudaMalloc(&c->d_tile_smax, sizeof(unsigned int) * (size_t)cap));
            c->tile_smax_cap = cap;
        }
    }
    if (c->prec == 32) {
        const int cap = max_tiles;
        if (cap > c->redo_cap) {
            cudaFree(c->d_redo);
            c->d_redo = nullptr;
            c->redo_cap = 0;
            HCK(c, cudaMalloc(&c->d_redo, sizeof(int) * 2 * (size_t)cap));
            c->redo_cap = cap;
        }
    }
    return HYDRO_OK;
}

void drop_graph(hydro_ctx* c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    c->gexec_steps = 0;
}

template <class T>
SweepArgs<T> sweep_args(hydro_ctx* c, int which, const Consts<T>& K) {
    SweepArgs<T> a;
    a.src = (const T*)c->buf[c->cur ^ which];
    a.dst = (T*)c->buf[c->cur ^ which ^ 1];
    a.grids = c->d_grids;
    a.tiles = nullptr;
    a.maps = c->d_maps;
    a.ntiles = 0;
    a.ngrids = (int)c->gd.size();
    a.ntiles_dev = nullptr;
    a.wclaim = nullptr;
    a.nsm = c->nsm;
    a.wcost = nullptr;
    a.tile_smax = c->d_tile_smax;
    a.wait_limit = c->wait_limit;
    a.which = which;
    a.src_buf = c->cur ^ which;
    a.redo_list = c->d_redo;
    a.redo_cap = c->redo_cap;
    a.run = c->d_run;
    a.ctr = c->d_ctr;
    a.K = K;
    a.Kd = c->Kd;
    return a;
}

// Enqueue one fused step (fused_tma.cuh): the dt prologue, the step kernel
// from buf[cur] to buf[cur ^ 1], and (FP64) the exact CFL pass over the new
// state or (FP32) the near-vacuum second pass; the state then lives in
// buf[cur ^ 1].  ev as in enqueue_step_t (the second interval is empty).
template <class T>
cudaError_t enqueue_fused_step_t(hydro_ctx* c, int parity, const double* ovr, double* log, cudaStream_t s,
                                 const Consts<T>& K, cudaEvent_t* ev) {
    cudaError_t e;
    if (ev && (e = cudaEventRecord(ev[0], s)) != cudaSuccess) return e;
    e = launch_step_prologue(c->d_run, c->d_grids, (int)c->gd.size(), c->d_ctr, ovr, c->cfl, log, s);
    if (e != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[1], s)) != cudaSuccess) return e;
    SweepArgs<T> a = sweep_args<T>(c, 0, K);
    a.which = 1;  // the new state's CFL speed is folded in
    a.tiles = c->d_tiles[DIR_FUSED];
    a.ntiles = c->ntiles[DIR_FUSED];
    if (sizeof(T) == 8) {
        e = launch_fused<T>(parity, VAR_F64, a, c->ctas[DIR_FUSED], s);
        if (e == cudaSuccess)
            e = launch_cfl_fp64((const double*)a.dst, c->d_grids, a.tiles, a.ntiles, nullptr, DIR_FUSED,
                                c->d_tile_smax, c->d_run, c->d_ctr, c->Kd, c->nsm * 8, s);
    } else {
        e = launch_fused<T>(parity, VAR_F32_MAIN, a, c->ctas[DIR_FUSED], s);
        if (e == cudaSuccess) e = launch_fused<T>(parity, VAR_F32_REDO, a, c->ctas_redo[DIR_FUSED], s);
    }
    if (e != cudaSuccess) return e;
    c->cur ^= 1;
    if (ev && (e = cudaEventRecord(ev[2], s)) != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[3], s)) != cudaSuccess) return e;
    return cudaSuccess;
}

// Enqueue one step of parity `parity` on stream s; ev (optional, 4 events)
// brackets the three launches for timing.
template <class T>
cudaError_t enqueue_step_t(hydro_ctx* c, int parity, const double* ovr, double* log,
                           cudaStream_t s, const Consts<T>& K, cudaEvent_t* ev) {
    if (c->tuning.fused) return enqueue_fused_step_t<T>(c, parity, ovr, log, s, K, ev);
    cudaError_t e;
    if (ev && (e = cudaEventRecord(ev[0], s)) != cudaSuccess) return e;
    e = launch_step_prologue(c->d_run, c->d_grids, (int)c->gd.size(), c->d_ctr, ovr, c->cfl, log, s);
    if (e != cudaSuccess) return e;
    for (int d = 0; d < 2; ++d) {
        if (!c->w_adaptive[d]) continue;
        e = launch_retile(d, c->d_grids, c->d_wstat[d], c->nwstat[d], c->d_wcost[d], c->d_ctr, c->d_tiles[d],
                          c->ntiles[d], c->w_cap[d], c->w_cap[d] * (kYBigJob / kYCostCap), kYBigOfMax, s);
        if (e != cudaSuccess) return e;
    }
    if (ev && (e = cudaEventRecord(ev[1], s)) != cudaSuccess) return e;
    const int first = parity == 0 ? DIR_X : DIR_Y;
    for (int which = 0; which < 2; ++which) {
        const int dir = which == 0 ? first : (first ^ 1);
        SweepArgs<T> a = sweep_args<T>(c, which, K);
        a.tiles = c->d_tiles[dir];
        a.ntiles = c->ntiles[dir];
        if (sizeof(T) == 8) a.wcost = c->d_wcost[dir];
        if (c->w_adaptive[dir]) {
            a.ntiles_dev = c->d_ctr->wtiles[dir];
            a.wclaim = c->d_wclaim[dir];
        }
        if (sizeof(T) == 8) {
            e = launch_sweep<T>(dir, VAR_F64, a, c->ctas[dir], s);
            // the second sweep's new state: its max wave speed (next dt)
            if (e == cudaSuccess && which == 1)
                e = launch_cfl_fp64((const double*)c->buf[c->cur], c->d_grids, a.tiles, a.ntiles, a.ntiles_dev, dir,
                                    c->d_tile_smax, c->d_run, c->d_ctr, c->Kd, c->nsm * 8, s);
        } else {
            // main FP32 pass, then the second pass over tiles it queued
            e = launch_sweep<T>(dir, VAR_F32_MAIN, a, c->ctas[dir], s);
            if (e == cudaSuccess) e = launch_sweep<T>(dir, VAR_F32_REDO, a, c->ctas_redo[dir], s);
        }
        if (e != cudaSuccess) return e;
        if (ev && (e = cudaEventRecord(ev[2 + which], s)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Kernels one step launches (enqueue_step_t): the dt prologue, a tiler per
// direction with adaptive tiles, and per sweep the sweep kernel plus, FP64, the CFL
// pass after the second sweep or, FP32, the near-vacuum second pass.  A
// fused step: the prologue, the step kernel and the CFL or second pass.
int launches_per_step(const hydro_ctx* c) {
    if (c->tuning.fused) return 3;
    return 1 + (c->w_adaptive[0] ? 1 : 0) + (c->w_adaptive[1] ? 1 : 0) + (c->prec == 64 ? 2 + 1 : 2 * 2);
}

cudaError_t enqueue_step(hydro_ctx* c, int parity, const double* ovr, double* log, cudaStream_t s,
                         cudaEvent_t* ev = nullptr) {
    if (c->prec == 64) return enqueue_step_t<double>(c, parity, ovr, log, s, c->Kd, ev);
    return enqueue_step_t<float>(c, parity, ovr, log, s, c->Kf, ev);
}

hydro_status ensure_graph(hydro_ctx* c, int steps) {
    if (c->gexec && c->gexec_steps == steps && c->gexec_cur == c->cur) return HYDRO_OK;
    drop_graph(c);
    cudaGraph_t graph = nullptr;
    HCK(c, cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    // the captured steps move `cur` as they will when the graph runs; an even
    // number of steps brings it back
    const int cur0 = c->cur;
    for (int k = 0; k < steps && e == cudaSuccess; ++k)
        e = enqueue_step(c, k & 1, nullptr, nullptr, c->capture_stream);
    c->cur = cur0;
    cudaError_t e2 = cudaStreamEndCapture(c->capture_stream, &graph);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return fail_cuda(c, "sweep launch during graph capture", e);
    }
    if (e2 != cudaSuccess) return fail_cuda(c, "cudaStreamEndCapture", e2);
    e = cudaGraphInstantiate(&c->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        c->gexec = nullptr;
        return fail_cuda(c, "cudaGraphInstantiate", e);
    }
    c->gexec_steps = steps;
    c->gexec_cur = cur0;
    return HYDRO_OK;
}

hydro_status check_grid(hydro_ctx* c, int grid) {
    if (!c) return fail(nullptr, HYDRO_EINVAL, "ctx is NULL");
    if (grid < 0 || grid >= (int)c->gd.size()) return fail(c, HYDRO_EINVAL, "grid index out of range");
    return HYDRO_OK;
}

template <class T>
T* state_ptr(hydro_ctx* c) { return (T*)c->buf[c->cur]; }

hydro_status status_result(hydro_ctx* c, unsigned int status) {
    if (status & STATUS_BAD_TILE)
        return fail(c, HYDRO_ECUDA, "internal error: a sweep tile lies outside its grid (tile skipped)");
    if (status & STATUS_TIMEOUT)
        return fail(c, HYDRO_ETIMEOUT, "a bounded wait for a TMA copy gave up (sweep kernel)");
    if (status) {
        char buf[120];
        snprintf(buf, sizeof buf, "non-positive or NaN %s detected", (status & STATUS_BAD_RHO) ? "density" : "energy");
        return fail(c, HYDRO_ENEGATIVE, buf);
    }
    return HYDRO_OK;
}

}  // namespace

extern "C" {

hydro_status hydro_init(const hydro_params* params, hydro_ctx** out) {
    if (!out) return fail(nullptr, HYDRO_EINVAL, "out is NULL");
    *out = nullptr;
    hydro_status st = validate_params(params);
    if (st != HYDRO_OK) return st;

    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev < 1)
        return fail(nullptr, HYDRO_ECUDA,
                    std::string("no CUDA device: ") + (e != cudaSuccess ? cudaGetErrorString(e) : "count 0"));

    hydro_ctx* c = new (std::nothrow) hydro_ctx();
    if (!c) return fail(nullptr, HYDRO_ENOMEM, "host allocation failed");
    auto bail = [&](hydro_status s) {
        g_init_error = c->err;
        hydro_destroy(c);
        return s;
    };

    c->prec = params->precision;
    c->esz = c->prec == 64 ? 8 : 4;
    c->cfl = params->cfl;
    // Newton convergence tolerances (godunov.cuh: riemann_star)
    c->Kd = make_consts<double>(*params, 1e-8);
    c->Kf = make_consts<float>(*params, 3e-4);
    c->grids.assign(params->grids, params->grids + params->ngrids);
    cudaGetDevice(&c->device);
    cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device);
    if (c->nsm <= 0) c->nsm = 1;

    // HBM layout (see kernels.h)
    long long off = 0, max_cells = 0, max_ny = 0;
    const long long align_elems = 256 / (long long)c->esz;
    for (const hydro_grid& G : c->grids) {
        GridDesc d{};
        d.nx = G.nx;
        d.ny = G.ny;
        d.pitch = (int)round_up(G.nx, 32);
        d.plane = (long long)d.pitch * G.ny;
        d.off = off;
        for (int k = 0; k < 4; ++k) d.bc[k] = G.bc[k];
        d.h = G.h;
        for (int dir = 0; dir < 2; ++dir) {
            const int nlines = dir == DIR_X ? G.ny : G.nx, ncells = dir == DIR_X ? G.nx : G.ny;
            d.wlg[dir] = (nlines + kWarpLines - 1) / kWarpLines;
            d.wnb[dir] = (ncells + walk_block(dir) - 1) / walk_block(dir);
            d.wblk[dir] = c->nwblocks[dir];
            c->nwblocks[dir] += (long long)d.wlg[dir] * d.wnb[dir];
        }
        off = round_up(off + 4 * d.plane, align_elems);
        max_cells = std::max(max_cells, (long long)G.nx * G.ny);
        max_ny = std::max(max_ny, (long long)G.ny);
        c->gd.push_back(d);
    }
    c->buf_elems = (size_t)off;

    if (params->cuda_stream) {
        c->stream = (cudaStream_t)params->cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { fail_cuda(c, "cudaStreamCreate", e); return bail(HYDRO_ECUDA); }
        c->own_stream = true;
    }
    e = cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { fail_cuda(c, "cudaStreamCreate", e); return bail(HYDRO_ECUDA); }

    auto alloc = [&](void** p, size_t bytes, const char* what) -> hydro_status {
        cudaError_t ea = cudaMalloc(p, bytes);
        if (ea != cudaSuccess) {
            cudaGetLastError();
            char buf[200];
            snprintf(buf, sizeof buf, "cudaMalloc(%s, %zu bytes): %s", what, bytes, cudaGetErrorString(ea));
            return fail(c, ea == cudaErrorMemoryAllocation ? HYDRO_ENOMEM : HYDRO_ECUDA, buf);
        }
        return HYDRO_OK;
    };
    for (int b = 0; b < 2; ++b)
        if ((st = alloc(&c->buf[b], c->buf_elems * c->esz, "state buffer")) != HYDRO_OK) return bail(st);
    if ((st = alloc((void**)&c->d_grids, sizeof(GridDesc) * c->gd.size(), "grids")) != HYDRO_OK) return bail(st);
    if ((st = alloc((void**)&c->d_run, sizeof(GridRun) * c->gd.size(), "run records")) != HYDRO_OK) return bail(st);
    if ((st = alloc((void**)&c->d_ctr, sizeof(DevCounters), "counters")) != HYDRO_OK) return bail(st);
    if ((st = alloc((void**)&c->d_rows, sizeof(double) * 4 * max_ny, "row sums")) != HYDRO_OK) return bail(st);
    if ((st = alloc((void**)&c->d_out4, sizeof(double) * 4, "sums")) != HYDRO_OK) return bail(st);
    if (c->prec == 32 &&
        (st = alloc((void**)&c->d_stage, sizeof(double) * 4 * max_cells, "staging")) != HYDRO_OK)
        return bail(st);
    for (int dir = 0; dir < 2; ++dir)
        if ((st = alloc((void**)&c->d_wcost[dir], sizeof(float) * c->nwblocks[dir], "cost blocks")) != HYDRO_OK)
            return bail(st);
    e = cudaMemcpy(c->d_grids, c->gd.data(), sizeof(GridDesc) * c->gd.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(c->d_run, 0, sizeof(GridRun) * c->gd.size());
    if (e == cudaSuccess) e = cudaMemset(c->d_ctr, 0, sizeof(DevCounters));
    if (e == cudaSuccess) e = cudaMemset(c->buf[0], 0, c->buf_elems * c->esz);
    if (e == cudaSuccess) e = cudaMemset(c->buf[1], 0, c->buf_elems * c->esz);
    if (e != cudaSuccess) { fail_cuda(c, "context set-up", e); return bail(HYDRO_ECUDA); }
    if ((st = build_tensor_maps(c)) != HYDRO_OK) return bail(st);
    if ((st = init_wcost(c)) != HYDRO_OK) return bail(st);
    if ((st = upload_tiles(c)) != HYDRO_OK) return bail(st);

    *out = c;
    return HYDRO_OK;
}

void hydro_destroy(hydro_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    drop_graph(c);
    for (int b = 0; b < 2; ++b) cudaFree(c->buf[b]);
    for (int d = 0; d < 3; ++d) cudaFree(c->d_tiles[d]);
    cudaFree(c->d_grids);
    cudaFree(c->d_run);
    cudaFree(c->d_ctr);
    cudaFree(c->d_stage);
    cudaFree(c->d_rows);
    cudaFree(c->d_out4);
    cudaFree(c->d_dt_ovr);
    cudaFree(c->d_dt_log);
    cudaFree(c->d_maps);
    cudaFree(c->d_redo);
    for (int dir = 0; dir < 2; ++dir) {
        cudaFree(c->d_wcost[dir]);
        cudaFree(c->d_wclaim[dir]);
        cudaFree(c->d_wstat[dir]);
    }
    cudaFree(c->d_tile_smax);
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

hydro_status hydro_set_tuning(hydro_ctx* c, const hydro_tuning* t) {
    if (!c || !t) return fail(c, HYDRO_EINVAL, "ctx or tuning is NULL");
    hydro_tuning n = *t;
    if (n.tile_len != 0 && (n.tile_len < 4 || n.tile_len > (1 << 24) || (n.tile_len & 3)))
        return fail(c, HYDRO_EINVAL, "tile_len must be 0 (automatic) or a multiple of 4 in [4, 2^24]");
    if (n.span_len != 0 && (n.span_len < kXStride || n.span_len > (1 << 24) || (n.span_len % kXStride)))
        return fail(c, HYDRO_EINVAL, "span_len must be 0 (automatic) or a multiple of 60 in [60, 2^24]");
    if (n.ctas_per_sm < 0 || n.ctas_per_sm > 64) return fail(c, HYDRO_EINVAL, "ctas_per_sm must be in [0, 64]");
    if (n.graph_steps < 0 || (n.graph_steps & 1) || n.graph_steps > 1000)
        return fail(c, HYDRO_EINVAL, "graph_steps must be even and in [0, 1000]");
    if (n.fused != 0 && n.fused != 1) return fail(c, HYDRO_EINVAL, "fused must be 0 or 1");
    HCK(c, cudaStreamSynchronize(c->stream));
    c->tuning = n;
    drop_graph(c);
    return upload_tiles(c);
}

hydro_status hydro_set_wait_limit(hydro_ctx* c, long long polls) {
    if (!c) return fail(nullptr, HYDRO_EINVAL, "ctx is NULL");
    if (polls > 0xffffffffLL) return fail(c, HYDRO_EINVAL, "polls must be below 2^32");
    HCK(c, cudaStreamSynchronize(c->stream));
    c->wait_limit = polls < 0 ? kWaitLimit : (unsigned)polls;
    drop_graph(c);  // the captured launches hold the previous limit
    return HYDRO_OK;
}

hydro_status hydro_set_state(hydro_ctx* c, int grid, const double* U, int on_device) {
    hydro_status st = check_grid(c, grid);
    if (st != HYDRO_OK) return st;
    if (!U) return fail(c, HYDRO_EINVAL, "U is NULL");
    const GridDesc& g = c->gd[grid];
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (c->prec == 64) {
        double* dst = state_ptr<double>(c) + g.off;
        HCK(c, cudaMemcpy2DAsync(dst, sizeof(double) * g.pitch, U, sizeof(double) * g.nx,
                                 sizeof(double) * g.nx, 4 * (size_t)g.ny, kind, c->stream));
        HCK(c, launch_cfl_init<double>(state_ptr<double>(c), c->d_grids, grid, g, c->d_run, c->d_ctr,
                                       c->Kd, c->stream));
    } else {
        HCK(c, cudaMemcpyAsync(c->d_stage, U, sizeof(double) * 4 * g.nx * (size_t)g.ny, kind, c->stream));
        HCK(c, launch_pack<float>(c->d_stage, state_ptr<float>(c), g, c->stream));
        HCK(c, launch_cfl_init<float>(state_ptr<float>(c), c->d_grids, grid, g, c->d_run, c->d_ctr,
                                      c->Kf, c->stream));
    }
    // time of this grid, step counter and status flags restart
    HCK(c, cudaMemsetAsync(&c->d_run[grid].t, 0, sizeof(double), c->stream));
    HCK(c, cudaMemsetAsync(&c->d_ctr->status, 0, sizeof(unsigned int), c->stream));
    HCK(c, cudaMemsetAsync(&c->d_ctr->wait_site, 0, 2 * sizeof(int), c->stream));
    HCK(c, cudaStreamSynchronize(c->stream));
    c->step = 0;
    return HYDRO_OK;
}

hydro_status hydro_get_state(hydro_ctx* c, int grid, double* U, int on_device) {
    hydro_status st = check_grid(c, grid);
    if (st != HYDRO_OK) return st;
    if (!U) return fail(c, HYDRO_EINVAL, "U_out is NULL");
    const GridDesc& g = c->gd[grid];
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (c->prec == 64) {
        const double* src = state_ptr<double>(c) + g.off;
        HCK(c, cudaMemcpy2DAsync(U, sizeof(double) * g.nx, src, sizeof(double) * g.pitch,
                                 sizeof(double) * g.nx, 4 * (size_t)g.ny, kind, c->stream));
    } else {
        HCK(c, launch_unpack<float>(state_ptr<float>(c), c->d_stage, g, c->stream));
        HCK(c, cudaMemcpyAsync(U, c->d_stage, sizeof(double) * 4 * g.nx * (size_t)g.ny, kind, c->stream));
    }
    HCK(c, cudaStreamSynchronize(c->stream));
    return HYDRO_OK;
}

hydro_status hydro_set_rows(hydro_ctx* c, int grid, int row0, int nrows, const double* U, int on_device) {
    hydro_status st = check_grid(c, grid);
    if (st != HYDRO_OK) return st;
    if (!U) return fail(c, HYDRO_EINVAL, "U is NULL");
    const GridDesc& g = c->gd[grid];
    if (row0 < 0 || nrows < 1 || row0 + nrows > g.ny) return fail(c, HYDRO_EINVAL, "rows out of range");
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const size_t n = (size_t)g.nx * nrows;
    if (c->prec == 64) {
        for (int q = 0; q < 4; ++q)
            HCK(c, cudaMemcpy2DAsync(state_ptr<double>(c) + g.off + q * g.plane + (long long)row0 * g.pitch,
                                     sizeof(double) * g.pitch, U + q * n, sizeof(double) * g.nx,
                                     sizeof(double) * g.nx, (size_t)nrows, kind, c->stream));
        HCK(c, launch_cfl_init<double>(state_ptr<double>(c), c->d_grids, grid, g, c->d_run, c->d_ctr, c->Kd,
                                       c->stream));
    } else {
        GridDesc rows = g;  // the row band as a grid of nrows rows
        rows.off = g.off + (long long)row0 * g.pitch;
        rows.ny = nrows;
        HCK(c, cudaMemcpyAsync(c->d_stage, U, sizeof(double) * 4 * n, kind, c->stream));
        HCK(c, launch_pack<float>(c->d_stage, state_ptr<float>(c), rows, c->stream));
        HCK(c, launch_cfl_init<float>(state_ptr<float>(c), c->d_grids, grid, g, c->d_run, c->d_ctr, c->Kf,
                                      c->stream));
    }
    HCK(c, cudaStreamSynchronize(c->stream));
    return HYDRO_OK;
}

hydro_status hydro_get_rows(hydro_ctx* c, int grid, int row0, int nrows, double* U, int on_device) {
    hydro_status st = check_grid(c, grid);
    if (st != HYDRO_OK) return st;
    if (!U) return fail(c, HYDRO_EINVAL, "U_out is NULL");
    const GridDesc& g = c->gd[grid];
    if (row0 < 0 || nrows < 1 || row0 + nrows > g.ny) return fail(c, HYDRO_EINVAL, "rows out of range");
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const size_t n = (size_t)g.nx * nrows;
    if (c->prec == 64) {
        for (int q = 0; q < 4; ++q)
            HCK(c, cudaMemcpy2DAsync(U + q * n, sizeof(double) * g.nx,
                                     state_ptr<double>(c) + g.off + q * g.plane + (long long)row0 * g.pitch,
                                     sizeof(double) * g.pitch, sizeof(double) * g.nx, (size_t)nrows, kind,
                                     c->stream));
    } else {
        GridDesc rows = g;
        rows.off = g.off + (long long)row0 * g.pitch;
        rows.ny = nrows;
        HCK(c, launch_unpack<float>(state_ptr<float>(c), c->d_stage, rows, c->stream));
        HCK(c, cudaMemcpyAsync(U, c->d_stage, sizeof(double) * 4 * n, kind, c->stream));
    }
    HCK(c, cudaStreamSynchronize(c->stream));
    return HYDRO_OK;
}

hydro_status hydro_step_dt(hydro_ctx* c, int nsteps, const double* dt_override, double* dt_used) {
    if (!c) return fail(nullptr, HYDRO_EINVAL, "ctx is NULL");
    if (nsteps < 0) return fail(c, HYDRO_EINVAL, "nsteps < 0");
    if (nsteps == 0) return HYDRO_OK;
    const size_t ng = c->gd.size();
    const size_t nval = (size_t)nsteps * ng;
    if (dt_override) {
        for (size_t k = 0; k < nval; ++k)
            if (!(dt_override[k] > 0.0) || !std::isfinite(dt_override[k]))
                return fail(c, HYDRO_EINVAL, "dt_override values must be finite and > 0");
        if (c->dt_ovr_cap < nval) {
            cudaFree(c->d_dt_ovr);
            c->d_dt_ovr = nullptr;
            c->dt_ovr_cap = 0;
            HCK(c, cudaMalloc(&c->d_dt_ovr, sizeof(double) * nval));
            c->dt_ovr_cap = nval;
        }
        HCK(c, cudaMemcpyAsync(c->d_dt_ovr, dt_override, sizeof(double) * nval,
                               cudaMemcpyHostToDevice, c->stream));
    }
    if (dt_used && c->dt_log_cap < nval) {
        cudaFree(c->d_dt_log);
        c->d_dt_log = nullptr;
        c->dt_log_cap = 0;
        HCK(c, cudaMalloc(&c->d_dt_log, sizeof(double) * nval));
        c->dt_log_cap = nval;
    }

    int s = 0;
    const int G = c->tuning.graph_steps;
    if (!dt_override && !dt_used && G > 0 && nsteps >= G) {
        if (c->step & 1) {
            HCK(c, enqueue_step(c, 1, nullptr, nullptr, c->stream));
            ++c->step;
            ++s;
        }
        if (nsteps - s >= G) {
            hydro_status st = ensure_graph(c, G);
            if (st != HYDRO_OK) return st;
            while (nsteps - s >= G) {
                HCK(c, cudaGraphLaunch(c->gexec, c->stream));
                c->step += G;
                s += G;
            }
        }
    }
    for (; s < nsteps; ++s) {
        const double* ovr = dt_override ? c->d_dt_ovr + (size_t)s * ng : nullptr;
        double* log = dt_used ? c->d_dt_log + (size_t)s * ng : nullptr;
        HCK(c, enqueue_step(c, (int)(c->step & 1), ovr, log, c->stream));
        ++c->step;
    }
    c->launches += (long long)nsteps * launches_per_step(c);
    unsigned int status = 0;
    HCK(c, cudaMemcpyAsync(&status, &c->d_ctr->status, sizeof status, cudaMemcpyDeviceToHost, c->stream));
    if (dt_used)
        HCK(c, cudaMemcpyAsync(dt_used, c->d_dt_log, sizeof(double) * nval, cudaMemcpyDeviceToHost,
                               c->stream));
    HCK(c, cudaStreamSynchronize(c->stream));
    return status_result(c, status);
}

hydro_status hydro_step(hydro_ctx* c, int nsteps, const double* dt_override) {
    return hydro_step_dt(c, nsteps, dt_override, nullptr);
}

hydro_status hydro_step_profiled(hydro_ctx* c, int nsteps, double* kernel_ms) {
    if (!c) return fail(nullptr, HYDRO_EINVAL, "ctx is NULL");
    if (nsteps < 0 || !kernel_ms) return fail(c, HYDRO_EINVAL, "nsteps < 0 or kernel_ms is NULL");
    std::vector<cudaEvent_t> ev(4 * (size_t)nsteps, nullptr);
    hydro_status st = HYDRO_OK;
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) { st = fail(c, HYDRO_ECUDA, "cudaEventCreate failed"); break; }
    for (int s = 0; s < nsteps && st == HYDRO_OK; ++s) {
        cudaError_t e = enqueue_step(c, (int)(c->step & 1), nullptr, nullptr, c->stream, &ev[4 * (size_t)s]);
        if (e != cudaSuccess) st = fail_cuda(c, "profiled step", e);
        else {
            ++c->step;
            c->launches += launches_per_step(c);
        }
    }
    if (st == HYDRO_OK) {
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) st = fail_cuda(c, "cudaStreamSynchronize", e);
    }
    for (int s = 0; s < nsteps && st == HYDRO_OK; ++s)
        for (int k = 0; k < 3; ++k) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[4 * (size_t)s + k], ev[4 * (size_t)s + k + 1]);
            kernel_ms[3 * (size_t)s + k] = ms;
        }
    for (auto& e : ev)
        if (e) cudaEventDestroy(e);
    if (st != HYDRO_OK) return st;
    unsigned int status = 0;
    HCK(c, cudaMemcpy(&status, &c->d_ctr->status, sizeof status, cudaMemcpyDeviceToHost));
    return status_result(c, status);
}

hydro_status hydro_cfl_dt(hydro_ctx* c, int grid, double* dt_out) {
    hydro_status st = check_grid(c, grid);
    if (st != HYDRO_OK) return st;
    if (!dt_out) return fail(c, HYDRO_EINVAL, "dt_out is NULL");
    DevCounters ctr;
    GridRun run;
    HCK(c, cudaMemcpyAsync(&ctr, c->d_ctr, sizeof ctr, cudaMemcpyDeviceToHost, c->stream));
    HCK(c, cudaMemcpyAsync(&run, &c->d_run[grid], sizeof run, cudaMemcpyDeviceToHost, c->stream));
    HCK(c, cudaStreamSynchronize(c->stream));
    double w;
    const unsigned long long bits = run.wmax[ctr.acc & 1u];
    std::memcpy(&w, &bits, sizeof w);
    *dt_out = c->cfl * c->gd[grid].h / w;
    return HYDRO_OK;
}

hydro_status hydro_get_time(hydro_ctx* c, int grid, double* t_out) {
    hydro_status st = check_grid(c, grid);
    if (st != HYDRO_OK) return st;
    if (!t_out) return fail(c, HYDRO_EINVAL, "t_out is NULL");
    HCK(c, cudaMemcpyAsync(t_out, &c->d_run[grid].t, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    HCK(c, cudaStreamSynchronize(c->stream));
    return HYDRO_OK;
}

hydro_status hydro_get_step(hydro_ctx* c, long long* step_out) {
    if (!c || !step_out) return fail(c, HYDRO_EINVAL, "ctx or step_out is NULL");
    *step_out = c->step;
    return HYDRO_OK;
}

hydro_status hydro_set_step(hydro_ctx* c, long long step) {
    if (!c) return fail(nullptr, HYDRO_EINVAL, "ctx is NULL");
    if (step < 0) return fail(c, HYDRO_EINVAL, "step < 0");
    c->step = step;
    return HYDRO_OK;
}

hydro_status hydro_set_time(hydro_ctx* c, int grid, double t) {
    hydro_status st = check_grid(c, grid);
    if (st != HYDRO_OK) return st;
    if (!std::isfinite(t)) return fail(c, HYDRO_EINVAL, "t must be finite");
    HCK(c, cudaMemcpyAsync(&c->d_run[grid].t, &t, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    HCK(c, cudaStreamSynchronize(c->stream));
    return HYDRO_OK;
}

hydro_status hydro_conservation(hydro_ctx* c, int grid, double sums[4]) {
    hydro_status st = check_grid(c, grid);
    if (st != HYDRO_OK) return st;
    if (!sums) return fail(c, HYDRO_EINVAL, "sums is NULL");
    const GridDesc& g = c->gd[grid];
    if (c->prec == 64) HCK(c, launch_conservation<double>(state_ptr<double>(c), g, c->d_rows, c->d_out4, c->stream));
    else HCK(c, launch_conservation<float>(state_ptr<float>(c), g, c->d_rows, c->d_out4, c->stream));
    HCK(c, cudaMemcpyAsync(sums, c->d_out4, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    HCK(c, cudaStreamSynchronize(c->stream));
    return HYDRO_OK;
}

hydro_status hydro_get_stats(hydro_ctx* c, hydro_stats* out) {
    if (!c || !out) return fail(c, HYDRO_EINVAL, "ctx or out is NULL");
    DevCounters ctr;
    HCK(c, cudaMemcpyAsync(&ctr, c->d_ctr, sizeof ctr, cudaMemcpyDeviceToHost, c->stream));
    HCK(c, cudaStreamSynchronize(c->stream));
    out->steps = (long long)ctr.steps;
    out->riemann_fp64 = (long long)ctr.riemann_fp64;
    out->status_flags = ctr.status;
    out->kernel_launches = c->launches;
    out->wait_site = ctr.wait_site;
    out->wait_tile = ctr.wait_tile;
    return HYDRO_OK;
}

const char* hydro_last_error(const hydro_ctx* c) {
    return c ? c->err.c_str() : g_init_error.c_str();
}

const char* hydro_version(void) { return "0.1.0"; }

}  // extern "C"
