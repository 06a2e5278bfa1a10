// godunov.cuh -- per-cell and per-interface arithmetic of the split Godunov
// sweep (§1; stencil of Figs. 1-2; COMPUTE step of Fig. 5), templated on the
// storage/arithmetic type T (double or float).
//
//   cons_to_prim   conserved (rho, m_n, m_t, E) -> primitive (rho, u_n, u_t, p)
//   trace          minmod slopes of the primitives + MUSCL-Hancock half step
//   godunov_flux   exact Riemann solver (Newton on the pressure function from
//                  the PVRS guess), sampled at x/t = 0, physical flux there
//
// Everything here is a pure function of its arguments, so a cell's update
// depends only on the cells i-2..i+2 of its line whatever the thread mapping.
// The kernels are built without automatic multiply-add contraction and every
// fused multiply-add is written out (tfma), so each inlined copy of these
// functions rounds identically: results are bit-identical for every tile
// shape, schedule, sweep direction and kernel variant.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hydro {

// Terms of the binomial series of (1 + x)^z used for |x| <= kBinomRadius.
constexpr int kBinomTerms = 8;
constexpr double kBinomRadius = 0.01;

// Constants of the scheme in the arithmetic type, derived once on the host.
template <class T>
struct Consts {
    T gamma;      // ratio of specific heats g
    T gm1;        // g - 1
    T g_gm1;      // g / (g - 1)
    T z;          // (g - 1) / (2 g): rarefaction exponent
    T zs;         // (g + 1) / (2 g): shock-speed factor
    T G3;         // 2 g / (g - 1)
    T G4;         // 2 / (g - 1)
    T G5;         // 2 / (g + 1)
    T G6;         // (g - 1) / (g + 1)
    T G7;         // (g - 1) / 2
    T inv_g;      // 1 / g
    T hgp1;       // (g + 1) / 2
    T sqg;        // sqrt(g)
    T rho_floor;  // density floor
    T cf2g;       // c_floor^2 / g: p >= rho * cf2g
    T pmin;       // smallest pressure of the Riemann iteration, rho_floor * cf2g
    T tol;        // Newton convergence test |p_new - p| <= tol * p_new
    int niter;    // maximum Newton iterations
    int g75;      // g = 7/5: z = 1/7, G4 = 5, G3 = 7 (a 7th root and integer powers)
    int two_shock;  // Riemann solver variant: the two-shock pressure function on both sides
    int slope;      // slope variant: SLOPE_MINMOD, SLOPE_MC or SLOPE_NONE
    int char_trace; // trace variant: characteristic tracing instead of MUSCL-Hancock
                    // (both read only by code compiled with SV = true: the kernels
                    // are instantiated once for the defaults, with no test of these
                    // flags, and once for any variant)
    T bz[kBinomTerms];  // binomial coefficients C(z, k), k = 1 .. kBinomTerms
    T pz_series;        // (1 - kBinomRadius)^z: (p/p_K)^z below it came from exp2/log2
    float f_gamma, f_gm1, f_rho_floor, f_cf2g;  // FP32 copies (the FP64 CFL estimate)
};

// Scheme variants (the HYDRO options the paper leaves to its ref. [5]).
enum { SLOPE_MINMOD = 0, SLOPE_MC = 1, SLOPE_NONE = 2 };

template <class T> struct Prim { T r, u, v, p; };     // u normal, v tangential
template <class T> struct Cons { T r, mn, mt, E; };   // (rho, m_n, m_t, E)

// ----------------------------------------------------------------- math --
// T = double: IEEE operations, except division (trcp / tdiv: within 1-2 ulp,
// a third of the FP64 instructions) and powers (below: within a few ulp).
// On this GPU every FP64 instruction of a warp occupies its FP64 unit for
// as long as a fused multiply-add, however few of its lanes are active, so
// the count of FP64 instructions is the cost.  For T = float the
// translation unit is built with fast single-precision division, square
// root and power (approximate hardware instructions); see the build script.
// FP32 a / b (tdiv) is the approximate division itself, a times the
// hardware reciprocal of b, within 2 ulp for 2^-126 <= |b| <= 2^126 (above,
// it returns 0); the build's fast division adds a rescaling for such
// divisors.  The divisors here -- p F'(p) of the Newton step (a speed),
// 1 + G6 p*/p_K, (p*/p_K)^(2z) <= 1, a sound speed, and the iterate p of
// a step that reached the pressure floor (an interface the FP64
// near-vacuum pass redoes) -- stay far inside that range for pressures and speeds well
// inside the FP32 range.  Measured on the 8192^2 random-mode field: the
// same 200-step L1 density error to all digits, FP32 sweeps 2.6 % faster.
// FP64 powers through exp2(e log2 x): within a few ulp, and cheaper on the
// FP64 pipe than the extra-precise pow
__device__ __forceinline__ double tpow(double x, double e) { return exp2(e * log2(x)); }
__device__ __forceinline__ float tpow(float x, float e) { return __powf(x, e); }
__device__ __forceinline__ double tsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float tsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double trsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float trsqrt(float x) { return rsqrtf(x); }
// FP64 1/b for a positive normal b with a normal reciprocal, within 1 ulp:
// the FP32 hardware reciprocal of b's significand (relative error below
// 2^-22 with its truncation), scaled by b's exponent on the integer pipe and
// refined by one third-order Newton step, r = r0 (1 + e + e^2) with
// e = 1 - b r0 (remainder e^3 < 2^-66) -- three FP64 operations where an
// IEEE division takes about nine.  Any other b: IEEE division.
__device__ __forceinline__ double trcp(double b) {
    const unsigned hi = (unsigned)__double2hiint(b), lo = (unsigned)__double2loint(b);
    const int ex = (int)(hi >> 20);  // with the sign bit: negative b gives ex > 0x7ff
    const float mf = __uint_as_float(0x3f800000u | ((hi & 0x000fffffu) << 3) | (lo >> 29));
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(mf));
    const unsigned fb = __float_as_uint(rf);  // in (1/2, 1]
    const int er = (int)(fb >> 23) - 127 - (ex - 1023) + 1023;  // biased exponent of r0
    if (ex == 0 || ex >= 0x7ff || er <= 0 || er >= 0x7ff) return 1.0 / b;
    const double r0 = __hiloint2double((int)(((unsigned)er << 20) | ((fb & 0x7fffffu) >> 3)), (int)(fb << 29));
    const double e = fma(-b, r0, 1.0);
    return fma(r0, fma(e, e, e), r0);
}
__device__ __forceinline__ float trcp(float b) { return 1.0f / b; }
// a / b through trcp (FP64: within 2 ulp for a positive normal b)
__device__ __forceinline__ double tdiv(double a, double b) { return a * trcp(b); }
__device__ __forceinline__ float tdiv(float a, float b) {
    float r;
    asm("div.approx.ftz.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ double tabs(double x) { return fabs(x); }
__device__ __forceinline__ float tabs(float x) { return fabsf(x); }
// Comparisons on the integer pipe (an FP64 compare costs an FP64 slot).
// For a, b >= +0 and not NaN the order of the bit patterns is the order of
// the values; the callers pass pressures (at least the floor) or their
// magnitudes, and a NaN there yields a NaN result whichever branch it takes.
__device__ __forceinline__ bool gt_pos(double a, double b) {
    return __double_as_longlong(a) > __double_as_longlong(b);
}
__device__ __forceinline__ bool gt_pos(float a, float b) { return a > b; }
// |x| > b for b >= +0 not NaN, on the magnitude's bit pattern (a NaN x
// counts as greater)
__device__ __forceinline__ bool abs_gt_pos(double x, double b) {
    return ((unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull) >
           (unsigned long long)__double_as_longlong(b);
}
__device__ __forceinline__ bool abs_gt_pos(float x, float b) { return !(fabsf(x) <= b); }
__device__ __forceinline__ bool eq_pos(double a, double b) {
    return __double_as_longlong(a) == __double_as_longlong(b);
}
__device__ __forceinline__ bool eq_pos(float a, float b) { return a == b; }
// x < c for a floor c >= +0, exactly as the IEEE comparison: the signed
// order of the patterns, with a NaN of either sign excluded and -0 < +0
// false
__device__ __forceinline__ bool below_floor(double x, double c) {
    const long long ix = __double_as_longlong(x), ic = __double_as_longlong(c);
    return ix < ic && (unsigned long long)ix <= 0xfff0000000000000ull &&
           (ic != 0 || ix != (long long)0x8000000000000000ull);
}
__device__ __forceinline__ bool below_floor(float x, float c) { return x < c; }
// x raised to the floor c.  FP64: x < c selects c (a NaN x stays NaN).
// FP32 (bound by instruction issue): one max instruction, which returns c
// for a NaN x -- a NaN state is still reported through its own cell's
// update, which reads the conserved state itself.
__device__ __forceinline__ double floor_at(double x, double c) { return below_floor(x, c) ? c : x; }
__device__ __forceinline__ float floor_at(float x, float c) { return fmaxf(x, c); }
// 0 <= x and x < 0 exactly as the IEEE comparisons (a NaN is neither), on
// the bit pattern: the sign bit, with -0 counted as zero
__device__ __forceinline__ bool ge_zero(double x) {
    const long long i = __double_as_longlong(x);
    return i >= 0 ? i <= 0x7ff0000000000000ll : i == (long long)0x8000000000000000ull;
}
__device__ __forceinline__ bool ge_zero(float x) { return 0.0f <= x; }
__device__ __forceinline__ bool lt_zero(double x) {
    const long long i = __double_as_longlong(x);
    return i < 0 && i != (long long)0x8000000000000000ull && (unsigned long long)i <= 0xfff0000000000000ull;
}
__device__ __forceinline__ bool lt_zero(float x) { return x < 0.0f; }
// x == +-0 exactly as the IEEE comparison
__device__ __forceinline__ bool is_zero(double x) { return (__double_as_longlong(x) << 1) == 0; }
__device__ __forceinline__ bool is_zero(float x) { return x == 0.0f; }
__device__ __forceinline__ double tfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float tfma(float a, float b, float c) { return fmaf(a, b, c); }

// x^(1/7) for a positive normal double, within 3 ulp (a 7th root by Newton's
// method for nth roots, taken to third order):  write x = m 2^(7q) with m in
// [1, 2^7); v0 ~ m^(-1/7) from the FP32 hardware log2 and exp2 (relative
// error below 1e-6), improved by one FP32 Newton step v0 (1 + (1 - m v0^7)/7)
// (relative error below 1e-7: the FP32 roundings and m's 24-bit FP32 copy);
// h = m v0^7 - 1 with one rounding (fused multiply-add), |h| < 1e-6; then
// m^(1/7) = m v0^6 (1 + h)^(-6/7), the binomial series to h^2 (the
// remainder is below 1e-18 of an ulp's 1.1e-16) -- nine FP64 operations, no
// division.  A rounding error d in v0^6 moves the result by only d/7, since
// it enters h as well.  The exponent q is added to the result's exponent
// field.  Other x: exp2/log2.
__device__ __forceinline__ double root7(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int ex = (int)((hi >> 20) & 0x7ffu);
    if (ex == 0 || ex == 0x7ff) return exp2(log2(x) * (1.0 / 7.0));
    const int e = ex - 1023;
    const int q = (e + 1029) / 7 - 147;  // floor(e / 7) for e in [-1022, 1023]
    const int r = e - 7 * q;             // 0 .. 6
    const unsigned mant = hi & 0x000fffffu;
    const double m = __hiloint2double((int)(mant | ((unsigned)(1023 + r) << 20)), (int)lo);
    const float mf = __uint_as_float(((unsigned)(127 + r) << 23) | (mant << 3) | (lo >> 29));
    float t;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(mf));
    t = t * (-1.0f / 7.0f);
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(t));
    {  // one FP32 Newton step (t stays in [1/2, 1])
        const float t2 = t * t, t4 = t2 * t2, t7 = t4 * t2 * t;
        t = fmaf(t * (1.0f / 7.0f), fmaf(-mf, t7, 1.0f), t);
    }
    // t in [1/2, 1]: exact conversion to double on the integer pipe
    const unsigned fb = __float_as_uint(t);
    const double v0 = __hiloint2double((int)((((fb >> 23) + (1023u - 127u)) << 20) | ((fb & 0x7fffffu) >> 3)),
                                       (int)(fb << 29));
    const double v2 = v0 * v0, v3 = v2 * v0, v6 = v3 * v3, v7 = v6 * v0;
    const double h = fma(m, v7, -1.0);
    const double P = fma(h, 39.0 / 49.0, -6.0 / 7.0);  // (1+h)^(-6/7) = 1 + h P + O(h^3)
    const double base = m * v6;
    const double y = fma(base, h * P, base);
    return __hiloint2double((int)((unsigned)__double2hiint(y) + ((unsigned)q << 20)), __double2loint(y));
}

// (p / p_K)^z, given 1/p_K.  FP64 with g = 7/5: the 7th root of p/p_K.
// Other FP64: where x = (p - p_K)/p_K has |x| <= 0.01,
// the binomial series (1 + x)^z = sum_k C(z, k) x^k summed to k = 8 by
// Horner's rule; for 0 < z < 1/2 the remainder is below 0.5 * 0.01^9, far
// under one unit in the last place; p = p_K gives 1 exactly.  This is the
// common case of the Newton iteration (iterates near p_K) and costs 8 fused
// multiply-adds instead of a logarithm and an exponential.  Farther from 1,
// and in FP32 (where the power is two hardware approximations), exp2/log2.
template <class T>
__device__ __forceinline__ T pow_z(const Consts<T>& K, T p, T pK, T ip) {
    if (eq_pos(p, pK)) return T(1);
    if constexpr (sizeof(T) == 8) {
        if (K.g75) return root7(p * ip);
        const T x = (p - pK) * ip;
        if (tabs(x) <= T(kBinomRadius)) {
            T s = K.bz[kBinomTerms - 1];
#pragma unroll
            for (int k = kBinomTerms - 2; k >= 0; --k) s = tfma(s, x, K.bz[k]);
            return tfma(s, x, T(1));
        }
    }
    return tpow(p * ip, K.z);
}

// ------------------------------------------------------------- EOS -----
// Floors compare with '<' so a NaN passes through and is reported.
template <class T>
__device__ __forceinline__ Prim<T> cons_to_prim(const Consts<T>& K, const Cons<T>& U, T& ir) {
    Prim<T> W;
    W.r = floor_at(U.r, K.rho_floor);
    ir = trcp(W.r);
    W.u = U.mn * ir;
    W.v = U.mt * ir;
    // p = (g-1) E - (g-1)/2 rho |u|^2, with rho |u|^2 = m_n u_n + m_t u_t
    T p = tfma(-K.G7, tfma(U.mn, W.u, U.mt * W.v), K.gm1 * U.E);
    const T pm = W.r * K.cf2g;
    W.p = floor_at(p, pm);
    return W;
}

template <class T>
__device__ __forceinline__ Prim<T> cons_to_prim(const Consts<T>& K, const Cons<T>& U) {
    T ir;
    return cons_to_prim(K, U, ir);
}

// CFL wave speed of a cell, max(|u|, |v|) + c with c = sqrt(g p / rho);
// in FP64 through one reciprocal square root, c = sqrt(g) p / sqrt(rho p).
template <class T>
__device__ __forceinline__ T cfl_speed(const Consts<T>& K, const Cons<T>& U) {
    T ir;
    const Prim<T> w = cons_to_prim(K, U, ir);
    const T au = tabs(w.u), av = tabs(w.v);
    T c;
    if (sizeof(T) == 8) c = K.sqg * w.p * trsqrt(w.r * w.p);
    else c = tsqrt(K.gamma * w.p * ir);
    if constexpr (sizeof(T) == 4) return fmaxf(au, av) + c;  // one instruction
    return ((au > av) ? au : av) + c;
}

// ---------------------------------------------------- slopes and trace --
// minmod(a, b): 0 unless a and b are both > 0 or both < 0, then the one of
// smaller magnitude.  The sign tests run on the bit patterns (integer
// pipe); the result is exactly a or b (or +0) as in the comparison form.
__device__ __forceinline__ double minmod(double a, double b) {
    const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
    const bool take = ((ia ^ ib) >= 0) && ((ia << 1) != 0) && ((ib << 1) != 0);
    // fmin of the magnitudes on the bit patterns (a NaN loses, as in fmin)
    const unsigned long long ma = (unsigned long long)ia & 0x7fffffffffffffffull;
    const unsigned long long mb = (unsigned long long)ib & 0x7fffffffffffffffull;
    const long long m = (long long)(ma < mb ? ma : mb) | (ia & (long long)0x8000000000000000ull);
    return take ? __longlong_as_double(m) : 0.0;
}
// FP32: minmod(a, b) is the median of a, b and 0 -- four min/max
// instructions, exactly a, b or a zero, with no product to underflow.
__device__ __forceinline__ float minmod(float a, float b) {
    return fmaxf(fminf(a, b), fminf(fmaxf(a, b), 0.0f));
}

// Monotonized central slope: 0 unless a and b are both > 0 or both < 0,
// then the one of 2a, 2b and (a + b)/2 of smallest magnitude (ties go to
// the earlier of (a + b)/2, 2a, 2b: the values are then equal).  FP64
// compares the magnitudes on the integer pipe, as minmod does.
__device__ __forceinline__ double mc_slope(double a, double b) {
    const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
    if (!(((ia ^ ib) >= 0) && ((ia << 1) != 0) && ((ib << 1) != 0))) return 0.0;
    const double c = 0.5 * (a + b), a2 = 2.0 * a, b2 = 2.0 * b;
    unsigned long long m = (unsigned long long)__double_as_longlong(c) & 0x7fffffffffffffffull;
    const unsigned long long ma = (unsigned long long)__double_as_longlong(a2) & 0x7fffffffffffffffull;
    const unsigned long long mb = (unsigned long long)__double_as_longlong(b2) & 0x7fffffffffffffffull;
    m = (ma < m) ? ma : m;
    m = (mb < m) ? mb : m;
    return __longlong_as_double((long long)m | (ia & (long long)0x8000000000000000ull));
}
__device__ __forceinline__ float mc_slope(float a, float b) {
    if (!(a * b > 0.0f)) return 0.0f;
    const float c = 0.5f * (a + b);
    float m = fabsf(c);
    m = (fabsf(2.0f * a) < m) ? fabsf(2.0f * a) : m;
    m = (fabsf(2.0f * b) < m) ? fabsf(2.0f * b) : m;
    return (a > 0.0f) ? m : -m;
}

// The limited slope of the one-sided differences a, b (the variant of K).
template <class T>
__device__ __forceinline__ T limited_slope(const Consts<T>& K, T a, T b) {
    if (K.slope == SLOPE_MINMOD) return minmod(a, b);
    if (K.slope == SLOPE_MC) return mc_slope(a, b);
    return T(0);
}

// Exact shortcuts for equal states, per arithmetic type: the trace of a cell
// whose one-sided differences vanish (trace), the Riemann problem of states
// equal bit for bit
// (equal_state_flux) and, in the sweeps, uniform 5-point stencils (a cell
// whose stencil is uniform is copied).  Each saves arithmetic where the state
// is uniform and costs a few integer instructions per cell elsewhere.  FP64
// takes them all: its bottleneck is the FP64 pipe and its issue slots are
// mostly idle.  FP32 is bound by instruction issue, so only the equal-state
// flux pays there (measured: it gains 15 % on the 512-grid batch for 1-2 % on
// fully non-uniform fields, where the other two cost 5-10 %).
template <class T>
struct Shortcuts {
    static constexpr bool trace = true;
    static constexpr bool flux = true;
    static constexpr bool stencil = true;
};
template <>
struct Shortcuts<float> {
    static constexpr bool trace = false;
    static constexpr bool flux = true;
    static constexpr bool stencil = false;
};

// Bitwise equality of states on the integer pipe (+0 and -0 differ, which
// only sends such a pair down the general path): the XORs of the fields are
// OR-ed together, which compiles to a few three-input logic operations.
__device__ __forceinline__ unsigned long long diff_bits(double a, double b) {
    return (unsigned long long)(__double_as_longlong(a) ^ __double_as_longlong(b));
}
__device__ __forceinline__ unsigned diff_bits(float a, float b) {
    return (unsigned)(__float_as_int(a) ^ __float_as_int(b));
}
__device__ __forceinline__ bool same_bits(double a, double b) { return diff_bits(a, b) == 0ull; }
__device__ __forceinline__ bool same_bits(float a, float b) { return diff_bits(a, b) == 0u; }
template <class T>
__device__ __forceinline__ auto diff_bits(const Prim<T>& a, const Prim<T>& b) {
    return diff_bits(a.r, b.r) | diff_bits(a.u, b.u) | diff_bits(a.v, b.v) | diff_bits(a.p, b.p);
}
template <class T>
__device__ __forceinline__ bool same_bits(const Prim<T>& a, const Prim<T>& b) {
    return diff_bits(a, b) == 0;
}

// x > 0 for x not NaN (positive finite or +inf); FP64 on the bit pattern
// (integer pipe), FP32 by one compare.
__device__ __forceinline__ bool positive(double x) {
    const long long i = __double_as_longlong(x);
    return i > 0 && i <= 0x7ff0000000000000ll;
}
__device__ __forceinline__ bool positive(float x) { return x > 0.0f; }  // one compare; NaN fails

// Characteristic tracing (the trace variant) of the cell W0 with limited
// slopes D: the slopes split into the waves of the primitive Jacobian
// (speeds u - c, u, u, u + c; amplitudes a1 = -rho/(2c) D_u + D_p/(2c^2),
// a2 = D_rho - D_p/c^2, a3 = D_ut, a4 = rho/(2c) D_u + D_p/(2c^2); right
// eigenvectors (1, -c/rho, 0, c^2), (1, 0, 0, 0), (0, 0, 1, 0),
// (1, c/rho, 0, c^2)); the right face takes (1 - nu_k)/2 a_k r_k of the
// waves with speed > 0, the left face -(1 + nu_k)/2 a_k r_k of those with
// speed < 0 (nu_k = speed dt/dx), in wave order; floored as the trace.
template <class T>
__device__ __forceinline__ void characteristic_trace(const Consts<T>& K, T hdtdx, const Prim<T>& W0, T ir0,
                                                     T Dr, T Du, T Dv, T Dp, Prim<T>& WL, Prim<T>& WR) {
    const T c = tsqrt(K.gamma * W0.p * ir0);
    const T ic = trcp(c);
    const T ic2 = ic * ic;
    const T rc = W0.r * ic, cr = c * ir0, c2 = c * c;
    const T hp = T(0.5) * Dp * ic2;
    const T a1 = tfma(T(-0.5) * rc, Du, hp), a2 = tfma(-Dp, ic2, Dr), a4 = tfma(T(0.5) * rc, Du, hp);
    const T dtdx = T(-2) * hdtdx;
    WL = W0;
    WR = W0;
    auto wave = [&](T lam, T a, T rr, T ru, T rv, T rp) {
        if (lam > T(0)) {
            const T s = T(0.5) * tfma(-lam, dtdx, T(1)) * a;
            WR.r = tfma(s, rr, WR.r); WR.u = tfma(s, ru, WR.u); WR.v = tfma(s, rv, WR.v); WR.p = tfma(s, rp, WR.p);
        }
        if (lam < T(0)) {
            const T s = T(-0.5) * tfma(lam, dtdx, T(1)) * a;
            WL.r = tfma(s, rr, WL.r); WL.u = tfma(s, ru, WL.u); WL.v = tfma(s, rv, WL.v); WL.p = tfma(s, rp, WL.p);
        }
    };
    wave(W0.u - c, a1, T(1), -cr, T(0), c2);
    wave(W0.u, a2, T(1), T(0), T(0), T(0));
    wave(W0.u, Dv, T(0), T(0), T(1), T(0));
    wave(W0.u + c, a4, T(1), cr, T(0), c2);
    WL.r = floor_at(WL.r, K.rho_floor);
    WR.r = floor_at(WR.r, K.rho_floor);
    const T pml = WL.r * K.cf2g, pmr = WR.r * K.cf2g;
    WL.p = floor_at(WL.p, pml);
    WR.p = floor_at(WR.p, pmr);
}

// Differences of primitive states, a - b.
template <class T>
__device__ __forceinline__ Prim<T> pdiff(const Prim<T>& a, const Prim<T>& b) {
    return Prim<T>{a.r - b.r, a.u - b.u, a.v - b.v, a.p - b.p};
}

// Whether every component of both differences is +-0 (bit patterns).
__device__ __forceinline__ bool zero_diffs(const Prim<double>& a, const Prim<double>& b) {
    const unsigned long long o =
        (unsigned long long)(__double_as_longlong(a.r) | __double_as_longlong(a.u) | __double_as_longlong(a.v) |
                             __double_as_longlong(a.p) | __double_as_longlong(b.r) | __double_as_longlong(b.u) |
                             __double_as_longlong(b.v) | __double_as_longlong(b.p));
    return (o << 1) == 0ull;
}
__device__ __forceinline__ bool zero_diffs(const Prim<float>& a, const Prim<float>& b) {
    const unsigned o = (unsigned)(__float_as_int(a.r) | __float_as_int(a.u) | __float_as_int(a.v) |
                                  __float_as_int(a.p) | __float_as_int(b.r) | __float_as_int(b.u) |
                                  __float_as_int(b.v) | __float_as_int(b.p));
    return (o << 1) == 0u;
}

// MUSCL-Hancock trace of the cell with primitive state W0 (§1, second
// order), given the one-sided differences dl = W0 - W_(i-1) and
// dr = W_(i+1) - W0 (a line walk passes a cell's dr on as the next cell's
// dl): slopes D = minmod(dl, dr); half-step predictor
// dW = -(dt/dx)/2 A(W0) D with the primitive Jacobian rows
//   rho: u D_rho + rho D_u,  u_n: u D_u + D_p/rho,  u_t: u D_ut,
//   p: g p D_u + u D_p;
// faces WL = W0 - D/2 + dW (left), WR = W0 + D/2 + dW (right), floored.
//
// Where every difference is zero every slope is 0 and each face is W0 (to
// the sign of a zero component; W0 is already floored): that case returns
// W0 without the arithmetic.
template <class T, bool SV = false>
__device__ __forceinline__ void trace(const Consts<T>& K, T hdtdx /* -dt/(2dx) */, const Prim<T>& W0,
                                      T ir0 /* 1/rho_0 */, const Prim<T>& dl, const Prim<T>& dr,
                                      Prim<T>& WL, Prim<T>& WR) {
    if (Shortcuts<T>::trace && zero_diffs(dl, dr)) {
        WL = W0;
        WR = W0;
        return;
    }
    T Dr, Du, Dv, Dp;
    if (!SV || K.slope == SLOPE_MINMOD) {
        Dr = minmod(dl.r, dr.r);
        Du = minmod(dl.u, dr.u);
        Dv = minmod(dl.v, dr.v);
        Dp = minmod(dl.p, dr.p);
    } else {
        Dr = limited_slope(K, dl.r, dr.r);
        Du = limited_slope(K, dl.u, dr.u);
        Dv = limited_slope(K, dl.v, dr.v);
        Dp = limited_slope(K, dl.p, dr.p);
    }
    if (SV && K.char_trace) {
        characteristic_trace(K, hdtdx, W0, ir0, Dr, Du, Dv, Dp, WL, WR);
        return;
    }
    // the predicted centre W0 + dW, each row of dW a chain of fused
    // multiply-adds on the scaled coefficients hu = -(dt/dx)/2 u and
    // -(dt/dx)/2 rho, 1/rho, g p (11 operations), then one fused
    // multiply-add per face (W0 + dW) -+ D/2
    const T hu = hdtdx * W0.u;
    const T cr = tfma(hu, Dr, tfma(hdtdx * W0.r, Du, W0.r));
    const T cu = tfma(hu, Du, tfma(hdtdx * ir0, Dp, W0.u));
    const T cv = tfma(hu, Dv, W0.v);
    const T cp = tfma(hu, Dp, tfma((hdtdx * K.gamma) * W0.p, Du, W0.p));
    WL.r = tfma(T(-0.5), Dr, cr);
    WL.u = tfma(T(-0.5), Du, cu);
    WL.v = tfma(T(-0.5), Dv, cv);
    WL.p = tfma(T(-0.5), Dp, cp);
    WR.r = tfma(T(0.5), Dr, cr);
    WR.u = tfma(T(0.5), Du, cu);
    WR.v = tfma(T(0.5), Dv, cv);
    WR.p = tfma(T(0.5), Dp, cp);
    WL.r = floor_at(WL.r, K.rho_floor);
    WR.r = floor_at(WR.r, K.rho_floor);
    const T pml = WL.r * K.cf2g, pmr = WR.r * K.cf2g;
    WL.p = floor_at(WL.p, pml);
    WR.p = floor_at(WR.p, pmr);
}

// ------------------------------------------------------ Riemann solver --
// Exact solver: Newton iteration on the pressure function
//   F(p) = f_L(p) + f_R(p) + (u_R - u_L) = 0,
//   shock (p > p_K):  f_K = (p - p_K) q,  q = sqrt(A_K/(p + B_K)),
//                     A_K = 2/((g+1) rho_K), B_K = (g-1)/(g+1) p_K,
//                     f_K' = q (1 - (p - p_K)/(2 (p + B_K)))
//   rarefaction:      f_K = 2 c_K/(g-1) ((p/p_K)^z - 1),
//                     f_K' = (p/p_K)^z / ((p/p_K) rho_K c_K).
// The arithmetic is arranged for few divisions: each side carries 1/p_K and
// 1/(rho_K c_K) = c_K/(g p_K); 1/(p + B) = q^2/A; and every derivative is
// written f_K' = a_K/p + b_K so one division per step gives the Newton
// update  dp = F p / (a_L + a_R + p (b_L + b_R)).
template <class T>
struct Side {
    T r, u, v, p;  // traced state
    T c;           // sound speed
    T ip;          // 1 / p_K
};

template <class T>
__device__ __forceinline__ Side<T> make_side(const Consts<T>& K, const Prim<T>& W) {
    Side<T> s;
    s.r = W.r; s.u = W.u; s.v = W.v; s.p = W.p;
    if (sizeof(T) == 8) {
        // y = 1/sqrt(rho p) gives c = sqrt(g) p y and 1/p = rho y^2: one
        // reciprocal square root per side
        const T y = trsqrt(W.r * W.p);
        s.c = K.sqg * W.p * y;
        s.ip = W.r * y * y;
    } else {
        // FP32: rho p can underflow at the floors, so two reciprocals
        const T ir = T(1) / W.r;
        s.ip = T(1) / W.p;
        s.c = tsqrt(K.gamma * W.p * ir);
    }
    return s;
}

// f_K(p) with f_K' = a/p + b; pz = (p/p_K)^z on the rarefaction branch, -1 on
// the shock branch.  p == p_K gives f = 0 and pz = 1 exactly.  The
// two-shock variant takes the shock branch for every p (the Lagrangian
// shock speed of both waves, f = (p - p_K)/W_K(p), the same expression).
template <class T, bool SV = false>
__device__ __forceinline__ void pressure_fn(const Consts<T>& K, const Side<T>& s, T p,
                                            T& f, T& a, T& b, T& pz) {
    if (gt_pos(p, s.p) || (SV && K.two_shock)) {
        const T iA = K.hgp1 * s.r;                        // 1 / A_K
        const T q = trsqrt(tfma(K.G6, s.p, p) * iA);      // p + B_K = p + G6 p_K
        const T dpk = p - s.p;
        f = dpk * q;
        a = T(0);
        b = q * tfma(T(-0.5) * dpk, q * q * iA, T(1));
        pz = T(-1);
    } else {
        // f_K = 2 c_K/(g-1) (pz - 1); a_K = pz p_K/(rho_K c_K) = pz c_K / g
        pz = pow_z(K, p, s.p, s.ip);
        const T cG4 = s.c * K.G4;
        f = tfma(cG4, pz, -cG4);
        a = pz * (s.c * K.inv_g);
        b = T(0);
    }
}

template <class T>
struct Star {
    T p, u;
    T pzl, pzr;    // (p*/p_K)^z of each side, -1 where not evaluated
    bool floored;  // the iterate reached the pressure floor
    int iters;     // pressure-function evaluations of each side
};

// (p*, u*) by Newton from the PVRS estimate
//   p0 = (pL+pR)/2 - (uR-uL)(rhoL+rhoR)(cL+cR)/8,
// every iterate clamped to pmin, at most niter steps.  The iteration stops
// once a step changes p by no more than tol * p.  Newton's method converges
// quadratically: after a step of relative size d the error of the new
// iterate is about (k/2) d^2, where k = p F''/F' is of order one for these
// pressure functions (at most 1 for the shock branch, 1 - z for the
// rarefaction branch).  tol = 1e-8 (FP64) and 3e-4 (FP32) therefore leave an
// error below the type's rounding, and f_K and (p/p_K)^z at the new iterate
// follow from their values at the previous one by a first-order update (the
// neglected term is of the same order).  Without convergence f_K is
// evaluated again at the last iterate.  u* = (uL+uR)/2 + (f_R(p*) - f_L(p*))/2.
template <class T, bool SV = false>
__device__ __forceinline__ Star<T> riemann_star(const Consts<T>& K, const Side<T>& L,
                                                const Side<T>& R) {
    T p = tfma(T(-0.125) * (R.u - L.u), (L.r + R.r) * (L.c + R.c), T(0.5) * (L.p + R.p));
    bool floored = false;
    if (below_floor(p, K.pmin)) { p = K.pmin; floored = true; }
    const T du = R.u - L.u;
    T fl, al, bl, pzl, fr, ar, br, pzr;
    bool conv = false;
    int iters = K.niter + 1;
    for (int it = 0; it < K.niter; ++it) {
        pressure_fn<T, SV>(K, L, p, fl, al, bl, pzl);
        pressure_fn<T, SV>(K, R, p, fr, ar, br, pzr);
        const T F = fl + fr + du;
        // Newton step / p (F == 0: p is the root, the step is exactly 0)
        const T g = is_zero(F) ? T(0) : tdiv(F, tfma(p, bl + br, al + ar));
        T d = g * p;                                    // the step p - p_new
        T pn = p - d;
        T rel = g;                                      // d / p
        if (below_floor(pn, K.pmin)) { pn = K.pmin; floored = true; d = p - pn; rel = tdiv(d, p); }
        if (!abs_gt_pos(rel, K.tol)) {
            if (!is_zero(d)) {
                // f_K(p - d) = f_K(p) - (a_K/p + b_K) d; (p/p_K)^z (1 - z d/p)
                fl = tfma(-al, rel, tfma(-bl, d, fl));
                fr = tfma(-ar, rel, tfma(-br, d, fr));
                const T zr = K.z * rel;
                if (positive(pzl)) pzl = tfma(-zr, pzl, pzl);
                if (positive(pzr)) pzr = tfma(-zr, pzr, pzr);
            }
            p = pn;
            conv = true;
            iters = it + 1;
            break;
        }
        p = pn;
    }
    if (!conv) {
        pressure_fn<T, SV>(K, L, p, fl, al, bl, pzl);
        pressure_fn<T, SV>(K, R, p, fr, ar, br, pzr);
    }
    Star<T> st;
    st.p = p;
    st.u = T(0.5) * ((fr - fl) + (L.u + R.u));
    st.pzl = pzl;
    st.pzr = pzr;
    st.floored = floored;
    st.iters = iters;
    return st;
}

// State of the Riemann solution at x/t = 0.  0 <= u* takes the left side of
// the contact (tangential velocity from the same side).  Left shock speed
// S_L = u_L - c_L sqrt(zs p*/p_L + z); rarefaction head u_L - c_L, tail
// u* - c*_L with c*_L = c_L (p*/p_L)^z.  Star densities: shock
// rho_L (p*/p_L + G6)/(G6 p*/p_L + 1), rarefaction
// rho_L (p*/p_L)^(1/g) = rho_L (p*/p_L) / ((p*/p_L)^z)^2.  Inside a fan at
// x/t = 0: c = G5 (c_L + G7 u_L), u = c (left); c = G5 (c_R - G7 u_R), u = -c
// (right); rho = rho_K (c/c_K)^G4, p = p_K (c/c_K)^G3.
template <class T>
__device__ __forceinline__ Prim<T> sample_side(const Consts<T>& K, const Side<T>& S, T pz,
                                               const Star<T>& st, T sgn) {
    // sgn = +1 for the left side, -1 for the right side (mirror formulas)
    Prim<T> W;
    W.v = S.v;
    const bool one = eq_pos(st.p, S.p);
    const T pr = one ? T(1) : st.p * S.ip;
    if (gt_pos(st.p, S.p)) {
        // sgn S_K = m - c_K sqrt(zs pr + z) with m = sgn u_K: it is >= 0 (the
        // shock moves away from x/t = 0 and the side's own state is sampled)
        // exactly when m >= 0 and m^2 >= c_K^2 (zs pr + z), which needs no
        // square root.  At a tie the two forms may round apart, but the flux
        // is continuous across a stationary shock (Rankine-Hugoniot with
        // zero speed), so either choice gives the same flux to rounding.
        const T m = sgn * S.u;
        if (ge_zero(m) && !gt_pos(S.c * S.c * tfma(K.zs, pr, K.z), m * m)) { W.r = S.r; W.u = S.u; W.p = S.p; }
        else { W.r = tdiv(S.r * (pr + K.G6), tfma(K.G6, pr, T(1))); W.u = st.u; W.p = st.p; }
    } else {
        const T hk = sgn * S.u - S.c;                              // head
        if (ge_zero(hk)) { W.r = S.r; W.u = S.u; W.p = S.p; }
        else {
            if (lt_zero(pz)) pz = pow_z(K, st.p, S.p, S.ip);
            const T tk = tfma(-S.c, pz, sgn * st.u);               // tail
            if (lt_zero(tk)) {
                W.r = one ? S.r : tdiv(S.r * pr, pz * pz);
                W.u = st.u; W.p = st.p;
            } else {
                const T c = K.G5 * tfma(sgn * K.G7, S.u, S.c);
                const T cc = tdiv(c, S.c);
                W.u = sgn * c;
                if (K.g75) {  // (c/c_K)^5 and (c/c_K)^7
                    const T c2 = cc * cc, c5 = c2 * c2 * cc;
                    W.r = S.r * c5;
                    W.p = S.p * (c5 * c2);
                } else {
                    W.r = S.r * tpow(cc, K.G4);
                    W.p = S.p * tpow(cc, K.G3);
                }
            }
        }
    }
    return W;
}

template <class T>
__device__ __forceinline__ Prim<T> sample0(const Consts<T>& K, const Side<T>& L,
                                           const Side<T>& R, const Star<T>& st) {
    if (ge_zero(st.u)) return sample_side(K, L, st.pzl, st, T(1));
    return sample_side(K, R, st.pzr, st, T(-1));
}

// Physical flux along the normal of a primitive state.
template <class T>
__device__ __forceinline__ Cons<T> physical_flux(const Consts<T>& K, const Prim<T>& W) {
    // E + p = rho |u|^2 / 2 + g/(g-1) p
    const T q2 = tfma(W.u, W.u, W.v * W.v);
    const T m = W.r * W.u;
    Cons<T> F;
    F.r = m;
    F.mn = tfma(m, W.u, W.p);
    F.mt = m * W.v;
    F.E = W.u * tfma(T(0.5) * W.r, q2, W.p * K.g_gm1);
    return F;
}

template <class T>
__device__ __forceinline__ T sound_speed(const Consts<T>& K, const Prim<T>& W) {
    return tsqrt(K.gamma * W.p / W.r);
}

// Work of a cell whose interface has equal states (solve_work units): its
// conversion, update and physical flux.
constexpr unsigned kEqualStateWork = 40u;

// A rough count of the FP64 operations of a cell and its interface solve,
// used only to schedule work (adaptive tiles): a fixed part (conversion,
// trace, update, sides, guess, sampling, flux), and per evaluation of the
// pressure functions the Newton update and both sides, where a rarefaction
// power far from p_K (exp2/log2) costs about four times the series near it.
template <class T>
__device__ __forceinline__ unsigned solve_work(const Consts<T>& K, const Star<T>& s) {
    // (on the integer pipe in FP64: both operands of gt_pos are >= +0 there)
    const unsigned pl = (positive(s.pzl) && gt_pos(K.pz_series, s.pzl)) ? 40u : 0u;
    const unsigned pr = (positive(s.pzr) && gt_pos(K.pz_series, s.pzr)) ? 40u : 0u;
    return 140u + (unsigned)s.iters * (40u + pl + pr);
}

// Equal states (bit for bit): the Riemann problem's solution is that state
// everywhere, so the flux is its physical flux.  The general path gives the
// same bits: p* = p and f_K = 0 exactly, u* = (u + u)/2 (which turns -0 into
// +0, reproduced here), and the sampling returns the state.
template <class T>
__device__ __forceinline__ Cons<T> equal_state_flux(const Consts<T>& K, Prim<T> W) {
    if (same_bits(W.u, -T(0))) W.u = T(0);
    return physical_flux(K, W);
}

// Godunov flux at one interface between the traced states L | R.
template <class T, bool SV = false>
__device__ __forceinline__ Cons<T> godunov_flux_exact(const Consts<T>& K, const Prim<T>& WL,
                                                      const Prim<T>& WR, bool* floored,
                                                      unsigned* work = nullptr) {
    if (Shortcuts<T>::flux && same_bits(WL, WR)) {
        if (floored) *floored = false;
        if (work) *work = kEqualStateWork;
        return equal_state_flux(K, WL);
    }
    const Side<T> L = make_side(K, WL), R = make_side(K, WR);
    const Star<T> s = riemann_star<T, SV>(K, L, R);
    if (floored) *floored = s.floored;
    if (work) *work = solve_work(K, s);
    return physical_flux(K, sample0(K, L, R, s));
}

}  // namespace hydro
