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
// depends only on the cells i-2..i+2 of its line whatever the thread mapping:
// results are identical for every tile shape and schedule.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hydro {

// Constants of the scheme in the arithmetic type, derived once on the host.
template <class T>
struct Consts {
    T gamma;      // ratio of specific heats g
    T gm1;        // g - 1
    T inv_gm1;    // 1 / (g - 1)
    T z;          // (g - 1) / (2 g): rarefaction exponent
    T zs;         // (g + 1) / (2 g): shock-speed factor
    T G3;         // 2 g / (g - 1)
    T G4;         // 2 / (g - 1)
    T G5;         // 2 / (g + 1)
    T G6;         // (g - 1) / (g + 1)
    T G7;         // (g - 1) / 2
    T inv_g;      // 1 / g
    T rho_floor;  // density floor
    T cf2g;       // c_floor^2 / g: p >= rho * cf2g
    T pmin;       // smallest pressure of the Riemann iteration, rho_floor * cf2g
    T tol;        // Newton convergence test |p_new - p| <= tol * p_new
    int niter;    // maximum Newton iterations
};

template <class T> struct Prim { T r, u, v, p; };     // u normal, v tangential
template <class T> struct Cons { T r, mn, mt, E; };   // (rho, m_n, m_t, E)

// ----------------------------------------------------------------- math --
// IEEE double operations for T = double.  For T = float the translation
// unit is built with fast single-precision division, square root and
// power (approximate hardware instructions); see the build script.
__device__ __forceinline__ double tpow(double x, double e) { return pow(x, e); }
__device__ __forceinline__ float tpow(float x, float e) { return __powf(x, e); }
__device__ __forceinline__ double tsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float tsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double tabs(double x) { return fabs(x); }
__device__ __forceinline__ float tabs(float x) { return fabsf(x); }

// x^e with the exact value 1 for x == 1 (pow(1, e) = 1 for every e).
template <class T>
__device__ __forceinline__ T pow_or_one(T x, T e) {
    return (x == T(1)) ? T(1) : tpow(x, e);
}

// ------------------------------------------------------------- EOS -----
// Floors compare with '<' so a NaN passes through and is reported.
template <class T>
__device__ __forceinline__ Prim<T> cons_to_prim(const Consts<T>& K, const Cons<T>& U) {
    Prim<T> W;
    W.r = (U.r < K.rho_floor) ? K.rho_floor : U.r;
    const T ir = T(1) / W.r;
    W.u = U.mn * ir;
    W.v = U.mt * ir;
    T p = K.gm1 * (U.E - T(0.5) * W.r * (W.u * W.u + W.v * W.v));
    const T pm = W.r * K.cf2g;
    W.p = (p < pm) ? pm : p;
    return W;
}

// ---------------------------------------------------- slopes and trace --
// minmod(a, b): 0 unless a and b are both > 0 or both < 0, then the one of
// smaller magnitude.
template <class T>
__device__ __forceinline__ T minmod(T a, T b) {
    T r = T(0);
    if (a > T(0) && b > T(0)) r = (a < b) ? a : b;
    if (a < T(0) && b < T(0)) r = (a > b) ? a : b;
    return r;
}

// MUSCL-Hancock trace of the cell with primitive state W0 between Wm and Wp
// (§1, second order): slopes D = minmod of one-sided differences; half-step
// predictor dW = -(dt/dx)/2 A(W0) D with the primitive Jacobian rows
//   rho: u D_rho + rho D_u,  u_n: u D_u + D_p/rho,  u_t: u D_ut,
//   p: g p D_u + u D_p;
// faces WL = W0 - D/2 + dW (left), WR = W0 + D/2 + dW (right), floored.
template <class T>
__device__ __forceinline__ void trace(const Consts<T>& K, T hdtdx /* -dt/(2dx) */,
                                      const Prim<T>& Wm, const Prim<T>& W0,
                                      const Prim<T>& Wp, Prim<T>& WL, Prim<T>& WR) {
    const T Dr = minmod(W0.r - Wm.r, Wp.r - W0.r);
    const T Du = minmod(W0.u - Wm.u, Wp.u - W0.u);
    const T Dv = minmod(W0.v - Wm.v, Wp.v - W0.v);
    const T Dp = minmod(W0.p - Wm.p, Wp.p - W0.p);
    const T dr = hdtdx * (W0.u * Dr + W0.r * Du);
    const T du = hdtdx * (W0.u * Du + Dp / W0.r);
    const T dv = hdtdx * (W0.u * Dv);
    const T dp = hdtdx * (K.gamma * W0.p * Du + W0.u * Dp);
    WL.r = W0.r - T(0.5) * Dr + dr;
    WL.u = W0.u - T(0.5) * Du + du;
    WL.v = W0.v - T(0.5) * Dv + dv;
    WL.p = W0.p - T(0.5) * Dp + dp;
    WR.r = W0.r + T(0.5) * Dr + dr;
    WR.u = W0.u + T(0.5) * Du + du;
    WR.v = W0.v + T(0.5) * Dv + dv;
    WR.p = W0.p + T(0.5) * Dp + dp;
    WL.r = (WL.r < K.rho_floor) ? K.rho_floor : WL.r;
    WR.r = (WR.r < K.rho_floor) ? K.rho_floor : WR.r;
    const T pml = WL.r * K.cf2g, pmr = WR.r * K.cf2g;
    WL.p = (WL.p < pml) ? pml : WL.p;
    WR.p = (WR.p < pmr) ? pmr : WR.p;
}

// ------------------------------------------------------ Riemann solver --
// Pressure function of side K and its derivative (exact solver):
//   shock (p > p_K):   f = (p - p_K) sqrt(A/(p+B)),  A = 2/((g+1) rho_K),
//                      B = (g-1)/(g+1) p_K,  f' = sqrt(A/(p+B)) (1 - (p-p_K)/(2(p+B)))
//   rarefaction:       f = 2 c_K/(g-1) ((p/p_K)^z - 1),
//                      f' = (p/p_K)^(z-1) / (rho_K c_K)
template <class T>
__device__ __forceinline__ void pressure_fn(const Consts<T>& K, T p, T rk, T pk, T ck,
                                            T& f, T& df) {
    if (p > pk) {
        const T A = K.G5 / rk;
        const T B = K.G6 * pk;
        const T ipb = T(1) / (p + B);
        const T q = tsqrt(A * ipb);
        const T dpk = p - pk;
        f = dpk * q;
        df = q * (T(1) - T(0.5) * dpk * ipb);
    } else {
        const T r = p / pk;
        const T pz = pow_or_one(r, K.z);
        f = ck * K.G4 * (pz - T(1));
        df = pz / (r * rk * ck);
    }
}

template <class T>
struct Star { T p, u; bool floored; };

// (p*, u*) by Newton from p0 = (pL+pR)/2 - (uR-uL)(rhoL+rhoR)(cL+cR)/8, each
// iterate clamped to pmin; at most niter steps, stopping once a step changes
// p by no more than tol * p (the iterate is then converged to rounding, so
// further steps would not move it); u* = (uL+uR)/2 + (f_R(p*) - f_L(p*))/2.
template <class T>
__device__ __forceinline__ Star<T> riemann_star(const Consts<T>& K, const Prim<T>& L,
                                                const Prim<T>& R, T cl, T cr) {
    T p = T(0.5) * (L.p + R.p) - T(0.125) * (R.u - L.u) * (L.r + R.r) * (cl + cr);
    bool floored = false;
    if (p < K.pmin) { p = K.pmin; floored = true; }
    const T du = R.u - L.u;
    T fl, dfl, fr, dfr;
    for (int it = 0; it < K.niter; ++it) {
        pressure_fn(K, p, L.r, L.p, cl, fl, dfl);
        pressure_fn(K, p, R.r, R.p, cr, fr, dfr);
        T pn = p - (fl + fr + du) / (dfl + dfr);
        if (pn < K.pmin) { pn = K.pmin; floored = true; }
        const bool done = tabs(pn - p) <= K.tol * pn;
        p = pn;
        if (done) break;
    }
    pressure_fn(K, p, L.r, L.p, cl, fl, dfl);
    pressure_fn(K, p, R.r, R.p, cr, fr, dfr);
    Star<T> s;
    s.p = p;
    s.u = T(0.5) * (L.u + R.u) + T(0.5) * (fr - fl);
    s.floored = floored;
    return s;
}

// State of the Riemann solution at x/t = 0.  0 <= u* takes the left side of
// the contact (tangential velocity from the same side).  Left shock speed
// S_L = u_L - c_L sqrt(zs p*/p_L + z); rarefaction head u_L - c_L, tail
// u* - c*_L with c*_L = c_L (p*/p_L)^z.  Star densities: shock
// rho_L (p*/p_L + G6)/(G6 p*/p_L + 1), rarefaction rho_L (p*/p_L)^(1/g).
// Inside a fan at x/t = 0: c = G5 (c_L + G7 u_L), u = c (left);
// c = G5 (c_R - G7 u_R), u = -c (right); rho = rho_K (c/c_K)^G4,
// p = p_K (c/c_K)^G3.  Mirror formulas on the right.
template <class T>
__device__ __forceinline__ Prim<T> sample0(const Consts<T>& K, const Prim<T>& L,
                                           const Prim<T>& R, T cl, T cr, const Star<T>& s) {
    Prim<T> W;
    if (T(0) <= s.u) {
        W.v = L.v;
        const T pr = s.p / L.p;
        if (s.p > L.p) {
            const T sl = L.u - cl * tsqrt(K.zs * pr + K.z);
            if (T(0) <= sl) { W.r = L.r; W.u = L.u; W.p = L.p; }
            else { W.r = L.r * (pr + K.G6) / (K.G6 * pr + T(1)); W.u = s.u; W.p = s.p; }
        } else {
            const T shl = L.u - cl;
            if (T(0) <= shl) { W.r = L.r; W.u = L.u; W.p = L.p; }
            else {
                const T cml = cl * pow_or_one(pr, K.z);
                const T stl = s.u - cml;
                if (T(0) > stl) { W.r = L.r * pow_or_one(pr, K.inv_g); W.u = s.u; W.p = s.p; }
                else {
                    const T c = K.G5 * (cl + K.G7 * L.u);
                    const T cc = c / cl;
                    W.u = c;
                    W.r = L.r * tpow(cc, K.G4);
                    W.p = L.p * tpow(cc, K.G3);
                }
            }
        }
    } else {
        W.v = R.v;
        const T pr = s.p / R.p;
        if (s.p > R.p) {
            const T sr = R.u + cr * tsqrt(K.zs * pr + K.z);
            if (T(0) >= sr) { W.r = R.r; W.u = R.u; W.p = R.p; }
            else { W.r = R.r * (pr + K.G6) / (K.G6 * pr + T(1)); W.u = s.u; W.p = s.p; }
        } else {
            const T shr = R.u + cr;
            if (T(0) >= shr) { W.r = R.r; W.u = R.u; W.p = R.p; }
            else {
                const T cmr = cr * pow_or_one(pr, K.z);
                const T str = s.u + cmr;
                if (T(0) <= str) { W.r = R.r * pow_or_one(pr, K.inv_g); W.u = s.u; W.p = s.p; }
                else {
                    const T c = K.G5 * (cr - K.G7 * R.u);
                    const T cc = c / cr;
                    W.u = -c;
                    W.r = R.r * tpow(cc, K.G4);
                    W.p = R.p * tpow(cc, K.G3);
                }
            }
        }
    }
    return W;
}

// Physical flux along the normal of a primitive state.
template <class T>
__device__ __forceinline__ Cons<T> physical_flux(const Consts<T>& K, const Prim<T>& W) {
    const T E = W.p * K.inv_gm1 + T(0.5) * W.r * (W.u * W.u + W.v * W.v);
    const T m = W.r * W.u;
    Cons<T> F;
    F.r = m;
    F.mn = m * W.u + W.p;
    F.mt = m * W.v;
    F.E = W.u * (E + W.p);
    return F;
}

template <class T>
__device__ __forceinline__ T sound_speed(const Consts<T>& K, const Prim<T>& W) {
    return tsqrt(K.gamma * W.p / W.r);
}

// Godunov flux at one interface between the traced states L | R.
template <class T>
__device__ __forceinline__ Cons<T> godunov_flux_exact(const Consts<T>& K, const Prim<T>& L,
                                                      const Prim<T>& R, bool* floored) {
    const T cl = sound_speed(K, L), cr = sound_speed(K, R);
    const Star<T> s = riemann_star(K, L, R, cl, cr);
    if (floored) *floored = s.floored;
    return physical_flux(K, sample0(K, L, R, cl, cr, s));
}

}  // namespace hydro
