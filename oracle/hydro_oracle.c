/*
 * hydro_oracle.c -- plain, single-threaded FP64 CPU oracle for the directionally
 * split second-order Godunov scheme of the HYDRO mini-application (§1).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the package's
 * smoke check and the benchmark's CPU-baseline leg may load this file's
 * library.  It shares no code, header, table or constant with the CUDA path,
 * and the CUDA path never calls it.
 *
 * What it computes (the paper states the structure; the arithmetic of each
 * stage is the textbook definition it refers to through its ref. [4]/[5]):
 *
 *   for each time step (§1, Fig. 5):
 *       dt = C h / max_cells( max(|u|,|v|) + c )                 (CFL)
 *       for each direction d in (x, y) on even steps, (y, x) on odd steps:
 *           apply boundary conditions along d            (Fig. 5, first item)
 *           for each line along d (row for x, column for y):
 *               READ    copy the line, 2 ghost cells per side, into a
 *                       1D buffer                        (Fig. 5, step 1)
 *               COMPUTE primitives, limited slopes, MUSCL-Hancock trace,
 *                       Riemann problem at every interface, interface
 *                       fluxes, conservative update      (Fig. 5, step 2)
 *               WRITE   copy the new values back         (Fig. 5, step 3)
 *
 * The update of a cell along d reads exactly the cells i-2..i+2 of its line
 * (Figs. 1-2).  Every numeric choice the paper leaves open (exact Newton
 * Riemann solver with 10 iterations from the PVRS guess, minmod slopes on the
 * primitive variables, primitive-form MUSCL-Hancock trace, ghost refresh before
 * each sweep, tie-break "0 <= u* samples the left side", floors) is fixed
 * in the comments of the function that makes it.
 *
 * Storage of a state handed across the API: interior cells only, SoA planes
 * U[4][ny][nx] in the order (rho, rho*u, rho*v, E), x fastest, FP64.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared hydro_oracle.c -lm
 * (no FMA contraction, so x86 and Arm hosts give the same bits); the same
 * source with -fopenmp shares the lines of each sweep among threads, with
 * bit-identical results (see sweep()).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double gamma;      /* ratio of specific heats */
    double cfl;        /* Courant number C in dt = C h / w */
    int niter;         /* Newton iterations of the Riemann solver (10) */
    double rho_floor;  /* density floor */
    double c_floor;    /* sound-speed floor: p >= rho c_floor^2 / gamma */
    int riemann;       /* ORC_RIEMANN_EXACT or ORC_RIEMANN_TWO_SHOCK */
    int slope;         /* ORC_SLOPE_MINMOD, ORC_SLOPE_MC or ORC_SLOPE_NONE */
    int trace;         /* ORC_TRACE_MUSCL_HANCOCK or ORC_TRACE_CHARACTERISTIC */
} orc_params;

/* Scheme variants (the HYDRO options the paper leaves to its ref. [5]):
 * the Riemann solver's pressure function -- exact (shock and rarefaction
 * branches) or the two-shock approximation (the shock branch on both
 * sides, whatever the sign of p - p_K) -- and the limited slope of the
 * MUSCL reconstruction -- minmod, monotonized central, or none (first-order
 * Godunov).  The defaults are the exact solver and minmod. */
enum { ORC_RIEMANN_EXACT = 0, ORC_RIEMANN_TWO_SHOCK = 1 };
enum { ORC_SLOPE_MINMOD = 0, ORC_SLOPE_MC = 1, ORC_SLOPE_NONE = 2 };
enum { ORC_TRACE_MUSCL_HANCOCK = 0, ORC_TRACE_CHARACTERISTIC = 1 };

enum { ORC_BC_REFLECT = 0, ORC_BC_TRANSMISSIVE = 1, ORC_BC_PERIODIC = 2 };
enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_ENEGATIVE = 4 };

/* --------------------------------------------------------------------------
 * Equation of state and conversions (ideal gas, p = (gamma-1) rho e).
 * A state along a line is (rho, m_n, m_t, E): m_n is the momentum component
 * normal to the sweep direction's interfaces, m_t the tangential one.
 * Primitive variables W = (rho, u_n, u_t, p).
 * ------------------------------------------------------------------------ */

/* Floors compare with '<' so that a NaN passes through and is reported. */
static double floor_rho(const orc_params *P, double rho)
{
    return (rho < P->rho_floor) ? P->rho_floor : rho;
}

static double floor_p(const orc_params *P, double rho, double p)
{
    double pmin = rho * P->c_floor * P->c_floor / P->gamma;
    return (p < pmin) ? pmin : p;
}

/* Smallest pressure the Riemann iteration may reach: the floor of the
 * lightest admissible state. */
static double riemann_pmin(const orc_params *P)
{
    return P->rho_floor * P->c_floor * P->c_floor / P->gamma;
}

/* conserved -> primitive (Fig. 5, "compute primitive variables") */
static void cons_to_prim(const orc_params *P, const double U[4], double W[4])
{
    double rho = floor_rho(P, U[0]);
    double un = U[1] / rho;
    double ut = U[2] / rho;
    double eint = U[3] - 0.5 * rho * (un * un + ut * ut);
    W[0] = rho;
    W[1] = un;
    W[2] = ut;
    W[3] = floor_p(P, rho, (P->gamma - 1.0) * eint);
}

static double sound_speed(const orc_params *P, const double W[4])
{
    return sqrt(P->gamma * W[3] / W[0]);
}

/* Physical flux of the Euler equations along the normal direction, evaluated
 * on a primitive state: (rho u_n, rho u_n^2 + p, rho u_n u_t, u_n (E + p)). */
static void physical_flux(const orc_params *P, const double W[4], double F[4])
{
    double rho = W[0], un = W[1], ut = W[2], p = W[3];
    double E = p / (P->gamma - 1.0) + 0.5 * rho * (un * un + ut * ut);
    F[0] = rho * un;
    F[1] = rho * un * un + p;
    F[2] = rho * un * ut;
    F[3] = un * (E + p);
}

/* --------------------------------------------------------------------------
 * Limited slopes and MUSCL-Hancock trace (second order in space and time, §1).
 * ------------------------------------------------------------------------ */

/* minmod(a, b): 0 when the signs differ or either is 0, else the argument of
 * smaller magnitude. */
static double minmod(double a, double b)
{
    if (a > 0.0 && b > 0.0) return (a < b) ? a : b;
    if (a < 0.0 && b < 0.0) return (a > b) ? a : b;
    return 0.0;
}

/* Monotonized central slope of the one-sided differences a, b: 0 when
 * their signs differ or either is 0, else the one of smallest magnitude
 * among 2a, 2b and (a + b)/2, with their common sign. */
static double mc_slope(double a, double b)
{
    if (!((a > 0.0 && b > 0.0) || (a < 0.0 && b < 0.0))) return 0.0;
    double c = 0.5 * (a + b);
    double m = fabs(c);
    if (fabs(2.0 * a) < m) m = fabs(2.0 * a);
    if (fabs(2.0 * b) < m) m = fabs(2.0 * b);
    return (a > 0.0) ? m : -m;
}

static double limited_slope(const orc_params *P, double a, double b)
{
    if (P->slope == ORC_SLOPE_MC) return mc_slope(a, b);
    if (P->slope == ORC_SLOPE_NONE) return 0.0;
    return minmod(a, b);
}

/* Trace of cell i from its primitive neighbours Wm = W_{i-1}, W0 = W_i,
 * Wp = W_{i+1}.  Slopes D = minmod of the one-sided differences of each
 * primitive; half-step predictor dW = -(dt/dx)/2 * A(W_i) D with the
 * primitive-variable Jacobian A of the 1D Euler equations (rows
 * rho: u D_rho + rho D_u;  u_n: u D_u + D_p / rho;  u_t: u D_ut;
 * p: gamma p D_u + u D_p).  Face states: WL = W - D/2 + dW at the cell's
 * left face, WR = W + D/2 + dW at its right face, each floored. */
static void characteristic_trace(const orc_params *P, double dtdx,
                                 const double W0[4], const double D[4],
                                 double WL[4], double WR[4]);

static void muscl_hancock_trace(const orc_params *P, double dtdx,
                                const double Wm[4], const double W0[4],
                                const double Wp[4], double WL[4], double WR[4])
{
    double D[4], dW[4];
    for (int q = 0; q < 4; q++) D[q] = limited_slope(P, W0[q] - Wm[q], Wp[q] - W0[q]);
    if (P->trace == ORC_TRACE_CHARACTERISTIC) {
        characteristic_trace(P, dtdx, W0, D, WL, WR);
        return;
    }

    double rho = W0[0], u = W0[1], p = W0[3];
    double half = -0.5 * dtdx;
    dW[0] = half * (u * D[0] + rho * D[1]);
    dW[1] = half * (u * D[1] + D[3] / rho);
    dW[2] = half * (u * D[2]);
    dW[3] = half * (P->gamma * p * D[1] + u * D[3]);

    for (int q = 0; q < 4; q++) {
        WL[q] = W0[q] - 0.5 * D[q] + dW[q];
        WR[q] = W0[q] + 0.5 * D[q] + dW[q];
    }
    WL[0] = floor_rho(P, WL[0]);
    WR[0] = floor_rho(P, WR[0]);
    WL[3] = floor_p(P, WL[0], WL[3]);
    WR[3] = floor_p(P, WR[0], WR[3]);
}

/* Characteristic tracing (the trace variant).  The limited slopes D are
 * split into the waves of the primitive Jacobian A(W) (speeds u - c, u, u,
 * u + c): amplitudes
 *   a1 = -rho/(2c) D_u + D_p/(2c^2),  a2 = D_rho - D_p/c^2,
 *   a3 = D_ut,                        a4 =  rho/(2c) D_u + D_p/(2c^2),
 * right eigenvectors r1 = (1, -c/rho, 0, c^2), r2 = (1, 0, 0, 0),
 * r3 = (0, 0, 1, 0), r4 = (1, c/rho, 0, c^2).  The MUSCL-Hancock faces are
 * W + 1/2 sum_k (1 - nu_k) a_k r_k (right) and W - 1/2 sum_k (1 + nu_k) a_k
 * r_k (left), nu_k = lambda_k dt/dx, over every wave; here each face takes
 * only the waves moving toward it: lambda_k > 0 for the right face,
 * lambda_k < 0 for the left one (a wave at rest reaches neither).  Faces
 * floored as in the MUSCL-Hancock trace. */
static void characteristic_trace(const orc_params *P, double dtdx,
                                 const double W0[4], const double D[4],
                                 double WL[4], double WR[4])
{
    double rho = W0[0], u = W0[1], p = W0[3];
    double c = sound_speed(P, W0);
    double a[4], lam[4], r[4][4];
    a[0] = -rho / (2.0 * c) * D[1] + D[3] / (2.0 * c * c);
    a[1] = D[0] - D[3] / (c * c);
    a[2] = D[2];
    a[3] = rho / (2.0 * c) * D[1] + D[3] / (2.0 * c * c);
    lam[0] = u - c; lam[1] = u; lam[2] = u; lam[3] = u + c;
    double r1[4] = {1.0, -c / rho, 0.0, c * c}, r2[4] = {1.0, 0.0, 0.0, 0.0};
    double r3[4] = {0.0, 0.0, 1.0, 0.0}, r4[4] = {1.0, c / rho, 0.0, c * c};
    for (int q = 0; q < 4; q++) {
        r[0][q] = r1[q]; r[1][q] = r2[q]; r[2][q] = r3[q]; r[3][q] = r4[q];
    }
    (void)p;
    for (int q = 0; q < 4; q++) {
        WL[q] = W0[q];
        WR[q] = W0[q];
    }
    for (int k = 0; k < 4; k++) {
        double nu = lam[k] * dtdx;
        for (int q = 0; q < 4; q++) {
            if (lam[k] > 0.0) WR[q] += 0.5 * (1.0 - nu) * a[k] * r[k][q];
            if (lam[k] < 0.0) WL[q] -= 0.5 * (1.0 + nu) * a[k] * r[k][q];
        }
    }
    WL[0] = floor_rho(P, WL[0]);
    WR[0] = floor_rho(P, WR[0]);
    WL[3] = floor_p(P, WL[0], WL[3]);
    WR[3] = floor_p(P, WR[0], WR[3]);
}

/* --------------------------------------------------------------------------
 * Exact Riemann solver (§1 and its ref. [4]): Newton iteration on the
 * pressure function  f_L(p) + f_R(p) + (u_R - u_L) = 0.
 * ------------------------------------------------------------------------ */

/* f_K(p) and f_K'(p) for the state K = (rho_K, p_K, c_K).
 * Shock branch (p > p_K):  f = (p - p_K) sqrt(A_K / (p + B_K)),
 *   A_K = 2 / ((gamma+1) rho_K),  B_K = (gamma-1)/(gamma+1) p_K,
 *   f' = sqrt(A_K/(p+B_K)) (1 - (p - p_K) / (2 (B_K + p))).
 * Rarefaction branch (p <= p_K):
 *   f = 2 c_K/(gamma-1) ((p/p_K)^((gamma-1)/(2 gamma)) - 1),
 *   f' = (p/p_K)^(-(gamma+1)/(2 gamma)) / (rho_K c_K).
 * The two-shock approximation takes the shock branch for every p: the
 * Lagrangian shock speed W_K = sqrt(gamma p_K rho_K (1 + (gamma+1)/(2 gamma)
 * (p - p_K)/p_K)) of both waves, f = (p - p_K)/W_K (the same expression). */
static void pressure_function(const orc_params *P, double p, double rk,
                              double pk, double ck, double *f, double *df)
{
    double g = P->gamma;
    if (p > pk || P->riemann == ORC_RIEMANN_TWO_SHOCK) {
        double A = 2.0 / ((g + 1.0) * rk);
        double B = (g - 1.0) / (g + 1.0) * pk;
        double q = sqrt(A / (p + B));
        *f = (p - pk) * q;
        *df = q * (1.0 - 0.5 * (p - pk) / (B + p));
    } else {
        double r = p / pk;
        *f = 2.0 * ck / (g - 1.0) * (pow(r, (g - 1.0) / (2.0 * g)) - 1.0);
        *df = 1.0 / (rk * ck) * pow(r, -(g + 1.0) / (2.0 * g));
    }
}

/* Star state (p*, u*) between WL and WR.  Start: the primitive-variable
 * (PVRS) estimate p0 = (pL+pR)/2 - (uR-uL)(rhoL+rhoR)(cL+cR)/8, clamped to
 * the floor.  Then exactly P->niter Newton steps, each clamped to the floor
 * (no vacuum state is formed: a vacuum-generating pair drives p* to the
 * floor).  u* = (uL+uR)/2 + (f_R(p*) - f_L(p*))/2. */
void orc_riemann_star(const orc_params *P, const double WL[4],
                      const double WR[4], double *pstar, double *ustar)
{
    double rl = WL[0], ul = WL[1], pl = WL[3];
    double rr = WR[0], ur = WR[1], pr = WR[3];
    double cl = sound_speed(P, WL), cr = sound_speed(P, WR);
    double pmin = riemann_pmin(P);

    double p = 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr);
    if (p < pmin) p = pmin;

    double fl, dfl, fr, dfr;
    for (int it = 0; it < P->niter; it++) {
        pressure_function(P, p, rl, pl, cl, &fl, &dfl);
        pressure_function(P, p, rr, pr, cr, &fr, &dfr);
        p = p - (fl + fr + (ur - ul)) / (dfl + dfr);
        if (p < pmin) p = pmin;
    }
    pressure_function(P, p, rl, pl, cl, &fl, &dfl);
    pressure_function(P, p, rr, pr, cr, &fr, &dfr);
    *pstar = p;
    *ustar = 0.5 * (ul + ur) + 0.5 * (fr - fl);
}

/* Sample the self-similar solution of the Riemann problem at xi = x/t.
 * Left of the contact when xi <= u* (so xi = 0 with u* = 0 takes the left
 * side); the tangential velocity is carried by the contact and comes from
 * the same side.  Waves: shock speeds
 *   S_L = u_L - c_L sqrt((g+1)/(2g) p* / p_L + (g-1)/(2g)),
 *   S_R = u_R + c_R sqrt((g+1)/(2g) p* / p_R + (g-1)/(2g));
 * rarefaction head/tail u_L - c_L / u* - c*_L (left) and u_R + c_R /
 * u* + c*_R (right), c*_K = c_K (p* / p_K)^((g-1)/(2g)).  Star densities:
 * shock rho*_K = rho_K (p* / p_K + G6)/(G6 p* / p_K + 1), G6 = (g-1)/(g+1);
 * rarefaction rho*_K = rho_K (p* / p_K)^(1/g).  Inside a fan the state is
 * fixed by the Riemann invariant and the isentrope:
 *   left:  c = 2/(g+1) (c_L + (g-1)/2 (u_L - xi)),  u = xi + c,
 *   right: c = 2/(g+1) (c_R - (g-1)/2 (u_R - xi)),  u = xi - c,
 * rho = rho_K (c/c_K)^(2/(g-1)),  p = p_K (c/c_K)^(2g/(g-1)). */
void orc_sample(const orc_params *P, const double WL[4], const double WR[4],
                double pstar, double ustar, double xi, double W[4])
{
    double g = P->gamma;
    double G6 = (g - 1.0) / (g + 1.0);
    double z = (g - 1.0) / (2.0 * g);

    if (xi <= ustar) {
        double rl = WL[0], ul = WL[1], pl = WL[3], cl = sound_speed(P, WL);
        W[2] = WL[2];
        if (pstar > pl) {
            double sl = ul - cl * sqrt((g + 1.0) / (2.0 * g) * pstar / pl + z);
            if (xi <= sl) {
                W[0] = rl; W[1] = ul; W[3] = pl;
            } else {
                double pr_ = pstar / pl;
                W[0] = rl * (pr_ + G6) / (G6 * pr_ + 1.0);
                W[1] = ustar; W[3] = pstar;
            }
        } else {
            double shl = ul - cl;
            if (xi <= shl) {
                W[0] = rl; W[1] = ul; W[3] = pl;
            } else {
                double cml = cl * pow(pstar / pl, z);
                double stl = ustar - cml;
                if (xi > stl) {
                    W[0] = rl * pow(pstar / pl, 1.0 / g);
                    W[1] = ustar; W[3] = pstar;
                } else {
                    double c = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * (ul - xi));
                    W[1] = xi + c;
                    W[0] = rl * pow(c / cl, 2.0 / (g - 1.0));
                    W[3] = pl * pow(c / cl, 2.0 * g / (g - 1.0));
                }
            }
        }
    } else {
        double rr = WR[0], ur = WR[1], pr = WR[3], cr = sound_speed(P, WR);
        W[2] = WR[2];
        if (pstar > pr) {
            double sr = ur + cr * sqrt((g + 1.0) / (2.0 * g) * pstar / pr + z);
            if (xi >= sr) {
                W[0] = rr; W[1] = ur; W[3] = pr;
            } else {
                double pr_ = pstar / pr;
                W[0] = rr * (pr_ + G6) / (G6 * pr_ + 1.0);
                W[1] = ustar; W[3] = pstar;
            }
        } else {
            double shr = ur + cr;
            if (xi >= shr) {
                W[0] = rr; W[1] = ur; W[3] = pr;
            } else {
                double cmr = cr * pow(pstar / pr, z);
                double str = ustar + cmr;
                if (xi <= str) {
                    W[0] = rr * pow(pstar / pr, 1.0 / g);
                    W[1] = ustar; W[3] = pstar;
                } else {
                    double c = 2.0 / (g + 1.0) * (cr - 0.5 * (g - 1.0) * (ur - xi));
                    W[1] = xi - c;
                    W[0] = rr * pow(c / cr, 2.0 / (g - 1.0));
                    W[3] = pr * pow(c / cr, 2.0 * g / (g - 1.0));
                }
            }
        }
    }
}

/* Godunov flux at one interface: solve the Riemann problem between the
 * traced states, sample it at x/t = 0, take the physical flux there. */
void orc_interface_flux(const orc_params *P, const double WL[4],
                        const double WR[4], double F[4])
{
    double ps, us, W[4];
    orc_riemann_star(P, WL, WR, &ps, &us);
    orc_sample(P, WL, WR, ps, us, 0.0, W);
    physical_flux(P, W, F);
}

/* --------------------------------------------------------------------------
 * One line: COMPUTE of Fig. 5.  `line` holds n+4 conserved states
 * (rho, m_n, m_t, E) for the cells -2 .. n+1 (index = cell + 2); `out`
 * receives the n updated interior states.
 * ------------------------------------------------------------------------ */
static int godunov_line(const orc_params *P, int n, double dtdx,
                        const double (*line)[4], double (*out)[4])
{
    int nb = n + 4;
    double (*W)[4] = malloc(sizeof(double[4]) * (size_t)nb);
    double (*WL)[4] = malloc(sizeof(double[4]) * (size_t)nb);
    double (*WR)[4] = malloc(sizeof(double[4]) * (size_t)nb);
    double (*F)[4] = malloc(sizeof(double[4]) * (size_t)(n + 1));
    if (!W || !WL || !WR || !F) {
        free(W); free(WL); free(WR); free(F);
        return ORC_ENOMEM;
    }

    /* primitive variables of every cell of the buffer */
    for (int b = 0; b < nb; b++) cons_to_prim(P, line[b], W[b]);

    /* slopes and trace for cells -1 .. n (buffer 1 .. n+2) */
    for (int b = 1; b <= n + 2; b++)
        muscl_hancock_trace(P, dtdx, W[b - 1], W[b], W[b + 1], WL[b], WR[b]);

    /* fluxes at interfaces i-1/2, i = 0 .. n: between cells i-1 and i */
    for (int i = 0; i <= n; i++)
        orc_interface_flux(P, WR[i + 1], WL[i + 2], F[i]);

    /* conservative update of the interior cells */
    for (int i = 0; i < n; i++)
        for (int q = 0; q < 4; q++)
            out[i][q] = line[i + 2][q] - dtdx * (F[i + 1][q] - F[i][q]);

    free(W); free(WL); free(WR); free(F);
    return ORC_OK;
}

/* --------------------------------------------------------------------------
 * Grid with 2 ghost layers on each side: G[4][ny+4][nx+4], x fastest.
 * ------------------------------------------------------------------------ */
typedef struct {
    int nx, ny, sx;      /* interior size, row stride = nx + 4 */
    size_t plane;        /* (ny + 4) * (nx + 4) */
    double *v;
} grid_t;

static double *gat(grid_t *g, int q, int i, int j)
{
    /* i, j: interior cell indices, -2 .. n+1 */
    return &g->v[(size_t)q * g->plane + (size_t)(j + 2) * g->sx + (size_t)(i + 2)];
}

/* Source cell of ghost index k (k < 0 or k >= n) along a line of n cells,
 * and whether the normal momentum flips sign. */
static int ghost_source(int bc_lo, int bc_hi, int n, int k, int *flip)
{
    int bc = (k < 0) ? bc_lo : bc_hi;
    *flip = 0;
    if (bc == ORC_BC_PERIODIC) return (k < 0) ? k + n : k - n;
    if (bc == ORC_BC_REFLECT) *flip = 1;
    /* reflective and transmissive: mirror image about the boundary face */
    return (k < 0) ? -1 - k : 2 * n - 1 - k;
}

/* Boundary conditions along direction dir (Fig. 5, "Apply boundary
 * conditions"), refreshed from the current state before each sweep.  Only
 * the two ghost layers along dir are written; corners are never read. */
static void apply_bc(grid_t *g, const int bc[4], int dir)
{
    if (dir == 0) {
        int n = g->nx;
        for (int j = 0; j < g->ny; j++)
            for (int k = -2; k < n + 2; k++) {
                if (k >= 0 && k < n) continue;
                int flip, s = ghost_source(bc[0], bc[1], n, k, &flip);
                for (int q = 0; q < 4; q++) {
                    double v = *gat(g, q, s, j);
                    if (flip && q == 1) v = -v;
                    *gat(g, q, k, j) = v;
                }
            }
    } else {
        int n = g->ny;
        for (int i = 0; i < g->nx; i++)
            for (int k = -2; k < n + 2; k++) {
                if (k >= 0 && k < n) continue;
                int flip, s = ghost_source(bc[2], bc[3], n, k, &flip);
                for (int q = 0; q < 4; q++) {
                    double v = *gat(g, q, i, s);
                    if (flip && q == 2) v = -v;
                    *gat(g, q, i, k) = v;
                }
            }
    }
}

/* One 1D Godunov sweep along dir (0 = x: rows, 1 = y: columns), Fig. 5:
 * boundary conditions, then READ / COMPUTE / WRITE line by line.  The x
 * sweep's normal momentum is rho*u, the y sweep's is rho*v.
 *
 * Lines are independent (a line reads only its own cells and ghosts and
 * writes only its own interior cells), so a build with -fopenmp shares the
 * lines of a sweep among threads, each with its own line buffers, as the
 * paper's Fine-Grain version shares the loop over lines (§2); every line is
 * computed by the same code either way, so the results are bit-identical to
 * the single-threaded build. */
static int sweep(const orc_params *P, grid_t *g, const int bc[4], int dir,
                 double dtdx)
{
    apply_bc(g, bc, dir);
    int n = dir == 0 ? g->nx : g->ny;
    int nlines = dir == 0 ? g->ny : g->nx;
    int qn = dir == 0 ? 1 : 2, qt = dir == 0 ? 2 : 1;
    int rc = ORC_OK;

#ifdef _OPENMP
#pragma omp parallel reduction(|:rc)
#endif
    {
        double (*line)[4] = malloc(sizeof(double[4]) * (size_t)(n + 4));
        double (*out)[4] = malloc(sizeof(double[4]) * (size_t)n);
        if (!line || !out) rc |= ORC_ENOMEM;
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int l = 0; l < nlines; l++) {
            if (!line || !out || rc != ORC_OK) continue;
            /* READ */
            for (int k = -2; k < n + 2; k++) {
                int i = dir == 0 ? k : l, j = dir == 0 ? l : k;
                line[k + 2][0] = *gat(g, 0, i, j);
                line[k + 2][1] = *gat(g, qn, i, j);
                line[k + 2][2] = *gat(g, qt, i, j);
                line[k + 2][3] = *gat(g, 3, i, j);
            }
            /* COMPUTE */
            rc |= godunov_line(P, n, dtdx, (const double (*)[4])line, out);
            /* WRITE */
            for (int k = 0; k < n; k++) {
                int i = dir == 0 ? k : l, j = dir == 0 ? l : k;
                *gat(g, 0, i, j) = out[k][0];
                *gat(g, qn, i, j) = out[k][1];
                *gat(g, qt, i, j) = out[k][2];
                *gat(g, 3, i, j) = out[k][3];
            }
        }
        free(line);
        free(out);
    }
    return rc;
}

/* CFL time step: dt = C h / w,  w = max over interior cells of
 * max(|u|, |v|) + c, with the primitives of cons_to_prim. */
static double cfl_dt_grid(const orc_params *P, grid_t *g, double h)
{
    double w = 0.0;
    for (int j = 0; j < g->ny; j++)
        for (int i = 0; i < g->nx; i++) {
            double U[4], W[4];
            for (int q = 0; q < 4; q++) U[q] = *gat(g, q, i, j);
            cons_to_prim(P, U, W);  /* (rho, u, v, p) */
            double c = sound_speed(P, W);
            double au = fabs(W[1]), av = fabs(W[2]);
            double s = ((au > av) ? au : av) + c;
            if (!(s <= w)) w = s;   /* NaN propagates */
        }
    return P->cfl * h / w;
}

static int valid_params(const orc_params *P, int nx, int ny, double h,
                        const int bc[4])
{
    if (!P || nx < 2 || ny < 2 || !(h > 0.0)) return 0;
    if (!(P->gamma > 1.0) || !(P->cfl > 0.0) || P->niter < 0) return 0;
    for (int k = 0; k < 4; k++)
        if (bc[k] < 0 || bc[k] > 2) return 0;
    if ((bc[0] == ORC_BC_PERIODIC) != (bc[1] == ORC_BC_PERIODIC)) return 0;
    if ((bc[2] == ORC_BC_PERIODIC) != (bc[3] == ORC_BC_PERIODIC)) return 0;
    return 1;
}

static int load_grid(grid_t *g, int nx, int ny, const double *U)
{
    g->nx = nx; g->ny = ny; g->sx = nx + 4;
    g->plane = (size_t)(ny + 4) * (size_t)(nx + 4);
    g->v = calloc(4 * g->plane, sizeof(double));
    if (!g->v) return ORC_ENOMEM;
    for (int q = 0; q < 4; q++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++)
                *gat(g, q, i, j) = U[((size_t)q * ny + j) * nx + i];
    return ORC_OK;
}

static int store_grid(grid_t *g, double *U)
{
    int bad = 0;
    for (int q = 0; q < 4; q++)
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++) {
                double v = *gat(g, q, i, j);
                U[((size_t)q * g->ny + j) * g->nx + i] = v;
                if (v != v || ((q == 0 || q == 3) && !(v > 0.0))) bad = 1;
            }
    return bad ? ORC_ENEGATIVE : ORC_OK;
}

/* ==========================================================================
 * Exported entry points
 * ======================================================================== */

/* Advance U (interior, SoA [4][ny][nx], in place) by nsteps steps.  Step
 * index k = step0 + s sets the sweep order: x then y for even k, y then x
 * for odd k.  dt_override: NULL, or nsteps values used instead of the CFL
 * dt.  dt_out (optional) receives the nsteps dt values used.  Returns
 * ORC_ENEGATIVE when the final state holds a NaN or a non-positive density
 * or energy. */
int orc_run(const orc_params *P, int nx, int ny, double h, const int bc[4],
            double *U, long step0, int nsteps, const double *dt_override,
            double *dt_out)
{
    if (!valid_params(P, nx, ny, h, bc) || !U || nsteps < 0) return ORC_EINVAL;
    grid_t g;
    int rc = load_grid(&g, nx, ny, U);
    if (rc) return rc;
    for (int s = 0; s < nsteps && rc == ORC_OK; s++) {
        double dt = dt_override ? dt_override[s] : cfl_dt_grid(P, &g, h);
        if (dt_out) dt_out[s] = dt;
        double dtdx = dt / h;
        if (((step0 + s) & 1) == 0) {
            rc = sweep(P, &g, bc, 0, dtdx);
            if (!rc) rc = sweep(P, &g, bc, 1, dtdx);
        } else {
            rc = sweep(P, &g, bc, 1, dtdx);
            if (!rc) rc = sweep(P, &g, bc, 0, dtdx);
        }
    }
    int rs = store_grid(&g, U);
    free(g.v);
    return rc ? rc : rs;
}

/* One sweep along dir (0 = x, 1 = y) with the given dt, in place. */
int orc_sweep(const orc_params *P, int nx, int ny, double h, const int bc[4],
              double *U, int dir, double dt)
{
    if (!valid_params(P, nx, ny, h, bc) || !U || dir < 0 || dir > 1) return ORC_EINVAL;
    grid_t g;
    int rc = load_grid(&g, nx, ny, U);
    if (rc) return rc;
    rc = sweep(P, &g, bc, dir, dt / h);
    int rs = store_grid(&g, U);
    free(g.v);
    return rc ? rc : rs;
}

/* CFL time step of the state U. */
double orc_cfl_dt(const orc_params *P, int nx, int ny, double h,
                  const double *U)
{
    grid_t g;
    if (load_grid(&g, nx, ny, U)) return -1.0;
    double dt = cfl_dt_grid(P, &g, h);
    free(g.v);
    return dt;
}

/* Domain totals h^2 * sum(U_q), rows in order, cells in order within a row. */
void orc_conservation(int nx, int ny, double h, const double *U,
                      double sums[4])
{
    for (int q = 0; q < 4; q++) {
        double s = 0.0;
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++)
                s += U[((size_t)q * ny + j) * nx + i];
        sums[q] = s * h * h;
    }
}

/* Godunov update of a single 1D line (n interior cells + 2 ghosts per side
 * given explicitly), exposed for the 1D pins. line: (n+4)*4 values
 * (rho, m_n, m_t, E) per cell; out: n*4 values. */
int orc_godunov_line(const orc_params *P, int n, double dtdx,
                     const double *line, double *out)
{
    if (!P || n < 1) return ORC_EINVAL;
    return godunov_line(P, n, dtdx, (const double (*)[4])line,
                        (double (*)[4])out);
}

/* The trace of one cell, exposed for the 1D pins. */
void orc_trace(const orc_params *P, double dtdx, const double Wm[4],
               const double W0[4], const double Wp[4], double WL[4],
               double WR[4])
{
    muscl_hancock_trace(P, dtdx, Wm, W0, Wp, WL, WR);
}

/* conserved (rho, m_n, m_t, E) -> primitive (rho, u_n, u_t, p) */
void orc_cons_to_prim(const orc_params *P, const double U[4], double W[4])
{
    cons_to_prim(P, U, W);
}

/* Threads of the -fopenmp build (0: the OpenMP default); returns the number
 * of threads a sweep will use, 1 in the single-threaded build. */
int orc_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}
