/*
 * rtlbfs_oracle.c -- plain FP64 CPU oracle of the reconstructed thermal
 * lattice Boltzmann flux solver (RTLBFS), 2D, structured rectilinear mesh.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, literal reference that
 * the CUDA path is checked against.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the product library never
 * links, includes or calls it, and it shares no code with the CUDA path.
 *
 * What it computes, step by step, in the paper's order (Section 3.2):
 *   1. ghost cells for the boundary conditions (Section 3.3 states only the
 *      physical conditions; the ghost-cell mirror rules are this oracle's
 *      reading, listed below);
 *   2. face values by inverse-distance weighting, Eq. 56;
 *   3. cell gradients by the discrete Gauss theorem, Eq. 55 (with 1/dV);
 *   4. per face: the 9-node unit lattice of Fig. 2, node values by the
 *      piecewise-linear interpolation of Eq. 29;
 *   5. per face: predicted variables from Eqs. 46-48, discretised by central
 *      differences on the 9 nodes;
 *   6. per face: fluxes of the corrector, the braces of Eqs. 57-59
 *      (including the (tau - 1.5)(X* - X^n) numerical-dissipation terms);
 *   7. explicit update of the cell conservatives, Eqs. 57-59, plus the
 *      Boussinesq source of Eq. 64;
 *   8. conservative -> primitive (Eqs. 11-13 with c_p = 1) and the steady
 *      residual (L2 analogue of Eq. 65).
 *
 * Readings where the paper is silent or garbled (each also used by the
 * CUDA path, which is written independently):
 *   R1  V_c = Ma * c with c = 1; nu = V_c L sqrt(Pr/Ra), chi = nu/Pr,
 *       beta_g = V_c^2/(dT L)                         (Eq. 63, Sec. 3.3)
 *   R2  lattice spacing per face: dt_f = kappa * min(width_L, width_R)
 *       normal to the face; tau_f = nu/(cs2 dt_f) + 1/2, tau_g likewise
 *       (Eqs. 9-10)
 *   R4  Eq. 55 carries the 1/dV that the printed form drops
 *   R5  node (a,b) of an x- or y-face sits at x_S + (a,b) dt_f in the
 *       global frame (D2Q9 is invariant under the 90-degree rotation)
 *   R6  the FD stencil of Eqs. 46-48: second-order central differences on
 *       the 9 nodes; products (rho u u etc.) are formed at the nodes
 *   R7  one ghost layer per side, mirror of the adjacent cell P with its
 *       width; rho even, velocity odd about the wall velocity, T odd about
 *       T_wall (Dirichlet) or even (adiabatic); even quantities mirror the
 *       normal gradient, odd ones the tangential gradient; periodic sides
 *       copy value, gradient and width from the opposite side
 *   R8  wall faces: after the predictor (rho u_n)* = 0,
 *       (rho u_t)* = rho* u_wall, and on Dirichlet walls (rho T)* = rho* T_w
 *       (the last enters no flux: T* only appears multiplied by u*_n = 0)
 *   R9  the time-n face state "( )^n" of Eqs. 58-59 is node (0,0) and the
 *       face derivatives are the central differences of R6
 *   R10 buoyancy F_y = + rho beta_g (T - T_ref): hot fluid rises (the sign
 *       printed in Eq. 64 would make it sink); body force (fx, fy) is an
 *       acceleration, source rho*(fx, fy)
 *   R12 residual: R_u = ||(|u|^{n+1} - |u|^n)||_2 / |||u|^{n+1}||_2,
 *       R_T likewise, plain sums over cells; a zero denominator gives inf,
 *       a sum that is not a number gives NaN (divergence)
 *
 * Second face stage, scheme = 1: the original TLBFS of Section 2.2 that
 * RTLBFS approximates -- steps 5-6 replaced by (a) D2Q9 equilibria (Eqs.
 * 3-4, c_p = 1) at the nodes x_S - e_i dt_f, whose values are the step-4
 * nodes (a, b) = -e_i; (b) the predicted variables as their moments, Eqs.
 * 30-32, with the wall rule R8; (c) the fluxes of Eqs. 38-40 from the
 * equilibria of the predicted variables and the non-equilibrium parts of
 * Eqs. 33-34.  The update (Eqs. 41-43) is step 7 with the same source.
 *   Nu  wall and mid-plane Nusselt numbers are the discrete energy flux of
 *       step 6 summed over a face column, / (chi dT); Nu_a follows Eq. 69
 *       with cell values and Green-Gauss dT/dx.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define CS2 (1.0 / 3.0) /* c_s^2 = c^2/3 with c = 1, Eq. 6 */

enum { SIDE_W = 0, SIDE_E = 1, SIDE_S = 2, SIDE_N = 3 };
enum { BC_DIRICHLET = 0, BC_ADIABATIC = 1, BC_PERIODIC = 2 };
enum { Q_RHO = 0, Q_U = 1, Q_V = 2, Q_T = 3 };

/* Problem description.  Field order of this struct is mirrored by the
 * Python ctypes binding in oracle/__init__.py. */
typedef struct {
    int nx, ny;
    const double* xf; /* nx+1 face coordinates, ascending */
    const double* yf; /* ny+1 */
    double nu, chi, beta_g, T_ref, dT;
    double dt;    /* macroscopic time step Delta t */
    double kappa; /* dt_f = kappa * min normal width (R2) */
    double fx, fy;
    int bc_kind[4];   /* per side W,E,S,N */
    double bc_T[4];   /* wall temperature (Dirichlet) */
    double bc_u[4];   /* tangential wall velocity */
    int scheme;       /* 0 RTLBFS (Section 3.2), 1 TLBFS (Section 2.2) */
} orc_problem;

/* ------------------------------------------------------------------ */
/* Mesh (Eq. 74) and parameters (Eq. 63, Eqs. 9-10)                    */
/* ------------------------------------------------------------------ */

/* Eq. 74: x_i = {tanh(phi) + tanh[2 phi (i/M - 1/2)]} L / (2 tanh(phi)).
 * phi <= 0 gives the uniform mesh x_i = i L / M. */
int orc_tanh_faces(int n, double L, double phi, double* out)
{
    if (n < 1 || !(L > 0.0) || !out) return -1;
    for (int i = 0; i <= n; ++i) {
        double s = (double)i / (double)n;
        if (phi > 0.0)
            out[i] = (tanh(phi) + tanh(2.0 * phi * (s - 0.5))) * L / (2.0 * tanh(phi));
        else
            out[i] = s * L;
    }
    return 0;
}

/* Eq. 63 solved for the transport coefficients, with V_c = Ma (R1):
 *   Ra = V_c^2 L^2 / (chi nu), Pr = nu / chi, V_c^2 = beta_g dT L. */
int orc_params(double Ra, double Pr, double Ma, double L, double dT, double* out3)
{
    if (!(Ra > 0.0) || !(Pr > 0.0) || !(Ma > 0.0) || !(L > 0.0) || !(dT > 0.0)) return -1;
    double Vc = Ma;
    double nu = Vc * L * sqrt(Pr / Ra);
    out3[0] = nu;
    out3[1] = nu / Pr;
    out3[2] = Vc * Vc / (dT * L);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Working storage: one ghost layer around the ny x nx cells           */
/* ------------------------------------------------------------------ */

typedef struct {
    int nx, ny, px;     /* px = nx + 2 */
    double* q[4];       /* padded primitives rho,u,v,T */
    double* g[4][2];    /* padded gradients d/dx, d/dy */
    double* wx;         /* padded widths in x (nx+2) */
    double* wy;         /* padded widths in y (ny+2) */
    double* fxf[4];     /* x-face fluxes, ny rows of nx+1 */
    double* fyf[4];     /* y-face fluxes, ny+1 rows of nx */
} work;

#define PIDX(w, i, j) (((j) + 1) * (w)->px + ((i) + 1))

static void work_free(work* w)
{
    for (int q = 0; q < 4; ++q) {
        free(w->q[q]);
        free(w->g[q][0]);
        free(w->g[q][1]);
        free(w->fxf[q]);
        free(w->fyf[q]);
    }
    free(w->wx);
    free(w->wy);
}

static int work_alloc(work* w, int nx, int ny)
{
    memset(w, 0, sizeof(*w));
    w->nx = nx;
    w->ny = ny;
    w->px = nx + 2;
    size_t np = (size_t)(nx + 2) * (size_t)(ny + 2);
    int ok = 1;
    for (int q = 0; q < 4; ++q) {
        w->q[q] = calloc(np, sizeof(double));
        w->g[q][0] = calloc(np, sizeof(double));
        w->g[q][1] = calloc(np, sizeof(double));
        w->fxf[q] = calloc((size_t)ny * (size_t)(nx + 1), sizeof(double));
        w->fyf[q] = calloc((size_t)(ny + 1) * (size_t)nx, sizeof(double));
        ok = ok && w->q[q] && w->g[q][0] && w->g[q][1] && w->fxf[q] && w->fyf[q];
    }
    w->wx = calloc((size_t)nx + 2, sizeof(double));
    w->wy = calloc((size_t)ny + 2, sizeof(double));
    ok = ok && w->wx && w->wy;
    if (!ok) {
        work_free(w);
        return -2;
    }
    return 0;
}

static int check_problem(const orc_problem* p)
{
    if (!p || (p->scheme != 0 && p->scheme != 1)) return -1;
    if (p->nx < 1 || p->ny < 1 || !p->xf || !p->yf) return -1;
    for (int i = 0; i < p->nx; ++i)
        if (!(p->xf[i + 1] > p->xf[i])) return -1;
    for (int j = 0; j < p->ny; ++j)
        if (!(p->yf[j + 1] > p->yf[j])) return -1;
    for (int s = 0; s < 4; ++s)
        if (p->bc_kind[s] < 0 || p->bc_kind[s] > 2) return -1;
    if ((p->bc_kind[SIDE_W] == BC_PERIODIC) != (p->bc_kind[SIDE_E] == BC_PERIODIC)) return -1;
    if ((p->bc_kind[SIDE_S] == BC_PERIODIC) != (p->bc_kind[SIDE_N] == BC_PERIODIC)) return -1;
    if (!(p->kappa > 0.0) || !(p->nu > 0.0) || !(p->chi > 0.0)) return -1;
    return 0;
}

/* Cell widths, ghosts included (R7: a mirror ghost has the width of its
 * partner cell; a periodic ghost has the width of the opposite cell). */
static void fill_widths(const orc_problem* p, work* w)
{
    int nx = p->nx, ny = p->ny;
    for (int i = 0; i < nx; ++i) w->wx[i + 1] = p->xf[i + 1] - p->xf[i];
    for (int j = 0; j < ny; ++j) w->wy[j + 1] = p->yf[j + 1] - p->yf[j];
    int perx = p->bc_kind[SIDE_W] == BC_PERIODIC;
    int pery = p->bc_kind[SIDE_S] == BC_PERIODIC;
    w->wx[0] = perx ? w->wx[nx] : w->wx[1];
    w->wx[nx + 1] = perx ? w->wx[1] : w->wx[nx];
    w->wy[0] = pery ? w->wy[ny] : w->wy[1];
    w->wy[ny + 1] = pery ? w->wy[1] : w->wy[ny];
}

/* Parity of quantity q about a wall of side s (R7): +1 even, -1 odd. */
static int wall_parity(const orc_problem* p, int s, int q)
{
    if (q == Q_RHO) return +1;
    if (q == Q_U || q == Q_V) return -1;
    return p->bc_kind[s] == BC_DIRICHLET ? -1 : +1; /* T */
}

/* Value that an odd quantity is mirrored about at wall s (R7). */
static double wall_value(const orc_problem* p, int s, int q)
{
    int normal_is_x = (s == SIDE_W || s == SIDE_E);
    if (q == Q_T) return p->bc_T[s];
    if (q == Q_U) return normal_is_x ? 0.0 : p->bc_u[s];
    if (q == Q_V) return normal_is_x ? p->bc_u[s] : 0.0;
    return 0.0;
}

/* Ghost value of quantity q at wall s given the partner cell value. */
static double ghost_value(const orc_problem* p, int s, int q, double phiP)
{
    if (wall_parity(p, s, q) > 0) return phiP;
    return 2.0 * wall_value(p, s, q) - phiP;
}

/* Step 1: ghost values on the four edges (no corner ghosts are needed). */
static void fill_ghost_values(const orc_problem* p, work* w)
{
    int nx = p->nx, ny = p->ny;
    for (int q = 0; q < 4; ++q) {
        double* a = w->q[q];
        for (int j = 0; j < ny; ++j) {
            if (p->bc_kind[SIDE_W] == BC_PERIODIC) {
                a[PIDX(w, -1, j)] = a[PIDX(w, nx - 1, j)];
                a[PIDX(w, nx, j)] = a[PIDX(w, 0, j)];
            } else {
                a[PIDX(w, -1, j)] = ghost_value(p, SIDE_W, q, a[PIDX(w, 0, j)]);
                a[PIDX(w, nx, j)] = ghost_value(p, SIDE_E, q, a[PIDX(w, nx - 1, j)]);
            }
        }
        for (int i = 0; i < nx; ++i) {
            if (p->bc_kind[SIDE_S] == BC_PERIODIC) {
                a[PIDX(w, i, -1)] = a[PIDX(w, i, ny - 1)];
                a[PIDX(w, i, ny)] = a[PIDX(w, i, 0)];
            } else {
                a[PIDX(w, i, -1)] = ghost_value(p, SIDE_S, q, a[PIDX(w, i, 0)]);
                a[PIDX(w, i, ny)] = ghost_value(p, SIDE_N, q, a[PIDX(w, i, ny - 1)]);
            }
        }
    }
}

/* Eq. 56: inverse-distance weighting between the two cell centres that
 * share a face; the centre-to-face distances are half the cell widths. */
static double eq56_face_value(double phiL, double phiR, double widthL, double widthR)
{
    double dL = 0.5 * widthL; /* |x_L - x_S| */
    double dR = 0.5 * widthR; /* |x_R - x_S| */
    return (phiL * dR + phiR * dL) / (dR + dL);
}

/* Steps 2-3: Eq. 55 with the 1/dV (R4), over the four faces of every
 * interior cell, outward face-area vectors dS = (+-dy, 0), (0, +-dx). */
static void interior_gradients(const orc_problem* p, work* w)
{
    int nx = p->nx, ny = p->ny;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            double dx = w->wx[i + 1], dy = w->wy[j + 1];
            double dV = dx * dy;
            for (int q = 0; q < 4; ++q) {
                const double* a = w->q[q];
                double c = a[PIDX(w, i, j)];
                double phi_e = eq56_face_value(c, a[PIDX(w, i + 1, j)], dx, w->wx[i + 2]);
                double phi_w = eq56_face_value(a[PIDX(w, i - 1, j)], c, w->wx[i], dx);
                double phi_n = eq56_face_value(c, a[PIDX(w, i, j + 1)], dy, w->wy[j + 2]);
                double phi_s = eq56_face_value(a[PIDX(w, i, j - 1)], c, w->wy[j], dy);
                /* sum_k phi_S dS_k,alpha */
                double sx = phi_e * (+dy) + phi_w * (-dy) + phi_n * 0.0 + phi_s * 0.0;
                double sy = phi_e * 0.0 + phi_w * 0.0 + phi_n * (+dx) + phi_s * (-dx);
                w->g[q][0][PIDX(w, i, j)] = sx / dV;
                w->g[q][1][PIDX(w, i, j)] = sy / dV;
            }
        }
    }
}

/* Ghost gradients (R7): even quantities keep the tangential gradient and
 * negate the normal one; odd quantities keep the normal and negate the
 * tangential.  Periodic ghosts copy the opposite cell's gradient. */
static void fill_ghost_gradients(const orc_problem* p, work* w)
{
    int nx = p->nx, ny = p->ny;
    for (int q = 0; q < 4; ++q) {
        double* gx = w->g[q][0];
        double* gy = w->g[q][1];
        for (int j = 0; j < ny; ++j) {
            if (p->bc_kind[SIDE_W] == BC_PERIODIC) {
                gx[PIDX(w, -1, j)] = gx[PIDX(w, nx - 1, j)];
                gy[PIDX(w, -1, j)] = gy[PIDX(w, nx - 1, j)];
                gx[PIDX(w, nx, j)] = gx[PIDX(w, 0, j)];
                gy[PIDX(w, nx, j)] = gy[PIDX(w, 0, j)];
            } else {
                int sW = wall_parity(p, SIDE_W, q), sE = wall_parity(p, SIDE_E, q);
                /* wall normal is x: normal gradient = gx */
                gx[PIDX(w, -1, j)] = (sW > 0 ? -1.0 : 1.0) * gx[PIDX(w, 0, j)];
                gy[PIDX(w, -1, j)] = (sW > 0 ? 1.0 : -1.0) * gy[PIDX(w, 0, j)];
                gx[PIDX(w, nx, j)] = (sE > 0 ? -1.0 : 1.0) * gx[PIDX(w, nx - 1, j)];
                gy[PIDX(w, nx, j)] = (sE > 0 ? 1.0 : -1.0) * gy[PIDX(w, nx - 1, j)];
            }
        }
        for (int i = 0; i < nx; ++i) {
            if (p->bc_kind[SIDE_S] == BC_PERIODIC) {
                gx[PIDX(w, i, -1)] = gx[PIDX(w, i, ny - 1)];
                gy[PIDX(w, i, -1)] = gy[PIDX(w, i, ny - 1)];
                gx[PIDX(w, i, ny)] = gx[PIDX(w, i, 0)];
                gy[PIDX(w, i, ny)] = gy[PIDX(w, i, 0)];
            } else {
                int sS = wall_parity(p, SIDE_S, q), sN = wall_parity(p, SIDE_N, q);
                /* wall normal is y: normal gradient = gy */
                gy[PIDX(w, i, -1)] = (sS > 0 ? -1.0 : 1.0) * gy[PIDX(w, i, 0)];
                gx[PIDX(w, i, -1)] = (sS > 0 ? 1.0 : -1.0) * gx[PIDX(w, i, 0)];
                gy[PIDX(w, i, ny)] = (sN > 0 ? -1.0 : 1.0) * gy[PIDX(w, i, ny - 1)];
                gx[PIDX(w, i, ny)] = (sN > 0 ? 1.0 : -1.0) * gx[PIDX(w, i, ny - 1)];
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* Steps 4-6: one face                                                  */
/* ------------------------------------------------------------------ */

/* Node-product indices used by the predictor and the flux. */
enum {
    P_RHO = 0, /* rho                    */
    P_MX,      /* rho u                  */
    P_MY,      /* rho v                  */
    P_E,       /* rho T (c_p = 1)        */
    P_XXX,     /* rho u u + rho cs2      */
    P_XXY,     /* rho u v                */
    P_XYY,     /* rho v v + rho cs2      */
    P_UT,      /* rho u T                */
    P_VT,      /* rho v T                */
    NPROD
};

/* Everything one face produces; exposed for the unit pins. */
typedef struct {
    double h;               /* lattice spacing dt_f (R2) */
    double tau_f, tau_g;    /* Eqs. 9-10 */
    double node[4][3][3];   /* primitives at node (a,b), indices [q][a+1][b+1] */
    double pred[4];         /* rho*, (rho u)*, (rho v)*, (rho T)* after R8 */
    double flux[4];         /* mass, x-momentum, y-momentum, energy */
} orc_face_out;

/* One cell seen from a face: its primitives, gradients and centre offset
 * x_cell - x_S. */
typedef struct {
    double q[4];
    double g[4][2];
    double off[2];
} cell_view;

static void take_cell(const work* w, int i, int j, double offx, double offy, cell_view* c)
{
    for (int q = 0; q < 4; ++q) {
        c->q[q] = w->q[q][PIDX(w, i, j)];
        c->g[q][0] = w->g[q][0][PIDX(w, i, j)];
        c->g[q][1] = w->g[q][1][PIDX(w, i, j)];
    }
    c->off[0] = offx;
    c->off[1] = offy;
}

/* Eq. 29: value at node position d (relative to x_S) extrapolated from a
 * cell with its Green-Gauss gradient. */
static double extrap(const cell_view* c, int q, const double d[2])
{
    return c->q[q] + c->g[q][0] * (d[0] - c->off[0]) + c->g[q][1] * (d[1] - c->off[1]);
}

/* Step 4: the 9 nodes x_S + (a,b) h (R5) with values by Eq. 29. */
static void face_nodes(int nd, const cell_view* L, const cell_view* R, double h,
                       double node[4][3][3])
{
    for (int a = -1; a <= 1; ++a) {
        for (int b = -1; b <= 1; ++b) {
            double d[2] = {a * h, b * h};
            int side = (nd == 0) ? a : b; /* normal offset decides the cell */
            for (int q = 0; q < 4; ++q) {
                double v;
                if (side < 0)
                    v = extrap(L, q, d);
                else if (side > 0)
                    v = extrap(R, q, d);
                else
                    v = 0.5 * (extrap(L, q, d) + extrap(R, q, d));
                node[q][a + 1][b + 1] = v;
            }
        }
    }
}

/*
 * Steps 5-6 from given node primitives o->node: the predictor and the
 * fluxes through a face with unit normal along axis `nd` (0 = x, 1 = y).
 * wall_side >= 0 marks a boundary face of that side (R8).
 */
static void face_from_nodes(const orc_problem* p, int nd, double h, int wall_side,
                            orc_face_out* o)
{
    o->h = h;
    o->tau_f = p->nu / (CS2 * h) + 0.5;  /* Eq. 9 */
    o->tau_g = p->chi / (CS2 * h) + 0.5; /* Eq. 10 */

    /* Products at the nodes (R6). */
    double P[NPROD][3][3];
    for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 3; ++b) {
            double r = o->node[Q_RHO][a][b], u = o->node[Q_U][a][b];
            double v = o->node[Q_V][a][b], T = o->node[Q_T][a][b];
            P[P_RHO][a][b] = r;
            P[P_MX][a][b] = r * u;
            P[P_MY][a][b] = r * v;
            P[P_E][a][b] = r * T;
            P[P_XXX][a][b] = r * u * u + r * CS2;
            P[P_XXY][a][b] = r * u * v;
            P[P_XYY][a][b] = r * v * v + r * CS2;
            P[P_UT][a][b] = r * u * T;
            P[P_VT][a][b] = r * v * T;
        }
    }

    /* Central differences on the nodes (R6): D[k][alpha], DD[k][alpha][beta]. */
    double D[NPROD][2], DD[NPROD][2][2];
    for (int k = 0; k < NPROD; ++k) {
        D[k][0] = (P[k][2][1] - P[k][0][1]) / (2.0 * h);
        D[k][1] = (P[k][1][2] - P[k][1][0]) / (2.0 * h);
        DD[k][0][0] = (P[k][2][1] - 2.0 * P[k][1][1] + P[k][0][1]) / (h * h);
        DD[k][1][1] = (P[k][1][2] - 2.0 * P[k][1][1] + P[k][1][0]) / (h * h);
        DD[k][0][1] = (P[k][2][2] - P[k][2][0] - P[k][0][2] + P[k][0][0]) / (4.0 * h * h);
        DD[k][1][0] = DD[k][0][1];
    }
    /* index maps for the tensor notation */
    const int M[2] = {P_MX, P_MY};                      /* rho u_alpha */
    const int X[2][2] = {{P_XXX, P_XXY}, {P_XXY, P_XYY}}; /* rho u_a u_b + rho cs2 delta */
    const int UT[2] = {P_UT, P_VT};                      /* rho u_alpha T */
#define C0(k) (P[(k)][1][1]) /* node (0,0) value = time-n face state (R9) */

    /* Step 5: predictor, Eqs. 46-48 with dt -> h. */
    double rho_s = C0(P_RHO);
    for (int al = 0; al < 2; ++al) rho_s -= h * D[M[al]][al];
    for (int al = 0; al < 2; ++al)
        for (int be = 0; be < 2; ++be) rho_s += 0.5 * h * h * DD[X[al][be]][al][be];

    double m_s[2];
    for (int al = 0; al < 2; ++al) {
        double s = C0(M[al]);
        for (int be = 0; be < 2; ++be) s -= h * D[X[al][be]][be];
        /* d_b[ d_b(rho u_a) + d_a(rho u_b) + d_g(rho u_g) delta_ab ] */
        double br = 0.0;
        for (int be = 0; be < 2; ++be) {
            br += DD[M[al]][be][be];
            br += DD[M[be]][al][be];
        }
        for (int ga = 0; ga < 2; ++ga) br += DD[M[ga]][al][ga];
        s += 0.5 * CS2 * h * h * br;
        m_s[al] = s;
    }

    double E_s = C0(P_E);
    for (int al = 0; al < 2; ++al) E_s -= h * D[UT[al]][al];
    for (int al = 0; al < 2; ++al) E_s += 0.5 * CS2 * h * h * DD[P_E][al][al];

    /* R8: wall override of the predicted variables. */
    if (wall_side >= 0) {
        int td = 1 - nd; /* tangential axis */
        m_s[nd] = 0.0;
        m_s[td] = rho_s * p->bc_u[wall_side];
        if (p->bc_kind[wall_side] == BC_DIRICHLET) E_s = rho_s * p->bc_T[wall_side];
    }
    o->pred[0] = rho_s;
    o->pred[1] = m_s[0];
    o->pred[2] = m_s[1];
    o->pred[3] = E_s;
    double us[2] = {m_s[0] / rho_s, m_s[1] / rho_s};
    double Ts = E_s / rho_s;

    /* Step 6: fluxes through the face, beta = nd (Eqs. 57-59 braces). */
    int be = nd;
    o->flux[0] = m_s[be]; /* Eq. 57 */
    double divm = D[P_MX][0] + D[P_MY][1];
    for (int al = 0; al < 2; ++al) {
        double X0 = C0(X[al][be]);
        double Xs = rho_s * us[al] * us[be] + (al == be ? rho_s * CS2 : 0.0);
        double visc = D[M[al]][be] + D[M[be]][al] + (al == be ? divm : 0.0);
        o->flux[1 + al] = X0 - p->nu * visc - (o->tau_f - 1.5) * (Xs - X0); /* Eq. 58 */
    }
    {
        double Q0 = C0(UT[be]);
        double Qs = rho_s * us[be] * Ts;
        o->flux[3] = Q0 - p->chi * D[P_E][be] - (o->tau_g - 1.5) * (Qs - Q0); /* Eq. 59 */
    }
#undef C0
}

/* D2Q9 (Eqs. 5-6): discrete velocities in the order printed, weights. */
static const int E9[9][2] = {{0, 0}, {1, 0},  {0, 1},   {-1, 0}, {0, -1},
                             {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
static const double W9[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

/* Eq. 3 */
static double f_equilibrium(int i, double r, double u, double v)
{
    double eu = E9[i][0] * u + E9[i][1] * v;
    return W9[i] * r * (1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - (u * u + v * v) / (2.0 * CS2));
}

/* Eq. 4 with c_p = 1 */
static double g_equilibrium(int i, double r, double u, double v, double T)
{
    double eu = E9[i][0] * u + E9[i][1] * v;
    return W9[i] * r * T * (1.0 + eu / CS2);
}

/*
 * TLBFS steps (a)-(c) of Section 2.2 for a face with normal along axis nd,
 * from the node primitives o->node (step 4).
 */
static void face_tlbfs_from_nodes(const orc_problem* p, int nd, double h, int wall_side,
                                  orc_face_out* o)
{
    o->h = h;
    o->tau_f = p->nu / (CS2 * h) + 0.5;  /* Eq. 9 */
    o->tau_g = p->chi / (CS2 * h) + 0.5; /* Eq. 10 */

    /* (a) equilibria at x_S - e_i dt: node (a, b) = -e_i (R5) */
    double fn[9], gn[9];
    for (int i = 0; i < 9; ++i) {
        int a = -E9[i][0] + 1, b = -E9[i][1] + 1;
        double r = o->node[Q_RHO][a][b], u = o->node[Q_U][a][b];
        double v = o->node[Q_V][a][b], T = o->node[Q_T][a][b];
        fn[i] = f_equilibrium(i, r, u, v);
        gn[i] = g_equilibrium(i, r, u, v, T);
    }

    /* (b) predicted variables, Eqs. 30-32 */
    double rho_s = 0.0, m_s[2] = {0.0, 0.0}, E_s = 0.0;
    for (int i = 0; i < 9; ++i) {
        rho_s += fn[i];
        m_s[0] += E9[i][0] * fn[i];
        m_s[1] += E9[i][1] * fn[i];
        E_s += gn[i];
    }
    if (wall_side >= 0) { /* R8 */
        int td = 1 - nd;
        m_s[nd] = 0.0;
        m_s[td] = rho_s * p->bc_u[wall_side];
        if (p->bc_kind[wall_side] == BC_DIRICHLET) E_s = rho_s * p->bc_T[wall_side];
    }
    o->pred[0] = rho_s;
    o->pred[1] = m_s[0];
    o->pred[2] = m_s[1];
    o->pred[3] = E_s;
    double us = m_s[0] / rho_s, vs = m_s[1] / rho_s, Ts = E_s / rho_s;

    /* (c) fluxes, Eqs. 38-40 (beta = nd), with the non-equilibrium parts of
     * Eqs. 33-34: f^(1) = -tau (f_eq(x_S, t+dt) - f_eq(x_S - e dt, t)) */
    double P = 0.0, Pi[2] = {0.0, 0.0}, Q = 0.0;
    for (int i = 0; i < 9; ++i) {
        double fs = f_equilibrium(i, rho_s, us, vs);
        double gs = g_equilibrium(i, rho_s, us, vs, Ts);
        double en = E9[i][nd];
        P += en * fs;
        for (int al = 0; al < 2; ++al)
            Pi[al] += E9[i][al] * en * (fs + (0.5 - o->tau_f) * (fs - fn[i]));
        Q += en * (gs + (0.5 - o->tau_g) * (gs - gn[i]));
    }
    o->flux[0] = P;
    o->flux[1] = Pi[0];
    o->flux[2] = Pi[1];
    o->flux[3] = Q;
}

/* One face from its two cells: steps 4-6. */
static void face_compute(const orc_problem* p, int nd, const cell_view* L, const cell_view* R,
                         double h, int wall_side, orc_face_out* o)
{
    face_nodes(nd, L, R, h, o->node);
    if (p->scheme == 1)
        face_tlbfs_from_nodes(p, nd, h, wall_side, o);
    else
        face_from_nodes(p, nd, h, wall_side, o);
}

/* Build the L/R views of x-face (i, j) (between cells i-1 and i) or of
 * y-face (i, j) (between cells j-1 and j) and compute it. */
static void face_at(const orc_problem* p, const work* w, int nd, int i, int j, orc_face_out* o)
{
    int nx = p->nx, ny = p->ny;
    cell_view L, R;
    double h;
    int wall = -1;
    if (nd == 0) {
        double wl = w->wx[i], wr = w->wx[i + 1]; /* padded: cell i-1 is index i */
        take_cell(w, i - 1, j, -0.5 * wl, 0.0, &L);
        take_cell(w, i, j, 0.5 * wr, 0.0, &R);
        h = p->kappa * (wl < wr ? wl : wr);
        if (p->bc_kind[SIDE_W] != BC_PERIODIC) {
            if (i == 0) wall = SIDE_W;
            if (i == nx) wall = SIDE_E;
        }
    } else {
        double wl = w->wy[j], wr = w->wy[j + 1];
        take_cell(w, i, j - 1, 0.0, -0.5 * wl, &L);
        take_cell(w, i, j, 0.0, 0.5 * wr, &R);
        h = p->kappa * (wl < wr ? wl : wr);
        if (p->bc_kind[SIDE_S] != BC_PERIODIC) {
            if (j == 0) wall = SIDE_S;
            if (j == ny) wall = SIDE_N;
        }
    }
    face_compute(p, nd, &L, &R, h, wall, o);
}

static void all_face_fluxes(const orc_problem* p, work* w)
{
    int nx = p->nx, ny = p->ny;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j) {
        orc_face_out o;
        for (int i = 0; i <= nx; ++i) {
            face_at(p, w, 0, i, j, &o);
            for (int k = 0; k < 4; ++k) w->fxf[k][(size_t)j * (nx + 1) + i] = o.flux[k];
        }
    }
#pragma omp parallel for schedule(static)
    for (int j = 0; j <= ny; ++j) {
        orc_face_out o;
        for (int i = 0; i < nx; ++i) {
            face_at(p, w, 1, i, j, &o);
            for (int k = 0; k < 4; ++k) w->fyf[k][(size_t)j * nx + i] = o.flux[k];
        }
    }
}

/* Steps 1-3 for the current padded state. */
static void prepare(const orc_problem* p, work* w)
{
    fill_ghost_values(p, w);
    interior_gradients(p, w);
    fill_ghost_gradients(p, w);
}

static void load_state(const orc_problem* p, work* w, const double* rho, const double* u,
                       const double* v, const double* T)
{
    const double* src[4] = {rho, u, v, T};
    for (int q = 0; q < 4; ++q)
        for (int j = 0; j < p->ny; ++j)
            for (int i = 0; i < p->nx; ++i)
                w->q[q][PIDX(w, i, j)] = src[q][(size_t)j * p->nx + i];
}

/* Steps 7-8 for every cell; writes the new primitives into the caller's
 * arrays and accumulates the residual sums of R12. */
static void update_cells(const orc_problem* p, work* w, double* rho, double* u, double* v,
                         double* T, double res[2])
{
    int nx = p->nx, ny = p->ny;
    double su_num = 0.0, su_den = 0.0, sT_num = 0.0, sT_den = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : su_num, su_den, sT_num, sT_den)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            double dx = w->wx[i + 1], dy = w->wy[j + 1], dV = dx * dy;
            double r = w->q[Q_RHO][PIDX(w, i, j)], uu = w->q[Q_U][PIDX(w, i, j)];
            double vv = w->q[Q_V][PIDX(w, i, j)], TT = w->q[Q_T][PIDX(w, i, j)];
            /* conservatives at time n */
            double Wc[4] = {r, r * uu, r * vv, r * TT};
            /* Sum_k F_k . dS_k with outward area vectors */
            double sum[4];
            for (int k = 0; k < 4; ++k) {
                double Fe = w->fxf[k][(size_t)j * (nx + 1) + i + 1];
                double Fw = w->fxf[k][(size_t)j * (nx + 1) + i];
                double Gn = w->fyf[k][(size_t)(j + 1) * nx + i];
                double Gs = w->fyf[k][(size_t)j * nx + i];
                sum[k] = Fe * dy - Fw * dy + Gn * dx - Gs * dx;
            }
            /* Boussinesq source (Eq. 64, sign by R10) and body force */
            double S[4] = {0.0, r * p->fx, r * (p->beta_g * (TT - p->T_ref) + p->fy), 0.0};
            double Wn[4];
            for (int k = 0; k < 4; ++k) Wn[k] = Wc[k] - p->dt / dV * sum[k] + p->dt * S[k];
            double r1 = Wn[0], u1 = Wn[1] / r1, v1 = Wn[2] / r1, T1 = Wn[3] / r1;
            size_t c = (size_t)j * nx + i;
            rho[c] = r1;
            u[c] = u1;
            v[c] = v1;
            T[c] = T1;
            double m0 = sqrt(uu * uu + vv * vv), m1 = sqrt(u1 * u1 + v1 * v1);
            su_num += (m1 - m0) * (m1 - m0);
            su_den += m1 * m1;
            sT_num += (T1 - TT) * (T1 - TT);
            sT_den += T1 * T1;
        }
    }
    res[0] = su_den > 0.0 ? sqrt(su_num) / sqrt(su_den) : INFINITY;
    res[1] = sT_den > 0.0 ? sqrt(sT_num) / sqrt(sT_den) : INFINITY;
    /* a state that is no longer a number has no residual: divergence */
    if (isnan(su_num) || isnan(su_den)) res[0] = NAN;
    if (isnan(sT_num) || isnan(sT_den)) res[1] = NAN;
}

/* ------------------------------------------------------------------ */
/* Public entry points                                                  */
/* ------------------------------------------------------------------ */

int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

static int all_finite(const orc_problem* p, const double* a)
{
    size_t n = (size_t)p->nx * p->ny;
    for (size_t c = 0; c < n; ++c)
        if (!isfinite(a[c])) return 0;
    return 1;
}

/* Advance nsteps explicit steps in place; res[0..1] = R_u, R_T of the
 * last step.  Returns 0, -1 on bad arguments, -2 on allocation failure,
 * -4 if the state became non-finite. */
int orc_step(const orc_problem* p, double* rho, double* u, double* v, double* T, long nsteps,
             double* res)
{
    if (check_problem(p) || !rho || !u || !v || !T || nsteps < 0) return -1;
    work w;
    if (work_alloc(&w, p->nx, p->ny)) return -2;
    fill_widths(p, &w);
    double r2[2] = {NAN, NAN};
    int rc = 0;
    for (long s = 0; s < nsteps; ++s) {
        load_state(p, &w, rho, u, v, T);
        prepare(p, &w);
        all_face_fluxes(p, &w);
        update_cells(p, &w, rho, u, v, T, r2);
        if (isnan(r2[0]) || isnan(r2[1])) { rc = -4; break; }
    }
    if (rc == 0 && !(all_finite(p, rho) && all_finite(p, u) && all_finite(p, v) && all_finite(p, T)))
        rc = -4;
    if (res) {
        res[0] = r2[0];
        res[1] = r2[1];
    }
    work_free(&w);
    return rc;
}

/* Step until max(R_u, R_T) < tol (checked after every step) or max_steps.
 * Returns 0 when converged, -5 when max_steps was reached, -4 diverged. */
int orc_run_to_steady(const orc_problem* p, double* rho, double* u, double* v, double* T,
                      double tol, long max_steps, long* steps, double* res)
{
    if (check_problem(p) || !rho || !u || !v || !T || max_steps < 0) return -1;
    work w;
    if (work_alloc(&w, p->nx, p->ny)) return -2;
    fill_widths(p, &w);
    double r2[2] = {INFINITY, INFINITY};
    long s = 0;
    int rc = -5;
    while (s < max_steps) {
        load_state(p, &w, rho, u, v, T);
        prepare(p, &w);
        all_face_fluxes(p, &w);
        update_cells(p, &w, rho, u, v, T, r2);
        ++s;
        if (isnan(r2[0]) || isnan(r2[1])) { rc = -4; break; }
        double m = r2[0] > r2[1] ? r2[0] : r2[1];
        if (m < tol) { rc = 0; break; }
    }
    if (steps) *steps = s;
    if (res) {
        res[0] = r2[0];
        res[1] = r2[1];
    }
    work_free(&w);
    return rc;
}

/* Cell gradients (Eq. 55) of the given state: out has 8 planes of ny*nx,
 * order d/dx rho, d/dy rho, d/dx u, d/dy u, d/dx v, d/dy v, d/dx T, d/dy T. */
int orc_gradients(const orc_problem* p, const double* rho, const double* u, const double* v,
                  const double* T, double* out)
{
    if (check_problem(p) || !out) return -1;
    work w;
    if (work_alloc(&w, p->nx, p->ny)) return -2;
    fill_widths(p, &w);
    load_state(p, &w, rho, u, v, T);
    prepare(p, &w);
    size_t n = (size_t)p->nx * p->ny;
    for (int q = 0; q < 4; ++q)
        for (int d = 0; d < 2; ++d)
            for (int j = 0; j < p->ny; ++j)
                for (int i = 0; i < p->nx; ++i)
                    out[(size_t)(2 * q + d) * n + (size_t)j * p->nx + i] = w.g[q][d][PIDX(&w, i, j)];
    work_free(&w);
    return 0;
}

/* One face of the given state (nd = 0: x-face between cells i-1 and i of
 * row j, i in [0, nx]; nd = 1: y-face between rows j-1 and j of column i,
 * j in [0, ny]); fills *o with its nodes, prediction and fluxes. */
int orc_face(const orc_problem* p, const double* rho, const double* u, const double* v,
             const double* T, int nd, int i, int j, orc_face_out* o)
{
    if (check_problem(p) || !o) return -1;
    if (nd == 0 && (i < 0 || i > p->nx || j < 0 || j >= p->ny)) return -1;
    if (nd == 1 && (i < 0 || i >= p->nx || j < 0 || j > p->ny)) return -1;
    if (nd != 0 && nd != 1) return -1;
    work w;
    if (work_alloc(&w, p->nx, p->ny)) return -2;
    fill_widths(p, &w);
    load_state(p, &w, rho, u, v, T);
    prepare(p, &w);
    face_at(p, &w, nd, i, j, o);
    work_free(&w);
    return 0;
}

/* Steps 5-6 alone, from caller-given node primitives nodes[q][a+1][b+1]
 * (q = rho,u,v,T; 36 values), lattice spacing h, face normal nd and
 * wall_side (-1 for an interior face).  Lets the tests feed node data
 * sampled from analytic fields. */
int orc_face_from_nodes(const orc_problem* p, int nd, const double* nodes, double h,
                        int wall_side, orc_face_out* o)
{
    if (!p || !nodes || !o || (nd != 0 && nd != 1) || !(h > 0.0) || wall_side < -1 ||
        wall_side > 3)
        return -1;
    memcpy(o->node, nodes, sizeof(o->node));
    if (p->scheme == 1)
        face_tlbfs_from_nodes(p, nd, h, wall_side, o);
    else
        face_from_nodes(p, nd, h, wall_side, o);
    return 0;
}

/* All face fluxes of the given state: fx has 4 planes of ny x (nx+1),
 * fy 4 planes of (ny+1) x nx (mass, x-mom, y-mom, energy). */
int orc_fluxes(const orc_problem* p, const double* rho, const double* u, const double* v,
               const double* T, double* fx, double* fy)
{
    if (check_problem(p) || !fx || !fy) return -1;
    work w;
    if (work_alloc(&w, p->nx, p->ny)) return -2;
    fill_widths(p, &w);
    load_state(p, &w, rho, u, v, T);
    prepare(p, &w);
    all_face_fluxes(p, &w);
    size_t nfx = (size_t)p->ny * (p->nx + 1), nfy = (size_t)(p->ny + 1) * p->nx;
    for (int k = 0; k < 4; ++k) {
        memcpy(fx + k * nfx, w.fxf[k], nfx * sizeof(double));
        memcpy(fy + k * nfy, w.fyf[k], nfy * sizeof(double));
    }
    work_free(&w);
    return 0;
}

/* Nusselt numbers of the given state.
 *   which = 0..3: wall side W,E,S,N -- the energy flux of step 6 through
 *                 that wall's faces, summed with the face areas, / (chi dT)
 *   which = 4:    Nu_a of Eq. 69, midpoint rule over cells, / (chi dT Lx)
 *   which = 5:    Nu_1/2 -- the same face-column sum at the x-face column
 *                 i = nx/2 (the plane x = L/2 on a symmetric mesh; nx even) */
int orc_nusselt(const orc_problem* p, const double* rho, const double* u, const double* v,
                const double* T, int which, double* nu_out)
{
    if (check_problem(p) || !nu_out || which < 0 || which > 5) return -1;
    if (which == 5 && (p->nx % 2)) return -1;
    work w;
    if (work_alloc(&w, p->nx, p->ny)) return -2;
    fill_widths(p, &w);
    load_state(p, &w, rho, u, v, T);
    prepare(p, &w);
    int nx = p->nx, ny = p->ny;
    double s = 0.0;
    orc_face_out o;
    if (which == SIDE_W || which == SIDE_E || which == 5) {
        int i = which == SIDE_W ? 0 : (which == SIDE_E ? nx : nx / 2);
        for (int j = 0; j < ny; ++j) {
            face_at(p, &w, 0, i, j, &o);
            s += o.flux[3] * w.wy[j + 1];
        }
        s /= p->chi * p->dT;
    } else if (which == SIDE_S || which == SIDE_N) {
        int j = which == SIDE_S ? 0 : ny;
        for (int i = 0; i < nx; ++i) {
            face_at(p, &w, 1, i, j, &o);
            s += o.flux[3] * w.wx[i + 1];
        }
        s /= p->chi * p->dT;
    } else {
        double Lx = p->xf[nx] - p->xf[0];
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double uc = w.q[Q_U][PIDX(&w, i, j)], Tc = w.q[Q_T][PIDX(&w, i, j)];
                double dTdx = w.g[Q_T][0][PIDX(&w, i, j)];
                s += (uc * Tc - p->chi * dTdx) * w.wx[i + 1] * w.wy[j + 1];
            }
        s /= p->chi * p->dT * Lx;
    }
    *nu_out = s;
    work_free(&w);
    return 0;
}
