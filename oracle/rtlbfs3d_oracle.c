/*
 * rtlbfs3d_oracle.c -- plain FP64 CPU oracle of the reconstructed thermal
 * lattice Boltzmann flux solver (RTLBFS) in 3D, on a structured rectilinear
 * (hexahedral) mesh, with the D3Q19 unit lattice at every face (Section 2.1,
 * Eqs. 5-6; Section 3.2; the 3D cubic cavity of Section 4.4).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, literal reference that
 * the CUDA path is checked against.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the product library never
 * links, includes or calls it, and it shares no code with the CUDA path.
 *
 * What it computes, step by step, in the paper's order (Section 3.2):
 *   1. ghost cells for the boundary conditions (one layer per side);
 *   2. face values by inverse-distance weighting, Eq. 56;
 *   3. cell gradients by the discrete Gauss theorem, Eq. 55 (with 1/dV),
 *      over the six faces of a cell;
 *   4. per face: the 19-node D3Q19 unit lattice x_S + e_i h, node values by
 *      the piecewise-linear interpolation of Eq. 29;
 *   5. per face: the predicted variables of Eqs. 46-48, discretised by
 *      second-order central differences on the 19 nodes;
 *   6. per face: the corrector fluxes, the braces of Eqs. 57-59 with their
 *      (tau - 1.5)(X* - X^n) numerical-dissipation terms;
 *   7. explicit update of the cell conservatives plus the Boussinesq source
 *      of Eq. 64;
 *   8. conservative -> primitive and the steady residual.
 *
 * Readings (the 2D oracle's readings, carried to three dimensions):
 *   R1  V_c = Ma * c, c = 1; nu = V_c L sqrt(Pr/Ra), chi = nu/Pr,
 *       beta_g = V_c^2/(dT L)                                     (Eq. 63)
 *   R2  lattice spacing per face h = kappa * min(width_L, width_R) normal
 *       to the face; tau_f = nu/(cs2 h) + 1/2, tau_g likewise (Eqs. 9-10)
 *   R4  Eq. 55 carries the 1/dV the printed form drops
 *   R5  node i of a face sits at x_S + e_i h in the global frame (D3Q19 is
 *       invariant under the 90-degree rotations that map the axes onto
 *       each other); the printed D3Q19 matrix repeats the velocity
 *       (-1, 0, 1) in columns 12 and 14 -- column 14 is read as (-1, 0, -1),
 *       which makes the set the 19 velocities of length 0, 1 and sqrt(2)
 *       with weights 1/3, 1/18, 1/36 (Eq. 6)
 *   R6  Eqs. 46-48 by central differences on the nodes: D_a from the
 *       nodes +-e_a, D_aa from +-e_a and the centre, D_ab (a != b) from the
 *       four nodes +-e_a +-e_b -- exactly the 19 nodes of D3Q19; products
 *       are formed at the nodes
 *   R7  ghosts mirror the adjacent cell with its width: rho even, velocity
 *       odd about the wall velocity, T odd about T_wall (Dirichlet) or even
 *       (adiabatic); ghost gradients: even quantities negate the normal
 *       component, odd ones the two tangential components; periodic sides
 *       copy the opposite cell
 *   R8  wall faces: (rho u_n)* = 0, (rho u_t)* = rho* u_wall,t for both
 *       tangents, and (rho T)* = rho* T_w on Dirichlet walls
 *   R9  the time-n face state of Eqs. 58-59 is the centre node, the face
 *       derivatives the central differences of R6
 *   R10 buoyancy + rho beta_g (T - T_ref) along +g_axis (hot fluid rises);
 *       body force (f_x, f_y, f_z) is an acceleration
 *   R12 residual: R_u = || |u|^{n+1} - |u|^n ||_2 / || |u|^{n+1} ||_2 with
 *       |u| = sqrt(u^2 + v^2 + w^2), R_T likewise; zero denominator -> inf,
 *       a sum that is not a number -> NaN (divergence)
 * Second face stage, scheme = 1: the original TLBFS of Section 2.2 that
 * RTLBFS approximates -- steps 5-6 replaced by (a) D3Q19 equilibria (Eqs.
 * 3-4, c_p = 1) at the nodes x_S - e_i h, i.e. node -e_i of step 4; (b) the
 * predicted variables as their moments, Eqs. 30-32, with the wall rule R8;
 * (c) the fluxes of Eqs. 38-40 with the non-equilibrium parts of Eqs. 33-34.
 *   Nu  a wall's Nusselt number is the energy flux of step 6 summed over
 *       the wall's faces with their areas, times the domain length normal
 *       to the wall, / (chi dT wall area): Eq. 76 with the conductive flux
 *       the scheme puts through the wall.  Eq. 75 takes the same flux
 *       along the wall line at the middle of its first tangential axis,
 *       integrated along the second; with an even cell count there the
 *       line is a face line and the two face rows beside it are averaged.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define CS2 (1.0 / 3.0) /* c_s^2 = c^2/3 with c = 1, Eq. 6 */

enum { BC_DIRICHLET = 0, BC_ADIABATIC = 1, BC_PERIODIC = 2 };
enum { Q_RHO = 0, Q_U = 1, Q_V = 2, Q_W = 3, Q_T = 4, NQ = 5 };

/* Problem description.  Field order is mirrored by the ctypes binding in
 * oracle/__init__.py.  Sides: 0 -x, 1 +x, 2 -y, 3 +y, 4 -z, 5 +z. */
typedef struct {
    int n[3];
    const double* f[3]; /* n[a]+1 face coordinates along axis a, ascending */
    double nu, chi, beta_g, T_ref, dT;
    double dt;    /* macroscopic time step Delta t */
    double kappa; /* h = kappa * min normal width (R2) */
    double force[3];
    int g_axis;        /* buoyancy acts along +g_axis (R10) */
    int bc_kind[6];
    double bc_T[6];
    double bc_u[6][3]; /* wall velocity; its normal component is ignored */
    int scheme;        /* 0 RTLBFS (Section 3.2), 1 TLBFS (Section 2.2) */
} orc3_problem;

/* D3Q19 (Eqs. 5-6 with the reading R5). */
static const int E19[19][3] = {
    {0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},   {0, 0, -1},
    {1, 1, 0},  {-1, 1, 0}, {1, -1, 0}, {-1, -1, 0}, {1, 0, 1},  {-1, 0, 1}, {1, 0, -1},
    {-1, 0, -1}, {0, 1, 1}, {0, -1, 1}, {0, 1, -1},  {0, -1, -1}};

/* ------------------------------------------------------------------ */
/* Working storage: one ghost layer around the nz x ny x nx cells      */
/* ------------------------------------------------------------------ */

typedef struct {
    int n[3], p[3];    /* cells and padded extents (n + 2) */
    double* q[NQ];     /* padded primitives */
    double* g[NQ][3];  /* padded gradients */
    double* w[3];      /* padded widths per axis */
    double* fl[3][NQ]; /* face fluxes normal to axis a: (n[a]+1) faces along a */
} work;

static size_t pidx(const work* w, int i, int j, int k)
{
    return ((size_t)(k + 1) * w->p[1] + (size_t)(j + 1)) * w->p[0] + (size_t)(i + 1);
}

/* flux index of the face normal to axis a at face position (i, j, k)
 * (the index along a runs over n[a]+1 faces) */
static size_t fidx(const work* w, int a, int i, int j, int k)
{
    int ex[3] = {w->n[0], w->n[1], w->n[2]};
    ex[a] += 1;
    return ((size_t)k * ex[1] + (size_t)j) * ex[0] + (size_t)i;
}

static void work_free(work* w)
{
    for (int q = 0; q < NQ; ++q) {
        free(w->q[q]);
        for (int a = 0; a < 3; ++a) {
            free(w->g[q][a]);
            free(w->fl[a][q]);
        }
    }
    for (int a = 0; a < 3; ++a) free(w->w[a]);
}

static int work_alloc(work* w, const int n[3])
{
    memset(w, 0, sizeof(*w));
    for (int a = 0; a < 3; ++a) {
        w->n[a] = n[a];
        w->p[a] = n[a] + 2;
    }
    size_t np = (size_t)w->p[0] * w->p[1] * w->p[2];
    int ok = 1;
    for (int q = 0; q < NQ; ++q) {
        w->q[q] = calloc(np, sizeof(double));
        ok = ok && w->q[q];
        for (int a = 0; a < 3; ++a) {
            w->g[q][a] = calloc(np, sizeof(double));
            size_t nf = (size_t)(n[0] + (a == 0)) * (n[1] + (a == 1)) * (n[2] + (a == 2));
            w->fl[a][q] = calloc(nf, sizeof(double));
            ok = ok && w->g[q][a] && w->fl[a][q];
        }
    }
    for (int a = 0; a < 3; ++a) {
        w->w[a] = calloc((size_t)n[a] + 2, sizeof(double));
        ok = ok && w->w[a];
    }
    if (!ok) {
        work_free(w);
        return -2;
    }
    return 0;
}

static int check_problem(const orc3_problem* p)
{
    if (!p) return -1;
    for (int a = 0; a < 3; ++a) {
        if (p->n[a] < 1 || !p->f[a]) return -1;
        for (int i = 0; i < p->n[a]; ++i)
            if (!(p->f[a][i + 1] > p->f[a][i])) return -1;
        if ((p->bc_kind[2 * a] == BC_PERIODIC) != (p->bc_kind[2 * a + 1] == BC_PERIODIC))
            return -1;
    }
    for (int s = 0; s < 6; ++s)
        if (p->bc_kind[s] < 0 || p->bc_kind[s] > 2) return -1;
    if (p->g_axis < 0 || p->g_axis > 2) return -1;
    if (p->scheme != 0 && p->scheme != 1) return -1;
    if (!(p->kappa > 0.0) || !(p->nu > 0.0) || !(p->chi > 0.0)) return -1;
    return 0;
}

static int periodic(const orc3_problem* p, int a) { return p->bc_kind[2 * a] == BC_PERIODIC; }

/* Cell widths, ghosts included (R7). */
static void fill_widths(const orc3_problem* p, work* w)
{
    for (int a = 0; a < 3; ++a) {
        int n = p->n[a];
        for (int i = 0; i < n; ++i) w->w[a][i + 1] = p->f[a][i + 1] - p->f[a][i];
        w->w[a][0] = periodic(p, a) ? w->w[a][n] : w->w[a][1];
        w->w[a][n + 1] = periodic(p, a) ? w->w[a][1] : w->w[a][n];
    }
}

/* Parity of quantity q about a wall (R7): +1 even, -1 odd. */
static int wall_parity(const orc3_problem* p, int s, int q)
{
    if (q == Q_RHO) return +1;
    if (q == Q_U || q == Q_V || q == Q_W) return -1;
    return p->bc_kind[s] == BC_DIRICHLET ? -1 : +1;
}

/* Value an odd quantity is mirrored about at wall s (R7). */
static double wall_value(const orc3_problem* p, int s, int q)
{
    if (q == Q_T) return p->bc_T[s];
    if (q >= Q_U && q <= Q_W) {
        int comp = q - Q_U;
        return comp == s / 2 ? 0.0 : p->bc_u[s][comp];
    }
    return 0.0;
}

/* Padded position of the ghost across side s of interior position c, and
 * of its partner (the cell it mirrors or copies). */
static void ghost_partner(const orc3_problem* p, int s, const int c[3], int gpos[3], int ppos[3])
{
    int a = s / 2, hi = s % 2, n = p->n[a];
    for (int b = 0; b < 3; ++b) gpos[b] = ppos[b] = c[b];
    gpos[a] = hi ? n : -1;
    if (periodic(p, a))
        ppos[a] = hi ? 0 : n - 1;
    else
        ppos[a] = hi ? n - 1 : 0;
}

/* Step 1: ghost values on the six faces of the box (no edge or corner
 * ghosts are needed: every stencil reaches across one side at a time). */
static void fill_ghost_values(const orc3_problem* p, work* w)
{
    for (int s = 0; s < 6; ++s) {
        int a = s / 2, b1 = (a + 1) % 3, b2 = (a + 2) % 3;
        for (int t2 = 0; t2 < p->n[b2]; ++t2)
            for (int t1 = 0; t1 < p->n[b1]; ++t1) {
                int c[3], gp[3], pp[3];
                c[a] = 0;
                c[b1] = t1;
                c[b2] = t2;
                ghost_partner(p, s, c, gp, pp);
                for (int q = 0; q < NQ; ++q) {
                    double v = w->q[q][pidx(w, pp[0], pp[1], pp[2])];
                    if (!periodic(p, a) && wall_parity(p, s, q) < 0) v = 2.0 * wall_value(p, s, q) - v;
                    w->q[q][pidx(w, gp[0], gp[1], gp[2])] = v;
                }
            }
    }
}

/* Eq. 56: inverse-distance weighting between the two centres sharing a
 * face; the centre-to-face distances are half the cell widths. */
static double eq56_face_value(double phiL, double phiR, double widthL, double widthR)
{
    double dL = 0.5 * widthL, dR = 0.5 * widthR;
    return (phiL * dR + phiR * dL) / (dR + dL);
}

/* Steps 2-3: Eq. 55 with 1/dV over the six faces of every interior cell,
 * outward face-area vectors +-(area) e_a. */
static void interior_gradients(const orc3_problem* p, work* w)
{
    int nx = p->n[0], ny = p->n[1], nz = p->n[2];
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int c[3] = {i, j, k};
                double wd[3] = {w->w[0][i + 1], w->w[1][j + 1], w->w[2][k + 1]};
                double dV = wd[0] * wd[1] * wd[2];
                for (int q = 0; q < NQ; ++q) {
                    const double* f = w->q[q];
                    double phiC = f[pidx(w, i, j, k)];
                    double sum[3] = {0.0, 0.0, 0.0};
                    for (int a = 0; a < 3; ++a) {
                        int cp[3] = {c[0], c[1], c[2]}, cm[3] = {c[0], c[1], c[2]};
                        cp[a] += 1;
                        cm[a] -= 1;
                        double phiP = f[pidx(w, cp[0], cp[1], cp[2])];
                        double phiM = f[pidx(w, cm[0], cm[1], cm[2])];
                        double wP = w->w[a][c[a] + 2], wM = w->w[a][c[a]];
                        double fp = eq56_face_value(phiC, phiP, wd[a], wP);
                        double fm = eq56_face_value(phiM, phiC, wM, wd[a]);
                        double area = dV / wd[a];
                        /* sum_k phi_S dS_k over the +a and -a faces */
                        sum[a] += fp * area - fm * area;
                    }
                    for (int a = 0; a < 3; ++a) w->g[q][a][pidx(w, i, j, k)] = sum[a] / dV;
                }
            }
}

/* Ghost gradients (R7). */
static void fill_ghost_gradients(const orc3_problem* p, work* w)
{
    for (int s = 0; s < 6; ++s) {
        int a = s / 2, b1 = (a + 1) % 3, b2 = (a + 2) % 3;
        for (int t2 = 0; t2 < p->n[b2]; ++t2)
            for (int t1 = 0; t1 < p->n[b1]; ++t1) {
                int c[3], gp[3], pp[3];
                c[a] = 0;
                c[b1] = t1;
                c[b2] = t2;
                ghost_partner(p, s, c, gp, pp);
                size_t gi = pidx(w, gp[0], gp[1], gp[2]), pi = pidx(w, pp[0], pp[1], pp[2]);
                for (int q = 0; q < NQ; ++q)
                    for (int d = 0; d < 3; ++d) {
                        double v = w->g[q][d][pi];
                        if (!periodic(p, a)) {
                            int even = wall_parity(p, s, q) > 0;
                            int normal = d == a;
                            /* even: negate the normal part; odd: the tangential parts */
                            if (even == normal) v = -v;
                        }
                        w->g[q][d][gi] = v;
                    }
            }
    }
}

/* ------------------------------------------------------------------ */
/* Steps 4-6: one face                                                  */
/* ------------------------------------------------------------------ */

enum {
    P_RHO = 0,
    P_M0, P_M1, P_M2,           /* rho u_a */
    P_E,                        /* rho T (c_p = 1) */
    P_X00, P_X01, P_X02, P_X11, P_X12, P_X22, /* rho u_a u_b + rho cs2 delta_ab */
    P_Q0, P_Q1, P_Q2,           /* rho u_a T */
    NPROD
};

/* Everything one face produces; exposed for the unit pins. */
typedef struct {
    double h, tau_f, tau_g;
    double node[NQ][19]; /* primitives at node i = x_S + e_i h */
    double pred[5];      /* rho*, (rho u)*, (rho v)*, (rho w)*, (rho T)* after R8 */
    double flux[5];      /* mass, x-, y-, z-momentum, energy along +normal */
} orc3_face_out;

typedef struct {
    double q[NQ];
    double g[NQ][3];
    double off[3]; /* x_cell - x_S */
} cell_view;

static void take_cell(const work* w, int i, int j, int k, const double off[3], cell_view* c)
{
    size_t id = pidx(w, i, j, k);
    for (int q = 0; q < NQ; ++q) {
        c->q[q] = w->q[q][id];
        for (int d = 0; d < 3; ++d) c->g[q][d] = w->g[q][d][id];
    }
    for (int d = 0; d < 3; ++d) c->off[d] = off[d];
}

/* Eq. 29 extrapolation from a cell to node offset d (relative to x_S). */
static double extrap(const cell_view* c, int q, const double d[3])
{
    double v = c->q[q];
    for (int b = 0; b < 3; ++b) v += c->g[q][b] * (d[b] - c->off[b]);
    return v;
}

/* Step 4 (R5): the 19 nodes x_S + e_i h; the normal component decides the
 * cell (Eq. 29), zero averages both. */
static void face_nodes(int nd, const cell_view* L, const cell_view* R, double h,
                       double node[NQ][19])
{
    for (int i = 0; i < 19; ++i) {
        double d[3] = {E19[i][0] * h, E19[i][1] * h, E19[i][2] * h};
        int side = E19[i][nd];
        for (int q = 0; q < NQ; ++q) {
            double v;
            if (side < 0)
                v = extrap(L, q, d);
            else if (side > 0)
                v = extrap(R, q, d);
            else
                v = 0.5 * (extrap(L, q, d) + extrap(R, q, d));
            node[q][i] = v;
        }
    }
}

/* index of the D3Q19 node with velocity (a, b, c), -1 if there is none;
 * filled by node_table_init() before any parallel region */
static int NODE[3][3][3];
static int node_table_ready = 0;

static void node_table_init(void)
{
    if (node_table_ready) return;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 3; ++c) NODE[a][b][c] = -1;
    for (int i = 0; i < 19; ++i) NODE[E19[i][0] + 1][E19[i][1] + 1][E19[i][2] + 1] = i;
    node_table_ready = 1;
}

static int node_of(int a, int b, int c) { return NODE[a + 1][b + 1][c + 1]; }

/* Steps 5-6 from given node primitives o->node for a face with normal
 * axis nd; wall_side >= 0 marks a boundary face of that side (R8). */
static void face_from_nodes(const orc3_problem* p, int nd, double h, int wall_side,
                            orc3_face_out* o)
{
    o->h = h;
    o->tau_f = p->nu / (CS2 * h) + 0.5;  /* Eq. 9 */
    o->tau_g = p->chi / (CS2 * h) + 0.5; /* Eq. 10 */

    const int M[3] = {P_M0, P_M1, P_M2};
    const int X[3][3] = {{P_X00, P_X01, P_X02}, {P_X01, P_X11, P_X12}, {P_X02, P_X12, P_X22}};
    const int UT[3] = {P_Q0, P_Q1, P_Q2};

    /* products at the nodes (R6) */
    double P[NPROD][19];
    for (int i = 0; i < 19; ++i) {
        double r = o->node[Q_RHO][i], T = o->node[Q_T][i];
        double u[3] = {o->node[Q_U][i], o->node[Q_V][i], o->node[Q_W][i]};
        P[P_RHO][i] = r;
        P[P_E][i] = r * T;
        for (int a = 0; a < 3; ++a) {
            P[M[a]][i] = r * u[a];
            P[UT[a]][i] = r * u[a] * T;
            for (int b = a; b < 3; ++b) P[X[a][b]][i] = r * u[a] * u[b] + (a == b ? r * CS2 : 0.0);
        }
    }

    /* central differences (R6) */
    int e0 = node_of(0, 0, 0);
    double D[NPROD][3], DD[NPROD][3][3];
    for (int k = 0; k < NPROD; ++k)
        for (int a = 0; a < 3; ++a) {
            int ep[3] = {0, 0, 0}, em[3] = {0, 0, 0};
            ep[a] = 1;
            em[a] = -1;
            double fp = P[k][node_of(ep[0], ep[1], ep[2])], fm = P[k][node_of(em[0], em[1], em[2])];
            D[k][a] = (fp - fm) / (2.0 * h);
            DD[k][a][a] = (fp - 2.0 * P[k][e0] + fm) / (h * h);
            for (int b = 0; b < 3; ++b) {
                if (b == a) continue;
                int v[4][3];
                const int sg[4][2] = {{1, 1}, {1, -1}, {-1, 1}, {-1, -1}};
                for (int m = 0; m < 4; ++m) {
                    v[m][0] = v[m][1] = v[m][2] = 0;
                    v[m][a] = sg[m][0];
                    v[m][b] = sg[m][1];
                }
                DD[k][a][b] = (P[k][node_of(v[0][0], v[0][1], v[0][2])] -
                               P[k][node_of(v[1][0], v[1][1], v[1][2])] -
                               P[k][node_of(v[2][0], v[2][1], v[2][2])] +
                               P[k][node_of(v[3][0], v[3][1], v[3][2])]) /
                              (4.0 * h * h);
            }
        }
#define C0(k) (P[(k)][e0]) /* centre node = time-n face state (R9) */

    /* Step 5: predictor, Eqs. 46-48 with dt -> h */
    double rho_s = C0(P_RHO);
    for (int a = 0; a < 3; ++a) rho_s -= h * D[M[a]][a];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) rho_s += 0.5 * h * h * DD[X[a][b]][a][b];

    double m_s[3];
    for (int a = 0; a < 3; ++a) {
        double s = C0(M[a]);
        for (int b = 0; b < 3; ++b) s -= h * D[X[a][b]][b];
        /* d_b[ d_b(rho u_a) + d_a(rho u_b) + d_g(rho u_g) delta_ab ] */
        double br = 0.0;
        for (int b = 0; b < 3; ++b) {
            br += DD[M[a]][b][b];
            br += DD[M[b]][a][b];
        }
        for (int g = 0; g < 3; ++g) br += DD[M[g]][a][g];
        s += 0.5 * CS2 * h * h * br;
        m_s[a] = s;
    }

    double E_s = C0(P_E);
    for (int a = 0; a < 3; ++a) E_s -= h * D[UT[a]][a];
    for (int a = 0; a < 3; ++a) E_s += 0.5 * CS2 * h * h * DD[P_E][a][a];

    /* R8 */
    if (wall_side >= 0) {
        for (int a = 0; a < 3; ++a) m_s[a] = a == nd ? 0.0 : rho_s * p->bc_u[wall_side][a];
        if (p->bc_kind[wall_side] == BC_DIRICHLET) E_s = rho_s * p->bc_T[wall_side];
    }
    o->pred[0] = rho_s;
    for (int a = 0; a < 3; ++a) o->pred[1 + a] = m_s[a];
    o->pred[4] = E_s;
    double us[3] = {m_s[0] / rho_s, m_s[1] / rho_s, m_s[2] / rho_s};
    double Ts = E_s / rho_s;

    /* Step 6: fluxes along the normal, beta = nd (Eqs. 57-59 braces) */
    int be = nd;
    o->flux[0] = m_s[be]; /* Eq. 57 */
    double divm = D[P_M0][0] + D[P_M1][1] + D[P_M2][2];
    for (int a = 0; a < 3; ++a) {
        double X0 = C0(X[a][be]);
        double Xs = rho_s * us[a] * us[be] + (a == be ? rho_s * CS2 : 0.0);
        double visc = D[M[a]][be] + D[M[be]][a] + (a == be ? divm : 0.0);
        o->flux[1 + a] = X0 - p->nu * visc - (o->tau_f - 1.5) * (Xs - X0); /* Eq. 58 */
    }
    {
        double Q0 = C0(UT[be]);
        double Qs = rho_s * us[be] * Ts;
        o->flux[4] = Q0 - p->chi * D[P_E][be] - (o->tau_g - 1.5) * (Qs - Q0); /* Eq. 59 */
    }
#undef C0
}

/* D3Q19 weights of Eq. 6 in the order of E19 */
static double w19(int i) { return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0); }

/* Eq. 3 */
static double f_equilibrium3(int i, double r, const double u[3])
{
    double eu = E19[i][0] * u[0] + E19[i][1] * u[1] + E19[i][2] * u[2];
    double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return w19(i) * r * (1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - usq / (2.0 * CS2));
}

/* Eq. 4 with c_p = 1 */
static double g_equilibrium3(int i, double r, const double u[3], double T)
{
    double eu = E19[i][0] * u[0] + E19[i][1] * u[1] + E19[i][2] * u[2];
    return w19(i) * r * T * (1.0 + eu / CS2);
}

/*
 * TLBFS steps (a)-(c) of Section 2.2 with D3Q19, for a face with normal
 * axis nd, from the node primitives o->node (step 4): (a) equilibria at
 * x_S - e_i dt, which is node -e_i of the lattice (R5); (b) the predicted
 * variables as their moments, Eqs. 30-32, then the wall rule R8; (c) the
 * fluxes of Eqs. 38-40 with the non-equilibrium parts of Eqs. 33-34.
 */
static void face_tlbfs_from_nodes(const orc3_problem* p, int nd, double h, int wall_side,
                                  orc3_face_out* o)
{
    o->h = h;
    o->tau_f = p->nu / (CS2 * h) + 0.5;  /* Eq. 9 */
    o->tau_g = p->chi / (CS2 * h) + 0.5; /* Eq. 10 */
    double fn[19], gn[19];
    for (int i = 0; i < 19; ++i) {
        int j = node_of(-E19[i][0], -E19[i][1], -E19[i][2]);
        double r = o->node[Q_RHO][j], T = o->node[Q_T][j];
        double u[3] = {o->node[Q_U][j], o->node[Q_V][j], o->node[Q_W][j]};
        fn[i] = f_equilibrium3(i, r, u);
        gn[i] = g_equilibrium3(i, r, u, T);
    }
    double rho_s = 0.0, m_s[3] = {0.0, 0.0, 0.0}, E_s = 0.0;
    for (int i = 0; i < 19; ++i) {
        rho_s += fn[i];
        for (int a = 0; a < 3; ++a) m_s[a] += E19[i][a] * fn[i];
        E_s += gn[i];
    }
    if (wall_side >= 0) { /* R8 */
        for (int a = 0; a < 3; ++a) m_s[a] = a == nd ? 0.0 : rho_s * p->bc_u[wall_side][a];
        if (p->bc_kind[wall_side] == BC_DIRICHLET) E_s = rho_s * p->bc_T[wall_side];
    }
    o->pred[0] = rho_s;
    for (int a = 0; a < 3; ++a) o->pred[1 + a] = m_s[a];
    o->pred[4] = E_s;
    double us[3] = {m_s[0] / rho_s, m_s[1] / rho_s, m_s[2] / rho_s};
    double Ts = E_s / rho_s;
    double P = 0.0, Pi[3] = {0.0, 0.0, 0.0}, Q = 0.0;
    for (int i = 0; i < 19; ++i) {
        double fs = f_equilibrium3(i, rho_s, us);
        double gs = g_equilibrium3(i, rho_s, us, Ts);
        double en = E19[i][nd];
        P += en * fs;
        for (int a = 0; a < 3; ++a) Pi[a] += E19[i][a] * en * (fs + (0.5 - o->tau_f) * (fs - fn[i]));
        Q += en * (gs + (0.5 - o->tau_g) * (gs - gn[i]));
    }
    o->flux[0] = P;
    for (int a = 0; a < 3; ++a) o->flux[1 + a] = Pi[a];
    o->flux[4] = Q;
}

/* Steps 5-6 of the selected face stage */
static void face_stage(const orc3_problem* p, int nd, double h, int wall_side, orc3_face_out* o)
{
    if (p->scheme == 1)
        face_tlbfs_from_nodes(p, nd, h, wall_side, o);
    else
        face_from_nodes(p, nd, h, wall_side, o);
}

/* One face normal to axis nd at face position (i, j, k): the face between
 * cell (i, j, k) - e_nd and cell (i, j, k). */
static void face_at(const orc3_problem* p, const work* w, int nd, int i, int j, int k,
                    orc3_face_out* o)
{
    int c[3] = {i, j, k}, cl[3] = {i, j, k};
    cl[nd] -= 1;
    double wl = w->w[nd][c[nd]], wr = w->w[nd][c[nd] + 1]; /* padded: cell c-1 is index c */
    double offL[3] = {0.0, 0.0, 0.0}, offR[3] = {0.0, 0.0, 0.0};
    offL[nd] = -0.5 * wl;
    offR[nd] = 0.5 * wr;
    cell_view L, R;
    take_cell(w, cl[0], cl[1], cl[2], offL, &L);
    take_cell(w, c[0], c[1], c[2], offR, &R);
    double h = p->kappa * (wl < wr ? wl : wr);
    int wall = -1;
    if (!periodic(p, nd)) {
        if (c[nd] == 0) wall = 2 * nd;
        if (c[nd] == p->n[nd]) wall = 2 * nd + 1;
    }
    face_nodes(nd, &L, &R, h, o->node);
    face_stage(p, nd, h, wall, o);
}

static void all_face_fluxes(const orc3_problem* p, work* w)
{
    for (int a = 0; a < 3; ++a) {
        int ex[3] = {p->n[0], p->n[1], p->n[2]};
        ex[a] += 1;
#pragma omp parallel for schedule(static)
        for (int k = 0; k < ex[2]; ++k) {
            orc3_face_out o;
            for (int j = 0; j < ex[1]; ++j)
                for (int i = 0; i < ex[0]; ++i) {
                    face_at(p, w, a, i, j, k, &o);
                    for (int q = 0; q < NQ; ++q) w->fl[a][q][fidx(w, a, i, j, k)] = o.flux[q];
                }
        }
    }
}

static void prepare(const orc3_problem* p, work* w)
{
    fill_ghost_values(p, w);
    interior_gradients(p, w);
    fill_ghost_gradients(p, w);
}

static void load_state(const orc3_problem* p, work* w, double* const st[NQ])
{
    int nx = p->n[0], ny = p->n[1], nz = p->n[2];
    for (int q = 0; q < NQ; ++q)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i)
                    w->q[q][pidx(w, i, j, k)] = st[q][((size_t)k * ny + j) * nx + i];
}

/* Steps 7-8 for every cell, residual sums of R12. */
static void update_cells(const orc3_problem* p, work* w, double* const st[NQ], double res[2])
{
    int nx = p->n[0], ny = p->n[1], nz = p->n[2];
    double su_num = 0.0, su_den = 0.0, sT_num = 0.0, sT_den = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : su_num, su_den, sT_num, sT_den)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int c[3] = {i, j, k};
                double wd[3] = {w->w[0][i + 1], w->w[1][j + 1], w->w[2][k + 1]};
                double dV = wd[0] * wd[1] * wd[2];
                size_t id = pidx(w, i, j, k);
                double r = w->q[Q_RHO][id], T = w->q[Q_T][id];
                double u[3] = {w->q[Q_U][id], w->q[Q_V][id], w->q[Q_W][id]};
                double Wc[5] = {r, r * u[0], r * u[1], r * u[2], r * T};
                double sum[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
                for (int a = 0; a < 3; ++a) {
                    int cp[3] = {c[0], c[1], c[2]};
                    cp[a] += 1;
                    double area = dV / wd[a];
                    for (int q = 0; q < NQ; ++q) {
                        double Fp = w->fl[a][q][fidx(w, a, cp[0], cp[1], cp[2])];
                        double Fm = w->fl[a][q][fidx(w, a, c[0], c[1], c[2])];
                        sum[q] += Fp * area - Fm * area;
                    }
                }
                /* Boussinesq source (Eq. 64, sign by R10) and body force */
                double S[5] = {0.0, r * p->force[0], r * p->force[1], r * p->force[2], 0.0};
                S[1 + p->g_axis] += r * p->beta_g * (T - p->T_ref);
                double Wn[5];
                for (int q = 0; q < 5; ++q) Wn[q] = Wc[q] - p->dt / dV * sum[q] + p->dt * S[q];
                double r1 = Wn[0], T1 = Wn[4] / r1;
                double u1[3] = {Wn[1] / r1, Wn[2] / r1, Wn[3] / r1};
                size_t o = ((size_t)k * ny + j) * nx + i;
                st[Q_RHO][o] = r1;
                st[Q_U][o] = u1[0];
                st[Q_V][o] = u1[1];
                st[Q_W][o] = u1[2];
                st[Q_T][o] = T1;
                double m0 = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
                double m1 = sqrt(u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
                su_num += (m1 - m0) * (m1 - m0);
                su_den += m1 * m1;
                sT_num += (T1 - T) * (T1 - T);
                sT_den += T1 * T1;
            }
    res[0] = su_den > 0.0 ? sqrt(su_num) / sqrt(su_den) : INFINITY;
    res[1] = sT_den > 0.0 ? sqrt(sT_num) / sqrt(sT_den) : INFINITY;
    if (isnan(su_num) || isnan(su_den)) res[0] = NAN;
    if (isnan(sT_num) || isnan(sT_den)) res[1] = NAN;
}

/* ------------------------------------------------------------------ */
/* Public entry points (the state is five arrays of nz*ny*nx, x fastest)*/
/* ------------------------------------------------------------------ */

static int all_finite(const orc3_problem* p, double* const st[NQ])
{
    size_t n = (size_t)p->n[0] * p->n[1] * p->n[2];
    for (int q = 0; q < NQ; ++q)
        for (size_t c = 0; c < n; ++c)
            if (!isfinite(st[q][c])) return 0;
    return 1;
}

/* Advance nsteps in place; res = (R_u, R_T) of the last step.  Returns 0,
 * -1 bad arguments, -2 allocation failure, -4 the state became non-finite. */
int orc3_step(const orc3_problem* p, double* rho, double* u, double* v, double* w_, double* T,
              long nsteps, double* res)
{
    node_table_init();
    double* st[NQ] = {rho, u, v, w_, T};
    if (check_problem(p) || !rho || !u || !v || !w_ || !T || nsteps < 0) return -1;
    work w;
    if (work_alloc(&w, p->n)) return -2;
    fill_widths(p, &w);
    double r2[2] = {NAN, NAN};
    int rc = 0;
    for (long s = 0; s < nsteps; ++s) {
        load_state(p, &w, st);
        prepare(p, &w);
        all_face_fluxes(p, &w);
        update_cells(p, &w, st, r2);
        if (isnan(r2[0]) || isnan(r2[1])) {
            rc = -4;
            break;
        }
    }
    if (rc == 0 && !all_finite(p, st)) rc = -4;
    if (res) {
        res[0] = r2[0];
        res[1] = r2[1];
    }
    work_free(&w);
    return rc;
}

/* Step until max(R_u, R_T) < tol or max_steps.  Returns 0 converged,
 * -5 max_steps reached, -4 diverged. */
int orc3_run_to_steady(const orc3_problem* p, double* rho, double* u, double* v, double* w_,
                       double* T, double tol, long max_steps, long* steps, double* res)
{
    node_table_init();
    double* st[NQ] = {rho, u, v, w_, T};
    if (check_problem(p) || !rho || !u || !v || !w_ || !T || max_steps < 0) return -1;
    work w;
    if (work_alloc(&w, p->n)) return -2;
    fill_widths(p, &w);
    double r2[2] = {INFINITY, INFINITY};
    long s = 0;
    int rc = -5;
    while (s < max_steps) {
        load_state(p, &w, st);
        prepare(p, &w);
        all_face_fluxes(p, &w);
        update_cells(p, &w, st, r2);
        ++s;
        if (isnan(r2[0]) || isnan(r2[1])) {
            rc = -4;
            break;
        }
        double m = r2[0] > r2[1] ? r2[0] : r2[1];
        if (m < tol) {
            rc = 0;
            break;
        }
    }
    if (steps) *steps = s;
    if (res) {
        res[0] = r2[0];
        res[1] = r2[1];
    }
    work_free(&w);
    return rc;
}

/* Eq. 55 gradients: out has 15 planes of nz*ny*nx, order
 * [q][d] = d/dx rho, d/dy rho, d/dz rho, d/dx u, ... d/dz T. */
int orc3_gradients(const orc3_problem* p, double* rho, double* u, double* v, double* w_,
                   double* T, double* out)
{
    node_table_init();
    double* st[NQ] = {rho, u, v, w_, T};
    if (check_problem(p) || !out) return -1;
    work w;
    if (work_alloc(&w, p->n)) return -2;
    fill_widths(p, &w);
    load_state(p, &w, st);
    prepare(p, &w);
    int nx = p->n[0], ny = p->n[1], nz = p->n[2];
    size_t n = (size_t)nx * ny * nz;
    for (int q = 0; q < NQ; ++q)
        for (int d = 0; d < 3; ++d)
            for (int k = 0; k < nz; ++k)
                for (int j = 0; j < ny; ++j)
                    for (int i = 0; i < nx; ++i)
                        out[(size_t)(3 * q + d) * n + ((size_t)k * ny + j) * nx + i] =
                            w.g[q][d][pidx(&w, i, j, k)];
    work_free(&w);
    return 0;
}

/* One face of the given state: normal axis nd, face position (i, j, k)
 * with the index along nd in [0, n[nd]] (the face between cells c - e_nd
 * and c); fills *o. */
int orc3_face(const orc3_problem* p, double* rho, double* u, double* v, double* w_, double* T,
              int nd, int i, int j, int k, orc3_face_out* o)
{
    node_table_init();
    double* st[NQ] = {rho, u, v, w_, T};
    if (check_problem(p) || !o || nd < 0 || nd > 2) return -1;
    int c[3] = {i, j, k};
    for (int a = 0; a < 3; ++a)
        if (c[a] < 0 || c[a] > p->n[a] - (a == nd ? 0 : 1)) return -1;
    work w;
    if (work_alloc(&w, p->n)) return -2;
    fill_widths(p, &w);
    load_state(p, &w, st);
    prepare(p, &w);
    face_at(p, &w, nd, i, j, k, o);
    work_free(&w);
    return 0;
}

/* Steps 5-6 alone from caller-given node primitives nodes[q][i] (q = rho,
 * u, v, w, T; i the D3Q19 index), spacing h, normal nd, wall_side (-1:
 * interior). */
int orc3_face_from_nodes(const orc3_problem* p, int nd, const double* nodes, double h,
                         int wall_side, orc3_face_out* o)
{
    node_table_init();
    if (!p || !nodes || !o || nd < 0 || nd > 2 || !(h > 0.0) || wall_side < -1 || wall_side > 5)
        return -1;
    memcpy(o->node, nodes, sizeof(o->node));
    face_stage(p, nd, h, wall_side, o);
    return 0;
}

/* The D3Q19 velocity set of R5, 57 ints [i][axis]. */
int orc3_lattice(int* out)
{
    if (!out) return -1;
    memcpy(out, E19, sizeof(E19));
    return 0;
}

/* All face fluxes: out[a] has 5 planes of the faces normal to axis a
 * ((nz + [a==2]) x (ny + [a==1]) x (nx + [a==0]), x fastest). */
int orc3_fluxes(const orc3_problem* p, double* rho, double* u, double* v, double* w_, double* T,
                double* fx, double* fy, double* fz)
{
    node_table_init();
    double* st[NQ] = {rho, u, v, w_, T};
    double* out[3] = {fx, fy, fz};
    if (check_problem(p) || !fx || !fy || !fz) return -1;
    work w;
    if (work_alloc(&w, p->n)) return -2;
    fill_widths(p, &w);
    load_state(p, &w, st);
    prepare(p, &w);
    all_face_fluxes(p, &w);
    for (int a = 0; a < 3; ++a) {
        size_t nf = (size_t)(p->n[0] + (a == 0)) * (p->n[1] + (a == 1)) * (p->n[2] + (a == 2));
        for (int q = 0; q < NQ; ++q) memcpy(out[a] + q * nf, w.fl[a][q], nf * sizeof(double));
    }
    work_free(&w);
    return 0;
}

/* Nusselt numbers (see "Nu" in the header comment).
 *   side 0..5, mid = 0: the whole wall (Eq. 76);
 *   side 0..5, mid = 1: the wall line at the middle of the first
 *                       tangential axis (Eq. 75);
 *   side 6,    mid = 0: the x-normal face plane at i = nx/2 (nx even), the
 *                       same sum as a wall of side 0 or 1.
 * Signed along +axis, so heat flowing towards +x is positive. */
int orc3_nusselt(const orc3_problem* p, double* rho, double* u, double* v, double* w_,
                 double* T, int side, int mid, double* nu_out)
{
    node_table_init();
    double* st[NQ] = {rho, u, v, w_, T};
    if (check_problem(p) || !nu_out || side < 0 || side > 6 || mid < 0 || mid > 1) return -1;
    if (side == 6 && (mid || p->n[0] % 2)) return -1;
    int a = side == 6 ? 0 : side / 2;
    if (side < 6 && periodic(p, a)) return -1;
    int b1 = (a + 1) % 3, b2 = (a + 2) % 3;
    int pos = side == 6 ? p->n[0] / 2 : (side % 2 ? p->n[a] : 0);
    work w;
    if (work_alloc(&w, p->n)) return -2;
    fill_widths(p, &w);
    load_state(p, &w, st);
    prepare(p, &w);
    double L[3];
    for (int d = 0; d < 3; ++d) L[d] = p->f[d][p->n[d]] - p->f[d][0];
    double s = 0.0;
    orc3_face_out o;
    if (!mid) {
        for (int t2 = 0; t2 < p->n[b2]; ++t2)
            for (int t1 = 0; t1 < p->n[b1]; ++t1) {
                int c[3];
                c[a] = pos;
                c[b1] = t1;
                c[b2] = t2;
                face_at(p, &w, a, c[0], c[1], c[2], &o);
                s += o.flux[4] * w.w[b1][t1 + 1] * w.w[b2][t2 + 1];
            }
        s *= L[a] / (p->chi * p->dT * L[b1] * L[b2]);
    } else {
        int n1 = p->n[b1];
        int rows[2] = {n1 / 2 - 1, n1 / 2};
        int nr = 2;
        if (n1 % 2) {
            rows[0] = n1 / 2;
            nr = 1;
        }
        for (int r = 0; r < nr; ++r)
            for (int t2 = 0; t2 < p->n[b2]; ++t2) {
                int c[3];
                c[a] = pos;
                c[b1] = rows[r];
                c[b2] = t2;
                face_at(p, &w, a, c[0], c[1], c[2], &o);
                s += o.flux[4] * w.w[b2][t2 + 1] / nr;
            }
        s *= L[a] / (p->chi * p->dT * L[b2]);
    }
    *nu_out = s;
    work_free(&w);
    return 0;
}
