/*
 * rtlbfs_curv_oracle.c -- plain FP64 CPU oracle of 2D RTLBFS on a structured
 * curvilinear (body-fitted) quadrilateral mesh: the O-type meshes of
 * Section 4.3 (the heated circular cylinder) and of concentric annuli.
 *
 * TEST INFRASTRUCTURE ONLY.  The slow, literal reference the CUDA path is
 * checked against; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark load it.  It shares no code with the CUDA path.
 *
 * Mesh: cells (i, j), i < ni, j < nj, with vertices X, Y of shape
 * (nj+1) x (ni+1), right-handed (i and j increase like x and y).  The i
 * direction is periodic -- the seam of an O-mesh, whose vertex column ni is
 * column 0, or a translation by X[j][ni] - X[j][0] -- or bounded by sides 0
 * (i = 0) and 1 (i = ni);
 * the j direction is bounded by sides 2 (j = 0, e.g. the cylinder) and 3
 * (j = nj, e.g. the far field).
 *
 * Steps, in the paper's order (Section 3.2), for general faces:
 *   1. ghost cells: a wall ghost is the mirror image of the adjacent cell P
 *      across the face line (centre reflected, rho even, velocity odd about
 *      the wall velocity, T odd about T_wall or even); a far-field ghost
 *      holds the free-stream state with zero gradient;
 *   2. face values by Eq. 56 with Euclidean centre-to-face distances;
 *   3. Eq. 55 with 1/dV: sum over the four faces of phi_S times the outward
 *      face vector;
 *   4. per face: the 9-node lattice in the face's local frame (n, t) --
 *      node (a, b) at x_S + (a n + b t) h -- with node values by Eq. 29 from
 *      the cell whose side of the face the node lies on (a < 0: L, a > 0:
 *      R, a = 0: their mean), using the full offset x_node - x_cell;
 *   5. Eqs. 46-48 by central differences on the nodes, with the velocity in
 *      the frame (u_n, u_t);
 *   6. the Eq. 57-59 braces along n, rotated back to x, y;
 *   7. the update with the face lengths and cell areas, plus the Boussinesq
 *      source along the gravity direction;
 *   8. the residual of R12.
 *
 * Readings (besides those of the rectilinear oracle):
 *   C1  cell centres are the vertex averages; cell areas the shoelace
 *       formula; face centres the edge midpoints
 *   C2  lattice spacing h = kappa * min(w_L, w_R), with w = twice the
 *       normal distance from a centre to the face (the cell width normal to
 *       the face on a rectilinear mesh)
 *   C3  the local frame is the face's unit normal n (from L to R) and
 *       t = (-n_y, n_x); the wall rule R8 acts on the frame components
 *   C4  wall ghost gradients: even quantities reflect the normal component
 *       (g - 2 (g.n) n), odd quantities the tangential one (2 (g.n) n - g);
 *       on a rectilinear mesh this is R7
 *   C5  the far field (Section 4.3: 52.5 D from the cylinder) is a ghost
 *       layer at the free-stream state with zero gradients
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define CS2 (1.0 / 3.0)

enum { CB_DIRICHLET = 0, CB_ADIABATIC = 1, CB_PERIODIC = 2, CB_FARFIELD = 3 };

/* Field order mirrored by the ctypes binding (oracle/curv.py). */
typedef struct {
    int ni, nj;
    const double* X; /* (nj+1) x (ni+1) vertex coordinates, row-major */
    const double* Y;
    double nu, chi, beta_g, T_ref, dT;
    double dt, kappa;
    double gdir[2];  /* unit direction of the buoyancy + rho beta_g (T - T_ref) */
    double force[2]; /* body acceleration */
    int bc_kind[4];  /* sides: 0 i = 0, 1 i = ni, 2 j = 0, 3 j = nj */
    double bc_T[4];
    double bc_u[4][2]; /* wall velocity (x, y) */
    double inf[4];     /* free-stream rho, u, v, T of far-field sides */
} orcc_problem;

typedef struct {
    int ni, nj, pi; /* padded row length ni + 2 */
    double *cx, *cy, *area;    /* padded cell centres and areas (ghosts mirrored) */
    double* q[4];              /* padded primitives rho, u, v, T */
    double* g[4][2];           /* padded gradients */
    double* fi[4];             /* fluxes of the i-faces: nj rows of ni + 1 */
    double* fj[4];             /* fluxes of the j-faces: nj + 1 rows of ni */
} cwork;

#define CP(w, i, j) ((size_t)((j) + 1) * (size_t)(w)->pi + (size_t)((i) + 1))
#define VX(p, i, j) ((p)->X[(size_t)(j) * ((p)->ni + 1) + (size_t)(i)])
#define VY(p, i, j) ((p)->Y[(size_t)(j) * ((p)->ni + 1) + (size_t)(i)])

static int iper(const orcc_problem* p) { return p->bc_kind[0] == CB_PERIODIC; }

static void cfree(cwork* w)
{
    free(w->cx);
    free(w->cy);
    free(w->area);
    for (int q = 0; q < 4; ++q) {
        free(w->q[q]);
        free(w->g[q][0]);
        free(w->g[q][1]);
        free(w->fi[q]);
        free(w->fj[q]);
    }
}

static int calloc_work(cwork* w, int ni, int nj)
{
    memset(w, 0, sizeof(*w));
    w->ni = ni;
    w->nj = nj;
    w->pi = ni + 2;
    size_t np = (size_t)(ni + 2) * (size_t)(nj + 2);
    int ok = 1;
    w->cx = calloc(np, sizeof(double));
    w->cy = calloc(np, sizeof(double));
    w->area = calloc(np, sizeof(double));
    ok = w->cx && w->cy && w->area;
    for (int q = 0; q < 4; ++q) {
        w->q[q] = calloc(np, sizeof(double));
        w->g[q][0] = calloc(np, sizeof(double));
        w->g[q][1] = calloc(np, sizeof(double));
        w->fi[q] = calloc((size_t)nj * (ni + 1), sizeof(double));
        w->fj[q] = calloc((size_t)(nj + 1) * ni, sizeof(double));
        ok = ok && w->q[q] && w->g[q][0] && w->g[q][1] && w->fi[q] && w->fj[q];
    }
    if (!ok) {
        cfree(w);
        return -2;
    }
    return 0;
}

static int check(const orcc_problem* p)
{
    if (!p || p->ni < 1 || p->nj < 1 || !p->X || !p->Y) return -1;
    for (int s = 0; s < 4; ++s)
        if (p->bc_kind[s] < 0 || p->bc_kind[s] > 3) return -1;
    if ((p->bc_kind[0] == CB_PERIODIC) != (p->bc_kind[1] == CB_PERIODIC)) return -1;
    if (p->bc_kind[2] == CB_PERIODIC || p->bc_kind[3] == CB_PERIODIC) return -1;
    if (!(p->kappa > 0.0) || !(p->nu > 0.0) || !(p->chi > 0.0)) return -1;
    return 0;
}

/* Face f of cell side: the edge from vertex A to vertex B.  i-face at
 * vertex column i, row j: (i, j) -> (i, j+1); j-face at vertex row j,
 * column i: (i, j) -> (i+1, j). */
static void iface_edge(const orcc_problem* p, int i, int j, double* ax, double* ay, double* bx,
                       double* by)
{
    *ax = VX(p, i, j);
    *ay = VY(p, i, j);
    *bx = VX(p, i, j + 1);
    *by = VY(p, i, j + 1);
}

static void jface_edge(const orcc_problem* p, int i, int j, double* ax, double* ay, double* bx,
                       double* by)
{
    *ax = VX(p, i, j);
    *ay = VY(p, i, j);
    *bx = VX(p, i + 1, j);
    *by = VY(p, i + 1, j);
}

/* Face vector of an edge pointing from the cell on the low-index side to
 * the high-index side: for an i-face (edge going up in j) it is the edge
 * rotated clockwise, for a j-face (edge going up in i) counter-clockwise;
 * on a right-handed mesh both point towards increasing index. */
static void face_vector(int kind, double ax, double ay, double bx, double by, double S[2])
{
    double dx = bx - ax, dy = by - ay;
    if (kind == 0) {
        S[0] = dy;
        S[1] = -dx;
    } else {
        S[0] = -dy;
        S[1] = dx;
    }
}

/* Reflection of point (px, py) across the line through (ax, ay), (bx, by). */
static void reflect(double px, double py, double ax, double ay, double bx, double by, double* rx,
                    double* ry)
{
    double dx = bx - ax, dy = by - ay, L2 = dx * dx + dy * dy;
    double s = ((px - ax) * dx + (py - ay) * dy) / L2;
    double fx = ax + s * dx, fy = ay + s * dy; /* foot of the perpendicular */
    *rx = 2.0 * fx - px;
    *ry = 2.0 * fy - py;
}

/* C1: centres and areas of all cells, ghosts mirrored (or wrapped).
 * Returns -1 unless every cell has a positive area (a right-handed mesh:
 * i and j increase like x and y), which the face orientation assumes. */
static int geometry(const orcc_problem* p, cwork* w)
{
    int ni = p->ni, nj = p->nj;
    for (int j = 0; j < nj; ++j)
        for (int i = 0; i < ni; ++i) {
            double x0 = VX(p, i, j), y0 = VY(p, i, j), x1 = VX(p, i + 1, j), y1 = VY(p, i + 1, j);
            double x2 = VX(p, i + 1, j + 1), y2 = VY(p, i + 1, j + 1), x3 = VX(p, i, j + 1),
                   y3 = VY(p, i, j + 1);
            size_t c = CP(w, i, j);
            w->cx[c] = 0.25 * (x0 + x1 + x2 + x3);
            w->cy[c] = 0.25 * (y0 + y1 + y2 + y3);
            w->area[c] = 0.5 * ((x0 * y1 - x1 * y0) + (x1 * y2 - x2 * y1) + (x2 * y3 - x3 * y2) +
                                (x3 * y0 - x0 * y3));
        }
    /* i-direction ghosts */
    for (int j = 0; j < nj; ++j) {
        if (iper(p)) {
            /* the opposite cell, moved by the seam's period (zero on an
             * O-mesh, whose last vertex column is its first) */
            double sx = VX(p, ni, j) - VX(p, 0, j), sy = VY(p, ni, j) - VY(p, 0, j);
            w->cx[CP(w, -1, j)] = w->cx[CP(w, ni - 1, j)] - sx;
            w->cy[CP(w, -1, j)] = w->cy[CP(w, ni - 1, j)] - sy;
            w->cx[CP(w, ni, j)] = w->cx[CP(w, 0, j)] + sx;
            w->cy[CP(w, ni, j)] = w->cy[CP(w, 0, j)] + sy;
        } else {
            double ax, ay, bx, by;
            iface_edge(p, 0, j, &ax, &ay, &bx, &by);
            reflect(w->cx[CP(w, 0, j)], w->cy[CP(w, 0, j)], ax, ay, bx, by, &w->cx[CP(w, -1, j)],
                    &w->cy[CP(w, -1, j)]);
            iface_edge(p, ni, j, &ax, &ay, &bx, &by);
            reflect(w->cx[CP(w, ni - 1, j)], w->cy[CP(w, ni - 1, j)], ax, ay, bx, by,
                    &w->cx[CP(w, ni, j)], &w->cy[CP(w, ni, j)]);
        }
        w->area[CP(w, -1, j)] = w->area[CP(w, iper(p) ? ni - 1 : 0, j)];
        w->area[CP(w, ni, j)] = w->area[CP(w, iper(p) ? 0 : ni - 1, j)];
    }
    for (int i = 0; i < ni; ++i) {
        double ax, ay, bx, by;
        jface_edge(p, i, 0, &ax, &ay, &bx, &by);
        reflect(w->cx[CP(w, i, 0)], w->cy[CP(w, i, 0)], ax, ay, bx, by, &w->cx[CP(w, i, -1)],
                &w->cy[CP(w, i, -1)]);
        jface_edge(p, i, nj, &ax, &ay, &bx, &by);
        reflect(w->cx[CP(w, i, nj - 1)], w->cy[CP(w, i, nj - 1)], ax, ay, bx, by,
                &w->cx[CP(w, i, nj)], &w->cy[CP(w, i, nj)]);
        w->area[CP(w, i, -1)] = w->area[CP(w, i, 0)];
        w->area[CP(w, i, nj)] = w->area[CP(w, i, nj - 1)];
    }
    for (int j = 0; j < nj; ++j)
        for (int i = 0; i < ni; ++i)
            if (!(w->area[CP(w, i, j)] > 0.0)) return -1;
    return 0;
}

static int odd_q(const orcc_problem* p, int side, int q)
{
    if (q == 0) return 0;
    if (q == 1 || q == 2) return 1;
    return p->bc_kind[side] == CB_DIRICHLET;
}

/* Step 1: ghost values (no corner ghosts are used). */
static void ghost_values(const orcc_problem* p, cwork* w)
{
    int ni = p->ni, nj = p->nj;
    for (int j = 0; j < nj; ++j)
        for (int s = 0; s < 2; ++s) {
            int gi = s ? ni : -1, pi_ = s ? ni - 1 : 0, wi = s ? 0 : ni - 1;
            for (int q = 0; q < 4; ++q) {
                double v;
                if (iper(p))
                    v = w->q[q][CP(w, wi, j)];
                else if (p->bc_kind[s] == CB_FARFIELD)
                    v = p->inf[q];
                else {
                    v = w->q[q][CP(w, pi_, j)];
                    if (odd_q(p, s, q)) {
                        double wv = q == 3 ? p->bc_T[s] : p->bc_u[s][q - 1];
                        v = 2.0 * wv - v;
                    }
                }
                w->q[q][CP(w, gi, j)] = v;
            }
        }
    for (int i = 0; i < ni; ++i)
        for (int s = 2; s < 4; ++s) {
            int gj = s == 3 ? nj : -1, pj = s == 3 ? nj - 1 : 0;
            for (int q = 0; q < 4; ++q) {
                double v;
                if (p->bc_kind[s] == CB_FARFIELD)
                    v = p->inf[q];
                else {
                    v = w->q[q][CP(w, i, pj)];
                    if (odd_q(p, s, q)) {
                        double wv = q == 3 ? p->bc_T[s] : p->bc_u[s][q - 1];
                        v = 2.0 * wv - v;
                    }
                }
                w->q[q][CP(w, i, gj)] = v;
            }
        }
}

/* Eq. 56 at the midpoint (mx, my) of a face between centres L and R. */
static double eq56(double phiL, double phiR, double xl, double yl, double xr, double yr, double mx,
                   double my)
{
    double dL = hypot(xl - mx, yl - my), dR = hypot(xr - mx, yr - my);
    return (phiL * dR + phiR * dL) / (dR + dL);
}

/* Steps 2-3: Eq. 55 over the four faces of every interior cell. */
static void gradients(const orcc_problem* p, cwork* w)
{
    int ni = p->ni, nj = p->nj;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < nj; ++j)
        for (int i = 0; i < ni; ++i) {
            size_t c = CP(w, i, j);
            /* the four faces: (neighbour, edge, sign of the face vector) */
            struct {
                int ni_, nj_;
                int kind, fi, fj;
                double sign;
            } F[4] = {{i - 1, j, 0, i, j, -1.0},
                      {i + 1, j, 0, i + 1, j, 1.0},
                      {i, j - 1, 1, i, j, -1.0},
                      {i, j + 1, 1, i, j + 1, 1.0}};
            for (int q = 0; q < 4; ++q) {
                double sx = 0.0, sy = 0.0;
                for (int k = 0; k < 4; ++k) {
                    double ax, ay, bx, by, S[2];
                    if (F[k].kind == 0)
                        iface_edge(p, F[k].fi, F[k].fj, &ax, &ay, &bx, &by);
                    else
                        jface_edge(p, F[k].fi, F[k].fj, &ax, &ay, &bx, &by);
                    face_vector(F[k].kind, ax, ay, bx, by, S);
                    size_t nb = CP(w, F[k].ni_, F[k].nj_);
                    double mx = 0.5 * (ax + bx), my = 0.5 * (ay + by);
                    double phiS = eq56(w->q[q][c], w->q[q][nb], w->cx[c], w->cy[c], w->cx[nb],
                                       w->cy[nb], mx, my);
                    sx += phiS * F[k].sign * S[0];
                    sy += phiS * F[k].sign * S[1];
                }
                w->g[q][0][c] = sx / w->area[c];
                w->g[q][1][c] = sy / w->area[c];
            }
        }
}

/* Ghost gradients: wrapped (periodic), zero (far field) or mirrored across
 * the boundary face with unit normal n (C4). */
static void ghost_gradients(const orcc_problem* p, cwork* w)
{
    int ni = p->ni, nj = p->nj;
    for (int j = 0; j < nj; ++j)
        for (int s = 0; s < 2; ++s) {
            int gi = s ? ni : -1, pi_ = s ? ni - 1 : 0, wi = s ? 0 : ni - 1;
            double ax, ay, bx, by, S[2];
            iface_edge(p, s ? ni : 0, j, &ax, &ay, &bx, &by);
            face_vector(0, ax, ay, bx, by, S);
            double L = hypot(S[0], S[1]), nx = S[0] / L, ny = S[1] / L;
            for (int q = 0; q < 4; ++q) {
                double gx, gy;
                if (iper(p)) {
                    gx = w->g[q][0][CP(w, wi, j)];
                    gy = w->g[q][1][CP(w, wi, j)];
                } else if (p->bc_kind[s] == CB_FARFIELD) {
                    gx = gy = 0.0;
                } else {
                    double px = w->g[q][0][CP(w, pi_, j)], py = w->g[q][1][CP(w, pi_, j)];
                    double gn = px * nx + py * ny;
                    gx = px - 2.0 * gn * nx;
                    gy = py - 2.0 * gn * ny;
                    if (odd_q(p, s, q)) {
                        gx = -gx;
                        gy = -gy;
                    }
                }
                w->g[q][0][CP(w, gi, j)] = gx;
                w->g[q][1][CP(w, gi, j)] = gy;
            }
        }
    for (int i = 0; i < ni; ++i)
        for (int s = 2; s < 4; ++s) {
            int gj = s == 3 ? nj : -1, pj = s == 3 ? nj - 1 : 0;
            double ax, ay, bx, by, S[2];
            jface_edge(p, i, s == 3 ? nj : 0, &ax, &ay, &bx, &by);
            face_vector(1, ax, ay, bx, by, S);
            double L = hypot(S[0], S[1]), nx = S[0] / L, ny = S[1] / L;
            for (int q = 0; q < 4; ++q) {
                double gx, gy;
                if (p->bc_kind[s] == CB_FARFIELD) {
                    gx = gy = 0.0;
                } else {
                    double px = w->g[q][0][CP(w, i, pj)], py = w->g[q][1][CP(w, i, pj)];
                    double gn = px * nx + py * ny;
                    gx = px - 2.0 * gn * nx;
                    gy = py - 2.0 * gn * ny;
                    if (odd_q(p, s, q)) {
                        gx = -gx;
                        gy = -gy;
                    }
                }
                w->g[q][0][CP(w, i, gj)] = gx;
                w->g[q][1][CP(w, i, gj)] = gy;
            }
        }
}

/* Everything one face produces (exposed for the pins). */
typedef struct {
    double h, tau_f, tau_g;
    double n[2];           /* unit normal, from L to R */
    double len;            /* face length |dS| */
    double node[4][3][3];  /* frame primitives rho, u_n, u_t, T at node (a, b) */
    double pred[4];        /* rho*, (rho u_n)*, (rho u_t)*, (rho T)* after R8 */
    double flux[4];        /* mass, x-momentum, y-momentum, energy along n */
} orcc_face_out;

/* Steps 4-6 for the face with centre (mx, my), unit normal n, between
 * padded cells cl and cr; wall_side >= 0 on a wall face. */
static void face_compute(const orcc_problem* p, const cwork* w, size_t cl, size_t cr, double mx,
                         double my, const double n[2], int wall_side, orcc_face_out* o)
{
    double t[2] = {-n[1], n[0]};
    /* C2: widths normal to the face */
    double wl = 2.0 * fabs((mx - w->cx[cl]) * n[0] + (my - w->cy[cl]) * n[1]);
    double wr = 2.0 * fabs((w->cx[cr] - mx) * n[0] + (w->cy[cr] - my) * n[1]);
    double h = p->kappa * (wl < wr ? wl : wr);
    o->h = h;
    o->n[0] = n[0];
    o->n[1] = n[1];
    o->tau_f = p->nu / (CS2 * h) + 0.5;
    o->tau_g = p->chi / (CS2 * h) + 0.5;
    /* step 4: nodes by Eq. 29 with the full offset, primitives in the frame */
    for (int a = -1; a <= 1; ++a)
        for (int b = -1; b <= 1; ++b) {
            double nxp = mx + (a * n[0] + b * t[0]) * h, nyp = my + (a * n[1] + b * t[1]) * h;
            double vL[4], vR[4];
            for (int q = 0; q < 4; ++q) {
                vL[q] = w->q[q][cl] + w->g[q][0][cl] * (nxp - w->cx[cl]) +
                        w->g[q][1][cl] * (nyp - w->cy[cl]);
                vR[q] = w->q[q][cr] + w->g[q][0][cr] * (nxp - w->cx[cr]) +
                        w->g[q][1][cr] * (nyp - w->cy[cr]);
            }
            double v[4];
            for (int q = 0; q < 4; ++q) v[q] = a < 0 ? vL[q] : (a > 0 ? vR[q] : 0.5 * (vL[q] + vR[q]));
            o->node[0][a + 1][b + 1] = v[0];
            o->node[1][a + 1][b + 1] = v[1] * n[0] + v[2] * n[1]; /* u_n */
            o->node[2][a + 1][b + 1] = v[1] * t[0] + v[2] * t[1]; /* u_t */
            o->node[3][a + 1][b + 1] = v[3];
        }
    /* step 5: products at the nodes and central differences, frame x = n, y = t */
    enum { RHO, MN, MT, E, XNN, XNT, XTT, QN, QT, NP };
    double P[NP][3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double r = o->node[0][a][b], un = o->node[1][a][b], ut = o->node[2][a][b],
                   T = o->node[3][a][b];
            P[RHO][a][b] = r;
            P[MN][a][b] = r * un;
            P[MT][a][b] = r * ut;
            P[E][a][b] = r * T;
            P[XNN][a][b] = r * un * un + r * CS2;
            P[XNT][a][b] = r * un * ut;
            P[XTT][a][b] = r * ut * ut + r * CS2;
            P[QN][a][b] = r * un * T;
            P[QT][a][b] = r * ut * T;
        }
    double D[NP][2], DD[NP][2][2];
    for (int k = 0; k < NP; ++k) {
        D[k][0] = (P[k][2][1] - P[k][0][1]) / (2.0 * h);
        D[k][1] = (P[k][1][2] - P[k][1][0]) / (2.0 * h);
        DD[k][0][0] = (P[k][2][1] - 2.0 * P[k][1][1] + P[k][0][1]) / (h * h);
        DD[k][1][1] = (P[k][1][2] - 2.0 * P[k][1][1] + P[k][1][0]) / (h * h);
        DD[k][0][1] = (P[k][2][2] - P[k][2][0] - P[k][0][2] + P[k][0][0]) / (4.0 * h * h);
        DD[k][1][0] = DD[k][0][1];
    }
    const int M[2] = {MN, MT};
    const int X[2][2] = {{XNN, XNT}, {XNT, XTT}};
    const int UT[2] = {QN, QT};
#define C0(k) (P[(k)][1][1])
    double rho_s = C0(RHO);
    for (int al = 0; al < 2; ++al) rho_s -= h * D[M[al]][al];
    for (int al = 0; al < 2; ++al)
        for (int be = 0; be < 2; ++be) rho_s += 0.5 * h * h * DD[X[al][be]][al][be];
    double m_s[2];
    for (int al = 0; al < 2; ++al) {
        double s = C0(M[al]);
        for (int be = 0; be < 2; ++be) s -= h * D[X[al][be]][be];
        double br = 0.0;
        for (int be = 0; be < 2; ++be) {
            br += DD[M[al]][be][be];
            br += DD[M[be]][al][be];
        }
        for (int ga = 0; ga < 2; ++ga) br += DD[M[ga]][al][ga];
        m_s[al] = s + 0.5 * CS2 * h * h * br;
    }
    double E_s = C0(E);
    for (int al = 0; al < 2; ++al) E_s -= h * D[UT[al]][al];
    for (int al = 0; al < 2; ++al) E_s += 0.5 * CS2 * h * h * DD[E][al][al];
    if (wall_side >= 0) { /* R8 in the frame */
        double uwt = p->bc_u[wall_side][0] * t[0] + p->bc_u[wall_side][1] * t[1];
        m_s[0] = 0.0;
        m_s[1] = rho_s * uwt;
        if (p->bc_kind[wall_side] == CB_DIRICHLET) E_s = rho_s * p->bc_T[wall_side];
    }
    o->pred[0] = rho_s;
    o->pred[1] = m_s[0];
    o->pred[2] = m_s[1];
    o->pred[3] = E_s;
    double us[2] = {m_s[0] / rho_s, m_s[1] / rho_s}, Ts = E_s / rho_s;
    /* step 6: braces of Eqs. 57-59 along n (frame axis 0) */
    double divm = D[MN][0] + D[MT][1];
    double Ff[2];
    for (int al = 0; al < 2; ++al) {
        double X0 = C0(X[al][0]);
        double Xs = rho_s * us[al] * us[0] + (al == 0 ? rho_s * CS2 : 0.0);
        double visc = D[M[al]][0] + D[M[0]][al] + (al == 0 ? divm : 0.0);
        Ff[al] = X0 - p->nu * visc - (o->tau_f - 1.5) * (Xs - X0);
    }
    double Q0 = C0(QN), Qs = rho_s * us[0] * Ts;
    o->flux[0] = m_s[0];
    o->flux[1] = Ff[0] * n[0] + Ff[1] * t[0]; /* back to x, y */
    o->flux[2] = Ff[0] * n[1] + Ff[1] * t[1];
    o->flux[3] = Q0 - p->chi * D[E][0] - (o->tau_g - 1.5) * (Qs - Q0);
#undef C0
}

/* i-face (i, j), i in [0, ni]: between cells (i-1, j) and (i, j). */
static void iface_at(const orcc_problem* p, const cwork* w, int i, int j, orcc_face_out* o)
{
    double ax, ay, bx, by, S[2];
    iface_edge(p, i, j, &ax, &ay, &bx, &by);
    face_vector(0, ax, ay, bx, by, S);
    double L = hypot(S[0], S[1]), n[2] = {S[0] / L, S[1] / L};
    int wall = -1;
    if (!iper(p)) {
        if (i == 0 && p->bc_kind[0] != CB_FARFIELD) wall = 0;
        if (i == p->ni && p->bc_kind[1] != CB_FARFIELD) wall = 1;
    }
    face_compute(p, w, CP(w, i - 1, j), CP(w, i, j), 0.5 * (ax + bx), 0.5 * (ay + by), n, wall, o);
    o->len = L;
}

/* j-face (i, j), j in [0, nj]: between cells (i, j-1) and (i, j). */
static void jface_at(const orcc_problem* p, const cwork* w, int i, int j, orcc_face_out* o)
{
    double ax, ay, bx, by, S[2];
    jface_edge(p, i, j, &ax, &ay, &bx, &by);
    face_vector(1, ax, ay, bx, by, S);
    double L = hypot(S[0], S[1]), n[2] = {S[0] / L, S[1] / L};
    int wall = -1;
    if (j == 0 && p->bc_kind[2] != CB_FARFIELD) wall = 2;
    if (j == p->nj && p->bc_kind[3] != CB_FARFIELD) wall = 3;
    face_compute(p, w, CP(w, i, j - 1), CP(w, i, j), 0.5 * (ax + bx), 0.5 * (ay + by), n, wall, o);
    o->len = L;
}

static void prepare(const orcc_problem* p, cwork* w)
{
    ghost_values(p, w);
    gradients(p, w);
    ghost_gradients(p, w);
}

static void all_faces(const orcc_problem* p, cwork* w)
{
    int ni = p->ni, nj = p->nj;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < nj; ++j) {
        orcc_face_out o;
        for (int i = 0; i <= ni; ++i) {
            iface_at(p, w, i, j, &o);
            for (int k = 0; k < 4; ++k) w->fi[k][(size_t)j * (ni + 1) + i] = o.flux[k] * o.len;
        }
    }
#pragma omp parallel for schedule(static)
    for (int j = 0; j <= nj; ++j) {
        orcc_face_out o;
        for (int i = 0; i < ni; ++i) {
            jface_at(p, w, i, j, &o);
            for (int k = 0; k < 4; ++k) w->fj[k][(size_t)j * ni + i] = o.flux[k] * o.len;
        }
    }
}

static void load(const orcc_problem* p, cwork* w, double* const st[4])
{
    for (int q = 0; q < 4; ++q)
        for (int j = 0; j < p->nj; ++j)
            for (int i = 0; i < p->ni; ++i) w->q[q][CP(w, i, j)] = st[q][(size_t)j * p->ni + i];
}

/* Steps 7-8: update with face lengths (fluxes above are already times the
 * length) and cell areas, Boussinesq source along gdir; residual of R12. */
static void update(const orcc_problem* p, cwork* w, double* const st[4], double res[2])
{
    int ni = p->ni, nj = p->nj;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : a0, a1, a2, a3)
    for (int j = 0; j < nj; ++j)
        for (int i = 0; i < ni; ++i) {
            size_t c = CP(w, i, j);
            double r = w->q[0][c], u = w->q[1][c], v = w->q[2][c], T = w->q[3][c];
            double Wc[4] = {r, r * u, r * v, r * T};
            double src = r * p->beta_g * (T - p->T_ref);
            double S[4] = {0.0, r * p->force[0] + src * p->gdir[0], r * p->force[1] + src * p->gdir[1],
                           0.0};
            double Wn[4];
            for (int k = 0; k < 4; ++k) {
                double sum = w->fi[k][(size_t)j * (ni + 1) + i + 1] - w->fi[k][(size_t)j * (ni + 1) + i] +
                             w->fj[k][(size_t)(j + 1) * ni + i] - w->fj[k][(size_t)j * ni + i];
                Wn[k] = Wc[k] - p->dt / w->area[c] * sum + p->dt * S[k];
            }
            double r1 = Wn[0], u1 = Wn[1] / r1, v1 = Wn[2] / r1, T1 = Wn[3] / r1;
            size_t o = (size_t)j * ni + i;
            st[0][o] = r1;
            st[1][o] = u1;
            st[2][o] = v1;
            st[3][o] = T1;
            double m0 = sqrt(u * u + v * v), m1 = sqrt(u1 * u1 + v1 * v1);
            a0 += (m1 - m0) * (m1 - m0);
            a1 += m1 * m1;
            a2 += (T1 - T) * (T1 - T);
            a3 += T1 * T1;
        }
    res[0] = a1 > 0.0 ? sqrt(a0) / sqrt(a1) : INFINITY;
    res[1] = a3 > 0.0 ? sqrt(a2) / sqrt(a3) : INFINITY;
    if (isnan(a0) || isnan(a1)) res[0] = NAN;
    if (isnan(a2) || isnan(a3)) res[1] = NAN;
}

int orcc_step(const orcc_problem* p, double* rho, double* u, double* v, double* T, long nsteps,
              double* res)
{
    double* st[4] = {rho, u, v, T};
    if (check(p) || !rho || !u || !v || !T || nsteps < 0) return -1;
    cwork w;
    if (calloc_work(&w, p->ni, p->nj)) return -2;
    if (geometry(p, &w)) {
        cfree(&w);
        return -1;
    }
    double r2[2] = {NAN, NAN};
    int rc = 0;
    for (long s = 0; s < nsteps; ++s) {
        load(p, &w, st);
        prepare(p, &w);
        all_faces(p, &w);
        update(p, &w, st, r2);
        if (isnan(r2[0]) || isnan(r2[1])) {
            rc = -4;
            break;
        }
    }
    if (res) {
        res[0] = r2[0];
        res[1] = r2[1];
    }
    cfree(&w);
    return rc;
}

int orcc_run_to_steady(const orcc_problem* p, double* rho, double* u, double* v, double* T,
                       double tol, long max_steps, long* steps, double* res)
{
    double* st[4] = {rho, u, v, T};
    if (check(p) || !rho || !u || !v || !T || max_steps < 0) return -1;
    cwork w;
    if (calloc_work(&w, p->ni, p->nj)) return -2;
    if (geometry(p, &w)) {
        cfree(&w);
        return -1;
    }
    double r2[2] = {INFINITY, INFINITY};
    long s = 0;
    int rc = -5;
    while (s < max_steps) {
        load(p, &w, st);
        prepare(p, &w);
        all_faces(p, &w);
        update(p, &w, st, r2);
        ++s;
        if (isnan(r2[0]) || isnan(r2[1])) {
            rc = -4;
            break;
        }
        if ((r2[0] > r2[1] ? r2[0] : r2[1]) < tol) {
            rc = 0;
            break;
        }
    }
    if (steps) *steps = s;
    if (res) {
        res[0] = r2[0];
        res[1] = r2[1];
    }
    cfree(&w);
    return rc;
}

/* Gradients (8 planes: d/dx, d/dy of rho, u, v, T) and geometry (centres
 * x, y and areas: 3 planes) of the interior cells. */
int orcc_gradients(const orcc_problem* p, double* rho, double* u, double* v, double* T,
                   double* grad, double* geom)
{
    double* st[4] = {rho, u, v, T};
    if (check(p) || !grad) return -1;
    cwork w;
    if (calloc_work(&w, p->ni, p->nj)) return -2;
    if (geometry(p, &w)) {
        cfree(&w);
        return -1;
    }
    load(p, &w, st);
    prepare(p, &w);
    size_t n = (size_t)p->ni * p->nj;
    for (int j = 0; j < p->nj; ++j)
        for (int i = 0; i < p->ni; ++i) {
            size_t c = CP(&w, i, j), o = (size_t)j * p->ni + i;
            for (int q = 0; q < 4; ++q) {
                grad[(2 * q) * n + o] = w.g[q][0][c];
                grad[(2 * q + 1) * n + o] = w.g[q][1][c];
            }
            if (geom) {
                geom[o] = w.cx[c];
                geom[n + o] = w.cy[c];
                geom[2 * n + o] = w.area[c];
            }
        }
    cfree(&w);
    return 0;
}

/* One face: kind 0 = i-face (i in [0, ni], j < nj), 1 = j-face. */
int orcc_face(const orcc_problem* p, double* rho, double* u, double* v, double* T, int kind, int i,
              int j, orcc_face_out* o)
{
    double* st[4] = {rho, u, v, T};
    if (check(p) || !o || kind < 0 || kind > 1) return -1;
    if (kind == 0 && (i < 0 || i > p->ni || j < 0 || j >= p->nj)) return -1;
    if (kind == 1 && (i < 0 || i >= p->ni || j < 0 || j > p->nj)) return -1;
    cwork w;
    if (calloc_work(&w, p->ni, p->nj)) return -2;
    if (geometry(p, &w)) {
        cfree(&w);
        return -1;
    }
    load(p, &w, st);
    prepare(p, &w);
    if (kind == 0)
        iface_at(p, &w, i, j, o);
    else
        jface_at(p, &w, i, j, o);
    cfree(&w);
    return 0;
}

/* Heat transfer through side s (2: j = 0, 3: j = nj): the energy flux of
 * step 6 times the face lengths, summed over the side's faces (along the
 * face vector, i.e. towards increasing j).  Divided by chi dT and the side's
 * length times a reference length lref, this is Eq. 73's mean Nusselt
 * number: Nu = -(lref / (chi dT perimeter)) sum (-chi dT/dn) dS. */
int orcc_heat(const orcc_problem* p, double* rho, double* u, double* v, double* T, int side,
              double* out, double* perimeter)
{
    double* st[4] = {rho, u, v, T};
    if (check(p) || !out || (side != 2 && side != 3)) return -1;
    cwork w;
    if (calloc_work(&w, p->ni, p->nj)) return -2;
    if (geometry(p, &w)) {
        cfree(&w);
        return -1;
    }
    load(p, &w, st);
    prepare(p, &w);
    int j = side == 3 ? p->nj : 0;
    double s = 0.0, per = 0.0;
    orcc_face_out o;
    for (int i = 0; i < p->ni; ++i) {
        jface_at(p, &w, i, j, &o);
        s += o.flux[3] * o.len;
        per += o.len;
    }
    *out = s;
    if (perimeter) *perimeter = per;
    cfree(&w);
    return 0;
}
