/*
 * FP64 CPU oracle of the lattice Boltzmann method with adaptive relaxation
 * parameter and Lax-Friedrichs-type equilibrium (Zhang, Lin, Zhao, Zhao,
 * arXiv 2609.18177).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is loaded by the tests, by the
 * package smoke check and by the CPU-baseline leg of the benchmark.  The
 * product path never links, loads or calls it, and it shares no code with the
 * CUDA path.
 *
 * Everything is plain FP64 loops over nodes in the order the paper states the
 * scheme (Section 2):
 *   1. U = sum_k f_k                                         Eq. (2.3)
 *   2. abar_j = max_x max_r |lambda_r(dF_j/dU)|              Eq. (2.17)/(2.19)
 *   3. dt = CFL dx / sum_j abar_j, lambda = dx/dt            Eq. (2.21)
 *   4. characteristic differences, theta, nu                 Eq. (2.9)/(2.13), (2.10)/(2.14)
 *   5. nu~ over the 3^d box, omega = 1 + 1/(1+nu~)           Eq. (2.11)/(2.15), (2.12)/(2.16)
 *   6. post_k = f_k - omega (f_k - f_k^eq) + dt/2 s_k        Eq. (2.2), (2.18)/(2.20), (2.6)
 *   7. pull streaming F_k(x) = post_k(x - e_k)               Section 2.1, implementation form
 *   8. U^{n+1} = sum_k F_k + dt/2 S(U^{n+1});
 *      f_k = F_k + dt/2 a_k S(U^{n+1})                       Eq. (2.8)
 *
 * Readings of points the paper leaves open (each is listed in the design notes):
 *   - abar, dt and lambda are recomputed every step from U^n; all coefficients
 *     of step n (including the second half-source) use alpha^n, lambda^n, dt^n.
 *   - the last step is clipped so that t hits T exactly (dt_cap argument).
 *   - nodes sit at cell centres x_i = x0 + (i + 1/2) dx.
 *   - boundaries: the distributions f^n are extended by 3 ghost layers whose
 *     values are read from the wrapped (periodic) or clamped (outflow) interior
 *     index; U, nu, omega and post at a ghost node are then computed from those
 *     ghost distributions exactly as at an interior node.  A ghost node takes
 *     the position of the interior node it copies (relevant only to the bed).
 *   - reflective wall (Example 5.13, y = +-15): a ghost node holds the
 *     distributions of its mirror node with the velocities normal to the wall
 *     exchanged (e_j <-> -e_j) and the normal momentum negated in every
 *     distribution, so its U is the mirror state with the normal velocity
 *     reversed; it sits at its own (mirrored) position.
 *   - fixed inflow (Example 5.13, x = 40): a ghost node holds f^eq(U_in)
 *     with the step's alpha and lambda.
 *   - sponge (Example 5.13, 0 <= x <= 6; the paper gives no formula): omega
 *     is blended toward 1, omega' = 1 + (omega - 1)(1 - sigma(x)), sigma =
 *     (1 + cos(pi (x - x0)/L))/2 on [x0, x0 + L], 1 to the left, 0 to the right.
 *   - L = R^{-1} with right eigenvectors normalised as in Toro's textbook
 *     (first component 1 for acoustic/entropy waves, unit tangential velocity
 *     for shear waves, unit Y for the species wave); this oracle inverts R
 *     numerically.
 *   - shallow water: h < h_dry is a dry node with u = v = 0; c in L is
 *     max(c, sqrt(g h_dry)).
 *   - bed-slope source S = (0, -g h db/dx, -g h db/dy) with the analytic
 *     gradient of a Gaussian bump; the paper's shallow-water tests have S = 0.
 *   - Arrhenius: (2.8) is a scalar equation in rho*Y; its largest root in the
 *     bracket between 0 and the streamed value is taken, found by a scan from
 *     the top followed by bisection.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_ADVECTION 0
#define ORC_EULER 1
#define ORC_SWE 2
#define ORC_REACTIVE 3
#define ORC_LINEAR 4

#define ORC_BC_PERIODIC 0
#define ORC_BC_OUTFLOW 1
#define ORC_BC_REFLECT 2
#define ORC_BC_INFLOW 3

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_MEM (-2)
/* positive return bits: non-physical states met during the step */
#define ORC_FLAG_NONPHYSICAL 1
#define ORC_FLAG_NOROOT 2

#define GHOST 3
#define MAXM 8

typedef struct {
    int system;
    int dim;
    int nx, ny;
    double x0, x1, y0, y1;
    int bc[4]; /* xlo, xhi, ylo, yhi */
    int nz;           /* 3D (D3Q7): nodes in z */
    double z0, z1;
    int bc_z[2];      /* zlo, zhi */
    double cfl, eps;
    double adv[3];
    double gamma, g;
    double bed_amp, bed_w2, bed_xc, bed_yc;
    double K, Ti, q;
    int m_linear;
    const double *A; /* LINEAR: dim matrices m x m, row-major */
    int omega_mode;  /* 0 adaptive (paper), 1 fixed */
    double omega_fixed;
    double h_dry;
    double sponge_width;  /* > 0: sponge layer of this width at x-lo */
    double u_in[MAXM];    /* conservative state held by inflow ghost nodes */
} orc_problem;

/* ------------------------------------------------------------------ */
/* problem geometry                                                     */
/* ------------------------------------------------------------------ */

int orc_nfields(const orc_problem *p) {
    switch (p->system) {
    case ORC_ADVECTION: return 1;
    case ORC_EULER: return p->dim + 2;
    case ORC_SWE: return p->dim + 1;
    case ORC_REACTIVE: return p->dim + 3;
    case ORC_LINEAR: return p->m_linear;
    }
    return -1;
}

static int nq(const orc_problem *p) { return 2 * p->dim + 1; }
static double mesh_dx(const orc_problem *p) { return (p->x1 - p->x0) / p->nx; }
static int ny_of(const orc_problem *p) { return p->dim >= 2 ? p->ny : 1; }
static int nz_of(const orc_problem *p) { return p->dim == 3 ? p->nz : 1; }
/* rows of the [Q][m][rows][nx] layout: y and z flattened (z outer) */
static int rows_of(const orc_problem *p) { return ny_of(p) * nz_of(p); }

static int check_problem(const orc_problem *p) {
    if (p->dim < 1 || p->dim > 3) return ORC_ERR_ARG;
    if (p->nx < 1 || (p->dim >= 2 && p->ny < 1) || (p->dim == 3 && p->nz < 1)) return ORC_ERR_ARG;
    if (p->dim == 3) {
        /* D3Q7: scalar advection, Euler and reactive Euler; periodic or outflow */
        if (p->system != ORC_ADVECTION && p->system != ORC_EULER && p->system != ORC_REACTIVE) return ORC_ERR_ARG;
        for (int b = 0; b < 4; b++)
            if (p->bc[b] != ORC_BC_PERIODIC && p->bc[b] != ORC_BC_OUTFLOW) return ORC_ERR_ARG;
        for (int b = 0; b < 2; b++)
            if (p->bc_z[b] != ORC_BC_PERIODIC && p->bc_z[b] != ORC_BC_OUTFLOW) return ORC_ERR_ARG;
        if ((p->bc_z[0] == ORC_BC_PERIODIC) != (p->bc_z[1] == ORC_BC_PERIODIC)) return ORC_ERR_ARG;
        double dx = mesh_dx(p), dz = (p->z1 - p->z0) / p->nz;
        if (fabs(dx - dz) > 1e-12 * dx) return ORC_ERR_ARG;
        if (p->sponge_width != 0.0) return ORC_ERR_ARG;
    }
    int m = orc_nfields(p);
    if (m < 1 || m > MAXM) return ORC_ERR_ARG;
    for (int b = 0; b < 2 * (p->dim < 2 ? p->dim : 2); b++)
        if (p->bc[b] < ORC_BC_PERIODIC || p->bc[b] > ORC_BC_INFLOW) return ORC_ERR_ARG;
    if ((p->bc[0] == ORC_BC_REFLECT || p->bc[1] == ORC_BC_REFLECT || p->bc[2] == ORC_BC_REFLECT ||
         p->bc[3] == ORC_BC_REFLECT) && (p->system == ORC_LINEAR || p->nx < GHOST || (p->dim == 2 && p->ny < GHOST)))
        return ORC_ERR_ARG;
    if (p->sponge_width < 0.0) return ORC_ERR_ARG;
    if ((p->bc[0] == ORC_BC_PERIODIC) != (p->bc[1] == ORC_BC_PERIODIC)) return ORC_ERR_ARG;
    if (p->dim >= 2 && (p->bc[2] == ORC_BC_PERIODIC) != (p->bc[3] == ORC_BC_PERIODIC)) return ORC_ERR_ARG;
    if (p->dim >= 2) {
        double dx = mesh_dx(p), dy = (p->y1 - p->y0) / p->ny;
        if (fabs(dx - dy) > 1e-12 * dx) return ORC_ERR_ARG; /* uniform mesh, Section 2.2.2 */
    }
    if (p->system == ORC_LINEAR && p->A == NULL) return ORC_ERR_ARG;
    return ORC_OK;
}

/* index of an extended (ghost) coordinate mapped back into the domain */
static int map_index(int e, int n, int bc_lo, int bc_hi) {
    if (e < 0) {
        if (bc_lo == ORC_BC_PERIODIC) return ((e % n) + n) % n;
        if (bc_lo == ORC_BC_REFLECT) return -1 - e;
        return 0;
    }
    if (e >= n) {
        if (bc_hi == ORC_BC_PERIODIC) return e % n;
        if (bc_hi == ORC_BC_REFLECT) return 2 * n - 1 - e;
        return n - 1;
    }
    return e;
}

/* the boundary type a ghost coordinate e lies across (-1: interior) */
static int ghost_side(int e, int n, int bc_lo, int bc_hi) {
    if (e < 0) return bc_lo;
    if (e >= n) return bc_hi;
    return -1;
}

/* index of the momentum component along direction dir, -1 if none */
static int momentum_index(const orc_problem *p, int dir) {
    if (p->system == ORC_EULER || p->system == ORC_SWE || p->system == ORC_REACTIVE) return 1 + dir;
    return -1;
}

/* sponge weight sigma(x): 1 left of x0, 0 beyond x0 + width */
static double sponge_sigma(const orc_problem *p, double x) {
    if (!(p->sponge_width > 0.0)) return 0.0;
    double r = (x - p->x0) / p->sponge_width;
    if (r <= 0.0) return 1.0;
    if (r >= 1.0) return 0.0;
    return 0.5 * (1.0 + cos(3.14159265358979323846 * r));
}

static double node_x(const orc_problem *p, int i) { return p->x0 + (i + 0.5) * mesh_dx(p); }
static double node_y(const orc_problem *p, int j) {
    if (p->dim < 2) return 0.0;
    return p->y0 + (j + 0.5) * ((p->y1 - p->y0) / p->ny);
}

/* ------------------------------------------------------------------ */
/* physical systems: primitive variables, flux, wave speeds, source     */
/* ------------------------------------------------------------------ */

typedef struct {
    double rho, u, v, w, p, Y, c, H; /* Euler-type */
    double h;                     /* shallow water */
    int dry;
} prim_t;

static prim_t primitives(const orc_problem *p, const double *U) {
    prim_t w;
    memset(&w, 0, sizeof w);
    if (p->system == ORC_EULER || p->system == ORC_REACTIVE) {
        int d = p->dim;
        w.rho = U[0];
        w.u = U[1] / w.rho;
        w.v = d >= 2 ? U[2] / w.rho : 0.0;
        w.w = d == 3 ? U[3] / w.rho : 0.0;
        double E = U[d + 1];
        double kin = 0.5 * w.rho * (w.u * w.u + w.v * w.v + w.w * w.w);
        double chem = 0.0;
        if (p->system == ORC_REACTIVE) {
            w.Y = U[d + 2] / w.rho;
            chem = p->q * U[d + 2];
        }
        w.p = (p->gamma - 1.0) * (E - kin - chem);
        w.c = sqrt(p->gamma * w.p / w.rho);
        w.H = (E + w.p) / w.rho;
    } else if (p->system == ORC_SWE) {
        w.h = U[0];
        w.dry = w.h < p->h_dry;
        if (!w.dry) {
            w.u = U[1] / w.h;
            w.v = p->dim == 2 ? U[2] / w.h : 0.0;
        }
        w.c = sqrt(p->g * (w.h > 0.0 ? w.h : 0.0));
    }
    return w;
}

/* physical flux F_dir(U); Section 5 (shallow water, reactive Euler) and the
 * textbook Euler flux (the reactive flux with q = 0 and no species). */
void orc_flux(const orc_problem *p, int dir, const double *U, double *F) {
    int m = orc_nfields(p), d = p->dim;
    if (p->system == ORC_ADVECTION) {
        F[0] = p->adv[dir] * U[0];
        return;
    }
    if (p->system == ORC_LINEAR) {
        const double *A = p->A + (size_t)dir * m * m;
        for (int r = 0; r < m; r++) {
            double s = 0.0;
            for (int c = 0; c < m; c++) s += A[r * m + c] * U[c];
            F[r] = s;
        }
        return;
    }
    prim_t w = primitives(p, U);
    if (p->system == ORC_SWE) {
        double vn = dir == 0 ? w.u : w.v;
        double pres = 0.5 * p->g * w.h * w.h;
        F[0] = w.h * vn;
        F[1] = w.h * w.u * vn + (dir == 0 ? pres : 0.0);
        if (d == 2) F[2] = w.h * w.v * vn + (dir == 1 ? pres : 0.0);
        return;
    }
    /* Euler / reactive Euler */
    double vn = dir == 0 ? w.u : (dir == 1 ? w.v : w.w);
    F[0] = w.rho * vn;
    F[1] = w.rho * w.u * vn + (dir == 0 ? w.p : 0.0);
    if (d >= 2) F[2] = w.rho * w.v * vn + (dir == 1 ? w.p : 0.0);
    if (d == 3) F[3] = w.rho * w.w * vn + (dir == 2 ? w.p : 0.0);
    F[d + 1] = vn * (U[d + 1] + w.p);
    if (p->system == ORC_REACTIVE) F[d + 2] = U[d + 2] * vn;
}

/* symmetric Jacobi eigen-solver for the constant matrices of LINEAR systems */
static void jacobi_eig(int m, const double *Ain, double *lam, double *V) {
    double A[MAXM * MAXM];
    memcpy(A, Ain, sizeof(double) * m * m);
    for (int i = 0; i < m; i++)
        for (int j = 0; j < m; j++) V[i * m + j] = (i == j);
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0.0;
        for (int i = 0; i < m; i++)
            for (int j = i + 1; j < m; j++) off += A[i * m + j] * A[i * m + j];
        if (off < 1e-300) break;
        for (int pp = 0; pp < m; pp++)
            for (int qq = pp + 1; qq < m; qq++) {
                double apq = A[pp * m + qq];
                if (apq == 0.0) continue;
                double theta = (A[qq * m + qq] - A[pp * m + pp]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < m; k++) { /* A <- A J */
                    double akp = A[k * m + pp], akq = A[k * m + qq];
                    A[k * m + pp] = c * akp - s * akq;
                    A[k * m + qq] = s * akp + c * akq;
                }
                for (int k = 0; k < m; k++) { /* A <- J^T A */
                    double apk = A[pp * m + k], aqk = A[qq * m + k];
                    A[pp * m + k] = c * apk - s * aqk;
                    A[qq * m + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < m; k++) {
                    double vkp = V[k * m + pp], vkq = V[k * m + qq];
                    V[k * m + pp] = c * vkp - s * vkq;
                    V[k * m + qq] = s * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < m; i++) lam[i] = A[i * m + i];
}

/* eigenvalues lambda_r(dF_dir/dU), closed forms of the textbook systems */
void orc_eigvals(const orc_problem *p, int dir, const double *U, double *lam) {
    int m = orc_nfields(p);
    if (p->system == ORC_ADVECTION) {
        lam[0] = p->adv[dir];
        return;
    }
    if (p->system == ORC_LINEAR) {
        double V[MAXM * MAXM];
        jacobi_eig(m, p->A + (size_t)dir * m * m, lam, V);
        return;
    }
    prim_t w = primitives(p, U);
    double vn = dir == 0 ? w.u : (dir == 1 ? w.v : w.w);
    lam[0] = vn - w.c;
    for (int r = 1; r < m - 1; r++) lam[r] = vn;
    lam[m - 1] = vn + w.c;
}

/* max_r |lambda_r| at one node (the inner max of Eq. (2.17)/(2.19)) */
double orc_max_speed(const orc_problem *p, int dir, const double *U) {
    int m = orc_nfields(p);
    double lam[MAXM], s = 0.0;
    orc_eigvals(p, dir, U, lam);
    for (int r = 0; r < m; r++) {
        double a = fabs(lam[r]);
        if (a > s || a != a) s = a; /* a NaN speed propagates */
    }
    return s;
}

/* right eigenvectors R (columns), normalisation described in the header */
void orc_right_eigvecs(const orc_problem *p, int dir, const double *U, double *R) {
    int m = orc_nfields(p), d = p->dim;
    memset(R, 0, sizeof(double) * m * m);
#define RS(row, col, val) R[(row) * m + (col)] = (val)
    if (p->system == ORC_ADVECTION) {
        R[0] = 1.0;
        return;
    }
    if (p->system == ORC_LINEAR) {
        double lam[MAXM];
        jacobi_eig(m, p->A + (size_t)dir * m * m, lam, R);
        return;
    }
    prim_t w = primitives(p, U);
    if (p->system == ORC_SWE) {
        double c = w.c, cmin = sqrt(p->g * p->h_dry);
        if (c < cmin) c = cmin;
        if (d == 1) {
            RS(0, 0, 1.0); RS(1, 0, w.u - c);
            RS(0, 1, 1.0); RS(1, 1, w.u + c);
        } else if (dir == 0) {
            RS(0, 0, 1.0); RS(1, 0, w.u - c); RS(2, 0, w.v);
            RS(2, 1, 1.0);
            RS(0, 2, 1.0); RS(1, 2, w.u + c); RS(2, 2, w.v);
        } else {
            RS(0, 0, 1.0); RS(1, 0, w.u); RS(2, 0, w.v - c);
            RS(1, 1, 1.0);
            RS(0, 2, 1.0); RS(1, 2, w.u); RS(2, 2, w.v + c);
        }
        return;
    }
    /* Euler / reactive: columns = (u-c), entropy, [shear], [species], (u+c) */
    double c = w.c, H = w.H, q2 = 0.5 * (w.u * w.u + w.v * w.v + w.w * w.w);
    double vel[3] = {w.u, w.v, w.w};
    double vn = vel[dir];
    int iE = d + 1, iY = d + 2, last = m - 1;
    int reactive = p->system == ORC_REACTIVE;
    double qY = reactive ? p->q * w.Y : 0.0;
    /* acoustic waves */
    for (int s = 0; s < 2; s++) {
        int col = s == 0 ? 0 : last;
        double sg = s == 0 ? -1.0 : 1.0;
        RS(0, col, 1.0);
        for (int t = 0; t < d; t++) RS(1 + t, col, vel[t] + (dir == t ? sg * c : 0.0));
        RS(iE, col, H + sg * vn * c);
        if (reactive) RS(iY, col, w.Y);
    }
    /* entropy wave */
    RS(0, 1, 1.0);
    for (int t = 0; t < d; t++) RS(1 + t, 1, vel[t]);
    RS(iE, 1, q2 + qY);
    if (reactive) RS(iY, 1, w.Y);
    int col = 2;
    for (int t = 0; t < d; t++) { /* shear waves: unit tangential velocity */
        if (t == dir) continue;
        RS(1 + t, col, 1.0);
        RS(iE, col, vel[t]);
        col++;
    }
    if (reactive) { /* species wave */
        RS(iE, col, p->q);
        RS(iY, col, 1.0);
    }
#undef RS
}

/* Gauss-Jordan inverse with partial pivoting; returns 0 on success */
static int invert(int m, const double *Ain, double *Inv) {
    double A[MAXM * MAXM];
    memcpy(A, Ain, sizeof(double) * m * m);
    for (int i = 0; i < m; i++)
        for (int j = 0; j < m; j++) Inv[i * m + j] = (i == j);
    for (int col = 0; col < m; col++) {
        int piv = col;
        for (int r = col + 1; r < m; r++)
            if (fabs(A[r * m + col]) > fabs(A[piv * m + col])) piv = r;
        if (A[piv * m + col] == 0.0) return -1;
        if (piv != col)
            for (int j = 0; j < m; j++) {
                double t = A[col * m + j]; A[col * m + j] = A[piv * m + j]; A[piv * m + j] = t;
                t = Inv[col * m + j]; Inv[col * m + j] = Inv[piv * m + j]; Inv[piv * m + j] = t;
            }
        double dgn = A[col * m + col];
        for (int j = 0; j < m; j++) { A[col * m + j] /= dgn; Inv[col * m + j] /= dgn; }
        for (int r = 0; r < m; r++) {
            if (r == col) continue;
            double fct = A[r * m + col];
            if (fct == 0.0) continue;
            for (int j = 0; j < m; j++) {
                A[r * m + j] -= fct * A[col * m + j];
                Inv[r * m + j] -= fct * Inv[col * m + j];
            }
        }
    }
    return 0;
}

/* left eigenvectors L = R^{-1} (Section 2.2) */
int orc_left_eigvecs(const orc_problem *p, int dir, const double *U, double *L) {
    int m = orc_nfields(p);
    double R[MAXM * MAXM];
    orc_right_eigvecs(p, dir, U, R);
    return invert(m, R, L);
}

/* Bed profile b(x, y) = amp * exp(-((x-xc)^2 + (y-yc)^2) / w2) and its gradient */
static void bed_gradient(const orc_problem *p, double x, double y, double *bx, double *by) {
    double dx = x - p->bed_xc, dy = p->dim == 2 ? y - p->bed_yc : 0.0;
    double b = p->bed_amp * exp(-(dx * dx + dy * dy) / p->bed_w2);
    *bx = -2.0 * dx / p->bed_w2 * b;
    *by = -2.0 * dy / p->bed_w2 * b;
}

static double arrhenius_rate(const orc_problem *p, double rho, double momsq, double E, double z) {
    /* R = K rho Y exp(-Ti / T), T = p / rho (Section 5.4) */
    double pres = (p->gamma - 1.0) * (E - 0.5 * momsq / rho - p->q * z);
    double T = pres / rho;
    return p->K * z * exp(-p->Ti / T);
}

/* source term S(U) at position (x, y) */
void orc_source(const orc_problem *p, const double *U, double x, double y, double *S) {
    int m = orc_nfields(p), d = p->dim;
    for (int c = 0; c < m; c++) S[c] = 0.0;
    if (p->system == ORC_SWE && p->bed_amp != 0.0) {
        double bx, by;
        bed_gradient(p, x, y, &bx, &by);
        S[1] = -p->g * U[0] * bx;
        if (d == 2) S[2] = -p->g * U[0] * by;
    } else if (p->system == ORC_REACTIVE && p->K != 0.0) {
        double momsq = 0.0;
        for (int t = 0; t < d; t++) momsq += U[1 + t] * U[1 + t];
        S[d + 2] = -arrhenius_rate(p, U[0], momsq, U[d + 1], U[d + 2]);
    }
}

/* Lax-Friedrichs-type equilibrium, Eq. (2.18)/(2.20), k = 0..2d */
void orc_equilibrium(const orc_problem *p, const double *U, const double *alpha, double lam,
                     double *feq) {
    int m = orc_nfields(p), d = p->dim;
    double F[MAXM], asum = 0.0;
    for (int j = 0; j < d; j++) asum += alpha[j];
    for (int c = 0; c < m; c++) feq[c] = (1.0 - asum / lam) * U[c];
    for (int j = 0; j < d; j++) {
        orc_flux(p, j, U, F);
        for (int c = 0; c < m; c++) {
            feq[(1 + j) * m + c] = (alpha[j] * U[c] + F[c]) / (2.0 * lam);
            feq[(1 + j + d) * m + c] = (alpha[j] * U[c] - F[c]) / (2.0 * lam);
        }
    }
}

/* weights a_k of Eq. (2.5) for the LF-type equilibrium: a_0 = 1 - sum alpha/lambda,
 * a_j = a_{j+d} = alpha_j / (2 lambda) */
static void weights_a(int d, const double *alpha, double lam, double *a) {
    double asum = 0.0;
    for (int j = 0; j < d; j++) asum += alpha[j];
    a[0] = 1.0 - asum / lam;
    for (int j = 0; j < d; j++) {
        a[1 + j] = alpha[j] / (2.0 * lam);
        a[1 + j + d] = alpha[j] / (2.0 * lam);
    }
}

/* Solve Eq. (2.8) for U^{n+1} given Ubar = sum_k F_k; returns flags */
static int solve_implicit_moment(const orc_problem *p, const double *Ubar, double x, double y,
                                 double dt, double *Un) {
    int m = orc_nfields(p), d = p->dim;
    for (int c = 0; c < m; c++) Un[c] = Ubar[c];
    if (p->system == ORC_SWE && p->bed_amp != 0.0) {
        /* S has no mass component, so h^{n+1} = hbar and the momentum equations
         * are explicit in h^{n+1} */
        double bx, by;
        bed_gradient(p, x, y, &bx, &by);
        Un[1] = Ubar[1] + 0.5 * dt * (-p->g * Un[0] * bx);
        if (d == 2) Un[2] = Ubar[2] + 0.5 * dt * (-p->g * Un[0] * by);
        return 0;
    }
    if (p->system == ORC_REACTIVE && p->K != 0.0) {
        /* only rho*Y carries a source; rho, momentum and rho*E equal their
         * streamed values.  g(z) = z - zbar + dt/2 R(z) = 0. */
        double rho = Ubar[0], E = Ubar[d + 1], zbar = Ubar[d + 2];
        double momsq = 0.0;
        for (int t = 0; t < d; t++) momsq += Ubar[t + 1] * Ubar[t + 1];
        double lo = zbar < 0.0 ? zbar : 0.0, hi = zbar < 0.0 ? 0.0 : zbar;
        if (zbar == 0.0) { Un[d + 2] = 0.0; return 0; }
#define GFUN(z) ((z) - zbar + 0.5 * dt * arrhenius_rate(p, rho, momsq, E, (z)))
        /* largest root: scan [lo, hi] downward from hi for the first sign change */
        const int nscan = 64;
        double b = hi, gb = GFUN(b), a = b, ga = gb;
        int found = 0;
        if (gb == 0.0) { Un[d + 2] = b; return 0; }
        for (int s = 1; s <= nscan; s++) {
            a = hi - (hi - lo) * s / nscan;
            ga = GFUN(a);
            if ((ga <= 0.0) != (gb <= 0.0) || ga == 0.0) { found = 1; break; }
            b = a; gb = ga;
        }
        if (!found || ga != ga || gb != gb) { Un[d + 2] = zbar; return ORC_FLAG_NOROOT; }
        /* bisection on [a, b] to full double precision */
        for (int it = 0; it < 200; it++) {
            double mid = 0.5 * (a + b);
            if (mid == a || mid == b) break;
            double gm = GFUN(mid);
            if (gm == 0.0) { a = b = mid; break; }
            if ((gm <= 0.0) == (ga <= 0.0)) { a = mid; ga = gm; } else { b = mid; gb = gm; }
        }
#undef GFUN
        Un[d + 2] = fabs(ga) <= fabs(gb) ? a : b;
        return 0;
    }
    return 0;
}

static int nonphysical(const orc_problem *p, const double *U) {
    int m = orc_nfields(p);
    for (int c = 0; c < m; c++)
        if (U[c] != U[c]) return 1;
    if (p->system == ORC_EULER || p->system == ORC_REACTIVE) {
        prim_t w = primitives(p, U);
        return !(w.rho > 0.0) || !(w.p > 0.0);
    }
    if (p->system == ORC_SWE) return U[0] < -1e-12;
    return 0;
}

/* ------------------------------------------------------------------ */
/* grid-level operations                                                */
/* ------------------------------------------------------------------ */

#define FIDX(k, c, j, i) ((((size_t)(k) * m + (c)) * ny + (j)) * nx + (i))
#define UIDX(c, j, i) (((size_t)(c) * ny + (j)) * nx + (i))

/* U = sum_k f_k, Eq. (2.3), summed in the order k = 0..Q-1 */
int orc_moments(const orc_problem *p, const double *f, double *U) {
    if (check_problem(p)) return ORC_ERR_ARG;
    int m = orc_nfields(p), Q = nq(p), nx = p->nx, ny = rows_of(p);
#pragma omp parallel for
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++)
            for (int c = 0; c < m; c++) {
                double s = 0.0;
                for (int k = 0; k < Q; k++) s += f[FIDX(k, c, j, i)];
                U[UIDX(c, j, i)] = s;
            }
    return ORC_OK;
}

/* abar_j = max over nodes of max_r |lambda_r(dF_j/dU)|, Eq. (2.17)/(2.19) */
int orc_alpha_bar_U(const orc_problem *p, const double *U, double *abar) {
    if (check_problem(p)) return ORC_ERR_ARG;
    int m = orc_nfields(p), nx = p->nx, ny = rows_of(p), d = p->dim;
    for (int j = 0; j < d; j++) abar[j] = 0.0;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            double Ui[MAXM];
            for (int c = 0; c < m; c++) Ui[c] = U[UIDX(c, j, i)];
            for (int dir = 0; dir < d; dir++) {
                double s = orc_max_speed(p, dir, Ui);
                if (s > abar[dir] || s != s) abar[dir] = s;
            }
        }
    return ORC_OK;
}

/* time step of Eq. (2.21), clipped to dt_cap (dt_cap <= 0 means no cap) */
static double time_step(const orc_problem *p, const double *abar, double dt_cap) {
    double asum = 0.0;
    for (int j = 0; j < p->dim; j++) asum += abar[j];
    double dt = p->cfl * mesh_dx(p) / asum;
    if (dt_cap > 0.0 && dt > dt_cap) dt = dt_cap;
    return dt;
}

/* f := f^eq(U) with alpha^0 and lambda^0 taken from U (uncapped dt) */
int orc_init(const orc_problem *p, const double *U, double *f, double *info) {
    if (check_problem(p)) return ORC_ERR_ARG;
    int m = orc_nfields(p), Q = nq(p), nx = p->nx, ny = rows_of(p), d = p->dim;
    double abar[3] = {0, 0, 0}, alpha[3];
    orc_alpha_bar_U(p, U, abar);
    double dt = time_step(p, abar, 0.0), lam = mesh_dx(p) / dt;
    for (int j = 0; j < d; j++) alpha[j] = abar[j] + p->eps;
#pragma omp parallel for
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            double Ui[MAXM], feq[7 * MAXM];
            for (int c = 0; c < m; c++) Ui[c] = U[UIDX(c, j, i)];
            orc_equilibrium(p, Ui, alpha, lam, feq);
            for (int k = 0; k < Q; k++)
                for (int c = 0; c < m; c++) f[FIDX(k, c, j, i)] = feq[k * m + c];
        }
    if (info) {
        info[0] = abar[0];
        info[1] = d >= 2 ? abar[1] : 0.0;
        info[2] = dt;
        info[3] = lam;
        if (d == 3) info[4] = abar[2];
    }
    return ORC_OK;
}

/* theta summed over the m characteristic fields for one direction, Eq. (2.9)/(2.13) */
static double theta_sum(int m, const double *L, const double *Um, const double *U0,
                        const double *Up, double dx) {
    double dm[MAXM], dp[MAXM];
    for (int c = 0; c < m; c++) {
        dm[c] = U0[c] - Um[c];
        dp[c] = Up[c] - U0[c];
    }
    double nu = 0.0;
    for (int r = 0; r < m; r++) {
        double wm = 0.0, wp = 0.0;
        for (int c = 0; c < m; c++) {
            wm += L[r * m + c] * dm[c];
            wp += L[r * m + c] * dp[c];
        }
        double am = fabs(wm), ap = fabs(wp);
        nu += fabs(wp - wm) / (am + ap + dx) + am + ap;
    }
    return nu;
}

/*
 * One time step f -> fn.  dt_cap > 0 clips the step; abar_in != NULL replaces
 * the global maximum of step 2 (used to check single nodes of a large grid).
 * info (optional, 4 doubles) receives abar_x, abar_y, dt, lambda; omega
 * (optional, nx*ny) receives the relaxation parameter of every node.
 * Returns 0, a positive flag mask, or a negative error.
 */
int orc_step(const orc_problem *p, const double *f, double *fn, double dt_cap, const double *abar_in,
             double *info, double *omega_out) {
    if (check_problem(p)) return ORC_ERR_ARG;
    const int m = orc_nfields(p), Q = nq(p), d = p->dim, nx = p->nx, ny = ny_of(p), nz = nz_of(p);
    const int G = GHOST;
    /* ghost-extended grid: G layers in every active direction */
    const int ex = nx + 2 * G, ey = d >= 2 ? ny + 2 * G : 1, ez = d == 3 ? nz + 2 * G : 1;
    const int gy = d >= 2 ? G : 0, gz = d == 3 ? G : 0;
    const double dx = mesh_dx(p);
    const size_t next = (size_t)ex * ey * ez;
    const size_t stride[3] = {1, (size_t)ex, (size_t)ex * ey};
    const int lo[3] = {G, gy, gz}, n_[3] = {nx, ny, nz};
    const int bclo[3] = {p->bc[0], p->bc[2], p->bc_z[0]}, bchi[3] = {p->bc[1], p->bc[3], p->bc_z[1]};
    int flags = 0;

    /* ghost-extended copies: fe[k][c][e], Ue[c][e], nu[e], om[e], post[k][c][e] */
    double *fe = malloc(sizeof(double) * Q * m * next);
    double *Ue = malloc(sizeof(double) * m * next);
    double *nu = malloc(sizeof(double) * next);
    double *om = malloc(sizeof(double) * next);
    double *post = malloc(sizeof(double) * Q * m * next);
    int *srci = malloc(sizeof(int) * ex), *srcj = malloc(sizeof(int) * ey), *srck = malloc(sizeof(int) * ez);
    double *posx = malloc(sizeof(double) * ex), *posy = malloc(sizeof(double) * ey);
    if (!fe || !Ue || !nu || !om || !post || !srci || !srcj || !srck || !posx || !posy) {
        free(fe); free(Ue); free(nu); free(om); free(post); free(srci); free(srcj); free(srck);
        free(posx); free(posy);
        return ORC_ERR_MEM;
    }
#define EI(kk, j, i) (((size_t)(kk) * ey + (j)) * ex + (i))
#define EF(k, c, e) (((size_t)(k) * m + (c)) * next + (e))
#define EU(c, e) ((size_t)(c) * next + (e))
#define FI(k, c, kk, j, i) (((((size_t)(k) * m + (c)) * nz + (kk)) * ny + (j)) * nx + (i))
    for (int ei = 0; ei < ex; ei++) srci[ei] = map_index(ei - G, nx, bclo[0], bchi[0]);
    for (int ej = 0; ej < ey; ej++) srcj[ej] = d >= 2 ? map_index(ej - gy, ny, bclo[1], bchi[1]) : 0;
    for (int ek = 0; ek < ez; ek++) srck[ek] = d == 3 ? map_index(ek - gz, nz, bclo[2], bchi[2]) : 0;
    /* node positions (bed source): a periodic or outflow ghost sits where the
     * node it copies sits, a reflecting ghost at its own position */
    for (int ei = 0; ei < ex; ei++)
        posx[ei] = ghost_side(ei - G, nx, bclo[0], bchi[0]) == ORC_BC_REFLECT ? node_x(p, ei - G) : node_x(p, srci[ei]);
    for (int ej = 0; ej < ey; ej++)
        posy[ej] = d >= 2 && ghost_side(ej - gy, ny, bclo[1], bchi[1]) == ORC_BC_REFLECT ? node_y(p, ej - gy)
                                                                                          : node_y(p, srcj[ej]);

    /* 1. ghost-extended distributions and moments U = sum_k f_k; across a
     * reflecting boundary the mirror node's distributions with the normal
     * velocities exchanged and the normal momentum negated */
#pragma omp parallel for collapse(2)
    for (int ek = 0; ek < ez; ek++)
        for (int ej = 0; ej < ey; ej++)
            for (int ei = 0; ei < ex; ei++) {
                const size_t e = EI(ek, ej, ei);
                const int i = srci[ei], j = srcj[ej], kk = srck[ek];
                const int ec[3] = {ei, ej, ek};
                int refl[3] = {0, 0, 0};
                for (int dir = 0; dir < d; dir++)
                    refl[dir] = ghost_side(ec[dir] - lo[dir], n_[dir], bclo[dir], bchi[dir]) == ORC_BC_REFLECT;
                for (int c = 0; c < m; c++) {
                    double sum = 0.0;
                    for (int k = 0; k < Q; k++) {
                        int ks = k; /* the velocity read from the mirror node */
                        double sign = 1.0;
                        for (int dir = 0; dir < d; dir++) {
                            if (!refl[dir]) continue;
                            if (ks == 1 + dir) ks = 1 + d + dir;
                            else if (ks == 1 + d + dir) ks = 1 + dir;
                            if (c == momentum_index(p, dir)) sign = -sign;
                        }
                        double v = sign * f[FI(ks, c, kk, j, i)];
                        fe[EF(k, c, e)] = v;
                        sum += v;
                    }
                    Ue[EU(c, e)] = sum;
                }
            }

    /* 2. global speed bound over the interior nodes */
    double abar[3] = {0.0, 0.0, 0.0}, alpha[3] = {0.0, 0.0, 0.0};
    if (abar_in) {
        for (int j = 0; j < d; j++) abar[j] = abar_in[j];
    } else {
        for (int ek = gz; ek < gz + nz; ek++)
            for (int ej = gy; ej < gy + ny; ej++)
                for (int ei = G; ei < G + nx; ei++) {
                    double Ui[MAXM];
                    for (int c = 0; c < m; c++) Ui[c] = Ue[EU(c, EI(ek, ej, ei))];
                    for (int dir = 0; dir < d; dir++) {
                        double sp = orc_max_speed(p, dir, Ui);
                        if (sp > abar[dir] || sp != sp) abar[dir] = sp;
                    }
                }
    }
    /* 3. time step, lattice speed, alpha_j = abar_j + eps */
    double dt = time_step(p, abar, dt_cap);
    double lam = dx / dt;
    for (int j = 0; j < d; j++) alpha[j] = abar[j] + p->eps;
    double a[7];
    weights_a(d, alpha, lam, a);

    /* 3b. ghost nodes across an inflow boundary: f^eq(U_in) with this step's
     * alpha and lambda */
    if (d <= 2) {
        double feq_in[7 * MAXM];
        orc_equilibrium(p, p->u_in, alpha, lam, feq_in);
        for (int ej = 0; ej < ey; ej++)
            for (int ei = 0; ei < ex; ei++) {
                int in = ghost_side(ei - G, nx, bclo[0], bchi[0]) == ORC_BC_INFLOW ||
                         (d == 2 && ghost_side(ej - gy, ny, bclo[1], bchi[1]) == ORC_BC_INFLOW);
                if (!in) continue;
                const size_t e = EI(0, ej, ei);
                for (int c = 0; c < m; c++) {
                    for (int k = 0; k < Q; k++) fe[EF(k, c, e)] = feq_in[k * m + c];
                    double sum = 0.0;
                    for (int k = 0; k < Q; k++) sum += feq_in[k * m + c];
                    Ue[EU(c, e)] = sum;
                }
            }
    }

    /* 4. smoothness indicator nu on nodes one layer inside the extension */
    for (size_t e = 0; e < next; e++) nu[e] = 0.0;
    const int in1[3][2] = {{1, ex - 1}, {d >= 2 ? 1 : 0, d >= 2 ? ey - 1 : 1}, {d == 3 ? 1 : 0, d == 3 ? ez - 1 : 1}};
#pragma omp parallel for collapse(2)
    for (int ek = in1[2][0]; ek < in1[2][1]; ek++)
        for (int ej = in1[1][0]; ej < in1[1][1]; ej++)
            for (int ei = in1[0][0]; ei < in1[0][1]; ei++) {
                const size_t e = EI(ek, ej, ei);
                double U0[MAXM], Um[MAXM], Up[MAXM], L[MAXM * MAXM];
                for (int c = 0; c < m; c++) U0[c] = Ue[EU(c, e)];
                double sum = 0.0;
                for (int dir = 0; dir < d; dir++) {
                    for (int c = 0; c < m; c++) {
                        Um[c] = Ue[EU(c, e - stride[dir])];
                        Up[c] = Ue[EU(c, e + stride[dir])];
                    }
                    orc_left_eigvecs(p, dir, U0, L);
                    sum += theta_sum(m, L, Um, U0, Up, dx);
                }
                nu[e] = sum;
            }

    /* 5. smoothed indicator over the 3^d box and the relaxation parameter,
     * on nodes two layers inside the extension */
    const int in2[3][2] = {{2, ex - 2}, {d >= 2 ? 2 : 0, d >= 2 ? ey - 2 : 1}, {d == 3 ? 2 : 0, d == 3 ? ez - 2 : 1}};
    const int bj0 = d >= 2 ? -1 : 0, bk0 = d == 3 ? -1 : 0;
#pragma omp parallel for collapse(2)
    for (int ek = in2[2][0]; ek < in2[2][1]; ek++)
        for (int ej = in2[1][0]; ej < in2[1][1]; ej++)
            for (int ei = in2[0][0]; ei < in2[0][1]; ei++) {
                double w;
                if (p->omega_mode == 1) {
                    w = p->omega_fixed;
                } else {
                    double nt = 0.0;
                    for (int bk = bk0; bk <= -bk0; bk++)
                        for (int bj = bj0; bj <= -bj0; bj++)
                            for (int bi = -1; bi <= 1; bi++) nt += nu[EI(ek + bk, ej + bj, ei + bi)];
                    w = 1.0 + 1.0 / (1.0 + nt);
                }
                if (p->sponge_width > 0.0) w = 1.0 + (w - 1.0) * (1.0 - sponge_sigma(p, node_x(p, ei - G)));
                om[EI(ek, ej, ei)] = w;
            }

    /* 6. collision with the first half of the source on the same nodes */
#pragma omp parallel for collapse(2)
    for (int ek = in2[2][0]; ek < in2[2][1]; ek++)
        for (int ej = in2[1][0]; ej < in2[1][1]; ej++)
            for (int ei = in2[0][0]; ei < in2[0][1]; ei++) {
                const size_t e = EI(ek, ej, ei);
                double Ui[MAXM], feq[7 * MAXM], S[MAXM];
                for (int c = 0; c < m; c++) Ui[c] = Ue[EU(c, e)];
                orc_equilibrium(p, Ui, alpha, lam, feq);
                orc_source(p, Ui, posx[ei], posy[ej], S);
                double w = om[e];
                for (int k = 0; k < Q; k++)
                    for (int c = 0; c < m; c++) {
                        double fk = fe[EF(k, c, e)];
                        post[EF(k, c, e)] = fk - w * (fk - feq[k * m + c]) + 0.5 * dt * a[k] * S[c];
                    }
            }

    /* 7-8. pull streaming, implicit moment (2.8), second half of the source */
#pragma omp parallel for collapse(2) reduction(| : flags)
    for (int kk = 0; kk < nz; kk++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                const size_t e = EI(kk + gz, j + gy, i + G);
                double Fk[7 * MAXM], Ubar[MAXM], Un[MAXM], S[MAXM];
                for (int k = 0; k < Q; k++) {
                    /* e_0 = 0, e_j = unit vector j, e_{j+d} = -e_j (Section 2.3) */
                    size_t src = e;
                    if (k >= 1 && k <= d) src = e - stride[k - 1];
                    if (k > d) src = e + stride[k - d - 1];
                    for (int c = 0; c < m; c++) Fk[k * m + c] = post[EF(k, c, src)];
                }
                for (int c = 0; c < m; c++) {
                    double sum = 0.0;
                    for (int k = 0; k < Q; k++) sum += Fk[k * m + c];
                    Ubar[c] = sum;
                }
                double xn = node_x(p, i), yn = node_y(p, j);
                flags |= solve_implicit_moment(p, Ubar, xn, yn, dt, Un);
                orc_source(p, Un, xn, yn, S);
                for (int k = 0; k < Q; k++)
                    for (int c = 0; c < m; c++)
                        fn[FI(k, c, kk, j, i)] = Fk[k * m + c] + 0.5 * dt * a[k] * S[c];
                if (nonphysical(p, Un)) flags |= ORC_FLAG_NONPHYSICAL;
                if (omega_out) omega_out[((size_t)kk * ny + j) * nx + i] = om[e];
            }

    if (info) {
        info[0] = abar[0];
        info[1] = abar[1];
        info[2] = dt;
        info[3] = lam;
        if (d == 3) info[4] = abar[2];
    }
    free(fe); free(Ue); free(nu); free(om); free(post); free(srci); free(srcj); free(srck);
    free(posx); free(posy);
    return flags;
#undef EI
#undef EF
#undef EU
#undef FI
}

/*
 * Advance f in place until t reaches T (clipping the last step) or nsteps_max
 * steps were taken.  t is updated.  Returns the OR of the step flags, or a
 * negative error; *nsteps receives the number of steps taken.
 */
int orc_advance(const orc_problem *p, double *f, double *t, double T, long nsteps_max, long *nsteps) {
    if (check_problem(p)) return ORC_ERR_ARG;
    int m = orc_nfields(p), Q = nq(p);
    size_t n = (size_t)Q * m * p->nx * rows_of(p);
    double *g = malloc(sizeof(double) * n);
    if (!g) return ORC_ERR_MEM;
    int flags = 0;
    long s = 0;
    double info[5];
    while (s < nsteps_max && (T <= 0.0 || *t < T)) {
        double cap = T > 0.0 ? T - *t : 0.0;
        int r = orc_step(p, f, g, cap, NULL, info, NULL);
        if (r < 0) { free(g); return r; }
        flags |= r;
        memcpy(f, g, sizeof(double) * n);
        *t = (T > 0.0 && info[2] == cap) ? T : *t + info[2];
        s++;
    }
    free(g);
    if (nsteps) *nsteps = s;
    return flags;
}

/* Threads of the OpenMP loops (for timing the oracle on one core or on all of
 * them); returns the number in effect.  Results do not depend on it: every
 * loop writes disjoint nodes and the one reduction is a bitwise OR. */
int orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
