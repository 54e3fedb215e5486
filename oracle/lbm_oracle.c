/*
 * FP64 CPU oracle of the coupled metaball-DEM / lattice-Boltzmann step of
 * Zhang, Qiu, Chen, Scheuermann, Li, Galindo-Torres, "Coupled Metaball
 * Discrete Element Lattice Boltzmann Method for fluid-particle systems with
 * non-spherical particle shapes: a sharp interface coupling scheme"
 * (arXiv 2206.11634).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference the CUDA path is
 * checked against.  Only the test suite, the smoke check and the timed CPU
 * baseline of the benchmark may load it.  It shares no code, header, table or
 * helper with the CUDA library, and the library never calls it.
 *
 * Plain, slow, obviously correct: every node and every link is visited in
 * index order, everything is double precision, and each function names the
 * passage of the paper it follows.  Equation numbers are the paper's, counted
 * in typeset order (Eq. (1) is the Newton-Euler system of §2.1.1, Eq. (32) the
 * missing-point torque of §2.3.5).  Where the paper is silent or ambiguous the
 * reading taken is stated at the spot ("Reading:").
 *
 * Units: lattice units, dx = dt = C = 1, c_s^2 = 1/3.  Node (i,j,k) sits at
 * position (i,j,k).  Non-periodic faces are no-slip walls halfway between the
 * last node and the next, at -1/2 and n-1/2.
 *
 * Pins (tests/test_oracle_*.py) tie every function here to a closed form, an
 * invariant, a textbook special case, or, for the whole lattice step, a
 * brute-force transcription written from the paper (tests/_bruteforce.py).
 * Parity unpinned: the numerical values of the contact constants k_n, eta_n,
 * k_t, eta_t, mu_s (the paper gives none; the law itself is pinned) and the
 * paper's experimental comparisons (their data are not in its text).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXCP 16
#define ORC_MAXQ 19
#define ORC_NWALL 6
#define ORC_ROT_ITERS 2

/* ------------------------------------------------------------------------- */
/* Public structs (mirrored by ctypes in oracle/oracle.py).                   */
/* ------------------------------------------------------------------------- */
typedef struct {
    int nx, ny, nz;
    int Q;              /* 19 (D3Q19) or 15 (D3Q15, the paper's lattice, §2.2) */
    int periodic[3];
    int n_sub;          /* DEM sub-steps per LBM step, §2.3.4 */
    int vibb;           /* 1: VIBB on particle links (§2.3.1); 0: halfway on all */
    int missing_force;  /* 1: missing-force-point treatment, §2.3.5 item 2 */
    int nthreads;       /* OpenMP threads for the lattice loops; 0 = default */
    int q_exact;        /* 1: link fraction q by Newton on Eq. (26); 0: Eq. (27) */
    double tau, rho0, c0;
    double u0[3];       /* initial uniform fluid velocity */
    double force[3];    /* body force density on the fluid (Guo forcing) */
    double gravity[3];  /* gravity, applied to particles only as (1-rho_f/rho_s) g */
    double kn, eta_n, kt, eta_t, mu_s, c_tol;  /* contact law, §2.1.1 / §2.1.3 */
    double mass_spacing; /* sample spacing of the mass-property integration */
} orc_config;

typedef struct {
    int ncp, fixed;
    double cp[ORC_MAXCP][3];  /* control points, body frame, about the centroid */
    double K[ORC_MAXCP];      /* weights K_i >= 0, Eq. (4) */
    double Rs;                /* sphero radius of the contact skin, §2.1.3 */
    double density;           /* rho_s */
    double mass;              /* <= 0: computed by orc_set_particles */
    double inertia[9];        /* body-frame inertia tensor about the centroid */
    double x[3];              /* centroid, world */
    double q[4];              /* orientation quaternion (w,x,y,z), body -> world */
    double v[3];              /* translational velocity */
    double w[3];              /* angular velocity, world frame */
} orc_particle;

typedef struct {
    orc_config c;
    int Q;
    int e[ORC_MAXQ][3];
    double wt[ORC_MAXQ];
    int opp[ORC_MAXQ];
    long N;
    double *f;    /* [Q][N] post-collision populations at the current time */
    double *g;    /* [Q][N] next populations */
    int *own;     /* [N] -1 fluid, else owning particle; geometry f is consistent with */
    int *own_new; /* [N] */
    double *rho;  /* [N] density used in the last collision */
    double *u;    /* [3][N] velocity used in the last collision */
    int np;
    orc_particle *p;
    double (*cpw)[ORC_MAXCP][3]; /* world control points */
    double (*Fh)[3], (*Th)[3];   /* hydrodynamic force / torque of the last step */
    double (*Fc)[3], (*Tc)[3];   /* contact force / torque of the last evaluation */
    /* contact history: tangential spring xi and Newton warm start */
    int *pair_on;
    double (*pair_xi)[3];
    double (*pair_xm)[3];
    int *wall_on;
    int *pair_warm;   /* the last evaluation of this potential collision found a valid x_m */
    int *wall_warm;   /* ... a valid x_cw */
    double (*wall_xi)[3];
    double (*wall_xcw)[3];
    long step;
    int nrefill;  /* new fluid nodes refilled in the last step */
    int nlinks;   /* particle boundary links in the last sweep */
    int frozen;   /* 1: node flags kept as they are (no classification, no refill) */
} orc_state;

/* ------------------------------------------------------------------------- */
/* Lattices.                                                                  */
/* ------------------------------------------------------------------------- */

/* D3Q15 as defined in §2.2: e_0 = 0, e_1..6 = (+-C,0,0),(0,+-C,0),(0,0,+-C),
 * e_7..14 = (+-C,+-C,+-C); weights 2/9, 1/9, 1/72. */
static const int D3Q15_E[15][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 1}, {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1},
    {1, -1, 1}, {-1, 1, -1}, {-1, 1, 1}, {1, -1, -1}};

/* D3Q19 (rest 1/3, six axis links 1/18, twelve face diagonals 1/36): the
 * lattice the build's workloads run on; the paper's method is lattice
 * independent apart from the weights. */
static const int D3Q19_E[19][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static int setup_lattice(orc_state *s, int Q) {
    const int(*E)[3];
    if (Q == 19) E = D3Q19_E;
    else if (Q == 15) E = D3Q15_E;
    else return -1;
    s->Q = Q;
    for (int i = 0; i < Q; i++) {
        for (int a = 0; a < 3; a++) s->e[i][a] = E[i][a];
        int len2 = E[i][0] * E[i][0] + E[i][1] * E[i][1] + E[i][2] * E[i][2];
        if (Q == 19) s->wt[i] = len2 == 0 ? 1.0 / 3.0 : (len2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        else s->wt[i] = len2 == 0 ? 2.0 / 9.0 : (len2 == 1 ? 1.0 / 9.0 : 1.0 / 72.0);
    }
    /* opposite direction i': e_i' = -e_i, found by search */
    for (int i = 0; i < Q; i++) {
        s->opp[i] = -1;
        for (int k = 0; k < Q; k++)
            if (E[k][0] == -E[i][0] && E[k][1] == -E[i][1] && E[k][2] == -E[i][2]) s->opp[i] = k;
        if (s->opp[i] < 0) return -1;
    }
    return 0;
}

/* Second-order equilibrium, Eq. (16), C = 1. */
static double feq(const orc_state *s, int i, double rho, const double u[3]) {
    double eu = s->e[i][0] * u[0] + s->e[i][1] * u[1] + s->e[i][2] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return s->wt[i] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
}

/* ------------------------------------------------------------------------- */
/* Small vector helpers.                                                      */
/* ------------------------------------------------------------------------- */
static void cross(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double norm(const double a[3]) { return sqrt(dot(a, a)); }

static int dim(const orc_state *s, int a) { return a == 0 ? s->c.nx : (a == 1 ? s->c.ny : s->c.nz); }

/* Minimum-image component along a periodic axis; identity on a walled axis. */
static double minimg(const orc_state *s, int a, double d) {
    if (s->c.periodic[a]) {
        double L = (double)dim(s, a);
        d -= L * floor(d / L + 0.5);
    }
    return d;
}

/* Rotation matrix of a unit quaternion (w,x,y,z), body -> world. */
static void quat_to_R(const double q[4], double R[9]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}
static void matvec(const double A[9], const double v[3], double r[3]) {
    r[0] = A[0] * v[0] + A[1] * v[1] + A[2] * v[2];
    r[1] = A[3] * v[0] + A[4] * v[1] + A[5] * v[2];
    r[2] = A[6] * v[0] + A[7] * v[1] + A[8] * v[2];
}
static void matTvec(const double A[9], const double v[3], double r[3]) {
    r[0] = A[0] * v[0] + A[3] * v[1] + A[6] * v[2];
    r[1] = A[1] * v[0] + A[4] * v[1] + A[7] * v[2];
    r[2] = A[2] * v[0] + A[5] * v[1] + A[8] * v[2];
}
/* Inverse of a 3x3 matrix by cofactors; returns 0 if singular. */
static int inv3(const double A[9], double B[9]) {
    double c0 = A[4] * A[8] - A[5] * A[7];
    double c1 = A[5] * A[6] - A[3] * A[8];
    double c2 = A[3] * A[7] - A[4] * A[6];
    double det = A[0] * c0 + A[1] * c1 + A[2] * c2;
    if (det == 0.0 || !isfinite(det)) return 0;
    double id = 1.0 / det;
    B[0] = c0 * id; B[1] = (A[2] * A[7] - A[1] * A[8]) * id; B[2] = (A[1] * A[5] - A[2] * A[4]) * id;
    B[3] = c1 * id; B[4] = (A[0] * A[8] - A[2] * A[6]) * id; B[5] = (A[2] * A[3] - A[0] * A[5]) * id;
    B[6] = c2 * id; B[7] = (A[1] * A[6] - A[0] * A[7]) * id; B[8] = (A[0] * A[4] - A[1] * A[3]) * id;
    return 1;
}

/* ------------------------------------------------------------------------- */
/* Metaball function, Eq. (4): M(x) = sum_i K_i / |x - x_i|^2.               */
/* ------------------------------------------------------------------------- */
static double metaball(const orc_state *s, int j, const double x[3]) {
    const orc_particle *p = &s->p[j];
    double M = 0.0;
    for (int k = 0; k < p->ncp; k++) {
        double dx = minimg(s, 0, x[0] - s->cpw[j][k][0]);
        double dy = minimg(s, 1, x[1] - s->cpw[j][k][1]);
        double dz = minimg(s, 2, x[2] - s->cpw[j][k][2]);
        double r2 = dx * dx + dy * dy + dz * dz;
        M += p->K[k] / r2;
    }
    return M;
}

/* Value, gradient and Hessian of Eq. (4) (used by the contact searches of
 * §2.1.3-2.1.4).  d/dx K/r^2 = -2K r/r^4; d2/dx2 = K(8 r r^T/r^6 - 2 I/r^4). */
static void metaball_dd(const orc_state *s, int j, const double x[3], double *M, double g[3], double H[9]) {
    const orc_particle *p = &s->p[j];
    *M = 0.0;
    for (int a = 0; a < 3; a++) g[a] = 0.0;
    for (int a = 0; a < 9; a++) H[a] = 0.0;
    for (int k = 0; k < p->ncp; k++) {
        double r[3];
        for (int a = 0; a < 3; a++) r[a] = minimg(s, a, x[a] - s->cpw[j][k][a]);
        double r2 = dot(r, r);
        double K = p->K[k];
        *M += K / r2;
        for (int a = 0; a < 3; a++) g[a] += -2.0 * K * r[a] / (r2 * r2);
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++)
                H[3 * a + b] += K * (8.0 * r[a] * r[b] / (r2 * r2 * r2) - (a == b ? 2.0 / (r2 * r2) : 0.0));
    }
}

static double sumK(const orc_particle *p) {
    double S = 0.0;
    for (int k = 0; k < p->ncp; k++) S += p->K[k];
    return S;
}

/* World positions of the control points, x_i = x_p + R(q) x_i^body. */
static void update_world_cps(orc_state *s) {
    for (int j = 0; j < s->np; j++) {
        double R[9];
        quat_to_R(s->p[j].q, R);
        for (int k = 0; k < s->p[j].ncp; k++) {
            double r[3];
            matvec(R, s->p[j].cp[k], r);
            for (int a = 0; a < 3; a++) s->cpw[j][k][a] = s->p[j].x[a] + r[a];
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Node classification, §2.3.1: a node is solid when it lies inside a metaball,
 * M_j(x) >= c0 (Eq. (26)); otherwise fluid.  Reading: c0 = 1 (the surface of
 * Eq. (4)); where several particles cover a node the owner is the one with the
 * largest M_j, ties to the lower index.  Only nodes inside the box
 * AABB(control points) +- sqrt(sum K / c0) are visited: M_j >= c0 forces
 * min_i |x - x_i|^2 <= sum K / c0, so no solid node lies outside it.          */
/* ------------------------------------------------------------------------- */
static long nidx(const orc_state *s, int x, int y, int z) {
    return (long)x + (long)s->c.nx * ((long)y + (long)s->c.ny * (long)z);
}

static void classify(orc_state *s, int *own) {
    long N = s->N;
    double *best = (double *)malloc(sizeof(double) * (size_t)N);
    for (long n = 0; n < N; n++) { own[n] = -1; best[n] = 0.0; }
    for (int j = 0; j < s->np; j++) {
        const orc_particle *p = &s->p[j];
        double bound = sqrt(sumK(p) / s->c.c0);
        int lo[3], hi[3];
        for (int a = 0; a < 3; a++) {
            double mn = s->cpw[j][0][a], mx = s->cpw[j][0][a];
            for (int k = 1; k < p->ncp; k++) {
                if (s->cpw[j][k][a] < mn) mn = s->cpw[j][k][a];
                if (s->cpw[j][k][a] > mx) mx = s->cpw[j][k][a];
            }
            lo[a] = (int)ceil(mn - bound);
            hi[a] = (int)floor(mx + bound);
            if (!s->c.periodic[a]) {
                if (lo[a] < 0) lo[a] = 0;
                if (hi[a] > dim(s, a) - 1) hi[a] = dim(s, a) - 1;
            } else if (hi[a] - lo[a] + 1 > dim(s, a)) {
                lo[a] = 0;
                hi[a] = dim(s, a) - 1;
            }
        }
        for (int zz = lo[2]; zz <= hi[2]; zz++)
            for (int yy = lo[1]; yy <= hi[1]; yy++)
                for (int xx = lo[0]; xx <= hi[0]; xx++) {
                    int ix = ((xx % s->c.nx) + s->c.nx) % s->c.nx;
                    int iy = ((yy % s->c.ny) + s->c.ny) % s->c.ny;
                    int iz = ((zz % s->c.nz) + s->c.nz) % s->c.nz;
                    double pos[3] = {ix, iy, iz};
                    double M = metaball(s, j, pos);
                    long n = nidx(s, ix, iy, iz);
                    if (M >= s->c.c0 && (own[n] < 0 || M > best[n])) {
                        own[n] = j;
                        best[n] = M;
                    }
                }
    }
    free(best);
}

/* Whether x lies in particle j's search box AABB(control points) +-
 * sqrt(sum K / c0) (minimum image on periodic axes); M_j(x) >= c0 only there. */
static int in_search_box(const orc_state *s, int j, const double x[3]) {
    const orc_particle *p = &s->p[j];
    double bound = sqrt(sumK(p) / s->c.c0);
    for (int a = 0; a < 3; a++) {
        double mn = s->cpw[j][0][a], mx = s->cpw[j][0][a];
        for (int k = 1; k < p->ncp; k++) {
            if (s->cpw[j][k][a] < mn) mn = s->cpw[j][k][a];
            if (s->cpw[j][k][a] > mx) mx = s->cpw[j][k][a];
        }
        double c = 0.5 * (mn + mx), hw = 0.5 * (mx - mn) + bound;
        if (fabs(minimg(s, a, x[a] - c)) > hw) return 0;
    }
    return 1;
}

/* Neighbour of node (x,y,z) along integer offset o.  Returns 1 and the wrapped
 * node index when it lies in the domain (periodic axes wrap), 0 when it lies
 * beyond a wall. */
static int neighbour(const orc_state *s, int x, int y, int z, const int o[3], long *n) {
    int c[3] = {x + o[0], y + o[1], z + o[2]};
    for (int a = 0; a < 3; a++) {
        int L = dim(s, a);
        if (c[a] < 0 || c[a] >= L) {
            if (!s->c.periodic[a]) return 0;
            c[a] = ((c[a] % L) + L) % L;
        }
    }
    *n = nidx(s, c[0], c[1], c[2]);
    return 1;
}

/* Surface velocity u_w = v_p + w_p x (x_w - x_p), §2.3.1. */
static void surface_velocity(const orc_state *s, int j, const double xw[3], double uw[3], double r[3]) {
    for (int a = 0; a < 3; a++) r[a] = minimg(s, a, xw[a] - s->p[j].x[a]);
    double wr[3];
    cross(s->p[j].w, r, wr);
    for (int a = 0; a < 3; a++) uw[a] = s->p[j].v[a] + wr[a];
}

/* ------------------------------------------------------------------------- */
/* Link fraction q.                                                           */
/* ------------------------------------------------------------------------- */

/* Linear approximation, Eq. (27): q = (c0 - M(x_f)) / (M(x_s) - M(x_f)). */
static double q_linear(double c0, double Mf, double Ms) { return (c0 - Mf) / (Ms - Mf); }

/* Exact root of Eq. (26), M(x_f + q d) = c0, by Newton's method with the
 * tolerance 1e-7 and iteration cap 100 quoted in §2.3.1, started from
 * Eq. (27).  Reading: the root sought is the one in [0,1] (M(x_f) < c0 <=
 * M(x_s) brackets it); the iteration stops when the Newton correction is
 * below the tolerance (taking it); a larger step that leaves the current
 * bracket is replaced by bisection, so grazing links cannot run off to the
 * far side of the particle.  Returns the iteration count, or -1 without
 * convergence. */
int orc_q_newton(const orc_state *s, int j, const double xf[3], const double d[3], double tol, int maxit,
                 double *q_out) {
    double xs[3] = {xf[0] + d[0], xf[1] + d[1], xf[2] + d[2]};
    double lo = 0.0, hi = 1.0;
    double q = q_linear(s->c.c0, metaball(s, j, xf), metaball(s, j, xs));
    for (int it = 0; it < maxit; it++) {
        double x[3] = {xf[0] + q * d[0], xf[1] + q * d[1], xf[2] + q * d[2]};
        double M, gr[3], H[9];
        metaball_dd(s, j, x, &M, gr, H);
        double r = M - s->c.c0;
        if (r < 0.0) lo = q; else hi = q;
        double slope = dot(gr, d);
        if (slope != 0.0 && fabs(r / slope) < tol) {
            *q_out = q - r / slope;
            return it + 1;
        }
        double qn = slope != 0.0 ? q - r / slope : 0.5 * (lo + hi);
        if (!(qn > lo && qn < hi)) qn = 0.5 * (lo + hi);
        double dq = qn - q;
        q = qn;
        if (fabs(dq) < tol) {
            *q_out = q;
            return it + 1;
        }
    }
    *q_out = q;
    return -1;
}

/* The link fraction the sweep uses for the link x_f -> x_f + d of particle j
 * (M_j(x_f) = Mf < c0 <= Ms = M_j(x_f + d)): Eq. (27), or, with q_exact, the
 * root of Eq. (26) by the Newton iteration above with the tolerance 1e-7 and
 * the cap of 100 iterations of §2.3.1 (the last iterate when the cap is hit). */
static double link_q(const orc_state *s, int j, const double xf[3], const double d[3], double Mf, double Ms) {
    double q = q_linear(s->c.c0, Mf, Ms);
    if (s->c.q_exact) orc_q_newton(s, j, xf, d, 1e-7, 100, &q);
    return q;
}

/* ------------------------------------------------------------------------- */
/* Local refilling of new fluid nodes, §2.3.3 (Eq. (30)).                     */
/* Reading: a population f_i' at x_new counts as known (Eq. (30)) when it
 * streams in from x_new + e_i and that node was fluid before the particle
 * moved; then f_i(x_new) = f_i'(x_new) + 6 w_i' rho_f e_i.u_w with u_w the
 * surface velocity at x_new of the particle that uncovered it and rho_f =
 * rho0.  Otherwise f_i(x_new) = f^eq_i(rho0, u_new).  The refilled values are
 * stored as the node's post-collision populations, so the next sweep streams
 * them like any other node's.                                                */
/* ------------------------------------------------------------------------- */
static void refill(orc_state *s) {
    int nref = 0;
    for (int z = 0; z < s->c.nz; z++)
        for (int y = 0; y < s->c.ny; y++)
            for (int x = 0; x < s->c.nx; x++) {
                long n = nidx(s, x, y, z);
                if (!(s->own[n] >= 0 && s->own_new[n] < 0)) continue;
                nref++;
                int j = s->own[n];
                double pos[3] = {x, y, z}, unew[3], r[3];
                surface_velocity(s, j, pos, unew, r);
                for (int i = 0; i < s->Q; i++) {
                    long nb;
                    int known = neighbour(s, x, y, z, s->e[i], &nb) && s->own[nb] < 0;
                    double val;
                    if (known) {
                        double eu = s->e[i][0] * unew[0] + s->e[i][1] * unew[1] + s->e[i][2] * unew[2];
                        int io = s->opp[i];
                        val = s->f[(long)io * s->N + nb] + 6.0 * s->wt[io] * s->c.rho0 * eu;
                    } else {
                        val = feq(s, i, s->c.rho0, unew);
                    }
                    s->f[(long)i * s->N + n] = val;
                }
            }
    s->nrefill = nref;
}

/* ------------------------------------------------------------------------- */
/* Unknown population on a particle link, §2.3.1.                            */
/* x_f fluid, x_s = x_f + d solid of particle j, d = e_i' points into the
 * solid; the unknown is f_i(x_f, t+1) with e_i = -d.  VIBB, Eqs. (19)-(25):
 *   f_i(x_f,t+1) = f+_i'(x_d,t) + 6 w_i' rho_f e_i.u_w                  (19)
 *   f+_i'(x_d,t) = f^eq_i'(rho_d,u_d) + f^neq_i'(x_d,t)                 (20)
 *   f^neq_i'(x_d) = 2q[f+_i'(x_f)-f^eq_i'(x_f)] + (1-2q)[f+_i'(x_ff)-f^eq_i'(x_ff)]  (21)
 *   rho_d = 2q rho_f + (1-2q) rho_ff (q<=1/2), rho_f (q>1/2)            (22)
 *   u*_d = 2q u_f + (1-2q) u_ff (q<=1/2), (1-q)/q u_f + (2q-1)/q u_w    (23)
 *   u**_d = (1-q)/(1+q) u_ff + 2q/(1+q) u_w                             (24)
 *   u_d = u*_d/3 + 2 u**_d/3                                            (25)
 * with x_ff = x_f - d.  Reading: Eq. (21) applies for every q (it
 * extrapolates for q > 1/2); rho_f, u_f, rho_ff, u_ff are the moments of the
 * time level of the stored post-collision populations f+: rho = sum f+ and,
 * since Guo's collision adds the body force F to the momentum, u =
 * (sum f+ e - F/2)/rho, the velocity that entered that collision (without a
 * body force this is Eq. (18) itself).  When x_ff is not a fluid node there
 * are not enough fluid nodes for VIBB and halfway bounce-back is used
 * (§2.3.5 item 1): f_i(x_f,t+1) = f+_i'(x_f,t) + 6 w_i' rho_f e_i.u_w.
 * Reading: u_w is taken at x_w = x_f + q d in both cases.                    */
/* ------------------------------------------------------------------------- */
/* The unknown f_i(x_f, t+1) of one particle link from the stored
 * populations of x_f and x_ff (fplus_ff == NULL when x_ff is not a fluid
 * node).  q is the link fraction, uw the surface velocity at x_w, io = i'. */
static double vibb_unknown(const orc_state *s, int i, double q, const double *fplus_f, const double *fplus_ff,
                           const double uw[3]) {
    int io = s->opp[i];
    double rho_f = 0.0, m_f[3] = {0, 0, 0}, u_f[3];
    for (int k = 0; k < s->Q; k++) {
        rho_f += fplus_f[k];
        for (int a = 0; a < 3; a++) m_f[a] += fplus_f[k] * s->e[k][a];
    }
    for (int a = 0; a < 3; a++) u_f[a] = (m_f[a] - 0.5 * s->c.force[a]) / rho_f;
    double eu_w = s->e[i][0] * uw[0] + s->e[i][1] * uw[1] + s->e[i][2] * uw[2];
    if (!s->c.vibb || fplus_ff == NULL) return fplus_f[io] + 6.0 * s->wt[io] * rho_f * eu_w;
    double rho_ff = 0.0, m_ff[3] = {0, 0, 0}, u_ff[3];
    for (int k = 0; k < s->Q; k++) {
        rho_ff += fplus_ff[k];
        for (int a = 0; a < 3; a++) m_ff[a] += fplus_ff[k] * s->e[k][a];
    }
    for (int a = 0; a < 3; a++) u_ff[a] = (m_ff[a] - 0.5 * s->c.force[a]) / rho_ff;
    double fneq_d = 2.0 * q * (fplus_f[io] - feq(s, io, rho_f, u_f)) +
                    (1.0 - 2.0 * q) * (fplus_ff[io] - feq(s, io, rho_ff, u_ff));
    double rho_d, us[3], uss[3], ud[3];
    if (q <= 0.5) {
        rho_d = 2.0 * q * rho_f + (1.0 - 2.0 * q) * rho_ff;
        for (int a = 0; a < 3; a++) us[a] = 2.0 * q * u_f[a] + (1.0 - 2.0 * q) * u_ff[a];
    } else {
        rho_d = rho_f;
        for (int a = 0; a < 3; a++) us[a] = (1.0 - q) / q * u_f[a] + (2.0 * q - 1.0) / q * uw[a];
    }
    for (int a = 0; a < 3; a++) uss[a] = (1.0 - q) / (1.0 + q) * u_ff[a] + 2.0 * q / (1.0 + q) * uw[a];
    for (int a = 0; a < 3; a++) ud[a] = us[a] / 3.0 + 2.0 * uss[a] / 3.0;
    double fplus_d = feq(s, io, rho_d, ud) + fneq_d;
    return fplus_d + 6.0 * s->wt[io] * rho_f * eu_w;
}

typedef struct {
    double fin;  /* the unknown f_i(x_f, t+1) */
    double xw[3], uw[3], rarm[3];
} link_result;

static link_result particle_link(const orc_state *s, int x, int y, int z, long n, int i, int j) {
    link_result L;
    int io = s->opp[i];
    double d[3] = {s->e[io][0], s->e[io][1], s->e[io][2]};
    double xf[3] = {x, y, z};
    double xs[3] = {x + d[0], y + d[1], z + d[2]};
    double q = link_q(s, j, xf, d, metaball(s, j, xf), metaball(s, j, xs));
    for (int a = 0; a < 3; a++) L.xw[a] = xf[a] + q * d[a];
    surface_velocity(s, j, L.xw, L.uw, L.rarm);
    double ff[ORC_MAXQ], fff[ORC_MAXQ];
    for (int k = 0; k < s->Q; k++) ff[k] = s->f[(long)k * s->N + n];
    long nff;
    int o_ff[3] = {s->e[i][0], s->e[i][1], s->e[i][2]}; /* x_ff = x_f - d = x_f + e_i */
    int ff_fluid = neighbour(s, x, y, z, o_ff, &nff) && s->own_new[nff] < 0;
    if (ff_fluid)
        for (int k = 0; k < s->Q; k++) fff[k] = s->f[(long)k * s->N + nff];
    L.fin = vibb_unknown(s, i, q, ff, ff_fluid ? fff : NULL, L.uw);
    return L;
}

/* ------------------------------------------------------------------------- */
/* Fused stream + bounce-back + collide over every fluid node (§2.2, §2.3),
 * with the Galilean-invariant momentum exchange of Eqs. (28)-(29) and the
 * missing force points of Eqs. (31)-(32).                                    */
/* ------------------------------------------------------------------------- */
static void sweep(orc_state *s) {
    const int Q = s->Q;
    const long N = s->N;
    const double tau = s->c.tau;
    const double *F = s->c.force;
    const int np = s->np;
    int nthr = 1;
#ifdef _OPENMP
    nthr = s->c.nthreads > 0 ? s->c.nthreads : omp_get_max_threads();
#endif
    /* per-thread partial sums, combined in thread order afterwards */
    double *acc = (double *)calloc((size_t)nthr * (size_t)(np > 0 ? np : 1) * 6, sizeof(double));
    int *links = (int *)calloc((size_t)nthr, sizeof(int));

#ifdef _OPENMP
#pragma omp parallel for num_threads(nthr) schedule(static)
#endif
    for (int z = 0; z < s->c.nz; z++) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *A = acc + (size_t)tid * (size_t)(np > 0 ? np : 1) * 6;
        for (int y = 0; y < s->c.ny; y++)
            for (int x = 0; x < s->c.nx; x++) {
                long n = nidx(s, x, y, z);
                int jn = s->own_new[n];
                if (jn >= 0) {
                    /* Missing force points, §2.3.5 item 2, Eqs. (31)-(32).
                     * Reading: the force points of particle j are the links
                     * y -> x_s = y + d that cross its surface (M_j(y) < c0 <=
                     * M_j(x_s)).  The momentum exchange of Eq. (28) sees those
                     * whose y is a fluid node and whose x_s is owned by j; every
                     * other one (y covered by another particle or beyond a box
                     * wall, or x_s inside j but owned by another particle) is a
                     * missing force point and gets the equilibrium term with
                     * rho0 and u_w.  q and x_w follow Eq. (27) with M_j. */
                    if (!s->c.missing_force) continue;
                    double xs[3] = {x, y, z};
                    for (int j = 0; j < np; j++) {
                        double Ms;
                        if (j != jn) {
                            if (!in_search_box(s, j, xs)) continue;
                            Ms = metaball(s, j, xs);
                            if (Ms < s->c.c0) continue;
                        } else {
                            Ms = metaball(s, j, xs);
                        }
                        for (int i = 1; i < Q; i++) {
                            int mo[3] = {-s->e[i][0], -s->e[i][1], -s->e[i][2]};
                            long ny_;
                            int inside = neighbour(s, x, y, z, mo, &ny_);
                            if (inside && s->own_new[ny_] < 0 && j == jn) continue; /* seen by Eq. (28) */
                            if (inside && s->own_new[ny_] == j) continue;           /* interior of j */
                            double yp[3] = {x + mo[0], y + mo[1], z + mo[2]};
                            double My = metaball(s, j, yp);
                            if (My >= s->c.c0) continue;
                            double d[3] = {s->e[i][0], s->e[i][1], s->e[i][2]};
                            double q = link_q(s, j, yp, d, My, Ms);
                            double xw[3], uw[3], r[3];
                            for (int c = 0; c < 3; c++) xw[c] = yp[c] + q * d[c];
                            surface_velocity(s, j, xw, uw, r);
                            double fi = feq(s, i, s->c.rho0, uw);          /* toward the solid, e_i = d */
                            double fo = feq(s, s->opp[i], s->c.rho0, uw);  /* bounced back, e_i' = -d */
                            double dP[3], tq[3];
                            for (int c = 0; c < 3; c++) dP[c] = (d[c] - uw[c]) * fi - (-d[c] - uw[c]) * fo;
                            cross(r, dP, tq);
                            for (int c = 0; c < 3; c++) {
                                A[6 * j + c] += dP[c];
                                A[6 * j + 3 + c] += tq[c];
                            }
                        }
                    }
                    continue;
                }
                double fin[ORC_MAXQ];
                for (int i = 0; i < Q; i++) {
                    int mo[3] = {-s->e[i][0], -s->e[i][1], -s->e[i][2]};
                    long src;
                    int io = s->opp[i];
                    if (!neighbour(s, x, y, z, mo, &src)) {
                        /* box wall: stationary halfway bounce-back */
                        fin[i] = s->f[(long)io * N + n];
                        continue;
                    }
                    int js = s->own_new[src];
                    if (js < 0) {
                        fin[i] = s->f[(long)i * N + src];
                        continue;
                    }
                    link_result L = particle_link(s, x, y, z, n, i, js);
                    fin[i] = L.fin;
                    links[tid]++;
                    /* Eqs. (28)-(29): force on particle js from this link;
                     * e_i' = d is the outgoing direction (toward the solid),
                     * f_i'(x_f,t) its post-collision population and f_i(x_f,
                     * t+1) the bounced one.  Reading of the time levels:
                     * Wen et al.'s outgoing/incoming pair. */
                    double dP[3], tq[3];
                    for (int a = 0; a < 3; a++) {
                        double d = s->e[io][a];
                        dP[a] = (d - L.uw[a]) * s->f[(long)io * N + n] - (-d - L.uw[a]) * L.fin;
                    }
                    cross(L.rarm, dP, tq);
                    for (int a = 0; a < 3; a++) {
                        A[6 * js + a] += dP[a];
                        A[6 * js + 3 + a] += tq[a];
                    }
                }
                /* moments, Eq. (18), with the half-force shift of Guo forcing */
                double rho = 0.0, m[3] = {0, 0, 0};
                for (int i = 0; i < Q; i++) {
                    rho += fin[i];
                    for (int a = 0; a < 3; a++) m[a] += fin[i] * s->e[i][a];
                }
                double u[3];
                for (int a = 0; a < 3; a++) u[a] = (m[a] + 0.5 * F[a]) / rho;
                s->rho[n] = rho;
                for (int a = 0; a < 3; a++) s->u[(long)a * N + n] = u[a];
                /* BGK, Eqs. (14)-(16), plus Guo's forcing term
                 * (1 - 1/(2 tau)) w_i [3(e_i - u) + 9 (e_i.u) e_i].F */
                for (int i = 0; i < Q; i++) {
                    double eu = s->e[i][0] * u[0] + s->e[i][1] * u[1] + s->e[i][2] * u[2];
                    double S = 0.0;
                    for (int a = 0; a < 3; a++) S += (3.0 * (s->e[i][a] - u[a]) + 9.0 * eu * s->e[i][a]) * F[a];
                    S *= (1.0 - 0.5 / tau) * s->wt[i];
                    s->g[(long)i * N + n] = fin[i] + (feq(s, i, rho, u) - fin[i]) / tau + S;
                }
            }
    }
    for (int j = 0; j < np; j++)
        for (int a = 0; a < 3; a++) { s->Fh[j][a] = 0.0; s->Th[j][a] = 0.0; }
    int nl = 0;
    for (int t = 0; t < nthr; t++) {
        nl += links[t];
        for (int j = 0; j < np; j++)
            for (int a = 0; a < 3; a++) {
                s->Fh[j][a] += acc[((size_t)t * np + j) * 6 + a];
                s->Th[j][a] += acc[((size_t)t * np + j) * 6 + 3 + a];
            }
    }
    s->nlinks = nl;
    free(acc);
    free(links);
}

/* ------------------------------------------------------------------------- */
/* DEM, §2.1.                                                                 */
/* ------------------------------------------------------------------------- */

/* Solve a 3x3 linear system H x = b by Cramer's rule; 0 if singular. */
static int solve3(const double H[9], const double b[3], double x[3]) {
    double Hi[9];
    if (!inv3(H, Hi)) return 0;
    matvec(Hi, b, x);
    return 1;
}

static double bounding_radius(const orc_particle *p, double c0) {
    double rmax = 0.0;
    for (int k = 0; k < p->ncp; k++) {
        double r = norm(p->cp[k]);
        if (r > rmax) rmax = r;
    }
    return rmax + sqrt(sumK(p) / c0) + p->Rs;
}

/* Contact law, §2.1.1: F_n = k_n delta + eta_n (v_j - v_i).n (Eq. (2)),
 * Coulomb-capped tangential spring-dashpot (Eq. (3)).  Reading: velocities
 * are those of the two bodies at the contact point; the tangential law is the
 * vector form F_t0 = -k_t xi - eta_t v_t with xi the tangential spring
 * (advanced by v_t h and kept in the tangent plane) and, when |F_t0| exceeds
 * mu_s F_n, F_t = mu_s F_n F_t0/|F_t0| with xi reset to match; F_n is not
 * allowed to become attractive.  Returns the force on body i. */
static void contact_law(const orc_state *s, double delta, const double n[3], const double vi[3], const double vj[3],
                        double xi[3], double h, double Fout[3]) {
    double vij[3] = {vi[0] - vj[0], vi[1] - vj[1], vi[2] - vj[2]};
    double vn = dot(vij, n);
    double Fn = s->c.kn * delta - s->c.eta_n * vn;
    if (Fn < 0.0) Fn = 0.0;
    double vt[3];
    for (int a = 0; a < 3; a++) vt[a] = vij[a] - vn * n[a];
    double xn = dot(xi, n);
    for (int a = 0; a < 3; a++) xi[a] = xi[a] - xn * n[a] + vt[a] * h;
    double Ft[3];
    for (int a = 0; a < 3; a++) Ft[a] = -s->c.kt * xi[a] - s->c.eta_t * vt[a];
    double ft = norm(Ft);
    if (ft > s->c.mu_s * Fn) {
        double sc = ft > 0.0 ? s->c.mu_s * Fn / ft : 0.0;
        for (int a = 0; a < 3; a++) {
            Ft[a] *= sc;
            xi[a] = s->c.kt > 0.0 ? -(Ft[a] + s->c.eta_t * vt[a]) / s->c.kt : 0.0;
        }
    }
    for (int a = 0; a < 3; a++) Fout[a] = Fn * n[a] + Ft[a];
}

static void point_velocity(const orc_state *s, int j, const double x[3], double v[3]) {
    double r[3], wr[3];
    for (int a = 0; a < 3; a++) r[a] = minimg(s, a, x[a] - s->p[j].x[a]);
    cross(s->p[j].w, r, wr);
    for (int a = 0; a < 3; a++) v[a] = s->p[j].v[a] + wr[a];
}

/* Metaball-metaball contact, §2.1.3, Eqs. (5)-(9).  Newton-Raphson on
 * grad(M_0 + M_1) = 0 (Eq. (6)) from xm_start (the caller passes the previous
 * minimum when the last evaluation of this potential collision found a valid
 * one), else from the midpoint of the closest pair of control points
 * (reading: the paper defers the start point to its ref. [zhang2021metaball];
 * the warm start follows what §2.1.4 states for walls).  *valid: Newton
 * converged to a minimum within Eq. (5)'s constraints.
 * The minimum must satisfy c_tol < M_k < 1 (Eq. (5)).  Closest points by
 * Eqs. (7)-(8), overlap, normal and contact point by Eq. (9).  Reading of
 * Eq. (9): the contact point is the middle of the overlap,
 * x_cp = x_c0 - (R_s0 - delta/2) n, n pointing from body 1 to body 0 (the
 * printed "+" places it outside the overlap for this n).
 * Returns 1 with delta, n (unit, from j to i) and x_cp when the dilated
 * shapes overlap. */
static int pair_geometry(const orc_state *s, int i, int j, const double *xm_start, double xm_out[3], double *delta,
                         double nvec[3], double xcp[3], int *valid) {
    double x[3];
    int converged = 0;
    *valid = 0;
    if (xm_start) {
        for (int a = 0; a < 3; a++) x[a] = xm_start[a];
    } else {
        double best = INFINITY;
        for (int a = 0; a < s->p[i].ncp; a++)
            for (int b = 0; b < s->p[j].ncp; b++) {
                double dd[3];
                for (int c = 0; c < 3; c++) dd[c] = minimg(s, c, s->cpw[j][b][c] - s->cpw[i][a][c]);
                double d2 = dot(dd, dd);
                if (d2 < best) {
                    best = d2;
                    for (int c = 0; c < 3; c++) x[c] = s->cpw[i][a][c] + 0.5 * dd[c];
                }
            }
    }
    for (int it = 0; it < 50; it++) {
        double M0, g0[3], H0[9], M1, g1[3], H1[9];
        metaball_dd(s, i, x, &M0, g0, H0);
        metaball_dd(s, j, x, &M1, g1, H1);
        double g[3], H[9], dx[3];
        for (int a = 0; a < 3; a++) g[a] = -(g0[a] + g1[a]);
        for (int a = 0; a < 9; a++) H[a] = H0[a] + H1[a];
        if (!solve3(H, g, dx)) break;
        for (int a = 0; a < 3; a++) x[a] += dx[a];
        if (norm(dx) < 1e-12) { converged = 1; break; }
    }
    for (int a = 0; a < 3; a++) xm_out[a] = x[a];
    double M0, g0[3], H0[9], M1, g1[3], H1[9];
    metaball_dd(s, i, x, &M0, g0, H0);
    metaball_dd(s, j, x, &M1, g1, H1);
    if (!(M0 > s->c.c_tol && M0 < 1.0 && M1 > s->c.c_tol && M1 < 1.0)) return 0;
    *valid = converged;   /* a local minimum of Eq. (5) within its constraints */
    double q0 = (1.0 - M0) / dot(g0, g0), q1 = (1.0 - M1) / dot(g1, g1);
    double xc0[3], xc1[3], dc[3];
    for (int a = 0; a < 3; a++) {
        xc0[a] = x[a] + q0 * g0[a];
        xc1[a] = x[a] + q1 * g1[a];
        dc[a] = xc0[a] - xc1[a];
    }
    double dist = norm(dc);
    *delta = s->p[i].Rs + s->p[j].Rs - dist;
    if (!(*delta > 0.0) || dist == 0.0) return 0;
    for (int a = 0; a < 3; a++) {
        nvec[a] = dc[a] / dist;
        xcp[a] = xc0[a] - (s->p[i].Rs - 0.5 * *delta) * nvec[a];
    }
    return 1;
}

int orc_pair_geometry(const orc_state *s, int i, int j, const double *xm_start, double xm_out[3], double *delta,
                      double nvec[3], double xcp[3]) {
    int valid;
    return pair_geometry(s, i, j, xm_start, xm_out, delta, nvec, xcp, &valid);
}

/* Metaball-plane contact, §2.1.4, Eqs. (10)-(13).  The plane is the box wall
 * wall = 2*axis + side (side 0 at -1/2, side 1 at n-1/2).  In the rotated
 * frame whose x axis is the wall normal m (pointing out of the fluid), Newton
 * solves the two tangential components of grad M = 0 on the plane (Eq. (10))
 * with dM/dm < 0; start from xcw_start (the caller passes the previous x_cw
 * when this potential collision existed at the previous evaluation and that
 * evaluation found a valid x_cw), else from the projection of the control
 * point nearest the plane.  *valid: Newton converged and dM/dm < 0 there.
 * Closest point by Eqs. (11)-(12), delta and n by Eq. (13) with n from x_cw
 * to x_cm.  Reading of Eq. (13): x_cp = x_cw - (delta/2) n, the middle of the
 * overlap. */
static int wall_geometry(const orc_state *s, int j, int wall, const double *xcw_start, double xcw_out[3],
                         double *delta, double nvec[3], double xcp[3], int *valid) {
    int converged = 0;
    *valid = 0;
    int ax = wall / 2, side = wall % 2;
    double plane = side ? dim(s, ax) - 0.5 : -0.5;
    double m[3] = {0, 0, 0};
    m[ax] = side ? 1.0 : -1.0;
    int t1 = (ax + 1) % 3, t2 = (ax + 2) % 3;
    double x[3];
    if (xcw_start) {
        for (int a = 0; a < 3; a++) x[a] = xcw_start[a];
    } else {
        int kbest = 0;
        double best = INFINITY;
        for (int k = 0; k < s->p[j].ncp; k++) {
            double dd = fabs(plane - s->cpw[j][k][ax]);
            if (dd < best) { best = dd; kbest = k; }
        }
        for (int a = 0; a < 3; a++) x[a] = s->cpw[j][kbest][a];
    }
    x[ax] = plane;
    for (int it = 0; it < 50; it++) {
        double M, g[3], H[9];
        metaball_dd(s, j, x, &M, g, H);
        double J00 = H[3 * t1 + t1], J01 = H[3 * t1 + t2], J10 = H[3 * t2 + t1], J11 = H[3 * t2 + t2];
        double det = J00 * J11 - J01 * J10;
        if (det == 0.0 || !isfinite(det)) break;
        double r0 = -g[t1], r1 = -g[t2];
        double d0 = (J11 * r0 - J01 * r1) / det, d1 = (-J10 * r0 + J00 * r1) / det;
        x[t1] += d0;
        x[t2] += d1;
        if (sqrt(d0 * d0 + d1 * d1) < 1e-12) { converged = 1; break; }
    }
    for (int a = 0; a < 3; a++) xcw_out[a] = x[a];
    double M, g[3], H[9];
    metaball_dd(s, j, x, &M, g, H);
    if (!(dot(g, m) < 0.0)) return 0;
    *valid = converged;   /* grad M along the outward normal at a converged x_cw */
    double qR = (1.0 - M) / dot(g, g);
    double xcm[3], dc[3];
    for (int a = 0; a < 3; a++) {
        xcm[a] = x[a] + qR * g[a];
        dc[a] = xcm[a] - x[a];
    }
    double dist = norm(dc);
    *delta = s->p[j].Rs - dist;
    if (!(*delta > 0.0) || dist == 0.0) return 0;
    for (int a = 0; a < 3; a++) {
        nvec[a] = dc[a] / dist;
        xcp[a] = x[a] - 0.5 * *delta * nvec[a];
    }
    return 1;
}

int orc_wall_geometry(const orc_state *s, int j, int wall, const double *xcw_start, double xcw_out[3],
                      double *delta, double nvec[3], double xcp[3]) {
    int valid;
    return wall_geometry(s, j, wall, xcw_start, xcw_out, delta, nvec, xcp, &valid);
}

/* All contact forces and torques at the current state (pairs, then walls),
 * advancing the tangential springs by h.  Pairs broad-phase on bounding
 * spheres (max |x_i^body| + sqrt(sum K / c0) + R_s). */
static void contacts(orc_state *s, double h) {
    int np = s->np;
    for (int j = 0; j < np; j++)
        for (int a = 0; a < 3; a++) { s->Fc[j][a] = 0.0; s->Tc[j][a] = 0.0; }
    for (int i = 0; i < np; i++)
        for (int j = i + 1; j < np; j++) {
            long pij = (long)i * np + j;
            double dx[3];
            for (int a = 0; a < 3; a++) dx[a] = minimg(s, a, s->p[j].x[a] - s->p[i].x[a]);
            double bi = bounding_radius(&s->p[i], s->c.c0), bj = bounding_radius(&s->p[j], s->c.c0);
            if (norm(dx) > bi + bj) {
                s->pair_on[pij] = 0;
                s->pair_warm[pij] = 0;
                continue;
            }
            /* Newton from the previous x_m when this potential collision
             * (overlapping bounding spheres) existed at the previous
             * evaluation and found a valid x_m, as for walls (§2.1.4) */
            double xm[3], delta, nv[3], xcp[3];
            int hit = pair_geometry(s, i, j, s->pair_warm[pij] ? s->pair_xm[pij] : NULL, xm, &delta, nv, xcp,
                                    &s->pair_warm[pij]);
            for (int a = 0; a < 3; a++) s->pair_xm[pij][a] = xm[a];
            if (!hit) {
                s->pair_on[pij] = 0;
                continue;
            }
            if (!s->pair_on[pij])
                for (int a = 0; a < 3; a++) s->pair_xi[pij][a] = 0.0;
            s->pair_on[pij] = 1;
            double vi[3], vj[3], Fi[3];
            point_velocity(s, i, xcp, vi);
            point_velocity(s, j, xcp, vj);
            contact_law(s, delta, nv, vi, vj, s->pair_xi[pij], h, Fi);
            double ri[3], rj[3], ti[3], tj[3], Fj[3];
            for (int a = 0; a < 3; a++) {
                ri[a] = minimg(s, a, xcp[a] - s->p[i].x[a]);
                rj[a] = minimg(s, a, xcp[a] - s->p[j].x[a]);
                Fj[a] = -Fi[a];
            }
            cross(ri, Fi, ti);
            cross(rj, Fj, tj);
            for (int a = 0; a < 3; a++) {
                s->Fc[i][a] += Fi[a]; s->Tc[i][a] += ti[a];
                s->Fc[j][a] += Fj[a]; s->Tc[j][a] += tj[a];
            }
        }
    for (int j = 0; j < np; j++)
        for (int wall = 0; wall < ORC_NWALL; wall++) {
            int ax = wall / 2, side = wall % 2;
            long wj = (long)j * ORC_NWALL + wall;
            if (s->c.periodic[ax]) { s->wall_on[wj] = 0; s->wall_warm[wj] = 0; continue; }
            double plane = side ? dim(s, ax) - 0.5 : -0.5;
            if (fabs(plane - s->p[j].x[ax]) > bounding_radius(&s->p[j], s->c.c0)) {
                s->wall_on[wj] = 0;
                s->wall_warm[wj] = 0;
                continue;
            }
            /* §2.1.4: Newton starts from the previous x_cw when this
             * potential collision (the plane within the bounding sphere)
             * already existed at the previous evaluation, in contact or
             * not, and that evaluation found a valid x_cw */
            double xcw[3], delta, nv[3], xcp[3];
            int hit = wall_geometry(s, j, wall, s->wall_warm[wj] ? s->wall_xcw[wj] : NULL, xcw, &delta, nv, xcp,
                                    &s->wall_warm[wj]);
            for (int a = 0; a < 3; a++) s->wall_xcw[wj][a] = xcw[a];
            if (!hit) { s->wall_on[wj] = 0; continue; }
            if (!s->wall_on[wj])
                for (int a = 0; a < 3; a++) s->wall_xi[wj][a] = 0.0;
            s->wall_on[wj] = 1;
            double vi[3], vw[3] = {0, 0, 0}, Fi[3], ri[3], ti[3];
            point_velocity(s, j, xcp, vi);
            contact_law(s, delta, nv, vi, vw, s->wall_xi[wj], h, Fi);
            for (int a = 0; a < 3; a++) ri[a] = minimg(s, a, xcp[a] - s->p[j].x[a]);
            cross(ri, Fi, ti);
            for (int a = 0; a < 3; a++) { s->Fc[j][a] += Fi[a]; s->Tc[j][a] += ti[a]; }
        }
}

/* Body-frame angular acceleration from Euler's equations (§2.1.1):
 * I dw_b/dt = T_b - w_b x (I w_b). */
static void euler_rhs(const orc_particle *p, const double Iinv[9], const double wb[3], const double Tb[3],
                      double out[3]) {
    double Iw[3], wIw[3], rhs[3];
    matvec(p->inertia, wb, Iw);
    cross(wb, Iw, wIw);
    for (int a = 0; a < 3; a++) rhs[a] = Tb[a] - wIw[a];
    matvec(Iinv, rhs, out);
}

/* q <- q (x) exp(h w_b / 2): rotation by the body-frame angular velocity. */
static void quat_advance(double q[4], const double wb[3], double h) {
    double th = norm(wb) * h;
    double dq[4];
    if (th > 0.0) {
        double sn = sin(0.5 * th) / norm(wb);
        dq[0] = cos(0.5 * th); dq[1] = sn * wb[0]; dq[2] = sn * wb[1]; dq[3] = sn * wb[2];
    } else {
        dq[0] = 1.0; dq[1] = dq[2] = dq[3] = 0.0;
    }
    double r[4];
    r[0] = q[0] * dq[0] - q[1] * dq[1] - q[2] * dq[2] - q[3] * dq[3];
    r[1] = q[0] * dq[1] + q[1] * dq[0] + q[2] * dq[3] - q[3] * dq[2];
    r[2] = q[0] * dq[2] - q[1] * dq[3] + q[2] * dq[0] + q[3] * dq[1];
    r[3] = q[0] * dq[3] + q[1] * dq[2] - q[2] * dq[1] + q[3] * dq[0];
    double nq = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3]);
    for (int a = 0; a < 4; a++) q[a] = r[a] / nq;
}

/* n_s DEM sub-steps with the hydrodynamic force and torque of the LBM step
 * held fixed (§2.3.4), velocity Verlet (§2.1.1) in kick-drift-kick form for
 * Eq. (1):  v += h/2 a; x += h v; [new contact forces]; v += h/2 a.  The
 * rotation follows the same pattern on Euler's equations in the body frame
 * with the orientation advanced by the half-step body angular velocity; the
 * closing half-kick is implicit in the gyroscopic term (a fixed number of
 * fixed-point sweeps) so that the rotation is second order like the
 * translation.
 * Gravity enters as the relative gravity (1 - rho_f/rho_s) g of §3.1. */
static void dem(orc_state *s) {
    int ns = s->c.n_sub;
    if (ns <= 0 || s->np == 0) return;
    double h = 1.0 / ns;
    contacts(s, 0.0);
    for (int sub = 0; sub < ns; sub++) {
        for (int j = 0; j < s->np; j++) {
            orc_particle *p = &s->p[j];
            if (p->fixed) continue;
            double gr = 1.0 - s->c.rho0 / p->density;
            double R[9], Iinv[9], wb[3], Tw[3], Tb[3], dw[3];
            for (int a = 0; a < 3; a++) {
                double Ftot = p->mass * gr * s->c.gravity[a] + s->Fh[j][a] + s->Fc[j][a];
                p->v[a] += 0.5 * h * Ftot / p->mass;
            }
            for (int a = 0; a < 3; a++) p->x[a] += h * p->v[a];
            quat_to_R(p->q, R);
            inv3(p->inertia, Iinv);
            matTvec(R, p->w, wb);
            for (int a = 0; a < 3; a++) Tw[a] = s->Th[j][a] + s->Tc[j][a];
            matTvec(R, Tw, Tb);
            euler_rhs(p, Iinv, wb, Tb, dw);
            for (int a = 0; a < 3; a++) wb[a] += 0.5 * h * dw[a];
            quat_advance(p->q, wb, h);
            quat_to_R(p->q, R);
            matvec(R, wb, p->w);
        }
        update_world_cps(s);
        contacts(s, h);
        for (int j = 0; j < s->np; j++) {
            orc_particle *p = &s->p[j];
            if (p->fixed) continue;
            double gr = 1.0 - s->c.rho0 / p->density;
            double R[9], Iinv[9], wb[3], Tw[3], Tb[3], dw[3];
            for (int a = 0; a < 3; a++) {
                double Ftot = p->mass * gr * s->c.gravity[a] + s->Fh[j][a] + s->Fc[j][a];
                p->v[a] += 0.5 * h * Ftot / p->mass;
            }
            quat_to_R(p->q, R);
            inv3(p->inertia, Iinv);
            matTvec(R, p->w, wb);
            for (int a = 0; a < 3; a++) Tw[a] = s->Th[j][a] + s->Tc[j][a];
            matTvec(R, Tw, Tb);
            /* closing half-kick evaluated at the end-of-step rate,
             * w1 = w_half + h/2 rhs(w1), by ORC_ROT_ITERS fixed-point sweeps */
            double w1[3] = {wb[0], wb[1], wb[2]};
            for (int it = 0; it < ORC_ROT_ITERS; it++) {
                euler_rhs(p, Iinv, w1, Tb, dw);
                for (int a = 0; a < 3; a++) w1[a] = wb[a] + 0.5 * h * dw[a];
            }
            matvec(R, w1, p->w);
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Mass properties: volume, centroid and inertia of {M >= c0} by sampling a
 * regular grid of spacing h at cell centres (the paper gives none; a sphere
 * of one control point has the closed form 4/3 pi K^(3/2)).  The control
 * points are shifted so that the body frame is centred on the centroid.     */
/* ------------------------------------------------------------------------- */
void orc_mass_properties(orc_particle *p, double c0, double h) {
    double B = 0.0;
    for (int k = 0; k < p->ncp; k++)
        for (int a = 0; a < 3; a++) {
            double v = fabs(p->cp[k][a]);
            if (v > B) B = v;
        }
    double Kt = 0.0;
    for (int k = 0; k < p->ncp; k++) Kt += p->K[k];
    B += sqrt(Kt / c0);
    int n = (int)ceil(B / h);
    double cnt = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
    double Sxx = 0, Syy = 0, Szz = 0, Sxy = 0, Sxz = 0, Syz = 0;
    for (int k = -n; k < n; k++)
        for (int j = -n; j < n; j++)
            for (int i = -n; i < n; i++) {
                double x = (i + 0.5) * h, y = (j + 0.5) * h, z = (k + 0.5) * h;
                double M = 0.0;
                for (int c = 0; c < p->ncp; c++) {
                    double dx = x - p->cp[c][0], dy = y - p->cp[c][1], dz = z - p->cp[c][2];
                    M += p->K[c] / (dx * dx + dy * dy + dz * dz);
                }
                if (M >= c0) {
                    cnt += 1.0;
                    sx += x; sy += y; sz += z;
                    Sxx += x * x; Syy += y * y; Szz += z * z;
                    Sxy += x * y; Sxz += x * z; Syz += y * z;
                }
            }
    double dV = h * h * h;
    double V = cnt * dV;
    double cx = sx / cnt, cy = sy / cnt, cz = sz / cnt;
    /* second moments about the centroid */
    double Cxx = Sxx / cnt - cx * cx, Cyy = Syy / cnt - cy * cy, Czz = Szz / cnt - cz * cz;
    double Cxy = Sxy / cnt - cx * cy, Cxz = Sxz / cnt - cx * cz, Cyz = Syz / cnt - cy * cz;
    double m = p->density * V;
    /* a cubic sample cell of side h adds h^2/12 per axis to each second moment */
    double cc = h * h / 12.0;
    Cxx += cc; Cyy += cc; Czz += cc;
    p->mass = m;
    p->inertia[0] = m * (Cyy + Czz); p->inertia[1] = -m * Cxy;        p->inertia[2] = -m * Cxz;
    p->inertia[3] = -m * Cxy;        p->inertia[4] = m * (Cxx + Czz); p->inertia[5] = -m * Cyz;
    p->inertia[6] = -m * Cxz;        p->inertia[7] = -m * Cyz;        p->inertia[8] = m * (Cxx + Cyy);
    double R[9], cw[3], cb[3] = {cx, cy, cz};
    quat_to_R(p->q, R);
    matvec(R, cb, cw);
    for (int k = 0; k < p->ncp; k++) {
        p->cp[k][0] -= cx; p->cp[k][1] -= cy; p->cp[k][2] -= cz;
    }
    for (int a = 0; a < 3; a++) p->x[a] += cw[a];
}

/* ------------------------------------------------------------------------- */
/* Public API.                                                                */
/* ------------------------------------------------------------------------- */
static void free_particles(orc_state *s) {
    free(s->p); free(s->cpw); free(s->Fh); free(s->Th); free(s->Fc); free(s->Tc);
    free(s->pair_on); free(s->pair_xi); free(s->pair_xm);
    free(s->wall_on); free(s->wall_warm); free(s->wall_xi); free(s->wall_xcw); free(s->pair_warm);
    s->p = NULL; s->cpw = NULL; s->Fh = s->Th = s->Fc = s->Tc = NULL;
    s->pair_on = NULL; s->pair_xi = s->pair_xm = NULL;
    s->wall_on = s->wall_warm = s->pair_warm = NULL; s->wall_xi = s->wall_xcw = NULL;
    s->np = 0;
}

orc_state *orc_create(const orc_config *c) {
    orc_state *s = (orc_state *)calloc(1, sizeof(orc_state));
    if (!s) return NULL;
    s->c = *c;
    if (setup_lattice(s, c->Q) != 0 || c->nx <= 0 || c->ny <= 0 || c->nz <= 0) {
        free(s);
        return NULL;
    }
    s->N = (long)c->nx * c->ny * c->nz;
    size_t QN = (size_t)s->Q * (size_t)s->N;
    s->f = (double *)malloc(sizeof(double) * QN);
    s->g = (double *)malloc(sizeof(double) * QN);
    s->own = (int *)malloc(sizeof(int) * (size_t)s->N);
    s->own_new = (int *)malloc(sizeof(int) * (size_t)s->N);
    s->rho = (double *)malloc(sizeof(double) * (size_t)s->N);
    s->u = (double *)malloc(sizeof(double) * 3 * (size_t)s->N);
    if (!s->f || !s->g || !s->own || !s->own_new || !s->rho || !s->u) {
        free(s->f); free(s->g); free(s->own); free(s->own_new); free(s->rho); free(s->u); free(s);
        return NULL;
    }
    for (long n = 0; n < s->N; n++) {
        s->own[n] = -1;
        s->own_new[n] = -1;
        s->rho[n] = c->rho0;
        for (int a = 0; a < 3; a++) s->u[(long)a * s->N + n] = c->u0[a];
        for (int i = 0; i < s->Q; i++) {
            double fi = feq(s, i, c->rho0, c->u0);
            s->f[(long)i * s->N + n] = fi;
            s->g[(long)i * s->N + n] = fi;
        }
    }
    return s;
}

void orc_destroy(orc_state *s) {
    if (!s) return;
    free_particles(s);
    free(s->f); free(s->g); free(s->own); free(s->own_new); free(s->rho); free(s->u);
    free(s);
}

/* Copy particles in; mass <= 0 asks for the mass properties to be computed
 * (which recentres the body frame on the centroid).  Contact history is reset. */
int orc_set_particles(orc_state *s, const orc_particle *p, int np) {
    free_particles(s);
    if (np < 0) return -1;
    s->np = np;
    size_t n1 = np > 0 ? (size_t)np : 1, n2 = n1 * n1;
    s->p = (orc_particle *)calloc(n1, sizeof(orc_particle));
    s->cpw = calloc(n1, sizeof(*s->cpw));
    s->Fh = calloc(n1, sizeof(*s->Fh)); s->Th = calloc(n1, sizeof(*s->Th));
    s->Fc = calloc(n1, sizeof(*s->Fc)); s->Tc = calloc(n1, sizeof(*s->Tc));
    s->pair_on = calloc(n2, sizeof(int));
    s->pair_xi = calloc(n2, sizeof(*s->pair_xi));
    s->pair_xm = calloc(n2, sizeof(*s->pair_xm));
    s->wall_on = calloc(n1 * ORC_NWALL, sizeof(int));
    s->wall_warm = calloc(n1 * ORC_NWALL, sizeof(int));
    s->pair_warm = calloc(n2, sizeof(int));
    s->wall_xi = calloc(n1 * ORC_NWALL, sizeof(*s->wall_xi));
    s->wall_xcw = calloc(n1 * ORC_NWALL, sizeof(*s->wall_xcw));
    for (int j = 0; j < np; j++) {
        s->p[j] = p[j];
        if (s->p[j].ncp < 1 || s->p[j].ncp > ORC_MAXCP) return -1;
        double qn = sqrt(s->p[j].q[0] * s->p[j].q[0] + s->p[j].q[1] * s->p[j].q[1] + s->p[j].q[2] * s->p[j].q[2] +
                         s->p[j].q[3] * s->p[j].q[3]);
        for (int a = 0; a < 4; a++) s->p[j].q[a] /= qn;
        if (s->p[j].mass <= 0.0) orc_mass_properties(&s->p[j], s->c.c0, s->c.mass_spacing);
    }
    update_world_cps(s);
    return 0;
}

int orc_get_particles(const orc_state *s, orc_particle *out) {
    for (int j = 0; j < s->np; j++) out[j] = s->p[j];
    return s->np;
}

/* One LBM step: classify with the current particle poses, refill the nodes
 * the particles uncovered (§2.3.3), stream + bounce back + collide with the
 * momentum exchange (§2.2, §2.3.1-2.3.2, §2.3.5), then n_s DEM sub-steps with
 * the new hydrodynamic force and torque held fixed (§2.3.4).  Reading: the
 * paper does not spell out this order; it is the standard sharp-interface
 * cycle. */
int orc_step(orc_state *s, int nsteps) {
    for (int t = 0; t < nsteps; t++) {
        update_world_cps(s);
        if (s->frozen) {
            /* flags held: the link set stays, while q follows the particles */
            memcpy(s->own_new, s->own, (size_t)s->N * sizeof(int));
        } else {
            classify(s, s->own_new);
            refill(s);
        }
        sweep(s);
        double *tmp = s->f; s->f = s->g; s->g = tmp;
        int *to = s->own; s->own = s->own_new; s->own_new = to;
        dem(s);
        update_world_cps(s);
        s->step++;
    }
    return 0;
}

/* Freeze the node flags (on = 1): classify the current particles once and
 * keep those flags for every later step, whatever the particles do; the link
 * fractions q still follow the particles.  This is the "flags frozen over
 * the window" setting of the drag gradient: a finite difference in the shape
 * then differentiates the method through q only.  on = 0 releases them. */
int orc_freeze_flags(orc_state *s, int on) {
    if (on) {
        update_world_cps(s);
        classify(s, s->own);
    }
    s->frozen = on != 0;
    return 0;
}

/* Stand-alone pieces, for the pins. */
int orc_classify(orc_state *s, int *own_out) {
    update_world_cps(s);
    classify(s, own_out);
    return 0;
}
double orc_metaball(const orc_state *s, int j, const double x[3]) { return metaball(s, j, x); }
void orc_metaball_dd(const orc_state *s, int j, const double x[3], double *M, double g[3], double H[9]) {
    metaball_dd(s, j, x, M, g, H);
}
double orc_q_linear(const orc_state *s, int j, const double xf[3], const double d[3]) {
    double xs[3] = {xf[0] + d[0], xf[1] + d[1], xf[2] + d[2]};
    return q_linear(s->c.c0, metaball(s, j, xf), metaball(s, j, xs));
}
/* The unknown population of one particle link from raw inputs (Eqs. (19)-(25),
 * or halfway bounce-back when fplus_ff is NULL). */
double orc_vibb_unknown(const orc_state *s, int i, double q, const double *fplus_f, const double *fplus_ff,
                        const double uw[3]) {
    return vibb_unknown(s, i, q, fplus_f, fplus_ff, uw);
}
void orc_lattice(const orc_state *s, int *Q, int *e, double *w, int *opp) {
    *Q = s->Q;
    for (int i = 0; i < s->Q; i++) {
        for (int a = 0; a < 3; a++) e[3 * i + a] = s->e[i][a];
        w[i] = s->wt[i];
        opp[i] = s->opp[i];
    }
}
void orc_equilibrium(const orc_state *s, double rho, const double u[3], double *out) {
    for (int i = 0; i < s->Q; i++) out[i] = feq(s, i, rho, u);
}
void orc_get_populations(const orc_state *s, double *out) {
    memcpy(out, s->f, sizeof(double) * (size_t)s->Q * (size_t)s->N);
}
void orc_set_populations(orc_state *s, const double *in) {
    memcpy(s->f, in, sizeof(double) * (size_t)s->Q * (size_t)s->N);
}
/* Geometry the stored populations are consistent with (-1 fluid, else owner). */
void orc_get_owner(const orc_state *s, int *out) { memcpy(out, s->own, sizeof(int) * (size_t)s->N); }
void orc_set_owner(orc_state *s, const int *in) { memcpy(s->own, in, sizeof(int) * (size_t)s->N); }
void orc_get_fields(const orc_state *s, double *rho, double *u) {
    memcpy(rho, s->rho, sizeof(double) * (size_t)s->N);
    memcpy(u, s->u, sizeof(double) * 3 * (size_t)s->N);
}
void orc_get_forces(const orc_state *s, double *F, double *T) {
    for (int j = 0; j < s->np; j++)
        for (int a = 0; a < 3; a++) {
            F[3 * j + a] = s->Fh[j][a];
            T[3 * j + a] = s->Th[j][a];
        }
}
/* Contact load of the current state (springs not advanced): the load the
 * next DEM step starts from.  Re-evaluating it leaves the state as the next
 * step's first evaluation would (the same geometry, an idempotent projection
 * of the springs onto the tangent plane). */
void orc_get_contact_forces(orc_state *s, double *F, double *T) {
    update_world_cps(s);
    contacts(s, 0.0);
    for (int j = 0; j < s->np; j++)
        for (int a = 0; a < 3; a++) {
            F[3 * j + a] = s->Fc[j][a];
            T[3 * j + a] = s->Tc[j][a];
        }
}
void orc_counters(const orc_state *s, long *step, int *nrefill, int *nlinks) {
    *step = s->step;
    *nrefill = s->nrefill;
    *nlinks = s->nlinks;
}
/* Smallest |M_j(x)/c0 - 1| over the nodes of every particle's search box: a
 * test input is rejected when some node lies this close to a surface. */
double orc_min_margin(orc_state *s) {
    update_world_cps(s);
    double best = INFINITY;
    for (int j = 0; j < s->np; j++) {
        const orc_particle *p = &s->p[j];
        double bound = sqrt(sumK(p) / s->c.c0) + 1.0;
        int lo[3], hi[3];
        for (int a = 0; a < 3; a++) {
            double mn = s->cpw[j][0][a], mx = s->cpw[j][0][a];
            for (int k = 1; k < p->ncp; k++) {
                if (s->cpw[j][k][a] < mn) mn = s->cpw[j][k][a];
                if (s->cpw[j][k][a] > mx) mx = s->cpw[j][k][a];
            }
            lo[a] = (int)ceil(mn - bound);
            hi[a] = (int)floor(mx + bound);
        }
        for (int zz = lo[2]; zz <= hi[2]; zz++)
            for (int yy = lo[1]; yy <= hi[1]; yy++)
                for (int xx = lo[0]; xx <= hi[0]; xx++) {
                    double pos[3] = {xx, yy, zz};
                    double M = metaball(s, j, pos);
                    double mg = fabs(M / s->c.c0 - 1.0);
                    if (mg < best) best = mg;
                }
    }
    return best;
}
