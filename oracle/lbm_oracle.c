/*
 * Plain FP64 CPU oracle for one time step of the two-component immiscible pseudopotential
 * lattice Boltzmann model with the improved solid-fluid interaction scheme of
 * Chen, Wang, Tao, Yang, Chen, "Improvement of Solid-Fluid Interaction Scheme in Lattice
 * Boltzmann Immiscible Pseudopotential Models" (arXiv 2505.22256).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark load this file's library.  It shares no code, header, table or constant with the
 * CUDA library; it is written to be read against the paper, not to be fast: every node is
 * visited with plain loops, in the order the method states its steps, in double precision.
 *
 * State convention: f[k][i][y][x] holds the post-streaming populations f_i^k(x, t) of component
 * k (0 = fluid 1 = "A", 1 = fluid 2 = "B"), i = 0..8 (D2Q9), row-major with x fastest.
 * Solid nodes hold 0 and are never updated.
 *
 * Readings of passages the paper leaves garbled or open are listed with the function that takes
 * them; the per-step order is
 *   (1) densities, Eq. 3               (2) E8 neighbourhood with second-layer copy, Sec. 2.4, Table 1
 *   (3) cohesion force, Eq. 8          (4) adhesion force, Eq. 9 with the local parameter of Eqs. 10-12
 *   (5) total force (+ body force, Sec. 3.1)
 *   (6) equilibrium velocity, Eqs. 4-5 with Guo's half-force shift
 *   (7) SRT collision with Guo forcing, Eqs. 1, 2, 6, 7
 *   (8) streaming with halfway bounce-back (Sec. 3.5), periodic wrap, open inlet/outlet (Sec. 3.3)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------------------------------
 * Configuration handed in from Python (layout mirrored there with ctypes).
 * ------------------------------------------------------------------------------------------- */
enum { BC_PERIODIC = 0, BC_WALL = 1, BC_OPEN = 2 };
enum { SCHEME_ORIGINAL = 0, SCHEME_IMPROVED = 1 };

typedef struct {
    int32_t nx, ny;
    int32_t bc_x;     /* BC_PERIODIC, BC_WALL (outside the array is solid), BC_OPEN (inlet x=0, outflow x=nx-1) */
    int32_t bc_y;     /* BC_PERIODIC or BC_WALL */
    int32_t scheme;   /* SCHEME_ORIGINAL (Eq. 9, constant G_w1) or SCHEME_IMPROVED (Eqs. 10-12) */
    int32_t nthreads; /* OpenMP threads for the node loops (each node is independent) */
    double tau[2];    /* relaxation times tau_k, Eq. 2 */
    double G;         /* G_12, Eq. 8 */
    double lambda;    /* strength coefficient lambda = G_w1 / G_w2, Sec. 2.3.2 */
    double Gw2;       /* adhesion parameter of fluid 2; the paper sets G_w2 = G_12 */
    double delta;     /* interpolation half-width delta of Eqs. 11-12 (0.8 in the paper) */
    double g[2];      /* body acceleration: F_k += rho_k g (Sec. 3.1 volume force) */
    double u_in;      /* inlet x-velocity (Sec. 3.3 velocity inlet) */
    double rho_in[2]; /* component densities imposed at the inlet */
    double wE8[5];    /* E8 weights w(|e|^2) for |e|^2 = 1, 2, 4, 5, 8 (derived in Python) */
    int32_t inlet_profile; /* 0: uniform u_in; 1: Poiseuille profile of peak u_in (Sec. 3.3) */
    int32_t second_layer;  /* what a replaced second-layer node takes from x + sign(e) (Sec. 2.4,
                              Table 1): 0 both psi and the solid switch, 1 psi only (the site keeps
                              its own solid switch in the adhesion sum of Eq. 9) */
    double u_wall[2]; /* x-velocity of the lower / upper wall of a walled y direction (Sec. 3.1 Couette) */
    int32_t adhesion_stencil; /* stencil of the adhesion sum of Eq. 9: ADHESION_E8 (the 24-node
                                 eighth-order stencil of the cohesion force, Sec. 2.4) or
                                 ADHESION_D2Q9 (Eq. 9 as printed: the D2Q9 weights w_i over the
                                 eight first-layer neighbours) */
    int32_t outlet;   /* OUTLET_COPY (entering populations copied from column nx-2) or
                         OUTLET_PRESSURE (Zou-He density condition, rho_out) at x = nx-1 */
    double rho_out[2]; /* component densities held at the outlet by OUTLET_PRESSURE */
} oracle_cfg;

enum { ADHESION_E8 = 0, ADHESION_D2Q9 = 1 };
enum { OUTLET_COPY = 0, OUTLET_PRESSURE = 1 };

/* ---------------------------------------------------------------------------------------------
 * Lattice tables.
 * D2Q9: e_0 = (0,0); e_1..e_4 = (1,0),(0,1),(-1,0),(0,-1); e_5..e_8 = (1,1),(-1,1),(-1,-1),(1,-1);
 * weights 4/9, 1/9, 1/36 and c_s^2 = 1/3 (Sec. 2.2, Eq. 6).
 * ------------------------------------------------------------------------------------------- */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double W9[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0;

/* E8 (eighth-order isotropic) 24-node stencil in the numbering of Fig. 2(a) / Table 1:
 * nodes 1-8 are the first layer (same order as the D2Q9 moving velocities), 9-16 the second-layer
 * nodes 2*e_(n-8), 17-20 and 21-24 the "knight" nodes whose first-layer partner is n-12 and n-16.
 * Index n-1 is stored. */
static const int EX[24] = {1, 0, -1, 0, 1, -1, -1, 1, 2, 0, -2, 0, 2, -2, -2, 2, 2, -2, -2, 2, 1, -1, -1, 1};
static const int EY[24] = {0, 1, 0, -1, 1, 1, -1, -1, 0, 2, 0, -2, 2, 2, -2, -2, 1, 1, -1, -1, 2, 2, -2, -2};

static int sgn(int v) { return (v > 0) - (v < 0); }

static double e8_weight(const oracle_cfg* c, int n) {
    int e2 = EX[n] * EX[n] + EY[n] * EY[n];
    switch (e2) {
        case 1: return c->wE8[0];
        case 2: return c->wE8[1];
        case 4: return c->wE8[2];
        case 5: return c->wE8[3];
        default: return c->wE8[4]; /* |e|^2 = 8 */
    }
}

/* Exposed so the tests can check the stencil numbering against Table 1. */
void oracle_e8_table(int32_t* ex, int32_t* ey) {
    for (int n = 0; n < 24; n++) { ex[n] = EX[n]; ey[n] = EY[n]; }
}

/* ---------------------------------------------------------------------------------------------
 * Equilibrium (Eq. 6) and Guo forcing term (Eq. 7), written as printed.
 * ------------------------------------------------------------------------------------------- */
void oracle_feq(double rho, double ux, double uy, double* feq) {
    for (int i = 0; i < 9; i++) {
        double eu = CX[i] * ux + CY[i] * uy;
        double uu = ux * ux + uy * uy;
        feq[i] = W9[i] * rho * (1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    }
}

/* F_i = w_i [ e_i.F / c_s^2 + (u F + F u) : (e_i e_i - c_s^2 I) / (2 c_s^4) ]  (Eq. 7). */
void oracle_guo(double ux, double uy, double Fx, double Fy, double* Fi) {
    double u[2] = {ux, uy}, F[2] = {Fx, Fy};
    for (int i = 0; i < 9; i++) {
        double e[2] = {(double)CX[i], (double)CY[i]};
        double contraction = 0.0;
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++) {
                double uF = u[a] * F[b] + F[a] * u[b];
                double ee = e[a] * e[b] - (a == b ? CS2 : 0.0);
                contraction += uF * ee;
            }
        Fi[i] = W9[i] * ((e[0] * F[0] + e[1] * F[1]) / CS2 + contraction / (2.0 * CS2 * CS2));
    }
}

/* ---------------------------------------------------------------------------------------------
 * Local adhesion parameter of the improved scheme, normalised by G_w2 (Eq. 12).
 * Reading of the garbled Eq. 12: branches {lambda; g1'; g2'; 1}, which is Eq. 11 divided by G_w2
 * with G_w1 = lambda G_w2.  The printed inequalities are kept; rho_e = -delta, which none of the
 * printed branches covers, falls to the last branch (the function is continuous there).
 * ------------------------------------------------------------------------------------------- */
double oracle_local_G(double rho_e, double lambda, double delta) {
    double s1 = 2.0 * lambda / (1.0 + lambda);
    double s2 = 2.0 * (lambda * lambda - lambda) / (delta * (1.0 + lambda));
    double s3 = (lambda - lambda * lambda) / (delta * delta * (1.0 + lambda));
    double t1 = s1;
    double t2 = 2.0 * (lambda - 1.0) / (delta * (1.0 + lambda));
    double t3 = (lambda - 1.0) / (delta * delta * (1.0 + lambda));
    if (rho_e > delta) return lambda;
    if (rho_e > 0.0) return s1 + s2 * rho_e + s3 * rho_e * rho_e;     /* delta >= rho_e > 0 */
    if (rho_e > -delta) return t1 + t2 * rho_e + t3 * rho_e * rho_e;  /* 0 >= rho_e > -delta */
    return 1.0;
}

/* ---------------------------------------------------------------------------------------------
 * Geometry helpers.
 * ------------------------------------------------------------------------------------------- */
static size_t idx(const oracle_cfg* c, int x, int y) { return (size_t)y * (size_t)c->nx + (size_t)x; }

/* Wrap (x, y) into the array along periodic directions.  Returns 0 when the site lies outside
 * the array along a non-periodic direction. */
static int wrap_site(const oracle_cfg* c, int* x, int* y) {
    if (*x < 0 || *x >= c->nx) {
        if (c->bc_x != BC_PERIODIC) return 0;
        *x = ((*x % c->nx) + c->nx) % c->nx;
    }
    if (*y < 0 || *y >= c->ny) {
        if (c->bc_y != BC_PERIODIC) return 0;
        *y = ((*y % c->ny) + c->ny) % c->ny;
    }
    return 1;
}

/* Effective pseudopotential psi~ (= rho, Sec. 1: psi_k = rho_k for immiscible fluids) and solid
 * switch s~ seen by node (x, y) along first-layer offset (dx, dy).
 * Solid site: psi~ = 0, s~ = 1 (Martys-Chen switch, Eq. 9).  A site outside the array along a wall
 * direction counts as solid.  Along an open (inlet/outlet) direction the site is clamped to the
 * boundary column. */
static void first_layer(const oracle_cfg* c, const uint8_t* solid, const double* rhoA,
                        const double* rhoB, int x, int y, int dx, int dy, double* pA, double* pB,
                        double* s) {
    int X = x + dx, Y = y + dy;
    if (c->bc_x == BC_OPEN) {
        if (X < 0) X = 0;
        if (X > c->nx - 1) X = c->nx - 1;
    }
    if (!wrap_site(c, &X, &Y) || solid[idx(c, X, Y)]) {
        *pA = 0.0; *pB = 0.0; *s = 1.0;
        return;
    }
    *pA = rhoA ? rhoA[idx(c, X, Y)] : 0.0;
    *pB = rhoB ? rhoB[idx(c, X, Y)] : 0.0;
    *s = 0.0;
}

/* Adhesion sum of Eq. 9 exactly as printed, a = sum_i w_i s(x + e_i) e_i over the eight moving
 * D2Q9 velocities with the lattice weights 1/9 (axes) and 1/36 (diagonals); s is the solid switch
 * of the first-layer site (as in first_layer(): outside a wall direction counts as solid, beyond an
 * open column is that column).  Opposite velocities are taken together, i = 1, 2, 5, 6 with opp(i). */
static void adhesion_d2q9(const oracle_cfg* c, const uint8_t* solid, int x, int y, double a[2]) {
    static const int HALF[4] = {1, 2, 5, 6};
    a[0] = 0.0;
    a[1] = 0.0;
    for (int h = 0; h < 4; h++) {
        int i = HALF[h], j = OPP[i];
        double pA, pB, si, sj;
        first_layer(c, solid, NULL, NULL, x, y, CX[i], CY[i], &pA, &pB, &si);
        first_layer(c, solid, NULL, NULL, x, y, CX[j], CY[j], &pA, &pB, &sj);
        a[0] += W9[i] * (si - sj) * CX[i];
        a[1] += W9[i] * (si - sj) * CY[i];
    }
}

/* E8 neighbourhood value for stencil node n (0-based) of fluid node (x, y).
 * Second-layer reconstruction (Sec. 2.4, Table 1): a second-layer node (|e|_inf = 2) that is not an
 * in-array fluid node takes the information of the first-layer node at x + sign(e): both psi and
 * the solid switch, or (second_layer = 1) psi alone, the site keeping its own solid switch (1 for a
 * solid site or one outside a wall direction; a site beyond an open column is that column).  (Table 1's
 * n -> n-8, n-12, n-16 is exactly sign(e) in this numbering.) */
static void e8_value(const oracle_cfg* c, const uint8_t* solid, const double* rhoA,
                     const double* rhoB, int x, int y, int n, double* pA, double* pB, double* s) {
    int ex = EX[n], ey = EY[n];
    int ring2 = (abs(ex) == 2 || abs(ey) == 2);
    if (!ring2) {
        first_layer(c, solid, rhoA, rhoB, x, y, ex, ey, pA, pB, s);
        return;
    }
    int X = x + ex, Y = y + ey;
    if (wrap_site(c, &X, &Y) && !solid[idx(c, X, Y)]) {
        *pA = rhoA[idx(c, X, Y)];
        *pB = rhoB[idx(c, X, Y)];
        *s = 0.0;
        return;
    }
    first_layer(c, solid, rhoA, rhoB, x, y, sgn(ex), sgn(ey), pA, pB, s);
    if (c->second_layer == 1) { /* the site's own switch (clamped along an open axis, as above) */
        double qA, qB;
        first_layer(c, solid, rhoA, rhoB, x, y, ex, ey, &qA, &qB, s);
    }
}

/* Is stencil node n of (x, y) taken from somewhere other than x + e?  (second layer only) */
static int substituted(const oracle_cfg* c, const uint8_t* solid, int x, int y, int n) {
    int ex = EX[n], ey = EY[n];
    if (!(abs(ex) == 2 || abs(ey) == 2)) return 0;
    int X = x + ex, Y = y + ey;
    return !(wrap_site(c, &X, &Y) && !solid[idx(c, X, Y)]);
}

/* Wall list: fluid nodes whose 24-node stencil reaches a non-fluid site (solid, or outside the
 * array along a non-periodic direction), in increasing node index y*nx + x.  Per entry: the
 * substitution mask (bit n set when stencil node n+1 is a second-layer node replaced by its
 * first-layer partner), the effective solid mask (bit n = s~ of stencil node n+1 when that node
 * enters the adhesion sum: all 24 on the E8 stencil, the first layer n < 8 for ADHESION_D2Q9) and
 * the static adhesion vector a(x) = sum_n w(|e_n|^2) s~_n e_n (ADHESION_D2Q9: adhesion_d2q9).
 * Returns the number of entries; arrays may be NULL to count only. */
int64_t oracle_wall_list(const oracle_cfg* c, const uint8_t* solid, int32_t* node, uint32_t* subst,
                         uint32_t* seff, double* ax, double* ay) {
    int64_t count = 0;
    double* zero = (double*)calloc((size_t)c->nx * (size_t)c->ny, sizeof(double));
    if (!zero) return -1;
    for (int y = 0; y < c->ny; y++)
        for (int x = 0; x < c->nx; x++) {
            if (solid[idx(c, x, y)]) continue;
            int touches = 0;
            for (int n = 0; n < 24 && !touches; n++) {
                int X = x + EX[n], Y = y + EY[n];
                if (!wrap_site(c, &X, &Y) || solid[idx(c, X, Y)]) touches = 1;
            }
            if (!touches) continue;
            uint32_t sm = 0, em = 0;
            double a[2] = {0.0, 0.0};
            /* pair (e, -e) first, as in the force sums */
            for (int n = 0; n < 24; n++) {
                double pA, pB, s;
                e8_value(c, solid, zero, zero, x, y, n, &pA, &pB, &s);
                if (substituted(c, solid, x, y, n)) sm |= 1u << n;
                /* the printed Eq. 9 sums the first layer only */
                if (s != 0.0 && (c->adhesion_stencil != ADHESION_D2Q9 || n < 8)) em |= 1u << n;
            }
            for (int p = 0; p < 12; p++) {
                int n = (p / 2) * 4 + (p % 2), m = n + 2; /* pairs (1,3),(2,4),(5,7),(6,8),... */
                double w = e8_weight(c, n);
                double sn = (em >> n) & 1u, sm2 = (em >> m) & 1u;
                a[0] += w * (sn - sm2) * EX[n];
                a[1] += w * (sn - sm2) * EY[n];
            }
            if (c->adhesion_stencil == ADHESION_D2Q9) adhesion_d2q9(c, solid, x, y, a);
            if (node) {
                node[count] = (int32_t)idx(c, x, y);
                subst[count] = sm;
                seff[count] = em;
                ax[count] = a[0];
                ay[count] = a[1];
            }
            count++;
        }
    free(zero);
    return count;
}

static void open_boundaries(const oracle_cfg* c, const uint8_t* solid, const double* fstar, double* f);

/* ---------------------------------------------------------------------------------------------
 * Initial state: f = f^eq(rho_k, u = 0) at fluid nodes, 0 at solid nodes.
 * ------------------------------------------------------------------------------------------- */
void oracle_init(const oracle_cfg* c, const uint8_t* solid, const double* rhoA0, const double* rhoB0,
                 double* f) {
    size_t N = (size_t)c->nx * (size_t)c->ny;
    for (size_t s = 0; s < N; s++) {
        double fe[9];
        for (int k = 0; k < 2; k++) {
            const double* r0 = k == 0 ? rhoA0 : rhoB0;
            oracle_feq(solid[s] ? 0.0 : r0[s], 0.0, 0.0, fe);
            for (int i = 0; i < 9; i++) f[((size_t)k * 9 + i) * N + s] = solid[s] ? 0.0 : fe[i];
        }
    }
    /* With open boundaries the entering populations of the boundary columns are, in every
     * post-streaming state, the ones the boundary rule gives -- the initial state included. */
    open_boundaries(c, solid, f, f);
}

/* Step (1): component densities rho_k = sum_i f_i^k (Eq. 3); 0 at solid nodes. */
static void densities(const oracle_cfg* c, const uint8_t* solid, const double* f, double* rhoA,
                      double* rhoB) {
    size_t N = (size_t)c->nx * (size_t)c->ny;
#pragma omp parallel for num_threads(c->nthreads) schedule(static)
    for (long long s = 0; s < (long long)N; s++) {
        double r[2] = {0.0, 0.0};
        if (!solid[s])
            for (int k = 0; k < 2; k++)
                for (int i = 0; i < 9; i++) r[k] += f[((size_t)k * 9 + i) * N + (size_t)s];
        rhoA[s] = r[0];
        rhoB[s] = r[1];
    }
}

/* Steps (2)-(6) at one fluid node: forces on both components and the equilibrium velocity. */
static void node_forces(const oracle_cfg* c, const uint8_t* solid, const double* f,
                        const double* rhoA, const double* rhoB, int x, int y, double FA[2],
                        double FB[2], double u[2]) {
    size_t N = (size_t)c->nx * (size_t)c->ny, s0 = idx(c, x, y);
    double rA = rhoA[s0], rB = rhoB[s0];

    /* (2) stencil values */
    double pA[24], pB[24], sw[24];
    for (int n = 0; n < 24; n++) e8_value(c, solid, rhoA, rhoB, x, y, n, &pA[n], &pB[n], &sw[n]);

    /* (3) cohesion, Eq. 8 read as F_k = -G_12 psi_k(x) sum_n w(|e_n|^2) psi_kbar(x + e_n) e_n
     *     (the force on one component comes from the other; E8 weights).  Symmetric pairs
     *     (e, -e) are summed first.
     * (4) adhesion, Eq. 9: F_k,ads = -G_w,k rho_k(x) a(x), with a(x) = sum_n w s~_n e_n on the same
     *     stencil, or (adhesion_stencil = ADHESION_D2Q9) the printed first-neighbour sum with the
     *     D2Q9 weights (adhesion_d2q9). */
    double gA[2] = {0.0, 0.0}, gB[2] = {0.0, 0.0}, a[2] = {0.0, 0.0};
    for (int p = 0; p < 12; p++) {
        int n = (p / 2) * 4 + (p % 2), m = n + 2;
        double w = e8_weight(c, n);
        double dA = pA[n] - pA[m], dB = pB[n] - pB[m], ds = sw[n] - sw[m];
        gA[0] += w * dA * EX[n]; gA[1] += w * dA * EY[n];
        gB[0] += w * dB * EX[n]; gB[1] += w * dB * EY[n];
        a[0] += w * ds * EX[n]; a[1] += w * ds * EY[n];
    }
    if (c->adhesion_stencil == ADHESION_D2Q9) adhesion_d2q9(c, solid, x, y, a);
    double GwA;
    if (c->scheme == SCHEME_IMPROVED) {
        double rho_e = (rA - rB) / (rA + rB);                 /* Eq. 10 */
        GwA = c->Gw2 * oracle_local_G(rho_e, c->lambda, c->delta); /* Eq. 12 */
    } else {
        GwA = c->lambda * c->Gw2;                               /* constant G_w1 (Eq. 9) */
    }
    double GwB = c->Gw2;
    for (int d = 0; d < 2; d++) {
        double FinA = -c->G * rA * gB[d];
        double FinB = -c->G * rB * gA[d];
        double FadsA = -GwA * rA * a[d];
        double FadsB = -GwB * rB * a[d];
        /* (5) total force with body force */
        FA[d] = FinA + FadsA + rA * c->g[d];
        FB[d] = FinB + FadsB + rB * c->g[d];
    }

    /* (6) equilibrium velocity: (sum_k sum_i f e + F_total / 2) / sum_k rho_k (Eqs. 4-5, Guo shift) */
    double mom[2] = {0.0, 0.0};
    for (int k = 0; k < 2; k++)
        for (int i = 0; i < 9; i++) {
            double fi = f[((size_t)k * 9 + i) * N + s0];
            mom[0] += fi * CX[i];
            mom[1] += fi * CY[i];
        }
    for (int d = 0; d < 2; d++) u[d] = (mom[d] + 0.5 * (FA[d] + FB[d])) / (rA + rB);
}

/* Steps (1)-(7): post-collision populations fstar from post-streaming f. */
int oracle_collide(const oracle_cfg* c, const uint8_t* solid, const double* f, double* fstar) {
    size_t N = (size_t)c->nx * (size_t)c->ny;
    double* rhoA = (double*)malloc(N * sizeof(double));
    double* rhoB = (double*)malloc(N * sizeof(double));
    if (!rhoA || !rhoB) { free(rhoA); free(rhoB); return -1; }
    densities(c, solid, f, rhoA, rhoB);
#pragma omp parallel for num_threads(c->nthreads) schedule(static)
    for (int y = 0; y < c->ny; y++)
        for (int x = 0; x < c->nx; x++) {
            size_t s0 = idx(c, x, y);
            if (solid[s0]) {
                for (int q = 0; q < 18; q++) fstar[(size_t)q * N + s0] = 0.0;
                continue;
            }
            double FA[2], FB[2], u[2];
            node_forces(c, solid, f, rhoA, rhoB, x, y, FA, FB, u);
            /* (7) Eq. 1 with Eq. 2: f* = f + (f^eq - f)/tau + (1 - 1/(2 tau)) F_i */
            for (int k = 0; k < 2; k++) {
                double rho = k == 0 ? rhoA[s0] : rhoB[s0];
                const double* F = k == 0 ? FA : FB;
                double fe[9], Fi[9];
                oracle_feq(rho, u[0], u[1], fe);
                oracle_guo(u[0], u[1], F[0], F[1], Fi);
                double tau = c->tau[k];
                for (int i = 0; i < 9; i++) {
                    size_t q = ((size_t)k * 9 + i) * N + s0;
                    fstar[q] = f[q] + (fe[i] - f[q]) / tau + (1.0 - 1.0 / (2.0 * tau)) * Fi[i];
                }
            }
        }
    free(rhoA);
    free(rhoB);
    return 0;
}

/* Inlet velocity of row y (Sec. 3.3).  Uniform: u_in.  Poiseuille: u_in 4 s (H - s) / H^2 with s the
 * distance from the lower wall, the walls being the halfway bounce-back planes below row 0 and above
 * row ny-1 (s = y + 1/2, H = ny), so u_in is the peak of the profile. */
static double inlet_velocity(const oracle_cfg* c, int y) {
    if (!c->inlet_profile) return c->u_in;
    double s = y + 0.5, H = (double)c->ny;
    return c->u_in * 4.0 * s * (H - s) / (H * H);
}

/* Open x boundaries (Sec. 3.3), applied to a post-streaming state f whose pre-streaming state was
 * fstar.  Populations entering through x = 0 are given by non-equilibrium bounce-back about
 * f^eq(rho_in,k, (u(y), 0)) (the reading of the two-component Zou-He inlet; u(y) from
 * inlet_velocity); populations entering through x = nx-1 are copied from column nx-2 (outflow), or
 * bounced back if that node is solid.
 * Pressure outlet (outlet = OUTLET_PRESSURE): per component the Zou-He density condition.  The three
 * populations entering through x = nx-1 (e_3, e_6, e_7) are those that give the node the density
 * rho_out[k] and no momentum along y, with non-equilibrium bounce-back along x: the first two
 * conditions leave rho u_x = f0 + f2 + f4 + 2 (f1 + f5 + f8) - rho_out, and then
 * f3 = f1 - (2/3) rho u_x, f7 = f5 + (f2 - f4)/2 - rho u_x / 6, f6 = f8 - (f2 - f4)/2 - rho u_x / 6. */
static void open_boundaries(const oracle_cfg* c, const uint8_t* solid, const double* fstar, double* f) {
    size_t N = (size_t)c->nx * (size_t)c->ny;
    if (c->bc_x != BC_OPEN) return;
    {
        for (int y = 0; y < c->ny; y++) {
            /* inlet, x = 0 */
            size_t s0 = idx(c, 0, y);
            if (!solid[s0])
                for (int k = 0; k < 2; k++) {
                    double fe[9];
                    oracle_feq(c->rho_in[k], inlet_velocity(c, y), 0.0, fe);
                    for (int i = 0; i < 9; i++)
                        if (CX[i] > 0) {
                            double fo = f[((size_t)k * 9 + OPP[i]) * N + s0];
                            f[((size_t)k * 9 + i) * N + s0] = fe[i] + (fo - fe[OPP[i]]);
                        }
                }
            /* outlet, x = nx-1 */
            size_t s1 = idx(c, c->nx - 1, y), s2 = idx(c, c->nx - 2, y);
            if (!solid[s1] && c->outlet == OUTLET_PRESSURE) {
                for (int k = 0; k < 2; k++) {
                    double* g = f + (size_t)k * 9 * N + s1; /* g[i * N] = f_i^k at the node */
                    double known = g[0] + g[2 * N] + g[4 * N] + 2.0 * (g[1 * N] + g[5 * N] + g[8 * N]);
                    double rho_ux = known - c->rho_out[k];
                    double dy = g[2 * N] - g[4 * N];
                    g[3 * N] = g[1 * N] - 2.0 / 3.0 * rho_ux;
                    g[7 * N] = g[5 * N] + 0.5 * dy - rho_ux / 6.0;
                    g[6 * N] = g[8 * N] - 0.5 * dy - rho_ux / 6.0;
                }
            } else if (!solid[s1])
                for (int k = 0; k < 2; k++)
                    for (int i = 0; i < 9; i++)
                        if (CX[i] < 0) {
                            size_t q = ((size_t)k * 9 + i) * N;
                            f[q + s1] = !solid[s2] ? f[q + s2]
                                                   : fstar[((size_t)k * 9 + OPP[i]) * N + s1];
                        }
        }
    }
}

/* Step (8): streaming with halfway bounce-back.
 * f_i(x, t+1) = f*_i(x - e_i) when x - e_i is a fluid node (periodic wrap), otherwise
 * f*_{opp(i)}(x) (halfway bounce-back, Sec. 3.5: the wall sits half a link from the fluid node).
 * A link that crosses a walled y edge of the array meets the lower (y < 0) or upper (y >= ny)
 * wall, which slides along x at u_wall (Sec. 3.1, Couette flow): the reflected population then
 * carries the wall's momentum, f_i = f*_opp(i) + 2 w_i rho_k (e_i . u_w) / c_s^2, with rho_k the
 * node's density sum_j f*_j(x) (the collision conserves it).
 * Open x boundaries: see open_boundaries(). */
int oracle_stream(const oracle_cfg* c, const uint8_t* solid, const double* fstar, double* f) {
    size_t N = (size_t)c->nx * (size_t)c->ny;
#pragma omp parallel for num_threads(c->nthreads) schedule(static)
    for (int y = 0; y < c->ny; y++)
        for (int x = 0; x < c->nx; x++) {
            size_t s0 = idx(c, x, y);
            for (int k = 0; k < 2; k++)
                for (int i = 0; i < 9; i++) {
                    size_t q = ((size_t)k * 9 + i) * N + s0;
                    if (solid[s0]) { f[q] = 0.0; continue; }
                    int X = x - CX[i], Y = y - CY[i];
                    if (c->bc_x == BC_OPEN && (X < 0 || X >= c->nx)) {
                        f[q] = NAN; /* unknown: set by the boundary rule below */
                        continue;
                    }
                    int Yraw = Y;
                    if (wrap_site(c, &X, &Y) && !solid[idx(c, X, Y)])
                        f[q] = fstar[((size_t)k * 9 + i) * N + idx(c, X, Y)];
                    else {
                        f[q] = fstar[((size_t)k * 9 + OPP[i]) * N + s0];
                        if (c->bc_y == BC_WALL && (Yraw < 0 || Yraw >= c->ny)) {
                            double uw = Yraw < 0 ? c->u_wall[0] : c->u_wall[1];
                            if (uw != 0.0) {
                                double rho = 0.0;
                                for (int j = 0; j < 9; j++) rho += fstar[((size_t)k * 9 + j) * N + s0];
                                f[q] += 6.0 * W9[i] * rho * CX[i] * uw;
                            }
                        }
                    }
                }
        }
    open_boundaries(c, solid, fstar, f);
    return 0;
}

/* n full time steps in place on f (scratch of the same size supplied by the caller). */
int oracle_run(const oracle_cfg* c, const uint8_t* solid, double* f, double* scratch, int64_t nsteps) {
    for (int64_t t = 0; t < nsteps; t++) {
        if (oracle_collide(c, solid, f, scratch)) return -1;
        if (oracle_stream(c, solid, scratch, f)) return -1;
    }
    return 0;
}

/* Macroscopic output fields at the current state: rho_A, rho_B (Eq. 3) and the equilibrium
 * velocity of step (6) (0 at solid nodes). */
int oracle_fields(const oracle_cfg* c, const uint8_t* solid, const double* f, double* rhoA,
                  double* rhoB, double* ux, double* uy) {
    densities(c, solid, f, rhoA, rhoB);
#pragma omp parallel for num_threads(c->nthreads) schedule(static)
    for (int y = 0; y < c->ny; y++)
        for (int x = 0; x < c->nx; x++) {
            size_t s0 = idx(c, x, y);
            if (solid[s0]) { ux[s0] = 0.0; uy[s0] = 0.0; continue; }
            double FA[2], FB[2], u[2];
            node_forces(c, solid, f, rhoA, rhoB, x, y, FA, FB, u);
            ux[s0] = u[0];
            uy[s0] = u[1];
        }
    return 0;
}

/* Forces on both components at every fluid node (0 at solid nodes), for the force pins. */
int oracle_forces(const oracle_cfg* c, const uint8_t* solid, const double* f, double* FAx,
                  double* FAy, double* FBx, double* FBy) {
    size_t N = (size_t)c->nx * (size_t)c->ny;
    double* rhoA = (double*)malloc(N * sizeof(double));
    double* rhoB = (double*)malloc(N * sizeof(double));
    if (!rhoA || !rhoB) { free(rhoA); free(rhoB); return -1; }
    densities(c, solid, f, rhoA, rhoB);
    for (int y = 0; y < c->ny; y++)
        for (int x = 0; x < c->nx; x++) {
            size_t s0 = idx(c, x, y);
            double FA[2] = {0, 0}, FB[2] = {0, 0}, u[2];
            if (!solid[s0]) node_forces(c, solid, f, rhoA, rhoB, x, y, FA, FB, u);
            FAx[s0] = FA[0]; FAy[s0] = FA[1]; FBx[s0] = FB[0]; FBy[s0] = FB[1];
        }
    free(rhoA);
    free(rhoB);
    return 0;
}
