/*
 * Plain FP64 CPU oracle for one time step of the three-dimensional form of the two-component
 * immiscible pseudopotential LBM with the improved solid-fluid interaction scheme (arXiv
 * 2505.22256, Sec. 3.5: contact angles on a spherical surface).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark load this file's library.  It shares no code, header, table or constant with the
 * CUDA library; it is written to be read against the paper, with plain loops over the nodes in
 * the order the method states its steps, in double precision.
 *
 * The paper gives the 3-D case only by its geometry and states that the physical parameters are
 * those of the 2-D tests.  Readings taken here (each the direct 3-D form of the 2-D step):
 *   - velocities D3Q19: e_0 = 0; 1..6 the axis unit vectors (+x, -x, +y, -y, +z, -z); 7..18 the
 *     twelve (+-1, +-1, 0)-type vectors, opposite vectors adjacent; weights 1/3, 1/18, 1/36,
 *     c_s^2 = 1/3;
 *   - gradient stencil: the 92 offsets with |e|_inf <= 2 and |e|^2 in {1, 2, 3, 4, 5, 6, 8}, with
 *     the weights w(|e|^2) of eighth-order isotropy (derived in Python by an exact rational solve
 *     and passed in);
 *   - second-layer reconstruction (Sec. 2.4, Table 1 in 2-D): a second-layer site x+e
 *     (|e|_inf = 2) that is not fluid takes the information of x + sign(e) componentwise;
 *   - adhesion sum of Eq. 9 on the same 92 offsets, or (adhesion_stencil = 1) as printed, with the
 *     D3Q19 weights over the 18 first-layer neighbours (the 3-D form of the 2-D option);
 *   - boundaries: periodic in x, y and z (the paper's case); solid nodes from the mask.
 *
 * State convention: f[k][i][z][y][x], k = 0 ("A") or 1 ("B"), i = 0..18, x fastest.  Solid nodes
 * hold 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { SCHEME3_ORIGINAL = 0, SCHEME3_IMPROVED = 1 };

typedef struct {
    int32_t nx, ny, nz;
    int32_t scheme;   /* original (Eq. 9, constant G_w1) or improved (Eqs. 10-12) */
    int32_t nthreads;
    int32_t second_layer; /* 0: a replaced second-layer site takes psi and the solid switch of
                             x + sign(e); 1: psi only, the (solid) site keeping s = 1 */
    int32_t adhesion_stencil; /* 0: the adhesion sum of Eq. 9 on the 92-offset stencil of the
                                 cohesion force; 1: Eq. 9 as printed, in 3-D: the D3Q19 weights
                                 w_i over the 18 first-layer neighbours */
    int32_t pad_;
    double tau[2];    /* Eq. 2 */
    double G;         /* Eq. 8 */
    double lambda;    /* G_w1 / G_w2 */
    double Gw2;
    double delta;     /* Eqs. 11-12 */
    double g[3];      /* body acceleration */
    double w[7];      /* stencil weights for |e|^2 = 1, 2, 3, 4, 5, 6, 8 */
} oracle3_cfg;

static const int C3X[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int C3Y[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int C3Z[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
static const double W19[19] = {1.0 / 3.0,  1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
                               1.0 / 18.0, 1.0 / 18.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
                               1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
                               1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

static int opp19(int i) { return i == 0 ? 0 : (i % 2 ? i + 1 : i - 1); }

static size_t nodes(const oracle3_cfg* c) { return (size_t)c->nx * (size_t)c->ny * (size_t)c->nz; }

static size_t id3(const oracle3_cfg* c, int x, int y, int z) {
    x = ((x % c->nx) + c->nx) % c->nx;
    y = ((y % c->ny) + c->ny) % c->ny;
    z = ((z % c->nz) + c->nz) % c->nz;
    return ((size_t)z * (size_t)c->ny + (size_t)y) * (size_t)c->nx + (size_t)x;
}

static int sgn(int v) { return (v > 0) - (v < 0); }

/* stencil weight of offset (ex, ey, ez); 0 outside the 92-offset stencil */
static double weight3(const oracle3_cfg* c, int ex, int ey, int ez) {
    switch (ex * ex + ey * ey + ez * ez) {
        case 1: return c->w[0];
        case 2: return c->w[1];
        case 3: return c->w[2];
        case 4: return c->w[3];
        case 5: return c->w[4];
        case 6: return c->w[5];
        case 8: return c->w[6];
        default: return 0.0;
    }
}

/* Eq. 12, as in the 2-D oracle: G_w1(x) / G_w2 as a function of rho^e */
static double local_G3(double rho_e, double lambda, double delta) {
    double s1 = 2.0 * lambda / (1.0 + lambda);
    double s2 = 2.0 * (lambda * lambda - lambda) / (delta * (1.0 + lambda));
    double s3 = (lambda - lambda * lambda) / (delta * delta * (1.0 + lambda));
    double t2 = 2.0 * (lambda - 1.0) / (delta * (1.0 + lambda));
    double t3 = (lambda - 1.0) / (delta * delta * (1.0 + lambda));
    if (rho_e > delta) return lambda;
    if (rho_e > 0.0) return s1 + s2 * rho_e + s3 * rho_e * rho_e;
    if (rho_e > -delta) return s1 + t2 * rho_e + t3 * rho_e * rho_e;
    return 1.0;
}

/* Eq. 6 in 3-D */
void oracle3_feq(double rho, double ux, double uy, double uz, double* fe) {
    double usq = ux * ux + uy * uy + uz * uz;
    for (int i = 0; i < 19; i++) {
        double eu = C3X[i] * ux + C3Y[i] * uy + C3Z[i] * uz;
        fe[i] = W19[i] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * usq);
    }
}

/* Eq. 7 (Guo): F_i = w_i [3 (e_i - u) . F + 9 (e_i . u)(e_i . F)] */
void oracle3_guo(double ux, double uy, double uz, double Fx, double Fy, double Fz, double* Fi) {
    for (int i = 0; i < 19; i++) {
        double eu = C3X[i] * ux + C3Y[i] * uy + C3Z[i] * uz;
        double eF = C3X[i] * Fx + C3Y[i] * Fy + C3Z[i] * Fz;
        double emuF = (C3X[i] - ux) * Fx + (C3Y[i] - uy) * Fy + (C3Z[i] - uz) * Fz;
        Fi[i] = W19[i] * (3.0 * emuF + 9.0 * eu * eF);
    }
}

static void densities3(const oracle3_cfg* c, const uint8_t* solid, const double* f, double* rA, double* rB) {
    size_t N = nodes(c);
#pragma omp parallel for num_threads(c->nthreads) schedule(static)
    for (long long s = 0; s < (long long)N; s++) {
        double r[2] = {0.0, 0.0};
        if (!solid[s])
            for (int k = 0; k < 2; k++)
                for (int i = 0; i < 19; i++) r[k] += f[((size_t)k * 19 + i) * N + (size_t)s];
        rA[s] = r[0];
        rB[s] = r[1];
    }
}

/* Steps (2)-(6) at one fluid node (x, y, z): the stencil sums with second-layer reconstruction,
 * cohesion (Eq. 8), adhesion (Eq. 9 with Eqs. 10-12), body force, and the velocity of Eq. 5 with
 * Guo's half-force shift. */
static void node_forces3(const oracle3_cfg* c, const uint8_t* solid, const double* f, const double* rA,
                         const double* rB, int x, int y, int z, double FA[3], double FB[3], double u[3]) {
    size_t N = nodes(c), s0 = id3(c, x, y, z);
    double gA[3] = {0, 0, 0}, gB[3] = {0, 0, 0}, a[3] = {0, 0, 0};
    for (int ez = -2; ez <= 2; ez++)
        for (int ey = -2; ey <= 2; ey++)
            for (int ex = -2; ex <= 2; ex++) {
                double w = weight3(c, ex, ey, ez);
                if (w == 0.0) continue;
                int sx = ex, sy = ey, sz = ez;
                int second = abs(ex) == 2 || abs(ey) == 2 || abs(ez) == 2;
                size_t s = id3(c, x + sx, y + sy, z + sz);
                int own_solid = solid[s] != 0;
                if (second && solid[s]) {  /* second-layer site not fluid: first-layer partner */
                    sx = sgn(ex);
                    sy = sgn(ey);
                    sz = sgn(ez);
                    s = id3(c, x + sx, y + sy, z + sz);
                }
                double pA = solid[s] ? 0.0 : rA[s], pB = solid[s] ? 0.0 : rB[s];
                double sw = (solid[s] || (c->second_layer == 1 && own_solid)) ? 1.0 : 0.0;
                gA[0] += w * pA * ex; gA[1] += w * pA * ey; gA[2] += w * pA * ez;
                gB[0] += w * pB * ex; gB[1] += w * pB * ey; gB[2] += w * pB * ez;
                a[0] += w * sw * ex; a[1] += w * sw * ey; a[2] += w * sw * ez;
            }
    if (c->adhesion_stencil == 1) { /* a = sum_i w_i s(x + e_i) e_i over the D3Q19 velocities */
        a[0] = a[1] = a[2] = 0.0;
        for (int i = 1; i < 19; i++) {
            double sw = solid[id3(c, x + C3X[i], y + C3Y[i], z + C3Z[i])] ? 1.0 : 0.0;
            a[0] += W19[i] * sw * C3X[i];
            a[1] += W19[i] * sw * C3Y[i];
            a[2] += W19[i] * sw * C3Z[i];
        }
    }
    double ra = rA[s0], rb = rB[s0];
    double GwA = c->scheme == SCHEME3_IMPROVED ? c->Gw2 * local_G3((ra - rb) / (ra + rb), c->lambda, c->delta)
                                               : c->lambda * c->Gw2;
    for (int d = 0; d < 3; d++) {
        FA[d] = -c->G * ra * gB[d] - GwA * ra * a[d] + ra * c->g[d];
        FB[d] = -c->G * rb * gA[d] - c->Gw2 * rb * a[d] + rb * c->g[d];
    }
    double mom[3] = {0, 0, 0};
    for (int k = 0; k < 2; k++)
        for (int i = 0; i < 19; i++) {
            double fi = f[((size_t)k * 19 + i) * N + s0];
            mom[0] += fi * C3X[i];
            mom[1] += fi * C3Y[i];
            mom[2] += fi * C3Z[i];
        }
    for (int d = 0; d < 3; d++) u[d] = (mom[d] + 0.5 * (FA[d] + FB[d])) / (ra + rb);
}

/* Forces and velocity at every node (zero at solid nodes): out[0..2] FA, [3..5] FB, [6..8] u,
 * each [N]. */
int oracle3_forces(const oracle3_cfg* c, const uint8_t* solid, const double* f, double* out) {
    size_t N = nodes(c);
    double* rA = (double*)malloc(N * sizeof(double));
    double* rB = (double*)malloc(N * sizeof(double));
    if (!rA || !rB) { free(rA); free(rB); return -1; }
    densities3(c, solid, f, rA, rB);
#pragma omp parallel for num_threads(c->nthreads) schedule(static)
    for (int z = 0; z < c->nz; z++)
        for (int y = 0; y < c->ny; y++)
            for (int x = 0; x < c->nx; x++) {
                size_t s = id3(c, x, y, z);
                double FA[3] = {0, 0, 0}, FB[3] = {0, 0, 0}, u[3] = {0, 0, 0};
                if (!solid[s]) node_forces3(c, solid, f, rA, rB, x, y, z, FA, FB, u);
                for (int d = 0; d < 3; d++) {
                    out[(size_t)d * N + s] = FA[d];
                    out[(size_t)(3 + d) * N + s] = FB[d];
                    out[(size_t)(6 + d) * N + s] = u[d];
                }
            }
    free(rA);
    free(rB);
    return 0;
}

/* Collision (Eqs. 1, 2, 6, 7): post-collision fstar from post-streaming f. */
int oracle3_collide(const oracle3_cfg* c, const uint8_t* solid, const double* f, double* fstar) {
    size_t N = nodes(c);
    double* rA = (double*)malloc(N * sizeof(double));
    double* rB = (double*)malloc(N * sizeof(double));
    if (!rA || !rB) { free(rA); free(rB); return -1; }
    densities3(c, solid, f, rA, rB);
#pragma omp parallel for num_threads(c->nthreads) schedule(static)
    for (int z = 0; z < c->nz; z++)
        for (int y = 0; y < c->ny; y++)
            for (int x = 0; x < c->nx; x++) {
                size_t s0 = id3(c, x, y, z);
                if (solid[s0]) {
                    for (int q = 0; q < 38; q++) fstar[(size_t)q * N + s0] = 0.0;
                    continue;
                }
                double FA[3], FB[3], u[3];
                node_forces3(c, solid, f, rA, rB, x, y, z, FA, FB, u);
                for (int k = 0; k < 2; k++) {
                    double rho = k == 0 ? rA[s0] : rB[s0];
                    const double* F = k == 0 ? FA : FB;
                    double fe[19], Fi[19];
                    oracle3_feq(rho, u[0], u[1], u[2], fe);
                    oracle3_guo(u[0], u[1], u[2], F[0], F[1], F[2], Fi);
                    double tau = c->tau[k];
                    for (int i = 0; i < 19; i++) {
                        size_t q = ((size_t)k * 19 + i) * N + s0;
                        fstar[q] = f[q] + (fe[i] - f[q]) / tau + (1.0 - 1.0 / (2.0 * tau)) * Fi[i];
                    }
                }
            }
    free(rA);
    free(rB);
    return 0;
}

/* Streaming with halfway bounce-back (Sec. 3.5): f_i(x) = f*_i(x - e_i) when x - e_i is fluid
 * (periodic wrap), otherwise f*_opp(i)(x). */
int oracle3_stream(const oracle3_cfg* c, const uint8_t* solid, const double* fstar, double* f) {
    size_t N = nodes(c);
#pragma omp parallel for num_threads(c->nthreads) schedule(static)
    for (int z = 0; z < c->nz; z++)
        for (int y = 0; y < c->ny; y++)
            for (int x = 0; x < c->nx; x++) {
                size_t s0 = id3(c, x, y, z);
                for (int k = 0; k < 2; k++)
                    for (int i = 0; i < 19; i++) {
                        size_t q = ((size_t)k * 19 + i) * N + s0;
                        if (solid[s0]) { f[q] = 0.0; continue; }
                        size_t sn = id3(c, x - C3X[i], y - C3Y[i], z - C3Z[i]);
                        f[q] = !solid[sn] ? fstar[((size_t)k * 19 + i) * N + sn]
                                          : fstar[((size_t)k * 19 + opp19(i)) * N + s0];
                    }
            }
    return 0;
}

/* n time steps in place on f. */
int oracle3_run(const oracle3_cfg* c, const uint8_t* solid, double* f, int n) {
    size_t N = nodes(c);
    double* fs = (double*)malloc(38 * N * sizeof(double));
    if (!fs) return -1;
    for (int t = 0; t < n; t++) {
        if (oracle3_collide(c, solid, f, fs)) { free(fs); return -1; }
        oracle3_stream(c, solid, fs, f);
    }
    free(fs);
    return 0;
}

/* Densities and the velocity of Eq. 5 at every node: out [5][N] = rho_A, rho_B, ux, uy, uz. */
int oracle3_fields(const oracle3_cfg* c, const uint8_t* solid, const double* f, double* out) {
    size_t N = nodes(c);
    double* fr = (double*)malloc(9 * N * sizeof(double));
    if (!fr) return -1;
    if (oracle3_forces(c, solid, f, fr)) { free(fr); return -1; }
    densities3(c, solid, f, out, out + N);
    memcpy(out + 2 * N, fr + 6 * N, 3 * N * sizeof(double));
    free(fr);
    return 0;
}

/* Initial state f = f^eq(rho_k, 0); 0 at solid nodes. */
void oracle3_init(const oracle3_cfg* c, const uint8_t* solid, const double* rA, const double* rB, double* f) {
    size_t N = nodes(c);
    for (size_t s = 0; s < N; s++)
        for (int k = 0; k < 2; k++) {
            double fe[19];
            oracle3_feq(solid[s] ? 0.0 : (k == 0 ? rA[s] : rB[s]), 0.0, 0.0, 0.0, fe);
            for (int i = 0; i < 19; i++) f[((size_t)k * 19 + i) * N + s] = fe[i];
        }
}
