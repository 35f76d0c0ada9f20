/*
 * C ABI of the three-dimensional form of the two-component pseudopotential LBM time step with the
 * improved solid-fluid interaction scheme (arXiv 2505.22256, Sec. 3.5: static contact angles on a
 * spherical surface), for NVIDIA GB300 (sm_103a).
 *
 * The paper gives the 3-D case by its geometry only.  This library takes the direct 3-D forms of
 * the 2-D steps: D3Q19 velocities (weights 1/3, 1/18, 1/36; c_s^2 = 1/3); the cohesion and
 * adhesion sums of Eqs. 8-9 over the 92 offsets with |e|_inf <= 2 and |e|^2 in {1, 2, 3, 4, 5,
 * 6, 8}, weighted for eighth-order isotropy (w = 4/45, 1/21, 2/105, 5/504, 1/315, 1/630, 1/5040,
 * normalised to sum_e w e_x^2 = 1); the second-layer copy of Sec. 2.4 (a non-fluid site x+e with
 * |e|_inf = 2 takes the density and the solid switch of x + sign(e), componentwise); the local
 * adhesion parameter of Eqs. 10-12 for component A; Guo-forced SRT collision (Eqs. 1, 2, 6, 7)
 * with the half-force velocity shift of Eq. 5; halfway bounce-back (Sec. 3.5).  The lattice is
 * periodic in x, y and z; solid nodes come from the mask.
 *
 * Conventions as in lbm.h: inputs are copied, outputs are caller-owned, every call returns an
 * lbm_status and sets lbm_last_error(); lbm3d_step is asynchronous on the context's stream.
 * Arrays are [nz][ny][nx] with x fastest; populations [2][19][nz][ny][nx] in the D3Q19 order
 * e_0 = 0, e_1..e_6 = +x, -x, +y, -y, +z, -z, e_7..e_18 = (1,1,0), (-1,-1,0), (1,-1,0), (-1,1,0),
 * (1,0,1), (-1,0,-1), (1,0,-1), (-1,0,1), (0,1,1), (0,-1,-1), (0,1,-1), (0,-1,1).
 */
#ifndef LBM3D_H
#define LBM3D_H

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm3d_ctx lbm3d_ctx;

typedef struct {
    int32_t nx, ny, nz; /* lattice size, each >= 5; periodic in every direction */
} lbm3d_grid;

/* Stencil of the adhesion sum a(x) of Eq. 9 in 3-D.  The default takes the 92 offsets and weights
 * of the cohesion sum (the same reading as the 2-D default); LBM3_ADHESION_D3Q19 takes the sum as
 * printed with the weights of the velocity set, w = 1/18 (axes) and 1/36 (face diagonals), over the
 * 18 first-layer neighbours.  Under LBM3_ADHESION_D3Q19 the second-layer reconstruction of Table 1
 * feeds the cohesion sum only, so both lbm_second_layer readings give the same state. */
typedef enum {
    LBM3_ADHESION_E8 = 0,
    LBM3_ADHESION_D3Q19 = 1
} lbm3d_adhesion_stencil;

typedef struct {
    double tau[2];   /* relaxation times (Eq. 2), each > 0.5 */
    double G_AB;     /* inter-component strength (Eq. 8) */
    int32_t mode;    /* lbm_ads_mode: LBM_ADS_ORIGINAL or LBM_ADS_IMPROVED */
    int32_t second_layer; /* lbm_second_layer (lbm.h): what a solid second-layer stencil site takes
                             from x + sign(e) (Sec. 2.4, Table 1); the box is periodic, so every
                             non-fluid site is solid */
    double lambda;   /* G_w1 / G_w2, > 0 */
    double G_w2;     /* adhesion parameter of component B */
    double delta;    /* half-width of Eqs. 11-12, in (0, 1] */
    double g[3];     /* body acceleration, F_k += rho_k g */
    int32_t adhesion_stencil; /* lbm3d_adhesion_stencil: the stencil of Eq. 9 */
    int32_t pad_;             /* set to 0 */
    double rho0_store[2];     /* reference densities of the shifted 16-bit storage modes: populations
                                 are stored as f_i^k - w_i rho0_store[k]; ignored for FP32/FP64 */
} lbm3d_params;

typedef struct {
    double mass_A, mass_B;       /* sum of rho_k over fluid nodes (FP64) */
    double mom_x, mom_y, mom_z;  /* sum of (rho_A + rho_B) u over fluid nodes */
    double umax;                 /* max |u| over fluid nodes */
    double rhoA_min, rhoA_max, rhoB_min, rhoB_max;
    int64_t n_fluid;
    int32_t unstable;            /* 1 when a density was non-finite or <= 0, or u non-finite */
    int32_t pad_;
} lbm3d_diag;

/* Create a lattice.  solid: host [nz][ny][nx], nonzero = solid, at least one fluid node.
 * rho_A0, rho_B0: host initial densities, finite and > 0 at fluid nodes; the state starts at
 * f^eq(rho_k, 0).  storage (lbm_storage, lbm.h): LBM_STORE_F64, LBM_STORE_F32 (FP32 arithmetic),
 * or LBM_STORE_F16_SHIFTED / LBM_STORE_BF16_SHIFTED (16-bit storage of f - w rho0_store, FP32
 * arithmetic).  cuda_stream may be NULL (the library creates its own).  LBM_EINVAL for bad sizes, parameters or fields;
 * LBM_ENOMEM when device memory runs out; LBM_ECUDA for other CUDA errors and for devices other
 * than sm_103. */
lbm_status lbm3d_create(const lbm3d_grid* grid, const uint8_t* solid, const lbm3d_params* params,
                        const double* rho_A0, const double* rho_B0, int32_t storage, void* cuda_stream,
                        lbm3d_ctx** out);

void lbm3d_destroy(lbm3d_ctx* ctx);

/* Advance n >= 0 time steps (two launches per step: densities, then the fused force / collision /
 * streaming pass).  Asynchronous. */
lbm_status lbm3d_step(lbm3d_ctx* ctx, int64_t n);

/* rho_A, rho_B, u (Eq. 5 with the half-force shift) of the current state, FP64, [nz][ny][nx]; zero
 * at solid nodes.  Any pointer may be NULL.  on_device = 1: device pointers, enqueued on the
 * context's stream; 0: host pointers, synchronises. */
lbm_status lbm3d_fields(lbm3d_ctx* ctx, double* rho_A, double* rho_B, double* ux, double* uy, double* uz,
                        int32_t on_device);

/* Post-streaming populations f (host, FP64, [2][19][nz][ny][nx]; zero at solid nodes) of the
 * current state, and the inverse: set the state so that the next step starts from f.
 * Synchronise. */
lbm_status lbm3d_get_populations(lbm3d_ctx* ctx, double* f);
lbm_status lbm3d_set_populations(lbm3d_ctx* ctx, const double* f);

/* Re-initialise the lattice from new densities, f = f^eq(rho_k, 0), as lbm3d_create does (the same
 * state bit for bit) but without rebuilding the geometry.  rho_A, rho_B: [nz][ny][nx] doubles on
 * the host (on_device = 0: copied before return; the first such call allocates 16 bytes per node,
 * held until lbm3d_destroy) or on the device (on_device = 1: read on the context's stream). */
lbm_status lbm3d_set_densities(lbm3d_ctx* ctx, const double* rho_A, const double* rho_B, int32_t on_device);

/* lbm3d_set_densities and lbm3d_fields with host arrays, overlapped with the context's work: the
 * calls only enqueue and return.  Host<->device copies run on two copy streams of the context
 * through double-buffered device staging, so that one call's fields travel to the host, and the
 * next call's densities to the device, while the context's stream steps the lattice.  In stream
 * order the state is set after all work enqueued before lbm3d_set_densities_async, and the fields
 * are those after all work enqueued before lbm3d_fields_async.  The host arrays (same layout as the
 * blocking calls) should be page-locked for the copies to overlap; the inputs must stay unchanged
 * and the outputs unread until lbm3d_synchronize returns.  The first call allocates 56 bytes per
 * node (LBM_ENOMEM when that fails), held until lbm3d_destroy.  Any field output may be NULL. */
lbm_status lbm3d_set_densities_async(lbm3d_ctx* ctx, const double* rho_A, const double* rho_B);
lbm_status lbm3d_fields_async(lbm3d_ctx* ctx, double* rho_A, double* rho_B, double* ux, double* uy, double* uz);

/* Wait for the context's stream and its copy streams; LBM_ECUDA for an error of earlier
 * asynchronous work. */
lbm_status lbm3d_synchronize(lbm3d_ctx* ctx);

/* FP64 diagnostics over the fluid nodes (host output; synchronises).  LBM_EUNSTABLE when a
 * density is non-finite or <= 0, or a velocity non-finite (the record is still written). */
lbm_status lbm3d_diagnostics(lbm3d_ctx* ctx, lbm3d_diag* out);

/* Contact angle of a droplet of A on a solid sphere of centre c[3] and effective radius R (the
 * mask's sphere radius + 1/2 for halfway bounce-back), in degrees: rho^e = 0 crossings
 * (Eq. 10) along x, y and z lines between fluid nodes more than three cells (Chebyshev) from any
 * solid node, linearly interpolated; an algebraic sphere fit refined by one Gauss-Newton step in
 * FP64 on the device; cos(theta) = (R^2 + r^2 - d^2) / (2 r R).  Host outputs (any may be NULL);
 * synchronises.  LBM_ESTATE with fewer than 8 points. */
lbm_status lbm3d_contact_angle(lbm3d_ctx* ctx, const double* c, double R, double* theta_deg, double* fit_rms,
                               int64_t* npoints);

#ifdef __cplusplus
}
#endif

#endif /* LBM3D_H */
