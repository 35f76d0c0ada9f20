/*
 * lbm.h -- C ABI of the GB300 two-component pseudopotential lattice Boltzmann library.
 *
 * The library advances the time-step loop of the two-component immiscible pseudopotential
 * (Shan-Chen-type) lattice Boltzmann model with the improved solid-fluid interaction scheme of
 * Chen, Wang, Tao, Yang and Chen, "Improvement of Solid-Fluid Interaction Scheme in Lattice
 * Boltzmann Immiscible Pseudopotential Models" (arXiv 2505.22256):
 *   per-component densities (Eq. 3), inter-component cohesion force on the eighth-order isotropic
 *   24-node stencil (Eq. 8, Sec. 2.4), solid-fluid adhesion force (Eq. 9) with the local adhesion
 *   parameter of the improved scheme (Eqs. 10-12), second-layer reconstruction at walls (Sec. 2.4,
 *   Table 1), SRT collision with Guo forcing (Eqs. 1, 2, 6, 7) and streaming with halfway
 *   bounce-back (Sec. 3.5), plus the open inlet/outlet of Sec. 3.3.
 *
 * Conventions shared by every call
 *   - Lattice: D2Q9, e_0 = (0,0), e_1..e_4 = (1,0),(0,1),(-1,0),(0,-1), e_5..e_8 = (1,1),(-1,1),
 *     (-1,-1),(1,-1); c_s^2 = 1/3; lattice units (dx = dt = 1).  Component 0 = "A" (the paper's
 *     fluid 1), component 1 = "B" (fluid 2).
 *   - 2-D arrays are row-major [ny][nx] with x fastest; populations are [2][9][ny][nx].
 *   - Every call returns an lbm_status and never throws; lbm_last_error() gives a message for the
 *     last failing call on the calling thread.
 *   - Host inputs are copied before the call returns; the caller keeps ownership of every buffer
 *     it passes.  The library does not retain caller pointers.
 *   - All device work is issued on the context's CUDA stream (the one given at creation, or a
 *     non-blocking stream the library creates when NULL is given).  lbm_step is asynchronous;
 *     calls that return data to the host synchronise that stream first.  A device-side error of
 *     an asynchronous call surfaces as LBM_ECUDA from the next call that synchronises.
 *   - Not thread-safe per context: one host thread at a time may use a given context.
 *   - There is no CPU fallback: every call that computes runs CUDA kernels for sm_103a and fails
 *     with LBM_ECUDA when no such device is present.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx; /* opaque; created by lbm_create / lbm_ensemble_create */

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,    /* invalid argument: sizes, parameters, NULL pointer, case index */
    LBM_ENOMEM = 2,    /* device or host allocation failed */
    LBM_ECUDA = 3,     /* a CUDA call or kernel failed (also: no usable sm_103a device, or a
                          bounded wait for a tensor load inside a kernel gave up) */
    LBM_EUNSTABLE = 4, /* a non-finite or non-positive density was found (lbm_diagnostics) */
    LBM_ETIMEOUT = 5,  /* lbm_synchronize gave up after its time limit */
    LBM_ESTATE = 6,    /* call not valid in the context's current state */
    LBM_EIO = 7        /* file error in lbm_save / lbm_load, or a file that does not match */
} lbm_status;

/* Boundary treatment along one axis. */
typedef enum {
    LBM_BC_PERIODIC = 0, /* wrap around */
    LBM_BC_WALL = 1,     /* outside the array is solid: halfway bounce-back, s = 1 for adhesion */
    LBM_BC_OPEN = 2      /* x only: velocity inlet at x = 0, outflow at x = nx-1 (Sec. 3.3) */
} lbm_bc;

typedef struct {
    int32_t nx, ny; /* lattice size; each >= 5 */
    int32_t bc_x;   /* lbm_bc */
    int32_t bc_y;   /* LBM_BC_PERIODIC or LBM_BC_WALL */
} lbm_grid;

/* Velocity profile of the open inlet (Sec. 3.3). */
typedef enum {
    LBM_INLET_UNIFORM = 0,   /* u_in on every row */
    LBM_INLET_POISEUILLE = 1 /* u_in 4 s (ny - s) / ny^2, s = y + 1/2: peak u_in, zero at walls half a
                                cell below row 0 and above row ny-1 (needs bc_y = LBM_BC_WALL) */
} lbm_inlet_profile;

/* Solid-fluid interaction scheme (Sec. 2.3). */
typedef enum {
    LBM_ADS_ORIGINAL = 0, /* Eq. 9 with constant G_w1 = lambda * G_w2 */
    LBM_ADS_IMPROVED = 1  /* Eq. 9 with G_w1(x) from the effective density, Eqs. 10-12 */
} lbm_ads_mode;

/* Second-layer reconstruction (Sec. 2.4, Table 1): a second-layer stencil node (|e|_inf = 2) that
 * is not a fluid node takes the "information" of the first-layer node x + sign(e).  The default
 * reads that as both the pseudopotential and the solid switch of Eq. 9.  The alternative copies the
 * pseudopotential only; the site keeps its own solid switch in the adhesion sum (1 for a solid site
 * or one outside a wall direction; a site beyond an open column is that column, as for the first
 * layer).  On curved walls it gives a wider range of contact angles.  The cohesion sum is the same
 * under both readings. */
typedef enum {
    LBM_SECOND_LAYER_PSI_AND_SOLID = 0, /* default */
    LBM_SECOND_LAYER_PSI = 1
} lbm_second_layer;

/* Stencil of the adhesion sum of Eq. 9, a(x) = sum_e w(e) s(x + e) e, F_k,ads = -G_w,k rho_k a(x).
 * Sec. 2.4 applies the eighth-order isotropy to both schemes; Eq. 9 itself is printed with the D2Q9
 * weights w_i over the first-layer neighbours.  Under LBM_ADHESION_D2Q9 the second-layer
 * reconstruction of Table 1 feeds the cohesion sum only, so both lbm_second_layer readings give the
 * same state. */
typedef enum {
    LBM_ADHESION_E8 = 0,  /* default: the 24-node stencil and weights of the cohesion force */
    LBM_ADHESION_D2Q9 = 1 /* as printed in Eq. 9: w_i = 1/9 (axes), 1/36 (diagonals), first layer only */
} lbm_adhesion_stencil;

/* Outflow at x = nx-1 of an open x (Sec. 3.3 names an outflow scheme without stating it).  The
 * copy rule takes the populations entering through the outlet from column nx-2, or bounces them
 * back when that node is solid; it leaves the pressure level free, so a channel driven by the
 * velocity inlet through a resistive medium keeps gaining mass.  The pressure rule is the Zou-He
 * density condition per component: the three entering populations give the node the densities
 * rho_out and no momentum along y, with non-equilibrium bounce-back along x. */
typedef enum {
    LBM_OUTLET_COPY = 0,    /* default */
    LBM_OUTLET_PRESSURE = 1
} lbm_outlet;

typedef struct {
    double tau[2];        /* relaxation times tau_A, tau_B (Eq. 2); each > 0.5 */
    double G_AB;          /* inter-component strength G_12 (Eq. 8), stencil weights with
                             sum_e w(|e|^2) e_x^2 = 1 */
    int32_t mode;         /* lbm_ads_mode */
    double lambda;        /* strength coefficient lambda = G_w1 / G_w2 (Sec. 2.3.2); > 0 */
    double G_w2;          /* adhesion parameter of component B; the paper sets G_w2 = G_12 */
    double delta;         /* half-width delta of the interpolation in Eqs. 11-12, in (0, 1] */
    double g[2];          /* body acceleration (force per unit density), F_k += rho_k g */
    double u_in;          /* inlet x-velocity (LBM_BC_OPEN) */
    double rho_in[2];     /* component densities imposed at the inlet (LBM_BC_OPEN) */
    double rho0_store[2]; /* reference densities of the shifted 16-bit storage modes: populations
                             are stored as f_i^k - w_i rho0_store[k]; ignored for FP32/FP64 */
    double u_wall[2];     /* x-velocity of the lower and upper wall when bc_y = LBM_BC_WALL (the
                             walls lie half a cell below row 0 and above row ny-1); links across
                             them bounce back with the wall's momentum, 2 w_i rho_k (e_i . u_w) / c_s^2,
                             rho_k the node's density (Sec. 3.1 Couette flow).  0, 0: resting walls.
                             Nonzero needs bc_y = LBM_BC_WALL and bc_x != LBM_BC_OPEN */
    int32_t inlet_profile; /* lbm_inlet_profile (LBM_BC_OPEN) */
    int32_t second_layer;  /* lbm_second_layer: what a second-layer stencil node that is not a fluid
                              node takes from its first-layer partner x + sign(e) (Sec. 2.4, Table 1) */
    int32_t adhesion_stencil; /* lbm_adhesion_stencil (Eq. 9) */
    int32_t outlet;           /* lbm_outlet (LBM_BC_OPEN): outflow rule at x = nx-1 */
    double rho_out[2];        /* component densities held by LBM_OUTLET_PRESSURE; each > 0 */
} lbm_params;

/* Storage and arithmetic precision of the populations. */
typedef enum {
    LBM_STORE_F64 = 0,         /* FP64 storage, FP64 arithmetic */
    LBM_STORE_F32 = 1,         /* FP32 storage, FP32 arithmetic */
    LBM_STORE_F16_SHIFTED = 2, /* FP16 storage of f - w rho0, FP32 arithmetic */
    LBM_STORE_BF16_SHIFTED = 3 /* BF16 storage of f - w rho0, FP32 arithmetic */
} lbm_storage;

/* Global diagnostics of one case over its fluid nodes, accumulated in FP64 (Sec. 3.2 measures:
 * maximum spurious velocity, Fig. 10; density extrema, Fig. 11). */
typedef struct {
    double mass_A, mass_B;       /* sum of rho_A, rho_B */
    double mom_x, mom_y;         /* sum of (rho_A + rho_B) u, u with the half-force shift */
    double umax;                 /* max |u| */
    double rhoA_min, rhoA_max;
    double rhoB_min, rhoB_max;
    int64_t n_fluid;             /* number of fluid nodes */
    int32_t unstable;            /* 1 when a density was non-finite or <= 0, or u non-finite */
    int32_t pad_;
} lbm_diag;

/* Solid surface a droplet rests on, for the contact angle. */
typedef enum { LBM_SURFACE_FLAT = 0, LBM_SURFACE_CIRCLE = 1, LBM_SURFACE_NONE = 2 } lbm_surface_kind;
typedef struct {
    int32_t kind;   /* lbm_surface_kind */
    int32_t normal; /* flat: +1 when the fluid lies at y > y_w, -1 when at y < y_w */
    double y_w;     /* flat: wall plane (halfway bounce-back: half a cell beyond the last fluid row) */
    double cx, cy;  /* circle: centre of the solid disk */
    double R;       /* circle: effective radius (disk radius + 0.5 for halfway bounce-back) */
} lbm_surface;

/* One case of an ensemble. */
typedef struct {
    lbm_grid grid;
    const uint8_t* solid;  /* host, [ny][nx], nonzero = solid */
    const double* rho_A0;  /* host, [ny][nx], initial density of A (ignored at solid nodes) */
    const double* rho_B0;  /* host, [ny][nx], initial density of B */
    lbm_params params;
} lbm_case;

typedef struct {
    int32_t ncases;
    int32_t storage;         /* lbm_storage */
    int64_t nodes;           /* sum of nx*ny over cases */
    int64_t fluid_nodes;     /* sum of fluid nodes */
    int64_t wall_nodes;      /* sum of wall-list entries */
    int64_t steps;           /* time steps taken since creation or the last state load */
    int64_t state_bytes;     /* bytes of one population buffer (all cases) */
    int64_t device_bytes;    /* device memory held by the context */
    int32_t block_threads;   /* launch shape of the step kernel: threads per block */
    int32_t block_rows;      /* rows per work item (guided list: rows of its long items) */
    int32_t grid_blocks;     /* blocks per launch */
    int32_t work_items;      /* work items per step */
    int32_t wall_inline;     /* 1: the wall-list correction is inlined in the step kernel, 0: called */
    int32_t pad_;
} lbm_info_t;

/* ---------------------------------------------------------------------------------------------
 * Creation and destruction
 * ------------------------------------------------------------------------------------------- */

/* Create a single-case context.
 *   grid: lattice size and axis boundary types.  solid: host [ny][nx] mask, nonzero = solid; must
 *   contain at least one fluid node.  params: model parameters (Eqs. 2, 8, 9, 11-12; invalid values
 *   give LBM_EINVAL: tau <= 0.5, lambda <= 0, delta outside (0, 1], non-finite numbers, bc_y open).
 *   rho_A0, rho_B0: host [ny][nx] initial densities (> 0 at fluid nodes); the populations start at
 *   f = f^eq(rho_k, u = 0) (Eq. 6).  storage: lbm_storage.  cuda_stream: a cudaStream_t to issue
 *   all work on, or NULL for a library-owned non-blocking stream.  *out receives the context.
 * Builds the node flags and the wall list (Sec. 2.4 second-layer reconstruction) on the device. */
lbm_status lbm_create(const lbm_grid* grid, const uint8_t* solid, const lbm_params* params,
                      const double* rho_A0, const double* rho_B0, int32_t storage,
                      void* cuda_stream, lbm_ctx** out);

/* Create a context holding ncases independent cases of any sizes, stepped together by one launch
 * per time step.  Each case is validated as in lbm_create.  All cases share one storage mode. */
lbm_status lbm_ensemble_create(int32_t ncases, const lbm_case* cases, int32_t storage,
                               void* cuda_stream, lbm_ctx** out);

/* Release every device and host resource of the context (synchronises its streams).  NULL is a
 * no-op. */
void lbm_destroy(lbm_ctx* ctx);

/* ---------------------------------------------------------------------------------------------
 * Time stepping
 * ------------------------------------------------------------------------------------------- */

/* Advance every case by n >= 0 time steps (Eq. 1: collide, force, stream; Sec. 2.2-2.4).
 * Asynchronous on the context's stream.  Repeated calls replay a captured CUDA graph of the step
 * launches. */
lbm_status lbm_step(lbm_ctx* ctx, int64_t n);

/* Wait for the context's stream and, once the overlapped transfers have been used, its copy
 * streams, giving up after timeout_s seconds (<= 0: wait without limit) with LBM_ETIMEOUT.
 * Reports LBM_ECUDA for a device error of earlier asynchronous work. */
lbm_status lbm_synchronize(lbm_ctx* ctx, double timeout_s);

/* Re-initialise one case from new densities: f = f^eq(rho_k, 0).  rho_A0 / rho_B0 are [ny][nx]
 * doubles on the host (on_device = 0) or on the device (on_device = 1); host buffers are copied
 * before return, device buffers are read on the context's stream. */
lbm_status lbm_set_densities(lbm_ctx* ctx, int32_t case_index, const double* rho_A0,
                             const double* rho_B0, int32_t on_device);

/* ---------------------------------------------------------------------------------------------
 * Outputs
 * ------------------------------------------------------------------------------------------- */

/* Macroscopic fields of one case at the current state: rho_A, rho_B (Eq. 3) and the equilibrium
 * velocity u = (sum_k sum_i f e + F/2) / (rho_A + rho_B) (Eqs. 4-5 with Guo's half-force shift);
 * 0 at solid nodes.  Each output is [ny][nx] doubles, on the host (on_device = 0; the call
 * synchronises) or on the device (on_device = 1; written asynchronously on the stream).  Any
 * output pointer may be NULL. */
lbm_status lbm_fields(lbm_ctx* ctx, int32_t case_index, double* rho_A, double* rho_B, double* ux,
                      double* uy, int32_t on_device);

/* Every case of the context at once (the same results as the per-case calls, bit for bit): arrays
 * of sum_i nx_i ny_i doubles holding the cases back to back in case order, each [ny][nx].  Host
 * arrays (on_device = 0) move in one copy per array and the call synchronises once; device arrays
 * (on_device = 1) are read or written on the context's stream.  The first host-array call (or a
 * device call with a NULL field output) allocates 32 bytes per node of all cases, held until
 * lbm_destroy (LBM_ENOMEM when that fails).
 * lbm_set_densities_all: f = f^eq(rho_k, 0) in every case, as lbm_set_densities.
 * lbm_fields_all: rho_A, rho_B, ux, uy of every case, as lbm_fields; any output may be NULL. */
lbm_status lbm_set_densities_all(lbm_ctx* ctx, const double* rho_A0, const double* rho_B0, int32_t on_device);
lbm_status lbm_fields_all(lbm_ctx* ctx, double* rho_A, double* rho_B, double* ux, double* uy, int32_t on_device);

/* The same two operations with host arrays, overlapped with the context's work: the calls only
 * enqueue and return.  Host<->device copies run on two copy streams of the context, through
 * double-buffered device staging, so that the copy of one call's fields to the host and of the
 * next call's densities to the device proceed while the context's stream steps the lattice.  In
 * stream order the state is set after all work enqueued before lbm_set_densities_all_async and
 * the fields are those after all work enqueued before lbm_fields_all_async.  The host arrays
 * (same layout as above) should be page-locked for the copies to overlap; the inputs must stay
 * unchanged and the outputs unread until lbm_synchronize returns (which waits for the copy
 * streams too).  The first call allocates 96 bytes per node of all cases (LBM_ENOMEM when that
 * fails), held until lbm_destroy.  LBM_EINVAL for NULL densities; any field output may be NULL. */
lbm_status lbm_set_densities_all_async(lbm_ctx* ctx, const double* rho_A0, const double* rho_B0);
lbm_status lbm_fields_all_async(lbm_ctx* ctx, double* rho_A, double* rho_B, double* ux, double* uy);

/* Global FP64 diagnostics of one case (host output; synchronises).  Returns LBM_EUNSTABLE, with
 * *out filled, when the state holds a non-finite or non-positive density. */
lbm_status lbm_diagnostics(lbm_ctx* ctx, int32_t case_index, lbm_diag* out);

/* Contact angle of the droplet of component A in one case (Sec. 3.2): interface points are the
 * linear-interpolated zeros of the effective density rho^e (Eq. 10) along lattice rows and columns,
 * away (> 3 cells) from non-fluid sites; an algebraic circle fit in FP64 refined by one
 * Gauss-Newton step gives the droplet circle, and theta follows from its geometry relative to
 * *surface (cos theta = (R^2 + r^2 - d^2) / (2 r R) on a circle, -normal (c_y - y_w) / r on a flat
 * wall).  Host outputs; synchronises.  theta_deg, fit_rms (rms distance of the points from the
 * fitted circle) and npoints may be NULL.  LBM_ESTATE when fewer than 8 interface points exist. */
lbm_status lbm_contact_angle(lbm_ctx* ctx, int32_t case_index, const lbm_surface* surface,
                             double* theta_deg, double* fit_rms, int64_t* npoints);

/* Diagnostics of every case of the context (the reductions of lbm_diagnostics over an ensemble) in
 * one launch over the state plus one reduction per case; the same per-item partial sums, reduced
 * in the same order, so each record equals lbm_diagnostics of that case bit for bit.  out: host,
 * one lbm_diag per case.  Synchronises once.  LBM_EUNSTABLE when any case is unstable (every record
 * is written; the message names the first such case). */
lbm_status lbm_diagnostics_all(lbm_ctx* ctx, lbm_diag* out);

/* Contact angle of every case (the measurement of lbm_contact_angle over an ensemble): one density
 * pass over all cases, then each fit pass as one launch over all cases, one synchronisation at the
 * end.  Per-case partial sums are formed and combined as in lbm_contact_angle, so each angle equals
 * the single-case result bit for bit.  surfaces: host, one per case; kind LBM_SURFACE_NONE skips a
 * case.  Host outputs, one per case, each may be NULL: theta_deg and fit_rms (NaN for a skipped case
 * or one with fewer than 8 interface points), npoints (0 when skipped).  The first call allocates
 * 16 bytes per lattice node of all cases (FP64 densities) plus small tables, held until
 * lbm_destroy (LBM_ENOMEM when that fails).  LBM_EINVAL for a bad surface, before any work. */
lbm_status lbm_contact_angle_all(lbm_ctx* ctx, const lbm_surface* surfaces, double* theta_deg,
                                 double* fit_rms, int64_t* npoints);

/* Wall list of one case (host outputs; synchronises): fluid nodes whose 24-node stencil reaches a
 * non-fluid site, in increasing node order y*nx + x.  Per entry: node index; subst = bit n-1 set
 * when second-layer stencil node n (numbering of Table 1: 1-8 first layer in the D2Q9 order, 9-16
 * = 2 e_(n-8), 17-20 and 21-24 the knight moves whose first-layer partner is n-12 and n-16) is
 * replaced by its first-layer partner; seff = bit n-1 set when stencil node n counts as solid in
 * the adhesion sum (first-layer bits only under LBM_ADHESION_D2Q9); a = sum_n w(e_n) seff_n e_n
 * with the weights of the adhesion stencil.  Call first with node = NULL to get *n; the
 * arrays must then hold *n entries (any of them may be NULL). */
lbm_status lbm_wall_list(lbm_ctx* ctx, int32_t case_index, int32_t* node, uint32_t* subst,
                         uint32_t* seff, double* ax, double* ay, int64_t* n);

/* Populations f_i^k(x, t) of one case after streaming (the state collision acts on), as host
 * doubles [2][9][ny][nx]; 0 at solid nodes.  Synchronises. */
lbm_status lbm_get_populations(lbm_ctx* ctx, int32_t case_index, double* f);

/* Replace the state of one case by the post-streaming populations f (host doubles [2][9][ny][nx]),
 * rounded to the storage type.  For LBM_BC_OPEN the populations that enter through the boundary
 * columns are recomputed by the boundary rule at the next step. */
lbm_status lbm_set_populations(lbm_ctx* ctx, int32_t case_index, const double* f);

/* Size and launch information. */
lbm_status lbm_info(lbm_ctx* ctx, lbm_info_t* out);

/* ---------------------------------------------------------------------------------------------
 * Launch shape
 * ------------------------------------------------------------------------------------------- */

/* Set the step kernel's launch shape: threads per block (128 or 64, the widths the kernel is built
 * for; a work item spans that many columns minus 8 halo columns; lbm_create picks the width that
 * launches fewer thread columns over all cases) and rows per work item: >= 1 for uniform items of
 * that height, or 0 (the default) for a guided list -- long items first, then 16-row items that
 * even out the end of the launch, the long height chosen to balance the list over the resident
 * blocks; -64 .. -1 for a guided list whose short items have -block_rows rows.  Rebuilds the work
 * list and drops the captured graph.  LBM_EINVAL for other widths or block_rows < -64. */
lbm_status lbm_set_launch(lbm_ctx* ctx, int32_t block_threads, int32_t block_rows);

/* Failure-detection self-test (no counterpart in the paper).  Runs a one-thread kernel whose
 * pipeline wait can never complete (an mbarrier that nothing arrives on), bounded by limit_ms
 * milliseconds (0 < limit_ms <= 1000) exactly like the step kernel's tensor-load waits.  On giving up
 * it sets the context's device error word, and the call synchronises and reports it the way a
 * stalled step would be reported: LBM_ECUDA with a message naming the wait.  No copy is issued and
 * nothing stays in flight, so the GPU and the CUDA context stay usable, but the error word stays
 * set: every later synchronising call on this context reports it, so destroy the context
 * afterwards.  LBM_EINVAL for a limit outside the range. */
lbm_status lbm_selftest_wait_timeout(lbm_ctx* ctx, double limit_ms);

/* Choose the step kernel's form for wall-list nodes (the second-layer correction of Table 1): 1
 * inlines it (faster where wall-list nodes are common, e.g. porous media), 0 calls an out-of-line
 * copy (keeps the loop of warps without wall-list nodes small).  lbm_create picks 1 when wall-list
 * nodes exceed 4 % of the fluid nodes; lbm_autotune tries both.  Results agree to FP rounding.
 * Drops the captured graph.  LBM_EINVAL for other values. */
lbm_status lbm_set_wall_path(lbm_ctx* ctx, int32_t inline_correction);

/* Time candidate launch shapes on the live state (the current shape first, then both widths x both
 * wall-list forms x the row settings 0, -8, 16, 32, 64, 128; each twice for `steps` steps after one
 * warm-up launch, keeping the faster time) and keep the fastest; a shape replaces the best so far
 * only when it is at least 1 % faster, so that shapes within the timing noise do not trade places
 * from run to run.  The state advances by the steps taken; best_ms (may be NULL)
 * receives the best time per step.  Synchronises. */
lbm_status lbm_autotune(lbm_ctx* ctx, int32_t steps, double* best_ms);

/* ---------------------------------------------------------------------------------------------
 * Checkpoints
 * ------------------------------------------------------------------------------------------- */

/* Write / read the raw populations of every case with a header (sizes, storage, step count and a
 * hash of the parameters).  lbm_load requires a context built with the same cases and storage
 * (LBM_EIO otherwise) and restores the state bit for bit. */
lbm_status lbm_save(lbm_ctx* ctx, const char* path);
lbm_status lbm_load(lbm_ctx* ctx, const char* path);

/* ---------------------------------------------------------------------------------------------
 * Diagnostics without allocation
 * ------------------------------------------------------------------------------------------- */

/* The paper has no counterpart to this call; it is a service for callers that cannot allocate
 * device memory: code running under a framework that owns all device memory through its own
 * pool, real-time loops that cannot afford the synchronisation and latency of cudaMalloc/cudaFree,
 * or tools attached to a process whose device memory is already committed.
 *
 * Computes the same global FP64 diagnostics as lbm_diagnostics, from fields the caller already
 * holds on the device: rho_A, rho_B, ux, uy as [ny][nx] doubles (for example written by lbm_fields
 * with on_device = 1) and the solid mask as [ny][nx] uint8 (nonzero = solid), all device pointers
 * owned by the caller and only read.  *out is a host struct, filled before return; the call
 * synchronises cuda_stream (NULL = the legacy default stream).  It allocates nothing: its partial
 * sums live in a fixed array inside the library's device image (about 384 KB, held by every GPU
 * that loads the library until the process exits).  Limits and rules:
 *   - nx * ny may not exceed 16,777,216 nodes (LBM_EINVAL otherwise);
 *   - all calls on a device share that array, so calls that overlap on the GPU race; serialise them;
 *   - the first call on each device looks up the array's device address (cudaGetSymbolAddress)
 *     with that device current; make that first call before any stream capture on the device.
 *     The address is kept for the life of the process and belongs to the device's primary
 *     context: after cudaDeviceReset (which destroys that context) it is no longer valid, so do
 *     not call this function again in that process.
 * Returns LBM_EUNSTABLE, with *out filled, when a fluid node has a non-finite or non-positive
 * density. */
lbm_status lbm_diagnostics_noalloc(const double* rho_A, const double* rho_B, const double* ux,
                                   const double* uy, const uint8_t* solid, int32_t nx, int32_t ny,
                                   void* cuda_stream, lbm_diag* out);

/* ---------------------------------------------------------------------------------------------
 * Errors
 * ------------------------------------------------------------------------------------------- */
const char* lbm_status_str(int32_t status);
const char* lbm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LBM_GB300_H */
