// Fused time-step kernel of the two-component pseudopotential LBM (arXiv 2505.22256) and the
// kernels that read and write its state.
//
// State: one buffer per time level holds the post-collision populations f*_i^k of every case,
// [2][9][ny][pitch] per case, of the storage type S.  One launch of k_step performs, for every
// fluid node x:
//   pull    f_i(x) = f*_i(x - e_i), or f*_opp(i)(x) across a blocked link (halfway bounce-back,
//           Sec. 3.5); open columns complete the entering populations (Sec. 3.3)
//   moments rho_k = sum_i f_i (Eq. 3), momentum sum_k sum_i f_i e_i (Eq. 4)
//   forces  cohesion on the eighth-order 24-node stencil (Eq. 8, Sec. 2.4) from a shared-memory
//           ring of densities; wall-list nodes take second-layer values from their first-layer
//           partner (Table 1) and add the adhesion force of Eq. 9 with the local parameter of
//           Eqs. 10-12; body force
//   collide u = (momentum + F/2) / rho (Eq. 5 with Guo's shift); f* = f + (f^eq - f)/tau +
//           (1 - 1/(2 tau)) F_i (Eqs. 1, 2, 6, 7), written to the other buffer.
//
// Work decomposition: a work item is a window of blockDim.x columns by a chunk of rows of one
// case.  Every thread owns one window column and marches down the rows: for row y+2 it pulls the
// populations and stores rho_A, rho_B in a six-row ring in shared memory, keeps the populations
// of rows y..y+2 in registers, and after one barrier collides row y with the 5x5 neighbourhood of
// densities it needs.  The two outermost columns on each side only supply densities (the window's
// halo); interior columns collide.  Densities of halo rows and columns are recomputed by the
// neighbouring items, so one launch needs no grid-wide synchronisation.
#include <math.h>

#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr int kRing = 6;  // rows of densities kept in shared memory

template <class R>
struct Params {
    int nx, ny, pitch, bc_x, bc_y, mode;
    long long plane;  // ny * pitch
    R omega[2], cF[2];
    R G, Gw2, lam, delta, s1, s2, s3, t2, t3;
    R gx, gy;
    R d1[2], d5[2];   // inlet: f_1 - f_3 and f_5 - f_7 (= f_8 - f_6) of f^eq(rho_in, u_in)
    R sh0[2], sh1[2], sh5[2];  // storage shift w_i rho0 for the rest, axis and diagonal weights
};

template <class R>
__device__ __forceinline__ Params<R> load_params(const DevCase& C) {
    Params<R> P;
    P.nx = C.nx; P.ny = C.ny; P.pitch = C.pitch; P.bc_x = C.bc_x; P.bc_y = C.bc_y; P.mode = C.mode;
    P.plane = (long long)C.ny * C.pitch;
    for (int k = 0; k < 2; ++k) {
        P.omega[k] = (R)C.omega[k];
        P.cF[k] = (R)C.cF[k];
        P.d1[k] = (R)(6.0 * wq(1) * C.rho_in[k] * C.u_in);
        P.d5[k] = (R)(6.0 * wq(5) * C.rho_in[k] * C.u_in);
        P.sh0[k] = (R)(wq(0) * C.rho0[k]);
        P.sh1[k] = (R)(wq(1) * C.rho0[k]);
        P.sh5[k] = (R)(wq(5) * C.rho0[k]);
    }
    P.G = (R)C.G; P.Gw2 = (R)C.Gw2; P.lam = (R)C.lam; P.delta = (R)C.delta;
    P.s1 = (R)C.s1; P.s2 = (R)C.s2; P.s3 = (R)C.s3; P.t2 = (R)C.t2; P.t3 = (R)C.t3;
    P.gx = (R)C.g[0]; P.gy = (R)C.g[1];
    return P;
}

template <class R>
__device__ __forceinline__ R shift_of(const Params<R>& P, int k, int i) {
    return i == 0 ? P.sh0[k] : (i <= 4 ? P.sh1[k] : P.sh5[k]);
}

// Pull the 18 post-streaming populations of fluid node (X, Y) from the post-collision buffer.
template <class S, class R>
__device__ __forceinline__ void pull_node(const S* __restrict__ fin, const Params<R>& P, int X, int Y,
                                          uint16_t fl, R (&f)[18]) {
    const bool open = P.bc_x == kOpen;
    const bool inlet = open && X == 0;
    const bool outlet = open && X == P.nx - 1;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        int sx = X, sy = Y, si = i;
        if (i != 0) {
            const bool blocked = (fl >> (i - 1)) & 1u;
            int bx = X;
            if (cx(i) < 0 && outlet) bx = (fl & kOutletOwnBit) ? X : X - 1;  // copied from upstream
            if (blocked) {
                sx = bx;
                si = opp(i);
            } else {
                sx = bx - cx(i);
                sy = Y - cy(i);
                sx += (sx < 0) ? P.nx : 0;
                sx -= (sx >= P.nx) ? P.nx : 0;
                sy += (sy < 0) ? P.ny : 0;
                sy -= (sy >= P.ny) ? P.ny : 0;
            }
        }
        if (cx(i) > 0 && inlet) continue;  // entering through the inlet: set below
        const long long o = (long long)sy * P.pitch + sx;
        R a = (R)Store<S>::ld(fin + (long long)si * P.plane + o);
        R b = (R)Store<S>::ld(fin + (long long)(9 + si) * P.plane + o);
        if constexpr (Store<S>::kShift) {
            a += shift_of(P, 0, i);  // w_si = w_i
            b += shift_of(P, 1, i);
        }
        f[i] = a;
        f[9 + i] = b;
    }
    if (inlet) {  // non-equilibrium bounce-back about f^eq(rho_in, (u_in, 0))
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            f[9 * k + 1] = f[9 * k + 3] + P.d1[k];
            f[9 * k + 5] = f[9 * k + 7] + P.d5[k];
            f[9 * k + 8] = f[9 * k + 6] + P.d5[k];
        }
    }
}

// Window column -> lattice column for density lookups; -1 when it lies outside a wall boundary.
template <class R>
__device__ __forceinline__ int map_col(const Params<R>& P, int x) {
    if (x >= 0 && x < P.nx) return x;
    if (P.bc_x == kPeriodic) return ((x % P.nx) + P.nx) % P.nx;
    if (P.bc_x == kOpen) return x < 0 ? 0 : P.nx - 1;  // clamp to the boundary column
    return -1;
}

__device__ __forceinline__ int ring_slot(int r) { return (r + kRing) % kRing; }

template <class R>
struct Diag {
    double v[kDiagN];
    __device__ void init() {
        for (int q = 0; q < kDiagN; ++q) v[q] = 0.0;
        v[5] = v[7] = INFINITY;
        v[6] = v[8] = -INFINITY;
    }
};

// Collide (or, in fields mode, evaluate) one interior fluid node.
template <class S, class R, bool kFields>
__device__ __forceinline__ void node_update(const Params<R>& P, const R* __restrict__ ringA,
                                            const R* __restrict__ ringB, int W, int tid, int y,
                                            int x, uint16_t fl, const R (&f)[18], long long w_entry,
                                            const uint32_t* __restrict__ wl_subst,
                                            const R* __restrict__ wl_a, long long nwall_total,
                                            S* __restrict__ fout, double* __restrict__ o_rA,
                                            double* __restrict__ o_rB, double* __restrict__ o_ux,
                                            double* __restrict__ o_uy, Diag<R>& dg) {
    int sb[5];
#pragma unroll
    for (int d = 0; d < 5; ++d) sb[d] = ring_slot(y + d - 2) * W + tid;
    const R rA = ringA[sb[2]];
    const R rB = ringB[sb[2]];

    uint32_t sub = 0;
    R ax = (R)0, ay = (R)0;
    const bool wall = (fl & kWallBit) != 0;
    if (wall) {
        sub = __ldg(wl_subst + w_entry);
        ax = __ldg(wl_a + w_entry);
        ay = __ldg(wl_a + nwall_total + w_entry);
    }

    // 24 stencil values psi~ of each component.  v[dy+2][dx+2]; second-layer sites flagged in
    // the substitution mask read their first-layer partner x + sign(e) (Table 1).
    R vA[5][5], vB[5][5];
#pragma unroll
    for (int dy = -2; dy <= 2; ++dy) {
#pragma unroll
        for (int dx = -2; dx <= 2; ++dx) {
            if (dx == 0 && dy == 0) continue;
            int addr = sb[dy + 2] + dx;
            if (dx == 2 || dx == -2 || dy == 2 || dy == -2) {
                // Table 1 node number of (dx, dy) minus one
                const int sx = (dx > 0) - (dx < 0), sy = (dy > 0) - (dy < 0);
                int n;
                if (dx == 2 * sx && dy == 2 * sy) {
                    // (+-2, 0), (0, +-2), (+-2, +-2): 2 e_m, m = first-layer partner
                    const int m = (sx == 1 && sy == 0) ? 1 : (sx == 0 && sy == 1) ? 2 : (sx == -1 && sy == 0) ? 3
                                : (sx == 0 && sy == -1) ? 4 : (sx == 1 && sy == 1) ? 5 : (sx == -1 && sy == 1) ? 6
                                : (sx == -1 && sy == -1) ? 7 : 8;
                    n = m + 7;
                } else {
                    const int m = (sx == 1 && sy == 1) ? 5 : (sx == -1 && sy == 1) ? 6 : (sx == -1 && sy == -1) ? 7 : 8;
                    n = (dx == 2 || dx == -2) ? m + 11 : m + 15;
                }
                const int alt = sb[sy + 2] + sx;
                addr = ((sub >> n) & 1u) ? alt : addr;
            }
            vA[dy + 2][dx + 2] = ringA[addr];
            vB[dy + 2][dx + 2] = ringB[addr];
        }
    }

    // sum_e w(|e|^2) psi~(x + e) e, grouping mirror images so a uniform field gives exactly 0
    R gAx = 0, gAy = 0, gBx = 0, gBy = 0;
#pragma unroll
    for (int dy = -2; dy <= 2; ++dy) {
#pragma unroll
        for (int dx = 1; dx <= 2; ++dx) {
            const R w = (R)(w8(dx * dx + dy * dy) * dx);
            gAx += w * (vA[dy + 2][2 + dx] - vA[dy + 2][2 - dx]);
            gBx += w * (vB[dy + 2][2 + dx] - vB[dy + 2][2 - dx]);
        }
    }
#pragma unroll
    for (int dx = -2; dx <= 2; ++dx) {
#pragma unroll
        for (int dy = 1; dy <= 2; ++dy) {
            const R w = (R)(w8(dx * dx + dy * dy) * dy);
            gAy += w * (vA[2 + dy][dx + 2] - vA[2 - dy][dx + 2]);
            gBy += w * (vB[2 + dy][dx + 2] - vB[2 - dy][dx + 2]);
        }
    }

    // cohesion: each component is pushed by the other's pseudopotential gradient (Eq. 8)
    R FAx = -P.G * rA * gBx, FAy = -P.G * rA * gBy;
    R FBx = -P.G * rB * gAx, FBy = -P.G * rB * gAy;
    // adhesion (Eq. 9); G_w1 local in the improved scheme (Eqs. 10, 12)
    if (wall) {
        R GA;
        if (P.mode == 1) {
            const R re = (rA - rB) / (rA + rB);
            R h;
            if (re > P.delta) h = P.lam;
            else if (re > (R)0) h = P.s1 + re * (P.s2 + re * P.s3);
            else if (re > -P.delta) h = P.s1 + re * (P.t2 + re * P.t3);
            else h = (R)1;
            GA = P.Gw2 * h;
        } else {
            GA = P.lam * P.Gw2;
        }
        FAx -= GA * rA * ax;
        FAy -= GA * rA * ay;
        FBx -= P.Gw2 * rB * ax;
        FBy -= P.Gw2 * rB * ay;
    }
    // body force
    FAx += rA * P.gx; FAy += rA * P.gy;
    FBx += rB * P.gx; FBy += rB * P.gy;

    // equilibrium velocity with the half-force shift
    R mx = 0, my = 0;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const R s = f[i] + f[9 + i];
        if (cx(i) != 0) mx += cx(i) > 0 ? s : -s;
        if (cy(i) != 0) my += cy(i) > 0 ? s : -s;
    }
    const R rho = rA + rB;
    const R inv = (R)1 / rho;
    const R ux = (mx + (R)0.5 * (FAx + FBx)) * inv;
    const R uy = (my + (R)0.5 * (FAy + FBy)) * inv;

    if constexpr (kFields) {
        const long long o = (long long)y * P.nx + x;
        o_rA[o] = (double)rA;
        o_rB[o] = (double)rB;
        o_ux[o] = (double)ux;
        o_uy[o] = (double)uy;
        const double dux = ux, duy = uy, drho = (double)rho;
        dg.v[0] += (double)rA;
        dg.v[1] += (double)rB;
        dg.v[2] += drho * dux;
        dg.v[3] += drho * duy;
        const double um = sqrt(dux * dux + duy * duy);
        dg.v[4] = fmax(dg.v[4], um);
        dg.v[5] = fmin(dg.v[5], (double)rA);
        dg.v[6] = fmax(dg.v[6], (double)rA);
        dg.v[7] = fmin(dg.v[7], (double)rB);
        dg.v[8] = fmax(dg.v[8], (double)rB);
        dg.v[9] += 1.0;
        if (!(rA > (R)0) || !(rB > (R)0) || !isfinite(um) || !isfinite((double)rA) || !isfinite((double)rB))
            dg.v[10] = 1.0;
    } else {
        // SRT collision with Guo forcing for each component (Eqs. 1, 2, 6, 7)
        const R usq15 = (R)1.5 * (ux * ux + uy * uy);
        const long long o = (long long)y * P.pitch + x;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const R rk = k == 0 ? rA : rB;
            const R Fx = k == 0 ? FAx : FBx, Fy = k == 0 ? FAy : FBy;
            const R om = P.omega[k], cf = P.cF[k];
            const R uF3 = (R)3 * (ux * Fx + uy * Fy);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                R eu = 0, eF = 0;
                if (cx(i) != 0) { eu += cx(i) > 0 ? ux : -ux; eF += cx(i) > 0 ? Fx : -Fx; }
                if (cy(i) != 0) { eu += cy(i) > 0 ? uy : -uy; eF += cy(i) > 0 ? Fy : -Fy; }
                const R w = (R)wq(i);
                const R feq = w * rk * ((R)1 - usq15 + eu * ((R)3 + (R)4.5 * eu));
                const R Fi = w * ((R)3 * eF - uF3 + (R)9 * eu * eF);
                const R fi = f[9 * k + i];
                R fo = fi + om * (feq - fi) + cf * Fi;
                if constexpr (Store<S>::kShift) fo -= shift_of(P, k, i);
                Store<S>::st(fout + (long long)(9 * k + i) * P.plane + o, fo);
            }
        }
    }
}

template <class S, class R, bool kFields>
__global__ void __launch_bounds__(256) k_step(const DevCase* __restrict__ cases, const int4* __restrict__ items,
                                              int item_begin, int item_end, const S* __restrict__ fin_all,
                                              S* __restrict__ fout_all, const uint16_t* __restrict__ flags_all,
                                              const int32_t* __restrict__ widx_all,
                                              const uint32_t* __restrict__ wl_subst,
                                              const R* __restrict__ wl_a, long long nwall_total,
                                              double* __restrict__ o_rA, double* __restrict__ o_rB,
                                              double* __restrict__ o_ux, double* __restrict__ o_uy,
                                              double* __restrict__ diag_part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int W = blockDim.x, tid = threadIdx.x;
    R* ringA = reinterpret_cast<R*>(smem_raw);
    R* ringB = ringA + kRing * W;

    for (int it = item_begin + blockIdx.x; it < item_end; it += gridDim.x) {
        const int4 item = items[it];
        const DevCase& C = cases[item.x];
        const Params<R> P = load_params<R>(C);
        const S* __restrict__ fin = fin_all + C.f_off;
        S* __restrict__ fout = fout_all + C.f_off;
        const uint16_t* __restrict__ flags = flags_all + C.n_off;
        const int32_t* __restrict__ widx = widx_all + C.n_off;
        const int x = item.y + tid;               // window column of this thread
        const int X = map_col(P, x);              // lattice column for the density ring
        const bool interior = tid >= 2 && tid < W - 2 && x < P.nx;
        const int y0 = item.z, y1 = item.w;

        Diag<R> dg;
        if constexpr (kFields) dg.init();

        // densities of row r into the ring; populations of row r kept in f, flags in fl
        auto rho_row = [&](int r, R(&f)[18], uint16_t& fl) {
            int Y = r;
            bool ok = X >= 0;
            if (Y < 0 || Y >= P.ny) {
                if (P.bc_y == kPeriodic) Y = (Y + P.ny) % P.ny;
                else ok = false;
            }
            R a = 0, b = 0;
            fl = kSolidBit;
            if (ok) {
                fl = __ldg(flags + (long long)Y * P.pitch + X);
                if (!(fl & kSolidBit)) {
                    pull_node<S, R>(fin, P, X, Y, fl, f);
#pragma unroll
                    for (int i = 0; i < 9; ++i) { a += f[i]; b += f[9 + i]; }
                }
            }
            const int s = ring_slot(r) * W + tid;
            ringA[s] = a;
            ringB[s] = b;
        };
        auto update_row = [&](int y, const R(&f)[18], uint16_t fl) {
            if (!interior) return;
            if (fl & kSolidBit) {
                if constexpr (kFields) {  // fields are 0 at solid nodes
                    const long long o = (long long)y * P.nx + x;
                    o_rA[o] = 0.0;
                    o_rB[o] = 0.0;
                    o_ux[o] = 0.0;
                    o_uy[o] = 0.0;
                }
                return;
            }
            long long we = 0;
            if (fl & kWallBit) {
                we = __ldg(widx + (long long)y * P.pitch + x);
                we = we < 0 ? 0 : (we >= nwall_total ? nwall_total - 1 : we);  // never read outside the list
            }
            node_update<S, R, kFields>(P, ringA, ringB, W, tid, y, x, fl, f, we, wl_subst, wl_a, nwall_total,
                                       fout, o_rA, o_rB, o_ux, o_uy, dg);
        };

        R fa[18], fb[18], fc[18];
        uint16_t la, lb, lc;
        __syncthreads();  // the previous item's readers are done with the ring
        rho_row(y0 - 2, fa, la);
        rho_row(y0 - 1, fa, la);
        rho_row(y0, fa, la);
        rho_row(y0 + 1, fb, lb);
        for (int y = y0; y < y1; y += 3) {
            rho_row(y + 2, fc, lc);
            __syncthreads();
            update_row(y, fa, la);
            if (y + 1 >= y1) break;
            rho_row(y + 3, fa, la);
            __syncthreads();
            update_row(y + 1, fb, lb);
            if (y + 2 >= y1) break;
            rho_row(y + 4, fb, lb);
            __syncthreads();
            update_row(y + 2, fc, lc);
        }

        if constexpr (kFields) {
            // block reduction of the item's partial diagnostics (sums, max, min), in FP64
            __shared__ double red[16][kDiagN];
            const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
            for (int q = 0; q < kDiagN; ++q) {
                double v = dg.v[q];
                for (int off = 16; off > 0; off >>= 1) {
                    const double o = __shfl_xor_sync(0xffffffffu, v, off);
                    v = (q == 4 || q == 6 || q == 8 || q == 10) ? fmax(v, o) : (q == 5 || q == 7) ? fmin(v, o) : v + o;
                }
                if (lane == 0) red[warp][q] = v;
            }
            __syncthreads();
            if (tid == 0) {
                const int nw = (W + 31) >> 5;
                for (int q = 0; q < kDiagN; ++q) {
                    double v = red[0][q];
                    for (int w2 = 1; w2 < nw; ++w2) {
                        const double o = red[w2][q];
                        v = (q == 4 || q == 6 || q == 8 || q == 10) ? fmax(v, o) : (q == 5 || q == 7) ? fmin(v, o) : v + o;
                    }
                    diag_part[(long long)it * kDiagN + q] = v;
                }
            }
        }
    }
}

// f = f^eq(rho_k, 0) = w_i rho_k at fluid nodes (dense doubles [2][9][ny][nx]).
__global__ void k_feq_rest(const DevCase* __restrict__ cases, int c, const uint8_t* __restrict__ solid_all,
                           const double* __restrict__ rhoA, const double* __restrict__ rhoB,
                           double* __restrict__ f) {
    const DevCase C = cases[c];
    const long long N = (long long)C.nx * C.ny;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N; s += (long long)gridDim.x * blockDim.x) {
        const bool sol = solid_all[C.d_off + s] != 0;
        const double a = sol ? 0.0 : rhoA[s], b = sol ? 0.0 : rhoB[s];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            f[(long long)i * N + s] = wq(i) * a;
            f[(long long)(9 + i) * N + s] = wq(i) * b;
        }
    }
}

// Post-streaming populations (dense doubles) -> post-collision buffer: the inverse of the pull, so
// that the next pull reproduces f exactly (up to the storage rounding).
template <class S>
__global__ void k_set_state(const DevCase* __restrict__ cases, int c, const uint16_t* __restrict__ flags_all,
                            const double* __restrict__ f, S* __restrict__ out_all) {
    const DevCase C = cases[c];
    using R = typename ComputeOf<S>::type;
    const long long N = (long long)C.nx * C.ny;
    const long long plane = (long long)C.ny * C.pitch;
    S* out = out_all + C.f_off;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N; s += (long long)gridDim.x * blockDim.x) {
        const int X = (int)(s % C.nx), Y = (int)(s / C.nx);
        const long long o = (long long)Y * C.pitch + X;
        const uint16_t fl = flags_all[C.n_off + o];
        for (int k = 0; k < 2; ++k) {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                double v = 0.0;
                if (!(fl & kSolidBit)) {
                    int tx = X + cx(i), ty = Y + cy(i);
                    if (C.bc_x == kOpen && (tx < 0 || tx >= C.nx)) {
                        const bool own = X == C.nx - 1 && (fl & kOutletOwnBit) && cx(i) > 0;
                        v = f[(long long)(9 * k + (own ? opp(i) : i)) * N + s];
                    } else if (i != 0 && ((fl >> (opp(i) - 1)) & 1u)) {
                        v = f[(long long)(9 * k + opp(i)) * N + s];
                    } else {
                        tx += (tx < 0) ? C.nx : 0;
                        tx -= (tx >= C.nx) ? C.nx : 0;
                        ty += (ty < 0) ? C.ny : 0;
                        ty -= (ty >= C.ny) ? C.ny : 0;
                        v = f[(long long)(9 * k + i) * N + (long long)ty * C.nx + tx];
                    }
                    if constexpr (Store<S>::kShift) v -= wq(i) * C.rho0[k];
                }
                Store<S>::st(out + (long long)(9 * k + i) * plane + o, (R)v);
            }
        }
    }
}

// Post-collision buffer -> post-streaming populations (dense doubles), 0 at solid nodes.
template <class S>
__global__ void k_get_state(const DevCase* __restrict__ cases, int c, const uint16_t* __restrict__ flags_all,
                            const S* __restrict__ fin_all, double* __restrict__ f) {
    using R = typename ComputeOf<S>::type;
    const DevCase C = cases[c];
    const Params<R> P = load_params<R>(C);
    const long long N = (long long)C.nx * C.ny;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N; s += (long long)gridDim.x * blockDim.x) {
        const int X = (int)(s % C.nx), Y = (int)(s / C.nx);
        const uint16_t fl = flags_all[C.n_off + (long long)Y * C.pitch + X];
        R v[18];
        if (fl & kSolidBit) {
#pragma unroll
            for (int q = 0; q < 18; ++q) v[q] = 0;
        } else {
            pull_node<S, R>(fin_all + C.f_off, P, X, Y, fl, v);
        }
#pragma unroll
        for (int q = 0; q < 18; ++q) f[(long long)q * N + s] = (double)v[q];
    }
}

// Per-case reduction of the per-item partials, in item order (deterministic).
__global__ void k_diag_reduce(const DevCase* __restrict__ cases, int c, const double* __restrict__ part,
                              double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const DevCase C = cases[c];
    double v[kDiagN];
    for (int q = 0; q < kDiagN; ++q) v[q] = part[(long long)C.item_begin * kDiagN + q];
    for (int it = C.item_begin + 1; it < C.item_end; ++it)
        for (int q = 0; q < kDiagN; ++q) {
            const double o = part[(long long)it * kDiagN + q];
            v[q] = (q == 4 || q == 6 || q == 8 || q == 10) ? fmax(v[q], o) : (q == 5 || q == 7) ? fmin(v[q], o) : v[q] + o;
        }
    for (int q = 0; q < kDiagN; ++q) out[(long long)c * kDiagN + q] = v[q];
}

template <class S>
void* kernel_ptr(bool fields) {
    using R = typename ComputeOf<S>::type;
    return fields ? (void*)k_step<S, R, true> : (void*)k_step<S, R, false>;
}

void* step_kernel(int storage, bool fields) {
    switch (storage) {
        case LBM_STORE_F64: return kernel_ptr<double>(fields);
        case LBM_STORE_F32: return kernel_ptr<float>(fields);
        case LBM_STORE_F16_SHIFTED: return kernel_ptr<__half>(fields);
        default: return kernel_ptr<__nv_bfloat16>(fields);
    }
}

size_t compute_size(int storage) { return storage == LBM_STORE_F64 ? 8 : 4; }

template <class S>
cudaError_t launch_step_t(Ctx& c, const void* fin, void* fout, cudaStream_t s, bool fields, int ib, int ie,
                          int grid, double* o4[4], double* part) {
    using R = typename ComputeOf<S>::type;
    const size_t smem = 2 * kRing * (size_t)c.block_threads * sizeof(R);
    if (fields)
        k_step<S, R, true><<<grid, c.block_threads, smem, s>>>(
            c.dcases, c.items, ib, ie, (const S*)fin, (S*)fout, c.flags, c.widx, c.wl_subst, (const R*)c.wl_ar,
            c.nwall, o4[0], o4[1], o4[2], o4[3], part);
    else
        k_step<S, R, false><<<grid, c.block_threads, smem, s>>>(
            c.dcases, c.items, ib, ie, (const S*)fin, (S*)fout, c.flags, c.widx, c.wl_subst, (const R*)c.wl_ar,
            c.nwall, nullptr, nullptr, nullptr, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t dispatch(Ctx& c, const void* fin, void* fout, cudaStream_t s, bool fields, int ib, int ie, int grid,
                     double* o4[4], double* part) {
    switch (c.storage) {
        case LBM_STORE_F64: return launch_step_t<double>(c, fin, fout, s, fields, ib, ie, grid, o4, part);
        case LBM_STORE_F32: return launch_step_t<float>(c, fin, fout, s, fields, ib, ie, grid, o4, part);
        case LBM_STORE_F16_SHIFTED: return launch_step_t<__half>(c, fin, fout, s, fields, ib, ie, grid, o4, part);
        default: return launch_step_t<__nv_bfloat16>(c, fin, fout, s, fields, ib, ie, grid, o4, part);
    }
}

int blocks_for(long long n) { return (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096); }

}  // namespace

int step_smem_bytes(int storage, int threads) { return (int)(2 * kRing * (size_t)threads * compute_size(storage)); }

cudaError_t step_occupancy(int storage, int threads, int* blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, step_kernel(storage, false), threads,
                                                         step_smem_bytes(storage, threads));
}

cudaError_t launch_step(Ctx& c, const void* fin, void* fout, cudaStream_t s) {
    double* o4[4] = {nullptr, nullptr, nullptr, nullptr};
    return dispatch(c, fin, fout, s, false, 0, c.nitems, c.grid_blocks, o4, nullptr);
}

cudaError_t launch_fields(Ctx& c, int ci, double* rhoA, double* rhoB, double* ux, double* uy, bool diag) {
    const DevCase& C = c.hcases[ci];
    const long long N = (long long)C.nx * C.ny;
    double* o4[4] = {rhoA ? rhoA : c.fields, rhoB ? rhoB : c.fields + N, ux ? ux : c.fields + 2 * N,
                     uy ? uy : c.fields + 3 * N};
    const int n = C.item_end - C.item_begin;
    const int grid = n < c.grid_blocks ? n : c.grid_blocks;
    (void)diag;
    return dispatch(c, c.f[c.cur], c.f[1 - c.cur], c.stream, true, C.item_begin, C.item_end, grid, o4, c.diag_part);
}

cudaError_t launch_diag_reduce(Ctx& c, int ci) {
    k_diag_reduce<<<1, 32, 0, c.stream>>>(c.dcases, ci, c.diag_part, c.diag_out);
    return cudaGetLastError();
}

cudaError_t launch_feq_rest(Ctx& c, int ci, const double* rhoA, const double* rhoB, double* dense_f) {
    const long long N = (long long)c.hcases[ci].nx * c.hcases[ci].ny;
    k_feq_rest<<<blocks_for(N), 256, 0, c.stream>>>(c.dcases, ci, c.solid, rhoA, rhoB, dense_f);
    return cudaGetLastError();
}

cudaError_t launch_set_state(Ctx& c, int ci, const double* dense_f) {
    const long long N = (long long)c.hcases[ci].nx * c.hcases[ci].ny;
    const int g = blocks_for(N);
    switch (c.storage) {
        case LBM_STORE_F64: k_set_state<double><<<g, 256, 0, c.stream>>>(c.dcases, ci, c.flags, dense_f, (double*)c.f[c.cur]); break;
        case LBM_STORE_F32: k_set_state<float><<<g, 256, 0, c.stream>>>(c.dcases, ci, c.flags, dense_f, (float*)c.f[c.cur]); break;
        case LBM_STORE_F16_SHIFTED: k_set_state<__half><<<g, 256, 0, c.stream>>>(c.dcases, ci, c.flags, dense_f, (__half*)c.f[c.cur]); break;
        default: k_set_state<__nv_bfloat16><<<g, 256, 0, c.stream>>>(c.dcases, ci, c.flags, dense_f, (__nv_bfloat16*)c.f[c.cur]); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_get_state(Ctx& c, int ci, double* dense_f) {
    const long long N = (long long)c.hcases[ci].nx * c.hcases[ci].ny;
    const int g = blocks_for(N);
    switch (c.storage) {
        case LBM_STORE_F64: k_get_state<double><<<g, 256, 0, c.stream>>>(c.dcases, ci, c.flags, (const double*)c.f[c.cur], dense_f); break;
        case LBM_STORE_F32: k_get_state<float><<<g, 256, 0, c.stream>>>(c.dcases, ci, c.flags, (const float*)c.f[c.cur], dense_f); break;
        case LBM_STORE_F16_SHIFTED: k_get_state<__half><<<g, 256, 0, c.stream>>>(c.dcases, ci, c.flags, (const __half*)c.f[c.cur], dense_f); break;
        default: k_get_state<__nv_bfloat16><<<g, 256, 0, c.stream>>>(c.dcases, ci, c.flags, (const __nv_bfloat16*)c.f[c.cur], dense_f); break;
    }
    return cudaGetLastError();
}

}  // namespace lbm
