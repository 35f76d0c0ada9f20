// Fused time-step kernel of the two-component pseudopotential LBM (arXiv 2505.22256) and the
// kernels that read and write its state.
//
// State: one buffer per time level holds the post-collision populations f*_i^k of every case as
// [ny][9][pitch] pairs (f*_i^A, f*_i^B) of the storage type S: the nine direction planes of a lattice
// row lie next to each other, and one vector access moves both components of a direction.  Column x of a row lives at pair x + G; the G ghost columns
// on each side repeat the opposite edge when x is periodic, so a tensor box never has to wrap.
//
// One launch of k_step performs, for every fluid node x:
//   pull    f_i(x) = f*_i(x - e_i), or f*_opp(i)(x) across a blocked link (halfway bounce-back,
//           Sec. 3.5); open columns complete the entering populations (Sec. 3.3)
//   moments rho_k = sum_i f_i (Eq. 3), momentum sum_k sum_i f_i e_i (Eq. 4)
//   forces  cohesion on the eighth-order 24-node stencil (Eq. 8, Sec. 2.4); wall-list nodes take
//           second-layer values from their first-layer partner (Table 1) and add the adhesion
//           force of Eq. 9 with the local parameter of Eqs. 10-12; body force
//   collide u = (momentum + F/2) / rho (Eq. 5 with Guo's shift); f* = f + (f^eq - f)/tau +
//           (1 - 1/(2 tau)) F_i (Eqs. 1, 2, 6, 7), written to the other buffer.
//
// Work decomposition.  A work item is a column window of one case (T - 8 interior columns) by a
// chunk of rows.  One thread per window column marches down the rows.  Data path per row:
//   * the tensor engine loads the whole row of f* (all 9 planes of pairs, T columns) into a ring of
//     kSlots shared-memory slots, about four rows ahead, each slot completing on its mbarrier;
//   * every thread pulls its 18 populations from the three slots around the row, sums rho_A,
//     rho_B into a six-row density ring and keeps the populations in registers;
//   * after one barrier, each interior thread forms the row sums of the density gradient
//     (D1 = rho(x+1) - rho(x-1), D2, and the |dy| = 1, 2 weighted sums) and adds them into a
//     five-row window of partial gradients; the row two rows up is then complete, is collided and
//     written straight to global memory (one coalesced pair store per plane and warp).
// Densities of halo rows and columns are recomputed by neighbouring items; one launch needs no
// grid-wide synchronisation.
#include <math.h>

#include "lbm_internal.h"
#include "lbm_tma.cuh"

namespace lbm {

namespace {

// Rows of densities kept in shared memory.  Each row is written twice, at ring slot m and m + kRing,
// so the five consecutive rows a collision reads sit at consecutive slots from one base.
constexpr int kRing = 6;
// Threads per block of the step kernel = window columns = density ring row length: 128, or 64 for
// lattices too narrow to fill a 120-column window (both are built; the context picks one).
// Rows of f* resident or in flight in shared memory (>= 4), per storage type: three rows feed a
// pull, the rest are loads in flight.  FP32 takes six (on the seven-case sweep 0.1743 ms per launch
// against 0.1772 with five; seven slots leave room for the 64-column form only); the 16-bit types
// five (six measured 0.1533 against 0.1513 ms, four the same as five).
#ifndef LBM_SLOTS
#define LBM_SLOTS 6
#endif
#ifndef LBM_MIN_BLOCKS
#define LBM_MIN_BLOCKS 3
#endif
#ifndef LBM_SLOTS_16
#define LBM_SLOTS_16 5
#endif
template <class S>
constexpr int slots_of() {
    return sizeof(S) == 2 ? LBM_SLOTS_16 : LBM_SLOTS;
}
static_assert(LBM_SLOTS >= 4 && LBM_SLOTS_16 >= 4, "the pull of a row needs three resident rows plus one in flight");

template <class R>
using Params = CaseParams<R>;

#ifdef LBM_BOUNDS_CHECK
// Checked build (a sanitizer of this kernel's own indexing): every shared- and global-memory index
// of the step kernel is tested before use; an index outside its buffer sets bit 4 of the context's
// error word and the access is skipped.  The normal build compiles the tests away.
__device__ __forceinline__ bool idx_ok(bool ok, int* err) {
    if (!ok) atomicOr(err, 4);
    return ok;
}
#define LBM_IDX_OK(cond) idx_ok((cond), a.err)
#else
#define LBM_IDX_OK(cond) true
#endif

template <class R>
__device__ __forceinline__ Params<R> load_params(const DevCase& C) {
    return case_params<R>(C);
}

template <class R>
__device__ __forceinline__ R shift_of(const Params<R>& P, int k, int i) {
    return i == 0 ? P.sh0[k] : (i <= 4 ? P.sh1[k] : P.sh5[k]);
}

// Load the pair of direction i at p.  16-bit types hold h_i = f_i - w_i rho0; kAddShift adds the
// shift back (f_i), otherwise the pair stays h_i (the step kernel works on h, see collide()).
template <bool kAddShift, class S, class R>
__device__ __forceinline__ V2<R> load_v2(const Pair<S>* p, const Params<R>& P, int i) {
    V2<R> v;
    if constexpr (Store<S>::kShift && kAddShift) load_pair<S, R>(p, shift_of(P, 0, i), shift_of(P, 1, i), v.x, v.y);
    else load_pair<S, R>(p, (R)0, (R)0, v.x, v.y);
    return v;
}

// ------------------------------------------------------------------------------------------------
// Pull of one node's 18 populations.  rm / r0 / rp point at the rows y-1, y, y+1 (plane stride ps
// pairs, column c of the node, lattice row y); used with the shared-memory row slots (step kernel)
// and with global memory (state read-back).  The plain form assumes no blocked link and no open
// column.  Pin: the rarely used constants (inlet).
// ------------------------------------------------------------------------------------------------
template <bool kGeneral, class S, class R, class I, bool kAddShift = true>
__device__ __forceinline__ void pull(const Pair<S>* __restrict__ rm, const Pair<S>* __restrict__ r0,
                                     const Pair<S>* __restrict__ rp, I ps, int c, uint16_t fl, bool inlet, bool outlet,
                                     const Params<R>& P, const Params<R>& Pin, int y, V2<R> (&f)[9]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const Pair<S>* src;
        I off;
        if (i == 0) {
            src = r0;
            off = c;
        } else if (!kGeneral) {
            src = cy(i) > 0 ? rm : (cy(i) < 0 ? rp : r0);
            off = (I)i * ps + c - cx(i);
        } else {
            if (cx(i) > 0 && inlet) continue;  // entering through the inlet: set below
            const bool blocked = (fl >> (i - 1)) & 1u;
            int b = c;
            if (cx(i) < 0 && outlet) b = (fl & kOutletOwnBit) ? c : c - 1;  // copied from upstream
            const Pair<S>* nsrc = cy(i) > 0 ? rm : (cy(i) < 0 ? rp : r0);
            src = blocked ? r0 : nsrc;
            off = blocked ? (I)opp(i) * ps + b : (I)i * ps + b - cx(i);
        }
        f[i] = load_v2<kAddShift, S, R>(src + off, P, i);
    }
    if (kGeneral && inlet) {  // non-equilibrium bounce-back about f^eq(rho_in, (u_in(y), 0))
        R sc = (R)1;
        if (Pin.inlet_profile) {  // Poiseuille profile of peak u_in (Sec. 3.3)
            const R s = (R)y + (R)0.5;
            sc = Pin.prof_c * s * ((R)Pin.ny - s);
        }
        const V2<R> s2 = vbc<R>(sc), d1 = V2<R>{Pin.d1[0], Pin.d1[1]}, d5 = V2<R>{Pin.d5[0], Pin.d5[1]};
        f[1] = vfma(d1, s2, f[3]);
        f[5] = vfma(d5, s2, f[7]);
        f[8] = vfma(d5, s2, f[6]);
    }
    if (kGeneral && outlet && Pin.outlet) {
        // Zou-He density condition per component (Sec. 3.3 outflow, pressure reading), replacing the
        // f3, f6, f7 the copy rule pulled above: the node gets the densities rho_out and no momentum
        // along y, with non-equilibrium bounce-back along x.  The known populations give
        // rho u_x = f0 + f2 + f4 + 2 (f1 + f5 + f8) - rho_out; shifted storage holds h = f - w rho0,
        // whose known sum misses rho0 (those weights sum to 1).
        V2<R> known = vadd(vadd(vadd(f[0], f[2]), f[4]), vmul(vbc<R>(2), vadd(vadd(f[1], f[5]), f[8])));
        if constexpr (Store<S>::kShift && !kAddShift) known = vadd(known, V2<R>{Pin.rho0[0], Pin.rho0[1]});
        const V2<R> rho_ux = vsub(known, V2<R>{Pin.rho_out[0], Pin.rho_out[1]});
        const V2<R> dy = vsub(f[2], f[4]);
        const V2<R> c6 = vmul(vbc<R>(1.0 / 6.0), rho_ux);
        f[3] = vsub(f[1], vmul(vbc<R>(2.0 / 3.0), rho_ux));
        f[7] = vsub(vfma(vbc<R>(0.5), dy, f[5]), c6);
        f[6] = vsub(vsub(f[8], vmul(vbc<R>(0.5), dy)), c6);
    }
}

// Window column -> lattice column; -1 when it lies outside a wall boundary.
template <class R>
__device__ __forceinline__ int map_col(const Params<R>& P, int x) {
    if (x >= 0 && x < P.nx) return x;
    if (P.bc_x == kPeriodic) return ((x % P.nx) + P.nx) % P.nx;
    if (P.bc_x == kOpen) return x < 0 ? 0 : P.nx - 1;  // clamp to the boundary column
    return -1;
}

__device__ __forceinline__ int ring_slot(int r) { return (r + 2 * kRing) % kRing; }

// Per-thread diagnostics of the fields pass: FP64 sums (mass, momentum); extrema and the largest
// |u|^2 in the compute type (exact: min / max only compare), one square root at the end.
template <class R>
struct Diag {
    double mA, mB, px, py;
    R u2, aMin, aMax, bMin, bMax;
    int n;
    bool bad;
    __device__ void init() {
        mA = mB = px = py = 0.0;
        u2 = (R)0;
        aMin = bMin = (R)INFINITY;
        aMax = bMax = (R)-INFINITY;
        n = 0;
        bad = false;
    }
    // record layout (kDiagN doubles): mass_A, mass_B, mom_x, mom_y, umax, rhoA min/max, rhoB min/max,
    // fluid nodes, unstable flag
    __device__ void to_record(double* v) const {
        v[0] = mA;
        v[1] = mB;
        v[2] = px;
        v[3] = py;
        v[4] = sqrt((double)u2);
        v[5] = (double)aMin;
        v[6] = (double)aMax;
        v[7] = (double)bMin;
        v[8] = (double)bMax;
        v[9] = (double)n;
        v[10] = bad ? 1.0 : 0.0;
        for (int q = 11; q < kDiagN; ++q) v[q] = 0.0;
    }
};

template <class R>
struct RowState {
    V2<R> f[9];  // (f_i^A, f_i^B)
    uint16_t fl;
    uint32_t sub;
    R ax, ay;
};

// five-row window of partial gradients, both components per entry (index 0 = the row being
// collided)
template <class R>
struct Grad {
    V2<R> x[5], y[5];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int j = 0; j < 5; ++j) x[j] = y[j] = vbc<R>(0);
    }
    __device__ __forceinline__ void shift() {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            x[j] = x[j + 1];
            y[j] = y[j + 1];
        }
        x[4] = vbc<R>(0);
        y[4] = vbc<R>(0);
    }
};

// Row sums of row r at this thread's column, added into the gradient window (the five target rows
// around r, in marching order):
// Gx(T) = sum_dy [w(1+dy^2) D1(T+dy) + 2 w(4+dy^2) D2(T+dy)],
// Gy(T) = R1(T+1) - R1(T-1) + 2 (R2(T+2) - R2(T-2)),
// D1 = rho(x+1) - rho(x-1), D2 = rho(x+2) - rho(x-2), R_k = w(k^2) rho + w(1+k^2) S1 + w(4+k^2) S2
// with S1, S2 the sums of the same pairs.
template <class R>
__device__ __forceinline__ void add_row(const V2<R>* __restrict__ ring, int base, Grad<R>& g, R dir) {
    using V = V2<R>;
    const V m2 = ring[base - 2], m1 = ring[base - 1], c0 = ring[base], p1 = ring[base + 1], p2 = ring[base + 2];
    const V D1 = vsub(p1, m1), D2 = vsub(p2, m2), S1 = vadd(p1, m1), S2 = vadd(p2, m2);
    const V X0 = vfma(vbc<R>(w8(1)), D1, vmul(vbc<R>(2 * w8(4)), D2));
    const V X1 = vfma(vbc<R>(w8(2)), D1, vmul(vbc<R>(2 * w8(5)), D2));
    const V X2 = vfma(vbc<R>(w8(5)), D1, vmul(vbc<R>(2 * w8(8)), D2));
    // window slot j holds target row r - 2 dir + j dir, i.e. dy = r - target = dir (2 - j)
    const V R1 = vmul(vbc<R>(dir), vfma(vbc<R>(w8(1)), c0, vfma(vbc<R>(w8(2)), S1, vmul(vbc<R>(w8(5)), S2))));
    const V R2 =
        vmul(vbc<R>((R)2 * dir), vfma(vbc<R>(w8(4)), c0, vfma(vbc<R>(w8(5)), S1, vmul(vbc<R>(w8(8)), S2))));
    g.x[0] = vadd(g.x[0], X2);
    g.y[0] = vadd(g.y[0], R2);
    g.x[1] = vadd(g.x[1], X1);
    g.y[1] = vadd(g.y[1], R1);
    g.x[2] = vadd(g.x[2], X0);
    g.x[3] = vadd(g.x[3], X1);
    g.y[3] = vsub(g.y[3], R1);
    g.x[4] = vadd(g.x[4], X2);
    g.y[4] = vsub(g.y[4], R2);
}

// Second-layer substitution of Table 1 on top of the bulk gradient.  The row sums give
// sum_e w e rho(x+e) with rho = 0 at every non-fluid site; a substituted second-layer site x+e
// (non-fluid) takes rho(x + sign e) instead, i.e. adds w e rho(x + sign e).  Grouped by the
// first-layer partner p = sign e: an axis partner has one second-layer site (2 e_p), a diagonal
// partner three (2 e_p and the two knight moves), so the correction is sum_p c_p rho(x + e_p) with
// c_p built from the substitution bits (bit n-1 for stencil node n: 2 e_p is n = p + 8, the
// knights are n = p + 12 and n = p + 16).
template <class R>
struct SubCoef {
    R x[8], y[8];
};

template <class R>
__device__ __forceinline__ void substitution_coefficients(uint32_t sub, SubCoef<R>& c) {
#pragma unroll
    for (int p = 1; p <= 8; ++p) {
        const R ex = (R)cx(p), ey = (R)cy(p);
        const bool b1 = (sub >> (p + 7)) & 1u;
        if (p <= 4) {
            const R w = (R)(2.0 * w8(4));
            c.x[p - 1] = b1 ? w * ex : (R)0;
            c.y[p - 1] = b1 ? w * ey : (R)0;
        } else {
            const bool b2 = (sub >> (p + 11)) & 1u, b3 = (sub >> (p + 15)) & 1u;
            const R wd = (R)(2.0 * w8(8)), wk = (R)w8(5);
            const R a = b1 ? wd : (R)0, kx = b2 ? wk : (R)0, ky = b3 ? wk : (R)0;
            // 2 e_p w8(8) + (2 ex, ey) w8(5) + (ex, 2 ey) w8(5)
            c.x[p - 1] = ex * (a + (R)2 * kx + ky);
            c.y[p - 1] = ey * (a + kx + (R)2 * ky);
        }
    }
}

template <class R>
struct Grad2 {
    V2<R> x, y;  // (A, B) gradient corrections
};

// Gradient correction of a wall-list node (ring slots from sb0 = row y-2 at this column).
// open_edge: the node lies within two columns of an open boundary, where the ring holds clamped
// densities beyond the edge.  The step kernel inlines it where wall-list nodes are common and calls
// the out-of-line copy otherwise, so that warps without wall-list nodes keep a small loop.
template <class R, int TC>
__device__ __forceinline__ Grad2<R> substitution_correction(const V2<R>* __restrict__ ring, int sb0, uint32_t sub,
                                                            bool open_edge) {
    SubCoef<R> sc;
    substitution_coefficients<R>(sub, sc);
    Grad2<R> g{vbc<R>(0), vbc<R>(0)};
#pragma unroll
    for (int p = 1; p <= 8; ++p) {
        const V2<R> n = ring[sb0 + (cy(p) + 2) * TC + cx(p)];
        g.x = vfma(vbc<R>(sc.x[p - 1]), n, g.x);
        g.y = vfma(vbc<R>(sc.y[p - 1]), n, g.y);
    }
    if (open_edge) {
        // beyond an open column a second-layer site is not fluid, but the ring holds the clamped
        // boundary-column density there: take it out again
#pragma unroll
        for (int n = 8; n < 24; ++n) {
            if ((sub >> n) & 1u) {
                const V2<R> v = ring[sb0 + (s24y(n) + 2) * TC + s24x(n)];
                const double w = w8(s24x(n) * s24x(n) + s24y(n) * s24y(n));
                g.x = vsub(g.x, vmul(vbc<R>(w * s24x(n)), v));
                g.y = vsub(g.y, vmul(vbc<R>(w * s24y(n)), v));
            }
        }
    }
    return g;
}

template <class R, int TC>
__device__ __noinline__ Grad2<R> substitution_correction_call(const V2<R>* __restrict__ ring, int sb0, uint32_t sub,
                                                              bool open_edge) {
    return substitution_correction<R, TC>(ring, sb0, sub, open_edge);
}

// SRT collision with Guo forcing (Eqs. 1, 2, 6, 7), both components at once and written per pair
// of directions (e, -e).  With a = e.u, b = e.F_k, c_s^2 = 1/3:
//   f^eq_i = w rho (1 + 3a + 4.5a^2 - 1.5u^2),   F_i = w (3b - 3 u.F + 9ab)   (Guo's term, Eq. 7)
// and f*_i = (1 - om) f_i + om f^eq_i + cF F_i splits into the part even in e,
//   w [C0 + 4.5 a (om rho a + 2 cF b)],   C0 = om rho (1 - 1.5u^2) - 3 cF u.F,
// and the odd part 3 w (om rho a + cF b).  With P = om rho a + cF b:
//   f*_+- = (1 - om) f_+- + w (C0 + 4.5 a (P + cF b)) +- 3 w P,   f*_0 = (1 - om) f_0 + w_0 C0.
// Lanes are the components: rho, F, om and cF are (A, B) pairs; u is shared.
// Lattice weights in the compute type.  FP64 takes 4/9, 1/9, 1/36 rounded to double.  In FP32 those
// roundings sum to 1 + 7.5e-9, and since every step redistributes each node's mass with them, the
// mass of an FP32 run grew by that much per step (3e-4 after 50,000 steps); the FP32 set below
// sums to 1 exactly (w_0 + 4 w_1 + 4 w_5 = (14913082 + 4 * 3728270 + 3728270) 2^-25), and 4.5 w and
// 3 w are exact in FP32 too.  Each weight is within 7.5e-8 (relative) of its value.
template <class R>
struct LatW {
    static constexpr double w0 = 4.0 / 9.0, w1 = 1.0 / 9.0, w5 = 1.0 / 36.0;
};
template <>
struct LatW<float> {
    static constexpr double w0 = 14913082.0 / 33554432.0, w1 = 3728270.0 / 33554432.0, w5 = 3728270.0 / 134217728.0;
};

// Shifted form (kShifted, 16-bit storage): f = h + w rho0 with rho0 per component, and the result
// is stored as f* - w rho0.  Since (1 - om) w rho0 - w rho0 = -om w rho0 in every direction, the
// same formula applies to h with C0 replaced by C0 - om rho0 (om_rho0 below), so neither the
// loads nor the stores handle the shift per population.
template <class R, bool kShifted = false>
__device__ __forceinline__ void collide(const V2<R>* f, V2<R> rho, R ux, R uy, V2<R> Fx, V2<R> Fy, V2<R> om,
                                        V2<R> cf, V2<R> (&out)[9], V2<R> om_rho0 = V2<R>{}) {
    using V = V2<R>;
    const V om1 = vsub(vbc<R>(1), om);
    const V wr = vmul(om, rho);
    const V ux2 = vbc<R>(ux), uy2 = vbc<R>(uy);
    const V t = vfma(vbc<R>(-1.5), vfma(ux2, ux2, vmul(uy2, uy2)), vbc<R>(1));
    const V uF = vfma(uy2, Fy, vmul(ux2, Fx));
    V C0 = vfma(wr, t, vmul(vmul(vbc<R>(-3), cf), uF));
    if constexpr (kShifted) C0 = vsub(C0, om_rho0);
    out[0] = vfma(om1, f[0], vmul(vbc<R>(LatW<R>::w0), C0));
    const V s1 = vmul(vbc<R>(LatW<R>::w1), C0), s5 = vmul(vbc<R>(LatW<R>::w5), C0);
#pragma unroll
    for (int p = 0; p < 4; ++p) {  // pairs (1,3): e = (1,0); (2,4): (0,1); (5,7): (1,1); (6,8): (-1,1)
        const V a = p == 0 ? ux2 : p == 1 ? uy2 : p == 2 ? vadd(ux2, uy2) : vsub(uy2, ux2);
        const V b = p == 0 ? Fx : p == 1 ? Fy : p == 2 ? vadd(Fx, Fy) : vsub(Fy, Fx);
        const double w = p < 2 ? LatW<R>::w1 : LatW<R>::w5;
        const V cb = vmul(cf, b);
        const V P = vfma(wr, a, cb);
        const V sym = vfma(vbc<R>(4.5 * w), vmul(a, vadd(P, cb)), p < 2 ? s1 : s5);
        const V anti = vmul(vbc<R>(3.0 * w), P);
        const int ip = p < 2 ? 1 + p : 3 + p, im = p < 2 ? 3 + p : 5 + p;
        out[ip] = vfma(om1, f[ip], vadd(sym, anti));
        out[im] = vfma(om1, f[im], vsub(sym, anti));
    }
}

template <class S>
struct Layout {
    static constexpr int G = 4;
};

template <class S, class R>
struct SmemPlan {
    size_t pop_bytes, slot_bytes, ring_off, bar_off, total;
    __host__ __device__ explicit SmemPlan(int T) {
        pop_bytes = ((size_t)T * 9 * sizeof(Pair<S>) + 127) / 128 * 128;
        slot_bytes = pop_bytes + ((size_t)(T + 8) * sizeof(uint16_t) + 127) / 128 * 128;  // + the flags row
        ring_off = slots_of<S>() * slot_bytes;
        bar_off = (ring_off + 4 * kRing * (size_t)T * sizeof(R) + 7) / 8 * 8;
        total = bar_off + slots_of<S>() * 8;
    }
};

struct StepArgs {
    const DevCase* cases;
    const int4* items;
    int item_begin, item_end;
    const CUtensorMap* tmaps;  // [case][3]: rows of buffer 0, rows of buffer 1, rows of the flags
    int in_buf;                // buffer holding the current state
    void* fout;                // the other buffer
    const uint32_t* wsub;      // dense: substitution mask of wall-list nodes
    const void* wa;            // dense: adhesion vectors [2][nodes] in the compute type
    long long dense_total;
    long long pop_pairs;       // pairs in one population buffer (index checks of the checked build)
    int* err;
    int* sched;                // [0] next work item, [1] blocks finished; both back to 0 at exit
    int fields_global;         // fields mode: outputs indexed over all cases (d_off + y nx + x)
    double *o_rA, *o_rB, *o_ux, *o_uy, *diag_part;
};

// blocks per SM the launch bounds ask for: the same registers per thread at either width.  16-bit
// storage fits four 128-thread blocks per SM in shared memory (FP32 three, FP64 two), and needs the
// warps: its launch is bound by instruction latency, not by DRAM.
#ifndef LBM_MIN_BLOCKS_16
#define LBM_MIN_BLOCKS_16 4
#endif
template <class S, int T>
constexpr int step_min_blocks() {
    return (sizeof(S) == 8 ? 2 : sizeof(S) == 2 ? LBM_MIN_BLOCKS_16 : LBM_MIN_BLOCKS) * (128 / T);
}

template <class S, class R, bool kFields, bool kWallInline, int T>
__global__ void __launch_bounds__(T, step_min_blocks<S, T>()) k_step(StepArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int kSlots = slots_of<S>();
    constexpr int Wi = T - 8;  // interior columns of a window
    const int t = threadIdx.x;
    constexpr int G = Layout<S>::G;
    constexpr int BX = T;  // pairs per plane of a row slot
    const SmemPlan<S, R> plan(T);
    V2<R>* ring = reinterpret_cast<V2<R>*>(smem + plan.ring_off);  // (rho_A, rho_B) per column
    const uint32_t bar0 = smem_u32(smem + plan.bar_off);
    const uint32_t slot0 = smem_u32(smem);
    const uint32_t box_bytes = (uint32_t)((size_t)BX * 9 * sizeof(Pair<S>) + (size_t)(T + 8) * sizeof(uint16_t));
    const R* wax = reinterpret_cast<const R*>(a.wa);
    const R* way = wax + a.dense_total;

    if (t == 0) {
        for (int s = 0; s < kSlots; ++s) mbar_init(bar0 + 8 * s, 1);
        fence_mbar_init();
        fence_proxy_async_smem();
    }
    __syncthreads();

    // Row loads are numbered per block: load n goes to slot n % kSlots and completes phase
    // n / kSlots of that slot's barrier.  (slot, parity) of the next load to issue and of the next
    // load to wait for advance incrementally; so_m / so_0 / so_p are the byte offsets of the slots
    // of the last three rows waited for.
    int issue_slot = 0;
    uint32_t issue_par = 0, wait_par = 0;
    uint32_t wait_off = 0, wait_bar = bar0;
    uint32_t so_m = 0, so_0 = 0, so_p = 0;
    bool failed = false;

    // Work items are claimed from a counter, so blocks that share a busy SM take fewer of them.  The
    // claiming thread also copies the item's case parameters to shared memory: the rarely used ones
    // (adhesion, inlet) are read from there where needed instead of occupying registers.
    __shared__ int s_claim;
    __shared__ Params<R> s_par;
    auto claim = [&]() {
        const int k = atomicAdd(a.sched, 1);
        s_claim = k;
        if (a.item_begin + k < a.item_end) s_par = load_params<R>(a.cases[a.items[a.item_begin + k].x & 0x7FFFFFFF]);
    };
    if (t == 0) claim();
    __syncthreads();
    int it = a.item_begin + s_claim;
    while (it < a.item_end) {
        const int4 item = a.items[it];
        const int ci = item.x & 0x7FFFFFFF;       // case
        const int dir = item.x < 0 ? -1 : 1;      // marching direction (neighbouring chunks alternate)
        const DevCase& C = a.cases[ci];
        const Params<R> P = s_par;
        const int xs = item.y, y0 = item.z, y1 = item.w;
        const CUtensorMap* lmap = a.tmaps + 3 * ci + a.in_buf;
        const CUtensorMap* fmap = a.tmaps + 3 * ci + 2;
        const int x = xs - 2 + t;                 // this thread's window column
        const bool rcol = t < Wi + 4;             // computes densities
        const int X = rcol ? map_col(P, x) : -1;  // lattice column
        const int sc = (P.bc_x == kPeriodic ? x : X) - (xs - G);  // column inside a row slot
        const bool interior = t >= 2 && t < Wi + 2 && x < P.nx;
        const bool inlet = P.bc_x == kOpen && X == 0;
        const bool outlet = P.bc_x == kOpen && X == P.nx - 1;
        const int nload = (y1 + 2) - (y0 - 3) + 1;  // f* rows y0-3 .. y1+2
        const int r_first = dir > 0 ? y0 - 3 : y1 + 2, r_last = dir > 0 ? y1 + 2 : y0 - 3;
        Pair<S>* fo = reinterpret_cast<Pair<S>*>(a.fout) + C.f_off;

        auto wrap_row = [&](int r) -> int {
            if (P.bc_y == kPeriodic) r += r < 0 ? P.ny : (r >= P.ny ? -P.ny : 0);
            return r;
        };
        int next_row = r_first;  // next f* row to load (thread 0 only)
        // load the next row of f* and of the flags into the next slot (outside a wall: zeros)
        auto issue = [&]() {
            const uint32_t dst = slot0 + issue_slot * (uint32_t)plan.slot_bytes;
            mbar_expect_tx(bar0 + 8 * issue_slot, box_bytes);
            if constexpr (sizeof(S) == 8) tma_load_4d(dst, lmap, 0, xs, 0, wrap_row(next_row), bar0 + 8 * issue_slot);
            else tma_load_3d(dst, lmap, xs, 0, wrap_row(next_row), bar0 + 8 * issue_slot);
            tma_load_2d(dst + (uint32_t)plan.pop_bytes, fmap, xs, wrap_row(next_row), bar0 + 8 * issue_slot);
            next_row += dir;
            if (++issue_slot == kSlots) {
                issue_slot = 0;
                issue_par ^= 1u;
            }
        };
        auto wait_next = [&]() -> bool {  // wait for the oldest load not yet waited for
            const bool okw = mbar_wait_bounded(wait_bar, wait_par);
            so_m = so_0;
            so_0 = so_p;
            so_p = wait_off;
            wait_off += (uint32_t)plan.slot_bytes;
            wait_bar += 8;
            if (wait_bar == bar0 + 8 * kSlots) {
                wait_bar = bar0;
                wait_off = 0;
                wait_par ^= 1u;
            }
            return okw;
        };

        // densities of row r into the ring, populations of row r into st
        auto rho_row = [&](int r, int m, RowState<R>& st) -> bool {
            const bool ok = wait_next();  // f* row r+dir; rows r and r-dir sit in the two slots before
            const unsigned char* s0 = smem + so_0;
            // node flags of row r; rows beyond a wall boundary are solid
            st.fl = (rcol && (P.bc_y == kPeriodic || (r >= 0 && r < P.ny)))
                        ? reinterpret_cast<const uint16_t*>(s0 + plan.pop_bytes)[t + 6]
                        : kSolidBit;
            V2<R> rho2 = vbc<R>(0);
            const bool general = __any_sync(0xffffffffu, (st.fl & 0xFFu) != 0 || inlet || outlet);
            if (!(st.fl & kSolidBit) && LBM_IDX_OK(sc >= 1 && sc + 1 < BX)) {  // reads columns sc - 1 .. sc + 1
                const Pair<S>* rm = reinterpret_cast<const Pair<S>*>(smem + (dir > 0 ? so_m : so_p));
                const Pair<S>* r0 = reinterpret_cast<const Pair<S>*>(s0);
                const Pair<S>* rp = reinterpret_cast<const Pair<S>*>(smem + (dir > 0 ? so_p : so_m));
                if (general) pull<true, S, R, int, false>(rm, r0, rp, BX, sc, st.fl, inlet, outlet, P, s_par, r, st.f);
                else pull<false, S, R, int, false>(rm, r0, rp, BX, sc, st.fl, inlet, outlet, P, s_par, r, st.f);
                // rho_k = sum_i f_i as a balanced tree (short dependency chains); 16-bit storage sums
                // h_i = f_i - w_i rho0 and adds rho0 once (the weights sum to 1)
                const V2<R>* f = st.f;
                rho2 = vadd(vadd(vadd(f[0], f[1]), vadd(f[2], f[3])),
                            vadd(vadd(f[4], f[5]), vadd(f[6], vadd(f[7], f[8]))));
                if constexpr (Store<S>::kShift) rho2 = vadd(rho2, V2<R>{s_par.rho0[0], s_par.rho0[1]});
                if (st.fl & kWallBit) {
                    const long long o = C.d_off + (long long)wrap_row(r) * P.nx + X;
                    if (LBM_IDX_OK(o >= 0 && o < a.dense_total)) {
                        st.sub = __ldg(a.wsub + o);
                        st.ax = __ldg(wax + o);
                        st.ay = __ldg(way + o);
                    }
                }
            }
            const int s = m * T + t;
            if (LBM_IDX_OK(m >= 0 && m < kRing)) {
                ring[s] = rho2;
                ring[s + kRing * T] = rho2;
            }
            return ok;
        };

        // collide row y (state st, complete gradient g[0]) and store it
        // lo: ring slot of row y - 2 (rows y-2 .. y+2 sit at slots lo .. lo+4)
        auto update_row = [&](int y, int lo, const RowState<R>& st, const Grad<R>& g, Diag<R>& dg) {
            if (!interior || (st.fl & kSolidBit)) {
                if constexpr (kFields) {
                    const long long o = (a.fields_global ? C.d_off : 0) + (long long)y * P.nx + x;
                    const long long on = a.fields_global ? a.dense_total : (long long)P.nx * P.ny;
                    if (interior && a.o_rA && LBM_IDX_OK(o >= 0 && o < on)) {
                        a.o_rA[o] = 0.0;
                        a.o_rB[o] = 0.0;
                        if (a.o_ux) {
                            a.o_ux[o] = 0.0;
                            a.o_uy[o] = 0.0;
                        }
                    }
                }
                return;
            }
            if (!LBM_IDX_OK(lo >= 0 && lo < kRing)) return;  // rows lo .. lo + 4, columns t - 2 .. t + 2
            const int sb0 = lo * T + t;
            const V2<R> r2 = ring[sb0 + 2 * T];
            const R rA = r2.x, rB = r2.y;
            V2<R> gx = g.x[0], gy = g.y[0];
            const bool wall = (st.fl & kWallBit) != 0;
            if (wall) {
                const bool open_edge = P.bc_x == kOpen && (X < 2 || X >= P.nx - 2);
                Grad2<R> c2;
                if constexpr (kWallInline) c2 = substitution_correction<R, T>(ring, sb0, st.sub, open_edge);
                else c2 = substitution_correction_call<R, T>(ring, sb0, st.sub, open_edge);
                gx = vadd(gx, c2.x);
                gy = vadd(gy, c2.y);
            }
            // cohesion: each component is pushed by the other's pseudopotential gradient (Eq. 8)
            const R nGA = -P.G * rA, nGB = -P.G * rB;
            R FAx = nGA * gx.y, FAy = nGA * gy.y;
            R FBx = nGB * gx.x, FBy = nGB * gy.x;
            if (wall) {  // adhesion (Eq. 9), G_w1 local in the improved scheme (Eqs. 10, 12)
                R GA;
                const Params<R>& Q = s_par;
                if (Q.mode == 1) {
                    const R re = (rA - rB) / (rA + rB);
                    R h;
                    if (re > Q.delta) h = Q.lam;
                    else if (re > (R)0) h = Q.s1 + re * (Q.s2 + re * Q.s3);
                    else if (re > -Q.delta) h = Q.s1 + re * (Q.t2 + re * Q.t3);
                    else h = (R)1;
                    GA = Q.Gw2 * h;
                } else {
                    GA = Q.lam * Q.Gw2;
                }
                FAx -= GA * rA * st.ax;
                FAy -= GA * rA * st.ay;
                FBx -= s_par.Gw2 * rB * st.ax;
                FBy -= s_par.Gw2 * rB * st.ay;
            }
            FAx += rA * P.gx;
            FAy += rA * P.gy;
            FBx += rB * P.gx;
            FBy += rB * P.gy;
            const V2<R>* f = st.f;
            // momentum per component, then summed over the components (Eq. 4)
            const V2<R> d13 = vsub(f[1], f[3]), d24 = vsub(f[2], f[4]), d57 = vsub(f[5], f[7]), d68 = vsub(f[6], f[8]);
            const V2<R> mx2 = vadd(d13, vsub(d57, d68)), my2 = vadd(d24, vadd(d57, d68));
            const R mx = mx2.x + mx2.y, my = my2.x + my2.y;
            const R rho = rA + rB;
            const R inv = recip(rho);
            const R ux = (mx + (R)0.5 * (FAx + FBx)) * inv;
            const R uy = (my + (R)0.5 * (FAy + FBy)) * inv;
            if constexpr (kFields) {
                const long long o = (a.fields_global ? C.d_off : 0) + (long long)y * P.nx + x;
                const long long on = a.fields_global ? a.dense_total : (long long)P.nx * P.ny;
                if (a.o_rA && LBM_IDX_OK(o >= 0 && o < on)) {  // null outputs: partial sums only
                    a.o_rA[o] = (double)rA;
                    a.o_rB[o] = (double)rB;
                    if (a.o_ux) {  // null velocity outputs: densities only
                        a.o_ux[o] = (double)ux;
                        a.o_uy[o] = (double)uy;
                    }
                }
                if (a.diag_part) {  // null: densities only
                    const double drho = (double)rho;
                    dg.mA += (double)rA;
                    dg.mB += (double)rB;
                    dg.px += drho * (double)ux;
                    dg.py += drho * (double)uy;
                    const R u2 = ux * ux + uy * uy;
                    dg.u2 = fmax(dg.u2, u2);
                    dg.aMin = fmin(dg.aMin, rA);
                    dg.aMax = fmax(dg.aMax, rA);
                    dg.bMin = fmin(dg.bMin, rB);
                    dg.bMax = fmax(dg.bMax, rB);
                    ++dg.n;
                    if (!(rA > (R)0) || !(rB > (R)0) || !isfinite(u2) || !isfinite(rA) || !isfinite(rB)) dg.bad = true;
                }
            } else {
                V2<R> o[9];
                collide<R, Store<S>::kShift>(f, r2, ux, uy, V2<R>{FAx, FBx}, V2<R>{FAy, FBy},
                                             V2<R>{P.omega[0], P.omega[1]}, V2<R>{P.cF[0], P.cF[1]}, o,
                                             V2<R>{s_par.om_rho0[0], s_par.om_rho0[1]});
                Pair<S>* out = fo + (long long)y * P.row + x + G;
                // the row's nine pairs at columns x + G of planes 0..8 lie inside the case's block
                const long long e0 = C.f_off + (long long)y * P.row + x + G;
                if (!LBM_IDX_OK(y >= 0 && y < P.ny && x + G >= 0 && x + G < P.plane && e0 >= 0 &&
                                e0 + 8 * P.plane < a.pop_pairs))
                    return;
#pragma unroll
                for (int i = 0; i < 9; ++i) store_pair<S, R>(out + i * P.plane, o[i].x, o[i].y);
                if (P.bc_x == kPeriodic && (x < G || x >= P.nx - G)) {  // copy for the periodic wrap
                    const int gx = x < G ? x + P.nx + G : x - P.nx + G;
                    if (!LBM_IDX_OK(gx >= 0 && gx < P.plane)) return;
                    Pair<S>* gout = fo + (long long)y * P.row + gx;
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        store_pair<S, R>(gout, o[i].x, o[i].y);
                        gout += P.plane;
                    }
                }
            }
        };

        Diag<R> dg;
        if constexpr (kFields) dg.init();
        Grad<R> g;
        g.zero();
        RowState<R> s0, s1, s2;
        s0.sub = s1.sub = s2.sub = 0;
        s0.ax = s0.ay = s1.ax = s1.ay = s2.ax = s2.ay = (R)0;

        if (t == 0) {
            const int n0 = nload < kSlots ? nload : kSlots;
            for (int k = 0; k < n0; ++k) issue();
        }
        bool ok = wait_next();   // f* row r_first
        ok = wait_next() && ok;  // f* row r_first + dir
        ok = !__syncthreads_or(!ok);  // the whole block takes a failed wait's exit path together
        const R rdir = (R)dir;

        // One row of the march: densities of row q into `cur`, barrier, refill of the slot that
        // held f* row q-dir, gradient row sums of row q, collision of row q-2 dir (`old`).
        auto iter = [&](int q, RowState<R>& old, RowState<R>& cur) -> bool {
            const int mq = ring_slot(q);
            const bool mine = rho_row(q, mq, cur);
            if (__syncthreads_or(!mine)) return false;
            if (t == 0 && (dir > 0 ? next_row <= r_last : next_row >= r_last)) issue();  // slot of q-dir is free
            if (interior && LBM_IDX_OK(mq >= 0 && mq < kRing && t >= 2 && t + 2 < T)) {
                add_row<R>(ring, mq * T + t, g, rdir);
            }
            const int y = q - 2 * dir;
            // slot of row y - 2: q - 4 when marching up (= mq + 2 mod kRing), q itself marching down
            if (y >= y0 && y < y1) update_row(y, dir > 0 ? (mq + 2 < kRing ? mq + 2 : mq + 2 - kRing) : mq, old, g, dg);
            g.shift();
            return true;
        };

        // row states rotate with period three: row q goes into cur, row q-2 dir is old
        int q = dir > 0 ? y0 - 2 : y1 + 1;
        int left = (y1 - y0) + 4;  // rows of densities to produce
        while (ok && left > 0) {
            ok = iter(q, s0, s2);
            q += dir;
            if (!ok || --left == 0) break;
            ok = iter(q, s1, s0);
            q += dir;
            if (!ok || --left == 0) break;
            ok = iter(q, s2, s1);
            q += dir;
            --left;
        }
        if (!ok) {
            failed = true;
            break;
        }
        __syncthreads();  // every thread is done with the slots before the next item refills them

        if (kFields && a.diag_part) {
            __shared__ double red[8][kDiagN];
            const int lane = t & 31, warp = t >> 5;
            double rec[kDiagN];
            dg.to_record(rec);
#pragma unroll
            for (int qq = 0; qq < kDiagN; ++qq) {
                double v = rec[qq];
                for (int off = 16; off > 0; off >>= 1) {
                    const double o = __shfl_xor_sync(0xffffffffu, v, off);
                    v = (qq == 4 || qq == 6 || qq == 8 || qq == 10) ? fmax(v, o) : (qq == 5 || qq == 7) ? fmin(v, o) : v + o;
                }
                if (lane == 0) red[warp][qq] = v;
            }
            __syncthreads();
            if (t == 0) {
                const int nw = (T + 31) >> 5;
                for (int qq = 0; qq < kDiagN; ++qq) {
                    double v = red[0][qq];
                    for (int w2 = 1; w2 < nw; ++w2) {
                        const double o = red[w2][qq];
                        v = (qq == 4 || qq == 6 || qq == 8 || qq == 10) ? fmax(v, o) : (qq == 5 || qq == 7) ? fmin(v, o) : v + o;
                    }
                    a.diag_part[(long long)it * kDiagN + qq] = v;
                }
            }
            __syncthreads();
        }
        if (t == 0) claim();  // every thread is past the previous claim and its parameters
        __syncthreads();
        it = a.item_begin + s_claim;
    }
    if (t == 0) {
        // the last block to finish sees every claim made and resets the counters for the next launch
        __threadfence();
        if (atomicAdd(a.sched + 1, 1) == (int)gridDim.x - 1) {
            atomicExch(a.sched, 0);
            atomicExch(a.sched + 1, 0);
        }
    }
    if (failed && t == 0) {
        atomicOr(a.err, 1);
        // give loads still in flight a bounded time to land before the block leaves
        const unsigned long long t0 = clock64();
        while (clock64() - t0 < 200000000ULL) {
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Sliding walls (Sec. 3.1, Couette flow), applied to a freshly written post-collision buffer.  At a
// node of row 0 (ny-1) of a walled y, the diagonals 7, 8 (5, 6) leave across the wall and come back
// only to the node itself, by halfway bounce-back, as f_opp(i) = f*_i + 2 w rho_k (e_opp(i) . u_w) /
// c_s^2 with rho_k = sum_j f*_j at the node.  Storing them reflected lets the pull take every
// bounce-back as it is, so the step kernel carries no code for it.  One thread per column of the
// two wall rows of each listed case (blockIdx.y = 2 * list index + upper); ghost copies of periodic
// x are rewritten with the node.
// ------------------------------------------------------------------------------------------------
template <class S>
__global__ void k_sliding_walls(const DevCase* __restrict__ cases, const int* __restrict__ list,
                                const uint16_t* __restrict__ flags_all, Pair<S>* __restrict__ buf_all) {
    using R = typename ComputeOf<S>::type;
    constexpr int G = Layout<S>::G;
    const int ci = list[blockIdx.y >> 1];
    const bool upper = blockIdx.y & 1;
    const DevCase& C = cases[ci];
    const int X = blockIdx.x * blockDim.x + threadIdx.x;
    if (X >= C.nx) return;
    const int Y = upper ? C.ny - 1 : 0;
    if (flags_all[C.d_off + (long long)Y * C.nx + X] & kSolidBit) return;
    const double uw = upper ? C.u_wall[1] : C.u_wall[0];
    if (uw == 0.0) return;
    const long long plane = C.pitch;
    Pair<S>* p = buf_all + C.f_off + (long long)Y * 9 * C.pitch + X + G;
    const int ip = upper ? 6 : 7, im = upper ? 5 : 8;  // returning as e_x = +1 / -1
    auto shift = [&](int k, int j) -> R { return Store<S>::kShift ? (R)(wq(j) * C.rho0[k]) : (R)0; };
    R v[2][9];
    R rho[2] = {(R)0, (R)0};
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        load_pair<S, R>(p + j * plane, shift(0, j), shift(1, j), v[0][j], v[1][j]);
        rho[0] += v[0][j];
        rho[1] += v[1][j];
    }
    const int q[2] = {ip, im};
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        R o[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const R a = (R)(6.0 * wq(5)) * rho[k] * (R)uw;
            o[k] = (m == 0 ? v[k][ip] + a : v[k][im] - a) - shift(k, q[m]);
        }
        Pair<S>* pq = p + q[m] * plane;
        store_pair<S, R>(pq, o[0], o[1]);
        if (C.bc_x == kPeriodic && X < G) store_pair<S, R>(pq + C.nx, o[0], o[1]);
        if (C.bc_x == kPeriodic && X >= C.nx - G) store_pair<S, R>(pq - C.nx, o[0], o[1]);
    }
}

// ------------------------------------------------------------------------------------------------
// State transfer kernels (dense doubles [2][9][ny][nx] <-> the post-collision buffer)
// ------------------------------------------------------------------------------------------------
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

// Post-streaming populations -> post-collision buffer: the inverse of the pull, so that the next
// pull reproduces f exactly (up to the storage rounding).  Ghost columns are filled as well.
template <class S>
__global__ void k_set_state(const DevCase* __restrict__ cases, int c, const uint16_t* __restrict__ flags_all,
                            const double* __restrict__ f, Pair<S>* __restrict__ out_all) {
    using R = typename ComputeOf<S>::type;
    constexpr int G = Layout<S>::G;
    const DevCase C = cases[c];
    const long long N = (long long)C.nx * C.ny;
    const long long plane = C.pitch;
    Pair<S>* out = out_all + C.f_off;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N; s += (long long)gridDim.x * blockDim.x) {
        const int X = (int)(s % C.nx), Y = (int)(s / C.nx);
        const uint16_t fl = flags_all[C.d_off + s];
        const long long o = (long long)Y * 9 * C.pitch + X + G;
        R ov[2][9];
        for (int k = 0; k < 2; ++k) {
            double vs[9];
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
                }
                vs[i] = v;
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                double v = vs[i];
                if (!(fl & kSolidBit)) {
                    if constexpr (Store<S>::kShift) v -= wq(i) * C.rho0[k];
                }
                ov[k][i] = (R)v;
            }
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            Pair<S>* p = out + i * plane;
            store_pair<S, R>(p + o, ov[0][i], ov[1][i]);
            if (C.bc_x == kPeriodic && X < G) store_pair<S, R>(p + o + C.nx, ov[0][i], ov[1][i]);
            if (C.bc_x == kPeriodic && X >= C.nx - G) store_pair<S, R>(p + o - C.nx, ov[0][i], ov[1][i]);
        }
    }
}

// Post-collision buffer -> post-streaming populations (dense doubles), 0 at solid nodes.
template <class S>
__global__ void k_get_state(const DevCase* __restrict__ cases, int c, const uint16_t* __restrict__ flags_all,
                            const Pair<S>* __restrict__ fin_all, double* __restrict__ f) {
    using R = typename ComputeOf<S>::type;
    constexpr int G = Layout<S>::G;
    const DevCase C = cases[c];
    const Params<R> P = load_params<R>(C);
    const long long N = (long long)C.nx * C.ny;
    const Pair<S>* fin = fin_all + C.f_off;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N; s += (long long)gridDim.x * blockDim.x) {
        const int X = (int)(s % C.nx), Y = (int)(s / C.nx);
        const uint16_t fl = flags_all[C.d_off + s];
        V2<R> v[9];
        if (fl & kSolidBit) {
#pragma unroll
            for (int i = 0; i < 9; ++i) v[i] = vbc<R>(0);
        } else {
            // rows beyond a wall are reached only through blocked links; clamping keeps the unused
            // row pointer inside the buffer
            const int ym = Y - 1 < 0 ? (C.bc_y == kPeriodic ? C.ny - 1 : 0) : Y - 1;
            const int yp = Y + 1 >= C.ny ? (C.bc_y == kPeriodic ? 0 : C.ny - 1) : Y + 1;
            const bool inlet = C.bc_x == kOpen && X == 0, outlet = C.bc_x == kOpen && X == C.nx - 1;
            const long long rs = 9LL * C.pitch;
            pull<true, S, R, long long>(fin + ym * rs, fin + Y * rs, fin + yp * rs, P.plane, X + G, fl, inlet, outlet, P,
                                        P, Y, v);
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            f[(long long)i * N + s] = (double)v[i].x;
            f[(long long)(9 + i) * N + s] = (double)v[i].y;
        }
    }
}

// Per-case reduction of the per-item partials in item order (one warp; deterministic).  c < 0:
// block b reduces case b.
__global__ void k_diag_reduce(const DevCase* __restrict__ cases, int c, const double* __restrict__ part,
                              double* __restrict__ out) {
    if (c < 0) c = blockIdx.x;
    const DevCase C = cases[c];
    const int lane = threadIdx.x;
    double v[kDiagN];
    for (int q = 0; q < kDiagN; ++q) v[q] = (q == 5 || q == 7) ? INFINITY : (q == 4 || q == 6 || q == 8) ? -INFINITY : 0.0;
    for (int it = C.item_begin + lane; it < C.item_end; it += 32)
        for (int q = 0; q < kDiagN; ++q) {
            const double o = part[(long long)it * kDiagN + q];
            v[q] = (q == 4 || q == 6 || q == 8 || q == 10) ? fmax(v[q], o) : (q == 5 || q == 7) ? fmin(v[q], o) : v[q] + o;
        }
    for (int q = 0; q < kDiagN; ++q) {
        double xv = v[q];
        for (int off = 16; off > 0; off >>= 1) {
            const double o = __shfl_xor_sync(0xffffffffu, xv, off);
            xv = (q == 4 || q == 6 || q == 8 || q == 10) ? fmax(xv, o) : (q == 5 || q == 7) ? fmin(xv, o) : xv + o;
        }
        if (lane == 0) out[(long long)c * kDiagN + q] = xv;
    }
}

template <class S, int T>
void* kernel_ptr(int variant) {
    using R = typename ComputeOf<S>::type;
    return variant == 2 ? (void*)k_step<S, R, true, false, T>
                        : (variant == 1 ? (void*)k_step<S, R, false, true, T> : (void*)k_step<S, R, false, false, T>);
}

template <class S>
void* kernel_ptr_w(int variant, int threads) {
    return threads == 64 ? kernel_ptr<S, 64>(variant) : kernel_ptr<S, 128>(variant);
}

// variant 0: step, wall path out of line; 1: step, wall path inline; 2: fields pass
void* step_kernel(int storage, int variant, int threads) {
    switch (storage) {
        case LBM_STORE_F64: return kernel_ptr_w<double>(variant, threads);
        case LBM_STORE_F32: return kernel_ptr_w<float>(variant, threads);
        case LBM_STORE_F16_SHIFTED: return kernel_ptr_w<__half>(variant, threads);
        default: return kernel_ptr_w<__nv_bfloat16>(variant, threads);
    }
}

template <class S>
size_t smem_for(int threads) {
    using R = typename ComputeOf<S>::type;
    return SmemPlan<S, R>(threads).total;
}

StepArgs make_args(Ctx& c, int ib, int ie, double* o4[4], double* part) {
    StepArgs a;
    a.cases = c.dcases;
    a.items = c.items;
    a.item_begin = ib;
    a.item_end = ie;
    a.tmaps = c.tmaps;
    a.in_buf = c.cur;
    a.fout = c.f[1 - c.cur];
    a.wsub = c.wsub;
    a.wa = c.wa;
    a.dense_total = c.dense_elems;
    a.pop_pairs = c.pop_elems / 2;
    a.err = c.err;
    a.sched = c.sched;
    a.fields_global = 0;
    a.o_rA = o4[0];
    a.o_rB = o4[1];
    a.o_ux = o4[2];
    a.o_uy = o4[3];
    a.diag_part = part;
    return a;
}

template <class S, int T>
cudaError_t launch_step_w(const Ctx& c, const StepArgs& a, cudaStream_t s, bool fields, int grid) {
    using R = typename ComputeOf<S>::type;
    const size_t smem = smem_for<S>(T);
    if (fields) k_step<S, R, true, false, T><<<grid, T, smem, s>>>(a);
    else if (c.wall_inline) k_step<S, R, false, true, T><<<grid, T, smem, s>>>(a);
    else k_step<S, R, false, false, T><<<grid, T, smem, s>>>(a);
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_step_t(Ctx& c, const StepArgs& a, cudaStream_t s, bool fields, int grid) {
    if (c.block_threads == 128) return launch_step_w<S, 128>(c, a, s, fields, grid);
    if (c.block_threads == 64) return launch_step_w<S, 64>(c, a, s, fields, grid);
    return cudaErrorInvalidConfiguration;
}

cudaError_t dispatch(Ctx& c, const StepArgs& a, cudaStream_t s, bool fields, int grid) {
    switch (c.storage) {
        case LBM_STORE_F64: return launch_step_t<double>(c, a, s, fields, grid);
        case LBM_STORE_F32: return launch_step_t<float>(c, a, s, fields, grid);
        case LBM_STORE_F16_SHIFTED: return launch_step_t<__half>(c, a, s, fields, grid);
        default: return launch_step_t<__nv_bfloat16>(c, a, s, fields, grid);
    }
}

int blocks_for(long long n) { return (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096); }

}  // namespace

int ghost_cols(int) { return Layout<float>::G; }
int box_extra_cols(int) { return 0; }

int step_smem_bytes(int storage, int threads) {
    switch (storage) {
        case LBM_STORE_F64: return (int)smem_for<double>(threads);
        case LBM_STORE_F32: return (int)smem_for<float>(threads);
        case LBM_STORE_F16_SHIFTED: return (int)smem_for<__half>(threads);
        default: return (int)smem_for<__nv_bfloat16>(threads);
    }
}

cudaError_t step_occupancy(int storage, int threads, int* blocks_per_sm) {
    const int bytes = step_smem_bytes(storage, threads);
    for (int v = 0; v < 3; ++v) {
        cudaError_t e =
            cudaFuncSetAttribute(step_kernel(storage, v, threads), cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
    }
    // the most restrictive of the three variants sets the resident blocks
    int m = 1 << 30;
    for (int v = 0; v < 3; ++v) {
        int b = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, step_kernel(storage, v, threads), threads, bytes);
        if (e != cudaSuccess) return e;
        m = b < m ? b : m;
    }
    *blocks_per_sm = m;
    return cudaSuccess;
}

cudaError_t launch_step(Ctx& c, int in_buf, cudaStream_t s) {
    double* o4[4] = {nullptr, nullptr, nullptr, nullptr};
    StepArgs a = make_args(c, 0, c.nitems, o4, nullptr);
    a.in_buf = in_buf;
    a.fout = c.f[1 - in_buf];
    cudaError_t e = dispatch(c, a, s, false, c.grid_blocks);
    if (e != cudaSuccess || c.slide_n == 0) return e;
    const dim3 grid((unsigned)((c.slide_max_nx + 127) / 128), (unsigned)(2 * c.slide_n));
    switch (c.storage) {
        case LBM_STORE_F64: k_sliding_walls<double><<<grid, 128, 0, s>>>(c.dcases, c.slide_list, c.flags, (Pair<double>*)a.fout); break;
        case LBM_STORE_F32: k_sliding_walls<float><<<grid, 128, 0, s>>>(c.dcases, c.slide_list, c.flags, (Pair<float>*)a.fout); break;
        case LBM_STORE_F16_SHIFTED: k_sliding_walls<__half><<<grid, 128, 0, s>>>(c.dcases, c.slide_list, c.flags, (Pair<__half>*)a.fout); break;
        default: k_sliding_walls<__nv_bfloat16><<<grid, 128, 0, s>>>(c.dcases, c.slide_list, c.flags, (Pair<__nv_bfloat16>*)a.fout); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_fields(Ctx& c, int ci, double* rhoA, double* rhoB, double* ux, double* uy, bool diag) {
    const DevCase& C = c.hcases[ci];
    const long long N = (long long)C.nx * C.ny;
    double* o4[4] = {rhoA ? rhoA : c.fields, rhoB ? rhoB : c.fields + N, ux ? ux : c.fields + 2 * N,
                     uy ? uy : c.fields + 3 * N};
    const int n = C.item_end - C.item_begin;
    const int grid = n < c.grid_blocks ? n : c.grid_blocks;
    (void)diag;
    StepArgs a = make_args(c, C.item_begin, C.item_end, o4, c.diag_part);
    return dispatch(c, a, c.stream, true, grid);
}

cudaError_t launch_diag_reduce(Ctx& c, int ci) {
    k_diag_reduce<<<1, 32, 0, c.stream>>>(c.dcases, ci, c.diag_part, c.diag_out);
    return cudaGetLastError();
}

cudaError_t launch_fields_all(Ctx& c, double* rhoA_all, double* rhoB_all, double* ux_all, double* uy_all) {
    double* o4[4] = {rhoA_all, rhoB_all, ux_all, uy_all};
    const int n = c.nitems_all - c.nitems;
    const int grid = n < c.grid_blocks ? n : c.grid_blocks;
    StepArgs a = make_args(c, c.nitems, c.nitems_all, o4, nullptr);
    a.fields_global = 1;
    return dispatch(c, a, c.stream, true, grid);
}

cudaError_t launch_densities_all(Ctx& c, double* rhoA_all, double* rhoB_all) {
    return launch_fields_all(c, rhoA_all, rhoB_all, nullptr, nullptr);
}

cudaError_t launch_diag_all(Ctx& c, double* rhoA_all, double* rhoB_all) {
    double* o4[4] = {rhoA_all, rhoB_all, nullptr, nullptr};  // densities too when given (all cases)
    const int n = c.nitems_all - c.nitems;
    const int grid = n < c.grid_blocks ? n : c.grid_blocks;
    StepArgs a = make_args(c, c.nitems, c.nitems_all, o4, c.diag_part);
    a.fields_global = 1;
    cudaError_t e = dispatch(c, a, c.stream, true, grid);
    if (e != cudaSuccess) return e;
    k_diag_reduce<<<(unsigned)c.hcases.size(), 32, 0, c.stream>>>(c.dcases, -1, c.diag_part, c.diag_out);
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
        case LBM_STORE_F64: k_set_state<double><<<g, 256, 0, c.stream>>>(c.dcases, ci, c.flags, dense_f, (Pair<double>*)c.f[c.cur]); break;
        case LBM_STORE_F32: k_set_state<float><<<g, 256, 0, c.stream>>>(c.dcases, ci, c.flags, dense_f, (Pair<float>*)c.f[c.cur]); break;
        case LBM_STORE_F16_SHIFTED: k_set_state<__half><<<g, 256, 0, c.stream>>>(c.dcases, ci, c.flags, dense_f, (Pair<__half>*)c.f[c.cur]); break;
        default: k_set_state<__nv_bfloat16><<<g, 256, 0, c.stream>>>(c.dcases, ci, c.flags, dense_f, (Pair<__nv_bfloat16>*)c.f[c.cur]); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_get_state(Ctx& c, int ci, double* dense_f) {
    const long long N = (long long)c.hcases[ci].nx * c.hcases[ci].ny;
    const int g = blocks_for(N);
    switch (c.storage) {
        case LBM_STORE_F64: k_get_state<double><<<g, 256, 0, c.stream>>>(c.dcases, ci, c.flags, (const Pair<double>*)c.f[c.cur], dense_f); break;
        case LBM_STORE_F32: k_get_state<float><<<g, 256, 0, c.stream>>>(c.dcases, ci, c.flags, (const Pair<float>*)c.f[c.cur], dense_f); break;
        case LBM_STORE_F16_SHIFTED: k_get_state<__half><<<g, 256, 0, c.stream>>>(c.dcases, ci, c.flags, (const Pair<__half>*)c.f[c.cur], dense_f); break;
        default: k_get_state<__nv_bfloat16><<<g, 256, 0, c.stream>>>(c.dcases, ci, c.flags, (const Pair<__nv_bfloat16>*)c.f[c.cur], dense_f); break;
    }
    return cudaGetLastError();
}

}  // namespace lbm
