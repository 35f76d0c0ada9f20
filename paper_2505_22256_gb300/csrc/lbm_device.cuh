// Device-side definitions shared by the library's kernels: lattice tables, the per-case
// descriptor, node flags and the storage-type traits.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

// ------------------------------------------------------------------------------------------------
// Boundary kinds (mirror lbm_bc) and node flags.
// ------------------------------------------------------------------------------------------------
enum : int { kPeriodic = 0, kWall = 1, kOpen = 2 };

// uint16 per node:
//   bits 0-7  link i = bit+1 is blocked: the node upstream along e_i (x - e_i) is not fluid, so
//             f_i arrives by halfway bounce-back of f*_opp(i) at the node itself.  At an outflow
//             node the bits of the entering populations (e_x < 0) describe the links of the
//             node one column upstream, from which those populations are copied.
//   bit 8     solid node
//   bit 9     wall-list node: the 24-node stencil reaches a non-fluid site
//   bit 10    outflow node whose upstream neighbour is solid: entering populations bounce back
//   bit 11    a non-fluid site lies within three cells (Chebyshev) -- excluded from the interface
//             points of the contact-angle measurement
constexpr uint16_t kSolidBit = 1u << 8;
constexpr uint16_t kWallBit = 1u << 9;
constexpr uint16_t kOutletOwnBit = 1u << 10;
constexpr uint16_t kNearSolidBit = 1u << 11;

// ------------------------------------------------------------------------------------------------
// D2Q9 (Sec. 2.1): 0 rest; 1-4 = (1,0),(0,1),(-1,0),(0,-1); 5-8 = (1,1),(-1,1),(-1,-1),(1,-1).
// Written as functions so fully unrolled loops fold them into immediates.
// ------------------------------------------------------------------------------------------------
__host__ __device__ __forceinline__ constexpr int cx(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0;
}
__host__ __device__ __forceinline__ constexpr int cy(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0;
}
__host__ __device__ __forceinline__ constexpr int opp(int i) {
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 5 + 2) % 4) + 5);
}
// lattice weights 4/9, 1/9, 1/36 as exact double quotients
__host__ __device__ __forceinline__ constexpr double wq(int i) {
    return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
}

// ------------------------------------------------------------------------------------------------
// 24-node eighth-order stencil in the numbering of Table 1 (index n-1 for node n): first layer in
// the D2Q9 order, then 2 e_(n-8) for n = 9..16, then the knight moves (2,1),(-2,1),(-2,-1),(2,-1)
// and (1,2),(-1,2),(-1,-2),(1,-2).  Used by the wall-list builder, whose masks are reported in
// this numbering.
// ------------------------------------------------------------------------------------------------
__host__ __device__ __forceinline__ constexpr int s24x(int n) {
    return n < 8 ? cx(n + 1) : n < 16 ? 2 * cx(n - 7) : n < 20 ? 2 * cx(n - 11) : cx(n - 15);
}
__host__ __device__ __forceinline__ constexpr int s24y(int n) {
    return n < 8 ? cy(n + 1) : n < 16 ? 2 * cy(n - 7) : n < 20 ? cy(n - 11) : 2 * cy(n - 15);
}
// E8 weights by squared length (normalised so that sum_e w e_x^2 = 1)
__host__ __device__ __forceinline__ constexpr double w8(int e2) {
    return e2 == 1 ? 4.0 / 21.0 : e2 == 2 ? 4.0 / 45.0 : e2 == 4 ? 1.0 / 60.0 : e2 == 5 ? 2.0 / 315.0 : 1.0 / 5040.0;
}

// ------------------------------------------------------------------------------------------------
// Per-case parameters in the compute type R, derived on the host once per case so that a kernel
// starting a work item only loads them.
// ------------------------------------------------------------------------------------------------
template <class R>
struct CaseParams {
    int nx, ny, row, bc_x, bc_y, mode;  // row: stride of lattice rows (9 planes x pitch pairs)
    long long plane;                    // stride of the planes of one row (pitch pairs)
    R omega[2], cF[2];
    R G, Gw2, lam, delta, s1, s2, s3, t2, t3;
    R gx, gy;
    R d1[2], d5[2];            // inlet: f_1 - f_3 and f_5 - f_7 (= f_8 - f_6) of f^eq(rho_in, u_in)
    R sh0[2], sh1[2], sh5[2];  // storage shift w_i rho0 for the rest, axis and diagonal weights
    R rho0[2], om_rho0[2];     // rho0 and omega rho0 of the shifted storage (0 for FP32 / FP64)
    int inlet_profile;         // 1: the inlet differences above scale with 4 s (ny - s) / ny^2, s = y + 1/2
    int outlet;                // 1: pressure outlet (Zou-He density condition holding rho_out)
    R rho_out[2];
    int moving;                // 1: a walled y edge slides (u_wall nonzero)
    R prof_c;                  // 4 / ny^2
    R uw[2];                   // x-velocity of the lower / upper wall
};

// ------------------------------------------------------------------------------------------------
// Per-case descriptor (device copy; built on the host).
// ------------------------------------------------------------------------------------------------
struct DevCase {
    int nx, ny, pitch;      // pitch: (A, B) pairs per row of one plane (ghost columns included)
    int bc_x, bc_y;
    int mode;               // 0 original, 1 improved
    long long f_off;        // pair offset of the case's [ny][9][pitch] block of (A, B) pairs in a buffer
    long long d_off;        // element offset of the case's [ny][nx] block in per-node arrays
    long long w_off;        // first wall-list entry of the case
    long long nwall;        // wall-list entries of the case
    int item_begin, item_end;
    double omega[2];        // 1 / tau_k
    double cF[2];           // 1 - 1 / (2 tau_k)
    double G, Gw2, lam;
    double delta;
    double s1, s2, s3, t2, t3;   // Eq. 12 coefficients s'_1 = t'_1, s'_2, s'_3, t'_2, t'_3
    double g[2];
    double u_in, rho_in[2];
    double rho0[2];         // storage shift per component
    double u_wall[2];       // x-velocity of the lower / upper wall of a walled y direction
    int inlet_profile;      // 0 uniform, 1 Poiseuille (peak u_in)
    int outlet;             // 0 copy, 1 pressure
    double rho_out[2];      // densities held by the pressure outlet
    CaseParams<float> pf;   // the above in FP32 and FP64 (filled by fill_case_params)
    CaseParams<double> pd;
};

// Derive pf / pd from the double fields above (host side, after pitch is known).
template <class R>
inline void fill_case_params_as(const DevCase& d, CaseParams<R>& P) {
    P.nx = d.nx; P.ny = d.ny; P.row = 9 * d.pitch; P.bc_x = d.bc_x; P.bc_y = d.bc_y; P.mode = d.mode;
    P.plane = d.pitch;
    for (int k = 0; k < 2; ++k) {
        P.omega[k] = (R)d.omega[k];
        P.cF[k] = (R)d.cF[k];
        P.d1[k] = (R)(6.0 * wq(1) * d.rho_in[k] * d.u_in);
        P.d5[k] = (R)(6.0 * wq(5) * d.rho_in[k] * d.u_in);
        P.sh0[k] = (R)(wq(0) * d.rho0[k]);
        P.sh1[k] = (R)(wq(1) * d.rho0[k]);
        P.sh5[k] = (R)(wq(5) * d.rho0[k]);
        P.rho0[k] = (R)d.rho0[k];
        P.om_rho0[k] = (R)(d.omega[k] * d.rho0[k]);
    }
    P.G = (R)d.G; P.Gw2 = (R)d.Gw2; P.lam = (R)d.lam; P.delta = (R)d.delta;
    P.s1 = (R)d.s1; P.s2 = (R)d.s2; P.s3 = (R)d.s3; P.t2 = (R)d.t2; P.t3 = (R)d.t3;
    P.gx = (R)d.g[0]; P.gy = (R)d.g[1];
    P.inlet_profile = d.inlet_profile;
    P.outlet = d.outlet;
    P.rho_out[0] = (R)d.rho_out[0];
    P.rho_out[1] = (R)d.rho_out[1];
    P.moving = (d.bc_y == kWall && (d.u_wall[0] != 0.0 || d.u_wall[1] != 0.0)) ? 1 : 0;
    P.prof_c = (R)(4.0 / ((double)d.ny * (double)d.ny));
    P.uw[0] = (R)d.u_wall[0];
    P.uw[1] = (R)d.u_wall[1];
}

inline void fill_case_params(DevCase& d) {
    fill_case_params_as<float>(d, d.pf);
    fill_case_params_as<double>(d, d.pd);
}

template <class R>
__device__ __forceinline__ const CaseParams<R>& case_params(const DevCase& C);
template <>
__device__ __forceinline__ const CaseParams<float>& case_params<float>(const DevCase& C) { return C.pf; }
template <>
__device__ __forceinline__ const CaseParams<double>& case_params<double>(const DevCase& C) { return C.pd; }

// ------------------------------------------------------------------------------------------------
// Storage traits: load/store one population value of storage type S as compute type R.
// 16-bit types hold f - w rho0; the kernels add and remove the shift around ld() and st().
// ------------------------------------------------------------------------------------------------
template <class S>
struct Store;

template <>
struct Store<double> {
    static constexpr bool kShift = false;
    __device__ __forceinline__ static double ld(const double* p) { return __ldg(p); }
    __device__ __forceinline__ static void st(double* p, double v) { *p = v; }
};
template <>
struct Store<float> {
    static constexpr bool kShift = false;
    __device__ __forceinline__ static float ld(const float* p) { return __ldg(p); }
    __device__ __forceinline__ static void st(float* p, float v) { *p = v; }
};
template <>
struct Store<__half> {
    static constexpr bool kShift = true;
    __device__ __forceinline__ static float ld(const __half* p) { return __half2float(__ldg(p)); }
    __device__ __forceinline__ static void st(__half* p, float v) { *p = __float2half_rn(v); }
};
template <>
struct Store<__nv_bfloat16> {
    static constexpr bool kShift = true;
    __device__ __forceinline__ static float ld(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
    __device__ __forceinline__ static void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};

// ------------------------------------------------------------------------------------------------
// The population buffers hold f*_i^A and f*_i^B of one node side by side: plane i (0..8) of a case
// is [ny][pitch] pairs (A, B).  One vector access moves both components of a direction.
// ------------------------------------------------------------------------------------------------
template <class S>
struct alignas(2 * sizeof(S)) Pair {
    S a, b;
};

// Load the pair at p as compute-type values; 16-bit types add the storage shifts (shA, shB) back
// with the mixed-precision add (the widening is exact, so each value is rounded once).
template <class S, class R>
__device__ __forceinline__ void load_pair(const Pair<S>* p, R shA, R shB, R& va, R& vb);
template <>
__device__ __forceinline__ void load_pair<double, double>(const Pair<double>* p, double, double, double& va,
                                                          double& vb) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    va = v.x;
    vb = v.y;
}
template <>
__device__ __forceinline__ void load_pair<float, float>(const Pair<float>* p, float, float, float& va, float& vb) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    va = v.x;
    vb = v.y;
}
template <>
__device__ __forceinline__ void load_pair<__half, float>(const Pair<__half>* p, float shA, float shB, float& va,
                                                         float& vb) {
    const uint32_t u = *reinterpret_cast<const uint32_t*>(p);
    asm("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\t"
        "add.rn.f32.f16 %0, lo, %3;\n\tadd.rn.f32.f16 %1, hi, %4;\n\t}"
        : "=f"(va), "=f"(vb)
        : "r"(u), "f"(shA), "f"(shB));
}
template <>
__device__ __forceinline__ void load_pair<__nv_bfloat16, float>(const Pair<__nv_bfloat16>* p, float shA, float shB,
                                                                float& va, float& vb) {
    const uint32_t u = *reinterpret_cast<const uint32_t*>(p);
    asm("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\t"
        "add.rn.f32.bf16 %0, lo, %3;\n\tadd.rn.f32.bf16 %1, hi, %4;\n\t}"
        : "=f"(va), "=f"(vb)
        : "r"(u), "f"(shA), "f"(shB));
}

// Store a pair (values already shifted for 16-bit types; round to nearest even).
template <class S, class R>
__device__ __forceinline__ void store_pair(Pair<S>* p, R va, R vb);
template <>
__device__ __forceinline__ void store_pair<double, double>(Pair<double>* p, double va, double vb) {
    *reinterpret_cast<double2*>(p) = make_double2(va, vb);
}
template <>
__device__ __forceinline__ void store_pair<float, float>(Pair<float>* p, float va, float vb) {
    *reinterpret_cast<float2*>(p) = make_float2(va, vb);
}
template <>
__device__ __forceinline__ void store_pair<__half, float>(Pair<__half>* p, float va, float vb) {
    *reinterpret_cast<__half2*>(p) = __floats2half2_rn(va, vb);
}
template <>
__device__ __forceinline__ void store_pair<__nv_bfloat16, float>(Pair<__nv_bfloat16>* p, float va, float vb) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(va, vb);
}

// ------------------------------------------------------------------------------------------------
// Component pairs.  Every per-component quantity of a step (the populations f_i^A, f_i^B, the
// densities, their gradients, forces and relaxation rates) is held as a pair (A, B), so that in
// FP32 one packed FP32x2 instruction (sm_100 and later) does the work of both components.  Each
// lane rounds exactly like the scalar operation.  FP64 pairs are two scalar operations.
// ------------------------------------------------------------------------------------------------
template <class R>
struct PairOf;
template <>
struct PairOf<float> {
    using T = float2;
};
template <>
struct PairOf<double> {
    using T = double2;
};
template <class R>
using V2 = typename PairOf<R>::T;

__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ double2 vadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 vsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 vmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ double2 vfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
template <class R, class T>
__device__ __forceinline__ V2<R> vbc(T v) {  // the same value in both lanes, in the compute type
    return V2<R>{(R)v, (R)v};
}

// 1 / x: FP32 takes the hardware reciprocal approximation (within 2 ulp; it only scales
// velocities), FP64 the correctly rounded division.
__device__ __forceinline__ float recip(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// Compute type for a storage type: FP64 storage computes in FP64, everything else in FP32.
template <class S>
struct ComputeOf {
    using type = float;
};
template <>
struct ComputeOf<double> {
    using type = double;
};

}  // namespace lbm
