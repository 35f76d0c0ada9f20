// Three-dimensional form of the time step (arXiv 2505.22256, Sec. 3.5) and its C ABI
// (include/lbm3d.h).
//
// State: the post-collision populations f*_i^k of one lattice, [19][N] pairs (f*_i^A, f*_i^B) in the
// storage / compute type R (float or double), N = nx ny nz, x fastest; two buffers.  One vector
// access moves both components of a direction.  One time step is two
// launches:
//   k3_rho    pull f_i(x) = f*_i(x - e_i), or f*_opp(i)(x) across a blocked link (halfway
//             bounce-back, Sec. 3.5); (rho_A, rho_B) = sum_i f_i (Eq. 3) into one interleaved
//             density array
//   k3_march  the same pull for the node's own populations and momentum (Eq. 4); cohesion (Eq. 8)
//             and adhesion (Eq. 9, local parameter of Eqs. 10-12) on the 92-offset eighth-order
//             stencil -- nodes with a solid node inside the stencil apply the second-layer copy
//             x + sign(e) (Sec. 2.4) and the solid switch; body force; velocity with Guo's
//             half-force shift (Eq. 5); SRT collision with Guo forcing (Eqs. 1, 2, 6, 7) written to
//             the other buffer.  Blocks march along z with the stencil's density planes in shared
//             memory.  Its fields form (kFields) writes rho and u in FP64 and per-block diagnostic
//             records instead of colliding.
// Periodic in x, y and z.
#include <math.h>
#include <stdarg.h>

#include <mutex>
#include <vector>

#include "lbm_internal.h"
#include "../../include/lbm3d.h"

namespace lbm {
lbm_status report_error(lbm_status s, const char* fmt, ...);
}

using namespace lbm;

namespace {

// D3Q19: 0 rest; 1..6 = +x, -x, +y, -y, +z, -z; 7..18 = (1,1,0), (-1,-1,0), (1,-1,0), (-1,1,0),
// (1,0,1), (-1,0,-1), (1,0,-1), (-1,0,1), (0,1,1), (0,-1,-1), (0,1,-1), (0,-1,1)
__host__ __device__ __forceinline__ constexpr int e3x(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1 : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ __forceinline__ constexpr int e3y(int i) {
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1 : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ __forceinline__ constexpr int e3z(int i) {
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1 : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
__host__ __device__ __forceinline__ constexpr int opp3(int i) { return i == 0 ? 0 : (i % 2 ? i + 1 : i - 1); }
__host__ __device__ __forceinline__ constexpr double w19(int i) { return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }
// The collision's weights in the compute type.  1/3, 1/18 and 1/36 rounded to FP32 one by one sum to
// 1 + 2e-8, and every step redistributes each node's mass with them, so an FP32 run gained that much
// mass per step; the FP32 set below sums to 1 exactly (w_0 + 6 w_1 + 12 w_2 = 1 with w_2 = w_1 / 2,
// w_1 = 7456540 2^-27, w_0 = 11184812 2^-25), each weight within 1.2e-7 (relative) of its value.
template <class R>
__host__ __device__ __forceinline__ constexpr double w19c(int i) { return w19(i); }
template <>
__host__ __device__ __forceinline__ constexpr double w19c<float>(int i) {
    return i == 0 ? 11184812.0 / 33554432.0 : (i <= 6 ? 7456540.0 / 134217728.0 : 3728270.0 / 134217728.0);
}
// eighth-order stencil weights by |e|^2 (0: not in the stencil)
__host__ __device__ __forceinline__ constexpr double w92(int q) {
    return q == 1 ? 4.0 / 45.0 : q == 2 ? 1.0 / 21.0 : q == 3 ? 2.0 / 105.0 : q == 4 ? 5.0 / 504.0
         : q == 5 ? 1.0 / 315.0 : q == 6 ? 1.0 / 630.0 : q == 8 ? 1.0 / 5040.0 : 0.0;
}

// node flags: bits 0..17 link i = bit+1 blocked (x - e_i solid); 18 solid; 19 a solid node lies in
// the 92-offset stencil; 20 a solid node within three cells (Chebyshev; contact-angle exclusion)
constexpr uint32_t k3Solid = 1u << 18;
constexpr uint32_t k3Wall = 1u << 19;
constexpr uint32_t k3Near = 1u << 20;

struct Geo3 {
    int nx, ny, nz;
    long long N;
};

__device__ __forceinline__ int wrapc(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }
__device__ __forceinline__ long long site(const Geo3& g, int x, int y, int z) {
    return ((long long)wrapc(z, g.nz) * g.ny + wrapc(y, g.ny)) * g.nx + wrapc(x, g.nx);
}

template <class R>
struct P3 {
    R omega[2], cF[2], G, Gw2, lam, delta, s1, s2, s3, t2, t3, g[3];
    R sh[3][2];  // storage shifts w rho0_store[k] of the 16-bit storage modes, by weight class
    int mode;
    int psi;  // second-layer reading: a replaced (solid) site copies psi only and keeps s = 1
    int adh;  // 1: adhesion sum of Eq. 9 with the D3Q19 weights over the first layer
};

// Stored populations: FP64 and FP32 pairs as computed; the 16-bit types hold h = f - w_i rho0_k per
// component (rho0 = lbm3d_params.rho0_store), which ld3 adds back (one rounding, the widening is
// exact) and st3 takes off before rounding to 16 bits.
__host__ __device__ __forceinline__ constexpr int wcls3(int i) { return i == 0 ? 0 : (i <= 6 ? 1 : 2); }
template <class S, class R>
__device__ __forceinline__ V2<R> ld3(const Pair<S>* p, const P3<R>& P, int i) {
    V2<R> v;
    if constexpr (Store<S>::kShift) load_pair<S, R>(p, P.sh[wcls3(i)][0], P.sh[wcls3(i)][1], v.x, v.y);
    else load_pair<S, R>(p, (R)0, (R)0, v.x, v.y);
    return v;
}
template <class S, class R>
__device__ __forceinline__ void st3(Pair<S>* p, V2<R> v, const P3<R>& P, int i) {
    if constexpr (Store<S>::kShift) store_pair<S, R>(p, v.x - P.sh[wcls3(i)][0], v.y - P.sh[wcls3(i)][1]);
    else store_pair<S, R>(p, v.x, v.y);
}

// Adhesion variants of the wall stencil: 0 the 92-offset sum with the solid switch of a replaced
// second-layer site, 1 the same keeping s = 1 there, 2 the D3Q19 first-layer sum (Eq. 9 as printed).
enum { kAdhE8 = 0, kAdhE8Psi = 1, kAdhD3Q19 = 2 };
__host__ __device__ constexpr double w19q(int q) { return q == 1 ? 1.0 / 18.0 : (q == 2 ? 1.0 / 36.0 : 0.0); }

__global__ void k3_flags(Geo3 g, const uint8_t* __restrict__ solid, uint32_t* __restrict__ flags) {
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 4 + threadIdx.y, z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const long long s = ((long long)z * g.ny + y) * g.nx + x;
    uint32_t f = 0;
    if (solid[s]) f |= k3Solid;
    for (int i = 1; i < 19; ++i)
        if (solid[site(g, x - e3x(i), y - e3y(i), z - e3z(i))]) f |= 1u << (i - 1);
    for (int dz = -3; dz <= 3; ++dz)
        for (int dy = -3; dy <= 3; ++dy)
            for (int dx = -3; dx <= 3; ++dx) {
                if (!solid[site(g, x + dx, y + dy, z + dz)]) continue;
                f |= k3Near;
                const int q = dx * dx + dy * dy + dz * dz;
                if (dx >= -2 && dx <= 2 && dy >= -2 && dy <= 2 && dz >= -2 && dz <= 2 && w92(q) != 0.0) f |= k3Wall;
            }
    flags[s] = f;
}

// Wrapped neighbourhood of one node: the x index and the y, z offsets (y nx, z nx ny) for the
// displacements -2..2, as 32-bit values, so every stencil site is one three-operand add.
struct Nb3 {
    int xw[5], yo[5], zo[5];
    __device__ __forceinline__ Nb3(const Geo3& g, int x, int y, int z) {
        const int nxy = g.nx * g.ny;
#pragma unroll
        for (int d = -2; d <= 2; ++d) {
            xw[d + 2] = wrapc(x + d, g.nx);
            yo[d + 2] = wrapc(y + d, g.ny) * g.nx;
            zo[d + 2] = wrapc(z + d, g.nz) * nxy;
        }
    }
    __device__ __forceinline__ int at(int dx, int dy, int dz) const { return zo[dz + 2] + yo[dy + 2] + xw[dx + 2]; }
};

// density pair (rho_A, rho_B) of a node, stored interleaved
template <class R>
struct Rho2;
template <>
struct Rho2<float> {
    using T = float2;
};
template <>
struct Rho2<double> {
    using T = double2;
};

// the node's 38 post-streaming populations (f[i]: component A, f[19 + i]: component B)
template <class S, class R>
__device__ __forceinline__ void pull3(const Geo3& g, const Nb3& nb, const Pair<S>* __restrict__ fs, const P3<R>& P,
                                      uint32_t fl, int s, R (&f)[38]) {
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        int src, q;
        if (i > 0 && ((fl >> (i - 1)) & 1u)) {
            src = s;
            q = opp3(i);
        } else {
            src = i == 0 ? s : nb.at(-e3x(i), -e3y(i), -e3z(i));
            q = i;
        }
        const V2<R> v = ld3<S, R>(fs + (long long)q * g.N + src, P, q);
        f[i] = v.x;
        f[19 + i] = v.y;
    }
}

template <class S, class R>
__global__ void __launch_bounds__(128) k3_rho(Geo3 g, P3<R> P, const uint32_t* __restrict__ flags,
                                              const Pair<S>* __restrict__ fs, typename Rho2<R>::T* __restrict__ rho) {
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 4 + threadIdx.y, z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const int s = (z * g.ny + y) * g.nx + x;
    const uint32_t fl = flags[s];
    typename Rho2<R>::T r;
    r.x = (R)-1;  // solid sites carry -1: the step kernel's wall path tells them apart by the sign
    r.y = (R)-1;
    if (!(fl & k3Solid)) {
        const Nb3 nb(g, x, y, z);
        V2<R> f[19];
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const bool bl = i > 0 && ((fl >> (i - 1)) & 1u);
            const int q = bl ? opp3(i) : i;
            f[i] = ld3<S, R>(fs + (long long)q * g.N + (bl || i == 0 ? s : nb.at(-e3x(i), -e3y(i), -e3z(i))), P, q);
        }
        // rho_k = sum_i f_i as a balanced tree (rounding grows with the depth, not the count), both
        // components at once
        const V2<R> a = vadd(vadd(vadd(f[0], f[1]), vadd(f[2], f[3])), vadd(vadd(f[4], f[5]), vadd(f[6], f[7])));
        const V2<R> b = vadd(vadd(vadd(f[8], f[9]), vadd(f[10], f[11])), vadd(vadd(f[12], f[13]), vadd(f[14], f[15])));
        r = vadd(vadd(a, b), vadd(f[16], vadd(f[17], f[18])));
    }
    rho[s] = r;
}

// record: mass A, mass B, mom x, y, z, max |u|^2 (|u| after the last combine), rhoA min/max, rhoB
// min/max, n, unstable
constexpr int k3DiagN = 12;

__device__ __forceinline__ double d3_combine(int q, double a, double b) {
    if (q == 5 || q == 7 || q == 9) return fmax(a, b);
    if (q == 6 || q == 8) return fmin(a, b);
    if (q == 11) return fmax(a, b);
    return a + b;
}
__device__ __forceinline__ double d3_neutral(int q) {
    return (q == 6 || q == 8) ? INFINITY : (q == 7 || q == 9) ? -INFINITY : 0.0;
}

// ------------------------------------------------------------------------------------------------
// Step kernel of the 3-D form.  A block of 32 x 4 columns (x, y) marches over a chunk of z planes.
// The density pairs (rho_A, rho_B) of the planes z-2 .. z+2 over the block's columns and a halo of
// two on each side (36 x 8 sites per plane) sit in a six-plane shared-memory ring; solid sites
// hold -1, so nodes near the wall take the second-layer copy and the solid switch out of the ring
// as well.  Each thread loads its share of the halo of plane z+4 into registers one plane before
// it enters the ring, and the flags of the next plane.  Per plane: pull of the node's 38
// populations, stencil sums out of the ring, moments, forces, collision, store; one barrier.  Both
// components share each instruction: densities, gradients, forces and populations are (A, B) pairs.
// ------------------------------------------------------------------------------------------------
constexpr int k3TX = 32, k3TY = 4, k3T = k3TX * k3TY;   // block = 32 x 4 columns
constexpr int k3HX = k3TX + 4, k3HY = k3TY + 4;           // halo region of one plane: 36 x 8
constexpr int k3HP = k3HX * k3HY;
constexpr int k3HN = (k3HP + k3T - 1) / k3T;              // halo sites loaded per thread
constexpr int k3Ring = 6;                                 // density planes resident

template <class R>
constexpr size_t k3_ring_bytes() {
    return (size_t)k3Ring * k3HP * sizeof(V2<R>);
}
template <class R>
constexpr size_t k3_march_smem() {
    return k3_ring_bytes<R>();
}

// Stencil sums of a node whose stencil reaches a solid site: second-layer copy of x + sign(e) for a
// solid second-layer site (Sec. 2.4), density 0 and solid switch 1 at a solid site; solid sites
// hold -1 in the ring.  b0..b4: ring rows of the planes z-2..z+2 at the node.  (Inlined: an
// out-of-line call measured 7 % slower on the full case and twice as slow on a small one.)
template <class R, int kAdh>
__device__ __forceinline__ void wall_stencil3(const V2<R>* b0, const V2<R>* b1, const V2<R>* b2, const V2<R>* b3,
                                           const V2<R>* b4, V2<R>& gx, V2<R>& gy, V2<R>& gz, R (&ad)[3]) {
    using V = V2<R>;
    const V* bs[5] = {b0, b1, b2, b3, b4};
#pragma unroll
    for (int dz = 0; dz <= 2; ++dz)
#pragma unroll
        for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
            for (int dx = -2; dx <= 2; ++dx) {
                if (dz == 0 && (dy < 0 || (dy == 0 && dx <= 0))) continue;
                const int q = dx * dx + dy * dy + dz * dz;
                const double wq = w92(q);
                if (wq == 0.0) continue;
                const bool second = dx == 2 || dx == -2 || dy == 2 || dy == -2 || dz == 2 || dz == -2;
                V v[2];
                R vs[2];
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    const int sg = side == 0 ? 1 : -1;
                    const int ex = sg * dx, ey = sg * dy, ez = sg * dz;
                    V w = bs[2 + ez][ey * k3HX + ex];
                    const bool own = w.x < (R)0;
                    if (second && own) {
                        const int fx = (ex > 0) - (ex < 0), fy = (ey > 0) - (ey < 0), fz = (ez > 0) - (ez < 0);
                        w = bs[2 + fz][fy * k3HX + fx];
                    }
                    const bool sol = w.x < (R)0;
                    v[side] = sol ? vbc<R>(0) : w;
                    vs[side] = (sol || (kAdh == kAdhE8Psi && own)) ? (R)1 : (R)0;
                }
                const V a = vsub(v[0], v[1]);
                gx = vfma(vbc<R>(wq * dx), a, gx);
                gy = vfma(vbc<R>(wq * dy), a, gy);
                gz = vfma(vbc<R>(wq * dz), a, gz);
                const double wa = kAdh == kAdhD3Q19 ? w19q(q) : wq;
                if (wa != 0.0) {
                    const R w = (R)wa, sw = vs[0] - vs[1];
                    ad[0] += w * dx * sw;
                    ad[1] += w * dy * sw;
                    ad[2] += w * dz * sw;
                }
            }
}

#ifndef LBM3_MIN_BLOCKS
#define LBM3_MIN_BLOCKS 3
#endif
// kFields: the fields form.  In place of the collision each node writes rho_A, rho_B and u (FP64, o5
// may be NULL) and adds its values to the thread's diagnostic record; each block writes one record
// (block index blockIdx.x + gridDim.x (blockIdx.y + gridDim.y blockIdx.z)) to part.
template <class S, class R, int kAdh, bool kFields = false>
__global__ void __launch_bounds__(k3T, sizeof(R) == 8 ? 2 : LBM3_MIN_BLOCKS)
    k3_march(Geo3 g, P3<R> P, int zc, const uint32_t* __restrict__ flags, const Pair<S>* __restrict__ fs,
             const V2<R>* __restrict__ rho, Pair<S>* __restrict__ fout, double* __restrict__ o5,
             double* __restrict__ part) {
    using V = V2<R>;
    extern __shared__ __align__(16) unsigned char smem3[];
    V* ring = reinterpret_cast<V*>(smem3);
    const int tx = threadIdx.x, ty = threadIdx.y, t = ty * k3TX + tx;
    const int x0 = blockIdx.x * k3TX, y0 = blockIdx.y * k3TY;
    const int x = x0 + tx, y = y0 + ty;
    const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, g.nz);
    const bool active = x < g.nx && y < g.ny;
    const int nxy = g.nx * g.ny;

    // this thread's halo sites: in-plane offsets of the wrapped columns
    int hoff[k3HN];
#pragma unroll
    for (int k = 0; k < k3HN; ++k) {
        const int j = t + k * k3T;
        const int hx = j % k3HX, hy = j / k3HX;
        const int gx = ((x0 - 2 + hx) % g.nx + g.nx) % g.nx, gy = ((y0 - 2 + hy) % g.ny + g.ny) % g.ny;
        hoff[k] = j < k3HP ? gy * g.nx + gx : -1;
    }
    auto load_plane = [&](int p, V (&v)[k3HN]) {
        const int zo = wrapc(p, g.nz) * nxy;
#pragma unroll
        for (int k = 0; k < k3HN; ++k)
            if (hoff[k] >= 0) v[k] = __ldg(rho + zo + hoff[k]);
    };
    auto slot = [&](int p) -> int { return wrapc(p % k3Ring, k3Ring); };  // ring slot of plane p >= -2
    auto store_plane = [&](int p, const V (&v)[k3HN]) {
        V* dst = ring + slot(p) * k3HP;
#pragma unroll
        for (int k = 0; k < k3HN; ++k)
            if (hoff[k] >= 0) dst[t + k * k3T] = v[k];
    };
    const int yx = active ? y * g.nx + x : 0;
    const Nb3 nb(g, active ? x : 0, active ? y : 0, 0);
    // the node's 38 populations at plane z: f_i(x) = f*_i(x - e_i), or f*_opp(i)(x) across a blocked link
    auto pull_plane = [&](int z, uint32_t fl, V (&f)[19]) {
        const int s = z * nxy + yx;
        const int zoff[3] = {wrapc(z - 1, g.nz) * nxy, z * nxy, wrapc(z + 1, g.nz) * nxy};
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            int src, q;
            if (i > 0 && ((fl >> (i - 1)) & 1u)) {
                src = s;
                q = opp3(i);
            } else {
                src = i == 0 ? s : zoff[1 - e3z(i)] + nb.yo[2 - e3y(i)] + nb.xw[2 - e3x(i)];
                q = i;
            }
            f[i] = ld3<S, R>(fs + (long long)q * g.N + src, P, q);
        }
    };

    double rec[k3DiagN];  // fields form: this thread's diagnostic record
    if constexpr (kFields) {
#pragma unroll
        for (int q = 0; q < k3DiagN; ++q) rec[q] = d3_neutral(q);
    }

    // prologue: planes z0-2 .. z0+2 into the ring, plane z0+3 into registers, populations of z0
    uint32_t fl_nx = active ? flags[z0 * nxy + yx] : k3Solid;
    {
        V v[5][k3HN];
#pragma unroll
        for (int d = 0; d < 5; ++d) load_plane(z0 - 2 + d, v[d]);
#pragma unroll
        for (int d = 0; d < 5; ++d) store_plane(z0 - 2 + d, v[d]);
    }
    V nxt[k3HN];
    load_plane(z0 + 3, nxt);
    __syncthreads();

    for (int z = z0; z < z1; ++z) {
        V nn[k3HN];
        if (z + 4 <= z1 + 1) load_plane(z + 4, nn);  // planes up to z1 + 1 are needed
        const uint32_t fl = fl_nx;  // the flags are loaded one plane ahead
        if (z + 1 < z1 && active) fl_nx = flags[(z + 1) * nxy + yx];
        const int s = z * nxy + yx;
        if (!(fl & k3Solid)) {
            V f[19];
            pull_plane(z, fl, f);
            // the node's stencil out of the ring: bs[d] = plane z - 2 + d at the node's column
            const V* bs[5];
#pragma unroll
            for (int d = 0; d < 5; ++d) bs[d] = ring + slot(z - 2 + d) * k3HP + (ty + 2) * k3HX + (tx + 2);
            const V r2 = bs[2][0];
            V gx = vbc<R>(0), gy = vbc<R>(0), gz = vbc<R>(0);  // (A, B) density gradients
            R ad[3] = {(R)0, (R)0, (R)0};
            if (!(fl & k3Wall)) {
                // symmetric pairs (e, -e): w e (rho(x+e) - rho(x-e)), the differences first; two sets
                // of partial sums (odd / even dx) shorten the dependency chains
                V hx[2] = {gx, gx}, hy[2] = {gy, gy}, hz[2] = {gz, gz};
#pragma unroll
                for (int dz = 0; dz <= 2; ++dz)
#pragma unroll
                    for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
                        for (int dx = -2; dx <= 2; ++dx) {
                            if (dz == 0 && (dy < 0 || (dy == 0 && dx <= 0))) continue;  // one of each pair
                            const int q = dx * dx + dy * dy + dz * dz;
                            if (w92(q) == 0.0) continue;
                            const int h = dx & 1;
                            const V a = vsub(bs[2 + dz][dy * k3HX + dx], bs[2 - dz][-dy * k3HX - dx]);
                            if (dx != 0) hx[h] = vfma(vbc<R>(w92(q) * dx), a, hx[h]);
                            if (dy != 0) hy[h] = vfma(vbc<R>(w92(q) * dy), a, hy[h]);
                            if (dz != 0) hz[h] = vfma(vbc<R>(w92(q) * dz), a, hz[h]);
                        }
                gx = vadd(hx[0], hx[1]);
                gy = vadd(hy[0], hy[1]);
                gz = vadd(hz[0], hz[1]);
            } else {
                wall_stencil3<R, kAdh>(bs[0], bs[1], bs[2], bs[3], bs[4], gx, gy, gz, ad);
            }
            const R rA = r2.x, rB = r2.y;
            R GA = (R)0;
            if (fl & k3Wall) {
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
            }
            // momentum per component from the differences of opposite populations (i odd, opp = i + 1)
            V mv[3] = {vbc<R>(0), vbc<R>(0), vbc<R>(0)};
#pragma unroll
            for (int i = 1; i < 19; i += 2) {
                const V d = vsub(f[i], f[i + 1]);
                if (e3x(i) != 0) mv[0] = e3x(i) > 0 ? vadd(mv[0], d) : vsub(mv[0], d);
                if (e3y(i) != 0) mv[1] = e3y(i) > 0 ? vadd(mv[1], d) : vsub(mv[1], d);
                if (e3z(i) != 0) mv[2] = e3z(i) > 0 ? vadd(mv[2], d) : vsub(mv[2], d);
            }
            const V gv[3] = {gx, gy, gz};
            const R inv = recip(rA + rB);
            V F[3];
            R u[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                // each component is pushed by the other's gradient (Eq. 8); adhesion (Eq. 9); body force
                const R FA = -P.G * rA * gv[d].y - GA * rA * ad[d] + rA * P.g[d];
                const R FB = -P.G * rB * gv[d].x - P.Gw2 * rB * ad[d] + rB * P.g[d];
                F[d] = V{FA, FB};
                u[d] = ((mv[d].x + mv[d].y) + (R)0.5 * (FA + FB)) * inv;
            }
            if constexpr (kFields) {
                if (o5) {
                    o5[s] = (double)rA;
                    o5[g.N + s] = (double)rB;
                    o5[2 * g.N + s] = (double)u[0];
                    o5[3 * g.N + s] = (double)u[1];
                    o5[4 * g.N + s] = (double)u[2];
                }
                const double dr = (double)(rA + rB);
                // |u|^2; the square root is taken once, of the maximum (it is monotonic)
                const double u2 = (double)u[0] * u[0] + (double)u[1] * u[1] + (double)u[2] * u[2];
                const bool bad = !(rA > (R)0) || !(rB > (R)0) || !isfinite(u2) || !isfinite((double)rA) ||
                                 !isfinite((double)rB);
                const double v[k3DiagN] = {(double)rA,       (double)rB, dr * (double)u[0], dr * (double)u[1],
                                           dr * (double)u[2], u2,         (double)rA,        (double)rA,
                                           (double)rB,        (double)rB, 1.0,               bad ? 1.0 : 0.0};
#pragma unroll
                for (int q = 0; q < k3DiagN; ++q) rec[q] = d3_combine(q, rec[q], v[q]);
            } else {
                // SRT collision with Guo forcing, per pair of directions (e, -e), both components at
                // once.  With a = e.u, b = e.F_k, P = om rho a + cF b, C0 = om rho (1 - 1.5u^2) - 3 cF u.F:
                //   f*_+- = (1 - om) f_+- + w (C0 + 4.5 a (P + cF b)) +- 3 w P,  f*_0 = (1 - om) f_0 + w_0 C0
                const V om = V{P.omega[0], P.omega[1]}, cf = V{P.cF[0], P.cF[1]};
                const V om1 = vsub(vbc<R>(1), om);
                const V wr = vmul(om, r2);
                const V u2v[3] = {vbc<R>(u[0]), vbc<R>(u[1]), vbc<R>(u[2])};
                const R tq = (R)1 - (R)1.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
                const V uF = vfma(u2v[2], F[2], vfma(u2v[1], F[1], vmul(u2v[0], F[0])));
                const V C0 = vfma(wr, vbc<R>(tq), vmul(vmul(vbc<R>(-3), cf), uF));
                V o[19];
                o[0] = vfma(om1, f[0], vmul(vbc<R>(w19c<R>(0)), C0));
                const V sAx = vmul(vbc<R>(w19c<R>(1)), C0), sDg = vmul(vbc<R>(w19c<R>(7)), C0);
#pragma unroll
                for (int i = 1; i < 19; i += 2) {
                    auto dot = [&](const V* vv) -> V {  // e_i . vv for a pair-valued vector
                        V r = vbc<R>(0);
                        bool first = true;
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            const int e = d == 0 ? e3x(i) : d == 1 ? e3y(i) : e3z(i);
                            if (e == 0) continue;
                            if (first) r = e > 0 ? vv[d] : vsub(vbc<R>(0), vv[d]);
                            else r = e > 0 ? vadd(r, vv[d]) : vsub(r, vv[d]);
                            first = false;
                        }
                        return r;
                    };
                    const double w = w19c<R>(i);
                    const V a = dot(u2v), b = dot(F);
                    const V cb = vmul(cf, b);
                    const V Pp = vfma(wr, a, cb);
                    const V sym = vfma(vbc<R>(4.5 * w), vmul(a, vadd(Pp, cb)), i <= 6 ? sAx : sDg);
                    const V anti = vmul(vbc<R>(3.0 * w), Pp);
                    o[i] = vfma(om1, f[i], vadd(sym, anti));
                    o[i + 1] = vfma(om1, f[i + 1], vsub(sym, anti));
                }
#pragma unroll
                for (int i = 0; i < 19; ++i) st3<S, R>(fout + (long long)i * g.N + s, o[i], P, i);
            }
        } else if constexpr (kFields) {  // solid node: zero fields
            if (active && o5)
                for (int q = 0; q < 5; ++q) o5[(long long)q * g.N + s] = 0.0;
        }
        if (z + 3 <= z1 + 1) store_plane(z + 3, nxt);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < k3HN; ++k) nxt[k] = nn[k];
    }
    if constexpr (kFields) {  // the block's record: warps by shuffles, then the warps in order
        __shared__ double red[k3T / 32][k3DiagN];
        const int lane = t & 31, warp = t >> 5;
#pragma unroll
        for (int q = 0; q < k3DiagN; ++q) {
            double v = rec[q];
            for (int off = 16; off > 0; off >>= 1) v = d3_combine(q, v, __shfl_xor_sync(0xffffffffu, v, off));
            if (lane == 0) red[warp][q] = v;
        }
        __syncthreads();
        if (t == 0) {
            const long long b = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
            for (int q = 0; q < k3DiagN; ++q) {
                double v = red[0][q];
                for (int w = 1; w < k3T / 32; ++w) v = d3_combine(q, v, red[w][q]);
                part[b * k3DiagN + q] = v;
            }
        }
    }
}

// Combine the per-block records in two levels, each in a fixed order (deterministic): k3DiagMid
// blocks each combine a contiguous range of records (a thread takes whole records, strided by the
// block size; then a shuffle tree and the warps in order), then one warp combines their k3DiagMid
// results (k3_diag_final).  A single warp over all records waited on one dependent load per record.
constexpr int k3DiagMid = 256, k3DiagMidThreads = 256;
__global__ void __launch_bounds__(k3DiagMidThreads) k3_diag_mid(long long nblocks, const double* __restrict__ part,
                                                               double* __restrict__ mid) {
    const long long per = (nblocks + gridDim.x - 1) / gridDim.x;
    const long long b0 = (long long)blockIdx.x * per, b1 = b0 + per < nblocks ? b0 + per : nblocks;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    double v[k3DiagN];
#pragma unroll
    for (int q = 0; q < k3DiagN; ++q) v[q] = d3_neutral(q);
    for (long long b = b0 + t; b < b1; b += k3DiagMidThreads) {
#pragma unroll
        for (int q = 0; q < k3DiagN; ++q) v[q] = d3_combine(q, v[q], part[b * k3DiagN + q]);
    }
    __shared__ double red[k3DiagMidThreads / 32][k3DiagN];
#pragma unroll
    for (int q = 0; q < k3DiagN; ++q) {
        double x = v[q];
        for (int off = 16; off > 0; off >>= 1) x = d3_combine(q, x, __shfl_xor_sync(0xffffffffu, x, off));
        if (lane == 0) red[warp][q] = x;
    }
    __syncthreads();
    if (t < k3DiagN) {
        double x = red[0][t];
        for (int w = 1; w < k3DiagMidThreads / 32; ++w) x = d3_combine(t, x, red[w][t]);
        mid[(long long)blockIdx.x * k3DiagN + t] = x;
    }
}

// Combine records in record order (one warp; deterministic); max |u| from max |u|^2.
__global__ void k3_diag_final(long long nblocks, const double* __restrict__ part, double* __restrict__ out) {
    const int lane = threadIdx.x;
    for (int q = 0; q < k3DiagN; ++q) {
        double v = d3_neutral(q);
        for (long long b = lane; b < nblocks; b += 32) v = d3_combine(q, v, part[b * k3DiagN + q]);
        for (int off = 16; off > 0; off >>= 1) v = d3_combine(q, v, __shfl_xor_sync(0xffffffffu, v, off));
        if (lane == 0) out[q] = q == 5 ? sqrt(v) : v;
    }
}

// post-streaming populations (FP64 [2][19][N]) <-> post-collision buffer
template <class S, class R>
__global__ void k3_get(Geo3 g, P3<R> P, const uint32_t* __restrict__ flags, const Pair<S>* __restrict__ fs,
                       double* __restrict__ f) {
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 4 + threadIdx.y, z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const long long s = ((long long)z * g.ny + y) * g.nx + x;
    const uint32_t fl = flags[s];
    R v[38];
    if (fl & k3Solid) {
        for (int q = 0; q < 38; ++q) v[q] = (R)0;
    } else {
        const Nb3 nb(g, x, y, z);
        pull3<S, R>(g, nb, fs, P, fl, (int)s, v);
    }
    for (int q = 0; q < 38; ++q) f[(long long)q * g.N + s] = (double)v[q];
}

template <class S, class R>
__global__ void k3_set(Geo3 g, P3<R> P, const uint32_t* __restrict__ flags, const double* __restrict__ f,
                       Pair<S>* __restrict__ fs) {
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 4 + threadIdx.y, z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const long long s = ((long long)z * g.ny + y) * g.nx + x;
    const uint32_t fl = flags[s];
    for (int i = 0; i < 19; ++i) {
        R v[2] = {(R)0, (R)0};
        for (int k = 0; k < 2; ++k)
            if (!(fl & k3Solid)) {
                // f*_i(x) streams to x + e_i; if that node is solid it comes back as f_opp(i)(x)
                if (i > 0 && ((fl >> (opp3(i) - 1)) & 1u)) v[k] = (R)f[(long long)(19 * k + opp3(i)) * g.N + s];
                else v[k] = (R)f[(long long)(19 * k + i) * g.N + (i == 0 ? s : site(g, x + e3x(i), y + e3y(i), z + e3z(i)))];
            }
        if (fl & k3Solid) store_pair<S, R>(fs + (long long)i * g.N + s, (R)0, (R)0);
        else st3<S, R>(fs + (long long)i * g.N + s, V2<R>{v[0], v[1]}, P, i);
    }
}

// f = f^eq(rho_k, 0) written straight into the post-collision buffer as the pull expects it (the
// state k3_feq + k3_set give, bit for bit, without the [38][N] transfer scratch): the stored f*_i
// at x is w_i rho(x + e_i), or w_i rho(x) when x + e_i is solid (the link comes back by
// bounce-back), and 0 at solid nodes.
template <class S, class R>
__global__ void k3_set_rest(Geo3 g, P3<R> P, const uint32_t* __restrict__ flags, const double* __restrict__ rA,
                            const double* __restrict__ rB, Pair<S>* __restrict__ fs) {
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 4 + threadIdx.y, z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const long long s = ((long long)z * g.ny + y) * g.nx + x;
    const uint32_t fl = flags[s];
    for (int i = 0; i < 19; ++i) {
        V2<R> v{(R)0, (R)0};
        if (!(fl & k3Solid)) {
            const bool bl = i > 0 && ((fl >> (opp3(i) - 1)) & 1u);
            const long long t = (bl || i == 0) ? s : site(g, x + e3x(i), y + e3y(i), z + e3z(i));
            v = V2<R>{(R)(w19(i) * rA[t]), (R)(w19(i) * rB[t])};
        }
        if (fl & k3Solid) store_pair<S, R>(fs + (long long)i * g.N + s, (R)0, (R)0);
        else st3<S, R>(fs + (long long)i * g.N + s, v, P, i);
    }
}

template <class R>
__global__ void k3_feq(Geo3 g, const uint8_t* __restrict__ solid, const double* __restrict__ rA, const double* __restrict__ rB,
                       double* __restrict__ f) {
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 4 + threadIdx.y, z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const long long s = ((long long)z * g.ny + y) * g.nx + x;
    const bool sol = solid[s] != 0;
    for (int i = 0; i < 19; ++i) {
        f[(long long)i * g.N + s] = sol ? 0.0 : w19(i) * rA[s];
        f[(long long)(19 + i) * g.N + s] = sol ? 0.0 : w19(i) * rB[s];
    }
}

// ------------------------------------------------------------------------------------------------
// Contact angle on a sphere (FP64): interface points, algebraic sphere fit, one Gauss-Newton step
// ------------------------------------------------------------------------------------------------
constexpr int kC3Threads = 256;
constexpr int kC3Blocks = 608;  // fixed (the summation order does not depend on the device): 4 x 152
constexpr int kC3Vals = 14;

template <class R>
struct Ca3 {
    Geo3 g;
    const uint32_t* flags;
    const typename Rho2<R>::T* rho;  // interleaved (rho_A, rho_B)
    uint8_t* cross;                  // per node: bit a set where the link to the +a neighbour crosses
};                                   // rho^e = 0 (written by pass 0, read by the later passes)

template <class R>
__device__ __forceinline__ bool ca3_usable(const Ca3<R>& c, long long s) { return (c.flags[s] & (k3Solid | k3Near)) == 0; }

__device__ __forceinline__ double phi3(double a, double b) { return (a - b) / (a + b); }
__device__ __forceinline__ bool phi3_pos(double a, double b) {
    const double sum = a + b;
    return (sum > 0.0 && sum < INFINITY) ? a > b : phi3(a, b) > 0.0;
}
// phi3_pos of densities in the compute type.  For finite FP32 values with a positive FP32 sum the
// FP64 test reduces to a > b (the FP64 sum of two floats is finite and has the sign of their FP32
// sum; the comparison is exact in either type), so FP32 takes it without the FP64 pipe; every other
// case goes through the FP64 form.  The decision is the FP64 one bit for bit.
__device__ __forceinline__ bool phi3_pos_r(float a, float b) {
    if (isfinite(a) && isfinite(b) && a + b > 0.0f) return a > b;
    return phi3_pos((double)a, (double)b);
}
__device__ __forceinline__ bool phi3_pos_r(double a, double b) { return phi3_pos(a, b); }

// st: 0 N, 1-3 centroid, 4-6 centre, 7 r, 8 rms, 9 theta, 10 status (1: too few points)
// One kernel per pass (kPass 0: count and centroid, 1: algebraic fit sums, 2: Gauss-Newton sums, 3:
// residual), so that each holds only the sums it needs: the pass is bound by the latency of its
// dependent loads, and fewer registers keep more warps resident.
template <class R, int kPass>
__global__ void __launch_bounds__(kC3Threads) k3_ca_pass(Ca3<R> c, const double* __restrict__ st,
                                                        double* __restrict__ part) {
    constexpr int pass = kPass;
    constexpr int nv = pass == 0 ? 4 : pass == 1 ? 13 : pass == 2 ? 14 : 1;  // sums this pass forms
    double acc[kC3Vals];
#pragma unroll
    for (int q = 0; q < kC3Vals; ++q) acc[q] = 0.0;
    const double m0 = st[1], m1 = st[2], m2 = st[3], c0 = st[4], c1 = st[5], c2 = st[6], r = st[7];
    const Geo3& g = c.g;
    const bool small = g.N < (1LL << 31);  // node index and coordinates in 32-bit arithmetic
    // one node: pass 0 tests its three links and records the crossings, the later passes take the
    // recorded ones (bits)
    auto node = [&](long long s, uint32_t bits) {
        int x, y, z;
        if (small) {
            const unsigned su = (unsigned)s, row = su / (unsigned)g.nx;
            x = (int)(su - row * (unsigned)g.nx);
            z = (int)(row / (unsigned)g.ny);
            y = (int)(row - (unsigned)z * (unsigned)g.ny);
        } else {
            x = (int)(s % g.nx);
            y = (int)((s / g.nx) % g.ny);
            z = (int)(s / ((long long)g.nx * g.ny));
        }
        const typename Rho2<R>::T r0 = c.rho[s];
        const double ra = (double)r0.x, rb = (double)r0.y;
        const bool pa = phi3_pos_r(r0.x, r0.y);
        uint32_t found = 0;
        for (int axis = 0; axis < 3; ++axis) {
            const long long sn = s + (axis == 0 ? 1 : (axis == 1 ? (long long)g.nx : (long long)g.nx * g.ny));
            if constexpr (pass == 0) {
                const int lim = axis == 0 ? g.nx : (axis == 1 ? g.ny : g.nz);
                const int coord = axis == 0 ? x : (axis == 1 ? y : z);
                if (coord + 1 >= lim) continue;  // no pair across the periodic seam
                if (!ca3_usable(c, sn)) continue;
                const typename Rho2<R>::T r1 = c.rho[sn];
                if (pa == phi3_pos_r(r1.x, r1.y)) continue;
                found |= 1u << axis;
            } else if (!((bits >> axis) & 1u)) {
                continue;
            }
            const typename Rho2<R>::T r1 = c.rho[sn];
            const double qa = (double)r1.x, qb = (double)r1.y;
            const double a = phi3(ra, rb), b = phi3(qa, qb);
            double p[3] = {(double)x, (double)y, (double)z};
            p[axis] += a / (a - b);
            if constexpr (pass == 0) {
                acc[0] += 1.0;
                acc[1] += p[0];
                acc[2] += p[1];
                acc[3] += p[2];
            } else if constexpr (pass == 1) {
                const double q0 = p[0] - m0, q1 = p[1] - m1, q2 = p[2] - m2, qq = q0 * q0 + q1 * q1 + q2 * q2;
                acc[0] += q0 * q0; acc[1] += q0 * q1; acc[2] += q0 * q2;
                acc[3] += q1 * q1; acc[4] += q1 * q2; acc[5] += q2 * q2;
                acc[6] += q0; acc[7] += q1; acc[8] += q2;
                acc[9] += q0 * qq; acc[10] += q1 * qq; acc[11] += q2 * qq; acc[12] += qq;
            } else if constexpr (pass == 2) {
                const double d0 = p[0] - c0, d1 = p[1] - c1, d2 = p[2] - c2;
                const double d = sqrt(d0 * d0 + d1 * d1 + d2 * d2), res = d - r;
                const double j[4] = {-d0 / d, -d1 / d, -d2 / d, -1.0};
                int k = 0;
                for (int a2 = 0; a2 < 4; ++a2)
                    for (int b2 = a2; b2 < 4; ++b2) acc[k++] += j[a2] * j[b2];
                for (int a2 = 0; a2 < 4; ++a2) acc[10 + a2] += j[a2] * res;
            } else {
                const double d0 = p[0] - c0, d1 = p[1] - c1, d2 = p[2] - c2;
                const double res = sqrt(d0 * d0 + d1 * d1 + d2 * d2) - r;
                acc[0] += res * res;
            }
        }
        if constexpr (pass == 0) c.cross[s] = (uint8_t)found;
    };
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x, nth = (long long)gridDim.x * blockDim.x;
    // one node per thread and step, so that the crossings of neighbouring nodes (they cluster along
    // the interface) go to neighbouring lanes
    if constexpr (pass == 0) {
        for (long long s = tid; s < g.N; s += nth) {
            if (ca3_usable(c, s)) node(s, 0u);
            else c.cross[s] = 0;
        }
    } else {  // the same order; the bits of four steps are loaded together
        for (long long s0 = tid; s0 < g.N; s0 += 4 * nth) {
            uint32_t b[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = s0 + j * nth < g.N ? c.cross[s0 + j * nth] : 0u;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (b[j]) node(s0 + j * nth, b[j]);
        }
    }
    __shared__ double red[kC3Threads / 32][kC3Vals];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < nv; ++q) {
        double v = acc[q];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) red[warp][q] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int q = 0; q < kC3Vals; ++q) {  // the sums a pass does not form are written as 0
            double v = 0.0;
            if (q < nv)
                for (int w = 0; w < kC3Threads / 32; ++w) v += red[w][q];
            part[blockIdx.x * kC3Vals + q] = v;
        }
}

__device__ void solve4(double A[4][4], double b[4], double x[4]) {
    for (int c = 0; c < 4; ++c) {
        int p = c;
        for (int r = c + 1; r < 4; ++r)
            if (fabs(A[r][c]) > fabs(A[p][c])) p = r;
        for (int k = 0; k < 4; ++k) {
            const double t = A[c][k];
            A[c][k] = A[p][k];
            A[p][k] = t;
        }
        const double t = b[c];
        b[c] = b[p];
        b[p] = t;
        for (int r = c + 1; r < 4; ++r) {
            const double f = A[r][c] / A[c][c];
            for (int k = c; k < 4; ++k) A[r][k] -= f * A[c][k];
            b[r] -= f * b[c];
        }
    }
    for (int r = 3; r >= 0; --r) {
        double s = b[r];
        for (int k = r + 1; k < 4; ++k) s -= A[r][k] * x[k];
        x[r] = s / A[r][r];
    }
}

__global__ void k3_ca_solve(int pass, int nblocks, const double* __restrict__ part, double* __restrict__ st, double sc0,
                            double sc1, double sc2, double R) {
    double S[kC3Vals];
    const int lane = threadIdx.x & 31;
    for (int q = 0; q < kC3Vals; ++q) {
        double v = 0.0;
        for (int b = lane; b < nblocks; b += 32) v += part[b * kC3Vals + q];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        S[q] = v;
    }
    if (lane != 0) return;
    if (pass == 0) {
        st[0] = S[0];
        st[10] = S[0] < 8.0 ? 1.0 : 0.0;
        for (int d = 0; d < 3; ++d) st[1 + d] = S[0] > 0.0 ? S[1 + d] / S[0] : 0.0;
    } else if (pass == 1) {
        if (st[10] != 0.0) return;
        // [2q, 1] [c; d] = |q|^2 in the least-squares sense
        double A[4][4] = {{4 * S[0], 4 * S[1], 4 * S[2], 2 * S[6]},
                          {4 * S[1], 4 * S[3], 4 * S[4], 2 * S[7]},
                          {4 * S[2], 4 * S[4], 4 * S[5], 2 * S[8]},
                          {2 * S[6], 2 * S[7], 2 * S[8], st[0]}};
        double b[4] = {2 * S[9], 2 * S[10], 2 * S[11], S[12]};
        double x[4];
        solve4(A, b, x);
        st[7] = sqrt(x[3] + x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        for (int d = 0; d < 3; ++d) st[4 + d] = st[1 + d] + x[d];
    } else if (pass == 2) {
        if (st[10] != 0.0) return;
        double A[4][4];
        int k = 0;
        for (int a = 0; a < 4; ++a)
            for (int b2 = a; b2 < 4; ++b2) {
                A[a][b2] = S[k];
                A[b2][a] = S[k];
                ++k;
            }
        double b[4] = {-S[10], -S[11], -S[12], -S[13]};
        double x[4];
        solve4(A, b, x);
        for (int d = 0; d < 3; ++d) st[4 + d] += x[d];
        st[7] += x[3];
    } else {
        if (st[10] != 0.0) return;
        st[8] = sqrt(S[0] / st[0]);
        const double d0 = st[4] - sc0, d1 = st[5] - sc1, d2 = st[6] - sc2, r = st[7];
        double cth = (R * R + r * r - (d0 * d0 + d1 * d1 + d2 * d2)) / (2.0 * r * R);
        cth = cth > 1.0 ? 1.0 : (cth < -1.0 ? -1.0 : cth);
        st[9] = acos(cth) * (180.0 / 3.14159265358979323846);
    }
}

}  // namespace

// ------------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------------
struct lbm3d_ctx {
    int storage = LBM_STORE_F32;
    size_t elem = 4;               // bytes per stored population value
    size_t relem = 4;              // bytes per value of the compute type (densities)
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Geo3 g{};
    P3<float> pf{};
    P3<double> pd{};
    long long nfluid = 0;
    uint8_t* solid = nullptr;
    uint32_t* flags = nullptr;
    unsigned char* f[2] = {nullptr, nullptr};
    int cur = 0;
    unsigned char* rho = nullptr;  // [2][N] in the compute type
    double* part = nullptr;        // per-block diagnostic records
    long long nparts = 0;
    double* dout = nullptr;        // [k3DiagN]
    double* ca = nullptr;          // contact angle: status record + block partials
    uint8_t* ca_cross = nullptr;   // contact angle: per-node crossing bits (N bytes)
    double* scratch = nullptr;     // [38][N] doubles for population transfers and fields (on demand)
    double* dens = nullptr;        // [2][N] doubles for lbm3d_set_densities from host arrays (on demand)
    // overlapped host transfers (lbm3d_set_densities_async, lbm3d_fields_async; on first use): copy
    // streams, double-buffered device staging and the events that order them with the stream
    cudaStream_t xs_in = nullptr, xs_out = nullptr;
    double* xin[2] = {nullptr, nullptr};   // [2][N] densities from the host
    double* xout[2] = {nullptr, nullptr};  // [5][N] fields for the host
    cudaEvent_t xin_ready[2] = {nullptr, nullptr}, xin_free[2] = {nullptr, nullptr};
    cudaEvent_t xout_ready[2] = {nullptr, nullptr}, xout_free[2] = {nullptr, nullptr};
    int xin_k = 0, xout_k = 0;
};

namespace {

bool fin(double v) { return isfinite(v) != 0; }

template <class R>
P3<R> make_p3(const lbm3d_params& p) {
    P3<R> P;
    for (int k = 0; k < 2; ++k) {
        P.omega[k] = (R)(1.0 / p.tau[k]);
        P.cF[k] = (R)(1.0 - 0.5 / p.tau[k]);
    }
    P.G = (R)p.G_AB;
    P.Gw2 = (R)p.G_w2;
    P.lam = (R)p.lambda;
    P.delta = (R)p.delta;
    const double l = p.lambda, dl = p.delta;
    P.s1 = (R)(2.0 * l / (1.0 + l));                          // Eq. 12 coefficients
    P.s2 = (R)(2.0 * (l * l - l) / (dl * (1.0 + l)));
    P.s3 = (R)((l - l * l) / (dl * dl * (1.0 + l)));
    P.t2 = (R)(2.0 * (l - 1.0) / (dl * (1.0 + l)));
    P.t3 = (R)((l - 1.0) / (dl * dl * (1.0 + l)));
    for (int d = 0; d < 3; ++d) P.g[d] = (R)p.g[d];
    for (int c = 0; c < 3; ++c)
        for (int k = 0; k < 2; ++k) P.sh[c][k] = (R)(w19(c == 0 ? 0 : (c == 1 ? 1 : 7)) * p.rho0_store[k]);
    P.mode = p.mode;
    P.psi = p.second_layer == LBM_SECOND_LAYER_PSI;
    P.adh = p.adhesion_stencil == LBM3_ADHESION_D3Q19;
    return P;
}

// Calls fn(S*, R*) (null pointers carrying the types) for the context's storage: the stored type S
// and the compute type R.
template <class Fn>
cudaError_t with_types3(int storage, Fn&& fn) {
    switch (storage) {
        case LBM_STORE_F64: return fn((double*)nullptr, (double*)nullptr);
        case LBM_STORE_F32: return fn((float*)nullptr, (float*)nullptr);
        case LBM_STORE_F16_SHIFTED: return fn((__half*)nullptr, (float*)nullptr);
        default: return fn((__nv_bfloat16*)nullptr, (float*)nullptr);
    }
}
#define TYPES3(s_, r_)                                   \
    using S = std::remove_pointer_t<decltype(s_)>;      \
    using R = std::remove_pointer_t<decltype(r_)>

// node kernels run blocks of 32 x 4 nodes (x, y), so that a block's stencil rows share L1
dim3 grid3(const Geo3& g) { return dim3((unsigned)((g.nx + 31) / 32), (unsigned)((g.ny + 3) / 4), (unsigned)g.nz); }
const dim3 kBlock3(32, 4, 1);

// z planes per block of the step kernel: about 16, spread evenly over nz
#ifndef LBM3_ZCHUNK
#define LBM3_ZCHUNK 16
#endif
int zchunk3(const Geo3& g) {
    const int chunks = (g.nz + LBM3_ZCHUNK - 1) / LBM3_ZCHUNK;
    return (g.nz + chunks - 1) / chunks;
}

cudaError_t scratch_for(lbm3d_ctx* c) {
    if (c->scratch) return cudaSuccess;
    return cudaMalloc(&c->scratch, (size_t)38 * c->g.N * sizeof(double));
}

// the context's parameters in the compute type R
template <class R>
const P3<R>& p3_of(const lbm3d_ctx* c) {
    return *reinterpret_cast<const P3<R>*>(sizeof(R) == 4 ? (const void*)&c->pf : (const void*)&c->pd);
}
template <class S>
Pair<S>* state3(const lbm3d_ctx* c, int buf) {
    return reinterpret_cast<Pair<S>*>(c->f[buf]);
}

// the step kernel instance of the adhesion variant (kFields: its fields form)
template <class S, class R, bool kFields = false>
auto march_kernel(const P3<R>& P) {
    return P.adh ? k3_march<S, R, kAdhD3Q19, kFields>
                 : (P.psi ? k3_march<S, R, kAdhE8Psi, kFields> : k3_march<S, R, kAdhE8, kFields>);
}

dim3 march_grid(const Geo3& g, int zc) {
    return dim3((unsigned)((g.nx + k3TX - 1) / k3TX), (unsigned)((g.ny + k3TY - 1) / k3TY), (unsigned)((g.nz + zc - 1) / zc));
}

template <class S, class R>
cudaError_t step_once(lbm3d_ctx* c) {
    const dim3 gr = grid3(c->g);
    const Pair<S>* fs = state3<S>(c, c->cur);
    auto* rho = reinterpret_cast<typename Rho2<R>::T*>(c->rho);
    const P3<R>& P = p3_of<R>(c);
    k3_rho<S, R><<<gr, kBlock3, 0, c->stream>>>(c->g, P, c->flags, fs, rho);
    const int zc = zchunk3(c->g);
    auto* kern = march_kernel<S, R>(P);
    kern<<<march_grid(c->g, zc), kBlock3, k3_march_smem<R>(), c->stream>>>(
        c->g, P, zc, c->flags, fs, reinterpret_cast<const V2<R>*>(rho), state3<S>(c, 1 - c->cur), nullptr, nullptr);
    c->cur ^= 1;
    return cudaGetLastError();
}

// densities of the current state into c->rho, then the fields form of the step kernel (o5 may be
// NULL): the same pull, stencil sums, moments and forces as a step, per-block diagnostic records
cudaError_t run_fields(lbm3d_ctx* c, double* o5, bool diag) {
    return with_types3(c->storage, [&](auto* s_, auto* r_) {
        TYPES3(s_, r_);
        const Pair<S>* fs = state3<S>(c, c->cur);
        auto* rho = reinterpret_cast<typename Rho2<R>::T*>(c->rho);
        const P3<R>& P = p3_of<R>(c);
        k3_rho<S, R><<<grid3(c->g), kBlock3, 0, c->stream>>>(c->g, P, c->flags, fs, rho);
        const int zc = zchunk3(c->g);
        const dim3 gm = march_grid(c->g, zc);
        auto* kern = march_kernel<S, R, true>(P);
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k3_march_smem<R>());
        if (e != cudaSuccess) return e;
        kern<<<gm, kBlock3, k3_march_smem<R>(), c->stream>>>(c->g, P, zc, c->flags, fs, reinterpret_cast<const V2<R>*>(rho),
                                                             nullptr, o5, c->part);
        if (diag) {
            const long long nb = (long long)gm.x * gm.y * gm.z;  // <= c->nparts (one record per block)
            double* mid = c->part + c->nparts * k3DiagN;         // k3DiagMid records after the per-block ones
            k3_diag_mid<<<k3DiagMid, k3DiagMidThreads, 0, c->stream>>>(nb, c->part, mid);
            k3_diag_final<<<1, 32, 0, c->stream>>>(k3DiagMid, mid, c->dout);
        }
        return cudaGetLastError();
    });
}

cudaError_t density_pass(lbm3d_ctx* c) {
    return with_types3(c->storage, [&](auto* s_, auto* r_) {
        TYPES3(s_, r_);
        k3_rho<S, R><<<grid3(c->g), kBlock3, 0, c->stream>>>(c->g, p3_of<R>(c), c->flags, state3<S>(c, c->cur),
                                                           reinterpret_cast<typename Rho2<R>::T*>(c->rho));
        return cudaGetLastError();
    });
}

// the state from post-streaming populations (FP64 [38][N] on the device) / from densities
cudaError_t set_state3(lbm3d_ctx* c, const double* f, int buf) {
    return with_types3(c->storage, [&](auto* s_, auto* r_) {
        TYPES3(s_, r_);
        k3_set<S, R><<<grid3(c->g), kBlock3, 0, c->stream>>>(c->g, p3_of<R>(c), c->flags, f, state3<S>(c, buf));
        return cudaGetLastError();
    });
}
cudaError_t set_rest3(lbm3d_ctx* c, const double* a, const double* b) {
    return with_types3(c->storage, [&](auto* s_, auto* r_) {
        TYPES3(s_, r_);
        k3_set_rest<S, R><<<grid3(c->g), kBlock3, 0, c->stream>>>(c->g, p3_of<R>(c), c->flags, a, b, state3<S>(c, c->cur));
        return cudaGetLastError();
    });
}

template <class R>
cudaError_t ca_passes(lbm3d_ctx* c, const double* sc, double R_) {
    Ca3<R> ca{c->g, c->flags, reinterpret_cast<const typename Rho2<R>::T*>(c->rho), c->ca_cross};
    double* st = c->ca;
    double* part = c->ca + 16;
    cudaError_t e = cudaMemsetAsync(st, 0, 16 * sizeof(double), c->stream);
    if (e != cudaSuccess) return e;
    for (int pass = 0; pass < 4; ++pass) {
        auto* kern = pass == 0 ? k3_ca_pass<R, 0> : pass == 1 ? k3_ca_pass<R, 1> : pass == 2 ? k3_ca_pass<R, 2> : k3_ca_pass<R, 3>;
        kern<<<kC3Blocks, kC3Threads, 0, c->stream>>>(ca, st, part);
        k3_ca_solve<<<1, 32, 0, c->stream>>>(pass, kC3Blocks, part, st, sc[0], sc[1], sc[2], R_);
    }
    return cudaGetLastError();
}

void free_xfer3(lbm3d_ctx* c) {
    for (cudaStream_t* st : {&c->xs_in, &c->xs_out})
        if (*st) {
            cudaStreamSynchronize(*st);
            cudaStreamDestroy(*st);
            *st = nullptr;
        }
    for (int k = 0; k < 2; ++k) {
        for (cudaEvent_t* ev : {&c->xin_ready[k], &c->xin_free[k], &c->xout_ready[k], &c->xout_free[k]})
            if (*ev) cudaEventDestroy(*ev), *ev = nullptr;
        if (c->xin[k]) cudaFree(c->xin[k]), c->xin[k] = nullptr;
        if (c->xout[k]) cudaFree(c->xout[k]), c->xout[k] = nullptr;
    }
}

void free3(lbm3d_ctx* c) {
    free_xfer3(c);
    void* ptrs[] = {c->solid, c->flags, c->f[0], c->f[1], c->rho, c->part, c->dout, c->ca, c->ca_cross, c->scratch, c->dens};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

}  // namespace

#define TRY3(call, what)                                                                                 \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) {                                                                         \
            lbm_status s_ = e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;                    \
            if (e_ == cudaErrorMemoryAllocation) cudaGetLastError();                                     \
            return report_error(s_, "%s: %s", what, cudaGetErrorString(e_));                              \
        }                                                                                                \
    } while (0)

extern "C" lbm_status lbm3d_create(const lbm3d_grid* grid, const uint8_t* solid, const lbm3d_params* p,
                                   const double* rA0, const double* rB0, int32_t storage, void* cuda_stream,
                                   lbm3d_ctx** out) {
    if (!out) return report_error(LBM_EINVAL, "NULL output pointer");
    *out = nullptr;
    if (!grid || !solid || !p || !rA0 || !rB0) return report_error(LBM_EINVAL, "NULL argument");
    if (grid->nx < 5 || grid->ny < 5 || grid->nz < 5) return report_error(LBM_EINVAL, "nx, ny, nz must be >= 5");
    if (grid->ny > 65535 || grid->nz > 65535) return report_error(LBM_EINVAL, "ny, nz must be <= 65535");
    if ((long long)grid->nx * grid->ny * grid->nz > (1LL << 31) - 1) return report_error(LBM_EINVAL, "lattice too large (2^31 nodes)");
    if (storage < LBM_STORE_F64 || storage > LBM_STORE_BF16_SHIFTED) return report_error(LBM_EINVAL, "bad storage %d", storage);
    for (int k = 0; k < 2; ++k)
        if (!fin(p->tau[k]) || p->tau[k] <= 0.5) return report_error(LBM_EINVAL, "tau[%d] must be > 0.5", k);
    if (!fin(p->G_AB) || !fin(p->G_w2) || !fin(p->g[0]) || !fin(p->g[1]) || !fin(p->g[2]) || !fin(p->rho0_store[0]) ||
        !fin(p->rho0_store[1]))
        return report_error(LBM_EINVAL, "non-finite parameter");
    if (!fin(p->lambda) || p->lambda <= 0.0) return report_error(LBM_EINVAL, "lambda must be > 0");
    if (!fin(p->delta) || p->delta <= 0.0 || p->delta > 1.0) return report_error(LBM_EINVAL, "delta must lie in (0, 1]");
    if (p->mode != LBM_ADS_ORIGINAL && p->mode != LBM_ADS_IMPROVED) return report_error(LBM_EINVAL, "bad mode");
    if (p->second_layer != LBM_SECOND_LAYER_PSI_AND_SOLID && p->second_layer != LBM_SECOND_LAYER_PSI)
        return report_error(LBM_EINVAL, "bad second_layer");
    if (p->adhesion_stencil != LBM3_ADHESION_E8 && p->adhesion_stencil != LBM3_ADHESION_D3Q19)
        return report_error(LBM_EINVAL, "bad adhesion_stencil");
    const long long N = (long long)grid->nx * grid->ny * grid->nz;
    long long nf = 0;
    for (long long s = 0; s < N; ++s) {
        if (solid[s]) continue;
        ++nf;
        if (!fin(rA0[s]) || !fin(rB0[s]) || rA0[s] <= 0.0 || rB0[s] <= 0.0)
            return report_error(LBM_EINVAL, "initial densities must be finite and > 0 at fluid node %lld", s);
    }
    if (nf == 0) return report_error(LBM_EINVAL, "the mask has no fluid node");
    int dev = 0;
    cudaDeviceProp prop;
    TRY3(cudaGetDevice(&dev), "cudaGetDevice");
    TRY3(cudaGetDeviceProperties(&prop, dev), "cudaGetDeviceProperties");
    if (!(prop.major == 10 && prop.minor == 3))
        return report_error(LBM_ECUDA, "this library is built for sm_103a (GB300); device %d is sm_%d%d", dev, prop.major, prop.minor);

    lbm3d_ctx* c = new (std::nothrow) lbm3d_ctx();
    if (!c) return report_error(LBM_ENOMEM, "host allocation");
    auto bail = [&](lbm_status s) {
        free3(c);
        delete c;
        return s;
    };
#define STEP3(call, what)                                                                            \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) {                                                                     \
            lbm_status s_ = e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;                \
            if (e_ == cudaErrorMemoryAllocation) cudaGetLastError();                                 \
            report_error(s_, "%s: %s", what, cudaGetErrorString(e_));                                 \
            return bail(s_);                                                                         \
        }                                                                                            \
    } while (0)
    c->storage = storage;
    c->elem = storage == LBM_STORE_F64 ? 8 : (storage == LBM_STORE_F32 ? 4 : 2);  // bytes per stored value
    c->relem = storage == LBM_STORE_F64 ? 8 : 4;                                  // bytes per computed value
    c->g = Geo3{grid->nx, grid->ny, grid->nz, N};
    c->pf = make_p3<float>(*p);
    c->pd = make_p3<double>(*p);
    c->nfluid = nf;
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        STEP3(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking), "stream");
        c->own_stream = true;
    }
    const dim3 gr = grid3(c->g);
    c->nparts = (long long)gr.x * gr.y * gr.z;
    STEP3(cudaMalloc(&c->solid, N), "mask");
    STEP3(cudaMalloc(&c->flags, N * sizeof(uint32_t)), "flags");
    STEP3(cudaMalloc(&c->f[0], 38 * N * c->elem), "population buffer");
    STEP3(cudaMalloc(&c->f[1], 38 * N * c->elem), "population buffer");
    STEP3(cudaMalloc(&c->rho, 2 * N * c->relem), "densities");
    STEP3(cudaMalloc(&c->part, (c->nparts + k3DiagMid) * k3DiagN * sizeof(double)), "diagnostics");
    STEP3(cudaMalloc(&c->dout, k3DiagN * sizeof(double)), "diagnostics");
    STEP3(cudaMalloc(&c->ca, (16 + kC3Blocks * kC3Vals) * sizeof(double)), "contact-angle scratch");
    STEP3(cudaMalloc(&c->ca_cross, (size_t)c->g.N), "contact-angle scratch");
    STEP3(cudaMemsetAsync(c->f[0], 0, 38 * N * c->elem, c->stream), "memset");
    STEP3(cudaMemsetAsync(c->f[1], 0, 38 * N * c->elem, c->stream), "memset");
    STEP3(cudaMemcpy(c->solid, solid, N, cudaMemcpyHostToDevice), "mask upload");
    k3_flags<<<gr, kBlock3, 0, c->stream>>>(c->g, c->solid, c->flags);
    STEP3(cudaGetLastError(), "flags kernel");
    STEP3(scratch_for(c), "transfer scratch");
    STEP3(cudaMemcpyAsync(c->scratch + 36 * N, rA0, N * sizeof(double), cudaMemcpyHostToDevice, c->stream), "density upload");
    STEP3(cudaMemcpyAsync(c->scratch + 37 * N, rB0, N * sizeof(double), cudaMemcpyHostToDevice, c->stream), "density upload");
    STEP3(cudaStreamSynchronize(c->stream), "upload");
    // f = f^eq(rho, 0) into scratch [0, 38 N) -- the densities sit in its last two planes and are
    // read before planes 36, 37 are overwritten by the same thread
    k3_feq<double><<<gr, kBlock3, 0, c->stream>>>(c->g, c->solid, c->scratch + 36 * N, c->scratch + 37 * N, c->scratch);
    STEP3(cudaGetLastError(), "init kernel");
    STEP3(set_state3(c, c->scratch, 0), "init kernel");
    STEP3(cudaGetLastError(), "init kernel");
    STEP3(cudaStreamSynchronize(c->stream), "initialisation");
    cudaFree(c->scratch);  // transfers allocate it again on demand
    c->scratch = nullptr;
#undef STEP3
    *out = c;
    return LBM_OK;
}

extern "C" void lbm3d_destroy(lbm3d_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    free3(c);
    delete c;
}

extern "C" lbm_status lbm3d_step(lbm3d_ctx* c, int64_t n) {
    NvtxRange nvtx_("lbm3d_step");
    if (!c) return report_error(LBM_EINVAL, "NULL context");
    if (n < 0) return report_error(LBM_EINVAL, "n must be >= 0");
    TRY3(with_types3(c->storage,
                     [&](auto* s_, auto* r_) {
                         TYPES3(s_, r_);
                         // the step kernel's shared-memory ring exceeds the default dynamic limit in FP64
                         cudaError_t e = cudaFuncSetAttribute(march_kernel<S, R>(p3_of<R>(c)),
                                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                              (int)k3_march_smem<R>());
                         for (int64_t t = 0; t < n && e == cudaSuccess; ++t) e = step_once<S, R>(c);
                         return e;
                     }),
         "step kernels");
    return LBM_OK;
}

extern "C" lbm_status lbm3d_fields(lbm3d_ctx* c, double* rA, double* rB, double* ux, double* uy, double* uz,
                                   int32_t on_device) {
    NvtxRange nvtx_("lbm3d_fields");
    if (!c) return report_error(LBM_EINVAL, "NULL context");
    TRY3(scratch_for(c), "fields scratch");
    TRY3(run_fields(c, c->scratch, false), "fields kernels");
    double* outs[5] = {rA, rB, ux, uy, uz};
    const long long N = c->g.N;
    for (int q = 0; q < 5; ++q)
        if (outs[q])
            TRY3(cudaMemcpyAsync(outs[q], c->scratch + q * N, N * sizeof(double),
                                 on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream),
                 "fields copy");
    if (!on_device) TRY3(cudaStreamSynchronize(c->stream), "fields");
    return LBM_OK;
}

namespace {
// copy streams, staging and events of the overlapped transfers
lbm_status xfer3_setup(lbm3d_ctx* c) {
    if (c->xs_in) return LBM_OK;
    const size_t N = (size_t)c->g.N;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaMalloc(&c->xin[k], 2 * N * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&c->xout[k], 5 * N * sizeof(double));
        for (cudaEvent_t* ev : {&c->xin_ready[k], &c->xin_free[k], &c->xout_ready[k], &c->xout_free[k]})
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->xs_out, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->xs_in, cudaStreamNonBlocking);  // set last: marks done
    if (e != cudaSuccess) {
        const bool oom = e == cudaErrorMemoryAllocation;
        cudaGetLastError();
        free_xfer3(c);
        return report_error(oom ? LBM_ENOMEM : LBM_ECUDA, "overlapped transfers: %s", cudaGetErrorString(e));
    }
    return LBM_OK;
}
}  // namespace

extern "C" lbm_status lbm3d_set_densities_async(lbm3d_ctx* c, const double* rho_A, const double* rho_B) {
    NvtxRange nvtx_("lbm3d_set_densities_async");
    if (!c || !rho_A || !rho_B) return report_error(LBM_EINVAL, "NULL argument");
    const lbm_status s = xfer3_setup(c);
    if (s != LBM_OK) return s;
    const long long N = c->g.N;
    const int k = c->xin_k;
    c->xin_k ^= 1;
    double* a = c->xin[k];
    double* b = c->xin[k] + N;
    // the copy may start once the kernel that read this staging buffer two calls ago has run
    TRY3(cudaStreamWaitEvent(c->xs_in, c->xin_free[k], 0), "transfer order");
    TRY3(cudaMemcpyAsync(a, rho_A, N * sizeof(double), cudaMemcpyHostToDevice, c->xs_in), "upload");
    TRY3(cudaMemcpyAsync(b, rho_B, N * sizeof(double), cudaMemcpyHostToDevice, c->xs_in), "upload");
    TRY3(cudaEventRecord(c->xin_ready[k], c->xs_in), "transfer order");
    TRY3(cudaStreamWaitEvent(c->stream, c->xin_ready[k], 0), "transfer order");
    TRY3(set_rest3(c, a, b), "state kernel");
    TRY3(cudaGetLastError(), "state kernel");
    TRY3(cudaEventRecord(c->xin_free[k], c->stream), "transfer order");
    return LBM_OK;
}

extern "C" lbm_status lbm3d_fields_async(lbm3d_ctx* c, double* rho_A, double* rho_B, double* ux, double* uy,
                                         double* uz) {
    NvtxRange nvtx_("lbm3d_fields_async");
    if (!c) return report_error(LBM_EINVAL, "NULL context");
    const lbm_status s = xfer3_setup(c);
    if (s != LBM_OK) return s;
    const long long N = c->g.N;
    const int k = c->xout_k;
    c->xout_k ^= 1;
    // the fields pass may overwrite this staging buffer once its previous copy to the host is done;
    // the copies then run on their own stream, beside the context's next work
    TRY3(cudaStreamWaitEvent(c->stream, c->xout_free[k], 0), "transfer order");
    TRY3(run_fields(c, c->xout[k], false), "fields kernels");
    TRY3(cudaEventRecord(c->xout_ready[k], c->stream), "transfer order");
    TRY3(cudaStreamWaitEvent(c->xs_out, c->xout_ready[k], 0), "transfer order");
    double* outs[5] = {rho_A, rho_B, ux, uy, uz};
    for (int q = 0; q < 5; ++q)
        if (outs[q])
            TRY3(cudaMemcpyAsync(outs[q], c->xout[k] + q * N, N * sizeof(double), cudaMemcpyDeviceToHost, c->xs_out),
                 "fields copy");
    TRY3(cudaEventRecord(c->xout_free[k], c->xs_out), "transfer order");
    return LBM_OK;
}

extern "C" lbm_status lbm3d_synchronize(lbm3d_ctx* c) {
    if (!c) return report_error(LBM_EINVAL, "NULL context");
    for (cudaStream_t st : {c->xs_in, c->xs_out, c->stream})
        if (st) TRY3(cudaStreamSynchronize(st), "synchronize");
    return LBM_OK;
}

extern "C" lbm_status lbm3d_get_populations(lbm3d_ctx* c, double* f) {
    if (!c || !f) return report_error(LBM_EINVAL, "NULL argument");
    TRY3(scratch_for(c), "transfer scratch");
    TRY3(with_types3(c->storage,
                     [&](auto* s_, auto* r_) {
                         TYPES3(s_, r_);
                         k3_get<S, R><<<grid3(c->g), kBlock3, 0, c->stream>>>(c->g, p3_of<R>(c), c->flags,
                                                                            state3<S>(c, c->cur), c->scratch);
                         return cudaGetLastError();
                     }),
         "read-back kernel");
    TRY3(cudaGetLastError(), "read-back kernel");
    TRY3(cudaMemcpyAsync(f, c->scratch, (size_t)38 * c->g.N * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "read-back");
    TRY3(cudaStreamSynchronize(c->stream), "read-back");
    return LBM_OK;
}

extern "C" lbm_status lbm3d_set_densities(lbm3d_ctx* c, const double* rho_A, const double* rho_B, int32_t on_device) {
    if (!c || !rho_A || !rho_B) return report_error(LBM_EINVAL, "NULL argument");
    const long long N = c->g.N;
    const double *a = rho_A, *b = rho_B;
    if (!on_device) {
        if (!c->dens) TRY3(cudaMalloc(&c->dens, (size_t)2 * N * sizeof(double)), "density buffer");
        TRY3(cudaMemcpyAsync(c->dens, rho_A, N * sizeof(double), cudaMemcpyHostToDevice, c->stream), "upload");
        TRY3(cudaMemcpyAsync(c->dens + N, rho_B, N * sizeof(double), cudaMemcpyHostToDevice, c->stream), "upload");
        a = c->dens;
        b = c->dens + N;
    }
    TRY3(set_rest3(c, a, b), "state kernel");
    TRY3(cudaGetLastError(), "state kernel");
    if (!on_device) TRY3(cudaStreamSynchronize(c->stream), "upload");
    return LBM_OK;
}

extern "C" lbm_status lbm3d_set_populations(lbm3d_ctx* c, const double* f) {
    if (!c || !f) return report_error(LBM_EINVAL, "NULL argument");
    TRY3(scratch_for(c), "transfer scratch");
    TRY3(cudaMemcpyAsync(c->scratch, f, (size_t)38 * c->g.N * sizeof(double), cudaMemcpyHostToDevice, c->stream), "upload");
    TRY3(set_state3(c, c->scratch, c->cur), "state kernel");
    TRY3(cudaGetLastError(), "state kernel");
    TRY3(cudaStreamSynchronize(c->stream), "upload");
    return LBM_OK;
}

extern "C" lbm_status lbm3d_diagnostics(lbm3d_ctx* c, lbm3d_diag* out) {
    if (!c || !out) return report_error(LBM_EINVAL, "NULL argument");
    TRY3(run_fields(c, nullptr, true), "diagnostics kernels");
    double v[k3DiagN];
    TRY3(cudaMemcpyAsync(v, c->dout, sizeof v, cudaMemcpyDeviceToHost, c->stream), "diagnostics read-back");
    TRY3(cudaStreamSynchronize(c->stream), "diagnostics");
    out->mass_A = v[0];
    out->mass_B = v[1];
    out->mom_x = v[2];
    out->mom_y = v[3];
    out->mom_z = v[4];
    out->umax = v[5];
    out->rhoA_min = v[6];
    out->rhoA_max = v[7];
    out->rhoB_min = v[8];
    out->rhoB_max = v[9];
    out->n_fluid = (int64_t)llround(v[10]);
    out->unstable = v[11] != 0.0;
    out->pad_ = 0;
    if (out->unstable) return report_error(LBM_EUNSTABLE, "non-finite or non-positive density");
    return LBM_OK;
}

extern "C" lbm_status lbm3d_contact_angle(lbm3d_ctx* c, const double* sc, double R, double* theta_deg, double* fit_rms,
                                          int64_t* npoints) {
    if (!c || !sc) return report_error(LBM_EINVAL, "NULL argument");
    if (!(R > 0.0) || !fin(sc[0]) || !fin(sc[1]) || !fin(sc[2])) return report_error(LBM_EINVAL, "bad sphere");
    cudaError_t e = density_pass(c);
    TRY3(e, "density kernel");
    e = c->storage == LBM_STORE_F64 ? ca_passes<double>(c, sc, R) : ca_passes<float>(c, sc, R);
    TRY3(e, "contact-angle kernels");
    double h[16];
    TRY3(cudaMemcpyAsync(h, c->ca, sizeof h, cudaMemcpyDeviceToHost, c->stream), "contact-angle read-back");
    TRY3(cudaStreamSynchronize(c->stream), "contact angle");
    if (npoints) *npoints = (int64_t)llround(h[0]);
    if (h[10] != 0.0) return report_error(LBM_ESTATE, "only %.0f interface points", h[0]);
    if (theta_deg) *theta_deg = h[9];
    if (fit_rms) *fit_rms = h[8];
    return LBM_OK;
}
