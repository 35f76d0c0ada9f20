// Contact angle of a droplet of component A (Sec. 3.2), measured on the device in FP64.
//
// Interface points: along every lattice row and column, between two neighbouring fluid nodes that
// lie more than three cells (Chebyshev) from any non-fluid site (flag bit kNearSolidBit), where the
// effective density rho^e = (rho_A - rho_B) / (rho_A + rho_B) (Eq. 10) changes sign (> 0 on one side, <= 0 on the
// other), the zero of its linear interpolation.  Pairs across a periodic seam are not used.
// Circle: algebraic (Kasa) fit in centroid coordinates, then one Gauss-Newton step on the geometric
// residuals |p - c| - r.  Angle: cos theta = (R^2 + r^2 - d^2) / (2 r R) for a circular solid of
// centre distance d; cos theta = -normal (c_y - y_w) / r for a flat wall.
//
// Every reduction writes one partial record per block, and a single thread combines the records in
// block order, so results do not depend on scheduling.
#include <math.h>

#include <vector>

#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr int kCaThreads = 256;
constexpr int kCaBlocks = 256;             // most blocks per case
constexpr int kCaNodesPerBlock = 4096;
constexpr int kCaVals = 9;

// blocks of one case's passes: one per 4,096 nodes, 1..256 (the same in the single-case and the
// batched call, so both sum the same partial records in the same order)
int ca_blocks(long long n) {
    const long long b = (n + kCaNodesPerBlock - 1) / kCaNodesPerBlock;
    return (int)(b < 1 ? 1 : (b > kCaBlocks ? kCaBlocks : b));
}

struct CaGeo {
    int nx, ny;
    const uint16_t* flags;  // node flags of the case
    const double* rA;
    const double* rB;
};

// fluid and more than three cells from any non-fluid site (precomputed by the flags kernel)
__device__ bool usable(const CaGeo& g, int X, int Y) {
    return (g.flags[(long long)Y * g.nx + X] & (kSolidBit | kNearSolidBit)) == 0;
}

__device__ double phi_of(double ra, double rb) { return (ra - rb) / (ra + rb); }

// phi > 0 without the division where 0 < rho_A + rho_B < inf: the quotient then has the sign of
// the difference, which is at least an ulp of the larger density and cannot underflow to zero.
__device__ bool phi_positive(double ra, double rb) {
    const double sum = ra + rb;
    return (sum > 0.0 && sum < INFINITY) ? ra > rb : phi_of(ra, rb) > 0.0;
}

// Up to two crossing points owned by node (X, Y): towards (X+1, Y) and towards (X, Y+1).  phi is
// formed only at the two ends of a crossing.
__device__ int node_points(const CaGeo& g, int X, int Y, double* px, double* py) {
    int n = 0;
    if (!usable(g, X, Y)) return 0;
    const long long s = (long long)Y * g.nx + X;
    const double ra = g.rA[s], rb = g.rB[s];
    const bool pa = phi_positive(ra, rb);
    if (X + 1 < g.nx && usable(g, X + 1, Y)) {
        const double qa = g.rA[s + 1], qb = g.rB[s + 1];
        if (pa != phi_positive(qa, qb)) {
            const double a = phi_of(ra, rb), b = phi_of(qa, qb);
            px[n] = X + a / (a - b);
            py[n] = (double)Y;
            ++n;
        }
    }
    if (Y + 1 < g.ny && usable(g, X, Y + 1)) {
        const double qa = g.rA[s + g.nx], qb = g.rB[s + g.nx];
        if (pa != phi_positive(qa, qb)) {
            const double a = phi_of(ra, rb), b = phi_of(qa, qb);
            px[n] = (double)X;
            py[n] = Y + a / (a - b);
            ++n;
        }
    }
    return n;
}

// st: 0 N, 1 xm, 2 ym, 3 cx, 4 cy, 5 r, 6 rms, 7 theta, 8 status (0 ok, 1 too few points)
// Block lb of nb of one case: nodes lb * threads + tid, strided by nb * threads; its partial record
// goes to out[0 .. kCaVals).
__device__ void ca_pass_block(const CaGeo& g, int lb, int nb, int pass, const double* __restrict__ st,
                              double* __restrict__ out) {
    double acc[kCaVals];
    for (int q = 0; q < kCaVals; ++q) acc[q] = 0.0;
    const long long N = (long long)g.nx * g.ny;
    const double xm = st[1], ym = st[2], cxv = st[3], cyv = st[4], r = st[5];
    // node s = Y nx + X advanced by a fixed stride: one division per thread, not per node
    const long long s0 = lb * (long long)blockDim.x + threadIdx.x, stride = (long long)nb * blockDim.x;
    const int dX = (int)(stride % g.nx), dY = (int)(stride / g.nx);
    int X = (int)(s0 % g.nx), Y = (int)(s0 / g.nx);
    for (long long s = s0; s < N; s += stride) {
        if (s != s0) {
            X += dX;
            Y += dY;
            if (X >= g.nx) {
                X -= g.nx;
                ++Y;
            }
        }
        double px[2], py[2];
        const int n = node_points(g, X, Y, px, py);
        for (int k = 0; k < n; ++k) {
            if (pass == 0) {
                acc[0] += 1.0;
                acc[1] += px[k];
                acc[2] += py[k];
            } else if (pass == 1) {
                const double u = px[k] - xm, v = py[k] - ym;
                acc[0] += u * u;
                acc[1] += u * v;
                acc[2] += v * v;
                acc[3] += u * u * u;
                acc[4] += u * v * v;
                acc[5] += v * v * v;
                acc[6] += v * u * u;
            } else if (pass == 2) {
                const double dx = px[k] - cxv, dy = py[k] - cyv;
                const double d = sqrt(dx * dx + dy * dy);
                const double res = d - r;
                const double j0 = -dx / d, j1 = -dy / d, j2 = -1.0;
                acc[0] += j0 * j0;
                acc[1] += j0 * j1;
                acc[2] += j0 * j2;
                acc[3] += j1 * j1;
                acc[4] += j1 * j2;
                acc[5] += j2 * j2;
                acc[6] += j0 * res;
                acc[7] += j1 * res;
                acc[8] += j2 * res;
            } else {
                const double dx = px[k] - cxv, dy = py[k] - cyv;
                const double res = sqrt(dx * dx + dy * dy) - r;
                acc[0] += res * res;
            }
        }
    }
    __shared__ double red[kCaThreads / 32][kCaVals];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = 0; q < kCaVals; ++q) {
        double v = acc[q];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) red[warp][q] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int q = 0; q < kCaVals; ++q) {
            double v = 0.0;
            for (int w = 0; w < kCaThreads / 32; ++w) v += red[w][q];
            out[q] = v;
        }
}

__global__ void k_ca_pass(CaGeo g, int pass, const double* __restrict__ st, double* __restrict__ part) {
    ca_pass_block(g, blockIdx.x, gridDim.x, pass, st, part + (long long)blockIdx.x * kCaVals);
}

// Batched passes: block b belongs to case blk_case[b], whose blocks are [blk0[case], blk0[case+1]).
struct CaBatch {
    const CaGeo* geo;          // per case
    const int* blk_case;       // per block
    const int* blk0;           // per case + 1
    const lbm_surface* surf;   // per case
    double* st;                // per case: 16-double status record
    double* part;              // per block: kCaVals partial sums
};

__global__ void k_ca_pass_all(CaBatch b, int pass) {
    const int ci = b.blk_case[blockIdx.x];
    if (b.surf[ci].kind == LBM_SURFACE_NONE) return;  // skipped: its partials are never read
    const int b0 = b.blk0[ci];
    ca_pass_block(b.geo[ci], blockIdx.x - b0, b.blk0[ci + 1] - b0, pass, b.st + 16 * (long long)ci,
                  b.part + (long long)blockIdx.x * kCaVals);
}

// Sum of the per-block partial records by one warp: lane l adds blocks l, l+32, ... in order, then
// a fixed butterfly combines the lanes (deterministic).
__device__ void sum_parts(const double* part, int nblocks, double* out) {
    const int lane = threadIdx.x & 31;
    for (int q = 0; q < kCaVals; ++q) {
        double v = 0.0;
        for (int b = lane; b < nblocks; b += 32) v += part[b * kCaVals + q];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        out[q] = v;
    }
}

// 3x3 solve by Gaussian elimination with partial pivoting.
__device__ void solve3(double A[3][3], double b[3], double x[3]) {
    for (int c = 0; c < 3; ++c) {
        int p = c;
        for (int r = c + 1; r < 3; ++r)
            if (fabs(A[r][c]) > fabs(A[p][c])) p = r;
        for (int k = 0; k < 3; ++k) {
            const double t = A[c][k];
            A[c][k] = A[p][k];
            A[p][k] = t;
        }
        const double t = b[c];
        b[c] = b[p];
        b[p] = t;
        for (int r = c + 1; r < 3; ++r) {
            const double f = A[r][c] / A[c][c];
            for (int k = c; k < 3; ++k) A[r][k] -= f * A[c][k];
            b[r] -= f * b[c];
        }
    }
    for (int r = 2; r >= 0; --r) {
        double s = b[r];
        for (int k = r + 1; k < 3; ++k) s -= A[r][k] * x[k];
        x[r] = s / A[r][r];
    }
}

__device__ void ca_solve(int pass, int nblocks, const double* __restrict__ part, double* __restrict__ st,
                         const lbm_surface& surf) {
    double S[kCaVals];
    sum_parts(part, nblocks, S);  // the whole warp
    if (threadIdx.x != 0) return;
    if (pass == 0) {
        st[0] = S[0];
        st[8] = S[0] < 8.0 ? 1.0 : 0.0;
        st[1] = S[0] > 0.0 ? S[1] / S[0] : 0.0;
        st[2] = S[0] > 0.0 ? S[2] / S[0] : 0.0;
    } else if (pass == 1) {
        if (st[8] != 0.0) return;
        const double Suu = S[0], Suv = S[1], Svv = S[2];
        const double b0 = 0.5 * (S[3] + S[4]), b1 = 0.5 * (S[5] + S[6]);
        const double det = Suu * Svv - Suv * Suv;
        const double uc = (b0 * Svv - Suv * b1) / det;
        const double vc = (Suu * b1 - Suv * b0) / det;
        st[5] = sqrt(uc * uc + vc * vc + (Suu + Svv) / st[0]);
        st[3] = st[1] + uc;
        st[4] = st[2] + vc;
    } else if (pass == 2) {
        if (st[8] != 0.0) return;
        double A[3][3] = {{S[0], S[1], S[2]}, {S[1], S[3], S[4]}, {S[2], S[4], S[5]}};
        double b[3] = {-S[6], -S[7], -S[8]};
        double d[3];
        solve3(A, b, d);
        st[3] += d[0];
        st[4] += d[1];
        st[5] += d[2];
    } else {
        if (st[8] != 0.0) return;
        st[6] = sqrt(S[0] / st[0]);
        const double cxv = st[3], cyv = st[4], r = st[5];
        double c;
        if (surf.kind == LBM_SURFACE_FLAT) {
            c = -(double)surf.normal * (cyv - surf.y_w) / r;
        } else {
            const double d2 = (cxv - surf.cx) * (cxv - surf.cx) + (cyv - surf.cy) * (cyv - surf.cy);
            c = (surf.R * surf.R + r * r - d2) / (2.0 * r * surf.R);
        }
        c = c > 1.0 ? 1.0 : (c < -1.0 ? -1.0 : c);
        st[7] = acos(c) * (180.0 / 3.14159265358979323846);
    }
}

__global__ void k_ca_solve(int pass, int nblocks, const double* __restrict__ part, double* __restrict__ st,
                           lbm_surface surf) {
    ca_solve(pass, nblocks, part, st, surf);
}

// one warp per case
__global__ void k_ca_solve_all(CaBatch b, int pass) {
    const int ci = blockIdx.x;
    const lbm_surface surf = b.surf[ci];
    if (surf.kind == LBM_SURFACE_NONE) return;
    const int b0 = b.blk0[ci];
    ca_solve(pass, b.blk0[ci + 1] - b0, b.part + (long long)b0 * kCaVals, b.st + 16 * (long long)ci, surf);
}

}  // namespace

// ctx->fields must already hold rho_A, rho_B of the case (dense).  host_out4 <- theta, rms, npoints,
// status.
cudaError_t enqueue_contact_angle(Ctx& c, int ci, const lbm_surface& surf, double* st) {
    const DevCase& C = c.hcases[ci];
    const long long N = (long long)C.nx * C.ny;
    CaGeo g{C.nx, C.ny, c.flags + C.d_off, c.fields, c.fields + N};
    double* part = c.ca_work + 16;
    const int nb = ca_blocks(N);
    cudaError_t e = cudaMemsetAsync(st, 0, 16 * sizeof(double), c.stream);
    if (e != cudaSuccess) return e;
    for (int pass = 0; pass < 4; ++pass) {
        k_ca_pass<<<nb, kCaThreads, 0, c.stream>>>(g, pass, st, part);
        k_ca_solve<<<1, 32, 0, c.stream>>>(pass, nb, part, st, surf);
    }
    return cudaGetLastError();
}

cudaError_t enqueue_contact_angle_all(Ctx& c, const lbm_surface* surf) {
    const int n = (int)c.hcases.size();
    // block tables
    std::vector<int> blk0(n + 1), blk_case;
    for (int i = 0; i < n; ++i) {
        blk0[i] = (int)blk_case.size();
        const int nb = ca_blocks((long long)c.hcases[i].nx * c.hcases[i].ny);
        blk_case.insert(blk_case.end(), nb, i);
    }
    blk0[n] = (int)blk_case.size();
    const int nblk = blk0[n];
    // one allocation: densities [2][dense_elems], geometry, tables, partials, surfaces
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t o_rho = 0, o_geo = al(2 * (size_t)c.dense_elems * sizeof(double));
    const size_t o_bc = o_geo + al(n * sizeof(CaGeo)), o_b0 = o_bc + al(nblk * sizeof(int));
    const size_t o_part = o_b0 + al((n + 1) * sizeof(int)), o_surf = o_part + al((size_t)nblk * kCaVals * sizeof(double));
    const size_t total = o_surf + al(n * sizeof(lbm_surface));
    cudaError_t e;
    if (!c.ca_batch) {
        e = cudaMalloc(&c.ca_batch, total);
        if (e != cudaSuccess) return e;
        c.ca_batch_bytes = total;
        c.device_bytes += (long long)total;
        double* rho = reinterpret_cast<double*>(c.ca_batch + o_rho);
        std::vector<CaGeo> geo(n);
        for (int i = 0; i < n; ++i) {
            const DevCase& d = c.hcases[i];
            geo[i] = CaGeo{d.nx, d.ny, c.flags + d.d_off, rho + d.d_off, rho + c.dense_elems + d.d_off};
        }
        e = cudaMemcpy(c.ca_batch + o_geo, geo.data(), n * sizeof(CaGeo), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c.ca_batch + o_bc, blk_case.data(), nblk * sizeof(int), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c.ca_batch + o_b0, blk0.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
    }
    e = cudaMemcpyAsync(c.ca_batch + o_surf, surf, n * sizeof(lbm_surface), cudaMemcpyHostToDevice, c.stream);
    if (e != cudaSuccess) return e;
    double* rho = reinterpret_cast<double*>(c.ca_batch + o_rho);
    if (c.ca_rho_version != c.version) {  // not already written at this state by the diagnostics
        e = launch_densities_all(c, rho, rho + c.dense_elems);
        if (e != cudaSuccess) return e;
        c.ca_rho_version = c.version;
    }
    e = cudaMemsetAsync(c.ca_all, 0, (size_t)16 * n * sizeof(double), c.stream);
    if (e != cudaSuccess) return e;
    CaBatch b{reinterpret_cast<const CaGeo*>(c.ca_batch + o_geo), reinterpret_cast<const int*>(c.ca_batch + o_bc),
              reinterpret_cast<const int*>(c.ca_batch + o_b0), reinterpret_cast<const lbm_surface*>(c.ca_batch + o_surf),
              c.ca_all, reinterpret_cast<double*>(c.ca_batch + o_part)};
    for (int pass = 0; pass < 4; ++pass) {
        k_ca_pass_all<<<nblk, kCaThreads, 0, c.stream>>>(b, pass);
        k_ca_solve_all<<<n, 32, 0, c.stream>>>(b, pass);
    }
    return cudaGetLastError();
}

cudaError_t launch_contact_angle(Ctx& c, int ci, const lbm_surface& surf, double* host_out4) {
    double* st = c.ca_work;
    cudaError_t e = enqueue_contact_angle(c, ci, surf, st);
    if (e != cudaSuccess) return e;
    double h[16];
    e = cudaMemcpyAsync(h, st, sizeof(h), cudaMemcpyDeviceToHost, c.stream);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return e;
    host_out4[0] = h[7];
    host_out4[1] = h[6];
    host_out4[2] = h[0];
    host_out4[3] = h[8];
    return cudaSuccess;
}

int contact_work_doubles() { return 16 + kCaBlocks * kCaVals; }

}  // namespace lbm
