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
// Two launches per call.  The point pass reads the flags and the FP64 densities of every node once
// and writes the crossings as keys (2 s + direction, s = Y nx + X) into a fixed segment per block of
// 4,096 nodes, in a fixed order; the sign test of rho^e is an integer compare of the densities' bit
// patterns (off the FP64 pipe, which is slow on this GPU), the interpolation is formed only at
// crossings.  The fit runs one block per case over those points: centroid, Kasa moments, the
// Gauss-Newton normal equations and the residual, each as a block sum in a fixed order, so results
// do not depend on scheduling and the single-case and the batched call agree bit for bit.
#include <math.h>

#include <vector>

#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr int kCaThreads = 256;                                  // threads of a point block
constexpr int kCaPerThread = 16;                                 // nodes per thread of a point block
constexpr int kCaNodesPerBlock = kCaThreads * kCaPerThread;      // 4,096 consecutive nodes
constexpr int kCaKeysPerBlock = 2 * kCaNodesPerBlock;            // at most two points per node
constexpr int kCaFitThreads = 256;
constexpr int kCaCache = 2048;                                   // points the fit keeps in shared memory
constexpr int kCaVals = 9;

// point blocks of one case: one per 4,096 nodes (the same in the single-case and the batched call,
// so that both find the same points in the same order)
int ca_blocks(long long n) { return (int)((n + kCaNodesPerBlock - 1) / kCaNodesPerBlock); }

// One case of a contact-angle launch.
struct CaCase {
    int nx, ny;
    const uint16_t* flags;  // node flags of the case
    const double* rA;       // FP64 densities of the case, [ny][nx]
    const double* rB;
    lbm_surface surf;
    long long blk;          // first point block: keys at blk * kCaKeysPerBlock, counts at blk
    long long pfx;          // first entry of the case's prefix of the block counts (nb + 1 entries)
    int nb;                 // point blocks
    double* st;             // 16-double status record
};

// fluid and more than three cells from any non-fluid site (precomputed by the flags kernel)
__device__ __forceinline__ bool usable(uint16_t fl) { return (fl & (kSolidBit | kNearSolidBit)) == 0; }

__device__ __forceinline__ double phi_of(double ra, double rb) { return (ra - rb) / (ra + rb); }

// phi > 0 without the division and off the FP64 pipe.  When both densities lie in (0, 2^1023) the
// sum is positive and finite, so phi has the sign of ra - rb (a difference of unequal doubles is
// never zero), and positive doubles order like their bit patterns read as integers.  Any other
// value (zero, negative, huge, non-finite) takes the quotient itself.
__device__ __forceinline__ bool phi_positive(double ra, double rb) {
    const long long ia = __double_as_longlong(ra), ib = __double_as_longlong(rb);
    constexpr long long kLo = 1, kHi = 0x7FDFFFFFFFFFFFFFLL;  // smallest subnormal .. largest double below 2^1023
    if (ia >= kLo && ia <= kHi && ib >= kLo && ib <= kHi) return ia > ib;
    return phi_of(ra, rb) > 0.0;
}

// Crossings owned by node s = Y nx + X: towards (X+1, Y) (h) and towards (X, Y+1) (v).
__device__ __forceinline__ void crossings(const CaCase& C, long long s, int X, int Y, int& h, int& v) {
    h = v = 0;
    if (!usable(C.flags[s])) return;
    const bool pa = phi_positive(C.rA[s], C.rB[s]);
    if (X + 1 < C.nx && usable(C.flags[s + 1])) h = pa != phi_positive(C.rA[s + 1], C.rB[s + 1]);
    if (Y + 1 < C.ny && usable(C.flags[s + C.nx])) v = pa != phi_positive(C.rA[s + C.nx], C.rB[s + C.nx]);
}

// Interface point of key = 2 s + dir: the zero of the linear interpolation of phi between node s
// and its neighbour along x (dir 0) or y (dir 1).
__device__ __forceinline__ void point_of(const CaCase& C, uint32_t key, double& px, double& py) {
    const int si = (int)(key >> 1);  // < 2^31: lattices hold at most 2^31 - 1 nodes
    const long long s = si;
    const long long q = (key & 1u) ? s + C.nx : s + 1;
    const int X = si % C.nx, Y = si / C.nx;
    const double a = phi_of(C.rA[s], C.rB[s]), b = phi_of(C.rA[q], C.rB[q]);
    const double f = a / (a - b);
    px = (key & 1u) ? (double)X : X + f;
    py = (key & 1u) ? Y + f : (double)Y;
}

// Point pass: block (lb, case) scans nodes [lb * 4096, +4096) of its case, thread t the nodes
// lb * 4096 + k * 256 + t (k = 0..15), and writes the keys of the crossings it finds to the block's
// segment in a fixed order (k, then node, horizontal before vertical), and their count.
__global__ void __launch_bounds__(kCaThreads) k_ca_points(const CaCase* __restrict__ cases, uint32_t* __restrict__ keys,
                                                          int* __restrict__ counts) {
    const CaCase& C = cases[blockIdx.y];
    const int lb = blockIdx.x;
    if (lb >= C.nb || C.surf.kind == LBM_SURFACE_NONE) return;
    const long long N = (long long)C.nx * C.ny;
    uint32_t* out = keys + (C.blk + lb) * (long long)kCaKeysPerBlock;
    __shared__ int wsum[2][kCaThreads / 32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const long long base = (long long)lb * kCaNodesPerBlock;
    // (X, Y) of this thread's node, advanced by a fixed stride: one division per thread
    int X = (int)((base + t) % C.nx), Y = (int)((base + t) / C.nx);
    int running = 0;
    for (int k = 0; k < kCaPerThread; ++k) {
        const long long s = base + k * kCaThreads + t;
        if (k > 0) {
            X += kCaThreads;
            while (X >= C.nx) {
                X -= C.nx;
                ++Y;
            }
        }
        int h = 0, v = 0;
        if (s < N) crossings(C, s, X, Y, h, v);
        const int c = h + v;
        int incl = c;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += o;
        }
        if (lane == 31) wsum[k & 1][warp] = incl;
        __syncthreads();  // (one buffer per parity: the next writer of this one is two barriers away)
        int before = running, total = 0;
#pragma unroll
        for (int w = 0; w < kCaThreads / 32; ++w) {
            const int x = wsum[k & 1][w];
            before += w < warp ? x : 0;
            total += x;
        }
        int pos = before + incl - c;
        if (h) out[pos++] = (uint32_t)(2 * s);
        if (v) out[pos] = (uint32_t)(2 * s + 1);
        running += total;
    }
    if (t == 0) counts[C.blk + lb] = running;
}

// Block-wide sum of kCaVals per-thread values in a fixed order (lane butterfly, then the warps in
// order); the result is valid in thread 0.
__device__ void block_sum(const double* acc, double (*red)[kCaVals], double* S) {
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
            for (int w = 0; w < kCaFitThreads / 32; ++w) v += red[w][q];
            S[q] = v;
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

// st: 0 N, 1 xm, 2 ym, 3 cx, 4 cy, 5 r, 6 rms, 7 theta, 8 status (0 ok, 1 too few points).
// Stage 0 centroid; 1 Kasa fit in centroid coordinates; 2 one Gauss-Newton step on |p - c| - r;
// 3 rms residual and the angle.
__device__ void ca_solve(int pass, const double* S, double* st, const lbm_surface& surf) {
    if (pass == 0) {
        st[1] = S[1] / st[0];
        st[2] = S[2] / st[0];
    } else if (pass == 1) {
        const double Suu = S[0], Suv = S[1], Svv = S[2];
        const double b0 = 0.5 * (S[3] + S[4]), b1 = 0.5 * (S[5] + S[6]);
        const double det = Suu * Svv - Suv * Suv;
        const double uc = (b0 * Svv - Suv * b1) / det;
        const double vc = (Suu * b1 - Suv * b0) / det;
        st[5] = sqrt(uc * uc + vc * vc + (Suu + Svv) / st[0]);
        st[3] = st[1] + uc;
        st[4] = st[2] + vc;
    } else if (pass == 2) {
        double A[3][3] = {{S[0], S[1], S[2]}, {S[1], S[3], S[4]}, {S[2], S[4], S[5]}};
        double b[3] = {-S[6], -S[7], -S[8]};
        double d[3];
        solve3(A, b, d);
        st[3] += d[0];
        st[4] += d[1];
        st[5] += d[2];
    } else {
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

// Fit: one block per case.  The block counts of the point pass are turned into a prefix, so that
// point j of the case (in the pass's order) is found by a binary search; thread t takes points
// t, t + 256, ... in every stage, so each stage's sums are formed in a fixed order.  The first
// kCaCache points are kept in shared memory after the first stage.
__global__ void __launch_bounds__(kCaFitThreads) k_ca_fit(const CaCase* __restrict__ cases,
                                                          const uint32_t* __restrict__ keys,
                                                          const int* __restrict__ counts, long long* __restrict__ pfx_all) {
    const CaCase& C = cases[blockIdx.x];
    if (C.surf.kind == LBM_SURFACE_NONE) return;
    __shared__ double2 cache[kCaCache];
    __shared__ double red[kCaFitThreads / 32][kCaVals];
    __shared__ double sst[16];
    __shared__ int scan_w[kCaFitThreads / 32];
    __shared__ long long carry;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    long long* P = pfx_all + C.pfx;
    if (t == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < C.nb; b0 += kCaFitThreads) {
        const int b = b0 + t;
        const int c = b < C.nb ? counts[C.blk + b] : 0;
        int incl = c;
        for (int off = 1; off < 32; off <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += o;
        }
        if (lane == 31) scan_w[warp] = incl;
        __syncthreads();
        long long before = carry, total = 0;
        for (int w = 0; w < kCaFitThreads / 32; ++w) {
            before += w < warp ? scan_w[w] : 0;
            total += scan_w[w];
        }
        if (b < C.nb) P[b] = before + incl - c;
        __syncthreads();
        if (t == 0) carry += total;
        __syncthreads();
    }
    const long long N = carry;
    if (t == 0) P[C.nb] = N;
    if (t < 16) sst[t] = 0.0;
    __syncthreads();
    if (t == 0) {
        sst[0] = (double)N;
        sst[8] = N < 8 ? 1.0 : 0.0;
    }
    __syncthreads();
    if (N >= 8) {
        auto point = [&](long long j, double& px, double& py) {
            int lo = 0, hi = C.nb - 1;  // the last block whose first point is at or before j
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (P[mid] <= j) lo = mid;
                else hi = mid - 1;
            }
            point_of(C, keys[(C.blk + lo) * (long long)kCaKeysPerBlock + (j - P[lo])], px, py);
        };
        for (int pass = 0; pass < 4; ++pass) {
            double acc[kCaVals];
            for (int q = 0; q < kCaVals; ++q) acc[q] = 0.0;
            const double xm = sst[1], ym = sst[2], cxv = sst[3], cyv = sst[4], r = sst[5];
            for (long long j = t; j < N; j += kCaFitThreads) {
                double px, py;
                if (pass > 0 && j < kCaCache) {
                    px = cache[j].x;
                    py = cache[j].y;
                } else {
                    point(j, px, py);
                    if (j < kCaCache) cache[j] = make_double2(px, py);
                }
                if (pass == 0) {
                    acc[1] += px;
                    acc[2] += py;
                } else if (pass == 1) {
                    const double u = px - xm, v = py - ym;
                    acc[0] += u * u;
                    acc[1] += u * v;
                    acc[2] += v * v;
                    acc[3] += u * u * u;
                    acc[4] += u * v * v;
                    acc[5] += v * v * v;
                    acc[6] += v * u * u;
                } else if (pass == 2) {
                    const double dx = px - cxv, dy = py - cyv;
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
                    const double dx = px - cxv, dy = py - cyv;
                    const double res = sqrt(dx * dx + dy * dy) - r;
                    acc[0] += res * res;
                }
            }
            double S[kCaVals];
            block_sum(acc, red, S);
            if (t == 0) ca_solve(pass, S, sst, C.surf);
            __syncthreads();
        }
    }
    if (t < 16) C.st[t] = sst[t];
}

// Device tables of the contact-angle launches: ncases + 1 case records (the last one serves the
// single-case call), the keys and counts of every case's point blocks, and the prefixes.
struct CaLayout {
    size_t o_cases, o_keys, o_counts, o_pfx, total;
    std::vector<long long> blk, pfx;
    std::vector<int> nb;
    long long nblk = 0;
    explicit CaLayout(const Ctx& c) {
        const int n = (int)c.hcases.size();
        blk.resize(n);
        pfx.resize(n);
        nb.resize(n);
        long long p = 0;
        for (int i = 0; i < n; ++i) {
            nb[i] = ca_blocks((long long)c.hcases[i].nx * c.hcases[i].ny);
            blk[i] = nblk;
            pfx[i] = p;
            nblk += nb[i];
            p += nb[i] + 1;
        }
        auto al = [](size_t x) { return (x + 255) / 256 * 256; };
        o_cases = 0;
        o_keys = al((size_t)(n + 1) * sizeof(CaCase));
        o_counts = o_keys + al((size_t)nblk * kCaKeysPerBlock * sizeof(uint32_t));
        o_pfx = o_counts + al((size_t)nblk * sizeof(int));
        total = o_pfx + al((size_t)p * sizeof(long long));
    }
};

cudaError_t ensure_points(Ctx& c) {
    if (c.ca_points) return cudaSuccess;
    const CaLayout L(c);
    cudaError_t e = cudaMalloc(&c.ca_points, L.total);
    if (e != cudaSuccess) {
        c.ca_points = nullptr;
        return e;
    }
    c.device_bytes += (long long)L.total;
    return cudaSuccess;
}

CaCase case_record(const Ctx& c, const CaLayout& L, int i, const double* rA, const double* rB,
                   const lbm_surface& surf, double* st) {
    const DevCase& d = c.hcases[i];
    return CaCase{d.nx, d.ny, c.flags + d.d_off, rA, rB, surf, L.blk[i], L.pfx[i], L.nb[i], st};
}

cudaError_t launch_ca(Ctx& c, const CaLayout& L, int first_record, int nrec, int max_nb) {
    const CaCase* cases = reinterpret_cast<const CaCase*>(c.ca_points + L.o_cases) + first_record;
    uint32_t* keys = reinterpret_cast<uint32_t*>(c.ca_points + L.o_keys);
    int* counts = reinterpret_cast<int*>(c.ca_points + L.o_counts);
    long long* pfx = reinterpret_cast<long long*>(c.ca_points + L.o_pfx);
    for (int c0 = 0; c0 < nrec; c0 += 65535) {  // grid y: at most 65,535 cases per launch
        const int m = nrec - c0 < 65535 ? nrec - c0 : 65535;
        k_ca_points<<<dim3((unsigned)max_nb, (unsigned)m), kCaThreads, 0, c.stream>>>(cases + c0, keys, counts);
    }
    k_ca_fit<<<(unsigned)nrec, kCaFitThreads, 0, c.stream>>>(cases, keys, counts, pfx);
    return cudaGetLastError();
}

}  // namespace

// ctx->fields must already hold rho_A, rho_B of the case (dense).  The 16-double status record st
// (device) receives theta at [7], rms at [6], points at [0], the too-few-points flag at [8].
cudaError_t enqueue_contact_angle(Ctx& c, int ci, const lbm_surface& surf, double* st) {
    cudaError_t e = ensure_points(c);
    if (e != cudaSuccess) return e;
    const CaLayout L(c);
    const int n = (int)c.hcases.size();
    const long long N = (long long)c.hcases[ci].nx * c.hcases[ci].ny;
    const CaCase rec = case_record(c, L, ci, c.fields, c.fields + N, surf, st);
    e = cudaMemcpyAsync(c.ca_points + L.o_cases + (size_t)n * sizeof(CaCase), &rec, sizeof rec,
                        cudaMemcpyHostToDevice, c.stream);
    if (e != cudaSuccess) return e;
    return launch_ca(c, L, n, 1, L.nb[ci]);
}

cudaError_t enqueue_contact_angle_all(Ctx& c, const lbm_surface* surf) {
    const int n = (int)c.hcases.size();
    cudaError_t e = ensure_points(c);
    if (e != cudaSuccess) return e;
    if (!c.ca_batch) {  // FP64 densities of all cases, [2][dense_elems]
        const size_t bytes = 2 * (size_t)c.dense_elems * sizeof(double);
        e = cudaMalloc(&c.ca_batch, bytes);
        if (e != cudaSuccess) {
            c.ca_batch = nullptr;
            return e;
        }
        c.ca_batch_bytes = bytes;
        c.device_bytes += (long long)bytes;
    }
    double* rho = reinterpret_cast<double*>(c.ca_batch);
    if (c.ca_rho_version != c.version) {  // not already written at this state by the diagnostics
        e = launch_densities_all(c, rho, rho + c.dense_elems);
        if (e != cudaSuccess) return e;
        c.ca_rho_version = c.version;
    }
    const CaLayout L(c);
    std::vector<CaCase> recs(n);
    int max_nb = 1;
    for (int i = 0; i < n; ++i) {
        const DevCase& d = c.hcases[i];
        recs[i] = case_record(c, L, i, rho + d.d_off, rho + c.dense_elems + d.d_off, surf[i], c.ca_all + 16 * (size_t)i);
        if (surf[i].kind != LBM_SURFACE_NONE && L.nb[i] > max_nb) max_nb = L.nb[i];
    }
    e = cudaMemcpyAsync(c.ca_points + L.o_cases, recs.data(), (size_t)n * sizeof(CaCase), cudaMemcpyHostToDevice,
                        c.stream);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(c.ca_all, 0, (size_t)16 * n * sizeof(double), c.stream);
    if (e != cudaSuccess) return e;
    return launch_ca(c, L, 0, n, max_nb);
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

int contact_work_doubles() { return 16; }

}  // namespace lbm
