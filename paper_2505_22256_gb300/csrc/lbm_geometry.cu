// Geometry preprocessing on the device: node flags (solid, blocked links for halfway bounce-back,
// wall-list membership) and the wall list with the second-layer reconstruction of Sec. 2.4.
//
// Wall list: the fluid nodes whose 24-node eighth-order stencil reaches a site that is not an
// in-array fluid node (solid, or outside the array along a non-periodic axis), in increasing node
// order y*nx + x.  For each entry:
//   subst  bit n-1 set when second-layer stencil node n (Table 1 numbering) is not a fluid node and
//          therefore takes the information of its first-layer partner x + sign(e_n)
//   seff   bit n-1 set when stencil node n counts as solid in the adhesion sum (Eq. 9): a solid or
//          outside first-layer site, or a replaced second-layer node whose partner is one (when it
//          copies the pseudopotential only: whose own site is one, clamped along an open axis)
//   a      sum_n w(|e_n|^2) seff_n e_n  (FP64)
// With the adhesion sum of Eq. 9 as printed (LBM_ADHESION_D2Q9) only the first layer enters it:
// seff keeps the first-layer bits and a = sum_i w_i s(x + e_i) e_i with the D2Q9 weights, opposite
// velocities taken together (i = 1, 2, 5, 6 with opp(i)).
// Along an open axis a first-layer site beyond the boundary column is the boundary column itself.
#include "lbm_internal.h"

namespace lbm {

namespace {

struct Geo {
    int nx, ny, bc_x, bc_y;
    const uint8_t* solid;  // dense [ny][nx]
};

// Is (X, Y) a fluid node after the periodic wrap?  Outside a non-periodic axis: no.
__device__ __forceinline__ bool fluid_at(const Geo& g, int X, int Y) {
    if (X < 0 || X >= g.nx) {
        if (g.bc_x != kPeriodic) return false;
        X = ((X % g.nx) + g.nx) % g.nx;
    }
    if (Y < 0 || Y >= g.ny) {
        if (g.bc_y != kPeriodic) return false;
        Y = ((Y % g.ny) + g.ny) % g.ny;
    }
    return g.solid[(long long)Y * g.nx + X] == 0;
}

// Solid switch of a first-layer site (dx, dy in {-1, 0, 1}).
__device__ __forceinline__ bool first_layer_solid(const Geo& g, int X, int Y, int dx, int dy) {
    int Xs = X + dx;
    if (g.bc_x == kOpen) Xs = Xs < 0 ? 0 : (Xs > g.nx - 1 ? g.nx - 1 : Xs);
    return !fluid_at(g, Xs, Y + dy);
}

__global__ void k_flags(const DevCase* __restrict__ cases, int c, const uint8_t* __restrict__ solid_all,
                        uint16_t* __restrict__ flags_all, int32_t* __restrict__ row_counts) {
    const DevCase C = cases[c];
    const Geo g{C.nx, C.ny, C.bc_x, C.bc_y, solid_all + C.d_off};
    const long long N = (long long)C.nx * C.ny;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N; s += (long long)gridDim.x * blockDim.x) {
        const int X = (int)(s % C.nx), Y = (int)(s / C.nx);
        const long long o = C.d_off + s;
        if (g.solid[s]) {
            flags_all[o] = kSolidBit;
            continue;
        }
        uint16_t fl = 0;
        for (int i = 1; i < 9; ++i) {
            const int sx = X - cx(i), sy = Y - cy(i);
            bool blocked;
            if (C.bc_x == kOpen && (sx < 0 || sx >= C.nx)) blocked = false;  // enters through the open boundary
            else blocked = !fluid_at(g, sx, sy);
            if (blocked) fl |= (uint16_t)(1u << (i - 1));
        }
        if (C.bc_x == kOpen && X == C.nx - 1) {
            // outflow: entering populations are those of the node one column upstream
            const bool base_fluid = fluid_at(g, X - 1, Y);
            if (!base_fluid) fl |= kOutletOwnBit;
            for (int i = 1; i < 9; ++i) {
                if (cx(i) >= 0) continue;
                const bool blocked = !base_fluid || !fluid_at(g, X, Y - cy(i));
                fl = blocked ? (uint16_t)(fl | (1u << (i - 1))) : (uint16_t)(fl & ~(1u << (i - 1)));
            }
        }
        bool near = false;
        for (int dy = -3; dy <= 3 && !near; ++dy)
            for (int dx = -3; dx <= 3 && !near; ++dx) near = !fluid_at(g, X + dx, Y + dy);
        if (near) fl |= kNearSolidBit;
        bool touches = false;
        for (int n = 0; n < 24 && !touches; ++n) touches = !fluid_at(g, X + s24x(n), Y + s24y(n));
        if (touches) {
            fl |= kWallBit;
            atomicAdd(row_counts + Y, 1);
        }
        flags_all[o] = fl;
    }
}

// Exclusive scan of n counts by one block; offsets[n] receives the total.
__global__ void k_scan(const int32_t* __restrict__ counts, int32_t* __restrict__ offsets, int n) {
    __shared__ int32_t warp_sums[32];
    __shared__ int32_t carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + tid;
        const int v = i < n ? counts[i] : 0;
        int incl = v;
        for (int off = 1; off < 32; off <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += t;
        }
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const int nw = blockDim.x >> 5;
            int ws = lane < nw ? warp_sums[lane] : 0;
            for (int off = 1; off < 32; off <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, ws, off);
                if (lane >= off) ws += t;
            }
            if (lane < nw) warp_sums[lane] = ws;  // inclusive warp prefix
        }
        __syncthreads();
        const int before = carry + (warp > 0 ? warp_sums[warp - 1] : 0);
        if (i < n) offsets[i] = before + incl - v;
        __syncthreads();
        if (tid == blockDim.x - 1) carry = before + incl;
        __syncthreads();
    }
    if (tid == 0) offsets[n] = carry;
}

// One block per row: wall nodes of the row in increasing x get consecutive entries.
__global__ void k_wall_fill(const DevCase* __restrict__ cases, int c, const uint8_t* __restrict__ solid_all,
                            const uint16_t* __restrict__ flags_all, uint32_t* __restrict__ wsub_all,
                            const int32_t* __restrict__ row_off, int32_t* __restrict__ wl_node,
                            uint32_t* __restrict__ wl_subst, uint32_t* __restrict__ wl_seff,
                            double* __restrict__ wl_a, long long nwall_total, int psi_only, int d2q9) {
    const DevCase C = cases[c];
    const Geo g{C.nx, C.ny, C.bc_x, C.bc_y, solid_all + C.d_off};
    const int Y = blockIdx.x;
    __shared__ int32_t warp_cnt[32];
    __shared__ int32_t running;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    if (tid == 0) running = 0;
    __syncthreads();
    for (int base = 0; base < C.nx; base += blockDim.x) {
        const int X = base + tid;
        bool is_wall = false;
        if (X < C.nx) is_wall = (flags_all[C.d_off + (long long)Y * C.nx + X] & kWallBit) != 0;
        const unsigned bal = __ballot_sync(0xffffffffu, is_wall);
        if (lane == 0) warp_cnt[warp] = __popc(bal);
        __syncthreads();
        int before = running;
        for (int w = 0; w < warp; ++w) before += warp_cnt[w];
        before += __popc(bal & ((1u << lane) - 1u));
        if (is_wall) {
            const long long e = C.w_off + row_off[Y] + before;
            uint32_t sm = 0, em = 0;
            for (int n = 0; n < 24; ++n) {
                const int ex = s24x(n), ey = s24y(n);
                bool s;
                if (ex >= -1 && ex <= 1 && ey >= -1 && ey <= 1) {
                    s = first_layer_solid(g, X, Y, ex, ey);
                } else if (fluid_at(g, X + ex, Y + ey)) {
                    s = false;
                } else {
                    sm |= 1u << n;
                    // psi only: the site keeps its own solid switch (clamped along an open axis)
                    s = psi_only ? first_layer_solid(g, X, Y, ex, ey)
                                 : first_layer_solid(g, X, Y, (ex > 0) - (ex < 0), (ey > 0) - (ey < 0));
                }
                if (s && (!d2q9 || n < 8)) em |= 1u << n;
            }
            double ax = 0.0, ay = 0.0;
            if (d2q9) {
                for (int h = 0; h < 4; ++h) {  // i = 1, 2, 5, 6 and opp(i); bit i-1 is first-layer node i
                    const int i = h < 2 ? 1 + h : 3 + h;
                    const double ds = (double)((em >> (i - 1)) & 1u) - (double)((em >> (opp(i) - 1)) & 1u);
                    ax += wq(i) * ds * cx(i);
                    ay += wq(i) * ds * cy(i);
                }
            } else {
                for (int p = 0; p < 12; ++p) {  // pairs (n, n+2): e_(n+2) = -e_n within each group of four
                    const int n = (p / 2) * 4 + (p % 2), m = n + 2;
                    const int ex = s24x(n), ey = s24y(n);
                    const double w = w8(ex * ex + ey * ey);
                    const double ds = (double)((em >> n) & 1u) - (double)((em >> m) & 1u);
                    ax += w * ds * ex;
                    ay += w * ds * ey;
                }
            }
            wl_node[e] = Y * C.nx + X;
            wl_subst[e] = sm;
            wl_seff[e] = em;
            wl_a[e] = ax;
            wl_a[nwall_total + e] = ay;
            wsub_all[C.d_off + (long long)Y * C.nx + X] = sm;
        }
        __syncthreads();
        if (tid == 0) {
            int tot = 0;
            for (int w = 0; w < nw; ++w) tot += warp_cnt[w];
            running += tot;
        }
        __syncthreads();
    }
}

// Flags with 8 ghost columns on each side, as the step kernel's tensor loads read them: column x
// at element x + 8; beyond the array a periodic axis wraps, a wall is solid and an open boundary
// repeats its boundary column.
__global__ void k_flags_ghost(const DevCase* __restrict__ cases, int c, const uint16_t* __restrict__ flags_all,
                              uint16_t* __restrict__ out, int pitch) {
    const DevCase C = cases[c];
    const long long n = (long long)C.ny * pitch;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const int Y = (int)(s / pitch), m = (int)(s % pitch), x = m - 8;
        uint16_t v;
        if (m >= C.nx + 16) v = 0;  // row padding
        else if (x >= 0 && x < C.nx) v = flags_all[C.d_off + (long long)Y * C.nx + x];
        else if (C.bc_x == kPeriodic) v = flags_all[C.d_off + (long long)Y * C.nx + ((x % C.nx) + C.nx) % C.nx];
        else if (C.bc_x == kOpen) v = flags_all[C.d_off + (long long)Y * C.nx + (x < 0 ? 0 : C.nx - 1)];
        else v = kSolidBit;
        out[s] = v;
    }
}

// Per-node copy of the adhesion vectors of one case's wall-list entries, in the compute type.
template <class R>
__global__ void k_wall_scatter(const DevCase* __restrict__ cases, int c, const int32_t* __restrict__ wl_node,
                               const double* __restrict__ wl_a, long long nwall_total, long long dense_total,
                               R* __restrict__ wa) {
    const DevCase C = cases[c];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < C.nwall; i += (long long)gridDim.x * blockDim.x) {
        const long long e = C.w_off + i;
        const long long o = C.d_off + wl_node[e];
        wa[o] = (R)wl_a[e];
        wa[dense_total + o] = (R)wl_a[nwall_total + e];
    }
}

// f = f^eq(rho_k, 0) in every case at once (cases along blockIdx.y): the stored populations that
// k_feq_rest followed by k_set_state write, computed straight from the densities (all cases back to
// back, case c at d_off) with the same double-precision products, so the state is the same bit for
// bit.  The stored f*_i at x is what the next pull takes: w_i rho(x + e_i) from a fluid neighbour,
// w_i rho(x) across a blocked link or beyond an open edge (the outlet column's own value where the
// copy rule keeps it); G ghost columns repeat the periodic edges.
template <class S>
__global__ void k_set_rest_all(const DevCase* __restrict__ cases, int G, const uint8_t* __restrict__ solid_all,
                               const uint16_t* __restrict__ flags_all, const double* __restrict__ rhoA_all,
                               const double* __restrict__ rhoB_all, Pair<S>* __restrict__ out_all) {
    using R = typename ComputeOf<S>::type;
    const DevCase C = cases[blockIdx.y];
    const long long N = (long long)C.nx * C.ny;
    const long long plane = C.pitch;
    Pair<S>* out = out_all + C.f_off;
    const double* rk[2] = {rhoA_all + C.d_off, rhoB_all + C.d_off};
    const uint8_t* sol = solid_all + C.d_off;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N; s += (long long)gridDim.x * blockDim.x) {
        const int X = (int)(s % C.nx), Y = (int)(s / C.nx);
        const uint16_t fl = flags_all[C.d_off + s];
        const long long o = (long long)Y * 9 * C.pitch + X + G;
        R ov[2][9];
        for (int k = 0; k < 2; ++k) {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                double v = 0.0;
                if (!(fl & kSolidBit)) {
                    int tx = X + cx(i), ty = Y + cy(i);
                    long long src = s;
                    int q = i;
                    if (C.bc_x == kOpen && (tx < 0 || tx >= C.nx)) {
                        q = (X == C.nx - 1 && (fl & kOutletOwnBit) && cx(i) > 0) ? opp(i) : i;
                    } else if (i != 0 && ((fl >> (opp(i) - 1)) & 1u)) {
                        q = opp(i);
                    } else {
                        tx += (tx < 0) ? C.nx : 0;
                        tx -= (tx >= C.nx) ? C.nx : 0;
                        ty += (ty < 0) ? C.ny : 0;
                        ty -= (ty >= C.ny) ? C.ny : 0;
                        src = (long long)ty * C.nx + tx;
                    }
                    v = wq(q) * (sol[src] ? 0.0 : rk[k][src]);  // the value k_feq_rest holds at src
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

}  // namespace

cudaError_t launch_flags(Ctx& c, int ci, int32_t* row_counts) {
    const long long N = (long long)c.hcases[ci].nx * c.hcases[ci].ny;
    const int g = (int)((N + 255) / 256 < 8192 ? (N + 255) / 256 : 8192);
    k_flags<<<g, 256, 0, c.stream>>>(c.dcases, ci, c.solid, c.flags, row_counts);
    return cudaGetLastError();
}

cudaError_t launch_scan_rows(const int32_t* counts, int32_t* offsets, int n, cudaStream_t s) {
    k_scan<<<1, 1024, 0, s>>>(counts, offsets, n);
    return cudaGetLastError();
}

cudaError_t launch_wall_fill(Ctx& c, int ci, const int32_t* row_offsets) {
    k_wall_fill<<<c.hcases[ci].ny, 256, 0, c.stream>>>(c.dcases, ci, c.solid, c.flags, c.wsub, row_offsets,
                                                        c.wl_node, c.wl_subst, c.wl_seff, c.wl_a, c.nwall,
                                                        c.cases[ci].params.second_layer == LBM_SECOND_LAYER_PSI,
                                                        c.cases[ci].params.adhesion_stencil == LBM_ADHESION_D2Q9);
    return cudaGetLastError();
}

cudaError_t launch_flags_ghost(Ctx& c, int ci) {
    const long long n = (long long)c.hcases[ci].ny * c.gf_pitch[ci];
    const int g = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    k_flags_ghost<<<g, 256, 0, c.stream>>>(c.dcases, ci, c.flags, c.gflags + c.gf_off[ci], c.gf_pitch[ci]);
    return cudaGetLastError();
}

cudaError_t launch_wall_cast(Ctx& c, int ci) {
    const long long n = c.hcases[ci].nwall;
    if (n == 0) return cudaSuccess;
    const int g = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    if (c.storage == LBM_STORE_F64)
        k_wall_scatter<double><<<g, 256, 0, c.stream>>>(c.dcases, ci, c.wl_node, c.wl_a, c.nwall, c.dense_elems, (double*)c.wa);
    else
        k_wall_scatter<float><<<g, 256, 0, c.stream>>>(c.dcases, ci, c.wl_node, c.wl_a, c.nwall, c.dense_elems, (float*)c.wa);
    return cudaGetLastError();
}

cudaError_t launch_set_rest_all(Ctx& c, const double* rhoA_all, const double* rhoB_all) {
    long long nmax = 0;
    for (const auto& h : c.hcases) nmax = nmax > (long long)h.nx * h.ny ? nmax : (long long)h.nx * h.ny;
    const int nc = (int)c.hcases.size(), G = ghost_cols(c.storage);
    for (int c0 = 0; c0 < nc; c0 += 65535) {  // cases along gridDim.y, at most 65535 per launch
        const int n = nc - c0 < 65535 ? nc - c0 : 65535;
        // about 4,096 blocks in all, at least one per case
        long long bx = ((nmax + 255) / 256 < 4096 ? (nmax + 255) / 256 : 4096);
        bx = bx * 8 / n > 0 ? (bx * 8 / n < bx ? bx * 8 / n : bx) : 1;
        const dim3 g((unsigned)bx, (unsigned)n);
        const DevCase* dc = c.dcases + c0;
        switch (c.storage) {
            case LBM_STORE_F64: k_set_rest_all<double><<<g, 256, 0, c.stream>>>(dc, G, c.solid, c.flags, rhoA_all, rhoB_all, (Pair<double>*)c.f[c.cur]); break;
            case LBM_STORE_F32: k_set_rest_all<float><<<g, 256, 0, c.stream>>>(dc, G, c.solid, c.flags, rhoA_all, rhoB_all, (Pair<float>*)c.f[c.cur]); break;
            case LBM_STORE_F16_SHIFTED: k_set_rest_all<__half><<<g, 256, 0, c.stream>>>(dc, G, c.solid, c.flags, rhoA_all, rhoB_all, (Pair<__half>*)c.f[c.cur]); break;
            default: k_set_rest_all<__nv_bfloat16><<<g, 256, 0, c.stream>>>(dc, G, c.solid, c.flags, rhoA_all, rhoB_all, (Pair<__nv_bfloat16>*)c.f[c.cur]); break;
        }
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace lbm
