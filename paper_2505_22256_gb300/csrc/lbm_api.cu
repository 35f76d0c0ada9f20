// C ABI of the library (include/lbm.h): validation, device layout, graph-captured stepping and the
// output calls.  All numerical work is done by the kernels in lbm_step.cu, lbm_geometry.cu and
// lbm_contact.cu.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <string>
#include <thread>
#include <vector>

#include <cudaTypedefs.h>

#include "lbm_internal.h"
#include "lbm_tma.cuh"

namespace lbm {
int contact_work_doubles();
}

using namespace lbm;

struct lbm_ctx {
    Ctx c;
};

namespace {

thread_local std::string g_err;
constexpr int kGraphSteps = 16;  // step launches per captured graph (even: ends on the same buffer)

lbm_status fail(lbm_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define CUDA_TRY(call)                                                                         \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) return fail(LBM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

template <class T>
cudaError_t dalloc(Ctx& c, T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    // Failure-injection hook for tests: with LBM_TEST_FAIL_ALLOC=k in the environment, the k-th
    // allocation of a context made here fails as if the device were out of memory.
    if (const char* k = getenv("LBM_TEST_FAIL_ALLOC")) {
        if (++c.alloc_count == atol(k)) return cudaErrorMemoryAllocation;
    }
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e == cudaSuccess) c.device_bytes += count * sizeof(T);
    return e;
}

bool finite(double v) { return isfinite(v) != 0; }

// FNV-1a over a solid mask read as fluid (0) / solid (1) per node.
uint64_t mask_hash(const uint8_t* solid, long long n) {
    uint64_t h = 1469598103934665603ULL;
    for (long long s = 0; s < n; ++s) h = (h ^ (uint64_t)(solid[s] != 0)) * 1099511628211ULL;
    return h;
}

lbm_status validate_case(const lbm_grid* g, const uint8_t* solid, const lbm_params* p, const double* rA,
                         const double* rB, int idx, int64_t* nfluid) {
    if (!g || !solid || !p || !rA || !rB) return fail(LBM_EINVAL, "case %d: NULL argument", idx);
    if (g->nx < 5 || g->ny < 5) return fail(LBM_EINVAL, "case %d: nx, ny must be >= 5 (got %d, %d)", idx, g->nx, g->ny);
    if ((long long)g->nx * g->ny > (1LL << 31) - 1) return fail(LBM_EINVAL, "case %d: lattice too large", idx);
    if (g->bc_x < 0 || g->bc_x > 2) return fail(LBM_EINVAL, "case %d: bad bc_x %d", idx, g->bc_x);
    if (g->bc_y < 0 || g->bc_y > 1) return fail(LBM_EINVAL, "case %d: bc_y must be periodic or wall", idx);
    for (int k = 0; k < 2; ++k) {
        if (!finite(p->tau[k]) || p->tau[k] <= 0.5) return fail(LBM_EINVAL, "case %d: tau[%d] must be > 0.5", idx, k);
        if (!finite(p->g[k]) || !finite(p->rho_in[k]) || !finite(p->rho0_store[k]))
            return fail(LBM_EINVAL, "case %d: non-finite parameter", idx);
    }
    if (!finite(p->G_AB) || !finite(p->G_w2) || !finite(p->u_in)) return fail(LBM_EINVAL, "case %d: non-finite parameter", idx);
    if (!finite(p->lambda) || p->lambda <= 0.0) return fail(LBM_EINVAL, "case %d: lambda must be > 0", idx);
    if (!finite(p->delta) || p->delta <= 0.0 || p->delta > 1.0) return fail(LBM_EINVAL, "case %d: delta must lie in (0, 1]", idx);
    if (p->mode != LBM_ADS_ORIGINAL && p->mode != LBM_ADS_IMPROVED) return fail(LBM_EINVAL, "case %d: bad mode", idx);
    if (p->second_layer != LBM_SECOND_LAYER_PSI_AND_SOLID && p->second_layer != LBM_SECOND_LAYER_PSI)
        return fail(LBM_EINVAL, "case %d: bad second_layer %d", idx, p->second_layer);
    if (p->adhesion_stencil != LBM_ADHESION_E8 && p->adhesion_stencil != LBM_ADHESION_D2Q9)
        return fail(LBM_EINVAL, "case %d: bad adhesion_stencil %d", idx, p->adhesion_stencil);
    if (p->outlet != LBM_OUTLET_COPY && p->outlet != LBM_OUTLET_PRESSURE)
        return fail(LBM_EINVAL, "case %d: bad outlet %d", idx, p->outlet);
    if (p->outlet == LBM_OUTLET_PRESSURE &&
        (g->bc_x != LBM_BC_OPEN || !finite(p->rho_out[0]) || !finite(p->rho_out[1]) || p->rho_out[0] <= 0.0 ||
         p->rho_out[1] <= 0.0))
        return fail(LBM_EINVAL, "case %d: the pressure outlet needs an open x and outlet densities > 0", idx);
    if (p->inlet_profile != LBM_INLET_UNIFORM && p->inlet_profile != LBM_INLET_POISEUILLE)
        return fail(LBM_EINVAL, "case %d: bad inlet profile", idx);
    if (p->inlet_profile == LBM_INLET_POISEUILLE && (g->bc_x != LBM_BC_OPEN || g->bc_y != LBM_BC_WALL))
        return fail(LBM_EINVAL, "case %d: the Poiseuille inlet needs an open x and walled y", idx);
    if (!finite(p->u_wall[0]) || !finite(p->u_wall[1])) return fail(LBM_EINVAL, "case %d: non-finite wall velocity", idx);
    if ((p->u_wall[0] != 0.0 || p->u_wall[1] != 0.0) && (g->bc_y != LBM_BC_WALL || g->bc_x == LBM_BC_OPEN))
        return fail(LBM_EINVAL, "case %d: sliding walls need a walled y and a closed x", idx);
    if (g->bc_x == LBM_BC_OPEN && (p->rho_in[0] <= 0.0 || p->rho_in[1] <= 0.0))
        return fail(LBM_EINVAL, "case %d: inlet densities must be > 0", idx);
    const long long N = (long long)g->nx * g->ny;
    int64_t nf = 0;
    for (long long s = 0; s < N; ++s) {
        if (solid[s]) continue;
        ++nf;
        if (!finite(rA[s]) || !finite(rB[s]) || rA[s] <= 0.0 || rB[s] <= 0.0)
            return fail(LBM_EINVAL, "case %d: initial densities must be finite and > 0 at fluid node %lld", idx, s);
    }
    if (nf == 0) return fail(LBM_EINVAL, "case %d: the mask has no fluid node", idx);
    *nfluid = nf;
    return LBM_OK;
}

DevCase make_desc(const lbm_grid& g, const lbm_params& p) {
    DevCase d;
    memset(&d, 0, sizeof d);
    d.nx = g.nx;
    d.ny = g.ny;
    d.bc_x = g.bc_x;
    d.bc_y = g.bc_y;
    d.mode = p.mode;
    for (int k = 0; k < 2; ++k) {
        d.omega[k] = 1.0 / p.tau[k];
        d.cF[k] = 1.0 - 0.5 / p.tau[k];
        d.g[k] = p.g[k];
        d.rho_in[k] = p.rho_in[k];
        d.rho0[k] = p.rho0_store[k];
    }
    d.G = p.G_AB;
    d.Gw2 = p.G_w2;
    d.lam = p.lambda;
    d.delta = p.delta;
    const double l = p.lambda, dl = p.delta;
    d.s1 = 2.0 * l / (1.0 + l);                          // s'_1 = t'_1
    d.s2 = 2.0 * (l * l - l) / (dl * (1.0 + l));          // s'_2
    d.s3 = (l - l * l) / (dl * dl * (1.0 + l));           // s'_3
    d.t2 = 2.0 * (l - 1.0) / (dl * (1.0 + l));            // t'_2
    d.t3 = (l - 1.0) / (dl * dl * (1.0 + l));             // t'_3
    d.u_in = p.u_in;
    d.u_wall[0] = p.u_wall[0];
    d.u_wall[1] = p.u_wall[1];
    d.inlet_profile = p.inlet_profile;
    d.outlet = p.outlet;
    d.rho_out[0] = p.rho_out[0];
    d.rho_out[1] = p.rho_out[1];
    return d;
}

size_t elem_size(int storage) {
    switch (storage) {
        case LBM_STORE_F64: return 8;
        case LBM_STORE_F32: return 4;
        default: return 2;
    }
}

void drop_graphs(Ctx& c) {
    if (c.graph) cudaGraphExecDestroy(c.graph);
    c.graph = nullptr;
    c.graph_steps = 0;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// Three tensor maps per case: one row of all 9 planes of (A, B) pairs of each population buffer, T
// columns from column x - G (the ghost columns included), and one row of the ghost-padded flags, as
// the step kernel loads them.  A pair is one tensor element (8-byte words for FP32, 4-byte for the
// 16-bit types); an FP64 pair is two 8-byte words along an extra innermost dimension.
lbm_status build_tmaps(Ctx& c) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return fail(LBM_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const int T = c.block_threads, G = ghost_cols(c.storage), XB = box_extra_cols(c.storage);
    if (T + XB > 256) return fail(LBM_EINVAL, "block of %d threads needs a tensor box wider than 256 columns", T);
    const bool f64 = c.storage == LBM_STORE_F64;
    const CUtensorMapDataType dt = c.elem == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT32 : CU_TENSOR_MAP_DATA_TYPE_UINT64;
    const cuuint64_t pb = 2 * c.elem;  // bytes of one pair
    std::vector<CUtensorMap> maps(3 * c.hcases.size());
    for (size_t ci = 0; ci < c.hcases.size(); ++ci) {
        const DevCase& d = c.hcases[ci];
        for (int buf = 0; buf < 2; ++buf) {
            void* base = (char*)c.f[buf] + (size_t)d.f_off * pb;
            const cuuint64_t plane = (cuuint64_t)d.pitch * pb, row = 9 * plane;  // [ny][9][pitch] pairs
            CUresult r;
            if (f64) {
                cuuint64_t dims[4] = {2, (cuuint64_t)(d.nx + 2 * G), 9, (cuuint64_t)d.ny};
                cuuint64_t strides[3] = {pb, plane, row};
                cuuint32_t box[4] = {2, (cuuint32_t)(T + XB), 9, 1};
                cuuint32_t estr[4] = {1, 1, 1, 1};
                r = enc(&maps[3 * ci + buf], dt, 4, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            } else {
                cuuint64_t dims[3] = {(cuuint64_t)(d.nx + 2 * G), 9, (cuuint64_t)d.ny};
                cuuint64_t strides[2] = {plane, row};
                cuuint32_t box[3] = {(cuuint32_t)(T + XB), 9, 1};
                cuuint32_t estr[3] = {1, 1, 1};
                r = enc(&maps[3 * ci + buf], dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            }
            if (r != CUDA_SUCCESS) return fail(LBM_ECUDA, "tensor map of case %zu rejected (CUresult %d)", ci, (int)r);
        }
        // flag rows: T + 8 columns from column x - 8 (8 ghost columns per side)
        cuuint64_t fdims[2] = {(cuuint64_t)(d.nx + 16), (cuuint64_t)d.ny};
        cuuint64_t fstr[1] = {(cuuint64_t)c.gf_pitch[ci] * sizeof(uint16_t)};
        cuuint32_t fbox[2] = {(cuuint32_t)(T + 8), 1};
        cuuint32_t festr[2] = {1, 1};
        CUresult r = enc(&maps[3 * ci + 2], CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, c.gflags + c.gf_off[ci], fdims, fstr, fbox,
                         festr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(LBM_ECUDA, "flag tensor map of case %zu rejected (CUresult %d)", ci, (int)r);
    }
    if (!c.tmaps) CUDA_TRY(cudaMalloc(&c.tmaps, maps.size() * sizeof(CUtensorMap)));
    CUDA_TRY(cudaMemcpy(c.tmaps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice));
    return LBM_OK;
}

#ifndef LBM_TAIL_ROWS
#define LBM_TAIL_ROWS 16  // height of the short items that end a launch
#endif

// Row chunks [y0, y1) of one case's column strips, chunk-major; odd chunks march upwards (sign bit
// of the case field), so the halo rows two neighbouring chunks share are read at about the same
// time, while they are still in L2.
void push_chunks(std::vector<int4>& out, int ci, int nstrip, int Wi, int y_begin, int y_end, int h) {
    const int n = (y_end - y_begin + h - 1) / h;
    for (int k = 0; k < n; ++k) {
        // balanced heights: the first (rows % n) chunks take one row more
        const int rows = y_end - y_begin, base = rows / n, extra = rows % n;
        const int y0 = y_begin + k * base + std::min(k, extra), y1 = y0 + base + (k < extra ? 1 : 0);
        for (int s = 0; s < nstrip; ++s)
            out.push_back(make_int4((int)((unsigned)ci | ((k & 1) ? 0x80000000u : 0u)), s * Wi, y0, y1));
    }
}

// Work lists.  A work item is a column window of block_threads - 8 interior columns by a chunk of
// rows of one case; blocks of the step kernel claim items in list order from a counter.
//  * Step list.  With block_rows > 0, uniform chunks of that height.  With block_rows = 0 (the
//    default; block_rows < 0 for a tail of -block_rows rows), a guided list: long chunks of height
//    Hb first, then short chunks of LBM_TAIL_ROWS
//    rows, enough of them to absorb the ragged end of the long ones, so that a launch lasts about
//    (rows marched, 5 halo rows per item included) / (resident blocks) + one short item.  Hb
//    minimises that estimate.
//  * Per-case list (after the step list): uniform chunks, contiguous per case, used by the fields
//    pass, whose per-item partial sums are reduced per case in item order.
lbm_status build_items(Ctx& c) {
    const int W = c.block_threads, Wi = W - 8;
    lbm_status ts = build_tmaps(c);
    if (ts != LBM_OK) return ts;
    int per_sm = 0;
    CUDA_TRY(step_occupancy(c.storage, W, &per_sm));
    if (per_sm < 1) return fail(LBM_ECUDA, "step kernel cannot be resident with %d threads", W);
    const long long resident = (long long)per_sm * c.num_sms;
    const int ncases = (int)c.hcases.size();
    std::vector<int> nstrip(ncases);
    long long strips = 0;
    for (int i = 0; i < ncases; ++i) {
        nstrip[i] = (c.hcases[i].nx + Wi - 1) / Wi;
        strips += nstrip[i];
    }
    std::vector<int4> items;
    if (c.block_rows > 0) {
        const int H = c.block_rows;
        for (int i = 0; i < ncases; ++i) push_chunks(items, i, nstrip[i], Wi, 0, c.hcases[i].ny, H);
        c.rows_used = H;
    } else {
        const int Hs = c.block_rows < 0 ? -c.block_rows : LBM_TAIL_ROWS;
        // rows of short chunks per strip of case i for a given long height hb
        auto tail_chunks = [&](int i, int hb) -> int {
            const long long need = (resident * (hb + 5) + strips * (Hs + 5) - 1) / (strips * (Hs + 5));
            return (int)std::min<long long>(need, c.hcases[i].ny / Hs);
        };
        double best = -1.0;
        int Hb = 32;
        for (int hb = 16; hb <= 256; ++hb) {
            double work = 0.0, tail = 0.0;
            for (int i = 0; i < ncases; ++i) {
                const int ns = tail_chunks(i, hb), bulk = c.hcases[i].ny - ns * Hs;
                const int nb = (bulk + hb - 1) / hb;
                work += (double)nstrip[i] * (bulk + 5.0 * nb + ns * (Hs + 5.0));
                tail += (double)nstrip[i] * ns * (Hs + 5.0);
            }
            const double cost = work / resident + (Hs + 5) + std::max(0.0, (hb + 5) - tail / resident);
            if (best < 0 || cost < best) {
                best = cost;
                Hb = hb;
            }
        }
        std::vector<int> ns(ncases);
        for (int i = 0; i < ncases; ++i) {
            ns[i] = tail_chunks(i, Hb);
            push_chunks(items, i, nstrip[i], Wi, 0, c.hcases[i].ny - ns[i] * Hs, Hb);
        }
        for (int i = 0; i < ncases; ++i)
            if (ns[i] > 0) push_chunks(items, i, nstrip[i], Wi, c.hcases[i].ny - ns[i] * Hs, c.hcases[i].ny, Hs);
        c.rows_used = Hb;
    }
    c.nitems = (int)items.size();
    for (int i = 0; i < ncases; ++i) {
        DevCase& d = c.hcases[i];
        // per-case chunk height: minimise (items + resident) x (h + 5) for this case alone
        long long bestc = -1;
        int Hf = 16;
        for (int h = 16; h <= 128; ++h) {
            const long long cost = ((long long)nstrip[i] * ((d.ny + h - 1) / h) + resident) * (h + 5);
            if (bestc < 0 || cost < bestc) {
                bestc = cost;
                Hf = h;
            }
        }
        d.item_begin = (int)items.size();
        push_chunks(items, i, nstrip[i], Wi, 0, d.ny, Hf);
        d.item_end = (int)items.size();
    }
    c.nitems_all = (int)items.size();
    if (c.items) {
        cudaFree(c.items);
        c.items = nullptr;
    }
    if (c.diag_part) {
        cudaFree(c.diag_part);
        c.diag_part = nullptr;
    }
    CUDA_TRY(cudaMalloc(&c.items, items.size() * sizeof(int4)));
    CUDA_TRY(cudaMemcpy(c.items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMalloc(&c.diag_part, items.size() * kDiagN * sizeof(double)));
    CUDA_TRY(cudaMemcpy(c.dcases, c.hcases.data(), c.hcases.size() * sizeof(DevCase), cudaMemcpyHostToDevice));
    c.grid_blocks = (int)std::min<long long>(c.nitems, resident);
    drop_graphs(c);
    return LBM_OK;
}

// After a synchronisation: report a pipeline wait inside a kernel that gave up.
lbm_status check_device_error(Ctx& c) {
    int e = 0;
    CUDA_TRY(cudaMemcpyAsync(&e, c.err, sizeof e, cudaMemcpyDeviceToHost, c.stream));
    CUDA_TRY(cudaStreamSynchronize(c.stream));
    if (e)
        return fail(LBM_ECUDA, "a bounded wait inside a kernel gave up (device error word %d: bit 1 a step kernel's "
                               "tensor-load wait, bit 2 the wait self-test)", e);
    return LBM_OK;
}

lbm_status check_case(lbm_ctx* ctx, int ci) {
    if (!ctx) return fail(LBM_EINVAL, "NULL context");
    if (ci < 0 || ci >= (int)ctx->c.cases.size()) return fail(LBM_EINVAL, "case index %d out of range", ci);
    return LBM_OK;
}

void free_ctx(Ctx& c) {
    drop_graphs(c);
    for (cudaStream_t st : {c.xs_in, c.xs_out})
        if (st) {
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
        }
    for (int k = 0; k < 2; ++k) {
        for (cudaEvent_t ev : {c.xin_ready[k], c.xin_free[k], c.xout_ready[k], c.xout_free[k]})
            if (ev) cudaEventDestroy(ev);
        if (c.xin[k]) cudaFree(c.xin[k]);
        if (c.xout[k]) cudaFree(c.xout[k]);
    }
    void* ptrs[] = {c.dcases, c.f[0], c.f[1], c.flags, c.wsub, c.wa, c.solid, c.wl_node, c.wl_subst, c.wl_seff,
                    c.wl_a, c.items, c.dense, c.fields, c.diag_part, c.diag_out, c.ca_work, c.ca_all, c.ca_batch, c.ca_points, c.fields_all, c.slide_list, c.tmaps, c.err, c.sched, c.gflags};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c.own_stream && c.stream) cudaStreamDestroy(c.stream);
}

lbm_status create_impl(int ncases, const lbm_case* cs, int storage, void* stream, lbm_ctx** out) {
    if (!out) return fail(LBM_EINVAL, "NULL output pointer");
    *out = nullptr;
    if (ncases < 1 || !cs) return fail(LBM_EINVAL, "need at least one case");
    if (storage < LBM_STORE_F64 || storage > LBM_STORE_BF16_SHIFTED) return fail(LBM_EINVAL, "bad storage %d", storage);
    std::vector<int64_t> nfluid(ncases);
    for (int i = 0; i < ncases; ++i) {
        lbm_status s = validate_case(&cs[i].grid, cs[i].solid, &cs[i].params, cs[i].rho_A0, cs[i].rho_B0, i, &nfluid[i]);
        if (s != LBM_OK) return s;
    }
    int dev = 0, ndev = 0;
    CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (ndev < 1) return fail(LBM_ECUDA, "no CUDA device");
    CUDA_TRY(cudaGetDevice(&dev));
    cudaDeviceProp prop;
    CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
    if (!(prop.major == 10 && prop.minor == 3))
        return fail(LBM_ECUDA, "this library is built for sm_103a (GB300); device %d is sm_%d%d", dev, prop.major, prop.minor);

    lbm_ctx* h = new (std::nothrow) lbm_ctx();
    if (!h) return fail(LBM_ENOMEM, "host allocation");
    Ctx& c = h->c;
    c.storage = storage;
    c.elem = elem_size(storage);
    c.device = dev;
    c.num_sms = prop.multiProcessorCount;
    auto bail = [&](lbm_status s) {
        free_ctx(c);
        delete h;
        return s;
    };
    if (stream) {
        c.stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(fail(LBM_ECUDA, "cudaStreamCreate failed"));
        c.own_stream = true;
    }

    long long max_nodes = 0;
    for (int i = 0; i < ncases; ++i) {
        HostCase hc;
        hc.grid = cs[i].grid;
        hc.params = cs[i].params;
        hc.nfluid = nfluid[i];
        hc.mask_hash = mask_hash(cs[i].solid, (long long)cs[i].grid.nx * cs[i].grid.ny);
        c.cases.push_back(hc);
        DevCase d = make_desc(cs[i].grid, cs[i].params);
        const int per_line = (int)(128 / (2 * c.elem));  // rows of pairs start on 128-byte boundaries
        d.pitch = (d.nx + 2 * ghost_cols(storage) + per_line - 1) / per_line * per_line;
        d.f_off = c.pop_elems / 2;
        d.d_off = c.dense_elems;
        fill_case_params(d);
        c.pop_elems += 18LL * d.ny * d.pitch;
        c.dense_elems += (long long)d.nx * d.ny;
        max_nodes = std::max(max_nodes, (long long)d.nx * d.ny);
        c.hcases.push_back(d);
    }
    auto cu = [&](cudaError_t e, const char* what) -> lbm_status {
        if (e == cudaErrorMemoryAllocation) return fail(LBM_ENOMEM, "%s: out of device memory", what);
        if (e != cudaSuccess) return fail(LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
        return LBM_OK;
    };
#define STEP(expr, what)                        \
    do {                                        \
        lbm_status s_ = cu((expr), what);       \
        if (s_ != LBM_OK) return bail(s_);      \
    } while (0)

    STEP(dalloc(c, (unsigned char**)&c.f[0], c.pop_elems * c.elem), "population buffer");
    STEP(dalloc(c, (unsigned char**)&c.f[1], c.pop_elems * c.elem), "population buffer");
    STEP(cudaMemsetAsync(c.f[0], 0, c.pop_elems * c.elem, c.stream), "memset");
    STEP(cudaMemsetAsync(c.f[1], 0, c.pop_elems * c.elem, c.stream), "memset");
    const size_t rsize = storage == LBM_STORE_F64 ? 8 : 4;
    STEP(dalloc(c, &c.flags, c.dense_elems), "flags");
    STEP(dalloc(c, &c.wsub, c.dense_elems), "wall masks");
    STEP(dalloc(c, (unsigned char**)&c.wa, 2 * c.dense_elems * rsize), "wall vectors");
    STEP(dalloc(c, &c.err, 1), "error word");
    STEP(dalloc(c, &c.sched, 2), "work counters");
    STEP(cudaMemsetAsync(c.flags, 0, c.dense_elems * sizeof(uint16_t), c.stream), "memset");
    STEP(cudaMemsetAsync(c.wsub, 0, c.dense_elems * sizeof(uint32_t), c.stream), "memset");
    STEP(cudaMemsetAsync(c.wa, 0, 2 * c.dense_elems * rsize, c.stream), "memset");
    STEP(cudaMemsetAsync(c.err, 0, sizeof(int), c.stream), "memset");
    STEP(cudaMemsetAsync(c.sched, 0, 2 * sizeof(int), c.stream), "memset");
    STEP(dalloc(c, &c.solid, c.dense_elems), "masks");
    STEP(dalloc(c, &c.dcases, ncases), "descriptors");
    STEP(dalloc(c, &c.dense, 18 * max_nodes), "transfer scratch");
    c.dense_cap = 18 * max_nodes;
    STEP(dalloc(c, &c.fields, 4 * max_nodes), "field scratch");
    STEP(dalloc(c, &c.diag_out, (size_t)ncases * kDiagN), "diagnostics");
    STEP(dalloc(c, &c.ca_work, (size_t)contact_work_doubles()), "contact-angle scratch");
    STEP(dalloc(c, &c.ca_all, (size_t)16 * ncases), "contact-angle records");
    for (int i = 0; i < ncases; ++i) {
        std::vector<uint8_t> m((size_t)c.hcases[i].nx * c.hcases[i].ny);
        for (size_t s = 0; s < m.size(); ++s) m[s] = cs[i].solid[s] ? 1 : 0;
        STEP(cudaMemcpy(c.solid + c.hcases[i].d_off, m.data(), m.size(), cudaMemcpyHostToDevice), "mask upload");
    }
    STEP(cudaMemcpy(c.dcases, c.hcases.data(), ncases * sizeof(DevCase), cudaMemcpyHostToDevice), "descriptors");

    // flags and per-row wall counts, then the wall list
    std::vector<int32_t*> offs(ncases, nullptr);
    int32_t* counts = nullptr;
    int max_ny = 0;
    for (auto& d : c.hcases) max_ny = std::max(max_ny, d.ny);
    STEP(cudaMalloc(&counts, (size_t)max_ny * sizeof(int32_t)), "row counts");
    lbm_status st = LBM_OK;
    for (int i = 0; i < ncases && st == LBM_OK; ++i) {
        const int ny = c.hcases[i].ny;
        st = cu(cudaMalloc(&offs[i], (size_t)(ny + 1) * sizeof(int32_t)), "row offsets");
        if (st == LBM_OK) st = cu(cudaMemsetAsync(counts, 0, (size_t)ny * sizeof(int32_t), c.stream), "memset");
        if (st == LBM_OK) st = cu(launch_flags(c, i, counts), "flags kernel");
        if (st == LBM_OK) st = cu(launch_scan_rows(counts, offs[i], ny, c.stream), "scan kernel");
        int32_t tot = 0;
        if (st == LBM_OK) st = cu(cudaMemcpyAsync(&tot, offs[i] + ny, sizeof tot, cudaMemcpyDeviceToHost, c.stream), "count");
        if (st == LBM_OK) st = cu(cudaStreamSynchronize(c.stream), "flags");
        c.hcases[i].w_off = c.nwall;
        c.hcases[i].nwall = tot;
        c.nwall += tot;
    }
    cudaFree(counts);
    long long gf_total = 0;
    for (int i = 0; i < ncases; ++i) {
        c.gf_off.push_back(gf_total);
        c.gf_pitch.push_back((c.hcases[i].nx + 16 + 63) / 64 * 64);
        gf_total += (long long)c.gf_pitch.back() * c.hcases[i].ny;
    }
    if (st == LBM_OK) st = cu(dalloc(c, &c.gflags, gf_total), "padded flags");
    for (int i = 0; i < ncases && st == LBM_OK; ++i) st = cu(launch_flags_ghost(c, i), "padded flags kernel");
    if (st == LBM_OK) st = cu(cudaMemcpy(c.dcases, c.hcases.data(), ncases * sizeof(DevCase), cudaMemcpyHostToDevice), "descriptors");
    if (st == LBM_OK) st = cu(dalloc(c, &c.wl_node, c.nwall), "wall list");
    if (st == LBM_OK) st = cu(dalloc(c, &c.wl_subst, c.nwall), "wall list");
    if (st == LBM_OK) st = cu(dalloc(c, &c.wl_seff, c.nwall), "wall list");
    if (st == LBM_OK) st = cu(dalloc(c, &c.wl_a, 2 * c.nwall), "wall list");
    for (int i = 0; i < ncases && st == LBM_OK; ++i) st = cu(launch_wall_fill(c, i, offs[i]), "wall-list kernel");
    for (int i = 0; i < ncases && st == LBM_OK; ++i) st = cu(launch_wall_cast(c, i), "wall-list scatter");
    if (st == LBM_OK) st = cu(cudaStreamSynchronize(c.stream), "wall list");
    for (auto p : offs)
        if (p) cudaFree(p);
    if (st != LBM_OK) return bail(st);

    // cases whose walls slide get the sliding-wall fix-up after every step
    {
        std::vector<int> sl;
        for (int i = 0; i < ncases; ++i)
            if (c.hcases[i].pf.moving) {
                sl.push_back(i);
                c.slide_max_nx = std::max(c.slide_max_nx, c.hcases[i].nx);
            }
        c.slide_n = (int)sl.size();
        if (c.slide_n) {
            STEP(dalloc(c, &c.slide_list, sl.size()), "sliding-wall list");
            STEP(cudaMemcpy(c.slide_list, sl.data(), sl.size() * sizeof(int), cudaMemcpyHostToDevice), "sliding-wall list");
        }
    }

    // work list and launch shape.  Block width: the one that launches fewer thread columns over all
    // cases (windows of width - 8 interior columns; 64 wins on lattices narrower than about 56
    // columns).  The wall-list correction is inlined where wall-list nodes are common (more than 4 %
    // of the fluid nodes), called out of line otherwise.
    {
        long long cols[2] = {0, 0};
        const int widths[2] = {128, 64};
        for (int w = 0; w < 2; ++w)
            for (const DevCase& d : c.hcases)
                cols[w] += (long long)((d.nx + widths[w] - 9) / (widths[w] - 8)) * widths[w] * d.ny;
        c.block_threads = cols[1] < cols[0] ? 64 : 128;
    }
    c.block_rows = 0;
    {
        long long fl = 0;
        for (const HostCase& h : c.cases) fl += h.nfluid;
        c.wall_inline = (double)c.nwall > 0.04 * (double)fl ? 1 : 0;
    }
    st = build_items(c);
    if (st != LBM_OK) return bail(st);

    // initial state f = f^eq(rho_k, 0)
    for (int i = 0; i < ncases; ++i) {
        const long long N = (long long)c.hcases[i].nx * c.hcases[i].ny;
        STEP(cudaMemcpyAsync(c.fields, cs[i].rho_A0, N * sizeof(double), cudaMemcpyHostToDevice, c.stream), "density upload");
        STEP(cudaMemcpyAsync(c.fields + N, cs[i].rho_B0, N * sizeof(double), cudaMemcpyHostToDevice, c.stream), "density upload");
        STEP(launch_feq_rest(c, i, c.fields, c.fields + N, c.dense), "init kernel");
        STEP(launch_set_state(c, i, c.dense), "init kernel");
    }
    STEP(cudaStreamSynchronize(c.stream), "initialisation");
#undef STEP
    *out = h;
    return LBM_OK;
}

}  // namespace

namespace lbm {
// Error reporting for entry points defined in other translation units.
lbm_status report_error(lbm_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}
}  // namespace lbm

extern "C" {

lbm_status lbm_create(const lbm_grid* grid, const uint8_t* solid, const lbm_params* params, const double* rho_A0,
                      const double* rho_B0, int32_t storage, void* cuda_stream, lbm_ctx** out) {
    if (!grid || !params) return fail(LBM_EINVAL, "NULL argument");
    lbm_case cs;
    cs.grid = *grid;
    cs.solid = solid;
    cs.rho_A0 = rho_A0;
    cs.rho_B0 = rho_B0;
    cs.params = *params;
    return create_impl(1, &cs, storage, cuda_stream, out);
}

lbm_status lbm_ensemble_create(int32_t ncases, const lbm_case* cases, int32_t storage, void* cuda_stream,
                               lbm_ctx** out) {
    return create_impl(ncases, cases, storage, cuda_stream, out);
}

void lbm_destroy(lbm_ctx* ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->c.stream);
    free_ctx(ctx->c);
    delete ctx;
}

lbm_status lbm_step(lbm_ctx* ctx, int64_t n) {
    NvtxRange nvtx_("lbm_step");
    if (!ctx) return fail(LBM_EINVAL, "NULL context");
    if (n < 0) return fail(LBM_EINVAL, "negative step count");
    Ctx& c = ctx->c;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CUDA_TRY(cudaStreamIsCapturing(c.stream, &cap));
    const bool may_graph = cap == cudaStreamCaptureStatusNone;
    while (n > 0) {
        if (may_graph && n >= kGraphSteps && c.cur == 0) {
            if (!c.graph) {
                cudaGraph_t g = nullptr;
                CUDA_TRY(cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal));
                cudaError_t le = cudaSuccess;
                for (int k = 0; k < kGraphSteps && le == cudaSuccess; ++k) le = launch_step(c, k & 1, c.stream);
                cudaError_t ee = cudaStreamEndCapture(c.stream, &g);
                if (le != cudaSuccess) {
                    if (g) cudaGraphDestroy(g);
                    return fail(LBM_ECUDA, "step launch during capture: %s", cudaGetErrorString(le));
                }
                if (ee != cudaSuccess) return fail(LBM_ECUDA, "graph capture: %s", cudaGetErrorString(ee));
                cudaError_t ie = cudaGraphInstantiate(&c.graph, g, 0);
                cudaGraphDestroy(g);
                if (ie != cudaSuccess) return fail(LBM_ECUDA, "graph instantiate: %s", cudaGetErrorString(ie));
                c.graph_steps = kGraphSteps;
            }
            CUDA_TRY(cudaGraphLaunch(c.graph, c.stream));
            n -= kGraphSteps;
            c.steps += kGraphSteps;
            ++c.version;
        } else {
            CUDA_TRY(launch_step(c, c.cur, c.stream));
            c.cur ^= 1;
            --n;
            ++c.steps;
            ++c.version;
        }
    }
    return LBM_OK;
}

lbm_status lbm_synchronize(lbm_ctx* ctx, double timeout_s) {
    if (!ctx) return fail(LBM_EINVAL, "NULL context");
    Ctx& c = ctx->c;
    // the overlapped transfers' copy streams first: their last copies follow the work they wait for
    if (timeout_s <= 0) {
        for (cudaStream_t st : {c.xs_in, c.xs_out})
            if (st) CUDA_TRY(cudaStreamSynchronize(st));
        CUDA_TRY(cudaStreamSynchronize(c.stream));
        return check_device_error(c);
    }
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaSuccess;
        for (cudaStream_t st : {c.xs_in, c.xs_out, c.stream})
            if (st && e == cudaSuccess) e = cudaStreamQuery(st);
        if (e == cudaSuccess) return check_device_error(c);
        if (e != cudaErrorNotReady) return fail(LBM_ECUDA, "stream: %s", cudaGetErrorString(e));
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > timeout_s) return fail(LBM_ETIMEOUT, "stream still busy after %.3f s", el);
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
}

lbm_status lbm_set_densities(lbm_ctx* ctx, int32_t ci, const double* rho_A0, const double* rho_B0, int32_t on_device) {
    lbm_status s = check_case(ctx, ci);
    if (s != LBM_OK) return s;
    if (!rho_A0 || !rho_B0) return fail(LBM_EINVAL, "NULL density");
    Ctx& c = ctx->c;
    const long long N = (long long)c.hcases[ci].nx * c.hcases[ci].ny;
    const double *a = rho_A0, *b = rho_B0;
    if (!on_device) {
        CUDA_TRY(cudaMemcpyAsync(c.fields, rho_A0, N * sizeof(double), cudaMemcpyHostToDevice, c.stream));
        CUDA_TRY(cudaMemcpyAsync(c.fields + N, rho_B0, N * sizeof(double), cudaMemcpyHostToDevice, c.stream));
        a = c.fields;
        b = c.fields + N;
    }
    CUDA_TRY(launch_feq_rest(c, ci, a, b, c.dense));
    CUDA_TRY(launch_set_state(c, ci, c.dense));
    ++c.version;
    if (!on_device) CUDA_TRY(cudaStreamSynchronize(c.stream));
    return LBM_OK;
}

lbm_status lbm_fields(lbm_ctx* ctx, int32_t ci, double* rho_A, double* rho_B, double* ux, double* uy, int32_t on_device) {
    NvtxRange nvtx_("lbm_fields");
    lbm_status s = check_case(ctx, ci);
    if (s != LBM_OK) return s;
    Ctx& c = ctx->c;
    const long long N = (long long)c.hcases[ci].nx * c.hcases[ci].ny;
    if (on_device) {
        c.fields_case = -1;  // NULL outputs land in the scratch
        CUDA_TRY(launch_fields(c, ci, rho_A, rho_B, ux, uy, false));
        return LBM_OK;
    }
    CUDA_TRY(launch_fields(c, ci, nullptr, nullptr, nullptr, nullptr, false));
    c.fields_case = ci;
    c.fields_version = c.version;
    double* outs[4] = {rho_A, rho_B, ux, uy};
    for (int q = 0; q < 4; ++q)
        if (outs[q]) CUDA_TRY(cudaMemcpyAsync(outs[q], c.fields + q * N, N * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    CUDA_TRY(cudaStreamSynchronize(c.stream));
    return check_device_error(c);
}

// Scratch of four doubles per node of all cases for the batched host transfers.
static lbm_status fields_all_scratch(Ctx& c) {
    if (c.fields_all) return LBM_OK;
    const cudaError_t e = cudaMalloc(&c.fields_all, (size_t)4 * c.dense_elems * sizeof(double));
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        c.fields_all = nullptr;
        return fail(LBM_ENOMEM, "batched transfer scratch: out of device memory");
    }
    CUDA_TRY(e);
    return LBM_OK;
}

lbm_status lbm_set_densities_all(lbm_ctx* ctx, const double* rho_A0, const double* rho_B0, int32_t on_device) {
    NvtxRange nvtx_("lbm_set_densities_all");
    if (!ctx) return fail(LBM_EINVAL, "NULL context");
    if (!rho_A0 || !rho_B0) return fail(LBM_EINVAL, "NULL density");
    Ctx& c = ctx->c;
    const long long total = c.dense_elems;
    const double *a = rho_A0, *b = rho_B0;
    if (!on_device) {
        lbm_status s = fields_all_scratch(c);
        if (s != LBM_OK) return s;
        CUDA_TRY(cudaMemcpyAsync(c.fields_all, rho_A0, total * sizeof(double), cudaMemcpyHostToDevice, c.stream));
        CUDA_TRY(cudaMemcpyAsync(c.fields_all + total, rho_B0, total * sizeof(double), cudaMemcpyHostToDevice, c.stream));
        a = c.fields_all;
        b = c.fields_all + total;
    }
    CUDA_TRY(launch_set_rest_all(c, a, b));
    ++c.version;
    if (!on_device) CUDA_TRY(cudaStreamSynchronize(c.stream));
    return LBM_OK;
}

lbm_status lbm_fields_all(lbm_ctx* ctx, double* rho_A, double* rho_B, double* ux, double* uy, int32_t on_device) {
    NvtxRange nvtx_("lbm_fields_all");
    if (!ctx) return fail(LBM_EINVAL, "NULL context");
    Ctx& c = ctx->c;
    const long long total = c.dense_elems;
    double* outs[4] = {rho_A, rho_B, ux, uy};
    if (!on_device || !rho_A || !rho_B || !ux || !uy) {
        lbm_status s = fields_all_scratch(c);
        if (s != LBM_OK) return s;
    }
    double* dst[4];
    for (int q = 0; q < 4; ++q) dst[q] = (on_device && outs[q]) ? outs[q] : c.fields_all + q * total;
    CUDA_TRY(launch_fields_all(c, dst[0], dst[1], dst[2], dst[3]));
    if (on_device) return LBM_OK;
    for (int q = 0; q < 4; ++q)
        if (outs[q]) CUDA_TRY(cudaMemcpyAsync(outs[q], dst[q], total * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    CUDA_TRY(cudaStreamSynchronize(c.stream));
    return check_device_error(c);
}

// Copy streams, staging buffers and events of the overlapped transfers.
static lbm_status xfer_setup(Ctx& c) {
    if (c.xs_in) return LBM_OK;
    const size_t total = (size_t)c.dense_elems;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaMalloc(&c.xin[k], 2 * total * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&c.xout[k], 4 * total * sizeof(double));
        for (cudaEvent_t* ev : {&c.xin_ready[k], &c.xin_free[k], &c.xout_ready[k], &c.xout_free[k]})
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c.xs_out, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c.xs_in, cudaStreamNonBlocking);  // set last: marks done
    if (e != cudaSuccess) {
        const bool oom = e == cudaErrorMemoryAllocation;
        cudaGetLastError();
        for (int k = 0; k < 2; ++k) {
            for (cudaEvent_t* ev : {&c.xin_ready[k], &c.xin_free[k], &c.xout_ready[k], &c.xout_free[k]})
                if (*ev) cudaEventDestroy(*ev), *ev = nullptr;
            if (c.xin[k]) cudaFree(c.xin[k]), c.xin[k] = nullptr;
            if (c.xout[k]) cudaFree(c.xout[k]), c.xout[k] = nullptr;
        }
        if (c.xs_out) cudaStreamDestroy(c.xs_out), c.xs_out = nullptr;
        if (c.xs_in) cudaStreamDestroy(c.xs_in), c.xs_in = nullptr;
        return fail(oom ? LBM_ENOMEM : LBM_ECUDA, "overlapped transfers: %s", cudaGetErrorString(e));
    }
    return LBM_OK;
}

lbm_status lbm_set_densities_all_async(lbm_ctx* ctx, const double* rho_A0, const double* rho_B0) {
    NvtxRange nvtx_("lbm_set_densities_all_async");
    if (!ctx) return fail(LBM_EINVAL, "NULL context");
    if (!rho_A0 || !rho_B0) return fail(LBM_EINVAL, "NULL density");
    Ctx& c = ctx->c;
    lbm_status s = xfer_setup(c);
    if (s != LBM_OK) return s;
    const long long total = c.dense_elems;
    const int k = c.xin_k;
    c.xin_k ^= 1;
    double* a = c.xin[k];
    double* b = c.xin[k] + total;
    // the copy may start as soon as the kernels that read this staging buffer last have run; the
    // state is set in stream order, after everything enqueued before
    CUDA_TRY(cudaStreamWaitEvent(c.xs_in, c.xin_free[k], 0));
    CUDA_TRY(cudaMemcpyAsync(a, rho_A0, total * sizeof(double), cudaMemcpyHostToDevice, c.xs_in));
    CUDA_TRY(cudaMemcpyAsync(b, rho_B0, total * sizeof(double), cudaMemcpyHostToDevice, c.xs_in));
    CUDA_TRY(cudaEventRecord(c.xin_ready[k], c.xs_in));
    CUDA_TRY(cudaStreamWaitEvent(c.stream, c.xin_ready[k], 0));
    CUDA_TRY(launch_set_rest_all(c, a, b));
    CUDA_TRY(cudaEventRecord(c.xin_free[k], c.stream));
    ++c.version;
    return LBM_OK;
}

lbm_status lbm_fields_all_async(lbm_ctx* ctx, double* rho_A, double* rho_B, double* ux, double* uy) {
    NvtxRange nvtx_("lbm_fields_all_async");
    if (!ctx) return fail(LBM_EINVAL, "NULL context");
    Ctx& c = ctx->c;
    lbm_status s = xfer_setup(c);
    if (s != LBM_OK) return s;
    const long long total = c.dense_elems;
    const int k = c.xout_k;
    c.xout_k ^= 1;
    double* dst[4];
    for (int q = 0; q < 4; ++q) dst[q] = c.xout[k] + q * total;
    // the fields pass may overwrite this staging buffer once its previous copy to the host is done;
    // the copies then run on their own stream, beside whatever the context's stream does next
    CUDA_TRY(cudaStreamWaitEvent(c.stream, c.xout_free[k], 0));
    CUDA_TRY(launch_fields_all(c, dst[0], dst[1], dst[2], dst[3]));
    CUDA_TRY(cudaEventRecord(c.xout_ready[k], c.stream));
    CUDA_TRY(cudaStreamWaitEvent(c.xs_out, c.xout_ready[k], 0));
    double* outs[4] = {rho_A, rho_B, ux, uy};
    for (int q = 0; q < 4; ++q)
        if (outs[q]) CUDA_TRY(cudaMemcpyAsync(outs[q], dst[q], total * sizeof(double), cudaMemcpyDeviceToHost, c.xs_out));
    CUDA_TRY(cudaEventRecord(c.xout_free[k], c.xs_out));
    return LBM_OK;
}

lbm_status lbm_diagnostics(lbm_ctx* ctx, int32_t ci, lbm_diag* out) {
    NvtxRange nvtx_("lbm_diagnostics");
    lbm_status s = check_case(ctx, ci);
    if (s != LBM_OK) return s;
    if (!out) return fail(LBM_EINVAL, "NULL output");
    Ctx& c = ctx->c;
    CUDA_TRY(launch_fields(c, ci, nullptr, nullptr, nullptr, nullptr, true));
    c.fields_case = ci;
    c.fields_version = c.version;
    CUDA_TRY(launch_diag_reduce(c, ci));
    double v[kDiagN];
    CUDA_TRY(cudaMemcpyAsync(v, c.diag_out + (size_t)ci * kDiagN, sizeof v, cudaMemcpyDeviceToHost, c.stream));
    CUDA_TRY(cudaStreamSynchronize(c.stream));
    {
        lbm_status es = check_device_error(c);
        if (es != LBM_OK) return es;
    }
    out->mass_A = v[0];
    out->mass_B = v[1];
    out->mom_x = v[2];
    out->mom_y = v[3];
    out->umax = v[4];
    out->rhoA_min = v[5];
    out->rhoA_max = v[6];
    out->rhoB_min = v[7];
    out->rhoB_max = v[8];
    out->n_fluid = (int64_t)llround(v[9]);
    out->unstable = v[10] != 0.0;
    out->pad_ = 0;
    if (out->unstable) return fail(LBM_EUNSTABLE, "case %d: non-finite or non-positive density", ci);
    return LBM_OK;
}

lbm_status lbm_contact_angle(lbm_ctx* ctx, int32_t ci, const lbm_surface* surface, double* theta_deg, double* fit_rms,
                             int64_t* npoints) {
    NvtxRange nvtx_("lbm_contact_angle");
    lbm_status s = check_case(ctx, ci);
    if (s != LBM_OK) return s;
    if (!surface) return fail(LBM_EINVAL, "NULL surface");
    if (surface->kind == LBM_SURFACE_CIRCLE && !(surface->R > 0)) return fail(LBM_EINVAL, "surface radius must be > 0");
    if (surface->kind != LBM_SURFACE_CIRCLE && surface->kind != LBM_SURFACE_FLAT) return fail(LBM_EINVAL, "bad surface kind");
    Ctx& c = ctx->c;
    if (!(c.fields_case == ci && c.fields_version == c.version)) {  // reuse fields of this very state
        CUDA_TRY(launch_fields(c, ci, nullptr, nullptr, nullptr, nullptr, false));
        c.fields_case = ci;
        c.fields_version = c.version;
    }
    double o[4];
    {
        const cudaError_t e = launch_contact_angle(c, ci, *surface, o);
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();  // clear the (non-sticky) allocation error
            return fail(LBM_ENOMEM, "contact angle: out of device memory for the interface points");
        }
        if (e != cudaSuccess) return fail(LBM_ECUDA, "contact angle: %s", cudaGetErrorString(e));
    }
    if (npoints) *npoints = (int64_t)llround(o[2]);
    if (o[3] != 0.0) return fail(LBM_ESTATE, "case %d: only %.0f interface points", ci, o[2]);
    if (theta_deg) *theta_deg = o[0];
    if (fit_rms) *fit_rms = o[1];
    return LBM_OK;
}

lbm_status lbm_diagnostics_all(lbm_ctx* ctx, lbm_diag* out) {
    NvtxRange nvtx_("lbm_diagnostics_all");
    if (!ctx) return fail(LBM_EINVAL, "NULL context");
    if (!out) return fail(LBM_EINVAL, "NULL output");
    Ctx& c = ctx->c;
    const int n = (int)c.hcases.size();
    if (c.ca_batch) {  // the batched contact angle has its density buffer: fill it in the same pass
        double* rho = reinterpret_cast<double*>(c.ca_batch);
        CUDA_TRY(launch_diag_all(c, rho, rho + c.dense_elems));
        c.ca_rho_version = c.version;
    } else {
        CUDA_TRY(launch_diag_all(c));
    }
    std::vector<double> v((size_t)n * kDiagN);
    CUDA_TRY(cudaMemcpyAsync(v.data(), c.diag_out, v.size() * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    CUDA_TRY(cudaStreamSynchronize(c.stream));
    {
        lbm_status es = check_device_error(c);
        if (es != LBM_OK) return es;
    }
    int first_bad = -1;
    for (int i = 0; i < n; ++i) {
        const double* r = v.data() + (size_t)i * kDiagN;
        lbm_diag& o = out[i];
        o.mass_A = r[0];
        o.mass_B = r[1];
        o.mom_x = r[2];
        o.mom_y = r[3];
        o.umax = r[4];
        o.rhoA_min = r[5];
        o.rhoA_max = r[6];
        o.rhoB_min = r[7];
        o.rhoB_max = r[8];
        o.n_fluid = (int64_t)llround(r[9]);
        o.unstable = r[10] != 0.0;
        o.pad_ = 0;
        if (o.unstable && first_bad < 0) first_bad = i;
    }
    if (first_bad >= 0) return fail(LBM_EUNSTABLE, "case %d: non-finite or non-positive density", first_bad);
    return LBM_OK;
}

lbm_status lbm_contact_angle_all(lbm_ctx* ctx, const lbm_surface* surfaces, double* theta_deg, double* fit_rms,
                                 int64_t* npoints) {
    NvtxRange nvtx_("lbm_contact_angle_all");
    if (!ctx) return fail(LBM_EINVAL, "NULL context");
    if (!surfaces) return fail(LBM_EINVAL, "NULL surfaces");
    Ctx& c = ctx->c;
    const int n = (int)c.hcases.size();
    for (int i = 0; i < n; ++i) {
        const lbm_surface& s = surfaces[i];
        if (s.kind != LBM_SURFACE_CIRCLE && s.kind != LBM_SURFACE_FLAT && s.kind != LBM_SURFACE_NONE)
            return fail(LBM_EINVAL, "case %d: bad surface kind", i);
        if (s.kind == LBM_SURFACE_CIRCLE && !(s.R > 0)) return fail(LBM_EINVAL, "case %d: surface radius must be > 0", i);
    }
    bool any = false;
    for (int i = 0; i < n; ++i) any = any || surfaces[i].kind != LBM_SURFACE_NONE;
    std::vector<double> h((size_t)16 * n, 0.0);
    if (!any) {
        for (int i = 0; i < n; ++i) {
            if (theta_deg) theta_deg[i] = NAN;
            if (fit_rms) fit_rms[i] = NAN;
            if (npoints) npoints[i] = 0;
        }
        return LBM_OK;
    }
    {
        const cudaError_t e = enqueue_contact_angle_all(c, surfaces);
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();  // clear the (non-sticky) allocation error
            return fail(LBM_ENOMEM, "batched contact angle: out of device memory for the densities and points");
        }
        if (e != cudaSuccess) return fail(LBM_ECUDA, "batched contact angle: %s", cudaGetErrorString(e));
    }
    CUDA_TRY(cudaMemcpyAsync(h.data(), c.ca_all, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    CUDA_TRY(cudaStreamSynchronize(c.stream));
    for (int i = 0; i < n; ++i) {
        const double* r = h.data() + (size_t)16 * i;
        const bool skip = surfaces[i].kind == LBM_SURFACE_NONE;
        const bool few = !skip && r[8] != 0.0;
        if (theta_deg) theta_deg[i] = (skip || few) ? NAN : r[7];
        if (fit_rms) fit_rms[i] = (skip || few) ? NAN : r[6];
        if (npoints) npoints[i] = skip ? 0 : (int64_t)llround(r[0]);
    }
    return LBM_OK;
}

lbm_status lbm_wall_list(lbm_ctx* ctx, int32_t ci, int32_t* node, uint32_t* subst, uint32_t* seff, double* ax,
                         double* ay, int64_t* n) {
    lbm_status s = check_case(ctx, ci);
    if (s != LBM_OK) return s;
    if (!n) return fail(LBM_EINVAL, "NULL count");
    Ctx& c = ctx->c;
    const DevCase& d = c.hcases[ci];
    *n = d.nwall;
    if (d.nwall == 0) return LBM_OK;
    if (node) CUDA_TRY(cudaMemcpyAsync(node, c.wl_node + d.w_off, d.nwall * sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
    if (subst) CUDA_TRY(cudaMemcpyAsync(subst, c.wl_subst + d.w_off, d.nwall * sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream));
    if (seff) CUDA_TRY(cudaMemcpyAsync(seff, c.wl_seff + d.w_off, d.nwall * sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream));
    if (ax) CUDA_TRY(cudaMemcpyAsync(ax, c.wl_a + d.w_off, d.nwall * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    if (ay) CUDA_TRY(cudaMemcpyAsync(ay, c.wl_a + c.nwall + d.w_off, d.nwall * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    CUDA_TRY(cudaStreamSynchronize(c.stream));
    return LBM_OK;
}

lbm_status lbm_get_populations(lbm_ctx* ctx, int32_t ci, double* f) {
    lbm_status s = check_case(ctx, ci);
    if (s != LBM_OK) return s;
    if (!f) return fail(LBM_EINVAL, "NULL output");
    Ctx& c = ctx->c;
    const long long N = (long long)c.hcases[ci].nx * c.hcases[ci].ny;
    CUDA_TRY(launch_get_state(c, ci, c.dense));
    CUDA_TRY(cudaMemcpyAsync(f, c.dense, 18 * N * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    CUDA_TRY(cudaStreamSynchronize(c.stream));
    return check_device_error(c);
}

lbm_status lbm_set_populations(lbm_ctx* ctx, int32_t ci, const double* f) {
    lbm_status s = check_case(ctx, ci);
    if (s != LBM_OK) return s;
    if (!f) return fail(LBM_EINVAL, "NULL input");
    Ctx& c = ctx->c;
    const long long N = (long long)c.hcases[ci].nx * c.hcases[ci].ny;
    CUDA_TRY(cudaMemcpyAsync(c.dense, f, 18 * N * sizeof(double), cudaMemcpyHostToDevice, c.stream));
    CUDA_TRY(launch_set_state(c, ci, c.dense));
    ++c.version;
    CUDA_TRY(cudaStreamSynchronize(c.stream));
    return LBM_OK;
}

lbm_status lbm_info(lbm_ctx* ctx, lbm_info_t* out) {
    if (!ctx || !out) return fail(LBM_EINVAL, "NULL argument");
    const Ctx& c = ctx->c;
    memset(out, 0, sizeof *out);
    out->ncases = (int32_t)c.cases.size();
    out->storage = c.storage;
    for (size_t i = 0; i < c.cases.size(); ++i) {
        out->nodes += (int64_t)c.cases[i].grid.nx * c.cases[i].grid.ny;
        out->fluid_nodes += c.cases[i].nfluid;
    }
    out->wall_nodes = c.nwall;
    out->steps = c.steps;
    out->state_bytes = (int64_t)(c.pop_elems * c.elem);
    out->device_bytes = (int64_t)c.device_bytes;
    out->block_threads = c.block_threads;
    out->block_rows = c.rows_used;
    out->grid_blocks = c.grid_blocks;
    out->work_items = c.nitems;
    out->wall_inline = c.wall_inline;
    out->pad_ = 0;
    return LBM_OK;
}

lbm_status lbm_set_launch(lbm_ctx* ctx, int32_t threads, int32_t rows) {
    if (!ctx) return fail(LBM_EINVAL, "NULL context");
    if (threads != 128 && threads != 64) return fail(LBM_EINVAL, "the step kernel is built for 64 or 128 threads per block");
    if (rows < -64) return fail(LBM_EINVAL, "rows must be >= -64 (0 or < 0: guided list, < 0 with tail items of -rows rows)");
    Ctx& c = ctx->c;
    CUDA_TRY(cudaStreamSynchronize(c.stream));
    c.block_threads = threads;
    c.block_rows = rows;
    return build_items(c);
}

namespace {
// ------------------------------------------------------------------------------------------------
// Self-test of the bounded pipeline wait: one thread initialises an mbarrier that nothing will ever
// arrive on, waits for it through the step kernel's bounded wait with a short limit, and on giving up
// records error bit 2 in the context's error word, as a step kernel records bit 1.  No copy is
// issued, so nothing is left in flight when the kernel returns.
// ------------------------------------------------------------------------------------------------
__global__ void k_wait_selftest(int* __restrict__ err, unsigned long long limit_cycles) {
    __shared__ __align__(8) unsigned long long bar_word;
    if (threadIdx.x != 0) return;
    const uint32_t bar = smem_u32(&bar_word);
    mbar_init(bar, 1);
    fence_mbar_init();
    if (!mbar_wait_bounded(bar, 0, limit_cycles)) atomicOr(err, 2);
}

}  // namespace

lbm_status lbm_selftest_wait_timeout(lbm_ctx* ctx, double limit_ms) {
    if (!ctx) return fail(LBM_EINVAL, "NULL context");
    if (!(limit_ms > 0.0) || limit_ms > 1000.0) return fail(LBM_EINVAL, "limit_ms must lie in (0, 1000]");
    Ctx& c = ctx->c;
    int rate_khz = 0;  // SM clock in kHz = cycles per millisecond
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (cudaDeviceGetAttribute(&rate_khz, cudaDevAttrClockRate, dev) != cudaSuccess || rate_khz <= 0) {
        cudaGetLastError();
        rate_khz = 2000000;
    }
    k_wait_selftest<<<1, 32, 0, c.stream>>>(c.err, (unsigned long long)(limit_ms * rate_khz));
    CUDA_TRY(cudaGetLastError());
    return check_device_error(c);
}

lbm_status lbm_set_wall_path(lbm_ctx* ctx, int32_t inline_correction) {
    if (!ctx) return fail(LBM_EINVAL, "NULL context");
    if (inline_correction != 0 && inline_correction != 1) return fail(LBM_EINVAL, "inline_correction must be 0 or 1");
    ctx->c.wall_inline = inline_correction;
    drop_graphs(ctx->c);
    return LBM_OK;
}

lbm_status lbm_autotune(lbm_ctx* ctx, int32_t steps, double* best_ms) {
    NvtxRange nvtx_("lbm_autotune");
    if (!ctx) return fail(LBM_EINVAL, "NULL context");
    if (steps < 1) return fail(LBM_EINVAL, "steps must be >= 1");
    Ctx& c = ctx->c;
    const int cand_t[] = {128, 64};
    const int cand_r[] = {0, -8, 16, 32, 64, 128};
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    // Candidates: the current shape first, then every other one.  Each is timed twice and keeps
    // the faster time; another shape replaces the best only when it is at least 1 % faster, so
    // that shapes within the timing noise of each other do not trade places from run to run.
    struct Cand {
        int w, t, r;
    };
    std::vector<Cand> cands{{c.wall_inline, c.block_threads, c.block_rows}};
    for (int w = 0; w < 2; ++w)
        for (int t : cand_t)
            for (int r : cand_r)
                if (!(w == cands[0].w && t == cands[0].t && r == cands[0].r)) cands.push_back({w, t, r});
    double best = 1e300;
    int bt = c.block_threads, br = c.block_rows, bw = c.wall_inline;
    for (const Cand& cd : cands) {
        c.wall_inline = cd.w;
        lbm_status s = lbm_set_launch(ctx, cd.t, cd.r);
        if (s != LBM_OK) continue;
        if (launch_step(c, c.cur, c.stream) != cudaSuccess) continue;
        c.cur ^= 1;
        ++c.steps;
        ++c.version;
        double ms_best = 1e300;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0, c.stream);
            for (int k = 0; k < steps; ++k) {
                launch_step(c, c.cur, c.stream);
                c.cur ^= 1;
                ++c.steps;
                ++c.version;
            }
            cudaEventRecord(e1, c.stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms_best = ms < ms_best ? ms : ms_best;
        }
        if (ms_best / steps < 0.99 * best || best == 1e300) {
            best = ms_best / steps;
            bt = cd.t;
            br = cd.r;
            bw = cd.w;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CUDA_TRY(cudaGetLastError());
    c.wall_inline = bw;
    lbm_status s = lbm_set_launch(ctx, bt, br);
    if (s != LBM_OK) return s;
    if (best_ms) *best_ms = best;
    return LBM_OK;
}

namespace {
struct CkptHeader {
    char magic[8];
    int32_t version, storage, ncases, pad;
    int64_t steps, bytes;
    uint64_t hash;
};

// FNV-1a over the grid, every parameter field by value (never the structs' padding bytes, which a C
// caller may leave undefined) and each case's solid-mask hash, so that a checkpoint only loads into
// a context with the same geometry and parameters.
uint64_t params_hash(const Ctx& c) {
    uint64_t h = 1469598103934665603ULL;
    auto mix = [&](const void* p, size_t n) {
        const unsigned char* b = (const unsigned char*)p;
        for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ULL;
    };
    auto mixi = [&](int64_t v) { mix(&v, sizeof v); };
    auto mixd = [&](double v) { mix(&v, sizeof v); };
    for (const auto& hc : c.cases) {
        const lbm_grid& g = hc.grid;
        const lbm_params& p = hc.params;
        mixi(g.nx); mixi(g.ny); mixi(g.bc_x); mixi(g.bc_y);
        mixd(p.tau[0]); mixd(p.tau[1]); mixd(p.G_AB); mixi(p.mode); mixd(p.lambda); mixd(p.G_w2); mixd(p.delta);
        mixd(p.g[0]); mixd(p.g[1]); mixd(p.u_in); mixd(p.rho_in[0]); mixd(p.rho_in[1]);
        mixd(p.rho0_store[0]); mixd(p.rho0_store[1]); mixd(p.u_wall[0]); mixd(p.u_wall[1]);
        mixi(p.inlet_profile); mixi(p.second_layer); mixi(p.adhesion_stencil);
        mixi(p.outlet); mixd(p.rho_out[0]); mixd(p.rho_out[1]);
        mixi((int64_t)hc.mask_hash);
    }
    return h;
}
}  // namespace

lbm_status lbm_save(lbm_ctx* ctx, const char* path) {
    if (!ctx || !path) return fail(LBM_EINVAL, "NULL argument");
    Ctx& c = ctx->c;
    std::vector<unsigned char> buf(c.pop_elems * c.elem);
    CUDA_TRY(cudaMemcpyAsync(buf.data(), c.f[c.cur], buf.size(), cudaMemcpyDeviceToHost, c.stream));
    CUDA_TRY(cudaStreamSynchronize(c.stream));
    CkptHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, "LBMGB300", 8);
    h.version = 3;  // 3: (A, B) pairs, the nine planes of a row side by side
    h.storage = c.storage;
    h.ncases = (int32_t)c.cases.size();
    h.steps = c.steps;
    h.bytes = (int64_t)buf.size();
    h.hash = params_hash(c);
    FILE* fp = fopen(path, "wb");
    if (!fp) return fail(LBM_EIO, "cannot open %s for writing", path);
    bool ok = fwrite(&h, sizeof h, 1, fp) == 1 && fwrite(buf.data(), 1, buf.size(), fp) == buf.size();
    ok = (fclose(fp) == 0) && ok;
    return ok ? LBM_OK : fail(LBM_EIO, "short write to %s", path);
}

lbm_status lbm_load(lbm_ctx* ctx, const char* path) {
    if (!ctx || !path) return fail(LBM_EINVAL, "NULL argument");
    Ctx& c = ctx->c;
    FILE* fp = fopen(path, "rb");
    if (!fp) return fail(LBM_EIO, "cannot open %s", path);
    CkptHeader h;
    std::vector<unsigned char> buf(c.pop_elems * c.elem);
    bool ok = fread(&h, sizeof h, 1, fp) == 1;
    if (ok && (memcmp(h.magic, "LBMGB300", 8) != 0 || h.version != 3 || h.storage != c.storage ||
               h.ncases != (int32_t)c.cases.size() || h.bytes != (int64_t)buf.size() || h.hash != params_hash(c))) {
        fclose(fp);
        return fail(LBM_EIO, "%s does not match this context", path);
    }
    ok = ok && fread(buf.data(), 1, buf.size(), fp) == buf.size();
    fclose(fp);
    if (!ok) return fail(LBM_EIO, "short read from %s", path);
    CUDA_TRY(cudaMemcpyAsync(c.f[c.cur], buf.data(), buf.size(), cudaMemcpyHostToDevice, c.stream));
    CUDA_TRY(cudaStreamSynchronize(c.stream));
    c.steps = h.steps;
    ++c.version;
    return LBM_OK;
}

const char* lbm_status_str(int32_t s) {
    switch (s) {
        case LBM_OK: return "LBM_OK";
        case LBM_EINVAL: return "LBM_EINVAL";
        case LBM_ENOMEM: return "LBM_ENOMEM";
        case LBM_ECUDA: return "LBM_ECUDA";
        case LBM_EUNSTABLE: return "LBM_EUNSTABLE";
        case LBM_ETIMEOUT: return "LBM_ETIMEOUT";
        case LBM_ESTATE: return "LBM_ESTATE";
        case LBM_EIO: return "LBM_EIO";
        default: return "LBM_UNKNOWN";
    }
}

const char* lbm_last_error(void) { return g_err.c_str(); }

}  // extern "C"
