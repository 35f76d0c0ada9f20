// Diagnostics of caller-held device fields without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs inside a framework which owns all device
// memory through its own pool and forbids allocations outside it, real-time loops where the
// implicit synchronisation and latency of cudaMalloc/cudaFree are not acceptable, or tools that
// attach to a process whose device memory is already fully committed.  lbm_diagnostics_noalloc
// serves them: it reads device arrays the caller already owns and keeps its per-block partial
// records in a fixed-size array placed in the library's own device image (file-scope
// __device__ storage), so it allocates nothing -- neither cudaMalloc/cudaFree nor any allocating
// library routine.
//
// The scratch array is shared by every call on a device and keeps the last call's contents.  Each
// call overwrites exactly the records it reads, so nothing has to be cleared first; calls whose
// work overlaps on the GPU (different streams, or different host threads on one stream without
// ordering) race on it.
#include <mutex>

#include "lbm_internal.h"

namespace lbm {
lbm_status report_error(lbm_status s, const char* fmt, ...);
}

using namespace lbm;

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaPerThread = 16;
constexpr int kNaNodesPerBlock = kNaThreads * kNaPerThread;                   // 4,096
constexpr int kNaMaxBlocks = 4096;
constexpr long long kNaMaxNodes = (long long)kNaMaxBlocks * kNaNodesPerBlock;  // 16,777,216
constexpr int kNaVals = 11;  // mass_A, mass_B, mom_x, mom_y, umax, rA min/max, rB min/max, n, unstable

// per-block partial records, then the final record (384 KB + 88 B)
static __device__ __align__(256) double g_na_scratch[(kNaMaxBlocks + 1) * kNaVals];

std::mutex g_na_mutex;
constexpr int kNaMaxDevices = 64;
double* g_na_ptr[kNaMaxDevices] = {nullptr};

__device__ __forceinline__ double na_combine(int q, double a, double b) {
    if (q == 4 || q == 6 || q == 8 || q == 10) return fmax(a, b);
    if (q == 5 || q == 7) return fmin(a, b);
    return a + b;
}

__device__ __forceinline__ double na_neutral(int q) {
    return (q == 5 || q == 7) ? INFINITY : (q == 4 || q == 6 || q == 8) ? -INFINITY : 0.0;
}

// One record per block over nodes [blockIdx.x * 4096, +4096); fixed reduction order.
__global__ void __launch_bounds__(kNaThreads) k_na_partial(const double* __restrict__ rA, const double* __restrict__ rB,
                                                          const double* __restrict__ ux, const double* __restrict__ uy,
                                                          const uint8_t* __restrict__ solid, long long n,
                                                          double* __restrict__ scratch) {
    double v[kNaVals];
    for (int q = 0; q < kNaVals; ++q) v[q] = na_neutral(q);
    const long long base = (long long)blockIdx.x * kNaNodesPerBlock;
    for (int k = 0; k < kNaPerThread; ++k) {
        const long long s = base + (long long)k * kNaThreads + threadIdx.x;
        if (s >= n || solid[s]) continue;
        const double a = rA[s], b = rB[s], x = ux[s], y = uy[s], rho = a + b;
        const double um = sqrt(x * x + y * y);
        v[0] += a;
        v[1] += b;
        v[2] += rho * x;
        v[3] += rho * y;
        v[4] = fmax(v[4], um);
        v[5] = fmin(v[5], a);
        v[6] = fmax(v[6], a);
        v[7] = fmin(v[7], b);
        v[8] = fmax(v[8], b);
        v[9] += 1.0;
        if (!(a > 0.0) || !(b > 0.0) || !isfinite(um) || !isfinite(a) || !isfinite(b)) v[10] = 1.0;
    }
    __shared__ double red[kNaThreads / 32][kNaVals];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = 0; q < kNaVals; ++q) {
        double x = v[q];
        for (int off = 16; off > 0; off >>= 1) x = na_combine(q, x, __shfl_xor_sync(0xffffffffu, x, off));
        if (lane == 0) red[warp][q] = x;
    }
    __syncthreads();
    if (threadIdx.x < kNaVals) {
        const int q = threadIdx.x;
        double x = red[0][q];
        for (int w = 1; w < kNaThreads / 32; ++w) x = na_combine(q, x, red[w][q]);
        scratch[(long long)blockIdx.x * kNaVals + q] = x;
    }
}

// One warp combines this call's block records in block order into the final record.
__global__ void k_na_final(int nblocks, double* __restrict__ scratch) {
    const int lane = threadIdx.x;
    for (int q = 0; q < kNaVals; ++q) {
        double x = na_neutral(q);
        for (int b = lane; b < nblocks; b += 32) x = na_combine(q, x, scratch[(long long)b * kNaVals + q]);
        for (int off = 16; off > 0; off >>= 1) x = na_combine(q, x, __shfl_xor_sync(0xffffffffu, x, off));
        if (lane == 0) scratch[(long long)kNaMaxBlocks * kNaVals + q] = x;
    }
}

// Device address of the scratch array on the current device, looked up once per device.
lbm_status na_scratch(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return report_error(LBM_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kNaMaxDevices) return report_error(LBM_ECUDA, "device ordinal %d not supported", dev);
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess || !p)
            return report_error(LBM_ECUDA, "cudaGetSymbolAddress of the diagnostics scratch: %s", cudaGetErrorString(e));
        g_na_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_na_ptr[dev];
    return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_diagnostics_noalloc(const double* rho_A, const double* rho_B, const double* ux,
                                              const double* uy, const uint8_t* solid, int32_t nx, int32_t ny,
                                              void* cuda_stream, lbm_diag* out) {
    if (!rho_A || !rho_B || !ux || !uy || !solid || !out) return report_error(LBM_EINVAL, "NULL argument");
    if (nx < 1 || ny < 1) return report_error(LBM_EINVAL, "nx, ny must be >= 1");
    const long long n = (long long)nx * ny;
    if (n > kNaMaxNodes)
        return report_error(LBM_EINVAL, "nx*ny = %lld exceeds the %lld-node limit of the no-allocation diagnostics",
                            n, kNaMaxNodes);
    double* scratch = nullptr;
    lbm_status s = na_scratch(&scratch);
    if (s != LBM_OK) return s;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int nblocks = (int)((n + kNaNodesPerBlock - 1) / kNaNodesPerBlock);
    k_na_partial<<<nblocks, kNaThreads, 0, st>>>(rho_A, rho_B, ux, uy, solid, n, scratch);
    k_na_final<<<1, 32, 0, st>>>(nblocks, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return report_error(LBM_ECUDA, "diagnostics kernels: %s", cudaGetErrorString(e));
    double v[kNaVals];
    e = cudaMemcpyAsync(v, scratch + (long long)kNaMaxBlocks * kNaVals, sizeof v, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return report_error(LBM_ECUDA, "diagnostics read-back: %s", cudaGetErrorString(e));
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
    if (out->unstable) return report_error(LBM_EUNSTABLE, "non-finite or non-positive density in the given fields");
    return LBM_OK;
}
