// Host-side internals of the library: the context and the kernel launch entry points that the
// C-ABI layer (lbm_api.cu) calls.
#pragma once

#include <nvtx3/nvToolsExt.h>
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_device.cuh"

namespace lbm {

constexpr int kDiagN = 12;  // per-item partial record: see diag_partial layout in lbm_step.cu

struct HostCase {
    lbm_grid grid;
    lbm_params params;
    int64_t nfluid = 0;
    uint64_t mask_hash = 0;  // hash of the solid mask (checkpoint matching)
};

// NVTX range over the host side of one entry point (visible in Nsight Systems timelines; NVTX v3
// is header-only and costs a few nanoseconds when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

struct Ctx {
    int storage = LBM_STORE_F32;
    size_t elem = 4;                 // bytes per stored population value
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    int num_sms = 0;
    long alloc_count = 0;            // allocations made through dalloc (failure-injection hook)

    std::vector<HostCase> cases;
    std::vector<DevCase> hcases;     // host copy of the descriptors
    DevCase* dcases = nullptr;

    long long pop_elems = 0;         // elements in one population buffer
    long long dense_elems = 0;       // sum of nx*ny (per-node arrays)
    long long nwall = 0;

    void* f[2] = {nullptr, nullptr}; // ping-pong population buffers (post-collision f*)
    int cur = 0;                     // f[cur] holds the current state
    uint16_t* flags = nullptr;       // [dense_elems] node flags
    uint32_t* wsub = nullptr;        // [dense_elems] substitution mask of wall-list nodes
    void* wa = nullptr;              // [2][dense_elems] adhesion vectors of wall-list nodes, compute type
    uint8_t* solid = nullptr;        // [dense_elems] copy of the masks
    CUtensorMap* tmaps = nullptr;    // [ncases][3] tensor maps: population buffers 0 and 1, flag rows
    uint16_t* gflags = nullptr;      // flags with 8 ghost columns per side ([ny][gpitch] per case)
    std::vector<long long> gf_off;   // element offset of each case's block in gflags
    std::vector<int> gf_pitch;       // its row pitch (elements)
    int* err = nullptr;              // device error word (pipeline wait gave up)
    int* sched = nullptr;            // step kernel's work-item and finished-block counters
    int32_t* wl_node = nullptr;      // wall list, all cases back to back
    uint32_t* wl_subst = nullptr;
    uint32_t* wl_seff = nullptr;
    double* wl_a = nullptr;          // [2][nwall] adhesion vectors in FP64

    // work list of the step kernel
    int block_threads = 128;
    int block_rows = 0;              // 0: automatic
    int wall_inline = 0;             // step kernel variant: wall-list correction inline (1) or called (0)
    int* slide_list = nullptr;       // cases with sliding walls (device), fixed up after each step
    int slide_n = 0;
    int slide_max_nx = 0;
    int rows_used = 0;
    int grid_blocks = 0;
    int4* items = nullptr;
    int nitems = 0;                  // step list: items [0, nitems)
    int nitems_all = 0;              // per-case lists follow: items [nitems, nitems_all)

    // scratch
    double* dense = nullptr;         // [18 * max case nodes] doubles for population transfers
    long long dense_cap = 0;
    double* fields = nullptr;        // [4][max case nodes]
    double* fields_all = nullptr;    // [4][all nodes] for the batched host transfers (on first use)
    // overlapped host transfers (lbm_set_densities_all_async, lbm_fields_all_async; on first use):
    // copy streams, double-buffered device staging and the events that order them with c.stream
    cudaStream_t xs_in = nullptr, xs_out = nullptr;
    double* xin[2] = {nullptr, nullptr};   // [2][all nodes] densities from the host
    double* xout[2] = {nullptr, nullptr};  // [4][all nodes] fields for the host
    cudaEvent_t xin_ready[2] = {nullptr, nullptr}, xin_free[2] = {nullptr, nullptr};
    cudaEvent_t xout_ready[2] = {nullptr, nullptr}, xout_free[2] = {nullptr, nullptr};
    int xin_k = 0, xout_k = 0;
    double* diag_part = nullptr;     // [nitems][kDiagN]
    double* diag_out = nullptr;      // [ncases][kDiagN]
    double* ca_work = nullptr;       // contact-angle reductions
    double* ca_all = nullptr;        // [ncases][16] contact-angle status records of the batched call
    unsigned char* ca_batch = nullptr;  // batched contact angle: FP64 densities of all cases
    size_t ca_batch_bytes = 0;          // (allocated by its first call)
    unsigned char* ca_points = nullptr; // contact angle: case records, interface-point keys (8 B per
                                        // node of all cases), counts (allocated by the first call)

    // CUDA graph of kGraphSteps step launches
    cudaGraphExec_t graph = nullptr;
    int graph_steps = 0;

    int64_t steps = 0;
    size_t device_bytes = 0;
    uint64_t version = 1;            // bumped by every change of the state
    int fields_case = -1;            // case whose fields the scratch holds ...
    uint64_t fields_version = 0;     // ... computed at this state version
    uint64_t ca_rho_version = 0;     // the batched contact angle's densities hold this state version
};

// lbm_step.cu
cudaError_t launch_step(Ctx& c, int in_buf, cudaStream_t s);
cudaError_t launch_fields(Ctx& c, int case_index, double* rhoA, double* rhoB, double* ux, double* uy,
                          bool diag);
cudaError_t launch_diag_reduce(Ctx& c, int case_index);
// partial sums of every case in one launch over the per-case lists, then one reduction per case
// per-case diagnostics of all cases; with rhoA_all / rhoB_all also the densities of all cases
// (case offsets as in the batched fields), in the same pass
cudaError_t launch_diag_all(Ctx& c, double* rhoA_all = nullptr, double* rhoB_all = nullptr);
// densities of every case into [dense_elems] arrays indexed d_off + y nx + x (zero at solid nodes)
// every case's fields at once (fields_global indexing: case d_off + y nx + x); ux_all / uy_all may be
// NULL for densities only
cudaError_t launch_fields_all(Ctx& c, double* rhoA_all, double* rhoB_all, double* ux_all, double* uy_all);
cudaError_t launch_densities_all(Ctx& c, double* rhoA_all, double* rhoB_all);
cudaError_t launch_set_state(Ctx& c, int case_index, const double* dense_f);
// f = f^eq(rho_k, 0) in every case from densities of all cases back to back (one launch per 65,535 cases)
cudaError_t launch_set_rest_all(Ctx& c, const double* rhoA_all, const double* rhoB_all);
cudaError_t launch_get_state(Ctx& c, int case_index, double* dense_f);
cudaError_t launch_feq_rest(Ctx& c, int case_index, const double* rhoA, const double* rhoB, double* dense_f);
int step_smem_bytes(int storage, int threads);
cudaError_t step_occupancy(int storage, int threads, int* blocks_per_sm);
int ghost_cols(int storage);      // ghost columns on each side of a stored population row
int box_extra_cols(int storage);  // tensor-box columns beyond the block width

// lbm_geometry.cu
cudaError_t launch_flags(Ctx& c, int case_index, int32_t* row_counts);
cudaError_t launch_scan_rows(const int32_t* counts, int32_t* offsets, int n, cudaStream_t s);
cudaError_t launch_wall_fill(Ctx& c, int case_index, const int32_t* row_offsets);
cudaError_t launch_wall_cast(Ctx& c, int case_index);
cudaError_t launch_flags_ghost(Ctx& c, int case_index);

// lbm_contact.cu
cudaError_t launch_contact_angle(Ctx& c, int case_index, const lbm_surface& surf, double* host_out4);
// Enqueue the contact-angle passes of one case (ctx->fields must hold its densities by then); the
// 16-double status record st (device) receives theta at [7], rms at [6], points at [0], the
// too-few-points flag at [8].  No synchronisation.
cudaError_t enqueue_contact_angle(Ctx& c, int case_index, const lbm_surface& surf, double* st);
// Contact angles of every case: densities of all cases, then each fit pass as one launch over all
// cases' blocks (per-case block counts as in the single-case call, so results agree bit for bit).
// surf: host, one per case (LBM_SURFACE_NONE skips).  Records land in ctx->ca_all; no
// synchronisation.
cudaError_t enqueue_contact_angle_all(Ctx& c, const lbm_surface* surf);

}  // namespace lbm
