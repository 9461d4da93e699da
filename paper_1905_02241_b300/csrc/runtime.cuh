// runtime.cuh -- host-side objects of the C ABI (contexts, mechanisms,
// fused-step plans, surrogates), shared by api.cu and api_surrogate.cu.
#pragma once

#include <cuda_bf16.h>

#include <memory>
#include <cstdint>
#include <vector>

#include "kernels.cuh"

struct nmodl_surrogate;
struct nmodl_cable;

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

template <typename T>
inline cudaError_t dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) return cudaSuccess;
    return cudaMalloc((void**)p, count * sizeof(T));
}

struct GraphEntry {
    double* v;
    double* rhs;
    double* d;
    double dt, cm;
    int nsteps, clamp;
    cudaGraphExec_t exec;
};

struct Plan {
    std::vector<nmodl_mech*> mechs;
    nmodl_cable* cable = nullptr;   // cable form: tiles of whole cells
    int precision = 0;
    int variant = 0;                // fused kernel: precision + 2 * (small systems / ions)
    int64_t n_nodes = 0;
    bool fused = false;
    // single-HH gate-warp form (k_hh.cu): nodes per block, 0 = not used
    int hh_per_block = 0;
    // one NMODL_KIN9 mechanism with a surrogate, instance i on node i: the
    // surrogate kernel runs the whole step (current, rhs/d, v, state)
    bool sur_step = false;
    // fused form
    int n_tiles = 0, block = 256, tile_stride = 0;
    size_t smem = 0;
    int32_t* d_tiles = nullptr;
    nmodl::MechD* d_md = nullptr;
    nmodl::Kin9D* d_k9 = nullptr;   // rate constants of the 9-state mechanisms
    int32_t* d_counter = nullptr;   // persistent form's tile queue
    uint16_t* d_sched = nullptr;    // cable form: level schedules of the tiles
    bool persistent = false;
    size_t budget = 0;
    int grid = 0;                   // blocks per launch
    std::vector<GraphEntry> graphs;
    ~Plan() {
        for (auto& g : graphs) cudaGraphExecDestroy(g.exec);
        cudaFree(d_tiles);
        cudaFree(d_md);
        cudaFree(d_k9);
        cudaFree(d_counter);
        cudaFree(d_sched);
    }
};

struct nmodl_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    nmodl_options opt{};
    int32_t* d_err = nullptr;
    std::vector<std::unique_ptr<Plan>> plans;
    int live_mechs = 0;
    int64_t epoch = 0;  // bumped when options, mechanisms or surrogates change
    double* ion[4] = {nullptr, nullptr, nullptr, nullptr};  // per-node ina, ik, ica (1..3)
    int64_t ion_nodes = 0;
    bool has_ions() const { return ion[1] || ion[2] || ion[3]; }
};

struct nmodl_mech {
    nmodl_ctx* ctx = nullptr;
    int type = 0;
    int64_t n = 0, n_nodes = 0, stride = 0;
    int n_states = 0;
    std::vector<double> params;
    int32_t* d_ni = nullptr;
    double* d_states = nullptr;
    int32_t* d_chunk = nullptr;
    int64_t n_chunks = 0;
    nmodl::MechD md{};
    nmodl::MechD* d_md = nullptr;
    nmodl::Kin9D kd{};
    nmodl::Kin9D* d_kd = nullptr;
    nmodl::KinCounters* d_cnt = nullptr;
    nmodl::Kin3D k3{};
    nmodl::Kin3D* d_k3 = nullptr;
    nmodl::CacumD cd{};
    nmodl::CacumD* d_cd = nullptr;
    int ion = NMODL_ION_NONE;       // USEION WRITE tag of the whole current
    int64_t calls = 0;
    // surrogate stand-in for the kinetic Newton solve (NMODL_KIN9 only)
    nmodl_surrogate* sur = nullptr;
    double sur_tol = 0.0;
    int32_t* d_fb_list = nullptr;   // fallback instance list (n entries)
    int32_t* d_fb_count = nullptr;  // its length
    int64_t sur_calls = 0;
};

struct nmodl_surrogate {
    nmodl_ctx* ctx = nullptr;
    int scaled = 1;
    int64_t max_batch = 0;
    int step = 0;
    float* params = nullptr;          // FP32 master, padded layout
    __nv_bfloat16* wbf = nullptr;     // bf16 weight copies
    unsigned char* img = nullptr;     // the training kernel's weight image (kTrImgBytes)
    float *grad = nullptr, *m = nullptr, *v = nullptr;
    __half2 *ds1 = nullptr, *ds2 = nullptr, *ds3 = nullptr;  // SiLU'(Z), whole 128-row tiles
    float *part = nullptr, *loss_part = nullptr, *loss = nullptr;
    int n_part_max = 0;                                     // CTAs of the training kernel
};


// shared helpers (api.cu)
int nmodl_cuda_status(cudaError_t e);
void nmodl_invalidate_plans(nmodl_ctx* c, nmodl_mech* m);
extern "C" {
void nmodl_enqueue_state(nmodl_mech* m, double dt, const double* v);
void nmodl_enqueue_cur(nmodl_mech* m, const double* v, double* rhs, double* d);
void nmodl_count_states(nmodl_mech* m, int64_t k);
void nmodl_zero_ions(nmodl_ctx* c, int64_t n_nodes);
// NMODL_OK when every mechanism's ion reads are satisfied by the context
int nmodl_check_ion_reads(nmodl_ctx* c, nmodl_mech* const* mechs, int n_mechs);
// step plan of a mechanism list (isolated, or the cable form of cb), built
// and autotuned on first use; fused windows run through nmodl_run_window
Plan* nmodl_get_plan(nmodl_ctx* c, nmodl_mech* const* mechs, int n_mechs, const double* v,
                     int* rc, nmodl_cable* cb);
cudaError_t nmodl_run_window(nmodl_ctx* c, Plan* p, nmodl_mech* const* mechs, int n_mechs,
                             double dt, double cm, double* v, double* rhs, double* d, int w);
}

struct nmodl_cable {
    nmodl_ctx* ctx = nullptr;
    int64_t n_nodes = 0, n_cells = 0;
    int32_t* d_parent = nullptr;
    double *d_ga = nullptr, *d_gb = nullptr;
    int64_t* d_cell_off = nullptr;
    std::vector<int64_t> cell_off;             // host copies: cell boundaries,
    std::vector<int32_t> parent;               // parents (for the tile schedules)
    double *d_d2 = nullptr, *d_r2 = nullptr;  // eliminated system (scratch)
    std::vector<GraphEntry> graphs;
    std::vector<nmodl_mech*> graph_mechs;      // mechanism list the graphs hold
    int64_t graph_epoch = -1;                  // context epoch they were made in
};
