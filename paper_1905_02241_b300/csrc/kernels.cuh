// kernels.cuh -- launch interfaces between the C-ABI runtime (api.cu) and
// the kernels of libnmodl_b300.so.
#pragma once

#include "nmodl_internal.cuh"
#include "small_systems.cuh"

namespace nmodl {

constexpr int kFusedMaxBlock = 1024;
// the fused variant with the 9-state scheme comes in two builds, picked by
// the block size of the launch: blocks of at most kFusedKinBlock threads
// run the register-rich build (the banded Newton solve in ~245 registers;
// MIXED two blocks per SM), larger blocks (up to fused_kin_wide_block) the
// one compiled for a single such block per SM (FP64 768 threads at 80
// registers, MIXED 512 at 128)
constexpr int kFusedKinBlock = 256;
__host__ __device__ constexpr int fused_kin_wide_block(int prec) {
    return prec == NMODL_MIXED ? 512 : 768;
}

// node-major slots per instance of the fused step's flat layout: one
// (e, g) per current (HH: sodium, potassium, leak; the calcium buffer none)
__host__ __device__ constexpr int flat_slots(int kind) {
    return kind == NMODL_HH ? 3 : kind == NMODL_CACUM ? 0 : 1;
}

// Arguments of the fused multi-step tile kernel (passed by value).
struct FusedArgs {
    const MechD* md;                       // n_types descriptors
    const Kin9D* k9d;                      // n_types (NMODL_KIN9 entries used)
    int32_t n_types;
    int32_t n_gates[kMaxMechsFused];
    double* states[kMaxMechsFused];        // SoA, row stride below
    int64_t stride[kMaxMechsFused];
    const int32_t* ni[kMaxMechsFused];
    const int32_t* tiles;                  // tile records (work list)
    int32_t tile_stride;                   // 2 + 2 * n_types
    int32_t n_tiles;
    int32_t* tile_counter;                 // persistent form: next tile
    int32_t nsteps;
    int32_t clamp_v;
    int32_t pade;                          // (1,1) Pade cnexp factor
    double* v;
    double* rhs;
    double* d;
    double dt, cm;
    int32_t* err;
    // cable form (tiles hold whole cells): per-node parent (-1 at roots),
    // axial conductances, and the tiles' level schedules of the tree solve
    // (tile record fields 2 + 2 T and 3 + 2 T: offset and length in sched)
    const int32_t* parent;
    const double* ga;
    const double* gb;
    const uint16_t* sched;
    int32_t cable;
    // ion currents (USEION): ion[1..3] = ina, ik, ica per node (null: not
    // recorded); with ions set, the step's ica is kept per node for the
    // state updates that read it (calcium buffer)
    double* ion[4];
    int32_t ions;
    int32_t newton_max_iter;
    double newton_tol;
    int32_t ir_max;  // refinements of the mixed small systems
    // Newton / refinement counters of the KIN9, KIN3 and CACUM mechanisms
    // (null: not counted, e.g. autotuning trials)
    struct KinCounters* cnt[kMaxMechsFused];
};

void launch_init_gates(const MechD* md, int n_gates, int64_t n, const int32_t* ni,
                       const double* v, double* st, int64_t stride, int32_t* err,
                       cudaStream_t s);
void launch_state_gates(int prec, const MechD* md, int n_gates, int64_t n,
                        const int32_t* ni, const double* v, double* st,
                        int64_t stride, double dt, int pade, int32_t* err,
                        cudaStream_t s);
// ion_a / ion_b (may be null): per-node ion currents accumulated with the
// same segmented reduction -- HH: ina and ik; other kinds: the whole current
// into ion_a (the array of the ion the mechanism is tagged with)
void launch_cur_seg(int kind, const void* desc, int64_t n_chunks,
                    const int32_t* chunk, const int32_t* ni, const double* v,
                    const double* st, int64_t stride, double* rhs, double* d,
                    double* ion_a, double* ion_b, int32_t* err, cudaStream_t s);
// variant = precision + 2 * ext + 2 * kin (ext: the kernel instantiated with
// the small systems KIN3 / CACUM and the ion sums; kin: ext and the 9-state
// scheme, variants 4 and 5, blocks of at most fused_kin_wide_block, the
// build chosen by the block size)
cudaError_t launch_fused(int variant, const FusedArgs& a, int grid, int block,
                         size_t smem, cudaStream_t s);
int fused_resident_grid(int variant, int n_tiles, int block, size_t smem);
size_t fused_static_smem(int variant);
cudaError_t fused_prepare(int variant, size_t max_smem);

// kinetic scheme
struct KinCounters {
    unsigned long long iters;     // total Newton / refinement updates
    unsigned long long nonconv;   // instances that hit the iteration cap
    int32_t max_iter_seen;
    int32_t pad;
    unsigned long long fallback;  // surrogate instances sent to Newton
};
// Warp-reduced update of the counters (every lane of the warp calls it).
__device__ __forceinline__ void warp_count(KinCounters* cnt, unsigned long long it,
                                           unsigned long long nc, int mx) {
    if (!cnt) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        it += __shfl_down_sync(0xffffffffu, it, o);
        nc += __shfl_down_sync(0xffffffffu, nc, o);
        mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (it) atomicAdd(&cnt->iters, it);
        if (nc) atomicAdd(&cnt->nonconv, nc);
        if (mx) atomicMax(&cnt->max_iter_seen, mx);
    }
}

void launch_kin9_init(const Kin9D* kd, int64_t n, const int32_t* ni,
                      const double* v, double* st, int64_t stride, int32_t* err,
                      cudaStream_t s);
// kd: the device descriptor; kh: the same on the host (the launch folds
// its rate constants with dt)
void launch_kin9_state(int prec, const Kin9D* kd, const Kin9D& kh, int64_t n, const int32_t* ni,
                       const double* v, double* st, int64_t stride, double dt,
                       const double* dt_arr, double tol, int max_iter, int ir_max,
                       const int32_t* list, int64_t n_list_max,
                       const int32_t* n_list_dev, KinCounters* cnt,
                       int32_t* err, cudaStream_t s);

// small systems: 3-state kinetic scheme and the calcium buffer
void launch_kin3_init(const Kin3D* kd, int64_t n, const int32_t* ni, const double* v,
                      double* st, int64_t stride, int32_t* err, cudaStream_t s);
// kd / cd: the device descriptor; kh / ch: the same on the host (its FP32
// copy is passed by value to the mixed form)
void launch_kin3_state(int prec, const Kin3D* kd, const Kin3D& kh, int64_t n, const int32_t* ni,
                       const double* v, double* st, int64_t stride, double dt, double tol,
                       int ir_max, KinCounters* cnt, int32_t* err, cudaStream_t s);
void launch_cacum_init(const CacumD* cd, int64_t n, double* st, int64_t stride,
                       cudaStream_t s);
void launch_cacum_state(int prec, const CacumD* cd, const CacumD& ch, int64_t n,
                        const int32_t* ni, const double* ica, double* st, int64_t stride,
                        double dt, double tol, int max_iter, int ir_max, KinCounters* cnt,
                        int32_t* err, cudaStream_t s);
// FP32 copies of the small systems' parameters (host)
Kin3F kin3_f32(const Kin3D& K);
CacumF cacum_f32(const CacumD& C);

// Arguments of the single-HH gate-warp step (k_hh.cu): n nodes, instance i
// on node i, per_block nodes per block of three warps.
struct HhArgs {
    GateD gate[3];         // m, h, n folded for this launch's dt (fold_gate)
    double g[3], e[3];     // gnabar, gkbar, gl; ena, ek, el
    int64_t n;
    int32_t per_block;     // 1..32
    int32_t nsteps;
    int32_t clamp_v;
    double dt, cm;
    double* v;
    double* states;        // m, h, n rows of the given stride
    int64_t stride;
    double* rhs;
    double* d;
    int32_t* err;
};
// nodes per block: the network spread over the SMs, at most 32
int hh_warps_per_block(int64_t n, int sms);
cudaError_t launch_hh_gate_warps(const HhArgs& a, cudaStream_t s);


// common
void launch_chunk_starts(const int32_t* ni, int64_t n, int64_t n_chunks,
                         int32_t* chunk, cudaStream_t s);
void launch_validate_index(const int32_t* ni, int64_t n, int64_t n_nodes,
                           int32_t* flags, cudaStream_t s);
void launch_vupdate(int64_t n_nodes, double* v, const double* rhs, double* d,
                    double cmdt, int clamp, int32_t* err, cudaStream_t s);
void launch_tile_bounds(const int32_t* ni, int64_t n, const int64_t* nodes,
                        int64_t n_bounds, int32_t* out, cudaStream_t s);
void launch_cable_solve(int64_t n_cells, const int64_t* cell_off, const int32_t* parent,
                        const double* ga, const double* gb, double cmdt, double* v,
                        double* rhs, double* d, double* d2, double* r2, int clamp,
                        int32_t* err, cudaStream_t s);

}  // namespace nmodl
