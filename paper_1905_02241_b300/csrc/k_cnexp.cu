// k_cnexp.cu -- cnexp-family kernels (HH and generic gates) and the fused
// step for sm_103a.
//
//  k_init_gates      INITIAL: gate := minf(v[node])
//  k_state_gates     nrn_state, one thread per (instance, gate): the cnexp
//                    exact exponential update (Section 5.2)
//  k_cur_seg         nrn_cur with the analytic conductance (Section 5.2,
//                    CONDUCTANCE) and a node_index-sorted segmented
//                    warp-shuffle reduction into rhs/d and the ion arrays
//                    (no atomics); HH, CNEXP, KIN9 and KIN3 currents
//  k_fused_tiles     nsteps whole network steps (cur -> v -> state) per node
//                    tile, with the tile's states resident in shared memory
//                    for the whole window (isolated compartments: tiles never
//                    exchange data; cable form: tiles of whole cells with the
//                    tree solve inside); HH, CNEXP and, in the EXT
//                    instantiation, the 3-state scheme, the calcium buffer
//                    and ion sums; in the KIN instantiation also the 9-state
//                    scheme (one thread per instance runs its banded Newton
//                    solve)
#include <algorithm>
#include <climits>

#include "kernels.cuh"
#include "kin9.cuh"
#include "small_systems.cuh"

namespace nmodl {

// ---------------------------------------------------------------- init

__global__ void k_init_gates(const MechD* __restrict__ md, int64_t n,
                             const int32_t* __restrict__ ni,
                             const double* __restrict__ v, double* states,
                             int64_t stride, int32_t* err) {
    const int g = blockIdx.y;
    const GateD G = md->gate[g];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double m = gate_inf_d(G, v[ni[i]]);
        if (!finite_int(m)) latch_error(err, NMODL_ERR_NONFINITE);
        states[g * stride + i] = m;
    }
}

// --------------------------------------------------------------- state

template <int PREC>
__global__ void k_state_gates(const MechD* __restrict__ md, int64_t n,
                              const int32_t* __restrict__ ni,
                              const double* __restrict__ v, double* states,
                              int64_t stride, double dt, int pade, int32_t* err) {
    const int g = blockIdx.y;
    const GateD G = md->gate[g];
    const double phidt = md->phi * dt;
    double* row = states + g * stride;
    if (PREC == NMODL_FP64) {
        // folded once per block (the fold takes a log per EXP rate)
        __shared__ GateD Gs;
        if (threadIdx.x == 0) {
            Gs = G;
            fold_gate(Gs, phidt);
        }
        __syncthreads();
        const GateD Gf = Gs;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
             i += (int64_t)gridDim.x * blockDim.x) {
            const double m = pade ? gate_step_pade_d<true>(Gf, 1.0, v[ni[i]], row[i])
                                  : gate_step_fast_d<true>(Gf, 1.0, v[ni[i]], row[i]);
            if (!finite_int(m)) latch_error(err, NMODL_ERR_NONFINITE);
            row[i] = m;
        }
    } else {
        const GateF F = gate_f(G);
        const float phidtf = (float)phidt;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
             i += (int64_t)gridDim.x * blockDim.x) {
            const double m = row[i];
            float minf, f;
            gate_coef_f(F, phidtf, d2f_int(v[ni[i]]), minf, f, pade != 0);
            // FP32 increment from the FP32-rounded state, added in FP64
            // (conversions on the integer pipe)
            const float delta = f * (minf - d2f_int(m));
            const double mn = m + f2d_int(delta);
            if (!finite_int(mn)) latch_error(err, NMODL_ERR_NONFINITE);
            row[i] = mn;
        }
    }
}

// ----------------------------------------------------------------- cur

// i and g of instance j of a cnexp-family mechanism at voltage vv (FP64)
__device__ __forceinline__ void cur_cnexp_d(const MechD& M, const double* st,
                                            int64_t stride, int64_t j,
                                            double vv, double& i, double& g) {
    if (M.kind == NMODL_HH) {
        const double m = st[j], h = st[stride + j], nn = st[2 * stride + j];
        const double gna = M.hh_g[0] * m * m * m * h;
        const double gk = M.hh_g[1] * nn * nn * nn * nn;
        const double gl = M.hh_g[2];
        i = gna * (vv - M.hh_e[0]) + gk * (vv - M.hh_e[1]) + gl * (vv - M.hh_e[2]);
        g = gna + gk + gl;
    } else {
        double gg = M.gbar;
        for (int q = 0; q < M.n_gates; ++q)
            gg = mul_pow_d(gg, st[q * stride + j], M.gate[q].power);
        i = gg * (vv - M.e);
        g = gg;
    }
}

__device__ __forceinline__ void cur_kin9_d(const Kin9D& K, const double* st,
                                           int64_t stride, int64_t j, double vv,
                                           double& i, double& g) {
    g = K.gbar * st[K.open * stride + j];
    i = g * (vv - K.e);
}

__device__ __forceinline__ void cur_kin3_d(const Kin3D& K, const double* st,
                                           int64_t stride, int64_t j, double vv,
                                           double& i, double& g) {
    g = K.gbar * st[K.open * stride + j];
    i = g * (vv - K.e);
}

// i, g and the ion parts (ia, ib) of instance j: HH splits its current into
// the sodium and potassium terms; the other kinds report the whole current
template <int KIND, bool ION>
__device__ __forceinline__ void cur_any_d(const void* desc, const double* st, int64_t stride,
                                          int64_t j, double vv, double& i, double& g,
                                          double& ia, double& ib) {
    if (KIND == NMODL_KIN9) {
        cur_kin9_d(*(const Kin9D*)desc, st, stride, j, vv, i, g);
        ia = i;
        ib = 0.0;
    } else if (KIND == NMODL_KIN3) {
        cur_kin3_d(*(const Kin3D*)desc, st, stride, j, vv, i, g);
        ia = i;
        ib = 0.0;
    } else {
        const MechD& M = *(const MechD*)desc;
        if (ION && M.kind == NMODL_HH) {
            const double m = st[j], h = st[stride + j], nn = st[2 * stride + j];
            const double gna = M.hh_g[0] * m * m * m * h;
            const double gk = M.hh_g[1] * nn * nn * nn * nn;
            const double gl = M.hh_g[2];
            ia = gna * (vv - M.hh_e[0]);
            ib = gk * (vv - M.hh_e[1]);
            i = ia + ib + gl * (vv - M.hh_e[2]);
            g = gna + gk + gl;
        } else {
            cur_cnexp_d(M, st, stride, j, vv, i, g);
            ia = i;
            ib = 0.0;
        }
    }
}

// One warp per segment-aligned chunk [chunk[w], chunk[w+1]) of instances:
// chunks start at segment heads, so every node's instances are reduced by a
// single warp and each node is written by exactly one lane (deterministic,
// no atomics).  Within a 32-wide piece a segmented inclusive scan on the
// sorted keys sums each node's terms; a segment that runs past the piece is
// carried into the next piece from lane 31.  The scan stops at the first
// offset that spans the longest segment of the piece (one level for
// segments of at most 2, two for at most 4, else five; a warp vote on the
// keys decides), since its FP64 additions are the kernel's main cost.  With
// ION the ion parts of the current (USEION WRITE) go through the same scan
// into ion_a / ion_b.
template <int KIND, bool ION>
__global__ void k_cur_seg(const void* __restrict__ desc, int64_t n_chunks,
                          const int32_t* __restrict__ chunk,
                          const int32_t* __restrict__ ni,
                          const double* __restrict__ v,
                          const double* __restrict__ st, int64_t stride,
                          double* rhs, double* d, double* ion_a, double* ion_b,
                          int32_t* err) {
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (w >= n_chunks) return;
    const int64_t s = chunk[w], e = chunk[w + 1];
    double ci = 0.0, cg = 0.0, ca = 0.0, cb = 0.0;
    int ckey = INT_MIN;
    for (int64_t base = s; base < e; base += 32) {
        const int64_t j = base + lane;
        const bool valid = j < e;
        const int key = valid ? ni[j] : -1 - lane;  // invalid lanes never match
        double vi = 0.0, vg = 0.0, va = 0.0, vb = 0.0;
        if (valid) cur_any_d<KIND, ION>(desc, st, stride, j, v[key], vi, vg, va, vb);
        // the carry into lane 0 behind a warp-uniform branch: a predicated
        // FP64 add would still take an FP64 issue slot of the whole warp
        if (__shfl_sync(0xffffffffu, key, 0) == ckey && lane == 0) {
            vi += ci;
            vg += cg;
            if (ION) {
                va += ca;
                vb += cb;
            }
        }
        int span;  // the scan's last offset: 2 * span covers every segment
        {          // (0: every node of the piece has one instance, no scan)
            const int k1 = __shfl_up_sync(0xffffffffu, key, 1);
            const int k2 = __shfl_up_sync(0xffffffffu, key, 2);
            const int k4 = __shfl_up_sync(0xffffffffu, key, 4);
            span = !__any_sync(0xffffffffu, lane >= 1 && k1 == key)   ? 0
                   : !__any_sync(0xffffffffu, lane >= 2 && k2 == key) ? 1
                   : !__any_sync(0xffffffffu, lane >= 4 && k4 == key) ? 2
                                                                      : 16;
        }
        for (int off = 1; off <= span; off <<= 1) {
            const double oi = __shfl_up_sync(0xffffffffu, vi, off);
            const double og = __shfl_up_sync(0xffffffffu, vg, off);
            double oa = 0.0, ob = 0.0;
            if (ION) {
                oa = __shfl_up_sync(0xffffffffu, va, off);
                ob = __shfl_up_sync(0xffffffffu, vb, off);
            }
            const int ok = __shfl_up_sync(0xffffffffu, key, off);
            if (lane >= off && ok == key) {
                vi += oi;
                vg += og;
                if (ION) {
                    va += oa;
                    vb += ob;
                }
            }
        }
        const int nkey = __shfl_down_sync(0xffffffffu, key, 1);
        const bool cont = valid && lane == 31 && (j + 1 < e) && ni[j + 1] == key;
        const bool tail = valid && (lane == 31 || nkey != key);
        if (tail && !cont) {
            const double r = rhs[key] - vi;
            const double dd = d[key] + vg;
            if (!finite_int(r) || !finite_int(dd)) latch_error(err, NMODL_ERR_NONFINITE);
            rhs[key] = r;
            d[key] = dd;
            if (ION) {
                if (ion_a) ion_a[key] += va;
                if (ion_b) ion_b[key] += vb;
            }
        }
        ci = __shfl_sync(0xffffffffu, vi, 31);
        cg = __shfl_sync(0xffffffffu, vg, 31);
        if (ION) {
            ca = __shfl_sync(0xffffffffu, va, 31);
            cb = __shfl_sync(0xffffffffu, vb, 31);
        }
        ckey = __shfl_sync(0xffffffffu, cont ? key : INT_MIN, 31);
    }
}

// ---------------------------------------------------- fused tile kernel

// first j in [0, n) with a[j] >= key (a sorted non-decreasing)
__device__ __forceinline__ int lower_bound_u16(const uint16_t* a, int n, int key) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// In-place inclusive prefix sum of a[0, n) in shared memory (the total fits
// uint16).  Each thread sums a contiguous chunk; the chunk sums are scanned
// with warp shuffles and one warp over the per-warp totals (wsum: 32 ints
// of shared memory).  Block size a multiple of 32; called by every thread.
__device__ void block_inclusive_scan_u16(uint16_t* a, int n, int* wsum) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int per = (n + nt - 1) / nt;
    const int b0 = min(n, tid * per), b1 = min(n, b0 + per);
    int s = 0;
    for (int k = b0; k < b1; ++k) s += a[k];
    const int lane = tid & 31, w = tid >> 5;
    int inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int nw = nt >> 5;
        int x = lane < nw ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane < nw) wsum[lane] = x;
    }
    __syncthreads();
    int run = (w ? wsum[w - 1] : 0) + inc - s;
    for (int k = b0; k < b1; ++k) {
        run += a[k];
        a[k] = (uint16_t)run;
    }
    __syncthreads();
}

// Shared-memory layout of one tile (built from the tile record):
//   double  v_s[NT]
//   state   st_s[sum_t gates_t * cnt_t]   (double, or float2 hi/lo in MIXED)
//   uint16  nid_s[sum_t cnt_t]            local node id of each instance
//   tables: uint16 seg_s[T][NT + 1]       per-type segment offsets
//   flat:   uint16 pos_s[sum_t cnt_t]     node-major slot of each instance
//           uint16 eoff_s[NT + 1]         slot range of each node
//           uint16 perm_s[NT]             owner order (by slot count)
//   float   vf_s[NT]                      (MIXED) float copy of v, 16-aligned
//   double  ica_s[NT]                     (EXT with ions) the step's ica
//   double  d2_s[NT], r2_s[NT], ga_s[NT], gb_s[NT]   (cable), 16-aligned
//   uint16  par_s[NT]                     (cable) local parent, 0xffff at roots
//   uint16  sched_s[...]                  (cable) level schedule of the solve
//   flat:   double2 xg_s[slots]           node-major (e, g) of each current
//           (HH three per instance); 16-aligned after the above
// "flat" is the layout on isolated compartments: one sum over contiguous
// slots per node, owners ordered by slot count.  The cable form keeps the
// per-type tables and computes each instance's conductance in its owner
// loop (tiles hold whole cells; the smaller footprint means fewer tiles,
// hence fewer tree solves, and lets the largest cells fit tiles small
// enough for two blocks per SM).
// Tile record (int32): n0, n1, then a_t, b_t per type (instance ranges).
// The host plan guarantees NT <= 65535, cnt_t <= 65535 (flat: the sum of
// cnt_t too) and that the layout fits the dynamic shared memory of the
// launch.
//
// Cable form: tiles hold whole cells.  After the current phase each node
// adds its own and its children's axial terms (in parallel).  The tree
// system is then solved by one warp in levels: nodes of equal height above
// the leaves are eliminated together (each gathers its children's
// eliminated rows, in a fixed order, and keeps 1/d' and r'/d'), then nodes
// of equal depth below the root are substituted together -- Hines'
// elimination (1984; no fill because parents precede children) scheduled by
// levels.  v += the solution.  On the last step of the window rhs and d
// report the assembled system.
// The KIN variant (the 9-state scheme) has two builds.  KIN == 1: blocks of
// at most 256 threads, the banded solve in registers (~245 in FP64, one
// block per SM; MIXED two blocks per SM at 128 registers, the FP32 solve
// spilling a few hundred bytes) -- best for lists of the 9-state scheme
// alone.  KIN == 2, the wide build: one block per SM, FP64 768 threads at
// 80 registers, MIXED 512 at 128, the solve keeping part of its state in
// local memory (about 1 KB per thread), so that cnexp items of the same
// tile run at more warps per SM (24 or 16 instead of 8).  Measured on the
// cortical mix with the 9-state scheme on a quarter of 1M nodes (in the
// fixed work order), FP64 instance-steps/s by block (registers): 256 (244)
// 7.07e9, 384 (168) 7.66e9, 512 (128) 8.13e9, 768 (80) 8.53e9, 1024 (64)
// 8.49e9; MIXED: 2 x 256 (128) 1.91e10, 512 (80) 2.03e10, 768 (80)
// 2.05e10, 1024 (64) 1.92e10; with the work chunks below, MIXED 512 at 128
// registers 2.59e10 against 2.41e10 for the register-rich build.  On the
// 9-state scheme alone (1M clamped instances, FP64) the wide build loses
// (it and the per-mechanism launches 1.07e9 vs 1.15e9).  The autotuner
// times block sizes of both builds.
template <int PREC, bool EXT, int KIN>
__global__ void __launch_bounds__(KIN == 0 ? kFusedMaxBlock
                                  : KIN == 1 ? kFusedKinBlock
                                             : fused_kin_wide_block(PREC),
                                  (KIN == 1 && PREC == NMODL_MIXED) ? 2 : 1)
    k_fused_tiles(FusedArgs A) {
    static_assert(!KIN || EXT, "the 9-state scheme comes with the extended variant");
    // MIXED on isolated compartments: each gate update writes its
    // instance's conductance factor into the instance's node-major slot
    // (gbar m^p for a type's first gate, h^q for the next ones; HH: gnabar
    // m^3 and h into the sodium slot, gkbar n^4 into the potassium slot; a
    // 3-state instance gbar x_open after its solve), the slot's fourth float
    // holds the id of its current (its reversal potential in efac_s), and
    // the owner pass multiplies the factors: no separate conductance pass,
    // two barriers per step, not three.  Not in the variant with the 9-state
    // scheme, whose 128-register bound the extra code pushed into more
    // spills (measured 0.92x there; 1.16x on the cnexp networks, 1.06x with
    // ion arrays and the small systems).
    constexpr bool FAC_V = PREC == NMODL_MIXED && !KIN;
    // MIXED with the 9-state scheme: the (e, g) slots hold both as float
    // pairs (e in the first 8 bytes, g in the second), summed as float
    // pairs by the owner
    constexpr bool XGF = PREC == NMODL_MIXED && KIN;
    __shared__ double efac_s[FAC_V ? 3 * kMaxMechsFused : 1];   // e of current 3 t + q
    __shared__ float2 efac2_s[FAC_V ? 3 * kMaxMechsFused : 1];  // the same as float pairs
    __shared__ float fmul_s[FAC_V ? kMaxMechsFused * kMaxGates : 1];
    __shared__ int fidx_s[FAC_V ? kMaxMechsFused * kMaxGates : 1];  // 4 slot + component
    __shared__ int fpow_s[FAC_V ? kMaxMechsFused * kMaxGates : 1];
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ MechD md_s[kMaxMechsFused];
    __shared__ GateF gf_s[kMaxMechsFused][kMaxGates];
    __shared__ int a_s[kMaxMechsFused], cnt_s[kMaxMechsFused];
    __shared__ int st_off[kMaxMechsFused], nid_off[kMaxMechsFused];
    __shared__ int pair_t[kMaxMechsFused * kMaxGates];
    __shared__ int pair_g[kMaxMechsFused * kMaxGates];
    __shared__ int pair_start[kMaxMechsFused * kMaxGates + 1];
    __shared__ int n_pairs;
    // work order of the state phase (see below): pair of each work slot and
    // its first work index
    __shared__ int wq_s[kMaxMechsFused * kMaxGates];
    __shared__ int wstart_s[kMaxMechsFused * kMaxGates + 1];
    __shared__ int wkey[kMaxMechsFused * kMaxGates];
    __shared__ int n_work;
    __shared__ int wctr_s;  // KIN: the next work slot of the state phase
    __shared__ float phidt_f[kMaxMechsFused];
    // MIXED: FP32 copies of the current parameters (gbar, e, HH g[3], e[3]),
    // converted once rather than per instance (FP64 -> FP32 conversions run
    // on the FP64 pipe)
    __shared__ float curf_s[kMaxMechsFused][8];
    // MIXED with the small systems: their parameters in FP32
    __shared__ Kin3F k3f_s[EXT ? kMaxMechsFused : 1];
    __shared__ CacumF cdf_s[EXT ? kMaxMechsFused : 1];
    // the 9-state scheme's rate constants folded with this launch's dt:
    // FP64 dt k = exp(b v + ln(dt a)) with ln(dt a) in place of a; MIXED the
    // FP32 b_f, b_b, ln(dt a_f), ln(dt a_b)
    __shared__ Kin9D k9_s[KIN ? kMaxMechsFused : 1];
    // per-block Newton / refinement counts of the coupled systems, added to
    // the mechanisms' counters once at the end
    __shared__ unsigned long long kit_s[EXT ? kMaxMechsFused : 1], knc_s[EXT ? kMaxMechsFused : 1];
    __shared__ int kmx_s[EXT ? kMaxMechsFused : 1];
    __shared__ float k9f_s[(KIN && PREC == NMODL_MIXED) ? kMaxMechsFused : 1][4 * kKinEdges];

    __shared__ int tile_s;
    __shared__ int inst_start[kMaxMechsFused + 1];  // instance offset of each type
    __shared__ int scan_s[32];                      // per-warp sums of the block scan
    __shared__ int n_slots_s;                       // node-major slots of the tile (flat)
    __shared__ int hist_s[64];                      // owner-order counting sort

    const int tid = threadIdx.x;
    const int T = A.n_types;
    for (int k = tid; k < T * (int)(sizeof(MechD) / 4); k += blockDim.x)
        ((int32_t*)md_s)[k] = ((const int32_t*)A.md)[k];
    if constexpr (EXT)
        if (tid < T) {
            kit_s[tid] = 0;
            knc_s[tid] = 0;
            kmx_s[tid] = 0;
        }
    // counts of one solve of type t: summed over the lanes of the warp that
    // solve the same type, then one shared atomic per warp and type (flushed
    // to the mechanisms' counters at the end)
    auto count_solve = [&](int t, int iters, bool failed) {
        if constexpr (EXT) {
            const unsigned same = __match_any_sync(__activemask(), t);
            const unsigned sum = __reduce_add_sync(same, (unsigned)iters);
            const unsigned nf = __reduce_add_sync(same, failed ? 1u : 0u);
            const unsigned mx = __reduce_max_sync(same, (unsigned)iters);
            if ((int)(threadIdx.x & 31) == __ffs(same) - 1) {
                atomicAdd(&kit_s[t], (unsigned long long)sum);
                if (nf) atomicAdd(&knc_s[t], (unsigned long long)nf);
                atomicMax(&kmx_s[t], (int)mx);
            }
        }
    };
    if constexpr (KIN)
        for (int k = tid; k < T * (int)(sizeof(Kin9D) / 4); k += blockDim.x)
            ((int32_t*)k9_s)[k] = ((const int32_t*)A.k9d)[k];
    if constexpr (PREC == NMODL_FP64) {
        // gate parameters folded for this launch (u by one multiply-add,
        // rates carrying phi dt); ordered by the first barrier of the loop
        __syncthreads();
        for (int k = tid; k < T * kMaxGates; k += blockDim.x) {
            MechD& M = md_s[k / kMaxGates];
            if (M.kind != NMODL_KIN9 && k % kMaxGates < M.n_gates)
                fold_gate(M.gate[k % kMaxGates], M.phi * A.dt);
        }
    }
    if constexpr (KIN) {
        __syncthreads();
        for (int k = tid; k < T * kKinEdges; k += blockDim.x) {
            const int t = k / kKinEdges, e = k % kKinEdges;
            if (md_s[t].kind != NMODL_KIN9) continue;
            Kin9D& K = k9_s[t];
            const double lf = log(A.dt * K.af[e]), lb = log(A.dt * K.ab[e]);
            if constexpr (PREC == NMODL_MIXED) {
                // scaled by log2(e) for the exp2 unit
                k9f_s[t][e] = (float)(K.bf[e] * 1.4426950408889634);
                k9f_s[t][kKinEdges + e] = (float)(K.bb[e] * 1.4426950408889634);
                k9f_s[t][2 * kKinEdges + e] = (float)(lf * 1.4426950408889634);
                k9f_s[t][3 * kKinEdges + e] = (float)(lb * 1.4426950408889634);
            } else {
                K.af[e] = lf;
                K.ab[e] = lb;
            }
        }
    }

    // Tiles come from the work list in order (largest first): either one
    // per block, or -- persistent form -- pulled from an atomic counter by
    // resident blocks until the list is exhausted.
    for (int round = 0;; ++round) {
    if (tid == 0) {
        if (A.tile_counter) tile_s = atomicAdd(A.tile_counter, 1);
        else tile_s = round == 0 ? (int)blockIdx.x : A.n_tiles;
    }
    __syncthreads();
    const int tile = tile_s;
    if (tile >= A.n_tiles) break;
    const int32_t* rec = A.tiles + (int64_t)tile * A.tile_stride;
    const int n0 = rec[0];
    const int NT = rec[1] - rec[0];

    if (tid == 0) {
        int so = 0, no = 0, q = 0;
        for (int t = 0; t < T; ++t) {
            a_s[t] = rec[2 + 2 * t];
            cnt_s[t] = rec[3 + 2 * t] - rec[2 + 2 * t];
            st_off[t] = so;
            nid_off[t] = no;
            const int ng = A.n_gates[t];
            for (int g = 0; g < ng; ++g) {
                pair_t[q] = t;
                pair_g[q] = g;
                pair_start[q] = so + g * cnt_s[t];
                ++q;
            }
            so += ng * cnt_s[t];
            no += cnt_s[t];
        }
        pair_start[q] = so;
        n_pairs = q;
        if (FAC_V) {  // the factor of each gate pair; the e of each current
            for (int p = 0; p < q; ++p) {
                const MechD& M = md_s[pair_t[p]];
                const int g = pair_g[p];
                const bool hh = M.kind == NMODL_HH;
                if (M.kind != NMODL_HH && M.kind != NMODL_CNEXP) {
                    // a coupled system: its open state's factor gbar x_open
                    // is written by the system's own update (power -1 here);
                    // gbar and the open row serve the window's first factors
                    const bool k3 = EXT && M.kind == NMODL_KIN3;
                    const int open = k3 ? M.k3.open : M.open;
                    fmul_s[p] = (float)(k3 ? M.k3.gbar : M.gbar);
                    fpow_s[p] = (M.kind == NMODL_CACUM || g != open) ? -2 : -1;
                    fidx_s[p] = 0;
                    continue;
                }
                fmul_s[p] = g == 0 ? (float)(hh ? M.hh_g[0] : M.gbar)
                                   : (hh && g == 2) ? (float)M.hh_g[1] : 1.f;
                fpow_s[p] = M.gate[g].power;
                fidx_s[p] = hh ? (g == 2 ? 4 : g) : g;
            }
            for (int t = 0; t < T; ++t)
                for (int c = 0; c < 3; ++c)
                    efac_s[3 * t + c] = md_s[t].kind == NMODL_HH     ? md_s[t].hh_e[c]
                                        : (EXT && md_s[t].kind == NMODL_KIN3) ? md_s[t].k3.e
                                                                        : md_s[t].e;
            for (int k = 0; k < 3 * T; ++k) {
                const float h = d2f_int(efac_s[k]);
                efac2_s[k] = make_float2(h, d2f_int(efac_s[k] - f2d_int(h)));
            }
        }
        // Work order of the FP64 state phase: the gates grouped by their pair
        // of rate forms (each pair of forms is one straight-line body), each
        // group padded to whole warps so that no warp runs two bodies; the
        // coupled systems one item per instance: the 9-state solve (about 13
        // gate updates' worth) first, since with it the warps take the work
        // in chunks as they come free, the 3-state solve and the buffer's
        // Newton last.  (MIXED, whose FP32 bodies are cheap and
        // issue-bound, keeps the storage order unless the 9-state scheme
        // is in the list.)
        int nw = 0;
        for (int p = 0; p < q; ++p) {
            const int t = pair_t[p], g = pair_g[p], kind = md_s[t].kind;
            int key;
            if (EXT && (kind == NMODL_KIN3 || kind == NMODL_CACUM || (KIN && kind == NMODL_KIN9))) {
                if (g != 0) continue;
                key = kind == NMODL_KIN3 ? 9 : kind == NMODL_CACUM ? 10 : -1;
            } else {
                key = md_s[t].gate[g].aform * 3 + md_s[t].gate[g].bform;
            }
            int i = nw++;  // insertion, stable in storage order
            while (i > 0 && wkey[i - 1] > key) {
                wkey[i] = wkey[i - 1];
                wq_s[i] = wq_s[i - 1];
                --i;
            }
            wkey[i] = key;
            wq_s[i] = p;
        }
        int w = 0;
        for (int i = 0; i < nw; ++i) {
            wstart_s[i] = w;
            w += cnt_s[pair_t[wq_s[i]]];
            if (i + 1 == nw || wkey[i + 1] != wkey[i]) w = (w + 31) & ~31;
        }
        wstart_s[nw] = w;
        n_work = nw;
        for (int t = 0; t < T; ++t) inst_start[t] = nid_off[t];
        inst_start[T] = no;
        int ns = 0;
        for (int t = 0; t < T; ++t) ns += flat_slots(md_s[t].kind) * cnt_s[t];
        n_slots_s = ns;
    }
    __syncthreads();
    if (PREC == NMODL_MIXED) {
        for (int k = tid; k < T; k += blockDim.x) {
            const MechD& M = md_s[k];
            phidt_f[k] = (float)(M.phi * A.dt);
            curf_s[k][0] = (float)((EXT && M.kind == NMODL_KIN3) ? M.k3.gbar : M.gbar);
            curf_s[k][1] = (float)M.e;
            for (int q = 0; q < 3; ++q) {
                curf_s[k][2 + q] = (float)M.hh_g[q];
                curf_s[k][5 + q] = (float)M.hh_e[q];
            }
        }
        if (EXT)
            for (int k = tid; k < T; k += blockDim.x) {
                const MechD& M = md_s[k];
                if (M.kind == NMODL_KIN3) {
                    for (int e = 0; e < 3; ++e) {
                        k3f_s[k].af[e] = (float)M.k3.af[e];
                        k3f_s[k].bf[e] = (float)(M.k3.bf[e] * 1.4426950408889634);  // log2(e)
                        k3f_s[k].ab[e] = (float)M.k3.ab[e];
                        k3f_s[k].bb[e] = (float)(M.k3.bb[e] * 1.4426950408889634);
                    }
                } else if (M.kind == NMODL_CACUM) {
                    const CacumD& C = M.cd;
                    cdf_s[k] = CacumF{(float)C.k, (float)C.rtau, (float)C.cai0, (float)C.kf,
                                      (float)C.kb, (float)C.btot};
                }
            }
        for (int k = tid; k < T * kMaxGates; k += blockDim.x) {
            const GateD& G = md_s[k / kMaxGates].gate[k % kMaxGates];
            gf_s[k / kMaxGates][k % kMaxGates] = gate_f(G);
        }
    }
    const int total_items = pair_start[n_pairs];
    int total_inst = 0;
    for (int t = 0; t < T; ++t) total_inst += cnt_s[t];

    double* v_s = reinterpret_cast<double*>(smem);
    double* st_d = v_s + NT;                                   // FP64 states
    float2* st_f = reinterpret_cast<float2*>(v_s + NT);        // MIXED states
    uint16_t* nid_s = reinterpret_cast<uint16_t*>(st_d + total_items);
    // Per-type tables (the cable form): the segment offsets of each node.
    // Flat (isolated compartments): the node-major slot of each instance, the
    // slot range of each node, the owner order, and (with ion arrays) the ion
    // of each slot.
    const bool flat = !A.cable;
    const bool FAC = FAC_V && flat;
    uint16_t* seg_s = nid_s + total_inst;
    uint16_t* pos_s = nid_s + total_inst;
    uint16_t* eoff_s = pos_s + total_inst;
    uint16_t* perm_s = eoff_s + NT + 1;
    uint8_t* tag_s = reinterpret_cast<uint8_t*>(perm_s + NT);
    void* idx_end = flat ? ((EXT && A.ions) ? (void*)(tag_s + n_slots_s) : (void*)(perm_s + NT))
                         : (void*)(seg_s + T * (NT + 1));
    // MIXED: a float copy of v per node follows at the next 16-byte boundary
    float* vf_s = reinterpret_cast<float*>(
        (reinterpret_cast<uintptr_t>(idx_end) + 15) & ~(uintptr_t)15);
    // ions: the step's ica per node; cable: the tree system -- each at the
    // next 16-byte boundary after the above
    uintptr_t end_p = reinterpret_cast<uintptr_t>(
        PREC == NMODL_MIXED ? (void*)(vf_s + NT) : idx_end);
    double* ica_s = reinterpret_cast<double*>((end_p + 15) & ~(uintptr_t)15);
    if (EXT && A.ions) end_p = reinterpret_cast<uintptr_t>(ica_s + NT);
    double* d2_s = reinterpret_cast<double*>((end_p + 15) & ~(uintptr_t)15);
    double* r2_s = d2_s + NT;
    double* ga_s = r2_s + NT;
    double* gb_s = ga_s + NT;
    uint16_t* par_s = reinterpret_cast<uint16_t*>(gb_s + NT);
    uint16_t* sched_s = par_s + NT;
    // Flat: the (e, g) node-major slots of the step (the cable form has none).
    // FAC (MIXED without the small systems): the factors and current id f_s
    // instead, at the same place
    double2* xg_s = reinterpret_cast<double2*>(
        (reinterpret_cast<uintptr_t>(d2_s) + 15) & ~(uintptr_t)15);
    float4* f_s = reinterpret_cast<float4*>(xg_s);
    if (A.cable) {
        const int32_t off = rec[2 + 2 * T], len = rec[3 + 2 * T];
        for (int k = tid; k < len; k += blockDim.x) sched_s[k] = A.sched[off + k];
    }
    // FAC: the conductance factor of gate pair q, instance j, from the gate's
    // FP32 state hi, into its component of the instance's slot
    auto put_factor = [&](int q, int j, float hi) {
        float f = fmul_s[q];
        const int pw = fpow_s[q];
        if (pw < 0) return;  // a coupled system's row
        if (pw >= 1) f *= hi;
        if (pw >= 2) f *= hi;
        if (pw >= 3) f *= hi;
        for (int k = 3; k < pw; ++k) f *= hi;
        reinterpret_cast<float*>(f_s)[4 * pos_s[nid_off[pair_t[q]] + j] + fidx_s[q]] = f;
    };

    // ---- load the tile
    for (int k = tid; k < NT; k += blockDim.x) {
        const double vv = A.v[n0 + k];
        v_s[k] = vv;
        if (PREC == NMODL_MIXED) vf_s[k] = d2f_int(vv);
        if (A.cable) {
            const int pp = A.parent[n0 + k];
            par_s[k] = pp < 0 ? (uint16_t)0xffffu : (uint16_t)(pp - n0);
            ga_s[k] = A.ga[n0 + k];
            gb_s[k] = A.gb[n0 + k];
        }
    }
    {
        int q = 0;
        for (int k = tid; k < total_items; k += blockDim.x) {
            while (k >= pair_start[q + 1]) ++q;
            const int t = pair_t[q], g = pair_g[q];
            const int j = k - pair_start[q];
            const double m = A.states[t][g * A.stride[t] + a_s[t] + j];
            if (PREC == NMODL_FP64) {
                st_d[k] = m;
            } else {
                const float hi = d2f_int(m);
                st_f[k] = make_float2(hi, d2f_int(m - f2d_int(hi)));
            }
        }
    }
    for (int t = 0; t < T; ++t)
        for (int j = tid; j < cnt_s[t]; j += blockDim.x)
            nid_s[nid_off[t] + j] = (uint16_t)(A.ni[t][a_s[t] + j] - n0);
    __syncthreads();
    if (!flat) {
        for (int t = 0; t < T; ++t) {
            const uint16_t* nid = nid_s + nid_off[t];
            uint16_t* seg = seg_s + t * (NT + 1);
            const int cnt = cnt_s[t];
            for (int n = tid; n <= NT; n += blockDim.x) seg[n] = (uint16_t)lower_bound_u16(nid, cnt, n);
        }
        __syncthreads();
    } else {
        // Node-major slots: node n owns slots [eoff[n], eoff[n+1]), its
        // instances in mechanism order, then ascending instance -- with ion
        // arrays the calcium-tagged currents after all others, so that the
        // owner sums them in a loop of their own; one slot (e, g) per
        // current (HH: three), e written here once per window.
        for (int n = tid; n < NT; n += blockDim.x) {
            int c = 0;
            for (int t = 0; t < T; ++t) {
                const uint16_t* nid = nid_s + nid_off[t];
                c += flat_slots(md_s[t].kind) *
                     (lower_bound_u16(nid, cnt_s[t], n + 1) - lower_bound_u16(nid, cnt_s[t], n));
            }
            eoff_s[n + 1] = (uint16_t)c;
        }
        if (tid == 0) eoff_s[0] = 0;
        __syncthreads();
        block_inclusive_scan_u16(eoff_s + 1, NT, scan_s);
        for (int n = tid; n < NT; n += blockDim.x) {
            int o = eoff_s[n];
            const int passes = (EXT && A.ions) ? 2 : 1;
            for (int pass = 0; pass < passes; ++pass)
            for (int t = 0; t < T; ++t) {
                const MechD& M = md_s[t];
                if (EXT && A.ions &&
                    (pass == 1) != (M.kind != NMODL_HH && M.ion == NMODL_ION_CA))
                    continue;
                const uint16_t* nid = nid_s + nid_off[t];
                const int hi = lower_bound_u16(nid, cnt_s[t], n + 1);
                for (int j = lower_bound_u16(nid, cnt_s[t], n); j < hi; ++j) {
                    pos_s[nid_off[t] + j] = (uint16_t)o;
                    if (FAC) {
                        // factors 1 except the constant conductances (the
                        // HH leak; a cnexp type without gates); the gate
                        // items and the systems' updates fill in the rest
                        if (M.kind == NMODL_HH) {
                            for (int q = 0; q < 3; ++q) {
                                f_s[o + q] = make_float4(q == 2 ? curf_s[t][4] : 1.f, 1.f, 1.f,
                                                         __int_as_float(3 * t + q));
                                if (EXT && A.ions)
                                    tag_s[o + q] = q == 0 ? NMODL_ION_NA : q == 1 ? NMODL_ION_K : NMODL_ION_NONE;
                            }
                            o += 3;
                        } else if (!EXT || M.kind != NMODL_CACUM) {
                            const bool konst = M.kind == NMODL_CNEXP && M.n_gates == 0;
                            f_s[o] = make_float4(konst ? curf_s[t][0] : 1.f, 1.f, 1.f,
                                                 __int_as_float(3 * t));
                            if (EXT && A.ions) tag_s[o] = (uint8_t)M.ion;
                            ++o;
                        }
                    } else if (M.kind == NMODL_HH) {
                        for (int q = 0; q < 3; ++q) {
                            if (XGF) {
                                const ff2 ep = ff_of(M.hh_e[q]);
                                reinterpret_cast<float2*>(xg_s)[2 * (o + q)] = make_float2(ep.h, ep.l);
                            } else {
                                xg_s[o + q].x = M.hh_e[q];
                            }
                            if (EXT && A.ions)
                                tag_s[o + q] = q == 0 ? NMODL_ION_NA : q == 1 ? NMODL_ION_K : NMODL_ION_NONE;
                        }
                        o += 3;
                    } else if (!EXT || M.kind != NMODL_CACUM) {
                        const double e = (EXT && M.kind == NMODL_KIN3) ? M.k3.e : M.e;
                        if (XGF) {
                            const ff2 ep = ff_of(e);
                            reinterpret_cast<float2*>(xg_s)[2 * o] = make_float2(ep.h, ep.l);
                        } else {
                            xg_s[o].x = e;
                        }
                        if (EXT && A.ions) tag_s[o] = (uint8_t)M.ion;
                        ++o;
                    }
                }
            }
        }
        // Owner order: nodes by decreasing slot count (counting sort on
        // min(count, 63)), so that the lanes of a warp run sums of similar
        // length.  Which thread owns a node does not change its result, so
        // the order within a count is free.
        for (int k = tid; k < 64; k += blockDim.x) hist_s[k] = 0;
        __syncthreads();
        for (int n = tid; n < NT; n += blockDim.x)
            atomicAdd(&hist_s[63 - min(eoff_s[n + 1] - eoff_s[n], 63)], 1);
        __syncthreads();
        if (tid == 0) {
            int acc = 0;
            for (int k = 0; k < 64; ++k) {
                const int h = hist_s[k];
                hist_s[k] = acc;
                acc += h;
            }
        }
        __syncthreads();
        for (int n = tid; n < NT; n += blockDim.x)
            perm_s[atomicAdd(&hist_s[63 - min(eoff_s[n + 1] - eoff_s[n], 63)], 1)] = (uint16_t)n;
        __syncthreads();
    }

    // FAC: a coupled system's factor gbar x_open into its slot
    auto put_open_factor = [&](int t, int j, float fmul, float x_open) {
        reinterpret_cast<float*>(f_s)[4 * pos_s[nid_off[t] + j]] = fmul * x_open;
    };
    if (FAC) {  // the factors of the loaded states
        int q = 0;
        for (int k = tid; k < total_items; k += blockDim.x) {
            while (k >= pair_start[q + 1]) ++q;
            const int j = k - pair_start[q];
            if (fpow_s[q] == -1) put_open_factor(pair_t[q], j, fmul_s[q], st_f[k].x);
            else put_factor(q, j, st_f[k].x);
        }
        __syncthreads();
    }

    // cable: the level schedule [H, D, EL, SL, E, S, coff, clist] of the tile
    // (offsets recomputed where used, to keep registers free)
    auto sched_coff = [&]() { return sched_s + 2 + (sched_s[0] + 1) + (sched_s[1] + 1) + 2 * NT; };
    const double cmdt = 1e-3 * A.cm / A.dt;
    // the same as a float pair (the mixed node update below)
    const float cmdt_h = d2f_int(cmdt), cmdt_l = d2f_int(cmdt - f2d_int(cmdt_h));
    // conductance(s) of instance j of type q from its states (HH: gna, gk;
    // not for the calcium buffer)
    auto inst_g = [&](int q, int j, double& g0, double& g1) {
        const MechD& M = md_s[q];
        const int cnt = cnt_s[q];
        g1 = 0.0;
        if constexpr (PREC == NMODL_FP64) {
            const double* st = st_d + st_off[q];
            if (M.kind == NMODL_HH) {
                const double m = st[j], h = st[cnt + j], nn = st[2 * cnt + j];
                g0 = M.hh_g[0] * m * m * m * h;
                g1 = M.hh_g[1] * nn * nn * nn * nn;
            } else if (EXT && M.kind == NMODL_KIN3) {
                g0 = M.k3.gbar * st[M.k3.open * cnt + j];
            } else if (KIN && M.kind == NMODL_KIN9) {
                g0 = M.gbar * st[M.open * cnt + j];
            } else {
                double gg = M.gbar;
                for (int gi = 0; gi < M.n_gates; ++gi)
                    gg = mul_pow_d(gg, st[gi * cnt + j], M.gate[gi].power);
                g0 = gg;
            }
        } else {
            const float2* st = st_f + st_off[q];
            const float* cf_p = curf_s[q];
            if (M.kind == NMODL_HH) {
                const float m = st[j].x, h = st[cnt + j].x, nn = st[2 * cnt + j].x;
                g0 = f2d_int(cf_p[2] * m * m * m * h);
                g1 = f2d_int(cf_p[3] * nn * nn * nn * nn);
            } else if (EXT && M.kind == NMODL_KIN3) {
                const float2 x = st[M.k3.open * cnt + j];
                g0 = M.k3.gbar * (f2d_int(x.x) + f2d_int(x.y));
            } else if (KIN && M.kind == NMODL_KIN9) {
                const float2 x = st[M.open * cnt + j];
                g0 = M.gbar * (f2d_int(x.x) + f2d_int(x.y));
            } else {
                float gf = cf_p[0];
                for (int gi = 0; gi < M.n_gates; ++gi) {
                    const float xs = st[gi * cnt + j].x;
                    for (int pw = 0; pw < M.gate[gi].power; ++pw) gf *= xs;
                }
                g0 = f2d_int(gf);
            }
        }
    };
    for (int step = 0; step < A.nsteps; ++step) {
        const bool last = (step == A.nsteps - 1);
        if (flat && !FAC) {
            // ---- conductances, one thread per instance (lane-efficient;
            // the owner loop below then spends two operations per instance).
            // MIXED: from the FP32 hi parts of the states, converted once.
            // (The cable form computes them in its owner loop instead: its
            // tiles of whole cells must stay small.)
            int q = 0;
            for (int k = tid; k < inst_start[T]; k += blockDim.x) {
                while (k >= inst_start[q + 1]) ++q;
                const int j = k - inst_start[q];
                const MechD& M = md_s[q];
                const int cnt = cnt_s[q];
                if (flat) {
                    // Flat: each current's g next to its e in the instance's
                    // node-major slots (the node forms sum(g e) - v sum(g)).
                    const int sl = pos_s[k];
                    if (EXT && M.kind == NMODL_CACUM) continue;  // no membrane current
                    if constexpr (PREC == NMODL_FP64) {
                        const double* st = st_d + st_off[q];
                        if (M.kind == NMODL_HH) {
                            const double m = st[j], h = st[cnt + j], nn = st[2 * cnt + j];
                            xg_s[sl].y = M.hh_g[0] * m * m * m * h;
                            xg_s[sl + 1].y = M.hh_g[1] * nn * nn * nn * nn;
                            xg_s[sl + 2].y = M.hh_g[2];
                        } else if (EXT && M.kind == NMODL_KIN3) {
                            xg_s[sl].y = M.k3.gbar * st[M.k3.open * cnt + j];
                        } else if (KIN && M.kind == NMODL_KIN9) {
                            xg_s[sl].y = M.gbar * st[M.open * cnt + j];
                        } else {
                            double gg = M.gbar;
                            for (int gi = 0; gi < M.n_gates; ++gi)
                                gg = mul_pow_d(gg, st[gi * cnt + j], M.gate[gi].power);
                            xg_s[sl].y = gg;
                        }
                    } else if constexpr (XGF) {
                        // g as a float pair beside e's (no FP64 instructions)
                        const float2* st = st_f + st_off[q];
                        const float* cf_p = curf_s[q];
                        float2* gp = reinterpret_cast<float2*>(xg_s) + 1;
                        if (M.kind == NMODL_HH) {
                            const float m = st[j].x, h = st[cnt + j].x, nn = st[2 * cnt + j].x;
                            const ff2 gl = ff_of(M.hh_g[2]);
                            gp[2 * sl] = make_float2(cf_p[2] * m * m * m * h, 0.f);
                            gp[2 * (sl + 1)] = make_float2(cf_p[3] * nn * nn * nn * nn, 0.f);
                            gp[2 * (sl + 2)] = make_float2(gl.h, gl.l);
                        } else if (M.kind == NMODL_KIN3 || M.kind == NMODL_KIN9) {
                            const bool k3 = M.kind == NMODL_KIN3;
                            const float2 x = st[(k3 ? M.k3.open : M.open) * cnt + j];
                            const ff2 g = ff_mul(ff_of(k3 ? M.k3.gbar : M.gbar), ff2{x.x, x.y});
                            gp[2 * sl] = make_float2(g.h, g.l);
                        } else {
                            float gf = cf_p[0];
                            for (int gi = 0; gi < M.n_gates; ++gi) {
                                const float xs = st[gi * cnt + j].x;
                                for (int pw = 0; pw < M.gate[gi].power; ++pw) gf *= xs;
                            }
                            gp[2 * sl] = make_float2(gf, 0.f);
                        }
                    } else {
                        const float2* st = st_f + st_off[q];
                        const float* cf_p = curf_s[q];
                        if (M.kind == NMODL_HH) {
                            const float m = st[j].x, h = st[cnt + j].x, nn = st[2 * cnt + j].x;
                            xg_s[sl].y = f2d_int(cf_p[2] * m * m * m * h);
                            xg_s[sl + 1].y = f2d_int(cf_p[3] * nn * nn * nn * nn);
                            xg_s[sl + 2].y = M.hh_g[2];
                        } else if (EXT && M.kind == NMODL_KIN3) {
                            const float2 x = st[M.k3.open * cnt + j];
                            xg_s[sl].y = M.k3.gbar * (f2d_int(x.x) + f2d_int(x.y));
                        } else if (KIN && M.kind == NMODL_KIN9) {
                            const float2 x = st[M.open * cnt + j];
                            xg_s[sl].y = M.gbar * (f2d_int(x.x) + f2d_int(x.y));
                        } else {
                            float gf = cf_p[0];
                            for (int gi = 0; gi < M.n_gates; ++gi) {
                                const float xs = st[gi * cnt + j].x;
                                for (int pw = 0; pw < M.gate[gi].power; ++pw) gf *= xs;
                            }
                            xg_s[sl].y = f2d_int(gf);
                        }
                    }
                }
            }
            __syncthreads();
        }
        // ---- current update and v update, one owner thread per node; the
        // terms are summed in mechanism order, then ascending instance (with
        // ion arrays the calcium-tagged currents apart, added last).
        for (int p = tid; p < NT; p += blockDim.x) {
            const int n = flat ? (int)perm_s[p] : p;
            const double vv = v_s[n];
            double r = 0.0, dd = 0.0;
            double s_na = 0.0, s_k = 0.0, s_ca = 0.0;  // ion sums (ions)
            if (flat) {
                double X = 0.0, G = 0.0, Xca = 0.0, Gca = 0.0;
                const int s0 = eoff_s[n], s1 = eoff_s[n + 1];
                // a slot's conductance and reversal potential: (e, g), or
                // (FAC) the product of its FP32 factors and its current's e
                auto slot_ge = [&](int sl, double& g, double& e) {
                    if (FAC) {
                        const float4 f = f_s[sl];
                        g = f2d_int((f.x * f.y) * f.z);
                        e = efac_s[__float_as_int(f.w)];
                    } else if (XGF) {
                        const float4 q = reinterpret_cast<const float4*>(xg_s)[sl];
                        g = ff2d_int_nf(q.z, q.w);
                        e = ff2d_int_nf(q.x, q.y);
                    } else {
                        const double2 eg = xg_s[sl];
                        g = eg.y;
                        e = eg.x;
                    }
                };
                // XGF: the same sums over the float-pair (e, g) slots
                auto ff_sums_xg = [&](int a, int b, double& Gs, double& Xs) {
                    ff2 G2{0.f, 0.f}, X2{0.f, 0.f};
                    for (int sl = a; sl < b; ++sl) {
                        const float4 q = reinterpret_cast<const float4*>(xg_s)[sl];
                        const ff2 g{q.z, q.w};
                        G2 = ff_add(G2, g);
                        X2 = ff_add(X2, ff_mul(g, ff2{q.x, q.y}));
                    }
                    Gs = ff2d_int_nf(G2.h, G2.l);
                    Xs = ff2d_int_nf(X2.h, X2.l);
                };
                // with ion arrays the calcium slots sit last: calcium every
                // step (the buffer reads it), in a loop of its own, then
                // added to the node's sums
                int sc = s1;
                if (EXT && A.ions)
                    while (sc > s0 && tag_s[sc - 1] == NMODL_ION_CA) --sc;
                // FAC (here flat, so FAC_V): sum(g) and sum(g e) over slots
                // [a, b) as float pairs on the FP32 pipe (TwoSum and the
                // products' exact errors, about 48 bits; each g is an FP32
                // product, e a float pair), widened to doubles once per node
                // -- the FP64 pipe, 1/64 of the FP32 rate, had carried two
                // instructions per slot here on a few warps per block
                auto ff_sums_f = [&](int a, int b, float& Gh, float& Gl, float& Xh, float& Xl) {
                    float gh = 0.f, gl = 0.f, xh = 0.f, xl = 0.f;
                    for (int sl = a; sl < b; ++sl) {
                        const float4 f = f_s[sl];
                        const float g = (f.x * f.y) * f.z;
                        const float2 e = efac2_s[__float_as_int(f.w)];
                        float sm, er;
                        two_sum_f(gh, g, sm, er);
                        gh = sm;
                        gl += er;
                        const float ph = __fmul_rn(g, e.x);
                        const float pl = fmaf(g, e.y, fmaf(g, e.x, -ph));
                        two_sum_f(xh, ph, sm, er);
                        xh = sm;
                        xl += er + pl;
                    }
                    two_sum_f(gh, gl, Gh, Gl);
                    two_sum_f(xh, xl, Xh, Xl);
                };
                auto ff_sums = [&](int a, int b, double& Gs, double& Xs) {
                    float Gh, Gl, Xh, Xl;
                    ff_sums_f(a, b, Gh, Gl, Xh, Xl);
                    Gs = ff2d_int_nf(Gh, Gl);
                    Xs = ff2d_int_nf(Xh, Xl);
                };
                if constexpr (FAC_V && !EXT) {
                    // without ion arrays the node update stays in float
                    // pairs too: r = X - v G, d = G + cm/dt and the change
                    // r/d (a quotient from the FP32 reciprocal and one
                    // remainder correction, about 46 bits), one FP64
                    // addition for v += dv (v split exactly to 47 bits for
                    // the product; the addition takes all of v)
                    float Gh, Gl, Xh, Xl;
                    ff_sums_f(s0, s1, Gh, Gl, Xh, Xl);
                    float vh, vl, sm, er, rh, rl, dh, dl;
                    split_d_ff(vv, vh, vl);
                    const float ph = __fmul_rn(vh, Gh);
                    const float pl = fmaf(vh, Gl, fmaf(vl, Gh, fmaf(vh, Gh, -ph)));
                    two_sum_f(Xh, -ph, sm, er);
                    two_sum_f(sm, er + (Xl - pl), rh, rl);
                    two_sum_f(Gh, cmdt_h, sm, er);
                    two_sum_f(sm, er + (Gl + cmdt_l), dh, dl);
                    if (last) {
                        A.rhs[n0 + n] = ff2d_int_nf(rh, rl);
                        A.d[n0 + n] = ff2d_int_nf(dh, dl);
                    }
                    double vn = vv;
                    if (!A.clamp_v) {
                        const float inv = __frcp_rn(dh);
                        const float q1 = __fmul_rn(rh, inv);
                        const float q2 = ((fmaf(-q1, dh, rh) + rl) - q1 * dl) * inv;
                        two_sum_f(q1, q2, sm, er);
                        vn = vv + ff2d_int_nf(sm, er);
                    }
                    v_s[n] = vn;
                    vf_s[n] = d2f_int(vn);
                    continue;
                } else if constexpr (FAC_V) {
                    ff_sums(s0, sc, G, X);
                } else if constexpr (XGF) {
                    ff_sums_xg(s0, sc, G, X);
                } else {
                    for (int sl = s0; sl < sc; ++sl) {
                        double g, e;
                        slot_ge(sl, g, e);
                        X = fma(g, e, X);
                        G += g;
                    }
                }
                if (EXT && A.ions) {
                    if constexpr (FAC_V) {
                        ff_sums(sc, s1, Gca, Xca);
                    } else if constexpr (XGF) {
                        ff_sums_xg(sc, s1, Gca, Xca);
                    } else {
                        for (int sl = sc; sl < s1; ++sl) {
                            double g, e;
                            slot_ge(sl, g, e);
                            Xca = fma(g, e, Xca);
                            Gca += g;
                        }
                    }
                    X += Xca;
                    G += Gca;
                }
                r = fma(-vv, G, X);  // -sum g (v - e)
                dd = G;
                if (EXT && A.ions) {
                    s_ca = fma(vv, Gca, -Xca);
                    if (last) {  // sodium and potassium, once per window
                        for (int sl = s0; sl < s1; ++sl) {
                            double g, e;
                            slot_ge(sl, g, e);
                            const int tg = tag_s[sl];
                            if (tg == NMODL_ION_NA) s_na = fma(g, vv - e, s_na);
                            else if (tg == NMODL_ION_K) s_k = fma(g, vv - e, s_k);
                        }
                    }
                }
            }
            for (int t = 0; !flat && t < T; ++t) {
                const MechD& M = md_s[t];
                const uint16_t* seg = seg_s + t * (NT + 1);
                const int j0 = seg[n], j1 = seg[n + 1];
                if (EXT && M.kind == NMODL_CACUM) continue;  // no membrane current
                {
                    if (M.kind == NMODL_HH) {
                        const double gl = M.hh_g[2];
                        for (int j = j0; j < j1; ++j) {
                            double gna, gk;
                            inst_g(t, j, gna, gk);
                            const double ina = gna * (vv - M.hh_e[0]);
                            const double ik = gk * (vv - M.hh_e[1]);
                            if (EXT && A.ions) {
                                s_na += ina;
                                s_k += ik;
                            }
                            r -= ina + ik + gl * (vv - M.hh_e[2]);
                            dd += gna + gk + gl;
                        }
                    } else {
                        const double ve = vv - ((EXT && M.kind == NMODL_KIN3) ? M.k3.e : M.e);
                        for (int j = j0; j < j1; ++j) {
                            double g, g1;
                            inst_g(t, j, g, g1);
                            if (EXT && M.ion) {  // tagged whole current
                                const double ci = g * ve;
                                if (M.ion == NMODL_ION_NA) s_na += ci;
                                else if (M.ion == NMODL_ION_K) s_k += ci;
                                else s_ca += ci;
                                r -= ci;
                            } else {
                                r = fma(-g, ve, r);
                            }
                            dd += g;
                        }
                    }
                }
            }
            if (EXT && A.ions) {
                ica_s[n] = s_ca;
                if (last) {
                    if (A.ion[NMODL_ION_NA]) A.ion[NMODL_ION_NA][n0 + n] = s_na;
                    if (A.ion[NMODL_ION_K]) A.ion[NMODL_ION_K][n0 + n] = s_k;
                    if (A.ion[NMODL_ION_CA]) A.ion[NMODL_ION_CA][n0 + n] = s_ca;
                }
            }
            dd += cmdt;
            if (A.cable) {
                // the node's row of the tree system: its own axial term, then
                // its children's (v is the step's old v throughout)
                const int pp = par_s[n];
                if (pp != 0xffff) {
                    r = fma(-ga_s[n], vv - v_s[pp], r);
                    dd += ga_s[n];
                }
                const uint16_t* coff = sched_coff();
                const uint16_t* clist = coff + NT + 1;
                for (int q = coff[n]; q < coff[n + 1]; ++q) {
                    const int c = clist[q];
                    r = fma(gb_s[c], v_s[c] - vv, r);
                    dd += gb_s[c];
                }
                // the row for the tree solve, as float pairs in the same
                // 8 bytes
                const ff2 rp = ff_of(r), dp = ff_of(dd);
                reinterpret_cast<float2*>(r2_s)[n] = make_float2(rp.h, rp.l);
                reinterpret_cast<float2*>(d2_s)[n] = make_float2(dp.h, dp.l);
                if (last) {  // rhs and d report the assembled system
                    A.rhs[n0 + n] = r;
                    A.d[n0 + n] = dd;
                }
                continue;
            }
            const double vn = A.clamp_v ? vv : fma(r, rcp_fast(dd), vv);
            if (last) {
                A.rhs[n0 + n] = r;
                A.d[n0 + n] = dd;
            }
            v_s[n] = vn;
            if (PREC == NMODL_MIXED) vf_s[n] = d2f_int(vn);
        }
        if (KIN && tid == 0) wctr_s = 0;  // the state phase's work counter
        __syncthreads();
        if (A.cable) {
            if (!A.clamp_v) {
                if (tid < 32) {
                    const int cH = sched_s[0], cD = sched_s[1];
                    const uint16_t* cEL = sched_s + 2;
                    const uint16_t* cSL = cEL + cH + 1;
                    const uint16_t* cE = cSL + cD + 1;
                    const uint16_t* cS = cE + NT;
                    const uint16_t* coff = cS + NT;
                    const uint16_t* clist = coff + NT + 1;
                    // The tree system in float pairs (rows r2/d2 as float2
                    // in the same storage): each level's chain of dependent
                    // FP32 operations has 4-cycle latencies where an FP64
                    // instruction takes about 64 cycles, and the FP64 pipe is
                    // left to the other warps' gate updates; the pairs carry
                    // about 46 bits, far inside the solve's error budget.
                    float2* d2f = reinterpret_cast<float2*>(d2_s);
                    float2* r2f = reinterpret_cast<float2*>(r2_s);
                    auto ld = [](const float2* a, int i) { const float2 x = a[i]; return ff2{x.x, x.y}; };
                    auto st = [](float2* a, int i, ff2 x) { a[i] = make_float2(x.h, x.l); };
                    // leaves -> roots by height: d2[i] := ga_i / d' of node i
                    // (0 at roots) and r2[i] := r'/d' once its children are
                    // eliminated; 1/d' is only ever needed times ga_i (by the
                    // parent, d'_p -= gb_c (ga_c / d'_c), and by the
                    // substitution), so each level's chain has one product
                    // and difference per child, the reciprocal and two
                    // products
                    for (int h = 0; h < cH; ++h) {
                        for (int k = cEL[h] + tid; k < cEL[h + 1]; k += 32) {
                            const int i = cE[k];
                            ff2 dd = ld(d2f, i), r = ld(r2f, i);
                            for (int q = coff[i]; q < coff[i + 1]; ++q) {
                                const int c = clist[q];
                                const ff2 gb = ff_of(gb_s[c]);
                                dd = ff_sub(dd, ff_mul(gb, ld(d2f, c)));
                                r = ff_add(r, ff_mul(gb, ld(r2f, c)));
                            }
                            const ff2 inv = ff_rcp(dd);
                            st(d2f, i, par_s[i] != 0xffff ? ff_mul(ff_of(ga_s[i]), inv) : ff2{0.f, 0.f});
                            st(r2f, i, ff_mul(r, inv));
                        }
                        __syncwarp();
                    }
                    // roots -> leaves by depth: r2[i] := the change of v,
                    // x_i = r'/d' + (ga_i / d') x_parent
                    for (int l = 0; l < cD; ++l) {
                        for (int k = cSL[l] + tid; k < cSL[l + 1]; k += 32) {
                            const int i = cS[k];
                            const int pp = par_s[i];
                            if (pp != 0xffff) st(r2f, i, ff_add(ff_mul(ld(d2f, i), ld(r2f, pp)), ld(r2f, i)));
                        }
                        __syncwarp();
                    }
                }
                __syncthreads();
                for (int n = tid; n < NT; n += blockDim.x) {
                    const float2 dv = reinterpret_cast<const float2*>(r2_s)[n];
                    const double vn = v_s[n] + ff2d_int_nf(dv.x, dv.y);
                    v_s[n] = vn;
                    if (PREC == NMODL_MIXED) vf_s[n] = d2f_int(vn);
                }
            }
            __syncthreads();
        }
        // MIXED gate update of item k: the increment f (minf - m) added to
        // the hi/lo pair compensated
        auto gate_update_f = [&](int k, float minf, float f) {
            float2 m = st_f[k];
            const float delta = f * ((minf - m.x) - m.y);
            float s, e;
            two_sum_f(m.x, delta, s, e);
            const float lo = m.y + e;
            const float hi2 = s + lo;
            m.y = lo - (hi2 - s);
            m.x = hi2;
            st_f[k] = m;
        };
        // ---- state update, one thread per (instance, gate) item k (storage
        // index) of gate g of type t, instance j
        auto item = [&](int k, int t, int g, int j) {
            const int kind = EXT ? md_s[t].kind : NMODL_CNEXP;
            if (KIN && kind == NMODL_KIN9) {
                // the implicit-Euler Newton solve of one instance (kin9.cuh)
                if (g != 0) return;
                const int cnt = cnt_s[t], nd = nid_s[nid_off[t] + j];
                double x[9], y[9];
#pragma unroll
                for (int a = 0; a < 9; ++a) {
                    const int o = st_off[t] + a * cnt + j;
                    x[a] = PREC == NMODL_FP64 ? st_d[o] : f2d_int(st_f[o].x) + f2d_int(st_f[o].y);
                }
                bool nonconv;
                int iters;
                if constexpr (PREC == NMODL_FP64) {
                    const Kin9D& K = k9_s[t];
                    const double vv = v_s[nd];
                    double dk_f[kKinEdges], dk_b[kKinEdges];
#pragma unroll
                    for (int e = 0; e < kKinEdges; ++e) {
                        dk_f[e] = exp_tang(fma(K.bf[e], vv, K.af[e]));
                        dk_b[e] = exp_tang(fma(-K.bb[e], vv, K.ab[e]));
                    }
                    iters = kin9_newton_d(dk_f, dk_b, x, y, A.newton_tol, A.newton_max_iter, nonconv);
                } else {
                    const float* kf = k9f_s[t];
                    const float vf = vf_s[nd];
                    float dk_f[kKinEdges], dk_b[kKinEdges];
#pragma unroll
                    for (int e = 0; e < kKinEdges; ++e) {
                        dk_f[e] = ex2_hw(fmaf(kf[e], vf, kf[2 * kKinEdges + e]));
                        dk_b[e] = ex2_hw(fmaf(-kf[kKinEdges + e], vf, kf[3 * kKinEdges + e]));
                    }
                    iters = kin9_refine_mixed(dk_f, dk_b, x, y, A.newton_tol, 1 + A.ir_max, nonconv);
                }
                if (nonconv) latch_error(A.err, NMODL_ERR_NOCONV);
                count_solve(t, iters, nonconv);
#pragma unroll
                for (int a = 0; a < 9; ++a) {
                    const int o = st_off[t] + a * cnt + j;
                    if (PREC == NMODL_FP64) {
                        st_d[o] = y[a];
                    } else {
                        const float hi = d2f_int(y[a]);
                        st_f[o] = make_float2(hi, d2f_int(y[a] - f2d_int(hi)));
                    }
                }
                if (FAC) {
                    double yo = y[0];
#pragma unroll
                    for (int a = 1; a < 9; ++a)
                        if (a == md_s[t].open) yo = y[a];
                    put_open_factor(t, j, curf_s[t][0], d2f_int(yo));
                }
                return;
            }
            if (EXT && (kind == NMODL_KIN3 || kind == NMODL_CACUM)) {
                // coupled states: the item of the first state updates all
                if (g != 0) return;
                const int cnt = cnt_s[t], nd = nid_s[nid_off[t] + j];
                double x[3];
                const int ns = kind == NMODL_KIN3 ? 3 : 2;
                for (int a = 0; a < ns; ++a) {
                    const int o = st_off[t] + a * cnt + j;
                    x[a] = PREC == NMODL_FP64 ? st_d[o] : f2d_int(st_f[o].x) + f2d_int(st_f[o].y);
                }
                // failed: the refinement or Newton iteration reached its cap
                bool failed = false, conv = true;
                int iters = 1;
                if (kind == NMODL_KIN3) {
                    if (PREC == NMODL_FP64)
                        kin3_step_d(md_s[t].k3, v_s[nd], A.dt, x);
                    else
                        iters = kin3_step_mixed(k3f_s[t], vf_s[nd], d2f_int(A.dt), A.newton_tol,
                                                A.ir_max, x, failed);
                } else if (PREC == NMODL_FP64) {
                    iters = cacum_newton_d(md_s[t].cd, ica_s[nd], A.dt, A.newton_tol,
                                           A.newton_max_iter, x[0], x[1], conv);
                } else {
                    iters = cacum_newton_mixed(md_s[t].cd, cdf_s[t], ica_s[nd], A.dt, A.newton_tol,
                                               A.newton_max_iter, A.ir_max, x[0], x[1], conv);
                }
                if (failed || !conv) latch_error(A.err, NMODL_ERR_NOCONV);
                count_solve(t, iters, failed || !conv);
                for (int a = 0; a < ns; ++a) {
                    const int o = st_off[t] + a * cnt + j;
                    if (PREC == NMODL_FP64) {
                        st_d[o] = x[a];
                    } else {
                        const float hi = d2f_int(x[a]);
                        st_f[o] = make_float2(hi, d2f_int(x[a] - f2d_int(hi)));
                    }
                }
                if (FAC && kind == NMODL_KIN3) {
                    const int open = md_s[t].k3.open;
                    put_open_factor(t, j, curf_s[t][0],
                                    d2f_int(open == 0 ? x[0] : open == 1 ? x[1] : x[2]));
                }
                return;
            }
            if (PREC == NMODL_FP64) {
                const double vv = v_s[nid_s[nid_off[t] + j]];
                const GateD& G = md_s[t].gate[g];
                st_d[k] = A.pade ? gate_step_pade_d<true>(G, 1.0, vv, st_d[k])
                                 : gate_step_fast_d<true>(G, 1.0, vv, st_d[k]);
            } else {
                float minf, f;
                gate_coef_f(gf_s[t][g], phidt_f[t], vf_s[nid_s[nid_off[t] + j]], minf, f,
                            A.pade != 0);
                gate_update_f(k, minf, f);
            }
        };
        if constexpr (PREC == NMODL_FP64 || KIN) {
            // work order (slots past a pair's count are a group's padding;
            // with the 9-state scheme MIXED takes it too, so that its one item
            // per instance does not leave eight of nine lanes idle)
            auto work = [&](int w, int& wi) {
                while (w >= wstart_s[wi + 1]) ++wi;
                const int q = wq_s[wi];
                const int t = pair_t[q], j = w - wstart_s[wi];
                if (j < cnt_s[t]) {
                    item(pair_start[q] + j, t, pair_g[q], j);
                    if (FAC) put_factor(q, j, st_f[pair_start[q] + j].x);
                }
            };
            int wi = 0;
            if constexpr (KIN != 0) {
                // warps take whole-warp chunks of work slots (groups are
                // padded to whole warps) from a counter as they come free:
                // the 9-state solves, first in the order, run beside the
                // gate updates instead of as a tail that leaves the rest of
                // the block idle (measured on the cortical mix with the
                // 9-state scheme on a quarter of 1M nodes: FP64 8.54e9 ->
                // 9.0e9, MIXED 2.05e10 -> 2.41e10; on the ion network, whose
                // 3-state and buffer solves are lighter, chunks from the
                // counter were 3-5 % slower -- one shared atomic per 32
                // cheap items -- so only this variant takes them)
                const int lane = tid & 31;
                for (;;) {
                    int base = 0;
                    if (lane == 0) base = atomicAdd(&wctr_s, 32);
                    base = __shfl_sync(0xffffffffu, base, 0);
                    if (base >= wstart_s[n_work]) break;
                    work(base + lane, wi);
                }
            } else {
                for (int w = tid; w < wstart_s[n_work]; w += blockDim.x) work(w, wi);
            }
        } else {
            // storage order (one group: the bodies are cheap and issue-bound)
            if constexpr (!EXT) {
                // gates only: the constants of a thread's current gate pair
                // (its FP32 rate parameters, phi dt, node-id and slot bases,
                // factor multiplier, power and component) kept in registers
                // and reloaded when its next item starts another pair, since
                // a thread's items stay in one pair for several rounds
                // Each warp takes a contiguous chunk of whole rounds of the
                // items, its lanes striding by 32 inside it, so that a
                // thread's next item is usually in the same pair (pairs are
                // a few hundred items; a block-wide stride would leave it
                // for another pair at almost every item)
                int q = -1, end = 0, base = 0, nb = 0, pw = 0, fx = 0;
                float pdt = 0.f, fm = 1.f;
                GateF G{};
                const bool pade = A.pade != 0;
                const int chunk = 32 * ((total_items + blockDim.x - 1) / blockDim.x);
                const int k_end = min(total_items, (tid >> 5) * chunk + chunk);
                for (int k = (tid >> 5) * chunk + (tid & 31); k < k_end; k += 32) {
                    if (k >= end) {
                        do {
                            ++q;
                        } while (k >= pair_start[q + 1]);
                        base = pair_start[q];
                        end = pair_start[q + 1];
                        const int t = pair_t[q];
                        G = gf_s[t][pair_g[q]];
                        pdt = phidt_f[t];
                        nb = nid_off[t];
                        if (FAC) {
                            fm = fmul_s[q];
                            pw = fpow_s[q];
                            fx = fidx_s[q];
                        }
                    }
                    const int j = k - base;
                    float minf, f;
                    gate_coef_f(G, pdt, vf_s[nid_s[nb + j]], minf, f, pade);
                    gate_update_f(k, minf, f);
                    if (FAC) {  // the gate's conductance factor (put_factor)
                        const float hi = st_f[k].x;
                        float fv = fm;
                        if (pw >= 1) fv *= hi;
                        if (pw >= 2) fv *= hi;
                        if (pw >= 3) fv *= hi;
                        for (int e = 3; e < pw; ++e) fv *= hi;
                        reinterpret_cast<float*>(f_s)[4 * pos_s[nb + j] + fx] = fv;
                    }
                }
            } else {
                int q = 0;
                for (int k = tid; k < total_items; k += blockDim.x) {
                    while (k >= pair_start[q + 1]) ++q;
                    item(k, pair_t[q], pair_g[q], k - pair_start[q]);
                    if (FAC) put_factor(q, k - pair_start[q], st_f[k].x);
                }
            }
        }
        __syncthreads();
    }

    // ---- write the tile back
    for (int k = tid; k < NT; k += blockDim.x) {
        const double vn = v_s[k];
        if (!finite_int(vn)) latch_error(A.err, NMODL_ERR_NONFINITE);
        A.v[n0 + k] = vn;
    }
    {
        int q = 0;
        for (int k = tid; k < total_items; k += blockDim.x) {
            while (k >= pair_start[q + 1]) ++q;
            const int t = pair_t[q], g = pair_g[q];
            const int j = k - pair_start[q];
            double m;
            if (PREC == NMODL_FP64) m = st_d[k];
            else m = f2d_int(st_f[k].x) + f2d_int(st_f[k].y);
            if (!finite_int(m)) latch_error(A.err, NMODL_ERR_NONFINITE);
            A.states[t][g * A.stride[t] + a_s[t] + j] = m;
        }
    }
    __syncthreads();  // shared memory is reused by the next tile
    }
    // every thread has left the tile loop after the same barrier: the
    // block's counts are complete
    if constexpr (EXT)
        if (tid < T && A.cnt[tid] && kit_s[tid]) {
            atomicAdd(&A.cnt[tid]->iters, kit_s[tid]);
            if (knc_s[tid]) atomicAdd(&A.cnt[tid]->nonconv, knc_s[tid]);
            atomicMax(&A.cnt[tid]->max_iter_seen, kmx_s[tid]);
        }
}

// ------------------------------------------------------------ launchers

static int grid_for(int64_t n, int block) {
    int64_t b = (n + block - 1) / block;
    if (b > 148 * 64) b = 148 * 64;
    return (int)(b < 1 ? 1 : b);
}

void launch_init_gates(const MechD* md, int n_gates, int64_t n, const int32_t* ni,
                       const double* v, double* st, int64_t stride, int32_t* err,
                       cudaStream_t s) {
    if (n == 0 || n_gates == 0) return;
    dim3 grid(grid_for(n, 256), n_gates);
    k_init_gates<<<grid, 256, 0, s>>>(md, n, ni, v, st, stride, err);
}

void launch_state_gates(int prec, const MechD* md, int n_gates, int64_t n,
                        const int32_t* ni, const double* v, double* st,
                        int64_t stride, double dt, int pade, int32_t* err,
                        cudaStream_t s) {
    if (n == 0 || n_gates == 0) return;
    dim3 grid(grid_for(n, 256), n_gates);
    if (prec == NMODL_FP64)
        k_state_gates<NMODL_FP64><<<grid, 256, 0, s>>>(md, n, ni, v, st, stride, dt, pade, err);
    else
        k_state_gates<NMODL_MIXED><<<grid, 256, 0, s>>>(md, n, ni, v, st, stride, dt, pade, err);
}

void launch_cur_seg(int kind, const void* desc, int64_t n_chunks,
                    const int32_t* chunk, const int32_t* ni, const double* v,
                    const double* st, int64_t stride, double* rhs, double* d,
                    double* ion_a, double* ion_b, int32_t* err, cudaStream_t s) {
    if (n_chunks == 0) return;
    const int block = 256;
    const int64_t threads = n_chunks * 32;
    const int grid = (int)((threads + block - 1) / block);
    const bool ion = ion_a || ion_b;
#define NMODL_CUR_SEG(K, I) \
    k_cur_seg<K, I><<<grid, block, 0, s>>>(desc, n_chunks, chunk, ni, v, st, stride, rhs, d, ion_a, ion_b, err)
    if (kind == NMODL_KIN9) {
        if (ion) NMODL_CUR_SEG(NMODL_KIN9, true); else NMODL_CUR_SEG(NMODL_KIN9, false);
    } else if (kind == NMODL_KIN3) {
        if (ion) NMODL_CUR_SEG(NMODL_KIN3, true); else NMODL_CUR_SEG(NMODL_KIN3, false);
    } else {
        if (ion) NMODL_CUR_SEG(NMODL_CNEXP, true); else NMODL_CUR_SEG(NMODL_CNEXP, false);
    }
#undef NMODL_CUR_SEG
}

// grid = blocks of this launch (one per tile, or the resident count in the
// persistent form)
// variant = precision + 2 * ext + 2 * kin: ext instantiates the kernel with
// the small systems and ion sums (EXT); kin adds the 9-state scheme (KIN),
// whose build follows the block size; plain HH/CNEXP plans use the leanest
// variant
using FusedKernel = void (*)(FusedArgs);
static FusedKernel fused_kernel(int variant, int block) {
    const bool wide = block > kFusedKinBlock;
    switch (variant) {
    case 0: return k_fused_tiles<NMODL_FP64, false, 0>;
    case 1: return k_fused_tiles<NMODL_MIXED, false, 0>;
    case 2: return k_fused_tiles<NMODL_FP64, true, 0>;
    case 3: return k_fused_tiles<NMODL_MIXED, true, 0>;
    case 4: return wide ? k_fused_tiles<NMODL_FP64, true, 2> : k_fused_tiles<NMODL_FP64, true, 1>;
    default: return wide ? k_fused_tiles<NMODL_MIXED, true, 2> : k_fused_tiles<NMODL_MIXED, true, 1>;
    }
}

cudaError_t launch_fused(int variant, const FusedArgs& a, int grid, int block, size_t smem,
                         cudaStream_t s) {
    fused_kernel(variant, block)<<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

int fused_resident_grid(int variant, int n_tiles, int block, size_t smem) {
    int dev = 0, sms = 148, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fused_kernel(variant, block), block,
                                                  smem);
    return std::min(n_tiles, std::max(1, per_sm) * sms);
}

// both builds of a 9-state variant (kFusedKinBlock and kFusedKinBlock + 32
// stand for the block sizes of the register-rich and the wide build)
cudaError_t fused_prepare(int variant, size_t max_smem) {
    cudaError_t e = cudaSuccess;
    for (int block : {kFusedKinBlock, kFusedKinBlock + 32})
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(fused_kernel(variant, block),
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem);
    return e;
}

size_t fused_static_smem(int variant) {
    size_t s = 0;
    for (int block : {kFusedKinBlock, kFusedKinBlock + 32}) {
        cudaFuncAttributes fa{};
        cudaFuncGetAttributes(&fa, fused_kernel(variant, block));
        s = std::max(s, fa.sharedSizeBytes);
    }
    return s;
}

}  // namespace nmodl
