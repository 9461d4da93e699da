// k_kin9.cu -- 9-state kinetic scheme: INITIAL and nrn_state for sm_103a.
//
// The KINETIC scheme is the linear ODE x' = A(v) x (Section 5.1); one
// implicit Euler step solves F(y) = y - x - dt A y = 0 by Newton iteration
// with the exact Jacobian J = I - dt A (Section 5.2 derivimplicit, Section
// 5.3 Newton + LU).  One thread owns one instance; the banded no-pivot LU
// and the Newton / refinement loops are in kin9.cuh (shared with the fused
// tile kernel).
//
// FP64 form: rates, J, LU, residual and update in double.
// MIXED form: rates and the LU factorisation in FP32; the FP64 residual and
// update refine y until max|delta| <= tol or ir_max refinements.
#include <algorithm>
#include <cmath>

#include "kernels.cuh"
#include "kin9.cuh"

namespace nmodl {

// ------------------------------------------------------------- INITIAL
// Stationary distribution: A pi = 0 with sum(pi) = 1, solved as the square
// system whose rows 0..7 are those of -A and whose last row is the
// normalisation.  The leading 8x8 block of -A is a nonsingular M-matrix
// (irreducible chain), so the dense no-pivot LU below is stable.
__global__ void k_kin9_init(const Kin9D* __restrict__ kd, int64_t n,
                            const int32_t* __restrict__ ni,
                            const double* __restrict__ v, double* st,
                            int64_t stride, int32_t* err) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Kin9D& K = *kd;
    const double vv = v[ni[i]];
    double M[9][9];
#pragma unroll
    for (int a = 0; a < 9; ++a)
#pragma unroll
        for (int b = 0; b < 9; ++b) M[a][b] = 0.0;
#pragma unroll
    for (int e = 0; e < kKinEdges; ++e) {
        const double kf = K.af[e] * exp(K.bf[e] * vv);
        const double kb = K.ab[e] * exp(-K.bb[e] * vv);
        const int lo = edge_lo(e), hi = edge_hi(e);
        M[hi][lo] -= kf;
        M[lo][lo] += kf;
        M[lo][hi] -= kb;
        M[hi][hi] += kb;
    }
#pragma unroll
    for (int b = 0; b < 9; ++b) M[8][b] = 1.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const double rp = 1.0 / M[k][k];
#pragma unroll
        for (int r = k + 1; r < 9; ++r) {
            const double l = M[r][k] * rp;
            M[r][k] = l;
#pragma unroll
            for (int c = k + 1; c < 9; ++c) M[r][c] -= l * M[k][c];
        }
    }
    double x[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) x[a] = (a == 8) ? 1.0 : 0.0;
#pragma unroll
    for (int a = 1; a < 9; ++a)
#pragma unroll
        for (int c = 0; c < a; ++c) x[a] -= M[a][c] * x[c];
#pragma unroll
    for (int a = 8; a >= 0; --a) {
#pragma unroll
        for (int c = a + 1; c < 9; ++c) x[a] -= M[a][c] * x[c];
        x[a] = x[a] / M[a][a];
    }
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        if (!finite_int(x[a])) latch_error(err, NMODL_ERR_NONFINITE);
        st[a * stride + i] = x[a];
    }
}

// ---------------------------------------------------------------- state

// One thread per instance (or per entry of the first *n_list_dev of list).  ni == nullptr means instance i reads v[i]; dt_arr != nullptr gives
// each instance its own step (used to generate training pairs).
// Rate constants of one launch, folded on the host and passed by value.
// With one dt for all instances dt k = exp(b v + ln(dt a)): one multiply-add
// and the exp (FP64: lnc = ln(dt af), ln(dt ab); MIXED: kf = bf, bb, then
// ln(dt af), ln(dt ab) in FP32, all scaled by log2(e) for the exp2 unit).
// With a dt per instance (training pairs) MIXED keeps af, ab in kf and
// scales by dt.  FP32 copies are made on the
// host because FP64 -> FP32 conversions run on the FP64 pipe.
struct Kin9Launch {
    double lnc[2 * kKinEdges];
    float kf[4 * kKinEdges];
};

// MIXED is compiled for four 128-thread blocks per SM (128 registers, about
// 190 bytes of spills): with the refinement's residual in float pairs the
// step is bound by issue latency more than by the FP64 pipe, and 16 warps
// per SM beat 12 at 168 registers without spills (measured 1.04x on 1M
// instances; before that change three blocks were best, 1.14x over two);
// the FP64 form keeps its ~240 registers, bound by the FP64 pipe already.
template <int PREC, bool LIST>
__global__ void __launch_bounds__(128, PREC == NMODL_MIXED ? 4 : 1)
    k_kin9_state(const Kin9D* __restrict__ kd, const Kin9Launch KL, int64_t n,
                 const int32_t* __restrict__ ni, const double* __restrict__ v,
                 double* st, int64_t stride, double dt_scalar,
                 const double* __restrict__ dt_arr, double tol, int max_iter,
                 int ir_max, const int32_t* __restrict__ list,
                 const int32_t* __restrict__ n_list_dev, KinCounters* cnt,
                 int32_t* err) {
    const double* lnc_s = KL.lnc;
    const float* kf_s = KL.kf;
    const int64_t n_work = LIST ? (int64_t)*n_list_dev : n;
    unsigned long long it_sum = 0, nc_sum = 0;
    int it_max = 0;
    // grid-stride: a fallback list of unknown length runs on a grid sized
    // for the device, not for the whole mechanism
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_work;
         t += (int64_t)gridDim.x * blockDim.x) {
        int iters = 0;
        bool nonconv = false;
        const int64_t i = LIST ? (int64_t)list[t] : t;
        const Kin9D& K = *kd;
        const double vv = ni ? v[ni[i]] : v[i];
        const double dt = dt_arr ? dt_arr[i] : dt_scalar;
        double x[9], y[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) x[a] = st[a * stride + i];
        if (PREC == NMODL_FP64) {
            double dk_f[kKinEdges], dk_b[kKinEdges];
            if (dt_arr) {
#pragma unroll
                for (int e = 0; e < kKinEdges; ++e) {
                    dk_f[e] = dt * (K.af[e] * exp_tang(K.bf[e] * vv));
                    dk_b[e] = dt * (K.ab[e] * exp_tang(-K.bb[e] * vv));
                }
            } else {
#pragma unroll
                for (int e = 0; e < kKinEdges; ++e) {
                    dk_f[e] = exp_tang(fma(K.bf[e], vv, lnc_s[e]));
                    dk_b[e] = exp_tang(fma(-K.bb[e], vv, lnc_s[kKinEdges + e]));
                }
            }
            iters = kin9_newton_d(dk_f, dk_b, x, y, tol, max_iter, nonconv);
        } else {
            float dk_f[kKinEdges], dk_b[kKinEdges];
            const float vf = d2f_int(vv);
            if (dt_arr) {
                const float dtf = d2f_int(dt);
#pragma unroll
                for (int e = 0; e < kKinEdges; ++e) {
                    dk_f[e] = dtf * (kf_s[2 * kKinEdges + e] * ex2_hw(kf_s[e] * vf));
                    dk_b[e] = dtf * (kf_s[3 * kKinEdges + e] * ex2_hw(-kf_s[kKinEdges + e] * vf));
                }
            } else {
#pragma unroll
                for (int e = 0; e < kKinEdges; ++e) {
                    dk_f[e] = ex2_hw(fmaf(kf_s[e], vf, kf_s[2 * kKinEdges + e]));
                    dk_b[e] = ex2_hw(fmaf(-kf_s[kKinEdges + e], vf, kf_s[3 * kKinEdges + e]));
                }
            }
            iters = kin9_refine_mixed(dk_f, dk_b, x, y, tol, 1 + ir_max, nonconv);
        }
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            if (!finite_int(y[a])) latch_error(err, NMODL_ERR_NONFINITE);
            st[a * stride + i] = y[a];
        }
        if (nonconv) latch_error(err, NMODL_ERR_NOCONV);
        it_sum += iters;
        nc_sum += nonconv ? 1 : 0;
        it_max = max(it_max, iters);
    }
    warp_count(cnt, it_sum, nc_sum, it_max);
}

void launch_kin9_init(const Kin9D* kd, int64_t n, const int32_t* ni,
                      const double* v, double* st, int64_t stride, int32_t* err,
                      cudaStream_t s) {
    if (n == 0) return;
    const int block = 128;
    k_kin9_init<<<(int)((n + block - 1) / block), block, 0, s>>>(kd, n, ni, v, st, stride, err);
}

void launch_kin9_state(int prec, const Kin9D* kd, const Kin9D& kh, int64_t n, const int32_t* ni,
                       const double* v, double* st, int64_t stride, double dt,
                       const double* dt_arr, double tol, int max_iter, int ir_max,
                       const int32_t* list, int64_t n_list_max,
                       const int32_t* n_list_dev, KinCounters* cnt,
                       int32_t* err, cudaStream_t s) {
    const int block = 128;
    const int64_t work = list ? n_list_max : n;
    if (work == 0) return;
    int grid = (int)((work + block - 1) / block);
    if (list) {
        // the list's length is known on the device only: exactly the
        // resident grid (one wave; its ~200 registers allow two or three
        // 128-thread blocks per SM), each thread striding over the list
        int dev = 0, sms = 148, per_sm = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (prec == NMODL_FP64)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_kin9_state<NMODL_FP64, true>,
                                                          block, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_kin9_state<NMODL_MIXED, true>,
                                                          block, 0);
        grid = (int)std::min<int64_t>(grid, (int64_t)sms * std::max(1, per_sm));
    }
    Kin9Launch KL;
    for (int e = 0; e < kKinEdges; ++e) {
        const double cf = dt_arr ? 0.0 : std::log(dt * kh.af[e]);
        const double cb = dt_arr ? 0.0 : std::log(dt * kh.ab[e]);
        KL.lnc[e] = cf;
        KL.lnc[kKinEdges + e] = cb;
        constexpr double kLog2e = 1.4426950408889634;
        KL.kf[e] = (float)(kh.bf[e] * kLog2e);
        KL.kf[kKinEdges + e] = (float)(kh.bb[e] * kLog2e);
        KL.kf[2 * kKinEdges + e] = (float)(dt_arr ? kh.af[e] : cf * kLog2e);
        KL.kf[3 * kKinEdges + e] = (float)(dt_arr ? kh.ab[e] : cb * kLog2e);
    }
    if (prec == NMODL_FP64) {
        if (list)
            k_kin9_state<NMODL_FP64, true><<<grid, block, 0, s>>>(kd, KL, n, ni, v, st, stride, dt, dt_arr, tol, max_iter, ir_max, list, n_list_dev, cnt, err);
        else
            k_kin9_state<NMODL_FP64, false><<<grid, block, 0, s>>>(kd, KL, n, ni, v, st, stride, dt, dt_arr, tol, max_iter, ir_max, list, n_list_dev, cnt, err);
    } else {
        if (list)
            k_kin9_state<NMODL_MIXED, true><<<grid, block, 0, s>>>(kd, KL, n, ni, v, st, stride, dt, dt_arr, tol, max_iter, ir_max, list, n_list_dev, cnt, err);
        else
            k_kin9_state<NMODL_MIXED, false><<<grid, block, 0, s>>>(kd, KL, n, ni, v, st, stride, dt, dt_arr, tol, max_iter, ir_max, list, n_list_dev, cnt, err);
    }
}

}  // namespace nmodl
