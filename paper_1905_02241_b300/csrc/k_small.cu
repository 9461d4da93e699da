// k_small.cu -- state updates of the small systems for sm_103a.
//
//  NMODL_KIN3   3-state kinetic scheme x' = A(v) x (edges 0-1, 1-2, 0-2).
//               Implicit Euler: (I - dt A) y = x.  For a linear scheme the
//               first Newton update from y = x is already the solution, so
//               the step is one solve, done by Gaussian elimination written
//               out for the 3x3 system ("sparse" with symbolic elimination,
//               Section 5.2).  J = I - dt A is an M-matrix whose columns sum
//               to one, so elimination without pivoting is stable (it is
//               the elimination partial pivoting would choose).
//  NMODL_CACUM  2-state calcium buffer, nonlinear (binding term kf cai
//               (btot - cab)).  Implicit Euler by Newton iteration with the
//               exact Jacobian, each update solved with the closed-form
//               inverse of the 2x2 matrix (the small-matrix direct inverse
//               of Section 5.3; no pivoting, no branches).  The calcium
//               current ica of the node is read from the ion array filled by
//               the current updates of the same step.
//
// One thread per instance; states are SoA rows of `stride` doubles.  MIXED:
// FP32 rates, eliminations and Newton updates, the residual and the
// refinement in FP64 (FP32 parameters passed by value from the host).  The
// per-instance math lives in small_systems.cuh (shared with the fused tile
// kernel).
#include "kernels.cuh"
#include "small_systems.cuh"

namespace nmodl {

// ------------------------------------------------------------- KIN3

// INITIAL: stationary distribution by the Markov chain tree theorem: pi_s
// is proportional to the sum, over the spanning trees directed to s, of the
// products of their rates (three trees per state for three states).
__global__ void k_kin3_init(const Kin3D* __restrict__ kd, int64_t n,
                            const int32_t* __restrict__ ni, const double* __restrict__ v,
                            double* st, int64_t stride, int32_t* err) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double kf[3], kb[3];
    kin3_rates_d(*kd, v[ni[i]], kf, kb);
    // k01 = kf0, k10 = kb0, k12 = kf1, k21 = kb1, k02 = kf2, k20 = kb2
    const double w0 = kb[0] * kb[2] + kb[0] * kb[1] + kf[1] * kb[2];
    const double w1 = kf[0] * kb[1] + kf[0] * kb[2] + kf[2] * kb[1];
    const double w2 = kf[2] * kf[1] + kf[2] * kb[0] + kf[0] * kf[1];
    const double r = 1.0 / (w0 + w1 + w2);
    const double p[3] = {w0 * r, w1 * r, w2 * r};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (!finite_int(p[a])) latch_error(err, NMODL_ERR_NONFINITE);
        st[a * stride + i] = p[a];
    }
}

// FP64: one solve.  MIXED: rates and the elimination in FP32, then
// iterative refinement with the FP64 residual x - J y (J's diagonal rebuilt
// in FP64 from the FP32 off-diagonals so that its columns sum to one) until
// max|delta| <= tol or ir_max refinements.
template <int PREC>
__global__ void __launch_bounds__(256)
    k_kin3_state(const Kin3D* __restrict__ kd, const Kin3F kf32, int64_t n,
                 const int32_t* __restrict__ ni, const double* __restrict__ v, double* st,
                 int64_t stride, double dt, double tol, int ir_max, KinCounters* cnt,
                 int32_t* err) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    unsigned long long it_sum = 0, nc_sum = 0;
    int it_max = 0;
    if (i < n) {
        const Kin3D& K = *kd;
        const double vv = v[ni[i]];
        double x[3], y[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) x[a] = st[a * stride + i];
        int iters = 1;
        if (PREC == NMODL_FP64) {
            double kf[3], kb[3], M[3][3];
            kin3_rates_d(K, vv, kf, kb);
            kin3_matrix(kf, kb, dt, M);
#pragma unroll
            for (int a = 0; a < 3; ++a) y[a] = x[a];
            solve3(M, y);
        } else {
            bool nonconv;
#pragma unroll
            for (int a = 0; a < 3; ++a) y[a] = x[a];
            iters = kin3_step_mixed(kf32, d2f_int(vv), d2f_int(dt), tol, ir_max, y, nonconv);
            if (nonconv) {
                nc_sum = 1;
                latch_error(err, NMODL_ERR_NOCONV);
            }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (!finite_int(y[a])) latch_error(err, NMODL_ERR_NONFINITE);
            st[a * stride + i] = y[a];
        }
        it_sum = iters;
        it_max = iters;
    }
    warp_count(cnt, it_sum, nc_sum, it_max);
}

// ------------------------------------------------------------ CACUM

__global__ void k_cacum_init(const CacumD* __restrict__ cd, int64_t n, double* st,
                             int64_t stride) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const CacumD& C = *cd;
    st[i] = C.cai0;
    st[stride + i] = C.kf * C.cai0 * C.btot / (C.kf * C.cai0 + C.kb);
}

// Newton with the closed-form 2x2 inverse (cacum_newton_d; MIXED:
// cacum_newton_mixed), reading the node's ica.
template <int PREC>
__global__ void __launch_bounds__(256)
    k_cacum_state(const CacumD* __restrict__ cd, const CacumF cf32, int64_t n,
                  const int32_t* __restrict__ ni, const double* __restrict__ ica, double* st,
                  int64_t stride, double dt, double tol, int max_iter, int ir_max,
                  KinCounters* cnt, int32_t* err) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    unsigned long long it_sum = 0, nc_sum = 0;
    int it_max = 0;
    if (i < n) {
        const CacumD C = *cd;
        double y0 = st[i], y1 = st[stride + i];
        bool conv = false;
        const int it = PREC == NMODL_FP64
                           ? cacum_newton_d(C, ica[ni[i]], dt, tol, max_iter, y0, y1, conv)
                           : cacum_newton_mixed(C, cf32, ica[ni[i]], dt, tol, max_iter, ir_max,
                                                y0, y1, conv);
        if (!finite_int(y0) || !finite_int(y1)) latch_error(err, NMODL_ERR_NONFINITE);
        if (!conv) latch_error(err, NMODL_ERR_NOCONV);
        st[i] = y0;
        st[stride + i] = y1;
        it_sum = it;
        nc_sum = conv ? 0 : 1;
        it_max = it;
    }
    warp_count(cnt, it_sum, nc_sum, it_max);
}

// ------------------------------------------------------------ launches

void launch_kin3_init(const Kin3D* kd, int64_t n, const int32_t* ni, const double* v,
                      double* st, int64_t stride, int32_t* err, cudaStream_t s) {
    if (n == 0) return;
    k_kin3_init<<<(int)((n + 255) / 256), 256, 0, s>>>(kd, n, ni, v, st, stride, err);
}

Kin3F kin3_f32(const Kin3D& K) {
    Kin3F f;
    for (int e = 0; e < 3; ++e) {
        f.af[e] = (float)K.af[e];
        f.bf[e] = (float)(K.bf[e] * 1.4426950408889634);  // log2(e): the exp2 unit
        f.ab[e] = (float)K.ab[e];
        f.bb[e] = (float)(K.bb[e] * 1.4426950408889634);
    }
    return f;
}
CacumF cacum_f32(const CacumD& C) {
    return CacumF{(float)C.k, (float)C.rtau, (float)C.cai0, (float)C.kf, (float)C.kb, (float)C.btot};
}

void launch_kin3_state(int prec, const Kin3D* kd, const Kin3D& kh, int64_t n, const int32_t* ni,
                       const double* v, double* st, int64_t stride, double dt, double tol,
                       int ir_max, KinCounters* cnt, int32_t* err, cudaStream_t s) {
    if (n == 0) return;
    const int grid = (int)((n + 255) / 256);
    const Kin3F f = kin3_f32(kh);
    if (prec == NMODL_FP64)
        k_kin3_state<NMODL_FP64><<<grid, 256, 0, s>>>(kd, f, n, ni, v, st, stride, dt, tol, ir_max, cnt, err);
    else
        k_kin3_state<NMODL_MIXED><<<grid, 256, 0, s>>>(kd, f, n, ni, v, st, stride, dt, tol, ir_max, cnt, err);
}

void launch_cacum_init(const CacumD* cd, int64_t n, double* st, int64_t stride,
                       cudaStream_t s) {
    if (n == 0) return;
    k_cacum_init<<<(int)((n + 255) / 256), 256, 0, s>>>(cd, n, st, stride);
}

void launch_cacum_state(int prec, const CacumD* cd, const CacumD& ch, int64_t n,
                        const int32_t* ni, const double* ica, double* st, int64_t stride,
                        double dt, double tol, int max_iter, int ir_max, KinCounters* cnt,
                        int32_t* err, cudaStream_t s) {
    if (n == 0) return;
    const int grid = (int)((n + 255) / 256);
    const CacumF f = cacum_f32(ch);
    if (prec == NMODL_FP64)
        k_cacum_state<NMODL_FP64><<<grid, 256, 0, s>>>(cd, f, n, ni, ica, st, stride, dt, tol,
                                                       max_iter, ir_max, cnt, err);
    else
        k_cacum_state<NMODL_MIXED><<<grid, 256, 0, s>>>(cd, f, n, ni, ica, st, stride, dt, tol,
                                                        max_iter, ir_max, cnt, err);
}

}  // namespace nmodl
