// k_kin9.cu -- 9-state kinetic scheme: INITIAL and nrn_state for sm_103a.
//
// The KINETIC scheme is the linear ODE x' = A(v) x (Section 5.1); one
// implicit Euler step solves F(y) = y - x - dt A y = 0 by Newton iteration
// with the exact Jacobian J = I - dt A (Section 5.2 derivimplicit, Section
// 5.3 Newton + LU).  One thread owns one instance.  J is a nonsingular
// M-matrix whose columns sum to one (columns of -dt A sum to 0), so LU with
// partial pivoting makes no row interchanges and the no-pivot LU below
// performs the same eliminations.  States are numbered 3a+b on a 3x3
// lattice whose edges join indices differing by 1 (same row) or 3, so J and
// its LU factors live inside the band |i - j| <= 3; every loop is unrolled
// at compile time and only band entries are ever touched.
//
// FP64 form: rates, J, LU, residual and update in double.
// MIXED form: rates and the LU factorisation in FP32; the residual
// F(y) = J y - x (with J's diagonal rebuilt in FP64 so that its columns keep
// summing exactly to one) and the update of y in FP64; the FP32 factors
// refine y until max|delta| <= tol or ir_max refinements.
#include <algorithm>
#include <cmath>

#include "kernels.cuh"

namespace nmodl {

namespace {


__host__ __device__ constexpr bool in_band(int i, int j) { return (i - j <= 3) && (j - i <= 3); }

// In-place no-pivot LU of the banded 9x9 matrix M (only band entries used);
// the diagonal is replaced by the reciprocals of the pivots, so that the
// triangular solves multiply instead of divide.
// pivot reciprocal: the refined hardware reciprocal in FP64, IEEE in FP32
__device__ __forceinline__ double recip(double x) { return rcp_fast(x); }
__device__ __forceinline__ float recip(float x) { return 1.0f / x; }

template <typename R>
__device__ __forceinline__ void lu_band(R (&M)[9][9]) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const R rp = recip(M[k][k]);
        M[k][k] = rp;
#pragma unroll
        for (int i = k + 1; i < 9; ++i) {
            if (!in_band(i, k)) continue;
            const R l = M[i][k] * rp;
            M[i][k] = l;
#pragma unroll
            for (int j = k + 1; j < 9; ++j) {
                if (!in_band(k, j) || !in_band(i, j)) continue;
                M[i][j] -= l * M[k][j];
            }
        }
    }
}

// Solve L U z = b in place (b -> z).
template <typename R>
__device__ __forceinline__ void lu_band_solve(const R (&M)[9][9], R (&b)[9]) {
#pragma unroll
    for (int i = 1; i < 9; ++i)
#pragma unroll
        for (int c = 0; c < i; ++c)
            if (in_band(i, c)) b[i] -= M[i][c] * b[c];
#pragma unroll
    for (int i = 8; i >= 0; --i) {
#pragma unroll
        for (int c = i + 1; c < 9; ++c)
            if (in_band(i, c)) b[i] -= M[i][c] * b[c];
        b[i] = b[i] * M[i][i];
    }
}

}  // namespace

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
        if (!isfinite(x[a])) latch_error(err, NMODL_ERR_NONFINITE);
        st[a * stride + i] = x[a];
    }
}

// ---------------------------------------------------------------- state

// One thread per instance (or per entry of the first *n_list_dev of list).  ni == nullptr means instance i reads v[i]; dt_arr != nullptr gives
// each instance its own step (used to generate training pairs).
// Rate constants of one launch, folded on the host and passed by value.
// With one dt for all instances dt k = exp(b v + ln(dt a)): one multiply-add
// and the exp (FP64: lnc = ln(dt af), ln(dt ab); MIXED: kf = bf, bb, then
// ln(dt af), ln(dt ab) in FP32).  With a dt per instance (training pairs)
// MIXED keeps af, ab in kf and scales by dt.  FP32 copies are made on the
// host because FP64 -> FP32 conversions run on the FP64 pipe.
struct Kin9Launch {
    double lnc[2 * kKinEdges];
    float kf[4 * kKinEdges];
};

template <int PREC, bool LIST>
__global__ void __launch_bounds__(128)
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
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n_work) {
        int iters = 0;
        bool nonconv = false;
        const int64_t i = LIST ? (int64_t)list[t] : t;
        const Kin9D& K = *kd;
        const double vv = ni ? v[ni[i]] : v[i];
        const double dt = dt_arr ? dt_arr[i] : dt_scalar;
        double x[9], y[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            x[a] = st[a * stride + i];
            y[a] = x[a];
        }
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
            double diag[9];
#pragma unroll
            for (int a = 0; a < 9; ++a) diag[a] = 1.0;
#pragma unroll
            for (int e = 0; e < kKinEdges; ++e) {
                diag[edge_lo(e)] += dk_f[e];
                diag[edge_hi(e)] += dk_b[e];
            }
            double M[9][9];
#pragma unroll
            for (int a = 0; a < 9; ++a)
#pragma unroll
                for (int b = 0; b < 9; ++b)
                    if (in_band(a, b)) M[a][b] = (a == b) ? diag[a] : 0.0;
#pragma unroll
            for (int e = 0; e < kKinEdges; ++e) {
                M[edge_hi(e)][edge_lo(e)] = -dk_f[e];
                M[edge_lo(e)][edge_hi(e)] = -dk_b[e];
            }
            lu_band(M);
            while (iters < max_iter) {
                // r = -(J y - x)
                double r[9];
#pragma unroll
                for (int a = 0; a < 9; ++a) r[a] = x[a] - diag[a] * y[a];
#pragma unroll
                for (int e = 0; e < kKinEdges; ++e) {
                    r[edge_hi(e)] += dk_f[e] * y[edge_lo(e)];
                    r[edge_lo(e)] += dk_b[e] * y[edge_hi(e)];
                }
                lu_band_solve(M, r);
                double dmax = 0.0;
#pragma unroll
                for (int a = 0; a < 9; ++a) {
                    y[a] += r[a];
                    dmax = fmax(dmax, fabs(r[a]));
                }
                ++iters;
                if (dmax <= tol) break;
                if (iters == max_iter) nonconv = true;
            }
        } else {
            float dk_f[kKinEdges], dk_b[kKinEdges];
            const float vf = d2f_int(vv);
            if (dt_arr) {
                const float dtf = d2f_int(dt);
#pragma unroll
                for (int e = 0; e < kKinEdges; ++e) {
                    dk_f[e] = dtf * (kf_s[2 * kKinEdges + e] * __expf(kf_s[e] * vf));
                    dk_b[e] = dtf * (kf_s[3 * kKinEdges + e] * __expf(-kf_s[kKinEdges + e] * vf));
                }
            } else {
#pragma unroll
                for (int e = 0; e < kKinEdges; ++e) {
                    dk_f[e] = __expf(fmaf(kf_s[e], vf, kf_s[2 * kKinEdges + e]));
                    dk_b[e] = __expf(fmaf(-kf_s[kKinEdges + e], vf, kf_s[3 * kKinEdges + e]));
                }
            }
            // FP64 copies of the FP32 rates (exact, integer pipe), and the
            // FP64 diagonal from them: columns of J sum to 1
            double dkd_f[kKinEdges], dkd_b[kKinEdges], diag[9];
#pragma unroll
            for (int e = 0; e < kKinEdges; ++e) {
                dkd_f[e] = f2d_int(dk_f[e]);
                dkd_b[e] = f2d_int(dk_b[e]);
            }
#pragma unroll
            for (int a = 0; a < 9; ++a) diag[a] = 1.0;
#pragma unroll
            for (int e = 0; e < kKinEdges; ++e) {
                diag[edge_lo(e)] += dkd_f[e];
                diag[edge_hi(e)] += dkd_b[e];
            }
            float M[9][9];
#pragma unroll
            for (int a = 0; a < 9; ++a)
#pragma unroll
                for (int b = 0; b < 9; ++b)
                    if (in_band(a, b)) M[a][b] = (a == b) ? d2f_int(diag[a]) : 0.0f;
#pragma unroll
            for (int e = 0; e < kKinEdges; ++e) {
                M[edge_hi(e)][edge_lo(e)] = -dk_f[e];
                M[edge_lo(e)][edge_hi(e)] = -dk_b[e];
            }
            lu_band(M);
            const int cap = 1 + ir_max;
            while (iters < cap) {
                double r[9];
#pragma unroll
                for (int a = 0; a < 9; ++a) r[a] = x[a] - diag[a] * y[a];
#pragma unroll
                for (int e = 0; e < kKinEdges; ++e) {
                    r[edge_hi(e)] += dkd_f[e] * y[edge_lo(e)];
                    r[edge_lo(e)] += dkd_b[e] * y[edge_hi(e)];
                }
                float rf[9];
#pragma unroll
                for (int a = 0; a < 9; ++a) rf[a] = d2f_int(r[a]);
                lu_band_solve(M, rf);
                float dmax = 0.0f;
#pragma unroll
                for (int a = 0; a < 9; ++a) {
                    y[a] += f2d_int(rf[a]);
                    dmax = fmaxf(dmax, fabsf(rf[a]));
                }
                ++iters;
                if (f2d_int(dmax) <= tol) break;
                if (iters == cap) nonconv = true;
            }
        }
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            if (!isfinite(y[a])) latch_error(err, NMODL_ERR_NONFINITE);
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
    const int grid = (int)((work + block - 1) / block);
    Kin9Launch KL;
    for (int e = 0; e < kKinEdges; ++e) {
        const double cf = dt_arr ? 0.0 : std::log(dt * kh.af[e]);
        const double cb = dt_arr ? 0.0 : std::log(dt * kh.ab[e]);
        KL.lnc[e] = cf;
        KL.lnc[kKinEdges + e] = cb;
        KL.kf[e] = (float)kh.bf[e];
        KL.kf[kKinEdges + e] = (float)kh.bb[e];
        KL.kf[2 * kKinEdges + e] = (float)(dt_arr ? kh.af[e] : cf);
        KL.kf[3 * kKinEdges + e] = (float)(dt_arr ? kh.ab[e] : cb);
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
