// kin9.cuh -- the implicit-Euler Newton solve of the 9-state kinetic scheme
// for one instance in one thread, shared by the standalone state kernel
// (k_kin9.cu) and the fused tile kernel (k_cnexp.cu).
//
// The KINETIC scheme is the linear ODE x' = A(v) x (Section 5.1); one
// implicit Euler step solves F(y) = y - x - dt A y = 0 by Newton iteration
// with the exact Jacobian J = I - dt A (Section 5.2 derivimplicit, Section
// 5.3 Newton + LU).  J is a nonsingular M-matrix whose columns sum to one
// (columns of -dt A sum to 0), so LU with partial pivoting makes no row
// interchanges and the no-pivot LU below performs the same eliminations.
// States are numbered 3a+b on a 3x3 lattice whose edges join indices
// differing by 1 (same row) or 3, so J and its LU factors live inside the
// band |i - j| <= 3; every loop is unrolled at compile time and only band
// entries are ever touched.
//
// Inputs are the 24 rates already multiplied by dt (dk_f forward, dk_b
// backward, per edge).  FP64 form: J, LU, residual and update in double.
// MIXED form: J and its LU in FP32; the residual F(y) = J y - x (with J's
// diagonal rebuilt in FP64 from the FP32 rates, so that its columns keep
// summing exactly to one) and the update of y in FP64; the FP32 factors
// refine y until max|delta| <= tol or cap updates.
#pragma once

#include "nmodl_internal.cuh"

namespace nmodl {

__host__ __device__ constexpr bool kin9_in_band(int i, int j) {
    return (i - j <= 3) && (j - i <= 3);
}

// pivot reciprocal: the refined hardware reciprocal in FP64, IEEE in FP32
__device__ __forceinline__ double kin9_recip(double x) { return rcp_fast(x); }
__device__ __forceinline__ float kin9_recip(float x) { return 1.0f / x; }

// In-place no-pivot LU of the banded 9x9 matrix M (only band entries used);
// the diagonal is replaced by the reciprocals of the pivots, so that the
// triangular solves multiply instead of divide.
template <typename R>
__device__ __forceinline__ void kin9_lu_band(R (&M)[9][9]) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const R rp = kin9_recip(M[k][k]);
        M[k][k] = rp;
#pragma unroll
        for (int i = k + 1; i < 9; ++i) {
            if (!kin9_in_band(i, k)) continue;
            const R l = M[i][k] * rp;
            M[i][k] = l;
#pragma unroll
            for (int j = k + 1; j < 9; ++j) {
                if (!kin9_in_band(k, j) || !kin9_in_band(i, j)) continue;
                M[i][j] -= l * M[k][j];
            }
        }
    }
}

// Solve L U z = b in place (b -> z).
template <typename R>
__device__ __forceinline__ void kin9_lu_band_solve(const R (&M)[9][9], R (&b)[9]) {
#pragma unroll
    for (int i = 1; i < 9; ++i)
#pragma unroll
        for (int c = 0; c < i; ++c)
            if (kin9_in_band(i, c)) b[i] -= M[i][c] * b[c];
#pragma unroll
    for (int i = 8; i >= 0; --i) {
#pragma unroll
        for (int c = i + 1; c < 9; ++c)
            if (kin9_in_band(i, c)) b[i] -= M[i][c] * b[c];
        b[i] = b[i] * M[i][i];
    }
}

// FP64 Newton from y = x: at most max_iter updates, stopping when
// max|delta| <= tol; returns the number of updates, nonconv when the cap
// was reached without meeting tol.
__device__ __forceinline__ int kin9_newton_d(const double (&dk_f)[kKinEdges],
                                             const double (&dk_b)[kKinEdges],
                                             const double (&x)[9], double (&y)[9], double tol,
                                             int max_iter, bool& nonconv) {
    nonconv = false;
#pragma unroll
    for (int a = 0; a < 9; ++a) y[a] = x[a];
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
            if (kin9_in_band(a, b)) M[a][b] = (a == b) ? diag[a] : 0.0;
#pragma unroll
    for (int e = 0; e < kKinEdges; ++e) {
        M[edge_hi(e)][edge_lo(e)] = -dk_f[e];
        M[edge_lo(e)][edge_hi(e)] = -dk_b[e];
    }
    kin9_lu_band(M);
    int iters = 0;
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
        kin9_lu_band_solve(M, r);
        // max|delta| and its test on the integer pipe
        unsigned long long dmax = 0;
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            y[a] += r[a];
            dmax = absmax_bits(dmax, r[a]);
        }
        ++iters;
        if (bits_le(dmax, tol)) break;
        if (iters == max_iter) nonconv = true;
    }
    return iters;
}

// MIXED: FP32 rates and LU, the residual to about 48 bits and the update in
// FP64; at most cap updates (the first solve and cap - 1 refinements).
// The residual x - J y = (x - y) - out .* y + (inflows), out_a the column's
// outflow rates (J's diagonal minus 1): x - y in FP64 (one subtraction per
// state, exact enough for the small increment), the rate products and sums
// as float pairs on the FP32 pipe from y split to 47 bits -- the same split
// y_a in column a's outflow and in the inflows it feeds, so that the sum of
// the residual stays the sum of x - y and the scheme keeps conserving to
// FP64 rounding.  (All in FP64 the residual took 57 FP64 instructions per
// refinement and the diagonal 48 per solve, the whole step's FP64 bound.)
__device__ __forceinline__ int kin9_refine_mixed(const float (&dk_f)[kKinEdges],
                                                 const float (&dk_b)[kKinEdges],
                                                 const double (&x)[9], double (&y)[9], double tol,
                                                 int cap, bool& nonconv) {
    nonconv = false;
#pragma unroll
    for (int a = 0; a < 9; ++a) y[a] = x[a];
    // each column's outflow as a float pair (TwoSum of the FP32 rates)
    ff2 out[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) out[a] = ff2{0.0f, 0.0f};
#pragma unroll
    for (int e = 0; e < kKinEdges; ++e) {
        out[edge_lo(e)] = ff_add(out[edge_lo(e)], ff2{dk_f[e], 0.0f});
        out[edge_hi(e)] = ff_add(out[edge_hi(e)], ff2{dk_b[e], 0.0f});
    }
    float M[9][9];
#pragma unroll
    for (int a = 0; a < 9; ++a)
#pragma unroll
        for (int b = 0; b < 9; ++b)
            if (kin9_in_band(a, b)) M[a][b] = (a == b) ? (1.0f + out[a].h) + out[a].l : 0.0f;
#pragma unroll
    for (int e = 0; e < kKinEdges; ++e) {
        M[edge_hi(e)][edge_lo(e)] = -dk_f[e];
        M[edge_lo(e)][edge_hi(e)] = -dk_b[e];
    }
    kin9_lu_band(M);
    // a float times a pair, renormalised
    auto mul_fp = [](float s, ff2 b) {
        const float p = __fmul_rn(s, b.h);
        return ff_renorm(p, fmaf(s, b.l, fmaf(s, b.h, -p)));
    };
    int iters = 0;
    while (iters < cap) {
        ff2 yp[9], r[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            yp[a] = ff_of(y[a]);
            r[a] = ff_sub(ff_of(x[a] - y[a]), ff_mul(out[a], yp[a]));
        }
#pragma unroll
        for (int e = 0; e < kKinEdges; ++e) {
            r[edge_hi(e)] = ff_add(r[edge_hi(e)], mul_fp(dk_f[e], yp[edge_lo(e)]));
            r[edge_lo(e)] = ff_add(r[edge_lo(e)], mul_fp(dk_b[e], yp[edge_hi(e)]));
        }
        float rf[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) rf[a] = r[a].h + r[a].l;
        kin9_lu_band_solve(M, rf);
        float dmax = 0.0f;
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            y[a] += f2d_int(rf[a]);
            dmax = fmaxf(dmax, fabsf(rf[a]));
        }
        ++iters;
        if (abs_le_int(f2d_int(dmax), tol)) break;
        if (iters == cap) nonconv = true;
    }
    return iters;
}

}  // namespace nmodl
