// small_systems.cuh -- per-instance math of the small systems (3-state
// kinetic scheme, calcium buffer), shared by their standalone kernels and
// the fused tile kernel.
#pragma once

#include "nmodl_internal.cuh"

namespace nmodl {

// rates of the three edges at v: kf[e] (lo -> hi) and kb[e] (hi -> lo)
__device__ __forceinline__ void kin3_rates_d(const Kin3D& K, double v, double (&kf)[3],
                                             double (&kb)[3]) {
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        kf[e] = K.af[e] * exp_tang(K.bf[e] * v);
        kb[e] = K.ab[e] * exp_tang(-K.bb[e] * v);
    }
}

// Row-major M = I - dt A from the edge rates: off-diagonals -dt k, the
// diagonal 1 + dt (outflow of the state).
template <typename R>
__device__ __forceinline__ void kin3_matrix(const R (&kf)[3], const R (&kb)[3], R dt,
                                            R (&M)[3][3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) M[a][b] = (a == b) ? R(1) : R(0);
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const int lo = kin3_lo(e), hi = kin3_hi(e);
        M[hi][lo] = -dt * kf[e];
        M[lo][hi] = -dt * kb[e];
        M[lo][lo] += dt * kf[e];
        M[hi][hi] += dt * kb[e];
    }
}

// reciprocal of a pivot: the refined hardware reciprocal in FP64 (within
// one ulp; IEEE division is a long sequence on the FP64 pipe), IEEE in FP32
__device__ __forceinline__ double pivot_rcp(double x) { return rcp_fast(x); }
__device__ __forceinline__ float pivot_rcp(float x) { return 1.0f / x; }

// Gaussian elimination of the 3x3 system, written out: M y = b.
template <typename R>
__device__ __forceinline__ void solve3(const R (&M)[3][3], R (&b)[3]) {
    const R r0 = pivot_rcp(M[0][0]);
    const R l10 = M[1][0] * r0, l20 = M[2][0] * r0;
    const R u11 = M[1][1] - l10 * M[0][1], u12 = M[1][2] - l10 * M[0][2];
    const R s21 = M[2][1] - l20 * M[0][1], s22 = M[2][2] - l20 * M[0][2];
    const R r1 = pivot_rcp(u11);
    const R l21 = s21 * r1;
    const R u22 = s22 - l21 * u12;
    const R z1 = b[1] - l10 * b[0];
    const R z2 = b[2] - l20 * b[0] - l21 * z1;
    b[2] = z2 * pivot_rcp(u22);
    b[1] = (z1 - u12 * b[2]) * r1;
    b[0] = (b[0] - M[0][1] * b[1] - M[0][2] * b[2]) * r0;
}


// One implicit Euler step of the 3-state scheme in FP64: for a linear scheme
// the first Newton update from y = x is the solution, (I - dt A) y = x.
__device__ __forceinline__ void kin3_step_d(const Kin3D& K, double v, double dt,
                                            double (&x)[3]) {
    double kf[3], kb[3], M[3][3];
    kin3_rates_d(K, v, kf, kb);
    kin3_matrix(kf, kb, dt, M);
    solve3(M, x);
}

// Calcium buffer: Newton on F(y) = y - x - dt f(y) with J = I - dt df/dy,
//   J = [[1 + dt (kf (btot - y1) + 1/tau), -dt (kf y0 + kb)],
//        [-dt kf (btot - y1),               1 + dt (kf y0 + kb)]]
// delta = J^-1 (-F) by the adjugate times the (refined hardware) reciprocal
// of the determinant; stops when both
// |delta| <= tol (conv = true) or after max_iter updates.  (y0, y1) enter
// as x and leave as the step's result; returns the number of updates.
__device__ __forceinline__ int cacum_newton_d(const CacumD& C, double ica, double dt,
                                              double tol, int max_iter, double& y0,
                                              double& y1, bool& conv) {
    const double x0 = y0, x1 = y1;
    const double src = C.rtau * C.cai0 - C.k * ica;  // constant part of f0
    int it = 0;
    conv = false;
    while (it < max_iter) {
        const double fr = C.btot - y1;
        const double on = C.kf * fr, off = fma(C.kf, y0, C.kb);
        const double bind = fma(on, y0, -C.kb * y1);
        const double f0 = src - bind - C.rtau * y0;
        const double r0 = fma(dt, f0, x0 - y0);
        const double r1 = fma(dt, bind, x1 - y1);
        const double a = fma(dt, on + C.rtau, 1.0), b = -dt * off;
        const double c = -dt * on, d = fma(dt, off, 1.0);
        const double rdet = rcp_fast(fma(a, d, -b * c));
        const double d0 = fma(d, r0, -b * r1) * rdet;
        const double d1 = fma(a, r1, -c * r0) * rdet;
        y0 += d0;
        y1 += d1;
        ++it;
        if (abs_le_int(d0, tol) && abs_le_int(d1, tol)) {  // integer pipe
            conv = true;
            break;
        }
    }
    return it;
}

// ------------------------------------------------------------ mixed forms
// Rates, matrices and eliminations in FP32; the residual and the
// refinement of the result in FP64 (conversions on the integer pipe).

// FP32 copies of the parameters, made once per launch or tile (Kin3F: the
// exponents' b scaled by log2(e) for the exp2 unit)
struct Kin3F {
    float af[3], bf[3], ab[3], bb[3];
};
struct CacumF {
    float k, rtau, cai0, kf, kb, btot;
};

// 3-state step: FP32 rates and elimination, then iterative refinement with
// the FP64 residual x - J y (J's diagonal rebuilt in FP64 from the FP32
// off-diagonals so that its columns sum to one) until max|delta| <= tol or
// ir_max refinements.  Returns the number of updates; nonconv when ir_max
// refinements did not reach tol.
__device__ __forceinline__ int kin3_step_mixed(const Kin3F& K, float vf, float dtf, double tol,
                                               int ir_max, double (&x)[3], bool& nonconv) {
    float kf[3], kb[3], M[3][3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        kf[e] = K.af[e] * ex2_hw(K.bf[e] * vf);
        kb[e] = K.ab[e] * ex2_hw(-K.bb[e] * vf);
    }
    kin3_matrix(kf, kb, dtf, M);
    // The refinement's residual x - J y = (x - y) - out .* y - off y (off:
    // J's off-diagonals, out_b = -sum_a off[a][b] the column's outflow, J's
    // diagonal minus 1): x - y in FP64, the rest as float pairs on the FP32
    // pipe from y split to 47 bits (the same split y_b in column b's outflow
    // and in its off-diagonal terms, so the residual's sum stays that of
    // x - y and the scheme conserves to FP64 rounding)
    ff2 out[3] = {ff2{0.f, 0.f}, ff2{0.f, 0.f}, ff2{0.f, 0.f}};
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (a != b) out[b] = ff_sub(out[b], ff2{M[a][b], 0.f});
    float yf[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) yf[a] = d2f_int(x[a]);
    solve3(M, yf);
    double y[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) y[a] = f2d_int(yf[a]);
    int iters = 1;
    bool done = false;
    for (int k = 0; k < ir_max && !done; ++k) {
        ff2 yp[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) yp[a] = ff_of(y[a]);
        float r[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            ff2 ra = ff_sub(ff_of(x[a] - y[a]), ff_mul(out[a], yp[a]));
#pragma unroll
            for (int b = 0; b < 3; ++b)
                if (b != a) {
                    const float p = __fmul_rn(M[a][b], yp[b].h);
                    ra = ff_sub(ra, ff_renorm(p, fmaf(M[a][b], yp[b].l, fmaf(M[a][b], yp[b].h, -p))));
                }
            r[a] = ra.h + ra.l;
        }
        solve3(M, r);
        float dmax = 0.0f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            y[a] += f2d_int(r[a]);
            dmax = fmaxf(dmax, fabsf(r[a]));
        }
        ++iters;
        done = abs_le_int(f2d_int(dmax), tol);
    }
    nonconv = !done && ir_max > 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) x[a] = y[a];
    return iters;
}

// The calcium buffer's implicit Euler step, mixed: the Newton updates of
// cacum_newton_d in FP32 until an update no longer changes y (or max_iter),
// then refinements with the FP64 residual F(y), solved through the FP32
// Jacobian at y, until both |delta| <= tol (conv) or ir_max refinements.
// Returns the number of updates (FP32 and refinements).
__device__ __forceinline__ int cacum_newton_mixed(const CacumD& C, const CacumF& F, double ica,
                                                  double dt, double tol, int max_iter,
                                                  int ir_max, double& y0, double& y1,
                                                  bool& conv) {
    const double x0 = y0, x1 = y1;
    const float dtf = d2f_int(dt);
    // 2x2 Jacobian of F at (z0, z1) in FP32, inverted by the adjugate
    auto jac_inv = [&](float z0, float z1, float& a, float& b, float& c, float& d) {
        const float on = F.kf * (F.btot - z1), off = fmaf(F.kf, z0, F.kb);
        a = fmaf(dtf, on + F.rtau, 1.0f);
        b = -dtf * off;
        c = -dtf * on;
        d = fmaf(dtf, off, 1.0f);
        const float rdet = 1.0f / fmaf(a, d, -b * c);
        a *= rdet; b *= rdet; c *= rdet; d *= rdet;
    };
    float z0 = d2f_int(y0), z1 = d2f_int(y1);
    const float x0f = z0, x1f = z1;
    const float srcf = F.rtau * F.cai0 - F.k * d2f_int(ica);
    int it = 0;
    while (it < max_iter) {
        const float fr = F.btot - z1;
        const float on = F.kf * fr;
        const float bind = fmaf(on, z0, -F.kb * z1);
        const float f0 = srcf - bind - F.rtau * z0;
        const float r0 = fmaf(dtf, f0, x0f - z0), r1 = fmaf(dtf, bind, x1f - z1);
        float a, b, c, d;
        jac_inv(z0, z1, a, b, c, d);
        const float d0 = fmaf(d, r0, -b * r1), d1 = fmaf(a, r1, -c * r0);
        ++it;
        const bool still = (z0 + d0 != z0) || (z1 + d1 != z1);
        z0 += d0;
        z1 += d1;
        if (!still) break;
    }
    y0 = f2d_int(z0);
    y1 = f2d_int(z1);
    conv = false;
    const double src = C.rtau * C.cai0 - C.k * ica;
    for (int k = 0; k < ir_max; ++k) {
        const double fr = C.btot - y1;
        const double on = C.kf * fr;
        const double bind = fma(on, y0, -C.kb * y1);
        const double f0 = src - bind - C.rtau * y0;
        const float r0 = d2f_int(fma(dt, f0, x0 - y0)), r1 = d2f_int(fma(dt, bind, x1 - y1));
        float a, b, c, d;
        jac_inv(d2f_int(y0), d2f_int(y1), a, b, c, d);
        const float d0 = fmaf(d, r0, -b * r1), d1 = fmaf(a, r1, -c * r0);
        y0 += f2d_int(d0);
        y1 += f2d_int(d1);
        ++it;
        if (abs_le_int(f2d_int(d0), tol) && abs_le_int(f2d_int(d1), tol)) {
            conv = true;
            break;
        }
    }
    return it;
}

}  // namespace nmodl
