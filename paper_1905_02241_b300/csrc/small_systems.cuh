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

// Gaussian elimination of the 3x3 system, written out: M y = b.
template <typename R>
__device__ __forceinline__ void solve3(const R (&M)[3][3], R (&b)[3]) {
    const R r0 = R(1) / M[0][0];
    const R l10 = M[1][0] * r0, l20 = M[2][0] * r0;
    const R u11 = M[1][1] - l10 * M[0][1], u12 = M[1][2] - l10 * M[0][2];
    const R s21 = M[2][1] - l20 * M[0][1], s22 = M[2][2] - l20 * M[0][2];
    const R r1 = R(1) / u11;
    const R l21 = s21 * r1;
    const R u22 = s22 - l21 * u12;
    const R z1 = b[1] - l10 * b[0];
    const R z2 = b[2] - l20 * b[0] - l21 * z1;
    b[2] = z2 / u22;
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
// delta = J^-1 (-F) by the adjugate over the determinant; stops when both
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
        const double rdet = 1.0 / fma(a, d, -b * c);
        const double d0 = fma(d, r0, -b * r1) * rdet;
        const double d1 = fma(a, r1, -c * r0) * rdet;
        y0 += d0;
        y1 += d1;
        ++it;
        if (fabs(d0) <= tol && fabs(d1) <= tol) {
            conv = true;
            break;
        }
    }
    return it;
}

}  // namespace nmodl
