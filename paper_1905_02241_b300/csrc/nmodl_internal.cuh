// nmodl_internal.cuh -- device descriptors and per-instance math shared by
// the kernels of libnmodl_b300.so (sm_103a).
//
// Gate rates use u = (v - vh) * (1/k) with three shapes (EXP, SIGMOID,
// LINOID); the Hodgkin-Huxley gates are mapped onto these shapes at create
// time.  A gate step is the cnexp update of Section 5.2: with
// s = alpha + beta, minf = alpha/s and dt/mtau = phi*dt*s,
//     m <- m + (1 - exp(-phi*dt*s)) * (minf - m).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nmodl_b300.h"

namespace nmodl {

constexpr int kMaxGates = 3;
constexpr int kMaxMechsFused = 16;
constexpr int kKinStates = 9;
constexpr int kKinEdges = 12;

enum RateForm : int32_t { kExp = 0, kSigmoid = 1, kLinoid = 2 };

struct GateD {
    double aA, avh, ark;  // alpha: A [1/ms], vh [mV], 1/k [1/mV]
    double bA, bvh, brk;  // beta
    int32_t aform, bform, power, pad;
};

// Device descriptor of one HH / CNEXP mechanism (staged in shared memory).
struct MechD {
    int32_t kind;     // NMODL_HH or NMODL_CNEXP
    int32_t n_gates;  // 3 for HH
    double phi;       // temperature factor
    double gbar, e;   // CNEXP single current
    double hh_g[3];   // HH gnabar, gkbar, gl
    double hh_e[3];   // HH ena, ek, el
    GateD gate[kMaxGates];
};

// Edge e of the 3x3 kinetic lattice joins state lo(e) and hi(e): edges
// 0..5 are horizontal (3a+b, 3a+b+1), edges 6..11 vertical (k, k+3).
__host__ __device__ constexpr int edge_lo(int e) {
    return e < 6 ? 3 * (e / 2) + (e % 2) : e - 6;
}
__host__ __device__ constexpr int edge_hi(int e) {
    return e < 6 ? edge_lo(e) + 1 : edge_lo(e) + 3;
}

struct Kin9D {
    double gbar, e;
    int32_t open, pad;
    double af[kKinEdges], bf[kKinEdges], ab[kKinEdges], bb[kKinEdges];
};

// ------------------------------------------------------------ FP64 math

__device__ __forceinline__ double rate_d(int form, double A, double vh,
                                         double rk, double v) {
    const double u = (v - vh) * rk;
    if (form == kExp) return A * exp(u);
    if (form == kSigmoid) return A / (1.0 + exp(-u));
    // LINOID: A u / (1 - exp(-u)); series 1 + u/2 + u^2/12 near u = 0
    if (fabs(u) < 1e-6) return A * (1.0 + u * (0.5 + u * (1.0 / 12.0)));
    return A * u / (-expm1(-u));
}

__device__ __forceinline__ double gate_step_d(const GateD& G, double phidt,
                                              double v, double m) {
    const double a = rate_d(G.aform, G.aA, G.avh, G.ark, v);
    const double b = rate_d(G.bform, G.bA, G.bvh, G.brk, v);
    const double s = a + b;
    const double minf = a / s;
    const double f = 1.0 - exp(-phidt * s);
    return m + f * (minf - m);
}

__device__ __forceinline__ double gate_inf_d(const GateD& G, double v) {
    const double a = rate_d(G.aform, G.aA, G.avh, G.ark, v);
    const double b = rate_d(G.bform, G.bA, G.bvh, G.brk, v);
    return a / (a + b);
}

__device__ __forceinline__ double ipow_d(double x, int p) {
    double r = 1.0;
    for (int k = 0; k < p; ++k) r *= x;
    return r;
}

// ------------------------------------------------------------ FP32 math
// Rates and the cnexp factor in single precision.  exp uses the hardware
// exp2 unit through __expf; the two cancelling differences (1 - exp(-u) in
// LINOID and 1 - exp(-x) in cnexp) switch to their Taylor series where the
// series is more accurate than the subtraction.

__device__ __forceinline__ float rate_f(int form, float A, float vh, float rk,
                                        float v) {
    const float u = (v - vh) * rk;
    if (form == kExp) return A * __expf(u);
    if (form == kSigmoid) return __fdividef(A, 1.0f + __expf(-u));
    // u/(1-e^-u) = 1 + u/2 + u^2/12 - u^4/720 + ...
    if (fabsf(u) < 0.1f) {
        const float u2 = u * u;
        return A * (1.0f + 0.5f * u + u2 * (1.0f / 12.0f - u2 * (1.0f / 720.0f)));
    }
    return __fdividef(A * u, 1.0f - __expf(-u));
}

// 1 - exp(-x) for x >= 0
__device__ __forceinline__ float one_minus_expneg_f(float x) {
    if (x < 0.1f) {
        // x - x^2/2 + x^3/6 - x^4/24 + x^5/120
        return x * (1.0f - x * (0.5f - x * (1.0f / 6.0f - x * (1.0f / 24.0f - x * (1.0f / 120.0f)))));
    }
    return 1.0f - __expf(-x);
}

struct GateF {
    float aA, avh, ark, bA, bvh, brk;
    int32_t aform, bform;
};

// (minf, 1 - exp(-dt/mtau)) of a gate in FP32
__device__ __forceinline__ void gate_coef_f(const GateF& G, float phidt, float v,
                                            float& minf, float& f) {
    const float a = rate_f(G.aform, G.aA, G.avh, G.ark, v);
    const float b = rate_f(G.bform, G.bA, G.bvh, G.brk, v);
    const float s = a + b;
    minf = __fdividef(a, s);
    f = one_minus_expneg_f(phidt * s);
}

// Knuth TwoSum: s + err == a + b exactly.
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& err) {
    s = a + b;
    const float bp = s - a;
    err = (a - (s - bp)) + (b - bp);
}

__device__ __forceinline__ void latch_error(int32_t* err, int32_t code) {
    if (err) atomicCAS(err, 0, code);
}

}  // namespace nmodl
