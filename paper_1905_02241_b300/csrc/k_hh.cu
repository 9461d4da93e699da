// k_hh.cu -- the time steps of one Hodgkin-Huxley mechanism with one
// instance on each node, for networks too small to fill the GPU (at most 32
// nodes per SM): one warp per gate.
//
// The FP64 unit of a B300 SM sub-partition takes one warp instruction
// about every 65 clocks, whatever the number of active lanes, and a
// dependent FP64 instruction waits about as long; independent FP64
// instructions of one warp do not overlap.  A network of a few thousand
// nodes gives each SM at most 32 nodes, so a step costs the length of its
// dependent chain, not the pipe's throughput.  The chain is cut three ways
// here: each block runs three warps, one per gate (m, h, n), on three
// sub-partitions, so that the three gate steps of a node run at the same
// time; each warp computes the node current itself from the three gates'
// exchanged factors (no second exchange for v); and the factors come
// folded by the producing warp (gnabar m^3; h; gk ek + gl el and
// gk + gl + cm/dt with gk = gkbar n^4), leaving the current update
//   gna = (gnabar m^3) h,  X = gna ena + (gk ek + gl el),
//   d = gna + (gk + gl + cm/dt),  v' = (v cm/dt + X) / d
// with five FP64 operations and one division.  v' equals v + rhs/d with
// rhs = X - v (gna + gk + gl) (Section 5.2's current form summed over the
// three currents, and the diagonal update), rounded differently.  One
// named barrier per step orders the exchange, double-buffered so that the
// next step's factors never overwrite ones still being read.
// Lanes past the block's nodes compute on node 0 and store nothing, so that
// every thread reaches every barrier.
#include <algorithm>

#include "kernels.cuh"

namespace nmodl {

__global__ void __launch_bounds__(96) k_hh_gate_warps(HhArgs A) {
    __shared__ double x_s[2][5][32];  // [buffer][factor][node of the block]
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t i0 = (int64_t)blockIdx.x * A.per_block + lane;
    const bool act = lane < A.per_block && i0 < A.n;
    const int64_t i = act ? i0 : 0;
    const GateD G = A.gate[w];
    const double gna_b = A.g[0], gk_b = A.g[1], gl = A.g[2];
    const double ena = A.e[0], ek = A.e[1], el = A.e[2];
    const double cmdt = 1e-3 * A.cm / A.dt;
    const double glel = gl * el, glc = gl + cmdt;
    double vv = A.v[i];
    double s = A.states[w * A.stride + i];
    // the factors of this warp's gate into buffer b; with_g: also
    // gk + gl, for the rhs of the last step
    auto produce = [&](int b, bool with_g) {
        if (w == 0) {
            x_s[b][0][lane] = gna_b * (s * s * s);
        } else if (w == 1) {
            x_s[b][1][lane] = s;
        } else {
            const double gk = gk_b * ((s * s) * (s * s));
            x_s[b][2][lane] = fma(gk, ek, glel);
            x_s[b][3][lane] = gk + glc;
            if (with_g) x_s[b][4][lane] = gk + gl;
        }
    };
    produce(0, A.nsteps == 1);
    asm volatile("bar.sync 1, 96;" ::: "memory");
    double X = 0.0, dd = 0.0, vold = vv;
    for (int k = 0; k < A.nsteps; ++k) {
        const int b = k & 1;
        const double gna = x_s[b][0][lane] * x_s[b][1][lane];
        X = fma(gna, ena, x_s[b][2][lane]);
        dd = gna + x_s[b][3][lane];
        vold = vv;
        if (!A.clamp_v) vv = ddiv_fast(fma(vv, cmdt, X), dd);
        if (k == A.nsteps - 1 && w == 0 && act) {
            // the last step's rhs and d (currents at the step's old v)
            A.rhs[i] = fma(-vold, gna + x_s[b][4][lane], X);
            A.d[i] = dd;
        }
        if (w == 1) s = gate_step_forms_d<kExp, kSigmoid, true>(G, 0.0, vv, s);
        else s = gate_step_forms_d<kLinoid, kExp, true>(G, 0.0, vv, s);
        produce(b ^ 1, k + 2 == A.nsteps);
        asm volatile("bar.sync 1, 96;" ::: "memory");
    }
    if (act) {
        if (!finite_int(s)) latch_error(A.err, NMODL_ERR_NONFINITE);
        A.states[w * A.stride + i] = s;
        if (w == 0) {
            if (!finite_int(vv)) latch_error(A.err, NMODL_ERR_NONFINITE);
            A.v[i] = vv;
        }
    }
}

int hh_warps_per_block(int64_t n, int sms) {
    const int64_t per = (n + sms - 1) / sms;
    return (int)std::max<int64_t>(1, std::min<int64_t>(32, per));
}

cudaError_t launch_hh_gate_warps(const HhArgs& a, cudaStream_t s) {
    if (a.n == 0 || a.nsteps == 0) return cudaSuccess;
    const int64_t grid = (a.n + a.per_block - 1) / a.per_block;
    k_hh_gate_warps<<<(unsigned)grid, 96, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace nmodl
