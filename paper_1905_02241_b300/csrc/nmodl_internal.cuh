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
#include "exp_tang_table.cuh"

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

// 3-state scheme: edge e in {0: (0,1), 1: (1,2), 2: (0,2)}
struct Kin3D {
    double gbar, e;
    int32_t open, pad;
    double af[3], bf[3], ab[3], bb[3];
};
__host__ __device__ constexpr int kin3_lo(int e) { return e == 1 ? 1 : 0; }
__host__ __device__ constexpr int kin3_hi(int e) { return e == 0 ? 1 : 2; }

// calcium buffer: k, 1/tau, cai0, kf, kb, btot
struct CacumD {
    double k, rtau, cai0, kf, kb, btot;
};

// Device descriptor of one mechanism of the fused step (staged in shared
// memory): HH, CNEXP, the small systems KIN3 and CACUM, and the current of
// NMODL_KIN9 (whose rate constants travel in a Kin9D).
struct MechD {
    int32_t kind;     // NMODL_HH, NMODL_CNEXP, NMODL_KIN3, NMODL_CACUM or NMODL_KIN9
    int32_t n_gates;  // states per instance (3 for HH)
    double phi;       // temperature factor
    double gbar, e;   // CNEXP single current
    double hh_g[3];   // HH gnabar, gkbar, gl
    double hh_e[3];   // HH ena, ek, el
    GateD gate[kMaxGates];
    int32_t ion;      // USEION WRITE tag of the whole current
    int32_t open;     // NMODL_KIN9: open state (gbar, e above hold its current)
    Kin3D k3;         // NMODL_KIN3
    CacumD cd;        // NMODL_CACUM
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

// Conversions between float and double on the integer pipe (the FP64 pipe
// of the B300 also executes the hardware conversions, at a low rate).
// float -> double is exact and handles every operand with integer
// operations (a subnormal float is a normal double; NaNs come out quiet);
// double -> float rounds to nearest even, and results that are zero,
// subnormal, infinite or NaN take the hardware conversion.
__device__ __forceinline__ double f2d_int(float x) {
    const unsigned f = __float_as_uint(x);
    const unsigned e = (f >> 23) & 0xffu, m = f & 0x7fffffu, s = f & 0x80000000u;
    if (e - 1u < 254u)
        return __hiloint2double((int)(s | ((e + (1023u - 127u)) << 20) | (m >> 3)), (int)(m << 29));
    if (e == 255u)  // infinity; NaN with the quiet bit set
        return __hiloint2double((int)(s | 0x7ff00000u | (m >> 3) | (m ? 0x80000u : 0u)),
                                (int)(m << 29));
    if (m == 0u) return __hiloint2double((int)s, 0);
    // subnormal m 2^-149: the leading one (bit p) becomes the implicit bit
    const int p = 31 - __clz((int)m);
    const unsigned long long b = ((unsigned long long)s << 32) |
                                 ((unsigned long long)(p + 874) << 52) |
                                 ((unsigned long long)(m ^ (1u << p)) << (52 - p));
    return __longlong_as_double((long long)b);
}
__device__ __forceinline__ float d2f_int(double d) {
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    const int e = (int)((hi >> 20) & 0x7ffu) - (1023 - 127);
    if (e >= 1 && e <= 254) {
        const unsigned m23 = ((hi & 0xfffffu) << 3) | (lo >> 29);
        const unsigned rem = lo & 0x1fffffffu;
        unsigned f = (hi & 0x80000000u) | ((unsigned)e << 23) | m23;
        if (rem > 0x10000000u || (rem == 0x10000000u && (m23 & 1u))) f += 1u;
        return __uint_as_float(f);
    }
    return (float)d;
}

// Knuth TwoSum: s + err == a + b exactly.
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& err) {
    s = a + b;
    const float bp = s - a;
    err = (a - (s - bp)) + (b - bp);
}

// ------------------------------------------------------------ FP64 math

// exp(x) by Tang's table-driven method (ACM TOMS 15(2), 1989): with
// N = 2048, n = round(N x / ln2) = N m + j and r = x - n ln2/N (two-constant
// Cody-Waite reduction, ln2/N = L1 + L2, |r| <= ln2/(2N) = 1.7e-4 up to the
// n choice below), exp(x) = 2^m 2^(j/N) (1 + p(r)), p(r) = r + r^2/2 +
// r^3/6 the degree-3 Taylor polynomial of exp(r) - 1 (truncation r^4/24 <
// 5.5e-17); error within 1.5 ulp (checked against mpmath on the GPU tests).
// The FP64 pipe of this GPU runs 1/64 of the FP32 rate and its issue slots
// are the scarce resource, so only 2 FP64 instructions remain:
//   r1 = x - n L1 (one fma, exact: L1 has 31 bits, |n| < 2^22), and
//   y  = T + T p (one fma).
// n is chosen in single precision from x split into two floats by integer
// operations (47 bits) times N/ln2 as a float pair with the product's exact
// error, so |x N/ln2 - n| <= 0.5 + 1e-7; n reaches FP64 as an exact
// integer-valued double by integer operations.  p (|p| < 1.8e-4) is needed
// to about 2^-42 of itself (its error enters y as T dp): it is formed as a
// normalized float pair (about 46 bits) from r1 split into two floats, n L2
// as a float pair and the products' exact errors, then widened to a double
// by integer operations.  2^m is applied to the exponent field; the 16 KB
// table stays in L1.
// x <= -708 returns 0 (the exact value is below 3.3e-308; this is the
// common case of the cnexp factor of very fast gates); x >= 708 and NaN go
// to the library exp.
// The rare arguments of exp_tang, out of line: a call boundary keeps their
// FP64 instructions out of the common path (not predicated into it).
static __device__ __noinline__ double exp_tang_rare(double x) {
    return (__double2hiint(x) < 0 && x == x) ? 0.0 : exp(x);
}
// An integer-valued float (normal or zero) as the equal double, integer
// operations only.
__device__ __forceinline__ double f2d_int_nz(float x) {
    const unsigned f = __float_as_uint(x), a = f & 0x7fffffffu;
    const unsigned hi = (f & 0x80000000u) | (a ? (a >> 3) + ((1023u - 127u) << 20) : 0u);
    return __hiloint2double((int)hi, (int)(f << 29));
}
// r = h + l to 47 bits (h: the leading 24 significand bits, l: the next 23),
// integer operations only; |r| < 2^-60 gives h = l = 0, |r| < 2^100 assumed.
__device__ __forceinline__ void split_d_ff(double r, float& h, float& l) {
    const unsigned hr = (unsigned)__double2hiint(r), lr = (unsigned)__double2loint(r);
    const unsigned ar = hr & 0x7fffffffu, sg = hr & 0x80000000u;
    h = __uint_as_float(__funnelshift_l(lr, ar - 0x38000000u, 3) | sg);
    // significand bits 6..28 of the low word, worth 2^(E - 1069) per unit
    const float m23 = __uint_as_float(0x4b000000u | ((lr >> 6) & 0x7fffffu)) - 8388608.0f;
    l = __uint_as_float(__float_as_uint(m23 * __uint_as_float(((ar >> 20) - 942u) << 23)) | sg);
    if (ar < 0x3c300000u) {
        h = 0.0f;
        l = 0.0f;
    }
}
// hi + lo as a double for a normalized float pair (|lo| <= ulp(hi)/2, hi
// normal or zero), integer operations only: hi's bits widened, then lo added
// in units of hi's double ulp, truncated toward zero (relative error below
// 2^-52 of the sum; a subnormal lo is dropped).  Where hi is a power of two
// and lo has the opposite sign, the sum lies in the binade below, whose ulp
// is half as large; otherwise |lo| <= ulp(hi)/2 keeps it in hi's binade, or
// carries into the exponent field exactly as the next binade requires.
__device__ __forceinline__ double ff2d_int(float hi, float lo) {
    const unsigned fh = __float_as_uint(hi), fl = __float_as_uint(lo);
    const unsigned ah = fh & 0x7fffffffu, al = fl & 0x7fffffffu;
    const int sh = (int)(al >> 23) - (int)(ah >> 23) + 29;  // <= 5
    const unsigned m = (al & 0x7fffffu) | 0x800000u;
    unsigned d = sh >= 0 ? m << sh : (sh > -24 ? m >> -sh : 0u);
    if ((al >> 23) == 0u) d = 0u;
    const bool opp = ((fh ^ fl) & 0x80000000u) != 0u;
    if (opp && (ah & 0x7fffffu) == 0u) d <<= 1;
    unsigned long long H = ((unsigned long long)((ah >> 3) + ((1023u - 127u) << 20)) << 32) |
                           (unsigned long long)(ah << 29);
    H = opp ? H - d : H + d;
    H |= (unsigned long long)(fh & 0x80000000u) << 32;
    return ah == 0u ? 0.0 : __longlong_as_double((long long)H);
}
// Float-pair arithmetic for dependent chains (the tree solve's levels): a
// value is h + l with |l| <= ulp(h)/2, about 46-48 significand bits in the
// FP32 exponent range, each operation a few FP32 instructions of 4-cycle
// latency where one FP64 instruction takes about 64 cycles on this GPU.
// Products keep the exact error of h h' from an fma; sums are TwoSum; each
// result is renormalised by a fast two-sum (|e| small against s, or s == 0).
struct ff2 {
    float h, l;
};
__device__ __forceinline__ ff2 ff_renorm(float s, float e) {
    const float h = s + e;
    return ff2{h, e - (h - s)};
}
__device__ __forceinline__ ff2 ff_of(double x) {  // to 47 bits (split_d_ff)
    ff2 r;
    split_d_ff(x, r.h, r.l);
    return r;
}
__device__ __forceinline__ ff2 ff_mul(ff2 a, ff2 b) {
    const float p = __fmul_rn(a.h, b.h);
    return ff_renorm(p, fmaf(a.h, b.l, fmaf(a.l, b.h, fmaf(a.h, b.h, -p))));
}
__device__ __forceinline__ ff2 ff_add(ff2 a, ff2 b) {
    float s, e;
    two_sum_f(a.h, b.h, s, e);
    return ff_renorm(s, e + (a.l + b.l));
}
__device__ __forceinline__ ff2 ff_sub(ff2 a, ff2 b) { return ff_add(a, ff2{-b.h, -b.l}); }
// 1/a: the correctly rounded FP32 reciprocal y of a.h and one Newton step
// y + y (1 - a y) (relative error about 2^-46)
__device__ __forceinline__ ff2 ff_rcp(ff2 a) {
    const float y = __frcp_rn(a.h);
    return ff_renorm(y, y * fmaf(-a.l, y, fmaf(-a.h, y, 1.0f)));
}

// ff2d_int, with a non-finite hi passed on as the equal double (an infinity,
// a quiet NaN) rather than widened as if finite, for sums whose non-finite
// values must reach the non-finite checks
__device__ __forceinline__ double ff2d_int_nf(float hi, float lo) {
    return (__float_as_uint(hi) & 0x7f800000u) == 0x7f800000u ? f2d_int(hi) : ff2d_int(hi, lo);
}
// e^x = 2^m T (1 + p) for |x| < 708: the table entry T, k (m = k >> kExpBits)
// and p, as described above.
__device__ __forceinline__ void exp_tang_core(double x, double& T, int& k, double& pr) {
    // x = xh + xl to 47 bits; x N/ln2 = kh + kl (kl: the product's exact
    // error, the low part of N/ln2 and xl's share); n = rint(kh), moved by
    // one where kh - n + kl passes +-1/2
    float xh, xl;
    split_d_ff(x, xh, xl);
    const float kh = __fmul_rn(xh, kExpInvLh);  // not contracted: kl holds its error
    const float kl = fmaf(xl, kExpInvLh, fmaf(xh, kExpInvLl, fmaf(xh, kExpInvLh, -kh)));
    const float t = kh + 0x1.8p23f;  // |kh| < 2^22: t's low bits hold rint(kh)
    const float nh = t - 0x1.8p23f;
    const float fr = (kh - nh) + kl;
    const int up = fr > 0.5f, dn = fr < -0.5f;
    k = (__float_as_int(t) - 0x4b400000) + up - dn;
    const float nf = nh + (up ? 1.0f : (dn ? -1.0f : 0.0f));
    const double r1 = fma(f2d_int_nz(nf), -kExpL1, x);
    // single-precision pairs: n L2 = a + ae, r = r1 - n L2 = R + Rl,
    // p = r + r^2/2 + r^3/6 = S + Sl (normalized), widened to a double
    float rh, rl;
    split_d_ff(r1, rh, rl);
    const float a = __fmul_rn(nf, kExpL2h);  // rounded products feed the TwoSums
    const float ae = fmaf(nf, kExpL2l, fmaf(nf, kExpL2h, -a));
    float R, Rl;
    two_sum_f(rh, -a, R, Rl);
    Rl += rl - ae;
    const float P = __fmul_rn(R, R);  // r^2 = P + Pe + 2 R Rl (+ Rl^2, below 2^-90)
    const float Pe = fmaf(R, R, -P);
    float S0, S0l, S, Sl;
    two_sum_f(R, 0.5f * P, S0, S0l);
    S0l += Rl + fmaf(0.5f, Pe, fmaf(R, Rl, (P * R) * (1.0f / 6.0f)));
    two_sum_f(S0, S0l, S, Sl);
    pr = ff2d_int(S, Sl);
    T = __ldg(&kExpTable[k & ((1 << kExpBits) - 1)]);
}
__device__ __forceinline__ double exp_tang(double x) {
    // |x| < 708 tested on the high word (integer pipe): 708 = 0x4086200000000000
    if (((unsigned)__double2hiint(x) & 0x7fffffffu) >= 0x40862000u) return exp_tang_rare(x);
    double T, pr;
    int k;
    exp_tang_core(x, T, k, pr);
    const double y = fma(T, pr, T);
    return __hiloint2double(__double2hiint(y) + ((k >> kExpBits) << 20), __double2loint(y));
}

// 1 + S e^x for S = +1 or -1 (the denominators of SIGMOID and LINOID
// rates) with one FP64 instruction after the exp's first: with e^x =
// 2^m T (1 + p), 1 + S e^x = S 2^m T p + C, C = 1 + S 2^m T formed by
// 64-bit integer operations on a common grid (exact, then rounded once to
// 53 bits; for m >= 53 the 1 is below half an ulp and C = S 2^m T).  Its
// error is within that of 1 + S exp_tang(x) (checked bit for bit on the
// CPU: 1.68 ulp worst for S = +1; for S = -1 the cancellation near x = 0
// amplifies e^x's own error alike).
template <int S>
static __device__ __noinline__ double one_pm_exp_rare(double x) {
    return 1.0 + (double)S * exp_tang_rare(x);
}
template <int S>
__device__ __forceinline__ double one_pm_exp(double x) {
    if (((unsigned)__double2hiint(x) & 0x7fffffffu) >= 0x40862000u) return one_pm_exp_rare<S>(x);
    double T, pr;
    int k;
    exp_tang_core(x, T, k, pr);
    const int m = k >> kExpBits;
    const long long Tb = __double_as_longlong(T);
    const double T2m = __longlong_as_double(Tb + ((long long)m << 52));
    double C;
    if (m >= 53) {
        C = S > 0 ? T2m : -T2m;
    } else {
        // grid 2^g, g = max(m - 52, -62): 1 = 2^-g, 2^m T = MT 2^(m - 52)
        const long long MT = (Tb & 0xfffffffffffffLL) | (1LL << 52);
        const int g = max(m - 52, -62);
        const int sh = max(0, -10 - m);
        const long long Tg = sh >= 63 ? 0LL : (MT >> sh);
        const long long one = 1LL << (-g);
        const long long Sv = S > 0 ? one + Tg : one - Tg;
        const unsigned long long A = (unsigned long long)(Sv < 0 ? -Sv : Sv);
        if (A == 0ULL) {
            C = 0.0;
        } else {
            const int lz = __clzll((long long)A);
            const int rs = 11 - lz;  // to a 53-bit significand, rounded half up
            const unsigned long long Ar = rs > 0 ? (A + (1ULL << (rs - 1))) >> rs : A << (-rs);
            const long long bits = ((long long)(63 - lz + g + 1022) << 52) + (long long)Ar;
            C = __longlong_as_double(Sv < 0 ? (bits | (long long)0x8000000000000000ULL) : bits);
        }
    }
    return fma(S > 0 ? T2m : -T2m, pr, C);
}

// 1/x with two FP64 instructions: a seed y0 good to about 2^-45 formed off
// the FP64 pipe, then one Newton step y = y0 + y0 e, e = 1 - x y0, whose
// result is within (1 + 2^-88) of 1/x before its one rounding, so within
// one ulp (exact at powers of two).  The seed: x's significand m = mh + ml
// split into two floats by integer operations, rh the FP32 hardware
// reciprocal of mh, d = 1 - m rh (the first product's residual is exact in
// an fma), 1/m = rh (1 + d + d^2 + ...) = rh + rh (d + d^2) as a float pair,
// widened to a double by integer operations and scaled by x's exponent
// (exponent field E in [1, 2043]).  Other x (zero, subnormals, |x| >=
// 2^1021, infinity, NaN) take the FP64 hardware seed and a third-order
// step, out of line: zero, infinity and subnormals then propagate as
// inf / 0 / NaN.
// 1/x for a dependent chain (the levels of a tree solve): the FP64
// hardware seed (relative error about 2^-22) and one third-order Newton
// step, 1/(1 - e) ~ 1 + e + e^2 with e = 1 - x y0 -- four FP64 pipe
// instructions but a short dependent path; within one ulp for normal-range
// x (zero, infinity and subnormals propagate as inf / 0 / NaN).
__device__ __forceinline__ double rcp_chain(double x) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double e = fma(-x, y, 1.0);
    return fma(y, fma(e, e, e), y);
}
static __device__ __noinline__ double rcp_rare(double x) { return rcp_chain(x); }
__device__ __forceinline__ double rcp_fast(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int E = (int)((hi >> 20) & 0x7ffu);
    if ((unsigned)E - 1u >= 2043u) return rcp_rare(x);
    float mh, ml;
    split_d_ff(__hiloint2double((int)((hi & 0xfffffu) | 0x3ff00000u), (int)lo), mh, ml);
    float rh;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rh) : "f"(mh));
    const float d = fmaf(-ml, rh, fmaf(-mh, rh, 1.0f));
    float h, l;
    two_sum_f(rh, __fmul_rn(rh, fmaf(d, d, d)), h, l);
    const double ym = ff2d_int(h, l);  // 1/m in (0.5, 1]
    const double y = __hiloint2double(
        (int)(((unsigned)(__double2hiint(ym) + (1023 - E) * (1 << 20))) | (hi & 0x80000000u)),
        __double2loint(ym));
    return fma(y, fma(-x, y, 1.0), y);
}

// x / y with two FP64 instructions: a quotient q0 good to about 2^-44
// formed off the FP64 pipe, then r = x - y q0 and q = q0 + r y0 with y0
// the FP32 reciprocal seed of y (the correction's error is that of q0
// times that of y0, about 2^-67), so q is within one ulp of x / y.  q0:
// the significands mx = mxh + mxl and my = myh + myl split into floats by
// integer operations, 1/my = rh + rh (d + d^2) with rh the FP32 hardware
// reciprocal of myh and d = 1 - my rh, mx/my as a float pair from the
// products' exact errors, widened to a double and scaled by 2^(Ex - Ey)
// with integer operations.  Zero, subnormal, huge or non-finite operands,
// and quotients near the ends of the range, take IEEE division out of line.
static __device__ __noinline__ double ddiv_rare(double x, double y) { return x / y; }
__device__ __forceinline__ double ddiv_fast(double x, double y) {
    const unsigned hx = (unsigned)__double2hiint(x), hy = (unsigned)__double2hiint(y);
    const int Ex = (int)((hx >> 20) & 0x7ffu), Ey = (int)((hy >> 20) & 0x7ffu);
    if ((unsigned)Ex - 1u >= 2046u || (unsigned)Ey - 1u >= 2043u ||
        (unsigned)(Ex - Ey + 1021) >= 2044u)
        return ddiv_rare(x, y);
    float mxh, mxl, myh, myl;
    split_d_ff(__hiloint2double((int)((hx & 0xfffffu) | 0x3ff00000u), __double2loint(x)), mxh, mxl);
    split_d_ff(__hiloint2double((int)((hy & 0xfffffu) | 0x3ff00000u), __double2loint(y)), myh, myl);
    float rh;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rh) : "f"(myh));
    const float d = fmaf(-myl, rh, fmaf(-myh, rh, 1.0f));
    const float c = __fmul_rn(rh, fmaf(d, d, d));
    const float qh = __fmul_rn(mxh, rh);
    float h, l;
    two_sum_f(qh, fmaf(mxh, rh, -qh) + fmaf(mxh, c, __fmul_rn(mxl, rh)), h, l);
    const double qm = ff2d_int(h, l);  // mx / my in (0.5, 2)
    const double q0 = __hiloint2double(
        (int)(((unsigned)(__double2hiint(qm) + (Ex - Ey) * (1 << 20))) | ((hx ^ hy) & 0x80000000u)),
        __double2loint(qm));
    const unsigned rb = __float_as_uint(rh);
    const double y0 = __hiloint2double(
        (int)((hy & 0x80000000u) | ((rb >> 3) + 0x77f00000u - (hy & 0x7ff00000u))), (int)(rb << 29));
    return fma(fma(-y, q0, x), y0, q0);
}

// x neither infinite nor NaN, from its exponent field on the integer pipe
// (an FP64 comparison would take an FP64 pipe slot)
__device__ __forceinline__ bool finite_int(double x) {
    return (__double2hiint(x) & 0x7ff00000) != 0x7ff00000;
}

// |x| <= t on the integer pipe (an FP64 comparison or max would take an
// FP64 pipe slot): for non-negative doubles the order of the values is the
// order of their bit patterns as unsigned integers.  A NaN |x| lies above
// every finite pattern and infinity, so it compares false, as the FP64
// comparison does; a negative t admits nothing.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
}
__device__ __forceinline__ bool bits_le(unsigned long long a, double t) {
    const unsigned long long tb = (unsigned long long)__double_as_longlong(t);
    return (tb >> 63) == 0 && a <= tb;
}
__device__ __forceinline__ bool abs_le_int(double x, double t) { return bits_le(abs_bits(x), t); }
// running maximum of magnitudes kept as a bit pattern; a NaN x leaves it
// unchanged, as fmax does
__device__ __forceinline__ unsigned long long absmax_bits(unsigned long long m, double x) {
    const unsigned long long b = abs_bits(x);
    return (b > m && b <= 0x7ff0000000000000ULL) ? b : m;
}

// -x by flipping the sign bit on the integer pipe: a negated argument that
// goes on to the integer steps of exp_tang / one_pm_exp has to exist in a
// register, and an FP64 negation there would take an FP64 pipe slot.
__device__ __forceinline__ double neg_int(double x) {
    return __hiloint2double(__double2hiint(x) ^ (int)0x80000000u, __double2loint(x));
}

// LINOID's series u/(1 - e^-u) = 1 + u/2 + u^2/12 - u^4/720 for |u| < 0.01,
// out of line like exp_tang_rare
static __device__ __noinline__ double linoid_series(double u) {
    const double s = u * u;
    return fma(u, 0.5, fma(s, fma(s, -1.0 / 720.0, 1.0 / 12.0), 1.0));
}

// A rate as numerator / denominator (so that a gate needs one reciprocal):
// EXP A e^u / 1; SIGMOID A / (1 + e^-u); LINOID A u / (1 - e^-u), with the
// series A (1 + u/2 + u^2/12 - u^4/720) / 1 for |u| < 0.01 (next term
// u^6/30240 < 4e-17).  FA: an EXP rate's |A| is folded into u (fold_gate)
// and A carries only its sign, applied to e^u by an integer operation.
template <bool FA = false>
__device__ __forceinline__ void rate_nd_u(int form, double A, double u, double& num,
                                          double& den) {
    if (form == kExp) {
        if (FA) {
            const double e = exp_tang(u);
            num = __hiloint2double(__double2hiint(e) ^ (__double2hiint(A) & (int)0x80000000u),
                                   __double2loint(e));
        } else {
            num = A * exp_tang(u);
        }
        den = 1.0;
    } else if (form == kSigmoid) {
        num = A;
        den = one_pm_exp<1>(neg_int(u));
    } else if ((__double2hiint(u) & 0x7fffffff) < 0x3f847ae1) {  // |u| < 0.01
        num = A * linoid_series(u);
        den = 1.0;
    } else {
        num = A * u;
        den = one_pm_exp<-1>(neg_int(u));
    }
}

// A gate's parameters folded for one launch: vh becomes c = -vh/k, so that
// u = v (1/k) + c is one multiply-add (its rounding moves u by at most a
// few units of |c| 2^-53: a few ulp in e^u, and in LINOID the same u enters
// numerator and denominator), and each A is multiplied by phi dt, so that
// alpha + beta comes out as phi dt (alpha + beta) and minf is unchanged.
// An EXP rate's A e^u becomes sign(A) e^(u + ln|A|): ln|A| joins c (one
// more rounding of the same kind) and A keeps its sign only (A = 0 gives
// e^-inf = 0).  Takes a log per rate: fold once per block, not per item.
__host__ __device__ __forceinline__ void fold_gate(GateD& G, double phidt) {
    G.avh = -G.avh * G.ark;
    G.bvh = -G.bvh * G.brk;
    G.aA *= phidt;
    G.bA *= phidt;
    if (G.aform == kExp) {
        G.avh += log(fabs(G.aA));
        G.aA = copysign(1.0, G.aA);
    }
    if (G.bform == kExp) {
        G.bvh += log(fabs(G.bA));
        G.bA = copysign(1.0, G.bA);
    }
}

// cnexp gate step from the rates as alpha = Pa/Da, beta = Pb/Db:
// N = Pa Db + Pb Da, D = Da Db, minf = Pa Db / N and alpha + beta = N / D,
// each one division of two FP64 instructions (ddiv_fast).  With the rate
// forms known at compile time an EXP rate's denominator 1 removes
// multiplications:
//   beta EXP:  N = Pa + Pb Da, minf = Pa / N,    s = N / Da
//   alpha EXP: N = Pb + Pa Db, minf = Pa Db / N, s = N / Db
//   both EXP:  s = Pa + Pb,    minf = Pa / s.
// The update m + (1 - e)(minf - m), e = exp(-phi dt s), is taken as
// minf + (m - minf) e (the same value; one operation fewer).
// FOLD: G folded by fold_gate (phidt unused).
template <int AF, int BF, bool FOLD>
__device__ __forceinline__ double gate_step_forms_d(const GateD& G, double phidt, double v,
                                                    double m) {
    double na, da, nb, db;
    rate_nd_u<FOLD>(AF, G.aA, FOLD ? fma(v, G.ark, G.avh) : (v - G.avh) * G.ark, na, da);
    rate_nd_u<FOLD>(BF, G.bA, FOLD ? fma(v, G.brk, G.bvh) : (v - G.bvh) * G.brk, nb, db);
    double minf, s;
    if constexpr (AF == kExp && BF == kExp) {
        s = na + nb;
        minf = ddiv_fast(na, s);
    } else if constexpr (BF == kExp) {
        const double N = fma(nb, da, na);
        minf = ddiv_fast(na, N);
        s = ddiv_fast(N, da);
    } else if constexpr (AF == kExp) {
        const double P = na * db;
        const double N = nb + P;
        minf = ddiv_fast(P, N);
        s = ddiv_fast(N, db);
    } else {
        const double P = na * db;
        const double N = fma(nb, da, P);
        minf = ddiv_fast(P, N);
        s = ddiv_fast(N, da * db);
    }
    return fma(m - minf, exp_tang(FOLD ? neg_int(s) : -phidt * s), minf);
}

// One form pair as a separate (not inlined) function: the call boundary
// keeps the compiler from merging the nine bodies into one predicated
// sequence, in which every lane would occupy the FP64 pipe for the
// instructions of all the forms.  A call costs integer instructions only.
template <int AF, int BF, bool FOLD>
__device__ __noinline__ double gate_step_call_d(double aA, double avh, double ark, double bA,
                                                double bvh, double brk, double phidt, double v,
                                                double m) {
    GateD G;
    G.aA = aA; G.avh = avh; G.ark = ark;
    G.bA = bA; G.bvh = bvh; G.brk = brk;
    return gate_step_forms_d<AF, BF, FOLD>(G, phidt, v, m);
}

// The gate step for the gate's forms: a switch that is uniform over the
// items of one gate, one straight-line body per form pair.  FOLD: G folded
// by fold_gate.
template <bool FOLD = false>
__device__ __forceinline__ double gate_step_fast_d(const GateD& G, double phidt, double v,
                                                   double m) {
#define NMODL_GATE_CASE(C, A, B) \
    case C: return gate_step_call_d<A, B, FOLD>(G.aA, G.avh, G.ark, G.bA, G.bvh, G.brk, phidt, v, m)
    switch (G.aform * 3 + G.bform) {
        NMODL_GATE_CASE(0, kExp, kExp);
        NMODL_GATE_CASE(1, kExp, kSigmoid);
        NMODL_GATE_CASE(2, kExp, kLinoid);
        NMODL_GATE_CASE(3, kSigmoid, kExp);
        NMODL_GATE_CASE(4, kSigmoid, kSigmoid);
        NMODL_GATE_CASE(5, kSigmoid, kLinoid);
        NMODL_GATE_CASE(6, kLinoid, kExp);
        NMODL_GATE_CASE(7, kLinoid, kSigmoid);
    default: return gate_step_call_d<kLinoid, kLinoid, FOLD>(G.aA, G.avh, G.ark, G.bA, G.bvh,
                                                             G.brk, phidt, v, m);
    }
#undef NMODL_GATE_CASE
}

__device__ __forceinline__ double rate_d(int form, double A, double vh,
                                         double rk, double v) {
    const double u = (v - vh) * rk;
    if (form == kExp) return A * exp(u);
    if (form == kSigmoid) return A / (1.0 + exp(-u));
    // LINOID: A u / (1 - exp(-u)); series 1 + u/2 + u^2/12 near u = 0
    if (fabs(u) < 1e-6) return A * (1.0 + u * (0.5 + u * (1.0 / 12.0)));
    return A * u / (-expm1(-u));
}


// The same step with exp(-x), x = phi dt (alpha + beta), replaced by its
// (1,1) Pade approximant: the factor 2x/(2 + x) folds into the one division,
// m += 2 c (Pa Db - m N) / (2 D + c N) with c = phi dt.
// FOLD: G folded by fold_gate (the rates carry phi dt; phidt unused).
template <bool FOLD = false>
__device__ __forceinline__ double gate_step_pade_d(const GateD& G, double phidt, double v,
                                                   double m) {
    double na, da, nb, db;
    rate_nd_u<FOLD>(G.aform, G.aA, FOLD ? fma(v, G.ark, G.avh) : (v - G.avh) * G.ark, na, da);
    rate_nd_u<FOLD>(G.bform, G.bA, FOLD ? fma(v, G.brk, G.bvh) : (v - G.bvh) * G.brk, nb, db);
    const double P = na * db;
    const double N = fma(nb, da, P);
    const double D = da * db;
    if (FOLD) return m + (2.0 * fma(-m, N, P)) * rcp_fast(N + (D + D));
    const double num = 2.0 * phidt * fma(-m, N, P);
    const double den = fma(phidt, N, D + D);
    return m + num * rcp_fast(den);
}

__device__ __forceinline__ double gate_inf_d(const GateD& G, double v) {
    const double a = rate_d(G.aform, G.aA, G.avh, G.ark, v);
    const double b = rate_d(G.bform, G.bA, G.bvh, G.brk, v);
    return a / (a + b);
}

// g x^p multiplied out from the left: p multiplications
__device__ __forceinline__ double mul_pow_d(double g, double x, int p) {
    for (int k = 0; k < p; ++k) g *= x;
    return g;
}

// ------------------------------------------------------------ FP32 math
// Rates and the cnexp factor in single precision.  exp uses the hardware
// exp2 unit; the two cancelling differences (1 - exp(-u) in LINOID and
// 1 - exp(-x) in cnexp) switch to their Taylor series where the series is
// more accurate than the subtraction.

__device__ __forceinline__ float ex2_hw(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// A rate with its parameters folded for the exp2 unit: w = u log2(e) =
// v k2 + c2 (k2 = rk log2(e), c2 = -vh rk log2(e): one multiply-add), and
// LINOID's prefactor as A ln2 (A u = (A ln2) w).
__device__ __forceinline__ float rate_f(int form, float A, float k2, float c2, float v) {
    const float w = fmaf(v, k2, c2);
    if (form == kExp) return A * ex2_hw(w);
    if (form == kSigmoid) return __fdividef(A, 1.0f + ex2_hw(-w));
    // u/(1-e^-u) = 1 + u/2 + u^2/12 - u^4/720 + ..., u = w ln2 and A = (A ln2) log2(e)
    if (fabsf(w) < 0.1f * 1.44269504f) {
        const float u = w * 0.693147181f, u2 = u * u;
        return (A * 1.44269504f) * (1.0f + 0.5f * u + u2 * (1.0f / 12.0f - u2 * (1.0f / 720.0f)));
    }
    return __fdividef(A * w, 1.0f - ex2_hw(-w));
}

// 1 - exp(-x) for x >= 0
__device__ __forceinline__ float one_minus_expneg_f(float x) {
    if (x < 0.1f) {
        // x - x^2/2 + x^3/6 - x^4/24 + x^5/120
        return x * (1.0f - x * (0.5f - x * (1.0f / 6.0f - x * (1.0f / 24.0f - x * (1.0f / 120.0f)))));
    }
    return 1.0f - __expf(-x);
}

// a gate's two rates in FP32, folded as rate_f takes them
struct GateF {
    float aA, ak2, ac2, bA, bk2, bc2;
    int32_t aform, bform;
};
__device__ __forceinline__ GateF gate_f(const GateD& G) {
    constexpr double kLog2e = 1.4426950408889634, kLn2 = 0.6931471805599453;
    return GateF{(float)(G.aform == kLinoid ? G.aA * kLn2 : G.aA), (float)(G.ark * kLog2e),
                 (float)(-G.avh * G.ark * kLog2e),
                 (float)(G.bform == kLinoid ? G.bA * kLn2 : G.bA), (float)(G.brk * kLog2e),
                 (float)(-G.bvh * G.brk * kLog2e), G.aform, G.bform};
}

// (minf, 1 - exp(-dt/mtau)) of a gate in FP32; with pade the factor is the
// (1,1) Pade form x/(1 + x/2)
__device__ __forceinline__ void gate_coef_f(const GateF& G, float phidt, float v,
                                            float& minf, float& f, bool pade = false) {
    const float a = rate_f(G.aform, G.aA, G.ak2, G.ac2, v);
    const float b = rate_f(G.bform, G.bA, G.bk2, G.bc2, v);
    const float s = a + b;
    minf = __fdividef(a, s);
    const float x = phidt * s;
    f = pade ? __fdividef(x, fmaf(0.5f, x, 1.0f)) : one_minus_expneg_f(x);
}

__device__ __forceinline__ void latch_error(int32_t* err, int32_t code) {
    if (err) atomicCAS(err, 0, code);
}

}  // namespace nmodl
