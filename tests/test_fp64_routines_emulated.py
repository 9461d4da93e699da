"""The FP64 routines of the state kernels, emulated step for step on the CPU.

The device exp, reciprocal, division and rate denominators keep two FP64
instructions each and do the rest of their work on the integer and FP32
pipes (float pairs, integer widening of pairs to doubles).  These tests
restate each routine in numpy -- integer steps on uint32/uint64 bit
patterns, FP32 steps in float32, the two FP64 instructions as one rounding
of the exact value -- and check its error bound against long double (64-bit
significand) over many more arguments than the GPU tests sample.  An fmaf is
modelled as the exact product rounded with the addend in float64, then to
float32 (a double rounding that can differ from the hardware's in rare
ties; the GPU tests measure the real routines).  Constants come from the
generated table header that the kernels include.
"""
import os
import re

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "..", "paper_1905_02241_b300", "csrc", "exp_tang_table.cuh")

f32 = np.float32
u32 = np.uint32
u64 = np.uint64


def _consts():
    src = open(TABLE).read()
    tab = np.array([float.fromhex(h) for h in re.findall(r"^\s+(-?0x[0-9a-fp.+-]+),", src, re.M)])

    def c(name):
        return float.fromhex(re.search(name + r" = (-?0x[0-9a-fp.+-]+)", src).group(1).rstrip("f"))
    return dict(tab=tab, InvLh=f32(c("kExpInvLh")), InvLl=f32(c("kExpInvLl")),
                L2h=f32(c("kExpL2h")), L2l=f32(c("kExpL2l")), L1=c("kExpL1"))


K = _consts()


def fmaf(a, b, c):
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def fma_d(a, b, c):
    """One FP64 fma: the exact value rounded once (long double first)."""
    return (np.longdouble(a) * np.longdouble(b) + np.longdouble(c)).astype(np.float64)


def bits_f(x):
    return np.asarray(x, dtype=np.float32).view(u32)


def from_bits_f(b):
    return np.asarray(b, dtype=u32).view(np.float32)


def hi_lo(d):
    b = np.asarray(d, dtype=np.float64).view(u64)
    return (b >> u64(32)).astype(u32), (b & u64(0xffffffff)).astype(u32)


def from_hi_lo(h, lo):
    return ((h.astype(u64) << u64(32)) | lo.astype(u64)).view(np.float64)


def funnel_l3(lo, hi):
    return ((hi << u32(3)) | (lo >> u32(29))).astype(u32)


def two_sum(a, b):
    s = f32(a + b)
    bp = f32(s - a)
    return s, f32(f32(a - f32(s - bp)) + f32(b - bp))


def split_d_ff(r):
    """r = h + l to 47 bits (h: leading 24 significand bits, l: the next 23)."""
    hr, lr = hi_lo(r)
    ar = hr & u32(0x7fffffff)
    sg = hr & u32(0x80000000)
    with np.errstate(over="ignore"):
        h = from_bits_f(funnel_l3(lr, (ar - u32(0x38000000)).astype(u32)) | sg)
        m23 = f32(from_bits_f(u32(0x4b000000) | ((lr >> u32(6)) & u32(0x7fffff))) - f32(8388608.0))
        scale = from_bits_f((((ar >> u32(20)) - u32(942)) << u32(23)).astype(u32))
        lo = from_bits_f(bits_f(f32(m23 * scale)) | sg)
    small = ar < u32(0x3c300000)
    return np.where(small, f32(0), h), np.where(small, f32(0), lo)


def ff2d(hi, lo):
    """hi + lo of a normalized float pair as a double (integer steps)."""
    fh = bits_f(hi).astype(u64)
    fl = bits_f(lo).astype(u64)
    ah, al = fh & u64(0x7fffffff), fl & u64(0x7fffffff)
    sh = (al >> u64(23)).astype(np.int64) - (ah >> u64(23)).astype(np.int64) + 29
    m = (al & u64(0x7fffff)) | u64(0x800000)
    d = np.where(sh >= 0, m << np.clip(sh, 0, 31).astype(u64),
                 np.where(sh > -24, m >> np.clip(-sh, 0, 31).astype(u64), u64(0)))
    d = np.where((al >> u64(23)) == 0, u64(0), d)
    opp = ((fh ^ fl) & u64(0x80000000)) != 0
    d = np.where(opp & ((ah & u64(0x7fffff)) == 0), d << u64(1), d)
    H = (((ah >> u64(3)) + u64(896 << 20)) << u64(32)) | ((ah << u64(29)) & u64(0xffffffff))
    H = np.where(opp, H - d, H + d) | ((fh & u64(0x80000000)) << u64(32))
    return np.where(ah == 0, 0.0, H.view(np.float64))


def exp_core(x):
    """e^x = 2^m T (1 + p): T, k (m = k >> 11) and p, |x| < 708."""
    xh, xl = split_d_ff(x)
    kh = f32(xh * K["InvLh"])
    kl = fmaf(xl, K["InvLh"], fmaf(xh, K["InvLl"], fmaf(xh, K["InvLh"], -kh)))
    t = f32(kh + f32(12582912.0))
    nh = f32(t - f32(12582912.0))
    fr = f32(f32(kh - nh) + kl)
    up, dn = fr > 0.5, fr < -0.5
    k = bits_f(t).astype(np.int64) - 0x4b400000 + up.astype(np.int64) - dn.astype(np.int64)
    nf = f32(nh + np.where(up, f32(1), np.where(dn, f32(-1), f32(0))))
    r1 = fma_d(nf, -K["L1"], x)                       # FP64 instruction 1 (exact)
    rh, rl = split_d_ff(r1)
    a = f32(nf * K["L2h"])
    ae = fmaf(nf, K["L2l"], fmaf(nf, K["L2h"], -a))
    R, Rl = two_sum(rh, -a)
    Rl = f32(Rl + f32(rl - ae))
    P = f32(R * R)
    Pe = fmaf(R, R, -P)
    S0, S0l = two_sum(R, f32(f32(0.5) * P))
    S0l = f32(S0l + f32(Rl + fmaf(f32(0.5), Pe, fmaf(R, Rl, f32(f32(P * R) * f32(1 / 6))))))
    S, Sl = two_sum(S0, S0l)
    return K["tab"][k & 2047], k, ff2d(S, Sl)


def exp_emulated(x):
    T, k, pr = exp_core(x)
    return np.ldexp(fma_d(T, pr, T), (k >> 11).astype(np.int32))   # FP64 instruction 2


def clz64(v):
    v = np.asarray(v, dtype=u64)
    out = np.full(v.shape, 64, dtype=np.int64)
    nz = v != 0
    _, e = np.frexp(v[nz].astype(np.float64))
    p = e.astype(np.int64) - 1                          # leading bit, maybe one too high
    p = np.where(v[nz] < (u64(1) << p.clip(0, 63).astype(u64)), p - 1, p)
    out[nz] = 63 - p
    return out


def one_pm_emulated(x, s):
    """1 + s e^x: the constant part 1 + s 2^m T on a common integer grid."""
    T, k, pr = exp_core(x)
    m = (k >> 11).astype(np.int64)
    Tb = T.view(u64)
    T2m = (Tb.astype(np.int64) + (m << 52)).astype(u64).view(np.float64)
    MT = ((Tb & u64((1 << 52) - 1)) | u64(1 << 52)).astype(np.int64)
    g = np.maximum(m - 52, -62)
    sh = np.maximum(0, -10 - m)
    Tg = np.where(sh >= 63, 0, MT >> np.minimum(sh, 62))
    one = np.int64(1) << (-g).clip(0, 62)
    Sv = one + s * Tg
    A = np.abs(Sv).astype(u64)
    lz = clz64(A)
    rs = 11 - lz
    Ar = np.where(rs > 0, (A + (u64(1) << (rs - 1).clip(0, 63).astype(u64))) >> rs.clip(0, 63).astype(u64),
                  A << (-rs).clip(0, 63).astype(u64))
    bits = ((63 - lz + g + 1022).astype(u64) << u64(52)) + Ar
    C = np.where(Sv < 0, -1.0, 1.0) * bits.view(np.float64)
    C = np.where(A == 0, 0.0, C)
    C = np.where(m >= 53, s * T2m, C)
    return fma_d(s * T2m, pr, C)


def rcp_seed_f32(mh, rng):
    """The FP32 hardware reciprocal, modelled as the correctly rounded one
    moved by one float ulp at random (its documented error is below 1 ulp)."""
    r = f32(np.float32(1.0) / mh)
    move = rng.random(r.size) < 0.5
    return np.where(move, np.nextafter(r, np.float32(0)), r).astype(np.float32)


def rcp_emulated(x, rng):
    hx, lx = hi_lo(x)
    E = ((hx >> u32(20)) & u32(0x7ff)).astype(np.int64)
    mh, ml = split_d_ff(from_hi_lo((hx & u32(0xfffff)) | u32(0x3ff00000), lx))
    rh = rcp_seed_f32(mh, rng)
    d = fmaf(-ml, rh, fmaf(-mh, rh, f32(1.0)))
    h, lo = two_sum(rh, f32(rh * fmaf(d, d, d)))
    hy, ly = hi_lo(ff2d(h, lo))
    hy = (hy.astype(np.int64) + (1023 - E) * (1 << 20)).astype(u32) | (hx & u32(0x80000000))
    y = from_hi_lo(hy, ly)
    return fma_d(y, fma_d(-x, y, 1.0), y)


def ddiv_emulated(x, y, rng):
    hx, lx = hi_lo(x)
    hy, ly = hi_lo(y)
    Ex = ((hx >> u32(20)) & u32(0x7ff)).astype(np.int64)
    Ey = ((hy >> u32(20)) & u32(0x7ff)).astype(np.int64)
    mxh, mxl = split_d_ff(from_hi_lo((hx & u32(0xfffff)) | u32(0x3ff00000), lx))
    myh, myl = split_d_ff(from_hi_lo((hy & u32(0xfffff)) | u32(0x3ff00000), ly))
    rh = rcp_seed_f32(myh, rng)
    d = fmaf(-myl, rh, fmaf(-myh, rh, f32(1.0)))
    c = f32(rh * fmaf(d, d, d))
    qh = f32(mxh * rh)
    h, lo = two_sum(qh, f32(fmaf(mxh, rh, -qh) + fmaf(mxh, c, f32(mxl * rh))))
    hq, lq = hi_lo(ff2d(h, lo))
    hq = (hq.astype(np.int64) + (Ex - Ey) * (1 << 20)).astype(u32) | ((hx ^ hy) & u32(0x80000000))
    q0 = from_hi_lo(hq, lq)
    rb = bits_f(rh).astype(np.int64)
    hy0 = (((rb >> 3) + 0x77f00000 - (hy & u32(0x7ff00000)).astype(np.int64)).astype(u32)
           | (hy & u32(0x80000000)))
    y0 = from_hi_lo(hy0, (rb << 29).astype(u32))
    return fma_d(fma_d(-y, q0, x), y0, q0)


def _ulps(got, ref):
    return np.abs((np.longdouble(got) - ref) / np.spacing(np.abs(ref).astype(np.float64))).astype(np.float64)


def test_emulated_pair_widening_is_exact_to_truncation():
    rng = np.random.default_rng(9)
    h = f32(rng.uniform(-1, 1, 100000) * 10.0 ** rng.uniform(-30, 0, 100000))
    h[:1000] = f32(2.0) ** rng.integers(-40, 0, 1000).astype(np.float32)
    h[:1000] *= rng.choice([-1, 1], 1000).astype(np.float32)
    lo = f32(np.spacing(np.abs(h)) * rng.uniform(-0.5, 0.5, h.size))
    hh, ll = two_sum(h, lo)
    keep = (np.abs(ll) >= np.float32(2.0 ** -126)) | (ll == 0)   # a subnormal lo is dropped
    exact = np.longdouble(hh) + np.longdouble(ll)
    got = ff2d(hh, ll)
    rel = np.abs((np.longdouble(got) - exact) / exact).astype(np.float64)
    assert rel[keep].max() <= 2.0 ** -52


def test_emulated_exp_within_its_bound():
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.uniform(-708, 708, 100000), rng.uniform(-30, 30, 100000),
                        rng.uniform(-1, 1, 50000),
                        (np.arange(-2000, 2000) + 0.5) * np.log(2) / 2048,   # near ties of n
                        [0.0, -0.0, 1e-300, 707.9, -707.9]])
    u = _ulps(exp_emulated(x), np.exp(x.astype(np.longdouble)))
    assert u.max() <= 1.5, u.max()


def test_emulated_reciprocal_and_division_within_one_ulp():
    rng = np.random.default_rng(7)
    n = 100000
    x = np.concatenate([rng.uniform(0.5, 2.0, n), rng.uniform(1, 10, n) * 10.0 ** rng.integers(-300, 300, n),
                        -rng.uniform(1e-6, 1e6, n // 2), 2.0 ** np.arange(-1000, 1000, 37)])
    y = rcp_emulated(x, np.random.default_rng(1))
    assert _ulps(y, 1 / np.longdouble(x)).max() <= 1.0
    p2 = np.arange(-1000, 1000, 37).size
    assert np.array_equal(y[-p2:], 1 / x[-p2:])
    a = rng.uniform(1, 10, n) * 10.0 ** rng.integers(-150, 150, n) * rng.choice([-1, 1], n)
    b = rng.uniform(1, 10, n) * 10.0 ** rng.integers(-150, 150, n) * rng.choice([-1, 1], n)
    q = ddiv_emulated(a, b, np.random.default_rng(2))
    assert _ulps(q, np.longdouble(a) / np.longdouble(b)).max() <= 1.0


def test_emulated_rate_denominators():
    rng = np.random.default_rng(21)
    x = np.concatenate([rng.uniform(-700, 700, 100000), rng.uniform(-40, 40, 100000),
                        rng.uniform(-1, 1, 50000), [0.0, 36.7, 37.5, -36.7]])
    e = np.exp(x.astype(np.longdouble))
    up = one_pm_emulated(x, 1)
    assert _ulps(up, 1 + e).max() <= 2.0
    um = one_pm_emulated(x, -1)
    keep = np.abs(x) >= 0.01           # LINOID takes its series below
    err = np.abs(np.longdouble(um[keep]) - (1 - e[keep])).astype(np.float64)
    bound = (2 * np.spacing(e[keep].astype(np.float64))
             + np.spacing(np.abs(1 - e[keep]).astype(np.float64)))
    assert np.all(err <= bound)


@pytest.mark.parametrize("s", [1, -1])
def test_emulated_denominator_constant_is_exact_where_representable(s):
    """On the grid, 1 + s 2^m T is formed exactly: with p = 0 the result is
    the correctly rounded 1 + s 2^m T whenever that sum fits 64 bits."""
    rng = np.random.default_rng(5)
    x = rng.uniform(-6, 30, 20000)
    T, k, _ = exp_core(x)
    m = (k >> 11).astype(np.int64)
    T2m = np.ldexp(T, m.astype(np.int32))
    exact = 1 + s * np.longdouble(T2m)
    got = one_pm_emulated(x, s) - s * (np.longdouble(T2m) * np.longdouble(exp_core(x)[2]))
    # the fma adds s 2^m T p to C; undoing that product leaves C to the fma's rounding
    assert np.all(np.abs(got - exact) <= 2 * np.spacing(np.abs(exact).astype(np.float64)))
