"""Generate exp_tang_table.cuh: constants of the table-driven FP64 exp.

Tang, "Table-driven implementation of the exponential function in IEEE
floating-point arithmetic", ACM TOMS 15(2), 1989: with N = 2^BITS,
x = (N m + j) ln2/N + r, exp(x) = 2^m 2^(j/N) exp(r).  The values are
mathematical constants evaluated with mpmath at 60 digits and rounded to
double:
  T[j] = 2^(j/N), j = 0..N-1
  L1 + L2 = ln2/N with L1 keeping L1_BITS significant bits (so n*L1 is exact
  for |n| < 2^(53 - L1_BITS), here |n| < 2^22, i.e. |x| < 1000), L2 the
  rounded remainder.
  InvLh + InvLl = N/ln2 as two floats (the leading float and the float
  nearest the remainder), for choosing n in single precision; L2h + L2l = L2
  as two floats likewise, for n L2 in single-precision pairs.
Run:  python gen_exp_table.py > exp_tang_table.cuh
"""
import mpmath
import numpy as np

mpmath.mp.dps = 60


def hexd(x):
    return float(x).hex()


BITS = 11          # table of 2^BITS entries
N = 1 << BITS
L1_BITS = 31


def main():
    lnN = mpmath.log(2) / N
    f = float(lnN)
    m, e = mpmath.frexp(mpmath.mpf(f))
    scale = mpmath.mpf(2) ** (L1_BITS - e)
    L1 = mpmath.floor(lnN * scale) / scale
    L2 = lnN - L1
    print("// Generated by gen_exp_table.py -- do not edit.")
    print("// Constants of the table-driven exp (Tang, ACM TOMS 1989).")
    print("#pragma once")
    print("namespace nmodl {")
    print(f"constexpr int kExpBits = {BITS};")
    print(f"constexpr double kExpInvL = {hexd(N / mpmath.log(2))};   // {N}/ln2")
    inv = N / mpmath.log(2)
    inv_h = np.float32(float(inv))
    inv_l = np.float32(float(inv - mpmath.mpf(float(inv_h))))
    print(f"constexpr float kExpInvLh = {float(inv_h).hex()}f;   // {N}/ln2, leading float")
    print(f"constexpr float kExpInvLl = {float(inv_l).hex()}f;   // {N}/ln2 - InvLh")
    l2_h = np.float32(float(L2))
    l2_l = np.float32(float(L2 - mpmath.mpf(float(l2_h))))
    print(f"constexpr float kExpL2h = {float(l2_h).hex()}f;   // L2, leading float")
    print(f"constexpr float kExpL2l = {float(l2_l).hex()}f;   // L2 - L2h")
    print(f"constexpr double kExpL1 = {hexd(L1)};   // ln2/{N}, {L1_BITS} leading bits")
    print(f"constexpr double kExpL2 = {hexd(L2)};   // ln2/{N} - L1")
    print(f"__device__ const double kExpTable[{N}] = {{")
    for j in range(N):
        print(f"    {hexd(mpmath.power(2, mpmath.mpf(j) / N))},  // 2^({j}/{N})")
    print("};")
    print("}  // namespace nmodl")


if __name__ == "__main__":
    main()
