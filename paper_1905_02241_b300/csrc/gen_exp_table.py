"""Generate exp_tang_table.cuh: constants of the table-driven FP64 exp.

Tang, "Table-driven implementation of the exponential function in IEEE
floating-point arithmetic", ACM TOMS 15(2), 1989: x = (64 m + j) ln2/64 + r,
exp(x) = 2^m 2^(j/64) exp(r).  The values are mathematical constants
evaluated with mpmath at 60 digits and rounded to double:
  T[j] = 2^(j/64), j = 0..63
  L1 + L2 = ln2/64 with L1 keeping 36 significant bits (so n*L1 is exact for
  |n| < 2^17), L2 the rounded remainder.
Run:  python gen_exp_table.py > exp_tang_table.cuh
"""
import mpmath

mpmath.mp.dps = 60


def hexd(x):
    return float(x).hex()


def main():
    ln2_32 = mpmath.log(2) / 64
    f = float(ln2_32)
    m, e = mpmath.frexp(mpmath.mpf(f))
    # keep 37 significant bits of ln2/32 in L1
    scale = mpmath.mpf(2) ** (36 - e)
    L1 = mpmath.floor(ln2_32 * scale) / scale
    L2 = ln2_32 - L1
    print("// Generated by gen_exp_table.py -- do not edit.")
    print("// Constants of the table-driven exp (Tang, ACM TOMS 1989).")
    print("#pragma once")
    print("namespace nmodl {")
    print(f"constexpr double kExpInvL = {hexd(64 / mpmath.log(2))};   // 64/ln2")
    print(f"constexpr double kExpL1 = {hexd(L1)};   // ln2/64, 36 leading bits")
    print(f"constexpr double kExpL2 = {hexd(L2)};   // ln2/64 - L1")
    print("__device__ const double kExpTable[64] = {")
    for j in range(64):
        print(f"    {hexd(mpmath.power(2, mpmath.mpf(j) / 64))},  // 2^({j}/64)")
    print("};")
    print("}  // namespace nmodl")


if __name__ == "__main__":
    main()
