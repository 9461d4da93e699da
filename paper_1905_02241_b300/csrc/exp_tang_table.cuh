// Generated by gen_exp_table.py -- do not edit.
// Constants of the table-driven exp (Tang, ACM TOMS 1989).
#pragma once
namespace nmodl {
constexpr double kExpInvL = 0x1.71547652b82fep+5;   // 32/ln2
constexpr double kExpL1 = 0x1.62e42fefa0000p-6;   // ln2/32, 37 leading bits
constexpr double kExpL2 = 0x1.cf79abc9e3b3ap-45;   // ln2/32 - L1
__device__ const double kExpTable[32] = {
    0x1.0000000000000p+0,  // 2^(0/32)
    0x1.059b0d3158574p+0,  // 2^(1/32)
    0x1.0b5586cf9890fp+0,  // 2^(2/32)
    0x1.11301d0125b51p+0,  // 2^(3/32)
    0x1.172b83c7d517bp+0,  // 2^(4/32)
    0x1.1d4873168b9aap+0,  // 2^(5/32)
    0x1.2387a6e756238p+0,  // 2^(6/32)
    0x1.29e9df51fdee1p+0,  // 2^(7/32)
    0x1.306fe0a31b715p+0,  // 2^(8/32)
    0x1.371a7373aa9cbp+0,  // 2^(9/32)
    0x1.3dea64c123422p+0,  // 2^(10/32)
    0x1.44e086061892dp+0,  // 2^(11/32)
    0x1.4bfdad5362a27p+0,  // 2^(12/32)
    0x1.5342b569d4f82p+0,  // 2^(13/32)
    0x1.5ab07dd485429p+0,  // 2^(14/32)
    0x1.6247eb03a5585p+0,  // 2^(15/32)
    0x1.6a09e667f3bcdp+0,  // 2^(16/32)
    0x1.71f75e8ec5f74p+0,  // 2^(17/32)
    0x1.7a11473eb0187p+0,  // 2^(18/32)
    0x1.82589994cce13p+0,  // 2^(19/32)
    0x1.8ace5422aa0dbp+0,  // 2^(20/32)
    0x1.93737b0cdc5e5p+0,  // 2^(21/32)
    0x1.9c49182a3f090p+0,  // 2^(22/32)
    0x1.a5503b23e255dp+0,  // 2^(23/32)
    0x1.ae89f995ad3adp+0,  // 2^(24/32)
    0x1.b7f76f2fb5e47p+0,  // 2^(25/32)
    0x1.c199bdd85529cp+0,  // 2^(26/32)
    0x1.cb720dcef9069p+0,  // 2^(27/32)
    0x1.d5818dcfba487p+0,  // 2^(28/32)
    0x1.dfc97337b9b5fp+0,  // 2^(29/32)
    0x1.ea4afa2a490dap+0,  // 2^(30/32)
    0x1.f50765b6e4540p+0,  // 2^(31/32)
};
}  // namespace nmodl
