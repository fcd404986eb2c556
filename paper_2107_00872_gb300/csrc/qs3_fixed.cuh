// qs3_fixed.cuh -- fixed-point images of binary64 values and exact integer
// sums, shared by the binary64 engine's dot products (qs3_engine64.cuh) and
// its H Phi (qs3_hphi.cu).
//
// A binary64 v on the grid of a biased exponent em (em >= the exponent of v,
// em >= 54) is P = round(v 2^(1075 - em)), |P| <= 2^53, split into balanced
// base-2^26 digits P = P1 2^26 + P0 (|P0| <= 2^25, |P1| <= 2^27).  Products
// of two such values are summed exactly with mad.wide.s32 on the digits.
// The digit store of the binary64 engine holds one image per stored vector:
// per 2048-row chunk and warp group q (the 128 rows base + 32 q + lane + 512 k,
// k < 4) one grid exponent, so row o of a chunk lies in group (o mod 512) / 32.
#pragma once

#include "qs3_internal.cuh"

namespace qs3 {

constexpr int XT = 512;                 // threads per chunk of k_dotx
constexpr int XR = BROWS / XT;          // rows per thread
constexpr int XW = XT / 32;             // warps per chunk
static_assert(XR * XT == BROWS, "k_dotx covers a chunk");

__device__ __forceinline__ int fx_exp(uint32_t h) { return (int)((h >> 20) & 0x7ffu); }

// the binary64 with high word h and low word l on the grid of em (em >= its
// biased exponent, em >= 54): balanced digits (p1, p0) of round(v 2^(1075-em)).
// A zero or subnormal v (exponent field 0) is at least 2^54 grid steps below
// em and rounds to 0.
__device__ __forceinline__ void fx_digits(uint32_t h, uint32_t l, int em, int &p1, int &p0) {
    const uint32_t sh = min((uint32_t)(em - fx_exp(h)), 63u);
    // 2m, m = 2^52 + the 52 stored significand bits: high word mh2, low l2
    const uint32_t mh2 = (__funnelshift_l(l, h, 1) & 0x1fffffu) | 0x200000u;
    const uint32_t l2 = l << 1;
    // t = floor(2m / 2^sh) = floor(m / 2^(sh-1)): words thi, tlo
    const uint32_t f = __funnelshift_rc(l2, mh2, sh);                  // (2m) >> min(sh, 32), low word
    const uint32_t thi = __funnelshift_rc(mh2, 0u, sh);                // its high word (0 for sh >= 32)
    const uint32_t tlo = f >> (max(sh, 32u) - 32u);                    // the rest of the shift (thi = 0 then)
    // Q = round(m / 2^sh) = floor((t + 1) / 2); Q1 = floor((Q + 2^25) / 2^26),
    // Q0 = Q - Q1 2^26 (the low 26 bits of Q, sign-extended)
    const uint64_t t = ((uint64_t)thi << 32) | tlo;
    const int q1 = (int)((t + 0x4000001ull) >> 27);
    const int q0 = ((int)(((tlo + 1u) >> 1) << 6)) >> 6;
    const int sg = ((int)h >> 31) | 1;
    p1 = q1 * sg;
    p0 = q0 * sg;
}

// a b + c with the 64-bit product of two 32-bit integers (one mad.wide.s32)
__device__ __forceinline__ long long mad_w(int a, int b, long long c) {
    long long d;
    asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
    return d;
}
// a 2^k rounded to the nearest binary64 (ties to even) in integer operations
// (the fp64 pipe issues one warp instruction per ~70 ALU ones, even for a
// single active lane); only a result below the normal range takes fp64 ops
__device__ __forceinline__ double i128_ldexp(__int128 a, int k) {
    if (a == 0) return 0.0;
    const unsigned long long sgn = a < 0 ? 0x8000000000000000ull : 0ull;
    const unsigned __int128 u = a < 0 ? (unsigned __int128)(-a) : (unsigned __int128)a;
    const unsigned long long hi = (unsigned long long)(u >> 64), lo = (unsigned long long)u;
    const int n = hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo);     // bit length
    unsigned long long mant;
    int e = n - 1 + k;                                                               // exponent of the top bit
    if (n <= 53) {
        mant = lo << (53 - n);
    } else {
        const int sh = n - 53;
        mant = (unsigned long long)(u >> sh);
        const unsigned __int128 rem = u & (((unsigned __int128)1 << sh) - 1);
        const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
        if (rem > half || (rem == half && (mant & 1ull))) {
            ++mant;
            if (mant == (1ull << 53)) {
                mant >>= 1;
                ++e;
            }
        }
    }
    if (e > 1023) return __longlong_as_double((long long)(sgn | 0x7ff0000000000000ull));
    if (e < -1022) {
        const double r = ldexp((double)mant, e - 52);
        return sgn ? -r : r;
    }
    return __longlong_as_double((long long)(sgn | ((unsigned long long)(e + 1023) << 52) | (mant & 0xfffffffffffffull)));
}

// the warp group of row o (0 <= o < BROWS) of a chunk in the digit store
__host__ __device__ __forceinline__ int dg_group(int o) { return (o & (XT - 1)) >> 5; }

}  // namespace qs3
