// Device helpers shared by the stage kernels: deconstruction of fp64 inputs
// into exponent-scaled integers, modular reduction, the Kulisch/lift finish
// and the correctly rounded pack.  All integer, no FP64 arithmetic.
#pragma once
#include <stdint.h>

#include "obfft_internal.h"

namespace obfft {

typedef unsigned __int128 u128;
typedef __int128 i128;

constexpr int LEAD_ZERO = -100000;  // ilogb stand-in for 0.0

// ilogb(|x|) from the bit pattern, exact for subnormals; LEAD_ZERO for 0.
__device__ __forceinline__ int lead_exponent(uint64_t bits) {
    uint32_t E = (uint32_t)(bits >> 52) & 0x7FFu;
    uint64_t f = bits & ((1ull << 52) - 1);
    if (E) return (int)E - 1023;
    if (f == 0) return LEAD_ZERO;
    return (63 - __clzll((long long)f)) - 1074;
}

// x~ = RNE(x * 2^(52 - e)) for a column exponent e >= ilogb(|x|) (Sec. deconstruction;
// |x~| < 2^53).  Pure integer: the significand shifted right with
// round-half-even on the dropped bits.
__device__ __forceinline__ int64_t scale_round(uint64_t bits, int e) {
    uint32_t E = (uint32_t)(bits >> 52) & 0x7FFu;
    uint64_t f = bits & ((1ull << 52) - 1);
    uint64_t sig = E ? (f | (1ull << 52)) : f;
    int Eeff = E ? (int)E : 1;
    int s = e + 1023 - Eeff;  // right shift amount
    uint64_t q;
    if (s <= 0) {
        q = sig << (-s);
    } else if (s >= 64) {
        q = 0;
    } else {
        q = sig >> s;
        uint64_t rem = sig & ((1ull << s) - 1);
        uint64_t half = 1ull << (s - 1);
        q += (rem > half) | ((rem == half) & (q & 1));
    }
    int64_t v = (int64_t)q;
    return (bits >> 63) ? -v : v;
}

// Residue of a deconstructed integer x~ (|x~| < 2^54) modulo m, canonical.
// v = x~ + 2^55 is split into 20/20/16-bit pieces; the piece weights are
// reduced mod m on the host, so one 32-bit sum and one Barrett step remain.
struct Pieces { uint32_t p0, p1, p2; };
__device__ __forceinline__ Pieces split_pieces(int64_t xt) {
    uint64_t v = (uint64_t)(xt + (1ll << 55));
    Pieces r;
    r.p0 = (uint32_t)v & 0xFFFFFu;
    r.p1 = (uint32_t)(v >> 20) & 0xFFFFFu;
    r.p2 = (uint32_t)(v >> 40);
    return r;
}
__device__ __forceinline__ uint32_t barrett(uint32_t t, uint32_t m, uint32_t mu) {
    uint32_t q = __umulhi(t, mu);
    uint32_t r = t - q * m;
    return r >= m ? r - m : r;
}
__device__ __forceinline__ uint32_t residue(const Pieces &pc, uint32_t m, uint32_t mu, uint32_t c20,
                                            uint32_t c40, uint32_t cneg) {
    uint32_t t = pc.p0 + cneg + pc.p1 * c20 + pc.p2 * c40;  // < 2^32
    return barrett(t, m, mu);
}
// Canonical residue of a signed 32-bit value with |x| < 2^27.
__device__ __forceinline__ uint32_t mod_signed27(int32_t x, uint32_t m, uint32_t mu, uint32_t off27) {
    return barrett((uint32_t)(x + (int32_t)off27), m, mu);
}

// RNE(R * 2^et) as an IEEE double, gradual underflow, |R| < 2^127.
__device__ __forceinline__ double pack_rne(i128 R, int et) {
    if (R == 0) return 0.0;
    uint64_t sign = 0;
    u128 a = (u128)R;
    if (R < 0) {
        sign = 1ull << 63;
        a = (u128)(-R);
    }
    uint64_t hi = (uint64_t)(a >> 64), lo = (uint64_t)a;
    int L = hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo);
    int d = L - 53;
    int dsub = -1074 - et;
    bool sub = dsub >= d;
    if (sub) d = dsub;
    uint64_t q;
    if (d <= 0) {
        q = (uint64_t)(a << (-d));
    } else if (d > L) {
        q = 0;
    } else {
        u128 qq = a >> d;
        u128 rem = a & ((((u128)1) << d) - 1);
        u128 half = ((u128)1) << (d - 1);
        q = (uint64_t)qq;
        q += (rem > half) | ((rem == half) & (q & 1));
    }
    uint64_t bits;
    if (sub) {
        bits = q;  // quantum 2^-1074: subnormal or (q >= 2^52) the smallest binades
    } else {
        if (q >> 53) {
            q >>= 1;
            d += 1;
        }
        int biased = et + d + 1075;
        if (biased >= 2047)
            bits = 0x7FF0000000000000ull;
        else
            bits = ((uint64_t)biased << 52) | (q & ((1ull << 52) - 1));
    }
    return __longlong_as_double((long long)(bits | sign));
}

__device__ __forceinline__ u128 u128_from_words(const uint32_t w[4]) {
    return ((u128)w[3] << 96) | ((u128)w[2] << 64) | ((u128)w[1] << 32) | (u128)w[0];
}

// Two-sided centered lift (Algorithm 2): R <- E - zhat M, then one correction
// towards [-M/2, M/2).  Arithmetic is modulo 2^128, valid because the centered
// result and every intermediate R are below 2^127 in magnitude.
__device__ __forceinline__ i128 lift_two_sided(u128 E, int64_t zhat, const ModConsts &mc) {
    u128 M = u128_from_words(mc.M32);
    i128 half = (i128)u128_from_words(mc.halfM32);
    i128 R = (i128)(E - (u128)(i128)zhat * M);
    if (R >= half) R -= (i128)M;
    if (R < -half) R += (i128)M;
    return R;
}

}  // namespace obfft
