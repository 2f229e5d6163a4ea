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
// Pieces of v = x~ + 2^55 for x~ = RNE(x * 2^(52 - e)) straight from the bit
// pattern (same value as split_pieces(scale_round(bits, e))): the significand
// shifted right by s = e - ilogb(x) with round-half-even folded into one add,
// q = (sig + 2^(s-1) - 1 + lsb) >> s, lsb = bit s of sig.
__device__ __forceinline__ Pieces scale_split(uint64_t bits, int e) {
    const uint32_t E = (uint32_t)(bits >> 52) & 0x7FFu;
    const uint64_t sig = (bits & ((1ull << 52) - 1)) | ((uint64_t)(E != 0) << 52);
    const int s = e + 1023 - (int)(E ? E : 1u);
    uint64_t q;
    if (s <= 0) {
        q = sig << (-s);  // only when x is subnormal and leads its column
    } else {
        const int sc = s < 63 ? s : 63;  // sig < 2^53: any shift >= 54 rounds to 0
        const uint64_t lsb = (sig >> sc) & 1ull;
        q = (sig + ((1ull << (sc - 1)) - 1ull) + lsb) >> sc;
    }
    const uint64_t v = (bits >> 63) ? (1ull << 55) - q : (1ull << 55) + q;
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
// Lazily reduced residue: t - floor(t mu / 2^32) m lies in [0, 2m) for the
// unbiased piece sum t = p0 + p1 2^20 + p2 2^40 (mod m) < 2^32 (no correction step).
__device__ __forceinline__ uint32_t residue_lazy(const Pieces &pc, uint32_t m, uint32_t mu, uint32_t c20,
                                                 uint32_t c40) {
    uint32_t t = pc.p0 + pc.p1 * c20 + pc.p2 * c40;
    return t - __umulhi(t, mu) * m;
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

// ---------------------------------------------------------------------------
// Lean Kulisch finish for the FP8 path (Algorithm 2), from the 21 FP32 Phase-A
// accumulators of one scalar output, each holding 2^23 + P_s (s < 15) or
// 2^23 + Q_t (t < 6) so that its bit pattern is 0x4B000000 + P (P < 2^23).
//   E = sum_s P_s 256^s (mod 2^128)       -- 15 wide multiply-adds
//   z_acc = sum_t Q_t 256^t (mod 2^64)    -- exact, z_acc < 2^63
//   zhat = floor((z_acc + 2^47) / 2^48);  R = E - zhat M  (mod 2^128)
// The two-sided correction is only needed when z_acc / 2^48 lies within 2^-33
// of a rounding boundary (the lift error is below 2^-34 for canonical
// residues); that rare case, and results that would be subnormal or overflow,
// take the general 128-bit path.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double kulisch_pack_fp8(const uint32_t *wv, const ModConsts &mc, int et,
                                                   const uint32_t (&ebias)[4], uint64_t zbias) {
    uint64_t a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    a0 += (uint64_t)wv[0];
    a0 += (uint64_t)wv[1] * 256u;
    a0 += (uint64_t)wv[2] * 65536u;
    a0 += (uint64_t)wv[3] * 16777216u;
    a1 += (uint64_t)wv[4];
    a1 += (uint64_t)wv[5] * 256u;
    a1 += (uint64_t)wv[6] * 65536u;
    a1 += (uint64_t)wv[7] * 16777216u;
    a2 += (uint64_t)wv[8];
    a2 += (uint64_t)wv[9] * 256u;
    a2 += (uint64_t)wv[10] * 65536u;
    a2 += (uint64_t)wv[11] * 16777216u;
    a3 += (uint64_t)wv[12];
    a3 += (uint64_t)wv[13] * 256u;
    a3 += (uint64_t)wv[14] * 65536u;
    // 128-bit words of the biased sum, then remove the constant bias
    uint32_t w0 = (uint32_t)a0;
    uint64_t t = (a0 >> 32) + a1;
    uint32_t w1 = (uint32_t)t;
    t = (t >> 32) + a2;
    uint32_t w2 = (uint32_t)t;
    t = (t >> 32) + a3;
    uint32_t w3 = (uint32_t)t;
    uint64_t z = (uint64_t)wv[15] + (uint64_t)wv[16] * 256u + (uint64_t)wv[17] * 65536u +
                 (uint64_t)wv[18] * 16777216u + ((uint64_t)wv[19] << 32) + ((uint64_t)wv[20] << 40);
    z -= zbias;
    const uint64_t zr = z + (1ull << 47);
    const uint32_t zhat = (uint32_t)(zr >> 48);
    const uint64_t frac = zr & ((1ull << 48) - 1);
    // R = E - bias - zhat M  (mod 2^128)
    uint64_t p0 = (uint64_t)zhat * mc.M32[0];
    uint64_t p1 = (uint64_t)zhat * mc.M32[1] + (p0 >> 32);
    uint64_t p2 = (uint64_t)zhat * mc.M32[2] + (p1 >> 32);
    uint32_t p3 = zhat * mc.M32[3] + (uint32_t)(p2 >> 32);
    uint32_t s0, s1, s2, s3;
    {
        // s = zhat M + bias (128-bit add), then r = w - s
        asm("add.cc.u32 %0, %4, %8;\n\taddc.cc.u32 %1, %5, %9;\n\taddc.cc.u32 %2, %6, %10;\n\taddc.u32 %3, %7, %11;"
            : "=r"(s0), "=r"(s1), "=r"(s2), "=r"(s3)
            : "r"((uint32_t)p0), "r"((uint32_t)p1), "r"((uint32_t)p2), "r"(p3), "r"(ebias[0]), "r"(ebias[1]),
              "r"(ebias[2]), "r"(ebias[3]));
    }
    uint32_t r0, r1, r2, r3;
    asm("sub.cc.u32 %0, %4, %8;\n\tsubc.cc.u32 %1, %5, %9;\n\tsubc.cc.u32 %2, %6, %10;\n\tsubc.u32 %3, %7, %11;"
        : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
        : "r"(w0), "r"(w1), "r"(w2), "r"(w3), "r"(s0), "r"(s1), "r"(s2), "r"(s3));
    const bool near = frac < (1ull << 15) || frac >= (1ull << 48) - (1ull << 15);
    if (near) {
        i128 R = (i128)((((u128)r3) << 96) | (((u128)r2) << 64) | (((u128)r1) << 32) | (u128)r0);
        u128 M = u128_from_words(mc.M32);
        i128 half = (i128)u128_from_words(mc.halfM32);
        if (R >= half) R -= (i128)M;
        if (R < -half) R += (i128)M;
        return pack_rne(R, et);
    }
    // fast pack: |R| < 2^117, normal result
    const bool neg = (int32_t)r3 < 0;
    if (neg) {
        asm("sub.cc.u32 %0, 0, %0;\n\tsubc.cc.u32 %1, 0, %1;\n\tsubc.cc.u32 %2, 0, %2;\n\tsubc.u32 %3, 0, %3;"
            : "+r"(r0), "+r"(r1), "+r"(r2), "+r"(r3));
    }
    uint64_t hi = ((uint64_t)r3 << 32) | r2, lo = ((uint64_t)r1 << 32) | r0;
    uint64_t top;
    bool sticky;
    int L;
    if (hi) {
        int lz = __clzll((long long)hi);
        top = lz ? (hi << lz) | (lo >> (64 - lz)) : hi;
        sticky = (lo << lz) != 0;
        L = 128 - lz;
    } else {
        if (lo == 0) return 0.0;
        int lz = __clzll((long long)lo);
        top = lo << lz;
        sticky = false;
        L = 64 - lz;
    }
    uint64_t mant = top >> 11;
    const uint32_t rbit = (uint32_t)(top >> 10) & 1u;
    sticky = sticky || (top & 0x3FFull);
    mant += rbit & (uint32_t)(sticky | (mant & 1));
    int E2 = L - 53 + et + 1075;  // biased exponent of the result
    if (mant >> 53) {
        mant >>= 1;
        E2 += 1;
    }
    if (E2 < 1 || E2 > 2046) {  // subnormal or overflow: general path
        i128 R = (i128)((((u128)r3) << 96) | (((u128)r2) << 64) | (((u128)r1) << 32) | (u128)r0);
        return pack_rne(neg ? -R : R, et);
    }
    const uint64_t bits = ((uint64_t)neg << 63) | ((uint64_t)E2 << 52) | (mant & ((1ull << 52) - 1));
    return __longlong_as_double((long long)bits);
}

// Straight-line lift and pack of the common case of kulisch_pack_fp8, from the
// words w0..w3 of the deposited sum (mod 2^128), the six w_k partials wq (FP32
// bit patterns 2^23 + Q_t) and the constant `ebias` to remove (deposit biases
// and the residue offset): no early exits, so the compiler can interleave two
// outputs' chains.  Sets `slow` (and returns an unspecified value) when the
// general finish is needed: lift near a rounding boundary, |R| < 2^64, or a
// result that is subnormal or overflows; Rw (R = E - ebias - zhat M mod 2^128)
// and near_out then feed kulisch_finish_general.
// zhat_out (debug builds): receives the lift quotient.
__device__ __forceinline__ double lift_pack_fast(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3,
                                                 const uint32_t *wq, const ModConsts &mc, int et,
                                                 const uint32_t (&ebias)[4], uint64_t zbias, bool &slow,
                                                 uint32_t (&Rw)[4], bool &near_out, uint32_t *zhat_out = nullptr) {
    uint64_t z = (uint64_t)wq[0] + (uint64_t)wq[1] * 256u + (uint64_t)wq[2] * 65536u +
                 (uint64_t)wq[3] * 16777216u + ((uint64_t)wq[4] << 32) + ((uint64_t)wq[5] << 40);
    z -= zbias;
    const uint64_t zr = z + (1ull << 47);
    const uint32_t zhat = (uint32_t)(zr >> 48);
    if (zhat_out) *zhat_out = zhat;
    const uint64_t frac = zr & ((1ull << 48) - 1);
    uint64_t p0 = (uint64_t)zhat * mc.M32[0];
    uint64_t p1 = (uint64_t)zhat * mc.M32[1] + (p0 >> 32);
    uint64_t p2 = (uint64_t)zhat * mc.M32[2] + (p1 >> 32);
    uint32_t p3 = zhat * mc.M32[3] + (uint32_t)(p2 >> 32);
    uint32_t s0, s1, s2, s3, r0, r1, r2, r3;
    asm("add.cc.u32 %0, %4, %8;\n\taddc.cc.u32 %1, %5, %9;\n\taddc.cc.u32 %2, %6, %10;\n\taddc.u32 %3, %7, %11;"
        : "=r"(s0), "=r"(s1), "=r"(s2), "=r"(s3)
        : "r"((uint32_t)p0), "r"((uint32_t)p1), "r"((uint32_t)p2), "r"(p3), "r"(ebias[0]), "r"(ebias[1]),
          "r"(ebias[2]), "r"(ebias[3]));
    asm("sub.cc.u32 %0, %4, %8;\n\tsubc.cc.u32 %1, %5, %9;\n\tsubc.cc.u32 %2, %6, %10;\n\tsubc.u32 %3, %7, %11;"
        : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
        : "r"(w0), "r"(w1), "r"(w2), "r"(w3), "r"(s0), "r"(s1), "r"(s2), "r"(s3));
    const bool near = frac < (1ull << 15) || frac >= (1ull << 48) - (1ull << 15);
    Rw[0] = r0;
    Rw[1] = r1;
    Rw[2] = r2;
    Rw[3] = r3;
    near_out = near;
    // |R| by a conditional two's-complement negation without branches
    const uint32_t neg = r3 >> 31, msk = 0u - neg;
    r0 ^= msk;
    r1 ^= msk;
    r2 ^= msk;
    r3 ^= msk;
    asm("add.cc.u32 %0, %0, %4;\n\taddc.cc.u32 %1, %1, 0;\n\taddc.cc.u32 %2, %2, 0;\n\taddc.u32 %3, %3, 0;"
        : "+r"(r0), "+r"(r1), "+r"(r2), "+r"(r3)
        : "r"(neg));
    const uint64_t hi = ((uint64_t)r3 << 32) | r2, lo = ((uint64_t)r1 << 32) | r0;
    const int lz = __clzll((long long)(hi | 1ull));
    const uint64_t top = (hi << lz) | ((lo >> 1) >> (63 - lz));
    bool sticky = (lo << lz) != 0;
    uint64_t mant = top >> 11;
    const uint32_t rbit = (uint32_t)(top >> 10) & 1u;
    sticky = sticky || (top & 0x3FFull);
    mant += rbit & (uint32_t)(sticky | (mant & 1));
    int E2 = (128 - lz) - 53 + et + 1075;
    const uint32_t ovf = (uint32_t)(mant >> 53);
    mant >>= ovf;
    E2 += (int)ovf;
    slow = near || hi == 0 || E2 < 1 || E2 > 2046;
    const uint64_t bits = ((uint64_t)neg << 63) | ((uint64_t)(uint32_t)E2 << 52) | (mant & ((1ull << 52) - 1));
    return __longlong_as_double((long long)bits);
}

// Straight-line form of the common case of kulisch_pack_fp8: the deposits of
// the 15 slices in four 64-bit partial sums of four slices each (Eq. accwidth's
// grouping), assembled into 128-bit words, then lift_pack_fast.  Otherwise the
// result equals kulisch_pack_fp8's bit for bit.
__device__ __forceinline__ double kulisch_pack_fp8_fast(const uint32_t *wv, const ModConsts &mc, int et,
                                                        const uint32_t (&ebias)[4], uint64_t zbias, bool &slow,
                                                        uint32_t (&Rw)[4], bool &near_out,
                                                        uint32_t *zhat_out = nullptr) {
    uint64_t a0 = (uint64_t)wv[0];
    a0 += (uint64_t)wv[1] * 256u;
    a0 += (uint64_t)wv[2] * 65536u;
    a0 += (uint64_t)wv[3] * 16777216u;
    uint64_t a1 = (uint64_t)wv[4];
    a1 += (uint64_t)wv[5] * 256u;
    a1 += (uint64_t)wv[6] * 65536u;
    a1 += (uint64_t)wv[7] * 16777216u;
    uint64_t a2 = (uint64_t)wv[8];
    a2 += (uint64_t)wv[9] * 256u;
    a2 += (uint64_t)wv[10] * 65536u;
    a2 += (uint64_t)wv[11] * 16777216u;
    uint64_t a3 = (uint64_t)wv[12];
    a3 += (uint64_t)wv[13] * 256u;
    a3 += (uint64_t)wv[14] * 65536u;
    const uint32_t w0 = (uint32_t)a0;
    uint64_t t = (a0 >> 32) + a1;
    const uint32_t w1 = (uint32_t)t;
    t = (t >> 32) + a2;
    const uint32_t w2 = (uint32_t)t;
    t = (t >> 32) + a3;
    const uint32_t w3 = (uint32_t)t;
    return lift_pack_fast(w0, w1, w2, w3, wv + 15, mc, et, ebias, zbias, slow, Rw, near_out, zhat_out);
}

// The centred CRT value from the lifted words of lift_pack_fast: the
// two-sided correction where the lift was near a rounding boundary (as
// kulisch_finish_general applies it before packing).
__device__ __forceinline__ i128 lift_centre(const uint32_t *Rw, bool near, const ModConsts &mc) {
    i128 R = (i128)((((u128)Rw[3]) << 96) | (((u128)Rw[2]) << 64) | (((u128)Rw[1]) << 32) | (u128)Rw[0]);
    if (near) {
        const u128 M = u128_from_words(mc.M32);
        const i128 half = (i128)u128_from_words(mc.halfM32);
        if (R >= half) R -= (i128)M;
        if (R < -half) R += (i128)M;
    }
    return R;
}

// General finish from R = E - bias - zhat M (mod 2^128): the two-sided
// correction when the lift was near a rounding boundary, then the correctly
// rounded pack with gradual underflow and overflow (as kulisch_pack_fp8).
__device__ __forceinline__ double kulisch_finish_general(uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3,
                                                         bool near, int et, const ModConsts &mc) {
    i128 R = (i128)((((u128)r3) << 96) | (((u128)r2) << 64) | (((u128)r1) << 32) | (u128)r0);
    if (near) {
        const u128 M = u128_from_words(mc.M32);
        const i128 half = (i128)u128_from_words(mc.halfM32);
        if (R >= half) R -= (i128)M;
        if (R < -half) R += (i128)M;
    }
    return pack_rne(R, et);
}

}  // namespace obfft
