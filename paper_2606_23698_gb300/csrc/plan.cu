// Host side of libobfft: constant generation, plan creation and the C ABI.
//
// Constants (all computed here, independently of any test code):
//   * moduli, M = prod m_k, CRT idempotents u_k = (M/m_k) y_k with
//     y_k = (M/m_k)^-1 mod m_k (Eq. fcrt), their byte slices (Eq. slicing),
//     lift weights w_k = round(2^48 u_k / M) = round(2^48 y_k / m_k).
//   * quantised DFT / twiddle-fused matrices RNE(2^52 omega) (Bailey
//     paragraph, Eq. twiddle-fusion), from double-double sin/cos with an exact
//     octant reduction of the rational angle m / N.
//   * INT8-mode limb tables in the register order of mma.m16n8k32 A fragments.
//   * FP64-comparator twiddle tables.
// Build flag: this file relies on separately rounded double operations
// (compile with -ffp-contract=off).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "obfft_internal.h"

namespace obfft {

const int kModuli[NMOD] = {2039, 2029, 2027, 1089, 1024, 961, 841, 625, 529, 511, 491, 487};
// The six-member subset of the Rev-34 set with log2 M = 62.6 (Sec. "Ozaki-II for FP32").
const int kModuli32[NMOD32] = {2039, 2029, 2027, 1024, 961, 841};

static thread_local std::string g_last_error = "no error";

obfft_status set_error(obfft_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

typedef unsigned __int128 u128;

// ------------------------------------------------------------ modular helpers
static int64_t inv_mod(int64_t a, int64_t m) {
    int64_t t = 0, newt = 1, r = m, newr = ((a % m) + m) % m;
    while (newr) {
        int64_t qq = r / newr, tmp;
        tmp = t - qq * newt; t = newt; newt = tmp;
        tmp = r - qq * newr; r = newr; newr = tmp;
    }
    return t < 0 ? t + m : t;
}
static int64_t pow2_mod(int e, int64_t m) {
    int64_t r = 1 % m;
    for (int i = 0; i < e; i++) r = (r * 2) % m;
    return r;
}

void make_mod_consts(ModConsts *mc) {
    memset(mc, 0, sizeof(*mc));
    u128 M = 1;
    for (int k = 0; k < NMOD; k++) M *= (u128)kModuli[k];
    for (int k = 0; k < NMOD; k++) {
        uint32_t m = (uint32_t)kModuli[k];
        mc->m[k] = m;
        mc->barrett[k] = (uint32_t)((1ull << 32) / m);
        mc->off27[k] = (uint32_t)((((1ull << 27) + m - 1) / m) * m);
        mc->c20[k] = (uint32_t)pow2_mod(20, m);
        mc->c40[k] = (uint32_t)pow2_mod(40, m);
        mc->c55neg[k] = (uint32_t)((m - pow2_mod(55, m)) % m);
        u128 Mk = M / m;
        int64_t y = inv_mod((int64_t)(Mk % m), m);
        u128 u = Mk * (u128)y;  // < M < 2^118
        for (int w = 0; w < 4; w++) mc->u32[k][w] = (uint32_t)(u >> (32 * w));
        for (int s = 0; s < S_RAW; s++) mc->us[k][s] = (uint8_t)(u >> (8 * s));
        // w_k = floor(2^48 y_k / m_k + 1/2) = floor((2^49 y_k + m_k) / (2 m_k))
        u128 wk = (((u128)y << 49) + m) / ((u128)2 * m);
        for (int t = 0; t < S_FRAC; t++) mc->ws[k][t] = (uint8_t)(wk >> (8 * t));
        mc->yk_over_mk[k] = (float)((double)y / (double)m);
        mc->fm[k] = (float)m;
        mc->finv[k] = (float)(1.0 / (double)m);
        mc->foff[k] = -(float)(8388608 + pow2_mod(55, m));
        int sq = 0;
        for (int t = 1; t * t <= (int)m; t++)
            if (t * t == (int)m) sq = t;
        mc->fsq[k] = (float)sq;
        mc->fc3[k] = (float)(4096 % m);
        mc->fc4[k] = (float)(65536 % m);
        for (int i = 0; i < 7; i++) {
            const uint32_t c = (uint32_t)pow2_mod(8 * i, m);  // < 2^11
            mc->b8lo[k][i / 4] |= (c & 0xFFu) << (8 * (i % 4));
            mc->b8hi[k][i / 4] |= (c >> 8) << (8 * (i % 4));
        }
    }
    for (int w = 0; w < 4; w++) {
        mc->M32[w] = (uint32_t)(M >> (32 * w));
        mc->halfM32[w] = (uint32_t)((M >> 1) >> (32 * w));
    }
    u128 kb = 0;
    for (int s = 0; s < S_RAW; s++) kb += (u128)0x4B000000u << (8 * s);  // wraps mod 2^128
    kb += (u128)RES_OFFSET;
    for (int w = 0; w < 4; w++) mc->kbias[w] = (uint32_t)(kb >> (32 * w));
    uint64_t zb = 0;
    for (int t = 0; t < S_FRAC; t++) zb += (uint64_t)0x4B000000u << (8 * t);  // mod 2^64
    mc->zbias[0] = (uint32_t)zb;
    mc->zbias[1] = (uint32_t)(zb >> 32);
}

// CRT constants of the FP32-precision variant: u_k < M < 2^63 as 8 byte
// slices, w_k = round(2^24 u_k / M) = round(2^24 y_k / m_k) as 3 byte slices.
static void make_crt_consts32(uint8_t us[NMOD32][S_RAW32], uint8_t ws[NMOD32][S_FRAC32], uint64_t *Mout) {
    u128 M = 1;
    for (int k = 0; k < NMOD32; k++) M *= (u128)kModuli32[k];
    for (int k = 0; k < NMOD32; k++) {
        const int64_t m = kModuli32[k];
        const u128 Mk = M / (u128)m;
        const int64_t y = inv_mod((int64_t)(Mk % (u128)m), m);
        const u128 u = Mk * (u128)y;
        for (int s = 0; s < S_RAW32; s++) us[k][s] = (uint8_t)(u >> (8 * s));
        const u128 wk = (((u128)y << 25) + (u128)m) / ((u128)2 * (u128)m);
        for (int t = 0; t < S_FRAC32; t++) ws[k][t] = (uint8_t)(wk >> (8 * t));
    }
    *Mout = (uint64_t)M;
}

// --------------------------------------------------- double-double sin / cos
struct dd { double hi, lo; };
static dd two_sum(double a, double b) {
    double s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
static dd qts(double a, double b) {
    double s = a + b;
    return {s, b - (s - a)};
}
static dd dd_add(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi), t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = qts(s.hi, s.lo);
    s.lo += t.lo;
    return qts(s.hi, s.lo);
}
static dd dd_mul(dd a, dd b) {
    double p = a.hi * b.hi;
    double e = fma(a.hi, b.hi, -p) + (a.hi * b.lo + a.lo * b.hi);
    return qts(p, e);
}
static dd dd_div_int(dd a, double d) {  // a / d for an exactly representable d
    double q1 = a.hi / d;
    dd prod = {q1 * d, fma(q1, d, -q1 * d)};
    dd r = dd_add(a, {-prod.hi, -prod.lo});
    double q2 = r.hi / d;
    return qts(q1, q2);
}
static const dd DD_PI = {3.141592653589793116, 1.2246467991473532e-16};

// cos and sin of phi = pi * num / den, |num / den| <= 1/4
static void dd_cos_sin(int64_t num, int64_t den, dd *c, dd *s) {
    dd r = dd_div_int({(double)num, 0.0}, (double)den);
    dd phi = dd_mul(DD_PI, r);
    dd phi2 = dd_mul(phi, phi);
    dd cs = {1.0, 0.0}, sn = phi;
    dd term = {1.0, 0.0};
    for (int n = 1; n < 30; n++) {  // cos: term_n = -term_{n-1} phi^2 / ((2n-1)(2n))
        term = dd_div_int(dd_mul(term, phi2), (double)((2 * n - 1) * (2 * n)));
        term = {-term.hi, -term.lo};
        cs = dd_add(cs, term);
    }
    term = phi;
    for (int n = 1; n < 30; n++) {
        term = dd_div_int(dd_mul(term, phi2), (double)((2 * n) * (2 * n + 1)));
        term = {-term.hi, -term.lo};
        sn = dd_add(sn, term);
    }
    *c = cs;
    *s = sn;
}

// cos / sin (2 pi m / N) with exact reduction to |phi| <= pi/4
static void dd_cos_sin_2pi(int64_t m, int64_t N, dd *c, dd *s) {
    m %= N;
    if (m < 0) m += N;
    int64_t k = (8 * m + N) / (2 * N);  // round(4 m / N)
    int64_t num = 4 * m - k * N;        // phi = pi num / (2N)
    dd cc, ss;
    if (num == 0) {
        cc = {1.0, 0.0};
        ss = {0.0, 0.0};
    } else {
        dd_cos_sin(num, 2 * N, &cc, &ss);
    }
    switch (k % 4) {
        case 0: *c = cc; *s = ss; break;
        case 1: *c = {-ss.hi, -ss.lo}; *s = cc; break;
        case 2: *c = {-cc.hi, -cc.lo}; *s = {-ss.hi, -ss.lo}; break;
        default: *c = ss; *s = {-cc.hi, -cc.lo}; break;
    }
}

static int64_t rne_dd_times_2p(dd v, int pexp) {
    double hi = ldexp(v.hi, pexp), lo = ldexp(v.lo, pexp);
    double n = rint(hi);
    double d = (hi - n) + lo;  // hi - n exact
    if (d > 0.5) n += 1.0;
    else if (d < -0.5) n -= 1.0;
    else if (d == 0.5 || d == -0.5) {
        double cand = d > 0 ? n + 1.0 : n - 1.0;
        if (fmod(cand, 2.0) == 0.0) n = cand;
    }
    return (int64_t)n;
}

void quantised_twiddle_scaled(int64_t m, int64_t N, int dir, int sexp, int64_t *re, int64_t *im) {
    dd c, s;
    dd_cos_sin_2pi(m, N, &c, &s);
    *re = rne_dd_times_2p(c, sexp);
    int64_t si = rne_dd_times_2p(s, sexp);
    *im = dir < 0 ? -si : si;
}
void quantised_twiddle(int64_t m, int64_t N, int dir, int64_t *re, int64_t *im) {
    quantised_twiddle_scaled(m, N, dir, 52, re, im);
}

// ------------------------------------------------------------ table building
static inline int64_t modc(int64_t x, int64_t m) {
    int64_t r = x % m;
    return r < 0 ? r + m : r;
}

// INT8 limb table for one stage.  F: [groups][Kout][K][2] int64, K == Kout.
// Output layout [g][mod][prod][mt][part][kb][lane] uint4 (16 bytes each).
static std::vector<uint32_t> build_int8_table(const std::vector<int64_t> &F, int groups, int K) {
    // K <= 16: the G and H columns share one k32 block (slots 0..15 and 16..31)
    const int KPAD = K <= 16 ? 16 : (K <= 32 ? 32 : 64);
    const int KB2 = 2 * KPAD / 32;
    const int MT = (K + 15) / 16;
    std::vector<uint32_t> out((size_t)groups * NMOD * 3 * MT * 2 * KB2 * 32 * 4, 0u);
    std::vector<int32_t> limb[2];  // [row 16*MT][2*KPAD] per part
    for (int g = 0; g < groups; g++)
        for (int k = 0; k < NMOD; k++) {
            const int64_t m = kModuli[k];
            for (int pd = 0; pd < 3; pd++) {
                limb[0].assign((size_t)16 * MT * 2 * KPAD, 0);
                limb[1].assign((size_t)16 * MT * 2 * KPAD, 0);
                for (int r = 0; r < K; r++)
                    for (int j = 0; j < K; j++) {
                        const int64_t *e = &F[(((size_t)g * K + r) * K + j) * 2];
                        int64_t a = pd == 0 ? e[0] : pd == 1 ? e[1] : e[0] + e[1];
                        int64_t G = modc(a, m), H = (256 * G) % m;
                        int64_t vals[2] = {G, H};
                        for (int gh = 0; gh < 2; gh++) {
                            int64_t v = vals[gh];
                            int64_t hi = (v + 128) >> 8, lo = v - 256 * hi;  // lo in [-128,127], hi in [0,8]
                            size_t col = (size_t)gh * KPAD + j;
                            limb[0][(size_t)r * 2 * KPAD + col] = (int32_t)lo;
                            limb[1][(size_t)r * 2 * KPAD + col] = (int32_t)hi;
                        }
                    }
                for (int mt = 0; mt < MT; mt++)
                    for (int part = 0; part < 2; part++)
                        for (int kb = 0; kb < KB2; kb++)
                            for (int lane = 0; lane < 32; lane++) {
                                size_t idx = ((((((size_t)g * NMOD + k) * 3 + pd) * MT + mt) * 2 + part) * KB2 + kb) * 32 + lane;
                                for (int reg = 0; reg < 4; reg++) {
                                    int row = mt * 16 + (lane >> 2) + ((reg & 1) ? 8 : 0);
                                    int kc = kb * 32 + 4 * (lane & 3) + ((reg & 2) ? 16 : 0);
                                    uint32_t word = 0;
                                    for (int b = 0; b < 4; b++) {
                                        int32_t v = limb[part][(size_t)row * 2 * KPAD + kc + b];
                                        word |= ((uint32_t)(uint8_t)(int8_t)v) << (8 * b);
                                    }
                                    out[idx * 4 + reg] = word;
                                }
                            }
            }
        }
    return out;
}

// ------------------------------------------------------------ FP8 tables
static uint8_t e4m3_of_int(int v) {  // exact for |v| <= 16
    if (v == 0) return 0;
    uint8_t sgn = v < 0 ? 0x80 : 0;
    int a = v < 0 ? -v : v;
    int e = 31 - __builtin_clz((unsigned)a);
    int mant = ((a << 3) >> e) & 7;
    return (uint8_t)(sgn | ((e + 7) << 3) | mant);
}
static uint16_t f16_of_small(int v) {  // exact for 0 <= v < 2048
    if (v == 0) return 0;
    int e = 31 - __builtin_clz((unsigned)v);
    int mant = ((v << 10) >> e) & 0x3FF;
    return (uint16_t)(((e + 15) << 10) | mant);
}
static uint16_t f16_of_small_int(int v) {  // exact for |v| < 2048
    return v < 0 ? (uint16_t)(0x8000u | f16_of_small(-v)) : f16_of_small(v);
}
static int64_t rne_div(int64_t v, int64_t d) {  // round-half-even of v / d, d > 0
    int64_t q = v >= 0 ? v / d : -((-v) / d);
    int64_t r = v - q * d;
    if (2 * r > d || (2 * r == d && (q & 1))) q += 1;
    if (2 * r < -d || (2 * r == -d && (q & 1))) q -= 1;
    return q;
}
// balanced digits of a residue for modulus index k (same decomposition rules
// as the device: m = s^2 -> (h, l); 9-bit -> (d0, d1); 11-bit -> (d0, d1, d2))
static int fp8_digits(int k, int64_t v, int dig[3]) {
    const int64_t m = kModuli[k];
    if (k >= 3 && k < 9) {
        int64_t s = 0;
        while ((s + 1) * (s + 1) <= m) s++;
        int64_t h = rne_div(v, s);
        dig[0] = (int)h;
        dig[1] = (int)(v - s * h);
        return 2;
    }
    if (k >= 9) {
        int64_t d1 = rne_div(v, 16);
        dig[0] = (int)(v - 16 * d1);
        dig[1] = (int)d1;
        return 2;
    }
    int64_t d2 = rne_div(v, 256), r = v - 256 * d2, d1 = rne_div(r, 16);
    dig[0] = (int)(r - 16 * d1);
    dig[1] = (int)d1;
    dig[2] = (int)d2;
    return 3;
}

std::vector<uint8_t> build_fp8_planes(const std::vector<int64_t> &F, int groups, int K) {
    // Per modulus: for the x_R half, digit pairs (a_R digit, a_I digit); for
    // the x_I half, (-a_I digit, a_R digit); digits in class order (squares:
    // l before h).  Each plane is npad rows (outputs) x 32 bytes (K) in the
    // no-swizzle K-major layout; a pair of planes is one N = 2 npad operand
    // whose rows give the Re and Im accumulators side by side.
    const int npad = K <= 16 ? 16 : 32;
    const size_t planeB = (size_t)npad * 32;
    std::vector<uint8_t> out((size_t)groups * FP8_PLANES_PER_GROUP * planeB, 0);
    size_t off = 0;
    for (int g = 0; g < groups; g++)
        for (int k = 0; k < NMOD; k++) {
            const int64_t m = kModuli[k];
            const int nd = k < 3 ? 3 : 2;
            const bool square = k >= 3 && k < 9;
            for (int h = 0; h < 2; h++)
                for (int di = 0; di < nd; di++) {
                    const int d = square ? 1 - di : di;  // digit index of this position
                    for (int tb = 0; tb < 2; tb++) {
                        // h = 0: (a_R, a_I); h = 1: (-a_I, a_R)
                        const int sel = h == 0 ? (tb == 0 ? 0 : 1) : (tb == 0 ? 2 : 0);
                        const size_t pbase = off + (size_t)((h * nd + di) * 2 + tb) * planeB;
                        for (int n = 0; n < K; n++)
                            for (int j = 0; j < K; j++) {
                                const int64_t *e = &F[(((size_t)g * K + n) * K + j) * 2];
                                const int64_t a = sel == 0 ? e[0] : sel == 1 ? e[1] : -e[1];
                                const int64_t r = modc(a, m);
                                const int64_t v = 2 * r > m ? r - m : r;  // balanced
                                int dig[3];
                                fp8_digits(k, v, dig);
                                const size_t pos = pbase + (size_t)(n / 8) * 256 + (size_t)(j / 16) * 128 +
                                                   (n % 8) * 16 + j % 16;
                                out[pos] = e4m3_of_int(dig[d]);
                            }
                    }
                }
            off += (size_t)4 * nd * planeB;
        }
    return out;
}

// FP16-carrier constant planes.  Each balanced constant residue a splits as
// a = c0 + 32 c1 (c1 = RNE(a / 32), |c0| <= 16, |c1| <= 32: FP16-exact).  Per
// modulus: for the x_R half, digit pairs (a_R, a_I), for the x_I half
// (-a_I, a_R), digits low to high; each plane is npad rows (outputs) x npad
// FP16 values (K) in the no-swizzle K-major layout of 16-bit operands (8 x 8
// core matrices of 16 bytes, LBO 128 between K neighbours, SBO 16 npad between
// 8-row groups), so consecutive planes continue the rows of one operand.
std::vector<uint8_t> build_fp16_planes(const std::vector<int64_t> &F, int groups, int K, const int *moduli,
                                       int nmod) {
    const int npad = K <= 16 ? 16 : 32;
    const size_t planeB = (size_t)npad * npad * 2, sbo = (size_t)16 * npad;
    std::vector<uint8_t> out((size_t)groups * nmod * 8 * planeB, 0);
    size_t off = 0;
    for (int g = 0; g < groups; g++)
        for (int k = 0; k < nmod; k++) {
            const int64_t m = moduli[k];
            for (int h = 0; h < 2; h++)
                for (int d = 0; d < 2; d++)
                    for (int tb = 0; tb < 2; tb++) {
                        const int sel = h == 0 ? (tb == 0 ? 0 : 1) : (tb == 0 ? 2 : 0);
                        const size_t pbase = off + (size_t)((h * 2 + d) * 2 + tb) * planeB;
                        for (int n = 0; n < K; n++)
                            for (int j = 0; j < K; j++) {
                                const int64_t *e = &F[(((size_t)g * K + n) * K + j) * 2];
                                const int64_t a = sel == 0 ? e[0] : sel == 1 ? e[1] : -e[1];
                                const int64_t r = modc(a, m);
                                const int64_t v = 2 * r > m ? r - m : r;  // balanced
                                const int64_t c1 = rne_div(v, 32);
                                const int digit = (int)(d == 0 ? v - 32 * c1 : c1);
                                const uint16_t hv = f16_of_small_int(digit);
                                const size_t pos = pbase + (size_t)(n / 8) * sbo + (size_t)(j / 8) * 128 +
                                                   (n % 8) * 16 + (j % 8) * 2;
                                out[pos] = (uint8_t)(hv & 0xFF);
                                out[pos + 1] = (uint8_t)(hv >> 8);
                            }
                    }
            off += (size_t)8 * planeB;
        }
    return out;
}

// Phase A B-matrix: 48 rows (Re: 15 u-slices, 6 w-slices, 3 zero; Im: same)
// x 32 K (the Re and Im residues of modulus k at K = 2k and 2k + 1, then 8
// zero), FP16, K-major canonical layout (LBO 128, SBO 512).
std::vector<uint8_t> build_phase_a_b() {
    ModConsts mc;
    make_mod_consts(&mc);
    std::vector<uint8_t> out(48 * 64, 0);
    for (int n = 0; n < 48; n++) {
        int part = n / 24, col = n % 24;
        for (int kk = 0; kk < 32; kk++) {
            int val = 0;
            if (kk < 24 && (kk & 1) == part && col < 21) {
                int k = kk >> 1;
                val = col < S_RAW ? mc.us[k][col] : mc.ws[k][col - S_RAW];
            }
            uint16_t h = f16_of_small(val);
            size_t pos = (size_t)(n / 8) * 512 + (size_t)(kk / 8) * 128 + (n % 8) * 16 + (kk % 8) * 2;
            out[pos] = (uint8_t)(h & 0xFF);
            out[pos + 1] = (uint8_t)(h >> 8);
        }
    }
    return out;
}

// FP32 variant's Phase A B-matrix: 32 rows (Re: 8 u-slices, 3 w-slices, 5
// zero; Im: same) x 16 K (Re residues 0..5, Im residues 6..11, 4 zero), FP16,
// K-major canonical layout (LBO 128, SBO 256).
std::vector<uint8_t> build_phase_a_b32() {
    uint8_t us[NMOD32][S_RAW32], ws[NMOD32][S_FRAC32];
    uint64_t M;
    make_crt_consts32(us, ws, &M);
    std::vector<uint8_t> out(32 * 32, 0);
    for (int n = 0; n < 32; n++) {
        const int part = n / 16, col = n % 16;
        for (int kk = 0; kk < 16; kk++) {
            int val = 0;
            if (kk < 2 * NMOD32 && kk / NMOD32 == part && col < S_RAW32 + S_FRAC32) {
                const int k = kk % NMOD32;
                val = col < S_RAW32 ? us[k][col] : ws[k][col - S_RAW32];
            }
            const uint16_t h = f16_of_small(val);
            const size_t pos = (size_t)(n / 8) * 256 + (size_t)(kk / 8) * 128 + (n % 8) * 16 + (kk % 8) * 2;
            out[pos] = (uint8_t)(h & 0xFF);
            out[pos + 1] = (uint8_t)(h >> 8);
        }
    }
    return out;
}

// Quantised F_q and twiddle-fused F_p^(k2) at 2^sexp (52: the FP64 method, 23:
// its FP32-precision variant).
static void fill_matrices(AxisTables &t, int sexp) {
    const int p = t.p, q = t.q, n = t.n, dir = t.dir;
    t.Fq.assign((size_t)q * q * 2, 0);
    for (int k2 = 0; k2 < q; k2++)
        for (int j2 = 0; j2 < q; j2++)
            quantised_twiddle_scaled((int64_t)j2 * k2 % q, q, dir, sexp, &t.Fq[((size_t)k2 * q + j2) * 2],
                                     &t.Fq[((size_t)k2 * q + j2) * 2 + 1]);
    t.Fp.assign((size_t)q * p * p * 2, 0);
    for (int k2 = 0; k2 < q; k2++)
        for (int k1 = 0; k1 < p; k1++)
            for (int j1 = 0; j1 < p; j1++) {
                int64_t e = ((int64_t)j1 * ((int64_t)q * k1 + k2)) % n;
                size_t idx = (((size_t)k2 * p + k1) * p + j1) * 2;
                quantised_twiddle_scaled(e, n, dir, sexp, &t.Fp[idx], &t.Fp[idx + 1]);
            }
}

// Stages with K <= 16 run lpv > 1 lines per TMEM lane in the tcgen05 stage
// kernel (FP8 and FP16-carrier modes): their constant operand is the
// block-diagonal 32 x 32 matrix with the K x K matrix of each group at rows
// and columns 32 b / lpv (b < lpv), zero elsewhere.
static std::vector<int64_t> lane_blocks(const std::vector<int64_t> &F, int groups, int K, int lpv) {
    const int ks = 32 / lpv;
    std::vector<int64_t> P((size_t)groups * 32 * 32 * 2, 0);
    for (int g = 0; g < groups; g++)
        for (int b = 0; b < lpv; b++)
            for (int n = 0; n < K; n++)
                for (int j = 0; j < K; j++)
                    for (int c = 0; c < 2; c++)
                        P[(((size_t)g * 32 + ks * b + n) * 32 + ks * b + j) * 2 + c] =
                            F[(((size_t)g * K + n) * K + j) * 2 + c];
    return P;
}

static cudaError_t upload(const void *host, size_t bytes, void **dev) {
    cudaError_t e = cudaMalloc(dev, bytes);
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dev, host, bytes, cudaMemcpyHostToDevice);
}

// Constant planes of both stages for the tcgen05 stage kernel: the layout for
// fp8_lines_per_lane(K) lines per lane, and for K <= 8 also the two-line one.
template <typename Build>
static cudaError_t upload_planes(AxisTables &t, Build build) {
    const int lq = fp8_lines_per_lane(t.q), lp = fp8_lines_per_lane(t.p);
    std::vector<uint8_t> s1 = build(t.Fq, 1, t.q, lq), s2 = build(t.Fp, t.q, t.p, lp);
    cudaError_t e = upload(s1.data(), s1.size(), &t.fp8_s1);
    if (e == cudaSuccess) e = upload(s2.data(), s2.size(), &t.fp8_s2);
    if (e == cudaSuccess && lq == 4) {
        s1 = build(t.Fq, 1, t.q, 2);
        e = upload(s1.data(), s1.size(), &t.fp8_s1_l2);
    }
    if (e == cudaSuccess && lp == 4) {
        s2 = build(t.Fp, t.q, t.p, 2);
        e = upload(s2.data(), s2.size(), &t.fp8_s2_l2);
    }
    return e;
}

static obfft_status build_tables(obfft_plan P, AxisTables &t) {
    fill_matrices(t, P->mode == OBFFT_MODE_FP32 ? 23 : 52);
    cudaError_t e = cudaSuccess;
    if (P->mode == OBFFT_MODE_INT8) {
        std::vector<uint32_t> s1 = build_int8_table(t.Fq, 1, t.q);
        std::vector<uint32_t> s2 = build_int8_table(t.Fp, t.q, t.p);
        t.int8_s1_bytes = s1.size() * 4;
        t.int8_s2_bytes = s2.size() * 4;
        e = upload(s1.data(), t.int8_s1_bytes, &t.int8_s1);
        if (e == cudaSuccess) e = upload(s2.data(), t.int8_s2_bytes, &t.int8_s2);
    } else if (P->mode == OBFFT_MODE_FP8) {
        e = fp8_upload_constants();
        if (e != cudaSuccess) return set_error(OBFFT_ERR_CUDA, std::string("FP8 constants: ") + cudaGetErrorString(e));
        e = upload_planes(t, [&](const std::vector<int64_t> &F, int groups, int K, int lpv) {
            return lpv > 1 ? build_fp8_planes(lane_blocks(F, groups, K, lpv), groups, 32) : build_fp8_planes(F, groups, K);
        });
    } else if (P->mode == OBFFT_MODE_FP16) {
        e = fp8_upload_constants();
        if (e != cudaSuccess) return set_error(OBFFT_ERR_CUDA, std::string("FP16 constants: ") + cudaGetErrorString(e));
        e = upload_planes(t, [&](const std::vector<int64_t> &F, int groups, int K, int lpv) {
            return lpv > 1 ? build_fp16_planes(lane_blocks(F, groups, K, lpv), groups, 32, kModuli, NMOD)
                           : build_fp16_planes(F, groups, K, kModuli, NMOD);
        });
    } else if (P->mode == OBFFT_MODE_FP32) {
        e = fp32_upload_constants();
        if (e != cudaSuccess) return set_error(OBFFT_ERR_CUDA, std::string("FP32 constants: ") + cudaGetErrorString(e));
        e = upload_planes(t, [&](const std::vector<int64_t> &F, int groups, int K, int lpv) {
            return lpv > 1 ? build_fp16_planes(lane_blocks(F, groups, K, lpv), groups, 32, kModuli32, NMOD32)
                           : build_fp16_planes(F, groups, K, kModuli32, NMOD32);
        });
    } else if (P->mode == OBFFT_MODE_FP32_NATIVE) {
        std::vector<float> tw;
        auto push = [&](int N) {
            for (int m = 0; m < N; m++) {
                dd c, s;
                dd_cos_sin_2pi(m, N, &c, &s);
                tw.push_back((float)c.hi);
                tw.push_back(t.dir < 0 ? -(float)s.hi : (float)s.hi);
            }
        };
        push(t.n);
        push(t.q);
        push(t.p);
        e = upload(tw.data(), tw.size() * sizeof(float), &t.tw);
    } else if (P->mode == OBFFT_MODE_FP64_NATIVE) {
        std::vector<double> tw;
        auto push = [&](int N) {
            for (int m = 0; m < N; m++) {
                dd c, s;
                dd_cos_sin_2pi(m, N, &c, &s);
                tw.push_back(c.hi);
                tw.push_back(t.dir < 0 ? -s.hi : s.hi);
            }
        };
        push(t.n);
        push(t.q);
        push(t.p);
        e = upload(tw.data(), tw.size() * sizeof(double), &t.tw);
    } else {
        return set_error(OBFFT_ERR_UNSUPPORTED_SIZE, "mode not available in this build");
    }
    if (e != cudaSuccess) return set_error(OBFFT_ERR_ALLOC, std::string("table upload: ") + cudaGetErrorString(e));
    return OBFFT_OK;
}

// FP64 twiddles exp(dir 2 pi i m / N), m < N, rounded from double-double
// (the values the FP64-native plans upload), for the no-allocation entry point.
void fp64_twiddles(int N, int dir, double2 *out) {
    for (int m = 0; m < N; m++) {
        dd c, s;
        dd_cos_sin_2pi(m, N, &c, &s);
        out[m] = make_double2(c.hi, dir < 0 ? -s.hi : s.hi);
    }
}

AxisTables *get_tables(obfft_plan P, int n, int pp, int qq, int dir) {
    for (auto &t : P->tables)
        if (t.n == n && t.p == pp && t.q == qq && t.dir == dir) return &t;
    return nullptr;
}

// Bailey split: q = smallest divisor >= sqrt(n), p = n / q; both <= kmax.
// Lengths above kmax^2 cannot factor within the limit and are rejected before
// the search, which then visits at most kmax candidates.
bool choose_split(int64_t n, AxisPlan *a, int kmax) {
    if (n < 1 || n > (int64_t)kmax * kmax) return false;
    if (n == 1) {
        a->n = 1; a->p = 1; a->q = 1;
        return true;
    }
    for (int64_t q = 1; q <= kmax; q++)
        if (n % q == 0 && q * q >= n) {
            const int64_t p = n / q;
            if (p > kmax) return false;
            a->n = (int)n; a->p = (int)p; a->q = (int)q;
            return true;
        }
    return false;
}

static void free_tables(obfft_plan P) {
    for (auto &t : P->tables) {
        cudaFree(t.int8_s1);
        cudaFree(t.int8_s2);
        cudaFree(t.fp8_s1);
        cudaFree(t.fp8_s2);
        cudaFree(t.fp8_s1_l2);
        cudaFree(t.fp8_s2_l2);
        cudaFree(t.tw);
    }
    P->tables.clear();
}

}  // namespace obfft

using namespace obfft;

// ------------------------------------------------------------------ autotune
// Multi-grid plans (and, with OBFFT_AUTOTUNE=1 in the environment, every
// plan; OBFFT_AUTOTUNE=0 turns it off) are tuned at creation:
//  * the Bailey split n = p * q (p, q within the mode's limit) of each distinct
//    axis length, timed on a synthetic batch of lines (stage 1 + stage 2
//    launches, CUDA events, best of 3 after a warm-up);
//  * for the tcgen05 stage kernels, the lines per TMEM lane of every stage
//    with K <= 8 (four or two), timed on the launch geometry of each group of
//    same-shape grids.
// Results remain exact for the chosen split; the oracle reads the split back
// through obfft_plan_get_splits, and obfft_plan_get_tuning reports both.
static bool autotune_enabled(obfft_plan P) {
    const char *env = getenv("OBFFT_AUTOTUNE");
    if (env && env[0] == '0') return false;
    if (env && env[0] == '1') return true;
    return P->grids.size() > 1;
}
// Bytes per complex element of the plan's data: complex128, or complex64 for
// the FP32-precision modes.
static size_t elem_bytes(int mode) {
    return (mode == OBFFT_MODE_FP32 || mode == OBFFT_MODE_FP32_NATIVE) ? 8 : 16;
}
// Largest Bailey factor of a mode: 32 for the tcgen05 stage kernels (one
// 128-column tile holds K <= 32), 64 otherwise.
static int mode_kmax(int mode) {
    return (mode == OBFFT_MODE_FP8 || mode == OBFFT_MODE_FP16 || mode == OBFFT_MODE_FP32) ? 32 : KMAX;
}
static bool mode_known(int mode) {
    return mode == OBFFT_MODE_FP8 || mode == OBFFT_MODE_INT8 || mode == OBFFT_MODE_FP64_NATIVE ||
           mode == OBFFT_MODE_FP16 || mode == OBFFT_MODE_FP32 || mode == OBFFT_MODE_FP32_NATIVE;
}

// One stage launch in the plan's mode.
static cudaError_t launch_stage_mode(obfft_plan P, const AxisTables &t, const StageGeom &g, int stage,
                                     const void *in, void *out, cudaStream_t s) {
    const double2 *i2 = (const double2 *)in;
    double2 *o2 = (double2 *)out;
    switch (P->mode) {
        case OBFFT_MODE_INT8: return launch_stage_int8(t, P->d_consts, g, stage, i2, o2, s);
        case OBFFT_MODE_FP8: return launch_stage_fp8(t, P->d_consts, P->d_pab, P->d_status, g, stage, i2, o2, s);
        case OBFFT_MODE_FP16: return launch_stage_fp16(t, P->d_consts, P->d_pab, P->d_status, g, stage, i2, o2, s);
        case OBFFT_MODE_FP64_NATIVE: return launch_stage_fp64(t, g, stage, i2, o2, s);
        case OBFFT_MODE_FP32:
            return launch_stage_fp32(t, P->d_pab, P->d_status, g, stage, (const float2 *)in, (float2 *)out, s);
        case OBFFT_MODE_FP32_NATIVE: return launch_stage_native32(t, g, stage, (const float2 *)in, (float2 *)out, s);
        default: return cudaErrorInvalidValue;
    }
}

static float time_split(obfft_plan P, int n, int pp, int qq, void *buf, void *tmp, void *outb, int64_t lines) {
    AxisTables t;
    t.n = n; t.p = pp; t.q = qq; t.dir = -1;
    if (build_tables(P, t) != OBFFT_OK) return 1e30f;
    StageGeom g;
    g.L = lines; g.P = lines; g.n = n; g.p = pp; g.q = qq;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    for (int rep = 0; rep < 4; rep++) {
        cudaEventRecord(a, 0);
        for (int st = 1; st <= 2; st++) launch_stage_mode(P, t, g, st, st == 1 ? buf : tmp, st == 1 ? tmp : outb, 0);
        cudaEventRecord(b, 0);
        cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        if (rep > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(t.int8_s1); cudaFree(t.int8_s2); cudaFree(t.fp8_s1); cudaFree(t.fp8_s2); cudaFree(t.tw);
    cudaFree(t.fp8_s1_l2); cudaFree(t.fp8_s2_l2);
    return best;
}

static void autotune_splits(obfft_plan P) {
    if (!autotune_enabled(P)) return;
    const int kmax = mode_kmax(P->mode);
    std::map<int, std::pair<int, int>> best;
    for (auto &gd : P->grids)
        for (int a = 0; a < 3; a++) {
            const int n = (int)gd.n[a];
            if (n == 1 || best.count(n)) continue;
            const int64_t lines = std::max<int64_t>(256, ((int64_t)1 << 21) / n);
            void *buf = nullptr, *tmp = nullptr, *outb = nullptr;
            size_t bytes = (size_t)lines * n * elem_bytes(P->mode);
            if (cudaMalloc(&buf, bytes) != cudaSuccess || cudaMalloc(&tmp, bytes) != cudaSuccess ||
                cudaMalloc(&outb, bytes) != cudaSuccess) {
                cudaFree(buf); cudaFree(tmp); cudaFree(outb);
                return;
            }
            cudaMemset(buf, 0, bytes);
            float tbest = 1e30f;
            std::pair<int, int> pick(gd.ax[a].p, gd.ax[a].q);
            for (int q = 1; q <= n; q++) {
                if (n % q) continue;
                int p = n / q;
                if (p > kmax || q > kmax) continue;
                float tm = time_split(P, n, p, q, buf, tmp, outb, lines);
                if (tm < tbest) {
                    tbest = tm;
                    pick = {p, q};
                }
            }
            cudaFree(buf); cudaFree(tmp); cudaFree(outb);
            best[n] = pick;
        }
    for (auto &gd : P->grids)
        for (int a = 0; a < 3; a++) {
            auto it = best.find((int)gd.n[a]);
            if (it != best.end()) {
                gd.ax[a].p = it->second.first;
                gd.ax[a].q = it->second.second;
            }
        }
}

static void autotune_lpv(obfft_plan P);

static obfft_status finish_create(obfft_plan P, obfft_plan *out) {
    autotune_splits(P);
    // tables for both directions of every distinct axis
    for (auto &gd : P->grids)
        for (int a = 0; a < 3; a++) {
            const AxisPlan &ap = gd.ax[a];
            if (ap.n == 1) continue;
            for (int dir : {-1, 1}) {
                if (get_tables(P, ap.n, ap.p, ap.q, dir)) continue;
                AxisTables t;
                t.n = ap.n; t.p = ap.p; t.q = ap.q; t.dir = dir;
                P->tables.push_back(t);
                obfft_status st = build_tables(P, P->tables.back());
                if (st != OBFFT_OK) {
                    free_tables(P);
                    cudaFree(P->d_consts);
                    delete P;
                    return st;
                }
            }
        }
    size_t maxel = 0, sumel = 0;
    for (auto &gd : P->grids) {
        maxel = std::max(maxel, (size_t)(gd.n[0] * gd.n[1] * gd.n[2]));
        sumel += (size_t)(gd.n[0] * gd.n[1] * gd.n[2]);
    }
    // several grids: those of identical shape and splits form a group that runs
    // as one batched transform (its stage launches cover all members); every
    // group gets its own memory so that the groups' launch chains are independent
    if (P->grids.size() > 1) {
        for (int g = 0; g < (int)P->grids.size(); g++) {
            const GridDesc &a = P->grids[g];
            int j = 0;
            for (; j < (int)P->groups.size(); j++) {
                const GridDesc &b = P->grids[P->groups[j][0]];
                bool same = true;
                for (int x = 0; x < 3; x++)
                    same = same && a.n[x] == b.n[x] && a.ax[x].p == b.ax[x].p && a.ax[x].q == b.ax[x].q;
                if (same) break;
            }
            if (j == (int)P->groups.size()) P->groups.push_back({});
            P->groups[j].push_back(g);
        }
        sumel = 0;
        for (auto &grp : P->groups) {
            const GridDesc &gd = P->grids[grp[0]];
            const size_t gel = (size_t)(gd.n[0] * gd.n[1] * gd.n[2]) * grp.size();
            sumel += grp.size() > 1 ? 3 * gel : gel;
        }
    }
    // single grid: one grid-sized scratch
    const size_t eb = elem_bytes(P->mode);
    P->scratch_bytes = (P->grids.size() == 1 ? maxel * (size_t)P->batch : sumel) * eb;
    cudaError_t e = cudaMalloc(&P->scratch, P->scratch_bytes ? P->scratch_bytes : 16);
    if (e != cudaSuccess) {
        free_tables(P);
        cudaFree(P->d_consts);
        delete P;
        return set_error(OBFFT_ERR_ALLOC, std::string("scratch: ") + cudaGetErrorString(e));
    }
    if (P->grids.size() > 1) {
        char *base = (char *)P->scratch;
        for (auto &grp : P->groups) {
            const GridDesc &gd = P->grids[grp[0]];
            const size_t gbytes = (size_t)(gd.n[0] * gd.n[1] * gd.n[2]) * grp.size() * eb;
            P->group_scratch.push_back(base);
            base += gbytes;
            if (grp.size() > 1) {
                P->group_in.push_back(base);
                base += gbytes;
                P->group_out.push_back(base);
                base += gbytes;
            } else {
                P->group_in.push_back(nullptr);
                P->group_out.push_back(nullptr);
            }
        }
    }
    autotune_lpv(P);
    *out = P;
    return OBFFT_OK;
}

static obfft_status new_plan(int mode, obfft_plan *P) {
    if (!mode_known(mode)) return set_error(OBFFT_ERR_ARG, "unknown mode");
    obfft_plan p = new obfft_plan_s();
    p->mode = mode;
    cudaGetDevice(&p->device);
    ModConsts mc;
    make_mod_consts(&mc);
    cudaError_t e = upload(&mc, sizeof(mc), (void **)&p->d_consts);
    if (e == cudaSuccess) {
        std::vector<uint8_t> pab = mode == OBFFT_MODE_FP32 ? build_phase_a_b32() : build_phase_a_b();
        e = upload(pab.data(), pab.size(), &p->d_pab);
    }
    if (e == cudaSuccess) {
        int zero = 0;
        e = upload(&zero, sizeof(int), (void **)&p->d_status);
    }
    if (e != cudaSuccess) {
        cudaFree(p->d_consts);
        cudaFree(p->d_pab);
        delete p;
        return set_error(OBFFT_ERR_ALLOC, std::string("constants: ") + cudaGetErrorString(e));
    }
    *P = p;
    return OBFFT_OK;
}

extern "C" obfft_status obfft_plan_create(obfft_plan *out, int64_t n0, int64_t n1, int64_t n2,
                                          int64_t batch, int mode) {
    if (!out) return set_error(OBFFT_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n0 < 1 || n1 < 1 || n2 < 1 || batch < 1) return set_error(OBFFT_ERR_ARG, "sizes must be >= 1");
    GridDesc gd;
    gd.n[0] = n0; gd.n[1] = n1; gd.n[2] = n2;
    if (!mode_known(mode)) return set_error(OBFFT_ERR_ARG, "unknown mode");
    const int kmax = mode_kmax(mode);
    for (int a = 0; a < 3; a++)
        if (!choose_split(gd.n[a], &gd.ax[a], kmax))
            return set_error(OBFFT_ERR_UNSUPPORTED_SIZE,
                             "axis " + std::to_string(a) + " of length " + std::to_string(gd.n[a]) +
                                 " does not factor as p*q with p, q <= " + std::to_string(kmax));
    obfft_plan P;
    obfft_status st = new_plan(mode, &P);
    if (st != OBFFT_OK) return st;
    P->batch = batch;
    P->grids.push_back(gd);
    return finish_create(P, out);
}

extern "C" obfft_status obfft_plan_create_many(obfft_plan *out, int count, const int64_t *dims, int mode) {
    if (!out) return set_error(OBFFT_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (count < 1 || !dims) return set_error(OBFFT_ERR_ARG, "count must be >= 1 and dims non-NULL");
    std::vector<GridDesc> grids;
    for (int g = 0; g < count; g++) {
        GridDesc gd;
        for (int a = 0; a < 3; a++) {
            gd.n[a] = dims[g * 3 + a];
            if (gd.n[a] < 1) return set_error(OBFFT_ERR_ARG, "sizes must be >= 1");
            if (!choose_split(gd.n[a], &gd.ax[a], mode_kmax(mode)))
                return set_error(OBFFT_ERR_UNSUPPORTED_SIZE, "axis length " + std::to_string(gd.n[a]) +
                                                                 " does not factor within the mode's p, q limit");
        }
        grids.push_back(gd);
    }
    obfft_plan P;
    obfft_status st = new_plan(mode, &P);
    if (st != OBFFT_OK) return st;
    P->grids = grids;
    return finish_create(P, out);
}

extern "C" obfft_status obfft_destroy(obfft_plan p) {
    if (!p) return OBFFT_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(p->device);
    free_tables(p);
    if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
    if (p->capture_stream) cudaStreamDestroy(p->capture_stream);
    for (cudaStream_t gs : p->group_streams) cudaStreamDestroy(gs);
    for (cudaEvent_t ev : p->group_events) cudaEventDestroy(ev);
    if (p->copy_stream) cudaStreamSynchronize(p->copy_stream), cudaStreamDestroy(p->copy_stream);
    for (cudaEvent_t ev : p->copy_events) cudaEventDestroy(ev);
    cudaFree(p->host_io[0]);
    cudaFree(p->host_io[1]);
    cudaFree(p->scratch);
    cudaFree(p->d_consts);
    cudaFree(p->d_pab);
    cudaFree(p->d_status);
    cudaSetDevice(cur);
    delete p;
    return OBFFT_OK;
}

extern "C" obfft_status obfft_plan_get_splits(obfft_plan p, int grid, int axis, int *p_out, int *q_out) {
    if (!p || !p_out || !q_out || axis < 0 || axis > 2 || grid < 0 || grid >= (int)p->grids.size())
        return set_error(OBFFT_ERR_ARG, "bad plan, grid, axis or output pointer");
    *p_out = p->grids[grid].ax[axis].p;
    *q_out = p->grids[grid].ax[axis].q;
    return OBFFT_OK;
}

// geometry of the pass over `axis` (0, 1, 2) of grid gd: lines, lines per batch item
static StageGeom pass_geom(const GridDesc &gd, int64_t batch, int axis) {
    StageGeom g;
    const AxisPlan &ap = gd.ax[axis];
    int64_t tot = gd.n[0] * gd.n[1] * gd.n[2];
    g.P = tot / gd.n[axis];
    g.L = g.P * batch;
    g.n = ap.n; g.p = ap.p; g.q = ap.q;
    return g;
}

static obfft_status run_stage_geom(obfft_plan P, const AxisPlan &ap, const StageGeom &g, int stage,
                                   const void *in, void *out, int dir, cudaStream_t s) {
    AxisTables *t = get_tables(P, ap.n, ap.p, ap.q, dir);
    if (!t) return set_error(OBFFT_ERR_INTERNAL, "missing tables");
    cudaError_t e = launch_stage_mode(P, *t, g, stage, in, out, s);
    if (e != cudaSuccess) return set_error(OBFFT_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return OBFFT_OK;
}

// Lines per TMEM lane of every stage with K <= 8 (four or two), timed on the
// launch geometry of each group of same-shape grids (the whole grid for
// one-grid plans): three launches per candidate after a warm-up, best of two.
static void autotune_lpv(obfft_plan P) {
    if (!autotune_enabled(P)) return;
    if (P->mode != OBFFT_MODE_FP8 && P->mode != OBFFT_MODE_FP16 && P->mode != OBFFT_MODE_FP32) return;
    std::vector<std::vector<int>> groups = P->groups;
    if (groups.empty()) groups.push_back({0});
    const size_t eb = elem_bytes(P->mode);
    cudaEvent_t ea, eb2;
    if (cudaEventCreate(&ea) != cudaSuccess) return;
    if (cudaEventCreate(&eb2) != cudaSuccess) {
        cudaEventDestroy(ea);
        return;
    }
    for (const auto &grp : groups) {
        const GridDesc &gd = P->grids[grp[0]];
        const int64_t batch = P->groups.empty() ? P->batch : (int64_t)grp.size();
        bool any = false;
        for (int a = 0; a < 3; a++) any = any || (gd.ax[a].n > 1 && (gd.ax[a].p <= 8 || gd.ax[a].q <= 8));
        if (!any) continue;
        const size_t bytes = (size_t)(gd.n[0] * gd.n[1] * gd.n[2] * batch) * eb;
        void *a = nullptr, *b = nullptr;
        if (cudaMalloc(&a, bytes) != cudaSuccess || cudaMalloc(&b, bytes) != cudaSuccess) {
            cudaFree(a);
            break;
        }
        cudaMemset(a, 0, bytes);
        int pick[3][2] = {{0, 0}, {0, 0}, {0, 0}};
        for (int axis = 2; axis >= 0; axis--) {
            const AxisPlan &ap = gd.ax[axis];
            AxisTables *t = ap.n > 1 ? get_tables(P, ap.n, ap.p, ap.q, -1) : nullptr;
            if (!t) continue;
            for (int stage = 1; stage <= 2; stage++) {
                const int K = stage == 1 ? ap.q : ap.p;
                if (K > 8 || !(stage == 1 ? t->fp8_s1_l2 : t->fp8_s2_l2)) continue;
                StageGeom g = pass_geom(gd, batch, axis);
                float best = 1e30f;
                for (int lpv : {4, 2}) {
                    g.lpv = lpv;
                    launch_stage_mode(P, *t, g, stage, a, b, 0);
                    for (int rep = 0; rep < 2; rep++) {
                        cudaEventRecord(ea, 0);
                        for (int i = 0; i < 3; i++) launch_stage_mode(P, *t, g, stage, a, b, 0);
                        cudaEventRecord(eb2, 0);
                        cudaEventSynchronize(eb2);
                        float ms = 0;
                        cudaEventElapsedTime(&ms, ea, eb2);
                        if (ms < best) {
                            best = ms;
                            pick[axis][stage - 1] = lpv;
                        }
                    }
                }
            }
        }
        for (int gi : grp)
            for (int axis = 0; axis < 3; axis++)
                for (int st = 0; st < 2; st++) P->grids[gi].lpv[axis][st] = pick[axis][st];
        cudaFree(a);
        cudaFree(b);
    }
    cudaEventDestroy(ea);
    cudaEventDestroy(eb2);
    cudaGetLastError();  // a failed candidate launch leaves no sticky error behind
}

extern "C" obfft_status obfft_plan_get_tuning(obfft_plan p, int grid, int axis, int *p_out, int *q_out,
                                              int *lpv_stage1, int *lpv_stage2) {
    if (!p || !p_out || !q_out || !lpv_stage1 || !lpv_stage2 || axis < 0 || axis > 2 || grid < 0 ||
        grid >= (int)p->grids.size())
        return set_error(OBFFT_ERR_ARG, "bad plan, grid, axis or output pointer");
    const GridDesc &gd = p->grids[grid];
    const AxisPlan &ap = gd.ax[axis];
    *p_out = ap.p;
    *q_out = ap.q;
    *lpv_stage1 = *lpv_stage2 = 0;
    const bool tc = p->mode == OBFFT_MODE_FP8 || p->mode == OBFFT_MODE_FP16 || p->mode == OBFFT_MODE_FP32;
    if (!tc || ap.n == 1) return OBFFT_OK;
    int64_t batch = p->batch;
    if (!p->groups.empty())
        for (const auto &grp : p->groups)
            for (int gi : grp)
                if (gi == grid) batch = (int64_t)grp.size();
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return set_error(OBFFT_ERR_CUDA, "device query failed");
    const AxisTables *t = get_tables(p, ap.n, ap.p, ap.q, -1);
    for (int stage = 1; stage <= 2; stage++) {
        StageGeom g = pass_geom(gd, batch, axis);
        g.lpv = gd.lpv[axis][stage - 1];
        const bool l2 = t && (stage == 1 ? t->fp8_s1_l2 : t->fp8_s2_l2);
        (stage == 1 ? *lpv_stage1 : *lpv_stage2) = pick_lpv(g, stage, l2, nsm);
    }
    return OBFFT_OK;
}

static obfft_status run_stage(obfft_plan P, const GridDesc &gd, int64_t batch, int axis, int stage,
                              const void *in, void *out, int dir, cudaStream_t s) {
    StageGeom g = pass_geom(gd, batch, axis);
    g.lpv = gd.lpv[axis][stage - 1];
    return run_stage_geom(P, gd.ax[axis], g, stage, in, out, dir, s);
}

// The axis passes first_axis, first_axis - 1, ..., last_axis (the full
// transform: 2 down to 0), each reading lines of its (contiguous) axis and
// writing them rotated, so that the next axis is contiguous.
static obfft_status exec_grid(obfft_plan P, const GridDesc &gd, int64_t batch, const void *in, void *out,
                              int dir, cudaStream_t s, void *scratch_override = nullptr, int first_axis = 2,
                              int last_axis = 0) {
    const void *src = in;
    void *scratch = scratch_override ? scratch_override : P->scratch;
    const int64_t total = gd.n[0] * gd.n[1] * gd.n[2] * batch;
    for (int axis = first_axis; axis >= last_axis; axis--) {
        const AxisPlan &ap = gd.ax[axis];
        if (ap.n == 1) {
            // length-1 axis: identity; the axis rotation [B][A1][A2][1] -> [B][1][A1][A2]
            // leaves the memory order unchanged
            if (src != out) {
                cudaError_t e = cudaMemcpyAsync(out, src, total * elem_bytes(P->mode), cudaMemcpyDeviceToDevice, s);
                if (e != cudaSuccess) return set_error(OBFFT_ERR_CUDA, cudaGetErrorString(e));
            }
        } else {
            obfft_status st = run_stage(P, gd, batch, axis, 1, src, scratch, dir, s);
            if (st != OBFFT_OK) return st;
            st = run_stage(P, gd, batch, axis, 2, scratch, out, dir, s);
            if (st != OBFFT_OK) return st;
        }
        src = out;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(OBFFT_ERR_CUDA, cudaGetErrorString(e));
    return OBFFT_OK;
}

static obfft_status check_ptrs(const void *in, void *out) {
    if (!in || !out) return set_error(OBFFT_ERR_ARG, "in/out is NULL");
    if (in == out) return set_error(OBFFT_ERR_ARG, "in == out: out-of-place only");
    if (((uintptr_t)in | (uintptr_t)out) & 15) return set_error(OBFFT_ERR_ARG, "in/out must be 16-byte aligned");
    return OBFFT_OK;
}

extern "C" obfft_status obfft_exec(obfft_plan p, const void *in, void *out, int dir, void *stream) {
    if (!p) return set_error(OBFFT_ERR_ARG, "plan is NULL");
    if (dir != -1 && dir != 1) return set_error(OBFFT_ERR_ARG, "dir must be -1 or +1");
    obfft_status st = check_ptrs(in, out);
    if (st != OBFFT_OK) return st;
    if (p->grids.size() != 1) return set_error(OBFFT_ERR_ARG, "plan has several grids: use obfft_exec_many");
    // the ranges must not overlap
    size_t bytes = (size_t)(p->grids[0].n[0] * p->grids[0].n[1] * p->grids[0].n[2] * p->batch) * elem_bytes(p->mode);
    uintptr_t a = (uintptr_t)in, b = (uintptr_t)out;
    if (a < b + bytes && b < a + bytes) return set_error(OBFFT_ERR_ARG, "in and out overlap");
    return exec_grid(p, p->grids[0], p->batch, in, out, dir, (cudaStream_t)stream);
}

// Host-to-host execution of a one-grid plan with the copies overlapped: the
// input arrives in chunks of lines of the first pass (axis 2), each chunk is
// transformed as soon as it has landed; the last pass (axis 0) runs in chunks
// of lines and each chunk's output (n0 runs of the chunk's lines, pitch P) is
// copied back while the next chunk computes.  A chunk lies inside one batch
// item, so the stage kernels address its output with the item's full line
// count P from pointers offset to the chunk.
static obfft_status cuda_err(cudaError_t e, const char *what) {
    return e == cudaSuccess ? OBFFT_OK : set_error(OBFFT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

extern "C" obfft_status obfft_exec_host(obfft_plan p, const void *host_in, void *host_out, int dir, void *stream) {
    if (!p) return set_error(OBFFT_ERR_ARG, "plan is NULL");
    if (dir != -1 && dir != 1) return set_error(OBFFT_ERR_ARG, "dir must be -1 or +1");
    if (!host_in || !host_out) return set_error(OBFFT_ERR_ARG, "host_in/host_out is NULL");
    if (host_in == host_out) return set_error(OBFFT_ERR_ARG, "host_in == host_out: out-of-place only");
    if (p->grids.size() != 1) return set_error(OBFFT_ERR_ARG, "plan has several grids: one grid only");
    const GridDesc &gd = p->grids[0];
    const int64_t B = p->batch;
    const int64_t total = gd.n[0] * gd.n[1] * gd.n[2] * B;
    const size_t eb = elem_bytes(p->mode);
    const size_t bytes = (size_t)total * eb;
    {
        uintptr_t a = (uintptr_t)host_in, b = (uintptr_t)host_out;
        if (a < b + bytes && b < a + bytes) return set_error(OBFFT_ERR_ARG, "host_in and host_out overlap");
    }
    cudaStream_t s = (cudaStream_t)stream;
    const char *hin = (const char *)host_in;
    char *hout = (char *)host_out;
    for (int i = 0; i < 2; i++)
        if (!p->host_io[i]) {
            cudaError_t e = cudaMalloc(&p->host_io[i], bytes);
            if (e != cudaSuccess) return set_error(OBFFT_ERR_ALLOC, std::string("host staging: ") + cudaGetErrorString(e));
        }
    char *d0 = (char *)p->host_io[0], *d1 = (char *)p->host_io[1];
    char *scr = (char *)p->scratch;
    // chunks: up to 64 per batch item (smaller chunks shorten the exposed
    // first copy and last copy-back), never fewer than 2^20 elements each
    const int64_t n2 = gd.ax[2].n, n0 = gd.ax[0].n;
    const int64_t P2 = gd.n[0] * gd.n[1], P0 = gd.n[1] * gd.n[2];
    auto nchunks = [](int64_t lines, int64_t len) {
        int64_t c = std::min<int64_t>(64, std::max<int64_t>(1, lines * len / ((int64_t)1 << 20)));
        return (int)std::min<int64_t>(c, lines);
    };
    const int c2 = nchunks(P2, n2), c0 = nchunks(P0, n0);
    const bool simple = gd.ax[2].n == 1 || gd.ax[0].n == 1 || (c2 == 1 && c0 == 1 && B == 1);
    obfft_status st;
    if (simple) {
        st = cuda_err(cudaMemcpyAsync(d0, hin, bytes, cudaMemcpyHostToDevice, s), "input copy");
        if (st != OBFFT_OK) return st;
        st = exec_grid(p, gd, B, d0, d1, dir, s);
        if (st != OBFFT_OK) return st;
        return cuda_err(cudaMemcpyAsync(hout, d1, bytes, cudaMemcpyDeviceToHost, s), "output copy");
    }
    if (!p->copy_stream) {
        st = cuda_err(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking), "copy stream");
        if (st != OBFFT_OK) return st;
    }
    const size_t nev = (size_t)B * (c2 + c0) + 2;
    while (p->copy_events.size() < nev) {
        cudaEvent_t ev;
        st = cuda_err(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
        if (st != OBFFT_OK) return st;
        p->copy_events.push_back(ev);
    }
    size_t ei = 0;
    cudaEvent_t start = p->copy_events[ei++];
    st = cuda_err(cudaEventRecord(start, s), "event record");
    if (st == OBFFT_OK) st = cuda_err(cudaStreamWaitEvent(p->copy_stream, start, 0), "stream wait");
    if (st != OBFFT_OK) return st;
    auto chunk = [](int64_t lines, int c, int i, int64_t *r0, int64_t *lc) {
        const int64_t per = (lines + c - 1) / c;
        *r0 = per * i;
        *lc = std::min(per, lines - *r0);
    };
    // pass 1 (axis 2): input copies on the copy stream, stages on `s` per chunk
    const AxisPlan &a2 = gd.ax[2];
    for (int64_t b = 0; b < B; b++)
        for (int i = 0; i < c2; i++) {
            int64_t r0, lc;
            chunk(P2, c2, i, &r0, &lc);
            if (lc <= 0) continue;
            const int64_t off = (b * P2 + r0) * n2;
            cudaEvent_t ev = p->copy_events[ei++];
            st = cuda_err(cudaMemcpyAsync(d0 + off * eb, hin + off * eb, (size_t)lc * n2 * eb, cudaMemcpyHostToDevice,
                                          p->copy_stream), "input copy");
            if (st == OBFFT_OK) st = cuda_err(cudaEventRecord(ev, p->copy_stream), "event record");
            if (st == OBFFT_OK) st = cuda_err(cudaStreamWaitEvent(s, ev, 0), "stream wait");
            if (st != OBFFT_OK) return st;
            StageGeom g;
            g.L = lc;
            g.P = P2;
            g.n = a2.n; g.p = a2.p; g.q = a2.q;
            st = run_stage_geom(p, a2, g, 1, d0 + off * eb, scr + off * eb, dir, s);
            if (st == OBFFT_OK)
                st = run_stage_geom(p, a2, g, 2, scr + off * eb, d1 + (b * n2 * P2 + r0) * eb, dir, s);
            if (st != OBFFT_OK) return st;
        }
    // pass 2 (axis 1), on the device only
    if (gd.ax[1].n == 1) {
        st = cuda_err(cudaMemcpyAsync(d0, d1, bytes, cudaMemcpyDeviceToDevice, s), "copy");
    } else {
        st = run_stage(p, gd, B, 1, 1, d1, scr, dir, s);
        if (st == OBFFT_OK) st = run_stage(p, gd, B, 1, 2, scr, d0, dir, s);
    }
    if (st != OBFFT_OK) return st;
    // pass 3 (axis 0): stages per chunk on `s`, output copies on the copy stream
    const AxisPlan &a0 = gd.ax[0];
    for (int64_t b = 0; b < B; b++)
        for (int i = 0; i < c0; i++) {
            int64_t r0, lc;
            chunk(P0, c0, i, &r0, &lc);
            if (lc <= 0) continue;
            const int64_t off = (b * P0 + r0) * n0;
            StageGeom g;
            g.L = lc;
            g.P = P0;
            g.n = a0.n; g.p = a0.p; g.q = a0.q;
            const int64_t ooff = b * n0 * P0 + r0;
            st = run_stage_geom(p, a0, g, 1, d0 + off * eb, scr + off * eb, dir, s);
            if (st == OBFFT_OK) st = run_stage_geom(p, a0, g, 2, scr + off * eb, d1 + ooff * eb, dir, s);
            if (st != OBFFT_OK) return st;
            cudaEvent_t ev = p->copy_events[ei++];
            st = cuda_err(cudaEventRecord(ev, s), "event record");
            if (st == OBFFT_OK) st = cuda_err(cudaStreamWaitEvent(p->copy_stream, ev, 0), "stream wait");
            if (st == OBFFT_OK)
                st = cuda_err(cudaMemcpy2DAsync(hout + ooff * eb, (size_t)P0 * eb, d1 + ooff * eb, (size_t)P0 * eb,
                                                (size_t)lc * eb, (size_t)n0, cudaMemcpyDeviceToHost, p->copy_stream),
                              "output copy");
            if (st != OBFFT_OK) return st;
        }
    // the caller's stream completes after the last output copy
    cudaEvent_t done = p->copy_events[ei++];
    st = cuda_err(cudaEventRecord(done, p->copy_stream), "event record");
    if (st == OBFFT_OK) st = cuda_err(cudaStreamWaitEvent(s, done, 0), "stream wait");
    if (st != OBFFT_OK) return st;
    return cuda_err(cudaGetLastError(), "launch");
}

// Multi-grid execution (the uneven batch).  Every grid gets its own slice of
// the plan scratch, so the grids' launch chains are independent; the whole
// sequence is captured once into a CUDA graph for a given set of pointers and
// direction, and later calls with the same arguments replay it with one
// cudaGraphLaunch on the caller's stream.
extern "C" obfft_status obfft_exec_many(obfft_plan p, const void *const *ins, void *const *outs, int dir,
                                        void *stream) {
    if (!p || !ins || !outs) return set_error(OBFFT_ERR_ARG, "NULL argument");
    if (dir != -1 && dir != 1) return set_error(OBFFT_ERR_ARG, "dir must be -1 or +1");
    const size_t G = p->grids.size();
    for (size_t g = 0; g < G; g++) {
        obfft_status st = check_ptrs(ins[g], outs[g]);
        if (st != OBFFT_OK) return st;
    }
    // the groups run as concurrent graph branches: no output may overlap any
    // input or any other output (inputs are only read and may share memory)
    {
        const size_t eb = elem_bytes(p->mode);
        std::vector<size_t> bytes(G);
        for (size_t g = 0; g < G; g++) {
            const GridDesc &gd = p->grids[g];
            bytes[g] = (size_t)(gd.n[0] * gd.n[1] * gd.n[2]) * (G == 1 ? (size_t)p->batch : 1) * eb;
        }
        auto overlap = [](const void *a, size_t na, const void *b, size_t nb) {
            const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
            return x < y + nb && y < x + na;
        };
        for (size_t h = 0; h < G; h++)
            for (size_t g = 0; g < G; g++) {
                if (overlap(outs[h], bytes[h], ins[g], bytes[g]))
                    return set_error(OBFFT_ERR_ARG, "output " + std::to_string(h) + " overlaps input " +
                                                        std::to_string(g));
                if (g != h && overlap(outs[h], bytes[h], outs[g], bytes[g]))
                    return set_error(OBFFT_ERR_ARG, "outputs " + std::to_string(h) + " and " + std::to_string(g) +
                                                        " overlap");
            }
    }
    cudaStream_t s = (cudaStream_t)stream;
    bool same = p->graph_exec && p->graph_dir == dir && p->graph_ins.size() == G;
    for (size_t g = 0; same && g < G; g++) same = p->graph_ins[g] == ins[g] && p->graph_outs[g] == outs[g];
    if (!same) {
        if (p->graph_exec) {
            cudaGraphExecDestroy(p->graph_exec);
            p->graph_exec = nullptr;
        }
        cudaError_t e = cudaSuccess;
        if (!p->capture_stream) e = cudaStreamCreateWithFlags(&p->capture_stream, cudaStreamNonBlocking);
        while (e == cudaSuccess && p->group_streams.size() < p->groups.size()) {
            cudaStream_t gs = nullptr;
            e = cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking);
            if (e == cudaSuccess) p->group_streams.push_back(gs);
        }
        while (e == cudaSuccess && p->group_events.size() < p->groups.size() + 1) {
            cudaEvent_t ev = nullptr;
            e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e == cudaSuccess) p->group_events.push_back(ev);
        }
        if (e != cudaSuccess) return set_error(OBFFT_ERR_CUDA, cudaGetErrorString(e));
        e = cudaStreamBeginCapture(p->capture_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return set_error(OBFFT_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
        obfft_status st = OBFFT_OK;
        const size_t eb = elem_bytes(p->mode);
        if (p->groups.empty())  // a one-grid plan: its own scratch
            st = exec_grid(p, p->grids[0], p->batch, ins[0], outs[0], dir, p->capture_stream, p->scratch);
        else
            st = cuda_err(cudaEventRecord(p->group_events[0], p->capture_stream), "fork");
        size_t forked = 0;  // groups whose stream joined the capture
        for (size_t j = 0; j < p->groups.size() && st == OBFFT_OK; j++) {
            const std::vector<int> &grp = p->groups[j];
            const GridDesc &gd = p->grids[grp[0]];
            cudaStream_t gs = p->group_streams[j];
            st = cuda_err(cudaStreamWaitEvent(gs, p->group_events[0], 0), "fork");
            if (st != OBFFT_OK) break;
            forked = j + 1;
            if (grp.size() == 1) {
                st = exec_grid(p, gd, 1, ins[grp[0]], outs[grp[0]], dir, gs, p->group_scratch[j]);
                continue;
            }
            // gather the members into one batch, transform, scatter the results
            const size_t bytes = (size_t)(gd.n[0] * gd.n[1] * gd.n[2]) * eb;
            for (size_t i = 0; i < grp.size() && st == OBFFT_OK; i++)
                st = cuda_err(cudaMemcpyAsync((char *)p->group_in[j] + i * bytes, ins[grp[i]], bytes,
                                              cudaMemcpyDeviceToDevice, gs), "gather");
            if (st == OBFFT_OK)
                st = exec_grid(p, gd, (int64_t)grp.size(), p->group_in[j], p->group_out[j], dir, gs,
                               p->group_scratch[j]);
            for (size_t i = 0; i < grp.size() && st == OBFFT_OK; i++)
                st = cuda_err(cudaMemcpyAsync(outs[grp[i]], (char *)p->group_out[j] + i * bytes, bytes,
                                              cudaMemcpyDeviceToDevice, gs), "scatter");
        }
        // join every forked branch back into the capture stream (also after an
        // error, so that the capture can end cleanly)
        for (size_t j = 0; j < forked; j++) {
            cudaError_t ej = cudaEventRecord(p->group_events[1 + j], p->group_streams[j]);
            if (ej == cudaSuccess) ej = cudaStreamWaitEvent(p->capture_stream, p->group_events[1 + j], 0);
            if (st == OBFFT_OK && ej != cudaSuccess) st = cuda_err(ej, "join");
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(p->capture_stream, &graph);
        if (st != OBFFT_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e2 != cudaSuccess) return set_error(OBFFT_ERR_CUDA, std::string("capture end: ") + cudaGetErrorString(e2));
        e2 = cudaGraphInstantiate(&p->graph_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e2 != cudaSuccess) {
            p->graph_exec = nullptr;
            return set_error(OBFFT_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e2));
        }
        p->graph_ins.assign(ins, ins + G);
        p->graph_outs.assign(outs, outs + G);
        p->graph_dir = dir;
    }
    cudaError_t e = cudaGraphLaunch(p->graph_exec, s);
    if (e != cudaSuccess) return set_error(OBFFT_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    return OBFFT_OK;
}

extern "C" obfft_status obfft_exec_axes(obfft_plan p, int first_axis, int last_axis, const void *in, void *out,
                                        int dir, void *stream) {
    if (!p) return set_error(OBFFT_ERR_ARG, "plan is NULL");
    if (dir != -1 && dir != 1) return set_error(OBFFT_ERR_ARG, "dir must be -1 or +1");
    if (first_axis < 0 || first_axis > 2 || last_axis < 0 || last_axis > first_axis)
        return set_error(OBFFT_ERR_ARG, "need 2 >= first_axis >= last_axis >= 0");
    obfft_status st = check_ptrs(in, out);
    if (st != OBFFT_OK) return st;
    if (p->grids.size() != 1) return set_error(OBFFT_ERR_ARG, "plan has several grids");
    const size_t bytes =
        (size_t)(p->grids[0].n[0] * p->grids[0].n[1] * p->grids[0].n[2] * p->batch) * elem_bytes(p->mode);
    const uintptr_t a = (uintptr_t)in, b = (uintptr_t)out;
    if (a < b + bytes && b < a + bytes) return set_error(OBFFT_ERR_ARG, "in and out overlap");
    return exec_grid(p, p->grids[0], p->batch, in, out, dir, (cudaStream_t)stream, nullptr, first_axis, last_axis);
}

extern "C" obfft_status obfft_transpose_blocks(const void *src, void *dst, int64_t nblocks, int64_t rows,
                                               int64_t row_bytes, void *stream) {
    if (!src || !dst || src == dst) return set_error(OBFFT_ERR_ARG, "src/dst NULL or equal");
    if (nblocks < 1 || rows < 0 || row_bytes < 1) return set_error(OBFFT_ERR_ARG, "bad block geometry");
    const size_t total = (size_t)nblocks * (size_t)rows * (size_t)row_bytes;
    const uintptr_t a = (uintptr_t)src, b = (uintptr_t)dst;
    if (a < b + total && b < a + total) return set_error(OBFFT_ERR_ARG, "src and dst overlap");
    cudaStream_t s = (cudaStream_t)stream;
    // block k of the source (rows x row_bytes, contiguous) becomes column
    // block k of the destination rows (pitch nblocks x row_bytes)
    for (int64_t k = 0; k < nblocks && rows > 0; k++) {
        cudaError_t e = cudaMemcpy2DAsync((char *)dst + k * row_bytes, (size_t)(nblocks * row_bytes),
                                          (const char *)src + k * rows * row_bytes, (size_t)row_bytes,
                                          (size_t)row_bytes, (size_t)rows, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return set_error(OBFFT_ERR_CUDA, std::string("block copy: ") + cudaGetErrorString(e));
    }
    return OBFFT_OK;
}

// Byte offsets of the sections of an obfft_exec_debug dump (16-byte aligned).
static void debug_layout(int64_t ncols, int K, int Kout, int nmod, int nacc, int64_t off[8]) {
    auto al = [](int64_t v) { return (v + 15) & ~(int64_t)15; };
    int64_t o = 0;
    off[0] = o; o = al(o + ncols * 4);                               // e
    off[1] = o; o = al(o + ncols * K * 2 * 8);                       // xt
    off[2] = o; o = al(o + ncols * Kout * nmod * 3 * 2);             // def
    off[3] = o; o = al(o + ncols * Kout * 2 * nmod * 2);             // res
    off[4] = o; o = al(o + ncols * Kout * 2 * nacc * 4);             // acc
    off[5] = o; o = al(o + ncols * Kout * 2 * 8);                    // zhat
    off[6] = o; o = al(o + ncols * Kout * 2 * 4 * 4);                // R
    off[7] = o;
}

static bool mode_has_integers(int mode) {
    return mode == OBFFT_MODE_FP8 || mode == OBFFT_MODE_INT8 || mode == OBFFT_MODE_FP16 || mode == OBFFT_MODE_FP32;
}

extern "C" obfft_status obfft_debug_layout(int mode, int K, int Kout, int64_t ncols, int64_t *offsets) {
    if (!offsets || !mode_has_integers(mode) || K < 1 || Kout < 1 || ncols < 0 || K > KMAX || Kout > KMAX)
        return set_error(OBFFT_ERR_ARG, "bad mode (native modes have no integer stages), size or NULL offsets");
    const int nm = mode == OBFFT_MODE_FP32 ? NMOD32 : NMOD;
    const int na = mode == OBFFT_MODE_FP32 ? S_RAW32 + S_FRAC32 : S_RAW + S_FRAC;
    debug_layout(ncols, K, Kout, nm, na, offsets);
    return OBFFT_OK;
}

extern "C" obfft_status obfft_exec_debug(obfft_plan p, int axis, int stage, const void *in, void *out, int dir,
                                         int64_t col0, int64_t ncols, void *dump, void *stream) {
    if (!p || axis < 0 || axis > 2 || (stage != 1 && stage != 2) || !dump) return set_error(OBFFT_ERR_ARG, "bad argument");
    if (dir != -1 && dir != 1) return set_error(OBFFT_ERR_ARG, "dir must be -1 or +1");
    if (!mode_has_integers(p->mode)) return set_error(OBFFT_ERR_ARG, "native modes have no integer stages to dump");
    if (p->grids.size() != 1) return set_error(OBFFT_ERR_ARG, "plan has several grids");
    obfft_status st = check_ptrs(in, out);
    if (st != OBFFT_OK) return st;
    const GridDesc &gd = p->grids[0];
    const AxisPlan &ap = gd.ax[axis];
    if (ap.n == 1) return set_error(OBFFT_ERR_ARG, "axis of length 1 has no stages");
    const StageGeom g = pass_geom(gd, p->batch, axis);
    const int K = stage == 1 ? ap.q : ap.p;
    const int64_t total_cols = stage == 1 ? g.L * ap.p : g.L * ap.q;
    if (col0 < 0 || ncols < 1 || col0 + ncols > total_cols)
        return set_error(OBFFT_ERR_ARG, "dumped columns outside [0, " + std::to_string(total_cols) + ")");
    AxisTables *t = get_tables(p, ap.n, ap.p, ap.q, dir);
    if (!t) return set_error(OBFFT_ERR_INTERNAL, "missing tables");
    const int nm = p->mode == OBFFT_MODE_FP32 ? NMOD32 : NMOD;
    const int na = p->mode == OBFFT_MODE_FP32 ? S_RAW32 + S_FRAC32 : S_RAW + S_FRAC;
    int64_t off[8];
    debug_layout(ncols, K, K, nm, na, off);
    char *b = (char *)dump;
    DebugDump d;
    d.e = (int32_t *)(b + off[0]);
    d.xt = (int64_t *)(b + off[1]);
    d.def = (uint16_t *)(b + off[2]);
    d.res = (uint16_t *)(b + off[3]);
    d.acc = (uint32_t *)(b + off[4]);
    d.zhat = (int64_t *)(b + off[5]);
    d.R = (uint32_t *)(b + off[6]);
    d.col0 = col0;
    d.ncols = ncols;
    d.K = K;
    d.Kout = K;
    d.nmod = nm;
    d.nacc = na;
    d.stage = stage;
    d.L = g.L;  // the launchers set Lpad (their own tile padding)
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(dump, 0, (size_t)off[7], s);
    if (e == cudaSuccess) {
        const double2 *i2 = (const double2 *)in;
        double2 *o2 = (double2 *)out;
        switch (p->mode) {
            case OBFFT_MODE_INT8: e = launch_stage_int8(*t, p->d_consts, g, stage, i2, o2, s, &d); break;
            case OBFFT_MODE_FP8: e = launch_stage_fp8(*t, p->d_consts, p->d_pab, p->d_status, g, stage, i2, o2, s, &d); break;
            case OBFFT_MODE_FP16: e = launch_stage_fp16(*t, p->d_consts, p->d_pab, p->d_status, g, stage, i2, o2, s, &d); break;
            case OBFFT_MODE_FP32:
                e = launch_stage_fp32(*t, p->d_pab, p->d_status, g, stage, (const float2 *)in, (float2 *)out, s, &d);
                break;
            default: e = cudaErrorInvalidValue;
        }
    }
    if (e != cudaSuccess) return set_error(OBFFT_ERR_CUDA, std::string("debug launch: ") + cudaGetErrorString(e));
    return OBFFT_OK;
}

extern "C" obfft_status obfft_exec_stage(obfft_plan p, int axis, int stage, const void *in, void *out, int dir,
                                         void *stream) {
    if (!p || axis < 0 || axis > 2 || (stage != 1 && stage != 2)) return set_error(OBFFT_ERR_ARG, "bad argument");
    if (dir != -1 && dir != 1) return set_error(OBFFT_ERR_ARG, "dir must be -1 or +1");
    obfft_status st = check_ptrs(in, out);
    if (st != OBFFT_OK) return st;
    if (p->grids[0].ax[axis].n == 1) return set_error(OBFFT_ERR_ARG, "axis of length 1 has no stages");
    st = run_stage(p, p->grids[0], p->batch, axis, stage, in, out, dir, (cudaStream_t)stream);
    return st;
}

extern "C" obfft_status obfft_plan_status(obfft_plan p, void *stream) {
    if (!p) return set_error(OBFFT_ERR_ARG, "plan is NULL");
    int v = 0, zero = 0;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(&v, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_error(OBFFT_ERR_CUDA, std::string("status read: ") + cudaGetErrorString(e));
    if (v == OBFFT_OK) return OBFFT_OK;
    cudaMemcpyAsync(p->d_status, &zero, sizeof(int), cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
    return set_error((obfft_status)v, "a device-side bounded wait gave up (the transform's output is invalid)");
}

extern "C" obfft_status obfft_selftest_bounded_wait(obfft_plan p, void *stream) {
    if (!p) return set_error(OBFFT_ERR_ARG, "plan is NULL");
    cudaError_t e = launch_bounded_wait_selftest(p->d_status, (cudaStream_t)stream);
    if (e != cudaSuccess) return set_error(OBFFT_ERR_CUDA, cudaGetErrorString(e));
    return OBFFT_OK;
}

extern "C" obfft_status obfft_host_twiddle(int64_t m, int64_t N, int dir, int64_t *re, int64_t *im) {
    if (N < 1 || !re || !im) return set_error(OBFFT_ERR_ARG, "bad argument");
    quantised_twiddle(m, N, dir, re, im);
    return OBFFT_OK;
}

extern "C" obfft_status obfft_host_crt_constants(uint32_t *moduli, uint8_t *u_slices, uint8_t *w_slices,
                                                 uint32_t *M4) {
    if (!moduli || !u_slices || !w_slices || !M4) return set_error(OBFFT_ERR_ARG, "NULL output");
    ModConsts mc;
    make_mod_consts(&mc);
    for (int k = 0; k < NMOD; k++) {
        moduli[k] = mc.m[k];
        for (int s = 0; s < S_RAW; s++) u_slices[k * S_RAW + s] = mc.us[k][s];
        for (int t = 0; t < S_FRAC; t++) w_slices[k * S_FRAC + t] = mc.ws[k][t];
    }
    for (int w = 0; w < 4; w++) M4[w] = mc.M32[w];
    return OBFFT_OK;
}

extern "C" obfft_status obfft_host_twiddle32(int64_t m, int64_t N, int dir, int64_t *re, int64_t *im) {
    if (N < 1 || !re || !im) return set_error(OBFFT_ERR_ARG, "bad argument");
    quantised_twiddle_scaled(m, N, dir, 23, re, im);
    return OBFFT_OK;
}

extern "C" obfft_status obfft_host_crt_constants32(uint32_t *moduli, uint8_t *u_slices, uint8_t *w_slices,
                                                   uint64_t *M) {
    if (!moduli || !u_slices || !w_slices || !M) return set_error(OBFFT_ERR_ARG, "NULL output");
    uint8_t us[NMOD32][S_RAW32], ws[NMOD32][S_FRAC32];
    make_crt_consts32(us, ws, M);
    for (int k = 0; k < NMOD32; k++) {
        moduli[k] = (uint32_t)kModuli32[k];
        for (int s = 0; s < S_RAW32; s++) u_slices[k * S_RAW32 + s] = us[k][s];
        for (int t = 0; t < S_FRAC32; t++) w_slices[k * S_FRAC32 + t] = ws[k][t];
    }
    return OBFFT_OK;
}

extern "C" obfft_status obfft_ablation_phase_b(int variant, int64_t n_unique, int64_t n_total, int reps,
                                              const void *acc, const void *et, void *out, void *checksum,
                                              void *stream) {
    if (variant != 0 && variant != 32 && variant != 16 && variant != 8)
        return set_error(OBFFT_ERR_ARG, "variant must be 0, 32, 16 or 8");
    if (n_unique < 1 || n_total < 0 || reps < 1 || !acc || !et || !checksum)
        return set_error(OBFFT_ERR_ARG, "bad argument");
    cudaError_t e = launch_phase_b_ablation(variant, n_unique, n_total, reps, (const uint32_t *)acc, (const int *)et,
                                            (double *)out, (unsigned long long *)checksum, (cudaStream_t)stream);
    return e == cudaSuccess ? OBFFT_OK : set_error(OBFFT_ERR_CUDA, cudaGetErrorString(e));
}

extern "C" obfft_status obfft_ablation_residues(int variant, int64_t n_unique, int64_t n_total, int reps,
                                               const void *xt, void *res, void *checksum, void *stream) {
    if (variant < 0 || variant > 3) return set_error(OBFFT_ERR_ARG, "variant must be 0, 1, 2 or 3");
    if (n_unique < 1 || n_total < 0 || reps < 1 || !xt || !checksum) return set_error(OBFFT_ERR_ARG, "bad argument");
    cudaError_t e = launch_residue_ablation(variant, n_unique, n_total, reps, (const int64_t *)xt, (uint16_t *)res,
                                            (unsigned long long *)checksum, (cudaStream_t)stream);
    return e == cudaSuccess ? OBFFT_OK : set_error(OBFFT_ERR_CUDA, cudaGetErrorString(e));
}

extern "C" const char *obfft_last_error(void) { return g_last_error.c_str(); }

extern "C" const char *obfft_version(void) { return "obfft 0.1 (sm_103a)"; }
