/*
 * ozaki_ref.c -- plain, slow CPU reference of the Ozaki-Bailey FFT.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product (the GPU library and its
 * Python binding) may include, link or call this file; only tests/, the
 * smoke check and the benchmark's CPU-baseline leg use it.  It shares no
 * code, header or table with the CUDA path.
 *
 * What it computes, per the paper:
 *   ob_ref_stage   one Ozaki-II complex GEMM per column (Algorithm 1, one of
 *                  its two halves): deconstruction (Sec. "Deconstruction
 *                  count"), per-modulus Karatsuba residue products
 *                  (Background, complex 3-real-GEMM split), residue-domain
 *                  combine + canonicalisation, Phase A slice sums P_s and
 *                  fractional partials Q_t (Eq. slicing, Eq. phaseAcost),
 *                  Kulisch Phase B with biased deposits in six radix-2^28
 *                  carry-save words, the two-sided modulo-M lift and the
 *                  correctly rounded pack (Algorithm 2).  Every output is also
 *                  computed as the plain exact integer product sum_j F~ x~
 *                  (the definition the CRT must reach) and the two are
 *                  compared; the count of mismatches is returned.
 *   ob_ref_pack    RNE of a signed 128-bit integer times 2^e, gradual underflow.
 *   ob_ref_stage32 / ob_ref_pack32   the same stage for the FP32-precision
 *                  variant (Sec. "Ozaki-II for FP32"): complex64 columns,
 *                  24-bit significands, r = 6 moduli, S = 8, f = 24.
 *   ob_ref_dft_dd_axis   direct O(N^2) DFT along the last axis in
 *                  double-double arithmetic (the high-precision reference).
 *   ob_ref_dft_dd_point  one output of the 3-D DFT in double-double.
 *   ob_ref_fft_lines     plain FP64 mixed-radix FFT along the last axis (the
 *                  FP64 reference transform and the timed CPU FFT).
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (contraction must be
 * off: the double-double kernels rely on separately rounded products/sums).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;
typedef unsigned __int128 u128;

#define NMOD 12
#define S_RAW 15
#define S_FRAC 6

/* Constants handed in by the Python side (computed there from definitions). */
typedef struct {
    int64_t m[NMOD];              /* moduli */
    uint8_t us[NMOD][S_RAW];      /* byte slices of the idempotents u_k */
    uint8_t ws[NMOD][S_FRAC];     /* byte slices of the lift weights w_k */
    uint32_t M[4];                /* M, little-endian 32-bit limbs */
} ob_consts;

/* Optional per-output dump of every integer stage (small tests only). */
typedef struct {
    int32_t *col_exp;     /* [ncols]                    e of each column          */
    int64_t *xt;          /* [ncols][K][2]              x~ = rint(x 2^(52-e))     */
    uint16_t *def;        /* [ncols][Kout][NMOD][3]     D, E, F mod m_k           */
    uint16_t *v;          /* [ncols][Kout][2][NMOD]     canonical R_k, I_k        */
    int64_t *P;           /* [ncols][Kout][2][S_RAW]    Phase A slice sums        */
    int64_t *Q;           /* [ncols][Kout][2][S_FRAC]   Phase A lift partials     */
    int64_t *zhat;        /* [ncols][Kout][2]           rounded lift quotient     */
    int64_t *Rlimbs;      /* [ncols][Kout][2][2]        lifted R (lo, hi 64 bits) */
} ob_dump;

/* ------------------------------------------------------------------------ */
/* A small signed 256-bit two's-complement integer (4 x 64-bit limbs).       */
/* ------------------------------------------------------------------------ */
typedef struct { uint64_t w[4]; } i256;

static i256 i256_add(i256 a, i256 b) {
    i256 r;
    u128 carry = 0;
    for (int i = 0; i < 4; i++) {
        u128 s = (u128)a.w[i] + b.w[i] + carry;
        r.w[i] = (uint64_t)s;
        carry = s >> 64;
    }
    return r;
}

static i256 i256_neg(i256 a) {
    i256 r;
    for (int i = 0; i < 4; i++) r.w[i] = ~a.w[i];
    i256 one = {{1, 0, 0, 0}};
    return i256_add(r, one);
}

static i256 i256_sub(i256 a, i256 b) { return i256_add(a, i256_neg(b)); }

static int i256_is_neg(i256 a) { return (int)(a.w[3] >> 63); }

/* signed compare: returns <0, 0, >0 */
static int i256_cmp(i256 a, i256 b) {
    i256 d = i256_sub(a, b);
    if (i256_is_neg(d)) return -1;
    if ((d.w[0] | d.w[1] | d.w[2] | d.w[3]) == 0) return 0;
    return 1;
}

/* a * small for 0 <= small < 2^63 */
static i256 i256_mul_small(i256 a, uint64_t small) {
    i256 r;
    u128 carry = 0;
    for (int i = 0; i < 4; i++) {
        u128 p = (u128)a.w[i] * small + carry;
        r.w[i] = (uint64_t)p;
        carry = p >> 64;
    }
    return r;
}

static i256 i256_shl(i256 a, int n) { /* 0 <= n < 256 */
    i256 r = {{0, 0, 0, 0}};
    int limbs = n / 64, bits = n % 64;
    for (int i = 3; i >= 0; i--) {
        int src = i - limbs;
        if (src < 0) continue;
        uint64_t v = a.w[src] << bits;
        if (bits && src - 1 >= 0) v |= a.w[src - 1] >> (64 - bits);
        r.w[i] = v;
    }
    return r;
}

static i256 i256_from_u32_limbs(const uint32_t *l, int n) {
    i256 r = {{0, 0, 0, 0}};
    for (int i = 0; i < n; i++) {
        i256 t = {{(uint64_t)l[i], 0, 0, 0}};
        r = i256_add(r, i256_shl(t, 32 * i));
    }
    return r;
}

/* value must fit in i128 */
static i128 i256_to_i128(i256 a) {
    u128 v = ((u128)a.w[1] << 64) | a.w[0];
    return (i128)v;
}

/* ------------------------------------------------------------------------ */
/* Correctly rounded pack: RNE(Rv * 2^e) with gradual underflow.             */
/* (Algorithm 2, last step: the single rounding of the pipeline.)            */
/* ------------------------------------------------------------------------ */
static int bitlen_u128(u128 a) {
    int n = 0;
    while (a) { a >>= 1; n++; }
    return n;
}

double ob_ref_pack(int64_t lo, int64_t hi, int e) {
    i128 Rv = (i128)(((u128)(uint64_t)hi << 64) | (uint64_t)lo);
    if (Rv == 0) return 0.0;
    int neg = Rv < 0;
    u128 a = neg ? (u128)(-Rv) : (u128)Rv;
    int L = bitlen_u128(a);
    /* drop d low bits: enough to keep 53 significant bits, and no bit below
       2^-1074 (the subnormal quantum). */
    int d = L - 53;
    int d_sub = -1074 - e;
    if (d_sub > d) d = d_sub;
    u128 q;
    if (d <= 0) {
        q = a; /* exact: at most 53 significant bits, above the subnormal quantum */
        d = 0;
    } else if (d > L) {
        q = 0; /* a < 2^(d-1): below half a quantum */
    } else { /* 1 <= d <= L <= 117 */
        q = a >> d;
        u128 rem = a & ((((u128)1) << d) - 1);
        u128 half = ((u128)1) << (d - 1);
        if (rem > half || (rem == half && (q & 1))) q += 1;
    }
    /* q <= 2^53: the conversion and the power-of-two scaling are exact
       (or overflow to infinity, which is the correctly rounded result). */
    double r = ldexp((double)(uint64_t)q, e + d);
    return neg ? -r : r;
}

/* ------------------------------------------------------------------------ */
/* Helpers                                                                  */
/* ------------------------------------------------------------------------ */
static int64_t modc(i128 x, int64_t m) { /* canonical residue in [0, m) */
    i128 r = x % m;
    if (r < 0) r += m;
    return (int64_t)r;
}

/* Kulisch Phase B for one scalar output (Algorithm 2).  P[s] signed slice
 * sums, Q[t] lift partials.  Returns the centered representative R. */
static i128 kulisch_lift(const int64_t P[S_RAW], const int64_t Q[S_FRAC],
                         const ob_consts *c, int64_t *zhat_out) {
    /* six radix-2^28 carry-save words, 4 guard bits each */
    uint32_t W[6] = {0, 0, 0, 0, 0, 0};
    const uint64_t MASK28 = (1u << 28) - 1;
    for (int s = 0; s < S_RAW; s++) {
        /* biased deposit (P_s + 2^23) << 8s: non-negative for P_s >= -2^23 */
        uint64_t d = (uint64_t)(P[s] + (1 << 23));
        int pos = 8 * s;
        int w = pos / 28, off = pos % 28;
        u128 t = (u128)d << off;
        W[w] += (uint32_t)(t & MASK28);
        W[w + 1] += (uint32_t)((t >> 28) & MASK28);
        if (w + 2 < 6) W[w + 2] += (uint32_t)(t >> 56);
    }
    /* one guard-bit carry sweep */
    for (int w = 0; w < 5; w++) {
        W[w + 1] += W[w] >> 28;
        W[w] &= (uint32_t)MASK28;
    }
    i256 E = {{0, 0, 0, 0}};
    for (int w = 0; w < 6; w++) {
        i256 t = {{(uint64_t)W[w], 0, 0, 0}};
        E = i256_add(E, i256_shl(t, 28 * w));
    }
    /* remove the compile-time bias B_tot = sum_s 2^23 256^s */
    for (int s = 0; s < S_RAW; s++) {
        i256 b = {{1ULL << 23, 0, 0, 0}};
        E = i256_sub(E, i256_shl(b, 8 * s));
    }
    /* fractional-CRT lift: zhat = round(2^-48 z_acc), half up */
    /* (signed: residues may also be signed, |v_k| < 2 m_k; floor division) */
    i128 zacc = 0;
    for (int t = 0; t < S_FRAC; t++) zacc += (i128)Q[t] * ((i128)1 << (8 * t));
    i128 zsum = zacc + ((i128)1 << 47);
    i128 zq = zsum / ((i128)1 << 48);
    if (zq * ((i128)1 << 48) > zsum) zq -= 1;
    int64_t zhat = (int64_t)zq;
    if (zhat_out) *zhat_out = zhat;
    i256 Mv = i256_from_u32_limbs(c->M, 4);
    i256 Rv = zhat >= 0 ? i256_sub(E, i256_mul_small(Mv, (uint64_t)zhat))
                        : i256_add(E, i256_mul_small(Mv, (uint64_t)(-zhat)));
    /* two-sided centered correction */
    i256 half = i256_from_u32_limbs(c->M, 4);
    /* M is even: M/2 exact */
    {
        uint64_t carry = 0;
        for (int i = 3; i >= 0; i--) {
            uint64_t v = half.w[i];
            half.w[i] = (v >> 1) | (carry << 63);
            carry = v & 1;
        }
    }
    if (i256_cmp(Rv, half) >= 0) Rv = i256_sub(Rv, Mv);
    if (i256_cmp(Rv, i256_neg(half)) < 0) Rv = i256_add(Rv, Mv);
    return i256_to_i128(Rv);
}

/* ------------------------------------------------------------------------ */
/* One Ozaki-II complex "GEMM" stage over independent columns.               */
/*   y[c][k] = RNE( 2^(e_c - 104) * sum_j F~[g(c)][k][j] * x~[c][j] )        */
/* ------------------------------------------------------------------------ */
int64_t ob_ref_stage(int64_t ncols, int K, int Kout,
                     const double *x,        /* [ncols][K][2] */
                     const int64_t *Ftab,    /* [ngroups][Kout][K][2] */
                     const int32_t *group,   /* [ncols] or NULL */
                     const ob_consts *c,
                     int use_crt,
                     double *y,              /* [ncols][Kout][2] */
                     ob_dump *dump) {
    int64_t mismatches = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : mismatches)
    for (int64_t col = 0; col < ncols; col++) {
        const double *xc = x + col * (int64_t)K * 2;
        int g = group ? group[col] : 0;
        const int64_t *F = Ftab + (int64_t)g * Kout * K * 2;
        /* ---- deconstruction: one power of two per column ---- */
        double amax = 0.0;
        for (int j = 0; j < 2 * K; j++) {
            double a = fabs(xc[j]);
            if (a > amax) amax = a;
        }
        int e = amax > 0.0 ? ilogb(amax) : 0;
        int64_t xt[2 * 64];
        for (int j = 0; j < 2 * K; j++) xt[j] = (int64_t)rint(ldexp(xc[j], 52 - e));
        if (dump && dump->col_exp) dump->col_exp[col] = e;
        if (dump && dump->xt) memcpy(dump->xt + col * (int64_t)K * 2, xt, sizeof(int64_t) * 2 * K);

        for (int k = 0; k < Kout; k++) {
            const int64_t *Fk = F + (int64_t)k * K * 2;
            /* plain definition: the exact complex integer product */
            i128 Cre = 0, Cim = 0;
            for (int j = 0; j < K; j++) {
                i128 fr = Fk[2 * j], fi = Fk[2 * j + 1];
                i128 xr = xt[2 * j], xi = xt[2 * j + 1];
                Cre += fr * xr - fi * xi;
                Cim += fr * xi + fi * xr;
            }
            i128 Rout[2] = {Cre, Cim};
            if (use_crt) {
                /* ---- per-modulus Karatsuba residue products ---- */
                int64_t v[2][NMOD];
                for (int i = 0; i < NMOD; i++) {
                    int64_t m = c->m[i];
                    int64_t D = 0, Ev = 0, Fv = 0;
                    for (int j = 0; j < K; j++) {
                        int64_t ar = modc(Fk[2 * j], m), ai = modc(Fk[2 * j + 1], m);
                        int64_t as = modc((i128)Fk[2 * j] + Fk[2 * j + 1], m);
                        int64_t br = modc(xt[2 * j], m), bi = modc(xt[2 * j + 1], m);
                        int64_t bs = modc((i128)xt[2 * j] + xt[2 * j + 1], m);
                        D += ar * br;
                        Ev += ai * bi;
                        Fv += as * bs;
                    }
                    D %= m;
                    Ev %= m;
                    Fv %= m;
                    if (dump && dump->def) {
                        uint16_t *p = dump->def + ((col * Kout + k) * NMOD + i) * 3;
                        p[0] = (uint16_t)D; p[1] = (uint16_t)Ev; p[2] = (uint16_t)Fv;
                    }
                    /* residue-domain combine, canonicalised once */
                    v[0][i] = modc((i128)D - Ev, m);
                    v[1][i] = modc((i128)Fv - D - Ev, m);
                }
                for (int part = 0; part < 2; part++) {
                    /* ---- Phase A: slice sums and lift partials ---- */
                    int64_t P[S_RAW], Q[S_FRAC];
                    for (int s = 0; s < S_RAW; s++) {
                        P[s] = 0;
                        for (int i = 0; i < NMOD; i++) P[s] += v[part][i] * c->us[i][s];
                    }
                    for (int t = 0; t < S_FRAC; t++) {
                        Q[t] = 0;
                        for (int i = 0; i < NMOD; i++) Q[t] += v[part][i] * c->ws[i][t];
                    }
                    int64_t zhat;
                    i128 Rv = kulisch_lift(P, Q, c, &zhat);
                    int64_t base = (col * Kout + k) * 2 + part;
                    if (dump) {
                        if (dump->v)
                            for (int i = 0; i < NMOD; i++) dump->v[base * NMOD + i] = (uint16_t)v[part][i];
                        if (dump->P) memcpy(dump->P + base * S_RAW, P, sizeof P);
                        if (dump->Q) memcpy(dump->Q + base * S_FRAC, Q, sizeof Q);
                        if (dump->zhat) dump->zhat[base] = zhat;
                        if (dump->Rlimbs) {
                            dump->Rlimbs[base * 2] = (int64_t)(uint64_t)Rv;
                            dump->Rlimbs[base * 2 + 1] = (int64_t)(uint64_t)((u128)Rv >> 64);
                        }
                    }
                    if (Rv != Rout[part]) mismatches++;
                    Rout[part] = Rv;
                }
            }
            double *yk = y + (col * Kout + k) * 2;
            for (int part = 0; part < 2; part++) {
                i128 Rv = Rout[part];
                yk[part] = ob_ref_pack((int64_t)(uint64_t)Rv, (int64_t)(uint64_t)((u128)Rv >> 64),
                                       e - 104);
            }
        }
    }
    return mismatches;
}

/* ------------------------------------------------------------------------ */
/* FP32-precision variant (Sec. "Ozaki-II for FP32"): complex64 columns,     */
/* 24-bit significands (constants RNE(2^23 omega), data x~ = x 2^(23-e)),    */
/* r = 6 moduli, S = 8 byte slices of u_k, f = 24 (three slices of w_k).     */
/* The lifted value fits the paper's 77-bit accumulator; here a 128-bit one. */
/* ------------------------------------------------------------------------ */
#define NMOD32 6
#define S_RAW32 8
#define S_FRAC32 3

typedef struct {
    int64_t m[NMOD32];
    uint8_t us[NMOD32][S_RAW32];
    uint8_t ws[NMOD32][S_FRAC32];
    uint64_t M;
} ob_consts32;

typedef struct {
    uint16_t *v;       /* [ncols][Kout][2][NMOD32]   canonical residues  */
    int64_t *P;        /* [ncols][Kout][2][S_RAW32]  Phase A slice sums  */
    int64_t *Q;        /* [ncols][Kout][2][S_FRAC32] lift partials        */
    int64_t *zhat;     /* [ncols][Kout][2]                                */
    int64_t *R;        /* [ncols][Kout][2]           lifted R (|R| < 2^63) */
    int32_t *col_exp;  /* [ncols]                    column exponent e       */
    int64_t *xt;       /* [ncols][K][2]              deconstructed integers  */
} ob_dump32;

/* RNE(R * 2^e) to binary32, gradual underflow (quantum 2^-149), overflow to
 * infinity.  Done in integers: the one rounding of the FP32 pipeline. */
float ob_ref_pack32(int64_t Rv, int e) {
    if (Rv == 0) return 0.0f;
    int neg = Rv < 0;
    u128 a = neg ? (u128)(-(i128)Rv) : (u128)Rv;
    int L = bitlen_u128(a);
    int d = L - 24;            /* keep 24 significant bits */
    int d_sub = -149 - e;      /* and no bit below 2^-149 */
    if (d_sub > d) d = d_sub;
    u128 q;
    if (d <= 0) {
        q = a;
        d = 0;
    } else if (d > L) {
        q = 0;
    } else {
        q = a >> d;
        u128 rem = a & ((((u128)1) << d) - 1);
        u128 half = ((u128)1) << (d - 1);
        if (rem > half || (rem == half && (q & 1))) q += 1;
    }
    /* q <= 2^24: q 2^(e+d) is a binary32 value or beyond its range; form it in
       double (exact) and narrow (exact, or infinity when too large). */
    double r = ldexp((double)(uint64_t)q, e + d);
    float f = (float)r;
    return neg ? -f : f;
}

/* y[c][k] = RNE32( 2^(e_c - 46) * sum_j F~[g(c)][k][j] * x~[c][j] ) */
int64_t ob_ref_stage32(int64_t ncols, int K, int Kout,
                       const float *x,         /* [ncols][K][2] */
                       const int64_t *Ftab,    /* [ngroups][Kout][K][2], |entry| <= 2^23 */
                       const int32_t *group,   /* [ncols] or NULL */
                       const ob_consts32 *c,
                       int use_crt,
                       float *y,               /* [ncols][Kout][2] */
                       ob_dump32 *dump) {
    int64_t mismatches = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : mismatches)
    for (int64_t col = 0; col < ncols; col++) {
        const float *xc = x + col * (int64_t)K * 2;
        int g = group ? group[col] : 0;
        const int64_t *F = Ftab + (int64_t)g * Kout * K * 2;
        /* deconstruction: one power of two per column, common to Re and Im */
        double amax = 0.0;
        for (int j = 0; j < 2 * K; j++) {
            double a = fabs((double)xc[j]);
            if (a > amax) amax = a;
        }
        int e = amax > 0.0 ? ilogb(amax) : 0;
        int64_t xt[2 * 64];
        for (int j = 0; j < 2 * K; j++) xt[j] = (int64_t)rint(ldexp((double)xc[j], 23 - e));
        if (dump && dump->col_exp) dump->col_exp[col] = e;
        if (dump && dump->xt) memcpy(dump->xt + col * (int64_t)K * 2, xt, sizeof(int64_t) * 2 * K);

        for (int k = 0; k < Kout; k++) {
            const int64_t *Fk = F + (int64_t)k * K * 2;
            i128 Cre = 0, Cim = 0;
            for (int j = 0; j < K; j++) {
                i128 fr = Fk[2 * j], fi = Fk[2 * j + 1];
                i128 xr = xt[2 * j], xi = xt[2 * j + 1];
                Cre += fr * xr - fi * xi;
                Cim += fr * xi + fi * xr;
            }
            i128 Rout[2] = {Cre, Cim};
            if (use_crt) {
                int64_t v[2][NMOD32];
                for (int i = 0; i < NMOD32; i++) {
                    int64_t m = c->m[i];
                    int64_t D = 0, Ev = 0, Fv = 0;
                    for (int j = 0; j < K; j++) {
                        int64_t ar = modc(Fk[2 * j], m), ai = modc(Fk[2 * j + 1], m);
                        int64_t as = modc((i128)Fk[2 * j] + Fk[2 * j + 1], m);
                        int64_t br = modc(xt[2 * j], m), bi = modc(xt[2 * j + 1], m);
                        int64_t bs = modc((i128)xt[2 * j] + xt[2 * j + 1], m);
                        D += ar * br;
                        Ev += ai * bi;
                        Fv += as * bs;
                    }
                    v[0][i] = modc((i128)(D % m) - (Ev % m), m);
                    v[1][i] = modc((i128)(Fv % m) - (D % m) - (Ev % m), m);
                }
                for (int part = 0; part < 2; part++) {
                    int64_t P[S_RAW32], Q[S_FRAC32];
                    for (int s = 0; s < S_RAW32; s++) {
                        P[s] = 0;
                        for (int i = 0; i < NMOD32; i++) P[s] += v[part][i] * c->us[i][s];
                    }
                    for (int t = 0; t < S_FRAC32; t++) {
                        Q[t] = 0;
                        for (int i = 0; i < NMOD32; i++) Q[t] += v[part][i] * c->ws[i][t];
                    }
                    /* Phase B: E = sum_s P_s 256^s, zhat = round(2^-24 sum_t Q_t 256^t),
                       R = E - zhat M, two-sided centered correction */
                    i128 E = 0, zacc = 0;
                    for (int s = 0; s < S_RAW32; s++) E += (i128)P[s] << (8 * s);
                    for (int t = 0; t < S_FRAC32; t++) zacc += (i128)Q[t] << (8 * t);
                    i128 zsum = zacc + ((i128)1 << 23);
                    i128 zq = zsum / ((i128)1 << 24);
                    if (zq * ((i128)1 << 24) > zsum) zq -= 1;
                    i128 Mv = (i128)c->M;
                    i128 Rv = E - zq * Mv;
                    if (2 * Rv >= Mv) Rv -= Mv;
                    if (2 * Rv < -Mv) Rv += Mv;
                    int64_t base = (col * Kout + k) * 2 + part;
                    if (dump) {
                        if (dump->v)
                            for (int i = 0; i < NMOD32; i++) dump->v[base * NMOD32 + i] = (uint16_t)v[part][i];
                        if (dump->P) memcpy(dump->P + base * S_RAW32, P, sizeof P);
                        if (dump->Q) memcpy(dump->Q + base * S_FRAC32, Q, sizeof Q);
                        if (dump->zhat) dump->zhat[base] = (int64_t)zq;
                        if (dump->R) dump->R[base] = (int64_t)Rv;
                    }
                    if (Rv != Rout[part]) mismatches++;
                    Rout[part] = Rv;
                }
            }
            float *yk = y + (col * Kout + k) * 2;
            for (int part = 0; part < 2; part++) yk[part] = ob_ref_pack32((int64_t)Rout[part], e - 46);
        }
    }
    return mismatches;
}

/* Standalone Kulisch + lift over a batch of (P, Q) vectors (regression tests). */
void ob_ref_kulisch(int64_t n, const int64_t *P, const int64_t *Q, const ob_consts *c,
                    int64_t *zhat, int64_t *Rlimbs) {
    for (int64_t i = 0; i < n; i++) {
        i128 Rv = kulisch_lift(P + i * S_RAW, Q + i * S_FRAC, c, zhat ? zhat + i : NULL);
        Rlimbs[2 * i] = (int64_t)(uint64_t)Rv;
        Rlimbs[2 * i + 1] = (int64_t)(uint64_t)((u128)Rv >> 64);
    }
}

/* ------------------------------------------------------------------------ */
/* Plain FP64 mixed-radix FFT along the last axis (the FP64 reference of the  */
/* transform): recursive decimation in time over the smallest prime factor  */
/* of the current length, a direct DFT for prime lengths.  tw: [N][2] =     */
/* exp(sign 2 pi i m / N) rounded to double; every sub-length's twiddle is  */
/* an entry of it (m scaled by N / length).  in/out: [nlines][N][2].        */
/* ------------------------------------------------------------------------ */
static int smallest_factor(int n) {
    for (int f = 2; f * f <= n; f++)
        if (n % f == 0) return f;
    return n;
}

/* y[k] = sum_j x[j stride] w^(j k), length n, w = tw[(N / n) m] */
static void fft_rec(int n, const double *x, int stride, double *y, const double *tw, int N, double *scratch) {
    if (n == 1) {
        y[0] = x[0];
        y[1] = x[1];
        return;
    }
    const int p = smallest_factor(n), m = n / p, step = N / n;
    if (p == n) { /* prime length: direct sum */
        for (int k = 0; k < n; k++) {
            double sr = 0.0, si = 0.0;
            for (int j = 0; j < n; j++) {
                const int e = (int)(((int64_t)j * k) % n) * step;
                const double wr = tw[2 * e], wi = tw[2 * e + 1];
                const double ar = x[2 * j * stride], ai = x[2 * j * stride + 1];
                sr += wr * ar - wi * ai;
                si += wr * ai + wi * ar;
            }
            y[2 * k] = sr;
            y[2 * k + 1] = si;
        }
        return;
    }
    /* p interleaved sub-transforms of length m: sub r holds x[(j p + r) stride] */
    double *sub = scratch;            /* [p][m][2] */
    double *rest = scratch + 2 * n;   /* scratch for the recursion */
    for (int r = 0; r < p; r++) fft_rec(m, x + 2 * r * stride, stride * p, sub + 2 * r * m, tw, N, rest);
    /* y[k1 + m k2] = sum_r w_n^(r k1) w_p^(r k2) sub_r[k1] */
    for (int k1 = 0; k1 < m; k1++)
        for (int k2 = 0; k2 < p; k2++) {
            const int k = k1 + m * k2;
            double sr = 0.0, si = 0.0;
            for (int r = 0; r < p; r++) {
                const int e = (int)(((int64_t)r * k) % n) * step;
                const double wr = tw[2 * e], wi = tw[2 * e + 1];
                const double ar = sub[2 * (r * m + k1)], ai = sub[2 * (r * m + k1) + 1];
                sr += wr * ar - wi * ai;
                si += wr * ai + wi * ar;
            }
            y[2 * k] = sr;
            y[2 * k + 1] = si;
        }
}

void ob_ref_fft_lines(int64_t nlines, int N, const double *tw, const double *in, double *out) {
#pragma omp parallel
    {
        /* scratch: 2n doubles per recursion level, at most log2 N + 1 levels */
        double *scratch = (double *)malloc(sizeof(double) * 2 * (size_t)N * 40);
#pragma omp for schedule(static)
        for (int64_t l = 0; l < nlines; l++)
            fft_rec(N, in + l * (int64_t)N * 2, 1, out + l * (int64_t)N * 2, tw, N, scratch);
        free(scratch);
    }
}

/* ------------------------------------------------------------------------ */
/* Double-double arithmetic (error-free transforms).                         */
/* ------------------------------------------------------------------------ */
typedef struct { double hi, lo; } dd;

static inline dd two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    double err = (a - (s - bb)) + (b - bb);
    dd r = {s, err};
    return r;
}
static inline dd quick_two_sum(double a, double b) {
    double s = a + b;
    dd r = {s, b - (s - a)};
    return r;
}
static inline dd dd_add(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi);
    dd t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}
static inline dd dd_mul(dd a, dd b) {
    double p = a.hi * b.hi;
    double e = fma(a.hi, b.hi, -p);
    e += a.hi * b.lo + a.lo * b.hi;
    return quick_two_sum(p, e);
}
static inline dd dd_neg(dd a) { dd r = {-a.hi, -a.lo}; return r; }

/* Direct DFT along the last (contiguous) axis of length N, for nlines lines,
 * in double-double.  in/out: [nlines][N][4] = (re_hi, re_lo, im_hi, im_lo);
 * tw: [N][4] = exp(sign 2 pi i m / N) in double-double. */
void ob_ref_dft_dd_axis(int64_t nlines, int N, const double *in, const double *tw, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t l = 0; l < nlines; l++) {
        const double *xl = in + l * (int64_t)N * 4;
        double *yl = out + l * (int64_t)N * 4;
        for (int k = 0; k < N; k++) {
            dd sr = {0, 0}, si = {0, 0};
            for (int j = 0; j < N; j++) {
                int m = (int)(((int64_t)j * k) % N);
                dd wr = {tw[4 * m], tw[4 * m + 1]}, wi = {tw[4 * m + 2], tw[4 * m + 3]};
                dd xr = {xl[4 * j], xl[4 * j + 1]}, xi = {xl[4 * j + 2], xl[4 * j + 3]};
                sr = dd_add(sr, dd_add(dd_mul(wr, xr), dd_neg(dd_mul(wi, xi))));
                si = dd_add(si, dd_add(dd_mul(wr, xi), dd_mul(wi, xr)));
            }
            yl[4 * k] = sr.hi; yl[4 * k + 1] = sr.lo;
            yl[4 * k + 2] = si.hi; yl[4 * k + 3] = si.lo;
        }
    }
}

/* One output Y[k0,k1,k2] of the 3-D DFT of a double grid x [n0][n1][n2][2],
 * in double-double, summed separably (innermost axis first). tw_a: [n_a][4].
 * The j0 slices are summed in parallel into per-slice partial results, which
 * are then combined in j0 order: the result does not depend on the thread
 * count. */
void ob_ref_dft_dd_point(int n0, int n1, int n2, const double *x,
                         const double *tw0, const double *tw1, const double *tw2,
                         int k0, int k1, int k2, double *res /* [4] */) {
    dd *Tr = (dd *)malloc(sizeof(dd) * (size_t)n0), *Ti = (dd *)malloc(sizeof(dd) * (size_t)n0);
#pragma omp parallel for schedule(dynamic, 1)
    for (int j0 = 0; j0 < n0; j0++) {
        dd tr = {0, 0}, ti = {0, 0};
        for (int j1 = 0; j1 < n1; j1++) {
            dd Sr = {0, 0}, Si = {0, 0};
            const double *xr = x + (((int64_t)j0 * n1 + j1) * n2) * 2;
            for (int j2 = 0; j2 < n2; j2++) {
                int m = (int)(((int64_t)j2 * k2) % n2);
                dd wr = {tw2[4 * m], tw2[4 * m + 1]}, wi = {tw2[4 * m + 2], tw2[4 * m + 3]};
                dd a = {xr[2 * j2], 0}, b = {xr[2 * j2 + 1], 0};
                Sr = dd_add(Sr, dd_add(dd_mul(wr, a), dd_neg(dd_mul(wi, b))));
                Si = dd_add(Si, dd_add(dd_mul(wr, b), dd_mul(wi, a)));
            }
            int m = (int)(((int64_t)j1 * k1) % n1);
            dd wr = {tw1[4 * m], tw1[4 * m + 1]}, wi = {tw1[4 * m + 2], tw1[4 * m + 3]};
            tr = dd_add(tr, dd_add(dd_mul(wr, Sr), dd_neg(dd_mul(wi, Si))));
            ti = dd_add(ti, dd_add(dd_mul(wr, Si), dd_mul(wi, Sr)));
        }
        Tr[j0] = tr;
        Ti[j0] = ti;
    }
    dd Ur = {0, 0}, Ui = {0, 0};
    for (int j0 = 0; j0 < n0; j0++) {
        int m = (int)(((int64_t)j0 * k0) % n0);
        dd wr = {tw0[4 * m], tw0[4 * m + 1]}, wi = {tw0[4 * m + 2], tw0[4 * m + 3]};
        Ur = dd_add(Ur, dd_add(dd_mul(wr, Tr[j0]), dd_neg(dd_mul(wi, Ti[j0]))));
        Ui = dd_add(Ui, dd_add(dd_mul(wr, Ti[j0]), dd_mul(wi, Tr[j0])));
    }
    free(Tr);
    free(Ti);
    res[0] = Ur.hi; res[1] = Ur.lo; res[2] = Ui.hi; res[3] = Ui.lo;
}
