// Epilogue ablation kernels: the two SIMT-heavy parts of the per-output
// integer epilogue, each in several exact forms with identical results, so
// that their instruction mix and throughput can be measured side by side
// (the paper's width-parameterised Kulisch accumulator, Sec. "The accumulator
// is substrate-agnostic" and Sec. "INT16 and INT8", Eq. kulisch-width, and
// the dp4a migration of the deconstruction bulk, Sec. "Deconstruction count").
//
// Phase B (Kulisch + two-sided lift + correctly rounded pack) of one scalar
// output from its 21 Phase-A accumulators (FP32 bit patterns 2^23 + P_s,
// s < 15, and 2^23 + Q_t, t < 6, of offset residues r_k + 1024):
//   variant 0: the stage kernel's own path (deposits grouped in four 64-bit
//              partial sums of four slices, 128-bit assembly);
//   variant W in {32, 16, 8}: Strategy A of Sec. "INT16 and INT8": the slices
//              deposited into W-bit words of radix 2^rho (rho = 28, 12, 6; the
//              W - rho guard bits absorb the carries), words packed 32 / W per
//              32-bit register and added as packed lanes, then one carry
//              sweep and the 128-bit assembly.
// All variants share the lift and the straight-line pack (lift_pack_fast,
// general finish for the rare cases); every result is exact.
//
// Deconstruction residues x~ mod m_k of the 12 moduli (|x~| < 2^53):
//   variant 0: the stage kernel's form: x~ + 2^55 split into 20/20/16-bit
//              pieces, two multiply-adds with 2^20 and 2^40 mod m, Barrett;
//   variant 1: dp4a: the 7 bytes of x~ + 2^55 against the bytes of
//              2^(8i) mod m (four dp4a per modulus), Barrett;
//   variant 2: the compiler's 64-bit remainder (reference form);
//   variant 3: dp4a as in variant 1, then the paper's H0 rung (Sec. on the
//              co-design ladder; the Rev-34 set's reduction-friendly members,
//              Sec. "Ozaki Scheme II"): fold-and-add t -> (t >> a) c + (t mod
//              2^a) for the seven members m = 2^a - c with small c (2039,
//              2029, 2027; 1024; 511, 491, 487), Barrett for the other five.
//
// Each kernel reads n_unique inputs (small enough to stay in L2) and processes
// n_total items, item i using input i mod n_unique, `reps` times each with the
// input perturbed by the repetition index (slice sum P_0 + r, or x~ + r), so
// that a timing launch does reps times the arithmetic per byte loaded.  The
// results of the first n_unique items (repetition 0) are stored when `out` is
// given; every result is folded into a 64-bit XOR checksum.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "obfft_internal.h"

namespace obfft {

__constant__ ModConsts c_abl_mc;

constexpr int ABL_THREADS = 256;

// The modulus set as compile-time constants for the H0 variant (the fold
// shifts and counts must be known to the compiler); checked against the
// plan's table before every launch.
__host__ __device__ constexpr int h0_modulus(int k) {
    return k == 0 ? 2039 : k == 1 ? 2029 : k == 2 ? 2027 : k == 3 ? 1089 : k == 4 ? 1024 : k == 5 ? 961
         : k == 6 ? 841 : k == 7 ? 625 : k == 8 ? 529 : k == 9 ? 511 : k == 10 ? 491 : 487;
}
// a of a reduction-friendly member m = 2^a - c (c <= 25), 0 for the others
__host__ __device__ constexpr int h0_shift(int k) {
    const int m = h0_modulus(k);
    return m > 2000 ? 11 : (m == 1024 ? 10 : (m >= 487 && m <= 511 ? 9 : 0));
}
// Folds that bring the dp4a sum t <= 7 x 255 x (m - 1) below 2m: each fold
// maps a bound T to (T >> a) c + 2^a - 1.
__host__ __device__ constexpr int h0_folds(int k) {
    const int a = h0_shift(k);
    if (a == 0) return 0;
    const uint64_t m = (uint64_t)h0_modulus(k), c = (1ull << a) - m;
    uint64_t t = 7ull * 255ull * (m - 1);
    int n = 0;
    while (t >= 2 * m && n < 8) {
        t = (t >> a) * c + ((1ull << a) - 1);
        n++;
    }
    return n;
}
static_assert(h0_folds(0) == 2 && h0_folds(4) == 1 && h0_folds(11) == 3, "fold counts");

// Kulisch accumulator of E = sum_s P_s 256^s in words of radix 2^RHO, LANES
// words of 32 / LANES bits packed per 32-bit register (word i in register
// i / LANES, lane i % LANES).
template <int RHO, int LANES>
struct KulischWords {
    static constexpr int WB = 32 / LANES;                 // word width
    static constexpr int TOP = 8 * (S_RAW - 1) + 23;      // highest deposited bit + 1
    static constexpr int NW = (TOP + RHO - 1) / RHO + 1;  // words (one spare for the carry sweep)
    static constexpr int NR = (NW + LANES - 1) / LANES;   // registers
    uint32_t r[NR];
};

// Deposit of P (< 2^23) at bit 8 s: the pieces of P << (8 s mod RHO) go to
// consecutive words, each piece below 2^RHO.  Positions are compile-time.
template <int RHO, int LANES, int S>
__device__ __forceinline__ void kw_deposit(KulischWords<RHO, LANES> &acc, uint32_t P) {
    constexpr int WB = 32 / LANES;
    constexpr int i0 = 8 * S / RHO, o = 8 * S % RHO;
    constexpr int NP = (23 + o + RHO - 1) / RHO;
    const uint64_t v = (uint64_t)P << o;
#pragma unroll
    for (int j = 0; j < NP; j++) {
        const uint32_t piece = (uint32_t)(v >> (RHO * j)) & ((1u << RHO) - 1u);
        const int i = i0 + j;
        acc.r[i / LANES] += piece << (WB * (i % LANES));
    }
}

template <int RHO, int LANES, int S = 0>
__device__ __forceinline__ void kw_deposit_all(KulischWords<RHO, LANES> &acc, const uint32_t *wv) {
    if constexpr (S < S_RAW) {
        kw_deposit<RHO, LANES, S>(acc, wv[S] - 0x4B000000u);
        kw_deposit_all<RHO, LANES, S + 1>(acc, wv);
    }
}

// Carry sweep and assembly of the exact E (mod 2^128) as four 32-bit words.
template <int RHO, int LANES>
__device__ __forceinline__ void kw_resolve(const KulischWords<RHO, LANES> &acc, uint32_t (&e)[4]) {
    using KW = KulischWords<RHO, LANES>;
    constexpr int WB = KW::WB;
    u128 E = 0;
    uint32_t carry = 0;
#pragma unroll
    for (int i = 0; i < KW::NW; i++) {
        uint32_t word;
        if constexpr (LANES == 1)
            word = acc.r[i];
        else
            word = (acc.r[i / LANES] >> (WB * (i % LANES))) & ((1u << WB) - 1u);
        const uint32_t t = word + carry;
        carry = t >> RHO;
        if (RHO * i < 128) E |= (u128)(t & ((1u << RHO) - 1u)) << (RHO * i);
    }
    e[0] = (uint32_t)E;
    e[1] = (uint32_t)(E >> 32);
    e[2] = (uint32_t)(E >> 64);
    e[3] = (uint32_t)(E >> 96);
}

template <int VARIANT>
__global__ void __launch_bounds__(ABL_THREADS) phase_b_ablation_kernel(const uint32_t *__restrict__ acc,
                                                                       const int *__restrict__ et,
                                                                       int64_t n_unique, int64_t n_total, int reps,
                                                                       double *__restrict__ out,
                                                                       unsigned long long *checksum) {
    const ModConsts &mc = c_abl_mc;
    const uint32_t ebias[4] = {mc.kbias[0], mc.kbias[1], mc.kbias[2], mc.kbias[3]};
    const uint64_t zbias = ((uint64_t)mc.zbias[1] << 32) | mc.zbias[0];
    uint64_t x = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = i % n_unique;
        uint32_t wv[21];
#pragma unroll
        for (int j = 0; j < 21; j++) wv[j] = acc[u * 21 + j];
        const int e = et[u];
        const uint32_t w00 = wv[0];
        for (int r = 0; r < reps; r++) {
        wv[0] = w00 + (uint32_t)r;
        double y;
        bool slow, near;
        uint32_t Rw[4];
        if constexpr (VARIANT == 0) {
            y = kulisch_pack_fp8_fast(wv, mc, e, ebias, zbias, slow, Rw, near);
        } else {
            constexpr int RHO = VARIANT == 32 ? 28 : (VARIANT == 16 ? 12 : 6);
            constexpr int LANES = 32 / VARIANT;
            KulischWords<RHO, LANES> kw;
#pragma unroll
            for (int r = 0; r < KulischWords<RHO, LANES>::NR; r++) kw.r[r] = 0u;
            kw_deposit_all<RHO, LANES>(kw, wv);
            uint32_t ew[4];
            kw_resolve<RHO, LANES>(kw, ew);
            // the deposits were unbiased: only the residue offset remains to remove
            const uint32_t off[4] = {(uint32_t)RES_OFFSET, 0u, 0u, 0u};
            y = lift_pack_fast(ew[0], ew[1], ew[2], ew[3], wv + S_RAW, mc, e, off, zbias, slow, Rw, near);
        }
        if (slow) y = kulisch_finish_general(Rw[0], Rw[1], Rw[2], Rw[3], near, e, mc);
        if (out && i < n_unique && r == 0) out[i] = y;
        x ^= (uint64_t)__double_as_longlong(y) + (uint64_t)(i + r);
        }
    }
    atomicXor(checksum, (unsigned long long)x);
}

template <int VARIANT>
__global__ void __launch_bounds__(ABL_THREADS) residue_ablation_kernel(const int64_t *__restrict__ xt,
                                                                       int64_t n_unique, int64_t n_total, int reps,
                                                                       uint16_t *__restrict__ res,
                                                                       unsigned long long *checksum) {
    const ModConsts &mc = c_abl_mc;
    uint64_t x = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = i % n_unique;
        const int64_t x0 = xt[u];
        for (int rp = 0; rp < reps; rp++) {
        const uint64_t v = (uint64_t)(x0 + rp + (1ll << 55));  // in [2^54, 2^56)
        uint32_t r[NMOD];
#pragma unroll
        for (int k = 0; k < NMOD; k++) {
            const uint32_t m = mc.m[k];
            uint32_t t;
            if constexpr (VARIANT == 0) {
                const uint32_t p0 = (uint32_t)v & 0xFFFFFu, p1 = (uint32_t)(v >> 20) & 0xFFFFFu,
                               p2 = (uint32_t)(v >> 40);
                t = p0 + p1 * mc.c20[k] + p2 * mc.c40[k];  // < 2^32
                t = t - __umulhi(t, mc.barrett[k]) * m;     // [0, 2m)
            } else if constexpr (VARIANT == 1) {
                const uint32_t lo = (uint32_t)v, hi = (uint32_t)(v >> 32);
                const uint32_t tl = __dp4a(lo, mc.b8lo[k][0], __dp4a(hi, mc.b8lo[k][1], 0u));
                const uint32_t th = __dp4a(lo, mc.b8hi[k][0], __dp4a(hi, mc.b8hi[k][1], 0u));
                t = tl + (th << 8);                       // < 7 x 255 x 2047 < 2^22
                t = t - __umulhi(t, mc.barrett[k]) * m;  // [0, 2m)
            } else if constexpr (VARIANT == 3) {
                const uint32_t lo = (uint32_t)v, hi = (uint32_t)(v >> 32);
                const uint32_t tl = __dp4a(lo, mc.b8lo[k][0], __dp4a(hi, mc.b8lo[k][1], 0u));
                const uint32_t th = __dp4a(lo, mc.b8hi[k][0], __dp4a(hi, mc.b8hi[k][1], 0u));
                t = tl + (th << 8);  // sum of the bytes times 2^(8i) mod m: <= 7 x 255 x (m - 1)
                const int a = h0_shift(k);
                if (a == 0) {
                    t = t - __umulhi(t, mc.barrett[k]) * m;  // [0, 2m)
                } else {
                    const uint32_t c = (1u << a) - (uint32_t)h0_modulus(k), mask = (1u << a) - 1u;
#pragma unroll
                    for (int f = 0; f < h0_folds(k); f++) t = (t >> a) * c + (t & mask);  // [0, 2m) after the last
                }
            } else {
                t = (uint32_t)(v % m);
            }
            t = t >= m ? t - m : t;
            // remove the 2^55 bias: x~ = v - 2^55, (-2^55) mod m = c55neg
            t += mc.c55neg[k];
            t = t >= m ? t - m : t;
            r[k] = t;
        }
        if (res && i < n_unique && rp == 0) {
#pragma unroll
            for (int k = 0; k < NMOD; k++) res[i * NMOD + k] = (uint16_t)r[k];
        }
        uint64_t h = (uint64_t)(i + rp);
#pragma unroll
        for (int k = 0; k < NMOD; k++) h = h * 0x9E3779B97F4A7C15ull + r[k];
        x ^= h;
        }
    }
    atomicXor(checksum, (unsigned long long)x);
}

static cudaError_t abl_upload() {
    for (int k = 0; k < NMOD; k++)
        if (h0_modulus(k) != kModuli[k]) return cudaErrorInvalidValue;
    ModConsts mc;
    make_mod_consts(&mc);
    return cudaMemcpyToSymbol(c_abl_mc, &mc, sizeof(mc));
}

static unsigned abl_blocks(int64_t n_total) {
    int dev = 0, nsm = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n_total + ABL_THREADS - 1) / ABL_THREADS;
    const int64_t cap = (int64_t)nsm * 8;  // 8 resident CTAs per SM, grid-stride beyond
    return (unsigned)(want < cap ? want : cap);
}

cudaError_t launch_phase_b_ablation(int variant, int64_t n_unique, int64_t n_total, int reps, const uint32_t *acc,
                                    const int *et, double *out, unsigned long long *checksum, cudaStream_t s) {
    cudaError_t e = abl_upload();
    if (e != cudaSuccess) return e;
    const unsigned nb = abl_blocks(n_total);
    switch (variant) {
        case 0: phase_b_ablation_kernel<0><<<nb, ABL_THREADS, 0, s>>>(acc, et, n_unique, n_total, reps, out, checksum); break;
        case 32: phase_b_ablation_kernel<32><<<nb, ABL_THREADS, 0, s>>>(acc, et, n_unique, n_total, reps, out, checksum); break;
        case 16: phase_b_ablation_kernel<16><<<nb, ABL_THREADS, 0, s>>>(acc, et, n_unique, n_total, reps, out, checksum); break;
        case 8: phase_b_ablation_kernel<8><<<nb, ABL_THREADS, 0, s>>>(acc, et, n_unique, n_total, reps, out, checksum); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_residue_ablation(int variant, int64_t n_unique, int64_t n_total, int reps, const int64_t *xt,
                                    uint16_t *res, unsigned long long *checksum, cudaStream_t s) {
    cudaError_t e = abl_upload();
    if (e != cudaSuccess) return e;
    const unsigned nb = abl_blocks(n_total);
    switch (variant) {
        case 0: residue_ablation_kernel<0><<<nb, ABL_THREADS, 0, s>>>(xt, n_unique, n_total, reps, res, checksum); break;
        case 1: residue_ablation_kernel<1><<<nb, ABL_THREADS, 0, s>>>(xt, n_unique, n_total, reps, res, checksum); break;
        case 2: residue_ablation_kernel<2><<<nb, ABL_THREADS, 0, s>>>(xt, n_unique, n_total, reps, res, checksum); break;
        case 3: residue_ablation_kernel<3><<<nb, ABL_THREADS, 0, s>>>(xt, n_unique, n_total, reps, res, checksum); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace obfft
