// FP8-mode Bailey stage on Blackwell tensor cores (tcgen05, sm_103a).
//
// One CTA transforms 128 columns (one Ozaki-II complex GEMM per column,
// Algorithm 1, one half), or 256 when K <= 16 (two columns per TMEM lane, see
// the kernel's LPV parameter).  Per modulus m_k:
//   * the data residues (x~ mod m_k, balanced) of the real and
//     imaginary parts are split into E4M3-exact digit planes by the SIMT
//     threads and written straight into tensor memory, where tcgen05.mma reads
//     them as its A operand (row = column of the DFT, 32 bytes of K);
//   * the constant DFT / twiddle-fused matrix digits (planes of a_R, a_I and
//     -a_I) arrive in shared memory by TMA bulk copy, double buffered;
//   * the complex product is formed in real form, Re = a_R b_R + (-a_I) b_I and
//     Im = a_I b_R + a_R b_I, in one pipelined step per modulus.  The constant
//     operand stacks, along N, the Re and Im rows of every constant digit, so
//     one tcgen05.mma kind::f8f6f4 (M = 128, N = 2 npad x digits, K = 32) per
//     data digit and half (x_R or x_I) adds its digit products to a window of
//     consecutive weight classes in TMEM (FP32, every partial sum an integer
//     below 2^17: exact): 4 to 6 MMAs per modulus.  On this GPU the tensor pipe
//     has ample headroom and the SIMT epilogue is the bottleneck, so the fourth
//     real product is cheaper than the Karatsuba operand a_R + a_I and the
//     residue-domain combine it would need (the INT8 mode keeps the paper's
//     Karatsuba split);
//   * the epilogue reads the classes back (tcgen05.ld), recombines them with
//     their weights, reduces mod m_k to |r| <= m_k/2 + 1 and writes r + 1024
//     as the FP16 CRT operand (Sec. tcgarner: integers below 2048 are
//     FP16-exact) to shared memory.  Any representative of the residue class
//     serves the CRT: sum_k u_k = 1 (mod M), so the offset lifts to C + 1024
//     and is removed with the Kulisch bias constant.
// The per-element and per-output arithmetic runs as packed two-lane FP32
// (fma/add.f32x2), on the Re/Im parts of an element or on two outputs.
// After the 12 moduli, CRT Phase A runs as tcgen05.mma kind::f16 (M = 128
// complex outputs, N = 48 = Re/Im x (15 byte slices of u_k + 6 of w_k + 3
// pad), K = 24 = Re/Im x 12 moduli, accumulators preset to 2^23, FP32
// accumulation exact below 2^24, Eq. phaseAcost), and each thread finishes its
// outputs with the Kulisch sum E = sum_s P_s 256^s, the lift quotient from the
// w_k columns, the two-sided modulo-M correction and the correctly rounded
// pack (Algorithm 2).
//
// Digit layouts (exhaustively verified on the host, see the FP8 layout tests):
//   m = s^2 (1089, 1024, 961, 841, 625, 529): v = s h + l, |h|, |l| <= 16;
//       a b = s (a_h b_l + a_l b_h) + a_l b_l (mod m): classes {s: 2 products, 1: 1}.
//   511, 491, 487: v = d0 + 16 d1, |d0| <= 8, |d1| <= 16: classes 16^w, w = 0..2.
//   2039, 2029, 2027: v = d0 + 16 d1 + 256 d2, |d0|,|d1| <= 8, |d2| <= 4:
//       classes 16^w (w = 0..4), 16^3 and 16^4 reduced mod m.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "obfft_internal.h"
#include "tc_common.cuh"
#include "tc_stage.cuh"

namespace obfft {

// modulus kinds, in the order of kModuli
enum : int { KIND_B11 = 0, KIND_SQ = 1, KIND_B9 = 2, KIND_F16 = 3 };  // KIND_F16: the FP16 carrier
__host__ __device__ constexpr int fp8_kind(int k) { return k < 3 ? KIND_B11 : (k < 9 ? KIND_SQ : KIND_B9); }
__host__ __device__ constexpr int fp8_ndig(int k) { return fp8_kind(k) == KIND_B11 ? 3 : 2; }
__host__ __device__ constexpr int fp8_ncls(int k) {
    return fp8_kind(k) == KIND_B11 ? 5 : (fp8_kind(k) == KIND_SQ ? 2 : 3);
}
// planes before modulus k in a per-group table: sum_{k' < k} 4 * ndig(k')
__host__ __device__ constexpr int fp8_plane_offset(int k) {
    int s = 0;
    for (int i = 0; i < k; i++) s += 4 * fp8_ndig(i);
    return s;
}
static_assert(fp8_plane_offset(NMOD) == FP8_PLANES_PER_GROUP, "plane table size");
constexpr int FP8_BPLANES = 12;  // planes of one modulus' constant operand buffer (at most 4 x 3)

constexpr int PA_N = 48;          // Phase A output columns (Re 24 | Im 24)
constexpr int PA_GSLOTS = 2;      // Phase-A accumulator slots per quarter-warp group (8 x 48 TMEM columns)
constexpr int PA_SLOTS = 4 * PA_GSLOTS;
// TMEM column of the first Phase-A slot in the FP16 carrier: the slots take
// columns 128..511, so they never overlap the accumulator set of the last
// modulus (columns 0..127), which other warps may still be reading when a warp
// presets its first slots.  The E4M3 pipeline ends every modulus with a CTA
// barrier, and its slots start at column 0 (measured 0.8 % faster than 128).
constexpr uint32_t PA_COL0 = 128;
static_assert(PA_COL0 + PA_SLOTS * PA_N <= 512, "Phase-A slots within the 512 TMEM columns");
constexpr int PA_ROWB = 384;      // bytes per 8-row group of the staging (3 K-chunks)
constexpr uint32_t WAIT_LIMIT = 1u << 22;


// byte offset of element (row, k) of the Phase-A staging (K-major, 3 chunks of 8 f16)
__device__ __forceinline__ uint32_t stage_off(uint32_t row, uint32_t k) {
    return (row >> 3) * PA_ROWB + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}


// ---------------------------------------------------------------------------
// Kernel: 512 threads.  Thread (sub = warp % 4, qd = warp / 4) owns TMEM lane
// c = 32 sub + lane (= DFT column c of the tile), deconstructs elements
// [EPT qd, EPT qd + EPT) of that column and finishes outputs [OPT qd, OPT qd +
// OPT) of the Re and Im products.  The per-modulus steps are software
// pipelined: the digits of modulus k+1 are generated (into the other TMEM
// A-buffer) while the MMAs of modulus k run; the TMA-loaded constant planes
// are double buffered.
// TMEM columns (E4M3 digits): class accumulators [0,320) (class cl: Re at
// cl 2 npad, Im at cl 2 npad + npad); A digit planes of x_R (planes 0..2) and
// x_I (planes 3..5) of one modulus in two buffers [320,368) and [368,416);
// the eight Phase-A slots reuse [0,384).  FP16 carrier: two accumulator sets
// [0,128) and [128,256), two A buffers from column 320, Phase-A slots
// [128,512).  One pipeline step per modulus: its MMAs run while the next
// modulus' digits are generated.
// ---------------------------------------------------------------------------
constexpr int FP8_WARPS = 16;

// Per-modulus constants (identical for every plan): read through the constant
// cache, uploaded once per device when the first FP8 plan is created.
__constant__ ModConsts c_fp8_mc;
constexpr uint32_t APL_BASE = 320, APL_COLS = 48;  // two A buffers
// FP16 carrier: TMEM columns of one accumulator set (two classes, Re | Im, at
// npad = 32); the second set follows the first, below the A buffers.  Modulus
// k uses set (k ^ (NMOD - 1)) & 1, so the last modulus uses set 0.
constexpr uint32_t F16_ACC = 128;
__device__ __forceinline__ uint32_t f16_acc_col(int k) { return (uint32_t)((k ^ (NMOD - 1)) & 1) * F16_ACC; }

template <int NPAD>
struct Fp8Cfg {
    static constexpr int EPT = NPAD / 4;  // elements per thread (K <= NPAD)
    static constexpr int OPT = NPAD / 4;  // outputs per thread per product
    static constexpr int WPP = EPT / 4;   // 32-bit TMEM words per plane per thread
};

// Digits of EPT balanced residue pairs (x_R, x_I) -> E4M3 words of up to 3
// planes each for x_R (wR) and x_I (wI); the digit arithmetic runs packed on
// both parts of an element.
template <int KIND, int EPT>
__device__ __forceinline__ void digits_to_words2(const float2 (&v)[EPT], float s, uint32_t (&wR)[3][EPT / 4],
                                                 uint32_t (&wI)[3][EPT / 4]) {
    float2 dg[3][EPT];
#pragma unroll
    for (int j = 0; j < EPT; j++) {
        const float2 x = v[j];
        if constexpr (KIND == KIND_SQ) {
            const float2 h = rint2_mul(x, f2splat(1.0f / s));
            dg[0][j] = h;
            dg[1][j] = __ffma2_rn(f2splat(-s), h, x);
        } else if constexpr (KIND == KIND_B9) {
            const float2 d1 = rint2_mul(x, f2splat(0.0625f));
            dg[1][j] = d1;
            dg[0][j] = __ffma2_rn(f2splat(-16.0f), d1, x);
        } else {
            const float2 d2 = rint2_mul(x, f2splat(0.00390625f));
            const float2 r = __ffma2_rn(f2splat(-256.0f), d2, x);
            const float2 d1 = rint2_mul(r, f2splat(0.0625f));
            dg[2][j] = d2;
            dg[1][j] = d1;
            dg[0][j] = __ffma2_rn(f2splat(-16.0f), d1, r);
        }
    }
    constexpr int ND = KIND == KIND_B11 ? 3 : 2;
#pragma unroll
    for (int d = 0; d < ND; d++)
#pragma unroll
        for (int q4 = 0; q4 < EPT / 4; q4++) {
            const int j = 4 * q4;
            wR[d][q4] = e4m3x2(dg[d][j].x, dg[d][j + 1].x) | (e4m3x2(dg[d][j + 2].x, dg[d][j + 3].x) << 16);
            wI[d][q4] = e4m3x2(dg[d][j].y, dg[d][j + 1].y) | (e4m3x2(dg[d][j + 2].y, dg[d][j + 3].y) << 16);
        }
}

// MMAs of one modulus, complex product in real form with the Re and Im
// outputs side by side along N: for the x_R half the constant rows are
// (a_R, a_I) per digit, for the x_I half (-a_I, a_R), so each MMA adds
// a_R b_R and a_I b_R (or -a_I b_I and a_R b_I) to the Re and Im columns of
// consecutive weight classes.  One MMA per data digit and half: its constant
// operand holds every constant digit (in class order), its accumulator window
// starts at the class of the data digit.  TMEM accumulator of class cl:
// columns [cl 2 npad, cl 2 npad + npad) Re, [.. + npad, .. + 2 npad) Im.
// Classes the window reaches beyond the first MMA's (B9: 2, B11: 3 and 4)
// must hold zero when the modulus starts.
template <int KIND>
__device__ __forceinline__ void issue_modulus_nm(uint32_t dacc, uint32_t apl, uint64_t bdesc, int npad) {
    constexpr int ND = KIND == KIND_B11 ? 3 : 2;
    const uint32_t planeB16 = (uint32_t)npad * 2;  // plane size in 16-byte descriptor units
    const uint32_t cls = 2u * (uint32_t)npad;       // TMEM columns per class
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const uint64_t bh = bdesc + (uint64_t)(h * 2 * ND) * planeB16;
        const uint32_t ah = apl + (uint32_t)(3 * h) * 8;  // data planes of x_R (h = 0) or x_I (h = 1)
        if (KIND == KIND_SQ) {  // data digit 0 = h, 1 = l; constant rows [l pair, h pair]
            tc_mma_f8_ta(dacc, ah + 8, bh, instr_desc(128, 4 * npad, 0), h ? 1u : 0u);  // classes 1, s
            tc_mma_f8_ta(dacc + cls, ah, bh, instr_desc(128, 2 * npad, 0), 1u);        // class s
        } else {
#pragma unroll
            for (int dj = 0; dj < ND; dj++)
                tc_mma_f8_ta(dacc + (uint32_t)dj * cls, ah + (uint32_t)dj * 8, bh,
                             instr_desc(128, 2 * ND * npad, 0), (h == 0 && dj == 0) ? 0u : 1u);
        }
    }
}


constexpr int fp8_ncls_of_kind(int kind) {
    return kind == KIND_B11 ? 5 : ((kind == KIND_SQ || kind == KIND_F16) ? 2 : 3);
}

// Issue the TMEM loads of the class accumulators of this thread's OPT outputs
// (completion: tmem_wait_ld, then regs_after_wait).
template <int KIND, int OPT>
__device__ __forceinline__ void load_classes(uint32_t tacc, int npad, uint32_t (&r)[5][OPT]) {
#pragma unroll
    for (int cl = 0; cl < fp8_ncls_of_kind(KIND); cl++) {
        if constexpr (OPT == 8)
            tmem_ld8(tacc + cl * 2 * npad, r[cl]);
        else
            tmem_ld4(tacc + cl * 2 * npad, r[cl]);
    }
}
// Zero this thread's columns of the classes >= 2 (they must start the next
// modulus at zero, see issue_modulus_nm).
template <int KIND, int OPT>
__device__ __forceinline__ void zero_high_classes(uint32_t tacc, int npad) {
#pragma unroll
    for (int cl = 2; cl < fp8_ncls_of_kind(KIND); cl++) {
        if constexpr (OPT == 8)
            tmem_st8_const(tacc + cl * 2 * npad, 0u);
        else
            tmem_st4_const(tacc + cl * 2 * npad, 0u);
    }
}
// Orders every later use of the loaded registers after the preceding tcgen05.wait::ld.
template <int KIND, int OPT>
__device__ __forceinline__ void regs_after_wait(uint32_t (&r)[5][OPT]) {
#pragma unroll
    for (int cl = 0; cl < fp8_ncls_of_kind(KIND); cl++)
#pragma unroll
        for (int i = 0; i < OPT; i++) asm volatile("" : "+r"(r[cl][i]));
}
// Class values -> their weighted sums (exact integers, |a| < 2^24, congruent
// to sum_j a_j b_j mod m), as packed pairs of consecutive outputs.
template <int KIND, int OPT>
__device__ __forceinline__ void combine_classes(const uint32_t (&r)[5][OPT], const ModConsts &mc, int k,
                                                float2 (&out)[OPT / 2]) {
    constexpr int NC = fp8_ncls_of_kind(KIND);
    if constexpr (KIND == KIND_F16) {
        // c0-class + 32 x c1-class exceeds 2^24: reduce the c1-class first
        // (|x| < 2^22, so x - m RNE(x / m) is exact and within m/2 + 1)
        const float2 nm2 = f2splat(-mc.fm[k]), im2 = f2splat(mc.finv[k]);
#pragma unroll
        for (int i = 0; i < OPT / 2; i++) {
            const float2 c1 = make_float2(__uint_as_float(r[1][2 * i]), __uint_as_float(r[1][2 * i + 1]));
            const float2 r1 = __ffma2_rn(nm2, rint2_mul(c1, im2), c1);
            out[i] = __ffma2_rn(f2splat(32.0f), r1,
                                make_float2(__uint_as_float(r[0][2 * i]), __uint_as_float(r[0][2 * i + 1])));
        }
        return;
    }
    float wts[5];
    if constexpr (KIND == KIND_SQ) {
        wts[0] = 1.f;
        wts[1] = mc.fsq[k];
    } else {
        wts[0] = 1.f;
        wts[1] = 16.f;
        wts[2] = 256.f;
        wts[3] = mc.fc3[k];
        wts[4] = mc.fc4[k];
    }
#pragma unroll
    for (int i = 0; i < OPT / 2; i++) {
        float2 a = make_float2(__uint_as_float(r[0][2 * i]), __uint_as_float(r[0][2 * i + 1]));
#pragma unroll
        for (int cl = 1; cl < NC; cl++)
            a = __ffma2_rn(f2splat(wts[cl]),
                           make_float2(__uint_as_float(r[cl][2 * i]), __uint_as_float(r[cl][2 * i + 1])), a);
        out[i] = a;
    }
}

// Epilogue of modulus k for this thread's OPT outputs of the Re and Im
// products: offset residues as FP16 into the Phase-A staging, where the Re
// and Im residues of modulus k are neighbours along K (columns 2k and 2k + 1
// of the output's row), so each output takes one 32-bit store.  The loads of
// the Im classes are in flight while the Re residues are reduced.
// dres (debug instantiations only): the dump row of this thread's column,
// receiving the offset residues of its outputs kl = slot - kbase < Kline.
template <int KIND, int OPT>
__device__ __forceinline__ void epilogue_modulus(uint32_t tacc_re, uint32_t tacc_im, int npad, const ModConsts &mc,
                                                 int k, uint8_t *sStage, int c, int qd, int Kout,
                                                 uint16_t *dres = nullptr, int kbase = 0, int Kline = 0) {
    const float2 nm2 = f2splat(-mc.fm[k]), im2 = f2splat(mc.finv[k]);
    uint32_t r[5][OPT];
    float2 res[OPT / 2], cvR[OPT / 2];
    load_classes<KIND, OPT>(tacc_re, npad, r);
    tmem_wait_ld();
    regs_after_wait<KIND, OPT>(r);
    combine_classes<KIND, OPT>(r, mc, k, res);
    zero_high_classes<KIND, OPT>(tacc_re, npad);
    load_classes<KIND, OPT>(tacc_im, npad, r);
#pragma unroll
    for (int o2 = 0; o2 < OPT / 2; o2++) cvR[o2] = offset_residue2(res[o2], nm2, im2);
    tmem_wait_ld();
    regs_after_wait<KIND, OPT>(r);
    combine_classes<KIND, OPT>(r, mc, k, res);
    zero_high_classes<KIND, OPT>(tacc_im, npad);
    // column 2k of the staging row (K-major: 8 FP16 per 16-byte core row)
    uint8_t *base = sStage + stage_off((uint32_t)(qd * OPT) * 128 + c, 0) + (uint32_t)(k >> 2) * 128 +
                    (uint32_t)(k & 3) * 4;
#pragma unroll
    for (int o2 = 0; o2 < OPT / 2; o2++) {
        const float2 cvI = offset_residue2(res[o2], nm2, im2);
        // exact: offset residues in [2, 2046]
        const uint32_t w0 = f16x2(cvR[o2].x, cvI.x), w1 = f16x2(cvR[o2].y, cvI.y);
        const int k0 = qd * OPT + 2 * o2;
        // each output slot is 128 staging rows = 16 row groups further on
        if (k0 < Kout) *reinterpret_cast<uint32_t *>(base + (uint32_t)(2 * o2) * (16 * PA_ROWB)) = w0;
        if (k0 + 1 < Kout) *reinterpret_cast<uint32_t *>(base + (uint32_t)(2 * o2 + 1) * (16 * PA_ROWB)) = w1;
        if (dres) {
            const float vr[2] = {cvR[o2].x, cvR[o2].y}, vi[2] = {cvI.x, cvI.y};
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int kl = k0 + h - kbase;
                if (kl >= 0 && kl < Kline) {
                    dres[(kl * 2 + 0) * NMOD + k] = (uint16_t)vr[h];
                    dres[(kl * 2 + 1) * NMOD + k] = (uint16_t)vi[h];
                }
            }
        }
    }
}

// Input tile of the columns [cb, cb + width): stage 1 reads whole or partial
// lines, one contiguous range [e0, e1) of elements; stage 2 reads K = p
// contiguous elements per column, at addresses in arithmetic progression.
struct InputTile {
    int64_t e0, e1;    // stage 1: element range
    int64_t src0, n;   // stage 2: column i starts at element src0 + i n
    int nvalid;        // stage 2: valid columns (the first nvalid of the tile)
};
__device__ __forceinline__ InputTile input_tile(const ColMapT &map, int64_t ncols, int64_t cb, int width) {
    InputTile t;
    if (map.stage == 1) {
        const int64_t l0 = cb / map.p, l1 = min(cb + width - 1, ncols - 1) / map.p;
        t.e0 = l0 * map.n;
        t.e1 = (l1 + 1) * map.n;
        t.src0 = 0;
        t.n = 0;
        t.nvalid = 0;
    } else {  // a stage-2 tile lies inside one group of Lpad columns
        const int64_t k2 = cb / map.Lpad, l0 = cb - k2 * map.Lpad;
        t.e0 = t.e1 = 0;
        t.src0 = l0 * map.n + k2 * map.p;
        t.n = map.n;
        t.nvalid = (int)max((int64_t)0, min((int64_t)width, map.L - l0));
    }
    return t;
}
// Stage 1: bulk copies of the input tile (one contiguous element range) into
// shared memory (warp-wide call), completing on mbar.
__device__ __forceinline__ void copy_input_tile(const InputTile &t, const double2 *in, uint8_t *sIn, uint32_t mbar,
                                                int lane) {
    if (lane == 0) mbar_expect_tx(mbar, (uint32_t)((t.e1 - t.e0) * 16));
    __syncwarp();
    // one copy per 64 KB (a tile is at most 64 KB: one copy); 4 KB copies
    // measured 0.6 % slower per stage-1 launch, the copy engine's per-copy
    // cost showing in the CTA set-up
    const int64_t chunk = 4096;
    for (int64_t e = t.e0 + (int64_t)lane * chunk; e < t.e1; e += 32 * chunk)
        tma_bulk_g2s(smem_u32(sIn + (e - t.e0) * 16), in + e, (uint32_t)(min(chunk, t.e1 - e) * 16), mbar);
}
// Stage 1: L2 prefetch of an input tile (warp-wide call)
__device__ __forceinline__ void prefetch_input_tile(const InputTile &t, const double2 *in, int lane) {
    const int64_t chunk = 4096;
    for (int64_t e = t.e0 + (int64_t)lane * chunk; e < t.e1; e += 32 * chunk)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(in + e), "r"((uint32_t)(min(chunk, t.e1 - e) * 16))
                     : "memory");
}

// The general Kulisch finish, out of line: it runs only for the rare outputs the
// straight-line form flags, and keeping it out of the hot code saves registers
// and instruction cache.
__device__ __noinline__ double kulisch_finish_slow(uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3, int near,
                                                   int et) {
    return kulisch_finish_general(r0, r1, r2, r3, near != 0, et, c_fp8_mc);
}

// Constant-plane geometry of the two carriers.  E4M3 (CAR 0): planes of npad
// rows x 32 bytes (K <= 32 one-byte digits), 4 x digits per modulus.  FP16
// (CAR 1): planes of npad rows x npad FP16 values, 8 per modulus.
template <int NPAD, int CAR>
struct CarrierCfg {
    static constexpr uint32_t PLANE_B = CAR ? NPAD * NPAD * 2 : NPAD * 32;
    static constexpr uint32_t SBO = CAR ? 16 * NPAD : 256;  // bytes between 8-row groups
    static constexpr int BUF_PLANES = CAR ? 8 : FP8_BPLANES;
    static constexpr int PLANES_PER_GROUP = CAR ? FP16_PLANES_PER_GROUP : FP8_PLANES_PER_GROUP;
    static constexpr uint32_t A_COLS = CAR ? NPAD : APL_COLS;  // TMEM columns of one A buffer
    __host__ __device__ static constexpr int plane_offset(int k) { return CAR ? 8 * k : fp8_plane_offset(k); }
    __host__ __device__ static constexpr int planes_of(int k) { return CAR ? 8 : 4 * fp8_ndig(k); }
};

// LPV = 2 or 4 (stages with K <= 16 or K <= 8, NPAD = 32): every TMEM lane
// carries LPV DFT columns (lines) side by side, line h in slots
// [KS h, KS h + KS), KS = 32 / LPV, of the 32 element and output slots, with
// a block-diagonal constant matrix (the K x K matrix at rows and columns
// KS h).  The threads of quarter-warp group qd work on line qd / (4 / LPV),
// so every thread still deconstructs, reduces and finishes elements of one
// line only; a CTA covers 128 LPV lines.
// DBG: also write the stage's integers of the dumped columns to `dbg` (the
// column exponent, x~, the offset residues, the Phase-A accumulators, zhat and
// the centred R); the transform itself is unchanged.
template <int NPAD, int CAR, int LPV, bool DBG>
__global__ void __launch_bounds__(FP8_WARPS * 32, 1)
    stage_fp8_kernel(const uint8_t *__restrict__ planes, const uint8_t *__restrict__ pab,
                     const ModConsts *__restrict__ gmc, ColMapT map, int64_t ncols, int K, int Kout,
                     const double2 *__restrict__ in, double2 *__restrict__ out, int *status, int pf_ahead,
                     DebugDump dbg) {
    using CF = Fp8Cfg<NPAD>;
    using CC = CarrierCfg<NPAD, CAR>;
    constexpr int EPT = CF::EPT, OPT = CF::OPT, WPP = CF::WPP;
    constexpr int NSTEP = NMOD;  // one pipeline step per modulus
    extern __shared__ __align__(1024) uint8_t smem[];
    const ModConsts &mc = c_fp8_mc;
    __shared__ int colpart[4][128];
    // 0,1: B planes (TMA, per buffer), 2 (and 3 in the FP16 carrier): MMA,
    // 4: Phase-A B, 5: input tile
    __shared__ __align__(8) uint64_t mbar[6];
    // Phase-A accumulator slots: MMAs complete (one commit) / slot read and
    // preset again (one arrival per warp of the owning quarter-warp group)
    __shared__ __align__(8) uint64_t pa_full[PA_SLOTS], pa_empty[PA_SLOTS];
    __shared__ uint32_t tmem_holder;

    static_assert(NPAD == 32 && (LPV == 1 || LPV == 2 || LPV == 4), "32 slots per lane, 1, 2 or 4 lines");
    constexpr int QPL = 4 / LPV;           // quarter-warp groups per line
    constexpr int TILE = 128 * LPV;        // columns (lines) per CTA
    constexpr int KS = NPAD / LPV;         // slots of one line
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int sub = w & 3, qd = w >> 2;
    const int c = 32 * sub + lane;
    const int hl = qd / QPL;  // this thread's line within its lane
    const uint32_t lanebase = (uint32_t)(32 * sub) << 16;
    const int64_t cbase = (int64_t)blockIdx.x * TILE;
    const int64_t cg = cbase + 128 * hl + c;
    const bool cvalid = map.valid(cg, ncols);
    const int group = map.group(cbase);

    const uint32_t stage_rows = (uint32_t)Kout * 128;
    // The E4M3 carrier keeps 128 zero bytes after the staging (read, times zero
    // Phase-A rows, by the last row group's padded K chunk); the FP16 carrier
    // has the Phase-A constants there instead (finite FP16 values), in the
    // first constant buffer, loaded after the last modulus has used it.
    const uint32_t stage_bytes = (stage_rows >> 3) * PA_ROWB + (CAR ? 0 : 128);
    uint8_t *sStage = smem;
    uint8_t *sB0 = smem + ((stage_bytes + 1023) & ~1023u);
    constexpr uint32_t planeB = CC::PLANE_B;
    uint8_t *sPAB = CAR ? sB0 : sB0 + 2 * CC::BUF_PLANES * planeB;
    const uint8_t *gplanes = planes + (size_t)group * CC::PLANES_PER_GROUP * planeB;

    // The input tile is copied into the front of the Phase-A staging, which the
    // epilogues overwrite only after every thread has read its elements.
    // Set-up runs on several warps at once: warp 0 allocates tensor memory,
    // warp 1 initialises the barriers and issues the copies of the first
    // constants and (stage 1) of the input tile, warps 4..7 (stage 2) copy the
    // input tile's columns, and warp 2 (stage 1) prefetches the input of the
    // CTA one wave ahead into L2.  Stage 2 prefetches that tile later, by
    // plain per-thread prefetches after the deconstruction: its 128 columns
    // would take one bulk prefetch each, and those held the set-up for about
    // 5,000 cycles (the whole change: 4 % per stage pair).
    uint8_t *sIn = sStage;
    __shared__ int64_t s_e0;  // stage 1: first element of the input tile
    __shared__ int64_t s_pf_src0;  // stage 2: the tile one wave ahead (first column's element; valid columns)
    __shared__ int s_pf_nvalid;
    (void)gmc;
    // Thread 32 issues every bulk copy of constants (and, in stage 1, of the
    // input tile; stage 2's input copies come from warps 4..7 and complete on
    // the same barrier); on the failure path it waits (bounded) for the last
    // copy into each barrier before the CTA exits.  Kept in shared memory
    // (written and read by thread 32 only, so no registers are held through
    // the pipeline): the last modulus whose constants went into B buffer 0 /
    // 1, and whether the Phase-A constants were requested.
    __shared__ int pf_last[3];
    if (w == 0) {
        tmem_alloc(smem_u32(&tmem_holder), 512);
    } else if (w == 1) {
        const InputTile itile = input_tile(map, ncols, cbase, TILE);
        if (lane == 0) {
            pf_last[0] = pf_last[1] = -1;
            pf_last[2] = 0;
            s_e0 = itile.e0;
            for (int b = 0; b < 6; b++) mbar_init(smem_u32(&mbar[b]), 1);
            for (int b = 0; b < PA_SLOTS; b++) {
                mbar_init(smem_u32(&pa_full[b]), 1);
                mbar_init(smem_u32(&pa_empty[b]), 4);
            }
            if (map.stage == 2) mbar_expect_tx(smem_u32(&mbar[5]), (uint32_t)(itile.nvalid * K * 16));
            mbar_fence_init();
        }
        __syncwarp();
        if (map.stage == 1) copy_input_tile(itile, in, sIn, smem_u32(&mbar[5]), lane);
        else asm volatile("bar.arrive 1, 160;" ::: "memory");  // barriers ready for warps 4..7
        if (lane == 0) {
            if (!CAR) {
                mbar_expect_tx(smem_u32(&mbar[4]), PA_N * 64);
                tma_bulk_g2s(smem_u32(sPAB), pab, PA_N * 64, smem_u32(&mbar[4]));
                pf_last[2] = 1;
            }
            const uint32_t bytes0 = CC::planes_of(0) * planeB;
            mbar_expect_tx(smem_u32(&mbar[0]), bytes0);
            tma_bulk_g2s(smem_u32(sB0), gplanes, bytes0, smem_u32(&mbar[0]));
            pf_last[0] = 0;
        }
    } else if (w == 2) {
        // the tile about one wave of CTAs ahead, most likely next on some SM
        const int64_t nb = (int64_t)blockIdx.x + pf_ahead;
        const bool pf = pf_ahead > 0 && nb < (int64_t)gridDim.x;
        if (map.stage == 1 && pf) {
            prefetch_input_tile(input_tile(map, ncols, nb * TILE, TILE), in, lane);
        } else if (CAR && map.stage == 2 && lane == 0) {
            // stage 2 prefetches after the deconstruction (below)
            const InputTile pt = pf ? input_tile(map, ncols, nb * TILE, TILE) : InputTile{0, 0, 0, 0, 0};
            s_pf_src0 = pt.src0;
            s_pf_nvalid = pt.nvalid;
        }
    } else if (w == 3 && !CAR) {
        reinterpret_cast<uint32_t *>(sStage + stage_bytes - 128)[lane] = 0u;
    } else if (w >= 4 && w < 8 && map.stage == 2) {
        // stage 2: one bulk copy per column (K elements of one line, to row i
        // of stride (K + 1) x 16 bytes: the padding keeps the 16-byte reads of
        // a warp free of bank conflicts), issued by four warps once warp 1 has
        // set up the barrier (one warp alone took 1 % longer per stage)
        const InputTile itile = input_tile(map, ncols, cbase, TILE);
        asm volatile("bar.sync 1, 160;" ::: "memory");
        for (int i = 32 * (w - 4) + lane; i < itile.nvalid; i += 128)
            tma_bulk_g2s(smem_u32(sIn + (int64_t)i * (K + 1) * 16), in + itile.src0 + (int64_t)i * itile.n,
                         (uint32_t)(K * 16), smem_u32(&mbar[5]));
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_holder;
    // E4M3 classes 2..4 start at zero (issue_modulus_nm)
    if (!CAR)
#pragma unroll
    for (int cl = 2; cl < 5; cl++)
#pragma unroll
        for (int part = 0; part < 2; part++) {
            const uint32_t ta = tmem + lanebase + (uint32_t)(cl * 2 * NPAD + part * NPAD + qd * OPT);
            if constexpr (OPT == 8)
                tmem_st8_const(ta, 0u);
            else
                tmem_st4_const(ta, 0u);
        }
    // ---------------- deconstruction of this thread's EPT elements ----------------
    Pieces pR[EPT], pI[EPT];
    int e;
    int64_t ibase, istride, obase, ostride;
    map.strides(cg, ibase, istride, obase, ostride);
    // tfail: this thread saw a bounded wait give up (or, thread 0, an issue
    // fail); the CTA learns of it at the next __syncthreads_or, so every thread
    // leaves the pipeline at the same barrier
    bool tfail = false;
    {
        const bool okin = mbar_wait(smem_u32(&mbar[5]), 0, WAIT_LIMIT);
        tfail = !okin;
        // element j of this column at sIn + (sbase + j sstride) * 16
        const int64_t sbase = map.stage == 1 ? ibase - s_e0 : (int64_t)(128 * hl + c) * (K + 1);
        const int64_t sstride = map.stage == 1 ? istride : 1;
        uint64_t xb[EPT][2];
        int lead = LEAD_ZERO;
#pragma unroll
        for (int jj = 0; jj < EPT; jj++) {
            int j = EPT * qd + jj - KS * hl;
            double2 x = make_double2(0.0, 0.0);
            if (okin && cvalid && j < K)
                x = *reinterpret_cast<const double2 *>(sIn + (sbase + (int64_t)j * sstride) * 16);
            xb[jj][0] = (uint64_t)__double_as_longlong(x.x);
            xb[jj][1] = (uint64_t)__double_as_longlong(x.y);
            lead = max(lead, max(lead_exponent(xb[jj][0]), lead_exponent(xb[jj][1])));
        }
        colpart[qd][c] = lead;
        __syncthreads();
        int l2 = colpart[QPL * hl][c];
#pragma unroll
        for (int i = 1; i < QPL; i++) l2 = max(l2, colpart[QPL * hl + i][c]);
        e = l2 == LEAD_ZERO ? 0 : l2;
#pragma unroll
        for (int jj = 0; jj < EPT; jj++) {
            pR[jj] = scale_split(xb[jj][0], e);
            pI[jj] = scale_split(xb[jj][1], e);
        }
    }
    const int64_t drow = DBG && cvalid ? dbg.row(cg) : -1;
    if (DBG && drow >= 0) {
        if (qd == QPL * hl) dbg.e[drow] = e;
        auto xt_of = [](const Pieces &pc) {
            return (int64_t)(((uint64_t)pc.p2 << 40) | ((uint64_t)pc.p1 << 20) | (uint64_t)pc.p0) - (1ll << 55);
        };
#pragma unroll
        for (int jj = 0; jj < EPT; jj++) {
            const int j = EPT * qd + jj - KS * hl;
            if (j < K) {
                dbg.xt[(drow * K + j) * 2] = xt_of(pR[jj]);
                dbg.xt[(drow * K + j) * 2 + 1] = xt_of(pI[jj]);
            }
        }
    }
    uint16_t *const dres = DBG && drow >= 0 ? dbg.res + drow * (int64_t)K * 2 * NMOD : nullptr;

    // digits of x_R and x_I for modulus k into A buffer (k & 1)
    auto gen = [&](int k) {
        const uint32_t m = mc.m[k], mu = mc.barrett[k], c20 = mc.c20[k], c40 = mc.c40[k];
        const float2 nm2 = f2splat(-mc.fm[k]), im2 = f2splat(mc.finv[k]), off2 = f2splat(mc.foff[k]);
        float2 v[EPT];
#pragma unroll
        for (int jj = 0; jj < EPT; jj++) {
            // lazily reduced residues in [0, 2m) of x~ + 2^55; as floats minus 2^55 mod m
            // they lie in (-m, 2m), and one packed rounding step balances them exactly
            // (the quotients are below 3, far from FP32 rounding trouble)
            const uint32_t rR = residue_lazy(pR[jj], m, mu, c20, c40);
            const uint32_t rI = residue_lazy(pI[jj], m, mu, c20, c40);
            float2 f = make_float2(__uint_as_float(0x4B000000u | rR), __uint_as_float(0x4B000000u | rI));
            f = __fadd2_rn(f, off2);
            v[jj] = __ffma2_rn(nm2, rint2_mul(f, im2), f);  // balanced, [-m/2, m/2]
        }
        if constexpr (CAR) {
            // FP16 carrier: each balanced residue is one FP16 operand (|v| <= 1020);
            // K-packed two per TMEM column, x_R at the buffer start, x_I npad / 2 later
            uint32_t fR[EPT / 2], fI[EPT / 2];
#pragma unroll
            for (int i = 0; i < EPT / 2; i++) {
                fR[i] = f16x2(v[2 * i].x, v[2 * i + 1].x);
                fI[i] = f16x2(v[2 * i].y, v[2 * i + 1].y);
            }
            const uint32_t ta = tmem + lanebase + APL_BASE + (uint32_t)(k & 1) * CC::A_COLS + (uint32_t)(qd * EPT / 2);
            if constexpr (EPT / 2 == 4) {
                tmem_st4(ta, fR);
                tmem_st4(ta + NPAD / 2, fI);
            } else {
                tmem_st2(ta, fR[0], fR[1]);
                tmem_st2(ta + NPAD / 2, fI[0], fI[1]);
            }
            return;
        }
        uint32_t wR[3][WPP], wI[3][WPP];
        const int kind = fp8_kind(k);
        if (kind == KIND_SQ)
            digits_to_words2<KIND_SQ, EPT>(v, mc.fsq[k], wR, wI);
        else if (kind == KIND_B9)
            digits_to_words2<KIND_B9, EPT>(v, 0.f, wR, wI);
        else
            digits_to_words2<KIND_B11, EPT>(v, 0.f, wR, wI);
        const uint32_t ta = tmem + lanebase + APL_BASE + (uint32_t)(k & 1) * APL_COLS + (uint32_t)(qd * WPP);
        const int nd = fp8_ndig(k);
#pragma unroll
        for (int d = 0; d < 3; d++) {
            if (d < nd) {
                if constexpr (WPP == 2) {
                    tmem_st2(ta + d * 8, wR[d][0], wR[d][1]);
                    tmem_st2(ta + (3 + d) * 8, wI[d][0], wI[d][1]);
                } else {
                    tmem_st1(ta + d * 8, wR[d][0]);
                    tmem_st1(ta + (3 + d) * 8, wI[d][0]);
                }
            }
        }
    };
    // MMAs of modulus k, Re then Im part (thread 0 only).  Constant planes of
    // modulus k live in B buffer k & 1; B(k+1) is prefetched here, into the
    // buffer of modulus k-1, whose MMAs have completed.
    const uint64_t bdesc0 = smem_desc(smem_u32(sB0), 128, CC::SBO);
    const uint64_t bdesc1 = smem_desc(smem_u32(sB0 + CC::BUF_PLANES * planeB), 128, CC::SBO);
    // Copy of the constant planes of modulus k into B buffer k & 1, whose
    // previous contents (modulus k - 2) are no longer read by any MMA.
    auto prefetch_b = [&](int k) {
        const uint32_t bytes = CC::planes_of(k) * planeB;
        mbar_expect_tx(smem_u32(&mbar[k & 1]), bytes);
        tma_bulk_g2s(smem_u32(sB0 + (k & 1) * CC::BUF_PLANES * planeB), gplanes + (size_t)CC::plane_offset(k) * planeB,
                     bytes, smem_u32(&mbar[k & 1]));
        pf_last[k & 1] = k;
    };
    auto issue = [&](int k) -> bool {
        if (!mbar_wait(smem_u32(&mbar[k & 1]), (uint32_t)((k >> 1) & 1), WAIT_LIMIT)) return false;
        const uint64_t bd = (k & 1) ? bdesc1 : bdesc0;
        const uint32_t apl = tmem + APL_BASE + (uint32_t)(k & 1) * CC::A_COLS;
        const int kind = fp8_kind(k);
        if constexpr (CAR)
            issue_modulus_f16<NPAD>(tmem + f16_acc_col(k), apl, bd);
        else if (kind == KIND_SQ)
            issue_modulus_nm<KIND_SQ>(tmem, apl, bd, NPAD);
        else if (kind == KIND_B9)
            issue_modulus_nm<KIND_B9>(tmem, apl, bd, NPAD);
        else
            issue_modulus_nm<KIND_B11>(tmem, apl, bd, NPAD);
        tc_commit(smem_u32(&mbar[CAR ? 2 + (k & 1) : 2]));
        return true;
    };

    if (map.stage == 2) {
        // stage 2: the tile one wave of CTAs ahead into L2 by plain prefetches,
        // one 128-byte line per thread (one bulk prefetch per column would hold
        // the copy engine, and the set-up with it, for microseconds)
        // the target tile was found by warp 2 during set-up (FP16 carrier) or
        // is found here by every thread (E4M3: the set-up form measured 0.5 %
        // slower there, though it only touches stage 2, and 1.4 % faster with
        // the FP16 carrier)
        int64_t src0 = 0;
        int nvalid = 0;
        if constexpr (CAR) {
            src0 = s_pf_src0;
            nvalid = s_pf_nvalid;
        } else {
            const int64_t nb = (int64_t)blockIdx.x + pf_ahead;
            if (pf_ahead > 0 && nb < (int64_t)gridDim.x) {
                const InputTile pt = input_tile(map, ncols, nb * TILE, TILE);
                src0 = pt.src0;
                nvalid = pt.nvalid;
            }
        }
        const int lpr = (K * 16 + 127) / 128;
        for (int r = tid; r < nvalid * lpr; r += FP8_WARPS * 32) {
            const int i = r / lpr, q = r - i * lpr;
            asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const char *>(in + src0 + (int64_t)i * map.n) + q * 128));
        }
    }
    gen(0);
    tmem_wait_st();
    tc_fence_before();
    bool ok = __syncthreads_or(tfail) == 0;
    if (ok && tid == 0) {
        tc_fence_after();
        // a failed first issue reaches the CTA at the first __syncthreads_or
        // of either pipeline (every thread's MMA wait then gives up as well)
        if (!issue(0)) tfail = true;
    } else if (ok && tid == 32 && NMOD > 1) {
        prefetch_b(1);  // buffer 1 is unused so far
    }
    uint32_t mph[1] = {0u};  // next phase parity of the MMA barrier mbar[2]
    int last_issued = 0, last_waited = -1;  // FP16 carrier, thread 0: MMA batches in flight
    if constexpr (CAR) {
        // FP16 carrier: two accumulator sets.  The MMAs of modulus k+1 (set
        // (k+1) & 1, committed to mbar[2 + ((k+1) & 1)]) are issued as soon as
        // every thread has written its data residues, and run while the
        // epilogue of modulus k reads set k & 1.  The constant planes of
        // modulus k+2 (after the last modulus: the Phase-A constants) go into
        // the B buffer of modulus k once its MMAs have completed.  A failure
        // stays in the thread's own tfail until the step's __syncthreads_or
        // (a shared flag read after one barrier measured 0.6 % slower).
        for (int k = 0; k < NSTEP && ok; k++) {
            if (k + 1 < NMOD) gen(k + 1);
            tmem_wait_st();
            tc_fence_before();
            if (__syncthreads_or(tfail)) {  // residues of modulus k+1 written; epilogue k-1 done
                ok = false;
                break;
            }
            if (tid == 0 && k + 1 < NSTEP) {
                tc_fence_after();
                if (issue(k + 1)) last_issued = k + 1;
                else tfail = true;
            }
            const bool okm = mbar_wait(smem_u32(&mbar[2 + (k & 1)]), (uint32_t)((k >> 1) & 1), WAIT_LIMIT);
            tc_fence_after();
            if (!okm) {
                tfail = true;
                continue;
            }
            last_waited = k;
            if (tid == 32) {
                if (k + 2 < NSTEP) {
                    prefetch_b(k + 2);
                } else if (k + 2 == NSTEP) {
                    mbar_expect_tx(smem_u32(&mbar[4]), PA_N * 64);
                    tma_bulk_g2s(smem_u32(sPAB), pab, PA_N * 64, smem_u32(&mbar[4]));
                    pf_last[2] = 1;
                }
            }
            const uint32_t tre = tmem + lanebase + f16_acc_col(k) + (uint32_t)(qd * OPT);
            epilogue_modulus<KIND_F16, OPT>(tre, tre + NPAD, NPAD, mc, k, sStage, c, qd, Kout, dres, KS * hl, K);
        }
    } else {
        // A failure (an MMA wait or, in thread 0, issue() giving up) stays in
        // the thread's own tfail and reaches the CTA through the next
        // __syncthreads_or: no shared flag is written while other threads may
        // still read it behind the same barrier.
        for (int k = 0; k < NSTEP && ok; k++) {
            if (k + 1 < NMOD) gen(k + 1);  // digits of the next modulus while this one's MMAs run
            const bool okm = mbar_wait(smem_u32(&mbar[2]), mph[0], WAIT_LIMIT);
            mph[0] ^= 1u;
            tc_fence_after();
            if (okm) {
                const uint32_t tre = tmem + lanebase + (uint32_t)(qd * OPT);
                const int kind = fp8_kind(k);
                if (kind == KIND_SQ)
                    epilogue_modulus<KIND_SQ, OPT>(tre, tre + NPAD, NPAD, mc, k, sStage, c, qd, Kout, dres, KS * hl, K);
                else if (kind == KIND_B9)
                    epilogue_modulus<KIND_B9, OPT>(tre, tre + NPAD, NPAD, mc, k, sStage, c, qd, Kout, dres, KS * hl, K);
                else
                    epilogue_modulus<KIND_B11, OPT>(tre, tre + NPAD, NPAD, mc, k, sStage, c, qd, Kout, dres, KS * hl, K);
            } else {
                tfail = true;
            }
            tmem_wait_st();
            tc_fence_before();
            if (__syncthreads_or(tfail)) {
                ok = false;
                break;
            }
            // MMAs of modulus k+1 from thread 0; the constant planes of modulus k+2
            // from another warp, into the buffer of modulus k (its MMAs completed:
            // every thread waited for them before this barrier)
            if (tid == 0 && k + 1 < NSTEP) {
                tc_fence_after();
                if (!issue(k + 1)) tfail = true;
            } else if (tid == 32 && k + 2 < NSTEP) {
                prefetch_b(k + 2);
            }
        }
    }

    // ---------------- CRT Phase A on FP16 tensor cores, then Kulisch + lift + pack ----
    // Row block b (one output slot for the 128 columns, N = 48 accumulators)
    // belongs to quarter-warp group g = b & 3 (its four warps cover the 128
    // TMEM lanes), which owns PA_GSLOTS accumulator slots of 48 columns: its
    // i-th block b = g + 4 i accumulates in slot PA_GSLOTS g + i % PA_GSLOTS.
    // Accumulators start at 2^23 (the FP32 bit pattern of 2^23 + P is
    // 0x4B000000 + P).  After its four warps have read block b and preset the
    // slot again (the slot's empty barrier), the group's issuing warp issues the
    // MMAs of block b + 4 PA_GSLOTS into it; they run while the group finishes
    // block b.  No CTA barrier separates the blocks, and the groups never wait
    // for one another.
    const int nblk = Kout;
    // the MMAs of a group's blocks are issued by lane 0 of its warp with
    // sub == qd, so the four issuing warps sit on the four schedulers (warps
    // 0, 5, 10, 15; all on scheduler 0 measured 1.1 to 1.6 % slower)
    const bool leader = sub == qd && lane == 0;
    int pa_last = -1;                            // leader: last block whose MMAs it issued
    auto gslot = [&](int b) { return PA_GSLOTS * (b & 3) + ((b >> 2) % PA_GSLOTS); };
    auto preset = [&](int b) {
        const uint32_t ta = tmem + lanebase + (CAR ? PA_COL0 : 0u) + (uint32_t)(gslot(b) * PA_N);
        tmem_st16_const(ta, 0x4B000000u);
        tmem_st16_const(ta + 16, 0x4B000000u);
        tmem_st16_const(ta + 32, 0x4B000000u);
    };
    if (ok) {
        for (int i = 0; i < PA_GSLOTS && qd + 4 * i < nblk; i++) preset(qd + 4 * i);
        tmem_wait_st();
        tc_fence_before();
        fence_async_smem();
        const int bad = mbar_wait(smem_u32(&mbar[4]), 0, WAIT_LIMIT) ? 0 : 1;
        // uniform decision across the CTA (including a failed wait in the last
        // pipeline step)
        ok = __syncthreads_or(bad | (int)tfail) == 0;
    }
    if (ok) {
        const uint32_t idescA = instr_desc(128, PA_N, 0);
        const uint64_t adescA = smem_desc(smem_u32(sStage), 128, PA_ROWB);
        const uint64_t bdescA0 = smem_desc(smem_u32(sPAB), 128, 512), bdescA1 = smem_desc(smem_u32(sPAB) + 256, 128, 512);
        const uint32_t ebias[4] = {mc.kbias[0], mc.kbias[1], mc.kbias[2], mc.kbias[3]};
        const uint64_t zbias = ((uint64_t)mc.zbias[1] << 32) | mc.zbias[0];
        // output slot of row block b.  With LPV lines per lane, block b
        // belongs to line (b & 3) / QPL, so the thread that finishes the
        // blocks b = qd (mod 4) stays on its own line; every 8 consecutive
        // blocks cover 8 / LPV consecutive outputs of every line (LPV = 2:
        // blocks 0, 1, 4, 5 are outputs 0 .. 3 of line 0)
        auto kout_of = [&](int b) -> int {
            const int b0 = b & ~7, bi = b & 7;
            if constexpr (LPV == 1) return b;
            else if constexpr (LPV == 2) return KS * ((bi & 3) >> 1) + (b0 >> 1) + 2 * (bi >> 2) + (bi & 1);
            else return KS * (bi & 3) + (b0 >> 2) + (bi >> 2);
        };
        // the two K-chunk MMAs of block b into its slot, committed to the slot's full barrier
        auto issue_block = [&](int b) {
            tc_fence_after();
            // a row block's descriptor lies 16 x PA_ROWB bytes (in 16-byte
            // units) per output slot past the staging start
            const uint64_t ad = adescA + (uint64_t)((uint32_t)kout_of(b) * (16 * PA_ROWB / 16));
            const uint32_t d = tmem + (CAR ? PA_COL0 : 0u) + (uint32_t)(gslot(b) * PA_N);
            tc_mma_f16(d, ad, bdescA0, idescA, 1);
            tc_mma_f16(d, ad + 16, bdescA1, idescA, 1);  // + 256 bytes: K 16..31
            tc_commit(smem_u32(&pa_full[gslot(b)]));
            pa_last = b;
        };
        // the 42 used accumulator words of a row block: Re 0..20, Im 24..44
        // (loaded straight into the word array: Re words 0..20 from columns
        // 0..20, Im words 21..41 from columns 24..44)
        auto load_block = [&](int b, uint32_t (&wv)[42]) {
            const uint32_t ta = tmem + lanebase + (CAR ? PA_COL0 : 0u) + (uint32_t)(gslot(b) * PA_N);
            tmem_ld16(ta, *reinterpret_cast<uint32_t(*)[16]>(&wv[0]));
            tmem_ld4(ta + 16, *reinterpret_cast<uint32_t(*)[4]>(&wv[16]));
            tmem_ld1(ta + 20, wv[20]);
            tmem_ld16(ta + 24, *reinterpret_cast<uint32_t(*)[16]>(&wv[21]));
            tmem_ld4(ta + 40, *reinterpret_cast<uint32_t(*)[4]>(&wv[37]));
            tmem_ld1(ta + 44, wv[41]);
        };
        auto after_wait = [&](uint32_t (&wv)[42]) {
#pragma unroll
            for (int i = 0; i < 42; i++) asm volatile("" : "+r"(wv[i]));
        };
        auto finish = [&](const uint32_t (&wv)[42], int kout) {
            bool slow_re, slow_im, near_re, near_im;
            uint32_t Rre[4], Rim[4], zre = 0, zim = 0;
            double re = kulisch_pack_fp8_fast(wv, mc, e - 104, ebias, zbias, slow_re, Rre, near_re, DBG ? &zre : nullptr);
            double im = kulisch_pack_fp8_fast(wv + 21, mc, e - 104, ebias, zbias, slow_im, Rim, near_im,
                                              DBG ? &zim : nullptr);
            if (slow_re) re = kulisch_finish_slow(Rre[0], Rre[1], Rre[2], Rre[3], near_re, e - 104);
            if (slow_im) im = kulisch_finish_slow(Rim[0], Rim[1], Rim[2], Rim[3], near_im, e - 104);
            const int kl = kout - KS * hl;  // the output index within this thread's line
            if (cvalid && kl < (LPV == 1 ? Kout : K)) out[obase + (int64_t)kl * ostride] = make_double2(re, im);
            if (DBG && drow >= 0 && kl < K) {
                const int64_t o = drow * K + kl;
#pragma unroll
                for (int i = 0; i < 21; i++) {
                    dbg.acc[(o * 2 + 0) * 21 + i] = wv[i];
                    dbg.acc[(o * 2 + 1) * 21 + i] = wv[21 + i];
                }
                dbg.zhat[o * 2] = zre;
                dbg.zhat[o * 2 + 1] = zim;
                const uint32_t *Rw[2] = {Rre, Rim};
                const bool nr[2] = {near_re, near_im};
#pragma unroll
                for (int part = 0; part < 2; part++) {
                    // the centred value: the two-sided correction where the lift was near a boundary
                    const u128 r = (u128)lift_centre(Rw[part], nr[part], mc);
                    dbg.put_R128(drow, kl, part, (uint32_t)r, (uint32_t)(r >> 32), (uint32_t)(r >> 64), (uint32_t)(r >> 96));
                }
            }
        };
        if (leader)
            for (int i = 0; i < PA_GSLOTS && qd + 4 * i < nblk; i++) issue_block(qd + 4 * i);
        for (int i = 0, b = qd; b < nblk; i++, b += 4) {
            const int sl = gslot(b);
            const uint32_t use = (uint32_t)((i / PA_GSLOTS) & 1);  // phase parity of this use of the slot
            const bool okb = mbar_wait(smem_u32(&pa_full[sl]), use, WAIT_LIMIT);
            tc_fence_after();
            uint32_t wv[42];
            load_block(b, wv);
            tmem_wait_ld();
            after_wait(wv);
            const int bn = b + 4 * PA_GSLOTS;  // the group's next block in this slot
            if (bn < nblk) {
                preset(bn);
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&pa_empty[sl]));
                if (leader) {
                    if (mbar_wait(smem_u32(&pa_empty[sl]), use, WAIT_LIMIT)) issue_block(bn);
                    else tfail = true;
                }
            }
            if (!okb) {
                tfail = true;
                continue;
            }
            finish(wv, kout_of(b));
        }
        ok = __syncthreads_or((int)tfail) == 0;
    }
    if (!ok && tid == 0) {
        atomicExch(status, (int)OBFFT_ERR_TIMEOUT);
        // let in-flight MMAs and copies drain (bounded) before the TMEM is freed
        // and the CTA exits
        if constexpr (CAR) {
            // modulus MMA batches issued and not yet waited for by this thread
            for (int j = last_waited + 1; j <= last_issued; j++)
                mbar_wait(smem_u32(&mbar[2 + (j & 1)]), (uint32_t)((j >> 1) & 1), WAIT_LIMIT);
        }
        if (!CAR) mbar_wait(smem_u32(&mbar[2]), mph[0], WAIT_LIMIT);
    }
    if (!ok && tid == 32) {
        // copies into shared memory: the input tile, the Phase-A constants and
        // the last constant planes of each B buffer (an earlier copy into the
        // same buffer completed before the MMAs that preceded the later copy)
        mbar_wait(smem_u32(&mbar[5]), 0, WAIT_LIMIT);
        if (pf_last[2]) mbar_wait(smem_u32(&mbar[4]), 0, WAIT_LIMIT);
        for (int b = 0; b < 2; b++)
            if (pf_last[b] >= 0) mbar_wait(smem_u32(&mbar[b]), (uint32_t)((pf_last[b] >> 1) & 1), WAIT_LIMIT);
    }
    // Phase A on the failure path: each leader's last commit completes once
    // every MMA it issued has (the waits are bounded)
    if (!ok && leader && pa_last >= 0)
        mbar_wait(smem_u32(&pa_full[gslot(pa_last)]), (uint32_t)(((pa_last >> 2) / PA_GSLOTS) & 1), WAIT_LIMIT);
    tc_fence_before();
    __syncthreads();
    if (w == 0) tmem_dealloc(tmem, 512);
}

// Failure-path self-test: waits (bounded) on an mbarrier phase that nothing
// completes, then records OBFFT_ERR_TIMEOUT in the status word -- the same
// path a real stalled wait takes, exercised without faulting or hanging.
__global__ void bounded_wait_selftest_kernel(int *status, uint32_t limit) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        mbar_fence_init();
    }
    __syncthreads();
    const bool ok = mbar_wait(smem_u32(&bar), 0, limit);  // never arrives
    if (!ok && threadIdx.x == 0) atomicExch(status, (int)OBFFT_ERR_TIMEOUT);
}

cudaError_t launch_bounded_wait_selftest(int *status, cudaStream_t s) {
    bounded_wait_selftest_kernel<<<1, 32, 0, s>>>(status, 1u << 12);
    return cudaGetLastError();
}

cudaError_t fp8_upload_constants() {
    ModConsts mc;
    make_mod_consts(&mc);
    return cudaMemcpyToSymbol(c_fp8_mc, &mc, sizeof(mc));
}

int pick_lpv(const StageGeom &g, int stage, bool have_l2_planes, int nsm) {
    const int K = stage == 1 ? g.q : g.p;
    const int top = fp8_lines_per_lane(K);
    if (g.lpv == top || (g.lpv == 2 && top == 4 && have_l2_planes)) return g.lpv;
    if (top == 4 && have_l2_planes) {
        // columns of the launch with lpv lines per lane (stage 2 pads each k2 group)
        auto cols = [&](int lpv) {
            const int64_t tile = 128 * lpv, Lpad = (g.L + tile - 1) / tile * tile;
            return stage == 1 ? g.L * g.p : Lpad * g.q;
        };
        const int64_t b4 = (cols(4) + 511) / 512, b2 = (cols(2) + 255) / 256;
        if ((b2 + nsm - 1) / nsm <= (b4 + nsm - 1) / nsm) return 2;
    }
    return top;
}

size_t fp8_smem_bytes(int Kout, int npad) {
    size_t stage_bytes = (size_t)Kout * 128 / 8 * PA_ROWB + 128;
    return ((stage_bytes + 1023) & ~(size_t)1023) + 2 * FP8_BPLANES * (size_t)npad * 32 + PA_N * 64;
}
static size_t fp16_smem_bytes(int Kout, int npad) {
    size_t stage_bytes = (size_t)Kout * 128 / 8 * PA_ROWB;  // Phase-A constants live in B buffer 0
    return ((stage_bytes + 1023) & ~(size_t)1023) + 2 * 8 * (size_t)npad * npad * 2;
}

template <int CAR, int LPV, bool DBG>
static cudaError_t launch_one(int smem, unsigned blocks, cudaStream_t s, const uint8_t *planes, const void *pab,
                              const ColMapT &map, int64_t ncols, int K, int kslots, const double2 *in, double2 *out,
                              int *status, int nsm, const DebugDump &dbg) {
    cudaError_t err = cudaFuncSetAttribute(stage_fp8_kernel<32, CAR, LPV, DBG>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (err != cudaSuccess) return err;
    stage_fp8_kernel<32, CAR, LPV, DBG><<<blocks, FP8_WARPS * 32, smem, s>>>(
        planes, (const uint8_t *)pab, nullptr, map, ncols, K, kslots, in, out, status, nsm, dbg);
    return cudaGetLastError();
}

template <int CAR>
static cudaError_t launch_stage_carrier(const AxisTables &t, const void *pab, int *status, const StageGeom &g,
                                        int stage, const double2 *in, double2 *out, cudaStream_t s,
                                        const DebugDump *dbg) {
    const int K = stage == 1 ? g.q : g.p;
    if (K > 32) return cudaErrorInvalidValue;
    int dev = 0, nsm = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    err = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    // K <= 16 (K <= 8): two (four) lines per TMEM lane, 128 x lpv lines per
    // CTA, all 32 output slots through the staging and Phase A; the constant
    // planes are block-diagonal 32 x 32, built by the plan for
    // fp8_lines_per_lane(K) lines and, at K <= 8, also for two.  One CTA runs
    // per SM at a time: four lines are used only when they need fewer rounds
    // of CTAs than two (a small launch keeps more SMs busy with two).
    auto columns = [&](int lpv, int64_t &Lpad) {
        const int64_t tile = 128 * lpv;
        Lpad = (g.L + tile - 1) / tile * tile;
        return stage == 1 ? g.L * g.p : Lpad * g.q;
    };
    const void *planes_l2 = stage == 1 ? t.fp8_s1_l2 : t.fp8_s2_l2;
    const int lpv = pick_lpv(g, stage, planes_l2 != nullptr, nsm);
    const int tile = 128 * lpv;
    const int kslots = lpv > 1 ? 32 : K;
    ColMapT map;
    map.stage = stage;
    map.L = g.L;
    map.P = g.P;
    map.n = g.n;
    map.p = g.p;
    map.q = g.q;
    const int64_t ncols = columns(lpv, map.Lpad);
    const uint8_t *planes = (const uint8_t *)(lpv == 2 && fp8_lines_per_lane(K) == 4
                                                  ? planes_l2
                                                  : (stage == 1 ? t.fp8_s1 : t.fp8_s2));
    const size_t smem = CAR ? fp16_smem_bytes(kslots, 32) : fp8_smem_bytes(kslots, 32);
    int64_t blocks = (ncols + tile - 1) / tile;
    if (blocks == 0) return cudaSuccess;
    DebugDump d;
    if (dbg) {
        d = *dbg;
        d.Lpad = map.Lpad;
    }
    const unsigned nb = (unsigned)blocks;
    if (dbg) {
        if (lpv == 4) return launch_one<CAR, 4, true>((int)smem, nb, s, planes, pab, map, ncols, K, kslots, in, out, status, nsm, d);
        if (lpv == 2) return launch_one<CAR, 2, true>((int)smem, nb, s, planes, pab, map, ncols, K, kslots, in, out, status, nsm, d);
        return launch_one<CAR, 1, true>((int)smem, nb, s, planes, pab, map, ncols, K, kslots, in, out, status, nsm, d);
    }
    if (lpv == 4) return launch_one<CAR, 4, false>((int)smem, nb, s, planes, pab, map, ncols, K, kslots, in, out, status, nsm, d);
    if (lpv == 2) return launch_one<CAR, 2, false>((int)smem, nb, s, planes, pab, map, ncols, K, kslots, in, out, status, nsm, d);
    return launch_one<CAR, 1, false>((int)smem, nb, s, planes, pab, map, ncols, K, kslots, in, out, status, nsm, d);
}

cudaError_t launch_stage_fp8(const AxisTables &t, const ModConsts *dmc, const void *pab, int *status,
                             const StageGeom &g, int stage, const double2 *in, double2 *out, cudaStream_t s,
                             const DebugDump *dbg) {
    (void)dmc;
    return launch_stage_carrier<0>(t, pab, status, g, stage, in, out, s, dbg);
}

cudaError_t launch_stage_fp16(const AxisTables &t, const ModConsts *dmc, const void *pab, int *status,
                              const StageGeom &g, int stage, const double2 *in, double2 *out, cudaStream_t s,
                              const DebugDump *dbg) {
    (void)dmc;
    return launch_stage_carrier<1>(t, pab, status, g, stage, in, out, s, dbg);
}

}  // namespace obfft
