// FP32-precision Ozaki-Bailey stage on Blackwell tensor cores (tcgen05,
// sm_103a): the variant of Sec. "Ozaki-II for FP32".  Complex64 columns,
// 24-bit significands (constants RNE(2^23 omega), data x~ = RNE(x 2^(23-e))
// with one power of two per column), r = 6 moduli {2039, 2029, 2027, 1024,
// 961, 841} (log2 M = 62.6 against the 56-bit capacity budget at K = 32),
// S = 8 byte slices of u_k, f = 24 (three slices of w_k), one rounding to
// binary32 at the end.
//
// One CTA transforms 128 columns, 512 threads, the same organisation as the
// FP64-precision stage kernel's FP16 carrier: per modulus the balanced data
// residues (|v| <= 1020) go into tensor memory as FP16 (the A operand), the
// constant residues arrive by TMA as two FP16 digits a = c0 + 32 c1, four
// tcgen05.mma kind::f16 form the complex product in real form into two class
// accumulators, and the epilogue reduces c0 + 32 (c1 mod m) to an offset
// residue r + 1024 in [2, 2046] (FP16-exact) in the shared-memory Phase-A
// staging.  After the six moduli Phase A is one tcgen05.mma kind::f16 per
// row block (M = 128 outputs, N = 32 = Re/Im x (8 u-slices + 3 w-slices + 5
// zero), K = 16 = Re/Im x 6 residues + 4 zero), accumulators preset to 2^23.
// Phase B per output: E = sum_s P_s 256^s and the lift quotient zhat =
// round(2^-24 sum_t Q_t 256^t) (Algorithm 2); the lifted value is within 2^54
// of zero, so E - zhat M is formed modulo 2^64 and is exact as a signed
// 64-bit integer; the two-sided correction and the offset follow, then the
// correctly rounded pack to binary32 with gradual underflow.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "obfft_internal.h"
#include "tc_common.cuh"
#include "tc_stage.cuh"

namespace obfft {

constexpr int F32_WARPS = 16;
constexpr int PA32_N = 32;       // Phase A accumulator columns per row block (Re 16 | Im 16)
constexpr int PA32_ROWB = 256;   // bytes per 8-row group of the staging (2 K-chunks of 8 FP16)
constexpr int PA32_GSLOTS = 2;   // Phase-A accumulator slots per quarter-warp group (8 x 32 TMEM columns)
constexpr uint32_t WAIT_LIMIT32 = 1u << 22;

struct ModConsts32 {
    float fm[NMOD32];    // m
    float finv[NMOD32];  // 1/m rounded to FP32
    uint64_t M;          // prod m_k (< 2^63)
    int64_t halfM;       // M / 2 (M is even)
};
__constant__ ModConsts32 c_fp32_mc;

// ilogb(|x|) of a binary32 bit pattern, exact for subnormals; LEAD_ZERO for 0.
__device__ __forceinline__ int lead_exponent32(uint32_t bits) {
    const uint32_t a = bits & 0x7FFFFFFFu;
    if (a == 0) return LEAD_ZERO;
    const int E = (int)(a >> 23);
    return E ? E - 127 : (31 - __clz((int)a)) - 149;
}
// 2^n as a binary32, n in [-126, 127]
__device__ __forceinline__ float pow2f(int n) { return __uint_as_float((uint32_t)(n + 127) << 23); }

// x~ = RNE(x 2^(23 - e)) for both parts, as exact FP32 integers (|x~| < 2^24).
// The scaling is split so that each factor is a normal power of two; every
// product that can round to a non-zero integer is exact.
__device__ __forceinline__ float2 scale_round2(float2 x, int e) {
    const int s = 23 - e;  // e in [-149, 127]: s in [-104, 172]
    const int a = s < 127 ? s : 127;
    float2 y = __fmul2_rn(x, f2splat(pow2f(a)));
    if (s > a) y = __fmul2_rn(y, f2splat(pow2f(s - a)));
    return make_float2(rintf(y.x), rintf(y.y));
}

// Balanced residue of an exact FP32 integer |x| < 2^24 (both parts): the
// first quotient (RNE of the exact product with the rounded reciprocal) is
// within one of RNE(x / m), the second one balances exactly: |v| <= m / 2.
__device__ __forceinline__ float2 balanced_residue2(float2 x, float2 nm, float2 im) {
    const float2 v1 = __ffma2_rn(nm, rint2_mul(x, im), x);
    return __ffma2_rn(nm, rint2_mul(v1, im), v1);
}

// RNE(R 2^et) to binary32 with gradual underflow (quantum 2^-149); overflow
// gives infinity.  |R| < 2^63.
__device__ __forceinline__ float pack32_rne(int64_t R, int et) {
    if (R == 0) return 0.0f;
    const bool neg = R < 0;
    const uint64_t a = neg ? 0ull - (uint64_t)R : (uint64_t)R;
    const int L = 64 - __clzll((long long)a);
    int d = L - 24;                 // keep 24 significant bits
    if (-149 - et > d) d = -149 - et;  // and none below 2^-149
    uint64_t q = a;
    if (d > 0) {  // d <= 46 here (et >= -195)
        q = a >> d;
        const uint64_t rem = a & ((1ull << d) - 1ull), half = 1ull << (d - 1);
        if (rem > half || (rem == half && (q & 1ull))) q += 1ull;
    } else {
        d = 0;
    }
    // q <= 2^24 and q 2^(et + d) lies on the binary32 grid (or beyond its range)
    const int n = et + d;  // >= -149
    const int n1 = n > -126 ? n : -126;
    float f = __fmul_rn(__uint2float_rn((uint32_t)q), pow2f(n1));
    if (n < n1) f = __fmul_rn(f, pow2f(n - n1));
    return neg ? -f : f;
}

// Phase B of one output: 8 u-slice and 3 w-slice accumulators (FP32 bit
// patterns 2^23 + P), the lift, the offset and the pack.
// zhat_out / R_out (debug builds): the lift quotient and the centred value.
__device__ __forceinline__ float crt_pack32(const uint32_t *w, int et, uint64_t M, int64_t halfM,
                                            int64_t *zhat_out = nullptr, int64_t *R_out = nullptr) {
    // sum_s (bits - 0x4B000000) 256^s = sum_s bits 256^s - 0x4B000000 sum_s 256^s (mod 2^64)
    constexpr uint64_t EB = 0x4B000000ull * 0x0101010101010101ull;
    constexpr uint64_t ZB = 0x4B000000ull * 0x010101ull;
    uint64_t E = 0;
#pragma unroll
    for (int s = 0; s < 8; s++) E += (uint64_t)w[s] << (8 * s);
    E -= EB;
    const uint64_t z = (uint64_t)w[8] + ((uint64_t)w[9] << 8) + ((uint64_t)w[10] << 16) - ZB;
    const uint64_t zhat = (z + (1ull << 23)) >> 24;
    int64_t R = (int64_t)(E - zhat * M);
    if (R >= halfM) R -= (int64_t)M;
    if (R < -halfM) R += (int64_t)M;
    if (zhat_out) *zhat_out = (int64_t)zhat;
    if (R_out) *R_out = R - RES_OFFSET;
    return pack32_rne(R - RES_OFFSET, et);
}

// byte offset of element (row, k) of the Phase-A staging (K-major, 2 chunks of 8 FP16)
__device__ __forceinline__ uint32_t stage32_off(uint32_t row, uint32_t k) {
    return (row >> 3) * PA32_ROWB + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// Input tile of the columns [cb, cb + width) (element = 8 bytes): stage 1 one
// contiguous element range [e0, e1), stage 2 K elements per column at
// src0 + i n.  In shared memory stage-2 column i starts at i (K + 2) elements.
struct InputTile32 {
    int64_t e0, e1, src0, n;
    int nvalid;
};
__device__ __forceinline__ InputTile32 input_tile32(const ColMapT &map, int64_t ncols, int64_t cb, int width) {
    InputTile32 t;
    if (map.stage == 1) {
        const int64_t l0 = cb / map.p, l1 = min(cb + width - 1, ncols - 1) / map.p;
        t.e0 = l0 * map.n;
        t.e1 = (l1 + 1) * map.n;
        t.src0 = 0;
        t.n = 0;
        t.nvalid = 0;
    } else {
        const int64_t k2 = cb / map.Lpad, l0 = cb - k2 * map.Lpad;
        t.e0 = t.e1 = 0;
        t.src0 = l0 * map.n + k2 * map.p;
        t.n = map.n;
        t.nvalid = (int)max((int64_t)0, min((int64_t)width, map.L - l0));
    }
    return t;
}
// Stage 1: TMA bulk copies of the tile (warp-wide call).  Only used when
// every copy starts and ends on a 16-byte boundary (even n and K, 16-byte
// aligned input).
__device__ __forceinline__ void copy_input_tile32(const InputTile32 &t, const float2 *in, uint8_t *sIn, uint32_t mbar,
                                                  int lane) {
    if (lane == 0) mbar_expect_tx(mbar, (uint32_t)((t.e1 - t.e0) * 8));
    __syncwarp();
    const int64_t chunk = 4096;  // elements (32 KB, a whole tile) per copy
    for (int64_t e = t.e0 + (int64_t)lane * chunk; e < t.e1; e += 32 * chunk)
        tma_bulk_g2s(smem_u32(sIn + (e - t.e0) * 8), in + e, (uint32_t)(min(chunk, t.e1 - e) * 8), mbar);
}
// The same tile with plain 8-byte loads by all threads of the CTA.
__device__ __forceinline__ void load_input_tile32(const ColMapT &map, const InputTile32 &t, int K, const float2 *in,
                                                  uint8_t *sIn, int tid) {
    float2 *s = reinterpret_cast<float2 *>(sIn);
    if (map.stage == 1) {
        for (int64_t e = tid; e < t.e1 - t.e0; e += F32_WARPS * 32) s[e] = in[t.e0 + e];
    } else {
        for (int idx = tid; idx < t.nvalid * K; idx += F32_WARPS * 32) {
            const int i = idx / K, j = idx - i * K;
            s[i * (K + 2) + j] = in[t.src0 + (int64_t)i * t.n + j];
        }
    }
}
// Stage 1: L2 prefetch of an input tile (warp-wide call)
__device__ __forceinline__ void prefetch_input_tile32(const InputTile32 &t, const float2 *in, int lane) {
    const int64_t chunk = 4096;
    for (int64_t e = t.e0 + (int64_t)lane * chunk; e < t.e1; e += 32 * chunk)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(in + e), "r"((uint32_t)(min(chunk, t.e1 - e) * 8))
                     : "memory");
}

// ---------------------------------------------------------------------------
// Kernel.  Thread (sub = warp % 4, qd = warp / 4) owns TMEM lane c = 32 sub +
// lane (DFT column c of the tile), deconstructs elements [EPT qd, EPT qd +
// EPT) of that column and finishes outputs [OPT qd, OPT qd + OPT).
// TMEM (512 columns): two sets of class accumulators, set b at [4 b npad,
// 4 (b + 1) npad) (class cl, Re at 2 cl npad, Im npad later), so that the MMAs
// of modulus k+1 run while the epilogue of modulus k reads its set; FP16 A
// buffers of the data residues at 8 npad + b npad (x_R in the first npad / 2
// columns, x_I in the next); the eight Phase-A slots take [256, 512).
// LPV = 2 or 4 (K <= 16 or K <= 8, NPAD = 32): LPV lines per TMEM lane, as
// in the FP8 / FP16-carrier stage kernel: line h in slots [KS h, KS h + KS)
// with block-diagonal constants; quarter-warp group qd works on line
// qd / (4 / LPV) only; a CTA covers 128 LPV lines.
// ---------------------------------------------------------------------------
// DBG: also write the stage's integers of the dumped columns to `dbg`.
template <int NPAD, int LPV, bool DBG>
__global__ void __launch_bounds__(F32_WARPS * 32, 1)
    stage_fp32_kernel(const uint8_t *__restrict__ planes, const uint8_t *__restrict__ pab, ColMapT map,
                      int64_t ncols, int K, int Kout, const float2 *__restrict__ in, float2 *__restrict__ out,
                      int *status, int pf_ahead, int tma_in, DebugDump dbg) {
    constexpr int EPT = NPAD / 4, OPT = NPAD / 4;
    constexpr uint32_t PLANE_B = NPAD * NPAD * 2, BUF_PLANES = 8, SBO = 16 * NPAD;
    constexpr uint32_t ACC = 4 * NPAD;  // columns of one accumulator set (two classes, Re | Im)
    constexpr uint32_t APL = 2 * ACC;   // first A buffer, after the two accumulator sets
    // Phase-A slots from column 256 on (over the A buffers, whose last MMAs
    // have completed): they never overlap an accumulator set, which other
    // warps may still be reading when a warp presets its first slots
    constexpr uint32_t PA_COL0 = 2 * ACC;
    static_assert(PA_COL0 + 4 * PA32_GSLOTS * PA32_N <= 512, "the Phase-A slots within the 512 TMEM columns");
    extern __shared__ __align__(1024) uint8_t smem[];
    const ModConsts32 &mc = c_fp32_mc;
    __shared__ int colpart[4][128];
    // 0,1: B planes (TMA, per buffer), 2,3: MMAs of modulus k (per accumulator
    // set k & 1), 4: Phase-A B, 5: input tile
    __shared__ __align__(8) uint64_t mbar[6];
    // Phase-A slots: MMAs complete (one commit) / slot read and preset again
    // (one arrival per warp of the owning quarter-warp group)
    __shared__ __align__(8) uint64_t pa_full[4 * PA32_GSLOTS], pa_empty[4 * PA32_GSLOTS];
    __shared__ uint32_t tmem_holder;

    static_assert(LPV == 1 || (NPAD == 32 && (LPV == 2 || LPV == 4)), "1, 2 or 4 lines per lane");
    constexpr int QPL = 4 / LPV;      // quarter-warp groups per line
    constexpr int TILE = 128 * LPV;   // columns (lines) per CTA
    constexpr int KS = NPAD / LPV;    // slots of one line
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int sub = w & 3, qd = w >> 2;
    const int c = 32 * sub + lane;
    const int hl = qd / QPL;  // this thread's line within its lane
    const uint32_t lanebase = (uint32_t)(32 * sub) << 16;
    const int64_t cbase = (int64_t)blockIdx.x * TILE;
    const int64_t cg = cbase + 128 * hl + c;
    const bool cvalid = map.valid(cg, ncols);
    const int group = map.group(cbase);

    const uint32_t stage_bytes = ((uint32_t)Kout * 128 >> 3) * PA32_ROWB;
    uint8_t *sStage = smem;
    uint8_t *sB0 = smem + ((stage_bytes + 1023) & ~1023u);
    uint8_t *sPAB = sB0 + 2 * BUF_PLANES * PLANE_B;
    const uint8_t *gplanes = planes + (size_t)group * NMOD32 * BUF_PLANES * PLANE_B;
    uint8_t *sIn = sStage;  // the input tile sits in the staging until every thread has read it
    __shared__ int64_t s_e0;
    __shared__ int64_t s_pf_src0;  // stage 2: the tile one wave ahead (first column's element; valid columns)
    __shared__ int s_pf_nvalid;

    if (w == 0) {
        tmem_alloc(smem_u32(&tmem_holder), 512);
    } else if (w == 1) {
        const InputTile32 itile = input_tile32(map, ncols, cbase, TILE);
        if (lane == 0) {
            s_e0 = itile.e0;
            for (int b = 0; b < 6; b++) mbar_init(smem_u32(&mbar[b]), 1);
            for (int b = 0; b < 4 * PA32_GSLOTS; b++) {
                mbar_init(smem_u32(&pa_full[b]), 1);
                mbar_init(smem_u32(&pa_empty[b]), 4);
            }
            if (tma_in && map.stage == 2) mbar_expect_tx(smem_u32(&mbar[5]), (uint32_t)(itile.nvalid * K * 8));
            mbar_fence_init();
        }
        __syncwarp();
        if (tma_in && map.stage == 1) copy_input_tile32(itile, in, sIn, smem_u32(&mbar[5]), lane);
        if (tma_in && map.stage == 2) asm volatile("bar.arrive 1, 160;" ::: "memory");  // barriers ready for warps 4..7
        if (lane == 0) {
            mbar_expect_tx(smem_u32(&mbar[4]), PA32_N * 32);
            tma_bulk_g2s(smem_u32(sPAB), pab, PA32_N * 32, smem_u32(&mbar[4]));
            mbar_expect_tx(smem_u32(&mbar[0]), BUF_PLANES * PLANE_B);
            tma_bulk_g2s(smem_u32(sB0), gplanes, BUF_PLANES * PLANE_B, smem_u32(&mbar[0]));
        }
    } else if (w == 2) {
        const int64_t nb = (int64_t)blockIdx.x + pf_ahead;
        const bool pf = pf_ahead > 0 && nb < (int64_t)gridDim.x;
        if (tma_in && map.stage == 1 && pf) {
            prefetch_input_tile32(input_tile32(map, ncols, nb * TILE, TILE), in, lane);
        } else if (map.stage == 2 && lane == 0) {
            // stage 2 prefetches after the deconstruction (below)
            const InputTile32 pt = pf ? input_tile32(map, ncols, nb * TILE, TILE) : InputTile32{0, 0, 0, 0, 0};
            s_pf_src0 = pt.src0;
            s_pf_nvalid = pt.nvalid;
        }
    } else if (w >= 4 && w < 8 && tma_in && map.stage == 2) {
        // stage 2: one bulk copy per column (K elements of one line), issued
        // by four warps once warp 1 has set up the barrier (as in the FP8
        // stage kernel)
        const InputTile32 itile = input_tile32(map, ncols, cbase, TILE);
        asm volatile("bar.sync 1, 160;" ::: "memory");
        for (int i = 32 * (w - 4) + lane; i < itile.nvalid; i += 128)
            tma_bulk_g2s(smem_u32(sIn + (int64_t)i * (K + 2) * 8), in + itile.src0 + (int64_t)i * itile.n,
                         (uint32_t)(K * 8), smem_u32(&mbar[5]));
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_holder;
    if (!tma_in) {
        load_input_tile32(map, input_tile32(map, ncols, cbase, TILE), K, in, sIn, tid);
        __syncthreads();
    }

    bool bad = false;  // this thread saw a bounded wait give up
    // ---------------- deconstruction of this thread's EPT elements ----------------
    float2 xt[EPT];
    int e;
    int64_t ibase, istride, obase, ostride;
    map.strides(cg, ibase, istride, obase, ostride);
    {
        const bool okin = tma_in ? mbar_wait(smem_u32(&mbar[5]), 0, WAIT_LIMIT32) : true;
        if (!okin) bad = true;
        const int64_t sbase = map.stage == 1 ? ibase - s_e0 : (int64_t)(128 * hl + c) * (K + 2);
        const int64_t sstride = map.stage == 1 ? istride : 1;
        float2 x[EPT];
        int lead = LEAD_ZERO;
#pragma unroll
        for (int jj = 0; jj < EPT; jj++) {
            const int j = EPT * qd + jj - KS * hl;
            x[jj] = make_float2(0.f, 0.f);
            if (okin && cvalid && j < K) x[jj] = *reinterpret_cast<const float2 *>(sIn + (sbase + (int64_t)j * sstride) * 8);
            lead = max(lead, max(lead_exponent32(__float_as_uint(x[jj].x)), lead_exponent32(__float_as_uint(x[jj].y))));
        }
        colpart[qd][c] = lead;
        __syncthreads();
        int l2 = colpart[QPL * hl][c];
#pragma unroll
        for (int i = 1; i < QPL; i++) l2 = max(l2, colpart[QPL * hl + i][c]);
        e = l2 == LEAD_ZERO ? 0 : l2;
#pragma unroll
        for (int jj = 0; jj < EPT; jj++) xt[jj] = scale_round2(x[jj], e);
    }
    const int64_t drow = DBG && cvalid ? dbg.row(cg) : -1;
    if (DBG && drow >= 0) {
        if (qd == QPL * hl) dbg.e[drow] = e;
#pragma unroll
        for (int jj = 0; jj < EPT; jj++) {
            const int j = EPT * qd + jj - KS * hl;
            if (j < K) {
                dbg.xt[(drow * K + j) * 2] = (int64_t)xt[jj].x;
                dbg.xt[(drow * K + j) * 2 + 1] = (int64_t)xt[jj].y;
            }
        }
    }

    // FP16 residues of x_R and x_I for modulus k into A buffer (k & 1)
    auto gen = [&](int k) {
        const float2 nm2 = f2splat(-mc.fm[k]), im2 = f2splat(mc.finv[k]);
        uint32_t fR[EPT / 2], fI[EPT / 2];
#pragma unroll
        for (int i = 0; i < EPT / 2; i++) {
            const float2 a = balanced_residue2(xt[2 * i], nm2, im2);
            const float2 b = balanced_residue2(xt[2 * i + 1], nm2, im2);
            fR[i] = f16x2(a.x, b.x);
            fI[i] = f16x2(a.y, b.y);
        }
        const uint32_t ta = tmem + lanebase + APL + (uint32_t)(k & 1) * NPAD + (uint32_t)(qd * EPT / 2);
        if constexpr (EPT / 2 == 4) {
            tmem_st4(ta, fR);
            tmem_st4(ta + NPAD / 2, fI);
        } else {
            tmem_st2(ta, fR[0], fR[1]);
            tmem_st2(ta + NPAD / 2, fI[0], fI[1]);
        }
    };
    const uint64_t bdesc0 = smem_desc(smem_u32(sB0), 128, SBO);
    const uint64_t bdesc1 = smem_desc(smem_u32(sB0 + BUF_PLANES * PLANE_B), 128, SBO);
    auto prefetch_b = [&](int k) {
        mbar_expect_tx(smem_u32(&mbar[k & 1]), BUF_PLANES * PLANE_B);
        tma_bulk_g2s(smem_u32(sB0 + (k & 1) * BUF_PLANES * PLANE_B), gplanes + (size_t)k * BUF_PLANES * PLANE_B,
                     BUF_PLANES * PLANE_B, smem_u32(&mbar[k & 1]));
    };
    auto issue = [&](int k) -> bool {
        if (!mbar_wait(smem_u32(&mbar[k & 1]), (uint32_t)((k >> 1) & 1), WAIT_LIMIT32)) return false;
        issue_modulus_f16<NPAD>(tmem + (uint32_t)(k & 1) * ACC, tmem + APL + (uint32_t)(k & 1) * NPAD,
                                (k & 1) ? bdesc1 : bdesc0);
        tc_commit(smem_u32(&mbar[2 + (k & 1)]));
        return true;
    };
    // Epilogue of modulus k: both classes of the Re and Im products of this
    // thread's outputs -> offset residues, FP16, into the staging.
    auto epilogue = [&](int k) {
        const float2 nm2 = f2splat(-mc.fm[k]), im2 = f2splat(mc.finv[k]);
#pragma unroll
        for (int part = 0; part < 2; part++) {
            const uint32_t ta = tmem + lanebase + (uint32_t)(k & 1) * ACC + (uint32_t)(part * NPAD + qd * OPT);
            uint32_t r0[OPT], r1[OPT];
            if constexpr (OPT == 8) {
                tmem_ld8(ta, r0);
                tmem_ld8(ta + 2 * NPAD, r1);
            } else {
                tmem_ld4(ta, r0);
                tmem_ld4(ta + 2 * NPAD, r1);
            }
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < OPT; i++) asm volatile("" : "+r"(r0[i]), "+r"(r1[i]));
            const int kk = part == 0 ? k : NMOD32 + k;  // staging column: Re residues, then Im
            const uint32_t koff = (uint32_t)(kk >> 3) * 128 + (uint32_t)(kk & 7) * 2;
#pragma unroll
            for (int o2 = 0; o2 < OPT / 2; o2++) {
                // class 1 (|x| < 2^21) reduced first: c0 + 32 c1 could exceed 2^24
                const float2 c1 = make_float2(__uint_as_float(r1[2 * o2]), __uint_as_float(r1[2 * o2 + 1]));
                const float2 c0 = make_float2(__uint_as_float(r0[2 * o2]), __uint_as_float(r0[2 * o2 + 1]));
                const float2 red1 = __ffma2_rn(nm2, rint2_mul(c1, im2), c1);
                const float2 sum = __ffma2_rn(f2splat(32.0f), red1, c0);
                const float2 cv = offset_residue2(sum, nm2, im2);
                const uint32_t hv = f16x2(cv.x, cv.y);  // exact: offset residues in [2, 2046]
                const int k0 = qd * OPT + 2 * o2;
                if (DBG && drow >= 0) {
                    const float vv[2] = {cv.x, cv.y};
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        const int kl = k0 + h - KS * hl;
                        if (kl >= 0 && kl < K) dbg.res[((drow * K + kl) * 2 + part) * NMOD32 + k] = (uint16_t)vv[h];
                    }
                }
                if (k0 < Kout)
                    *reinterpret_cast<uint16_t *>(sStage + stage32_off((uint32_t)k0 * 128 + c, 0) + koff) =
                        (uint16_t)(hv & 0xFFFFu);
                if (k0 + 1 < Kout)
                    *reinterpret_cast<uint16_t *>(sStage + stage32_off((uint32_t)(k0 + 1) * 128 + c, 0) + koff) =
                        (uint16_t)(hv >> 16);
            }
        }
        if (k == NMOD32 - 1) {
            // K columns 12..15 of this thread's staging rows are read by Phase A
            // (times zero constants): they must hold finite values
#pragma unroll
            for (int o = 0; o < OPT; o++) {
                const int ko = qd * OPT + o;
                if (ko < Kout)
                    *reinterpret_cast<uint2 *>(sStage + stage32_off((uint32_t)ko * 128 + c, 12)) = make_uint2(0u, 0u);
            }
        }
    };

    // Pipeline: the MMAs of modulus k+1 (accumulator set (k+1) & 1) are issued
    // as soon as every thread has written its data residues, and run while the
    // epilogue of modulus k reads set k & 1.  The constant planes of modulus
    // k+2 go into the B buffer of modulus k once its MMAs have completed.
    // Failures (a bounded wait that gave up) are combined at each CTA barrier
    // (__syncthreads_or), so every thread leaves the loop at the same step.
    int last_issued = -1;    // thread 0: the last modulus whose MMAs it issued
    int last_waited = -1;    // the last modulus whose MMAs this thread waited for
    if (map.stage == 2) {
        // stage 2: the tile one wave of CTAs ahead into L2 by plain prefetches
        // after the deconstruction, one 128-byte line per thread (as in the
        // FP8 stage kernel)
        const int lpr = (K * 8 + 127) / 128;
        const int64_t src0 = s_pf_src0;
        for (int r = tid; r < s_pf_nvalid * lpr; r += F32_WARPS * 32) {
            const int i = r / lpr, q = r - i * lpr;
            asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const char *>(in + src0 + (int64_t)i * map.n) + q * 128));
        }
    }
    gen(0);
    tmem_wait_st();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
        tc_fence_after();
        if (issue(0)) last_issued = 0;
        else bad = true;
    } else if (tid == 32) {
        prefetch_b(1);
    }
    bool ok = true;
    for (int k = 0; k < NMOD32; k++) {
        if (k + 1 < NMOD32) gen(k + 1);
        tmem_wait_st();
        tc_fence_before();
        if (__syncthreads_or(bad)) {  // residues of modulus k+1 written; epilogue k-1 done
            ok = false;
            break;
        }
        if (tid == 0 && k + 1 < NMOD32) {
            tc_fence_after();
            if (issue(k + 1)) last_issued = k + 1;
            else bad = true;
        }
        const bool okm = mbar_wait(smem_u32(&mbar[2 + (k & 1)]), (uint32_t)((k >> 1) & 1), WAIT_LIMIT32);
        tc_fence_after();
        if (!okm) {
            bad = true;
            continue;
        }
        last_waited = k;
        if (tid == 32 && k + 2 < NMOD32) prefetch_b(k + 2);  // B buffer k & 1 is free again
        epilogue(k);
    }
    // ---------------- CRT Phase A (FP16 tensor cores), then Phase B + pack ----------------
    // As in the FP8 / FP16-carrier stage kernel: row block b (one output slot,
    // N = 32 accumulators) belongs to quarter-warp group g = b & 3, which owns
    // PA32_GSLOTS slots of 32 columns; its issuing warp (sub == qd, one per
    // scheduler) issues the MMA of block b + 4 PA32_GSLOTS into the slot of
    // block b once the group's four warps have read and preset it.
    const int nblk = Kout;
    const bool leader = sub == qd && lane == 0;
    int pa_last = -1;  // leader: last block whose MMA it issued
    auto gslot = [&](int b) { return PA32_GSLOTS * (b & 3) + ((b >> 2) % PA32_GSLOTS); };
    auto preset = [&](int b) {
        const uint32_t ta = tmem + lanebase + PA_COL0 + (uint32_t)(gslot(b) * PA32_N);
        tmem_st16_const(ta, 0x4B000000u);
        tmem_st16_const(ta + 16, 0x4B000000u);
    };
    if (ok) {
        for (int i = 0; i < PA32_GSLOTS && qd + 4 * i < nblk; i++) preset(qd + 4 * i);
        tmem_wait_st();
        tc_fence_before();
        fence_async_smem();
        const bool okp = mbar_wait(smem_u32(&mbar[4]), 0, WAIT_LIMIT32);
        ok = __syncthreads_or(bad || !okp) == 0;
    }
    if (ok) {
        const uint32_t idescA = instr_desc(128, PA32_N, 0);
        const uint64_t adescA = smem_desc(smem_u32(sStage), 128, PA32_ROWB);
        const uint64_t bdescA = smem_desc(smem_u32(sPAB), 128, 256);
        const uint64_t M = mc.M;
        const int64_t halfM = mc.halfM;
        // output slot of row block b (with LPV lines per lane, the thread
        // finishing the blocks b = qd (mod 4) stays on its own line; see the
        // FP8 stage kernel)
        auto kout_of = [&](int b) -> int {
            const int b0 = b & ~7, bi = b & 7;
            if constexpr (LPV == 1) return b;
            else if constexpr (LPV == 2) return KS * ((bi & 3) >> 1) + (b0 >> 1) + 2 * (bi >> 2) + (bi & 1);
            else return KS * (bi & 3) + (b0 >> 2) + (bi >> 2);
        };
        auto issue_block = [&](int b) {
            tc_fence_after();
            // a row block is 16 row groups: 16 x PA32_ROWB bytes per output slot
            const uint64_t ad = adescA + (uint64_t)((uint32_t)kout_of(b) * (16 * PA32_ROWB / 16));
            tc_mma_f16(tmem + PA_COL0 + (uint32_t)(gslot(b) * PA32_N), ad, bdescA, idescA, 1);
            tc_commit(smem_u32(&pa_full[gslot(b)]));
            pa_last = b;
        };
        if (leader)
            for (int i = 0; i < PA32_GSLOTS && qd + 4 * i < nblk; i++) issue_block(qd + 4 * i);
        for (int i = 0, b = qd; b < nblk; i++, b += 4) {
            const int sl = gslot(b);
            const uint32_t use = (uint32_t)((i / PA32_GSLOTS) & 1);  // phase parity of this use of the slot
            const bool okb = mbar_wait(smem_u32(&pa_full[sl]), use, WAIT_LIMIT32);
            tc_fence_after();
            const uint32_t ta = tmem + lanebase + PA_COL0 + (uint32_t)(sl * PA32_N);
            uint32_t a8[8], a4[4], b8[8], b4[4];
            tmem_ld8(ta, a8);
            tmem_ld4(ta + 8, a4);
            tmem_ld8(ta + 16, b8);
            tmem_ld4(ta + 24, b4);
            tmem_wait_ld();
            uint32_t wr[11], wi[11];
#pragma unroll
            for (int j = 0; j < 8; j++) {
                wr[j] = a8[j];
                wi[j] = b8[j];
            }
#pragma unroll
            for (int j = 0; j < 3; j++) {
                wr[8 + j] = a4[j];
                wi[8 + j] = b4[j];
            }
#pragma unroll
            for (int j = 0; j < 11; j++) asm volatile("" : "+r"(wr[j]), "+r"(wi[j]));
            const int bn = b + 4 * PA32_GSLOTS;  // the group's next block in this slot
            if (bn < nblk) {
                preset(bn);
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&pa_empty[sl]));
                if (leader) {
                    if (mbar_wait(smem_u32(&pa_empty[sl]), use, WAIT_LIMIT32)) issue_block(bn);
                    else bad = true;
                }
            }
            if (!okb) {
                bad = true;
                continue;
            }
            int64_t zr = 0, zi = 0, Rr = 0, Ri = 0;
            const float re = crt_pack32(wr, e - 46, M, halfM, DBG ? &zr : nullptr, DBG ? &Rr : nullptr);
            const float im = crt_pack32(wi, e - 46, M, halfM, DBG ? &zi : nullptr, DBG ? &Ri : nullptr);
            const int kl = kout_of(b) - KS * hl;  // output index within this thread's line
            if (cvalid && kl < K) out[obase + (int64_t)kl * ostride] = make_float2(re, im);
            if (DBG && drow >= 0 && kl < K) {
                const int64_t o = drow * K + kl;
#pragma unroll
                for (int j = 0; j < 11; j++) {
                    dbg.acc[(o * 2 + 0) * 11 + j] = wr[j];
                    dbg.acc[(o * 2 + 1) * 11 + j] = wi[j];
                }
                dbg.zhat[o * 2] = zr;
                dbg.zhat[o * 2 + 1] = zi;
                const uint32_t sr = (uint32_t)(Rr >> 63), si = (uint32_t)(Ri >> 63);
                dbg.put_R128(drow, kl, 0, (uint32_t)Rr, (uint32_t)((uint64_t)Rr >> 32), sr, sr);
                dbg.put_R128(drow, kl, 1, (uint32_t)Ri, (uint32_t)((uint64_t)Ri >> 32), si, si);
            }
        }
        ok = __syncthreads_or(bad) == 0;
    }
    if (!ok && tid == 0) {
        atomicExch(status, (int)OBFFT_ERR_TIMEOUT);
        // let this thread's in-flight MMAs and copies drain (bounded) before the
        // TMEM is freed and the CTA exits
        for (int j = last_waited + 1; j <= last_issued; j++)
            mbar_wait(smem_u32(&mbar[2 + (j & 1)]), (uint32_t)((j >> 1) & 1), WAIT_LIMIT32);
        if (tma_in) mbar_wait(smem_u32(&mbar[5]), 0, WAIT_LIMIT32);
        mbar_wait(smem_u32(&mbar[4]), 0, WAIT_LIMIT32);
    }
    // Phase A on the failure path: each leader's last commit completes once
    // every MMA it issued has (the waits are bounded)
    if (!ok && leader && pa_last >= 0)
        mbar_wait(smem_u32(&pa_full[gslot(pa_last)]), (uint32_t)(((pa_last >> 2) / PA32_GSLOTS) & 1), WAIT_LIMIT32);
    tc_fence_before();
    __syncthreads();
    if (w == 0) tmem_dealloc(tmem, 512);
}

cudaError_t fp32_upload_constants() {
    ModConsts32 mc;
    uint64_t M = 1;
    for (int k = 0; k < NMOD32; k++) M *= (uint64_t)kModuli32[k];
    for (int k = 0; k < NMOD32; k++) {
        mc.fm[k] = (float)kModuli32[k];
        mc.finv[k] = (float)(1.0 / (double)kModuli32[k]);
    }
    mc.M = M;
    mc.halfM = (int64_t)(M / 2);
    return cudaMemcpyToSymbol(c_fp32_mc, &mc, sizeof(mc));
}

size_t fp32_smem_bytes(int Kout, int npad) {
    const size_t stage_bytes = (size_t)Kout * 128 / 8 * PA32_ROWB;
    return ((stage_bytes + 1023) & ~(size_t)1023) + 2 * 8 * (size_t)npad * npad * 2 + PA32_N * 32;
}

template <int LPV, bool DBG>
static cudaError_t launch32(int smem, unsigned blocks, cudaStream_t s, const uint8_t *planes, const void *pab,
                            const ColMapT &map, int64_t ncols, int K, int kslots, const float2 *in, float2 *out,
                            int *status, int nsm, int tma_in, const DebugDump &dbg) {
    cudaError_t err =
        cudaFuncSetAttribute(stage_fp32_kernel<32, LPV, DBG>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (err != cudaSuccess) return err;
    stage_fp32_kernel<32, LPV, DBG><<<blocks, F32_WARPS * 32, smem, s>>>(planes, (const uint8_t *)pab, map, ncols, K,
                                                                        kslots, in, out, status, nsm, tma_in, dbg);
    return cudaGetLastError();
}

cudaError_t launch_stage_fp32(const AxisTables &t, const void *pab, int *status, const StageGeom &g, int stage,
                              const float2 *in, float2 *out, cudaStream_t s, const DebugDump *dbg) {
    const int K = stage == 1 ? g.q : g.p;
    if (K > 32) return cudaErrorInvalidValue;
    int dev = 0, nsm = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    err = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    // lines per TMEM lane, chosen as in the FP8 / FP16-carrier launcher: four
    // (K <= 8) only when they need fewer rounds of CTAs than two
    auto columns = [&](int lpv, int64_t &Lpad) {
        const int64_t tile = 128 * lpv;
        Lpad = (g.L + tile - 1) / tile * tile;
        return stage == 1 ? g.L * g.p : Lpad * g.q;
    };
    const void *planes_l2 = stage == 1 ? t.fp8_s1_l2 : t.fp8_s2_l2;
    const int lpv = pick_lpv(g, stage, planes_l2 != nullptr, nsm);
    const int tile = 128 * lpv, kslots = lpv > 1 ? 32 : K;
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
    const size_t smem = fp32_smem_bytes(kslots, 32);
    const int64_t blocks = (ncols + tile - 1) / tile;
    if (blocks == 0) return cudaSuccess;
    // TMA bulk copies of the input need 16-byte aligned starts and sizes: an
    // even line length (stage 1), even n and K (stage 2), aligned base
    const int tma_in = ((uintptr_t)in % 16 == 0) && (g.n % 2 == 0) && (stage == 1 || K % 2 == 0);
    DebugDump d;
    if (dbg) {
        d = *dbg;
        d.Lpad = map.Lpad;
    }
    const unsigned nb = (unsigned)blocks;
    const int sm = (int)smem;
    if (dbg) {
        if (lpv == 4) return launch32<4, true>(sm, nb, s, planes, pab, map, ncols, K, kslots, in, out, status, nsm, tma_in, d);
        if (lpv == 2) return launch32<2, true>(sm, nb, s, planes, pab, map, ncols, K, kslots, in, out, status, nsm, tma_in, d);
        return launch32<1, true>(sm, nb, s, planes, pab, map, ncols, K, kslots, in, out, status, nsm, tma_in, d);
    }
    if (lpv == 4) return launch32<4, false>(sm, nb, s, planes, pab, map, ncols, K, kslots, in, out, status, nsm, tma_in, d);
    if (lpv == 2) return launch32<2, false>(sm, nb, s, planes, pab, map, ncols, K, kslots, in, out, status, nsm, tma_in, d);
    return launch32<1, false>(sm, nb, s, planes, pab, map, ncols, K, kslots, in, out, status, nsm, tma_in, d);
}

}  // namespace obfft
