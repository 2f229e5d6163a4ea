// INT8-mode Bailey stage: Ozaki-II complex GEMM over independent columns with
// the per-modulus residue products on INT8 tensor cores (warp-level
// mma.sync.m16n8k32 s8 x s8 -> s32, exact integer accumulation), followed by
// the residue-domain Karatsuba combine, CRT and correctly rounded pack.
//
// Paper map: Algorithm 1 (one half: decompose -> per-modulus complex
// Karatsuba products -> combine -> tcCRT), INT8 substrate (Background, Ozaki
// Scheme II paragraph), two-limb residue split v = v0 + 256 v1 with
// v0 in [-128, 128), v1 in [0, 8] (Eq. h1-group), direct CRT with idempotents
// (Eq. fcrt) and the two-sided lift + pack (Algorithm 2).
//
// Residue products.  For modulus m, constant residues a_j and data residues
// b_j (both canonical): b_j = b0_j + 256 b1_j, and with G_j = a_j, H_j = 256 a_j
// mod m, sum_j a_j b_j = sum_j G_j b0_j + H_j b1_j (mod m).  G and H are split
// into limbs g0 + 256 g1 on the host, giving two K = 2*KPAD limb GEMMs whose
// int32 sums T_lo, T_hi combine as T_lo + 256 T_hi (|.| < 2^25): no rounding
// anywhere.  In this mode the CRT's E = sum_k v_k u_k is accumulated in
// registers (four 32-bit words of u_k, 64-bit partial sums) and the lift
// quotient is estimated in FP32 (error < 0.01 < 1/2, so the two-sided
// correction still lands on the unique centered value).
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "obfft_internal.h"

namespace obfft {

__device__ __forceinline__ void mma_s8(int (&c)[4], const uint4 &a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

struct ColMap {
    // element j of column c and output k of column c, for both stages
    int stage;
    int64_t L, Lpad, P;
    int n, p, q;
    __device__ __forceinline__ bool valid(int64_t c, int64_t ncols) const {
        if (c >= ncols) return false;
        if (stage == 2) return (c % Lpad) < L;
        return true;
    }
    __device__ __forceinline__ int64_t in_index(int64_t c, int j) const {
        if (stage == 1) {
            int64_t l = c / p, j1 = c % p;
            return l * n + j1 + (int64_t)p * j;
        }
        int64_t k2 = c / Lpad, l = c % Lpad;
        return l * n + k2 * p + j;
    }
    __device__ __forceinline__ int64_t out_index(int64_t c, int k) const {
        if (stage == 1) {
            int64_t l = c / p, j1 = c % p;
            return l * n + (int64_t)k * p + j1;
        }
        int64_t k2 = c / Lpad, l = c % Lpad;
        int64_t b = l / P, r = l % P;
        return (b * n + k2 + (int64_t)q * k) * P + r;
    }
    __device__ __forceinline__ int group(int64_t c) const { return stage == 1 ? 0 : (int)(c / Lpad); }
};

// smem layout of the data B fragments: [gi 4][mod 12][prod 3][kb KB][limb 2][lane 32] uint2.
// KPAD = 16 (K <= 16): the b0 and b1 limbs of the 16 elements share one k32
// block (k slots 0..15: G b0, 16..31: H b1), so each residue product is one
// limb GEMM block instead of two half-empty ones: [gi][mod][prod][lane] uint2
// holding (b0 word, b1 word).
// DBG: also write the stage's integers (column exponent, x~, D/E/F, the
// canonical residues v, zhat and R) of the dumped columns to `dbg`.
template <int KPAD, int MT, bool DBG>
__global__ void __launch_bounds__(128 * MT) stage_int8_kernel(const uint4 *__restrict__ table,
                                                              const ModConsts *__restrict__ gmc,
                                                              ColMap map, int64_t ncols, int K,
                                                              int Kout,
                                                              const double2 *__restrict__ in,
                                                              double2 *__restrict__ out, int64_t pf_cols,
                                                              DebugDump dbg) {
    constexpr bool PK = KPAD == 16;         // b0 and b1 limbs in one k32 block
    constexpr int KB = PK ? 1 : KPAD / 32;  // k32 blocks of data elements
    constexpr int KB2 = PK ? 1 : 2 * KB;    // limb GEMM blocks (b0 limbs then b1 limbs)
    constexpr int HN = PK ? 1 : 2;          // 16-element halves of a k32 block that hold data
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint2 *sB = reinterpret_cast<uint2 *>(smem_raw);
    __shared__ ModConsts mc;
    __shared__ int colexp[CT_COLS];
    __shared__ int64_t s_pf_src;  // stage 2: first element of the CTA one wave ahead (-1: none)
    __shared__ int s_pf_nv;       // and its valid columns

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gi = warp & 3, sub = warp >> 2;
    const int tig = lane & 3, grp = lane >> 2;
    const int64_t c0 = (int64_t)blockIdx.x * CT_COLS;

    for (int i = threadIdx.x; i < (int)(sizeof(ModConsts) / 4); i += blockDim.x)
        reinterpret_cast<uint32_t *>(&mc)[i] = reinterpret_cast<const uint32_t *>(gmc)[i];
    if (map.stage == 2 && threadIdx.x == 0) {
        const int64_t cn = c0 + pf_cols;
        s_pf_src = -1;
        if (pf_cols > 0 && cn < ncols) {
            const int64_t k2 = cn / map.Lpad, l0 = cn - k2 * map.Lpad;
            s_pf_src = l0 < map.L ? l0 * map.n + k2 * map.p : -1;
            s_pf_nv = (int)min((int64_t)CT_COLS, map.L - l0);
        }
    }
    if (map.stage == 1 && pf_cols > 0 && c0 + pf_cols < ncols) {
        // stage 1: the input of the CTA one wave ahead (whole lines, one
        // contiguous range) into L2, one 128-byte line per thread (6 % per
        // stage-1 launch).  Stage 2 prefetches after the set-up barrier, from
        // a target thread 0 found once (per-thread target arithmetic there
        // cost more than the prefetch saved).
        const int64_t cn = c0 + pf_cols;
        const int64_t e0 = (cn / map.p) * map.n;
        const int64_t e1 = (min(cn + CT_COLS - 1, ncols - 1) / map.p + 1) * map.n;
        for (int64_t off = (int64_t)threadIdx.x * 8; e0 + off < e1; off += (int64_t)blockDim.x * 8)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(in + e0 + off));
    }

    // ---------------- phase 1: deconstruct this lane's column elements -------------
    const int col_local = gi * 8 + grp;
    const int64_t c = c0 + col_local;
    const bool cvalid = map.valid(c, ncols);
    // elements owned: j = kb*32 + h*16 + 4*tig + i
    uint64_t xb[KB][2][4][2];
    int lead = LEAD_ZERO;
#pragma unroll
    for (int kb = 0; kb < KB; kb++)
#pragma unroll
        for (int h = 0; h < HN; h++)
#pragma unroll
            for (int i = 0; i < 4; i++) {
                int j = kb * 32 + h * 16 + 4 * tig + i;
                double2 x = make_double2(0.0, 0.0);
                if (cvalid && j < K) x = in[map.in_index(c, j)];
                uint64_t br = (uint64_t)__double_as_longlong(x.x), bi = (uint64_t)__double_as_longlong(x.y);
                xb[kb][h][i][0] = br;
                xb[kb][h][i][1] = bi;
                lead = max(lead, max(lead_exponent(br), lead_exponent(bi)));
            }
    lead = max(lead, __shfl_xor_sync(0xffffffffu, lead, 1));
    lead = max(lead, __shfl_xor_sync(0xffffffffu, lead, 2));
    const int e = lead == LEAD_ZERO ? 0 : lead;
    if (sub == 0 && tig == 0) colexp[col_local] = e;
    const int64_t drow = DBG && cvalid ? dbg.row(c) : -1;
    if (DBG && drow >= 0 && sub == 0 && tig == 0) dbg.e[drow] = e;
    __syncthreads();  // mc ready
    if (map.stage == 2 && s_pf_src >= 0) {
        // stage 2: the CTA one wave ahead (its columns' K-element pieces)
        const int lpr = (K * 16 + 127) / 128;
        for (int r = threadIdx.x; r < s_pf_nv * lpr; r += blockDim.x) {
            const int i = r / lpr, q = r - i * lpr;
            asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const char *>(in + s_pf_src + (int64_t)i * map.n) + q * 128));
        }
    }

#pragma unroll
    for (int kb = 0; kb < KB; kb++) {
        Pieces pr[2][4], pi[2][4];
#pragma unroll
        for (int h = 0; h < HN; h++)
#pragma unroll
            for (int i = 0; i < 4; i++) {
                int64_t a = scale_round(xb[kb][h][i][0], e);
                int64_t b = scale_round(xb[kb][h][i][1], e);
                if (DBG && drow >= 0 && sub == 0) {
                    const int j = kb * 32 + h * 16 + 4 * tig + i;
                    if (j < K) {
                        dbg.xt[(drow * K + j) * 2] = a;
                        dbg.xt[(drow * K + j) * 2 + 1] = b;
                    }
                }
                pr[h][i] = split_pieces(a);
                pi[h][i] = split_pieces(b);
            }
        for (int k = sub; k < NMOD; k += MT) {
            const uint32_t m = mc.m[k], mu = mc.barrett[k], c20 = mc.c20[k], c40 = mc.c40[k],
                           cn = mc.c55neg[k];
            uint32_t w[3][2][2] = {};  // [prod][limb][h]
#pragma unroll
            for (int h = 0; h < HN; h++) {
                uint32_t l0[3] = {0, 0, 0}, l1[3] = {0, 0, 0};
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    uint32_t rr = residue(pr[h][i], m, mu, c20, c40, cn);
                    uint32_t ri = residue(pi[h][i], m, mu, c20, c40, cn);
                    uint32_t rs = rr + ri;
                    rs = rs >= m ? rs - m : rs;
                    uint32_t r3[3] = {rr, ri, rs};
#pragma unroll
                    for (int pd = 0; pd < 3; pd++) {
                        l0[pd] |= (r3[pd] & 0xFFu) << (8 * i);          // v0 byte (two's complement)
                        l1[pd] |= ((r3[pd] + 128u) >> 8) << (8 * i);    // v1 in [0, 8]
                    }
                }
#pragma unroll
                for (int pd = 0; pd < 3; pd++) {
                    w[pd][0][h] = l0[pd];
                    w[pd][1][h] = l1[pd];
                }
            }
#pragma unroll
            for (int pd = 0; pd < 3; pd++) {
                if constexpr (PK) {
                    sB[((gi * NMOD + k) * 3 + pd) * 32 + lane] = make_uint2(w[pd][0][0], w[pd][1][0]);
                } else {
#pragma unroll
                    for (int limb = 0; limb < 2; limb++) {
                        int idx = ((((gi * NMOD + k) * 3 + pd) * KB + kb) * 2 + limb) * 32 + lane;
                        sB[idx] = make_uint2(w[pd][limb][0], w[pd][limb][1]);
                    }
                }
            }
        }
    }
    __syncthreads();

    // ---------------- phase 2: residue GEMMs, combine, CRT accumulation ------------
    const int mt = sub;
    const int64_t cw = c0 + gi * 8;  // first column of this warp's group
    const int g = map.valid(cw, ncols) ? map.group(cw) : 0;
    uint64_t accE[8][4];
    float zf[8];
#pragma unroll
    for (int o = 0; o < 8; o++) {
        zf[o] = 0.f;
#pragma unroll
        for (int w4 = 0; w4 < 4; w4++) accE[o][w4] = 0;
    }
    const size_t per_prod = (size_t)MT * 2 * KB2 * 32;  // uint4 entries per (mod, prod)
    for (int k = 0; k < NMOD; k++) {
        int T[3][4];
#pragma unroll
        for (int pd = 0; pd < 3; pd++) {
            int lo[4] = {0, 0, 0, 0}, hi[4] = {0, 0, 0, 0};
            const uint4 *tb = table + ((size_t)(g * NMOD + k) * 3 + pd) * per_prod +
                              (size_t)mt * 2 * KB2 * 32;
#pragma unroll
            for (int kb = 0; kb < KB2; kb++) {
                uint2 b = PK ? sB[((gi * NMOD + k) * 3 + pd) * 32 + lane]
                             : sB[((((gi * NMOD + k) * 3 + pd) * KB + (kb % KB)) * 2 + kb / KB) * 32 + lane];
                uint4 alo = __ldg(tb + (size_t)(0 * KB2 + kb) * 32 + lane);
                uint4 ahi = __ldg(tb + (size_t)(1 * KB2 + kb) * 32 + lane);
                mma_s8(lo, alo, b.x, b.y);
                mma_s8(hi, ahi, b.x, b.y);
            }
#pragma unroll
            for (int i = 0; i < 4; i++) T[pd][i] = lo[i] + (hi[i] << 8);
        }
        const uint32_t m = mc.m[k], mu = mc.barrett[k], off = mc.off27[k];
        const uint32_t u0 = mc.u32[k][0], u1 = mc.u32[k][1], u2 = mc.u32[k][2], u3 = mc.u32[k][3];
        const float ym = mc.yk_over_mk[k];
#pragma unroll
        for (int i = 0; i < 4; i++) {
            int32_t D = T[0][i], Ev = T[1][i], Fv = T[2][i];
            uint32_t vr = mod_signed27(D - Ev, m, mu, off);       // Re = D - E
            uint32_t vi = mod_signed27(Fv - D - Ev, m, mu, off);  // Im = F - D - E
            if constexpr (DBG) {
                const int kout = mt * 16 + grp + ((i >> 1) << 3);
                const int64_t cc = c0 + gi * 8 + 2 * tig + (i & 1);
                const int64_t d = map.valid(cc, ncols) ? dbg.row(cc) : -1;
                if (d >= 0 && kout < Kout) {
                    uint16_t *pd = dbg.def + ((d * Kout + kout) * NMOD + k) * 3;
                    pd[0] = (uint16_t)mod_signed27(D, m, mu, off);
                    pd[1] = (uint16_t)mod_signed27(Ev, m, mu, off);
                    pd[2] = (uint16_t)mod_signed27(Fv, m, mu, off);
                    dbg.res[((d * Kout + kout) * 2 + 0) * NMOD + k] = (uint16_t)vr;
                    dbg.res[((d * Kout + kout) * 2 + 1) * NMOD + k] = (uint16_t)vi;
                }
            }
            uint32_t vv[2] = {vr, vi};
#pragma unroll
            for (int part = 0; part < 2; part++) {
                int o = i * 2 + part;
                uint32_t v = vv[part];
                accE[o][0] += (uint64_t)v * u0;
                accE[o][1] += (uint64_t)v * u1;
                accE[o][2] += (uint64_t)v * u2;
                accE[o][3] += (uint64_t)v * u3;
                zf[o] = fmaf((float)v, ym, zf[o]);
            }
        }
    }

    // ---------------- finish: E, lift, pack, store ----------------------------------
#pragma unroll
    for (int i = 0; i < 4; i++) {
        int kout = mt * 16 + grp + ((i >> 1) << 3);
        int cl = gi * 8 + 2 * tig + (i & 1);
        int64_t cc = c0 + cl;
        if (kout >= Kout || !map.valid(cc, ncols)) continue;
        double res[2];
#pragma unroll
        for (int part = 0; part < 2; part++) {
            int o = i * 2 + part;
            u128 E = (u128)accE[o][0] + ((u128)accE[o][1] << 32) + ((u128)accE[o][2] << 64) +
                     ((u128)accE[o][3] << 96);
            int64_t zhat = (int64_t)__float2int_rn(zf[o]);
            i128 R = lift_two_sided(E, zhat, mc);
            res[part] = pack_rne(R, colexp[cl] - 104);
            if constexpr (DBG) {
                const int64_t d = dbg.row(cc);
                if (d >= 0) {
                    dbg.zhat[(d * Kout + kout) * 2 + part] = zhat;
                    const u128 ur = (u128)R;
                    dbg.put_R128(d, kout, part, (uint32_t)ur, (uint32_t)(ur >> 32), (uint32_t)(ur >> 64),
                                 (uint32_t)(ur >> 96));
                }
            }
        }
        out[map.out_index(cc, kout)] = make_double2(res[0], res[1]);
    }
}

template <int KPAD, int MT>
static cudaError_t launch_t(const AxisTables &t, const ModConsts *dmc, const ColMap &map,
                            int64_t ncols, int K, int Kout, const double2 *in, double2 *out,
                            cudaStream_t s, const DebugDump *dbg) {
    const void *table = map.stage == 1 ? t.int8_s1 : t.int8_s2;
    size_t smem = (size_t)4 * NMOD * 3 * (KPAD == 16 ? 1 : (KPAD / 32) * 2) * 32 * sizeof(uint2);
    auto kern = dbg ? stage_int8_kernel<KPAD, MT, true> : stage_int8_kernel<KPAD, MT, false>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int64_t blocks = (ncols + CT_COLS - 1) / CT_COLS;
    if (blocks == 0) return cudaSuccess;
    // columns one wave of CTAs ahead (resident CTAs per SM x SMs), for the
    // stage-1 L2 prefetch
    int dev = 0, nsm = 0, per_sm = 0;
    err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (err == cudaSuccess) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128 * MT, smem);
    if (err != cudaSuccess) return err;
    const int64_t pf_cols = (int64_t)nsm * per_sm * CT_COLS;
    DebugDump d;
    if (dbg) {
        d = *dbg;
        d.stage = map.stage;
        d.L = map.L;
        d.Lpad = map.Lpad;
    }
    kern<<<(unsigned)blocks, 128 * MT, smem, s>>>((const uint4 *)table, dmc, map, ncols, K, Kout, in, out, pf_cols,
                                                   d);
    return cudaGetLastError();
}

cudaError_t launch_stage_int8(const AxisTables &t, const ModConsts *dmc, const StageGeom &g,
                              int stage, const double2 *in, double2 *out, cudaStream_t s, const DebugDump *dbg) {
    ColMap map;
    map.stage = stage;
    map.L = g.L;
    map.Lpad = (g.L + 7) / 8 * 8;
    map.P = g.P;
    map.n = g.n;
    map.p = g.p;
    map.q = g.q;
    int K = stage == 1 ? g.q : g.p;
    int64_t ncols = stage == 1 ? g.L * g.p : map.Lpad * g.q;
    int MT = (K + 15) / 16;
    bool wide = K > 32;
    if (!wide) {
        if (MT == 1) return launch_t<16, 1>(t, dmc, map, ncols, K, K, in, out, s, dbg);
        return launch_t<32, 2>(t, dmc, map, ncols, K, K, in, out, s, dbg);
    }
    if (MT == 3) return launch_t<64, 3>(t, dmc, map, ncols, K, K, in, out, s, dbg);
    return launch_t<64, 4>(t, dmc, map, ncols, K, K, in, out, s, dbg);
}

}  // namespace obfft
