// Pieces shared by the tcgen05 Bailey stage kernels (E4M3 / FP16 carriers of
// the FP64-precision method and the FP32-precision variant): the column map
// of a stage, the offset residue of an exact class sum and the MMAs of one
// modulus in the FP16 carrier.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "obfft_internal.h"
#include "tc_common.cuh"

namespace obfft {

// Columns of one Bailey stage (Algorithm 1).  Stage 1: column c = (line l,
// j1) transforms the q elements j1 + p j2 of line l; stage 2: column c =
// (k2, line l) in groups of Lpad columns per k2 transforms the p elements
// k2 p + j1 of the stage-1 output and writes the pass output rotated.
struct ColMapT {
    int stage;
    int64_t L, Lpad, P;
    int n, p, q;
    __device__ __forceinline__ bool valid(int64_t c, int64_t ncols) const {
        if (c >= ncols) return false;
        if (stage == 2) return (c % Lpad) < L;
        return true;
    }
    __device__ __forceinline__ int group(int64_t c) const { return stage == 1 ? 0 : (int)(c / Lpad); }
    // element j of column c lives at ibase + j * istride; output k at obase + k * ostride
    __device__ __forceinline__ void strides(int64_t c, int64_t &ibase, int64_t &istride, int64_t &obase,
                                            int64_t &ostride) const {
        if (stage == 1) {
            int64_t l = c / p, j1 = c - l * p;
            ibase = l * n + j1;
            istride = p;
            obase = ibase;
            ostride = p;
        } else {
            int64_t k2 = c / Lpad, l = c - k2 * Lpad;
            int64_t b = l / P, r = l - b * P;
            ibase = l * n + k2 * p;
            istride = 1;
            obase = (b * n + k2) * P + r;
            ostride = (int64_t)q * P;
        }
    }
};

// Reduced residue plus RES_OFFSET of two exact integers |x| < 2^24 (packed):
// q = RNE(x / m) from the rounded reciprocal is within one of the true
// quotient, so x - m q lies in [-m/2 - 1, m/2 + 1] and the offset value in
// [2, 2046]: exact in FP16, non-negative for the biased Phase-A deposits.
__device__ __forceinline__ float2 offset_residue2(float2 x, float2 nm, float2 im) {
    const float2 q = rint2_mul(x, im);
    return __fadd2_rn(__ffma2_rn(nm, q, x), f2splat((float)RES_OFFSET));
}

// FP16 carrier: per half (x_R, x_I) and K chunk of 16 elements one
// tcgen05.mma kind::f16 (M = 128, N = 4 npad: digit c0 then c1, Re and Im rows
// side by side, K = 16) into the two class accumulators (class 1 at 2 npad).
template <int NPAD>
__device__ __forceinline__ void issue_modulus_f16(uint32_t dacc, uint32_t apl, uint64_t bdesc) {
    constexpr uint32_t planeB16 = NPAD * NPAD * 2 / 16;  // plane size in 16-byte descriptor units
#pragma unroll
    for (int h = 0; h < 2; h++)
#pragma unroll
        for (int kc = 0; kc < NPAD / 16; kc++)
            tc_mma_f16_ta(dacc, apl + (uint32_t)(h * NPAD / 2 + kc * 8),
                          bdesc + (uint64_t)(h * 4) * planeB16 + (uint64_t)(kc * 16), instr_desc(128, 4 * NPAD, 0),
                          (h == 0 && kc == 0) ? 0u : 1u);
}

}  // namespace obfft
