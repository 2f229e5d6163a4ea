// Internal declarations shared by the library's host and device translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "obfft.h"

namespace obfft {

constexpr int NMOD = 12;     // r = 12 moduli (Rev-34 set)
constexpr int S_RAW = 15;    // byte slices of the CRT idempotents (Eq. slicing)
constexpr int S_FRAC = 6;    // byte slices of the 48-bit lift weights
constexpr int KMAX = 64;     // largest Bailey factor p or q
constexpr int CT_COLS = 32;  // columns per CTA of the INT8 stage kernel

// Rev-34 modulus set (Background, Ozaki Scheme II paragraph).
extern const int kModuli[NMOD];

// FP32-precision variant (Sec. "Ozaki-II for FP32"): six of the Rev-34 moduli
// (the subset with log2 M = 62.6), 8 byte slices of u_k, f = 24 (3 slices of w_k).
constexpr int NMOD32 = 6;
constexpr int S_RAW32 = 8;
constexpr int S_FRAC32 = 3;
extern const int kModuli32[NMOD32];

// Per-modulus constants used on the device (one copy in __constant__ memory).
// Offset added to the FP8 mode's reduced residues (|r| <= m/2 + 1) so that the
// FP16 CRT operands are non-negative: r + RES_OFFSET lies in [2, 2046].
constexpr int RES_OFFSET = 1024;

// FP8-mode constant digit planes per matrix group: per modulus 4 planes per
// digit (x_R half: a_R, a_I; x_I half: -a_I, a_R), 3 digits for the three
// 11-bit moduli and 2 for the other nine.
constexpr int FP8_PLANES_PER_GROUP = 4 * (3 * 3 + 9 * 2);
// FP16-carrier mode: per modulus 8 planes (2 halves x 2 constant digits x Re/Im rows)
constexpr int FP16_PLANES_PER_GROUP = 8 * 12;

struct ModConsts {
    uint32_t m[NMOD];         // moduli
    uint32_t barrett[NMOD];   // floor(2^32 / m)
    uint32_t off27[NMOD];     // smallest multiple of m >= 2^27 (makes |x| < 2^27 non-negative)
    uint32_t c20[NMOD];       // 2^20 mod m
    uint32_t c40[NMOD];       // 2^40 mod m
    uint32_t c55neg[NMOD];    // (-2^55) mod m : removes the +2^55 bias of deconstructed integers
    uint32_t u32[NMOD][4];    // u_k as four little-endian 32-bit words (u_k < M < 2^118)
    float yk_over_mk[NMOD];   // u_k / M = y_k / m_k rounded to float (lift quotient estimate)
    uint32_t M32[4];          // M
    uint32_t halfM32[4];      // M / 2 (M is even)
    uint8_t us[NMOD][S_RAW];  // byte slices of u_k (Phase A B-matrix)
    uint8_t ws[NMOD][S_FRAC]; // byte slices of w_k = round(2^48 u_k / M)
    // FP8-mode epilogue constants (exact small integers as floats)
    float fm[NMOD];    // m
    float finv[NMOD];  // 1/m rounded
    float foff[NMOD];  // -(2^23 + (2^55 mod m)): float bias of a lazily reduced data residue
    float fsq[NMOD];   // s for m = s^2, else 0
    float fc3[NMOD];   // 16^3 mod m
    float fc4[NMOD];   // 16^4 mod m
    // Kulisch deposit biases of the FP32-bit-pattern deposits:
    // sum_{s<15} 0x4B000000 * 256^s + RES_OFFSET mod 2^128 (the CRT of residues
    // r_k + RES_OFFSET lifts to C + RES_OFFSET, since sum_k u_k = 1 mod M) and
    // sum_{t<6} 0x4B000000 * 256^t mod 2^64
    uint32_t kbias[4];
    uint32_t zbias[2];
    // dp4a form of the deconstruction (epilogue ablation): the bytes of
    // 2^(8i) mod m, i < 7, low 8 bits (b8lo) and bits 8..10 (b8hi), packed four
    // per word: [0] = i 0..3, [1] = i 4..6
    uint32_t b8lo[NMOD][2];
    uint32_t b8hi[NMOD][2];
};

// Host-side constant generation (plan.cpp).
void make_mod_consts(ModConsts *mc);
// RNE(2^52 * cos / sin(2 pi m / N)) with the sign of the imaginary part
// chosen by dir (-1: exp(-i theta)); returns false on internal inconsistency.
void quantised_twiddle(int64_t m, int64_t N, int dir, int64_t *re, int64_t *im);
// The same at 2^sexp (sexp = 23: the FP32-precision variant's 24-bit significands).
void quantised_twiddle_scaled(int64_t m, int64_t N, int dir, int sexp, int64_t *re, int64_t *im);

// One axis of a grid: n = p * q.
struct AxisPlan {
    int n = 1, p = 1, q = 1;
};

// Device tables for one (n, p, q, dir, mode) axis.
struct AxisTables {
    int n = 0, p = 0, q = 0, dir = 0;
    // INT8 mode: fragment-native s8 limb tables, stage 1 (1 group) / stage 2 (q groups)
    void *int8_s1 = nullptr, *int8_s2 = nullptr;
    size_t int8_s1_bytes = 0, int8_s2_bytes = 0;
    // FP8 mode: E4M3 digit planes of the constant matrices, stage 1 / stage 2
    // (FP16-carrier and FP32 modes: their FP16 planes), laid out for
    // fp8_lines_per_lane(K) lines per TMEM lane; stages with K <= 8 also get
    // planes for two lines per lane (the launch picks the layout that needs
    // fewer rounds of CTAs)
    void *fp8_s1 = nullptr, *fp8_s2 = nullptr;
    void *fp8_s1_l2 = nullptr, *fp8_s2_l2 = nullptr;
    // native comparators: twiddles exp(dir 2 pi i m / n) for m < n, then the
    // q and p tables, as double pairs (FP64) or float pairs (FP32)
    void *tw = nullptr;
    // quantised int64 constants (kept for the FP8 path and for debugging)
    std::vector<int64_t> Fq, Fp;  // [q][q][2], [q][p][p][2]
};

struct GridDesc {
    int64_t n[3];
    AxisPlan ax[3];
    int lpv[3][2] = {{0, 0}, {0, 0}, {0, 0}};  // tuned lines per TMEM lane per axis and stage (0: default)
};

// Default Bailey split of an axis of length n: q = smallest divisor with
// q^2 >= n, p = n / q, both <= kmax; false when n does not factor that way.
bool choose_split(int64_t n, AxisPlan *a, int kmax = KMAX);

}  // namespace obfft

struct obfft_plan_s {
    int mode = 0;
    int device = 0;
    int64_t batch = 1;
    std::vector<obfft::GridDesc> grids;   // one for create, count for create_many
    std::vector<obfft::AxisTables> tables;  // one per distinct (n, dir)
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    obfft::ModConsts *d_consts = nullptr;
    void *d_pab = nullptr;     // Phase A B-matrix (FP16 u_k / w_k byte slices)
    int *d_status = nullptr;   // device status word (bounded-wait timeouts)
    // multi-grid execution: the whole launch sequence captured once per
    // (input pointers, output pointers, direction) and replayed as one graph
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t capture_stream = nullptr;
    std::vector<const void *> graph_ins;
    std::vector<void *> graph_outs;
    int graph_dir = 0;
    // multi-grid plans: grids of identical shape and splits run together as
    // one batched transform.  Group j lists its grid indices; a group of one
    // grid has only a scratch slice, a larger group also a gather buffer and a
    // result buffer (all offsets into `scratch`).
    std::vector<std::vector<int>> groups;
    std::vector<void *> group_in, group_out, group_scratch;
    // the groups' launch chains are captured on streams of their own, forked
    // from and joined back into the capture stream, so the graph runs them as
    // parallel branches (one stream and one join event per group)
    std::vector<cudaStream_t> group_streams;
    std::vector<cudaEvent_t> group_events;  // [0]: fork, [1 + j]: join of group j
    // host-to-host execution: two grid-sized device buffers, a copy stream and
    // its events, created on the first obfft_exec_host call
    void *host_io[2] = {nullptr, nullptr};
    cudaStream_t copy_stream = nullptr;
    std::vector<cudaEvent_t> copy_events;
};

namespace obfft {
// Integer dump of one Bailey stage (obfft_exec_debug): device pointers into the
// caller's buffer (sections as in include/obfft.h), written by the DBG
// instantiations of the stage kernels for the logical columns
// [col0, col0 + ncols).  Logical column: stage 1, c = line * p + j1 (the
// kernel's own column index); stage 2, c = k2 * L + line (the kernel pads
// each k2 group of columns to Lpad).
struct DebugDump {
    int32_t *e = nullptr;      // [ncols]                    column exponent
    int64_t *xt = nullptr;     // [ncols][K][2]              deconstructed integers (Re, Im)
    uint16_t *def = nullptr;   // [ncols][Kout][nmod][3]     INT8: D, E, F mod m_k (canonical)
    uint16_t *res = nullptr;   // [ncols][Kout][2][nmod]     the CRT operands (Re, Im)
    uint32_t *acc = nullptr;   // [ncols][Kout][2][nacc]     Phase-A accumulator words (FP32 bits)
    int64_t *zhat = nullptr;   // [ncols][Kout][2]           lift quotient
    uint32_t *R = nullptr;     // [ncols][Kout][2][4]        centred CRT value, 128-bit two's complement
    int64_t col0 = 0, ncols = 0;
    int K = 0, Kout = 0, nmod = 0, nacc = 0;
    int stage = 1;
    int64_t L = 0, Lpad = 0;
    // dump row of the kernel's column c, or -1 when c is not dumped
    __host__ __device__ __forceinline__ int64_t row(int64_t c) const {
        const int64_t lc = stage == 1 ? c : (c / Lpad) * L + (c % Lpad);
        const int64_t d = lc - col0;
        return (d >= 0 && d < ncols) ? d : -1;
    }
    __host__ __device__ __forceinline__ void put_R128(int64_t d, int k, int part, uint32_t r0, uint32_t r1,
                                                      uint32_t r2, uint32_t r3) const {
        uint32_t *p = R + ((d * Kout + k) * 2 + part) * 4;
        p[0] = r0; p[1] = r1; p[2] = r2; p[3] = r3;
    }
};

// error reporting
obfft_status set_error(obfft_status st, const std::string &msg);
AxisTables *get_tables(obfft_plan p, int n, int pp, int qq, int dir);

// Launchers (one CUDA translation unit each).
// Stage geometry: `lines` lines of length n = p*q per batch-slice structure.
struct StageGeom {
    int64_t L;       // total lines = batch * P
    int64_t P;       // lines per batch item (A1 * A2)
    int n, p, q;
    int lpv = 0;     // tcgen05 stage kernels: lines per TMEM lane (0: pick_lpv's default)
};
// Lines per TMEM lane of a tcgen05 stage launch (FP8, FP16-carrier and FP32
// modes): the caller's choice when valid (lpv <= fp8_lines_per_lane(K); two
// at K <= 8 needs the two-line planes), else fp8_lines_per_lane(K), with four
// lines only when they need fewer rounds of CTAs than two.
int pick_lpv(const StageGeom &g, int stage, bool have_l2_planes, int nsm);
cudaError_t launch_stage_int8(const AxisTables &t, const ModConsts *dmc, const StageGeom &g,
                              int stage, const double2 *in, double2 *out, cudaStream_t s,
                              const DebugDump *dbg = nullptr);
cudaError_t launch_stage_fp8(const AxisTables &t, const ModConsts *dmc, const void *pab, int *status,
                             const StageGeom &g, int stage, const double2 *in, double2 *out, cudaStream_t s,
                             const DebugDump *dbg = nullptr);
cudaError_t launch_stage_fp16(const AxisTables &t, const ModConsts *dmc, const void *pab, int *status,
                              const StageGeom &g, int stage, const double2 *in, double2 *out, cudaStream_t s,
                              const DebugDump *dbg = nullptr);
std::vector<uint8_t> build_fp16_planes(const std::vector<int64_t> &F, int groups, int K, const int *moduli,
                                       int nmod);
// FP32-precision variant
cudaError_t launch_stage_fp32(const AxisTables &t, const void *pab, int *status, const StageGeom &g, int stage,
                              const float2 *in, float2 *out, cudaStream_t s, const DebugDump *dbg = nullptr);
cudaError_t fp32_upload_constants();  // once per device, outside any stream capture
size_t fp32_smem_bytes(int Kout, int npad);
std::vector<uint8_t> build_phase_a_b32();
cudaError_t launch_stage_native32(const AxisTables &t, const StageGeom &g, int stage, const float2 *in,
                                  float2 *out, cudaStream_t s);
size_t fp8_smem_bytes(int Kout, int npad);
// Lines per TMEM lane of the tcgen05 stage kernel (FP8 and FP16-carrier
// modes) for a DFT of length K <= 32: the 32 element and output slots of a
// lane hold 4 lines of up to 8, 2 of up to 16, or 1 of up to 32.
inline int fp8_lines_per_lane(int K) { return K <= 8 ? 4 : (K <= 16 ? 2 : 1); }
cudaError_t fp8_upload_constants();  // once per device, outside any stream capture
cudaError_t launch_bounded_wait_selftest(int *status, cudaStream_t s);
std::vector<uint8_t> build_fp8_planes(const std::vector<int64_t> &F, int groups, int K);
std::vector<uint8_t> build_phase_a_b();
// Epilogue ablation kernels (ablation.cu)
cudaError_t launch_phase_b_ablation(int variant, int64_t n_unique, int64_t n_total, int reps, const uint32_t *acc,
                                    const int *et, double *out, unsigned long long *checksum, cudaStream_t s);
cudaError_t launch_residue_ablation(int variant, int64_t n_unique, int64_t n_total, int reps, const int64_t *xt,
                                    uint16_t *res, unsigned long long *checksum, cudaStream_t s);
cudaError_t launch_stage_fp64(const AxisTables &t, const StageGeom &g, int stage,
                              const double2 *in, double2 *out, cudaStream_t s);
}  // namespace obfft
