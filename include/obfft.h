/*
 * obfft.h -- C ABI of the GB300 Ozaki-Bailey FFT library (libobfft.so).
 *
 * The library computes full-FP64-accurate complex128 3-D FFTs as a Bailey
 * six-step transform whose DFT stages are Ozaki-Scheme-II residue GEMMs on
 * tensor cores (paper: "FP8 is All You Need (Part 2)", Algorithm 1), with the
 * exact CRT reconstruction (Eq. fcrt, Eq. slicing, Algorithm 2) and one
 * correctly rounded conversion per stage output.
 *
 * Conventions shared by every entry point
 *  - Transform (Bailey paragraph of the Background; the sign is this
 *    library's reading, the paper leaves it open):
 *      forward  (dir = -1): Y[k] = sum_j X[j] exp(-2 pi i sum_a j_a k_a / n_a)
 *      inverse  (dir = +1): the conjugate kernel, unnormalised (so the inverse
 *               is also the adjoint of the forward transform).
 *  - Layout: contiguous C-order [batch][n0][n1][n2] complex128, interleaved
 *    (re, im) doubles, 16-byte aligned; complex64 (interleaved floats, still
 *    16-byte aligned) for the FP32-precision modes OBFFT_MODE_FP32 and
 *    OBFFT_MODE_FP32_NATIVE.  Axis 2 is transformed first, then 1,
 *    then 0; each axis of length n = p * q uses the Bailey indices
 *    j = j1 + p j2, k = k2 + q k1 with 1 <= p, q <= 64.
 *  - Pointers passed to obfft_exec / obfft_exec_many are DEVICE pointers
 *    (cudaMalloc'd or torch CUDA tensors) on the plan's device; the caller
 *    owns them.  in == out is rejected (out-of-place only).
 *  - Errors are returned as obfft_status, never by aborting; a thread-local
 *    message is available from obfft_last_error().
 *  - obfft_exec is asynchronous on `stream`.  One plan must not run on two
 *    streams at the same time (it owns one scratch buffer).
 */
#ifndef OBFFT_H
#define OBFFT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct obfft_plan_s *obfft_plan; /* opaque, owned by the library */

typedef enum {
    OBFFT_OK = 0,
    OBFFT_ERR_ARG = 1,              /* bad pointer, size, direction or mode */
    OBFFT_ERR_UNSUPPORTED_SIZE = 2, /* an axis does not factor as p*q, p,q <= 64 */
    OBFFT_ERR_ALLOC = 3,            /* device or host allocation failed */
    OBFFT_ERR_CUDA = 4,             /* a CUDA call failed (message has details) */
    OBFFT_ERR_TIMEOUT = 5,          /* a device-side bounded wait gave up */
    OBFFT_ERR_INTERNAL = 6
} obfft_status;

typedef enum {
    /* residue GEMMs on tcgen05 FP8 E4M3 tensor cores (kind::f8f6f4), exact digit
       planes; Phase A on tcgen05 FP16 */
    OBFFT_MODE_FP8 = 0,
    /* residue GEMMs on INT8 tensor cores through warp-level mma.sync s8 x s8
       (the INT8 kind sm_103a accepts), two-limb residues */
    OBFFT_MODE_INT8 = 1,
    /* comparator: plain FP64 six-step FFT (radix butterflies + FP64 twiddles) */
    OBFFT_MODE_FP64_NATIVE = 2,
    /* residue GEMMs on tcgen05 FP16 tensor cores (kind::f16), the FP16-carrier
       variant: each balanced data residue is one FP16 operand (no digit split),
       each constant residue two FP16 digits c0 + 32 c1; Phase A as in FP8 mode */
    OBFFT_MODE_FP16 = 3,
    /* FP32-precision variant (Sec. "Ozaki-II for FP32"): complex64 in and out,
       24-bit significands, r = 6 moduli {2039, 2029, 2027, 1024, 961, 841},
       S = 8 byte slices, f = 24; residue GEMMs on tcgen05 FP16 tensor cores
       (FP16 carrier), Phase A on tcgen05 FP16, one correctly rounded binary32
       conversion per stage output.  Axis factors p, q <= 32. */
    OBFFT_MODE_FP32 = 4,
    /* comparator of the FP32 variant: plain FP32 six-step FFT on complex64 */
    OBFFT_MODE_FP32_NATIVE = 5
} obfft_mode;

/*
 * Create a plan for `batch` grids of n0 x n1 x n2 (each n_a >= 1, and each
 * n_a must factor as p*q with p, q <= 64, so n_a <= 4096).  Generates the
 * quantised DFT and twiddle-fused matrices (Eq. twiddle-fusion, constants
 * scaled by 2^52), their residue planes for the Rev-34 modulus set, the CRT
 * constants (u_k byte slices, w_k, M) and allocates one device scratch buffer
 * of the grid's size (paper: Algorithm 1 "Require" clause; Sec. tcgarner).
 * The plan is bound to the CUDA device current at creation.
 * Returns OBFFT_ERR_ARG for null `out` or non-positive sizes,
 * OBFFT_ERR_UNSUPPORTED_SIZE for an axis that does not factor, OBFFT_ERR_ALLOC
 * when device memory is short.
 */
obfft_status obfft_plan_create(obfft_plan *out, int64_t n0, int64_t n1, int64_t n2,
                               int64_t batch, int mode);

/*
 * Run the transform: in/out are device pointers to batch*n0*n1*n2 complex128
 * values (16-byte aligned, distinct buffers).  dir = -1 forward, +1 inverse.
 * `stream` is a cudaStream_t (0 = legacy default stream).  Asynchronous:
 * returns after enqueueing; kernel faults surface on a later synchronising
 * call.  OBFFT_ERR_ARG for null/aliased/misaligned pointers or a bad dir.
 */
obfft_status obfft_exec(obfft_plan p, const void *in, void *out, int dir, void *stream);

/* Release the plan's device tables and scratch.  NULL is accepted. */
obfft_status obfft_destroy(obfft_plan p);

/*
 * Splits chosen for one axis (0, 1 or 2) of grid `grid` (0 for single-grid
 * plans): n = (*p) * (*q).  The oracle takes them from here.
 */
obfft_status obfft_plan_get_splits(obfft_plan p, int grid, int axis, int *p_out, int *q_out);

/*
 * The choices a plan runs with for one axis of one grid: the Bailey split
 * n = p * q and, for the tcgen05 stage kernels (OBFFT_MODE_FP8, _FP16,
 * _FP32), the lines per TMEM lane of the stage-1 and stage-2 launches (1, 2
 * or 4 lines of up to 32, 16 or 8 elements side by side in each lane; 0 for
 * the other modes and length-1 axes).  Not part of the paper: multi-grid plans
 * choose both by timing at creation (see obfft_plan_create_many).
 */
obfft_status obfft_plan_get_tuning(obfft_plan p, int grid, int axis, int *p_out, int *q_out, int *lpv_stage1,
                                   int *lpv_stage2);

/*
 * Plan for `count` independent grids of possibly different sizes
 * (dims[g][0..2]) executed together (the uneven batch).  Same size rules as
 * obfft_plan_create.  Unless OBFFT_AUTOTUNE=0 is set in the environment, the
 * plan is tuned when it is created (OBFFT_AUTOTUNE=1 tunes one-grid plans
 * too): the split of each distinct axis length and, for the tcgen05 stage
 * kernels, the lines per TMEM lane of every stage with K <= 8 are chosen by
 * timing launches on this GPU (obfft_plan_get_tuning reports them; every
 * choice gives exact results for its split).  Grids of identical shape and
 * splits form a group that runs as one batched transform; the plan owns
 * device memory of about the total size of the grids, three times that for
 * grids that share their shape.
 */
obfft_status obfft_plan_create_many(obfft_plan *out, int count, const int64_t *dims /* [count][3] */,
                                    int mode);

/*
 * Transform every grid of a _many plan: ins[g] / outs[g] are device pointers
 * (arrays of `count` pointers in HOST memory).  Every output range must be
 * disjoint from every input range and from every other output range (inputs
 * may share memory); OBFFT_ERR_ARG otherwise.  Asynchronous on `stream`.
 * The work (per group: device-to-device gathers of the members, six batched
 * stage launches, scatters of the results) is captured once into a CUDA
 * graph per set of pointers and direction, and replayed by later calls.  The
 * groups are independent branches of the graph, so their launches can run
 * concurrently.
 */
obfft_status obfft_exec_many(obfft_plan p, const void *const *ins, void *const *outs, int dir,
                             void *stream);

/*
 * Run the axis passes first_axis, first_axis - 1, ..., last_axis of a
 * one-grid plan (2 >= first_axis >= last_axis >= 0; obfft_exec is (2, 0)).
 * Each pass transforms the lines of the contiguous axis (Bailey six-step,
 * Algorithm 1) and writes them rotated, [batch][A1][A2][n_axis] ->
 * [batch][n_axis][A1][A2], so the data layouts are: before the pass over
 * axis 2 (natural) [batch][n0][n1][n2]; before axis 1 [batch][n2][n0][n1];
 * before axis 0 [batch][n1][n2][n0]; after axis 0 [batch][n0][n1][n2].
 * `in` must hold the layout of the first pass.  Used by the slab
 * decomposition of one grid over several GPUs (local passes over axes 2 and
 * 1, an all-to-all exchange, then the pass over axis 0; the paper has no
 * multi-GPU design).  Same pointer rules and errors as obfft_exec.
 */
obfft_status obfft_exec_axes(obfft_plan p, int first_axis, int last_axis, const void *in, void *out, int dir,
                             void *stream);

/*
 * Device-to-device block transpose used around the all-to-all exchange of
 * the slab decomposition (not part of the paper): `src` holds `nblocks`
 * contiguous blocks of `rows` rows of `row_bytes` bytes; `dst` receives, for
 * each row r, the rows r of blocks 0 .. nblocks-1 side by side:
 *   dst[r][k][0 .. row_bytes) = src[k][r][0 .. row_bytes).
 * Device pointers, disjoint ranges; asynchronous on `stream`.  OBFFT_ERR_ARG
 * for NULL, equal or overlapping buffers or a bad geometry.
 */
obfft_status obfft_transpose_blocks(const void *src, void *dst, int64_t nblocks, int64_t rows, int64_t row_bytes,
                                    void *stream);

/*
 * Run ONE Bailey stage of ONE axis pass on the current contents of `in`
 * (debug / parity entry): stage 1 or 2 of the pass over axis `axis`.  `in`
 * holds the pass input laid out [batch][A1][A2][n_axis] (axis contiguous),
 * `out` receives:
 *   stage 1: Y'[line][k2][j1] (complex128, lines x n_axis)
 *   stage 2 (with in = the stage-1 output): the pass output, rotated to
 *            [batch][n_axis][A1][A2].
 * Grid sizes are those of the plan; A1, A2 are the other two axes in rotated
 * order (pass over axis 2: A1 = n0, A2 = n1; axis 1: A1 = n2, A2 = n0;
 * axis 0: A1 = n1, A2 = n2).
 */
obfft_status obfft_exec_stage(obfft_plan p, int axis, int stage, const void *in, void *out, int dir,
                              void *stream);

/*
 * Integer dump of one Bailey stage, for parity checks of every integer step
 * against an independent implementation (Algorithm 1, one half: the
 * deconstruction, the residue GEMMs, the combine; Algorithm 2: the CRT with
 * Phase A, the Kulisch sum and the two-sided lift).  Runs stage `stage` of
 * the pass over `axis` exactly as obfft_exec_stage (same output in `out`) and
 * writes, for the logical columns [col0, col0 + ncols) of that stage, the
 * stage's integers into the device buffer `dump` (zeroed first by the call).
 * A logical column is one length-K DFT input vector: stage 1, c = line * p +
 * j1 (K = q, elements j2); stage 2, c = k2 * L + line (K = p, elements j1),
 * L = lines of the pass.  K outputs per column.  Sections (byte offsets from
 * obfft_debug_layout; nm moduli: 12, or 6 for OBFFT_MODE_FP32):
 *   [0] int32  e[ncols]                   column exponent (x~ = RNE(x 2^(52 - e)),
 *                                          2^(23 - e) for OBFFT_MODE_FP32)
 *   [1] int64  xt[ncols][K][2]            x~ of each element (Re, Im)
 *   [2] uint16 def[ncols][K][nm][3]       INT8 mode: the residue products D, E,
 *                                          F mod m_k (Karatsuba, canonical);
 *                                          other modes: zero (real-form products)
 *   [3] uint16 res[ncols][K][2][nm]       the CRT operand of each output part and
 *                                          modulus: INT8 the canonical v_k; the
 *                                          tensor-core modes the offset residue
 *                                          r + 1024, r = v_k (mod m_k), |r| <= m_k/2 + 1
 *   [4] uint32 acc[ncols][K][2][na]       tensor-core modes: the Phase-A
 *                                          accumulators as FP32 bit patterns
 *                                          0x4B000000 + P_s (s < S) then + Q_t
 *                                          (t < F) of the offset residues (na =
 *                                          21, or 11 for OBFFT_MODE_FP32); INT8: zero
 *   [5] int64  zhat[ncols][K][2]          the lift quotient the kernel used
 *   [6] uint32 R[ncols][K][2][4]          the centred CRT value R (|R| < M/2), the
 *                                          integer the output is rounded from:
 *                                          128-bit two's complement, little-endian
 *                                          words
 * offsets[7] is the total size.  Native modes have no integer stages
 * (OBFFT_ERR_ARG).  Errors as obfft_exec_stage, plus OBFFT_ERR_ARG for
 * columns outside the stage.
 */
obfft_status obfft_debug_layout(int mode, int K, int Kout, int64_t ncols, int64_t *offsets /* [8] */);
obfft_status obfft_exec_debug(obfft_plan p, int axis, int stage, const void *in, void *out, int dir, int64_t col0,
                              int64_t ncols, void *dump, void *stream);

/*
 * Transform from host memory to host memory (one-grid plans): in and out are
 * host pointers to batch * n0 * n1 * n2 complex128 values in the layout of
 * obfft_exec (page-locked memory makes the copies asynchronous; pageable
 * memory works, with copies that block the host thread).  Not part of the
 * paper: the copies are overlapped with the transform.  The input is copied in
 * chunks of lines of the first axis pass (axis 2), each chunk transformed as
 * soon as it has arrived; the last pass (axis 0) runs in chunks of lines and
 * each chunk's output is copied back while the next one computes.  The plan
 * allocates two device buffers of the grid's size on the first call and keeps
 * them, with an internal copy stream and events, until obfft_destroy.  Work is
 * ordered after prior work on `stream` (a cudaStream_t, NULL = legacy default)
 * and the host output is complete once `stream` reaches the point after the
 * call.  Calls on one plan must not overlap in time on different streams
 * (they share the device buffers).  Errors: OBFFT_ERR_ARG (NULL pointers,
 * in == out, overlapping ranges, multi-grid plan, bad dir), OBFFT_ERR_ALLOC,
 * OBFFT_ERR_CUDA.
 */
obfft_status obfft_exec_host(obfft_plan p, const void *in, void *out, int dir, void *stream);

/*
 * Device status of the plan: synchronises `stream` (a cudaStream_t), reads the
 * plan's status word and returns OBFFT_ERR_TIMEOUT if a kernel's bounded wait
 * on a tensor-core completion or a TMA copy gave up since the last call (the
 * output of that transform is invalid), OBFFT_OK otherwise.  The word is reset.
 * Not part of the paper: the kernels' waits have iteration limits so that a
 * stalled wait ends with an error instead of hanging the GPU.
 */
obfft_status obfft_plan_status(obfft_plan p, void *stream);

/*
 * Exercise the failure path: launch a one-block kernel that waits, with a
 * short iteration limit, on an mbarrier phase nothing completes, and records
 * OBFFT_ERR_TIMEOUT in the plan's status word exactly as a stalled stage
 * kernel would.  Nothing faults or hangs; obfft_plan_status then reports it.
 */
obfft_status obfft_selftest_bounded_wait(obfft_plan p, void *stream);

/*
 * Host-only introspection (no GPU needed): the quantised constant
 * RNE(2^52 exp(dir 2 pi i m / N)) the plans use (Bailey paragraph and
 * Eq. twiddle-fusion: 53-bit signed significands, |re|, |im| <= 2^52), written
 * to *re, *im.  OBFFT_ERR_ARG for N < 1 or null outputs.
 */
obfft_status obfft_host_twiddle(int64_t m, int64_t N, int dir, int64_t *re, int64_t *im);

/*
 * Host-only introspection of the CRT constants (Eq. fcrt, Eq. slicing, and the
 * lift weights of Sec. "Exact Phase B"): moduli[12]; u_slices[12][15] = byte s
 * of u_k (little-endian); w_slices[12][6] = byte t of w_k = round(2^48 u_k / M);
 * M4[4] = M as little-endian 32-bit words.  Caller-owned host buffers.
 */
obfft_status obfft_host_crt_constants(uint32_t *moduli, uint8_t *u_slices, uint8_t *w_slices,
                                      uint32_t *M4);

/*
 * The same two introspection calls for the FP32-precision variant:
 * RNE(2^23 exp(dir 2 pi i m / N)) (24-bit signed significands), and
 * moduli[6], u_slices[6][8], w_slices[6][3] (w_k = round(2^24 u_k / M)) and M
 * (< 2^63).  Caller-owned host buffers; OBFFT_ERR_ARG for bad arguments.
 */
obfft_status obfft_host_twiddle32(int64_t m, int64_t N, int dir, int64_t *re, int64_t *im);
obfft_status obfft_host_crt_constants32(uint32_t *moduli, uint8_t *u_slices, uint8_t *w_slices, uint64_t *M);

/*
 * Epilogue ablation (the paper's width-parameterised Kulisch accumulator,
 * Sec. "The accumulator is substrate-agnostic", Sec. "INT16 and INT8",
 * Eq. kulisch-width; and the dp4a migration of the deconstruction bulk,
 * Sec. "Deconstruction count").  Exact alternative forms of two epilogue
 * parts, run stand-alone on device buffers so that their instruction mix and
 * throughput can be measured; every variant gives bit-identical results.
 *
 * obfft_ablation_phase_b: Phase B (Kulisch sum, two-sided lift, correctly
 * rounded pack) of scalar outputs.  acc: device uint32 [n_unique][21], the
 * Phase-A accumulators of one output as FP32 bit patterns 2^23 + P_s (s < 15)
 * then 2^23 + Q_t (t < 6), of offset residues r_k + 1024 (P_s, Q_t < 2^23);
 * et: device int32 [n_unique], the output is RNE(C 2^et) where C is the value
 * the residues encode.  variant: 0 = the stage kernels' path (four 64-bit
 * partial sums), 32 / 16 / 8 = deposits into words of that width (radix 2^28,
 * 2^12, 2^6), packed 32 / variant per register.
 * obfft_ablation_residues: canonical residues x~ mod m_k of the 12 moduli.
 * xt: device int64 [n_unique], |x~| < 2^53; variant 0 = the stage kernels'
 * 20/20/16-bit pieces with Barrett, 1 = dp4a over the bytes of x~ + 2^55,
 * 2 = 64-bit remainder, 3 = dp4a followed by the H0 reduction (fold-and-add
 * t -> (t >> a) c + (t mod 2^a) for the seven moduli m = 2^a - c with small c,
 * Barrett for the other five; the co-design ladder's rung H0).
 * Both: item i < n_total uses input i mod n_unique, computed `reps` times
 * (reps >= 1) with the input perturbed by the repetition index r (slice sum
 * P_0 + r, or x~ + r), so that a timing launch is bound by the arithmetic
 * rather than by loading inputs; the repetition-0 results of the first
 * n_unique items go to out (double [n_unique]) / res (uint16 [n_unique][12])
 * when those are non-NULL; *checksum (device uint64, caller-initialised) is
 * XOR-combined with a hash of every result.  Asynchronous on `stream`.
 * OBFFT_ERR_ARG for an unknown variant, n_unique < 1, n_total < 0, reps < 1
 * or NULL inputs.
 */
obfft_status obfft_ablation_phase_b(int variant, int64_t n_unique, int64_t n_total, int reps, const void *acc,
                                    const void *et, void *out, void *checksum, void *stream);
obfft_status obfft_ablation_residues(int variant, int64_t n_unique, int64_t n_total, int reps, const void *xt,
                                     void *res, void *checksum, void *stream);

/*
 * Largest grid (n0 * n1 * n2 complex128 values) obfft_exec_fp64_noalloc accepts.
 */
#define OBFFT_NOALLOC_MAX_ELEMS (1 << 21)

/*
 * Forward or inverse 3-D transform that allocates no memory (the paper has no
 * counterpart; this entry point exists for callers that are not allowed to
 * allocate device memory while they run -- code where cudaMalloc/cudaFree are
 * forbidden or where their implicit device synchronisation is unacceptable,
 * or applications that hand a library only the buffers it works on).
 *
 * It runs the native-FP64 six-step path (the kernels of OBFFT_MODE_FP64_NATIVE
 * plans with their default Bailey splits, so results are bit-identical to a
 * plan created without OBFFT_AUTOTUNE=1) on one n0 x n1 x n2 grid, with the stage-to-
 * stage scratch and the twiddle tables in device memory that the library
 * reserves at load time (file-scope device arrays, about 32 MiB per GPU that
 * loads the library, held until the process exits).  in/out: device pointers
 * to n0*n1*n2 complex128 values, 16-byte aligned, distinct.  dir = -1 forward,
 * +1 inverse (unnormalised).  stream: a cudaStream_t (0 = default stream).
 *
 * Limits and behaviour:
 *  - n0 * n1 * n2 <= OBFFT_NOALLOC_MAX_ELEMS, each axis p*q with p, q <= 64;
 *    larger or unfactorable grids return OBFFT_ERR_UNSUPPORTED_SIZE.
 *  - Calls no cudaMalloc, cudaFree or any allocating routine.  The first call
 *    on a device looks up the device addresses of the reserved arrays
 *    (cudaGetSymbolAddress, with that device current); with the CUDA driver's
 *    lazy module loading this first call is also when the driver places the
 *    arrays in device memory.  Make that first call during set-up; later calls
 *    leave free device memory unchanged.  The addresses are kept per device
 *    and CUDA context: after cudaDeviceReset the next call looks them up again.
 *  - Not for stream capture: every call uploads the twiddles of its three
 *    axes from a static pageable host table (a copy a captured graph could not
 *    replay with the right contents).
 *  - Every call on a device shares the same reserved arrays, which keep the
 *    last call's contents.  Nothing in them needs to start at zero (the scratch
 *    is fully written before it is read, the twiddles are rewritten by every
 *    call).  Calls whose work overlaps on the GPU (e.g. on two streams) race
 *    on these arrays and give wrong results: serialise them.
 *  - The twiddle upload is a host-to-device copy from pageable memory of
 *    the n + p + q entries each transformed axis uses.
 */
obfft_status obfft_exec_fp64_noalloc(const void *in, void *out, int64_t n0, int64_t n1, int64_t n2, int dir,
                                     void *stream);

/* Thread-local text of the last error (never NULL). */
const char *obfft_last_error(void);

/* Library version string. */
const char *obfft_version(void);

#ifdef __cplusplus
}
#endif
#endif /* OBFFT_H */
