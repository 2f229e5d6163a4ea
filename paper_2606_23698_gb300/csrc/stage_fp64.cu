// Native Bailey stage (the comparator paths), in FP64 for complex128 and in
// FP32 for complex64: the same column maps as the Ozaki stages, with the
// length-K sub-DFT done as a Stockham FFT (radix 4 / 2 / 3 butterflies,
// generic small radix otherwise) and the inter-stage twiddle omega_N^(j1 k2)
// applied as a complex multiply on the stage-2 input (Bailey paragraph,
// steps 2-5; no Ozaki emulation).
#include <cuda_runtime.h>

#include "obfft_internal.h"

namespace obfft {

constexpr int FP64_COLS = 64;  // columns (threads) per CTA

struct ColMap64 {
    int stage;
    int64_t L, P;
    int n, p, q;
    __device__ __forceinline__ int64_t in_index(int64_t c, int j) const {
        if (stage == 1) {
            int64_t l = c / p, j1 = c % p;
            return l * n + j1 + (int64_t)p * j;
        }
        int64_t k2 = c / L, l = c % L;
        return l * n + k2 * p + j;
    }
    __device__ __forceinline__ int64_t out_index(int64_t c, int k) const {
        if (stage == 1) {
            int64_t l = c / p, j1 = c % p;
            return l * n + (int64_t)k * p + j1;
        }
        int64_t k2 = c / L, l = c % L;
        int64_t b = l / P, r = l % P;
        return (b * n + k2 + (int64_t)q * k) * P + r;
    }
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
template <typename T2>
__device__ __forceinline__ T2 cmake(decltype(T2::x) re, decltype(T2::x) im) {
    T2 v;
    v.x = re;
    v.y = im;
    return v;
}

// twK: exp(dir 2 pi i m / K) for m < K; twN: exp(dir 2 pi i m / n) for m < n
template <typename T2>
__global__ void __launch_bounds__(FP64_COLS) stage_native_kernel(ColMap64 map, int64_t ncols, int K, int dir,
                                                                 const T2 *__restrict__ twK,
                                                                 const T2 *__restrict__ twN,
                                                                 const T2 *__restrict__ in, T2 *__restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2 *bufA = reinterpret_cast<T2 *>(smem_raw);
    T2 *bufB = bufA + (size_t)FP64_COLS * K;
    const int t = threadIdx.x;
    const int64_t c = (int64_t)blockIdx.x * FP64_COLS + t;
    if (c >= ncols) return;
    // column-interleaved: element j of thread t at [j * FP64_COLS + t] (conflict-free)
    T2 *x = bufA, *y = bufB;
    int64_t k2 = map.stage == 2 ? c / map.L : 0;
    for (int j = 0; j < K; j++) {
        T2 v = in[map.in_index(c, j)];
        if (map.stage == 2) v = cmul(v, twN[(int)(((int64_t)j * k2) % map.n)]);
        x[j * FP64_COLS + t] = v;
    }
    // Stockham autosort passes
    int Ns = 1;
    int rem = K;
    while (rem > 1) {
        int R;
        if (rem % 4 == 0) R = 4;
        else if (rem % 2 == 0) R = 2;
        else if (rem % 3 == 0) R = 3;
        else {
            R = rem;
            for (int f = 5; f * f <= rem; f++)
                if (rem % f == 0) { R = f; break; }
        }
        const int stride = K / R;
        for (int j = 0; j < stride; j++) {
            const int jm = j % Ns;
            const int base = (j / Ns) * Ns * R + jm;
            const int tws = K / (Ns * R);
            if (R == 4) {
                T2 v0 = x[j * FP64_COLS + t], v1 = x[(j + stride) * FP64_COLS + t];
                T2 v2 = x[(j + 2 * stride) * FP64_COLS + t], v3 = x[(j + 3 * stride) * FP64_COLS + t];
                if (jm) {
                    v1 = cmul(v1, twK[(jm * tws) % K]);
                    v2 = cmul(v2, twK[(2 * jm * tws) % K]);
                    v3 = cmul(v3, twK[(3 * jm * tws) % K]);
                }
                T2 s02 = cadd(v0, v2), d02 = csub(v0, v2);
                T2 s13 = cadd(v1, v3), d13 = csub(v1, v3);
                // d13 * exp(dir i pi / 2) = d13 * (dir i)
                T2 rd13 = dir < 0 ? cmake<T2>(d13.y, -d13.x) : cmake<T2>(-d13.y, d13.x);
                y[(base) * FP64_COLS + t] = cadd(s02, s13);
                y[(base + Ns) * FP64_COLS + t] = cadd(d02, rd13);
                y[(base + 2 * Ns) * FP64_COLS + t] = csub(s02, s13);
                y[(base + 3 * Ns) * FP64_COLS + t] = csub(d02, rd13);
            } else if (R == 2) {
                T2 v0 = x[j * FP64_COLS + t], v1 = x[(j + stride) * FP64_COLS + t];
                if (jm) v1 = cmul(v1, twK[(jm * tws) % K]);
                y[(base) * FP64_COLS + t] = cadd(v0, v1);
                y[(base + Ns) * FP64_COLS + t] = csub(v0, v1);
            } else {
                T2 v[64];
                for (int r = 0; r < R; r++) {
                    T2 a = x[(j + r * stride) * FP64_COLS + t];
                    if (jm && r) a = cmul(a, twK[(r * jm * tws) % K]);
                    v[r] = a;
                }
                for (int s2 = 0; s2 < R; s2++) {
                    T2 acc = v[0];
                    for (int r = 1; r < R; r++) acc = cadd(acc, cmul(v[r], twK[((r * s2) % R) * (K / R)]));
                    y[(base + s2 * Ns) * FP64_COLS + t] = acc;
                }
            }
        }
        T2 *tmp = x;
        x = y;
        y = tmp;
        Ns *= R;
        rem /= R;
    }
    for (int k = 0; k < K; k++) out[map.out_index(c, k)] = x[k * FP64_COLS + t];
}

template <typename T2>
static cudaError_t launch_native(const AxisTables &t, const StageGeom &g, int stage, const T2 *in, T2 *out,
                                 cudaStream_t s) {
    ColMap64 map;
    map.stage = stage;
    map.L = g.L;
    map.P = g.P;
    map.n = g.n;
    map.p = g.p;
    map.q = g.q;
    int K = stage == 1 ? g.q : g.p;
    int64_t ncols = stage == 1 ? g.L * g.p : g.L * g.q;
    // twiddle tables: t.tw holds [n] entries of exp(dir 2 pi i m / n), then [q], then [p]
    const T2 *twN = reinterpret_cast<const T2 *>(t.tw);
    const T2 *twK = twN + g.n + (stage == 1 ? 0 : g.q);
    size_t smem = (size_t)2 * FP64_COLS * K * sizeof(T2);
    cudaError_t err = cudaFuncSetAttribute(stage_native_kernel<T2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int64_t blocks = (ncols + FP64_COLS - 1) / FP64_COLS;
    if (blocks == 0) return cudaSuccess;
    stage_native_kernel<T2><<<(unsigned)blocks, FP64_COLS, smem, s>>>(map, ncols, K, t.dir, twK, twN, in, out);
    return cudaGetLastError();
}

cudaError_t launch_stage_fp64(const AxisTables &t, const StageGeom &g, int stage, const double2 *in,
                              double2 *out, cudaStream_t s) {
    return launch_native<double2>(t, g, stage, in, out, s);
}

cudaError_t launch_stage_native32(const AxisTables &t, const StageGeom &g, int stage, const float2 *in,
                                  float2 *out, cudaStream_t s) {
    return launch_native<float2>(t, g, stage, in, out, s);
}

}  // namespace obfft
