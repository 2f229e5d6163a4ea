// Standalone measurement program (not part of libobfft.so): checks that
// tcgen05.mma kind::f16 and kind::f8f6f4 (E4M3) accumulate small-integer
// operands exactly in FP32 up to the magnitudes the Ozaki stages use, and
// measures the dense issue rate of both kinds on every SM (M = 128, N = 256,
// K = 32 bytes per instruction, back to back from one thread per CTA).
// Build and run on one GPU:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O2 -std=c++17 \
//        -o tcgen05_peak paper_2606_23698_gb300/probes/tcgen05_peak.cu && ./tcgen05_peak
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <vector>
#include <cmath>

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t make_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                 "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_f8(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                 "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}
__device__ __forceinline__ bool wait_parity(uint32_t mbar, uint32_t parity, long long limit) {
    uint32_t done = 0;
    for (long long it = 0; it < limit; it++) {
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

// A: [128][K] elements (esz bytes), B: [N][K]; D out: [128][N] float
// smem layout K-major no-swizzle: core (i = row/8, j = kbyte/16) at i*SBO + j*LBO, row%8 * 16 + kbyte%16
template <int ESZ>
__global__ void probe_kernel(const uint8_t *A, const uint8_t *B, float *D, int N, int K, int reps, int *err) {
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ uint32_t tmem_holder;
    __shared__ __align__(8) uint64_t mbar;
    const int KB = K * ESZ;                 // bytes per row
    const int LBO = 128, SBO = (KB / 16) * 128;
    uint8_t *sA = sm;
    uint8_t *sB = sm + 128 * KB;
    for (int i = threadIdx.x; i < 128 * KB; i += blockDim.x) {
        int r = i / KB, kb = i % KB;
        sA[(r / 8) * SBO + (kb / 16) * LBO + (r % 8) * 16 + kb % 16] = A[i];
    }
    for (int i = threadIdx.x; i < N * KB; i += blockDim.x) {
        int r = i / KB, kb = i % KB;
        sB[(r / 8) * SBO + (kb / 16) * LBO + (r % 8) * 16 + kb % 16] = B[i];
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                     "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    uint32_t tmem = tmem_holder;
    if (threadIdx.x == 0) {
        uint32_t idesc = (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
        const int kstep_bytes = 32;  // one MMA covers 32 bytes of K (16 f16 or 32 f8)
        for (int r = 0; r < reps; r++)
            for (int kk = 0; kk < KB / kstep_bytes; kk++) {
                uint64_t ad = make_desc(smem_u32(sA) + kk * 2 * LBO, LBO, SBO);
                uint64_t bd = make_desc(smem_u32(sB) + kk * 2 * LBO, LBO, SBO);
                if (ESZ == 2) mma_f16(tmem, ad, bd, idesc, (r | kk) ? 1u : 0u);
                else mma_f8(tmem, ad, bd, idesc, (r | kk) ? 1u : 0u);
            }
        commit(smem_u32(&mbar));
    }
    bool ok = wait_parity(smem_u32(&mbar), 0, 1ll << 26);
    if (!ok && threadIdx.x == 0) atomicExch(err, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (ok) {
        for (int c = 0; c < N; c += 8) {
            uint32_t v[8];
            uint32_t taddr = tmem + ((uint32_t)(32 * w) << 16) + c;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                           "=r"(v[7])
                         : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            for (int j = 0; j < 8; j++) D[(32 * w + lane) * N + c + j] = __uint_as_float(v[j]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
}

// rate: each CTA issues iters MMAs M=128,N=256,K=32B on garbage-free zero smem
template <int ESZ>
__global__ void rate_kernel(int iters, int *err) {
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ uint32_t tmem_holder;
    __shared__ __align__(8) uint64_t mbar;
    for (int i = threadIdx.x; i < (128 + 256) * 32 / 4; i += blockDim.x) ((uint32_t *)sm)[i] = 0x3c003c00u & (ESZ == 2 ? 0xffffffffu : 0x38383838u);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)), "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    uint32_t tmem = tmem_holder;
    if (threadIdx.x == 0) {
        const int N = 256;
        uint32_t idesc = (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
        uint64_t ad = make_desc(smem_u32(sm), 128, 256);
        uint64_t bd = make_desc(smem_u32(sm + 128 * 32), 128, 256);
        for (int i = 0; i < iters; i++) {
            if (ESZ == 2) mma_f16(tmem, ad, bd, idesc, 1u);
            else mma_f8(tmem, ad, bd, idesc, 1u);
        }
        commit(smem_u32(&mbar));
    }
    bool ok = wait_parity(smem_u32(&mbar), 0, 1ll << 30);
    if (!ok && threadIdx.x == 0) atomicExch(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
}

static uint16_t f2h(float f) {  // exact for small integers
    if (f == 0) return 0;
    uint32_t u; memcpy(&u, &f, 4);
    uint32_t s = (u >> 16) & 0x8000; int e = ((u >> 23) & 0xff) - 127 + 15; uint32_t m = (u >> 13) & 0x3ff;
    return (uint16_t)(s | (e << 10) | m);
}
static uint8_t f2e4m3(int v) {  // exact for |v| <= 16 or 4-sig-bit ints <= 448
    if (v == 0) return 0;
    uint8_t s = v < 0 ? 0x80 : 0; int a = abs(v);
    int e = 31 - __builtin_clz(a);  // floor log2
    int mant = (a << 3 >> e) & 7;   // 3 bits
    if ((((mant | 8) << e) >> 3) != a) { printf("not e4m3 exact %d\n", v); exit(1); }
    return s | ((e + 7) << 3) | mant;
}

int main() {
    int *derr; cudaMalloc(&derr, 4); cudaMemset(derr, 0, 4);
    srand(1);
    // ---- FP16 exactness: A in [0,2038] (K=12 + bias column), B in [0,255], K padded 32
    {
        const int K = 32, N = 48;
        std::vector<uint16_t> A(128 * K), B(N * K);
        std::vector<long long> Ai(128 * K), Bi(N * K);
        for (int r = 0; r < 128; r++) for (int k = 0; k < K; k++) {
            int v = k < 12 ? (r < 4 ? 2038 : rand() % 2039) : (k == 12 ? 2048 : 0);
            Ai[r * K + k] = v; A[r * K + k] = f2h((float)v);
        }
        for (int n = 0; n < N; n++) for (int k = 0; k < K; k++) {
            int v = k < 12 ? (n < 4 ? 255 : rand() % 256) : (k == 12 ? 4096 : 0);
            Bi[n * K + k] = v; B[n * K + k] = f2h((float)v);
        }
        uint8_t *dA, *dB; float *dD;
        cudaMalloc(&dA, A.size() * 2); cudaMalloc(&dB, B.size() * 2); cudaMalloc(&dD, 128 * N * 4);
        cudaMemcpy(dA, A.data(), A.size() * 2, cudaMemcpyHostToDevice);
        cudaMemcpy(dB, B.data(), B.size() * 2, cudaMemcpyHostToDevice);
        size_t smem = (128 + N) * K * 2;
        cudaFuncSetAttribute(probe_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        probe_kernel<2><<<1, 128, smem>>>(dA, dB, dD, N, K, 1, derr);
        cudaError_t e = cudaDeviceSynchronize();
        int herr; cudaMemcpy(&herr, derr, 4, cudaMemcpyDeviceToHost);
        std::vector<float> D(128 * N); cudaMemcpy(D.data(), dD, D.size() * 4, cudaMemcpyDeviceToHost);
        long long bad = 0, maxv = 0;
        for (int r = 0; r < 128; r++) for (int n = 0; n < N; n++) {
            long long s = 0; for (int k = 0; k < K; k++) s += Ai[r * K + k] * Bi[n * K + k];
            maxv = s > maxv ? s : maxv;
            if ((long long)D[r * N + n] != s || D[r * N + n] != (float)s) { if (bad < 5) printf("f16 mismatch r%d n%d got %.1f want %lld\n", r, n, D[r*N+n], s); bad++; }
            uint32_t bits; memcpy(&bits, &D[r * N + n], 4);
            if (r == 5 && n == 7) printf("f16 sample bits 0x%08x value %lld\n", bits, s);
        }
        printf("F16 probe: cuda=%s timeout=%d mismatches=%lld max=%lld\n", cudaGetErrorString(e), herr, bad, maxv);
    }
    // ---- FP8 exactness: digits in [-16,16], K = 32*KBLK, reps to push magnitudes
    for (int trial = 0; trial < 4; trial++) {
        const int KBLK = trial == 3 ? 8 : 2, K = 32 * KBLK, N = 32;
        const int reps = trial == 0 ? 1 : trial == 1 ? 8 : trial == 2 ? 64 : 16;
        std::vector<uint8_t> A(128 * K), B(N * K);
        std::vector<long long> Ai(128 * K), Bi(N * K);
        for (int r = 0; r < 128; r++) for (int k = 0; k < K; k++) {
            int v = r < 8 ? 16 : (r < 16 ? -16 : (rand() % 33) - 16);
            if (trial >= 2 && r >= 16 && r < 24) v = (k % 2) ? 16 : -16;
            Ai[r * K + k] = v; A[r * K + k] = f2e4m3(v);
        }
        for (int n = 0; n < N; n++) for (int k = 0; k < K; k++) {
            int v = n < 4 ? 16 : (rand() % 33) - 16;
            if (trial >= 2 && n >= 4 && n < 8) v = 1;
            Bi[n * K + k] = v; B[n * K + k] = f2e4m3(v);
        }
        uint8_t *dA, *dB; float *dD;
        cudaMalloc(&dA, A.size()); cudaMalloc(&dB, B.size()); cudaMalloc(&dD, 128 * N * 4);
        cudaMemcpy(dA, A.data(), A.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(dB, B.data(), B.size(), cudaMemcpyHostToDevice);
        size_t smem = (128 + N) * K;
        cudaFuncSetAttribute(probe_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        probe_kernel<1><<<1, 128, smem>>>(dA, dB, dD, N, K, reps, derr);
        cudaError_t e = cudaDeviceSynchronize();
        int herr; cudaMemcpy(&herr, derr, 4, cudaMemcpyDeviceToHost);
        std::vector<float> D(128 * N); cudaMemcpy(D.data(), dD, D.size() * 4, cudaMemcpyDeviceToHost);
        long long bad = 0, maxv = 0;
        for (int r = 0; r < 128; r++) for (int n = 0; n < N; n++) {
            long long s = 0; for (int k = 0; k < K; k++) s += Ai[r * K + k] * Bi[n * K + k];
            s *= reps;
            maxv = llabs(s) > maxv ? llabs(s) : maxv;
            if ((double)D[r * N + n] != (double)s) { if (bad < 5) printf("f8 t%d mismatch r%d n%d got %.1f want %lld\n", trial, r, n, D[r*N+n], s); bad++; }
        }
        printf("F8 probe trial %d K=%d reps=%d: cuda=%s timeout=%d mismatches=%lld max|sum|=%lld\n", trial, K, reps, cudaGetErrorString(e), herr, bad, maxv);
    }
    // ---- rates
    for (int esz = 1; esz <= 2; esz++) {
        int iters = 20000;
        size_t smem = (128 + 256) * 32;
        cudaEvent_t a, b; cudaEventCreate(&a); cudaEventCreate(&b);
        if (esz == 1) cudaFuncSetAttribute(rate_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        else cudaFuncSetAttribute(rate_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        for (int rep = 0; rep < 2; rep++) {
            cudaEventRecord(a);
            if (esz == 1) rate_kernel<1><<<152, 128, smem>>>(iters, derr); else rate_kernel<2><<<152, 128, smem>>>(iters, derr);
            cudaEventRecord(b);
            cudaError_t e = cudaEventSynchronize(b);
            float ms; cudaEventElapsedTime(&ms, a, b);
            double flops = 2.0 * 128 * 256 * (esz == 1 ? 32 : 16) * (double)iters * 152;
            printf("rate %s: %.3f ms -> %.1f TFLOP/s (%s)\n", esz == 1 ? "f8f6f4 e4m3" : "f16", ms, flops / ms / 1e9, cudaGetErrorString(e));
        }
    }
    int herr; cudaMemcpy(&herr, derr, 4, cudaMemcpyDeviceToHost);
    printf("final err flag %d\n", herr);
    return 0;
}
