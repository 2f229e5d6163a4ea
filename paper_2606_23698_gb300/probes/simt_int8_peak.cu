// Peak-rate probe for the two rooflines the tcgen05 probe does not cover:
//   * INT8 tensor rate of warp-level mma.sync.m16n8k32.s32.s8.s8.s32 (the INT8
//     MMA form sm_103a accepts; the INT8 mode's residue GEMMs use it), with an
//     exactness check of one tile against integer arithmetic;
//   * SIMT integer issue rate: independent chains of 32-bit integer
//     multiply-adds (IMAD) and of three-input adds / logic ops, the kinds of
//     instructions the per-output integer epilogue consists of.
// Every kernel is a bounded loop with in-range stores.
//
// Build and run (one GPU):
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o simt_int8_peak \
//        paper_2606_23698_gb300/probes/simt_int8_peak.cu && ./simt_int8_peak
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include <cuda_runtime.h>

#define CK(x)                                                                                    \
    do {                                                                                         \
        cudaError_t e_ = (x);                                                                    \
        if (e_ != cudaSuccess) {                                                                 \
            printf("CUDA error %s at line %d\n", cudaGetErrorString(e_), __LINE__);              \
            exit(1);                                                                             \
        }                                                                                        \
    } while (0)

__device__ __forceinline__ void mma_s8(int (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One m16n8k32 tile from A [16][32] and B [32][8] (row-major s8), result D [16][8].
// Fragment layout of mma.m16n8k32 (s8): a[r] holds 4 consecutive k of row
// (lane / 4) + 8 (r & 1), k offset 4 (lane % 4) + 16 (r >> 1); b[r] holds 4
// consecutive k of column lane / 4, k offset 4 (lane % 4) + 16 r; c[r] is row
// (lane / 4) + 8 (r >> 1), column 2 (lane % 4) + (r & 1).
__global__ void mma_check_kernel(const int8_t *A, const int8_t *B, int *D) {
    const int lane = threadIdx.x;
    uint32_t a[4], b[2];
    for (int r = 0; r < 4; r++) {
        const int row = lane / 4 + 8 * (r & 1), k0 = 4 * (lane % 4) + 16 * (r >> 1);
        uint32_t w = 0;
        for (int i = 0; i < 4; i++) w |= (uint32_t)(uint8_t)A[row * 32 + k0 + i] << (8 * i);
        a[r] = w;
    }
    for (int r = 0; r < 2; r++) {
        const int col = lane / 4, k0 = 4 * (lane % 4) + 16 * r;
        uint32_t w = 0;
        for (int i = 0; i < 4; i++) w |= (uint32_t)(uint8_t)B[(k0 + i) * 8 + col] << (8 * i);
        b[r] = w;
    }
    int c[4] = {0, 0, 0, 0};
    mma_s8(c, a, b[0], b[1]);
    for (int r = 0; r < 4; r++) D[(lane / 4 + 8 * (r >> 1)) * 8 + 2 * (lane % 4) + (r & 1)] = c[r];
}

// Throughput: every warp issues 4 independent accumulator chains.
__global__ void mma_rate_kernel(int iters, uint32_t seed, int *out) {
    uint32_t a[4], b0 = seed * 7u + threadIdx.x, b1 = seed * 13u + threadIdx.x;
    for (int r = 0; r < 4; r++) a[r] = seed + threadIdx.x * 3u + r;
    int c0[4] = {0, 0, 0, 0}, c1[4] = {0, 0, 0, 0}, c2[4] = {0, 0, 0, 0}, c3[4] = {0, 0, 0, 0};
    for (int it = 0; it < iters; it++) {
        mma_s8(c0, a, b0, b1);
        mma_s8(c1, a, b1, b0);
        mma_s8(c2, a, b0, b0);
        mma_s8(c3, a, b1, b1);
    }
    int s = 0;
    for (int r = 0; r < 4; r++) s += c0[r] + c1[r] + c2[r] + c3[r];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Integer issue rate: 8 independent chains per thread.  kind 0: IMAD
// (x = x * a + b); kind 1: IADD3 + LOP3 (x = (x ^ y) + z + w).
template <int KIND>
__global__ void int_rate_kernel(int iters, uint32_t seed, uint32_t *out) {
    uint32_t x[8];
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    for (int i = 0; i < 8; i++) x[i] = seed ^ (t * 2654435761u + i);
    const uint32_t a = seed | 1u, b = seed >> 3, y = seed * 5u, z = seed * 11u;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < 8; i++) {
            if (KIND == 0)
                asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[i]) : "r"(a), "r"(b));
            else
                asm volatile("{ .reg .b32 t; xor.b32 t, %0, %1; add.u32 %0, t, %2; }" : "+r"(x[i]) : "r"(y), "r"(z));
        }
    }
    uint32_t s = 0;
    for (int i = 0; i < 8; i++) s += x[i];
    out[t] = s;
}

int main() {
    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    // ---- exactness of one s8 tile ----
    {
        std::vector<int8_t> A(16 * 32), B(32 * 8);
        uint32_t st = 12345;
        for (auto &v : A) v = (int8_t)((st = st * 1664525u + 1013904223u) >> 24);
        for (auto &v : B) v = (int8_t)((st = st * 1664525u + 1013904223u) >> 24);
        int8_t *dA, *dB;
        int *dD;
        CK(cudaMalloc(&dA, A.size()));
        CK(cudaMalloc(&dB, B.size()));
        CK(cudaMalloc(&dD, 16 * 8 * sizeof(int)));
        CK(cudaMemcpy(dA, A.data(), A.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(dB, B.data(), B.size(), cudaMemcpyHostToDevice));
        mma_check_kernel<<<1, 32>>>(dA, dB, dD);
        CK(cudaGetLastError());
        std::vector<int> D(16 * 8);
        CK(cudaMemcpy(D.data(), dD, D.size() * sizeof(int), cudaMemcpyDeviceToHost));
        int bad = 0;
        for (int r = 0; r < 16; r++)
            for (int n = 0; n < 8; n++) {
                int s = 0;
                for (int k = 0; k < 32; k++) s += (int)A[r * 32 + k] * (int)B[k * 8 + n];
                if (s != D[r * 8 + n]) bad++;
            }
        printf("mma.sync s8 tile check: %d mismatches of 128\n", bad);
        CK(cudaFree(dA));
        CK(cudaFree(dB));
        CK(cudaFree(dD));
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    // ---- mma.sync s8 rate ----
    for (int wpb : {4, 8, 16}) {
        const int blocks = nsm * (32 / wpb) * 2, threads = 32 * wpb, iters = 20000;
        int *dout;
        CK(cudaMalloc(&dout, (size_t)blocks * threads * sizeof(int)));
        mma_rate_kernel<<<blocks, threads>>>(100, 1u, dout);
        CK(cudaEventRecord(e0));
        mma_rate_kernel<<<blocks, threads>>>(iters, 2u, dout);
        CK(cudaEventRecord(e1));
        CK(cudaEventSynchronize(e1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        const double ops = (double)blocks * wpb * iters * 4 * (2.0 * 16 * 8 * 32);
        printf("mma.sync m16n8k32 s8: %d warps/block x %d blocks: %.3f ms -> %.1f TOPS\n", wpb, blocks, ms,
               ops / ms / 1e9);
        CK(cudaFree(dout));
    }
    // ---- integer issue rate ----
    for (int kind = 0; kind < 2; kind++) {
        const int blocks = nsm * 8, threads = 256, iters = 20000;
        uint32_t *dout;
        CK(cudaMalloc(&dout, (size_t)blocks * threads * sizeof(uint32_t)));
        if (kind == 0) int_rate_kernel<0><<<blocks, threads>>>(100, 3u, dout);
        else int_rate_kernel<1><<<blocks, threads>>>(100, 3u, dout);
        CK(cudaEventRecord(e0));
        if (kind == 0) int_rate_kernel<0><<<blocks, threads>>>(iters, 4u, dout);
        else int_rate_kernel<1><<<blocks, threads>>>(iters, 4u, dout);
        CK(cudaEventRecord(e1));
        CK(cudaEventSynchronize(e1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        const double inst = (double)blocks * threads * iters * 8 * (kind == 0 ? 1 : 2);
        printf("integer %s: %.3f ms -> %.1f T lane-instructions/s\n", kind == 0 ? "IMAD chains" : "XOR+ADD chains",
               ms, inst / ms / 1e9);
        CK(cudaFree(dout));
    }
    int clk = 0;
    CK(cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev));
    printf("SMs %d, max SM clock %d MHz\n", nsm, clk / 1000);
    return 0;
}
