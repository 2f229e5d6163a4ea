// A transform entry point that allocates no memory.
//
// Who needs it: callers that may not allocate device memory once they are
// running -- code executing inside a region where cudaMalloc is forbidden or
// would stall (for example a latency-critical loop that must never synchronise
// the device, which cudaMalloc/cudaFree can do), or an embedding application
// that owns every byte of device memory through its own pool and gives a
// library only its input and output buffers.  The regular plan API allocates
// its tables and its scratch buffer when the plan is created; this entry point
// instead keeps its scratch in memory reserved when the library is loaded.
//
// What it runs: the native-FP64 six-step path (the same stage kernels the
// OBFFT_MODE_FP64_NATIVE plans launch), whose two stages per axis pass
// exchange data through a scratch buffer.  That scratch and the twiddle tables
// live in the file-scope device arrays below, sized for grids of at most
// OBFFT_NOALLOC_MAX_ELEMS complex128 values.  Every GPU that loads the library
// holds these arrays (about 32 MiB) until the process exits.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "obfft_internal.h"

namespace obfft {

constexpr int64_t NOALLOC_MAX_ELEMS = (int64_t)1 << 21;   // complex128 values per call
constexpr int NOALLOC_TW_PER_AXIS = 4096 + 2 * 64;        // n + q + p twiddles per axis
constexpr int NOALLOC_MAX_DEVICES = 64;

// Scratch shared by every call of obfft_exec_fp64_noalloc on this device.
static __device__ __align__(256) double2 g_noalloc_scratch[NOALLOC_MAX_ELEMS];
// Twiddle tables of the three axes of the current call.
static __device__ __align__(256) double2 g_noalloc_tw[3 * NOALLOC_TW_PER_AXIS];

// Device addresses of the two arrays, looked up once per device and CUDA
// context.  In host code the array names are only host-side stand-ins; the
// kernels must be given these addresses instead.  The context's unique ID is
// kept beside them: after cudaDeviceReset the device gets a new primary
// context, its arrays live at new addresses, and the next call looks them up
// again instead of using the stale ones.
static void *g_scratch_addr[NOALLOC_MAX_DEVICES];
static void *g_tw_addr[NOALLOC_MAX_DEVICES];
static unsigned long long g_ctx_id[NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mutex;
// host staging of the twiddle tables (static: no heap allocation per call)
static double2 g_tw_host[3 * NOALLOC_TW_PER_AXIS];

// Unique ID of the CUDA context current on this thread (0 if none or if the
// driver does not provide one).  The two driver calls are resolved through the
// runtime, so the library does not link the driver library itself and still
// loads on machines without a GPU.
static unsigned long long current_context_id() {
    typedef CUresult (*get_current_t)(CUcontext *);
    typedef CUresult (*get_id_t)(CUcontext, unsigned long long *);
    static get_current_t get_current = nullptr;
    static get_id_t get_id = nullptr;
    if (!get_current || !get_id) {
        void *f = nullptr, *g = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &g, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess)
            return 0;
        get_current = (get_current_t)f;
        get_id = (get_id_t)g;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

static obfft_status noalloc_setup(int dev) {
    // the context current on this thread: the device's primary context once
    // the runtime has initialised it (cudaGetDevice in the caller does not;
    // cudaGetSymbolAddress below does, and the ID is read again afterwards)
    unsigned long long id = current_context_id();
    if (g_scratch_addr[dev] && g_tw_addr[dev] && id != 0 && id == g_ctx_id[dev]) return OBFFT_OK;
    void *s = nullptr, *t = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&s, g_noalloc_scratch);
    if (e != cudaSuccess)
        return set_error(OBFFT_ERR_CUDA, std::string("no-alloc set-up (scratch address): ") + cudaGetErrorString(e));
    e = cudaGetSymbolAddress(&t, g_noalloc_tw);
    if (e != cudaSuccess)
        return set_error(OBFFT_ERR_CUDA, std::string("no-alloc set-up (twiddle address): ") + cudaGetErrorString(e));
    if (id == 0) id = current_context_id();
    g_scratch_addr[dev] = s;
    g_tw_addr[dev] = t;
    g_ctx_id[dev] = id;
    return OBFFT_OK;
}

// exp(dir 2 pi i m / N) for m < N, double precision (same generator as the plans)
void fp64_twiddles(int N, int dir, double2 *out);

}  // namespace obfft

using namespace obfft;

extern "C" obfft_status obfft_exec_fp64_noalloc(const void *in, void *out, int64_t n0, int64_t n1, int64_t n2,
                                                int dir, void *stream) {
    if (!in || !out) return set_error(OBFFT_ERR_ARG, "in/out is NULL");
    if (in == out) return set_error(OBFFT_ERR_ARG, "in == out: out-of-place only");
    if (((uintptr_t)in | (uintptr_t)out) & 15) return set_error(OBFFT_ERR_ARG, "in/out must be 16-byte aligned");
    if (dir != -1 && dir != 1) return set_error(OBFFT_ERR_ARG, "dir must be -1 or +1");
    if (n0 < 1 || n1 < 1 || n2 < 1) return set_error(OBFFT_ERR_ARG, "sizes must be >= 1");
    GridDesc gd;
    gd.n[0] = n0; gd.n[1] = n1; gd.n[2] = n2;
    // every axis within the factor limit first (so the product below cannot
    // wrap around), with the split the FP64-native plans choose by default
    for (int a = 0; a < 3; a++)
        if (!choose_split(gd.n[a], &gd.ax[a], KMAX))
            return set_error(OBFFT_ERR_UNSUPPORTED_SIZE, "axis length " + std::to_string(gd.n[a]) +
                                                             " does not factor as p*q with p, q <= 64");
    if (n0 * n1 * n2 > NOALLOC_MAX_ELEMS)
        return set_error(OBFFT_ERR_UNSUPPORTED_SIZE,
                         "obfft_exec_fp64_noalloc: n0*n1*n2 = " + std::to_string(n0 * n1 * n2) +
                             " exceeds the fixed scratch of " + std::to_string(NOALLOC_MAX_ELEMS) +
                             " complex128 values; use a plan for larger grids");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(OBFFT_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return set_error(OBFFT_ERR_ARG, "device index out of range");

    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    obfft_status st = noalloc_setup(dev);
    if (st != OBFFT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    double2 *scratch = (double2 *)g_scratch_addr[dev];
    double2 *twdev = (double2 *)g_tw_addr[dev];

    // twiddle tables of the three axes, packed: [n][q][p] of each axis in turn
    AxisTables tabs[3];
    size_t used = 0;
    for (int a = 0; a < 3; a++) {
        const AxisPlan &ap = gd.ax[a];
        if (ap.n == 1) continue;
        double2 *h = g_tw_host + used;
        fp64_twiddles(ap.n, dir, h);
        fp64_twiddles(ap.q, dir, h + ap.n);
        fp64_twiddles(ap.p, dir, h + ap.n + ap.q);
        tabs[a].n = ap.n; tabs[a].p = ap.p; tabs[a].q = ap.q; tabs[a].dir = dir;
        tabs[a].tw = (double *)(twdev + used);
        used += (size_t)ap.n + ap.q + ap.p;
    }
    // pageable-source copy of the entries in use: returns once the host buffer
    // has been staged, so the static host table can be reused by the next call
    if (used) {
        e = cudaMemcpyAsync(twdev, g_tw_host, used * sizeof(double2), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return set_error(OBFFT_ERR_CUDA, std::string("twiddle upload: ") + cudaGetErrorString(e));
    }

    const double2 *src = (const double2 *)in;
    double2 *dst = (double2 *)out;
    const int64_t total = n0 * n1 * n2;
    for (int axis = 2; axis >= 0; axis--) {
        const AxisPlan &ap = gd.ax[axis];
        if (ap.n == 1) {
            if (src != dst) {
                e = cudaMemcpyAsync(dst, src, total * 16, cudaMemcpyDeviceToDevice, s);
                if (e != cudaSuccess) return set_error(OBFFT_ERR_CUDA, cudaGetErrorString(e));
            }
        } else {
            StageGeom g;
            g.P = total / ap.n;
            g.L = g.P;
            g.n = ap.n; g.p = ap.p; g.q = ap.q;
            e = launch_stage_fp64(tabs[axis], g, 1, src, scratch, s);
            if (e == cudaSuccess) e = launch_stage_fp64(tabs[axis], g, 2, scratch, dst, s);
            if (e != cudaSuccess) return set_error(OBFFT_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
        }
        src = dst;
    }
    return OBFFT_OK;
}
