// Residual norms without any allocation.
//
// Some callers cannot allocate device memory at the point where they need
// the residual: real-time loops that must not hit the allocator's locks or
// latency spikes, and host programs embedded in a framework that owns every
// device byte through its own pool, so that a cudaMalloc of the library
// would fail or fragment that pool.
// For them this file offers the FP64 residual-norm reduction of the library
// (the same definition as dg_residual: per-variable max |L| and sqrt(sum
// L^2)) with its per-block partial results in a fixed, file-scope device
// array instead of memory from cudaMalloc.  The caller passes the values
// and the output buffer.
//
// The array holds NOALLOC_MAX_BLOCKS x 8 doubles (1 MiB); every GPU that
// loads the library keeps it until the process exits.  All calls share it
// and it keeps the contents of the last call, so calls that overlap on the
// GPU (different streams, or different host threads on one device) race;
// calls issued in order on one stream do not.  Nothing in it needs to start
// at zero: each call writes every partial slot it later reads.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>
#include <string>

#include "dgcurved.h"

namespace dgc {
void set_global_error(const std::string& msg);   // dg_api.cu: read back by dg_last_error(NULL)
}

namespace {

constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_VALUES_PER_BLOCK = 4096;     // 16 values per thread
constexpr int NOALLOC_MAX_BLOCKS = 16384;
constexpr long long NOALLOC_MAX_VALUES = (long long)NOALLOC_MAX_BLOCKS * NOALLOC_VALUES_PER_BLOCK;
constexpr int NOALLOC_MAX_DEVICES = 64;

// Partial results: 8 doubles per block (4 maxima, 4 sums of squares).
static __device__ __align__(256) double g_noalloc_partials[NOALLOC_MAX_BLOCKS * 8];

__device__ __forceinline__ double nan_max(double a, double b) { return (b > a || b != b) ? b : a; }

// Block b reduces values [4096 b, 4096 (b + 1)) of x[K][4][Np].
__global__ void __launch_bounds__(NOALLOC_THREADS) noalloc_partial(const float* x, long long n, int Np,
                                                                  double* partial) {
    double mx[4] = {0, 0, 0, 0}, ss[4] = {0, 0, 0, 0};
    const long long b0 = (long long)blockIdx.x * NOALLOC_VALUES_PER_BLOCK;
    for (int i = threadIdx.x; i < NOALLOC_VALUES_PER_BLOCK; i += NOALLOC_THREADS) {
        const long long g = b0 + i;
        if (g >= n) break;
        const int v = (int)((g / Np) & 3);
        const double val = (double)x[g];
#pragma unroll
        for (int w = 0; w < 4; ++w)
            if (w == v) {
                mx[w] = nan_max(mx[w], fabs(val));
                ss[w] += val * val;
            }
    }
    __shared__ double sm[8][NOALLOC_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        double a = mx[w], s = ss[w];
        for (int o = 16; o > 0; o >>= 1) {
            a = nan_max(a, __shfl_xor_sync(0xffffffffu, a, o));
            s += __shfl_xor_sync(0xffffffffu, s, o);
        }
        if (lane == 0) {
            sm[w][warp] = a;
            sm[4 + w][warp] = s;
        }
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        const int w = threadIdx.x;
        double acc = 0.0;
        for (int i = 0; i < NOALLOC_THREADS / 32; ++i) acc = (w < 4) ? nan_max(acc, sm[w][i]) : acc + sm[w][i];
        partial[(long long)blockIdx.x * 8 + w] = acc;
    }
}

__global__ void __launch_bounds__(NOALLOC_THREADS) noalloc_final(const double* partial, int nblocks, double* out8) {
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += NOALLOC_THREADS)
#pragma unroll
        for (int w = 0; w < 8; ++w) acc[w] = (w < 4) ? nan_max(acc[w], partial[(long long)b * 8 + w])
                                                     : acc[w] + partial[(long long)b * 8 + w];
    __shared__ double sm[8][NOALLOC_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        double a = acc[w];
        for (int o = 16; o > 0; o >>= 1) {
            const double y = __shfl_xor_sync(0xffffffffu, a, o);
            a = (w < 4) ? nan_max(a, y) : a + y;
        }
        if (lane == 0) sm[w][warp] = a;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        const int w = threadIdx.x;
        double a = 0.0;
        for (int i = 0; i < NOALLOC_THREADS / 32; ++i) a = (w < 4) ? nan_max(a, sm[w][i]) : a + sm[w][i];
        out8[w] = (w < 4) ? a : sqrt(a);
    }
}

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// Device address of the static array on the current device, looked up once
// per device (with that device current) and kept for the life of the
// process: like every handle of this library it does not survive a
// cudaDeviceReset of that device.
int noalloc_scratch(int dev, double** out) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) {
            dgc::set_global_error(std::string("cudaGetSymbolAddress of the static scratch failed: ") +
                                  cudaGetErrorString(e));
            return DG_ECUDA;
        }
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return DG_OK;
}

}  // namespace

extern "C" int dg_residual_norms_noalloc(const float* values_dev, int64_t K, int32_t Np, double* out8_dev,
                                         void* cuda_stream) {
    if (!values_dev || !out8_dev || K <= 0 || Np <= 0) {
        dgc::set_global_error("dg_residual_norms_noalloc: NULL pointer or non-positive size");
        return DG_EINVAL;
    }
    // compare before multiplying: K * 4 * Np must not overflow
    if (K > NOALLOC_MAX_VALUES / (4LL * Np)) {
        dgc::set_global_error("dg_residual_norms_noalloc: K = " + std::to_string(K) + ", Np = " + std::to_string(Np) +
                              ": K*4*Np exceeds the static scratch limit of " + std::to_string(NOALLOC_MAX_VALUES) +
                              " values");
        return DG_EINVAL;
    }
    const long long n = (long long)K * 4 * Np;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        cudaGetLastError();
        dgc::set_global_error("dg_residual_norms_noalloc: no usable current CUDA device");
        return DG_ECUDA;
    }
    double* scratch = nullptr;
    const int st = noalloc_scratch(dev, &scratch);
    if (st != DG_OK) return st;
    const int nblocks = (int)((n + NOALLOC_VALUES_PER_BLOCK - 1) / NOALLOC_VALUES_PER_BLOCK);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    noalloc_partial<<<nblocks, NOALLOC_THREADS, 0, s>>>(values_dev, n, Np, scratch);
    noalloc_final<<<1, NOALLOC_THREADS, 0, s>>>(scratch, nblocks, out8_dev);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        dgc::set_global_error(std::string("dg_residual_norms_noalloc: launch failed: ") + cudaGetErrorString(e));
        return DG_ECUDA;
    }
    return DG_OK;
}
