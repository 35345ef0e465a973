// Degree-independent kernels: FP64 residual reduction and element
// permutation between the caller's order and the device order.
#include <cuda_runtime.h>
#include <math.h>

#include "dg_device.h"
#include "tc_ptx.cuh"

namespace dgc {

namespace {

constexpr int RED_THREADS = 256;

// Per-variable max |L| and sum L^2 of L[K][NV][NP] in FP64 (NV = 4 on
// triangles, 5 on tetrahedra).  Each block writes 2 NV partials; the order
// of accumulation is fixed by the launch shape, so the result is
// deterministic.
template <typename Real, int NV>
__global__ void __launch_bounds__(RED_THREADS) residual_partial(const Real* L, long long total, int NP,
                                                                 double* partial) {
    double mx[NV], ss[NV];
#pragma unroll
    for (int w = 0; w < NV; ++w) mx[w] = ss[w] = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < total; n += stride) {
        const int v = (int)((n / NP) % NV);
        const double x = (double)L[n];
        const double ax = fabs(x);
#pragma unroll
        for (int w = 0; w < NV; ++w) {
            if (w == v) {
                mx[w] = (ax > mx[w] || ax != ax) ? ax : mx[w];
                ss[w] += x * x;
            }
        }
    }
    __shared__ double sm[2 * NV][RED_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int w = 0; w < NV; ++w) {
        double a = mx[w], b = ss[w];
        for (int o = 16; o > 0; o >>= 1) {
            const double ao = __shfl_xor_sync(0xffffffffu, a, o);
            a = (ao > a || ao != ao) ? ao : a;
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (lane == 0) {
            sm[w][warp] = a;
            sm[NV + w][warp] = b;
        }
    }
    __syncthreads();
    if (threadIdx.x < 2 * NV) {
        const int w = threadIdx.x;
        double acc = 0.0;
        for (int i = 0; i < RED_THREADS / 32; ++i) {
            const double x = sm[w][i];
            if (w < NV)
                acc = (x > acc || x != x) ? x : acc;
            else
                acc += x;
        }
        partial[(long long)blockIdx.x * 2 * NV + w] = acc;
    }
}

__global__ void residual_final(const double* partial, int nblocks, int nv, double* out) {
    if (threadIdx.x < 2 * nv) {
        const int w = threadIdx.x;
        double acc = 0.0;
        for (int b = 0; b < nblocks; ++b) {
            const double x = partial[(long long)b * 2 * nv + w];
            if (w < nv)
                acc = (x > acc || x != x) ? x : acc;
            else
                acc += x;
        }
        out[w] = (w < nv) ? acc : sqrt(acc);
    }
}

template <typename Real>
__global__ void permute_rows(const Real* src, Real* dst, const long long* map, long long K, int rowlen) {
    const long long total = K * rowlen;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < total; n += stride) {
        const long long row = n / rowlen;
        const int c = (int)(n - row * rowlen);
        dst[n] = src[map[row] * rowlen + c];
    }
}

// dst row r <- src row map[r], converted from S to D; one warp per row at a
// time, its lanes along the row.  Either side may be host memory that the
// device reaches coherently (pageable memory through the host's page
// tables): each row is one contiguous read and one contiguous write.
template <typename S, typename D>
__global__ void __launch_bounds__(256) gather_rows_convert(const S* src, D* dst, const long long* map, long long K,
                                                           int rowlen) {
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < K; r += nw) {
        const S* s = src + map[r] * rowlen;
        D* d = dst + r * rowlen;
        for (int c = lane; c < rowlen; c += 32) d[c] = (D)s[c];
    }
}

// Prolongation of a state between degrees: out[k][v][i] = sum_j P[i][j]
// in[src[k]][v][j] (nvar variables; src null: src[k] = k), one thread per
// output value.
template <typename Real>
__global__ void __launch_bounds__(256) prolong_kernel(const Real* in, Real* out, const Real* P, long long K, int nvar,
                                                     int npf, int npt, const long long* src) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= K * nvar * npt) return;
    const long long row = n / npt;
    const int i = (int)(n - row * npt);
    const long long k = row / nvar;
    const Real* x = in + ((src ? src[k] : k) * nvar + (row - k * nvar)) * npf;
    const Real* pr = P + (long long)i * npf;
    Real acc = 0;
    for (int j = 0; j < npf; ++j) acc += pr[j] * x[j];
    out[n] = acc;
}

}  // namespace

template <typename Real>
int launch_prolong(const Real* in, Real* out, const Real* P, long long K, int nvar, int npf, int npt,
                   const long long* src, cudaStream_t st) {
    const long long total = K * nvar * npt;
    if (total == 0) return 0;
    prolong_kernel<Real><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(in, out, P, K, nvar, npf, npt, src);
    return (int)cudaGetLastError();
}

int residual_blocks() { return 304; }

template <typename Real>
int launch_residual(const Real* L, int nvar, long long K, int NP, double* partial, double* out, cudaStream_t st) {
    const int nb = residual_blocks();
    if (nvar == 5)
        residual_partial<Real, 5><<<nb, RED_THREADS, 0, st>>>(L, K * 5 * NP, NP, partial);
    else
        residual_partial<Real, 4><<<nb, RED_THREADS, 0, st>>>(L, K * 4 * NP, NP, partial);
    residual_final<<<1, 32, 0, st>>>(partial, nb, nvar, out);
    return (int)cudaGetLastError();
}

template <typename Real>
int launch_permute(const Real* src, Real* dst, const long long* map, long long K, int rowlen, cudaStream_t st) {
    if (K == 0) return 0;
    const long long total = K * rowlen;
    const unsigned grid = (unsigned)((total + 255) / 256 < 152 * 16 ? (total + 255) / 256 : 152 * 16);
    permute_rows<Real><<<grid, 256, 0, st>>>(src, dst, map, K, rowlen);
    return (int)cudaGetLastError();
}

template <typename S, typename D>
int launch_gather_convert(const S* src, D* dst, const long long* map, long long K, int rowlen, cudaStream_t st) {
    if (K == 0) return 0;
    const long long warps = K < 152LL * 64 ? K : 152LL * 64;   // 8 warps a block, up to 8 blocks an SM
    gather_rows_convert<S, D><<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(src, dst, map, K, rowlen);
    return (int)cudaGetLastError();
}

template int launch_residual<float>(const float*, int, long long, int, double*, double*, cudaStream_t);
template int launch_residual<double>(const double*, int, long long, int, double*, double*, cudaStream_t);
template int launch_permute<float>(const float*, float*, const long long*, long long, int, cudaStream_t);
template int launch_permute<double>(const double*, double*, const long long*, long long, int, cudaStream_t);
template int launch_prolong<float>(const float*, float*, const float*, long long, int, int, int, const long long*,
                                   cudaStream_t);
template int launch_prolong<double>(const double*, double*, const double*, long long, int, int, int,
                                    const long long*, cudaStream_t);

namespace {

// One thread waits, with the bounded mbarrier wait every kernel of the
// library uses, on a barrier of one expected arrival; with arrive = 0
// nothing arrives, so the wait runs out after `limit` polls and the kernel
// records that in *status (1) instead of hanging.
__global__ void bounded_wait_kernel(uint32_t limit, int arrive, int* status) {
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    tc::mbar_init(&bar, 1);
    tc::mbar_fence_init();
    if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(tc::smem_addr(&bar)) : "memory");
    *status = tc::mbar_wait(&bar, 0, limit) ? 0 : 1;
}

}  // namespace

int launch_bounded_wait(uint32_t limit, int arrive, int* status, cudaStream_t st) {
    bounded_wait_kernel<<<1, 32, 0, st>>>(limit, arrive, status);
    return (int)cudaGetLastError();
}

template int launch_gather_convert<double, float>(const double*, float*, const long long*, long long, int,
                                                  cudaStream_t);
template int launch_gather_convert<float, double>(const float*, double*, const long long*, long long, int,
                                                  cudaStream_t);
template int launch_gather_convert<double, double>(const double*, double*, const long long*, long long, int,
                                                   cudaStream_t);

}  // namespace dgc
