// Device-side data layout and kernel launch interface shared by the host
// library (dg_api.cpp) and the per-degree kernel translation units.
#pragma once
#include <utility>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace dgc {

constexpr int THREADS = 256;

// Reciprocal and square root of the flux evaluations.  FP32: the hardware
// approximations (relative error a few units in the last place, far below
// the FP32 and tensor-core tolerances); FP64 (the debug path): correctly
// rounded.
__device__ __forceinline__ float recip(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double recip(double x) { return __drcp_rn(x); }
__device__ __forceinline__ float fsqrt(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double fsqrt(double x) { return sqrt(x); }

__host__ __device__ constexpr int np_of(int N) { return (N + 1) * (N + 2) / 2; }
__host__ __device__ constexpr int q_of(int N) { return (3 * N + 2) / 2; }
__host__ __device__ constexpr int nq_of(int N) { return q_of(N) * q_of(N); }
__host__ __device__ constexpr int ng_of(int N) { return q_of(N); }
__host__ __device__ constexpr int nf_of(int N) { return 3 * q_of(N); }

// Packed operator table of degree N (offsets in elements of the real type).
// All tables are stored transposed so that the thread index runs along the
// contiguous dimension in the kernels.
struct OpsLayout {
    int icub, mrt, mst, drt, dst, igt, mlt, lt, qrt, qst, vinvt, itopt, w, total;
};
__host__ __device__ constexpr OpsLayout ops_layout(int N) {
    const int NP = np_of(N), NQ = nq_of(N), NF = nf_of(N);
    OpsLayout o{};
    o.icub = 0;                    // IcubT [NP][NQ]
    o.mrt = o.icub + NP * NQ;      // (Mref^-1 D_r^T W)^T [NQ][NP]
    o.mst = o.mrt + NQ * NP;
    o.drt = o.mst + NQ * NP;       // (D_r^T W)^T [NQ][NP]
    o.dst = o.drt + NQ * NP;
    o.igt = o.dst + NQ * NP;       // I_g^T [NP][NF]
    o.mlt = o.igt + NP * NF;       // (Mref^-1 Lift)^T [NF][NP]
    o.lt = o.mlt + NF * NP;        // Lift^T [NF][NP]
    o.qrt = o.lt + NF * NP;        // (Mref^-1 D_r^T W I_cub)^T [NP][NP]
    o.qst = o.qrt + NP * NP;
    o.vinvt = o.qst + NP * NP;     // (V^-1)^T [NP][NP]
    o.itopt = o.vinvt + NP * NP;   // Itop^T [NP][NQ]
    o.w = o.itopt + NP * NQ;       // cubature weights [NQ]
    o.total = o.w + NQ;
    return o;
}

// Curved-element geometry record (per element, stride curved_stride):
//   [c * NQ + qn]          c = 0..4: J r_x, J r_y, J s_x, J s_y, J at cubature nodes
//   [5 NQ + c * NF + fg]   c = 0..2: n_x, n_y, sJ at face points
//   [5 NQ + 3 NF + j NP + i]  (M_k^-1)^T
__host__ __device__ constexpr int curved_stride(int N) {
    return 5 * nq_of(N) + 3 * nf_of(N) + np_of(N) * np_of(N);
}

// Connectivity word per element: int4 {nb0, nb1, nb2, code}, with
// code bits [4f, 4f+1] = neighbour face of face f, [4f+2, 4f+3] = bc of face f.
__host__ __device__ constexpr int code_face(int code, int f) { return (code >> (4 * f)) & 3; }
__host__ __device__ constexpr int code_bc(int code, int f) { return (code >> (4 * f + 2)) & 3; }

template <typename Real>
struct StageArgs {
    const Real* Us;     // stage input [K][4][NP] (device order)
    const Real* Un;     // U^n (read when a != 0)
    Real* Uout;         // output
    Real a, b, dt;      // Uout = a Un + b (Us + dt L(Us));  rhs_only: Uout = L(Us)
    int flux;           // numerical flux: 0 local Lax-Friedrichs, 1 HLLC
    Real* dU;           // low-storage RK register: dU = a dU + dt L(Us), Uout = Us + b dU (null: the form above)
    int rhs_only;
    const int4* conn;   // [K]
    const Real* geoA;   // [K_aff][4]: x_r, x_s, y_r, y_s
    const Real* geoC;   // [Kc][curved_stride]
    const Real* ops;    // packed operator table
    const Real* eps;    // [K] viscosity (AV)
    Real* eps_next;     // AV, tensor-core path: eps of the state this stage writes (null: none)
    // AV: count of tiles (sensor kernel: elements) with eps > 0 -- incremented
    // where eps is written (eps_next or a sensor launch); the tensor-core
    // gradient kernel reads it and does nothing when it is 0 (null: none)
    int* visc;
    int* visc_in;       // AV stage kernel: the count of the eps it reads (its last CTA resets it; null: viscous)
    const Real* q;      // [K][2][4][NP] sqrt(eps) grad U (AV)
    long long K, Kaff;
    Real gamma;
    Real uinf[4];
    // sensor parameters (AV); ramp band of S = 10^(s0 -+ kappa), set on the host
    double s0, kappa, eps0;
    double S_lo, S_hi;
    // elements per CUDA-core tile (0: the degree's default); sets the grid,
    // the shared-memory layout and the launch's shared memory
    int tile_e;
};

// Per-degree launchers (kernels_n<N>.cu).  Return cudaError_t as int.
template <int N, typename Real> int launch_stage(const StageArgs<Real>& a, int av, cudaStream_t st);
template <int N, typename Real> int launch_sensor(const StageArgs<Real>& a, Real* eps_out, cudaStream_t st);
template <int N, typename Real> int launch_grad(const StageArgs<Real>& a, Real* q_out, cudaStream_t st);
// Set the dynamic shared-memory limits of the degree-N kernels (call once
// per device before the first launch or stream capture).
template <int N, typename Real> int prepare_kernels();
// CUDA-core tile sizes: the default, and whether a tile of e elements fits
// the shared-memory limit of one CTA in both the stage and gradient kernels.
template <int N, typename Real> int tile_e_default();
template <int N, typename Real> bool tile_e_fits(int e, int av);

// Tensor-core stage kernel (tc_kernels.cuh, instantiated per degree and
// precision in tc_stage_n<N>_<prec>.cu): PREC 1 = TF32, 2 = BF16 x3; cfg =
// the tile-pipeline configuration 10 C + P (C CTAs per SM of P pipelines),
// 0 = the default; tc_configs lists the fitting ones (at most 4).
template <int N, int PREC>
int launch_stage_tc_prec(const StageArgs<float>& a, int av, const unsigned char* ops_tc, int* err, cudaStream_t st,
                         int cfg);
template <int N, int PREC> int prepare_tc_prec();
template <int N> int tc_configs_n(int av, int* out4);
#ifdef DGC_PHASE_CLOCKS
template <int N> int tc_phase_cycles(unsigned long long* out16, bool reset);
#endif
template <int N>
int launch_grad_tc(const StageArgs<float>& a, float* q_out, int prec, const unsigned char* ops_tc, int* err,
                   cudaStream_t st);
template <int N> int prepare_grad_tc();
struct RefOps;
template <int N> std::vector<uint8_t> pack_ops_tc(const RefOps& R, int prec);

// Resident CTAs per SM of a kernel from its attributes and the device
// limits (registers, shared memory incl. the per-block reservation, warps),
// and the larger of that and the runtime's occupancy estimate.
inline int resident_ctas(const void* kern, int threads, size_t dyn_smem) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return 0;
    int dev = 0, smem_sm = 0, reserved = 0, regs_sm = 0, warps_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&warps_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    warps_sm /= 32;
    const size_t per_block = dyn_smem + fa.sharedSizeBytes + (size_t)reserved;
    int by_smem = per_block ? (int)(smem_sm / per_block) : 64;
    const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
    int by_regs = regs_warp ? regs_sm / (regs_warp * ((threads + 31) / 32)) : 64;
    int by_warps = warps_sm / ((threads + 31) / 32);
    int manual = by_smem < by_regs ? by_smem : by_regs;
    manual = manual < by_warps ? manual : by_warps;
    int api = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&api, kern, threads, dyn_smem) != cudaSuccess) api = 0;
    cudaGetLastError();
    return api > manual ? api : manual;
}

// Launch with programmatic stream serialization: the kernel may begin
// before the previous kernel of the stream has finished and must wait for it
// (griddepcontrol.wait) before touching that kernel's results.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), unsigned grid, unsigned threads, size_t smem, cudaStream_t st,
                       Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// Generic kernels (kernels_common.cu)
// Diagnostics: one bounded mbarrier wait (see dg_selftest_bounded_wait).
int launch_bounded_wait(uint32_t limit, int arrive, int* status, cudaStream_t st);

template <typename Real>
int launch_residual(const Real* L, int nvar, long long K, int NP, double* partial, double* out,
                    cudaStream_t st);   // out: nvar max-norms, then nvar Euclidean norms
template <typename Real>
int launch_permute(const Real* src, Real* dst, const long long* map, long long K, int rowlen, cudaStream_t st);
template <typename Real>
int launch_prolong(const Real* in, Real* out, const Real* P, long long K, int nvar, int npf, int npt,
                   const long long* src, cudaStream_t st);
int residual_blocks();

}  // namespace dgc
