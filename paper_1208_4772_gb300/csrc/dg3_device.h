// Device-side data layout and launch interface of the tetrahedral stage
// kernel (the method of paper Sec. 2 with d = 3: five conserved variables,
// triangle faces).
#pragma once
#include "dg_device.h"

namespace dgc {

__host__ __device__ constexpr int np3_of(int N) { return (N + 1) * (N + 2) * (N + 3) / 6; }
__host__ __device__ constexpr int nfp3_of(int N) { return (N + 1) * (N + 2) / 2; }
__host__ __device__ constexpr int nq3_of(int N) { return q_of(N) * q_of(N) * q_of(N); }
__host__ __device__ constexpr int ng3_of(int N) { return q_of(N) * q_of(N); }

__host__ __device__ constexpr int pad4(int n) { return (n + 3) / 4 * 4; }

// Operator table of degree N in the real type (offsets in elements, each a
// multiple of 4; NPP = pad4(NP), NQP = pad4(NQ), NFPP = pad4(NFP),
// NGP = pad4(NG), padding entries zero):
//   Icub as [NPP/4][NQP][4]: (j, q) at ((j/4) NQP + q) 4 + j%4
//   D_r^T W, D_s^T W, D_t^T W as [NQP/4][NPP][4]: (q, n) at ((q/4) NPP + n) 4 + q%4
//   I2 [6][NG][NFPP]: face nodes -> face-frame points, by orientation
//   I2^T [6][NFP][NGP]: its transpose (the lift to the face nodes)
//   face weights [NG], (M_ref^-1)^T [NP][NP].
struct Ops3Layout {
    int icub, drw, dsw, dtw, i2, i2t, wg, mi, total;
};
__host__ __device__ constexpr Ops3Layout ops3_layout(int N) {
    const int NP = np3_of(N), NQ = nq3_of(N), NG = ng3_of(N), NFP = nfp3_of(N);
    const int NPP = pad4(NP), NQP = pad4(NQ), NFPP = pad4(NFP), NGP = pad4(NG);
    Ops3Layout o{};
    o.icub = 0;
    o.drw = o.icub + NPP * NQP;
    o.dsw = o.drw + NQP * NPP;
    o.dtw = o.dsw + NQP * NPP;
    o.i2 = o.dtw + NQP * NPP;
    o.i2t = o.i2 + 6 * NG * NFPP;
    o.wg = o.i2t + 6 * NFP * NGP;
    o.mi = pad4(o.wg + NG);
    o.total = pad4(o.mi + NP * NP);
    return o;
}
// Sensor table: the high-degree filter F_h = I - V diag(deg <= N-1) V^-1
// [NP][NP] (row-major), then the cubature weights [NQP].
__host__ __device__ constexpr int av3_size(int N) { return np3_of(N) * np3_of(N) + pad4(nq3_of(N)); }

// Integer table: fmask [4][NFP] (element node of each face node),
// fpos [4][NP] (face-local index of each element node, -1 off the face).
__host__ __device__ constexpr int opsi3_size(int N) { return 4 * nfp3_of(N) + 4 * np3_of(N); }

// Curved-element record (stride curved3_stride):
//   [(3 d + a) NQ + q]          J dr_a/dx_d at cubature point q (cofactors)
//   [9 NQ + c 4NG + f NG + g]   c = 0..3: n_x, n_y, n_z, sJ at face-frame point g of face f
//   [9 NQ + 16 NG + i NP + j]   M_k^-1
__host__ __device__ constexpr int curved3_stride(int N) {
    return 9 * nq3_of(N) + 16 * ng3_of(N) + np3_of(N) * np3_of(N);
}

// Per-element face codes: int2 {faces 0 and 1, faces 2 and 3}, 16 bits per
// face: neighbour face (2) | bc (2) << 2 | own orientation (3) << 4 |
// neighbour's orientation (3) << 7.
__host__ __device__ constexpr int code3_face(int c) { return c & 3; }
__host__ __device__ constexpr int code3_bc(int c) { return (c >> 2) & 3; }
__host__ __device__ constexpr int code3_own(int c) { return (c >> 4) & 7; }
__host__ __device__ constexpr int code3_nbr(int c) { return (c >> 7) & 7; }

template <typename Real>
struct StageArgs3 {
    const Real* Us;     // stage input [K][5][NP] (device order)
    const Real* Un;     // U^n (read when a != 0, SSP form)
    Real* Uout;
    Real* dU;           // low-storage register (null: SSP form)
    Real a, b, dt;      // SSP: Uout = a Un + b (Us + dt L); low-storage: dU = a dU + dt L, Uout = Us + b dU
    int rhs_only;       // Uout = L(Us)
    int flux;           // 0 local Lax-Friedrichs, 1 HLLC
    const int4* conn;   // [K] neighbours of faces 0..3 (own index on boundary faces)
    const int2* code;   // [K] face codes
    const Real* geoA;   // [Kaff][9] dx_d/dr_a, row d
    const Real* geoC;   // [Kc][curved3_stride]
    const Real* ops;    // ops3_layout
    const int* opsi;    // fmask, fpos
    long long K, Kaff;
    Real gamma;
    Real uinf[5];
    int tile_e;         // elements per tile (0: the default of the degree and real type)
    int* err;           // device error word (tensor-core kernel: a bounded wait ran out)
    // artificial viscosity (CUDA-core kernels): eps [K]; q [K][3][5][NP]
    // (rows m * 5 + v: sqrt(eps) dU_v/dx_m), read by the viscous stage and
    // written, one direction grad_m per launch, by the gradient pass
    const Real* eps;
    const Real* q;
    Real* qout;
    int grad_m;
};

bool supported_degree3(int N);
int prepare_stage3(int N, int rsize);
int tile3_default(int N, int rsize);
bool tile3_fits(int N, int rsize, int E);
// mode 0: the Euler stage; 1: the stage with the viscous terms (eps, q);
// 2: the gradient pass for direction grad_m (q out, no stage update).
int launch_stage3(int N, const StageArgs3<float>& a, cudaStream_t st, int mode = 0);
int launch_stage3(int N, const StageArgs3<double>& a, cudaStream_t st, int mode = 0);
// The element sensor (paper Sec. 2): eps [K] of the state U [K][5][NP];
// ops_av = av3_layout(N).
int launch_sensor3(int N, const float* U, float* eps, const float* ops, const float* ops_av, const float* geoC,
                   long long K, long long Kaff, double kappa, double eps0, double s0, cudaStream_t st);
int launch_sensor3(int N, const double* U, double* eps, const double* ops, const double* ops_av,
                   const double* geoC, long long K, long long Kaff, double kappa, double eps0, double s0,
                   cudaStream_t st);

// Tensor-core variant (TF32 products for the two volume terms, FP32 state;
// degrees 2 and 3, fixed tiles of tile3_tc(N) elements).
bool supported_degree3_tc(int N);
int tile3_tc(int N);
int prepare_stage3_tc(int N);
int launch_stage3_tc(int N, const StageArgs3<float>& a, cudaStream_t st);

}  // namespace dgc
