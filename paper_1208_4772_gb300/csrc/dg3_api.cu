// Host side of the tetrahedral method (paper Sec. 2 with d = 3): reference
// operators (refops3.cpp), face matching and orientation from global vertex
// numbers, per-element geometry in FP64, and the stage launch.  The meshes
// it uploads share the rest of the C ABI (state I/O, dg_step, dg_step_lserk,
// dg_eval_rhs, dg_residual) with the triangle path; see include/dgcurved.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "dg3_device.h"
#include "dg_internal.h"
#include "dgcurved.h"
#include "refops.h"
#include "refops3.h"

using namespace dgc;

namespace {

const RefOps3* get_refops3(int N, std::string& err) {
    static std::mutex mu;
    static std::map<int, std::unique_ptr<RefOps3>> cache;
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(N);
    if (it != cache.end()) return it->second.get();
    auto R = std::make_unique<RefOps3>();
    if (!build_refops3(N, *R, err)) return nullptr;
    const RefOps3* p = R.get();
    cache[N] = std::move(R);
    return p;
}

// Operator tables in the kernel's layout (ops3_layout): the volume products
// in blocks of four along their summation index, so that one 16-byte load
// gives a thread four consecutive terms.
std::vector<double> pack_ops3(const RefOps3& R) {
    const int NP = R.Np, NQ = R.Nq, NG = R.Ng;
    const int NPP = pad4(NP), NQP = pad4(NQ);
    const Ops3Layout L = ops3_layout(R.N);
    std::vector<double> o((size_t)L.total, 0.0);
    for (int j = 0; j < NP; ++j)
        for (int q = 0; q < NQ; ++q)
            o[L.icub + ((size_t)(j / 4) * NQP + q) * 4 + j % 4] = R.Icub[(size_t)q * NP + j];
    for (int q = 0; q < NQ; ++q)
        for (int n = 0; n < NP; ++n) {
            const size_t at = ((size_t)(q / 4) * NPP + n) * 4 + q % 4;
            o[L.drw + at] = R.DrW[(size_t)n * NQ + q];
            o[L.dsw + at] = R.DsW[(size_t)n * NQ + q];
            o[L.dtw + at] = R.DtW[(size_t)n * NQ + q];
        }
    const int NFP = R.Nfp, NFPP = pad4(NFP), NGP = pad4(NG);
    for (int c = 0; c < 6; ++c)
        for (int g = 0; g < NG; ++g)
            for (int i = 0; i < NFP; ++i) {
                const double v = R.I2[((size_t)c * NG + g) * NFP + i];
                o[L.i2 + ((size_t)c * NG + g) * NFPP + i] = v;
                o[L.i2t + ((size_t)c * NFP + i) * NGP + g] = v;
            }
    for (int g = 0; g < NG; ++g) o[L.wg + g] = R.wg[g];
    for (int j = 0; j < NP; ++j)
        for (int n = 0; n < NP; ++n) o[L.mi + (size_t)j * NP + n] = R.Mrefinv[(size_t)n * NP + j];
    return o;
}

template <typename Real>
int copy_table(const std::vector<double>& v, void** dst) {
    std::vector<Real> h(v.begin(), v.end());
    if (cudaMalloc(dst, h.size() * sizeof(Real)) != cudaSuccess) {
        cudaGetLastError();
        *dst = nullptr;
        return DG_ENOMEM;
    }
    if (cudaMemcpy(*dst, h.data(), h.size() * sizeof(Real), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(*dst);
        *dst = nullptr;
        return DG_ECUDA;
    }
    return DG_OK;
}

template <typename Real>
StageArgs3<Real> make_args3(const MeshData& m, const void* Us, const void* Un, void* out, double a, double b,
                            double dt, int rhs_only, void* dU) {
    StageArgs3<Real> s{};
    s.Us = (const Real*)Us;
    s.Un = (const Real*)Un;
    s.Uout = (Real*)out;
    s.dU = (Real*)dU;
    s.a = (Real)a;
    s.b = (Real)b;
    s.dt = (Real)dt;
    s.rhs_only = rhs_only;
    s.flux = m.p.flux;
    s.conn = m.conn;
    s.code = m.code3;
    s.geoA = (const Real*)m.geoA;
    s.geoC = (const Real*)m.geoC;
    s.ops = (const Real*)m.ops;
    s.opsi = m.opsi3;
    s.K = m.K;
    s.Kaff = m.Kaff;
    s.gamma = (Real)m.p.gamma;
    for (int v = 0; v < 5; ++v) s.uinf[v] = (Real)m.p.u_inf[v];
    s.tile_e = m.tile_e;
    s.err = m.err;
    s.eps = (const Real*)m.eps;
    s.q = (const Real*)m.q;
    s.qout = (Real*)m.q;
    s.grad_m = 0;
    return s;
}

struct FaceKey {
    std::array<int64_t, 3> v;
    int64_t kf;
    bool operator<(const FaceKey& o) const { return v < o.v || (v == o.v && kf < o.kf); }
};

}  // namespace

namespace dgc {

// With artificial viscosity a stage is: the sensor of U_s into eps, the
// gradient pass q = sqrt(eps) grad U_s (one launch per direction), the
// stage with the viscous terms.
template <typename Real>
int enqueue_av_stage3(const MeshData& m, const void* Us, const void* Un, void* out, double a, double b, double dt,
                      int rhs_only, cudaStream_t st, void* dU) {
    int e = launch_sensor3(m.N, (const Real*)Us, (Real*)m.eps, (const Real*)m.ops, (const Real*)m.ops_av3,
                           (const Real*)m.geoC, m.K, m.Kaff, m.p.kappa, m.p.eps0, m.s0, st);
    StageArgs3<Real> s = make_args3<Real>(m, Us, Un, out, a, b, dt, rhs_only, dU);
    for (int d = 0; d < 3 && !e; ++d) {
        s.grad_m = d;
        e = launch_stage3(m.N, s, st, 2);
    }
    if (!e) e = launch_stage3(m.N, s, st, 1);
    return e;
}

int enqueue_stage3(const MeshData& m, const void* Us, const void* Un, void* out, double a, double b, double dt,
                   int rhs_only, cudaStream_t st, void* dU) {
    if (m.p.av_on)
        return m.rsize == 8 ? enqueue_av_stage3<double>(m, Us, Un, out, a, b, dt, rhs_only, st, dU)
                            : enqueue_av_stage3<float>(m, Us, Un, out, a, b, dt, rhs_only, st, dU);
    if (m.rsize == 8) return launch_stage3(m.N, make_args3<double>(m, Us, Un, out, a, b, dt, rhs_only, dU), st);
    if (m.prec == DG_TF32)
        return launch_stage3_tc(m.N, make_args3<float>(m, Us, Un, out, a, b, dt, rhs_only, dU), st);
    return launch_stage3(m.N, make_args3<float>(m, Us, Un, out, a, b, dt, rhs_only, dU), st);
}

}  // namespace dgc

extern "C" {

int dg_tet_reference_nodes(int N, double* rst_out) {
    if (!rst_out) return api_fail(nullptr, DG_EINVAL, "rst_out is NULL");
    if (N < 1 || N > 6) return api_fail(nullptr, DG_EINVAL, "N out of range");
    std::string err;
    const RefOps3* R = get_refops3(N, err);
    if (!R) return api_fail(nullptr, DG_EINVAL, err);
    for (int i = 0; i < R->Np; ++i) {
        rst_out[3 * i] = R->r[i];
        rst_out[3 * i + 1] = R->s[i];
        rst_out[3 * i + 2] = R->t[i];
    }
    return DG_OK;
}

int dg_tet_sizes(int N, int32_t* out4) {
    if (!out4 || N < 1 || N > 6) return api_fail(nullptr, DG_EINVAL, "bad argument");
    const int q = default_q(N);
    out4[0] = n_modes3(N);
    out4[1] = q * q * q;
    out4[2] = q * q;
    out4[3] = n_face_nodes3(N);
    return DG_OK;
}

static int dg_tet_mesh_upload_body(dg_ctx* ctx, int N, int64_t K, const int64_t* EToV, const int8_t* bc, const double* node_xyz,
                                   const dg_params* p, dg_mesh* out) {
    if (!ctx) return api_fail(nullptr, DG_EINVAL, "ctx is NULL");
    if (!EToV || !bc || !node_xyz || !p || !out) return api_fail(ctx, DG_EINVAL, "NULL argument");
    if (!supported_degree3(N)) return api_fail(ctx, DG_EINVAL, "tetrahedral device path supports 2 <= N <= 4");
    if (K <= 0 || K > (int64_t)1 << 30) return api_fail(ctx, DG_EINVAL, "K out of range");
    if (p->cub_q != 0 && p->cub_q != default_q(N))
        return api_fail(ctx, DG_EINVAL, "device path uses cub_q = ceil((3N+1)/2) only");
    if (p->prec != DG_FP32 && p->prec != DG_FP64_DEBUG && p->prec != DG_TF32)
        return api_fail(ctx, DG_EINVAL, "the tetrahedral path computes in DG_FP32, DG_TF32 or DG_FP64_DEBUG");
    if (p->prec == DG_TF32 && !supported_degree3_tc(N))
        return api_fail(ctx, DG_EINVAL, "DG_TF32 on tetrahedra supports N = 2 and 3");
    if (p->av_on && p->prec == DG_TF32)
        return api_fail(ctx, DG_EINVAL, "artificial viscosity on tetrahedra runs in DG_FP32 or DG_FP64_DEBUG");
    if (p->av_on && !(p->kappa > 0.0 && p->eps0 >= 0.0))
        return api_fail(ctx, DG_EINVAL, "artificial viscosity needs kappa > 0 and eps0 >= 0");
    if (p->flux != 0 && p->flux != 1)
        return api_fail(ctx, DG_EINVAL, "flux must be 0 (local Lax-Friedrichs) or 1 (HLLC)");
    if (!(p->gamma > 1.0)) return api_fail(ctx, DG_EINVAL, "gamma must exceed 1");
    std::string err;
    const RefOps3* R = get_refops3(N, err);
    if (!R) return api_fail(ctx, DG_EINVAL, err);
    const int NP = R->Np, NQ = R->Nq, NG = R->Ng, NFP = R->Nfp;

    // face matching by sorted global vertex numbers
    std::vector<FaceKey> faces((size_t)K * 4);
    std::vector<int> own((size_t)K * 4);
    for (int64_t k = 0; k < K; ++k)
        for (int f = 0; f < 4; ++f) {
            int64_t G[3];
            for (int m = 0; m < 3; ++m) G[m] = EToV[4 * k + FACE3[f][m]];
            if (G[0] == G[1] || G[1] == G[2] || G[0] == G[2])
                return api_fail(ctx, DG_EINVAL, "degenerate face at element " + std::to_string(k));
            int order[3] = {0, 1, 2};
            std::sort(order, order + 3, [&](int x, int y) { return G[x] < G[y]; });
            int o = -1;
            for (int c = 0; c < 6; ++c)
                if (PERM3[c][0] == order[0] && PERM3[c][1] == order[1] && PERM3[c][2] == order[2]) o = c;
            own[4 * k + f] = o;
            faces[4 * k + f] = FaceKey{{G[order[0]], G[order[1]], G[order[2]]}, 4 * k + f};
        }
    std::vector<int64_t> mate((size_t)K * 4, -1);
    {
        std::vector<FaceKey> sorted = faces;
        std::sort(sorted.begin(), sorted.end());
        for (size_t i = 0; i < sorted.size();) {
            size_t j = i + 1;
            while (j < sorted.size() && sorted[j].v == sorted[i].v) ++j;
            if (j - i > 2) return api_fail(ctx, DG_EINVAL, "a face is shared by more than two elements");
            if (j - i == 2) {
                mate[sorted[i].kf] = sorted[i + 1].kf;
                mate[sorted[i + 1].kf] = sorted[i].kf;
            }
            i = j;
        }
    }
    for (int64_t kf = 0; kf < K * 4; ++kf) {
        const int b = bc[kf];
        if (b < 0 || b > 2) return api_fail(ctx, DG_EINVAL, "bad bc code at element " + std::to_string(kf / 4));
        if ((b == DG_BC_INTERIOR) != (mate[kf] >= 0))
            return api_fail(ctx, DG_EINVAL, "bc must mark exactly the unmatched faces, element " +
                                                std::to_string(kf / 4));
    }

    // affine classification against the vertex nodes
    const int iv[4] = {0, N, NFP - 1, NP - 1};
    std::vector<char> curved(K, 0);
    for (int64_t k = 0; k < K; ++k) {
        const double* X = node_xyz + (size_t)k * NP * 3;
        double diam = 0.0, dev = 0.0;
        for (int v = 1; v < 4; ++v)
            for (int d = 0; d < 3; ++d) diam += std::fabs(X[3 * iv[v] + d] - X[3 * iv[0] + d]);
        for (int i = 0; i < NP; ++i) {
            const double lam[4] = {-(1.0 + R->r[i] + R->s[i] + R->t[i]) / 2.0, (1.0 + R->r[i]) / 2.0,
                                   (1.0 + R->s[i]) / 2.0, (1.0 + R->t[i]) / 2.0};
            for (int d = 0; d < 3; ++d) {
                double y = 0.0;
                for (int v = 0; v < 4; ++v) y += lam[v] * X[3 * iv[v] + d];
                dev = std::max(dev, std::fabs(X[3 * i + d] - y));
            }
        }
        if (!(dev <= 1e-12 * diam)) curved[k] = 1;
    }

    auto* m = new MeshData();
    m->dim = 3;
    m->nvar = 5;
    m->N = N; m->Np = NP; m->Nq = NQ; m->Ng = NG; m->Nf = 4 * NG; m->Nfp = NFP;
    m->K = K;
    m->p = *p;
    m->prec = p->prec;
    m->rsize = (p->prec == DG_FP64_DEBUG) ? 8 : 4;
    m->perm.reserve(K);
    for (int64_t k = 0; k < K; ++k)
        if (!curved[k]) m->perm.push_back(k);
    m->Kaff = (long long)m->perm.size();
    for (int64_t k = 0; k < K; ++k)
        if (curved[k]) m->perm.push_back(k);
    m->Kc = K - m->Kaff;
    std::vector<long long> iperm(K);
    for (int64_t d = 0; d < K; ++d) iperm[m->perm[d]] = d;

    std::vector<int4> conn(K);
    std::vector<int2> code(K);
    for (int64_t d = 0; d < K; ++d) {
        const int64_t k = m->perm[d];
        int nb[4], c[4];
        for (int f = 0; f < 4; ++f) {
            const int64_t kf = 4 * k + f, mt = mate[kf];
            const int b = bc[kf];
            nb[f] = mt >= 0 ? (int)iperm[mt / 4] : (int)d;
            const int fn = mt >= 0 ? (int)(mt % 4) : f;
            const int on = mt >= 0 ? own[mt] : 0;
            c[f] = fn | (b << 2) | (own[kf] << 4) | (on << 7);
        }
        conn[d] = make_int4(nb[0], nb[1], nb[2], nb[3]);
        code[d] = make_int2(c[0] | (c[1] << 16), c[2] | (c[3] << 16));
    }

    // geometry (FP64)
    std::vector<double> geoA((size_t)m->Kaff * 9);
    for (long long d = 0; d < m->Kaff; ++d) {
        const double* X = node_xyz + (size_t)m->perm[d] * NP * 3;
        double* g = geoA.data() + 9 * d;
        for (int dd = 0; dd < 3; ++dd)
            for (int a = 0; a < 3; ++a) g[3 * dd + a] = 0.5 * (X[3 * iv[a + 1] + dd] - X[3 * iv[0] + dd]);
        const double det = g[0] * (g[4] * g[8] - g[5] * g[7]) - g[1] * (g[3] * g[8] - g[5] * g[6]) +
                           g[2] * (g[3] * g[7] - g[4] * g[6]);
        if (!(det > 0.0)) {
            api_free_mesh(m);
            return api_fail(ctx, DG_EINVAL, "non-positive Jacobian at element " + std::to_string(m->perm[d]));
        }
    }
    const int CS = curved3_stride(N);
    std::vector<double> geoC((size_t)m->Kc * CS);
    {
        std::vector<double> M((size_t)NP * NP), Mi((size_t)NP * NP), J(NQ);
        double tu[4][3], tv[4][3];
        for (int f = 0; f < 4; ++f)
            for (int d = 0; d < 3; ++d) {
                tu[f][d] = 0.5 * (VERT3[FACE3[f][1]][d] - VERT3[FACE3[f][0]][d]);
                tv[f][d] = 0.5 * (VERT3[FACE3[f][2]][d] - VERT3[FACE3[f][0]][d]);
            }
        for (long long c = 0; c < m->Kc; ++c) {
            const long long k = m->perm[m->Kaff + c];
            const double* X = node_xyz + (size_t)k * NP * 3;
            double* g = geoC.data() + (size_t)c * CS;
            auto jacobian = [&](const double* Dr, const double* Ds, const double* Dt, double* Jm) {
                for (int i = 0; i < 9; ++i) Jm[i] = 0.0;
                for (int j = 0; j < NP; ++j)
                    for (int d = 0; d < 3; ++d) {
                        Jm[3 * d + 0] += Dr[j] * X[3 * j + d];
                        Jm[3 * d + 1] += Ds[j] * X[3 * j + d];
                        Jm[3 * d + 2] += Dt[j] * X[3 * j + d];
                    }
            };
            for (int q = 0; q < NQ; ++q) {
                double a[9];
                jacobian(&R->Dr[(size_t)q * NP], &R->Ds[(size_t)q * NP], &R->Dt[(size_t)q * NP], a);
                const double cof[9] = {a[4] * a[8] - a[5] * a[7], a[5] * a[6] - a[3] * a[8], a[3] * a[7] - a[4] * a[6],
                                       a[2] * a[7] - a[1] * a[8], a[0] * a[8] - a[2] * a[6], a[1] * a[6] - a[0] * a[7],
                                       a[1] * a[5] - a[2] * a[4], a[2] * a[3] - a[0] * a[5], a[0] * a[4] - a[1] * a[3]};
                J[q] = a[0] * cof[0] + a[1] * cof[1] + a[2] * cof[2];
                if (!(J[q] > 0.0)) {
                    api_free_mesh(m);
                    return api_fail(ctx, DG_EINVAL, "non-positive Jacobian at a cubature point of element " +
                                                        std::to_string(k));
                }
                for (int i = 0; i < 9; ++i) g[(size_t)i * NQ + q] = cof[i];
            }
            for (int f = 0; f < 4; ++f) {
                const int o = own[4 * k + f];
                const size_t off = (size_t)(f * 6 + o) * NG * NP;
                for (int gg = 0; gg < NG; ++gg) {
                    double a[9];
                    jacobian(&R->Dfr[off + (size_t)gg * NP], &R->Dfs[off + (size_t)gg * NP],
                             &R->Dft[off + (size_t)gg * NP], a);
                    double au[3], av[3];
                    for (int d = 0; d < 3; ++d) {
                        au[d] = a[3 * d] * tu[f][0] + a[3 * d + 1] * tu[f][1] + a[3 * d + 2] * tu[f][2];
                        av[d] = a[3 * d] * tv[f][0] + a[3 * d + 1] * tv[f][1] + a[3 * d + 2] * tv[f][2];
                    }
                    const double nr[3] = {au[1] * av[2] - au[2] * av[1], au[2] * av[0] - au[0] * av[2],
                                          au[0] * av[1] - au[1] * av[0]};
                    const double sJ = std::sqrt(nr[0] * nr[0] + nr[1] * nr[1] + nr[2] * nr[2]);
                    double* gf = g + 9 * NQ + f * NG + gg;
                    gf[0] = nr[0] / sJ;
                    gf[4 * NG] = nr[1] / sJ;
                    gf[8 * NG] = nr[2] / sJ;
                    gf[12 * NG] = sJ;
                }
            }
            for (int i = 0; i < NP; ++i)
                for (int j = 0; j < NP; ++j) {
                    double v = 0.0;
                    for (int q = 0; q < NQ; ++q)
                        v += R->Icub[(size_t)q * NP + i] * R->wq[q] * J[q] * R->Icub[(size_t)q * NP + j];
                    M[(size_t)i * NP + j] = v;
                }
            if (!spd_inverse(M.data(), Mi.data(), NP)) {
                api_free_mesh(m);
                return api_fail(ctx, DG_EINVAL, "curved mass matrix not SPD at element " + std::to_string(k));
            }
            for (int j = 0; j < NP; ++j)
                for (int i = 0; i < NP; ++i) g[9 * NQ + 16 * NG + (size_t)j * NP + i] = Mi[(size_t)i * NP + j];
        }
    }

    // device buffers
    cudaSetDevice(ctx->device);
    const size_t rs = m->rsize, nstate = (size_t)K * 5 * NP;
    int e;
    for (int b = 0; b < 3; ++b)
        if ((e = api_alloc(ctx, *m, &m->U[b], nstate * rs))) { api_free_mesh(m); return e; }
    if ((e = api_alloc(ctx, *m, &m->rhs, nstate * rs))) { api_free_mesh(m); return e; }
    if (p->av_on) {   // eps [K] and q [K][3][5][NP]
        if ((e = api_alloc(ctx, *m, &m->eps, (size_t)K * rs))) { api_free_mesh(m); return e; }
        if ((e = api_alloc(ctx, *m, &m->q, 3 * nstate * rs))) { api_free_mesh(m); return e; }
        m->s0 = std::isnan(p->s0) ? std::log10(1.0 / std::pow((double)N, 4)) : p->s0;
    }
    if ((e = api_alloc(ctx, *m, (void**)&m->conn, (size_t)K * sizeof(int4)))) { api_free_mesh(m); return e; }
    if ((e = api_alloc(ctx, *m, (void**)&m->code3, (size_t)K * sizeof(int2)))) { api_free_mesh(m); return e; }
    if ((e = api_alloc(ctx, *m, &m->geoA, geoA.size() * rs))) { api_free_mesh(m); return e; }
    if ((e = api_alloc(ctx, *m, &m->geoC, geoC.size() * rs))) { api_free_mesh(m); return e; }
    if ((e = api_alloc(ctx, *m, (void**)&m->dperm, (size_t)K * sizeof(long long)))) { api_free_mesh(m); return e; }
    if ((e = api_alloc(ctx, *m, (void**)&m->diperm, (size_t)K * sizeof(long long)))) { api_free_mesh(m); return e; }
    if ((e = api_alloc(ctx, *m, (void**)&m->red, (size_t)(residual_blocks() * 10 + 10) * sizeof(double)))) {
        api_free_mesh(m);
        return e;
    }
    if ((e = api_alloc(ctx, *m, (void**)&m->err, ERR_WORDS * sizeof(int)))) { api_free_mesh(m); return e; }
    if (cudaMemset(m->err, 0, ERR_WORDS * sizeof(int)) != cudaSuccess) {
        api_free_mesh(m);
        return api_fail(ctx, DG_ECUDA, "memset failed");
    }
    // operator tables, shared per context, degree and state type
    const int okey = 100000 + N * 16 + (rs == 8 ? 1 : 0), ikey = 200000 + N;
    if (ctx->ops.find(okey) == ctx->ops.end()) {
        void* d = nullptr;
        const std::vector<double> packed = pack_ops3(*R);
        const int ce = rs == 8 ? copy_table<double>(packed, &d) : copy_table<float>(packed, &d);
        if (ce) {
            api_free_mesh(m);
            return api_fail(ctx, ce, "operator table upload failed");
        }
        ctx->ops[okey] = d;
        const int pe = prepare_stage3(N, (int)rs);
        if (pe) {
            api_free_mesh(m);
            return api_fail(ctx, DG_ECUDA, std::string("tetrahedral kernel attribute set-up failed: ") +
                                               cudaGetErrorString((cudaError_t)pe));
        }
    }
    if (ctx->ops.find(ikey) == ctx->ops.end()) {
        std::vector<int> it(R->fmask.begin(), R->fmask.end());
        it.insert(it.end(), R->fpos.begin(), R->fpos.end());
        void* d = nullptr;
        if (cudaMalloc(&d, it.size() * sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            api_free_mesh(m);
            return api_fail(ctx, DG_ENOMEM, "face table allocation failed");
        }
        if (cudaMemcpy(d, it.data(), it.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaFree(d);
            api_free_mesh(m);
            return api_fail(ctx, DG_ECUDA, "face table copy failed");
        }
        ctx->ops[ikey] = d;
    }
    if (p->prec == DG_TF32) {
        const int pe = prepare_stage3_tc(N);
        if (pe) {
            api_free_mesh(m);
            return api_fail(ctx, DG_ECUDA, std::string("tetrahedral tensor-core kernel set-up failed: ") +
                                               cudaGetErrorString((cudaError_t)pe));
        }
    }
    // the sensor's table: F_h = I - V diag(deg <= N-1) V^-1, cubature weights
    const int akey = 300000 + N * 16 + (rs == 8 ? 1 : 0);
    if (p->av_on && ctx->ops.find(akey) == ctx->ops.end()) {
        const int nlow = n_modes3(N - 1);
        std::vector<double> av((size_t)av3_size(N), 0.0);
        for (int i = 0; i < NP; ++i)
            for (int j = 0; j < NP; ++j) {
                double lowp = 0.0;
                for (int k = 0; k < nlow; ++k) lowp += R->V[(size_t)i * NP + k] * R->Vinv[(size_t)k * NP + j];
                av[(size_t)i * NP + j] = (i == j ? 1.0 : 0.0) - lowp;
            }
        for (int q = 0; q < NQ; ++q) av[(size_t)NP * NP + q] = R->wq[q];
        void* d = nullptr;
        const int ce = rs == 8 ? copy_table<double>(av, &d) : copy_table<float>(av, &d);
        if (ce) {
            api_free_mesh(m);
            return api_fail(ctx, ce, "sensor table upload failed");
        }
        ctx->ops[akey] = d;
    }
    if (p->av_on) m->ops_av3 = ctx->ops[akey];
    m->ops = ctx->ops[okey];
    m->opsi3 = (const int*)ctx->ops[ikey];

    auto upload = [&](void* dst, const std::vector<double>& src) -> cudaError_t {
        if (src.empty()) return cudaSuccess;
        if (rs == 8) return cudaMemcpy(dst, src.data(), src.size() * 8, cudaMemcpyHostToDevice);
        std::vector<float> f(src.begin(), src.end());
        return cudaMemcpy(dst, f.data(), f.size() * 4, cudaMemcpyHostToDevice);
    };
    if (upload(m->geoA, geoA) != cudaSuccess || upload(m->geoC, geoC) != cudaSuccess ||
        cudaMemcpy(m->conn, conn.data(), (size_t)K * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m->code3, code.data(), (size_t)K * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m->dperm, m->perm.data(), (size_t)K * sizeof(long long), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m->diperm, iperm.data(), (size_t)K * sizeof(long long), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(m->U[0], 0, nstate * rs) != cudaSuccess) {
        api_free_mesh(m);
        return api_fail(ctx, DG_ECUDA, "mesh upload copy failed");
    }
    if (p->prec != DG_TF32) {   // a tile size tuned earlier for this kind of mesh
        auto it = ctx->tuned_e.find(3000 + N * 32 + (int)rs * 2);
        if (it != ctx->tuned_e.end()) m->tile_e = it->second;
    }
    // the copies and memsets above ran on the legacy default stream, which
    // the context's non-blocking stream does not wait for: complete them
    // before any work of the context can touch the mesh
    if (cudaStreamSynchronize(cudaStreamLegacy) != cudaSuccess) {
        api_free_mesh(m);
        return api_fail(ctx, DG_ECUDA, "mesh upload synchronisation failed");
    }
    const dg_mesh h = ctx->next_id++;
    ctx->meshes[h] = m;
    *out = h;
    return DG_OK;
}

int dg_tet_mesh_upload(dg_ctx* ctx, int N, int64_t K, const int64_t* EToV, const int8_t* bc, const double* node_xyz,
                    const dg_params* p, dg_mesh* out) {
    try {
        return dg_tet_mesh_upload_body(ctx, N, K, EToV, bc, node_xyz, p, out);
    } catch (...) {
        return exception_status(ctx);
    }
}

int dg_mesh_info(dg_ctx* ctx, dg_mesh h, int64_t* out6) {
    if (!ctx || !out6) return api_fail(ctx, DG_EINVAL, "NULL argument");
    auto it = ctx->meshes.find(h);
    if (it == ctx->meshes.end()) return api_fail(ctx, DG_ENOTFOUND, "unknown mesh handle");
    const MeshData* m = it->second;
    out6[0] = m->dim;
    out6[1] = m->nvar;
    out6[2] = m->N;
    out6[3] = m->Np;
    out6[4] = m->K;
    out6[5] = m->Kc;
    return DG_OK;
}

}  // extern "C"
