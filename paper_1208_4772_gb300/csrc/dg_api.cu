// Host side of libdgcurved.so: the C ABI of include/dgcurved.h.
//
// Set-up (paper Sec. 4 flowchart: "setup operators and transfer to GPU"):
// reference operators per degree (refops.cpp), per-element geometric
// factors computed in FP64 from the collocation-node coordinates, elements
// reordered affine-first, everything copied to the device once.  The time
// loop enqueues the stage kernels (kernels.cuh) and replays a captured CUDA
// graph per (mesh, dt).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <exception>
#include <map>
#include <memory>
#include <functional>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "dg3_device.h"
#include "dg_device.h"
#include "dgcurved.h"
#include "refops.h"
#include "refops3.h"
#include "dg_internal.h"
#include "dg_batch.h"

using namespace dgc;

namespace {

thread_local std::string g_err;  // errors of calls without a context

int fail(dg_ctx* ctx, int code, const std::string& msg) {
    if (ctx)
        ctx->err = msg;
    else
        g_err = msg;
    return code;
}

#define CUDA_OK(ctx, call)                                                                  \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) return fail((ctx), DG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

bool supported_degree(int N) { return N >= 2 && N <= 6; }

template <typename Real>
int dispatch_prepare(int N) {
    switch (N) {
        case 2: return prepare_kernels<2, Real>();
        case 3: return prepare_kernels<3, Real>();
        case 4: return prepare_kernels<4, Real>();
        case 5: return prepare_kernels<5, Real>();
        case 6: return prepare_kernels<6, Real>();
    }
    return (int)cudaErrorInvalidValue;
}
template <typename Real>
int dispatch_tile_default(int N) {
    switch (N) {
        case 2: return tile_e_default<2, Real>();
        case 3: return tile_e_default<3, Real>();
        case 4: return tile_e_default<4, Real>();
        case 5: return tile_e_default<5, Real>();
        case 6: return tile_e_default<6, Real>();
    }
    return 0;
}
template <typename Real>
bool dispatch_tile_fits(int N, int e, int av) {
    switch (N) {
        case 2: return tile_e_fits<2, Real>(e, av);
        case 3: return tile_e_fits<3, Real>(e, av);
        case 4: return tile_e_fits<4, Real>(e, av);
        case 5: return tile_e_fits<5, Real>(e, av);
        case 6: return tile_e_fits<6, Real>(e, av);
    }
    return false;
}
int tune_key(int dim, int N, size_t rsize, int av) { return dim * 1000 + N * 32 + (int)rsize * 2 + (av ? 1 : 0); }

template <typename Real>
int dispatch_stage(int N, const StageArgs<Real>& a, int av, cudaStream_t st) {
    switch (N) {
        case 2: return launch_stage<2, Real>(a, av, st);
        case 3: return launch_stage<3, Real>(a, av, st);
        case 4: return launch_stage<4, Real>(a, av, st);
        case 5: return launch_stage<5, Real>(a, av, st);
        case 6: return launch_stage<6, Real>(a, av, st);
    }
    return (int)cudaErrorInvalidValue;
}
template <typename Real>
int dispatch_sensor(int N, const StageArgs<Real>& a, Real* out, cudaStream_t st) {
    switch (N) {
        case 2: return launch_sensor<2, Real>(a, out, st);
        case 3: return launch_sensor<3, Real>(a, out, st);
        case 4: return launch_sensor<4, Real>(a, out, st);
        case 5: return launch_sensor<5, Real>(a, out, st);
        case 6: return launch_sensor<6, Real>(a, out, st);
    }
    return (int)cudaErrorInvalidValue;
}
template <typename Real>
int dispatch_grad(int N, const StageArgs<Real>& a, Real* out, cudaStream_t st) {
    switch (N) {
        case 2: return launch_grad<2, Real>(a, out, st);
        case 3: return launch_grad<3, Real>(a, out, st);
        case 4: return launch_grad<4, Real>(a, out, st);
        case 5: return launch_grad<5, Real>(a, out, st);
        case 6: return launch_grad<6, Real>(a, out, st);
    }
    return (int)cudaErrorInvalidValue;
}

int dispatch_stage_tc(int N, const StageArgs<float>& a, int av, int prec, const unsigned char* ops, int* err,
                      cudaStream_t st, int cfg) {
#define DGC_TC_CASE(n)                                                              \
    case n:                                                                         \
        return prec == 1 ? launch_stage_tc_prec<n, 1>(a, av, ops, err, st, cfg)   \
                         : launch_stage_tc_prec<n, 2>(a, av, ops, err, st, cfg);
    switch (N) {
        DGC_TC_CASE(2) DGC_TC_CASE(3) DGC_TC_CASE(4) DGC_TC_CASE(5) DGC_TC_CASE(6)
    }
#undef DGC_TC_CASE
    return (int)cudaErrorInvalidValue;
}

int dispatch_tc_configs(int N, int av, int* out4) {
    switch (N) {
        case 2: return tc_configs_n<2>(av, out4);
        case 3: return tc_configs_n<3>(av, out4);
        case 4: return tc_configs_n<4>(av, out4);
        case 5: return tc_configs_n<5>(av, out4);
        case 6: return tc_configs_n<6>(av, out4);
    }
    return 0;
}

int dispatch_prepare_tc(int N) {
#define DGC_TC_PREP(n)                                                  \
    case n: {                                                           \
        int e = prepare_tc_prec<n, 1>();                                \
        if (!e) e = prepare_tc_prec<n, 2>();                            \
        return e ? e : prepare_grad_tc<n>();                            \
    }
    switch (N) {
        DGC_TC_PREP(2) DGC_TC_PREP(3) DGC_TC_PREP(4) DGC_TC_PREP(5) DGC_TC_PREP(6)
    }
#undef DGC_TC_PREP
    return (int)cudaErrorInvalidValue;
}

int dispatch_grad_tc(int N, const StageArgs<float>& a, float* q, int prec, const unsigned char* ops, int* err,
                     cudaStream_t st) {
    switch (N) {
        case 2: return launch_grad_tc<2>(a, q, prec, ops, err, st);
        case 3: return launch_grad_tc<3>(a, q, prec, ops, err, st);
        case 4: return launch_grad_tc<4>(a, q, prec, ops, err, st);
        case 5: return launch_grad_tc<5>(a, q, prec, ops, err, st);
        case 6: return launch_grad_tc<6>(a, q, prec, ops, err, st);
    }
    return (int)cudaErrorInvalidValue;
}
std::vector<uint8_t> dispatch_pack_tc(int N, const RefOps& R, int prec) {
    switch (N) {
        case 2: return pack_ops_tc<2>(R, prec);
        case 3: return pack_ops_tc<3>(R, prec);
        case 4: return pack_ops_tc<4>(R, prec);
        case 5: return pack_ops_tc<5>(R, prec);
        case 6: return pack_ops_tc<6>(R, prec);
    }
    return {};
}
bool tensor_prec(int prec) { return prec == DG_TF32 || prec == DG_BF16X3; }

// Packed operator table (layout of ops_layout) in FP64.
std::vector<double> pack_ops(const RefOps& R) {
    const int NP = R.Np, NQ = R.Nq, NF = R.Nf;
    const OpsLayout L = ops_layout(R.N);
    std::vector<double> o(L.total, 0.0);
    for (int j = 0; j < NP; ++j)
        for (int q = 0; q < NQ; ++q) {
            o[L.icub + j * NQ + q] = R.Icub[(size_t)q * NP + j];
            o[L.itopt + j * NQ + q] = R.Itop[(size_t)q * NP + j];
        }
    for (int q = 0; q < NQ; ++q)
        for (int i = 0; i < NP; ++i) {
            o[L.mrt + q * NP + i] = R.MrW[(size_t)i * NQ + q];
            o[L.mst + q * NP + i] = R.MsW[(size_t)i * NQ + q];
            o[L.drt + q * NP + i] = R.DrW[(size_t)i * NQ + q];
            o[L.dst + q * NP + i] = R.DsW[(size_t)i * NQ + q];
        }
    for (int j = 0; j < NP; ++j)
        for (int fg = 0; fg < NF; ++fg) o[L.igt + j * NF + fg] = R.Ig[(size_t)fg * NP + j];
    for (int fg = 0; fg < NF; ++fg)
        for (int i = 0; i < NP; ++i) {
            o[L.mlt + fg * NP + i] = R.MLift[(size_t)i * NF + fg];
            o[L.lt + fg * NP + i] = R.Lift[(size_t)i * NF + fg];
        }
    for (int j = 0; j < NP; ++j)
        for (int i = 0; i < NP; ++i) {
            o[L.qrt + j * NP + i] = R.Qr[(size_t)i * NP + j];
            o[L.qst + j * NP + i] = R.Qs[(size_t)i * NP + j];
            o[L.vinvt + j * NP + i] = R.Vinv[(size_t)i * NP + j];
        }
    for (int q = 0; q < NQ; ++q) o[L.w + q] = R.wq[q];
    return o;
}

const RefOps* get_refops(int N, std::string& err) {
    static std::mutex mu;
    static std::map<int, std::unique_ptr<RefOps>> cache;
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(N);
    if (it != cache.end()) return it->second.get();
    auto R = std::make_unique<RefOps>();
    if (!build_refops(N, 0, *R, err)) return nullptr;
    const RefOps* p = R.get();
    cache[N] = std::move(R);
    return p;
}

// Device order of a set of elements: consecutive patches of `tile`
// elements grown breadth-first across interior faces, each new patch seeded
// from the frontier the previous one left, so that most face neighbours of
// a tile lie in the same tile and consecutive tiles are adjacent in space.
void compact_order(const std::vector<long long>& elems, const int32_t* EToE, const int8_t* bc, int64_t K, int tile,
                   std::vector<long long>& out) {
    std::vector<char> member(K, 0), placed(K, 0), queued(K, 0);
    for (long long e : elems) member[e] = 1;
    std::vector<long long> queue, frontier;
    size_t scan = 0, done = 0;
    auto next_seed = [&]() -> long long {
        while (!frontier.empty()) {
            const long long c = frontier.back();
            frontier.pop_back();
            if (!placed[c]) return c;
        }
        while (scan < elems.size() && placed[elems[scan]]) ++scan;
        return scan < elems.size() ? elems[scan] : -1;
    };
    while (done < elems.size()) {
        int count = 0;
        queue.clear();
        size_t head = 0;
        while (count < tile && done < elems.size()) {
            if (head == queue.size()) {
                const long long seed = next_seed();
                if (seed < 0) break;
                queue.push_back(seed);
                queued[seed] = 1;
            }
            const long long e = queue[head++];
            if (placed[e]) continue;
            placed[e] = 1;
            out.push_back(e);
            ++done;
            ++count;
            for (int f = 0; f < 3; ++f) {
                if (bc[3 * e + f] != DG_BC_INTERIOR) continue;
                const long long nb = EToE[3 * e + f];
                if (member[nb] && !placed[nb] && !queued[nb]) {
                    queued[nb] = 1;
                    queue.push_back(nb);
                }
            }
        }
        // discovered but not placed: seeds for the next patch
        for (size_t i = head; i < queue.size(); ++i) {
            queued[queue[i]] = 0;
            if (!placed[queue[i]]) frontier.push_back(queue[i]);
        }
    }
}

template <typename Real>
std::vector<Real> to_real(const std::vector<double>& v) {
    return std::vector<Real>(v.begin(), v.end());
}

int alloc(dg_ctx* ctx, MeshData& m, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return DG_OK;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(ctx, DG_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    m.bytes += bytes;
    m.allocs.push_back(*p);
    return DG_OK;
}

void free_mesh(MeshData* m) {
    if (!m) return;
    for (cudaEvent_t e : m->prof_ev) cudaEventDestroy(e);
    drop_graphs(*m);
    for (void* p : m->allocs) cudaFree(p);
    delete m;
}

void reset_batch(dg_ctx* ctx) {
    if (ctx->batch_gexec) cudaGraphExecDestroy(ctx->batch_gexec);
    if (ctx->batch_graph) cudaGraphDestroy(ctx->batch_graph);
    ctx->batch_gexec = nullptr;
    ctx->batch_graph = nullptr;
    for (void* b : ctx->batch_bufs) cudaFree(b);
    ctx->batch_bufs.clear();
    ctx->batch_key_meshes.clear();
    ctx->batch_key_dts.clear();
}

// Error words written by kernels whose bounded waits ran out.
int check_device_errors(dg_ctx* ctx) {
    for (auto& kv : ctx->meshes) {
        int w = 0;
        if (kv.second->err && cudaMemcpy(&w, kv.second->err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess &&
            w != 0)
            return fail(ctx, DG_ETIMEOUT, "a device-side wait ran out (error word " + std::to_string(w) + ")");
    }
    return DG_OK;
}

MeshData* find(dg_ctx* ctx, dg_mesh h) {
    auto it = ctx->meshes.find(h);
    return it == ctx->meshes.end() ? nullptr : it->second;
}

template <typename Real>
StageArgs<Real> make_args(const MeshData& m, const void* Us, const void* Un, void* out, double a, double b,
                          double dt, int rhs_only) {
    StageArgs<Real> s{};
    s.Us = (const Real*)Us;
    s.Un = (const Real*)Un;
    s.Uout = (Real*)out;
    s.a = (Real)a;
    s.b = (Real)b;
    s.dt = (Real)dt;
    s.rhs_only = rhs_only;
    s.conn = m.conn;
    s.geoA = (const Real*)m.geoA;
    s.geoC = (const Real*)m.geoC;
    s.ops = (const Real*)m.ops;
    s.eps = (const Real*)m.eps;
    s.q = (const Real*)m.q;
    s.K = m.K;
    s.Kaff = m.Kaff;
    s.gamma = (Real)m.p.gamma;
    for (int v = 0; v < 4; ++v) s.uinf[v] = (Real)m.p.u_inf[v];
    s.s0 = m.s0;
    s.kappa = m.p.kappa;
    s.eps0 = m.p.eps0;
    s.S_lo = std::pow(10.0, m.s0 - m.p.kappa);
    s.S_hi = std::pow(10.0, m.s0 + m.p.kappa);
    s.tile_e = tensor_prec(m.prec) ? 0 : m.tile_e;   // the tensor-core path has fixed tiles
    s.flux = m.p.flux;
    return s;
}

// Event pair around one kernel when the mesh is being profiled.
struct ProfScope {
    const MeshData& m;
    cudaStream_t st;
    int idx = -1;
    ProfScope(const MeshData& m_, cudaStream_t s, int kind) : m(m_), st(s) {
        if (m.prof_capturing && m.prof_next >= 0 && (size_t)m.prof_next < m.prof_kind.size()) {
            idx = m.prof_next++;
            const_cast<MeshData&>(m).prof_kind[idx] = kind;
            cudaEventRecordWithFlags(m.prof_ev[2 * idx], st, cudaEventRecordExternal);
        }
    }
    ~ProfScope() {
        if (idx >= 0) cudaEventRecordWithFlags(m.prof_ev[2 * idx + 1], st, cudaEventRecordExternal);
    }
};

template <typename Real>
int enqueue_stage_t(const MeshData& m, const void* Us, const void* Un, void* out, double a, double b, double dt,
                    int rhs_only, cudaStream_t st, int stage, void* dU, int ring) {
    StageArgs<Real> s = make_args<Real>(m, Us, Un, out, a, b, dt, rhs_only);
    s.dU = (Real*)dU;
    int e;
    const bool fused = fused_sensor(m) && stage >= 0 && !rhs_only;
    if (m.p.av_on) {
        if (fused) {
            // eps of this stage's input was written by the previous stage
            // kernel, with the count of its viscous tiles
            s.eps = (const Real*)m.eps_ring[stage];
            s.eps_next = (Real*)m.eps_ring[(stage + 1) % ring];
            s.visc = m.err + VISC_SLOT + stage;
        } else {
            // a right-hand-side evaluation on the tensor-core path uses the
            // ring slot that the next step's first stage rewrites
            Real* ebuf = (Real*)(fused_sensor(m) ? m.eps_ring[1] : m.eps);
            ProfScope ps(m, st, 0);
            if ((e = dispatch_sensor<Real>(m.N, s, ebuf, st))) return e;
            s.eps = ebuf;
        }
        {
            ProfScope ps(m, st, 1);
            if constexpr (sizeof(Real) == 4) {
                if (tensor_prec(m.prec)) {
                    if ((e = dispatch_grad_tc(m.N, s, (float*)m.q, m.prec == DG_TF32 ? 1 : 2,
                                              (const unsigned char*)m.ops_tc, m.err, st)))
                        return e;
                } else if ((e = dispatch_grad<Real>(m.N, s, (Real*)m.q, st))) {
                    return e;
                }
            } else if ((e = dispatch_grad<Real>(m.N, s, (Real*)m.q, st))) {
                return e;
            }
        }
    }
    s.visc = fused ? m.err + VISC_SLOT + (stage + 1) % ring : nullptr;   // counts the tiles eps_next makes viscous
    s.visc_in = fused ? m.err + VISC_SLOT + stage : nullptr;          // the count of this stage's eps
    ProfScope ps(m, st, 2);
    if constexpr (sizeof(Real) == 4) {
        if (tensor_prec(m.prec))
            return dispatch_stage_tc(m.N, s, m.p.av_on, m.prec == DG_TF32 ? 1 : 2,
                                     (const unsigned char*)m.ops_tc, m.err, st, m.tc_cfg);
    }
    return dispatch_stage<Real>(m.N, s, m.p.av_on, st);
}

}  // namespace

namespace dgc {

void set_global_error(const std::string& msg) { g_err = msg; }

int api_fail(dg_ctx* ctx, int code, const std::string& msg) { return fail(ctx, code, msg); }
int exception_status(dg_ctx* ctx) {
    try {
        throw;
    } catch (const std::bad_alloc&) {
        return fail(ctx, DG_ENOMEM, "host allocation failed");
    } catch (const std::exception& e) {
        return fail(ctx, DG_ENOMEM, std::string("host resources exhausted: ") + e.what());
    } catch (...) {
        return fail(ctx, DG_ENOMEM, "host resources exhausted");
    }
}
int api_alloc(dg_ctx* ctx, MeshData& m, void** p, size_t bytes) { return alloc(ctx, m, p, bytes); }
void api_free_mesh(MeshData* m) { free_mesh(m); }

int enqueue_stage(const MeshData& m, const void* Us, const void* Un, void* out, double a, double b, double dt,
                  int rhs_only, cudaStream_t st, int stage, void* dU, int ring) {
    if (m.dim == 3) {
        ProfScope ps(m, st, 2);
        return enqueue_stage3(m, Us, Un, out, a, b, dt, rhs_only, st, dU);
    }
    if (m.prec == DG_FP64_DEBUG)
        return enqueue_stage_t<double>(m, Us, Un, out, a, b, dt, rhs_only, st, stage, dU, ring);
    return enqueue_stage_t<float>(m, Us, Un, out, a, b, dt, rhs_only, st, stage, dU, ring);
}

// The tensor-core path with AV computes each stage's eps in the previous
// stage kernel's epilogue (no sensor kernel in the step graph).
bool fused_sensor(const MeshData& m) { return m.dim == 2 && m.p.av_on && tensor_prec(m.prec); }

int enqueue_sensor(const MeshData& m, const void* U, void* eps_out, cudaStream_t st, int* visc) {
    if (m.prec == DG_FP64_DEBUG) {
        StageArgs<double> s = make_args<double>(m, U, nullptr, nullptr, 0.0, 0.0, 0.0, 1);
        s.visc = visc;
        return dispatch_sensor<double>(m.N, s, (double*)eps_out, st);
    }
    StageArgs<float> s = make_args<float>(m, U, nullptr, nullptr, 0.0, 0.0, 0.0, 1);
    s.visc = visc;
    return dispatch_sensor<float>(m.N, s, (float*)eps_out, st);
}

// One SSP-RK3 step: U0 -> U1 -> U2 -> U0 (stage 3 writes U^n in place; each
// thread reads U^n only for the value it overwrites).
int enqueue_step(const MeshData& m, double dt, cudaStream_t st) {
    int e;
    if ((e = enqueue_stage(m, m.U[0], nullptr, m.U[1], 0.0, 1.0, dt, 0, st, 0))) return e;
    if ((e = enqueue_stage(m, m.U[1], m.U[0], m.U[2], 0.75, 0.25, dt, 0, st, 1))) return e;
    return enqueue_stage(m, m.U[2], m.U[0], m.U[0], 1.0 / 3.0, 2.0 / 3.0, dt, 0, st, 2);
}

// One step of Carpenter and Kennedy's five-stage fourth-order low-storage
// RK (the paper's integrator): dU <- A_i dU + dt L(U), U <- U + B_i dU.  Each
// stage reads one state buffer and writes another (neighbours read a state
// no tile is writing): U0 -> U1 -> U2 -> U1 -> U2 -> U0; dU lives in the
// right-hand-side scratch.  On the tensor-core path with AV the eps of each
// stage comes from the previous stage kernel through a ring of five
// buffers, so that the step begins and ends with eps(U^n) in buffer 0, as
// the three-stage step does.
int enqueue_step_lserk(const MeshData& m, double dt, cudaStream_t st) {
    static const double A[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                                -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
    static const double Bc[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                                 1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                                 2277821191437.0 / 14882151754819.0};
    static const int in[5] = {0, 1, 2, 1, 2}, out[5] = {1, 2, 1, 2, 0};
    for (int i = 0; i < 5; ++i) {
        const int e = enqueue_stage(m, m.U[in[i]], nullptr, m.U[out[i]], A[i], Bc[i], dt, 0, st, i, m.rhs, EPS_RING);
        if (e) return e;
    }
    return 0;
}

void drop_graphs(MeshData& m) {
    if (m.gexec) { cudaGraphExecDestroy(m.gexec); m.gexec = nullptr; }
    if (m.graph) { cudaGraphDestroy(m.graph); m.graph = nullptr; }
    if (m.gexec_ls) { cudaGraphExecDestroy(m.gexec_ls); m.gexec_ls = nullptr; }
    if (m.graph_ls) { cudaGraphDestroy(m.graph_ls); m.graph_ls = nullptr; }
}

}  // namespace dgc


template <typename Real>
static int build_batch(dg_ctx* ctx, const std::vector<MeshData*>& ms, const double* dts) {
    const int n = (int)ms.size();
    std::vector<BatchItem> items;
    int e_by_n[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < n; ++i) {
        const MeshData& m = *ms[i];
        const int E = m.tile_e > 0 ? m.tile_e : batch_tile_e(m.N, (int)m.rsize);
        e_by_n[m.N] = std::max(e_by_n[m.N], E);
        for (long long e0 = 0; e0 < m.Kaff; e0 += E)
            items.push_back(BatchItem{i, m.N, e0, (int)std::min<long long>(E, m.Kaff - e0), 0});
        for (long long e0 = m.Kaff; e0 < m.K; e0 += E)
            items.push_back(BatchItem{i, m.N, e0, (int)std::min<long long>(E, m.K - e0), 1});
    }
    // largest work first: curved tiles, then by degree
    std::stable_sort(items.begin(), items.end(), [&](const BatchItem& a, const BatchItem& b) {
        const double ca = (double)a.ne * np_of(a.N) * nq_of(a.N) * (a.curved ? 2.0 : 1.0);
        const double cb = (double)b.ne * np_of(b.N) * nq_of(b.N) * (b.curved ? 2.0 : 1.0);
        return ca > cb;
    });
    std::vector<StageArgs<Real>> args(3 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        const MeshData& m = *ms[i];
        args[i] = make_args<Real>(m, m.U[0], nullptr, m.U[1], 0.0, 1.0, dts[i], 0);
        args[n + i] = make_args<Real>(m, m.U[1], m.U[0], m.U[2], 0.75, 0.25, dts[i], 0);
        args[2 * n + i] = make_args<Real>(m, m.U[2], m.U[0], m.U[0], 1.0 / 3.0, 2.0 / 3.0, dts[i], 0);
    }
    void *dargs = nullptr, *ditems = nullptr, *dcnt = nullptr;
    if (cudaMalloc(&dargs, args.size() * sizeof(StageArgs<Real>)) != cudaSuccess ||
        cudaMalloc(&ditems, items.size() * sizeof(BatchItem)) != cudaSuccess ||
        cudaMalloc(&dcnt, 4 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        if (dargs) cudaFree(dargs);
        if (ditems) cudaFree(ditems);
        return fail(ctx, DG_ENOMEM, "batch work-list allocation failed");
    }
    ctx->batch_bufs = {dargs, ditems, dcnt};
    CUDA_OK(ctx, cudaMemcpy(dargs, args.data(), args.size() * sizeof(StageArgs<Real>), cudaMemcpyHostToDevice));
    CUDA_OK(ctx, cudaMemcpy(ditems, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice));
    CUDA_OK(ctx, cudaStreamSynchronize(cudaStreamLegacy));   // before the context's stream reads them
    const size_t smem = batch_smem_bytes<Real>(e_by_n);
    const int grid = batch_grid<Real>(ctx->device, 0, smem);
    if (grid <= 0) return fail(ctx, DG_ECUDA, "batch kernel occupancy query failed");
    // the capture of the step graph opens here; dg_batch_step adds the
    // meshes with artificial viscosity and closes it
    CUDA_OK(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    int e = (int)cudaMemsetAsync(dcnt, 0, 4 * sizeof(int), ctx->stream);
    const size_t as = sizeof(StageArgs<Real>);
    for (int st = 0; st < 3 && !e; ++st)
        e = launch_batch_stage<Real>((const char*)dargs + (size_t)st * n * as, (const BatchItem*)ditems,
                                     (int)items.size(), (int*)dcnt + st, grid, smem, ctx->stream);
    return e ? fail(ctx, DG_ECUDA, std::string("batched stage launch failed: ") +
                                       cudaGetErrorString((cudaError_t)e))
             : DG_OK;
}

// Tensor-core batch: affine tiles of 32 elements and curved tiles of the
// CUDA-core size; degrees 2..5 in one persistent launch per stage, degree 6
// (a larger shared-memory layout) in a second one.
static int build_batch_tc(dg_ctx* ctx, const std::vector<MeshData*>& ms, const double* dts) {
    const int n = (int)ms.size();
    const int prec = ms[0]->prec == DG_TF32 ? 1 : 2;
    std::vector<BatchItem> lo, hi;
    for (int i = 0; i < n; ++i) {
        const MeshData& m = *ms[i];
        std::vector<BatchItem>& v = (m.N == 6) ? hi : lo;
        const int EC = batch_tile_e(m.N, 4);
        for (long long e0 = m.Kaff; e0 < m.K; e0 += EC)
            v.push_back(BatchItem{i, m.N, e0, (int)std::min<long long>(EC, m.K - e0), 1});
        for (long long e0 = 0; e0 < m.Kaff; e0 += 32)
            v.push_back(BatchItem{i, m.N, e0, (int)std::min<long long>(32, m.Kaff - e0), 0});
    }
    // curved tiles first (slowest), then affine tiles grouped by degree,
    // highest first, so that each CTA reloads its operators rarely
    auto order = [](const BatchItem& a, const BatchItem& b) {
        if (a.curved != b.curved) return a.curved > b.curved;
        return a.N > b.N;
    };
    std::stable_sort(lo.begin(), lo.end(), order);
    std::stable_sort(hi.begin(), hi.end(), order);
    std::vector<StageArgs<float>> args(3 * (size_t)n);
    std::vector<const unsigned char*> ops(7, nullptr);
    for (int i = 0; i < n; ++i) {
        const MeshData& m = *ms[i];
        args[i] = make_args<float>(m, m.U[0], nullptr, m.U[1], 0.0, 1.0, dts[i], 0);
        args[n + i] = make_args<float>(m, m.U[1], m.U[0], m.U[2], 0.75, 0.25, dts[i], 0);
        args[2 * n + i] = make_args<float>(m, m.U[2], m.U[0], m.U[0], 1.0 / 3.0, 2.0 / 3.0, dts[i], 0);
        ops[m.N] = (const unsigned char*)m.ops_tc;
    }
    std::vector<BatchItem> items(lo);
    items.insert(items.end(), hi.begin(), hi.end());
    void *dargs = nullptr, *ditems = nullptr, *dops = nullptr, *dcnt = nullptr;
    if (cudaMalloc(&dargs, args.size() * sizeof(StageArgs<float>)) != cudaSuccess ||
        cudaMalloc(&ditems, items.size() * sizeof(BatchItem)) != cudaSuccess ||
        cudaMalloc(&dops, ops.size() * sizeof(void*)) != cudaSuccess ||
        cudaMalloc(&dcnt, 8 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        for (void* b : {dargs, ditems, dops, dcnt})
            if (b) cudaFree(b);
        return fail(ctx, DG_ENOMEM, "batch work-list allocation failed");
    }
    ctx->batch_bufs = {dargs, ditems, dops, dcnt};
    CUDA_OK(ctx, cudaMemcpy(dargs, args.data(), args.size() * sizeof(StageArgs<float>), cudaMemcpyHostToDevice));
    CUDA_OK(ctx, cudaMemcpy(ditems, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice));
    CUDA_OK(ctx, cudaMemcpy(dops, ops.data(), ops.size() * sizeof(void*), cudaMemcpyHostToDevice));
    CUDA_OK(ctx, cudaStreamSynchronize(cudaStreamLegacy));   // before the context's stream reads them
    const int glo = lo.empty() ? 0 : batch_tc_grid(ctx->device, prec, false);
    const int ghi = hi.empty() ? 0 : batch_tc_grid(ctx->device, prec, true);
    if ((!lo.empty() && glo <= 0) || (!hi.empty() && ghi <= 0))
        return fail(ctx, DG_ECUDA, "tensor-core batch kernel set-up failed");
    // the capture of the step graph opens here; dg_batch_step adds the
    // meshes with artificial viscosity and closes it
    CUDA_OK(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    int e = (int)cudaMemsetAsync(dcnt, 0, 8 * sizeof(int), ctx->stream);
    const size_t as = sizeof(StageArgs<float>);
    const BatchItem* dl = (const BatchItem*)ditems;
    for (int st = 0; st < 3 && !e; ++st) {
        const char* a = (const char*)dargs + (size_t)st * n * as;
        e = launch_batch_stage_tc(prec, false, a, dl, (int)lo.size(), (const unsigned char* const*)dops, ms[0]->err,
                                  (int*)dcnt + 2 * st, glo, ctx->stream);
        if (!e)
            e = launch_batch_stage_tc(prec, true, a, dl + lo.size(), (int)hi.size(),
                                      (const unsigned char* const*)dops, ms[0]->err, (int*)dcnt + 2 * st + 1, ghi,
                                      ctx->stream);
    }
    return e ? fail(ctx, DG_ECUDA, std::string("batched stage launch failed: ") +
                                       cudaGetErrorString((cudaError_t)e))
             : DG_OK;
}

// Meshes with artificial viscosity in a batch: each runs its own stage
// chain (sensor, gradient and stage kernels, or the tensor-core gradient and
// fused-sensor stage kernels) on a branch of the step graph forked from the
// context's stream, on a side stream of the context; the branches of
// different meshes and the persistent launches of the other meshes run
// concurrently and join at the end of the step.
static int enqueue_av_branches(dg_ctx* ctx, const std::vector<MeshData*>& av, const std::vector<double>& dts) {
    if (av.empty()) return DG_OK;
    while (ctx->side_streams.size() < std::min<size_t>(av.size(), 8)) {
        cudaStream_t s = nullptr;
        CUDA_OK(ctx, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        ctx->side_streams.push_back(s);
    }
    const size_t nb = std::min<size_t>(av.size(), ctx->side_streams.size());
    while (ctx->side_events.size() < nb + 1) {
        cudaEvent_t ev = nullptr;
        CUDA_OK(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        ctx->side_events.push_back(ev);
    }
    CUDA_OK(ctx, cudaEventRecord(ctx->side_events[nb], ctx->stream));   // the fork
    for (size_t b = 0; b < nb; ++b) CUDA_OK(ctx, cudaStreamWaitEvent(ctx->side_streams[b], ctx->side_events[nb], 0));
    for (size_t i = 0; i < av.size(); ++i) {
        cudaStream_t st = ctx->side_streams[i % nb];
        const int e = enqueue_step(*av[i], dts[i], st);
        if (e) return fail(ctx, DG_ECUDA, "stage launch of a mesh with artificial viscosity failed");
    }
    for (size_t b = 0; b < nb; ++b) {   // the join
        CUDA_OK(ctx, cudaEventRecord(ctx->side_events[b], ctx->side_streams[b]));
        CUDA_OK(ctx, cudaStreamWaitEvent(ctx->stream, ctx->side_events[b], 0));
    }
    return DG_OK;
}

static int dg_batch_step_body(dg_ctx* ctx, int n, const dg_mesh* hs, const double* dts, int nsteps) {
    if (!ctx) return fail(nullptr, DG_EINVAL, "ctx is NULL");
    if (n <= 0 || !hs || !dts || nsteps < 0) return fail(ctx, DG_EINVAL, "bad argument");
    std::vector<MeshData*> ms(n);
    for (int i = 0; i < n; ++i) {
        ms[i] = find(ctx, hs[i]);
        if (!ms[i]) return fail(ctx, DG_ENOTFOUND, "unknown mesh handle in batch");
        if (ms[i]->dim != 2) return fail(ctx, DG_EINVAL, "batched path runs triangle meshes only");
        if (ms[i]->prec != ms[0]->prec) return fail(ctx, DG_EINVAL, "batch mixes precision modes");
        if (!std::isfinite(dts[i])) return fail(ctx, DG_EINVAL, "bad dt");
        for (int j = 0; j < i; ++j)
            if (hs[j] == hs[i]) return fail(ctx, DG_EINVAL, "mesh listed twice in batch");
    }
    if (nsteps == 0) return DG_OK;
    cudaSetDevice(ctx->device);
    // meshes without viscosity share the persistent launches; the others
    // run their own stage chains on branches of the same step graph
    std::vector<MeshData*> plain, av;
    std::vector<double> dplain, dav;
    for (int i = 0; i < n; ++i) {
        (ms[i]->p.av_on ? av : plain).push_back(ms[i]);
        (ms[i]->p.av_on ? dav : dplain).push_back(dts[i]);
    }
    const std::vector<int> key(hs, hs + n);
    const std::vector<double> kdt(dts, dts + n);
    if (!ctx->batch_gexec || key != ctx->batch_key_meshes || kdt != ctx->batch_key_dts) {
        CUDA_OK(ctx, cudaStreamSynchronize(ctx->stream));
        reset_batch(ctx);
        int e = DG_OK;
        if (!plain.empty()) {   // these open the capture
            e = tensor_prec(ms[0]->prec) ? build_batch_tc(ctx, plain, dplain.data())
                : (ms[0]->rsize == 8)    ? build_batch<double>(ctx, plain, dplain.data())
                                         : build_batch<float>(ctx, plain, dplain.data());
        } else {
            CUDA_OK(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        }
        if (!e) e = enqueue_av_branches(ctx, av, dav);
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(ctx->stream, &cs);
        cudaGraph_t g = nullptr;
        const cudaError_t ce = (cs != cudaStreamCaptureStatusNone) ? cudaStreamEndCapture(ctx->stream, &g)
                                                                   : cudaErrorStreamCaptureInvalidated;
        if (e || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            reset_batch(ctx);
            return e ? e : fail(ctx, DG_ECUDA, "graph capture of the batched step failed");
        }
        ctx->batch_graph = g;
        if (cudaGraphInstantiate(&ctx->batch_gexec, g, 0) != cudaSuccess) {
            cudaGetLastError();
            reset_batch(ctx);
            return fail(ctx, DG_ECUDA, "instantiation of the batched step graph failed");
        }
        ctx->batch_key_meshes = key;
        ctx->batch_key_dts = kdt;
    }
    for (MeshData* m : av) {   // eps(U^n) of the first stage where a state was set from outside
        if (fused_sensor(*m) && !m->eps_valid) {
            CUDA_OK(ctx, cudaMemsetAsync(m->err + VISC_SLOT, 0, sizeof(int), ctx->stream));
            const int e = enqueue_sensor(*m, m->U[0], m->eps_ring[0], ctx->stream, m->err + VISC_SLOT);
            if (e) return fail(ctx, DG_ECUDA, std::string("sensor launch failed: ") + cudaGetErrorString((cudaError_t)e));
            m->eps_valid = true;
        }
    }
    for (int s = 0; s < nsteps; ++s) CUDA_OK(ctx, cudaGraphLaunch(ctx->batch_gexec, ctx->stream));
    return DG_OK;
}

extern "C" extern "C" int dg_batch_step(dg_ctx* ctx, int n, const dg_mesh* hs, const double* dts, int nsteps) {
    try {
        return dg_batch_step_body(ctx, n, hs, dts, nsteps);
    } catch (...) {
        return exception_status(ctx);
    }
}

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int dg_create(dg_ctx** out, int device, void* cuda_stream) {
    if (!out) return fail(nullptr, DG_EINVAL, "out is NULL");
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return fail(nullptr, DG_EINVAL, "no such CUDA device: " + std::to_string(device));
    }
    if (cudaSetDevice(device) != cudaSuccess) return fail(nullptr, DG_ECUDA, "cudaSetDevice failed");
    auto* c = new dg_ctx();
    c->device = device;
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
        c->own_stream = false;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return fail(nullptr, DG_ECUDA, "cudaStreamCreate failed");
        }
        c->own_stream = true;
    }
    int pageable = 0, host_tables = 0;
    if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&host_tables, cudaDevAttrPageableMemoryAccessUsesHostPageTables, device) !=
            cudaSuccess) {
        cudaGetLastError();
        pageable = host_tables = 0;
    }
    c->host_coherent = pageable == 1 && host_tables == 1;
    c->host_io = DG_HOST_IO_STAGED;
    *out = c;
    return DG_OK;
}

int dg_set_host_io(dg_ctx* ctx, int mode) {
    if (!ctx) return fail(nullptr, DG_EINVAL, "ctx is NULL");
    // the staged path is the faster of the two on GB300 (the device path's
    // kernel runs at well under the link's bandwidth on pageable memory)
    if (mode == DG_HOST_IO_AUTO) mode = DG_HOST_IO_STAGED;
    if (mode != DG_HOST_IO_STAGED && mode != DG_HOST_IO_DEVICE)
        return fail(ctx, DG_EINVAL, "unknown host I/O mode " + std::to_string(mode));
    if (mode == DG_HOST_IO_DEVICE && !ctx->host_coherent)
        return fail(ctx, DG_EINVAL, "the device has no coherent access to pageable host memory");
    ctx->host_io = mode;
    return DG_OK;
}

int dg_host_io(dg_ctx* ctx, int32_t* out) {
    if (!ctx || !out) return fail(ctx, DG_EINVAL, "NULL argument");
    *out = ctx->host_io;
    return DG_OK;
}

int dg_destroy(dg_ctx* ctx) {
    if (!ctx) return DG_OK;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto& kv : ctx->meshes) free_mesh(kv.second);
    ctx->meshes.clear();
    for (auto& kv : ctx->ops) cudaFree(kv.second);
    reset_batch(ctx);
    for (cudaStream_t s : ctx->side_streams) cudaStreamDestroy(s);
    if (ctx->res_host) cudaFreeHost(ctx->res_host);
    for (cudaEvent_t ev : ctx->side_events) cudaEventDestroy(ev);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return DG_OK;
}

int dg_reference_nodes(int N, double* rs_out) {
    if (!rs_out) return fail(nullptr, DG_EINVAL, "rs_out is NULL");
    if (N < 1 || N > 8) return fail(nullptr, DG_EINVAL, "N out of range");
    std::string err;
    const RefOps* R = get_refops(N, err);
    if (!R) return fail(nullptr, DG_EINVAL, err);
    for (int i = 0; i < R->Np; ++i) {
        rs_out[2 * i] = R->r[i];
        rs_out[2 * i + 1] = R->s[i];
    }
    return DG_OK;
}

int dg_sizes(int N, int cub_q, int32_t* out4) {
    if (!out4 || N < 1 || N > 8 || cub_q < 0) return fail(nullptr, DG_EINVAL, "bad argument");
    const int q = cub_q ? cub_q : default_q(N);
    out4[0] = n_modes(N);
    out4[1] = q * q;
    out4[2] = q;
    out4[3] = q;
    return DG_OK;
}

// The host half of an upload (no context, no device): checks, element
// classification and device order, connectivity words and the FP64
// geometric factors.  Errors go to ctx when given, else to the calling
// thread's message (dg_last_error(NULL)).
static int prepare_mesh(dg_ctx* ctx, int N, int64_t K, const int32_t* EToE, const int8_t* EToF, const int8_t* bc,
                        const double* node_xy, const dg_params* p, dg_prepared* pr) {
    if (!EToE || !EToF || !bc || !node_xy || !p) return fail(ctx, DG_EINVAL, "NULL argument");
    if (!supported_degree(N)) return fail(ctx, DG_EINVAL, "device path supports 2 <= N <= 6");
    if (K <= 0 || K > (int64_t)1 << 31) return fail(ctx, DG_EINVAL, "K out of range");
    if (p->cub_q != 0 && p->cub_q != default_q(N))
        return fail(ctx, DG_EINVAL, "device path uses cub_q = ceil((3N+1)/2) only");
    if (p->prec != DG_FP32 && p->prec != DG_FP64_DEBUG && p->prec != DG_TF32 && p->prec != DG_BF16X3)
        return fail(ctx, DG_EINVAL, "unknown precision mode");
    if (p->flux != 0 && p->flux != 1) return fail(ctx, DG_EINVAL, "flux must be 0 (local Lax-Friedrichs) or 1 (HLLC)");
    if (!(p->gamma > 1.0)) return fail(ctx, DG_EINVAL, "gamma must exceed 1");
    std::string err;
    const RefOps* R = get_refops(N, err);
    if (!R) return fail(ctx, DG_EINVAL, err);
    const int NP = R->Np, NQ = R->Nq, NF = R->Nf, NG = R->Ng;

    // connectivity checks
    for (int64_t k = 0; k < K; ++k)
        for (int f = 0; f < 3; ++f) {
            const int64_t nb = EToE[3 * k + f];
            const int fn = EToF[3 * k + f], b = bc[3 * k + f];
            if (b < 0 || b > 2) return fail(ctx, DG_EINVAL, "bad bc code at element " + std::to_string(k));
            if (b == DG_BC_INTERIOR) {
                if (nb < 0 || nb >= K || fn < 0 || fn > 2)
                    return fail(ctx, DG_EINVAL, "bad neighbour at element " + std::to_string(k));
                if (EToE[3 * nb + fn] != k || EToF[3 * nb + fn] != f)
                    return fail(ctx, DG_EINVAL, "non-reciprocal connectivity at element " + std::to_string(k));
            }
        }

    // classify: affine if the nodes are the affine image of the three vertex nodes
    const int iv1 = N, iv2 = NP - 1;
    std::vector<char> curved(K, 0);
    for (int64_t k = 0; k < K; ++k) {
        const double* X = node_xy + (size_t)k * NP * 2;
        const double x0 = X[0], y0 = X[1], x1 = X[2 * iv1], y1 = X[2 * iv1 + 1], x2 = X[2 * iv2], y2 = X[2 * iv2 + 1];
        const double diam = std::fabs(x1 - x0) + std::fabs(y1 - y0) + std::fabs(x2 - x0) + std::fabs(y2 - y0);
        double dev = 0.0;
        for (int i = 0; i < NP; ++i) {
            const double l1 = -(R->r[i] + R->s[i]) / 2, l2 = (1 + R->r[i]) / 2, l3 = (1 + R->s[i]) / 2;
            dev = std::max(dev, std::fabs(X[2 * i] - (l1 * x0 + l2 * x1 + l3 * x2)));
            dev = std::max(dev, std::fabs(X[2 * i + 1] - (l1 * y0 + l2 * y1 + l3 * y2)));
        }
        if (!(dev <= 1e-12 * diam)) curved[k] = 1;
    }
    auto* m = new MeshData();
    pr->m = m;
    m->N = N; m->Np = NP; m->Nq = NQ; m->Ng = NG; m->Nf = NF;
    m->perm.reserve(K);
    m->K = K;
    m->p = *p;
    m->prec = p->prec;
    m->rsize = (p->prec == DG_FP64_DEBUG) ? 8 : 4;
    m->s0 = std::isnan(p->s0) ? std::log10(1.0 / std::pow((double)N, 4)) : p->s0;
    {
        std::vector<long long> affine;
        affine.reserve(K);
        for (int64_t k = 0; k < K; ++k)
            if (!curved[k]) affine.push_back(k);
        compact_order(affine, EToE, bc, K, 32, m->perm);
    }
    m->Kaff = (long long)m->perm.size();
    for (int64_t k = 0; k < K; ++k)
        if (curved[k]) m->perm.push_back(k);
    m->Kc = K - m->Kaff;
    std::vector<long long>& iperm = pr->iperm;
    iperm.assign(K, 0);
    for (int64_t d = 0; d < K; ++d) iperm[m->perm[d]] = d;

    // connectivity in device order
    std::vector<int4>& conn = pr->conn;
    conn.assign(K, int4{});
    for (int64_t d = 0; d < K; ++d) {
        const int64_t k = m->perm[d];
        int nb[3], code = 0;
        for (int f = 0; f < 3; ++f) {
            const int b = bc[3 * k + f];
            nb[f] = (b == DG_BC_INTERIOR) ? (int)iperm[EToE[3 * k + f]] : (int)d;
            const int fn = (b == DG_BC_INTERIOR) ? EToF[3 * k + f] : f;
            code |= (fn | (b << 2)) << (4 * f);
        }
        conn[d] = make_int4(nb[0], nb[1], nb[2], code);
    }

    // geometry (FP64)
    std::vector<double>& geoA = pr->geoA;
    geoA.assign((size_t)m->Kaff * 4, 0.0);
    for (long long d = 0; d < m->Kaff; ++d) {
        const double* X = node_xy + (size_t)m->perm[d] * NP * 2;
        const double xr = 0.5 * (X[2 * iv1] - X[0]), xs = 0.5 * (X[2 * iv2] - X[0]);
        const double yr = 0.5 * (X[2 * iv1 + 1] - X[1]), ys = 0.5 * (X[2 * iv2 + 1] - X[1]);
        if (!(xr * ys - xs * yr > 0.0)) {
            const long long bad = m->perm[d];
            free_mesh(m);
            pr->m = nullptr;
            return fail(ctx, DG_EINVAL, "non-positive Jacobian at element " + std::to_string(bad));
        }
        geoA[4 * d] = xr; geoA[4 * d + 1] = xs; geoA[4 * d + 2] = yr; geoA[4 * d + 3] = ys;
    }
    const int CS = curved_stride(N);
    std::vector<double>& geoC = pr->geoC;
    geoC.assign((size_t)m->Kc * CS, 0.0);
    {
        std::vector<double> M((size_t)NP * NP), Mi((size_t)NP * NP);
        const double drdt[3] = {1.0, -1.0, 0.0}, dsdt[3] = {0.0, 1.0, -1.0};
        for (long long c = 0; c < m->Kc; ++c) {
            const long long k = m->perm[m->Kaff + c];
            const double* X = node_xy + (size_t)k * NP * 2;
            double* g = geoC.data() + (size_t)c * CS;
            std::vector<double> J(NQ);
            for (int q = 0; q < NQ; ++q) {
                double xr = 0, xs = 0, yr = 0, ys = 0;
                for (int j = 0; j < NP; ++j) {
                    xr += R->Dr[(size_t)q * NP + j] * X[2 * j];
                    xs += R->Ds[(size_t)q * NP + j] * X[2 * j];
                    yr += R->Dr[(size_t)q * NP + j] * X[2 * j + 1];
                    ys += R->Ds[(size_t)q * NP + j] * X[2 * j + 1];
                }
                J[q] = xr * ys - xs * yr;
                if (!(J[q] > 0.0)) {
                    free_mesh(m);
                    pr->m = nullptr;
                    return fail(ctx, DG_EINVAL, "non-positive Jacobian at a cubature node of element " +
                                                    std::to_string(k));
                }
                g[q] = ys; g[NQ + q] = -xs; g[2 * NQ + q] = -yr; g[3 * NQ + q] = xr; g[4 * NQ + q] = J[q];
            }
            for (int fg = 0; fg < NF; ++fg) {
                const int f = fg / NG;
                double xr = 0, xs = 0, yr = 0, ys = 0;
                for (int j = 0; j < NP; ++j) {
                    xr += R->Drg[(size_t)fg * NP + j] * X[2 * j];
                    xs += R->Dsg[(size_t)fg * NP + j] * X[2 * j];
                    yr += R->Drg[(size_t)fg * NP + j] * X[2 * j + 1];
                    ys += R->Dsg[(size_t)fg * NP + j] * X[2 * j + 1];
                }
                const double xt = xr * drdt[f] + xs * dsdt[f], yt = yr * drdt[f] + ys * dsdt[f];
                const double sJ = std::sqrt(xt * xt + yt * yt);
                g[5 * NQ + fg] = yt / sJ;
                g[5 * NQ + NF + fg] = -xt / sJ;
                g[5 * NQ + 2 * NF + fg] = sJ;
            }
            for (int i = 0; i < NP; ++i)
                for (int j = 0; j < NP; ++j) {
                    double v = 0;
                    for (int q = 0; q < NQ; ++q)
                        v += R->Icub[(size_t)q * NP + i] * R->wq[q] * J[q] * R->Icub[(size_t)q * NP + j];
                    M[(size_t)i * NP + j] = v;
                }
            if (!spd_inverse(M.data(), Mi.data(), NP)) {
                free_mesh(m);
                pr->m = nullptr;
                return fail(ctx, DG_EINVAL, "curved mass matrix not SPD at element " + std::to_string(k));
            }
            for (int j = 0; j < NP; ++j)
                for (int i = 0; i < NP; ++i) g[5 * NQ + 3 * NF + j * NP + i] = Mi[(size_t)i * NP + j];
        }
    }
    pr->R = R;
    return DG_OK;
}

// The device half of an upload: buffers, operator tables, copies.  The
// prepared host mesh moves into the context on success.
static int upload_prepared(dg_ctx* ctx, dg_prepared* pr, dg_mesh* out) {
    MeshData* m = pr->m;
    const RefOps* R = pr->R;
    const dg_params* p = &m->p;
    const int N = m->N, NP = m->Np;
    const int64_t K = m->K;
    const std::vector<long long>& iperm = pr->iperm;
    const std::vector<int4>& conn = pr->conn;
    const std::vector<double>& geoA = pr->geoA;
    const std::vector<double>& geoC = pr->geoC;
    pr->m = nullptr;   // from here on freed by this function or owned by the context
    // device buffers
    cudaSetDevice(ctx->device);
    const size_t rs = m->rsize, nstate = (size_t)K * 4 * NP;
    int e;
    for (int b = 0; b < 3; ++b)
        if ((e = alloc(ctx, *m, &m->U[b], nstate * rs))) { free_mesh(m); return e; }
    if ((e = alloc(ctx, *m, &m->rhs, nstate * rs))) { free_mesh(m); return e; }
    if ((e = alloc(ctx, *m, (void**)&m->conn, (size_t)K * sizeof(int4)))) { free_mesh(m); return e; }
    if ((e = alloc(ctx, *m, &m->geoA, geoA.size() * rs))) { free_mesh(m); return e; }
    if ((e = alloc(ctx, *m, &m->geoC, geoC.size() * rs))) { free_mesh(m); return e; }
    if ((e = alloc(ctx, *m, (void**)&m->dperm, (size_t)K * sizeof(long long)))) { free_mesh(m); return e; }
    if ((e = alloc(ctx, *m, (void**)&m->diperm, (size_t)K * sizeof(long long)))) { free_mesh(m); return e; }
    if ((e = alloc(ctx, *m, (void**)&m->red, (size_t)(residual_blocks() * 10 + 10) * sizeof(double)))) {
        free_mesh(m);
        return e;
    }
    // error word, the persistent kernels' tile / done counters, viscous counts
    if ((e = alloc(ctx, *m, (void**)&m->err, ERR_WORDS * sizeof(int)))) { free_mesh(m); return e; }
    if (cudaMemset(m->err, 0, ERR_WORDS * sizeof(int)) != cudaSuccess) {
        free_mesh(m);
        return fail(ctx, DG_ECUDA, "memset failed");
    }
    if (tensor_prec(p->prec)) {
        const int tkey = N * 16 + 4 + p->prec;
        auto tit = ctx->ops.find(tkey);
        if (tit == ctx->ops.end()) {
            const std::vector<uint8_t> packed = dispatch_pack_tc(N, *R, p->prec == DG_TF32 ? 1 : 2);
            if (packed.empty()) {
                free_mesh(m);
                return fail(ctx, DG_EINVAL, "face traces do not reduce to the face nodes");
            }
            void* d = nullptr;
            if (cudaMalloc(&d, packed.size()) != cudaSuccess) {
                cudaGetLastError();
                free_mesh(m);
                return fail(ctx, DG_ENOMEM, "tensor-core operator table allocation failed");
            }
            if (cudaMemcpy(d, packed.data(), packed.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
                cudaFree(d);
                free_mesh(m);
                return fail(ctx, DG_ECUDA, "tensor-core operator table copy failed");
            }
            ctx->ops[tkey] = d;
            const int pe = dispatch_prepare_tc(N);
            if (pe) {
                free_mesh(m);
                return fail(ctx, DG_ECUDA, "tensor-core kernel attribute set-up failed");
            }
            tit = ctx->ops.find(tkey);
        }
        m->ops_tc = tit->second;
    }
    if (p->av_on) {
        // padded to whole tiles of 32: the tensor-core kernels copy eps per tile
        const size_t eb = (size_t)((K + 31) / 32 * 32) * rs;
        if ((e = alloc(ctx, *m, &m->eps, eb))) { free_mesh(m); return e; }
        m->eps_ring[0] = m->eps;
        if (tensor_prec(p->prec))
            for (int b = 1; b < EPS_RING; ++b)
                if ((e = alloc(ctx, *m, &m->eps_ring[b], eb))) { free_mesh(m); return e; }
        if ((e = alloc(ctx, *m, &m->q, (size_t)K * 8 * NP * rs))) { free_mesh(m); return e; }
    }
    // operators (shared per context, degree and precision)
    const int okey = N * 16 + (m->rsize == 8 ? 1 : 0);
    auto oit = ctx->ops.find(okey);
    if (oit == ctx->ops.end()) {
        const std::vector<double> packed = pack_ops(*R);
        void* d = nullptr;
        if (cudaMalloc(&d, packed.size() * rs) != cudaSuccess) {
            cudaGetLastError();
            free_mesh(m);
            return fail(ctx, DG_ENOMEM, "operator table allocation failed");
        }
        cudaError_t ce;
        if (rs == 8)
            ce = cudaMemcpy(d, packed.data(), packed.size() * 8, cudaMemcpyHostToDevice);
        else {
            const auto f = to_real<float>(packed);
            ce = cudaMemcpy(d, f.data(), f.size() * 4, cudaMemcpyHostToDevice);
        }
        if (ce != cudaSuccess) {
            cudaFree(d);
            free_mesh(m);
            return fail(ctx, DG_ECUDA, "operator table copy failed");
        }
        ctx->ops[okey] = d;
        const int pe = (rs == 8) ? dispatch_prepare<double>(N) : dispatch_prepare<float>(N);
        if (pe) {
            free_mesh(m);
            return fail(ctx, DG_ECUDA, std::string("kernel attribute set-up failed: ") +
                                           cudaGetErrorString((cudaError_t)pe));
        }
        oit = ctx->ops.find(okey);
    }
    m->ops = oit->second;

    auto upload = [&](void* dst, const std::vector<double>& src) -> cudaError_t {
        if (src.empty()) return cudaSuccess;
        if (rs == 8) return cudaMemcpy(dst, src.data(), src.size() * 8, cudaMemcpyHostToDevice);
        const auto f = to_real<float>(src);
        return cudaMemcpy(dst, f.data(), f.size() * 4, cudaMemcpyHostToDevice);
    };
    if (upload(m->geoA, geoA) != cudaSuccess || upload(m->geoC, geoC) != cudaSuccess ||
        cudaMemcpy(m->conn, conn.data(), (size_t)K * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m->dperm, m->perm.data(), (size_t)K * sizeof(long long), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m->diperm, iperm.data(), (size_t)K * sizeof(long long), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(m->U[0], 0, nstate * rs) != cudaSuccess) {
        free_mesh(m);
        return fail(ctx, DG_ECUDA, "mesh upload copy failed");
    }
    for (int b = 1; b < EPS_RING; ++b)
        if (m->eps_ring[b] && cudaMemset(m->eps_ring[b], 0, (size_t)((K + 31) / 32 * 32) * rs) != cudaSuccess) {
            free_mesh(m);
            return fail(ctx, DG_ECUDA, "mesh upload memset failed");
        }
    if (p->av_on && (cudaMemset(m->eps, 0, (size_t)((K + 31) / 32 * 32) * rs) != cudaSuccess ||
                     cudaMemset(m->q, 0, (size_t)K * 8 * NP * rs) != cudaSuccess)) {
        free_mesh(m);
        return fail(ctx, DG_ECUDA, "mesh upload memset failed");
    }
    if (!tensor_prec(m->prec)) {   // a tile size tuned earlier for this kind of mesh
        auto it = ctx->tuned_e.find(tune_key(m->dim, m->N, m->rsize, m->p.av_on));
        if (it != ctx->tuned_e.end()) m->tile_e = it->second;
    } else {                       // a tile-pipeline configuration tuned earlier
        auto it = ctx->tuned_e.find(tune_key(m->dim, m->N, 16 + m->prec, m->p.av_on));
        if (it != ctx->tuned_e.end()) m->tc_cfg = it->second;
    }
    // the copies and memsets above ran on the legacy default stream, which
    // the context's non-blocking stream does not wait for: complete them
    // before any work of the context can touch the mesh
    if (cudaStreamSynchronize(cudaStreamLegacy) != cudaSuccess) {
        free_mesh(m);
        return fail(ctx, DG_ECUDA, "mesh upload synchronisation failed");
    }
    const dg_mesh h = ctx->next_id++;
    ctx->meshes[h] = m;
    *out = h;
    return DG_OK;
}

static int dg_mesh_upload_body(dg_ctx* ctx, int N, int64_t K, const int32_t* EToE, const int8_t* EToF, const int8_t* bc,
                               const double* node_xy, const dg_params* p, dg_mesh* out) {
    if (!ctx) return fail(nullptr, DG_EINVAL, "ctx is NULL");
    if (!out) return fail(ctx, DG_EINVAL, "NULL argument");
    dg_prepared pr;
    const int e = prepare_mesh(ctx, N, K, EToE, EToF, bc, node_xy, p, &pr);
    if (e) return e;
    return upload_prepared(ctx, &pr, out);
}

int dg_mesh_upload(dg_ctx* ctx, int N, int64_t K, const int32_t* EToE, const int8_t* EToF, const int8_t* bc,
                   const double* node_xy, const dg_params* p, dg_mesh* out) {
    try {
        return dg_mesh_upload_body(ctx, N, K, EToE, EToF, bc, node_xy, p, out);
    } catch (...) {
        return exception_status(ctx);
    }
}

static int dg_mesh_prepare_body(int N, int64_t K, const int32_t* EToE, const int8_t* EToF, const int8_t* bc,
                                const double* node_xy, const dg_params* p, dg_prepared** out) {
    if (!out) return fail(nullptr, DG_EINVAL, "NULL argument");
    *out = nullptr;
    auto* pr = new dg_prepared();
    const int e = prepare_mesh(nullptr, N, K, EToE, EToF, bc, node_xy, p, pr);
    if (e) {
        delete pr;
        return e;
    }
    *out = pr;
    return DG_OK;
}

int dg_mesh_prepare(int N, int64_t K, const int32_t* EToE, const int8_t* EToF, const int8_t* bc,
                    const double* node_xy, const dg_params* p, dg_prepared** out) {
    try {
        return dg_mesh_prepare_body(N, K, EToE, EToF, bc, node_xy, p, out);
    } catch (...) {
        return exception_status(nullptr);
    }
}

static int dg_mesh_upload_prepared_body(dg_ctx* ctx, dg_prepared* prep, dg_mesh* out) {
    if (!prep) return fail(ctx, DG_EINVAL, "NULL prepared mesh");
    if (!ctx || !out || !prep->m) {
        dg_prepared_free(prep);
        return fail(ctx, DG_EINVAL, !prep->m ? "prepared mesh already uploaded" : "NULL argument");
    }
    const int e = upload_prepared(ctx, prep, out);
    delete prep;
    return e;
}

int dg_mesh_upload_prepared(dg_ctx* ctx, dg_prepared* prep, dg_mesh* out) {
    try {
        return dg_mesh_upload_prepared_body(ctx, prep, out);
    } catch (...) {
        return exception_status(ctx);
    }
}

int dg_prepared_free(dg_prepared* prep) {
    if (!prep) return DG_OK;
    if (prep->m) free_mesh(prep->m);
    delete prep;
    return DG_OK;
}

int dg_mesh_free(dg_ctx* ctx, dg_mesh h) {
    if (!ctx) return fail(nullptr, DG_EINVAL, "ctx is NULL");
    MeshData* m = find(ctx, h);
    if (!m) return fail(ctx, DG_ENOTFOUND, "unknown mesh handle");
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    free_mesh(m);
    ctx->meshes.erase(h);
    reset_batch(ctx);
    return DG_OK;
}

int dg_mesh_bytes(dg_ctx* ctx, dg_mesh h, int64_t* out) {
    if (!ctx || !out) return fail(ctx, DG_EINVAL, "NULL argument");
    MeshData* m = find(ctx, h);
    if (!m) return fail(ctx, DG_ENOTFOUND, "unknown mesh handle");
    *out = (int64_t)m->bytes;
    return DG_OK;
}

// host FP64 canonical <-> device order in the mesh precision.  Staged
// (DG_HOST_IO_STAGED): the rows are converted and reordered by up to 16
// host threads (about a million values or more each) in a host buffer,
// which is copied to or from the device in one transfer.  Device
// (DG_HOST_IO_DEVICE, where the device reaches pageable host memory
// coherently): one kernel reads (writes) the caller's FP64 rows in place,
// converting and reordering them on the device; the call returns when it
// has completed.
static void parallel_rows(long long K, size_t row, const std::function<void(long long, long long)>& body) {
    const size_t n = (size_t)K * row;
    unsigned T = std::thread::hardware_concurrency();
    T = std::max(1u, std::min(std::min(T, 16u), (unsigned)std::min<size_t>(n >> 20, 1u << 20) + 1u));
    if (T <= 1) {
        body(0LL, K);
        return;
    }
    const long long per = (K + T - 1) / T;
    std::vector<std::thread> th;
    th.reserve(T);
    for (unsigned t = 0; t < T; ++t) {
        const long long d0 = (long long)t * per, d1 = std::min<long long>(K, d0 + per);
        if (d0 >= d1) break;
        try {
            th.emplace_back([&body, d0, d1] { body(d0, d1); });
        } catch (...) {   // no thread to be had: the remaining rows on this one
            body(d0, K);
            break;
        }
    }
    for (auto& x : th) x.join();
}

static int put_host(dg_ctx* ctx, MeshData* m, const double* U, void* dst) {
    const size_t row = (size_t)m->nvar * m->Np, n = (size_t)m->K * row;
    const long long* perm = m->perm.data();
    cudaError_t ce;
    if (ctx->host_io == DG_HOST_IO_DEVICE) {   // device row d <- canonical row perm[d]
        const int e = m->rsize == 8
                          ? launch_gather_convert<double, double>(U, (double*)dst, m->dperm, m->K, (int)row, ctx->stream)
                          : launch_gather_convert<double, float>(U, (float*)dst, m->dperm, m->K, (int)row, ctx->stream);
        ce = e ? (cudaError_t)e : cudaStreamSynchronize(ctx->stream);
    } else if (m->rsize == 8) {
        std::unique_ptr<double[]> buf(new double[n]);   // not zero-filled: every value is written
        double* b = buf.get();
        parallel_rows(m->K, row, [&](long long d0, long long d1) {
            for (long long d = d0; d < d1; ++d) std::memcpy(&b[d * row], U + perm[d] * row, row * 8);
        });
        ce = cudaMemcpyAsync(dst, buf.get(), n * 8, cudaMemcpyHostToDevice, ctx->stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
    } else {
        std::unique_ptr<float[]> buf(new float[n]);   // not zero-filled: every value is written
        float* b = buf.get();
        parallel_rows(m->K, row, [&](long long d0, long long d1) {
            for (long long d = d0; d < d1; ++d)
                for (size_t i = 0; i < row; ++i) b[d * row + i] = (float)U[perm[d] * row + i];
        });
        ce = cudaMemcpyAsync(dst, buf.get(), n * 4, cudaMemcpyHostToDevice, ctx->stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
    }
    if (ce != cudaSuccess) return fail(ctx, DG_ECUDA, std::string("state upload: ") + cudaGetErrorString(ce));
    return DG_OK;
}

static int get_host(dg_ctx* ctx, MeshData* m, const void* src, double* U) {
    const size_t row = (size_t)m->nvar * m->Np, n = (size_t)m->K * row;
    const long long* perm = m->perm.data();
    cudaError_t ce;
    if (ctx->host_io == DG_HOST_IO_DEVICE) {   // canonical row k <- device row iperm[k]
        const int e = m->rsize == 8
                          ? launch_gather_convert<double, double>((const double*)src, U, m->diperm, m->K, (int)row,
                                                                  ctx->stream)
                          : launch_gather_convert<float, double>((const float*)src, U, m->diperm, m->K, (int)row,
                                                                 ctx->stream);
        ce = e ? (cudaError_t)e : cudaStreamSynchronize(ctx->stream);
    } else if (m->rsize == 8) {
        std::unique_ptr<double[]> buf(new double[n]);   // not zero-filled: every value is written
        ce = cudaMemcpyAsync(buf.get(), src, n * 8, cudaMemcpyDeviceToHost, ctx->stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
        if (ce == cudaSuccess) {
            const double* b = buf.get();
            parallel_rows(m->K, row, [&](long long d0, long long d1) {
                for (long long d = d0; d < d1; ++d) std::memcpy(U + perm[d] * row, &b[d * row], row * 8);
            });
        }
    } else {
        std::unique_ptr<float[]> buf(new float[n]);   // not zero-filled: every value is written
        ce = cudaMemcpyAsync(buf.get(), src, n * 4, cudaMemcpyDeviceToHost, ctx->stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
        if (ce == cudaSuccess) {
            const float* b = buf.get();
            parallel_rows(m->K, row, [&](long long d0, long long d1) {
                for (long long d = d0; d < d1; ++d)
                    for (size_t i = 0; i < row; ++i) U[perm[d] * row + i] = b[d * row + i];
            });
        }
    }
    if (ce != cudaSuccess) return fail(ctx, DG_ECUDA, std::string("state download: ") + cudaGetErrorString(ce));
    return DG_OK;
}

static int dg_set_state_body(dg_ctx* ctx, dg_mesh h, const double* U) {
    if (!ctx || !U) return fail(ctx, DG_EINVAL, "NULL argument");
    MeshData* m = find(ctx, h);
    if (!m) return fail(ctx, DG_ENOTFOUND, "unknown mesh handle");
    cudaSetDevice(ctx->device);
    m->eps_valid = false;
    return put_host(ctx, m, U, m->U[0]);
}

int dg_set_state(dg_ctx* ctx, dg_mesh h, const double* U) {
    try {
        return dg_set_state_body(ctx, h, U);
    } catch (...) {
        return exception_status(ctx);
    }
}

static int dg_get_state_body(dg_ctx* ctx, dg_mesh h, double* U_out) {
    if (!ctx || !U_out) return fail(ctx, DG_EINVAL, "NULL argument");
    MeshData* m = find(ctx, h);
    if (!m) return fail(ctx, DG_ENOTFOUND, "unknown mesh handle");
    cudaSetDevice(ctx->device);
    return get_host(ctx, m, m->U[0], U_out);
}

int dg_get_state(dg_ctx* ctx, dg_mesh h, double* U_out) {
    try {
        return dg_get_state_body(ctx, h, U_out);
    } catch (...) {
        return exception_status(ctx);
    }
}

int dg_set_state_device(dg_ctx* ctx, dg_mesh h, const float* U_dev) {
    if (!ctx || !U_dev) return fail(ctx, DG_EINVAL, "NULL argument");
    MeshData* m = find(ctx, h);
    if (!m) return fail(ctx, DG_ENOTFOUND, "unknown mesh handle");
    if (m->rsize != 4) return fail(ctx, DG_EINVAL, "device state I/O needs an FP32 precision mode");
    cudaSetDevice(ctx->device);
    m->eps_valid = false;
    // device row d <- canonical row perm[d]
    int e = launch_permute<float>(U_dev, (float*)m->U[0], m->dperm, m->K, m->nvar * m->Np, ctx->stream);
    if (e) return fail(ctx, DG_ECUDA, cudaGetErrorString((cudaError_t)e));
    return DG_OK;
}

int dg_get_state_device(dg_ctx* ctx, dg_mesh h, float* U_dev_out) {
    if (!ctx || !U_dev_out) return fail(ctx, DG_EINVAL, "NULL argument");
    MeshData* m = find(ctx, h);
    if (!m) return fail(ctx, DG_ENOTFOUND, "unknown mesh handle");
    if (m->rsize != 4) return fail(ctx, DG_EINVAL, "device state I/O needs an FP32 precision mode");
    cudaSetDevice(ctx->device);
    // canonical row k <- device row iperm[k]
    int e = launch_permute<float>((const float*)m->U[0], U_dev_out, m->diperm, m->K, m->nvar * m->Np, ctx->stream);
    if (e) return fail(ctx, DG_ECUDA, cudaGetErrorString((cudaError_t)e));
    return DG_OK;
}

static int dg_eval_rhs_body(dg_ctx* ctx, dg_mesh h, double* rhs_out) {
    if (!ctx || !rhs_out) return fail(ctx, DG_EINVAL, "NULL argument");
    MeshData* m = find(ctx, h);
    if (!m) return fail(ctx, DG_ENOTFOUND, "unknown mesh handle");
    cudaSetDevice(ctx->device);
    int e = enqueue_stage(*m, m->U[0], nullptr, m->rhs, 0.0, 0.0, 0.0, 1, ctx->stream);
    if (e) return fail(ctx, DG_ECUDA, std::string("stage launch: ") + cudaGetErrorString((cudaError_t)e));
    return get_host(ctx, m, m->rhs, rhs_out);
}

int dg_eval_rhs(dg_ctx* ctx, dg_mesh h, double* rhs_out) {
    try {
        return dg_eval_rhs_body(ctx, h, rhs_out);
    } catch (...) {
        return exception_status(ctx);
    }
}

static int dg_step_body(dg_ctx* ctx, dg_mesh h, double dt, int nsteps) {
    if (!ctx) return fail(nullptr, DG_EINVAL, "ctx is NULL");
    MeshData* m = find(ctx, h);
    if (!m) return fail(ctx, DG_ENOTFOUND, "unknown mesh handle");
    if (nsteps < 0 || !std::isfinite(dt)) return fail(ctx, DG_EINVAL, "bad dt or nsteps");
    if (nsteps == 0) return DG_OK;
    cudaSetDevice(ctx->device);
    if (!m->gexec || m->gdt != dt) {
        if (m->gexec) { cudaGraphExecDestroy(m->gexec); m->gexec = nullptr; }
        if (m->graph) { cudaGraphDestroy(m->graph); m->graph = nullptr; }
        CUDA_OK(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        m->prof_next = 0;
        m->prof_capturing = m->profiling;
        const int e = enqueue_step(*m, dt, ctx->stream);
        m->prof_capturing = false;   // no event records outside the profiled step graph
        m->prof_count = m->profiling ? m->prof_next : 0;
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(ctx->stream, &g);
        if (e || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return fail(ctx, DG_ECUDA, "graph capture of the RK step failed");
        }
        m->graph = g;
        CUDA_OK(ctx, cudaGraphInstantiate(&m->gexec, g, 0));
        m->gdt = dt;
    }
    if (fused_sensor(*m) && !m->eps_valid) {   // eps(U^n) for the first stage, with its viscous count
        CUDA_OK(ctx, cudaMemsetAsync(m->err + VISC_SLOT, 0, sizeof(int), ctx->stream));
        const int e = enqueue_sensor(*m, m->U[0], m->eps_ring[0], ctx->stream, m->err + VISC_SLOT);
        if (e) return fail(ctx, DG_ECUDA, std::string("sensor launch failed: ") + cudaGetErrorString((cudaError_t)e));
        m->eps_valid = true;
    }
    for (int s = 0; s < nsteps; ++s) CUDA_OK(ctx, cudaGraphLaunch(m->gexec, ctx->stream));
    return DG_OK;
}

int dg_step(dg_ctx* ctx, dg_mesh h, double dt, int nsteps) {
    try {
        return dg_step_body(ctx, h, dt, nsteps);
    } catch (...) {
        return exception_status(ctx);
    }
}

int dg_residual(dg_ctx* ctx, dg_mesh h, double* out_linf, double* out_l2) {
    if (!ctx || !out_linf || !out_l2) return fail(ctx, DG_EINVAL, "NULL argument");
    MeshData* m = find(ctx, h);
    if (!m) return fail(ctx, DG_ENOTFOUND, "unknown mesh handle");
    cudaSetDevice(ctx->device);
    int e = enqueue_stage(*m, m->U[0], nullptr, m->rhs, 0.0, 0.0, 0.0, 1, ctx->stream);
    if (e) return fail(ctx, DG_ECUDA, std::string("stage launch failed: ") + cudaGetErrorString((cudaError_t)e));
    const int nv = m->nvar;
    double* out = m->red + residual_blocks() * 10;
    if (m->rsize == 8)
        e = launch_residual<double>((const double*)m->rhs, nv, m->K, m->Np, m->red, out, ctx->stream);
    else
        e = launch_residual<float>((const float*)m->rhs, nv, m->K, m->Np, m->red, out, ctx->stream);
    if (e) return fail(ctx, DG_ECUDA, "residual launch failed");
    double hv[10];
    CUDA_OK(ctx, cudaMemcpyAsync(hv, out, 2 * nv * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_OK(ctx, cudaStreamSynchronize(ctx->stream));
    bool finite = true;
    for (int v = 0; v < nv; ++v) {
        out_linf[v] = hv[v];
        out_l2[v] = hv[nv + v];
        finite = finite && std::isfinite(hv[v]) && std::isfinite(hv[nv + v]);
    }
    return finite ? DG_OK : fail(ctx, DG_ENONFINITE, "non-finite residual norm");
}

static int dg_batch_residual_body(dg_ctx* ctx, int n, const dg_mesh* hs, double* out10) {
    if (!ctx || n <= 0 || !hs || !out10) return fail(ctx, DG_EINVAL, "bad argument");
    std::vector<MeshData*> ms(n);
    for (int i = 0; i < n; ++i) {
        ms[i] = find(ctx, hs[i]);
        if (!ms[i]) return fail(ctx, DG_ENOTFOUND, "unknown mesh handle");
    }
    cudaSetDevice(ctx->device);
    if (ctx->res_host_n < n) {   // pinned host slots, one per mesh
        if (ctx->res_host) cudaFreeHost(ctx->res_host);
        ctx->res_host = nullptr;
        ctx->res_host_n = 0;
        CUDA_OK(ctx, cudaMallocHost((void**)&ctx->res_host, (size_t)n * 10 * sizeof(double)));
        ctx->res_host_n = n;
    }
    for (int i = 0; i < n; ++i) {
        MeshData* m = ms[i];
        int e = enqueue_stage(*m, m->U[0], nullptr, m->rhs, 0.0, 0.0, 0.0, 1, ctx->stream);
        if (e) return fail(ctx, DG_ECUDA, std::string("stage launch failed: ") + cudaGetErrorString((cudaError_t)e));
        double* dout = m->red + residual_blocks() * 10;
        if (m->rsize == 8)
            e = launch_residual<double>((const double*)m->rhs, m->nvar, m->K, m->Np, m->red, dout, ctx->stream);
        else
            e = launch_residual<float>((const float*)m->rhs, m->nvar, m->K, m->Np, m->red, dout, ctx->stream);
        if (e) return fail(ctx, DG_ECUDA, "residual launch failed");
        CUDA_OK(ctx, cudaMemcpyAsync(ctx->res_host + 10 * i, dout, 2 * m->nvar * sizeof(double),
                                     cudaMemcpyDeviceToHost, ctx->stream));
    }
    CUDA_OK(ctx, cudaStreamSynchronize(ctx->stream));
    bool finite = true;
    for (int i = 0; i < n; ++i) {
        const int nv = ms[i]->nvar;
        const double* hv = ctx->res_host + 10 * i;
        double* o = out10 + 10 * i;
        for (int v = 0; v < 5; ++v) {
            o[v] = v < nv ? hv[v] : 0.0;
            o[5 + v] = v < nv ? hv[nv + v] : 0.0;
            if (v < nv) finite = finite && std::isfinite(hv[v]) && std::isfinite(hv[nv + v]);
        }
    }
    return finite ? DG_OK : fail(ctx, DG_ENONFINITE, "non-finite residual norm");
}

int dg_batch_residual(dg_ctx* ctx, int n, const dg_mesh* hs, double* out10) {
    try {
        return dg_batch_residual_body(ctx, n, hs, out10);
    } catch (...) {
        return exception_status(ctx);
    }
}

int dg_av_count(dg_ctx* ctx, dg_mesh h, int64_t* out) {
    if (!ctx || !out) return fail(ctx, DG_EINVAL, "NULL argument");
    MeshData* m = find(ctx, h);
    if (!m) return fail(ctx, DG_ENOTFOUND, "unknown mesh handle");
    if (!m->p.av_on) return fail(ctx, DG_EINVAL, "the mesh has no artificial viscosity");
    cudaSetDevice(ctx->device);
    if (m->dim == 3) {   // the sensor of U^n into the scratch, counted on the host
        const int e = m->rsize == 8
            ? launch_sensor3(m->N, (const double*)m->U[0], (double*)m->rhs, (const double*)m->ops,
                             (const double*)m->ops_av3, (const double*)m->geoC, m->K, m->Kaff, m->p.kappa,
                             m->p.eps0, m->s0, ctx->stream)
            : launch_sensor3(m->N, (const float*)m->U[0], (float*)m->rhs, (const float*)m->ops,
                             (const float*)m->ops_av3, (const float*)m->geoC, m->K, m->Kaff, m->p.kappa,
                             m->p.eps0, m->s0, ctx->stream);
        if (e) return fail(ctx, DG_ECUDA, std::string("sensor launch failed: ") + cudaGetErrorString((cudaError_t)e));
        std::vector<double> ev((size_t)m->K);
        if (m->rsize == 8) {
            CUDA_OK(ctx, cudaMemcpyAsync(ev.data(), m->rhs, (size_t)m->K * 8, cudaMemcpyDeviceToHost, ctx->stream));
            CUDA_OK(ctx, cudaStreamSynchronize(ctx->stream));
        } else {
            std::vector<float> ef((size_t)m->K);
            CUDA_OK(ctx, cudaMemcpyAsync(ef.data(), m->rhs, (size_t)m->K * 4, cudaMemcpyDeviceToHost, ctx->stream));
            CUDA_OK(ctx, cudaStreamSynchronize(ctx->stream));
            ev.assign(ef.begin(), ef.end());
        }
        int64_t c = 0;
        for (double x : ev) c += x > 0.0;
        *out = c;
        return DG_OK;
    }
    // the sensor of U^n into the right-hand-side scratch, counting its
    // elements with eps > 0 in a scratch word of the error block
    int* cnt = m->err + VISC_SLOT + EPS_RING;
    CUDA_OK(ctx, cudaMemsetAsync(cnt, 0, sizeof(int), ctx->stream));
    const int e = enqueue_sensor(*m, m->U[0], m->rhs, ctx->stream, cnt);
    if (e) return fail(ctx, DG_ECUDA, std::string("sensor launch failed: ") + cudaGetErrorString((cudaError_t)e));
    int hv = 0;
    CUDA_OK(ctx, cudaMemcpyAsync(&hv, cnt, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_OK(ctx, cudaStreamSynchronize(ctx->stream));
    *out = hv;
    return DG_OK;
}

int dg_sync(dg_ctx* ctx, double timeout_s) {
    if (!ctx) return fail(nullptr, DG_EINVAL, "ctx is NULL");
    cudaSetDevice(ctx->device);
    if (timeout_s <= 0) {
        CUDA_OK(ctx, cudaStreamSynchronize(ctx->stream));
        return check_device_errors(ctx);
    }
    const auto t0 = std::chrono::steady_clock::now();
    while (true) {
        const cudaError_t q = cudaStreamQuery(ctx->stream);
        if (q == cudaSuccess) return check_device_errors(ctx);
        if (q != cudaErrorNotReady) return fail(ctx, DG_ECUDA, cudaGetErrorString(q));
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > timeout_s) return fail(ctx, DG_ETIMEOUT, "work still in flight after the timeout");
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
}

int dg_selftest_bounded_wait(dg_ctx* ctx, uint32_t limit, int arrive, int32_t* out) {
    if (!ctx || !out) return fail(ctx, DG_EINVAL, "NULL argument");
    if (limit == 0 || limit > (1u << 26)) return fail(ctx, DG_EINVAL, "limit must be in 1..2^26");
    cudaSetDevice(ctx->device);
    int* d = nullptr;
    CUDA_OK(ctx, cudaMalloc(&d, sizeof(int)));
    int h = -1;
    cudaError_t e = cudaMemsetAsync(d, 0xff, sizeof(int), ctx->stream);
    if (e == cudaSuccess) e = (cudaError_t)launch_bounded_wait(limit, arrive ? 1 : 0, d, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(d);
    if (e != cudaSuccess) return fail(ctx, DG_ECUDA, std::string("bounded-wait self-test: ") + cudaGetErrorString(e));
    *out = h;
    return DG_OK;
}

static int dg_step_lserk_body(dg_ctx* ctx, dg_mesh h, double dt, int nsteps) {
    if (!ctx) return fail(nullptr, DG_EINVAL, "ctx is NULL");
    MeshData* m = find(ctx, h);
    if (!m) return fail(ctx, DG_ENOTFOUND, "unknown mesh handle");
    if (nsteps < 0 || !std::isfinite(dt)) return fail(ctx, DG_EINVAL, "bad dt or nsteps");
    if (nsteps == 0) return DG_OK;
    cudaSetDevice(ctx->device);
    if (!m->gexec_ls || m->gdt_ls != dt) {
        if (m->gexec_ls) { cudaGraphExecDestroy(m->gexec_ls); m->gexec_ls = nullptr; }
        if (m->graph_ls) { cudaGraphDestroy(m->graph_ls); m->graph_ls = nullptr; }
        CUDA_OK(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        m->prof_capturing = false;
        const int e = enqueue_step_lserk(*m, dt, ctx->stream);
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(ctx->stream, &g);
        if (e || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return fail(ctx, DG_ECUDA, "graph capture of the low-storage RK step failed");
        }
        m->graph_ls = g;
        CUDA_OK(ctx, cudaGraphInstantiate(&m->gexec_ls, g, 0));
        m->gdt_ls = dt;
    }
    if (fused_sensor(*m) && !m->eps_valid) {   // eps(U^n) for the first stage, with its viscous count
        CUDA_OK(ctx, cudaMemsetAsync(m->err + VISC_SLOT, 0, sizeof(int), ctx->stream));
        const int e = enqueue_sensor(*m, m->U[0], m->eps_ring[0], ctx->stream, m->err + VISC_SLOT);
        if (e) return fail(ctx, DG_ECUDA, std::string("sensor launch failed: ") + cudaGetErrorString((cudaError_t)e));
        m->eps_valid = true;
    }
    for (int s = 0; s < nsteps; ++s) CUDA_OK(ctx, cudaGraphLaunch(m->gexec_ls, ctx->stream));
    return DG_OK;
}

int dg_step_lserk(dg_ctx* ctx, dg_mesh h, double dt, int nsteps) {
    try {
        return dg_step_lserk_body(ctx, h, dt, nsteps);
    } catch (...) {
        return exception_status(ctx);
    }
}

static int dg_prolong_body(dg_ctx* ctx, dg_mesh from, dg_mesh to) {
    if (!ctx) return fail(nullptr, DG_EINVAL, "ctx is NULL");
    MeshData* a = find(ctx, from);
    MeshData* b = find(ctx, to);
    if (!a || !b) return fail(ctx, DG_ENOTFOUND, "unknown mesh handle");
    if (a == b || a->dim != b->dim || a->K != b->K || a->N > b->N || a->rsize != b->rsize)
        return fail(ctx, DG_EINVAL,
                    "prolongation needs two uploads of one mesh, the target of degree >= the source, one state type");
    // the device orders of the two uploads (affine elements first) may
    // differ where an element is curved at one degree only: target element
    // d takes source element src[d]
    std::vector<long long> src;
    if (a->perm != b->perm) {
        std::vector<long long> ia((size_t)a->K);
        for (long long d = 0; d < a->K; ++d) ia[(size_t)a->perm[d]] = d;
        src.resize((size_t)b->K);
        for (long long d = 0; d < b->K; ++d) src[(size_t)d] = ia[(size_t)b->perm[d]];
    }
    std::vector<double> P;
    std::string err;
    const bool ok = a->dim == 3 ? build_prolongation3(a->N, b->N, P, err) : build_prolongation(a->N, b->N, P, err);
    if (!ok) return fail(ctx, DG_EINVAL, err);
    cudaSetDevice(ctx->device);
    void* dP = nullptr;
    const size_t rs = a->rsize;
    if (cudaMalloc(&dP, P.size() * rs) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, DG_ENOMEM, "prolongation operator allocation failed");
    }
    cudaError_t ce;
    if (rs == 8) {
        ce = cudaMemcpy(dP, P.data(), P.size() * 8, cudaMemcpyHostToDevice);
    } else {
        std::vector<float> Pf(P.begin(), P.end());
        ce = cudaMemcpy(dP, Pf.data(), Pf.size() * 4, cudaMemcpyHostToDevice);
    }
    long long* dsrc = nullptr;
    if (ce == cudaSuccess && !src.empty()) {
        ce = cudaMalloc((void**)&dsrc, src.size() * sizeof(long long));
        if (ce == cudaSuccess)
            ce = cudaMemcpy(dsrc, src.data(), src.size() * sizeof(long long), cudaMemcpyHostToDevice);
    }
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(cudaStreamLegacy);   // copies complete before the kernel
    int e = (int)ce;
    if (!e)
        e = rs == 8 ? launch_prolong<double>((const double*)a->U[0], (double*)b->U[0], (const double*)dP, a->K,
                                             a->nvar, a->Np, b->Np, dsrc, ctx->stream)
                    : launch_prolong<float>((const float*)a->U[0], (float*)b->U[0], (const float*)dP, a->K, a->nvar,
                                            a->Np, b->Np, dsrc, ctx->stream);
    if (!e) e = (int)cudaStreamSynchronize(ctx->stream);
    if (dsrc) cudaFree(dsrc);
    cudaFree(dP);
    if (e) return fail(ctx, DG_ECUDA, std::string("prolongation failed: ") + cudaGetErrorString((cudaError_t)e));
    b->eps_valid = false;
    return DG_OK;
}

int dg_prolong(dg_ctx* ctx, dg_mesh from, dg_mesh to) {
    try {
        return dg_prolong_body(ctx, from, to);
    } catch (...) {
        return exception_status(ctx);
    }
}

// Time nsteps SSP-RK3 steps of m (dt = 0: the full work, the state
// unchanged, and saved and restored as well) with each of the values set by
// apply(c) for c in cands; returns the times (ms per nsteps) or an error.
static int time_candidates(dg_ctx* ctx, MeshData* m, int nsteps, const std::vector<int>& cands,
                           const std::function<void(int)>& apply, std::vector<double>& ms) {
    const size_t bytes = (size_t)m->K * m->nvar * m->Np * m->rsize;
    CUDA_OK(ctx, cudaStreamSynchronize(ctx->stream));
    CUDA_OK(ctx, cudaMemcpyAsync(m->rhs, m->U[0], bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    cudaEvent_t ea = nullptr, eb = nullptr;
    CUDA_OK(ctx, cudaEventCreate(&ea));
    if (cudaEventCreate(&eb) != cudaSuccess) {
        cudaEventDestroy(ea);
        return fail(ctx, DG_ECUDA, "event creation failed");
    }
    ms.assign(cands.size(), 0.0);
    int err = 0;
    for (size_t c = 0; c < cands.size() && !err; ++c) {
        apply(cands[c]);
        err = enqueue_step(*m, 0.0, ctx->stream);   // warm-up
        if (!err) err = (int)cudaEventRecord(ea, ctx->stream);
        for (int k = 0; k < nsteps && !err; ++k) err = enqueue_step(*m, 0.0, ctx->stream);
        if (!err) err = (int)cudaEventRecord(eb, ctx->stream);
        if (!err) err = (int)cudaEventSynchronize(eb);
        float t = 0.f;
        if (!err) err = (int)cudaEventElapsedTime(&t, ea, eb);
        ms[c] = t;
    }
    cudaEventDestroy(ea);
    cudaEventDestroy(eb);
    const cudaError_t ce = cudaMemcpyAsync(m->U[0], m->rhs, bytes, cudaMemcpyDeviceToDevice, ctx->stream);
    const cudaError_t cs = cudaStreamSynchronize(ctx->stream);
    if (err) return fail(ctx, DG_ECUDA, std::string("autotune step failed: ") + cudaGetErrorString((cudaError_t)err));
    if (ce != cudaSuccess || cs != cudaSuccess) return fail(ctx, DG_ECUDA, "autotune state restore failed");
    return DG_OK;
}

// The tensor-core path: the tile-pipeline configuration of the stage kernel
// (C CTAs per SM of P tile pipelines, code 10 C + P) among those that fit.
static int autotune_tc(dg_ctx* ctx, MeshData* m, int nsteps, int32_t* tile_e_out, int32_t* cand_out, double* ms_out,
                       int32_t* ncand_out) {
    int list[4];
    const int nl = dispatch_tc_configs(m->N, m->p.av_on, list);
    if (nl <= 0) return fail(ctx, DG_EINVAL, "no tile-pipeline configuration fits");
    const std::vector<int> cands(list, list + nl);
    if (fused_sensor(*m) && !m->eps_valid) {   // eps(U^n) for the timed steps' first stage
        CUDA_OK(ctx, cudaMemsetAsync(m->err + VISC_SLOT, 0, sizeof(int), ctx->stream));
        const int se = enqueue_sensor(*m, m->U[0], m->eps_ring[0], ctx->stream, m->err + VISC_SLOT);
        if (se) return fail(ctx, DG_ECUDA, "sensor launch failed");
        m->eps_valid = true;
    }
    // dt = 0 leaves the state (and so its eps) unchanged
    std::vector<double> ms;
    const int e = time_candidates(ctx, m, nsteps, cands, [&](int c) {
        m->tc_cfg = c;
        drop_graphs(*m);
    }, ms);
    size_t best = 0;
    for (size_t c = 1; c < cands.size(); ++c)
        if (ms[c] < ms[best]) best = c;
    m->tc_cfg = e ? 0 : cands[best];
    drop_graphs(*m);
    reset_batch(ctx);
    if (e) return e;
    const int key = tune_key(m->dim, m->N, 16 + m->prec, m->p.av_on);
    ctx->tuned_e[key] = m->tc_cfg;
    for (auto& kv : ctx->meshes) {   // the context's other meshes of this kind follow
        MeshData* o = kv.second;
        if (o == m || o->dim != m->dim || o->prec != m->prec || o->N != m->N || o->p.av_on != m->p.av_on) continue;
        o->tc_cfg = m->tc_cfg;
        drop_graphs(*o);
    }
    *tile_e_out = 32;
    if (ncand_out) *ncand_out = (int32_t)cands.size();
    for (size_t c = 0; c < cands.size() && c < 8; ++c) {
        if (cand_out) cand_out[c] = cands[c];
        if (ms_out) ms_out[c] = ms[c] / nsteps;
    }
    return check_device_errors(ctx);
}

int dg_set_tc_config(dg_ctx* ctx, dg_mesh h, int32_t cfg, int32_t* cands_out, int32_t* ncand_out) {
    if (!ctx) return fail(ctx, DG_EINVAL, "NULL argument");
    MeshData* m = find(ctx, h);
    if (!m) return fail(ctx, DG_ENOTFOUND, "unknown mesh handle");
    if (ncand_out) *ncand_out = 0;
    if (!tensor_prec(m->prec) || m->dim != 2) return fail(ctx, DG_EINVAL, "not a tensor-core mesh of triangles");
    int list[4];
    const int nl = dispatch_tc_configs(m->N, m->p.av_on, list);
    if (nl <= 0) return fail(ctx, DG_EINVAL, "no tile-pipeline configuration fits");
    if (cfg != 0 && std::find(list, list + nl, (int)cfg) == list + nl)
        return fail(ctx, DG_EINVAL, "configuration does not fit this mesh's kernel");
    for (int c = 0; c < nl; ++c)
        if (cands_out) cands_out[c] = list[c];
    if (ncand_out) *ncand_out = nl;
    m->tc_cfg = cfg;
    drop_graphs(*m);
    reset_batch(ctx);
    return DG_OK;
}

static int dg_autotune_body(dg_ctx* ctx, dg_mesh h, int nsteps, int32_t* tile_e_out, int32_t* cand_out, double* ms_out,
                            int32_t* ncand_out) {
    if (!ctx || !tile_e_out) return fail(ctx, DG_EINVAL, "NULL argument");
    MeshData* m = find(ctx, h);
    if (!m) return fail(ctx, DG_ENOTFOUND, "unknown mesh handle");
    if (nsteps < 1 || nsteps > 1000) return fail(ctx, DG_EINVAL, "nsteps must be in 1..1000");
    if (ncand_out) *ncand_out = 0;
    if (tensor_prec(m->prec) && m->dim == 3) {   // fixed tiles: 5 E <= 128 rows of the products
        *tile_e_out = tile3_tc(m->N);
        return DG_OK;
    }
    cudaSetDevice(ctx->device);
    if (tensor_prec(m->prec)) return autotune_tc(ctx, m, nsteps, tile_e_out, cand_out, ms_out, ncand_out);
    const bool dbl = m->rsize == 8;
    const int av = m->p.av_on;
    const int E0 = m->dim == 3 ? tile3_default(m->N, (int)m->rsize)
                   : dbl       ? dispatch_tile_default<double>(m->N)
                               : dispatch_tile_default<float>(m->N);
    std::vector<int> cands;
    for (int quarters : {1, 2, 4, 6, 8, 12}) {   // E0/4, E0/2, E0, 3E0/2, 2E0, 3E0
        const int e = std::max(1, E0 * quarters / 4);
        const bool fits = m->dim == 3 ? tile3_fits(m->N, (int)m->rsize, e)
                          : dbl       ? dispatch_tile_fits<double>(m->N, e, av)
                                      : dispatch_tile_fits<float>(m->N, e, av);
        if (fits && std::find(cands.begin(), cands.end(), e) == cands.end()) cands.push_back(e);
    }
    if (cands.empty()) return fail(ctx, DG_EINVAL, "no tile size fits the shared memory");
    // timed steps with dt = 0 (the full work of a step, the state unchanged);
    // the state is saved and restored all the same
    const size_t bytes = (size_t)m->K * m->nvar * m->Np * m->rsize;
    CUDA_OK(ctx, cudaStreamSynchronize(ctx->stream));
    CUDA_OK(ctx, cudaMemcpyAsync(m->rhs, m->U[0], bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    cudaEvent_t ea = nullptr, eb = nullptr;
    CUDA_OK(ctx, cudaEventCreate(&ea));
    if (cudaEventCreate(&eb) != cudaSuccess) {
        cudaEventDestroy(ea);
        return fail(ctx, DG_ECUDA, "event creation failed");
    }
    std::vector<double> ms(cands.size(), 0.0);
    int err = 0;
    for (size_t c = 0; c < cands.size() && !err; ++c) {
        m->tile_e = cands[c];
        err = enqueue_step(*m, 0.0, ctx->stream);   // warm-up
        if (!err) err = (int)cudaEventRecord(ea, ctx->stream);
        for (int k = 0; k < nsteps && !err; ++k) err = enqueue_step(*m, 0.0, ctx->stream);
        if (!err) err = (int)cudaEventRecord(eb, ctx->stream);
        if (!err) err = (int)cudaEventSynchronize(eb);
        float t = 0.f;
        if (!err) err = (int)cudaEventElapsedTime(&t, ea, eb);
        ms[c] = t;
    }
    cudaEventDestroy(ea);
    cudaEventDestroy(eb);
    const cudaError_t ce = cudaMemcpyAsync(m->U[0], m->rhs, bytes, cudaMemcpyDeviceToDevice, ctx->stream);
    const cudaError_t cs = cudaStreamSynchronize(ctx->stream);
    size_t best = 0;
    for (size_t c = 1; c < cands.size(); ++c)
        if (ms[c] < ms[best]) best = c;
    m->tile_e = err ? 0 : cands[best];
    // graphs captured with the old tile size are rebuilt on their next use
    drop_graphs(*m);
    reset_batch(ctx);
    if (err) return fail(ctx, DG_ECUDA, std::string("autotune step failed: ") + cudaGetErrorString((cudaError_t)err));
    if (ce != cudaSuccess || cs != cudaSuccess) return fail(ctx, DG_ECUDA, "autotune state restore failed");
    const int key = tune_key(m->dim, m->N, m->rsize, av);
    ctx->tuned_e[key] = m->tile_e;
    for (auto& kv : ctx->meshes) {   // the context's other meshes of this kind follow
        MeshData* o = kv.second;
        if (o == m || tensor_prec(o->prec) || tune_key(o->dim, o->N, o->rsize, o->p.av_on) != key) continue;
        o->tile_e = m->tile_e;
        drop_graphs(*o);
    }
    *tile_e_out = m->tile_e;
    if (ncand_out) *ncand_out = (int32_t)cands.size();
    for (size_t c = 0; c < cands.size() && c < 8; ++c) {
        if (cand_out) cand_out[c] = cands[c];
        if (ms_out) ms_out[c] = ms[c] / nsteps;
    }
    return check_device_errors(ctx);
}

int dg_autotune(dg_ctx* ctx, dg_mesh h, int nsteps, int32_t* tile_e_out, int32_t* cand_out, double* ms_out,
                int32_t* ncand_out) {
    try {
        return dg_autotune_body(ctx, h, nsteps, tile_e_out, cand_out, ms_out, ncand_out);
    } catch (...) {
        return exception_status(ctx);
    }
}

int dg_set_profiling(dg_ctx* ctx, dg_mesh h, int on) {
    if (!ctx) return fail(nullptr, DG_EINVAL, "ctx is NULL");
    MeshData* m = find(ctx, h);
    if (!m) return fail(ctx, DG_ENOTFOUND, "unknown mesh handle");
    cudaSetDevice(ctx->device);
    CUDA_OK(ctx, cudaStreamSynchronize(ctx->stream));
    if (on && m->prof_ev.empty()) {
        const int pairs = 9;  // up to three kernels per stage, three stages
        m->prof_ev.resize(2 * pairs);
        m->prof_kind.assign(pairs, -1);
        for (auto& e : m->prof_ev) CUDA_OK(ctx, cudaEventCreate(&e));
    }
    m->profiling = on != 0;
    m->prof_capturing = false;
    m->prof_next = 0;
    m->prof_count = 0;
    if (m->gexec) { cudaGraphExecDestroy(m->gexec); m->gexec = nullptr; }
    if (m->graph) { cudaGraphDestroy(m->graph); m->graph = nullptr; }
    return DG_OK;
}

int dg_kernel_times(dg_ctx* ctx, dg_mesh h, double out_ms[4]) {
    if (!ctx || !out_ms) return fail(ctx, DG_EINVAL, "NULL argument");
    MeshData* m = find(ctx, h);
    if (!m) return fail(ctx, DG_ENOTFOUND, "unknown mesh handle");
    if (!m->profiling || m->prof_count == 0) return fail(ctx, DG_EINVAL, "profiling is off or no step has run");
    out_ms[0] = out_ms[1] = out_ms[2] = 0.0;
    for (int i = 0; i < m->prof_count; ++i) {
        float ms = 0.0f;
        CUDA_OK(ctx, cudaEventElapsedTime(&ms, m->prof_ev[2 * i], m->prof_ev[2 * i + 1]));
        if (m->prof_kind[i] >= 0 && m->prof_kind[i] < 3) out_ms[m->prof_kind[i]] += ms;
    }
    out_ms[3] = m->prof_count;
    return DG_OK;
}

const char* dg_last_error(dg_ctx* ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

#ifdef DGC_PHASE_CLOCKS
// Profiling builds only: the per-phase cycle counts of the degree-N
// tensor-core tile body (see DGC_PHASE_CLOCKS in tc_kernels.cuh), reset after
// reading when reset != 0.
int dg_debug_tc_phase_cycles(int N, unsigned long long out16[16], int reset) {
    switch (N) {
        case 2: return dgc::tc_phase_cycles<2>(out16, reset != 0);
        case 3: return dgc::tc_phase_cycles<3>(out16, reset != 0);
        case 4: return dgc::tc_phase_cycles<4>(out16, reset != 0);
        case 5: return dgc::tc_phase_cycles<5>(out16, reset != 0);
        case 6: return dgc::tc_phase_cycles<6>(out16, reset != 0);
    }
    return DG_EINVAL;
}
#endif

}  // extern "C"
