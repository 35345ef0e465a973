// Host-side structures of the library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include "dgcurved.h"

namespace dgc {

// dst row r <- src row map[r] (rows of rowlen values), converted from S to
// D, on the device; either side may be host memory that the device reaches
// coherently (kernels_common.cu)
template <typename S, typename D>
int launch_gather_convert(const S* src, D* dst, const long long* map, long long K, int rowlen, cudaStream_t st);

struct MeshData {
    int dim = 2;                  // 2: triangles, 4 variables; 3: tetrahedra, 5 variables
    int nvar = 4;
    int N = 0, Np = 0, Nq = 0, Ng = 0, Nf = 0;
    int Nfp = 0;                  // tetrahedra: nodes per face
    int2* code3 = nullptr;        // tetrahedra: face codes [K]
    const int* opsi3 = nullptr;   // tetrahedra: fmask / fpos table (owned by the context)
    long long K = 0, Kaff = 0, Kc = 0;
    dg_params p{};
    int prec = 0;
    size_t rsize = 4;             // bytes of the device real type
    int tile_e = 0;               // elements per CUDA-core tile (0: default; see dg_autotune)
    int tc_cfg = 0;               // tensor-core tile-pipeline configuration 10 C + P (0: default; dg_autotune)
    double s0 = 0.0;              // sensor offset actually used
    std::vector<long long> perm;  // device element d is caller element perm[d]
    void* U[3] = {nullptr, nullptr, nullptr};  // U^n, stage buffers
    void* rhs = nullptr;          // L(U) scratch
    void* eps = nullptr;          // [K] viscosity (AV); eps_ring[0]
    // tensor-core path with AV: the stage kernel of stage s reads eps_ring[s]
    // and writes the sensor of its new state to eps_ring[(s+1) % R] (R = 3
    // for SSP-RK3, 5 for the low-storage RK), so that a step of either kind
    // starts and ends with eps_ring[0] = eps(U^n)
    void* eps_ring[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    bool eps_valid = false;       // eps_ring[0] holds eps(U^n)
    void* q = nullptr;            // [K][2][4][Np] (AV; tetrahedra [K][3][5][Np])
    const void* ops_av3 = nullptr;   // tetrahedral sensor table (AV)
    void* geoA = nullptr;         // [Kaff][4]
    void* geoC = nullptr;         // [Kc][curved_stride]
    void* ops = nullptr;          // shared operator table (owned by the context)
    void* ops_tc = nullptr;       // tensor-core operator table (owned by the context)
    int* err = nullptr;           // device error words (ERR_WORDS ints; see below)
    int4* conn = nullptr;         // [K]
    long long* dperm = nullptr;   // device copy of perm
    long long* diperm = nullptr;  // inverse permutation
    double* red = nullptr;        // residual partials + 8 results
    size_t bytes = 0;
    std::vector<void*> allocs;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    double gdt = 0.0;
    cudaGraph_t graph_ls = nullptr;       // low-storage RK(5,4) step
    cudaGraphExec_t gexec_ls = nullptr;
    double gdt_ls = 0.0;
    // profiling: event pairs around each kernel of one step, with its kind
    bool profiling = false;
    std::vector<cudaEvent_t> prof_ev;
    std::vector<int> prof_kind;
    mutable int prof_next = 0;    // next event pair while capturing
    bool prof_capturing = false;  // true only while a profiled step is being captured
    int prof_count = 0;
};

int enqueue_stage(const MeshData& m, const void* Us, const void* Un, void* out, double a, double b, double dt,
                  int rhs_only, cudaStream_t st, int stage = -1, void* dU = nullptr, int ring = 3);
int enqueue_stage3(const MeshData& m, const void* Us, const void* Un, void* out, double a, double b, double dt,
                   int rhs_only, cudaStream_t st, void* dU);
// helpers of the C ABI shared by dg_api.cu and dg3_api.cu
int api_fail(dg_ctx* ctx, int code, const std::string& msg);
// the status of an exception caught around an entry point's body (called
// inside the catch handler): none may cross the C ABI
int exception_status(dg_ctx* ctx);
int api_alloc(dg_ctx* ctx, MeshData& m, void** p, size_t bytes);
void api_free_mesh(MeshData* m);
bool fused_sensor(const MeshData& m);
int enqueue_sensor(const MeshData& m, const void* U, void* eps_out, cudaStream_t st, int* visc = nullptr);
// error word block: [0] error bits, [1..4] tile / done counters of the
// persistent kernels, [VISC_SLOT + s] viscous-tile count of eps ring slot s
// (s < 5), [VISC_SLOT + 5] scratch count of dg_av_count
constexpr int ERR_WORDS = 16, VISC_SLOT = 8, EPS_RING = 5;
int enqueue_step(const MeshData& m, double dt, cudaStream_t st);
int enqueue_step_lserk(const MeshData& m, double dt, cudaStream_t st);
void drop_graphs(MeshData& m);

}  // namespace dgc

namespace dgc {
struct RefOps;
}

// The host half of a mesh upload (dg_mesh_prepare): the mesh's host fields
// and device order, and the connectivity words and FP64 geometric factors
// waiting to be copied.
struct dg_prepared {
    dgc::MeshData* m = nullptr;
    const dgc::RefOps* R = nullptr;
    std::vector<long long> iperm;
    std::vector<int4> conn;
    std::vector<double> geoA, geoC;
};

struct dg_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::map<int, dgc::MeshData*> meshes;
    int next_id = 1;
    std::map<int, void*> ops;         // operator tables by (N, precision)
    std::map<int, int> tuned_e;       // tile sizes found by dg_autotune, by (N, real size, av)
    std::vector<void*> batch_bufs;    // work lists of the batched path
    // batched-step graph cache
    std::vector<int> batch_key_meshes;
    std::vector<double> batch_key_dts;
    cudaGraph_t batch_graph = nullptr;
    cudaGraphExec_t batch_gexec = nullptr;
    // side streams and fork / join events of the batched step's branches
    // (meshes with artificial viscosity)
    std::vector<cudaStream_t> side_streams;
    std::vector<cudaEvent_t> side_events;
    double* res_host = nullptr;       // pinned slots of dg_batch_residual
    int res_host_n = 0;
    // host state I/O: the device reaches pageable host memory coherently
    // through the host's page tables (host_coherent), and the mode in
    // effect (DG_HOST_IO_STAGED or DG_HOST_IO_DEVICE)
    bool host_coherent = false;
    int host_io = 1;
    std::string err;
};
