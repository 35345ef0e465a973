/*
 * dgcurved.h -- C ABI of libdgcurved.so, a GB300 (sm_103a) implementation of
 * the right-hand side and Runge-Kutta stage update of the curved-element
 * discontinuous Galerkin method for the Euler equations of Siebenborn,
 * Schulz & Schmidt, "A curved-element unstructured discontinuous Galerkin
 * method on GPUs for the Euler equations" (arXiv 1208.4772): on triangles
 * (2D, four variables; every entry point) and on tetrahedra (the paper's 3D
 * setting, five variables; dg_tet_mesh_upload and the state, stepping and
 * residual calls, see "Tetrahedra" below).
 *
 * Conventions (all calls)
 *   - Every function returns an int status: DG_OK (0) or a negative DG_E*
 *     code.  No C++ exception crosses the ABI: a host allocation or thread
 *     that cannot be had inside a call returns DG_ENOMEM.  dg_last_error(ctx) returns a
 *     NUL-terminated description of the last failure on that context (valid
 *     until the next call on the same context; ctx may be NULL for calls
 *     that take none).
 *   - Reference triangle T: vertices (-1,-1), (1,-1), (-1,1).  Elements are
 *     counter-clockwise; face f joins local vertices f and (f+1) mod 3.  On a
 *     shared face the neighbour runs the edge the other way, so face point g
 *     meets the neighbour's point N_g - 1 - g.
 *   - N is the polynomial degree, 2 <= N <= 6; N_p = (N+1)(N+2)/2.
 *   - Canonical host state layout: double U[K][4][N_p], variables
 *     (rho, rho u, rho v, E), nodes in the order of dg_reference_nodes.  The
 *     device layout is private to the library.
 *   - Pointers passed in are only read during the call (the library copies
 *     what it keeps); pointers passed out are caller-owned buffers of the
 *     stated size.  All calls on one context are issued on its stream and
 *     are not thread-safe with respect to each other.
 *   - Calls that read results back (dg_get_state, dg_eval_rhs, dg_residual)
 *     synchronise the context's stream; dg_step and dg_batch_step only
 *     enqueue work (use dg_sync to wait).
 *
 * Tetrahedra (paper Sec. 2 with d = 3)
 *   - Reference tetrahedron: vertices (-1,-1,-1), (1,-1,-1), (-1,1,-1),
 *     (-1,-1,1); elements positively oriented (det[v1-v0, v2-v0, v3-v0] >
 *     0).  Face f has the local vertices (0,2,1), (0,1,3), (1,2,3), (0,3,2)
 *     for f = 0..3.
 *   - N_p = (N+1)(N+2)(N+3)/6, 2 <= N <= 4 on the device; state layout
 *     double U[K][5][N_p], variables (rho, rho u, rho v, rho w, E), nodes in
 *     the order of dg_tet_reference_nodes.
 *   - Face integrals use the triangle rule (q^2 points) placed in each
 *     face's canonical frame, its vertices ordered by global vertex number,
 *     so both elements of a face evaluate the flux at the same points.
 *   - dg_set_state, dg_get_state, dg_set_state_device, dg_get_state_device,
 *     dg_eval_rhs, dg_step, dg_step_lserk, dg_residual, dg_mesh_info,
 *     dg_mesh_bytes, dg_mesh_free, dg_set_profiling, dg_kernel_times and
 *     dg_autotune and dg_prolong accept tetrahedral meshes with the
 *     five-variable layout; dg_batch_step returns DG_EINVAL for them.  Precisions
 *     DG_FP32, DG_FP64_DEBUG and, for N = 2 and 3, DG_TF32 (the
 *     interpolation to the cubature points and the three weighted
 *     derivative products on the tensor cores, on deviations from each
 *     element's mean state and its flux; the face terms in FP32).
 *   - Artificial viscosity (av_on, DG_FP32 or DG_FP64_DEBUG): per stage the
 *     element sensor, the gradient pass q = sqrt(eps) grad U (BR1, one
 *     launch per direction) and the stage with the viscous terms, all on
 *     the CUDA cores; dg_av_count counts eps > 0.
 */
#ifndef DGCURVED_H
#define DGCURVED_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum dg_status {
    DG_OK = 0,
    DG_EINVAL = -1,      /* bad argument, malformed mesh, non-positive Jacobian */
    DG_ENOMEM = -2,      /* device or host allocation failed, or budget exceeded */
    DG_ECUDA = -3,       /* a CUDA runtime call failed */
    DG_ENONFINITE = -4,  /* a residual norm came back NaN or Inf */
    DG_ETIMEOUT = -5,    /* dg_sync gave up waiting */
    DG_EBUSY = -6,       /* work is still in flight where none may be */
    DG_ENOTFOUND = -7    /* unknown mesh handle */
};

/* Arithmetic of the operator products.  DG_FP32: FP32 state, FP32 FMA
 * products.  DG_FP64_DEBUG: every device quantity in FP64 (slow; used to
 * check the kernels' logic against the FP64 oracle to round-off).
 * DG_TF32 and DG_BF16X3: FP32 state, operator products on the tensor
 * cores (TF32 inputs, or each FP32 operand split into three BF16 parts),
 * FP32 accumulate. */
enum dg_prec { DG_FP32 = 0, DG_TF32 = 1, DG_BF16X3 = 2, DG_FP64_DEBUG = 3 };

/* Face codes of the bc array.  Periodic faces are interior faces whose
 * neighbour is the periodic image. */
enum dg_bc { DG_BC_INTERIOR = 0, DG_BC_WALL = 1, DG_BC_FARFIELD = 2 };

typedef struct dg_ctx dg_ctx;   /* opaque: device, stream, meshes, graphs */
typedef int32_t dg_mesh;        /* mesh handle within one context */

/* Physical and numerical parameters of one mesh (paper Sec. 2 and Sec. 5).
 *   gamma      adiabatic index
 *   flux       0 = local Lax-Friedrichs (Sec. 2 approximate Riemann solver);
 *              1 = HLLC (the alternative Sec. 2 names; Davis wave speeds)
 *   av_on      1 = Persson-Peraire artificial viscosity (Sec. 2)
 *   kappa, eps0, s0   sensor ramp parameters; s0 = NaN -> log10(1/N^4)
 *   u_inf      conserved farfield state used by DG_BC_FARFIELD faces: the
 *              first four entries on triangles, all five on tetrahedra
 *   prec       enum dg_prec
 *   cub_q      points per direction of the volume rule and points per edge
 *              of the face rule; 0 -> ceil((3N+1)/2) (exact to degree 3N) */
typedef struct {
    double gamma;
    int32_t flux;
    int32_t av_on;
    double kappa, eps0, s0;
    double u_inf[5];
    int32_t prec;
    int32_t cub_q;
} dg_params;

/* Create a context on CUDA device `device`.  cuda_stream: a cudaStream_t to
 * issue work on, or NULL for a stream owned by the context.  *out is set on
 * success.  Errors: DG_EINVAL (out NULL, bad device), DG_ECUDA. */
int dg_create(dg_ctx** out, int device, void* cuda_stream);

/* Free every mesh, graph and buffer of ctx, then ctx itself.  NULL is a no-op. */
int dg_destroy(dg_ctx* ctx);

/* How dg_set_state, dg_get_state and dg_eval_rhs move the host FP64 state
 * (the conversion to and from the mesh precision and the reordering
 * between the canonical and the device element order):
 *   DG_HOST_IO_STAGED  up to 16 host threads convert and reorder the rows
 *                      in a host buffer, copied in one transfer;
 *   DG_HOST_IO_DEVICE  one kernel reads (writes) the caller's rows in
 *                      place and converts and reorders them on the device.
 *                      Needs coherent device access to pageable host memory
 *                      through the host's page tables (as on Grace systems
 *                      over NVLink-C2C): the device attributes
 *                      PageableMemoryAccess and
 *                      PageableMemoryAccessUsesHostPageTables both 1.
 *   DG_HOST_IO_AUTO    STAGED (the mode a new context starts in): the
 *                      faster of the two on GB300 with the caller's
 *                      buffers in pageable memory.
 * Either way the call returns when the data has arrived, so the caller's
 * buffer may be reused at once; the results are the same bit for bit.
 * dg_set_host_io errors: DG_EINVAL (ctx NULL, unknown mode, DEVICE without
 * that access).  dg_host_io writes the mode in effect (STAGED or DEVICE)
 * to *out; DG_EINVAL for NULL arguments. */
enum dg_host_io_mode { DG_HOST_IO_AUTO = 0, DG_HOST_IO_STAGED = 1, DG_HOST_IO_DEVICE = 2 };
int dg_set_host_io(dg_ctx* ctx, int mode);
int dg_host_io(dg_ctx* ctx, int32_t* out);

/* Collocation nodes of degree N on T (paper Sec. 2: nodes after Warburton
 * 2006, the warp & blend construction, blending parameter 0), written as
 * rs_out[N_p][2] (caller-owned).  The order is j (the s index) outer, i
 * inner, starting at (-1,-1).  Host-only; needs no GPU.  Errors: DG_EINVAL. */
int dg_reference_nodes(int N, double* rs_out);

/* Sizes for degree N with cub_q points per direction (0 = default):
 * out4 = {N_p, N_q, N_g, q}.  Host-only. */
int dg_sizes(int N, int cub_q, int32_t* out4);

/* Upload one mesh (paper Sec. 4 flowchart: "setup operators and transfer to
 * GPU").  K elements of degree N:
 *   EToE[K][3]   neighbour element across each face (self on boundary faces)
 *   EToF[K][3]   the neighbour's face index (0..2)
 *   bc[K][3]     enum dg_bc per face
 *   node_xy[K][N_p][2]  collocation-node coordinates (FP64), curved
 *                elements by isoparametric node displacement (paper Sec. 3)
 *   p            parameters (copied)
 * The library builds the reference operators, computes the geometric
 * factors in FP64 (J = |det D Psi|, r_x, ..., face normals and sJ, and the
 * mass matrix with its Cholesky-based inverse for curved elements, paper
 * Sec. 2 eqs. stiffness, mass, face_mass), classifies each element as affine
 * or curved, and copies everything to the device.  The state is set to 0.
 * There is no argument for caller-computed geometric factors: on
 * isoparametric elements they are a function of the node coordinates
 * (paper Sec. 2, the mapping of the reference element by the collocation
 * nodes), and the library always derives them from node_xy, so that the
 * factors and the nodes cannot disagree (free-stream preservation rests on
 * their consistency).
 * Errors: DG_EINVAL (bad sizes or connectivity, J <= 0 at a cubature node,
 * unsupported N or prec), DG_ENOMEM, DG_ECUDA. */
int dg_mesh_upload(dg_ctx* ctx, int N, int64_t K, const int32_t* EToE, const int8_t* EToF,
                   const int8_t* bc, const double* node_xy, const dg_params* p, dg_mesh* out);

/* dg_mesh_upload in two halves, so that the host work of one mesh can run
 * while the device works on others (the serving loop prepares arriving
 * requests on a worker thread).  dg_mesh_prepare does everything
 * dg_mesh_upload does on the host -- the checks, the affine / curved
 * classification and device order, the FP64 geometric factors and curved
 * mass inverses (paper Sec. 2, Sec. 4 "setup operators") -- with the same
 * arguments and errors, needs no context or GPU, is safe to call from
 * several threads at once, and returns an opaque host object in *out
 * (errors in dg_last_error(NULL) of the calling thread).
 * dg_mesh_upload_prepared allocates the device buffers and copies; it takes
 * ownership of prep and frees it whatever the outcome.  dg_prepared_free
 * discards a prepared mesh that is not uploaded.  Together they give the
 * mesh dg_mesh_upload gives. */
typedef struct dg_prepared dg_prepared;
int dg_mesh_prepare(int N, int64_t K, const int32_t* EToE, const int8_t* EToF, const int8_t* bc,
                    const double* node_xy, const dg_params* p, dg_prepared** out);
int dg_mesh_upload_prepared(dg_ctx* ctx, dg_prepared* prep, dg_mesh* out);
int dg_prepared_free(dg_prepared* prep);

/* Tetrahedral counterparts of dg_reference_nodes, dg_sizes and
 * dg_mesh_upload (paper Sec. 2 with d = 3).
 *
 * dg_tet_reference_nodes: collocation nodes of degree N (1..6) on the
 * reference tetrahedron, the warp & blend construction with blending
 * parameter 0 (each face carries the triangle's nodes, each edge the
 * Gauss-Lobatto-Legendre points), written as rst_out[N_p][3]; order: the
 * equidistant lattice index of t outer, of s, of r inner.  Host-only.
 *
 * dg_tet_sizes: out4 = {N_p, N_q = q^3, N_g = q^2 (points per face),
 * N_fp = (N+1)(N+2)/2 (nodes per face)}, q = ceil((3N+1)/2).  Host-only.
 *
 * dg_tet_mesh_upload: K tetrahedra of degree N (2..4):
 *   EToV[K][4]   global vertex numbers (periodic images share a number); the
 *                library matches faces by their vertex sets and orients the
 *                face rule by them
 *   bc[K][4]     enum dg_bc per face; exactly the unmatched faces must be
 *                DG_BC_WALL or DG_BC_FARFIELD
 *   node_xyz[K][N_p][3]  collocation-node coordinates (FP64); elements
 *                whose nodes are not the affine image of their vertex nodes
 *                are treated as curved (per-point geometric factors and their
 *                own mass matrix)
 *   p            parameters (copied); prec DG_FP32, DG_FP64_DEBUG, or DG_TF32
 *                with N <= 3 and av_on 0
 * The state is set to 0.  Errors: DG_EINVAL (N, K, prec or av_on out of
 * range, a face shared by more than two elements, bc inconsistent with the
 * face matching, J <= 0 at a cubature point), DG_ENOMEM, DG_ECUDA. */
int dg_tet_reference_nodes(int N, double* rst_out);
int dg_tet_sizes(int N, int32_t* out4);
int dg_tet_mesh_upload(dg_ctx* ctx, int N, int64_t K, const int64_t* EToV, const int8_t* bc,
                       const double* node_xyz, const dg_params* p, dg_mesh* out);

/* Shape of mesh m: out6 = {dimension (2 or 3), variables (4 or 5), N, N_p,
 * K, curved elements}. */
int dg_mesh_info(dg_ctx* ctx, dg_mesh m, int64_t* out6);

/* Release a mesh and its device memory. */
int dg_mesh_free(dg_ctx* ctx, dg_mesh m);

/* Device bytes held by mesh m (state buffers, geometry, operators, scratch). */
int dg_mesh_bytes(dg_ctx* ctx, dg_mesh m, int64_t* out);

/* Set / read the state U^n from / to host memory, canonical layout
 * double[K][4][N_p] (tetrahedra: [K][5][N_p]).  The device holds it in the
 * precision of p->prec. */
int dg_set_state(dg_ctx* ctx, dg_mesh m, const double* U);
int dg_get_state(dg_ctx* ctx, dg_mesh m, double* U_out);

/* Device-resident variants: U is a device pointer to float[K][4][N_p] (tetrahedra [K][5][N_p]) in
 * canonical order (FP32 precision modes only).  Asynchronous on the
 * context's stream.  Errors: DG_EINVAL for DG_FP64_DEBUG meshes. */
int dg_set_state_device(dg_ctx* ctx, dg_mesh m, const float* U_dev);
int dg_get_state_device(dg_ctx* ctx, dg_mesh m, float* U_dev_out);

/* Right-hand side L(U^n) of the semi-discrete system (paper Sec. 2, eq.
 * semidiscrete; with the artificial-viscosity terms when av_on) written to
 * rhs_out[K][4][N_p] (tetrahedra [K][5][N_p]; host, FP64, canonical layout). */
int dg_eval_rhs(dg_ctx* ctx, dg_mesh m, double* rhs_out);

/* Advance U^n by nsteps SSP-RK3 steps of size dt (three right-hand-side
 * evaluations with the stage combination fused into each; a fixed step
 * replayed from a captured CUDA graph).  Asynchronous. */
int dg_step(dg_ctx* ctx, dg_mesh m, double dt, int nsteps);

/* Advance U^n by nsteps steps of the paper's integrator (Sec. 2): the
 * five-stage, fourth-order low-storage Runge-Kutta of Carpenter and
 * Kennedy, dU <- A_i dU + dt L(U), U <- U + B_i dU (i = 1..5), each stage's
 * combination fused into its right-hand-side kernel; a fixed step replayed
 * from its own captured CUDA graph.  Same arguments and errors as dg_step.
 * Asynchronous. */
int dg_step_lserk(dg_ctx* ctx, dg_mesh m, double dt, int nsteps);

/* Residual norms of L(U^n) per variable, accumulated in FP64 on the device
 * (paper Sec. 5 checks the residual norm): out_linf[v] = max |L|,
 * out_l2[v] = sqrt(sum L^2) over all nodal values, v over the mesh's 4
 * (triangles) or 5 (tetrahedra) variables: out_linf and out_l2 hold that
 * many doubles each.  Returns DG_ENONFINITE (with the norms still written)
 * if any norm is NaN or Inf. */
int dg_residual(dg_ctx* ctx, dg_mesh m, double* out_linf, double* out_l2);

/* dg_residual of n meshes with one synchronisation: every mesh's
 * right-hand side and FP64 norms are enqueued, the norms copied to pinned
 * host slots, and the stream synchronised once.  out10: caller-owned
 * double[n][10]; mesh i's max norms in out10[10 i + v] and Euclidean norms in
 * out10[10 i + 5 + v] for its variables v (4 on triangles, 5 on tetrahedra;
 * unused slots 0).  Returns DG_ENONFINITE (all norms still written) if any
 * norm is NaN or Inf; DG_EINVAL, DG_ENOTFOUND, DG_ECUDA. */
int dg_batch_residual(dg_ctx* ctx, int n, const dg_mesh* ms, double* out10);

/* Advance n meshes (any mix of N and K) by nsteps SSP-RK3 steps each, with
 * per-mesh step sizes dts[n], replayed from one captured CUDA graph.  The
 * meshes without artificial viscosity share one persistent launch per RK
 * stage that walks a work list over all of them: DG_FP32 and DG_FP64_DEBUG
 * run the CUDA-core tile body, DG_TF32 and DG_BF16X3 the tensor-core tile
 * body (degrees 2..5 in one launch per stage, degree 6 in a second).  Each
 * mesh with artificial viscosity (paper Sec. 2) runs its own sensor,
 * gradient and stage kernels on a branch of the same graph (up to eight
 * side streams of the context), concurrently with the other meshes; a
 * state set from outside gets its sensor before the graph runs.  All meshes
 * must share one precision mode.  Each mesh ends in the state dg_step would
 * give it.  Asynchronous. */
int dg_batch_step(dg_ctx* ctx, int n, const dg_mesh* ms, const double* dts, int nsteps);

/* p-refinement (paper Sec. 5, Table 2: converge at a low degree, then raise
 * it): sets the state of mesh `to` to the state of mesh `from` embedded
 * exactly at the higher degree -- the nodal values at to's nodes of from's
 * degree-N polynomial in every element, i.e. the modal coefficients of
 * degree <= N carried over and the higher ones zero (the basis is
 * hierarchical).  `from` and `to` must be two uploads of the same mesh
 * (both triangle or both tetrahedral meshes; same K and connectivity, the
 * elements in the same caller order -- the library maps its own device
 * orders, which may differ where an element is curved at one degree only)
 * with N_from <= N_to and the same state type (FP32 precisions together, or
 * FP64_DEBUG with FP64_DEBUG).
 * DG_EINVAL otherwise.  Synchronises the context's stream. */
int dg_prolong(dg_ctx* ctx, dg_mesh from, dg_mesh to);

/* Autotuner of the work distribution over CTAs: times nsteps (1..1000)
 * SSP-RK3 steps of mesh m with dt = 0 (the full work of a step, the state
 * unchanged; it is also saved and restored) for each candidate and keeps the
 * fastest for m.  The choice also applies to the context's other meshes of
 * the same kind (dimension, degree, precision, viscosity setting), and to
 * those uploaded later.
 *   - CUDA-core paths (DG_FP32, DG_FP64_DEBUG; triangles and tetrahedra):
 *     the tile size -- E/4, E/2, E, 3E/2, 2E, 3E elements per CTA around the
 *     degree's default E, where the tile's layout fits one CTA (and so also
 *     dg_batch_step's tiles).  *tile_e_out = the chosen size.
 *   - Tensor-core path on triangles (DG_TF32, DG_BF16X3): the tiles are
 *     fixed by the 128 rows of the products (32 elements, *tile_e_out = 32);
 *     the candidates are the stage kernel's tile-pipeline configurations
 *     10 C + P that fit an SM: C CTAs per SM of P groups of 256 threads, each
 *     group working on its own tile and sharing the CTA's operator tables
 *     (21, 13, 12, or 11 where nothing larger fits), and 113: three groups
 *     with a lean per-tile layout (one operand buffer for the flux
 *     products), offered for inviscid meshes where 13 does not fit.
 *   - Tensor-core path on tetrahedra: fixed tiles (8 tetrahedra at N = 3,
 *     16 at N = 2), nothing timed.
 * Optional outputs cand_out[8], ms_out[8] (candidates and milliseconds per
 * step) and *ncand_out (number of candidates), each may be NULL.
 * Synchronises the context's stream.  The paper has no counterpart (its
 * block per element is fixed); a step's work distribution over the SMs is
 * the tuned quantity. */
int dg_autotune(dg_ctx* ctx, dg_mesh m, int nsteps, int32_t* tile_e_out, int32_t* cand_out, double* ms_out,
                int32_t* ncand_out);

/* Set the stage kernel's tile-pipeline configuration of one tensor-core
 * mesh of triangles (DG_TF32, DG_BF16X3) by hand: cfg one of the codes that
 * fit its kernel (see dg_autotune), or 0 for the built-in default.  The
 * other meshes of its kind keep theirs.  Optional outputs cands_out[4] (the
 * codes that fit) and *ncand_out (their number).  Every configuration gives
 * the same state bit for bit: a tile's arithmetic does not depend on which
 * pipeline runs it.  Returns DG_EINVAL for another precision, a tetrahedral
 * mesh or a code that does not fit, with nothing changed. */
int dg_set_tc_config(dg_ctx* ctx, dg_mesh m, int32_t cfg, int32_t* cands_out, int32_t* ncand_out);

/* Kernel timing for profiling (paper Sec. 4 reports run times of the time
 * loop).  dg_set_profiling(ctx, m, 1) puts CUDA event-record nodes around
 * every kernel of the step graph of mesh m (the graph is re-captured);
 * after a dg_step has completed, dg_kernel_times writes the device time in
 * milliseconds of the last step's kernels, summed per kind:
 * out_ms[0] sensor, [1] gradient, [2] stage, [3] kernels launched per step.
 * Errors: DG_EINVAL if profiling is off. */
int dg_set_profiling(dg_ctx* ctx, dg_mesh m, int on);
int dg_kernel_times(dg_ctx* ctx, dg_mesh m, double out_ms[4]);

/* Residual norms of a caller's device array with no allocation at all.  The
 * paper has no counterpart: this serves callers that cannot allocate device
 * memory where they need the norms -- real-time loops that must stay off the
 * allocator's locks and latency, and hosts whose framework owns every device
 * byte through its own pool.  values_dev: device float[K][4][Np]
 * (any element order); out8_dev: device double[8] receiving max |x| for
 * the four variables, then sqrt(sum x^2) for the four variables, in FP64
 * (the definition dg_residual uses).  Runs on the calling thread's current
 * device, asynchronously on cuda_stream (NULL = legacy default stream); both
 * pointers must belong to that device.  The reduction's partial results
 * live in a fixed 1 MiB file-scope device array that every GPU loading the
 * library keeps until the process exits, so K*4*Np may not exceed
 * 67,108,864 values (DG_EINVAL beyond that, and for NULL pointers or
 * non-positive sizes).  The first call on a device looks up that array's
 * address (cudaGetSymbolAddress), so make it before any stream capture;
 * the address is kept for the process's life and, like every handle of this
 * library, does not survive a cudaDeviceReset.
 * All calls share the array: calls that overlap on the GPU race; calls in
 * order on one stream are safe.  No cudaMalloc, cudaFree or allocating
 * library routine is called.  Errors: DG_EINVAL, DG_ECUDA (message in
 * dg_last_error(NULL)). */
int dg_residual_norms_noalloc(const float* values_dev, int64_t K, int32_t Np, double* out8_dev,
                              void* cuda_stream);

/* Number of elements of mesh m whose artificial viscosity is positive for
 * the current state U^n (the sensor of paper Sec. 2, eps_k > 0), in *out.
 * The stage kernels compute the viscous terms only where they are non-zero
 * (a launch with none runs the inviscid tile body), so this is also a
 * measure of the viscous work.  Synchronises the context's stream.  Errors:
 * DG_EINVAL for meshes without artificial viscosity. */
int dg_av_count(dg_ctx* ctx, dg_mesh m, int64_t* out);

/* Wait for the context's stream, polling at most timeout_s seconds
 * (<= 0: wait without limit).  DG_ETIMEOUT if work is still in flight then;
 * the work itself is not cancelled. */
int dg_sync(dg_ctx* ctx, double timeout_s);

/* Diagnostics of the device-side waits.  Every wait inside the library's
 * kernels (on an mbarrier: tensor-core products, bulk copies) polls a
 * bounded number of times; a wait that runs out sets a bit in the mesh's
 * error word, the kernel finishes without the result, and the next call
 * that checks the word returns DG_ETIMEOUT.  This call runs one such wait
 * on a barrier of one expected arrival -- with arrive = 0 nothing arrives --
 * polling at most `limit` (1..2^26) times, on the context's stream, and
 * stores 1 in *out if the wait ran out, 0 if it completed.  The context
 * stays usable either way.  Synchronises the context's stream. */
int dg_selftest_bounded_wait(dg_ctx* ctx, uint32_t limit, int arrive, int32_t* out);

/* Description of the last failure on ctx (or of the last failure of a call
 * without a context when ctx is NULL). */
const char* dg_last_error(dg_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* DGCURVED_H */
