/*
 * hho.h -- C ABI of the GB300 (sm_103a) library for the statically condensed
 * HHO Stokes system and its p-multilevel V-cycle / FGMRES solve
 * (Botti & Di Pietro, arXiv 2009.13840).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every call returns an hho_status; no call aborts the process.  On error
 *    hho_last_error() returns a one-line message.
 *  - Host pointers ("host") are read during the call only and stay owned by the
 *    caller.  Device pointers ("device") are caller-owned CUDA allocations on
 *    the context's device; the library never frees them.
 *  - All device work is enqueued on the stream given to hho_setup.  Calls that
 *    return host data synchronise that stream.
 *  - The context owns every internal device buffer and frees them in
 *    hho_destroy.
 *  - Vector layout of a condensed vector at level l (degree k_l): one block of
 *    b_l = d * dim P^{k_l}_{d-1} values per face (component-major, each
 *    component's coefficients in the hierarchical orthonormal face basis), then
 *    one block of n_P values per element (n_P = 1 for v&p-cond, the mean
 *    pressure coefficient; n_P = dim P^{k_l}_d for v-cond).
 */
#ifndef HHO_H
#define HHO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HHO_OK = 0,
    HHO_ERR_ARG = 1,           /* invalid argument (null pointer, size, option) */
    HHO_ERR_MESH = 2,          /* inconsistent mesh arrays */
    HHO_ERR_CUDA = 3,          /* a CUDA runtime call failed */
    HHO_ERR_NOMEM = 4,         /* device allocation failed */
    HHO_ERR_SINGULAR = 5,      /* a local or coarse factorisation met a zero pivot */
    HHO_ERR_NOT_CONVERGED = 6, /* FGMRES stopped at maxit above the tolerance */
    HHO_ERR_TIMEOUT = 7,       /* a bounded device wait expired */
    HHO_ERR_STATE = 8,         /* call out of order (e.g. solve before pmg_setup) */
    HHO_ERR_UNSUPPORTED = 9    /* element shape, degree or dimension not built */
} hho_status;

/* HHO_VCOND, HHO_VPCOND: Scheme 1 (HHO-dp, k' = k) with velocity-only or
 * velocity-and-pressure condensation (Sec. 4.1.2).  HHO_HPCOND: Scheme 2
 * (HHO-hp, Sec. 2.3.2: element velocity of degree k+1, hybrid element/face
 * pressure) with every element unknown condensed; its condensed unknowns are
 * one block of (d+1) n_F per face (velocity components, then the face
 * pressure) and no element rows.  HHO_UNCOND: Scheme 1 uncondensed (the
 * reference formulation of Sec. 5.4): face blocks of d n_F, then one block of
 * (d+1) n_E per element ([U_T (d components) | P_T]); its p-multilevel
 * hierarchy truncates every element component like a face component, and its
 * V-cycle needs the block ILU(0) smoother (hho_set_option "smoother" = 1).
 * HHO_DGCOND: the DG scheme (Scheme 3, Sec. 2.4: BR2 vector Laplacian,
 * stabilised equal-order pressure), k >= 1, element unknowns only: one block
 * of (d+1) n_E per element ([u_T (d components) | p_T]) in element order;
 * at most 10 coefficients per component (2D k <= 3, 3D k <= 2, else
 * HHO_ERR_UNSUPPORTED), planar faces.  Its hierarchy truncates every
 * component; its V-cycle takes the element block-Jacobi smoother and the
 * dense coarse solve (a coarse level above coarse_dense_max unknowns, the ILU
 * smoother, the two-level coarse solve, batches and the learned smoother are
 * HHO_ERR_UNSUPPORTED).  hho_element_schur returns the element data the
 * couplings are formed from (K, D_c, then per face the trace matrices), and
 * hho_recover copies the element blocks. */
typedef enum { HHO_VCOND = 0, HHO_VPCOND = 1, HHO_HPCOND = 2, HHO_UNCOND = 3, HHO_DGCOND = 4 } hho_cond;
typedef enum { HHO_FP64 = 0, HHO_FP32 = 1 } hho_prec;
/* Preconditioner of the smoother's GMRES, selected by hho_set_option("smoother", v) before pmg_setup. */
typedef enum { HHO_SMOOTH_BJACOBI = 0, HHO_SMOOTH_ILU = 1 } hho_smoother;
typedef enum { HHO_NODES_ELEM = 0, HHO_NODES_FACE = 1 } hho_node_set;

typedef struct hho_ctx hho_ctx;

/* Mesh of Sec. 2.1 (host arrays, copied by hho_setup).
 *   dim            2 or 3
 *   xyz            n_vert*dim vertex coordinates
 *   elem_face_ptr  n_elem+1 CSR offsets into elem_face; elem_face lists the
 *                  faces of each element (any order; it fixes the local order)
 *   face_vert_ptr  n_face+1 CSR offsets into face_vert; a face is a segment
 *                  (2 vertices) in 2D, a planar polygon with vertices in cyclic
 *                  order in 3D
 *   face_elem      2*n_face: the one or two elements of each face (T1 < T2),
 *                  -1 in the second slot for a boundary face
 *   face_bc        n_face tags: 0 interior, 1 Dirichlet, 2 Neumann
 * Supported: 2D triangles and convex polygons with up to 8 faces, 3D convex
 * polyhedra with up to 6 faces of up to 4 vertices (hexahedra). */
typedef struct {
    int32_t dim;
    int64_t n_vert;
    const double* xyz;
    int64_t n_elem;
    const int64_t* elem_face_ptr;
    const int64_t* elem_face;
    int64_t n_face;
    const int64_t* face_vert_ptr;
    const int64_t* face_vert;
    const int64_t* face_elem;
    const int8_t* face_bc;
} hho_mesh;

typedef struct {
    int32_t iterations;        /* FGMRES iterations (one V-cycle each) */
    int32_t coarse_iterations; /* total coarse-solver iterations (1 per V-cycle for LU) */
    double rel_residual;       /* true ||b - S x|| / ||b|| in FP64 */
    double solve_ms;           /* device time of the solve (CUDA events) */
    int32_t status;            /* hho_status of the solve */
} hho_solve_info;

/* Build the context: copy and check the mesh, compute on the GPU the element
 * and face geometry, hierarchical orthonormal bases (Secs. 2.1, 4.2), the
 * local operators of Scheme 1 with k' = k (Sec. 2.2, Eq. HHOdiscr:residuals,
 * Eq. def:HHOAB) or of Scheme 2 (cond = HHO_HPCOND, Sec. 2.3.2), the element
 * static condensation (v-cond Eq. ST.1, v&p-cond Eq. ST.2, or every element
 * unknown for Scheme 2, none for HHO_UNCOND) and the assembled level-0
 * operator in the face-block layout.  k in 0..5 (2D) or 0..3 (3D).  Scheme 2
 * contexts support one problem (no hho_set_batch), the block-Jacobi smoother,
 * no learned smoother, and the dense or multifrontal coarse solve;
 * uncondensed contexts likewise one problem, no learned smoother and the dense
 * or multifrontal coarse solve, with element blocks of at most 32 unknowns
 * (2D k <= 3, 3D k <= 1).  stream: a
 * cudaStream_t (NULL = legacy default stream).  *out receives the new
 * context. */
hho_status hho_setup(const hho_mesh* mesh, int k, int cond, void* stream, hho_ctx** out);

/* Number of condensed unknowns at level `level` (0 = fine) after pmg_setup, or
 * at level 0 before it. */
hho_status hho_ndof(const hho_ctx* ctx, int level, int64_t* ndof);

/* Quadrature nodes where the data of hho_assemble are sampled (degree 2k+2
 * rules on the element and face simplex fans).  which = HHO_NODES_ELEM or
 * HHO_NODES_FACE.  *n_nodes receives the count.  If d_xyz (device,
 * n_nodes*dim) is not NULL the coordinates are written there; for the face
 * set, d_normals (device, n_nodes*dim, may be NULL) receives the unit normal
 * pointing out of the face's first element. */
hho_status hho_quad_nodes(hho_ctx* ctx, int which, int64_t* n_nodes, double* d_xyz, double* d_normals);

/* Condensed right-hand side (Eq. ST.1 / Eq. ST.2 right-hand sides) from the
 * body force and boundary data sampled at the nodes of hho_quad_nodes:
 *   d_f   device, n_elem_nodes*dim   f at the element nodes
 *   d_gD  device, n_face_nodes*dim   g_D (read on Dirichlet faces only)
 *   d_gN  device, n_face_nodes*dim   traction (grad u - p I) n_TF1 (read on
 *                                    Neumann faces only)
 *   d_rhs device, ndof(0) or NULL    receives a copy of the condensed RHS. */
hho_status hho_assemble(hho_ctx* ctx, const double* d_f, const double* d_gD, const double* d_gN, double* d_rhs);

/* hho_assemble without allocating memory.  The paper has no counterpart: this
 * entry point serves callers that cannot call cudaMalloc when they refresh the
 * right-hand side -- programs that give all device memory to their own pool,
 * or loops in which a device allocation (which may synchronise the device or
 * fail) is not acceptable.  It computes the same condensed right-hand side as
 * hho_assemble, from the same arguments, but the element kernel's working
 * memory is a fixed array of 2^17 doubles (1 MiB) inside the library, held on
 * every GPU that loads the library until the process exits, instead of memory
 * allocated per call.
 *  - No allocation of any kind is made on success (cudaMalloc, cudaFree,
 *    pools or host heap); on failure the message is stored in the context.
 *  - The first call on a context looks up the device address of the array
 *    with the context's device current and keeps it in the context; if you
 *    capture streams, make that first call before any capture begins.  The
 *    current device must be the context's device.
 *  - The work is only enqueued on the context's stream: the call returns
 *    before the right-hand side is ready (hho_assemble synchronises).
 *  - Every call on a device shares the one array.  The kernel clears what it
 *    reads, so the contents left by the previous call do not matter, but two
 *    calls whose kernels overlap on the GPU (different streams or contexts on
 *    one device, not ordered by events) race on the array; order them.
 *  - Returns HHO_ERR_ARG when one element's local system would need more than
 *    the 2^17 doubles (never for the degrees and element shapes built). */
hho_status hho_assemble_noalloc(hho_ctx* ctx, const double* d_f, const double* d_gD, const double* d_gN,
                                double* d_rhs);

/* Build the p-hierarchy: levels of degrees degrees[0] = k > degrees[1] > ...
 * > degrees[n_levels-1] >= 0, coarse operators by Galerkin block extraction
 * from the fine condensed operator (Sec. 4.2), smoother data (face-block
 * Jacobi with element pressure pivot blocks, or block ILU(0) with option
 * "smoother" = HHO_SMOOTH_ILU), and the exact coarse solver (dense inverse up
 * to "coarse_dense_max" coarse unknowns, nested-dissection multifrontal solver
 * above).  prec: HHO_FP64 (every V-cycle operation in FP64) or HHO_FP32
 * (mixed precision: the level operators, smoother blocks and smoother vectors
 * of every level above the coarse one are stored and multiplied in FP32, and
 * the smoother's arithmetic is FP32 too -- dot products are summed in FP32 per
 * thread, warp and block, the block partials stored as FP64 and added in FP64,
 * the Givens recurrence and basis scaling in FP32; the coarse solve stays FP64
 * unless option "coarse_fp32" = 1; the outer FGMRES, its operator and its CGS2
 * stay FP64).  smooth_its: GMRES iterations per pre/post smoothing (the paper
 * uses 2). */
hho_status pmg_setup(hho_ctx* ctx, int n_levels, const int* degrees, int prec, int smooth_its);

/* Solver options.  "coarse_dense_max", "mf_leaf", "coarse_twolevel",
 * "dd_elements", "coarse_fp32" and "smoother" take effect at the next
 * pmg_setup.  Keys:
 *   "coarse_dense_max"  largest coarse level solved by the dense inverse
 *                       (default 10000 unknowns); larger coarse levels use
 *                       the substructured direct solver
 *   "mf_leaf"           elements per leaf of the nested-dissection tree of
 *                       the multifrontal coarse solver (default 16 in 2D, 8 in
 *                       3D); pmg_setup returns HHO_ERR_UNSUPPORTED when one
 *                       front exceeds the shared-memory staging of its solve
 *                       kernels (about 28000 FP64 unknowns)
 *   "coarse_twolevel"   1: coarse levels above "coarse_dense_max" use the
 *                       two-level substructured solver (subdomain interiors
 *                       eliminated, dense interface inverse; its setup grows
 *                       with the cube of the interface size) instead of the
 *                       multifrontal one; 0 (default): multifrontal
 *   "dd_elements"       target number of elements per subdomain of the
 *                       two-level solver (default 128 in 2D, 64 in 3D;
 *                       rounded so the subdomain count is a power of two);
 *                       pmg_setup returns HHO_ERR_UNSUPPORTED when a subdomain
 *                       has more than 5632 interior unknowns (the interior
 *                       solve stages them in 48 KB of shared memory)
 *   "graphs"            1 (default): pmg_vcycle and hho_solve replay a CUDA
 *                       graph of the V-cycle captured on first use for each
 *                       (input, output) pair of device buffers; 0: launch
 *                       kernels directly.  The legacy default stream is never
 *                       captured.
 *   "spmv_rows"         0 (default): operator kernels specialised for the
 *                       face block size (2, 3, 4, 6, 8, 9, 10, 12, 18, 30
 *                       unknowns), generic kernel for other sizes; 1..4: the
 *                       generic kernel with that many rows of a face or
 *                       element per thread
 *   "spmv_grid"         blocks of 256 threads of the operator kernels,
 *                       1..8192 (0 = automatic: about one 32-row tile per warp)
 *   "smoother"          0 (default): block-Jacobi preconditioner in the
 *                       smoother's GMRES; 1: block ILU(0) (faces in greedy
 *                       multicolour order, element pressures last; factored
 *                       at pmg_setup on every level above the coarse one,
 *                       face blocks of at most 18 and pressure blocks of at
 *                       most 32 unknowns).  Takes effect at the next pmg_setup.
 *   "learned_smoother"  1: add the learned correction (hho_mlp_*) to the
 *                       block-Jacobi output in the finest-level post-smoother;
 *                       0 (default): plain smoother.  HHO_ERR_STATE without
 *                       hho_mlp_init.
 *   "spmv_warp"         1 (default): the FP32 operator and block-Jacobi
 *                       kernels of face blocks of 18, 24, 30 and 40 unknowns
 *                       (3D, k = 2, 3; HHO-hp k = 2, 3) use one warp per
 *                       face; 0: one thread per face
 *   "solve_graph"       1 (default): hho_solve_batch on a non-default stream
 *                       runs as one CUDA graph captured on first use for each
 *                       (x, rtol, maxit, restart): restart cycles in a WHILE
 *                       node, Arnoldi steps in IF nodes, every convergence
 *                       test on the device; 0: host-driven loop (one 16-byte
 *                       read per problem and iteration)
 *   "solve_graph_single" 1: hho_solve (no declared batch, non-default stream)
 *                       runs the same graph-captured FGMRES with one problem;
 *                       0 (default): the host-driven FGMRES of hho_solve
 *   "coarse_fp32"       with HHO_FP32: 1 keeps FP32 copies of the coarse
 *                       solver's inverse blocks and runs the coarse solve in
 *                       FP32 (FP32 multiply-adds, no FP64 round trip);
 *                       0 (default): FP64 coarse solve.  The FP32 coarse
 *                       solve can cost FGMRES iterations when the coarse
 *                       operator is badly conditioned (velocity-pressure
 *                       condensation).  Copies are made at pmg_setup;
 *                       setting 0 afterwards switches back at once.
 * "graphs", "spmv_rows", "spmv_grid", "spmv_warp", "solve_graph" and a later
 * "coarse_fp32" = 0 act at the next V-cycle or solve.  Returns HHO_ERR_ARG for an unknown key or an invalid value. */
hho_status hho_set_option(hho_ctx* ctx, const char* key, double value);

/* One V-cycle MG_V(0, r, 0) of the Algorithm of Sec. 3.3: d_z = MG(d_r).
 * d_r, d_z: device, ndof(0) doubles, may not alias. */
hho_status pmg_vcycle(hho_ctx* ctx, const double* d_r, double* d_z);

/* y = S^l x with the level-l condensed operator (device vectors of ndof(l)). */
hho_status hho_spmv(hho_ctx* ctx, int level, const double* d_x, double* d_y);

/* y = S^l x with the FP32 copy of the level-l operator that a mixed-precision
 * hierarchy (pmg_setup with HHO_FP32) keeps for every level above the coarse
 * one (device vectors of ndof(l) floats).  HHO_ERR_STATE if there is none. */
hho_status hho_spmv_f32(hho_ctx* ctx, int level, const float* d_x, float* d_y);

/* FGMRES (Sec. 3.3) on S x = rhs (the RHS of the last hho_assemble) with one
 * V-cycle per iteration, CGS2 orthogonalisation, x0 = 0, restart `restart`,
 * stopping at ||rhs - S x|| <= rtol ||rhs||.  d_x: device, ndof(0).  info may
 * be NULL.  Returns HHO_ERR_NOT_CONVERGED if maxit is reached. */
hho_status hho_solve(hho_ctx* ctx, double rtol, int maxit, int restart, double* d_x, hho_solve_info* info);

/* Batches of independent problems (no counterpart in the paper).  Declares the
 * context's mesh a disjoint union of n_prob (1..65535) problems: problem p owns faces
 * [face_off[p], face_off[p+1]) and elements [elem_off[p], elem_off[p+1])
 * (host arrays of n_prob + 1, copied; face_off[0] = elem_off[0] = 0, last
 * entries the face and element counts; no face may touch an element of
 * another problem: HHO_ERR_MESH).  Call between hho_setup and pmg_setup
 * (HHO_ERR_STATE afterwards, and pmg_setup must then be called again).
 * Every level operator is block diagonal, so one launch of each V-cycle kernel
 * serves all problems; a problem without Neumann face gets its own constant-
 * pressure kernel treatment (projection, coarse pin). */
hho_status hho_set_batch(hho_ctx* ctx, int n_prob, const int64_t* face_off, const int64_t* elem_off);

/* One FGMRES per problem of a declared batch (Sec. 3.3: one V-cycle per
 * iteration, CGS2, x0 = 0), all advanced in lockstep with per-problem
 * (segmented) dot products, each stopping at ||rhs_p - S_p x_p|| <=
 * rtol ||rhs_p||; a converged problem is frozen while the others go on.
 * With option "solve_graph" (default) and a non-default stream the whole
 * solve is one graph launch with device-side control; the results are read
 * back once it has finished.  The
 * V-cycle is the union's (its smoother's Krylov coefficients are shared by the
 * batch, which flexible GMRES admits).  d_x: device, ndof(0).  h_iters
 * (host, n_prob, may be NULL): iteration at which each problem converged;
 * h_relres (host, n_prob, may be NULL): each problem's final true relative
 * residual.  info: batch totals (iterations of the lockstep loop, the largest
 * relative residual, wall time).  HHO_ERR_NOT_CONVERGED if some problem is
 * above rtol after maxit iterations. */
hho_status hho_solve_batch(hho_ctx* ctx, double rtol, int maxit, int restart, double* d_x, int32_t* h_iters,
                           double* h_relres, hho_solve_info* info);

/* Learned block smoother (no counterpart in the paper).  A two-layer MLP
 * (hidden width `hidden`, BF16 weights, FP32 accumulation) maps the residual
 * of a face's neighbourhood -- the residual blocks of the faces in the face's
 * operator slots (the face, the other faces of its first element, of its
 * second) and the pressure blocks of its two elements, divided by their norm
 * s_F -- to a correction s_F y_F of the block-Jacobi output on the face's rows
 * in the finest-level post-smoother (option "learned_smoother" = 1; the plain
 * smoother is the fallback).  All entry points need pmg_setup first.
 *
 * hho_mlp_init: sizes from the finest level (d_in = slots*b + 2 nP padded to
 * a multiple of 16, at most 256; d_out = b padded to a multiple of 8) and a
 * seeded initialisation; hidden in 8..256, multiple of 8. */
hho_status hho_mlp_init(hho_ctx* ctx, int hidden, uint64_t seed);

/* dims (host, 4): {d_in, hidden, d_out, raw feature count}. */
hho_status hho_mlp_dims(hho_ctx* ctx, int32_t* dims);

/* Get (set = 0) or set (set = 1) the FP32 master parameters (host, row-major:
 * W1 d_in x hidden, b1 hidden, W2 hidden x d_out, b2 d_out); setting refreshes
 * the BF16 copies. */
hho_status hho_mlp_weights(hho_ctx* ctx, int set, double* W1, double* b1, double* W2, double* b2);

/* Network inputs of a finest-level vector d_r (device, ndof(0)): d_X (device,
 * nf x d_in floats holding the BF16-rounded normalised features) and d_s
 * (device, nf floats: the norms s_F). */
hho_status hho_mlp_features(hho_ctx* ctx, const double* d_r, float* d_X, float* d_s);

/* The learned correction as the finest-level post-smoother applies it (test
 * hook): d_z[F's rows] += s_F y_F for every face F, y = the network's output
 * on the normalised BF16 features of d_v (device, ndof(0) doubles each;
 * element rows of d_z are left unchanged; d_v and d_z may not alias). */
hho_status hho_mlp_apply(hho_ctx* ctx, const double* d_v, double* d_z);

/* Training set from the FP64 V-cycle (pmg_setup with HHO_FP64, learned
 * smoother off) applied to r0 = S e0 for n_vec (1..4096) seeded white-noise
 * errors e0: kind 0 takes the pair it is applied to (e = e0, r = r0), kind 1
 * the pair it leaves (e = e0 - MG(r0), r = S e), kind 2 the pair its
 * finest-level post-smoother meets (e = e0 - x with x the iterate after the
 * coarse correction, r = S e; the distribution the learned correction acts
 * on).  One sample per face, target (e_F - (M_J^{-1} r)_F) / s_F.
 * *n_samples (may be NULL) = n_vec * nf. */
hho_status hho_mlp_generate(hho_ctx* ctx, int n_vec, uint64_t seed, int kind, int64_t* n_samples);

/* `steps` Adam steps (lr, beta = 0.9 / 0.999) on minibatches of `batch` samples
 * drawn with `seed`; loss = mean over samples of ||y - t||^2.  h_loss (host,
 * steps doubles, may be NULL) receives each step's loss. */
hho_status hho_mlp_train(hho_ctx* ctx, int steps, int batch, double lr, uint64_t seed, double* h_loss);

/* Loss and parameter gradients of the training kernels for a given
 * minibatch: d_X (device, batch x d_in floats), d_T (device, batch x d_out);
 * host outputs as in hho_mlp_weights. */
hho_status hho_mlp_grads(hho_ctx* ctx, const float* d_X, const float* d_T, int batch, double* h_loss, double* h_gW1,
                         double* h_gb1, double* h_gW2, double* h_gb2);

/* Block ILU(0) smoother preconditioner of level `level` (option "smoother" = 1
 * before pmg_setup): d_z = (L U)^{-1} d_v (device, ndof(level) doubles, FP64
 * factors).  HHO_ERR_STATE if the level has no factors. */
hho_status hho_ilu_apply(hho_ctx* ctx, int level, const double* d_v, double* d_z);

/* Autotuner (after pmg_setup): times `reps` V-cycles for every candidate of
 * "spmv_rows" (0, 2, 4) x "spmv_grid" (automatic, 1216, 2432) and, for a
 * declared batch, `reps` segmented update kernels for tile sizes 1024 ..
 * 8192 unknowns, and keeps the fastest.  h_choice (host, 3 doubles, may be
 * NULL) receives {spmv_rows, spmv_grid, tile_rows}.  reps in 1..1000. */
hho_status hho_autotune(hho_ctx* ctx, int reps, double* h_choice);

/* Back-substitution of the eliminated unknowns (Eq. ST.1 / ST.2): for every
 * element the full local vector [U_T | U_F1 .. U_FN | P_T] (velocity
 * component-major, orthonormal element/face bases) from the condensed
 * solution d_x (device, ndof(0)).  d_local: device, sum over elements of
 * (d*n_E + N*d*n_F + n_E) doubles, elements in order. */
hho_status hho_recover(hho_ctx* ctx, const double* d_x, double* d_local);

/* L2 errors of Sec. 5.2.2 from recovered local vectors and exact values at the
 * element nodes of hho_quad_nodes: d_u (n*dim), d_gradu (n*dim*dim, row i =
 * d u_i / d x_j), d_p (n).  out[4] (host) = ||P u_h - u||, ||grad(P u_h - u)||,
 * ||p_h - p|| (both means removed when no Neumann face exists), ||div u_T||. */
hho_status hho_errors(hho_ctx* ctx, const double* d_local, const double* d_u, const double* d_gradu,
                      const double* d_p, double out[4]);

/* Test hooks (exact-input parity checks).  Copy to host the element Schur
 * complements S_T (elements in order, each n_k*n_k row-major over the kept
 * local unknowns [U_F1 .. U_FN | pressure block]); *count receives the total
 * number of doubles (host_out may be NULL to query). */
hho_status hho_get_element_schur(hho_ctx* ctx, double* host_out, int64_t* count);

/* Copy the level-l operator to host as COO triplets of its stored blocks
 * (explicit zeros included).  Query with null arrays to get *nnz. */
hho_status hho_get_level_coo(hho_ctx* ctx, int level, int64_t* rows, int64_t* cols, double* vals, int64_t* nnz);

/* Replace the element Schur complements by host values (same layout as
 * hho_get_element_schur) and re-assemble the level-0 operator; the RHS and
 * hierarchy must be rebuilt afterwards (hho_assemble is unaffected). */
hho_status hho_set_element_schur(hho_ctx* ctx, const double* host_in);

/* Coarse solver of the current hierarchy (after pmg_setup): info (host, 4)
 * = {kind: 0 dense inverse, 1 two-level substructuring, 2 multifrontal;
 * stored operator values one coarse solve reads; kernel launches per coarse
 * solve (without the pressure-kernel projection); values of the dense
 * factorisation workspace (multifrontal: freed after pmg_setup)}. */
hho_status hho_coarse_info(hho_ctx* ctx, int64_t* info);

/* Number of kernels the library has launched on this context since setup
 * (counts every launch of the solver, V-cycle and SpMV entry points). */
hho_status hho_launch_count(const hho_ctx* ctx, int64_t* launches);

hho_status hho_destroy(hho_ctx* ctx);
const char* hho_last_error(const hho_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* HHO_H */
