// Internal declarations shared by the translation units of libhho.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/hho.h"

namespace hho {

constexpr int MAX_K2 = 5;       // highest face degree built in 2D
constexpr int MAX_K3 = 3;       // highest face degree built in 3D
constexpr int MAX_NFACE = 8;    // faces per element
constexpr int MAX_FVERT = 4;    // vertices per 3D face
constexpr int MAX_GL = 16;      // Gauss-Legendre tables 1..MAX_GL points

__host__ __device__ inline int dimP(int nvar, int deg) {
    if (deg < 0) return 0;
    if (nvar == 0) return 1;
    if (nvar == 1) return deg + 1;
    if (nvar == 2) return (deg + 1) * (deg + 2) / 2;
    return (deg + 1) * (deg + 2) * (deg + 3) / 6;
}

// Geometry of a face (written by the face kernel, read by the element kernels).
struct FaceGeo {
    double xF[3];   // vertex average
    double n[3];    // fixed unit normal
    double t1[3];   // tangent frame
    double t2[3];
    double bc[2];   // bounding-box centre in the frame
    double br[2];   // bounding-box half widths in the frame
    double hF;      // diameter
    double meas;    // measure
};

// Device-resident mesh and per-element/per-face data of the fine discretisation.
struct Disc {
    int d = 0, k = 0, cond = 0;
    int64_t nv = 0, ne = 0, nf = 0;
    int nR = 0, nE = 0, nF = 0, b = 0, nP = 0;
    int maxN = 0;                 // most faces of one element
    // mesh (device)
    double* xyz = nullptr;
    int32_t* ef_ptr = nullptr;    // element -> faces CSR
    int32_t* ef = nullptr;
    int32_t* fv_ptr = nullptr;    // face -> vertices CSR
    int32_t* fv = nullptr;
    int32_t* fe = nullptr;        // 2 per face
    int32_t* flf = nullptr;       // local index of the face in each of its elements, 2 per face
    int8_t* fbc = nullptr;
    // geometry and bases (device)
    FaceGeo* fgeo = nullptr;
    double* fC = nullptr;         // face basis coefficients, nF*nF per face
    double* eC = nullptr;         // element basis coefficients, nR*nR per element
    double* emeas = nullptr;      // |T|
    // local operators (device), per element offsets in the arrays below
    int64_t* off_S = nullptr;     // S_T (nk*nk)
    int64_t* off_X = nullptr;     // X = Kee^{-1} Kek (ne_el*nk)
    int64_t* off_Kei = nullptr;   // Kee^{-1} (ne_el*ne_el)
    int64_t* off_P = nullptr;     // reconstruction (nR*ns)
    int64_t* off_loc = nullptr;   // full local vector offsets (recovery output)
    double* S = nullptr;
    double* X = nullptr;
    double* Kei = nullptr;
    double* P = nullptr;
    double* gT = nullptr;         // condensed local RHS, nk per element (off_gT)
    double* yT = nullptr;         // Kee^{-1} rhs_e (recovery), per element (off_yT)
    int64_t* off_gT = nullptr;
    int64_t* off_yT = nullptr;
    std::vector<int64_t> h_off_S, h_off_loc, h_off_gT;
    int64_t tot_S = 0, tot_X = 0, tot_Kei = 0, tot_P = 0, tot_loc = 0, tot_gT = 0, tot_yT = 0;
    // data nodes
    int64_t n_enodes = 0, n_fnodes = 0;
    int64_t* enode_off = nullptr; // per element
    int64_t* fnode_off = nullptr; // per face
    std::vector<int64_t> h_enode_off, h_fnode_off;
    // Gauss-Legendre tables on [0,1]
    double* gl = nullptr;         // [MAX_GL+1][MAX_GL] nodes then weights
    // host copies of topology
    std::vector<int32_t> h_ef_ptr, h_ef, h_fe, h_flf, h_fv_ptr, h_fv;
    std::vector<double> h_xyz;
    std::vector<int8_t> h_fbc;
};

// Block layout of one level operator (face-block ELL, values innermost over rows).
struct LevelMat {
    int k = 0, nF = 0, b = 0, nP = 0;
    int64_t nf = 0, ne = 0, n = 0;
    int S_max = 0;    // face slots per face row
    int N_max = 0;    // face slots per element row
    // topology (device, shared layout across levels)
    const int32_t* ff_col = nullptr;  // [S_max][nf]
    const int32_t* ff_nsl = nullptr;  // [nf]
    const int32_t* fp_col = nullptr;  // [2][nf]  (-1 = none)
    const int32_t* pf_col = nullptr;  // [N_max][ne]
    const int32_t* pf_nsl = nullptr;  // [ne]
    // values (device, FP64)
    double* ff = nullptr;   // [S_max][b c][b r][nf]
    double* fp = nullptr;   // [2][nP c][b r][nf]
    double* pf = nullptr;   // [N_max][b c][nP r][ne]
    double* pp = nullptr;   // [nP c][nP r][ne]
    // smoother data
    double* dinv = nullptr; // [b c][b r][nf]
    double* minv = nullptr; // [nP c][nP r][ne]
    // FP32 copies used by a mixed-precision V-cycle: the layouts above, or with
    // ilv set the row-interleaved layouts (rows of one face / element block
    // contiguous for each column: ff[s][c][F][r], fp[p][c][F][r], pf[f][c][T][r],
    // pp[c][T][r], dinv[c][F][r], minv[c][T][r]) read by the one-thread-per-block kernels
    float *ff32 = nullptr, *fp32 = nullptr, *pf32 = nullptr, *pp32 = nullptr, *dinv32 = nullptr, *minv32 = nullptr;
    bool ilv = false;
};

struct Topo {
    int S_max = 0, N_max = 0;
    int32_t *ff_col = nullptr, *ff_nsl = nullptr, *fp_col = nullptr, *pf_col = nullptr, *pf_nsl = nullptr;
    // assembly sources for level 0
    int32_t* asm_T = nullptr;   // [S_max][nf] element of the off-diagonal / first diag source
    int32_t* asm_lf = nullptr;  // [S_max][nf] local index of the row face in that element
    int32_t* asm_lg = nullptr;  // [S_max][nf] local index of the column face in that element
    std::vector<int32_t> h_ff_col, h_ff_nsl, h_fp_col, h_pf_col, h_pf_nsl;
};

struct Workspace;     // solver work vectors (solve.cu)
struct CoarseSolver;  // coarse-level solver (coarse.cu)
struct BatchWork;     // segmented FGMRES state of a batch (batch.cu)
struct Learned;       // learned block smoother (learned.cu)
struct IluLevel;      // block ILU(0) factors of one level (ilu.cu)
struct MFSolver;      // multifrontal coarse solver (multifrontal.cu)

// Partition of the mesh into independent problems (a disjoint union): problem
// p owns faces [face_off[p], face_off[p+1]) and elements [elem_off[p],
// elem_off[p+1]).  A context without a declared batch is one problem.
struct Problems {
    int P = 1;
    std::vector<int64_t> face_off, elem_off;
    std::vector<int32_t> elem_prob;  // problem of every element
    std::vector<char> has_null;      // no Neumann face: constant pressure in the kernel
    bool declared = false;           // hho_set_batch was called
};

}  // namespace hho

struct hho_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    hho::Disc disc;
    hho::Topo topo;
    std::vector<hho::LevelMat> levels;   // levels[0] always present after setup
    bool have_rhs = false, have_pmg = false;
    double* rhs = nullptr;               // condensed RHS (level 0)
    int smooth_its = 2;
    int prec = 0;
    std::vector<int> degrees;
    double* null_vec0 = nullptr;         // per-problem unit constant-pressure vectors at level 0 (or null)
    bool has_null = false;               // some problem has a pressure kernel
    hho::Problems probs;                 // problem partition (one problem unless a batch is declared)
    double* null_w = nullptr;            // per kernel slot: its weight in its problem's unit kernel vector
                                         // (0 for problems without kernel).  Slots: every element's first
                                         // pressure unknown (Scheme 1) or every face's constant face-pressure
                                         // coefficient (HHO-hp)
    std::vector<double> h_null_w;        // host copy of null_w
    int64_t* d_null_off = nullptr;       // device copy of the slot ranges per problem (probs.elem_off, or
                                         // probs.face_off for HHO-hp)
    int null_nch = 1;                    // chunks per problem of the projection kernels
    double* null_part = nullptr;         // their partial products (problems x chunks)
    hho::BatchWork* batch = nullptr;
    int tile_rows = 2048;                // rows of the condensed vector per block in the segmented kernels
    hho::Learned* learned = nullptr;     // learned smoother network (or null)
    int smoother_kind = 0;               // 0 block Jacobi, 1 block ILU(0) (from the next pmg_setup)
    std::vector<hho::IluLevel*> ilu;     // ILU factors per level (smoother_kind 1)
    int use_learned = 0;                 // apply it in the finest-level post-smoother
    void* capture = nullptr;             // when set: the finest-level iterate after the coarse correction
                                         // is copied here (direct V-cycles only)
    hho::Workspace* ws = nullptr;
    hho::CoarseSolver* coarse = nullptr;
    int64_t coarse_its_total = 0;
    int* d_flag = nullptr;               // device status word for bounded waits / breakdowns
    int64_t launches = 0;                // kernels launched by the solver entry points
    double* noalloc_scratch = nullptr;   // device address of the no-alloc assembly array, looked up
                                         // on this context's first hho_assemble_noalloc call
    int64_t coarse_dense_max = 10000;    // options
    int64_t dd_elements = 0;             // 0 = default per dimension
    int coarse_fp32 = 0;                 // mixed precision: FP32 coarse solve operators
    int coarse_twolevel = 0;             // coarse levels above coarse_dense_max: 1 two-level substructuring,
                                         // 0 multifrontal (default)
    int64_t mf_leaf = 0;                 // elements per leaf of the multifrontal tree (0 = default per dimension)
    bool use_graphs = true;              // replay captured V-cycles
    int spmv_rows = 0;                   // rows per thread of the operator kernels (0 = automatic)
    int spmv_grid = 0;                   // blocks of the operator kernels (0 = automatic)
    int solve_graph = 1;                 // hho_solve_batch as one captured CUDA graph (device-side control)
    int solve_graph_single = 0;          // hho_solve through the same graph (one problem) instead of the
                                         // host-driven FGMRES
    int spmv_warp = 1;                   // FP32 operator of large 3D face blocks: warp per face (1) or
                                         // a face's rows split over two threads (0)
};

// ---- helpers shared across units ----
#define HHO_CUDA(call)                                                          \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) {                                                 \
            ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);       \
            return HHO_ERR_CUDA;                                                 \
        }                                                                        \
    } while (0)

#define HHO_TRY(call)                   \
    do {                                \
        hho_status s_ = (call);         \
        if (s_ != HHO_OK) return s_;    \
    } while (0)

namespace hho {
hho_status device_alloc(hho_ctx* ctx, void** p, size_t bytes);
template <class T>
inline hho_status dalloc(hho_ctx* ctx, T** p, size_t count) {
    return device_alloc(ctx, reinterpret_cast<void**>(p), count * sizeof(T));
}
void dfree(void* p);
// streaming multiprocessors of the current device (queried once per device)
int sm_count();
// largest dynamic shared memory a block may opt in to on the current device
int smem_optin();
// Allow `fn` the device's largest dynamic shared memory.  The limit is a
// process-wide attribute of the kernel, not of a context, so every context
// raises it to the maximum rather than to its own need (a later context with
// smaller fronts must not lower it below an earlier one's); occupancy follows
// the shared memory a launch actually requests.  HHO_ERR_UNSUPPORTED when
// `need` exceeds the device's limit.
template <class F>
inline hho_status allow_smem(hho_ctx* ctx, F* fn, size_t need) {
    const int mx = smem_optin();
    if ((int64_t)need > (int64_t)mx) {
        ctx->err = "a kernel needs " + std::to_string(need) + " bytes of shared memory, more than the device's " +
                   std::to_string(mx);
        return HHO_ERR_UNSUPPORTED;
    }
    // the limit covers static and dynamic shared memory together
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e == cudaSuccess && need + fa.sharedSizeBytes > (size_t)mx) {
        ctx->err = "a kernel needs " + std::to_string(need + fa.sharedSizeBytes) +
                   " bytes of shared memory, more than the device's " + std::to_string(mx);
        return HHO_ERR_UNSUPPORTED;
    }
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, mx - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess) {
        ctx->err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
        return HHO_ERR_CUDA;
    }
    return HHO_OK;
}

// setup.cu
hho_status build_discretisation(hho_ctx* ctx, const hho_mesh* m, int k, int cond);
hho_status build_rhs(hho_ctx* ctx, const double* f, const double* gD, const double* gN);
hho_status build_rhs_scratch(hho_ctx* ctx, const double* f, const double* gD, const double* gN, double* scratch,
                             int64_t capacity);
hho_status quad_nodes(hho_ctx* ctx, int which, int64_t* n, double* xyz, double* normals);
hho_status recover_local(hho_ctx* ctx, const double* x, double* local);
hho_status compute_errors(hho_ctx* ctx, const double* local, const double* u, const double* gu,
                          const double* p, double out[4]);
// assemble.cu
hho_status build_topology(hho_ctx* ctx);
hho_status assemble_level0(hho_ctx* ctx);
// DG scheme: element-block level-0 operator (setup.cu)
hho_status dg_assemble_level0(hho_ctx* ctx, double* ff, int S_max);
hho_status assemble_rhs_vector(hho_ctx* ctx, double* rhs);
hho_status build_level(hho_ctx* ctx, int l, int k_l);
hho_status build_smoother(hho_ctx* ctx, int l);
hho_status level_coo(hho_ctx* ctx, int l, int64_t* rows, int64_t* cols, double* vals, int64_t* nnz);
void free_level(hho::LevelMat& L);
// solve.cu
hho_status pmg_build(hho_ctx* ctx);
hho_status spmv(hho_ctx* ctx, int l, const double* x, double* y);
hho_status spmv_f32(hho_ctx* ctx, int l, const float* x, float* y);
hho_status vcycle(hho_ctx* ctx, const double* r, double* z);
hho_status fgmres(hho_ctx* ctx, double rtol, int maxit, int restart, double* x, hho_solve_info* info);
void free_workspace(hho_ctx* ctx);
void invalidate_graphs(hho_ctx* ctx);
hho_status residual(hho_ctx* ctx, int l, const double* x, const double* b, double* r);
hho_status null_build(hho_ctx* ctx);
// x -= (n_p . x) n_p for every problem p with a pressure kernel, x a vector of
// level L (one block per problem)
template <typename T>
hho_status null_project(hho_ctx* ctx, const LevelMat& L, T* x);
// components of an element block, each truncated on its own by the
// restriction: d + 1 (velocity, pressure) uncondensed, else 1 (a prefix of
// kept pressure coefficients)
inline int elem_comp(int cond, int d) { return cond == HHO_UNCOND ? d + 1 : 1; }
// position of the constant pressure mode in an element block of nP unknowns
inline int mean_slot(int cond, int d, int nP) { return cond == HHO_UNCOND ? d * (nP / (d + 1)) : 0; }
// index of kernel slot i (element or face, see hho_ctx::null_w) in a vector of level L
// HHO-hp (face pressure) and DG (element pressure in the block rows): the
// constant pressure sits in component d of the block rows
inline bool null_in_blocks(int cond) { return cond == HHO_HPCOND || cond == HHO_DGCOND; }
inline int64_t null_slot(const hho_ctx* ctx, const LevelMat& L, int64_t i) {
    if (null_in_blocks(ctx->disc.cond)) return i * L.b + (int64_t)ctx->disc.d * L.nF;
    return L.nf * L.b + i * L.nP + mean_slot(ctx->disc.cond, ctx->disc.d, L.nP);
}
// v = r / *den, z = M^{-1} v with the level-0 block-Jacobi preconditioner (FP64)
hho_status jacobi_apply(hho_ctx* ctx, const double* r, const double* den, double* v, double* z);
// learned.cu
hho_status mlp_init(hho_ctx* ctx, int hidden, uint64_t seed);
void mlp_free(hho_ctx* ctx);
hho_status mlp_dims(hho_ctx* ctx, int* dims);
hho_status mlp_weights(hho_ctx* ctx, int set, double* W1, double* b1, double* W2, double* b2);
hho_status mlp_features(hho_ctx* ctx, const double* r, float* X, float* s);
template <typename T>
hho_status mlp_apply(hho_ctx* ctx, const T* v, T* z);
hho_status mlp_status(hho_ctx* ctx);
hho_status mlp_generate(hho_ctx* ctx, int n_vec, uint64_t seed, int kind, int64_t* nsamp);
hho_status mlp_train(hho_ctx* ctx, int steps, int batch, double lr, uint64_t seed, double* h_loss);
hho_status mlp_grads(hho_ctx* ctx, const float* X, const float* T, int B, double* loss, double* gW1, double* gb1,
                     double* gW2, double* gb2);
// ilu.cu
hho_status ilu_setup(hho_ctx* ctx, int l, bool fp32);
template <typename T>
hho_status ilu_apply(hho_ctx* ctx, int l, const T* v, T* z, T* tmp);
void ilu_free(hho_ctx* ctx);
// batch.cu
hho_status batch_set(hho_ctx* ctx, int P, const int64_t* face_off, const int64_t* elem_off);
hho_status batch_solve(hho_ctx* ctx, double rtol, int maxit, int restart, double* x, int32_t* its,
                       double* relres, hho_solve_info* info);
hho_status autotune(hho_ctx* ctx, int reps, double* choice);
void batch_free(hho_ctx* ctx);
void batch_graph_free(hho_ctx* ctx);
// coarse.cu
hho_status coarse_setup(hho_ctx* ctx);
hho_status coarse_apply(hho_ctx* ctx, const double* d, double* c);
// FP32 coarse solve (FP32 copies of the solve operators; only when they exist)
bool coarse_has_f32(const hho_ctx* ctx);
hho_status coarse_apply_f32(hho_ctx* ctx, const float* d, float* c);
void coarse_free(hho_ctx* ctx);
// bytes of the stored operators one coarse solve reads
int64_t coarse_solve_bytes(const hho_ctx* ctx, int value_bytes);
// multifrontal.cu
hho_status mf_build(hho_ctx* ctx, int64_t leaf, MFSolver** out);
hho_status mf_make_f32(hho_ctx* ctx, MFSolver* S);
bool mf_has_f32(const MFSolver* S);
int mf_levels(const MFSolver* S);
// kernel launches of one solve with values of value_bytes (8 FP64, 4 FP32)
int mf_launches(const MFSolver* S, int value_bytes);
int64_t mf_factor_doubles(const MFSolver* S);
hho_status coarse_info(const hho_ctx* ctx, int64_t out[4]);
int64_t mf_solve_bytes(const MFSolver* S, int value_bytes);
template <typename T>
hho_status mf_apply(hho_ctx* ctx, MFSolver* S, const T* d, T* c);
void mf_free(MFSolver* S);
}  // namespace hho
