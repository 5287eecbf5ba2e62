// C ABI entry points of libhho (declared in include/hho.h).
#include <cstring>
#include <new>
#include <string>

#include "internal.h"

namespace hho {

hho_status device_alloc(hho_ctx* ctx, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 8;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->err = std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e);
        *p = nullptr;
        return HHO_ERR_NOMEM;
    }
    return HHO_OK;
}

int sm_count() {
    constexpr int kMaxDev = 64;
    static int cache[kMaxDev] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) dev = -1;
    if (dev >= 0 && cache[dev] > 0) return cache[dev];
    int s = 0;
    if (dev < 0 || cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || s <= 0)
        return 1;  // no device answer: a one-SM grid cap is always valid
    cache[dev] = s;
    return s;
}

int smem_optin() {
    constexpr int kMaxDev = 64;
    static int cache[kMaxDev] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) dev = -1;
    if (dev >= 0 && cache[dev] > 0) return cache[dev];
    int s = 0;
    if (dev < 0 || cudaDeviceGetAttribute(&s, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || s <= 0)
        return 48 * 1024;
    cache[dev] = s;
    return s;
}

void dfree(void* p) {
    if (p) cudaFree(p);
}

static hho_status check_mesh(hho_ctx* ctx, const hho_mesh* m, int k) {
    auto bad = [&](const char* why) {
        ctx->err = std::string("hho_setup: ") + why;
        return HHO_ERR_MESH;
    };
    if (m->dim != 2 && m->dim != 3) return bad("dim must be 2 or 3");
    if ((m->dim == 2 && (k < 0 || k > MAX_K2)) || (m->dim == 3 && (k < 0 || k > MAX_K3))) {
        ctx->err = "hho_setup: degree k not built for this dimension";
        return HHO_ERR_UNSUPPORTED;
    }
    if (m->n_vert <= 0 || m->n_elem <= 0 || m->n_face <= 0) return bad("empty mesh");
    if (!m->xyz || !m->elem_face_ptr || !m->elem_face || !m->face_vert_ptr || !m->face_vert || !m->face_elem || !m->face_bc)
        return bad("null mesh array");
    if (m->n_elem > INT32_MAX || m->n_face > INT32_MAX || m->n_vert > INT32_MAX) return bad("mesh too large");
    if (m->elem_face_ptr[0] != 0 || m->face_vert_ptr[0] != 0) return bad("CSR offsets must start at 0");
    for (int64_t t = 0; t < m->n_elem; ++t) {
        int64_t N = m->elem_face_ptr[t + 1] - m->elem_face_ptr[t];
        if (N < m->dim + 1 || N > MAX_NFACE || (m->dim == 3 && N > 6)) return bad("unsupported number of element faces");
        for (int64_t i = m->elem_face_ptr[t]; i < m->elem_face_ptr[t + 1]; ++i)
            if (m->elem_face[i] < 0 || m->elem_face[i] >= m->n_face) return bad("element face index out of range");
    }
    std::vector<int> seen(m->n_face, 0);
    for (int64_t t = 0; t < m->n_elem; ++t)
        for (int64_t i = m->elem_face_ptr[t]; i < m->elem_face_ptr[t + 1]; ++i) {
            int64_t F = m->elem_face[i];
            if (m->face_elem[2 * F] != t && m->face_elem[2 * F + 1] != t) return bad("face_elem does not list an element of the face");
            ++seen[F];
        }
    for (int64_t F = 0; F < m->n_face; ++F) {
        int64_t nv = m->face_vert_ptr[F + 1] - m->face_vert_ptr[F];
        if ((m->dim == 2 && nv != 2) || (m->dim == 3 && (nv < 3 || nv > MAX_FVERT))) return bad("unsupported face vertex count");
        for (int64_t i = m->face_vert_ptr[F]; i < m->face_vert_ptr[F + 1]; ++i)
            if (m->face_vert[i] < 0 || m->face_vert[i] >= m->n_vert) return bad("face vertex index out of range");
        int64_t T1 = m->face_elem[2 * F], T2 = m->face_elem[2 * F + 1];
        if (T1 < 0 || T1 >= m->n_elem || T2 >= m->n_elem || T2 == T1) return bad("invalid face_elem entry");
        int expect = (T2 >= 0) ? 2 : 1;
        if (seen[F] != expect) return bad("face_elem inconsistent with elem_face");
        int8_t bc = m->face_bc[F];
        if (bc < 0 || bc > 2) return bad("face_bc must be 0, 1 or 2");
        if ((T2 >= 0) != (bc == 0)) return bad("boundary tag on an interior face or interior tag on a boundary face");
    }
    return HHO_OK;
}

}  // namespace hho

using namespace hho;

extern "C" {

hho_status hho_setup(const hho_mesh* mesh, int k, int cond, void* stream, hho_ctx** out) {
    if (!out) return HHO_ERR_ARG;
    *out = nullptr;
    hho_ctx* ctx = new (std::nothrow) hho_ctx();
    if (!ctx) return HHO_ERR_NOMEM;
    *out = ctx;
    if (!mesh) {
        ctx->err = "hho_setup: null mesh";
        return HHO_ERR_ARG;
    }
    if (cond != HHO_VCOND && cond != HHO_VPCOND && cond != HHO_HPCOND && cond != HHO_UNCOND && cond != HHO_DGCOND) {
        ctx->err = "hho_setup: cond must be HHO_VCOND, HHO_VPCOND, HHO_HPCOND, HHO_UNCOND or HHO_DGCOND";
        return HHO_ERR_ARG;
    }
    HHO_TRY(check_mesh(ctx, mesh, k));
    if (cond == HHO_DGCOND && (k < 1 || (mesh->dim == 2 && k > 3) || (mesh->dim == 3 && k > 2))) {
        ctx->err = "hho_setup: the DG scheme takes k >= 1 with at most 10 coefficients per component (2D k <= 3, 3D k <= 2)";
        return HHO_ERR_UNSUPPORTED;
    }
    HHO_CUDA(cudaGetDevice(&ctx->device));
    ctx->stream = reinterpret_cast<cudaStream_t>(stream);
    HHO_TRY(dalloc(ctx, &ctx->d_flag, 4));
    HHO_TRY(build_discretisation(ctx, mesh, k, cond));
    HHO_TRY(build_topology(ctx));
    HHO_TRY(assemble_level0(ctx));
    HHO_TRY(dalloc(ctx, &ctx->rhs, (size_t)ctx->levels[0].n));
    // one problem until a batch is declared
    Problems& pr = ctx->probs;
    pr.P = 1;
    pr.face_off = {0, ctx->disc.nf};
    pr.elem_off = {0, ctx->disc.ne};
    pr.elem_prob.assign(ctx->disc.ne, 0);
    pr.declared = false;
    return HHO_OK;
}

hho_status hho_set_batch(hho_ctx* ctx, int n_prob, const int64_t* face_off, const int64_t* elem_off) {
    if (!ctx || !face_off || !elem_off) return HHO_ERR_ARG;
    if (ctx->disc.cond == HHO_HPCOND || ctx->disc.cond == HHO_UNCOND || ctx->disc.cond == HHO_DGCOND) {
        ctx->err = "hho_set_batch: HHO-hp, uncondensed and DG contexts hold one problem";
        return HHO_ERR_UNSUPPORTED;
    }
    HHO_TRY(batch_set(ctx, n_prob, face_off, elem_off));
    return HHO_OK;
}

hho_status hho_solve_batch(hho_ctx* ctx, double rtol, int maxit, int restart, double* d_x, int32_t* h_iters,
                           double* h_relres, hho_solve_info* info) {
    if (!ctx || !d_x) return HHO_ERR_ARG;
    if (!ctx->have_pmg || !ctx->have_rhs) {
        ctx->err = "hho_solve_batch: call hho_assemble and pmg_setup first";
        return HHO_ERR_STATE;
    }
    return batch_solve(ctx, rtol, maxit, restart, d_x, h_iters, h_relres, info);
}

hho_status hho_mlp_init(hho_ctx* ctx, int hidden, uint64_t seed) {
    if (ctx && (ctx->disc.cond == HHO_HPCOND || ctx->disc.cond == HHO_UNCOND || ctx->disc.cond == HHO_DGCOND)) {
        ctx->err = "hho_mlp_init: the learned smoother is built for condensed Scheme 1 (element pressure rows)";
        return HHO_ERR_UNSUPPORTED;
    }
    if (!ctx) return HHO_ERR_ARG;
    return mlp_init(ctx, hidden, seed);
}

hho_status hho_mlp_dims(hho_ctx* ctx, int32_t* dims) {
    if (!ctx || !dims) return HHO_ERR_ARG;
    int d[4];
    HHO_TRY(mlp_dims(ctx, d));
    for (int i = 0; i < 4; ++i) dims[i] = d[i];
    return HHO_OK;
}

hho_status hho_mlp_weights(hho_ctx* ctx, int set, double* W1, double* b1, double* W2, double* b2) {
    if (!ctx || !W1 || !b1 || !W2 || !b2 || (set != 0 && set != 1)) return HHO_ERR_ARG;
    return mlp_weights(ctx, set, W1, b1, W2, b2);
}

hho_status hho_mlp_features(hho_ctx* ctx, const double* d_r, float* d_X, float* d_s) {
    if (!ctx || !d_r || !d_X || !d_s) return HHO_ERR_ARG;
    return mlp_features(ctx, d_r, d_X, d_s);
}

hho_status hho_mlp_apply(hho_ctx* ctx, const double* d_v, double* d_z) {
    if (!ctx || !d_v || !d_z) return HHO_ERR_ARG;
    if (d_v == d_z) {
        ctx->err = "hho_mlp_apply: d_v and d_z may not alias";
        return HHO_ERR_ARG;
    }
    if (!ctx->learned) {
        ctx->err = "learned smoother: call hho_mlp_init first";
        return HHO_ERR_STATE;
    }
    HHO_TRY(mlp_apply<double>(ctx, d_v, d_z));
    HHO_CUDA(cudaStreamSynchronize(ctx->stream));
    return mlp_status(ctx);
}

hho_status hho_mlp_generate(hho_ctx* ctx, int n_vec, uint64_t seed, int kind, int64_t* n_samples) {
    if (!ctx) return HHO_ERR_ARG;
    if (!ctx->have_pmg) {
        ctx->err = "hho_mlp_generate: call pmg_setup first";
        return HHO_ERR_STATE;
    }
    return mlp_generate(ctx, n_vec, seed, kind, n_samples);
}

hho_status hho_mlp_train(hho_ctx* ctx, int steps, int batch, double lr, uint64_t seed, double* h_loss) {
    if (!ctx) return HHO_ERR_ARG;
    return mlp_train(ctx, steps, batch, lr, seed, h_loss);
}

hho_status hho_mlp_grads(hho_ctx* ctx, const float* d_X, const float* d_T, int batch, double* h_loss, double* h_gW1,
                         double* h_gb1, double* h_gW2, double* h_gb2) {
    if (!ctx || !d_X || !d_T || !h_loss || !h_gW1 || !h_gb1 || !h_gW2 || !h_gb2) return HHO_ERR_ARG;
    return mlp_grads(ctx, d_X, d_T, batch, h_loss, h_gW1, h_gb1, h_gW2, h_gb2);
}

hho_status hho_ilu_apply(hho_ctx* ctx, int level, const double* d_v, double* d_z) {
    if (!ctx || !d_v || !d_z || d_v == d_z) return HHO_ERR_ARG;
    if (!ctx->have_pmg || level < 0 || level >= (int)ctx->ilu.size() || !ctx->ilu[level]) {
        ctx->err = "hho_ilu_apply: no ILU factors on this level (option smoother = 1, then pmg_setup)";
        return HHO_ERR_STATE;
    }
    const LevelMat& L = ctx->levels[level];
    double* tmp = nullptr;
    HHO_TRY(dalloc(ctx, &tmp, (size_t)std::max<int64_t>(L.ne * L.nP, 1)));
    hho_status st = ilu_apply<double>(ctx, level, d_v, d_z, tmp);
    cudaError_t se = cudaStreamSynchronize(ctx->stream);
    dfree(tmp);
    HHO_TRY(st);
    HHO_CUDA(se);
    return HHO_OK;
}

hho_status hho_autotune(hho_ctx* ctx, int reps, double* h_choice) {
    if (!ctx || reps < 1 || reps > 1000) return HHO_ERR_ARG;
    if (!ctx->have_pmg) {
        ctx->err = "hho_autotune: call pmg_setup first";
        return HHO_ERR_STATE;
    }
    return autotune(ctx, reps, h_choice);
}

hho_status hho_ndof(const hho_ctx* ctx, int level, int64_t* ndof) {
    if (!ctx || !ndof) return HHO_ERR_ARG;
    if (level < 0 || level >= (int)ctx->levels.size()) return HHO_ERR_ARG;
    *ndof = ctx->levels[level].n;
    return HHO_OK;
}

hho_status hho_quad_nodes(hho_ctx* ctx, int which, int64_t* n_nodes, double* d_xyz, double* d_normals) {
    if (!ctx || !n_nodes) return HHO_ERR_ARG;
    return quad_nodes(ctx, which, n_nodes, d_xyz, d_normals);
}

hho_status hho_assemble(hho_ctx* ctx, const double* d_f, const double* d_gD, const double* d_gN, double* d_rhs) {
    if (!ctx) return HHO_ERR_ARG;
    if (!d_f || !d_gD || !d_gN) {
        ctx->err = "hho_assemble: null data array";
        return HHO_ERR_ARG;
    }
    HHO_TRY(build_rhs(ctx, d_f, d_gD, d_gN));
    HHO_TRY(assemble_rhs_vector(ctx, ctx->rhs));
    if (d_rhs)
        HHO_CUDA(cudaMemcpyAsync(d_rhs, ctx->rhs, ctx->levels[0].n * sizeof(double), cudaMemcpyDeviceToDevice,
                                 ctx->stream));
    HHO_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->have_rhs = true;
    return HHO_OK;
}

hho_status pmg_setup(hho_ctx* ctx, int n_levels, const int* degrees, int prec, int smooth_its) {
    if (!ctx) return HHO_ERR_ARG;
    if (!degrees || n_levels < 1 || n_levels > 8 || degrees[0] != ctx->disc.k) {
        ctx->err = "pmg_setup: degrees must start at k and have 1..8 entries";
        return HHO_ERR_ARG;
    }
    for (int l = 1; l < n_levels; ++l)
        if (!(degrees[l] < degrees[l - 1] && degrees[l] >= 0)) {
            ctx->err = "pmg_setup: degrees must decrease strictly to >= 0";
            return HHO_ERR_ARG;
        }
    if (prec != HHO_FP64 && prec != HHO_FP32) {
        ctx->err = "pmg_setup: prec must be HHO_FP64 or HHO_FP32";
        return HHO_ERR_ARG;
    }
    if (smooth_its < 0 || smooth_its > 16) {
        ctx->err = "pmg_setup: smooth_its must be in 0..16";
        return HHO_ERR_ARG;
    }
    if (ctx->disc.cond == HHO_HPCOND && (ctx->smoother_kind != 0 || ctx->coarse_twolevel)) {
        ctx->err = "pmg_setup: HHO-hp contexts use the block-Jacobi smoother and the dense or multifrontal coarse solve";
        return HHO_ERR_UNSUPPORTED;
    }
    if (ctx->disc.cond == HHO_DGCOND && (ctx->smoother_kind != 0 || ctx->coarse_twolevel)) {
        ctx->err = "pmg_setup: DG contexts use the element block-Jacobi smoother and the dense coarse solve";
        return HHO_ERR_UNSUPPORTED;
    }
    if (ctx->disc.cond == HHO_UNCOND && ctx->coarse_twolevel) {
        ctx->err = "pmg_setup: uncondensed contexts use the dense or multifrontal coarse solve";
        return HHO_ERR_UNSUPPORTED;
    }
    ctx->have_pmg = false;
    while ((int)ctx->levels.size() > 1) {
        free_level(ctx->levels.back());
        ctx->levels.pop_back();
    }
    ctx->degrees.assign(degrees, degrees + n_levels);
    ctx->prec = prec;
    ctx->smooth_its = smooth_its;
    for (int l = 1; l < n_levels; ++l) HHO_TRY(build_level(ctx, l, degrees[l]));
    for (int l = 0; l < n_levels; ++l) HHO_TRY(build_smoother(ctx, l));
    HHO_TRY(pmg_build(ctx));
    HHO_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->have_pmg = true;
    return HHO_OK;
}

hho_status hho_set_option(hho_ctx* ctx, const char* key, double value) {
    if (!ctx || !key) return HHO_ERR_ARG;
    std::string k(key);
    invalidate_graphs(ctx);  // captured V-cycles embed the old settings
    if (k == "graphs") {
        if (value != 0.0 && value != 1.0) {
            ctx->err = "hho_set_option: graphs must be 0 or 1";
            return HHO_ERR_ARG;
        }
        ctx->use_graphs = value != 0.0;
        return HHO_OK;
    }
    if (k == "smoother") {
        if (value != 0.0 && value != 1.0) {
            ctx->err = "hho_set_option: smoother must be 0 (block Jacobi) or 1 (block ILU(0))";
            return HHO_ERR_ARG;
        }
        ctx->smoother_kind = (int)value;
        return HHO_OK;
    }
    if (k == "learned_smoother") {
        if (value != 0.0 && value != 1.0) {
            ctx->err = "hho_set_option: learned_smoother must be 0 or 1";
            return HHO_ERR_ARG;
        }
        if (value != 0.0 && !ctx->learned) {
            ctx->err = "hho_set_option: learned_smoother needs hho_mlp_init (and training) first";
            return HHO_ERR_STATE;
        }
        ctx->use_learned = value != 0.0 ? 1 : 0;
        return HHO_OK;
    }
    if (k == "coarse_fp32") {
        if (value != 0.0 && value != 1.0) {
            ctx->err = "hho_set_option: coarse_fp32 must be 0 or 1";
            return HHO_ERR_ARG;
        }
        ctx->coarse_fp32 = value != 0.0 ? 1 : 0;
        return HHO_OK;
    }
    if (k == "spmv_rows" || k == "spmv_grid") {
        if (value < 0.0 || (k == "spmv_rows" && value > 4.0) || (k == "spmv_grid" && value > 8192.0)) {
            ctx->err = "hho_set_option: spmv_rows must be 0..4 and spmv_grid 0..8192";
            return HHO_ERR_ARG;
        }
        if (k == "spmv_rows") ctx->spmv_rows = (int)value;
        else ctx->spmv_grid = (int)value;
        return HHO_OK;
    }
    if (k == "solve_graph") {
        ctx->solve_graph = value != 0.0 ? 1 : 0;
        return HHO_OK;
    }
    if (k == "solve_graph_single") {
        ctx->solve_graph_single = value != 0.0 ? 1 : 0;
        return HHO_OK;
    }
    if (k == "spmv_warp") {
        ctx->spmv_warp = value != 0.0 ? 1 : 0;
        return HHO_OK;
    }
    if (k == "coarse_twolevel") {
        ctx->coarse_twolevel = value != 0.0 ? 1 : 0;
        return HHO_OK;
    }
    if (!(value > 0.0) || value > 9.0e18) {
        ctx->err = "hho_set_option: value must be positive";
        return HHO_ERR_ARG;
    }
    if (k == "coarse_dense_max") ctx->coarse_dense_max = (int64_t)value;
    else if (k == "dd_elements") ctx->dd_elements = (int64_t)value;
    else if (k == "mf_leaf") ctx->mf_leaf = (int64_t)value;
    else {
        ctx->err = "hho_set_option: unknown key " + k;
        return HHO_ERR_ARG;
    }
    return HHO_OK;
}

hho_status pmg_vcycle(hho_ctx* ctx, const double* d_r, double* d_z) {
    if (!ctx) return HHO_ERR_ARG;
    if (!ctx->have_pmg) {
        ctx->err = "pmg_vcycle: call pmg_setup first";
        return HHO_ERR_STATE;
    }
    if (!d_r || !d_z || d_r == d_z) {
        ctx->err = "pmg_vcycle: null or aliased vectors";
        return HHO_ERR_ARG;
    }
    HHO_TRY(vcycle(ctx, d_r, d_z));
    HHO_CUDA(cudaGetLastError());
    return HHO_OK;
}

hho_status hho_spmv(hho_ctx* ctx, int level, const double* d_x, double* d_y) {
    if (!ctx || !d_x || !d_y || d_x == d_y) return HHO_ERR_ARG;
    if (level < 0 || level >= (int)ctx->levels.size()) {
        ctx->err = "hho_spmv: no such level";
        return HHO_ERR_ARG;
    }
    return spmv(ctx, level, d_x, d_y);
}

hho_status hho_spmv_f32(hho_ctx* ctx, int level, const float* d_x, float* d_y) {
    if (!ctx || !d_x || !d_y || (const void*)d_x == (const void*)d_y) return HHO_ERR_ARG;
    if (level < 0 || level >= (int)ctx->levels.size()) {
        ctx->err = "hho_spmv_f32: no such level";
        return HHO_ERR_ARG;
    }
    return spmv_f32(ctx, level, d_x, d_y);
}

hho_status hho_solve(hho_ctx* ctx, double rtol, int maxit, int restart, double* d_x, hho_solve_info* info) {
    if (!ctx || !d_x) return HHO_ERR_ARG;
    if (!ctx->have_pmg || !ctx->have_rhs) {
        ctx->err = "hho_solve: call hho_assemble and pmg_setup first";
        return HHO_ERR_STATE;
    }
    const hho_status st = (ctx->solve_graph_single && ctx->stream != nullptr && !ctx->probs.declared)
                              ? batch_solve(ctx, rtol, maxit, restart, d_x, nullptr, nullptr, info)
                              : fgmres(ctx, rtol, maxit, restart, d_x, info);
    if (ctx->use_learned && ctx->learned) HHO_TRY(mlp_status(ctx));
    return st;
}

hho_status hho_recover(hho_ctx* ctx, const double* d_x, double* d_local) {
    if (!ctx || !d_x || !d_local) return HHO_ERR_ARG;
    if (!ctx->have_rhs) {
        ctx->err = "hho_recover: call hho_assemble first";
        return HHO_ERR_STATE;
    }
    HHO_TRY(recover_local(ctx, d_x, d_local));
    HHO_CUDA(cudaStreamSynchronize(ctx->stream));
    return HHO_OK;
}

hho_status hho_errors(hho_ctx* ctx, const double* d_local, const double* d_u, const double* d_gradu, const double* d_p,
                      double out[4]) {
    if (!ctx || !d_local || !d_u || !d_gradu || !d_p || !out) return HHO_ERR_ARG;
    return compute_errors(ctx, d_local, d_u, d_gradu, d_p, out);
}

hho_status hho_get_element_schur(hho_ctx* ctx, double* host_out, int64_t* count) {
    if (!ctx || !count) return HHO_ERR_ARG;
    *count = ctx->disc.tot_S;
    if (!host_out) return HHO_OK;
    HHO_CUDA(cudaMemcpyAsync(host_out, ctx->disc.S, ctx->disc.tot_S * sizeof(double), cudaMemcpyDeviceToHost,
                             ctx->stream));
    HHO_CUDA(cudaStreamSynchronize(ctx->stream));
    return HHO_OK;
}

hho_status hho_set_element_schur(hho_ctx* ctx, const double* host_in) {
    if (!ctx || !host_in) return HHO_ERR_ARG;
    HHO_CUDA(cudaMemcpyAsync(ctx->disc.S, host_in, ctx->disc.tot_S * sizeof(double), cudaMemcpyHostToDevice,
                             ctx->stream));
    HHO_TRY(assemble_level0(ctx));
    ctx->have_pmg = false;
    return HHO_OK;
}

hho_status hho_get_level_coo(hho_ctx* ctx, int level, int64_t* rows, int64_t* cols, double* vals, int64_t* nnz) {
    if (!ctx || !nnz) return HHO_ERR_ARG;
    return level_coo(ctx, level, rows, cols, vals, nnz);
}

hho_status hho_coarse_info(hho_ctx* ctx, int64_t* info) {
    if (!ctx || !info) return HHO_ERR_ARG;
    if (!ctx->have_pmg) {
        ctx->err = "hho_coarse_info: call pmg_setup first";
        return HHO_ERR_STATE;
    }
    return coarse_info(ctx, info);
}

hho_status hho_launch_count(const hho_ctx* ctx, int64_t* launches) {
    if (!ctx || !launches) return HHO_ERR_ARG;
    *launches = ctx->launches;
    return HHO_OK;
}

hho_status hho_destroy(hho_ctx* ctx) {
    if (!ctx) return HHO_OK;
    free_workspace(ctx);
    coarse_free(ctx);
    for (auto& L : ctx->levels) free_level(L);
    Disc& D = ctx->disc;
    void* ps[] = {D.xyz, D.ef_ptr, D.ef, D.fv_ptr, D.fv, D.fe, D.flf, D.fbc, D.fgeo, D.fC, D.eC, D.emeas,
                  D.off_S, D.off_X, D.off_Kei, D.off_P, D.off_loc, D.S, D.X, D.Kei, D.P, D.gT, D.yT, D.off_gT,
                  D.off_yT, D.enode_off, D.fnode_off, D.gl};
    for (void* p : ps) dfree(p);
    Topo& T = ctx->topo;
    void* pt[] = {T.ff_col, T.ff_nsl, T.fp_col, T.pf_col, T.pf_nsl, T.asm_T, T.asm_lf, T.asm_lg};
    for (void* p : pt) dfree(p);
    batch_free(ctx);
    mlp_free(ctx);
    ilu_free(ctx);
    dfree(ctx->rhs);
    dfree(ctx->null_vec0);
    dfree(ctx->null_w);
    dfree(ctx->d_null_off);
    dfree(ctx->null_part);
    dfree(ctx->d_flag);
    delete ctx;
    return HHO_OK;
}

const char* hho_last_error(const hho_ctx* ctx) {
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

}  // extern "C"
