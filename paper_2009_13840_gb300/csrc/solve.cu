// p-multilevel V-cycle and FGMRES on the GPU (Sec. 3.3, Algorithm MG_V).
//
//   smoother      m iterations of right-preconditioned GMRES (the paper uses two,
//                 Sec. 5.2.2) with the block-Jacobi preconditioner (face blocks
//                 D_F^{-1}, element pressure pivot blocks M_T^{-1})
//   restriction   per face and component keep the leading coefficients,
//                 fused with the defect computation d = I(b - S w) (Sec. 3.1)
//   prolongation  zero padding, added to the iterate (Sec. 3.1)
//   coarse level  explicit inverse from a dense Gauss-Jordan factorisation
//                 (at most 10^4 unknowns) with a rank-one fix of the constant
//                 pressure kernel, else block-Jacobi GMRES to a 1e-3 relative
//                 residual decrease (Sec. 5.2.2)
//   outer solver  flexible GMRES, one V-cycle per iteration (Sec. 3.3)
//
// Every Arnoldi step uses classical Gram-Schmidt applied twice (CGS2).  All
// reductions are two-stage with a fixed grid, so results are bitwise
// reproducible run to run.  Small Hessenberg algebra (Givens rotations,
// back-substitution) runs in single-thread device kernels; the host reads only
// the residual estimate of the outer and coarse iterations.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace hho {

namespace {

constexpr int RED_BLOCKS = 304;  // fixed grid of the two-stage reductions
constexpr int RED_TPB = 256;
constexpr int MDOT_MAX = 8;

int grid1d(int64_t n, int tpb) {
    int64_t g = (n + tpb - 1) / tpb;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152LL * 64));
}

// ---------------------------------------------------------------------------
// SpMV-type kernels (one thread per scalar row; 32 consecutive faces per warp)
// mode 0: y = S x     mode 1: y = bv - S x
// ---------------------------------------------------------------------------
struct LevelView {
    int64_t nf, ne;
    int b, nP, S_max, N_max;
    const int32_t *ff_col, *ff_nsl, *fp_col, *pf_col, *pf_nsl;
    const double *ff, *fp, *pf, *pp, *dinv, *minv;
};

LevelView view(const LevelMat& L) {
    LevelView v;
    v.nf = L.nf;
    v.ne = L.ne;
    v.b = L.b;
    v.nP = L.nP;
    v.S_max = L.S_max;
    v.N_max = L.N_max;
    v.ff_col = L.ff_col;
    v.ff_nsl = L.ff_nsl;
    v.fp_col = L.fp_col;
    v.pf_col = L.pf_col;
    v.pf_nsl = L.pf_nsl;
    v.ff = L.ff;
    v.fp = L.fp;
    v.pf = L.pf;
    v.pp = L.pp;
    v.dinv = L.dinv;
    v.minv = L.minv;
    return v;
}

__device__ __forceinline__ double face_row(const LevelView& L, int64_t F, int r, const double* __restrict__ x) {
    const int b = L.b, nP = L.nP;
    const int64_t nf = L.nf;
    double acc = 0.0;
    const int ns = L.ff_nsl[F];
    for (int s = 0; s < ns; ++s) {
        const int64_t G = L.ff_col[s * nf + F];
        const double* xv = x + G * b;
        const double* a = L.ff + ((int64_t)s * b * b + r) * nf + F;
        for (int c = 0; c < b; ++c) acc += a[(int64_t)c * b * nf] * xv[c];
    }
    const double* xp = x + nf * b;
    for (int p = 0; p < 2; ++p) {
        const int T = L.fp_col[p * nf + F];
        if (T < 0) continue;
        const double* a = L.fp + ((int64_t)p * nP * b + r) * nf + F;
        for (int c = 0; c < nP; ++c) acc += a[(int64_t)c * b * nf] * xp[(int64_t)T * nP + c];
    }
    return acc;
}

__device__ __forceinline__ double elem_row(const LevelView& L, int64_t T, int r, const double* __restrict__ x) {
    const int b = L.b, nP = L.nP;
    const int64_t ne = L.ne;
    double acc = 0.0;
    const int N = L.pf_nsl[T];
    for (int f = 0; f < N; ++f) {
        const int64_t G = L.pf_col[f * ne + T];
        const double* a = L.pf + ((int64_t)f * b * nP + r) * ne + T;
        for (int c = 0; c < b; ++c) acc += a[(int64_t)c * nP * ne] * x[G * b + c];
    }
    const double* xp = x + L.nf * b + T * nP;
    const double* a = L.pp + (int64_t)r * ne + T;
    for (int c = 0; c < nP; ++c) acc += a[(int64_t)c * nP * ne] * xp[c];
    return acc;
}

__global__ void k_spmv(LevelView L, const double* __restrict__ x, const double* __restrict__ bv, double* __restrict__ y,
                       int mode) {
    const int64_t nfr = L.nf * L.b, ner = L.ne * L.nP;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nfr + ner; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < nfr) {
            int r = (int)(i / L.nf);
            int64_t F = i % L.nf;
            double v = face_row(L, F, r, x);
            int64_t o = F * L.b + r;
            y[o] = mode ? bv[o] - v : v;
        } else {
            int64_t j = i - nfr;
            int r = (int)(j / L.ne);
            int64_t T = j % L.ne;
            double v = elem_row(L, T, r, x);
            int64_t o = nfr + T * L.nP + r;
            y[o] = mode ? bv[o] - v : v;
        }
    }
}

// d (coarse layout) = I (bv - S x): only the rows kept by the restriction are formed.
__global__ void k_residual_restrict(LevelView L, int nFf, int bc, int nFc, int nPc, const double* __restrict__ x,
                                    const double* __restrict__ bv, double* __restrict__ d) {
    const int64_t nfr = L.nf * bc, ner = L.ne * nPc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nfr + ner; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < nfr) {
            int rc = (int)(i / L.nf);
            int64_t F = i % L.nf;
            int rf = (rc / nFc) * nFf + rc % nFc;
            int64_t o = F * L.b + rf;
            d[F * bc + rc] = bv[o] - face_row(L, F, rf, x);
        } else {
            int64_t j = i - nfr;
            int r = (int)(j / L.ne);
            int64_t T = j % L.ne;
            int64_t o = L.nf * L.b + T * L.nP + r;
            d[nfr + T * nPc + r] = bv[o] - elem_row(L, T, r, x);
        }
    }
}

// x (fine) += zero-padded xc (coarse)
__global__ void k_prolong_add(int64_t nf, int64_t ne, int bf, int nFf, int nPf, int bc, int nFc, int nPc,
                              const double* __restrict__ xc, double* __restrict__ x) {
    const int64_t nfr = nf * bc, ner = ne * nPc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nfr + ner; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < nfr) {
            int64_t F = i / bc;
            int rc = (int)(i % bc);
            int rf = (rc / nFc) * nFf + rc % nFc;
            x[F * bf + rf] += xc[i];
        } else {
            int64_t j = i - nfr, T = j / nPc;
            int r = (int)(j % nPc);
            x[nf * bf + T * nPf + r] += xc[i];
        }
    }
}

// z = M^{-1} v (block Jacobi)
__global__ void k_jacobi(LevelView L, const double* __restrict__ v, double* __restrict__ z) {
    const int64_t nfr = L.nf * L.b, ner = L.ne * L.nP;
    const int b = L.b, nP = L.nP;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nfr + ner; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < nfr) {
            int r = (int)(i / L.nf);
            int64_t F = i % L.nf;
            const double* a = L.dinv + (int64_t)r * L.nf + F;
            const double* vv = v + F * b;
            double s = 0.0;
            for (int c = 0; c < b; ++c) s += a[(int64_t)c * b * L.nf] * vv[c];
            z[F * b + r] = s;
        } else {
            int64_t j = i - nfr;
            int r = (int)(j / L.ne);
            int64_t T = j % L.ne;
            const double* a = L.minv + (int64_t)r * L.ne + T;
            const double* vv = v + nfr + T * nP;
            double s = 0.0;
            for (int c = 0; c < nP; ++c) s += a[(int64_t)c * nP * L.ne] * vv[c];
            z[nfr + T * nP + r] = s;
        }
    }
}

// ---------------------------------------------------------------------------
// Deterministic reductions: dots of w with up to MDOT_MAX vectors V_i (stride ld)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(RED_TPB) k_mdot_partial(int64_t n, const double* __restrict__ V, int64_t ld, int nv,
                                                          const double* __restrict__ w, double* __restrict__ partial) {
    double acc[MDOT_MAX];
#pragma unroll
    for (int v = 0; v < MDOT_MAX; ++v) acc[v] = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double wi = w[i];
#pragma unroll
        for (int v = 0; v < MDOT_MAX; ++v)
            if (v < nv) acc[v] += V[v * ld + i] * wi;
    }
    __shared__ double sm[RED_TPB / 32][MDOT_MAX];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < MDOT_MAX; ++v) {
        double a = acc[v];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) sm[wid][v] = a;
    }
    __syncthreads();
    if (threadIdx.x < nv) {
        double s = 0.0;
        for (int i = 0; i < RED_TPB / 32; ++i) s += sm[i][threadIdx.x];
        partial[threadIdx.x * RED_BLOCKS + blockIdx.x] = s;
    }
}

__global__ void k_mdot_final(int nv, const double* __restrict__ partial, double* __restrict__ out) {
    __shared__ double sm[RED_BLOCKS];
    for (int v = 0; v < nv; ++v) {
        for (int i = threadIdx.x; i < RED_BLOCKS; i += blockDim.x) sm[i] = partial[v * RED_BLOCKS + i];
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int i = 0; i < RED_BLOCKS; ++i) s += sm[i];
            out[v] = s;
        }
        __syncthreads();
    }
}

// out = a0 * out + sgn * sum_i coef[i] * V_i
__global__ void k_combine(int64_t n, double* __restrict__ out, double a0, const double* __restrict__ V, int64_t ld,
                          int nv, const double* __restrict__ coef, double sgn) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = (a0 == 0.0) ? 0.0 : a0 * out[i];
        for (int v = 0; v < nv; ++v) s += sgn * coef[v] * V[v * ld + i];
        out[i] = s;
    }
}

// dst = src / *den  (zero if the denominator is zero)
__global__ void k_scale(int64_t n, const double* __restrict__ src, double* __restrict__ dst, const double* __restrict__ den) {
    double dv = *den;
    double inv = (dv == 0.0) ? 0.0 : 1.0 / dv;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i] * inv;
}

__global__ void k_copy(int64_t n, const double* __restrict__ src, double* __restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

__global__ void k_zero(int64_t n, double* __restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = 0.0;
}

// ---------------------------------------------------------------------------
// Small Hessenberg algebra (single thread).  Scalar area layout for restart m:
//   [0] beta^2   [1] beta   [2] m_eff   [3] residual estimate   [4] breakdown
//   [8 ..)       H (m+1) x m column-major
//   then cs[m], sn[m], g[m+1], y[m], t1[m+1], t2[m+1], nrm2[1]
// ---------------------------------------------------------------------------
struct GS {
    int m;
    int H, cs, sn, g, y, t1, t2, nrm;
    int total;
};
GS gs_layout(int m) {
    GS s;
    s.m = m;
    int o = 8;
    s.H = o;
    o += (m + 1) * m;
    s.cs = o;
    o += m;
    s.sn = o;
    o += m;
    s.g = o;
    o += m + 1;
    s.y = o;
    o += m;
    s.t1 = o;
    o += m + 1;
    s.t2 = o;
    o += m + 1;
    s.nrm = o;
    o += 1;
    s.total = o;
    return s;
}

__global__ void k_gs_start(double* sc, GS L) {
    double b2 = sc[0];
    double beta = sqrt(b2);
    sc[1] = beta;
    sc[2] = 0.0;
    sc[3] = beta;
    sc[4] = (beta == 0.0) ? 1.0 : 0.0;
    for (int i = 0; i <= L.m; ++i) sc[L.g + i] = 0.0;
    sc[L.g] = beta;
}

// Finish column j: H[:,j] = t1 + t2, H[j+1,j] = sqrt(nrm2); Givens update.
__global__ void k_gs_column(double* sc, GS L, int j) {
    double* H = sc + L.H;
    const int ld = L.m + 1;
    if (sc[4] != 0.0) {  // after a breakdown the remaining columns are ignored
        for (int i = 0; i <= L.m; ++i) H[j * ld + i] = 0.0;
        sc[L.nrm + 0] = 0.0;
        return;
    }
    for (int i = 0; i <= j; ++i) H[j * ld + i] = sc[L.t1 + i] + sc[L.t2 + i];
    double hn = sqrt(sc[L.nrm]);
    H[j * ld + j + 1] = hn;
    sc[L.nrm] = hn;  // denominator for v_{j+1}
    // apply previous rotations
    for (int i = 0; i < j; ++i) {
        double c = sc[L.cs + i], s = sc[L.sn + i];
        double a = H[j * ld + i], bb = H[j * ld + i + 1];
        H[j * ld + i] = c * a + s * bb;
        H[j * ld + i + 1] = -s * a + c * bb;
    }
    double a = H[j * ld + j], bb = H[j * ld + j + 1];
    double r = hypot(a, bb);
    double c = (r == 0.0) ? 1.0 : a / r, s = (r == 0.0) ? 0.0 : bb / r;
    sc[L.cs + j] = c;
    sc[L.sn + j] = s;
    H[j * ld + j] = r;
    H[j * ld + j + 1] = 0.0;
    double gj = sc[L.g + j];
    sc[L.g + j] = c * gj;
    sc[L.g + j + 1] = -s * gj;
    sc[3] = fabs(sc[L.g + j + 1]);
    sc[2] = j + 1;
    if (hn == 0.0) sc[4] = 1.0;
}

// y = R^{-1} g over the first m_eff columns (zeros beyond).
__global__ void k_gs_solve(double* sc, GS L) {
    const double* H = sc + L.H;
    const int ld = L.m + 1;
    int me = (int)sc[2];
    if (sc[1] == 0.0) me = 0;
    for (int i = 0; i < L.m; ++i) sc[L.y + i] = 0.0;
    for (int i = me - 1; i >= 0; --i) {
        double s = sc[L.g + i];
        for (int l = i + 1; l < me; ++l) s -= H[l * ld + i] * sc[L.y + l];
        double d = H[i * ld + i];
        sc[L.y + i] = (d == 0.0) ? 0.0 : s / d;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Workspace
// ---------------------------------------------------------------------------
struct LevelWork {
    double *bv = nullptr, *x = nullptr, *r = nullptr, *V = nullptr, *Z = nullptr, *w = nullptr, *sc = nullptr;
};

struct Workspace {
    std::vector<LevelWork> lv;
    double* partial = nullptr;
    // FGMRES
    int restart = 0;
    double *fV = nullptr, *fZ = nullptr, *fw = nullptr, *fr = nullptr, *fsc = nullptr;
    double* h_sc = nullptr;  // pinned host scalars
};

void free_workspace(hho_ctx* ctx) {
    Workspace* W = ctx->ws;
    if (!W) return;
    for (auto& l : W->lv) {
        dfree(l.bv);
        dfree(l.x);
        dfree(l.r);
        dfree(l.V);
        dfree(l.Z);
        dfree(l.w);
        dfree(l.sc);
    }
    dfree(W->partial);
    dfree(W->fV);
    dfree(W->fZ);
    dfree(W->fw);
    dfree(W->fr);
    dfree(W->fsc);
    if (W->h_sc) cudaFreeHost(W->h_sc);
    delete W;
    ctx->ws = nullptr;
}

static hho_status mdot(hho_ctx* ctx, int64_t n, const double* V, int64_t ld, int nv, const double* w, double* out) {
    Workspace* W = ctx->ws;
    for (int v0 = 0; v0 < nv; v0 += MDOT_MAX) {
        int cnt = std::min(MDOT_MAX, nv - v0);
        k_mdot_partial<<<RED_BLOCKS, RED_TPB, 0, ctx->stream>>>(n, V + v0 * ld, ld, cnt, w, W->partial);
        ++ctx->launches;
        k_mdot_final<<<1, 256, 0, ctx->stream>>>(cnt, W->partial, out + v0);
        ++ctx->launches;
    }
    HHO_CUDA(cudaGetLastError());
    return HHO_OK;
}

hho_status spmv(hho_ctx* ctx, int l, const double* x, double* y) {
    const LevelMat& L = ctx->levels[l];
    k_spmv<<<grid1d(L.n, 256), 256, 0, ctx->stream>>>(view(L), x, nullptr, y, 0);
    ++ctx->launches;
    HHO_CUDA(cudaGetLastError());
    return HHO_OK;
}

static hho_status residual(hho_ctx* ctx, int l, const double* x, const double* bv, double* r) {
    const LevelMat& L = ctx->levels[l];
    k_spmv<<<grid1d(L.n, 256), 256, 0, ctx->stream>>>(view(L), x, bv, r, 1);
    ++ctx->launches;
    HHO_CUDA(cudaGetLastError());
    return HHO_OK;
}

static hho_status jacobi(hho_ctx* ctx, int l, const double* v, double* z) {
    const LevelMat& L = ctx->levels[l];
    k_jacobi<<<grid1d(L.n, 256), 256, 0, ctx->stream>>>(view(L), v, z);
    ++ctx->launches;
    HHO_CUDA(cudaGetLastError());
    return HHO_OK;
}

// One Arnoldi step j with CGS2: w = A z_j is given in w; V holds v_0..v_j.
static hho_status arnoldi_finish(hho_ctx* ctx, int64_t n, double* V, double* w, double* sc, const GS& G, int j) {
    HHO_TRY(mdot(ctx, n, V, n, j + 1, w, sc + G.t1));
    k_combine<<<grid1d(n, 256), 256, 0, ctx->stream>>>(n, w, 1.0, V, n, j + 1, sc + G.t1, -1.0);
    ++ctx->launches;
    HHO_TRY(mdot(ctx, n, V, n, j + 1, w, sc + G.t2));
    k_combine<<<grid1d(n, 256), 256, 0, ctx->stream>>>(n, w, 1.0, V, n, j + 1, sc + G.t2, -1.0);
    ++ctx->launches;
    HHO_TRY(mdot(ctx, n, w, n, 1, w, sc + G.nrm));
    k_gs_column<<<1, 1, 0, ctx->stream>>>(sc, G, j);
    ++ctx->launches;
    k_scale<<<grid1d(n, 256), 256, 0, ctx->stream>>>(n, w, V + (int64_t)(j + 1) * n, sc + G.nrm);
    ++ctx->launches;
    HHO_CUDA(cudaGetLastError());
    return HHO_OK;
}

// m iterations of right-preconditioned GMRES on level l: x <- x + Z y (x = Z y when x_zero).
static hho_status smooth(hho_ctx* ctx, int l, const double* bv, double* x, bool x_zero) {
    const LevelMat& L = ctx->levels[l];
    LevelWork& lw = ctx->ws->lv[l];
    const int m = ctx->smooth_its;
    const int64_t n = L.n;
    if (m == 0) {
        if (x_zero) {
            k_zero<<<grid1d(n, 256), 256, 0, ctx->stream>>>(n, x);
            ++ctx->launches;
        }
        return HHO_OK;
    }
    GS G = gs_layout(m);
    double* sc = lw.sc;
    if (x_zero) {
        k_copy<<<grid1d(n, 256), 256, 0, ctx->stream>>>(n, bv, lw.r);
        ++ctx->launches;
    } else {
        HHO_TRY(residual(ctx, l, x, bv, lw.r));
    }
    HHO_TRY(mdot(ctx, n, lw.r, n, 1, lw.r, sc + 0));
    k_gs_start<<<1, 1, 0, ctx->stream>>>(sc, G);
    ++ctx->launches;
    k_scale<<<grid1d(n, 256), 256, 0, ctx->stream>>>(n, lw.r, lw.V, sc + 1);
    ++ctx->launches;
    for (int j = 0; j < m; ++j) {
        HHO_TRY(jacobi(ctx, l, lw.V + (int64_t)j * n, lw.Z + (int64_t)j * n));
        HHO_TRY(spmv(ctx, l, lw.Z + (int64_t)j * n, lw.w));
        HHO_TRY(arnoldi_finish(ctx, n, lw.V, lw.w, sc, G, j));
    }
    k_gs_solve<<<1, 1, 0, ctx->stream>>>(sc, G);
    ++ctx->launches;
    k_combine<<<grid1d(n, 256), 256, 0, ctx->stream>>>(n, x, x_zero ? 0.0 : 1.0, lw.Z, n, m, sc + G.y, 1.0);
    ++ctx->launches;
    HHO_CUDA(cudaGetLastError());
    return HHO_OK;
}

static hho_status host_read(hho_ctx* ctx, const double* dsrc, double* hdst, int count) {
    HHO_CUDA(cudaMemcpyAsync(hdst, dsrc, count * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    HHO_CUDA(cudaStreamSynchronize(ctx->stream));
    return HHO_OK;
}

static hho_status coarse_solve(hho_ctx* ctx, int l, const double* d, double* c) {
    (void)l;
    return coarse_apply(ctx, d, c);
}

// MG_V(l, b, w) with the iterate held in lv[l].x (zero initial guess when x_zero).
static hho_status vcycle_level(hho_ctx* ctx, int l, const double* bv, double* x, bool x_zero) {
    const int Lc = (int)ctx->levels.size() - 1;
    const LevelMat& F = ctx->levels[l];
    const LevelMat& C = ctx->levels[l + 1];
    LevelWork& cw = ctx->ws->lv[l + 1];
    HHO_TRY(smooth(ctx, l, bv, x, x_zero));
    k_residual_restrict<<<grid1d(C.n, 256), 256, 0, ctx->stream>>>(view(F), F.nF, C.b, C.nF, C.nP, x, bv, cw.bv);
    ++ctx->launches;
    HHO_CUDA(cudaGetLastError());
    if (l + 1 == Lc) HHO_TRY(coarse_solve(ctx, l + 1, cw.bv, cw.x));
    else HHO_TRY(vcycle_level(ctx, l + 1, cw.bv, cw.x, true));
    k_prolong_add<<<grid1d(C.n, 256), 256, 0, ctx->stream>>>(F.nf, F.ne, F.b, F.nF, F.nP, C.b, C.nF, C.nP, cw.x, x);
    ++ctx->launches;
    HHO_CUDA(cudaGetLastError());
    HHO_TRY(smooth(ctx, l, bv, x, false));
    return HHO_OK;
}

hho_status vcycle(hho_ctx* ctx, const double* r, double* z) {
    if (ctx->levels.size() == 1) return coarse_solve(ctx, 0, r, z);
    return vcycle_level(ctx, 0, r, z, true);
}

__global__ void k_null_project(int64_t n, double* __restrict__ x, const double* __restrict__ nv, const double* __restrict__ dot) {
    double a = *dot;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] -= a * nv[i];
}

static hho_status project_null(hho_ctx* ctx, int64_t n, double* x, const double* nv, double* tmp) {
    HHO_TRY(mdot(ctx, n, nv, n, 1, x, tmp));
    k_null_project<<<grid1d(n, 256), 256, 0, ctx->stream>>>(n, x, nv, tmp);
    ++ctx->launches;
    HHO_CUDA(cudaGetLastError());
    return HHO_OK;
}

static std::vector<double> null_vector_host(hho_ctx* ctx, const LevelMat& L) {
    std::vector<double> meas(L.ne), v(L.n, 0.0);
    cudaMemcpy(meas.data(), ctx->disc.emeas, L.ne * sizeof(double), cudaMemcpyDeviceToHost);
    double s = 0.0;
    for (int64_t T = 0; T < L.ne; ++T) s += meas[T];
    double inv = 1.0 / std::sqrt(s);
    for (int64_t T = 0; T < L.ne; ++T) v[L.nf * L.b + T * L.nP] = std::sqrt(meas[T]) * inv;
    return v;
}

hho_status pmg_build(hho_ctx* ctx) {
    free_workspace(ctx);
    Workspace* W = new Workspace();
    ctx->ws = W;
    const int nl = (int)ctx->levels.size();
    W->lv.resize(nl);
    const int m = std::max(ctx->smooth_its, 1);
    GS G = gs_layout(m);
    for (int l = 0; l < nl; ++l) {
        const int64_t n = ctx->levels[l].n;
        LevelWork& w = W->lv[l];
        HHO_TRY(dalloc(ctx, &w.bv, n));
        HHO_TRY(dalloc(ctx, &w.x, n));
        HHO_TRY(dalloc(ctx, &w.r, n));
        HHO_TRY(dalloc(ctx, &w.V, (size_t)(m + 1) * n));
        HHO_TRY(dalloc(ctx, &w.Z, (size_t)m * n));
        HHO_TRY(dalloc(ctx, &w.w, n));
        HHO_TRY(dalloc(ctx, &w.sc, G.total));
    }
    HHO_TRY(dalloc(ctx, &W->partial, (size_t)MDOT_MAX * RED_BLOCKS));
    HHO_CUDA(cudaMallocHost(&W->h_sc, 64 * sizeof(double)));
    bool neumann = false;
    for (auto b : ctx->disc.h_fbc) neumann |= (b == 2);
    ctx->has_null = !neumann;
    // level-0 null vector
    dfree(ctx->null_vec0);
    ctx->null_vec0 = nullptr;
    if (ctx->has_null) {
        auto v = null_vector_host(ctx, ctx->levels[0]);
        HHO_TRY(dalloc(ctx, &ctx->null_vec0, v.size()));
        HHO_CUDA(cudaMemcpy(ctx->null_vec0, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    HHO_TRY(coarse_setup(ctx));
    return HHO_OK;
}

hho_status fgmres(hho_ctx* ctx, double rtol, int maxit, int restart, double* x, hho_solve_info* info) {
    Workspace* W = ctx->ws;
    const LevelMat& L0 = ctx->levels[0];
    const int64_t n = L0.n;
    if (restart < 1 || restart > 200 || maxit < 0 || !(rtol > 0.0)) {
        ctx->err = "hho_solve: invalid restart, maxit or rtol";
        return HHO_ERR_ARG;
    }
    if (W->restart != restart) {
        dfree(W->fV);
        dfree(W->fZ);
        dfree(W->fw);
        dfree(W->fr);
        dfree(W->fsc);
        HHO_TRY(dalloc(ctx, &W->fV, (size_t)(restart + 1) * n));
        HHO_TRY(dalloc(ctx, &W->fZ, (size_t)restart * n));
        HHO_TRY(dalloc(ctx, &W->fw, n));
        HHO_TRY(dalloc(ctx, &W->fr, n));
        HHO_TRY(dalloc(ctx, &W->fsc, gs_layout(restart).total + 8));
        W->restart = restart;
    }
    GS G = gs_layout(restart);
    double* sc = W->fsc;
    double* hs = W->h_sc;
    double* bvec = W->fr;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, ctx->stream);
    ctx->coarse_its_total = 0;
    // b (projected on the complement of the constant-pressure kernel when it exists)
    k_copy<<<grid1d(n, 256), 256, 0, ctx->stream>>>(n, ctx->rhs, bvec);
    ++ctx->launches;
    if (ctx->has_null) HHO_TRY(project_null(ctx, n, bvec, ctx->null_vec0, sc + G.total));
    k_zero<<<grid1d(n, 256), 256, 0, ctx->stream>>>(n, x);
    ++ctx->launches;
    HHO_TRY(mdot(ctx, n, bvec, n, 1, bvec, sc + 0));
    HHO_TRY(host_read(ctx, sc, hs, 1));
    const double bnorm = std::sqrt(hs[0]);
    int it = 0;
    double relres = 0.0;
    hho_status st = HHO_OK;
    if (bnorm > 0.0) {
        k_copy<<<grid1d(n, 256), 256, 0, ctx->stream>>>(n, bvec, W->fw);
        ++ctx->launches;
        bool conv = false;
        while (it < maxit) {
            // r = b - S x is in fw
            HHO_TRY(mdot(ctx, n, W->fw, n, 1, W->fw, sc + 0));
            k_gs_start<<<1, 1, 0, ctx->stream>>>(sc, G);
            ++ctx->launches;
            HHO_TRY(host_read(ctx, sc + 1, hs, 1));
            if (hs[0] <= rtol * bnorm) {
                conv = true;
                break;
            }
            k_scale<<<grid1d(n, 256), 256, 0, ctx->stream>>>(n, W->fw, W->fV, sc + 1);
            ++ctx->launches;
            int j = 0;
            for (; j < restart; ++j) {
                HHO_TRY(vcycle(ctx, W->fV + (int64_t)j * n, W->fZ + (int64_t)j * n));
                HHO_TRY(spmv(ctx, 0, W->fZ + (int64_t)j * n, W->fw));
                HHO_TRY(arnoldi_finish(ctx, n, W->fV, W->fw, sc, G, j));
                ++it;
                HHO_TRY(host_read(ctx, sc + 3, hs, 2));
                if (hs[0] <= rtol * bnorm || hs[1] != 0.0 || it >= maxit) break;
            }
            k_gs_solve<<<1, 1, 0, ctx->stream>>>(sc, G);
            ++ctx->launches;
            k_combine<<<grid1d(n, 256), 256, 0, ctx->stream>>>(n, x, 1.0, W->fZ, n, std::min(j + 1, restart), sc + G.y,
                                                              1.0);
            ++ctx->launches;
            HHO_TRY(residual(ctx, 0, x, bvec, W->fw));
        }
        if (ctx->has_null) HHO_TRY(project_null(ctx, n, x, ctx->null_vec0, sc + G.total));
        HHO_TRY(residual(ctx, 0, x, bvec, W->fw));
        HHO_TRY(mdot(ctx, n, W->fw, n, 1, W->fw, sc + 0));
        HHO_TRY(host_read(ctx, sc, hs, 1));
        relres = std::sqrt(hs[0]) / bnorm;
        if (!conv && relres > rtol) st = HHO_ERR_NOT_CONVERGED;
    }
    cudaEventRecord(e1, ctx->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (info) {
        info->iterations = it;
        info->coarse_iterations = (int32_t)ctx->coarse_its_total;
        info->rel_residual = relres;
        info->solve_ms = ms;
        info->status = st;
    }
    HHO_CUDA(cudaGetLastError());
    if (st != HHO_OK) ctx->err = "hho_solve: FGMRES reached maxit above the tolerance";
    return st;
}

}  // namespace hho
