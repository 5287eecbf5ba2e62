// Assembly of the condensed operator into the face-block layout, Galerkin
// coarse operators by block extraction, and block-Jacobi smoother data.
//
//   Sec. 4.1.2 end: element Schur complements are assembled face by face.
//   Sec. 4.2: with hierarchical orthonormal bases the restriction is the
//   unit-diagonal selection of the leading coefficients, so the level-(l+1)
//   operator is the sub-block extraction of the level-l operator (recursive,
//   matrix-free: no transfer matrix is formed).
//
// Layout of a level operator with face block b and pressure block nP (one
// thread later reads one row, 32 consecutive faces per warp, so every value
// array is innermost over faces or elements):
//   ff[s][c][r][F]  face row F, slot s (s=0 is the diagonal block), column c
//   fp[p][c][r][F]  face row F, pressure block of its p-th element
//   pf[f][c][r][T]  element row T, its f-th face
//   pp[c][r][T]     element row T, its own pressure block
// Every block of the global matrix receives its element contributions in a
// fixed order (first element of the face, then the second), so the assembly is
// deterministic without atomics.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace hho {

namespace {

__global__ void k_assemble_ff(int64_t nf, int b, int S_max, const int32_t* __restrict__ ff_nsl,
                              const int32_t* __restrict__ asm_T, const int32_t* __restrict__ asm_lf,
                              const int32_t* __restrict__ asm_lg, const int32_t* __restrict__ fe,
                              const int32_t* __restrict__ flf, const int64_t* __restrict__ off_S,
                              const int32_t* __restrict__ ef_ptr, int nP, const double* __restrict__ S,
                              double* __restrict__ ff) {
    int64_t tot = (int64_t)S_max * b * b * nf;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t F = i % nf;
        int64_t rest = i / nf;
        int r = rest % b;
        rest /= b;
        int c = rest % b;
        int s = (int)(rest / b);
        double v = 0.0;
        if (s < ff_nsl[F]) {
            if (s == 0) {
                for (int e = 0; e < 2; ++e) {
                    int T = fe[2 * F + e];
                    if (T < 0) continue;
                    int lf = flf[2 * F + e];
                    int N = ef_ptr[T + 1] - ef_ptr[T];
                    int nk = N * b + nP;
                    v += S[off_S[T] + (int64_t)(lf * b + r) * nk + (lf * b + c)];
                }
            } else {
                int T = asm_T[s * nf + F], lf = asm_lf[s * nf + F], lg = asm_lg[s * nf + F];
                int N = ef_ptr[T + 1] - ef_ptr[T];
                int nk = N * b + nP;
                v = S[off_S[T] + (int64_t)(lf * b + r) * nk + (lg * b + c)];
            }
        }
        ff[i] = v;
    }
}

__global__ void k_assemble_p(int64_t nf, int64_t ne, int b, int nP, int N_max, const int32_t* __restrict__ fe,
                             const int32_t* __restrict__ flf, const int64_t* __restrict__ off_S,
                             const int32_t* __restrict__ ef_ptr, const double* __restrict__ S, double* __restrict__ fp,
                             double* __restrict__ pf, double* __restrict__ pp) {
    int64_t n_fp = 2LL * nP * b * nf, n_pf = (int64_t)N_max * b * nP * ne, n_pp = (int64_t)nP * nP * ne;
    int64_t tot = n_fp + n_pf + n_pp;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < n_fp) {
            int64_t F = i % nf, rest = i / nf;
            int r = rest % b;
            rest /= b;
            int c = rest % nP;
            int p = (int)(rest / nP);
            int T = fe[2 * F + p];
            double v = 0.0;
            if (T >= 0) {
                int lf = flf[2 * F + p], N = ef_ptr[T + 1] - ef_ptr[T], nk = N * b + nP;
                v = S[off_S[T] + (int64_t)(lf * b + r) * nk + (N * b + c)];
            }
            fp[i] = v;
        } else if (i < n_fp + n_pf) {
            int64_t j = i - n_fp;
            int64_t T = j % ne, rest = j / ne;
            int r = rest % nP;
            rest /= nP;
            int c = rest % b;
            int f = (int)(rest / b);
            int N = ef_ptr[T + 1] - ef_ptr[T], nk = N * b + nP;
            double v = 0.0;
            if (f < N) v = S[off_S[T] + (int64_t)(N * b + r) * nk + (f * b + c)];
            pf[j] = v;
        } else {
            int64_t j = i - n_fp - n_pf;
            int64_t T = j % ne, rest = j / ne;
            int r = rest % nP;
            int c = (int)(rest / nP);
            int N = ef_ptr[T + 1] - ef_ptr[T], nk = N * b + nP;
            pp[j] = S[off_S[T] + (int64_t)(N * b + r) * nk + (N * b + c)];
        }
    }
}

// coarse index within a face block -> fine index (component-major prefix)
__device__ __forceinline__ int face_map(int i, int nFc, int nFf) { return (i / nFc) * nFf + (i % nFc); }

// Element blocks hold ec components (1: a prefix of pressure coefficients;
// d + 1 when nothing is condensed: velocity components and pressure), each
// truncated like a face component.
__global__ void k_extract(int64_t nf, int64_t ne, int S_max, int N_max, int bf, int nFf, int nPf, int bc, int nFc,
                          int nPc, int ec, const double* __restrict__ ff0, const double* __restrict__ fp0,
                          const double* __restrict__ pf0, const double* __restrict__ pp0, double* __restrict__ ff,
                          double* __restrict__ fp, double* __restrict__ pf, double* __restrict__ pp) {
    int64_t n_ff = (int64_t)S_max * bc * bc * nf, n_fp = 2LL * nPc * bc * nf, n_pf = (int64_t)N_max * bc * nPc * ne,
            n_pp = (int64_t)nPc * nPc * ne;
    int64_t tot = n_ff + n_fp + n_pf + n_pp;
    const int nEc = nPc / ec, nEf = nPf / ec;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < n_ff) {
            int64_t F = i % nf, rest = i / nf;
            int r = rest % bc;
            rest /= bc;
            int c = rest % bc;
            int s = (int)(rest / bc);
            int rf = face_map(r, nFc, nFf), cf = face_map(c, nFc, nFf);
            ff[i] = ff0[(((int64_t)s * bf + cf) * bf + rf) * nf + F];
        } else if (i < n_ff + n_fp) {
            int64_t j = i - n_ff;
            int64_t F = j % nf, rest = j / nf;
            int r = rest % bc;
            rest /= bc;
            int c = rest % nPc;
            int p = (int)(rest / nPc);
            fp[j] = fp0[(((int64_t)p * nPf + face_map(c, nEc, nEf)) * bf + face_map(r, nFc, nFf)) * nf + F];
        } else if (i < n_ff + n_fp + n_pf) {
            int64_t j = i - n_ff - n_fp;
            int64_t T = j % ne, rest = j / ne;
            int r = rest % nPc;
            rest /= nPc;
            int c = rest % bc;
            int f = (int)(rest / bc);
            pf[j] = pf0[(((int64_t)f * bf + face_map(c, nFc, nFf)) * nPf + face_map(r, nEc, nEf)) * ne + T];
        } else {
            int64_t j = i - n_ff - n_fp - n_pf;
            int64_t T = j % ne, rest = j / ne;
            int r = rest % nPc;
            int c = (int)(rest / nPc);
            pp[j] = pp0[((int64_t)face_map(c, nEc, nEf) * nPf + face_map(r, nEc, nEf)) * ne + T];
        }
    }
}

// In-register Gauss-Jordan inverse of an n x n matrix (row-major in A, result in Ai), n <= NMAX.
template <int NMAX>
__device__ bool small_inverse(double* A, double* Ai, int n) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Ai[i * n + j] = (i == j) ? 1.0 : 0.0;
    for (int j = 0; j < n; ++j) {
        int p = j;
        double best = fabs(A[j * n + j]);
        for (int i = j + 1; i < n; ++i)
            if (fabs(A[i * n + j]) > best) {
                best = fabs(A[i * n + j]);
                p = i;
            }
        if (best == 0.0) return false;
        if (p != j)
            for (int c = 0; c < n; ++c) {
                double t = A[j * n + c];
                A[j * n + c] = A[p * n + c];
                A[p * n + c] = t;
                t = Ai[j * n + c];
                Ai[j * n + c] = Ai[p * n + c];
                Ai[p * n + c] = t;
            }
        double inv = 1.0 / A[j * n + j];
        for (int c = 0; c < n; ++c) {
            A[j * n + c] *= inv;
            Ai[j * n + c] *= inv;
        }
        for (int i = 0; i < n; ++i) {
            if (i == j) continue;
            double f = A[i * n + j];
            if (f == 0.0) continue;
            for (int c = 0; c < n; ++c) {
                A[i * n + c] -= f * A[j * n + c];
                Ai[i * n + c] -= f * Ai[j * n + c];
            }
        }
    }
    return true;
}

// Face block inverses D_F^{-1} (one thread per face; scratch 2*b*b per thread).
__global__ void k_face_inverse(int64_t nf, int b, const double* __restrict__ ff, double* __restrict__ dinv,
                               double* __restrict__ scratch, int* __restrict__ status) {
    int64_t F = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (F >= nf) return;
    double* A = scratch + F * 2 * b * b;
    double* Ai = A + b * b;
    for (int r = 0; r < b; ++r)
        for (int c = 0; c < b; ++c) A[r * b + c] = ff[((int64_t)c * b + r) * nf + F];
    if (!small_inverse<64>(A, Ai, b)) {
        atomicExch(status, (int)HHO_ERR_SINGULAR);
        return;
    }
    for (int r = 0; r < b; ++r)
        for (int c = 0; c < b; ++c) dinv[((int64_t)c * b + r) * nf + F] = Ai[r * b + c];
}

// Element pressure pivot blocks M_T = S_TT - sum_F S_TF D_F^{-1} S_FT and their inverses.
__global__ void k_elem_pivot(int64_t ne, int64_t nf, int b, int nP, int N_max, const int32_t* __restrict__ pf_col,
                             const int32_t* __restrict__ pf_nsl, const int32_t* __restrict__ fe,
                             const double* __restrict__ fp, const double* __restrict__ pf, const double* __restrict__ pp,
                             const double* __restrict__ dinv, double* __restrict__ minv, double* __restrict__ scratch,
                             int* __restrict__ status) {
    int64_t T = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (T >= ne) return;
    double* M = scratch + T * (2 * nP * nP + b * nP);
    double* Mi = M + nP * nP;
    double* DS = Mi + nP * nP;  // D_F^{-1} S_FT  (b x nP)
    for (int r = 0; r < nP; ++r)
        for (int c = 0; c < nP; ++c) M[r * nP + c] = pp[((int64_t)c * nP + r) * ne + T];
    for (int f = 0; f < pf_nsl[T]; ++f) {
        int F = pf_col[f * ne + T];
        int p = (fe[2 * F] == T) ? 0 : 1;
        // DS = D_F^{-1} S_FT
        for (int r = 0; r < b; ++r)
            for (int c = 0; c < nP; ++c) {
                double s = 0.0;
                for (int l = 0; l < b; ++l)
                    s += dinv[((int64_t)l * b + r) * nf + F] * fp[(((int64_t)p * nP + c) * b + l) * nf + F];
                DS[r * nP + c] = s;
            }
        for (int r = 0; r < nP; ++r)
            for (int c = 0; c < nP; ++c) {
                double s = 0.0;
                for (int l = 0; l < b; ++l) s += pf[(((int64_t)f * b + l) * nP + r) * ne + T] * DS[l * nP + c];
                M[r * nP + c] -= s;
            }
    }
    if (!small_inverse<32>(M, Mi, nP)) {
        atomicExch(status, (int)HHO_ERR_SINGULAR);
        return;
    }
    for (int r = 0; r < nP; ++r)
        for (int c = 0; c < nP; ++c) minv[((int64_t)c * nP + r) * ne + T] = Mi[r * nP + c];
}

__global__ void k_rhs_gather(int64_t nf, int64_t ne, int b, int nP, const int32_t* __restrict__ fe,
                             const int32_t* __restrict__ flf, const int32_t* __restrict__ ef_ptr,
                             const int64_t* __restrict__ off_gT, const double* __restrict__ gT, double* __restrict__ rhs) {
    int64_t n = nf * b + ne * nP;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        if (i < nf * b) {
            int64_t F = i / b;
            int r = i % b;
            for (int e = 0; e < 2; ++e) {
                int T = fe[2 * F + e];
                if (T < 0) continue;
                v += gT[off_gT[T] + flf[2 * F + e] * b + r];
            }
        } else {
            int64_t j = i - nf * b, T = j / nP;
            int r = j % nP;
            int N = ef_ptr[T + 1] - ef_ptr[T];
            v = gT[off_gT[T] + N * b + r];
        }
        rhs[i] = v;
    }
}

int grid_for(int64_t n, int tpb) {
    int64_t g = (n + tpb - 1) / tpb;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)sm_count() * 32));
}

}  // namespace

// DG scheme: the block rows are the elements.  Row block of element T: slot 0
// is T, slot 1 + i the neighbour across T's i-th interior face (local order;
// boundary faces couple nothing), padding slots repeat T with zero blocks.
// No element rows (nP = 0): the element-row arrays hold one dummy slot.
static hho_status build_topology_dg(hho_ctx* ctx) {
    Disc& D = ctx->disc;
    Topo& P = ctx->topo;
    const int64_t ne = D.ne;
    auto neighbour = [&](int64_t T, int g) -> int32_t {
        const int F = D.h_ef[g];
        const int a = D.h_fe[2 * F], b = D.h_fe[2 * F + 1];
        if (a < 0 || b < 0) return -1;
        return a == T ? b : a;
    };
    int S_max = 1;
    for (int64_t T = 0; T < ne; ++T) {
        int s = 1;
        for (int g = D.h_ef_ptr[T]; g < D.h_ef_ptr[T + 1]; ++g) s += neighbour(T, g) >= 0;
        S_max = std::max(S_max, s);
    }
    P.S_max = S_max;
    P.N_max = 1;
    std::vector<int32_t> col((size_t)S_max * ne), nsl(ne), fpc(2 * ne, -1), pfc(ne), pfn(ne, 0);
    for (int64_t T = 0; T < ne; ++T) {
        int s = 0;
        col[T] = (int32_t)T;
        ++s;
        for (int g = D.h_ef_ptr[T]; g < D.h_ef_ptr[T + 1]; ++g) {
            const int32_t G = neighbour(T, g);
            if (G >= 0) col[(size_t)s++ * ne + T] = G;
        }
        nsl[T] = s;
        for (; s < S_max; ++s) col[(size_t)s * ne + T] = (int32_t)T;
        pfc[T] = (int32_t)T;
    }
    P.h_ff_col = col;
    P.h_ff_nsl = nsl;
    P.h_fp_col = fpc;
    P.h_pf_col = pfc;
    P.h_pf_nsl = pfn;
    auto up = [&](int32_t** dst, const std::vector<int32_t>& v) -> hho_status {
        HHO_TRY(dalloc(ctx, dst, v.size()));
        HHO_CUDA(cudaMemcpyAsync(*dst, v.data(), v.size() * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
        return HHO_OK;
    };
    HHO_TRY(up(&P.ff_col, col));
    HHO_TRY(up(&P.ff_nsl, nsl));
    HHO_TRY(up(&P.fp_col, fpc));
    HHO_TRY(up(&P.pf_col, pfc));
    HHO_TRY(up(&P.pf_nsl, pfn));
    HHO_CUDA(cudaStreamSynchronize(ctx->stream));
    return HHO_OK;
}

hho_status build_topology(hho_ctx* ctx) {
    Disc& D = ctx->disc;
    if (D.cond == HHO_DGCOND) return build_topology_dg(ctx);
    Topo& P = ctx->topo;
    const int64_t nf = D.nf, ne = D.ne;
    int S_max = 1;
    for (int64_t F = 0; F < nf; ++F) {
        int s = 1;
        for (int e = 0; e < 2; ++e) {
            int T = D.h_fe[2 * F + e];
            if (T >= 0) s += D.h_ef_ptr[T + 1] - D.h_ef_ptr[T] - 1;
        }
        S_max = std::max(S_max, s);
    }
    P.S_max = S_max;
    P.N_max = D.maxN;
    std::vector<int32_t> col((size_t)S_max * nf), nsl(nf), aT((size_t)S_max * nf, -1), alf((size_t)S_max * nf, -1),
        alg((size_t)S_max * nf, -1), fpc(2 * nf), pfc((size_t)P.N_max * ne), pfn(ne);
    for (int64_t F = 0; F < nf; ++F) {
        int s = 0;
        col[s * nf + F] = (int32_t)F;
        ++s;
        for (int e = 0; e < 2; ++e) {
            int T = D.h_fe[2 * F + e];
            fpc[e * nf + F] = T;
            if (T < 0) continue;
            int lf = D.h_flf[2 * F + e];
            for (int g = D.h_ef_ptr[T]; g < D.h_ef_ptr[T + 1]; ++g) {
                int lg = g - D.h_ef_ptr[T];
                if (lg == lf) continue;
                col[s * nf + F] = D.h_ef[g];
                aT[s * nf + F] = T;
                alf[s * nf + F] = lf;
                alg[s * nf + F] = lg;
                ++s;
            }
        }
        nsl[F] = s;
        for (; s < S_max; ++s) col[s * nf + F] = (int32_t)F;
    }
    for (int64_t T = 0; T < ne; ++T) {
        int N = D.h_ef_ptr[T + 1] - D.h_ef_ptr[T];
        pfn[T] = N;
        for (int f = 0; f < P.N_max; ++f) pfc[f * ne + T] = (f < N) ? D.h_ef[D.h_ef_ptr[T] + f] : D.h_ef[D.h_ef_ptr[T]];
    }
    P.h_ff_col = col;
    P.h_ff_nsl = nsl;
    P.h_fp_col = fpc;
    P.h_pf_col = pfc;
    P.h_pf_nsl = pfn;
    auto up = [&](int32_t** dst, const std::vector<int32_t>& v) -> hho_status {
        HHO_TRY(dalloc(ctx, dst, v.size()));
        HHO_CUDA(cudaMemcpyAsync(*dst, v.data(), v.size() * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
        return HHO_OK;
    };
    HHO_TRY(up(&P.ff_col, col));
    HHO_TRY(up(&P.ff_nsl, nsl));
    HHO_TRY(up(&P.fp_col, fpc));
    HHO_TRY(up(&P.pf_col, pfc));
    HHO_TRY(up(&P.pf_nsl, pfn));
    HHO_TRY(up(&P.asm_T, aT));
    HHO_TRY(up(&P.asm_lf, alf));
    HHO_TRY(up(&P.asm_lg, alg));
    HHO_CUDA(cudaStreamSynchronize(ctx->stream));
    return HHO_OK;
}

static hho_status alloc_level(hho_ctx* ctx, LevelMat& L) {
    const Topo& P = ctx->topo;
    L.S_max = P.S_max;
    L.N_max = P.N_max;
    L.ff_col = P.ff_col;
    L.ff_nsl = P.ff_nsl;
    L.fp_col = P.fp_col;
    L.pf_col = P.pf_col;
    L.pf_nsl = P.pf_nsl;
    HHO_TRY(dalloc(ctx, &L.ff, (size_t)L.S_max * L.b * L.b * L.nf));
    HHO_TRY(dalloc(ctx, &L.fp, (size_t)2 * L.nP * L.b * L.nf));
    HHO_TRY(dalloc(ctx, &L.pf, (size_t)L.N_max * L.b * L.nP * L.ne));
    HHO_TRY(dalloc(ctx, &L.pp, (size_t)L.nP * L.nP * L.ne));
    return HHO_OK;
}

void free_level(LevelMat& L) {
    dfree(L.ff);
    dfree(L.fp);
    dfree(L.pf);
    dfree(L.pp);
    dfree(L.dinv);
    dfree(L.minv);
    L.ff = L.fp = L.pf = L.pp = L.dinv = L.minv = nullptr;
    dfree(L.ff32);
    dfree(L.fp32);
    dfree(L.pf32);
    dfree(L.pp32);
    dfree(L.dinv32);
    dfree(L.minv32);
    L.ff32 = L.fp32 = L.pf32 = L.pp32 = L.dinv32 = L.minv32 = nullptr;
    L.ilv = false;
}

hho_status assemble_level0(hho_ctx* ctx) {
    Disc& D = ctx->disc;
    const Topo& P = ctx->topo;
    const bool dg = D.cond == HHO_DGCOND;
    if (ctx->levels.empty()) {
        LevelMat L;
        L.k = D.k;
        L.nF = dg ? D.nE : D.nF;  // DG: element blocks of d + 1 components of P^k(T)
        L.b = D.b;
        L.nP = D.nP;
        L.nf = dg ? D.ne : D.nf;
        L.ne = D.ne;
        L.n = L.nf * L.b + L.ne * L.nP;
        HHO_TRY(alloc_level(ctx, L));
        ctx->levels.push_back(L);
    }
    LevelMat& L = ctx->levels[0];
    if (dg) {
        HHO_TRY(dg_assemble_level0(ctx, L.ff, P.S_max));
        HHO_CUDA(cudaStreamSynchronize(ctx->stream));
        return HHO_OK;
    }
    int64_t tot = (int64_t)P.S_max * L.b * L.b * L.nf;
    k_assemble_ff<<<grid_for(tot, 256), 256, 0, ctx->stream>>>(L.nf, L.b, P.S_max, P.ff_nsl, P.asm_T, P.asm_lf,
                                                               P.asm_lg, D.fe, D.flf, D.off_S, D.ef_ptr, L.nP, D.S,
                                                               L.ff);
    HHO_CUDA(cudaGetLastError());
    int64_t tp = 2LL * L.nP * L.b * L.nf + (int64_t)P.N_max * L.b * L.nP * L.ne + (int64_t)L.nP * L.nP * L.ne;
    k_assemble_p<<<grid_for(tp, 256), 256, 0, ctx->stream>>>(L.nf, L.ne, L.b, L.nP, P.N_max, D.fe, D.flf, D.off_S,
                                                             D.ef_ptr, D.S, L.fp, L.pf, L.pp);
    HHO_CUDA(cudaGetLastError());
    HHO_CUDA(cudaStreamSynchronize(ctx->stream));
    return HHO_OK;
}

hho_status assemble_rhs_vector(hho_ctx* ctx, double* rhs) {
    Disc& D = ctx->disc;
    if (D.cond == HHO_DGCOND) {  // the element blocks of the right-hand side, in element order
        HHO_CUDA(cudaMemcpyAsync(rhs, D.gT, (size_t)D.ne * D.b * sizeof(double), cudaMemcpyDeviceToDevice,
                                 ctx->stream));
        return HHO_OK;
    }
    int64_t n = D.nf * D.b + D.ne * D.nP;
    k_rhs_gather<<<grid_for(n, 256), 256, 0, ctx->stream>>>(D.nf, D.ne, D.b, D.nP, D.fe, D.flf, D.ef_ptr, D.off_gT,
                                                            D.gT, rhs);
    HHO_CUDA(cudaGetLastError());
    return HHO_OK;
}

hho_status build_level(hho_ctx* ctx, int l, int k_l) {
    Disc& D = ctx->disc;
    LevelMat L;
    L.k = k_l;
    const bool dg = D.cond == HHO_DGCOND;
    L.nF = dg ? dimP(D.d, k_l) : dimP(D.d - 1, k_l);  // DG: element blocks, every component truncated
    L.b = (D.cond == HHO_HPCOND || dg ? D.d + 1 : D.d) * L.nF;  // HHO-hp: the face pressure is one more component
    L.nP = (D.cond == HHO_HPCOND || dg) ? 0
           : (D.cond == HHO_VPCOND)     ? 1
           : (D.cond == HHO_UNCOND)     ? (D.d + 1) * dimP(D.d, k_l)  // velocity components and pressure
                                        : dimP(D.d, k_l);
    L.nf = dg ? D.ne : D.nf;
    L.ne = D.ne;
    L.n = L.nf * L.b + L.ne * L.nP;
    HHO_TRY(alloc_level(ctx, L));
    const LevelMat& Fm = ctx->levels[l - 1];
    int64_t tot = (int64_t)L.S_max * L.b * L.b * L.nf + 2LL * L.nP * L.b * L.nf + (int64_t)L.N_max * L.b * L.nP * L.ne +
                  (int64_t)L.nP * L.nP * L.ne;
    k_extract<<<grid_for(tot, 256), 256, 0, ctx->stream>>>(L.nf, L.ne, L.S_max, L.N_max, Fm.b, Fm.nF, Fm.nP, L.b, L.nF,
                                                           L.nP, elem_comp(D.cond, D.d), Fm.ff, Fm.fp, Fm.pf, Fm.pp,
                                                           L.ff, L.fp, L.pf, L.pp);
    HHO_CUDA(cudaGetLastError());
    if ((int)ctx->levels.size() > l) {
        free_level(ctx->levels[l]);
        ctx->levels[l] = L;
    } else {
        ctx->levels.push_back(L);
    }
    return HHO_OK;
}

hho_status build_smoother(hho_ctx* ctx, int l) {
    LevelMat& L = ctx->levels[l];
    if (L.b > 64 || L.nP > 32) {
        ctx->err = "pmg_setup: block too large for the block-Jacobi setup";
        return HHO_ERR_UNSUPPORTED;
    }
    dfree(L.dinv);
    dfree(L.minv);
    L.dinv = L.minv = nullptr;
    HHO_TRY(dalloc(ctx, &L.dinv, (size_t)L.b * L.b * L.nf));
    HHO_TRY(dalloc(ctx, &L.minv, (size_t)L.nP * L.nP * L.ne));
    double* scratch = nullptr;
    size_t need = std::max<size_t>((size_t)L.nf * 2 * L.b * L.b, (size_t)L.ne * (2 * L.nP * L.nP + L.b * L.nP));
    HHO_TRY(dalloc(ctx, &scratch, need));
    HHO_CUDA(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream));
    k_face_inverse<<<(unsigned)((L.nf + 127) / 128), 128, 0, ctx->stream>>>(L.nf, L.b, L.ff, L.dinv, scratch,
                                                                               ctx->d_flag);
    cudaError_t e1 = cudaGetLastError();
    if (L.nP > 0)  // element pressure pivot blocks (none under HHO-hp)
        k_elem_pivot<<<(unsigned)((L.ne + 127) / 128), 128, 0, ctx->stream>>>(L.ne, L.nf, L.b, L.nP, L.N_max,
                                                                                L.pf_col, L.pf_nsl, ctx->disc.fe, L.fp,
                                                                                L.pf, L.pp, L.dinv, L.minv, scratch,
                                                                                ctx->d_flag);
    cudaError_t e2 = cudaGetLastError();
    int flag = 0;
    cudaError_t e3 = cudaMemcpyAsync(&flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    cudaError_t e4 = cudaStreamSynchronize(ctx->stream);
    dfree(scratch);
    HHO_CUDA(e1);
    HHO_CUDA(e2);
    HHO_CUDA(e3);
    HHO_CUDA(e4);
    if (flag) {
        ctx->err = "pmg_setup: singular smoother block";
        return HHO_ERR_SINGULAR;
    }
    return HHO_OK;
}

hho_status level_coo(hho_ctx* ctx, int l, int64_t* rows, int64_t* cols, double* vals, int64_t* nnz) {
    if (l < 0 || l >= (int)ctx->levels.size()) {
        ctx->err = "hho_get_level_coo: no such level";
        return HHO_ERR_ARG;
    }
    const LevelMat& L = ctx->levels[l];
    const Topo& P = ctx->topo;
    const int64_t nf = L.nf, ne = L.ne;
    int b = L.b, nP = L.nP;
    int64_t count = 0;
    for (int64_t F = 0; F < nf; ++F) {
        count += (int64_t)P.h_ff_nsl[F] * b * b;
        for (int p = 0; p < 2; ++p)
            if (P.h_fp_col[p * nf + F] >= 0) count += (int64_t)b * nP;
    }
    for (int64_t T = 0; T < ne; ++T) count += (int64_t)P.h_pf_nsl[T] * b * nP + (int64_t)nP * nP;
    *nnz = count;
    if (!rows || !cols || !vals) return HHO_OK;
    std::vector<double> ff((size_t)L.S_max * b * b * nf), fp((size_t)2 * nP * b * nf), pf((size_t)L.N_max * b * nP * ne),
        pp((size_t)nP * nP * ne);
    HHO_CUDA(cudaMemcpyAsync(ff.data(), L.ff, ff.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
    HHO_CUDA(cudaMemcpyAsync(fp.data(), L.fp, fp.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
    HHO_CUDA(cudaMemcpyAsync(pf.data(), L.pf, pf.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
    HHO_CUDA(cudaMemcpyAsync(pp.data(), L.pp, pp.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
    HHO_CUDA(cudaStreamSynchronize(ctx->stream));
    int64_t o = 0;
    const int64_t pbase = nf * b;
    for (int64_t F = 0; F < nf; ++F) {
        for (int s = 0; s < P.h_ff_nsl[F]; ++s) {
            int64_t G = P.h_ff_col[s * nf + F];
            for (int c = 0; c < b; ++c)
                for (int r = 0; r < b; ++r) {
                    rows[o] = F * b + r;
                    cols[o] = G * b + c;
                    vals[o++] = ff[(((int64_t)s * b + c) * b + r) * nf + F];
                }
        }
        for (int p = 0; p < 2; ++p) {
            int64_t T = P.h_fp_col[p * nf + F];
            if (T < 0) continue;
            for (int c = 0; c < nP; ++c)
                for (int r = 0; r < b; ++r) {
                    rows[o] = F * b + r;
                    cols[o] = pbase + T * nP + c;
                    vals[o++] = fp[(((int64_t)p * nP + c) * b + r) * nf + F];
                }
        }
    }
    for (int64_t T = 0; T < ne; ++T) {
        for (int f = 0; f < P.h_pf_nsl[T]; ++f) {
            int64_t G = P.h_pf_col[f * ne + T];
            for (int c = 0; c < b; ++c)
                for (int r = 0; r < nP; ++r) {
                    rows[o] = pbase + T * nP + r;
                    cols[o] = G * b + c;
                    vals[o++] = pf[(((int64_t)f * b + c) * nP + r) * ne + T];
                }
        }
        for (int c = 0; c < nP; ++c)
            for (int r = 0; r < nP; ++r) {
                rows[o] = pbase + T * nP + r;
                cols[o] = pbase + T * nP + c;
                vals[o++] = pp[((int64_t)c * nP + r) * ne + T];
            }
    }
    return HHO_OK;
}

}  // namespace hho
