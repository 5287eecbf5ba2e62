// Block ILU(0) smoother preconditioner on the GPU (Sec. 3.3 / Sec. 5.2.2: the
// paper smooths with ILU-preconditioned GMRES; fill, ordering and block size are
// not given).  Reading: block ILU(0) on the block pattern of the level
// operator S (face blocks of b unknowns, element pressure blocks of nP), no
// fill, with the faces first in a greedy multicolour order (faces sharing an
// element get different colours; face F, in index order, takes the smallest
// colour not used by an already coloured adjacent face; faces sorted by
// (colour, index)) and the element pressure blocks last, so the zero
// mean-pressure diagonal is pivoted on its Schur-like block.
//
// Because no two faces of one colour are in each other's pattern, every colour
// is factored, and swept in the triangular solves, in parallel:
//   factorisation (IKJ on the pattern, once per pmg_setup): one CTA per block
//     row, colour after colour, then all element rows;
//   application z = U^{-1} L^{-1} v: forward sweep colour by colour, then the
//     element rows; backward sweep over the element rows, then colours in
//     reverse; one thread per block row.
// Factors keep the level layouts ([slot][col][row][position]) with the face
// index replaced by the face's position in colour order, so that the faces of
// one colour are contiguous and their reads coalesce.  Integer bookkeeping
// (colouring, orders, pattern lookups) is done on the host once.
#include <algorithm>
#include <numeric>
#include <vector>

#include "dense.cuh"
#include "internal.h"

namespace hho {

struct IluLevel {
    int b = 0, nP = 0, S_max = 0, N_max = 0, ncol = 0;
    int64_t nf = 0, ne = 0;
    std::vector<int32_t> coff;            // host: colour c owns positions [coff[c], coff[c+1])
    int32_t *pos = nullptr, *face_at = nullptr;  // face -> position, position -> face
    int32_t *lorder = nullptr, *nlow = nullptr;  // per face: lower slots in rank order
    int8_t *fpos = nullptr, *fepos = nullptr;    // pattern lookups of the face rows
    int8_t *torder = nullptr, *tpos = nullptr, *tside = nullptr;  // of the element rows
    double *lff = nullptr, *lfp = nullptr, *lpf = nullptr, *lpp = nullptr, *uf = nullptr, *ue = nullptr;
    float *lff32 = nullptr, *lfp32 = nullptr, *lpf32 = nullptr, *lpp32 = nullptr, *uf32 = nullptr, *ue32 = nullptr;
};

namespace {

int g1(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 32)); }

// dst[p * nf + pos[F]] = src[p * nf + F] for every plane p (face-indexed arrays to colour order)
__global__ void k_perm_faces(int64_t planes, int64_t nf, const int32_t* __restrict__ pos, const double* __restrict__ src,
                             double* __restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < planes * nf;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = i / nf, F = i % nf;
        dst[p * nf + pos[F]] = src[i];
    }
}

__global__ void k_copy_d(int64_t n, const double* __restrict__ a, double* __restrict__ b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = a[i];
}

__global__ void k_to_f32(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

struct IluView {
    int b, nP, S_max, N_max;
    int64_t nf, ne;
    const int32_t *ff_col, *ff_nsl, *fp_col, *pf_col, *pf_nsl;  // level topology (natural face ids)
    const int32_t *pos, *face_at, *lorder, *nlow;
    const int8_t *fpos, *fepos, *torder, *tpos, *tside;
};

// Block accessors on the factor layouts (positions, not face ids, for face rows)
__device__ __forceinline__ double& FF(double* a, const IluView& v, int s, int r, int c, int64_t P) {
    return a[(((int64_t)s * v.b + c) * v.b + r) * v.nf + P];
}
__device__ __forceinline__ double& FP(double* a, const IluView& v, int p, int r, int c, int64_t P) {
    return a[(((int64_t)p * v.nP + c) * v.b + r) * v.nf + P];
}
__device__ __forceinline__ double& PF(double* a, const IluView& v, int f, int r, int c, int64_t T) {
    return a[(((int64_t)f * v.b + c) * v.nP + r) * v.ne + T];
}
__device__ __forceinline__ double& PP(double* a, const IluView& v, int r, int c, int64_t T) {
    return a[((int64_t)c * v.nP + r) * v.ne + T];
}
__device__ __forceinline__ double& UFI(double* a, const IluView& v, int r, int c, int64_t P) {
    return a[((int64_t)c * v.b + r) * v.nf + P];
}
__device__ __forceinline__ double& UEI(double* a, const IluView& v, int r, int c, int64_t T) {
    return a[((int64_t)c * v.nP + r) * v.ne + T];
}

constexpr int IB = 128;  // threads per CTA of the factorisation kernels
constexpr int MB = 32;   // largest block handled (b, nP <= 32)

// inverse of the n x n block held in sA (row-major, ld MB) into global through put(r, c, value)
__device__ bool cta_inverse(double* sW, int n) {
    __shared__ int s_piv;
    return cta_gauss_jordan(sW, 2 * MB, n, n, &s_piv);
}

// Face rows of one colour: L_FG = A_FG U_GG^{-1} for the lower slots in rank
// order, the pattern updates of the later blocks, then U_FF^{-1}.
__global__ void __launch_bounds__(IB) k_ilu_face_rows(IluView v, int p0, int p1, double* __restrict__ lff,
                                                      double* __restrict__ lfp, double* __restrict__ uf,
                                                      int* __restrict__ status) {
    __shared__ double sL[MB * MB], sU[MB * MB], sW[MB * 2 * MB];
    const int b = v.b, nP = v.nP;
    for (int P = p0 + blockIdx.x; P < p1; P += gridDim.x) {
        const int F = v.face_at[P];
        const int ns = v.ff_nsl[F];
        for (int li = 0; li < v.nlow[F]; ++li) {
            const int s = v.lorder[(int64_t)F * v.S_max + li];
            const int G = v.ff_col[(int64_t)s * v.nf + F];
            const int64_t PG = v.pos[G];
            // L = A_FG U_GG^{-1}
            for (int i = threadIdx.x; i < b * b; i += blockDim.x) {
                const int r = i / b, c = i % b;
                sU[r * MB + c] = UFI(uf, v, r, c, PG);
                sW[r * MB + c] = FF(lff, v, s, r, c, P);
            }
            __syncthreads();
            for (int i = threadIdx.x; i < b * b; i += blockDim.x) {
                const int r = i / b, c = i % b;
                double a = 0.0;
                for (int q = 0; q < b; ++q) a += sW[r * MB + q] * sU[q * MB + c];
                sL[r * MB + c] = a;
                FF(lff, v, s, r, c, P) = a;
            }
            __syncthreads();
            // later face blocks of the row that row G also holds
            for (int t = 0; t < ns; ++t) {
                const int u = v.fpos[((int64_t)F * v.S_max + s) * v.S_max + t];
                if (u < 0) continue;
                for (int i = threadIdx.x; i < b * b; i += blockDim.x) {
                    const int r = i / b, c = i % b;
                    double a = 0.0;
                    for (int q = 0; q < b; ++q) a += sL[r * MB + q] * FF(lff, v, u, q, c, PG);
                    FF(lff, v, t, r, c, P) -= a;
                }
                __syncthreads();
            }
            // the row's element blocks that row G also holds
            for (int p = 0; p < 2; ++p) {
                const int q2 = v.fepos[((int64_t)F * v.S_max + s) * 2 + p];
                if (q2 < 0) continue;
                for (int i = threadIdx.x; i < b * nP; i += blockDim.x) {
                    const int r = i / nP, c = i % nP;
                    double a = 0.0;
                    for (int q = 0; q < b; ++q) a += sL[r * MB + q] * FP(lfp, v, q2, q, c, PG);
                    FP(lfp, v, p, r, c, P) -= a;
                }
                __syncthreads();
            }
        }
        // U_FF^{-1}
        for (int i = threadIdx.x; i < b * 2 * b; i += blockDim.x) {
            const int r = i / (2 * b), c = i % (2 * b);
            sW[r * 2 * MB + c] = (c < b) ? FF(lff, v, 0, r, c, P) : ((c - b == r) ? 1.0 : 0.0);
        }
        __syncthreads();
        if (!cta_inverse(sW, b)) {
            if (threadIdx.x == 0) atomicExch(status, (int)HHO_ERR_SINGULAR);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < b * b; i += blockDim.x) {
            const int r = i / b, c = i % b;
            UFI(uf, v, r, c, P) = sW[r * 2 * MB + b + c];
        }
        __syncthreads();
    }
}

// Element rows (after every face): L_TF = A_TF U_FF^{-1} over the element's
// faces in rank order, updates of its later faces and of A_TT, then U_TT^{-1}.
__global__ void __launch_bounds__(IB) k_ilu_elem_rows(IluView v, double* __restrict__ lff, double* __restrict__ lfp,
                                                      double* __restrict__ lpf, double* __restrict__ lpp,
                                                      const double* __restrict__ uf, double* __restrict__ ue,
                                                      int* __restrict__ status) {
    __shared__ double sL[MB * MB], sU[MB * MB], sW[MB * 2 * MB];
    const int b = v.b, nP = v.nP;
    for (int64_t T = blockIdx.x; T < v.ne; T += gridDim.x) {
        const int N = v.pf_nsl[T];
        for (int li = 0; li < N; ++li) {
            const int f = v.torder[T * v.N_max + li];
            const int F = v.pf_col[(int64_t)f * v.ne + T];
            const int64_t PF_ = v.pos[F];
            for (int i = threadIdx.x; i < b * b; i += blockDim.x) {
                const int r = i / b, c = i % b;
                sU[r * MB + c] = UFI(const_cast<double*>(uf), v, r, c, PF_);
            }
            for (int i = threadIdx.x; i < nP * b; i += blockDim.x) {
                const int r = i / b, c = i % b;
                sW[r * MB + c] = PF(lpf, v, f, r, c, T);
            }
            __syncthreads();
            for (int i = threadIdx.x; i < nP * b; i += blockDim.x) {
                const int r = i / b, c = i % b;
                double a = 0.0;
                for (int q = 0; q < b; ++q) a += sW[r * MB + q] * sU[q * MB + c];
                sL[r * MB + c] = a;
                PF(lpf, v, f, r, c, T) = a;
            }
            __syncthreads();
            for (int gi = li + 1; gi < N; ++gi) {
                const int g = v.torder[T * v.N_max + gi];
                const int u = v.tpos[(T * v.N_max + f) * v.N_max + g];
                if (u < 0) continue;
                for (int i = threadIdx.x; i < nP * b; i += blockDim.x) {
                    const int r = i / b, c = i % b;
                    double a = 0.0;
                    for (int q = 0; q < b; ++q) a += sL[r * MB + q] * FF(lff, v, u, q, c, PF_);
                    PF(lpf, v, g, r, c, T) -= a;
                }
                __syncthreads();
            }
            const int side = v.tside[T * v.N_max + f];
            for (int i = threadIdx.x; i < nP * nP; i += blockDim.x) {
                const int r = i / nP, c = i % nP;
                double a = 0.0;
                for (int q = 0; q < b; ++q) a += sL[r * MB + q] * FP(lfp, v, side, q, c, PF_);
                PP(lpp, v, r, c, T) -= a;
            }
            __syncthreads();
        }
        for (int i = threadIdx.x; i < nP * 2 * nP; i += blockDim.x) {
            const int r = i / (2 * nP), c = i % (2 * nP);
            sW[r * 2 * MB + c] = (c < nP) ? PP(lpp, v, r, c, T) : ((c - nP == r) ? 1.0 : 0.0);
        }
        __syncthreads();
        if (!cta_inverse(sW, nP)) {
            if (threadIdx.x == 0) atomicExch(status, (int)HHO_ERR_SINGULAR);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nP * nP; i += blockDim.x) {
            const int r = i / nP, c = i % nP;
            UEI(ue, v, r, c, T) = sW[r * 2 * MB + nP + c];
        }
        __syncthreads();
    }
}

// ---- application, one thread per block row ----
template <typename T>
struct IluData {
    const T *lff, *lfp, *lpf, *lpp, *uf, *ue;
};

// forward sweep of one colour: z_F = v_F - sum over lower slots of L_FG z_G
template <int B, typename T>
__global__ void k_ilu_fwd_face(IluView v, IluData<T> d, int p0, int p1, const int32_t* __restrict__ rank,
                               const T* __restrict__ vin, T* __restrict__ z) {
    const int64_t nf = v.nf;
    for (int P = p0 + blockIdx.x * blockDim.x + threadIdx.x; P < p1; P += gridDim.x * blockDim.x) {
        const int F = v.face_at[P];
        T acc[B];
#pragma unroll
        for (int r = 0; r < B; ++r) acc[r] = vin[(int64_t)F * B + r];
        const int ns = v.ff_nsl[F];
        for (int s = 1; s < ns; ++s) {
            const int G = v.ff_col[(int64_t)s * nf + F];
            if (rank[G] >= P) continue;  // rank = colour position; earlier colours only
            const T* zg = z + (int64_t)G * B;
#pragma unroll
            for (int c = 0; c < B; ++c) {
                const T x = zg[c];
#pragma unroll
                for (int r = 0; r < B; ++r) acc[r] -= d.lff[(((int64_t)s * B + c) * B + r) * nf + P] * x;
            }
        }
#pragma unroll
        for (int r = 0; r < B; ++r) z[(int64_t)F * B + r] = acc[r];
    }
}

// element rows of the forward sweep: z_T = v_T - sum_F L_TF z_F
template <int B, typename T>
__global__ void k_ilu_fwd_elem(IluView v, IluData<T> d, const T* __restrict__ vin, T* __restrict__ z) {
    const int64_t nf = v.nf, ne = v.ne;
    const int nP = v.nP;
    for (int64_t E = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; E < ne * nP;
         E += (int64_t)gridDim.x * blockDim.x) {
        const int64_t Te = E % ne;
        const int r = (int)(E / ne);
        T acc = vin[nf * B + Te * nP + r];
        const int N = v.pf_nsl[Te];
        for (int f = 0; f < N; ++f) {
            const T* zf = z + (int64_t)v.pf_col[(int64_t)f * ne + Te] * B;
#pragma unroll
            for (int c = 0; c < B; ++c) acc -= d.lpf[(((int64_t)f * B + c) * nP + r) * ne + Te] * zf[c];
        }
        z[nf * B + Te * nP + r] = acc;
    }
}

// element rows of the backward sweep: z_T = U_TT^{-1} z_T (elements are last: nothing after them)
template <int B, typename T>
__global__ void k_ilu_bwd_elem(IluView v, IluData<T> d, T* __restrict__ z, T* __restrict__ tmp) {
    const int64_t nf = v.nf, ne = v.ne;
    const int nP = v.nP;
    for (int64_t E = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; E < ne * nP;
         E += (int64_t)gridDim.x * blockDim.x) {
        const int64_t Te = E % ne;
        const int r = (int)(E / ne);
        T acc = 0;
        for (int c = 0; c < nP; ++c) acc += d.ue[((int64_t)c * nP + r) * ne + Te] * z[nf * B + Te * nP + c];
        tmp[Te * nP + r] = acc;
    }
}

__global__ void k_ilu_elem_store(int64_t n, int64_t off, const double* __restrict__ tmp, double* __restrict__ z) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        z[off + i] = tmp[i];
}
__global__ void k_ilu_elem_store(int64_t n, int64_t off, const float* __restrict__ tmp, float* __restrict__ z) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        z[off + i] = tmp[i];
}

// backward sweep of one colour: z_F = U_FF^{-1} (z_F - sum over upper slots U_FG z_G - sum_p U_FT z_T)
template <int B, typename T>
__global__ void k_ilu_bwd_face(IluView v, IluData<T> d, int p0, int p1, const int32_t* __restrict__ rank,
                               T* __restrict__ z) {
    const int64_t nf = v.nf;
    const int nP = v.nP;
    for (int P = p0 + blockIdx.x * blockDim.x + threadIdx.x; P < p1; P += gridDim.x * blockDim.x) {
        const int F = v.face_at[P];
        T t[B];
#pragma unroll
        for (int r = 0; r < B; ++r) t[r] = z[(int64_t)F * B + r];
        const int ns = v.ff_nsl[F];
        for (int s = 1; s < ns; ++s) {
            const int G = v.ff_col[(int64_t)s * nf + F];
            if (rank[G] <= P) continue;  // later colours only
            const T* zg = z + (int64_t)G * B;
#pragma unroll
            for (int c = 0; c < B; ++c) {
                const T x = zg[c];
#pragma unroll
                for (int r = 0; r < B; ++r) t[r] -= d.lff[(((int64_t)s * B + c) * B + r) * nf + P] * x;
            }
        }
        for (int p = 0; p < 2; ++p) {
            const int Te = v.fp_col[(int64_t)p * nf + F];
            if (Te < 0) continue;
            const T* zt = z + nf * B + (int64_t)Te * nP;
            for (int c = 0; c < nP; ++c) {
                const T x = zt[c];
#pragma unroll
                for (int r = 0; r < B; ++r) t[r] -= d.lfp[(((int64_t)p * nP + c) * B + r) * nf + P] * x;
            }
        }
        T o[B];
#pragma unroll
        for (int r = 0; r < B; ++r) {
            T a = 0;
#pragma unroll
            for (int c = 0; c < B; ++c) a += d.uf[((int64_t)c * B + r) * nf + P] * t[c];
            o[r] = a;
        }
#pragma unroll
        for (int r = 0; r < B; ++r) z[(int64_t)F * B + r] = o[r];
    }
}

IluView view_of(const hho_ctx* ctx, const LevelMat& L, const IluLevel& I) {
    return IluView{I.b, I.nP, I.S_max, I.N_max, I.nf, I.ne, L.ff_col, L.ff_nsl, L.fp_col, L.pf_col, L.pf_nsl,
                   I.pos, I.face_at, I.lorder, I.nlow, I.fpos, I.fepos, I.torder, I.tpos, I.tside};
}

template <typename T>
IluData<T> data_of(const IluLevel& I);
template <>
IluData<double> data_of<double>(const IluLevel& I) {
    return IluData<double>{I.lff, I.lfp, I.lpf, I.lpp, I.uf, I.ue};
}
template <>
IluData<float> data_of<float>(const IluLevel& I) {
    return IluData<float>{I.lff32, I.lfp32, I.lpf32, I.lpp32, I.uf32, I.ue32};
}

template <typename Tv>
hho_status upload_vec(hho_ctx* ctx, Tv** dst, const std::vector<Tv>& v) {
    HHO_TRY(dalloc(ctx, dst, std::max<size_t>(v.size(), 1)));
    if (!v.empty()) HHO_CUDA(cudaMemcpy(*dst, v.data(), v.size() * sizeof(Tv), cudaMemcpyHostToDevice));
    return HHO_OK;
}

}  // namespace

void ilu_free(hho_ctx* ctx) {
    for (IluLevel* I : ctx->ilu) {
        if (!I) continue;
        void* ps[] = {I->pos, I->face_at, I->lorder, I->nlow, I->fpos, I->fepos, I->torder, I->tpos, I->tside,
                      I->lff, I->lfp, I->lpf, I->lpp, I->uf, I->ue, I->lff32, I->lfp32, I->lpf32, I->lpp32,
                      I->uf32, I->ue32};
        for (void* p : ps) dfree(p);
        delete I;
    }
    ctx->ilu.clear();
}

// Factor level l (FP64; FP32 copies when fp32).
hho_status ilu_setup(hho_ctx* ctx, int l, bool fp32) {
    const LevelMat& L = ctx->levels[l];
    const Disc& D = ctx->disc;
    const Topo& Tp = ctx->topo;
    if (L.b > MB || L.nP > MB) {
        ctx->err = "ILU smoother: blocks larger than 32 unknowns are not supported";
        return HHO_ERR_UNSUPPORTED;
    }
    if ((int)ctx->ilu.size() <= l) ctx->ilu.resize(l + 1, nullptr);
    IluLevel* I = new IluLevel();
    ctx->ilu[l] = I;
    const int64_t nf = L.nf, ne = L.ne;
    I->b = L.b;
    I->nP = L.nP;
    I->S_max = L.S_max;
    I->N_max = L.N_max;
    I->nf = nf;
    I->ne = ne;
    // greedy colouring of the faces in index order (adjacent = sharing an element)
    std::vector<int32_t> col(nf, -1);
    int ncol = 0;
    for (int64_t F = 0; F < nf; ++F) {
        std::vector<char> used(64, 0);
        for (int e = 0; e < 2; ++e) {
            const int T = D.h_fe[2 * F + e];
            if (T < 0) continue;
            for (int g = D.h_ef_ptr[T]; g < D.h_ef_ptr[T + 1]; ++g) {
                const int G = D.h_ef[g];
                if (G != F && col[G] >= 0) {
                    if (col[G] >= (int)used.size()) used.resize(col[G] + 1, 0);
                    used[col[G]] = 1;
                }
            }
        }
        int c = 0;
        while (c < (int)used.size() && used[c]) ++c;
        col[F] = c;
        ncol = std::max(ncol, c + 1);
    }
    std::vector<int32_t> face_at(nf), pos(nf);
    std::iota(face_at.begin(), face_at.end(), 0);
    std::stable_sort(face_at.begin(), face_at.end(), [&](int32_t a, int32_t b) { return col[a] < col[b]; });
    for (int64_t P = 0; P < nf; ++P) pos[face_at[P]] = (int32_t)P;
    I->ncol = ncol;
    I->coff.assign(ncol + 1, 0);
    for (int64_t F = 0; F < nf; ++F) I->coff[col[F] + 1]++;
    for (int c = 0; c < ncol; ++c) I->coff[c + 1] += I->coff[c];
    // pattern lookups (rank of a face = its position; elements rank after all faces)
    const int S = L.S_max, NM = L.N_max;
    const std::vector<int32_t>& fc = Tp.h_ff_col;
    const std::vector<int32_t>& fn = Tp.h_ff_nsl;
    const std::vector<int32_t>& fpc = Tp.h_fp_col;
    const std::vector<int32_t>& pfc = Tp.h_pf_col;
    const std::vector<int32_t>& pfn = Tp.h_pf_nsl;
    std::vector<int32_t> lorder((size_t)nf * S, -1), nlow(nf, 0);
    std::vector<int8_t> fpos((size_t)nf * S * S, -1), fepos((size_t)nf * S * 2, -1);
    auto slot_of = [&](int64_t G, int64_t H) -> int {
        for (int u = 0; u < fn[G]; ++u)
            if (fc[(size_t)u * nf + G] == H) return u;
        return -1;
    };
    auto side_of = [&](int64_t G, int64_t T) -> int {
        for (int p = 0; p < 2; ++p)
            if (fpc[(size_t)p * nf + G] == T) return p;
        return -1;
    };
    for (int64_t F = 0; F < nf; ++F) {
        std::vector<int> low;
        for (int s = 1; s < fn[F]; ++s)
            if (pos[fc[(size_t)s * nf + F]] < pos[F]) low.push_back(s);
        std::sort(low.begin(), low.end(), [&](int a, int b2) {
            return pos[fc[(size_t)a * nf + F]] < pos[fc[(size_t)b2 * nf + F]];
        });
        nlow[F] = (int32_t)low.size();
        for (size_t i = 0; i < low.size(); ++i) lorder[(size_t)F * S + i] = low[i];
        for (int s : low) {
            const int64_t G = fc[(size_t)s * nf + F];
            for (int t = 0; t < fn[F]; ++t) {
                const int64_t H = fc[(size_t)t * nf + F];
                if (pos[H] > pos[G]) fpos[((size_t)F * S + s) * S + t] = (int8_t)slot_of(G, H);
            }
            for (int p = 0; p < 2; ++p) {
                const int64_t T = fpc[(size_t)p * nf + F];
                if (T >= 0) fepos[((size_t)F * S + s) * 2 + p] = (int8_t)side_of(G, T);
            }
        }
    }
    std::vector<int8_t> torder((size_t)ne * NM, -1), tpos((size_t)ne * NM * NM, -1), tside((size_t)ne * NM, -1);
    for (int64_t T = 0; T < ne; ++T) {
        const int N = pfn[T];
        std::vector<int> fs(N);
        std::iota(fs.begin(), fs.end(), 0);
        std::sort(fs.begin(), fs.end(), [&](int a, int b2) {
            return pos[pfc[(size_t)a * ne + T]] < pos[pfc[(size_t)b2 * ne + T]];
        });
        for (int i = 0; i < N; ++i) torder[(size_t)T * NM + i] = (int8_t)fs[i];
        for (int f = 0; f < N; ++f) {
            const int64_t F = pfc[(size_t)f * ne + T];
            tside[(size_t)T * NM + f] = (int8_t)side_of(F, T);
            for (int g = 0; g < N; ++g)
                if (g != f) tpos[((size_t)T * NM + f) * NM + g] = (int8_t)slot_of(F, pfc[(size_t)g * ne + T]);
        }
    }
    HHO_TRY(upload_vec(ctx, &I->pos, pos));
    HHO_TRY(upload_vec(ctx, &I->face_at, face_at));
    HHO_TRY(upload_vec(ctx, &I->lorder, lorder));
    HHO_TRY(upload_vec(ctx, &I->nlow, nlow));
    HHO_TRY(upload_vec(ctx, &I->fpos, fpos));
    HHO_TRY(upload_vec(ctx, &I->fepos, fepos));
    HHO_TRY(upload_vec(ctx, &I->torder, torder));
    HHO_TRY(upload_vec(ctx, &I->tpos, tpos));
    HHO_TRY(upload_vec(ctx, &I->tside, tside));
    // factor storage: copies of the level blocks, face rows in colour order
    const int64_t nff = (int64_t)S * L.b * L.b, nfp = (int64_t)2 * L.nP * L.b;
    const int64_t npf = (int64_t)NM * L.b * L.nP * ne, npp = (int64_t)L.nP * L.nP * ne;
    HHO_TRY(dalloc(ctx, &I->lff, (size_t)(nff * nf)));
    HHO_TRY(dalloc(ctx, &I->lfp, (size_t)(nfp * nf)));
    HHO_TRY(dalloc(ctx, &I->lpf, (size_t)npf));
    HHO_TRY(dalloc(ctx, &I->lpp, (size_t)npp));
    HHO_TRY(dalloc(ctx, &I->uf, (size_t)L.b * L.b * nf));
    HHO_TRY(dalloc(ctx, &I->ue, (size_t)L.nP * L.nP * ne));
    k_perm_faces<<<g1(nff * nf), 256, 0, ctx->stream>>>(nff, nf, I->pos, L.ff, I->lff);
    k_perm_faces<<<g1(nfp * nf), 256, 0, ctx->stream>>>(nfp, nf, I->pos, L.fp, I->lfp);
    k_copy_d<<<g1(npf), 256, 0, ctx->stream>>>(npf, L.pf, I->lpf);
    k_copy_d<<<g1(npp), 256, 0, ctx->stream>>>(npp, L.pp, I->lpp);
    HHO_CUDA(cudaGetLastError());
    HHO_CUDA(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream));
    const IluView v = view_of(ctx, L, *I);
    for (int c = 0; c < ncol; ++c) {
        const int n = I->coff[c + 1] - I->coff[c];
        if (n == 0) continue;
        k_ilu_face_rows<<<std::min(n, sm_count() * 16), IB, 0, ctx->stream>>>(v, I->coff[c], I->coff[c + 1], I->lff, I->lfp,
                                                                       I->uf, ctx->d_flag);
    }
    k_ilu_elem_rows<<<(int)std::min<int64_t>(ne, (int64_t)sm_count() * 16), IB, 0, ctx->stream>>>(v, I->lff, I->lfp, I->lpf, I->lpp,
                                                                                 I->uf, I->ue, ctx->d_flag);
    HHO_CUDA(cudaGetLastError());
    int flag = 0;
    HHO_CUDA(cudaMemcpyAsync(&flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    HHO_CUDA(cudaStreamSynchronize(ctx->stream));
    if (flag) {
        ctx->err = "ILU smoother: zero pivot in the block factorisation";
        return HHO_ERR_SINGULAR;
    }
    if (fp32) {
        struct Pair {
            const double* s;
            float** d;
            int64_t n;
        } prs[] = {{I->lff, &I->lff32, nff * nf}, {I->lfp, &I->lfp32, nfp * nf}, {I->lpf, &I->lpf32, npf},
                   {I->lpp, &I->lpp32, npp},       {I->uf, &I->uf32, (int64_t)L.b * L.b * nf},
                   {I->ue, &I->ue32, (int64_t)L.nP * L.nP * ne}};
        for (auto& q : prs) {
            HHO_TRY(dalloc(ctx, q.d, (size_t)q.n));
            k_to_f32<<<g1(q.n), 256, 0, ctx->stream>>>(q.n, q.s, *q.d);
        }
        HHO_CUDA(cudaGetLastError());
        HHO_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    return HHO_OK;
}

// z = (L U)^{-1} v on level l; tmp: element-block scratch (ne * nP of T)
template <int B, typename T>
static void ilu_apply_B(hho_ctx* ctx, int l, const T* v, T* z, T* tmp) {
    const LevelMat& L = ctx->levels[l];
    const IluLevel& I = *ctx->ilu[l];
    const IluView vw = view_of(ctx, L, I);
    const IluData<T> d = data_of<T>(I);
    for (int c = 0; c < I.ncol; ++c) {
        const int n = I.coff[c + 1] - I.coff[c];
        if (n == 0) continue;
        k_ilu_fwd_face<B, T><<<(n + 127) / 128, 128, 0, ctx->stream>>>(vw, d, I.coff[c], I.coff[c + 1], I.pos, v, z);
    }
    const int64_t ner = I.ne * I.nP;
    k_ilu_fwd_elem<B, T><<<g1(ner), 256, 0, ctx->stream>>>(vw, d, v, z);
    k_ilu_bwd_elem<B, T><<<g1(ner), 256, 0, ctx->stream>>>(vw, d, z, tmp);
    k_ilu_elem_store<<<g1(ner), 256, 0, ctx->stream>>>(ner, I.nf * B, tmp, z);
    for (int c = I.ncol - 1; c >= 0; --c) {
        const int n = I.coff[c + 1] - I.coff[c];
        if (n == 0) continue;
        k_ilu_bwd_face<B, T><<<(n + 127) / 128, 128, 0, ctx->stream>>>(vw, d, I.coff[c], I.coff[c + 1], I.pos, z);
    }
    ctx->launches += 2 * I.ncol + 3;
}

template <typename T>
hho_status ilu_apply(hho_ctx* ctx, int l, const T* v, T* z, T* tmp) {
    if ((int)ctx->ilu.size() <= l || !ctx->ilu[l]) {
        ctx->err = "ILU smoother: level not factored";
        return HHO_ERR_STATE;
    }
    switch (ctx->levels[l].b) {
        case 2: ilu_apply_B<2, T>(ctx, l, v, z, tmp); break;
        case 3: ilu_apply_B<3, T>(ctx, l, v, z, tmp); break;
        case 4: ilu_apply_B<4, T>(ctx, l, v, z, tmp); break;
        case 6: ilu_apply_B<6, T>(ctx, l, v, z, tmp); break;
        case 8: ilu_apply_B<8, T>(ctx, l, v, z, tmp); break;
        case 9: ilu_apply_B<9, T>(ctx, l, v, z, tmp); break;
        case 10: ilu_apply_B<10, T>(ctx, l, v, z, tmp); break;
        case 12: ilu_apply_B<12, T>(ctx, l, v, z, tmp); break;
        case 18: ilu_apply_B<18, T>(ctx, l, v, z, tmp); break;
        default:
            ctx->err = "ILU smoother: face block size without a kernel";
            return HHO_ERR_UNSUPPORTED;
    }
    HHO_CUDA(cudaGetLastError());
    return HHO_OK;
}
template hho_status ilu_apply<double>(hho_ctx*, int, const double*, double*, double*);
template hho_status ilu_apply<float>(hho_ctx*, int, const float*, float*, float*);

}  // namespace hho
