// Many independent problems in one context: the mesh is a disjoint union of
// problems (contiguous face and element ranges per problem), so every level
// operator is block diagonal and one launch of each V-cycle kernel works on all
// problems at once.  What must stay per problem is the outer Krylov method:
// hho_solve_batch runs one FP64 FGMRES (Sec. 3.3) per problem, in lockstep,
// with segmented reductions -- every dot product is split by problem -- and a
// per-problem convergence test; a problem that has converged is frozen (its
// Arnoldi recurrence stops, its iterate is kept) while the others go on.
//
// The V-cycle preconditioner is the union's: levels, transfers and coarse
// solve are block diagonal and act on each problem exactly as alone, while the
// smoother's two GMRES iterations take their Krylov coefficients from the
// whole batch.  That makes the preconditioner of one problem depend on the
// others' residuals, which flexible GMRES admits (its minimal-residual
// property holds for any preconditioned vectors).
//
// Segmented kernels work on tiles: a tile is a contiguous run of at most
// tile_rows unknowns of the level-0 vector that belong to one problem (face
// unknowns and element unknowns of a problem form two runs).  One block per
// tile writes partial sums; a second kernel (one block of 32 threads per
// problem) adds its tiles' partials in index order and runs the GMRES scalar
// recurrence of that problem, so results are reproducible run to run.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"
#include "krylov.cuh"

namespace hho {

namespace {

constexpr int BT = 256;  // threads per block of the segmented kernels
constexpr int NVB = 8;   // dot products per segmented kernel

struct TileView {
    int nt;
    const int32_t* prob;
    const int64_t* r0;
    const int32_t* len;
};

// w = w + sgn sum_{q<ncomb} c_{p,q} V_q on the tile (c_p = fsc_p[coef_off..]),
// then partial sums of Vd_q . w (q < nv) and of w . w (self) per tile.
__global__ void __launch_bounds__(BT) k_seg_upd_dot(TileView T, double* __restrict__ w, const double* __restrict__ V,
                                                    int64_t ld, int ncomb, const double* __restrict__ fsc, int64_t GT,
                                                    int coef_off, double sgn, const double* __restrict__ Vd, int nv,
                                                    int self, double* __restrict__ partial) {
    __shared__ double s_c[MMAX];
    __shared__ double sm[BT / 32][NVB + 1];
    const int p = T.prob[blockIdx.x];
    const int64_t r0 = T.r0[blockIdx.x], r1 = r0 + T.len[blockIdx.x];
    for (int q = threadIdx.x; q < ncomb; q += blockDim.x) s_c[q] = sgn * fsc[p * GT + coef_off + q];
    __syncthreads();
    double acc[NVB + 1];
#pragma unroll
    for (int v = 0; v <= NVB; ++v) acc[v] = 0.0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        double s = w[i];
        for (int q = 0; q < ncomb; ++q) s += s_c[q] * V[q * ld + i];
        if (ncomb > 0) w[i] = s;
#pragma unroll
        for (int q = 0; q < NVB; ++q)
            if (q < nv) acc[q] += Vd[q * ld + i] * s;
        if (self) acc[NVB] += s * s;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v <= NVB; ++v) {
        if (v < nv || (self && v == NVB)) {
            double a = acc[v];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0) sm[wid][v] = a;
        }
    }
    __syncthreads();
    if ((int)threadIdx.x < nv + self) {
        const int src = ((int)threadIdx.x < nv) ? (int)threadIdx.x : NVB;
        double s = 0.0;
        for (int k = 0; k < BT / 32; ++k) s += sm[k][src];
        partial[(int64_t)threadIdx.x * T.nt + blockIdx.x] = s;
    }
}

// Per problem (block of 32): out_p[v] = sum over the problem's tiles of the
// partials, in tile order; then the scalar recurrence of the problem's GMRES.
// stat[2p] = beta (START) or the residual estimate (COLUMN), stat[2p+1] = the
// breakdown / frozen flag.
__global__ void __launch_bounds__(32) k_seg_finish(const int32_t* __restrict__ prob_t0,
                                                   const double* __restrict__ partial, int nt, int nout, int self,
                                                   double* __restrict__ fsc, int64_t GT, int out_off, int hook, GS G,
                                                   int j, double* __restrict__ stat) {
    __shared__ double s_fresh;
    const int p = blockIdx.x, lane = threadIdx.x;
    const int t0 = prob_t0[p], t1 = prob_t0[p + 1];
    double* sc = fsc + p * GT;
    for (int v = 0; v < nout; ++v) {
        double s = 0.0;
        for (int t = t0 + lane; t < t1; t += 32) s += partial[(int64_t)v * nt + t];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            sc[out_off + v] = s;
            if (v == (self ? nout - 1 : 0)) s_fresh = s;
        }
    }
    __syncthreads();
    run_hook<double>(hook, sc, G, j, s_fresh);
    if (threadIdx.x == 0 && stat) {
        stat[2 * p] = (hook == HOOK_START) ? sc[1] : sc[3];
        stat[2 * p + 1] = sc[4];
    }
}

// v = w / beta_p on the tile (0 when beta_p = 0)
__global__ void __launch_bounds__(BT) k_seg_scale(TileView T, const double* __restrict__ w, double* __restrict__ v,
                                                  const double* __restrict__ fsc, int64_t GT) {
    const int p = T.prob[blockIdx.x];
    const double inv = block_inverse<double>(fsc + p * GT + 5);
    const int64_t r0 = T.r0[blockIdx.x], r1 = r0 + T.len[blockIdx.x];
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) v[i] = w[i] * inv;
}

// x += Z y_p on the tile, y_p = R_p^{-1} g_p of the problem's GMRES (staged
// in shared memory, back-substituted by one thread).  Dynamic shared memory:
// ((m+1) m + m) doubles.
__global__ void __launch_bounds__(BT) k_seg_update_x(TileView T, double* __restrict__ x, const double* __restrict__ Z,
                                                     int64_t ld, const double* __restrict__ fsc, int64_t GT, GS G) {
    extern __shared__ double s_dyn[];
    const int p = T.prob[blockIdx.x];
    const double* sc = fsc + p * GT;
    const int ld2 = G.m + 1;
    double* Hs = s_dyn;
    double* y = s_dyn + ld2 * G.m;
    const int me = (sc[1] == 0.0) ? 0 : (int)sc[2];
    for (int i = threadIdx.x; i < ld2 * me; i += blockDim.x) Hs[i] = sc[G.H + i];
    for (int i = threadIdx.x; i < me; i += blockDim.x) y[i] = sc[G.g + i];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = me - 1; i >= 0; --i) {
            double s = y[i];
            for (int l = i + 1; l < me; ++l) s -= Hs[l * ld2 + i] * y[l];
            const double dd = Hs[i * ld2 + i];
            y[i] = (dd == 0.0) ? 0.0 : s / dd;
        }
    }
    __syncthreads();
    const int64_t r0 = T.r0[blockIdx.x], r1 = r0 + T.len[blockIdx.x];
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        double s = x[i];
        for (int q = 0; q < me; ++q) s += y[q] * Z[q * ld + i];
        x[i] = s;
    }
}

// fsc_p[4] = 1 (breakdown flag: the problem's recurrence stops) for the listed problems
__global__ void k_freeze(const int32_t* __restrict__ list, int n, double* __restrict__ fsc, int64_t GT) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double* sc = fsc + list[i] * GT;
        sc[4] = 1.0;
        sc[5] = 0.0;
    }
}

__global__ void k_copy(int64_t n, const double* __restrict__ a, double* __restrict__ b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = a[i];
}

__global__ void k_zero(int64_t n, double* __restrict__ b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = 0.0;
}

int grid1d(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 32)); }

}  // namespace

// Device state of the graph-captured batch solve (one FGMRES per problem, all
// control on the device).
struct BGState {
    int it;      // FGMRES iterations so far
    int cycles;  // restart cycles so far
};

struct BatchWork {
    int restart = 0, tile_rows = 0;
    int nt = 0;
    int32_t *tile_prob = nullptr, *tile_len = nullptr, *prob_t0 = nullptr, *frz = nullptr;
    int64_t* tile_r0 = nullptr;
    double *V = nullptr, *Z = nullptr, *w = nullptr, *b = nullptr, *fsc = nullptr, *partial = nullptr,
           *stat = nullptr;
    double* h_stat = nullptr;  // pinned
    int32_t* h_frz = nullptr;  // pinned
    // graph-captured solve: the captured graph, what it was captured for, and its device state
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    double* g_x = nullptr;
    double g_rtol = 0.0;
    int g_maxit = -1, g_restart = 0;
    int64_t g_launch_fixed = 0, g_launch_cycle = 0, g_launch_iter = 0;  // kernels per part of the graph
    double *d_bnorm = nullptr, *d_relres = nullptr;
    int32_t *d_conv = nullptr, *d_convit = nullptr, *d_its = nullptr;
    BGState* d_state = nullptr;
    cudaGraphConditionalHandle* d_handles = nullptr;  // the restart cycle's IF nodes
    cudaStream_t s_body = nullptr;                    // streams that capture the nested bodies
    int gP = 0;
};

void batch_graph_free(hho_ctx* ctx) {
    BatchWork* B = ctx->batch;
    if (!B) return;
    if (B->gexec) cudaGraphExecDestroy(B->gexec);
    if (B->graph) cudaGraphDestroy(B->graph);
    B->gexec = nullptr;
    B->graph = nullptr;
    B->g_x = nullptr;
    B->g_maxit = -1;
}

void batch_free(hho_ctx* ctx) {
    BatchWork* B = ctx->batch;
    if (!B) return;
    batch_graph_free(ctx);
    if (B->s_body) cudaStreamDestroy(B->s_body);
    void* ps[] = {B->tile_prob, B->tile_len, B->prob_t0, B->frz, B->tile_r0, B->V, B->Z, B->w, B->b, B->fsc,
                  B->partial, B->stat, B->d_bnorm, B->d_relres, B->d_conv, B->d_convit, B->d_its, B->d_state,
                  B->d_handles};
    for (void* p : ps) dfree(p);
    if (B->h_stat) cudaFreeHost(B->h_stat);
    if (B->h_frz) cudaFreeHost(B->h_frz);
    delete B;
    ctx->batch = nullptr;
}

hho_status batch_set(hho_ctx* ctx, int P, const int64_t* face_off, const int64_t* elem_off) {
    const Disc& D = ctx->disc;
    if (P < 1 || P > 65535) {
        ctx->err = "hho_set_batch: n_prob must be in 1..65535";
        return HHO_ERR_ARG;
    }
    if (face_off[0] != 0 || elem_off[0] != 0 || face_off[P] != D.nf || elem_off[P] != D.ne) {
        ctx->err = "hho_set_batch: offsets must start at 0 and end at the face / element counts";
        return HHO_ERR_ARG;
    }
    std::vector<int32_t> eprob(D.ne);
    for (int p = 0; p < P; ++p) {
        if (face_off[p + 1] <= face_off[p] || elem_off[p + 1] <= elem_off[p]) {
            ctx->err = "hho_set_batch: every problem needs at least one face and one element";
            return HHO_ERR_ARG;
        }
        for (int64_t T = elem_off[p]; T < elem_off[p + 1]; ++T) eprob[T] = p;
    }
    // the problems must be uncoupled: each face's elements, and each element's faces, in one problem
    for (int p = 0; p < P; ++p)
        for (int64_t F = face_off[p]; F < face_off[p + 1]; ++F)
            for (int s = 0; s < 2; ++s) {
                const int T = D.h_fe[2 * F + s];
                if (T >= 0 && eprob[T] != p) {
                    ctx->err = "hho_set_batch: face " + std::to_string(F) + " of problem " + std::to_string(p) +
                               " touches an element of another problem";
                    return HHO_ERR_MESH;
                }
            }
    Problems& pr = ctx->probs;
    pr.P = P;
    pr.face_off.assign(face_off, face_off + P + 1);
    pr.elem_off.assign(elem_off, elem_off + P + 1);
    pr.elem_prob = eprob;
    pr.declared = true;
    batch_free(ctx);
    if (ctx->have_pmg) {  // the coarse solver and kernel vectors depend on the partition
        ctx->err = "hho_set_batch: declare the batch before pmg_setup";
        ctx->have_pmg = false;
        return HHO_ERR_STATE;
    }
    return HHO_OK;
}

// tiles of the level-0 vector: per problem, its face run then its element run
static hho_status build_tiles(hho_ctx* ctx, BatchWork* B, int tile_rows) {
    const Problems& pr = ctx->probs;
    const LevelMat& L = ctx->levels[0];
    std::vector<int32_t> tp, tl, t0(pr.P + 1, 0);
    std::vector<int64_t> tr;
    for (int p = 0; p < pr.P; ++p) {
        t0[p] = (int32_t)tp.size();
        const int64_t runs[2][2] = {{pr.face_off[p] * L.b, pr.face_off[p + 1] * L.b},
                                    {L.nf * L.b + pr.elem_off[p] * L.nP, L.nf * L.b + pr.elem_off[p + 1] * L.nP}};
        for (auto& run : runs)
            for (int64_t r = run[0]; r < run[1]; r += tile_rows) {
                tp.push_back(p);
                tr.push_back(r);
                tl.push_back((int32_t)std::min<int64_t>(tile_rows, run[1] - r));
            }
    }
    t0[pr.P] = (int32_t)tp.size();
    B->tile_rows = 0;  // set again once every tile buffer below exists
    dfree(B->tile_prob);
    dfree(B->tile_len);
    dfree(B->tile_r0);
    dfree(B->prob_t0);
    dfree(B->partial);
    B->tile_prob = B->tile_len = B->prob_t0 = nullptr;
    B->tile_r0 = nullptr;
    B->partial = nullptr;
    B->nt = (int)tp.size();
    HHO_TRY(dalloc(ctx, &B->tile_prob, tp.size()));
    HHO_TRY(dalloc(ctx, &B->tile_len, tl.size()));
    HHO_TRY(dalloc(ctx, &B->tile_r0, tr.size()));
    HHO_TRY(dalloc(ctx, &B->prob_t0, t0.size()));
    HHO_TRY(dalloc(ctx, &B->partial, (size_t)(NVB + 1) * B->nt));
    HHO_CUDA(cudaMemcpy(B->tile_prob, tp.data(), tp.size() * 4, cudaMemcpyHostToDevice));
    HHO_CUDA(cudaMemcpy(B->tile_len, tl.data(), tl.size() * 4, cudaMemcpyHostToDevice));
    HHO_CUDA(cudaMemcpy(B->tile_r0, tr.data(), tr.size() * 8, cudaMemcpyHostToDevice));
    HHO_CUDA(cudaMemcpy(B->prob_t0, t0.data(), t0.size() * 4, cudaMemcpyHostToDevice));
    B->tile_rows = tile_rows;
    return HHO_OK;
}

static hho_status batch_work(hho_ctx* ctx, int restart) {
    BatchWork* B = ctx->batch;
    const int64_t n = ctx->levels[0].n;
    const int P = ctx->probs.P;
    if (B && B->restart == restart && B->tile_rows == ctx->tile_rows) return HHO_OK;
    if (!B) {
        B = new BatchWork();
        ctx->batch = B;
    }
    HHO_TRY(build_tiles(ctx, B, ctx->tile_rows));
    if (B->restart != restart) {
        B->restart = 0;  // until every buffer below exists (a failed allocation must not leave stale ones)
        void* ps[] = {B->V, B->Z, B->w, B->b, B->fsc, B->stat, B->frz};
        for (void* p : ps) dfree(p);
        B->V = B->Z = B->w = B->b = B->fsc = B->stat = nullptr;
        B->frz = nullptr;
        const int64_t GT = (gs_layout(restart).total + 7) / 8 * 8;
        HHO_TRY(dalloc(ctx, &B->V, (size_t)(restart + 1) * n));
        HHO_TRY(dalloc(ctx, &B->Z, (size_t)restart * n));
        HHO_TRY(dalloc(ctx, &B->w, (size_t)n));
        HHO_TRY(dalloc(ctx, &B->b, (size_t)n));
        HHO_TRY(dalloc(ctx, &B->fsc, (size_t)P * GT));
        HHO_CUDA(cudaMemset(B->fsc, 0, (size_t)P * GT * sizeof(double)));
        HHO_TRY(dalloc(ctx, &B->stat, (size_t)2 * P));
        HHO_TRY(dalloc(ctx, &B->frz, (size_t)P));
        if (!B->h_stat) HHO_CUDA(cudaMallocHost(&B->h_stat, (size_t)2 * P * sizeof(double)));
        if (!B->h_frz) HHO_CUDA(cudaMallocHost(&B->h_frz, (size_t)P * sizeof(int32_t)));
        B->restart = restart;
    }
    return HHO_OK;
}

namespace {

struct Seg {
    hho_ctx* ctx;
    BatchWork* B;
    TileView tv;
    int64_t n, GT;
    GS G;
    int P;

    // w += sgn c_p V (ncomb columns), then dots of w with Vd (nv columns, in
    // chunks) and optionally with itself, reduced into fsc_p[out_off + ...]
    hho_status upd_dot(double* w, const double* Vu, int ncomb, int coef_off, double sgn, const double* Vd, int nv,
                       int self, int out_off, int hook, int j, bool want_stat) {
        int done = 0;
        bool first = true;
        do {
            const int cnt = std::min(NVB, nv - done);
            const int me = (done + cnt >= nv) ? self : 0;
            k_seg_upd_dot<<<B->nt, BT, 0, ctx->stream>>>(tv, w, Vu, n, first ? ncomb : 0, B->fsc, GT, coef_off, sgn,
                                                        Vd ? Vd + (int64_t)done * n : nullptr, cnt, me, B->partial);
            const bool last = done + cnt >= nv;
            k_seg_finish<<<P, 32, 0, ctx->stream>>>(B->prob_t0, B->partial, B->nt, cnt + me, me, B->fsc, GT,
                                                    out_off + done, last ? hook : HOOK_NONE, G, j,
                                                    (last && want_stat) ? B->stat : nullptr);
            ctx->launches += 2;
            done += cnt;
            first = false;
        } while (done < nv);
        HHO_CUDA(cudaGetLastError());
        return HHO_OK;
    }
    hho_status read_stat() {
        HHO_CUDA(cudaMemcpyAsync(B->h_stat, B->stat, 2 * P * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        HHO_CUDA(cudaStreamSynchronize(ctx->stream));
        return HHO_OK;
    }
    hho_status freeze(const std::vector<int32_t>& list) {
        if (list.empty()) return HHO_OK;
        for (size_t i = 0; i < list.size(); ++i) B->h_frz[i] = list[i];
        HHO_CUDA(cudaMemcpyAsync(B->frz, B->h_frz, list.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                                 ctx->stream));
        k_freeze<<<1, 256, 0, ctx->stream>>>(B->frz, (int)list.size(), B->fsc, GT);
        ++ctx->launches;
        HHO_CUDA(cudaGetLastError());
        return HHO_OK;
    }
};

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// Graph-captured batch solve.  The whole solve (every restart cycle and every
// Arnoldi step of every problem's FGMRES) is one CUDA graph: a WHILE node runs
// the restart cycles and, inside it, one IF node per Arnoldi step skips the
// rest of a cycle once every problem has met its tolerance.  The tests that
// the host-driven loop does on copied scalars run in the single-block kernels
// below, which set the graph's conditions; nothing is read on the host until
// the graph has finished.
// ---------------------------------------------------------------------------
constexpr int BG_T = 256;

__device__ __forceinline__ void bg_freeze(double* fsc, int64_t GT, int p) {
    fsc[p * GT + 4] = 1.0;
    fsc[p * GT + 5] = 0.0;
}

// after ||b_p|| (START statistics in stat): tolerances and the first condition
__global__ void __launch_bounds__(BG_T) k_bg_init(int P, const double* __restrict__ stat, double* __restrict__ bnorm,
                                                  int32_t* __restrict__ conv, int32_t* __restrict__ convit,
                                                  BGState* st, int maxit, cudaGraphConditionalHandle h_outer) {
    int open = 0;
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        const double bn = stat[2 * p];
        bnorm[p] = bn;
        const int c = bn > 0.0 ? 0 : 1;
        conv[p] = c;
        convit[p] = c ? 0 : -1;
        open |= !c;
    }
    open = __syncthreads_or(open);
    if (threadIdx.x == 0) {
        st->it = 0;
        st->cycles = 0;
        cudaGraphSetConditional(h_outer, (open && maxit > 0) ? 1u : 0u);
    }
}

// start of a restart cycle: freeze the problems that have converged, open the
// first Arnoldi step and close the others
__global__ void __launch_bounds__(BG_T) k_bg_cycle_start(int P, const int32_t* __restrict__ conv,
                                                         double* __restrict__ fsc, int64_t GT,
                                                         const cudaGraphConditionalHandle* __restrict__ hs, int m) {
    for (int p = threadIdx.x; p < P; p += blockDim.x)
        if (conv[p]) bg_freeze(fsc, GT, p);
    for (int j = threadIdx.x; j < m; j += blockDim.x) cudaGraphSetConditional(hs[j], j == 0 ? 1u : 0u);
}

// after Arnoldi step j: problems whose residual estimate meets the tolerance
// are frozen for the rest of the cycle; step j + 1 runs unless every problem
// is frozen or broken down, maxit is reached or the cycle is full
__global__ void __launch_bounds__(BG_T) k_bg_iter(int P, const double* __restrict__ stat,
                                                  const double* __restrict__ bnorm, const int32_t* __restrict__ conv,
                                                  int32_t* __restrict__ convit, BGState* st, double rtol, int maxit,
                                                  int j, int m, double* __restrict__ fsc, int64_t GT,
                                                  const cudaGraphConditionalHandle* __restrict__ hs) {
    __shared__ int s_it;
    if (threadIdx.x == 0) s_it = ++st->it;
    __syncthreads();
    const int it = s_it;
    int open = 0;
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        if (conv[p]) continue;
        const double est = stat[2 * p];
        const bool brk = stat[2 * p + 1] != 0.0;
        if (est <= rtol * bnorm[p]) {
            if (convit[p] < 0) convit[p] = it;
            bg_freeze(fsc, GT, p);
        } else if (!brk) {
            open = 1;
        }
    }
    open = __syncthreads_or(open);
    if (threadIdx.x == 0 && j + 1 < m) cudaGraphSetConditional(hs[j + 1], (open && it < maxit) ? 1u : 0u);
}

// end of a cycle (START statistics of the true residuals in stat): converged
// problems, and whether another cycle runs
__global__ void __launch_bounds__(BG_T) k_bg_cycle_end(int P, const double* __restrict__ stat,
                                                       const double* __restrict__ bnorm, int32_t* __restrict__ conv,
                                                       int32_t* __restrict__ convit, BGState* st, double rtol,
                                                       int maxit, cudaGraphConditionalHandle h_outer) {
    const int it = st->it;
    int open = 0;
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        const double beta = stat[2 * p];
        if (beta <= rtol * bnorm[p] || !(bnorm[p] > 0.0)) {
            if (!conv[p] && convit[p] < 0) convit[p] = it;
            conv[p] = 1;
        } else {
            conv[p] = 0;  // the estimate was optimistic: iterate again
            convit[p] = -1;
            open = 1;
        }
    }
    open = __syncthreads_or(open);
    if (threadIdx.x == 0) {
        ++st->cycles;
        cudaGraphSetConditional(h_outer, (open && it < maxit) ? 1u : 0u);
    }
}

// per-problem results from the final START statistics
__global__ void __launch_bounds__(BG_T) k_bg_final(int P, const double* __restrict__ stat,
                                                   const double* __restrict__ bnorm,
                                                   const int32_t* __restrict__ convit, const BGState* st,
                                                   int32_t* __restrict__ its, double* __restrict__ relres) {
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        relres[p] = bnorm[p] > 0.0 ? stat[2 * p] / bnorm[p] : 0.0;
        its[p] = convit[p] >= 0 ? convit[p] : st->it;
    }
}

// a conditional node appended to the graph the stream is capturing; returns its body
hho_status add_conditional(hho_ctx* ctx, cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType ty,
                           cudaGraph_t* body) {
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    cudaGraph_t cg = nullptr;
    HHO_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, &deps, nullptr, &nd));
    if (cs != cudaStreamCaptureStatusActive || !cg) {
        ctx->err = "hho_solve_batch: the solve graph's capture was invalidated";
        return HHO_ERR_CUDA;
    }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = ty;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    HHO_CUDA(cudaGraphAddNode(&node, cg, deps, nullptr, nd, &cp));
    *body = cp.conditional.phGraph_out[0];
    HHO_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return HHO_OK;
}

}  // namespace

// Capture the graph of a batch solve (x, restart, rtol and maxit are baked in).
// The library's kernels are launched on ctx->stream, which is pointed at the
// stream capturing each part in turn; the V-cycle is captured by its direct
// launches.
static hho_status batch_graph_build(hho_ctx* ctx, BatchWork* B, double rtol, int maxit, int restart, double* x) {
    const LevelMat& L0 = ctx->levels[0];
    const int P = ctx->probs.P;
    const int64_t n = L0.n;
    Seg S{ctx, B, TileView{B->nt, B->tile_prob, B->tile_r0, B->tile_len}, n, (gs_layout(restart).total + 7) / 8 * 8,
          gs_layout(restart), P};
    const GS& G = S.G;
    if (B->gP != P || !B->d_bnorm) {
        void* ps[] = {B->d_bnorm, B->d_relres, B->d_conv, B->d_convit, B->d_its, B->d_state, B->d_handles};
        for (void* q : ps) dfree(q);
        B->d_bnorm = B->d_relres = nullptr;
        B->d_conv = B->d_convit = B->d_its = nullptr;
        B->d_state = nullptr;
        B->d_handles = nullptr;
        B->gP = 0;
        HHO_TRY(dalloc(ctx, &B->d_bnorm, (size_t)P));
        HHO_TRY(dalloc(ctx, &B->d_relres, (size_t)P));
        HHO_TRY(dalloc(ctx, &B->d_conv, (size_t)P));
        HHO_TRY(dalloc(ctx, &B->d_convit, (size_t)P));
        HHO_TRY(dalloc(ctx, &B->d_its, (size_t)P));
        HHO_TRY(dalloc(ctx, &B->d_state, 1));
        HHO_TRY(dalloc(ctx, &B->d_handles, (size_t)MMAX));
        B->gP = P;
    }
    if (!B->s_body) HHO_CUDA(cudaStreamCreateWithFlags(&B->s_body, cudaStreamNonBlocking));
    batch_graph_free(ctx);
    {
        // one direct V-cycle first: a kernel that cannot run is reported here as
        // an error instead of invalidating the capture
        const bool g0 = ctx->use_graphs;
        ctx->use_graphs = false;
        hho_status e = vcycle(ctx, B->V, B->Z);
        ctx->use_graphs = g0;
        HHO_TRY(e);
        HHO_CUDA(cudaStreamSynchronize(ctx->stream));
        HHO_CUDA(cudaGetLastError());
    }
    cudaStream_t main = ctx->stream;
    const bool saved_graphs = ctx->use_graphs;
    const int64_t saved_launches = ctx->launches;
    ctx->use_graphs = false;  // the V-cycle's own kernels go into this graph
    cudaGraph_t g = nullptr;
    hho_status st = HHO_OK;
    auto fail = [&](hho_status e) {
        st = e;
        return e;
    };
    do {
        if (cudaGraphCreate(&g, 0) != cudaSuccess) { fail(HHO_ERR_CUDA); break; }
        cudaGraphConditionalHandle h_outer;
        if (cudaGraphConditionalHandleCreate(&h_outer, g, 0, 0) != cudaSuccess) { fail(HHO_ERR_CUDA); break; }
        // prologue: b, x = 0, ||b_p||, w = b, tolerances
        if (cudaStreamBeginCaptureToGraph(main, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
            fail(HHO_ERR_CUDA);
            break;
        }
        int64_t l0 = ctx->launches;
        k_copy<<<grid1d(n), 256, 0, main>>>(n, ctx->rhs, B->b);
        k_zero<<<grid1d(n), 256, 0, main>>>(n, x);
        ctx->launches += 2;
        hho_status e = null_project<double>(ctx, L0, B->b);
        if (e == HHO_OK) e = S.upd_dot(B->b, nullptr, 0, 0, 0.0, B->b, 1, 0, 0, HOOK_START, 0, true);
        k_copy<<<grid1d(n), 256, 0, main>>>(n, B->b, B->w);
        k_bg_init<<<1, BG_T, 0, main>>>(P, B->stat, B->d_bnorm, B->d_conv, B->d_convit, B->d_state, maxit, h_outer);
        ctx->launches += 2;
        cudaGraph_t body = nullptr;
        if (e == HHO_OK) e = add_conditional(ctx, main, h_outer, cudaGraphCondTypeWhile, &body);
        if (e != HHO_OK) { fail(e); cudaGraph_t t; cudaStreamEndCapture(main, &t); break; }
        // epilogue: the pressure kernels' projection and the final statistics
        if (ctx->has_null) {
            e = null_project<double>(ctx, L0, x);
            if (e == HHO_OK) e = residual(ctx, 0, x, B->b, B->w);
            if (e == HHO_OK) e = S.upd_dot(B->w, nullptr, 0, 0, 0.0, B->w, 1, 0, 0, HOOK_START, 0, true);
        }
        k_bg_final<<<1, BG_T, 0, main>>>(P, B->stat, B->d_bnorm, B->d_convit, B->d_state, B->d_its, B->d_relres);
        ++ctx->launches;
        cudaGraph_t tmp = nullptr;
        if (cudaStreamEndCapture(main, &tmp) != cudaSuccess || e != HHO_OK) { fail(e != HHO_OK ? e : HHO_ERR_CUDA); break; }
        B->g_launch_fixed = ctx->launches - l0;
        // the restart cycle (WHILE body)
        std::vector<cudaGraphConditionalHandle> hs(restart);
        bool ok = true;
        for (int j = 0; j < restart && ok; ++j) ok = cudaGraphConditionalHandleCreate(&hs[j], body, 0, 0) == cudaSuccess;
        if (!ok || cudaMemcpy(B->d_handles, hs.data(), restart * sizeof(cudaGraphConditionalHandle),
                              cudaMemcpyHostToDevice) != cudaSuccess) { fail(HHO_ERR_CUDA); break; }
        ctx->stream = B->s_body;
        if (cudaStreamBeginCaptureToGraph(B->s_body, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) !=
            cudaSuccess) { fail(HHO_ERR_CUDA); break; }
        l0 = ctx->launches;
        k_bg_cycle_start<<<1, BG_T, 0, B->s_body>>>(P, B->d_conv, B->fsc, S.GT, B->d_handles, restart);
        k_seg_scale<<<B->nt, BT, 0, B->s_body>>>(S.tv, B->w, B->V, B->fsc, S.GT);
        ctx->launches += 2;
        std::vector<cudaGraph_t> ifb(restart, nullptr);
        for (int j = 0; j < restart && e == HHO_OK; ++j) e = add_conditional(ctx, B->s_body, hs[j], cudaGraphCondTypeIf, &ifb[j]);
        k_seg_update_x<<<B->nt, BT, (size_t)((G.m + 1) * G.m + G.m) * sizeof(double), B->s_body>>>(S.tv, x, B->Z, n,
                                                                                                 B->fsc, S.GT, G);
        ++ctx->launches;
        if (e == HHO_OK) e = residual(ctx, 0, x, B->b, B->w);
        if (e == HHO_OK) e = S.upd_dot(B->w, nullptr, 0, 0, 0.0, B->w, 1, 0, 0, HOOK_START, 0, true);
        k_bg_cycle_end<<<1, BG_T, 0, B->s_body>>>(P, B->stat, B->d_bnorm, B->d_conv, B->d_convit, B->d_state, rtol,
                                                  maxit, h_outer);
        ++ctx->launches;
        if (cudaStreamEndCapture(B->s_body, &tmp) != cudaSuccess || e != HHO_OK) { fail(e != HHO_OK ? e : HHO_ERR_CUDA); break; }
        B->g_launch_cycle = ctx->launches - l0;
        // the Arnoldi steps (IF bodies)
        for (int j = 0; j < restart && e == HHO_OK; ++j) {
            if (cudaStreamBeginCaptureToGraph(B->s_body, ifb[j], nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) !=
                cudaSuccess) { e = HHO_ERR_CUDA; break; }
            l0 = ctx->launches;
            double* vj = B->V + (int64_t)j * n;
            double* zj = B->Z + (int64_t)j * n;
            if (j > 0) {
                k_seg_scale<<<B->nt, BT, 0, B->s_body>>>(S.tv, B->w, vj, B->fsc, S.GT);
                ++ctx->launches;
            }
            e = vcycle(ctx, vj, zj);
            if (e == HHO_OK) e = spmv(ctx, 0, zj, B->w);
            const int nv = j + 1;
            if (e == HHO_OK) e = S.upd_dot(B->w, nullptr, 0, 0, 0.0, B->V, nv, 0, G.t1, HOOK_NONE, j, false);
            if (e == HHO_OK) e = S.upd_dot(B->w, B->V, nv, G.t1, -1.0, B->V, nv, 0, G.t2, HOOK_NONE, j, false);
            if (e == HHO_OK) e = S.upd_dot(B->w, B->V, nv, G.t2, -1.0, nullptr, 0, 1, G.nrm, HOOK_COLUMN, j, true);
            // the step's test: freezes the problems that met the tolerance and opens step j + 1
            k_bg_iter<<<1, BG_T, 0, B->s_body>>>(P, B->stat, B->d_bnorm, B->d_conv, B->d_convit, B->d_state, rtol,
                                                 maxit, j, restart, B->fsc, S.GT, B->d_handles);
            ++ctx->launches;
            if (cudaStreamEndCapture(B->s_body, &tmp) != cudaSuccess && e == HHO_OK) e = HHO_ERR_CUDA;
            if (j == 0) B->g_launch_iter = ctx->launches - l0 + 1;  // + the scaling of the later steps
        }
        if (e != HHO_OK) { fail(e); break; }
        if (cudaGraphInstantiate(&B->gexec, g, 0) != cudaSuccess) { fail(HHO_ERR_CUDA); break; }
        B->graph = g;
        g = nullptr;
        B->g_x = x;
        B->g_rtol = rtol;
        B->g_maxit = maxit;
        B->g_restart = restart;
    } while (false);
    ctx->stream = main;
    ctx->use_graphs = saved_graphs;
    ctx->launches = saved_launches;
    if (g) cudaGraphDestroy(g);
    if (st != HHO_OK) {
        cudaGetLastError();
        if (ctx->err.empty() || st == HHO_ERR_CUDA) ctx->err = "hho_solve_batch: capturing the solve graph failed";
    }
    return st;
}

static hho_status batch_solve_graph(hho_ctx* ctx, double rtol, int maxit, int restart, double* x, int32_t* its,
                                    double* relres, hho_solve_info* info) {
    BatchWork* B = ctx->batch;
    const int P = ctx->probs.P;
    if (!B->gexec || B->g_x != x || B->g_rtol != rtol || B->g_maxit != maxit || B->g_restart != restart)
        HHO_TRY(batch_graph_build(ctx, B, rtol, maxit, restart, x));
    cudaEvent_t e0, e1;
    HHO_CUDA(cudaEventCreate(&e0));
    HHO_CUDA(cudaEventCreate(&e1));
    HHO_CUDA(cudaEventRecord(e0, ctx->stream));
    HHO_CUDA(cudaGraphLaunch(B->gexec, ctx->stream));
    HHO_CUDA(cudaEventRecord(e1, ctx->stream));
    std::vector<int32_t> hits(P);
    std::vector<double> hrr(P);
    BGState hst{};
    HHO_CUDA(cudaMemcpyAsync(hits.data(), B->d_its, P * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    HHO_CUDA(cudaMemcpyAsync(hrr.data(), B->d_relres, P * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    HHO_CUDA(cudaMemcpyAsync(&hst, B->d_state, sizeof(BGState), cudaMemcpyDeviceToHost, ctx->stream));
    HHO_CUDA(cudaStreamSynchronize(ctx->stream));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->launches += B->g_launch_fixed + (int64_t)hst.cycles * B->g_launch_cycle + (int64_t)hst.it * B->g_launch_iter;
    ctx->coarse_its_total = hst.it;
    double worst = 0.0;
    bool ok = true;
    for (int p = 0; p < P; ++p) {
        if (relres) relres[p] = hrr[p];
        if (its) its[p] = hits[p];
        worst = std::max(worst, hrr[p]);
        ok &= hrr[p] <= rtol;
    }
    const hho_status st = ok ? HHO_OK : HHO_ERR_NOT_CONVERGED;
    if (info) {
        info->iterations = hst.it;
        info->coarse_iterations = hst.it;
        info->rel_residual = worst;
        info->solve_ms = ms;
        info->status = st;
    }
    if (st != HHO_OK) ctx->err = "hho_solve_batch: some problem reached maxit above the tolerance";
    return st;
}

hho_status batch_solve(hho_ctx* ctx, double rtol, int maxit, int restart, double* x, int32_t* its, double* relres,
                       hho_solve_info* info) {
    if (restart < 1 || restart > MMAX || maxit < 0 || !(rtol > 0.0)) {
        ctx->err = "hho_solve_batch: invalid restart (1..64), maxit or rtol";
        return HHO_ERR_ARG;
    }
    HHO_TRY(batch_work(ctx, restart));
    if (ctx->solve_graph && ctx->stream != nullptr) return batch_solve_graph(ctx, rtol, maxit, restart, x, its, relres, info);
    BatchWork* B = ctx->batch;
    const LevelMat& L0 = ctx->levels[0];
    const int P = ctx->probs.P;
    Seg S{ctx, B, TileView{B->nt, B->tile_prob, B->tile_r0, B->tile_len}, L0.n,
          (gs_layout(restart).total + 7) / 8 * 8, gs_layout(restart), P};
    const int64_t n = L0.n;
    const GS& G = S.G;
    cudaEvent_t e0, e1;
    HHO_CUDA(cudaEventCreate(&e0));
    HHO_CUDA(cudaEventCreate(&e1));
    HHO_CUDA(cudaEventRecord(e0, ctx->stream));
    ctx->coarse_its_total = 0;
    k_copy<<<grid1d(n), 256, 0, ctx->stream>>>(n, ctx->rhs, B->b);
    k_zero<<<grid1d(n), 256, 0, ctx->stream>>>(n, x);
    ctx->launches += 2;
    HHO_TRY(null_project<double>(ctx, L0, B->b));
    // ||b_p|| with the START recurrence of every problem
    HHO_TRY(S.upd_dot(B->b, nullptr, 0, 0, 0.0, B->b, 1, 0, 0, HOOK_START, 0, true));
    HHO_TRY(S.read_stat());
    std::vector<double> bnorm(P), beta(P), est(P);
    std::vector<int> conv_it(P, -1);
    std::vector<char> conv(P, 0);
    std::vector<int32_t> frz;
    for (int p = 0; p < P; ++p) {
        bnorm[p] = beta[p] = B->h_stat[2 * p];
        if (!(bnorm[p] > 0.0)) {
            conv[p] = 1;
            conv_it[p] = 0;
        }
    }
    int it = 0;
    bool all_conv = std::all_of(conv.begin(), conv.end(), [](char c) { return c != 0; });
    const double* r = B->b;
    while (!all_conv && it < maxit) {
        // problems already converged keep their iterate: freeze their recurrence
        frz.clear();
        for (int p = 0; p < P; ++p)
            if (conv[p]) frz.push_back(p);
        HHO_TRY(S.freeze(frz));
        k_seg_scale<<<B->nt, BT, 0, ctx->stream>>>(S.tv, r, B->V, B->fsc, S.GT);
        ++ctx->launches;
        for (int j = 0; j < restart; ++j) {
            double* vj = B->V + (int64_t)j * n;
            double* zj = B->Z + (int64_t)j * n;
            HHO_TRY(vcycle(ctx, vj, zj));
            HHO_TRY(spmv(ctx, 0, zj, B->w));
            const int nv = j + 1;
            // t1 = V^T w;  w -= V t1, t2 = V^T w;  w -= V t2, ||w||^2 and the Hessenberg column
            HHO_TRY(S.upd_dot(B->w, nullptr, 0, 0, 0.0, B->V, nv, 0, G.t1, HOOK_NONE, j, false));
            HHO_TRY(S.upd_dot(B->w, B->V, nv, G.t1, -1.0, B->V, nv, 0, G.t2, HOOK_NONE, j, false));
            HHO_TRY(S.upd_dot(B->w, B->V, nv, G.t2, -1.0, nullptr, 0, 1, G.nrm, HOOK_COLUMN, j, true));
            ++it;
            HHO_TRY(S.read_stat());
            bool all = true;
            frz.clear();
            for (int p = 0; p < P; ++p) {
                if (conv[p]) continue;
                est[p] = B->h_stat[2 * p];
                const bool brk = B->h_stat[2 * p + 1] != 0.0;
                if (est[p] <= rtol * bnorm[p]) {
                    if (conv_it[p] < 0) conv_it[p] = it;
                    frz.push_back(p);
                } else if (!brk) {
                    all = false;
                }
            }
            HHO_TRY(S.freeze(frz));
            if (all || it >= maxit || j + 1 == restart) break;
            k_seg_scale<<<B->nt, BT, 0, ctx->stream>>>(S.tv, B->w, B->V + (int64_t)(j + 1) * n, B->fsc, S.GT);
            ++ctx->launches;
        }
        // x_p += Z y_p, then the true residuals and the START state of the next cycle
        k_seg_update_x<<<B->nt, BT, (size_t)((G.m + 1) * G.m + G.m) * sizeof(double), ctx->stream>>>(
            S.tv, x, B->Z, n, B->fsc, S.GT, G);
        ++ctx->launches;
        HHO_TRY(residual(ctx, 0, x, B->b, B->w));
        HHO_TRY(S.upd_dot(B->w, nullptr, 0, 0, 0.0, B->w, 1, 0, 0, HOOK_START, 0, true));
        HHO_TRY(S.read_stat());
        all_conv = true;
        for (int p = 0; p < P; ++p) {
            beta[p] = B->h_stat[2 * p];
            if (beta[p] <= rtol * bnorm[p] || !(bnorm[p] > 0.0)) {
                if (!conv[p] && conv_it[p] < 0) conv_it[p] = it;
                conv[p] = 1;
            } else {
                conv[p] = 0;  // the estimate was optimistic: iterate again
                conv_it[p] = -1;
                all_conv = false;
            }
        }
        r = B->w;
    }
    if (ctx->has_null) {
        HHO_TRY(null_project<double>(ctx, L0, x));
        HHO_TRY(residual(ctx, 0, x, B->b, B->w));
        HHO_TRY(S.upd_dot(B->w, nullptr, 0, 0, 0.0, B->w, 1, 0, 0, HOOK_START, 0, true));
        HHO_TRY(S.read_stat());
        for (int p = 0; p < P; ++p) beta[p] = B->h_stat[2 * p];
    }
    HHO_CUDA(cudaEventRecord(e1, ctx->stream));
    HHO_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    double worst = 0.0;
    bool ok = true;
    for (int p = 0; p < P; ++p) {
        const double rr = bnorm[p] > 0.0 ? beta[p] / bnorm[p] : 0.0;
        if (relres) relres[p] = rr;
        const int ip = conv_it[p] >= 0 ? conv_it[p] : it;
        if (its) its[p] = ip;
        worst = std::max(worst, rr);
        ok &= rr <= rtol;
    }
    const hho_status st = ok ? HHO_OK : HHO_ERR_NOT_CONVERGED;
    if (info) {
        info->iterations = it;
        info->coarse_iterations = (int32_t)ctx->coarse_its_total;
        info->rel_residual = worst;
        info->solve_ms = ms;
        info->status = st;
    }
    HHO_CUDA(cudaGetLastError());
    if (st != HHO_OK) ctx->err = "hho_solve_batch: some problem reached maxit above the tolerance";
    return st;
}

// Pick the operator kernel variant, its grid and the tile size by timing:
// every candidate runs `reps` V-cycles (and, for a batch, `reps` segmented
// update kernels) on a fixed input; the fastest is kept.  choice (host, may be
// NULL) receives {spmv_rows, spmv_grid, tile_rows}.
static hho_status autotune_run(hho_ctx* ctx, int reps, double* r, double* z, cudaEvent_t e0, cudaEvent_t e1,
                               double* choice) {
    const int64_t n = ctx->levels[0].n;
    HHO_CUDA(cudaMemcpyAsync(r, ctx->rhs, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    auto time_vcycles = [&](float* ms) -> hho_status {
        HHO_TRY(vcycle(ctx, r, z));  // capture / warm up
        HHO_CUDA(cudaEventRecord(e0, ctx->stream));
        for (int i = 0; i < reps; ++i) HHO_TRY(vcycle(ctx, r, z));
        HHO_CUDA(cudaEventRecord(e1, ctx->stream));
        HHO_CUDA(cudaEventSynchronize(e1));
        HHO_CUDA(cudaEventElapsedTime(ms, e0, e1));
        return HHO_OK;
    };
    const int rows_c[] = {0, 2, 4};
    const int grid_c[] = {0, sm_count() * 8, sm_count() * 16};
    float best = 1e30f;
    int br = ctx->spmv_rows, bg = ctx->spmv_grid;
    for (int rr : rows_c)
        for (int gg : grid_c) {
            ctx->spmv_rows = rr;
            ctx->spmv_grid = gg;
            invalidate_graphs(ctx);
            float ms = 0.f;
            HHO_TRY(time_vcycles(&ms));
            if (ms < best) {
                best = ms;
                br = rr;
                bg = gg;
            }
        }
    ctx->spmv_rows = br;
    ctx->spmv_grid = bg;
    invalidate_graphs(ctx);
    int bt = ctx->tile_rows;
    if (ctx->probs.declared) {
        const int tile_c[] = {1024, 2048, 4096, 8192};
        float bt_ms = 1e30f;
        for (int tr : tile_c) {
            ctx->tile_rows = tr;
            HHO_TRY(batch_work(ctx, ctx->batch ? ctx->batch->restart : 30));
            BatchWork* B = ctx->batch;
            const GS G = gs_layout(B->restart);
            Seg S{ctx, B, TileView{B->nt, B->tile_prob, B->tile_r0, B->tile_len}, n, (G.total + 7) / 8 * 8, G,
                  ctx->probs.P};
            HHO_TRY(S.upd_dot(z, nullptr, 0, 0, 0.0, r, 1, 1, G.t1, HOOK_NONE, 0, false));
            HHO_CUDA(cudaEventRecord(e0, ctx->stream));
            for (int i = 0; i < reps; ++i) HHO_TRY(S.upd_dot(z, nullptr, 0, 0, 0.0, r, 1, 1, G.t1, HOOK_NONE, 0, false));
            HHO_CUDA(cudaEventRecord(e1, ctx->stream));
            HHO_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            HHO_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < bt_ms) {
                bt_ms = ms;
                bt = tr;
            }
        }
        ctx->tile_rows = bt;
        HHO_TRY(batch_work(ctx, ctx->batch->restart));
    }
    if (choice) {
        choice[0] = br;
        choice[1] = bg;
        choice[2] = bt;
    }
    return HHO_OK;
}

// The timing buffers and events are released on every path; a failed run
// restores the kernel choices the context had before.
hho_status autotune(hho_ctx* ctx, int reps, double* choice) {
    const int64_t n = ctx->levels[0].n;
    const int rows0 = ctx->spmv_rows, grid0 = ctx->spmv_grid, tile0 = ctx->tile_rows;
    double *r = nullptr, *z = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    hho_status st = dalloc(ctx, &r, (size_t)n);
    if (st == HHO_OK) st = dalloc(ctx, &z, (size_t)n);
    if (st == HHO_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) {
        ctx->err = "hho_autotune: cudaEventCreate failed";
        st = HHO_ERR_CUDA;
    }
    if (st == HHO_OK) st = autotune_run(ctx, reps, r, z, e0, e1, choice);
    if (st != HHO_OK) {
        ctx->spmv_rows = rows0;
        ctx->spmv_grid = grid0;
        ctx->tile_rows = tile0;
        invalidate_graphs(ctx);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dfree(r);
    dfree(z);
    return st;
}

}  // namespace hho
