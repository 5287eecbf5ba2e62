// Exact coarse solve of the p-multilevel V-cycle (Sec. 3.3, Algorithm MG_V:
// c = A_L^{-1} d on the coarsest level) by a nested-dissection multifrontal
// factorisation, for coarse levels too large for one dense inverse.
//
// Elimination tree.  The elements of every problem are split by recursive
// coordinate bisection (longest extent of the centroids, median cut) down to
// leaves of at most `leaf` elements.  Every coarse unknown is eliminated at one
// tree node:
//  * a face's unknowns at the lowest common ancestor of the leaves of its one or
//    two elements (boundary faces and faces inside a leaf at the leaf);
//  * an element's pressure coefficients other than the first at its leaf;
//  * the first pressure coefficient at the lowest node where the element is not
//    the representative (smallest element) of its connected component, the
//    components of a node being its elements joined by the faces eliminated in
//    its subtree.  The constant pressure of such a component does not act on
//    the component's interior velocity unknowns, so one mean pressure per
//    component is kept for the parent; the last one reaches the problem's root.
// Node v then has the eliminated set I (owned unknowns) and the boundary set B
// (unknowns of its elements owned by an ancestor), and its dense frontal matrix
// over [I | B] is the sum of its elements' contributions (leaves: prefixes of
// the fine element Schur complements, as the Galerkin coarse operator of
// Sec. 4.2) or of its children's Schur updates (internal nodes, extend-add).
//
// Factorisation of a front F = [F_II F_IB; F_BI F_BB]: Gauss-Jordan with partial
// pivoting restricted to the I rows on [F | E_I] (E_I the identity on the I
// rows) gives [I X Finv; 0 U -W] with Finv = F_II^{-1}, X = Finv F_IB,
// W = F_BI Finv and the Schur update U = F_BB - F_BI X passed to the parent.
// Solve: forward, leaves to roots, f = (own d entries on I) + extend-add of the
// children's u; y = Finv f_I; u = f_B - W f_I.  Backward, roots to leaves,
// x_I = y - X x_B.  A problem with a constant-pressure kernel (no Neumann face)
// gets alpha = mean |diag| added on the diagonal of its root's kept pressure;
// the caller projects the result on the complement of the kernel, which gives
// the same solution as the rank-one fix of the dense path.
//
// Levels of the tree with at least one node per SM are factored one CTA per
// node; the few large fronts near the roots are factored by all SMs, one pivot
// column per pair of launches.  The tree, the index maps and the offsets are
// integer bookkeeping done once on the host; every floating-point operation
// runs in the kernels below.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "internal.h"

namespace hho {

namespace {

constexpr int MF_T = 256;           // threads per CTA
constexpr int MF_WARPS = MF_T / 32;

__host__ __device__ inline int64_t mf_ld(int64_t n) { return (n + 3) & ~int64_t(3); }

int mf_grid(int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + MF_T - 1) / MF_T, (int64_t)sm_count() * 16));
}

// Per-node device data.
struct MFView {
    const int32_t* m;        // front size
    const int32_t* nI;       // eliminated unknowns (the first nI front positions)
    const int32_t* child;    // 2 per node, -1 = none
    const int32_t* pin;      // front position that gets +alpha on its diagonal, -1 = none
    const int64_t* offW;     // factorisation workspace: m x (m + nI) row-major
    const int64_t* offM1;    // [Finv; -W]: m x nI column-major, ld mf_ld(m)
    const int64_t* offX;     // X: nI x (m - nI) column-major, ld mf_ld(nI)
    const int64_t* offP;     // front positions: glob[], cpos[2][] start
    const int64_t* offY;     // forward buffer y (nI)
    const int64_t* offU;     // forward buffer u (m - nI)
    const int32_t* glob;     // global coarse index of every front position
    const int32_t* cpos;     // 2 per front position: index in child 0 / 1's B set, -1 = none
    // leaves
    const int32_t* leaf_elem_ptr;  // per node: range in leaf_elem (empty for internal nodes)
    const int32_t* leaf_elem;
    const int64_t* elem_loc_off;   // per element: offset in elem_loc
    const int32_t* elem_loc;       // per element local unknown: front position in its leaf
    const int32_t* ef_ptr;
    const int64_t* off_S;
    const double* S;               // fine element Schur complements
    int b0, nF0, nP0, bL, nFL, nPL;
    int ec;  // components of an element block (1, or d + 1 uncondensed), each truncated on its own
    const double* alpha;
};

// Entry (i, j) of a child's Schur update U, read from its workspace.
__device__ __forceinline__ double child_u(const MFView& V, const double* __restrict__ Wall, int c, int a, int b) {
    const int m = V.m[c], nI = V.nI[c];
    return Wall[V.offW[c] + (int64_t)(nI + a) * (m + nI) + (nI + b)];
}

// Front entry (i, j) of an internal node from its children's updates (extend-add
// as a gather: child 0 then child 1, fixed order).
__device__ __forceinline__ double gather_entry(const MFView& V, const double* __restrict__ Wall, int v, int i, int j) {
    const int32_t* cp = V.cpos + 2 * V.offP[v];
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int c = V.child[2 * v + q];
        if (c < 0) continue;
        const int a = cp[2 * i + q], b = cp[2 * j + q];
        if (a >= 0 && b >= 0) s += child_u(V, Wall, c, a, b);
    }
    return s;
}

// Assemble the augmented front [F | E_I] of node v into its workspace with the
// threads [t0, t0 + nt) (one CTA, or one CTA of a grid over the node).
__device__ void assemble_internal(const MFView& V, double* __restrict__ Wall, int v, int64_t t0, int64_t nt) {
    const int m = V.m[v], nI = V.nI[v], w = m + nI;
    double* W = Wall + V.offW[v];
    const int pin = V.pin[v];
    const double al = pin >= 0 ? *V.alpha : 0.0;
    for (int64_t idx = t0; idx < (int64_t)m * w; idx += nt) {
        const int i = (int)(idx / w), j = (int)(idx % w);
        double x;
        if (j < m) {
            x = gather_entry(V, Wall, v, i, j);
            if (i == pin && j == pin) x += al;
        } else {
            x = (j - m == i) ? 1.0 : 0.0;
        }
        W[idx] = x;
    }
}

// Leaf front: element contributions (prefix of the fine element Schur
// complements at the coarse degree), elements in order.  One CTA.
__device__ void assemble_leaf(const MFView& V, double* __restrict__ Wall, int v) {
    const int m = V.m[v], nI = V.nI[v], w = m + nI;
    double* W = Wall + V.offW[v];
    for (int64_t idx = threadIdx.x; idx < (int64_t)m * w; idx += blockDim.x) {
        const int i = (int)(idx / w), j = (int)(idx % w);
        W[idx] = (j >= m && j - m == i) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int e = V.leaf_elem_ptr[v]; e < V.leaf_elem_ptr[v + 1]; ++e) {
        const int T = V.leaf_elem[e];
        const int N = V.ef_ptr[T + 1] - V.ef_ptr[T];
        const int nk0 = N * V.b0 + V.nP0, nkL = N * V.bL + V.nPL;
        const double* ST = V.S + V.off_S[T];
        const int32_t* loc = V.elem_loc + V.elem_loc_off[T];
        for (int idx = threadIdx.x; idx < nkL * nkL; idx += blockDim.x) {
            const int a = idx / nkL, bb = idx % nkL;
            const int nEL = V.nPL / V.ec, nE0 = V.nP0 / V.ec;
            const int ea = a - N * V.bL, eb = bb - N * V.bL;
            const int fa = a < N * V.bL ? (a / V.bL) * V.b0 + ((a % V.bL) / V.nFL) * V.nF0 + (a % V.bL) % V.nFL
                                        : N * V.b0 + (ea / nEL) * nE0 + ea % nEL;
            const int fb = bb < N * V.bL ? (bb / V.bL) * V.b0 + ((bb % V.bL) / V.nFL) * V.nF0 + (bb % V.bL) % V.nFL
                                         : N * V.b0 + (eb / nEL) * nE0 + eb % nEL;
            W[(int64_t)loc[a] * w + loc[bb]] += ST[(int64_t)fa * nk0 + fb];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && V.pin[v] >= 0) W[(int64_t)V.pin[v] * w + V.pin[v]] += *V.alpha;
    __syncthreads();
}

// Gauss-Jordan of one front by one CTA: pivots in the first nI columns, chosen
// among the I rows (largest magnitude, lowest row on ties), elimination from
// all m rows.  Columns left of the pivot column are already reduced and are
// not touched.  Returns false on a zero pivot.
__device__ bool cta_front_gj(double* __restrict__ W, int m, int nI) {
    __shared__ double s_best[MF_WARPS];
    __shared__ int s_arg[MF_WARPS];
    __shared__ int s_piv, s_ok;
    const int w = m + nI;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int j = 0; j < nI; ++j) {
        double best = -1.0;
        int arg = nI;
        for (int i = j + threadIdx.x; i < nI; i += blockDim.x) {
            const double a = fabs(W[(int64_t)i * w + j]);
            if (a > best) {
                best = a;
                arg = i;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
            if (ob > best || (ob == best && oa < arg)) {
                best = ob;
                arg = oa;
            }
        }
        if (lane == 0) {
            s_best[wid] = best;
            s_arg[wid] = arg;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = s_best[0];
            int a = s_arg[0];
            for (int q = 1; q < MF_WARPS; ++q)
                if (s_best[q] > b || (s_best[q] == b && s_arg[q] < a)) {
                    b = s_best[q];
                    a = s_arg[q];
                }
            s_piv = a;
            s_ok = (b > 0.0);
        }
        __syncthreads();
        if (!s_ok) return false;
        const int p = s_piv;
        if (p != j)
            for (int c = j + threadIdx.x; c < w; c += blockDim.x) {
                const double t = W[(int64_t)j * w + c];
                W[(int64_t)j * w + c] = W[(int64_t)p * w + c];
                W[(int64_t)p * w + c] = t;
            }
        __syncthreads();
        const double inv = 1.0 / W[(int64_t)j * w + j];
        __syncthreads();
        for (int c = j + threadIdx.x; c < w; c += blockDim.x) W[(int64_t)j * w + c] = (c == j) ? 1.0 : W[(int64_t)j * w + c] * inv;
        __syncthreads();
        const double* wj = W + (int64_t)j * w;
        for (int i = wid; i < m; i += MF_WARPS) {
            if (i == j) continue;
            double* wi = W + (int64_t)i * w;
            const double f = wi[j];
            if (f == 0.0) continue;
            for (int c = j + 1 + lane; c < w; c += 32) wi[c] -= f * wj[c];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += blockDim.x)
            if (i != j) W[(int64_t)i * w + j] = 0.0;
        __syncthreads();
    }
    return true;
}

// Copy [Finv; -W] and X of node v from its workspace into the solve arrays.
__device__ void extract(const MFView& V, const double* __restrict__ Wall, double* __restrict__ M1all,
                        double* __restrict__ Xall, int v, int64_t t0, int64_t nt) {
    const int m = V.m[v], nI = V.nI[v], nB = m - nI, w = m + nI;
    const double* W = Wall + V.offW[v];
    double* M1 = M1all + V.offM1[v];
    double* X = Xall + V.offX[v];
    const int64_t ld1 = mf_ld(m), ldx = mf_ld(nI);
    for (int64_t idx = t0; idx < (int64_t)ld1 * nI; idx += nt) {
        const int jj = (int)(idx / ld1), i = (int)(idx % ld1);
        M1[idx] = i < m ? W[(int64_t)i * w + m + jj] : 0.0;
    }
    for (int64_t idx = t0; idx < ldx * nB; idx += nt) {
        const int jj = (int)(idx / ldx), i = (int)(idx % ldx);
        X[idx] = i < nI ? W[(int64_t)i * w + nI + jj] : 0.0;
    }
}

// One CTA per node: assemble, factor, extract.
__global__ void __launch_bounds__(MF_T) k_mf_factor_cta(MFView V, const int32_t* __restrict__ nodes, int nn,
                                                       double* __restrict__ Wall, double* __restrict__ M1all,
                                                       double* __restrict__ Xall, int* __restrict__ status) {
    for (int q = blockIdx.x; q < nn; q += gridDim.x) {
        const int v = nodes[q];
        if (V.leaf_elem_ptr[v + 1] > V.leaf_elem_ptr[v]) {
            assemble_leaf(V, Wall, v);
        } else {
            assemble_internal(V, Wall, v, threadIdx.x, blockDim.x);
            __syncthreads();
        }
        if (!cta_front_gj(Wall + V.offW[v], V.m[v], V.nI[v])) {
            if (threadIdx.x == 0) atomicExch(status, (int)HHO_ERR_SINGULAR);
            continue;
        }
        extract(V, Wall, M1all, Xall, v, threadIdx.x, blockDim.x);
        __syncthreads();
    }
}

// Grid-wide front assembly of internal nodes: blockIdx.y = node of the level.
__global__ void __launch_bounds__(MF_T) k_mf_assemble(MFView V, const int32_t* __restrict__ nodes,
                                                     double* __restrict__ Wall) {
    const int v = nodes[blockIdx.y];
    assemble_internal(V, Wall, v, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

// Pivot step j of every node of a level (one CTA per node): choose the pivot
// row, swap, scale, and store the multipliers of column j in colbuf.
__global__ void __launch_bounds__(MF_T) k_mf_pivot(MFView V, const int32_t* __restrict__ nodes, int j,
                                                  double* __restrict__ Wall, double* __restrict__ colbuf,
                                                  const int64_t* __restrict__ coloff, int* __restrict__ status) {
    __shared__ double s_best[MF_WARPS];
    __shared__ int s_arg[MF_WARPS];
    __shared__ int s_piv, s_ok;
    const int v = nodes[blockIdx.x];
    const int m = V.m[v], nI = V.nI[v], w = m + nI;
    if (j >= nI) return;
    double* W = Wall + V.offW[v];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double best = -1.0;
    int arg = nI;
    for (int i = j + threadIdx.x; i < nI; i += blockDim.x) {
        const double a = fabs(W[(int64_t)i * w + j]);
        if (a > best) {
            best = a;
            arg = i;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
        if (ob > best || (ob == best && oa < arg)) {
            best = ob;
            arg = oa;
        }
    }
    if (lane == 0) {
        s_best[wid] = best;
        s_arg[wid] = arg;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = s_best[0];
        int a = s_arg[0];
        for (int q = 1; q < MF_WARPS; ++q)
            if (s_best[q] > b || (s_best[q] == b && s_arg[q] < a)) {
                b = s_best[q];
                a = s_arg[q];
            }
        s_piv = a;
        s_ok = (b > 0.0);
        if (!s_ok) atomicExch(status, (int)HHO_ERR_SINGULAR);
    }
    __syncthreads();
    double* cb = colbuf + coloff[blockIdx.x];
    if (!s_ok) {  // leave the node unchanged: the elimination kernel reads zero multipliers
        for (int i = threadIdx.x; i < m; i += blockDim.x) cb[i] = 0.0;
        return;
    }
    const int p = s_piv;
    if (p != j)
        for (int c = j + threadIdx.x; c < w; c += blockDim.x) {
            const double t = W[(int64_t)j * w + c];
            W[(int64_t)j * w + c] = W[(int64_t)p * w + c];
            W[(int64_t)p * w + c] = t;
        }
    __syncthreads();
    const double inv = 1.0 / W[(int64_t)j * w + j];
    __syncthreads();
    for (int c = j + threadIdx.x; c < w; c += blockDim.x) W[(int64_t)j * w + c] = (c == j) ? 1.0 : W[(int64_t)j * w + c] * inv;
    for (int i = threadIdx.x; i < m; i += blockDim.x) cb[i] = (i == j) ? 0.0 : W[(int64_t)i * w + j];
}

// Elimination of column j: W[i][c] -= colbuf[i] W[j][c] for i != j, c > j, and
// W[i][j] = 0 (blockIdx.y = node of the level).  One warp per row (rows with a
// zero multiplier are skipped whole), lanes over the columns.
__global__ void __launch_bounds__(MF_T) k_mf_elim(MFView V, const int32_t* __restrict__ nodes, int j,
                                                 double* __restrict__ Wall, const double* __restrict__ colbuf,
                                                 const int64_t* __restrict__ coloff) {
    const int v = nodes[blockIdx.y];
    const int m = V.m[v], nI = V.nI[v], w = m + nI;
    if (j >= nI) return;
    double* W = Wall + V.offW[v];
    const double* cb = colbuf + coloff[blockIdx.y];
    const double* wj = W + (int64_t)j * w;
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < m; i += nw) {
        const double f = cb[i];
        if (i == j || f == 0.0) continue;
        double* wi = W + i * w;
        for (int c = j + 1 + lane; c < w; c += 32) wi[c] -= f * wj[c];
        if (lane == 0) wi[j] = 0.0;
    }
}

__global__ void __launch_bounds__(MF_T) k_mf_extract(MFView V, const int32_t* __restrict__ nodes,
                                                    const double* __restrict__ Wall, double* __restrict__ M1all,
                                                    double* __restrict__ Xall) {
    const int v = nodes[blockIdx.y];
    extract(V, Wall, M1all, Xall, v, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

__global__ void k_mf_mean_abs_diag(int64_t nf, int64_t ne, int b, int nP, const double* __restrict__ ff,
                                   const double* __restrict__ pp, double* __restrict__ alpha) {
    __shared__ double red[MF_T];
    double s = 0.0;
    const int64_t nfr = nf * b, n = nfr + ne * nP;
    // fixed assignment of rows to threads and a fixed-order tree: deterministic
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        if (i < nfr) {
            const int64_t F = i / b;
            const int r = (int)(i % b);
            s += fabs(ff[((int64_t)r * b + r) * nf + F]);
        } else {
            const int64_t T = (i - nfr) / nP;
            const int r = (int)((i - nfr) % nP);
            s += fabs(pp[((int64_t)r * nP + r) * ne + T]);
        }
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *alpha = red[0] / (double)n;
}

// ---------------------------------------------------------------------------
// solve kernels (FP64, or FP32 copies of M1 / X)
// ---------------------------------------------------------------------------
// W consecutive rows per lane: the widest 16-byte vector (2 FP64, 4 FP32) on
// levels with enough row blocks to fill the GPU, one row per lane (32 rows
// per CTA, 4x / 2x more CTAs) on the few large fronts near the roots
template <typename T, int W> struct MFVec;
template <> struct MFVec<double, 2> {
    using V = double2;
    __device__ static void fma(double* a, const double2& q, double x) {
        a[0] += q.x * x;
        a[1] += q.y * x;
    }
};
template <> struct MFVec<float, 4> {
    using V = float4;
    __device__ static void fma(float* a, const float4& q, float x) {
        a[0] += q.x * x;
        a[1] += q.y * x;
        a[2] += q.z * x;
        a[3] += q.w * x;
    }
};
template <typename T> struct MFVec<T, 1> {
    using V = T;
    __device__ static void fma(T* a, const T& q, T x) { a[0] += q * x; }
};
template <typename T> constexpr int mf_wide() { return std::is_same<T, float>::value ? 4 : 2; }
constexpr int MF_UNROLL = 4;

// rows [rb*RB, rb*RB + RB) of the column-major matrix A (ld, ncol columns)
// times the vector xs (shared memory); lane l of every warp owns W consecutive
// rows (one 16-byte load per column), warp w takes columns w, w + 8, ...; the
// warp partials are added in warp order (deterministic).  Results in sred[0..RB).
template <typename T, int W>
__device__ void block_colmajor_gemv(const T* __restrict__ A, int64_t ld, int nrow, int ncol, const T* xs, int rb,
                                    T* sred) {
    using DV = MFVec<T, W>;
    using V = typename DV::V;
    constexpr int RB = 32 * W;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int r0 = rb * RB + lane * W;
    T acc[W];
#pragma unroll
    for (int q = 0; q < W; ++q) acc[q] = T(0);
    if (r0 < nrow) {
        const T* a = A + r0;
        int j = w;
        for (; j + MF_WARPS * (MF_UNROLL - 1) < ncol; j += MF_WARPS * MF_UNROLL) {
            V q4[MF_UNROLL];
#pragma unroll
            for (int u = 0; u < MF_UNROLL; ++u) q4[u] = __ldg(reinterpret_cast<const V*>(a + (int64_t)(j + MF_WARPS * u) * ld));
#pragma unroll
            for (int u = 0; u < MF_UNROLL; ++u) DV::fma(acc, q4[u], xs[j + MF_WARPS * u]);
        }
        for (; j < ncol; j += MF_WARPS) DV::fma(acc, __ldg(reinterpret_cast<const V*>(a + (int64_t)j * ld)), xs[j]);
    }
#pragma unroll
    for (int q = 0; q < W; ++q) sred[w * RB + lane * W + q] = acc[q];
    __syncthreads();
    for (int r = threadIdx.x; r < RB; r += blockDim.x) {
        T t = sred[r];
#pragma unroll
        for (int q = 1; q < MF_WARPS; ++q) t += sred[q * RB + r];
        sred[MF_WARPS * RB + r] = t;
    }
    __syncthreads();
}

// Forward step of one tree level: one CTA per (node, block of RB front rows).
template <typename T, int W>
__global__ void __launch_bounds__(MF_T) k_mf_fwd(MFView V, const int32_t* __restrict__ nodes, int rb_max,
                                                const T* __restrict__ M1all, const T* __restrict__ d,
                                                T* __restrict__ Y, T* __restrict__ U) {
    constexpr int RB = 32 * W;
    extern __shared__ unsigned char mf_smem[];
    T* sred = reinterpret_cast<T*>(mf_smem);           // (MF_WARPS + 1) * RB
    T* f = sred + (MF_WARPS + 1) * RB;                 // m
    const int q = blockIdx.x / rb_max, rb = blockIdx.x % rb_max;
    const int v = nodes[q];
    const int m = V.m[v], nI = V.nI[v];
    if (rb * RB >= m) return;
    const int32_t* gl = V.glob + V.offP[v];
    const int32_t* cp = V.cpos + 2 * V.offP[v];
    const int c0 = V.child[2 * v], c1 = V.child[2 * v + 1];
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        T s = i < nI ? d[gl[i]] : T(0);
        if (c0 >= 0 && cp[2 * i] >= 0) s += U[V.offU[c0] + cp[2 * i]];
        if (c1 >= 0 && cp[2 * i + 1] >= 0) s += U[V.offU[c1] + cp[2 * i + 1]];
        f[i] = s;
    }
    __syncthreads();
    block_colmajor_gemv<T, W>(M1all + V.offM1[v], mf_ld(m), m, nI, f, rb, sred);
    const T* res = sred + MF_WARPS * RB;
    for (int r = threadIdx.x; r < RB; r += blockDim.x) {
        const int i = rb * RB + r;
        if (i >= m) continue;
        if (i < nI) Y[V.offY[v] + i] = res[r];
        else U[V.offU[v] + (i - nI)] = res[r] + f[i];
    }
}

// Backward step of one tree level: x_I = y - X x_B, written to the global
// solution (one CTA per (node, block of RB eliminated rows)).
template <typename T, int W>
__global__ void __launch_bounds__(MF_T) k_mf_bwd(MFView V, const int32_t* __restrict__ nodes, int rb_max,
                                                const T* __restrict__ Xall, const T* __restrict__ Y,
                                                T* __restrict__ c) {
    constexpr int RB = 32 * W;
    extern __shared__ unsigned char mf_smem[];
    T* sred = reinterpret_cast<T*>(mf_smem);
    T* xb = sred + (MF_WARPS + 1) * RB;
    const int q = blockIdx.x / rb_max, rb = blockIdx.x % rb_max;
    const int v = nodes[q];
    const int m = V.m[v], nI = V.nI[v], nB = m - nI;
    if (rb * RB >= nI) return;
    const int32_t* gl = V.glob + V.offP[v];
    for (int j = threadIdx.x; j < nB; j += blockDim.x) xb[j] = c[gl[nI + j]];
    __syncthreads();
    block_colmajor_gemv<T, W>(Xall + V.offX[v], mf_ld(nI), nI, nB, xb, rb, sred);
    const T* res = sred + MF_WARPS * RB;
    for (int r = threadIdx.x; r < RB; r += blockDim.x) {
        const int i = rb * RB + r;
        if (i < nI) c[gl[i]] = Y[V.offY[v] + i] - res[r];
    }
}

// Entry i of the forward right-hand side f of node v: own d entries on I plus
// the children's updates (extend-add as a gather, child 0 then child 1).
template <typename T>
__device__ __forceinline__ T mf_f_entry(const MFView& V, int v, int i, int nI, const T* __restrict__ d,
                                        const T* __restrict__ U) {
    const int32_t* gl = V.glob + V.offP[v];
    const int32_t* cp = V.cpos + 2 * V.offP[v];
    const int c0 = V.child[2 * v], c1 = V.child[2 * v + 1];
    T s = i < nI ? d[gl[i]] : T(0);
    if (c0 >= 0 && cp[2 * i] >= 0) s += U[V.offU[c0] + cp[2 * i]];
    if (c1 >= 0 && cp[2 * i + 1] >= 0) s += U[V.offU[c1] + cp[2 * i + 1]];
    return s;
}

// Levels with too few (node, row block) pairs to fill the GPU (the large
// fronts near the roots) also split the columns: CTA (node q, row block rb,
// column chunk cc) writes the partial product of its chunk to part[(q rb_max +
// rb) cs + cc][RB]; the finishing kernel adds the cs partials in chunk order
// (deterministic) and applies the step's epilogue.
template <typename T, int W>
__global__ void __launch_bounds__(MF_T) k_mf_fwd_part(MFView V, const int32_t* __restrict__ nodes, int rb_max, int cs,
                                                     const T* __restrict__ M1all, const T* __restrict__ d,
                                                     const T* __restrict__ U, T* __restrict__ part) {
    constexpr int RB = 32 * W;
    extern __shared__ unsigned char mf_smem[];
    T* sred = reinterpret_cast<T*>(mf_smem);
    T* f = sred + (MF_WARPS + 1) * RB;  // the chunk's columns of f
    const int cc = blockIdx.x % cs, rest = blockIdx.x / cs;
    const int q = rest / rb_max, rb = rest % rb_max;
    const int v = nodes[q];
    const int m = V.m[v], nI = V.nI[v];
    if (rb * RB >= m) return;
    const int chunk = (nI + cs - 1) / cs;
    const int j0 = min(nI, cc * chunk), j1 = min(nI, j0 + chunk);
    for (int j = j0 + (int)threadIdx.x; j < j1; j += blockDim.x) f[j - j0] = mf_f_entry<T>(V, v, j, nI, d, U);
    __syncthreads();
    const int64_t ld = mf_ld(m);
    block_colmajor_gemv<T, W>(M1all + V.offM1[v] + (int64_t)j0 * ld, ld, m, j1 - j0, f, rb, sred);
    const T* res = sred + MF_WARPS * RB;
    T* out = part + (int64_t)blockIdx.x * RB;
    for (int r = threadIdx.x; r < RB; r += blockDim.x) out[r] = res[r];
}

template <typename T>
__global__ void k_mf_fwd_fin(MFView V, const int32_t* __restrict__ nodes, int cnt, int rb_max, int RB, int cs,
                             const T* __restrict__ part, const T* __restrict__ d, T* __restrict__ Y,
                             T* __restrict__ U) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)cnt * rb_max * RB) return;
    const int r = (int)(t % RB);
    const int64_t rest = t / RB;
    const int rb = (int)(rest % rb_max), q = (int)(rest / rb_max);
    const int v = nodes[q];
    const int m = V.m[v], nI = V.nI[v], i = rb * RB + r;
    if (i >= m) return;
    const T* p = part + ((int64_t)q * rb_max + rb) * cs * RB + r;
    T s = T(0);
    for (int c = 0; c < cs; ++c) s += p[(int64_t)c * RB];
    if (i < nI) Y[V.offY[v] + i] = s;
    else U[V.offU[v] + (i - nI)] = s + mf_f_entry<T>(V, v, i, nI, d, U);
}

template <typename T, int W>
__global__ void __launch_bounds__(MF_T) k_mf_bwd_part(MFView V, const int32_t* __restrict__ nodes, int rb_max, int cs,
                                                     const T* __restrict__ Xall, const T* __restrict__ c,
                                                     T* __restrict__ part) {
    constexpr int RB = 32 * W;
    extern __shared__ unsigned char mf_smem[];
    T* sred = reinterpret_cast<T*>(mf_smem);
    T* xb = sred + (MF_WARPS + 1) * RB;
    const int cc = blockIdx.x % cs, rest = blockIdx.x / cs;
    const int q = rest / rb_max, rb = rest % rb_max;
    const int v = nodes[q];
    const int m = V.m[v], nI = V.nI[v], nB = m - nI;
    if (rb * RB >= nI) return;
    const int chunk = (nB + cs - 1) / cs;
    const int j0 = min(nB, cc * chunk), j1 = min(nB, j0 + chunk);
    const int32_t* gl = V.glob + V.offP[v];
    for (int j = j0 + (int)threadIdx.x; j < j1; j += blockDim.x) xb[j - j0] = c[gl[nI + j]];
    __syncthreads();
    const int64_t ld = mf_ld(nI);
    block_colmajor_gemv<T, W>(Xall + V.offX[v] + (int64_t)j0 * ld, ld, nI, j1 - j0, xb, rb, sred);
    const T* res = sred + MF_WARPS * RB;
    T* out = part + (int64_t)blockIdx.x * RB;
    for (int r = threadIdx.x; r < RB; r += blockDim.x) out[r] = res[r];
}

template <typename T>
__global__ void k_mf_bwd_fin(MFView V, const int32_t* __restrict__ nodes, int cnt, int rb_max, int RB, int cs,
                             const T* __restrict__ part, const T* __restrict__ Y, T* __restrict__ c) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)cnt * rb_max * RB) return;
    const int r = (int)(t % RB);
    const int64_t rest = t / RB;
    const int rb = (int)(rest % rb_max), q = (int)(rest / rb_max);
    const int v = nodes[q];
    const int nI = V.nI[v], i = rb * RB + r;
    if (i >= nI) return;
    const T* p = part + ((int64_t)q * rb_max + rb) * cs * RB + r;
    T s = T(0);
    for (int k = 0; k < cs; ++k) s += p[(int64_t)k * RB];
    c[V.glob[V.offP[v] + i]] = Y[V.offY[v] + i] - s;
}

__global__ void k_mf_to_f32(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

template <class T>
hho_status mf_upload(hho_ctx* ctx, T** dst, const std::vector<T>& v) {
    HHO_TRY(dalloc(ctx, dst, std::max<size_t>(v.size(), 1)));
    if (!v.empty()) HHO_CUDA(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return HHO_OK;
}

}  // namespace

struct MFSolver {
    int nnodes = 0;
    std::vector<int32_t> h_level_ptr, h_level_nodes;  // nodes grouped by height (leaves first)
    std::vector<int> level_rbf64, level_rbf32, level_rbb64, level_rbb32;  // row blocks per node per level
    std::vector<int> level_mmax, level_nBmax, level_nImax;
    int32_t *m = nullptr, *nI = nullptr, *child = nullptr, *pin = nullptr, *glob = nullptr, *cpos = nullptr,
            *level_nodes = nullptr, *leaf_elem_ptr = nullptr, *leaf_elem = nullptr, *elem_loc = nullptr;
    int64_t *offW = nullptr, *offM1 = nullptr, *offX = nullptr, *offP = nullptr, *offY = nullptr, *offU = nullptr,
            *elem_loc_off = nullptr;
    double* alpha = nullptr;
    int64_t nM1 = 0, nX = 0, nY = 0, nU = 0;
    double *M1 = nullptr, *X = nullptr, *Y = nullptr, *U = nullptr;
    float *M1f = nullptr, *Xf = nullptr, *Yf = nullptr, *Uf = nullptr;
    size_t smem_fwd64 = 0, smem_fwd32 = 0, smem_bwd64 = 0, smem_bwd32 = 0;
    int64_t factor_doubles = 0;  // workspace used by the factorisation (freed after it)
    // partial products of the column-split levels (see k_mf_fwd_part), FP64 and FP32
    int64_t npart64 = 0, npart32 = 0;
    double* part64 = nullptr;
    float* part32 = nullptr;
    MFView view() const {
        MFView V{};
        V.m = m;
        V.nI = nI;
        V.child = child;
        V.pin = pin;
        V.offW = nullptr;
        V.offM1 = offM1;
        V.offX = offX;
        V.offP = offP;
        V.offY = offY;
        V.offU = offU;
        V.glob = glob;
        V.cpos = cpos;
        V.leaf_elem_ptr = leaf_elem_ptr;
        V.leaf_elem = leaf_elem;
        V.elem_loc_off = elem_loc_off;
        V.elem_loc = elem_loc;
        V.alpha = alpha;
        V.ec = 1;
        return V;
    }
};

// Launch shape of one solve step on a tree level of cnt nodes with `rows` rows
// and `cols` columns per node (the largest): rb row blocks of 32 W rows per
// node; levels with at least 2 CTAs per SM use them as they are (cs = 1,
// wide), smaller ones split the columns into cs chunks of at least 32 columns
// for about 4 CTAs per SM (cs > 1), or, when the columns are too few for that,
// take one row per lane (wide = false).
struct MFShape {
    int rb, cs;
    bool wide;
};
static MFShape mf_shape(int64_t cnt, int rows, int cols, int W) {
    MFShape sh;
    sh.rb = (rows + 32 * W - 1) / (32 * W);
    sh.cs = 1;
    sh.wide = true;
    const int64_t nsm = sm_count();
    if (rows == 0 || cnt * sh.rb >= 2 * nsm) return sh;
    const int64_t want = (4 * nsm + cnt * sh.rb - 1) / (cnt * sh.rb);
    const int64_t cap = std::max<int64_t>(1, cols / 32);
    sh.cs = (int)std::min(want, cap);
    if (sh.cs == 1) {
        sh.wide = false;
        sh.rb = (rows + 31) / 32;
    }
    return sh;
}

void mf_free(MFSolver* S) {
    if (!S) return;
    void* ps[] = {S->m, S->nI, S->child, S->pin, S->glob, S->cpos, S->level_nodes, S->leaf_elem_ptr, S->leaf_elem,
                  S->elem_loc, S->offW, S->offM1, S->offX, S->offP, S->offY, S->offU, S->elem_loc_off, S->alpha,
                  S->M1, S->X, S->Y, S->U, S->M1f, S->Xf, S->Yf, S->Uf, S->part64, S->part32};
    for (void* p : ps) dfree(p);
    delete S;
}

namespace {

struct HostNode {
    int parent = -1, child[2] = {-1, -1}, height = 0, depth = 0, prob = 0;
    int64_t e0 = 0, e1 = 0;  // range in the element permutation
    std::vector<int32_t> I, B;
    int pin = -1;
};

// Recursive coordinate bisection; returns the node index.
int mf_split(std::vector<HostNode>& nodes, std::vector<int32_t>& perm, int64_t lo, int64_t hi, int parent, int depth,
             int prob, int64_t leaf, const std::vector<double>& cen, int d) {
    const int id = (int)nodes.size();
    nodes.emplace_back();
    nodes[id].parent = parent;
    nodes[id].depth = depth;
    nodes[id].prob = prob;
    nodes[id].e0 = lo;
    nodes[id].e1 = hi;
    if (hi - lo <= leaf) return id;
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = lo; i < hi; ++i)
        for (int j = 0; j < d; ++j) {
            mn[j] = std::min(mn[j], cen[(size_t)perm[i] * d + j]);
            mx[j] = std::max(mx[j], cen[(size_t)perm[i] * d + j]);
        }
    int ax = 0;
    for (int j = 1; j < d; ++j)
        if (mx[j] - mn[j] > mx[ax] - mn[ax]) ax = j;
    std::stable_sort(perm.begin() + lo, perm.begin() + hi, [&](int32_t a, int32_t b) {
        const double ca = cen[(size_t)a * d + ax], cb = cen[(size_t)b * d + ax];
        return ca < cb || (ca == cb && a < b);
    });
    const int64_t mid = lo + (hi - lo) / 2;
    const int c0 = mf_split(nodes, perm, lo, mid, id, depth + 1, prob, leaf, cen, d);
    const int c1 = mf_split(nodes, perm, mid, hi, id, depth + 1, prob, leaf, cen, d);
    nodes[id].child[0] = c0;
    nodes[id].child[1] = c1;
    nodes[id].height = 1 + std::max(nodes[c0].height, nodes[c1].height);
    return id;
}

int64_t pos_in(const std::vector<int32_t>& sorted, int32_t g) {
    auto it = std::lower_bound(sorted.begin(), sorted.end(), g);
    return (it != sorted.end() && *it == g) ? (int64_t)(it - sorted.begin()) : -1;
}

}  // namespace

// Build and factor the multifrontal solver of the coarse level.  leaf: target
// elements per leaf.  project_null: problems with a pressure kernel get a pin.
hho_status mf_build(hho_ctx* ctx, int64_t leaf, MFSolver** out) {
    *out = nullptr;
    const Disc& D = ctx->disc;
    const LevelMat& L = ctx->levels.back();
    const int d = D.d;
    const int64_t ne = D.ne, nf = D.nf;
    const int bL = L.b, nPL = L.nP;
    const int pm = mean_slot(D.cond, d, nPL);  // the constant pressure mode in an element block
    const Problems& pr = ctx->probs;
    // element centroids (vertex averages)
    std::vector<double> cen((size_t)ne * d, 0.0);
    for (int64_t T = 0; T < ne; ++T) {
        std::vector<int32_t> vs;
        for (int i = D.h_ef_ptr[T]; i < D.h_ef_ptr[T + 1]; ++i) {
            const int F = D.h_ef[i];
            for (int v = D.h_fv_ptr[F]; v < D.h_fv_ptr[F + 1]; ++v) vs.push_back(D.h_fv[v]);
        }
        std::sort(vs.begin(), vs.end());
        vs.erase(std::unique(vs.begin(), vs.end()), vs.end());
        for (int32_t v : vs)
            for (int j = 0; j < d; ++j) cen[(size_t)T * d + j] += D.h_xyz[(size_t)v * d + j];
        for (int j = 0; j < d; ++j) cen[(size_t)T * d + j] /= (double)vs.size();
    }
    // elimination forest: one tree per problem
    std::vector<HostNode> nodes;
    std::vector<int32_t> perm(ne);
    std::iota(perm.begin(), perm.end(), 0);
    std::vector<int> roots;
    for (int q = 0; q < pr.P; ++q)
        roots.push_back(mf_split(nodes, perm, pr.elem_off[q], pr.elem_off[q + 1], -1, 0, q, std::max<int64_t>(leaf, 1),
                                 cen, d));
    const int nn = (int)nodes.size();
    std::vector<int32_t> leaf_of(ne, -1);
    for (int v = 0; v < nn; ++v)
        if (nodes[v].child[0] < 0)
            for (int64_t i = nodes[v].e0; i < nodes[v].e1; ++i) leaf_of[perm[i]] = v;
    auto lca = [&](int a, int b) {
        while (nodes[a].depth > nodes[b].depth) a = nodes[a].parent;
        while (nodes[b].depth > nodes[a].depth) b = nodes[b].parent;
        while (a != b) {
            a = nodes[a].parent;
            b = nodes[b].parent;
        }
        return a;
    };
    std::vector<int32_t> face_owner(nf);
    for (int64_t F = 0; F < nf; ++F) {
        const int T1 = D.h_fe[2 * F], T2 = D.h_fe[2 * F + 1];
        face_owner[F] = T2 < 0 ? leaf_of[T1] : lca(leaf_of[T1], leaf_of[T2]);
    }
    // nodes by height; pressure owners by union-find over the faces owned so far
    int hmax = 0;
    for (const HostNode& nd : nodes) hmax = std::max(hmax, nd.height);
    std::vector<std::vector<int>> by_h(hmax + 1);
    for (int v = 0; v < nn; ++v) by_h[nodes[v].height].push_back(v);
    std::vector<std::vector<int64_t>> owned_faces(nn);
    for (int64_t F = 0; F < nf; ++F) owned_faces[face_owner[F]].push_back(F);
    std::vector<int32_t> uf(ne);
    std::iota(uf.begin(), uf.end(), 0);
    auto find = [&](int32_t a) {
        while (uf[a] != a) {
            uf[a] = uf[uf[a]];
            a = uf[a];
        }
        return a;
    };
    std::vector<int32_t> p_owner(ne, -1);
    for (int h = 0; h <= hmax; ++h)
        for (int v : by_h[h]) {
            for (int64_t F : owned_faces[v]) {
                const int T2 = D.h_fe[2 * F + 1];
                if (T2 < 0) continue;
                const int a = find(D.h_fe[2 * F]), b = find(T2);
                if (a != b) uf[std::max(a, b)] = std::min(a, b);
            }
            for (int64_t i = nodes[v].e0; i < nodes[v].e1; ++i) {
                const int32_t T = perm[i];
                if (p_owner[T] < 0 && find(T) != T) p_owner[T] = v;
            }
        }
    for (int64_t T = 0; T < ne; ++T)
        if (p_owner[T] < 0) p_owner[T] = roots[pr.elem_prob[T]];
    // I and B sets (global coarse indices, sorted)
    auto in_subtree = [&](int o, int v) { return nodes[o].e0 >= nodes[v].e0 && nodes[o].e1 <= nodes[v].e1 &&
                                                 nodes[o].depth >= nodes[v].depth; };
    const int64_t pbase = nf * bL;
    for (int v = 0; v < nn; ++v) {
        HostNode& nd = nodes[v];
        for (int64_t F : owned_faces[v])
            for (int r = 0; r < bL; ++r) nd.I.push_back((int32_t)(F * bL + r));
        std::vector<int64_t> bfaces;
        for (int64_t i = nd.e0; i < nd.e1; ++i) {
            const int32_t T = perm[i];
            if (nd.child[0] < 0)
                for (int c = 0; c < nPL; ++c)
                    if (c != pm) nd.I.push_back((int32_t)(pbase + (int64_t)T * nPL + c));
            if (nPL > 0) {  // HHO-hp has no element rows
                if (p_owner[T] == v) nd.I.push_back((int32_t)(pbase + (int64_t)T * nPL + pm));
                else if (!in_subtree(p_owner[T], v)) nd.B.push_back((int32_t)(pbase + (int64_t)T * nPL + pm));
            }
            for (int q = D.h_ef_ptr[T]; q < D.h_ef_ptr[T + 1]; ++q) {
                const int F = D.h_ef[q];
                if (!in_subtree(face_owner[F], v)) bfaces.push_back(F);
            }
        }
        std::sort(bfaces.begin(), bfaces.end());
        bfaces.erase(std::unique(bfaces.begin(), bfaces.end()), bfaces.end());
        for (int64_t F : bfaces)
            for (int r = 0; r < bL; ++r) nd.B.push_back((int32_t)(F * bL + r));
        std::sort(nd.I.begin(), nd.I.end());
        std::sort(nd.B.begin(), nd.B.end());
    }
    for (int rt : roots)
        if (!nodes[rt].B.empty()) {
            ctx->err = "pmg_setup: multifrontal coarse solver: a root has boundary unknowns";
            return HHO_ERR_MESH;
        }
    // pins: the root's kept pressure of every problem with a pressure kernel
    // (HHO-hp: the constant face-pressure coefficient of the first face the root
    // eliminates; the kernel vector is non-zero there)
    for (int q = 0; q < pr.P; ++q) {
        if (!ctx->has_null || !pr.has_null[q]) continue;
        HostNode& rt = nodes[roots[q]];
        int32_t g = -1;
        if (nPL == 0) {
            if (!owned_faces[roots[q]].empty()) g = (int32_t)(owned_faces[roots[q]][0] * bL + (int64_t)d * L.nF);
        } else {
            for (int64_t i = rt.e0; i < rt.e1 && g < 0; ++i)
                if (p_owner[perm[i]] == roots[q]) g = (int32_t)(pbase + (int64_t)perm[i] * nPL + pm);
        }
        if (g < 0) {
            ctx->err = "pmg_setup: multifrontal coarse solver: no kept pressure at a root";
            return HHO_ERR_MESH;
        }
        rt.pin = (int)pos_in(rt.I, g);
    }
    // every unknown eliminated exactly once
    {
        std::vector<char> seen((size_t)L.n, 0);
        for (const HostNode& nd : nodes)
            for (int32_t g : nd.I) {
                if (g < 0 || g >= L.n || seen[g]) {
                    ctx->err = "pmg_setup: multifrontal coarse solver: inconsistent elimination sets";
                    return HHO_ERR_MESH;
                }
                seen[g] = 1;
            }
        for (int64_t g = 0; g < L.n; ++g)
            if (!seen[g]) {
                ctx->err = "pmg_setup: multifrontal coarse solver: an unknown is never eliminated";
                return HHO_ERR_MESH;
            }
    }
    // flat device arrays
    MFSolver* S = new MFSolver();
    S->nnodes = nn;
    std::vector<int32_t> h_m(nn), h_nI(nn), h_child(2 * nn), h_pin(nn), h_glob, h_cpos, h_leaf_ptr(nn + 1, 0),
        h_leaf_elem, h_elem_loc;
    std::vector<int64_t> h_offW(nn), h_offM1(nn), h_offX(nn), h_offP(nn), h_offY(nn), h_offU(nn), h_elem_loc_off(ne, 0);
    int64_t tW = 0, tM1 = 0, tX = 0, tP = 0, tY = 0, tU = 0;
    for (int v = 0; v < nn; ++v) {
        const HostNode& nd = nodes[v];
        const int m = (int)(nd.I.size() + nd.B.size()), nIv = (int)nd.I.size();
        h_m[v] = m;
        h_nI[v] = nIv;
        h_child[2 * v] = nd.child[0];
        h_child[2 * v + 1] = nd.child[1];
        h_pin[v] = nd.pin;
        h_offW[v] = tW;
        tW += (int64_t)m * (m + nIv);
        h_offM1[v] = tM1;
        tM1 += mf_ld(m) * nIv;
        h_offX[v] = tX;
        tX += mf_ld(nIv) * (m - nIv);
        h_offP[v] = tP;
        tP += m;
        h_offY[v] = tY;
        tY += nIv;
        h_offU[v] = tU;
        tU += m - nIv;
        for (int32_t g : nd.I) h_glob.push_back(g);
        for (int32_t g : nd.B) h_glob.push_back(g);
        // positions of every front entry in the children's B sets
        for (int i = 0; i < m; ++i) {
            const int32_t g = i < nIv ? nd.I[i] : nd.B[i - nIv];
            for (int q = 0; q < 2; ++q) {
                const int c = nd.child[q];
                h_cpos.push_back(c < 0 ? -1 : (int32_t)pos_in(nodes[c].B, g));
            }
        }
        if (nd.child[0] < 0) {
            for (int64_t i = nd.e0; i < nd.e1; ++i) h_leaf_elem.push_back(perm[i]);
        }
        h_leaf_ptr[v + 1] = (int32_t)h_leaf_elem.size();
    }
    // children's B sets must map into the parent's front
    for (int v = 0; v < nn; ++v)
        for (int q = 0; q < 2; ++q) {
            const int c = nodes[v].child[q];
            if (c < 0) continue;
            int64_t hits = 0;
            for (int i = 0; i < h_m[v]; ++i) hits += h_cpos[2 * (h_offP[v] + i) + q] >= 0;
            if (hits != (int64_t)nodes[c].B.size()) {
                delete S;
                ctx->err = "pmg_setup: multifrontal coarse solver: a child's boundary is not in its parent's front";
                return HHO_ERR_MESH;
            }
        }
    // leaf element maps
    {
        int64_t o = 0;
        for (int64_t T = 0; T < ne; ++T) {
            h_elem_loc_off[T] = o;
            o += (int64_t)(D.h_ef_ptr[T + 1] - D.h_ef_ptr[T]) * bL + nPL;
        }
        h_elem_loc.assign(o, -1);
        for (int v = 0; v < nn; ++v) {
            const HostNode& nd = nodes[v];
            if (nd.child[0] >= 0) continue;
            auto front_pos = [&](int32_t g) -> int32_t {
                int64_t p = pos_in(nd.I, g);
                if (p >= 0) return (int32_t)p;
                p = pos_in(nd.B, g);
                return p >= 0 ? (int32_t)(nd.I.size() + p) : -1;
            };
            for (int64_t i = nd.e0; i < nd.e1; ++i) {
                const int32_t T = perm[i];
                const int N = D.h_ef_ptr[T + 1] - D.h_ef_ptr[T];
                int32_t* lo = h_elem_loc.data() + h_elem_loc_off[T];
                for (int f = 0; f < N; ++f) {
                    const int F = D.h_ef[D.h_ef_ptr[T] + f];
                    for (int r = 0; r < bL; ++r) lo[f * bL + r] = front_pos((int32_t)(F * bL + r));
                }
                for (int c = 0; c < nPL; ++c) lo[N * bL + c] = front_pos((int32_t)(pbase + (int64_t)T * nPL + c));
            }
        }
        for (int32_t x : h_elem_loc)
            if (x < 0) {
                delete S;
                ctx->err = "pmg_setup: multifrontal coarse solver: inconsistent leaf maps";
                return HHO_ERR_MESH;
            }
    }
    // levels (heights), their sizes and row blocks of the solve kernels
    S->h_level_ptr.assign(1, 0);
    for (int h = 0; h <= hmax; ++h) {
        int mmax = 0, nBmax = 0, nImax = 0;
        for (int v : by_h[h]) {
            S->h_level_nodes.push_back(v);
            mmax = std::max(mmax, h_m[v]);
            nImax = std::max(nImax, h_nI[v]);
            nBmax = std::max(nBmax, h_m[v] - h_nI[v]);
        }
        S->h_level_ptr.push_back((int32_t)S->h_level_nodes.size());
        S->level_mmax.push_back(mmax);
        S->level_nBmax.push_back(nBmax);
        S->level_nImax.push_back(nImax);
        S->level_rbf64.push_back((mmax + 63) / 64);
        S->level_rbf32.push_back((mmax + 127) / 128);
        S->level_rbb64.push_back((nImax + 63) / 64);
        S->level_rbb32.push_back((nImax + 127) / 128);
        S->smem_fwd64 = std::max(S->smem_fwd64, (size_t)((MF_WARPS + 1) * 64 + mmax) * 8);
        S->smem_fwd32 = std::max(S->smem_fwd32, (size_t)((MF_WARPS + 1) * 128 + mmax) * 4);
        S->smem_bwd64 = std::max(S->smem_bwd64, (size_t)((MF_WARPS + 1) * 64 + nBmax) * 8);
        S->smem_bwd32 = std::max(S->smem_bwd32, (size_t)((MF_WARPS + 1) * 128 + nBmax) * 4);
    }
    // partial-product buffers of the column-split levels (one level at a time)
    for (int h = 0; h <= hmax; ++h) {
        const int64_t cnt = S->h_level_ptr[h + 1] - S->h_level_ptr[h];
        for (int W : {2, 4}) {
            const MFShape f = mf_shape(cnt, S->level_mmax[h], S->level_nImax[h], W);
            const MFShape b = mf_shape(cnt, S->level_nImax[h], S->level_nBmax[h], W);
            int64_t need = 0;
            if (f.cs > 1) need = std::max<int64_t>(need, cnt * f.rb * f.cs * 32 * W);
            if (b.cs > 1) need = std::max<int64_t>(need, cnt * b.rb * b.cs * 32 * W);
            int64_t& slot = (W == 2) ? S->npart64 : S->npart32;
            slot = std::max(slot, need);
        }
    }
    const size_t smem_cap = (size_t)smem_optin();
    if (S->smem_fwd64 > smem_cap || S->smem_bwd64 > smem_cap) {
        delete S;
        ctx->err = "pmg_setup: multifrontal coarse solver: a front exceeds the shared-memory staging of the solve";
        return HHO_ERR_UNSUPPORTED;
    }
    *out = S;
    HHO_TRY(mf_upload(ctx, &S->m, h_m));
    HHO_TRY(mf_upload(ctx, &S->nI, h_nI));
    HHO_TRY(mf_upload(ctx, &S->child, h_child));
    HHO_TRY(mf_upload(ctx, &S->pin, h_pin));
    HHO_TRY(mf_upload(ctx, &S->glob, h_glob));
    HHO_TRY(mf_upload(ctx, &S->cpos, h_cpos));
    HHO_TRY(mf_upload(ctx, &S->level_nodes, S->h_level_nodes));
    HHO_TRY(mf_upload(ctx, &S->leaf_elem_ptr, h_leaf_ptr));
    HHO_TRY(mf_upload(ctx, &S->leaf_elem, h_leaf_elem));
    HHO_TRY(mf_upload(ctx, &S->elem_loc, h_elem_loc));
    HHO_TRY(mf_upload(ctx, &S->offW, h_offW));
    HHO_TRY(mf_upload(ctx, &S->offM1, h_offM1));
    HHO_TRY(mf_upload(ctx, &S->offX, h_offX));
    HHO_TRY(mf_upload(ctx, &S->offP, h_offP));
    HHO_TRY(mf_upload(ctx, &S->offY, h_offY));
    HHO_TRY(mf_upload(ctx, &S->offU, h_offU));
    HHO_TRY(mf_upload(ctx, &S->elem_loc_off, h_elem_loc_off));
    HHO_TRY(dalloc(ctx, &S->alpha, 1));
    HHO_TRY(dalloc(ctx, &S->part64, (size_t)std::max<int64_t>(S->npart64, 1)));
    S->nM1 = tM1;
    S->nX = tX;
    S->nY = tY;
    S->nU = tU;
    HHO_TRY(dalloc(ctx, &S->M1, (size_t)std::max<int64_t>(tM1, 1)));
    HHO_TRY(dalloc(ctx, &S->X, (size_t)std::max<int64_t>(tX, 1)));
    HHO_TRY(dalloc(ctx, &S->Y, (size_t)std::max<int64_t>(tY, 1)));
    HHO_TRY(dalloc(ctx, &S->U, (size_t)std::max<int64_t>(tU, 1)));
    S->factor_doubles = tW;
    double* Wall = nullptr;
    HHO_TRY(dalloc(ctx, &Wall, (size_t)std::max<int64_t>(tW, 1)));
    // factorisation, level by level
    MFView V = S->view();
    V.offW = S->offW;
    V.ef_ptr = D.ef_ptr;
    V.off_S = D.off_S;
    V.S = D.S;
    V.b0 = D.b;
    V.nF0 = D.nF;
    V.nP0 = D.nP;
    V.bL = bL;
    V.nFL = L.nF;
    V.nPL = nPL;
    V.ec = elem_comp(D.cond, d);
    if (ctx->has_null) k_mf_mean_abs_diag<<<1, MF_T, 0, ctx->stream>>>(L.nf, L.ne, L.b, L.nP, L.ff, L.pp, S->alpha);
    else HHO_CUDA(cudaMemsetAsync(S->alpha, 0, sizeof(double), ctx->stream));
    HHO_CUDA(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream));
    double* colbuf = nullptr;
    int64_t* d_coloff = nullptr;
    hho_status st = HHO_OK;
    const int nsm = sm_count();
    for (int h = 0; h <= hmax && st == HHO_OK; ++h) {
        const int l0 = S->h_level_ptr[h], cnt = S->h_level_ptr[h + 1] - l0;
        const int32_t* lnodes = S->level_nodes + l0;
        int nImax = 0;
        for (int q = 0; q < cnt; ++q) nImax = std::max(nImax, h_nI[S->h_level_nodes[l0 + q]]);
        if (h == 0 || cnt >= nsm) {
            k_mf_factor_cta<<<cnt, MF_T, 0, ctx->stream>>>(V, lnodes, cnt, Wall, S->M1, S->X, ctx->d_flag);
            if (cudaGetLastError() != cudaSuccess) st = HHO_ERR_CUDA;
            continue;
        }
        // few large fronts: every SM on every pivot column
        int64_t wmax = 0, mmax = 0;
        std::vector<int64_t> coloff(cnt + 1, 0);
        for (int q = 0; q < cnt; ++q) {
            const int v = S->h_level_nodes[l0 + q];
            wmax = std::max<int64_t>(wmax, (int64_t)h_m[v] * (h_m[v] + h_nI[v]));
            mmax = std::max<int64_t>(mmax, h_m[v]);
            coloff[q + 1] = coloff[q] + h_m[v];
        }
        dfree(colbuf);
        dfree(d_coloff);
        colbuf = nullptr;
        d_coloff = nullptr;
        if ((st = dalloc(ctx, &colbuf, (size_t)coloff[cnt])) != HHO_OK) break;
        if ((st = mf_upload(ctx, &d_coloff, coloff)) != HHO_OK) break;
        const int gx = (int)std::max<int64_t>(1, std::min<int64_t>((wmax + MF_T - 1) / MF_T,
                                                                   (int64_t)std::max(1, 4 * nsm / cnt)));
        k_mf_assemble<<<dim3(gx, cnt), MF_T, 0, ctx->stream>>>(V, lnodes, Wall);
        const int ge = (int)std::max<int64_t>(1, std::min<int64_t>((mmax + MF_WARPS - 1) / MF_WARPS,
                                                                   (int64_t)std::max(1, 8 * nsm / cnt)));
        for (int j = 0; j < nImax; ++j) {
            k_mf_pivot<<<cnt, MF_T, 0, ctx->stream>>>(V, lnodes, j, Wall, colbuf, d_coloff, ctx->d_flag);
            k_mf_elim<<<dim3(ge, cnt), MF_T, 0, ctx->stream>>>(V, lnodes, j, Wall, colbuf, d_coloff);
        }
        k_mf_extract<<<dim3(gx, cnt), MF_T, 0, ctx->stream>>>(V, lnodes, Wall, S->M1, S->X);
        if (cudaGetLastError() != cudaSuccess) st = HHO_ERR_CUDA;
    }
    int flag = 0;
    cudaError_t ce = cudaMemcpyAsync(&flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    cudaError_t se = cudaStreamSynchronize(ctx->stream);
    dfree(Wall);
    dfree(colbuf);
    dfree(d_coloff);
    if (st == HHO_ERR_CUDA) {
        ctx->err = "pmg_setup: multifrontal coarse solver: kernel launch failed";
        return st;
    }
    HHO_TRY(st);
    HHO_CUDA(ce);
    HHO_CUDA(se);
    if (flag) {
        ctx->err = "pmg_setup: multifrontal coarse solver: singular front";
        return HHO_ERR_SINGULAR;
    }
    HHO_TRY(allow_smem(ctx, k_mf_fwd<double, 2>, S->smem_fwd64));
    HHO_TRY(allow_smem(ctx, k_mf_bwd<double, 2>, S->smem_bwd64));
    HHO_TRY(allow_smem(ctx, k_mf_fwd<float, 4>, S->smem_fwd32));
    HHO_TRY(allow_smem(ctx, k_mf_bwd<float, 4>, S->smem_bwd32));
    HHO_TRY(allow_smem(ctx, k_mf_fwd<double, 1>, S->smem_fwd64));
    HHO_TRY(allow_smem(ctx, k_mf_bwd<double, 1>, S->smem_bwd64));
    HHO_TRY(allow_smem(ctx, k_mf_fwd<float, 1>, S->smem_fwd32));
    HHO_TRY(allow_smem(ctx, k_mf_bwd<float, 1>, S->smem_bwd32));
    HHO_TRY(allow_smem(ctx, k_mf_fwd_part<double, 2>, S->smem_fwd64));
    HHO_TRY(allow_smem(ctx, k_mf_bwd_part<double, 2>, S->smem_bwd64));
    HHO_TRY(allow_smem(ctx, k_mf_fwd_part<float, 4>, S->smem_fwd32));
    HHO_TRY(allow_smem(ctx, k_mf_bwd_part<float, 4>, S->smem_bwd32));
    return HHO_OK;
}

hho_status mf_make_f32(hho_ctx* ctx, MFSolver* S) {
    if (S->M1f) return HHO_OK;
    HHO_TRY(dalloc(ctx, &S->M1f, (size_t)std::max<int64_t>(S->nM1, 1)));
    HHO_TRY(dalloc(ctx, &S->Xf, (size_t)std::max<int64_t>(S->nX, 1)));
    HHO_TRY(dalloc(ctx, &S->Yf, (size_t)std::max<int64_t>(S->nY, 1)));
    HHO_TRY(dalloc(ctx, &S->Uf, (size_t)std::max<int64_t>(S->nU, 1)));
    HHO_TRY(dalloc(ctx, &S->part32, (size_t)std::max<int64_t>(S->npart32, 1)));
    k_mf_to_f32<<<mf_grid(S->nM1), MF_T, 0, ctx->stream>>>(S->nM1, S->M1, S->M1f);
    k_mf_to_f32<<<mf_grid(S->nX), MF_T, 0, ctx->stream>>>(S->nX, S->X, S->Xf);
    HHO_CUDA(cudaGetLastError());
    return HHO_OK;
}

bool mf_has_f32(const MFSolver* S) { return S && S->M1f; }

int mf_levels(const MFSolver* S) { return (int)S->level_mmax.size(); }

int mf_launches(const MFSolver* S, int value_bytes) {
    const int W = value_bytes == 4 ? 4 : 2;
    int n = 0;
    for (size_t h = 0; h < S->level_mmax.size(); ++h) {
        const int64_t cnt = S->h_level_ptr[h + 1] - S->h_level_ptr[h];
        n += mf_shape(cnt, S->level_mmax[h], S->level_nImax[h], W).cs > 1 ? 2 : 1;
        if (S->level_nImax[h] > 0) n += mf_shape(cnt, S->level_nImax[h], S->level_nBmax[h], W).cs > 1 ? 2 : 1;
    }
    return n;
}

int64_t mf_factor_doubles(const MFSolver* S) { return S->factor_doubles; }

int64_t mf_solve_bytes(const MFSolver* S, int value_bytes) { return (S->nM1 + S->nX) * value_bytes; }

template <typename T>
hho_status mf_apply(hho_ctx* ctx, MFSolver* S, const T* d, T* c) {
    constexpr bool F32 = std::is_same<T, float>::value;
    constexpr int WW = mf_wide<T>();
    const T* M1 = F32 ? (const T*)S->M1f : (const T*)S->M1;
    const T* X = F32 ? (const T*)S->Xf : (const T*)S->X;
    T* Y = F32 ? (T*)S->Yf : (T*)S->Y;
    T* U = F32 ? (T*)S->Uf : (T*)S->U;
    const MFView V = S->view();
    const int H = (int)S->level_mmax.size();
    T* part = F32 ? (T*)S->part32 : (T*)S->part64;
    const size_t red1 = (size_t)(MF_WARPS + 1) * 32 * sizeof(T), redw = (size_t)(MF_WARPS + 1) * 32 * WW * sizeof(T);
    int launches = 0;
    for (int h = 0; h < H; ++h) {
        const int l0 = S->h_level_ptr[h], cnt = S->h_level_ptr[h + 1] - l0;
        const int mm = S->level_mmax[h];
        const MFShape sh = mf_shape(cnt, mm, S->level_nImax[h], WW);
        const unsigned g = (unsigned)((int64_t)cnt * sh.rb * sh.cs);
        if (sh.cs > 1) {
            const size_t vec = (size_t)((S->level_nImax[h] + sh.cs - 1) / sh.cs) * sizeof(T);
            k_mf_fwd_part<T, WW><<<g, MF_T, redw + vec, ctx->stream>>>(V, S->level_nodes + l0, sh.rb, sh.cs, M1, d, U,
                                                                       part);
            const int64_t nt = (int64_t)cnt * sh.rb * 32 * WW;
            k_mf_fwd_fin<T><<<(unsigned)((nt + 255) / 256), 256, 0, ctx->stream>>>(V, S->level_nodes + l0, cnt, sh.rb,
                                                                                    32 * WW, sh.cs, part, d, Y, U);
            launches += 2;
        } else {
            const size_t vec = (size_t)mm * sizeof(T);
            if (sh.wide)
                k_mf_fwd<T, WW><<<g, MF_T, redw + vec, ctx->stream>>>(V, S->level_nodes + l0, sh.rb, M1, d, Y, U);
            else
                k_mf_fwd<T, 1><<<g, MF_T, red1 + vec, ctx->stream>>>(V, S->level_nodes + l0, sh.rb, M1, d, Y, U);
            launches += 1;
        }
    }
    for (int h = H - 1; h >= 0; --h) {
        const int l0 = S->h_level_ptr[h], cnt = S->h_level_ptr[h + 1] - l0;
        const int nImax = S->level_nImax[h];
        if (nImax == 0) continue;
        const MFShape sh = mf_shape(cnt, nImax, S->level_nBmax[h], WW);
        const unsigned g = (unsigned)((int64_t)cnt * sh.rb * sh.cs);
        if (sh.cs > 1) {
            const size_t vec = (size_t)((S->level_nBmax[h] + sh.cs - 1) / sh.cs) * sizeof(T);
            k_mf_bwd_part<T, WW><<<g, MF_T, redw + vec, ctx->stream>>>(V, S->level_nodes + l0, sh.rb, sh.cs, X, c,
                                                                       part);
            const int64_t nt = (int64_t)cnt * sh.rb * 32 * WW;
            k_mf_bwd_fin<T><<<(unsigned)((nt + 255) / 256), 256, 0, ctx->stream>>>(V, S->level_nodes + l0, cnt, sh.rb,
                                                                                    32 * WW, sh.cs, part, Y, c);
            launches += 2;
        } else {
            const size_t vec = (size_t)S->level_nBmax[h] * sizeof(T);
            if (sh.wide)
                k_mf_bwd<T, WW><<<g, MF_T, redw + vec, ctx->stream>>>(V, S->level_nodes + l0, sh.rb, X, Y, c);
            else
                k_mf_bwd<T, 1><<<g, MF_T, red1 + vec, ctx->stream>>>(V, S->level_nodes + l0, sh.rb, X, Y, c);
            launches += 1;
        }
    }
    ctx->launches += launches;
    HHO_CUDA(cudaGetLastError());
    return HHO_OK;
}
template hho_status mf_apply<double>(hho_ctx*, MFSolver*, const double*, double*);
template hho_status mf_apply<float>(hho_ctx*, MFSolver*, const float*, float*);

}  // namespace hho
