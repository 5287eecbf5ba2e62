// Krylov building blocks shared by the solver translation units: the scalar
// area of one GMRES instance (Hessenberg matrix, Givens rotations, residual
// estimates), the scalar recurrences run once a kernel's reductions are final
// (the "hooks"), and per-block helpers.  Every includer gets its own copy
// (anonymous namespace).
#pragma once

#include <cstdint>

namespace hho {
namespace {

constexpr int MMAX = 64;  // largest GMRES restart

// Scalar area of one GMRES instance with restart m.
//   [0] beta^2  [1] beta  [2] m_eff  [3] residual estimate  [4] breakdown  [5] norm of the pending w
//   H (m+1) x m column-major, cs[m], sn[m], g[m+1], t1[m+1], t2[m+1], nrm
struct GS {
    int m, H, cs, sn, g, t1, t2, nrm, total;
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
    s.t1 = o;
    o += m + 1;
    s.t2 = o;
    o += m + 1;
    s.nrm = o;
    o += 1;
    s.total = o;
    return s;
}

enum Hook { HOOK_NONE = 0, HOOK_START = 1, HOOK_COLUMN = 2, HOOK_COLUMN_PY = 3, HOOK_COLUMN_1R = 4 };

// Type of the per-thread and per-warp part of a dot product: FP32 inside the
// FP32 V-cycle (FP64 arithmetic is a narrow pipe on this part), FP64 otherwise.
template <typename T>
struct AccT {
    using type = double;
};
template <>
struct AccT<float> {
    using type = float;
};


// 1 / *den (0 when *den is 0) computed once per block: divisions, FP64 ones in
// particular, are costly per thread.  Call from all threads of the block.
template <typename T>
__device__ __forceinline__ T block_inverse(const double* __restrict__ den) {
    __shared__ T s_inv;
    if (threadIdx.x == 0) {
        const T dv = (T)*den;
        s_inv = (dv == T(0)) ? T(0) : T(1) / dv;
    }
    __syncthreads();
    return s_inv;
}

// Coefficients of a pending second Gram-Schmidt pass (FP64 storage) staged in
// shared memory in the level type.  Call from all threads of the block.
template <typename T>
__device__ __forceinline__ const T* stage_pending(const double* __restrict__ pc, int npend) {
    __shared__ T s_pc[MMAX];
    for (int q = threadIdx.x; q < npend; q += blockDim.x) s_pc[q] = (T)pc[q];
    __syncthreads();
    return s_pc;
}

// w''[o] = w'[o] - sum_{q < npend} pc_q Vp_q[o]: the second pass of the last
// Arnoldi step, applied where w'' is consumed
template <typename T>
__device__ __forceinline__ T pending(const T* __restrict__ w, const T* __restrict__ Vp, int64_t ld, int npend,
                                     const T* s_pc, int64_t o) {
    T u = w[o];
    for (int q = 0; q < npend; ++q) u -= s_pc[q] * Vp[q * ld + o];
    return u;
}

// Scalar work once the reductions of a kernel are final, run by the whole last
// block: the operands are first staged in shared memory by all threads in one
// round of loads, then one thread does the short serial recurrence there, in
// the arithmetic type A of the kernel (FP32 for the FP32 V-cycle: FP64
// arithmetic is scarce on this part, and storage stays FP64).
//   START   fresh = ||r||^2: beta, residual estimate, g = beta e_1
//   COLUMN  fresh = ||w||^2 after the second projection: Hessenberg column j
//           (t1 + t2, ||w||), the earlier Givens rotations applied to it, the
//           new rotation, and the updated residual estimate |g_{j+1}|
//   COLUMN_PY  the same with fresh = ||w'||^2 before the second projection
//           w'' = w' - V t2 (t2 = V^T w'), which is left to the consumer of
//           w'': ||w''||^2 = ||w'||^2 - ||t2||^2 for orthonormal V (the
//           correction t2 is small against w', so the difference is benign)
//   COLUMN_1R  one-reduction classical Gram-Schmidt: t2 = V^T w of the
//           unprojected w (the only pass, t1 unused), fresh = ||w||^2; the
//           column is t2 with ||w - V t2||^2 = ||w||^2 - ||t2||^2, and the
//           projection w - V t2 is left to the consumer
template <typename A>
__device__ __forceinline__ void run_hook(int hook, double* sc, GS L, int j, A fresh) {
    __shared__ A s_h[MMAX + 2], s_cs[MMAX], s_sn[MMAX], s_misc[2];
    if (hook == HOOK_START) {
        const A beta = sqrt(fresh);
        for (int i = threadIdx.x; i <= L.m; i += blockDim.x) sc[L.g + i] = (i == 0) ? (double)beta : 0.0;
        if (threadIdx.x == 0) {
            sc[1] = beta;
            sc[2] = 0.0;
            sc[3] = beta;
            sc[4] = (beta == A(0)) ? 1.0 : 0.0;
            sc[5] = beta;
        }
        return;
    }
    if (hook != HOOK_COLUMN && hook != HOOK_COLUMN_PY && hook != HOOK_COLUMN_1R) return;
    const int ld = L.m + 1;
    double* H = sc + L.H;
    __shared__ A s_t2sq[MMAX + 1];
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        const A t2 = (A)sc[L.t2 + i];
        s_h[i] = (hook == HOOK_COLUMN_1R) ? t2 : (A)sc[L.t1 + i] + t2;
        s_t2sq[i] = t2 * t2;
        if (i < j) {
            s_cs[i] = (A)sc[L.cs + i];
            s_sn[i] = (A)sc[L.sn + i];
        }
    }
    if (threadIdx.x == 0) {
        s_misc[0] = (A)sc[4];
        s_misc[1] = (A)sc[L.g + j];
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    if (s_misc[0] != A(0)) {  // after a breakdown the remaining columns are ignored
        for (int i = 0; i <= L.m; ++i) H[j * ld + i] = 0.0;
        sc[5] = 0.0;
        return;
    }
    A hn2 = fresh;
    if (hook == HOOK_COLUMN_PY || hook == HOOK_COLUMN_1R) {
        for (int i = 0; i <= j; ++i) hn2 -= s_t2sq[i];
        hn2 = hn2 > A(0) ? hn2 : A(0);
    }
    const A hn = sqrt(hn2);
    s_h[j + 1] = hn;
    sc[5] = hn;
    for (int i = 0; i < j; ++i) {
        const A c = s_cs[i], s = s_sn[i];
        const A a = s_h[i], bb = s_h[i + 1];
        s_h[i] = c * a + s * bb;
        s_h[i + 1] = -s * a + c * bb;
    }
    const A a = s_h[j], bb = s_h[j + 1];
    const A r = hypot(a, bb);
    const A c = (r == A(0)) ? A(1) : a / r, s = (r == A(0)) ? A(0) : bb / r;
    s_h[j] = r;
    s_h[j + 1] = A(0);
    for (int i = 0; i <= j + 1; ++i) H[j * ld + i] = s_h[i];
    sc[L.cs + j] = c;
    sc[L.sn + j] = s;
    const A gj = s_misc[1];
    sc[L.g + j] = c * gj;
    sc[L.g + j + 1] = -s * gj;
    sc[3] = fabs(s * gj);
    sc[2] = j + 1;
    if (hn == A(0)) sc[4] = 1.0;
}

}  // namespace
}  // namespace hho
