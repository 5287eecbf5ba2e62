// CTA-level dense linear algebra shared by the element and coarse-level kernels.
#pragma once

#include <cuda_runtime.h>

namespace hho {

// Gauss-Jordan with partial pivoting on the n x (n+m) row-major matrix W (ld):
// on return the right block holds A^{-1} B.  Returns false on a zero pivot.
// The pivot is the first row (lowest index) of largest magnitude, so the
// result does not depend on the number of threads.
__device__ inline bool cta_gauss_jordan(double* W, int ld, int n, int m, int* s_piv) {
    __shared__ double s_best[32];
    __shared__ int s_arg[32];
    __shared__ int s_ok;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (threadIdx.x == 0) s_ok = 1;
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        double best = -1.0;
        int arg = n;
        for (int i = j + threadIdx.x; i < n; i += blockDim.x) {
            double v = fabs(W[(int64_t)i * ld + j]);
            if (v > best) {
                best = v;
                arg = i;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            double ob = __shfl_xor_sync(0xffffffffu, best, o);
            int oa = __shfl_xor_sync(0xffffffffu, arg, o);
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
            for (int w = 1; w < nw; ++w)
                if (s_best[w] > b || (s_best[w] == b && s_arg[w] < a)) {
                    b = s_best[w];
                    a = s_arg[w];
                }
            *s_piv = a;
            if (!(b > 0.0)) s_ok = 0;
        }
        __syncthreads();
        if (!s_ok) return false;
        const int p = *s_piv;
        if (p != j)
            for (int c = threadIdx.x; c < n + m; c += blockDim.x) {
                double t = W[(int64_t)j * ld + c];
                W[(int64_t)j * ld + c] = W[(int64_t)p * ld + c];
                W[(int64_t)p * ld + c] = t;
            }
        __syncthreads();
        const double inv = 1.0 / W[(int64_t)j * ld + j];
        __syncthreads();
        for (int c = threadIdx.x; c < n + m; c += blockDim.x) W[(int64_t)j * ld + c] *= inv;
        __syncthreads();
        // eliminate column j from every other row: one warp per row, lanes over columns
        for (int i = wid; i < n; i += nw) {
            if (i == j) continue;
            const double f = W[(int64_t)i * ld + j];
            if (f == 0.0) continue;
            double* wi = W + (int64_t)i * ld;
            const double* wj = W + (int64_t)j * ld;
            for (int c = lane; c < n + m; c += 32)
                if (c != j) wi[c] -= f * wj[c];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x)
            if (i != j) W[(int64_t)i * ld + j] = 0.0;
        __syncthreads();
    }
    return true;
}

}  // namespace hho
