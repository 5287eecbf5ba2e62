// p-multilevel V-cycle and FGMRES on the GPU (Sec. 3.3, Algorithm MG_V).
//
//   smoother      m iterations of right-preconditioned GMRES (the paper uses two,
//                 Sec. 5.2.2) with the block-Jacobi preconditioner (face blocks
//                 D_F^{-1}, element pressure pivot blocks M_T^{-1})
//   restriction   per face and component keep the leading coefficients,
//                 fused with the defect computation d = I(b - S w) (Sec. 3.1)
//   prolongation  zero padding, added to the iterate (Sec. 3.1)
//   coarse level  exact solve in FP64 (coarse.cu)
//   outer solver  flexible GMRES in FP64, one V-cycle per iteration (Sec. 3.3)
//
// The V-cycle runs in FP64 or, for the mixed-precision option, with FP32
// level operators, smoother blocks and smoother vectors (FP32 multiply-adds).
// In the FP32 V-cycle a dot product is summed in FP32 inside a thread (a few
// terms), across the 32 lanes of a warp and across the warps of a block, and
// each block's partial is stored in FP64 and added in the last block; the
// relative rounding error stays near (terms per thread + 13) FP32 ulps of
// sum |x_i y_i|, far below what the smoother needs, and the FP64 pipe (about
// 1/64 of the FP32 rate on this part) stays off the FP32 kernels.  The
// smoother's Hessenberg recurrence runs in the level type; the outer FGMRES
// with its operator stays FP64.
//
// Arnoldi steps use classical Gram-Schmidt applied twice (CGS2).  Kernel
// structure of one Arnoldi step (j) of the outer FGMRES:
//   apply      v_j = w / ||w||, z_j = MG(v_j)  (a V-cycle)
//   spmv+dot   w = S z_j,  t1 = V^T w
//   upd+dot    w -= V t1,  t2 = V^T w
//   upd+norm   w -= V t2,  ||w||^2, then the Hessenberg column, Givens rotation
//              and residual estimate in the last block of the grid
// and of the FP64 smoother, one kernel shorter:
//   apply      w'' = w' - V t2 (second pass of step j-1), v_j = w'' / ||w''||,
//              z_j = M^{-1} v_j  (block Jacobi)
//   spmv+dot   w = S z_j,  t1 = V^T w
//   upd+dot    w' = w - V t1,  t2 = V^T w',  ||w'||^2, then the Hessenberg
//              column with ||w''||^2 = ||w'||^2 - ||t2||^2
// and of the FP32 smoother (at most m = 2 basis vectors), one more kernel
// shorter, by one-reduction classical Gram-Schmidt:
//   apply      w' = w - V t (step j-1), v_j = w' / ||w'||, z_j = M^{-1} v_j
//   spmv+dot   w = S z_j,  t = V^T w,  ||w||^2, then the Hessenberg column
//              with ||w'||^2 = ||w||^2 - ||t||^2
// Every dot product is a deterministic two-level reduction inside the kernel
// that produces its operand: each block writes a partial sum and the last
// block to finish adds the partials in index order, so results are bitwise
// reproducible run to run.  The V-cycle is captured once per (input, output)
// buffer pair into a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <type_traits>

#include "internal.h"
#include "krylov.cuh"

namespace hho {

namespace {

constexpr int GMAX = 8192;  // largest grid of any reduction kernel
constexpr int RT = 256;     // threads per block of the reduction kernels
constexpr int NVMAX = 8;    // dot products per kernel
constexpr int EPT = 4;      // elements per thread of the streaming vector kernels (see vgrid)
constexpr int NCCH = 4;     // combination vectors whose loads a streaming kernel issues together

int grid1d(int64_t n, int tpb) {
    int64_t g = (n + tpb - 1) / tpb;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)sm_count() * 64));
}

// grid of the streaming vector kernels: about 4 elements per thread
int vgrid(int64_t n) {
    int64_t g = (n + (int64_t)EPT * RT - 1) / ((int64_t)EPT * RT);
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, GMAX));
}

template <typename T>
struct LV {
    int64_t nf, ne;
    int b, nP;
    const int32_t *ff_col, *ff_nsl, *fp_col, *pf_col, *pf_nsl;
    const T *ff, *fp, *pf, *pp, *dinv, *minv;
};

template <typename T>
LV<T> view(const LevelMat& L);

template <>
LV<double> view<double>(const LevelMat& L) {
    return LV<double>{L.nf, L.ne, L.b, L.nP, L.ff_col, L.ff_nsl, L.fp_col, L.pf_col, L.pf_nsl,
                      L.ff, L.fp, L.pf, L.pp, L.dinv, L.minv};
}

template <>
LV<float> view<float>(const LevelMat& L) {
    return LV<float>{L.nf, L.ne, L.b, L.nP, L.ff_col, L.ff_nsl, L.fp_col, L.pf_col, L.pf_nsl,
                     L.ff32, L.fp32, L.pf32, L.pp32, L.dinv32, L.minv32};
}

// Block reduction of the accumulators acc[0..nv0-1] and, when self is set, of
// acc[NV-1] as output nv0; partial sums per block; the last block adds the
// partials in a fixed order into out[0..nv0+self-1] and runs the hook on the
// self output (on output 0 without one).  All
// arithmetic is in A (partials are stored as FP64).  Output slots are mapped
// in shared memory, so that no register array is indexed by a run-time value,
// and warps shuffle only the slots in use.
template <int NV, typename A>
__device__ __forceinline__ void reduce_finish(A (&acc)[NV], int nv0, int self, double* __restrict__ partial,
                                              unsigned* __restrict__ counter, double* __restrict__ out, int hook,
                                              double* sc, GS L, int j) {
    const int nv = nv0 + self;
    __shared__ A sm[RT / 32][NV];
    __shared__ bool s_last;
    __shared__ A s_fresh;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        if (v < nv0 || (self && v == NV - 1)) {
            A a = acc[v];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0) sm[wid][v] = a;
        }
    }
    __syncthreads();
    if (threadIdx.x < nv) {
        const int src = ((int)threadIdx.x < nv0) ? (int)threadIdx.x : NV - 1;
        A s = A(0);
        for (int w = 0; w < RT / 32; ++w) s += sm[w][src];
        partial[threadIdx.x * GMAX + blockIdx.x] = (double)s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // thread t adds the partials of blocks t, t + RT, ...; then a fixed shuffle
    // tree per warp and the warps in index order
    A ps[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) ps[v] = A(0);
    for (int b = threadIdx.x; b < (int)gridDim.x; b += RT) {
#pragma unroll
        for (int v = 0; v < NV; ++v)
            if (v < nv) ps[v] += (A)__ldcg(partial + v * GMAX + b);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        if (v < nv) {
            A a = ps[v];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0) sm[wid][v] = a;
        }
    }
    __syncthreads();
    if (threadIdx.x < nv) {
        A s = A(0);
        for (int w = 0; w < RT / 32; ++w) s += sm[w][threadIdx.x];
        out[threadIdx.x] = (double)s;
        if ((int)threadIdx.x == (self ? nv0 : 0)) s_fresh = s;
    }
    if (threadIdx.x == 0) *counter = 0u;
    __syncthreads();
    run_hook<A>(hook, sc, L, j, s_fresh);
}

// dacc[q] += V_q[o] * v for q < nv, dacc[NVMAX] += v * v: fully unrolled with
// predicates so the accumulators stay in registers.
template <typename T, typename A>
__device__ __forceinline__ void accumulate_dots(A (&dacc)[NVMAX + 1], const T* __restrict__ V, int64_t ld,
                                                int64_t o, int nv, int self, T v) {
    const A dv = (A)v;
#pragma unroll
    for (int q = 0; q < NVMAX; ++q)
        if (q < nv) dacc[q] += (A)V[q * ld + o] * dv;
    if (self) dacc[NVMAX] += dv * dv;
}

// accumulate_dots with a compile-time number of dot vectors (no predicated
// FMAs: the FP64 pipe of this part is narrow enough for them to matter)
template <int NVC, typename T, typename A>
__device__ __forceinline__ void accumulate_dots_n(A (&dacc)[NVMAX + 1], const T* __restrict__ V, int64_t ld,
                                                  int64_t o, int self, T v) {
    const A dv = (A)v;
#pragma unroll
    for (int q = 0; q < NVC; ++q) dacc[q] += (A)V[q * ld + o] * dv;
    if (self) dacc[NVMAX] += dv * dv;
}

// Finish the nv dots and the self product (output nv).
template <typename A>
__device__ __forceinline__ void finish_dots(A (&dacc)[NVMAX + 1], int nv, int self, double* partial,
                                            unsigned* counter, double* out, int hook, double* sc, GS gsl, int j) {
    reduce_finish<NVMAX + 1>(dacc, nv, self, partial, counter, out, hook, sc, gsl, j);
}

// ---------------------------------------------------------------------------
// Operator rows.  A warp handles 32 consecutive faces (or elements) and R rows
// of each, so every value load of the operator is one coalesced access and
// each gathered x value serves R rows.  Accumulation is in the level type T.
// ---------------------------------------------------------------------------
template <int R, typename T>
__device__ __forceinline__ void face_rows(const LV<T>& L, int64_t F, const int (&rows)[R], int nr,
                                          const T* __restrict__ x, T (&acc)[R]) {
    const int b = L.b, nP = L.nP;
    const int64_t nf = L.nf;
#pragma unroll
    for (int i = 0; i < R; ++i) acc[i] = T(0);
    const int ns = L.ff_nsl[F];
    for (int s = 0; s < ns; ++s) {
        const int64_t G = L.ff_col[s * nf + F];
        const T* xv = x + G * b;
        const T* a = L.ff + (int64_t)s * b * b * nf + F;
#pragma unroll 4
        for (int c = 0; c < b; ++c) {
            const T xc = xv[c];
            const T* ac = a + (int64_t)c * b * nf;
#pragma unroll
            for (int i = 0; i < R; ++i)
                if (i < nr) acc[i] += __ldg(ac + (int64_t)rows[i] * nf) * xc;
        }
    }
    const T* xp = x + nf * b;
    for (int p = 0; p < 2; ++p) {
        const int Tl = L.fp_col[p * nf + F];
        if (Tl < 0) continue;
        const T* a = L.fp + (int64_t)p * nP * b * nf + F;
        for (int c = 0; c < nP; ++c) {
            const T xc = xp[(int64_t)Tl * nP + c];
            const T* ac = a + (int64_t)c * b * nf;
#pragma unroll
            for (int i = 0; i < R; ++i)
                if (i < nr) acc[i] += __ldg(ac + (int64_t)rows[i] * nf) * xc;
        }
    }
}

template <int R, typename T>
__device__ __forceinline__ void elem_rows(const LV<T>& L, int64_t E, const int (&rows)[R], int nr,
                                          const T* __restrict__ x, T (&acc)[R]) {
    const int b = L.b, nP = L.nP;
    const int64_t ne = L.ne;
#pragma unroll
    for (int i = 0; i < R; ++i) acc[i] = T(0);
    const int N = L.pf_nsl[E];
    for (int f = 0; f < N; ++f) {
        const int64_t G = L.pf_col[f * ne + E];
        const T* xv = x + G * b;
        const T* a = L.pf + (int64_t)f * b * nP * ne + E;
#pragma unroll 4
        for (int c = 0; c < b; ++c) {
            const T xc = xv[c];
            const T* ac = a + (int64_t)c * nP * ne;
#pragma unroll
            for (int i = 0; i < R; ++i)
                if (i < nr) acc[i] += __ldg(ac + (int64_t)rows[i] * ne) * xc;
        }
    }
    const T* xp = x + L.nf * b + E * nP;
    for (int c = 0; c < nP; ++c) {
        const T xc = xp[c];
        const T* ac = L.pp + (int64_t)c * nP * ne + E;
#pragma unroll
        for (int i = 0; i < R; ++i)
            if (i < nr) acc[i] += __ldg(ac + (int64_t)rows[i] * ne) * xc;
    }
}

// Work items of a level: (32-face tile, row group) then (32-element tile, row group).
struct Items {
    int64_t ftiles, etiles;
    int fgroups, egroups;
    __host__ __device__ int64_t total() const { return ftiles * fgroups + etiles * egroups; }
};

// y = S x (mode 0) or y = bv - S x (mode 1) on all rows; optional FP64 dots of y
// with V_0..V_{nv-1} and with itself (self), finished by reduce_finish.
template <int R, typename T>
__global__ void __launch_bounds__(RT) k_spmv_dot(LV<T> L, Items it, const T* __restrict__ x, const T* __restrict__ bv,
                                                  T* __restrict__ y, int mode, const T* __restrict__ V, int64_t ld,
                                                  int nv, int self, double* __restrict__ partial,
                                                  unsigned* __restrict__ counter, double* __restrict__ out, int hook,
                                                  double* sc, GS gsl, int j) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    using A = typename AccT<T>::type;
    A dacc[NVMAX + 1];
#pragma unroll
    for (int v = 0; v <= NVMAX; ++v) dacc[v] = A(0);
    const int64_t nfi = it.ftiles * it.fgroups;
    for (int64_t w = warp; w < it.total(); w += nwarps) {
        const bool face = w < nfi;
        const int64_t ww = face ? w : w - nfi;
        const int groups = face ? it.fgroups : it.egroups;
        const int64_t tile = ww / groups;
        const int g = (int)(ww % groups);
        const int64_t id = tile * 32 + lane;
        const int nrow = face ? L.b : L.nP;
        if (id >= (face ? L.nf : L.ne)) continue;
        int rows[R];
        int nr = 0;
#pragma unroll
        for (int i = 0; i < R; ++i) {
            rows[i] = g * R + i;
            if (rows[i] < nrow) nr = i + 1;
        }
        T acc[R];
        if (face) face_rows<R, T>(L, id, rows, nr, x, acc);
        else elem_rows<R, T>(L, id, rows, nr, x, acc);
        const int64_t base = face ? id * L.b : L.nf * L.b + id * L.nP;
#pragma unroll
        for (int i = 0; i < R; ++i) {
            if (i >= nr) break;
            const int64_t o = base + rows[i];
            const T v = mode ? T(bv[o] - acc[i]) : acc[i];
            y[o] = v;
            accumulate_dots(dacc, V, ld, o, nv, self, v);
        }
    }
    if (nv + self > 0) finish_dots(dacc, nv, self, partial, counter, out, hook, sc, gsl, j);
}

// Row selection of the restriction d = I(bv - S x) (mode 2 of k_spmv_b): of a
// fine face block (components of nFf unknowns each) the first nFc of every
// component are kept, of a fine element block (components of nEf unknowns:
// one pressure prefix, or velocity and pressure when nothing is condensed) the
// first nEc of every component; d is written in the coarse layout (face blocks
// of bc, then element blocks of nPc).
struct Restr {
    int nFf, nFc, bc, nPc, nEf, nEc;
};
__device__ __forceinline__ int restr_elem_row(const Restr& rs, int r) {  // coarse position of fine element row r, or -1
    const int comp = r / rs.nEf, rr = r - comp * rs.nEf;
    return rr < rs.nEc ? comp * rs.nEc + rr : -1;
}

// Same operator with the face block size B known at compile time: a thread
// holds RF consecutive rows of one face (RF = B up to B = 12), the column loops
// are fully unrolled and the B gathered x values of a neighbour face are loaded
// once per slot.  Element rows: RP rows per thread.
template <int B, int RF, int RP, typename T>
__global__ void __launch_bounds__(RT) k_spmv_b(LV<T> L, Items it, const T* __restrict__ x, const T* __restrict__ bv,
                                                T* __restrict__ y, int mode, const T* __restrict__ V, int64_t ld, int nv,
                                                int self, double* __restrict__ partial, unsigned* __restrict__ counter,
                                                double* __restrict__ out, int hook, double* sc, GS gsl, int j,
                                                Restr rs) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nf = L.nf, ne = L.ne;
    const int nP = L.nP;
    constexpr int CU = B <= 12 ? B : 2;  // column unrolling
    using A = typename AccT<T>::type;
    A dacc[NVMAX + 1];
#pragma unroll
    for (int v = 0; v <= NVMAX; ++v) dacc[v] = A(0);
    const int64_t nfi = it.ftiles * it.fgroups;
    for (int64_t w = warp; w < it.total(); w += nwarps) {
        if (w < nfi) {
            const int64_t tile = w / it.fgroups;
            const int r0 = (int)(w % it.fgroups) * RF;
            const int64_t F = tile * 32 + lane;
            if (F >= nf) continue;
            T acc[RF];
#pragma unroll
            for (int i = 0; i < RF; ++i) acc[i] = T(0);
            const int ns = L.ff_nsl[F];
            for (int s = 0; s < ns; ++s) {
                const T* xv = x + (int64_t)L.ff_col[s * nf + F] * B;
                const T* a = L.ff + ((int64_t)s * B * B + r0) * nf + F;
#pragma unroll(CU)
                for (int c = 0; c < B; ++c) {
                    const T xc = xv[c];
#pragma unroll
                    for (int i = 0; i < RF; ++i) acc[i] += __ldg(a + (int64_t)(c * B + i) * nf) * xc;
                }
            }
            for (int p = 0; p < 2; ++p) {
                const int Tl = L.fp_col[p * nf + F];
                if (Tl < 0) continue;
                const T* xp = x + nf * B + (int64_t)Tl * nP;
                const T* a = L.fp + ((int64_t)p * nP * B + r0) * nf + F;
                for (int c = 0; c < nP; ++c) {
                    const T xc = xp[c];
#pragma unroll
                    for (int i = 0; i < RF; ++i) acc[i] += __ldg(a + (int64_t)(c * B + i) * nf) * xc;
                }
            }
#pragma unroll
            for (int i = 0; i < RF; ++i) {
                const int64_t o = F * B + r0 + i;
                const T v = mode ? T(bv[o] - acc[i]) : acc[i];
                if (mode == 2) {
                    const int r = r0 + i, comp = r / rs.nFf, rr = r - comp * rs.nFf;
                    if (rr < rs.nFc) {
                        y[F * rs.bc + comp * rs.nFc + rr] = v;
                        if (self) dacc[NVMAX] += (A)v * (A)v;
                    }
                } else {
                    y[o] = v;
                    accumulate_dots(dacc, V, ld, o, nv, self, v);
                }
            }
        } else {
            const int64_t ww = w - nfi;
            const int64_t tile = ww / it.egroups;
            const int r0 = (int)(ww % it.egroups) * RP;
            const int64_t E = tile * 32 + lane;
            if (E >= ne) continue;
            T acc[RP];
#pragma unroll
            for (int i = 0; i < RP; ++i) acc[i] = T(0);
            const int N = L.pf_nsl[E];
            for (int f = 0; f < N; ++f) {
                const T* xv = x + (int64_t)L.pf_col[f * ne + E] * B;
                const T* a = L.pf + ((int64_t)f * B * nP + r0) * ne + E;
#pragma unroll 2
                for (int c = 0; c < B; ++c) {
                    const T xc = xv[c];
#pragma unroll
                    for (int i = 0; i < RP; ++i) acc[i] += __ldg(a + (int64_t)(c * nP + i) * ne) * xc;
                }
            }
            const T* xp = x + nf * B + E * nP;
#pragma unroll 2
            for (int c = 0; c < nP; ++c) {
                const T xc = xp[c];
                const T* a = L.pp + ((int64_t)c * nP + r0) * ne + E;
#pragma unroll
                for (int i = 0; i < RP; ++i) acc[i] += __ldg(a + (int64_t)i * ne) * xc;
            }
#pragma unroll
            for (int i = 0; i < RP; ++i) {
                const int64_t o = nf * B + E * nP + r0 + i;
                const T v = mode ? T(bv[o] - acc[i]) : acc[i];
                if (mode == 2) {
                    const int rc = restr_elem_row(rs, r0 + i);
                    if (rc >= 0) {
                        y[nf * rs.bc + E * rs.nPc + rc] = v;
                        if (self) dacc[NVMAX] += (A)v * (A)v;
                    }
                } else {
                    y[o] = v;
                    accumulate_dots(dacc, V, ld, o, nv, self, v);
                }
            }
        }
    }
    if (nv + self > 0) finish_dots(dacc, nv, self, partial, counter, out, hook, sc, gsl, j);
}

// d (coarse layout) = I (bv - S x): only the rows kept by the restriction are
// formed; optionally ||d||^2 with the START hook of the coarse smoother.
template <int R, typename T>
__global__ void __launch_bounds__(RT) k_residual_restrict(LV<T> L, Items it, int nFf, int bc, int nFc, int nPc,
                                                           int nEf, int nEc, const T* __restrict__ x, const T* __restrict__ bv,
                                                           T* __restrict__ d, int do_norm, double* __restrict__ partial,
                                                           unsigned* __restrict__ counter, double* __restrict__ out,
                                                           double* sc, GS gsl) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    using A = typename AccT<T>::type;
    A dacc[1] = {A(0)};
    const int64_t nfi = it.ftiles * it.fgroups;
    for (int64_t w = warp; w < it.total(); w += nwarps) {
        const bool face = w < nfi;
        const int64_t ww = face ? w : w - nfi;
        const int groups = face ? it.fgroups : it.egroups;
        const int64_t tile = ww / groups;
        const int g = (int)(ww % groups);
        const int64_t id = tile * 32 + lane;
        const int nrow = face ? bc : nPc;
        if (id >= (face ? L.nf : L.ne)) continue;
        int rows[R];
        int nr = 0;
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int rc = g * R + i;
            rows[i] = face ? (rc / nFc) * nFf + rc % nFc : (rc / nEc) * nEf + rc % nEc;
            if (rc < nrow) nr = i + 1;
        }
        T acc[R];
        if (face) face_rows<R, T>(L, id, rows, nr, x, acc);
        else elem_rows<R, T>(L, id, rows, nr, x, acc);
#pragma unroll
        for (int i = 0; i < R; ++i) {
            if (i >= nr) break;
            const int rc = g * R + i;
            const int64_t of = face ? id * L.b + rows[i] : L.nf * L.b + id * L.nP + rows[i];
            const int64_t oc = face ? id * bc + rc : L.nf * bc + id * nPc + rc;
            const T v = bv[of] - acc[i];
            d[oc] = v;
            dacc[0] += (A)v * (A)v;
        }
    }
    if (do_norm) reduce_finish<1>(dacc, 1, 0, partial, counter, out, HOOK_START, sc, gsl, 0);
}

// v = w / den, z = M^{-1} v (block Jacobi): z is computed from w and scaled.
template <typename T>
__global__ void k_apply_jacobi(LV<T> L, const T* __restrict__ w, const double* __restrict__ den, T* __restrict__ v,
                               T* __restrict__ z, const T* __restrict__ Vp, int64_t ld, int npend,
                               const double* __restrict__ pc) {
    const T inv = block_inverse<T>(den);
    const T* s_pc = stage_pending<T>(pc, npend);
    const int64_t nfr = L.nf * L.b, ner = L.ne * L.nP;
    const int b = L.b, nP = L.nP;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nfr + ner; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < nfr) {
            const int r = (int)(i / L.nf);
            const int64_t F = i % L.nf;
            const T* a = L.dinv + (int64_t)r * L.nf + F;
            T s = T(0);
            for (int c = 0; c < b; ++c) s += a[(int64_t)c * b * L.nf] * pending(w, Vp, ld, npend, s_pc, F * b + c);
            z[F * b + r] = s * inv;
            v[F * b + r] = pending(w, Vp, ld, npend, s_pc, F * b + r) * inv;
        } else {
            const int64_t jj = i - nfr;
            const int r = (int)(jj / L.ne);
            const int64_t E = jj % L.ne;
            const T* a = L.minv + (int64_t)r * L.ne + E;
            const int64_t ob = nfr + E * nP;
            T s = T(0);
            for (int c = 0; c < nP; ++c) s += a[(int64_t)c * nP * L.ne] * pending(w, Vp, ld, npend, s_pc, ob + c);
            z[ob + r] = s * inv;
            v[ob + r] = pending(w, Vp, ld, npend, s_pc, ob + r) * inv;
        }
    }
}

// Same operation with the face block size B known at compile time: a thread
// holds RF rows of one face (its B values of w loaded once) or RP rows of one
// element; the block values are read coalesced across the 32 faces (elements)
// of a warp.  Work items as in k_spmv_b.
template <int B, int RF, int RP, typename T>
__global__ void __launch_bounds__(RT) k_jacobi_b(LV<T> L, Items it, const T* __restrict__ w,
                                                  const double* __restrict__ den, T* __restrict__ v,
                                                  T* __restrict__ z, const T* __restrict__ Vp, int64_t ld,
                                                  int npend, const double* __restrict__ pc) {
    const T inv = block_inverse<T>(den);
    const T* s_pc = stage_pending<T>(pc, npend);
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nf = L.nf, ne = L.ne;
    const int nP = L.nP;
    constexpr int CU = B <= 12 ? B : 2;  // column unrolling
    const int64_t nfi = it.ftiles * it.fgroups;
    for (int64_t wi = warp; wi < it.total(); wi += nwarps) {
        if (wi < nfi) {
            const int64_t F = (wi / it.fgroups) * 32 + lane;
            const int r0 = (int)(wi % it.fgroups) * RF;
            if (F >= nf) continue;
            T acc[RF];
#pragma unroll
            for (int i = 0; i < RF; ++i) acc[i] = T(0);
            const T* a = L.dinv + (int64_t)r0 * nf + F;
#pragma unroll(CU)
            for (int c = 0; c < B; ++c) {
                const T wc = pending(w, Vp, ld, npend, s_pc, F * B + c);
#pragma unroll
                for (int i = 0; i < RF; ++i) acc[i] += __ldg(a + (int64_t)(c * B + i) * nf) * wc;
            }
#pragma unroll
            for (int i = 0; i < RF; ++i) {
                z[F * B + r0 + i] = acc[i] * inv;
                v[F * B + r0 + i] = pending(w, Vp, ld, npend, s_pc, F * B + r0 + i) * inv;
            }
        } else {
            const int64_t ww = wi - nfi;
            const int64_t E = (ww / it.egroups) * 32 + lane;
            const int r0 = (int)(ww % it.egroups) * RP;
            if (E >= ne) continue;
            const int64_t ob = nf * B + E * nP;
            T acc[RP];
#pragma unroll
            for (int i = 0; i < RP; ++i) acc[i] = T(0);
            const T* a = L.minv + (int64_t)r0 * ne + E;
#pragma unroll 2
            for (int c = 0; c < nP; ++c) {
                const T wc = pending(w, Vp, ld, npend, s_pc, ob + c);
#pragma unroll
                for (int i = 0; i < RP; ++i) acc[i] += __ldg(a + (int64_t)(c * nP + i) * ne) * wc;
            }
#pragma unroll
            for (int i = 0; i < RP; ++i) {
                const int64_t o = ob + r0 + i;
                z[o] = acc[i] * inv;
                v[o] = pending(w, Vp, ld, npend, s_pc, o) * inv;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// FP32 kernels on the row-interleaved layouts (LevelMat::ilv): one thread owns
// a whole face block (B rows) or element block (NP rows); for every column the
// block's rows are contiguous, so a thread reads them with 16- or 8-byte
// loads and a warp reads one contiguous span per column.  NP is the pressure
// block size the degree behind B gives under velocity-only condensation, or 1.
// ---------------------------------------------------------------------------
constexpr int np_full(int B) {
    return B == 2 ? 1 : B == 4 ? 3 : B == 6 ? 6 : B == 8 ? 10 : B == 10 ? 15 : B == 12 ? 21 : B == 3 ? 1 : B == 9 ? 4
         : B == 18 ? 10 : B == 30 ? 20 : 0;
}

// v[0..N) = p[0..N), 16-byte loads when N % 4 == 0, 8-byte when N is even
// (operator values only: every run starts at a multiple of N floats of a
// separately allocated array, so it is aligned for the chosen width)
template <int N>
__device__ __forceinline__ void load_run(const float* __restrict__ p, float (&v)[N]) {
    if constexpr (N % 4 == 0) {
#pragma unroll
        for (int i = 0; i < N / 4; ++i) {
            const float4 t = __ldg(reinterpret_cast<const float4*>(p) + i);
            v[4 * i] = t.x;
            v[4 * i + 1] = t.y;
            v[4 * i + 2] = t.z;
            v[4 * i + 3] = t.w;
        }
    } else if constexpr (N % 2 == 0) {
#pragma unroll
        for (int i = 0; i < N / 2; ++i) {
            const float2 t = __ldg(reinterpret_cast<const float2*>(p) + i);
            v[2 * i] = t.x;
            v[2 * i + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] = __ldg(p + i);
    }
}

// v[0..N) = p[0..N) with scalar loads: vectors of the smoother (the Arnoldi
// and preconditioned vectors sit at offsets j n that need not be 16-byte
// aligned), read through L1
template <int N>
__device__ __forceinline__ void load_run_plain(const float* __restrict__ p, float (&v)[N]) {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = p[i];
}

// acc[r] += sum_c A_c[r] xv[c] for a block of R rows and C columns; column c's
// R rows start at a + c * cs
template <int R, int C>
__device__ __forceinline__ void block_mv(const float* __restrict__ a, int64_t cs, const float (&xv)[C],
                                         float (&acc)[R]) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
        float col[R];
        load_run<R>(a + (int64_t)c * cs, col);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] += col[r] * xv[c];
    }
}

// The level operator on the interleaved FP32 layout, with the modes, dots and
// hooks of k_spmv_b (mode 0: y = S x, 1: y = bv - S x, 2: restriction).
template <int B, int NP, int RF>
__global__ void __launch_bounds__(RT, 4) k_spmv_v(LV<float> L, Items it, const float* __restrict__ x,
                                                const float* __restrict__ bv, float* __restrict__ y, int mode,
                                                const float* __restrict__ V, int64_t ld, int nv, int self,
                                                double* __restrict__ partial, unsigned* __restrict__ counter,
                                                double* __restrict__ out, int hook, double* sc, GS gsl, int j,
                                                Restr rs) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nf = L.nf, ne = L.ne;
    float dacc[NVMAX + 1];
#pragma unroll
    for (int v = 0; v <= NVMAX; ++v) dacc[v] = 0.f;
    const int64_t nfi = it.ftiles * it.fgroups;
    for (int64_t w = warp; w < it.total(); w += nwarps) {
        if (w < nfi) {
            const int64_t F = (w / it.fgroups) * 32 + lane;
            const int r0 = (int)(w % it.fgroups) * RF;
            if (F >= nf) continue;
            float acc[RF];
#pragma unroll
            for (int r = 0; r < RF; ++r) acc[r] = 0.f;
            // the next slot's column index is fetched one slot ahead, so that
            // each slot waits for one round of loads (x and values) only
            const int ns = L.ff_nsl[F];
            int64_t G = (ns > 0) ? L.ff_col[F] : 0;
            for (int s = 0; s < ns; ++s) {
                const int64_t Gn = (s + 1 < ns) ? L.ff_col[(s + 1) * nf + F] : 0;
                float xv[B];
                load_run_plain<B>(x + G * B, xv);
                block_mv<RF, B>(L.ff + ((int64_t)s * B * nf + F) * B + r0, nf * B, xv, acc);
                G = Gn;
            }
            if constexpr (NP > 0) {  // HHO-hp levels have no element rows (NP = 0)
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    const int T = L.fp_col[p * nf + F];
                    if (T < 0) continue;
                    float xp[NP];
                    load_run_plain<NP>(x + nf * B + (int64_t)T * NP, xp);
                    block_mv<RF, NP>(L.fp + ((int64_t)p * NP * nf + F) * B + r0, nf * B, xp, acc);
                }
            }
#pragma unroll
            for (int i = 0; i < RF; ++i) {
                const int r = r0 + i;
                const int64_t o = F * B + r;
                const float v = mode ? bv[o] - acc[i] : acc[i];
                if (mode == 2) {
                    const int comp = r / rs.nFf, rr = r - comp * rs.nFf;
                    if (rr < rs.nFc) {
                        y[F * rs.bc + comp * rs.nFc + rr] = v;
                        if (self) dacc[NVMAX] += v * v;
                    }
                } else {
                    y[o] = v;
                    accumulate_dots(dacc, V, ld, o, nv, self, v);
                }
            }
        } else if constexpr (NP > 0) {
            const int64_t E = (w - nfi) * 32 + lane;  // one thread per element block (egroups = 1)
            if (E >= ne) continue;
            float acc[NP];
#pragma unroll
            for (int r = 0; r < NP; ++r) acc[r] = 0.f;
            const int N = L.pf_nsl[E];
            int64_t G = (N > 0) ? L.pf_col[E] : 0;
            for (int f = 0; f < N; ++f) {
                const int64_t Gn = (f + 1 < N) ? L.pf_col[(f + 1) * ne + E] : 0;
                float xv[B];
                load_run_plain<B>(x + G * B, xv);
                block_mv<NP, B>(L.pf + ((int64_t)f * B * ne + E) * NP, ne * NP, xv, acc);
                G = Gn;
            }
            {
                float xp[NP];
                load_run_plain<NP>(x + nf * B + E * NP, xp);
                block_mv<NP, NP>(L.pp + E * NP, ne * NP, xp, acc);
            }
#pragma unroll
            for (int r = 0; r < NP; ++r) {
                const int64_t o = nf * B + E * NP + r;
                const float v = mode ? bv[o] - acc[r] : acc[r];
                if (mode == 2) {
                    const int rc = restr_elem_row(rs, r);
                    if (rc >= 0) {
                        y[nf * rs.bc + E * rs.nPc + rc] = v;
                        if (self) dacc[NVMAX] += v * v;
                    }
                } else {
                    y[o] = v;
                    accumulate_dots(dacc, V, ld, o, nv, self, v);
                }
            }
        }
    }
    if (nv + self > 0) finish_dots(dacc, nv, self, partial, counter, out, hook, sc, gsl, j);
}

// Lane layout of the warp-per-face kernels for the large 3D face blocks (B = 18
// and 30 unknowns; smaller blocks keep one thread per face, which measured
// faster for B = 9): a lane loads VW consecutive rows of one column with one
// VW * 4-byte load; RL = B / VW lanes cover a column and GC = 32 / RL columns
// are read by one warp instruction (lane = g * RL + rr: column group g, rows
// rr * VW ..); each lane accumulates its rows over the columns c = g (mod GC)
// and the GC partial sums of a row are added across the lane groups in group
// order (deterministic).
// The 3D HHO-hp blocks (24 and 40 unknowns, multiples of 4) take 16-byte loads
// of 4 rows: RL = 6 or 10 lanes per column, 5 or 3 columns per load.
constexpr int wv_vw(int B) { return (B >= 24 && B % 4 == 0) ? 4 : (B % 2 == 0 && B / 2 <= 16) ? 2 : 1; }
constexpr int wv_rl(int B) { return B / wv_vw(B); }
constexpr int wv_gc(int B) { return 32 / wv_rl(B); }
constexpr int wv_nk(int B) { return (B + wv_gc(B) - 1) / wv_gc(B); }
constexpr int wv_xr(int B) { return (B + 31) / 32; }  // registers per lane holding a column block of x
// resident blocks of 256 threads per SM the operator kernel is compiled for
// (the largest count without register spills): 4 (64 registers a thread) for
// the blocks of 18 and 24 unknowns, 3 for 30 with one pressure per element, 2
// for 30 with element pressure blocks and for 40
constexpr int wv_minb(int B, int NP) { return (B == 18 || B == 24) ? 4 : (B == 30 && NP <= 1) ? 3 : 2; }
static_assert(wv_rl(30) == 15 && wv_gc(30) == 2 && wv_rl(18) == 9 && wv_gc(18) == 3 && wv_rl(9) == 9 &&
                  wv_gc(9) == 3 && wv_nk(30) * wv_gc(30) == 30 && wv_nk(18) * wv_gc(18) == 18 &&
                  wv_rl(40) == 10 && wv_gc(40) == 3 && wv_nk(40) == 14 && wv_rl(24) == 6 && wv_gc(24) == 5 &&
                  wv_xr(40) == 2 && wv_xr(30) == 1,
              "warp lane layout");

// entry c (0 <= c < 32 XR, lane-dependent) of a column block held as XR
// registers per lane (register i of lane l holds entry 32 i + l); every lane
// takes part in every shuffle
template <int XR>
__device__ __forceinline__ float wv_bcast(const float (&xr)[XR], int c) {
    float v = __shfl_sync(0xffffffffu, xr[0], c & 31);
#pragma unroll
    for (int i = 1; i < XR; ++i) {
        const float t = __shfl_sync(0xffffffffu, xr[i], c & 31);
        if ((c >> 5) == i) v = t;
    }
    return v;
}

template <int VW>
__device__ __forceinline__ void load_vw(const float* __restrict__ p, float (&v)[VW]) {
    if constexpr (VW == 4) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(p));
        v[0] = t.x;
        v[1] = t.y;
        v[2] = t.z;
        v[3] = t.w;
    } else if constexpr (VW == 2) {
        const float2 t = __ldg(reinterpret_cast<const float2*>(p));
        v[0] = t.x;
        v[1] = t.y;
    } else {
#pragma unroll
        for (int q = 0; q < VW; ++q) v[q] = __ldg(p + q);
    }
}

// sum over the GC column groups of acc (every lane gets the total of its rows)
template <int B, int VW>
__device__ __forceinline__ void wv_group_sum(float (&acc)[VW], int rr) {
    constexpr int RL = wv_rl(B), GC = wv_gc(B);
#pragma unroll
    for (int q = 0; q < VW; ++q) {
        float t = 0.f;
#pragma unroll
        for (int g2 = 0; g2 < GC; ++g2) t += __shfl_sync(0xffffffffu, acc[q], g2 * RL + rr);
        acc[q] = t;
    }
}

// The level operator for the 3D face blocks: one warp per face row block
// (lane layout above).  Per slot, lane c < B loads x's entry c of the slot's
// column block once and the values are broadcast by shuffles; the face's
// block is read as NK wide coalesced loads per slot.  Element rows stay one
// thread per element (their values are contiguous across elements).
template <int B, int NP>
__global__ void __launch_bounds__(RT, wv_minb(B, NP)) k_spmv_w(LV<float> L, int64_t nfw, int64_t etiles,
                                                          const float* __restrict__ x,
                                             const float* __restrict__ bv, float* __restrict__ y, int mode,
                                             const float* __restrict__ V, int64_t ld, int nv, int self,
                                             double* __restrict__ partial, unsigned* __restrict__ counter,
                                             double* __restrict__ out, int hook, double* sc, GS gsl, int j,
                                             Restr rs) {
    constexpr int VW = wv_vw(B), RL = wv_rl(B), GC = wv_gc(B), NK = wv_nk(B), XR = wv_xr(B);
    constexpr int SU = (NK * VW <= 12) ? 2 : 1;  // slots in flight per warp
    const int lane = threadIdx.x & 31;
    const int g = lane / RL, rr = lane - g * RL;
    const bool lane_ok = g < GC;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nf = L.nf, ne = L.ne;
    float dacc[NVMAX + 1];
#pragma unroll
    for (int v = 0; v <= NVMAX; ++v) dacc[v] = 0.f;
    for (int64_t w = warp; w < nfw + etiles; w += nwarps) {
        if (w < nfw) {
            const int64_t F = w;
            const int ns = L.ff_nsl[F];
            float acc[VW];
#pragma unroll
            for (int q = 0; q < VW; ++q) acc[q] = 0.f;
            // SU slots per iteration: their column-index -> x chains and their
            // value loads are all issued before the first multiply
            for (int s0 = 0; s0 < ns; s0 += SU) {
                float xl[SU][XR];
                float av[SU][NK][VW];
#pragma unroll
                for (int u = 0; u < SU; ++u) {
                    const int s = s0 + u;
                    const bool has = s < ns;
                    const int64_t G = has ? L.ff_col[(int64_t)s * nf + F] : 0;
#pragma unroll
                    for (int i = 0; i < XR; ++i) xl[u][i] = (has && 32 * i + lane < B) ? x[G * B + 32 * i + lane] : 0.f;
                    const float* a = L.ff + ((int64_t)s * B * nf + F) * B + rr * VW;
#pragma unroll
                    for (int k = 0; k < NK; ++k) {
                        const int c = k * GC + g;
                        if (has && lane_ok && c < B) load_vw<VW>(a + (int64_t)c * nf * B, av[u][k]);
                        else
#pragma unroll
                            for (int q = 0; q < VW; ++q) av[u][k][q] = 0.f;
                    }
                }
#pragma unroll
                for (int u = 0; u < SU; ++u)
#pragma unroll
                    for (int k = 0; k < NK; ++k) {
                        const float xc = wv_bcast<XR>(xl[u], k * GC + g);
#pragma unroll
                        for (int q = 0; q < VW; ++q) acc[q] += av[u][k][q] * xc;
                    }
            }
            if constexpr (NP > 0) {  // HHO-hp levels have no element rows (NP = 0)
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    const int T = L.fp_col[p * nf + F];
                    if (T < 0) continue;
                    const float* xp = x + nf * B + (int64_t)T * NP;
                    const float* a = L.fp + ((int64_t)p * NP * nf + F) * B + rr * VW;
                    for (int c = g; c < NP; c += GC) {
                        if (!lane_ok) break;
                        float av[VW];
                        load_vw<VW>(a + (int64_t)c * nf * B, av);
                        const float xc = xp[c];
#pragma unroll
                        for (int q = 0; q < VW; ++q) acc[q] += av[q] * xc;
                    }
                }
            }
            wv_group_sum<B, VW>(acc, rr);
            if (lane_ok && g == 0) {
#pragma unroll
                for (int q = 0; q < VW; ++q) {
                    const int r = rr * VW + q;
                    const int64_t o = F * B + r;
                    const float v = mode ? bv[o] - acc[q] : acc[q];
                    if (mode == 2) {
                        const int comp = r / rs.nFf, rq = r - comp * rs.nFf;
                        if (rq < rs.nFc) {
                            y[F * rs.bc + comp * rs.nFc + rq] = v;
                            if (self) dacc[NVMAX] += v * v;
                        }
                    } else {
                        y[o] = v;
                        accumulate_dots(dacc, V, ld, o, nv, self, v);
                    }
                }
            }
        } else if constexpr (NP > 0) {
            const int64_t E = (w - nfw) * 32 + lane;
            if (E >= ne) continue;
            float acc[NP];
#pragma unroll
            for (int q = 0; q < NP; ++q) acc[q] = 0.f;
            const int N = L.pf_nsl[E];
            for (int f = 0; f < N; ++f) {
                const int64_t G = L.pf_col[(int64_t)f * ne + E];
                const float* xv = x + G * B;
                const float* a = L.pf + ((int64_t)f * B * ne + E) * NP;
#pragma unroll 6
                for (int c = 0; c < B; ++c) {
                    const float xc = xv[c];
                    float col[NP];
                    load_run<NP>(a + (int64_t)c * ne * NP, col);
#pragma unroll
                    for (int q = 0; q < NP; ++q) acc[q] += col[q] * xc;
                }
            }
            {
                float xp[NP];
                load_run_plain<NP>(x + nf * B + E * NP, xp);
                block_mv<NP, NP>(L.pp + E * NP, ne * NP, xp, acc);
            }
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const int64_t o = nf * B + E * NP + q;
                const float v = mode ? bv[o] - acc[q] : acc[q];
                if (mode == 2) {
                    const int rc = restr_elem_row(rs, q);
                    if (rc >= 0) {
                        y[nf * rs.bc + E * rs.nPc + rc] = v;
                        if (self) dacc[NVMAX] += v * v;
                    }
                } else {
                    y[o] = v;
                    accumulate_dots(dacc, V, ld, o, nv, self, v);
                }
            }
        }
    }
    if (nv + self > 0) finish_dots(dacc, nv, self, partial, counter, out, hook, sc, gsl, j);
}

// Block Jacobi for the 3D face blocks with the lane layout above (one warp per
// face), element blocks one thread per element; the pending second
// Gram-Schmidt pass as in k_jacobi_v.
template <int B, int NP>
__global__ void __launch_bounds__(RT) k_jacobi_w(LV<float> L, int64_t etiles, const float* __restrict__ w,
                                               const double* __restrict__ den, float* __restrict__ v,
                                               float* __restrict__ z, const float* __restrict__ Vp, int64_t ld,
                                               int npend, const double* __restrict__ pc) {
    constexpr int VW = wv_vw(B), RL = wv_rl(B), GC = wv_gc(B), NK = wv_nk(B), XR = wv_xr(B);
    const float inv = block_inverse<float>(den);
    const float* s_pc = stage_pending<float>(pc, npend);
    const int lane = threadIdx.x & 31;
    const int g = lane / RL, rr = lane - g * RL;
    const bool lane_ok = g < GC;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nf = L.nf, ne = L.ne;
    for (int64_t wi = warp; wi < nf + etiles; wi += nwarps) {
        if (wi < nf) {
            const int64_t F = wi;
            float ul[XR];
#pragma unroll
            for (int i = 0; i < XR; ++i)
                ul[i] = 32 * i + lane < B ? pending(w, Vp, ld, npend, s_pc, F * B + 32 * i + lane) : 0.f;
            const float* a = L.dinv + F * B + rr * VW;
            float av[NK][VW];
#pragma unroll
            for (int k = 0; k < NK; ++k) {
                const int c = k * GC + g;
                if (lane_ok && c < B) load_vw<VW>(a + (int64_t)c * nf * B, av[k]);
                else
#pragma unroll
                    for (int q = 0; q < VW; ++q) av[k][q] = 0.f;
            }
            float acc[VW];
#pragma unroll
            for (int q = 0; q < VW; ++q) acc[q] = 0.f;
#pragma unroll
            for (int k = 0; k < NK; ++k) {
                const float uc = wv_bcast<XR>(ul, k * GC + g);
#pragma unroll
                for (int q = 0; q < VW; ++q) acc[q] += av[k][q] * uc;
            }
            wv_group_sum<B, VW>(acc, rr);
            if (lane_ok && g == 0)
#pragma unroll
                for (int q = 0; q < VW; ++q) z[F * B + rr * VW + q] = acc[q] * inv;
#pragma unroll
            for (int i = 0; i < XR; ++i)
                if (32 * i + lane < B) v[F * B + 32 * i + lane] = ul[i] * inv;
        } else if constexpr (NP > 0) {
            const int64_t E = (wi - nf) * 32 + lane;
            if (E >= ne) continue;
            const int64_t ob = nf * B + E * NP;
            float u[NP], acc[NP];
#pragma unroll
            for (int c = 0; c < NP; ++c) {
                u[c] = pending(w, Vp, ld, npend, s_pc, ob + c);
                acc[c] = 0.f;
            }
            block_mv<NP, NP>(L.minv + E * NP, ne * NP, u, acc);
#pragma unroll
            for (int r = 0; r < NP; ++r) {
                z[ob + r] = acc[r] * inv;
                v[ob + r] = u[r] * inv;
            }
        }
    }
}

// Block Jacobi on the interleaved FP32 layout, with the pending second
// Gram-Schmidt pass of k_jacobi_b.
template <int B, int NP>
__global__ void __launch_bounds__(RT) k_jacobi_v(LV<float> L, Items it, const float* __restrict__ w,
                                                  const double* __restrict__ den, float* __restrict__ v,
                                                  float* __restrict__ z, const float* __restrict__ Vp, int64_t ld,
                                                  int npend, const double* __restrict__ pc) {
    const float inv = block_inverse<float>(den);
    const float* s_pc = stage_pending<float>(pc, npend);
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nf = L.nf, ne = L.ne;
    for (int64_t wi = warp; wi < it.total(); wi += nwarps) {
        if (wi < it.ftiles) {
            const int64_t F = wi * 32 + lane;
            if (F >= nf) continue;
            float u[B], acc[B];
#pragma unroll
            for (int c = 0; c < B; ++c) {
                u[c] = pending(w, Vp, ld, npend, s_pc, F * B + c);
                acc[c] = 0.f;
            }
            block_mv<B, B>(L.dinv + F * B, nf * B, u, acc);
#pragma unroll
            for (int r = 0; r < B; ++r) {
                z[F * B + r] = acc[r] * inv;
                v[F * B + r] = u[r] * inv;
            }
        } else if constexpr (NP > 0) {
            const int64_t E = (wi - it.ftiles) * 32 + lane;
            if (E >= ne) continue;
            const int64_t ob = nf * B + E * NP;
            float u[NP], acc[NP];
#pragma unroll
            for (int c = 0; c < NP; ++c) {
                u[c] = pending(w, Vp, ld, npend, s_pc, ob + c);
                acc[c] = 0.f;
            }
            block_mv<NP, NP>(L.minv + E * NP, ne * NP, u, acc);
#pragma unroll
            for (int r = 0; r < NP; ++r) {
                z[ob + r] = acc[r] * inv;
                v[ob + r] = u[r] * inv;
            }
        }
    }
}

// dst[(p N + i) R + r] = src[(p R + r) N + i]: FP32 row-interleaved copy of a
// [planes][R][N] FP64 array
__global__ void k_interleave(int64_t planes, int R, int64_t N, const double* __restrict__ src,
                             float* __restrict__ dst) {
    const int64_t tot = planes * R * N;
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < tot; o += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = o % R, i = (o / R) % N, p = o / ((int64_t)R * N);
        dst[o] = (float)src[(p * R + r) * N + i];
    }
}

// v = (w' - sum_{q < npend} pc_q Vp_q) / den: the pending second pass and the
// basis scaling of a smoother step whose preconditioner is not block Jacobi
template <typename T>
__global__ void k_pend_scale(int64_t n, const T* __restrict__ w, const double* __restrict__ den, T* __restrict__ v,
                             const T* __restrict__ Vp, int64_t ld, int npend, const double* __restrict__ pc) {
    const T inv = block_inverse<T>(den);
    const T* s_pc = stage_pending<T>(pc, npend);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = pending(w, Vp, ld, npend, s_pc, i) * inv;
}

// v = w / den (FGMRES basis vector)
__global__ void k_scale(int64_t n, const double* __restrict__ w, const double* __restrict__ den, double* __restrict__ v) {
    const double inv = block_inverse<double>(den);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = w[i] * inv;
}

// w += sgn * sum_{q<ncomb} coef[q] V_q, then FP64 dots of the new w with Vd_0..Vd_{nv-1} and itself.
template <typename T, int NVC>
__global__ void __launch_bounds__(RT) k_update_dot(int64_t n, T* __restrict__ w, const T* __restrict__ V, int64_t ld,
                                                    int ncomb, const double* __restrict__ coef, double sgn,
                                                    const T* __restrict__ Vd, int self,
                                                    double* __restrict__ partial, unsigned* __restrict__ counter,
                                                    double* __restrict__ out, int hook, double* sc, GS gsl, int j) {
    __shared__ T s_coef[MMAX + NCCH];
    for (int q = threadIdx.x; q < MMAX + NCCH; q += blockDim.x) s_coef[q] = (q < ncomb) ? T(sgn * coef[q]) : T(0);
    __syncthreads();
    using A = typename AccT<T>::type;
    A dacc[NVMAX + 1];
#pragma unroll
    for (int v = 0; v <= NVMAX; ++v) dacc[v] = A(0);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T v = w[i];
        for (int q = 0; q < ncomb; ++q) v += s_coef[q] * V[q * ld + i];
        if (ncomb > 0) w[i] = v;
        accumulate_dots_n<NVC>(dacc, Vd, ld, i, self, v);
    }
    if (NVC + self > 0) finish_dots(dacc, NVC, self, partial, counter, out, hook, sc, gsl, j);
}

// x = a0 x + Z y with y = R^{-1} g solved redundantly by every block (m <= 64):
// the triangle of H and g are staged in shared memory by all threads, then one
// thread back-substitutes there.  Dynamic shared memory: xupd_smem(m) bytes.
template <typename T>
__global__ void k_update_x(int64_t n, T* __restrict__ x, double a0, const T* __restrict__ Z, int64_t ld,
                           const double* __restrict__ sc, GS L) {
    extern __shared__ double s_dyn[];
    using A = typename AccT<T>::type;
    __shared__ A ya[MMAX + NCCH];
    const int ld2 = L.m + 1;
    double* Hs = s_dyn;
    double* y = s_dyn + ld2 * L.m;
    const int me = (sc[1] == 0.0) ? 0 : (int)sc[2];
    for (int i = threadIdx.x; i < ld2 * me; i += blockDim.x) Hs[i] = sc[L.H + i];
    for (int i = threadIdx.x; i < me; i += blockDim.x) y[i] = sc[L.g + i];
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
    if (threadIdx.x < MMAX + NCCH) ya[threadIdx.x] = ((int)threadIdx.x < me) ? (A)y[threadIdx.x] : A(0);
    __syncthreads();
    const A a0a = (A)a0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < n; i0 += EPT * stride) {
        A sv[EPT];
#pragma unroll
        for (int e = 0; e < EPT; ++e)
            sv[e] = (a0 == 0.0 || i0 + e * stride >= n) ? A(0) : a0a * (A)x[i0 + e * stride];
        for (int q0 = 0; q0 < me; q0 += NCCH) {
            T z[NCCH][EPT];
#pragma unroll
            for (int q = 0; q < NCCH; ++q)
#pragma unroll
                for (int e = 0; e < EPT; ++e)
                    z[q][e] = (q0 + q < me && i0 + e * stride < n) ? __ldg(Z + (q0 + q) * ld + i0 + e * stride) : T(0);
#pragma unroll
            for (int q = 0; q < NCCH; ++q)
#pragma unroll
                for (int e = 0; e < EPT; ++e) sv[e] += ya[q0 + q] * (A)z[q][e];
        }
#pragma unroll
        for (int e = 0; e < EPT; ++e)
            if (i0 + e * stride < n) x[i0 + e * stride] = T(sv[e]);
    }
}

size_t xupd_smem(int m) { return (size_t)((m + 1) * m + m) * sizeof(double); }

// x += zero-padded xc (prolongation)
template <typename T>
__global__ void k_prolong_add(int64_t nf, int64_t ne, int bf, int nFf, int nPf, int bc, int nFc, int nPc, int nEf,
                              int nEc, const T* __restrict__ xc, T* __restrict__ x) {
    const int64_t nfr = nf * bc, ner = ne * nPc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nfr + ner; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < nfr) {
            const int64_t F = i / bc;
            const int rc = (int)(i % bc);
            x[F * bf + (rc / nFc) * nFf + rc % nFc] += xc[i];
        } else {
            const int64_t jj = i - nfr, E = jj / nPc;
            const int rc = (int)(jj % nPc);
            x[nf * bf + E * nPf + (rc / nEc) * nEf + rc % nEc] += xc[i];
        }
    }
}

template <typename S, typename D>
__global__ void k_convert(int64_t n, const S* __restrict__ src, D* __restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = D(src[i]);
}

template <typename T>
__global__ void k_zero(int64_t n, T* __restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = T(0);
}

// x -= (n_p . x) n_p for every problem p: n_p is non-zero only on one unknown
// per kernel slot E (the first pressure unknown of an element, or the
// constant face-pressure coefficient of a face for HHO-hp), xp[E * stride],
// with weight w[E] (0 throughout for a problem without pressure kernel).
// Problem p's slots are split into nch chunks of NP_CHUNK; block (p, c) of
// k_null_dot writes the chunk's partial product, block (p, c) of k_null_sub
// adds the nch partials of p in chunk order (fixed-order trees: deterministic)
// and updates its chunk.
constexpr int NP_CHUNK = 2048;

template <typename T>
__global__ void __launch_bounds__(512) k_null_dot(const int64_t* __restrict__ slot_off, int nch,
                                                  const double* __restrict__ w, const T* __restrict__ xp, int stride,
                                                  double* __restrict__ part) {
    __shared__ double sm[512];
    const int p = blockIdx.x / nch, c = blockIdx.x % nch;
    const int64_t e0 = slot_off[p] + (int64_t)c * NP_CHUNK, e1 = min(slot_off[p + 1], e0 + NP_CHUNK);
    double s = 0.0;
    for (int64_t E = e0 + threadIdx.x; E < e1; E += blockDim.x) s += w[E] * (double)xp[E * stride];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

template <typename T>
__global__ void __launch_bounds__(512) k_null_sub(const int64_t* __restrict__ slot_off, int nch,
                                                  const double* __restrict__ w, T* __restrict__ xp, int stride,
                                                  const double* __restrict__ part) {
    __shared__ double s_a;
    const int p = blockIdx.x / nch, c = blockIdx.x % nch;
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int q = 0; q < nch; ++q) a += part[p * nch + q];
        s_a = a;
    }
    __syncthreads();
    const double a = s_a;
    if (a == 0.0) return;
    const int64_t e0 = slot_off[p] + (int64_t)c * NP_CHUNK, e1 = min(slot_off[p + 1], e0 + NP_CHUNK);
    for (int64_t E = e0 + threadIdx.x; E < e1; E += blockDim.x) xp[E * stride] = T((double)xp[E * stride] - a * w[E]);
}

int rows_per_thread(int nrow) {
    if (nrow % 4 == 0) return 4;
    if (nrow % 3 == 0) return 3;
    if (nrow % 2 == 0) return 2;
    return nrow >= 4 ? 4 : nrow;
}

Items items_for(const LevelMat& L, int R, int frows, int erows) {
    Items it;
    it.ftiles = (L.nf + 31) / 32;
    it.etiles = (L.ne + 31) / 32;
    it.fgroups = (frows + R - 1) / R;
    it.egroups = (erows + R - 1) / R;
    return it;
}

}  // namespace

// ---------------------------------------------------------------------------
// Workspace
// ---------------------------------------------------------------------------
struct LevelWork {
    // smoother vectors in the V-cycle type (double or float)
    void *bv = nullptr, *x = nullptr, *w = nullptr, *V = nullptr, *Z = nullptr;
    void* ilu_tmp = nullptr;  // element-block scratch of the ILU backward sweep
    double* sc = nullptr;
    double *cd = nullptr, *cc = nullptr;  // FP64 coarse right-hand side and solution (mixed precision)
};

struct Workspace {
    std::vector<LevelWork> lv;
    double* partial = nullptr;
    unsigned* counter = nullptr;
    // FGMRES
    int restart = 0;
    double *fV = nullptr, *fZ = nullptr, *fw = nullptr, *fb = nullptr, *fsc = nullptr;
    double* h_sc = nullptr;  // pinned host scalars
    // captured V-cycles
    std::map<std::pair<const double*, double*>, cudaGraphExec_t> graphs;
    std::map<std::pair<const double*, double*>, int64_t> graph_launches;
};

static void free_graphs(Workspace* W) {
    for (auto& g : W->graphs) cudaGraphExecDestroy(g.second);
    W->graphs.clear();
    W->graph_launches.clear();
}

void invalidate_graphs(hho_ctx* ctx) {
    if (ctx->ws) free_graphs(ctx->ws);
    batch_graph_free(ctx);
}

void free_workspace(hho_ctx* ctx) {
    Workspace* W = ctx->ws;
    if (!W) return;
    free_graphs(W);
    for (auto& l : W->lv) {
        dfree(l.bv);
        dfree(l.x);
        dfree(l.w);
        dfree(l.V);
        dfree(l.Z);
        dfree(l.ilu_tmp);
        dfree(l.sc);
        dfree(l.cd);
        dfree(l.cc);
    }
    dfree(W->partial);
    dfree(W->counter);
    dfree(W->fV);
    dfree(W->fZ);
    dfree(W->fw);
    dfree(W->fb);
    dfree(W->fsc);
    if (W->h_sc) cudaFreeHost(W->h_sc);
    delete W;
    ctx->ws = nullptr;
}

// ---- launch helpers (each counts its kernel) ----
static int op_rows(const hho_ctx* ctx, int nrow) {
    return ctx->spmv_rows > 0 ? ctx->spmv_rows : rows_per_thread(nrow);
}

static int op_grid(const hho_ctx* ctx, const Items& it) {
    if (ctx->spmv_grid > 0) return ctx->spmv_grid;
    const int64_t g = (it.total() + (RT / 32) - 1) / (RT / 32);
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, GMAX));
}

// rows of a face held by one thread in k_spmv_b: small blocks whole, larger
// ones split in two or three row groups so that enough warps are in flight
constexpr int face_rows_for(int B) {
    return B <= 4 ? B
                  : (B % 2 == 0 && B <= 12 ? B / 2
                                           : (B % 3 == 0 ? (B / 3 <= 10 ? B / 3 : B / 6) : (B % 4 == 0 ? B / 4 : B)));
}
static_assert(face_rows_for(40) == 10 && face_rows_for(24) == 8 && face_rows_for(30) == 10, "face row groups");

// rows of an element held by one thread: a divisor of the pressure block size
// that the degree behind B gives under velocity-only condensation
// (2D: B = 2(k+1), nP = (k+1)(k+2)/2; 3D: B = 3(k+1)(k+2)/2,
// nP = (k+1)(k+2)(k+3)/6); a level whose nP it does not divide (one pressure
// per element under velocity-pressure condensation) uses RP = 1
constexpr int elem_rows_for(int B) {
    return B == 4 ? 3 : B == 6 ? 3 : B == 8 ? 5 : B == 10 ? 5 : B == 12 ? 7 : B == 9 ? 4 : B == 18 ? 5 : B == 30 ? 5 : 1;
}

template <int B>
static Items items_b(const LevelMat& L, int RP) {
    Items it;
    it.ftiles = (L.nf + 31) / 32;
    it.etiles = (L.ne + 31) / 32;
    it.fgroups = B / face_rows_for(B);
    it.egroups = (L.nP + RP - 1) / RP;
    return it;
}

template <int B, typename T>
static bool launch_spmv_b_B(hho_ctx* ctx, const LevelMat& L, const T* x, const T* bv, T* y, int mode, const T* V,
                            int64_t ld, int nv, int self, double* partial, unsigned* counter, double* out, int hook,
                            double* sc, GS gsl, int j, Restr rs) {
    constexpr int RF = face_rows_for(B);
    constexpr int RPB = elem_rows_for(B);
    const int RP = (L.nP % RPB == 0) ? RPB : 1;  // element row groups are always full
    const Items it = items_b<B>(L, RP);
    const int g = op_grid(ctx, it);
    const LV<T> lv = view<T>(L);
    if (RP == 1)
        k_spmv_b<B, RF, 1, T><<<g, RT, 0, ctx->stream>>>(lv, it, x, bv, y, mode, V, ld, nv, self, partial, counter, out,
                                                         hook, sc, gsl, j, rs);
    else
        k_spmv_b<B, RF, RPB, T><<<g, RT, 0, ctx->stream>>>(lv, it, x, bv, y, mode, V, ld, nv, self, partial, counter,
                                                           out, hook, sc, gsl, j, rs);
    return true;
}

template <int B, typename T>
static void launch_jacobi_b_B(hho_ctx* ctx, const LevelMat& L, const T* w, const double* den, T* v, T* z,
                              const T* Vp, int64_t ld, int npend, const double* pc) {
    constexpr int RF = face_rows_for(B);
    constexpr int RPB = elem_rows_for(B);
    const int RP = (L.nP % RPB == 0) ? RPB : 1;  // element row groups are always full
    const Items it = items_b<B>(L, RP);
    const int64_t g = std::max<int64_t>(1, std::min<int64_t>((it.total() + RT / 32 - 1) / (RT / 32), GMAX));
    const LV<T> lv = view<T>(L);
    if (RP == 1) k_jacobi_b<B, RF, 1, T><<<(int)g, RT, 0, ctx->stream>>>(lv, it, w, den, v, z, Vp, ld, npend, pc);
    else k_jacobi_b<B, RF, RPB, T><<<(int)g, RT, 0, ctx->stream>>>(lv, it, w, den, v, z, Vp, ld, npend, pc);
}

// v = w / den, z = M^{-1} v, with w = w' - sum_{q < npend} pc_q Vp_q when a
// second Gram-Schmidt pass is pending: the compile-time block size kernel where
// B is one of the instantiated sizes, else the generic one
template <typename T>
static void launch_jacobi(hho_ctx* ctx, const LevelMat& L, const T* w, const double* den, T* v, T* z, const T* Vp,
                          int64_t ld, int npend, const double* pc) {
    if constexpr (std::is_same<T, float>::value) {
        if (L.ilv && launch_jacobi_v(ctx, L, w, den, v, z, Vp, ld, npend, pc)) {
            ++ctx->launches;
            return;
        }
    }
    switch (L.b) {
        case 2: launch_jacobi_b_B<2, T>(ctx, L, w, den, v, z, Vp, ld, npend, pc); break;
        case 3: launch_jacobi_b_B<3, T>(ctx, L, w, den, v, z, Vp, ld, npend, pc); break;
        case 4: launch_jacobi_b_B<4, T>(ctx, L, w, den, v, z, Vp, ld, npend, pc); break;
        case 6: launch_jacobi_b_B<6, T>(ctx, L, w, den, v, z, Vp, ld, npend, pc); break;
        case 8: launch_jacobi_b_B<8, T>(ctx, L, w, den, v, z, Vp, ld, npend, pc); break;
        case 9: launch_jacobi_b_B<9, T>(ctx, L, w, den, v, z, Vp, ld, npend, pc); break;
        case 10: launch_jacobi_b_B<10, T>(ctx, L, w, den, v, z, Vp, ld, npend, pc); break;
        case 12: launch_jacobi_b_B<12, T>(ctx, L, w, den, v, z, Vp, ld, npend, pc); break;
        case 18: launch_jacobi_b_B<18, T>(ctx, L, w, den, v, z, Vp, ld, npend, pc); break;
        case 24: launch_jacobi_b_B<24, T>(ctx, L, w, den, v, z, Vp, ld, npend, pc); break;
        case 30: launch_jacobi_b_B<30, T>(ctx, L, w, den, v, z, Vp, ld, npend, pc); break;
        case 40: launch_jacobi_b_B<40, T>(ctx, L, w, den, v, z, Vp, ld, npend, pc); break;
        default:
            k_apply_jacobi<T><<<grid1d(L.n, 256), 256, 0, ctx->stream>>>(view<T>(L), w, den, v, z, Vp, ld, npend,
                                                                         pc);
    }
    ++ctx->launches;
}

// ---- interleaved FP32 kernels (LevelMat::ilv) ----
// Scheme 1 levels with the block sizes of np_full, and the HHO-hp levels above
// the coarse one (no element rows; 2D b = 3 (k+1), 3D b = 12, 24, 40)
static bool ilv_supported(int b, int nP) {
    if (nP == 0) return b == 3 || b == 6 || b == 9 || b == 12 || b == 24 || b == 40;
    return np_full(b) > 0 && (nP == 1 || nP == np_full(b));
}

static Items items_v(const LevelMat& L) {
    Items it;
    it.ftiles = (L.nf + 31) / 32;
    it.etiles = (L.ne + 31) / 32;
    it.fgroups = 1;
    it.egroups = 1;
    return it;
}

// rows of a face block per thread in k_spmv_v: even blocks of 8 or more
// unknowns are split in two halves, others are kept whole.  The half must
// divide B, and a vector load of it must stay aligned: load_run uses 16-byte
// loads only when RF % 4 == 0 (then B % 8 == 0, so every half starts at a
// multiple of 4 floats) and 8-byte loads only when RF is even (B even, every
// run starts at an even float); odd RF (B = 10, 18, 30 halves; B = 3, 9 whole)
// uses scalar loads.
constexpr int rf_v(int B) { return (B >= 8 && B % 2 == 0) ? B / 2 : B; }
static_assert(rf_v(9) == 9 && rf_v(8) == 4 && rf_v(12) == 6 && rf_v(18) == 9 && rf_v(30) == 15, "row split");

template <int B, int NP>
static void launch_spmv_v_BN(hho_ctx* ctx, const LevelMat& L, const float* x, const float* bv, float* y, int mode,
                             const float* V, int64_t ld, int nv, int self, double* partial, unsigned* counter,
                             double* out, int hook, double* sc, GS gsl, int j, Restr rs) {
    if constexpr (B == 18 || B == 30 || B == 24 || B == 40) {  // large 3D face blocks: warp per face
        if (ctx->spmv_warp) {
            Items it;
            it.ftiles = L.nf;
            it.etiles = NP > 0 ? (L.ne + 31) / 32 : 0;
            it.fgroups = it.egroups = 1;
            const int g = op_grid(ctx, it);
            k_spmv_w<B, NP><<<g, RT, 0, ctx->stream>>>(view<float>(L), it.ftiles, it.etiles, x, bv, y, mode, V, ld,
                                                       nv, self, partial, counter, out, hook, sc, gsl, j, rs);
            return;
        }
    }
    constexpr int RF = rf_v(B);
    Items it = items_v(L);
    it.fgroups = B / RF;
    if constexpr (NP == 0) it.etiles = 0;
    const int g = op_grid(ctx, it);
    k_spmv_v<B, NP, RF><<<g, RT, 0, ctx->stream>>>(view<float>(L), it, x, bv, y, mode, V, ld, nv, self, partial,
                                                   counter, out, hook, sc, gsl, j, rs);
}

template <int B, int NP>
static void launch_jacobi_v_BN(hho_ctx* ctx, const LevelMat& L, const float* w, const double* den, float* v,
                               float* z, const float* Vp, int64_t ld, int npend, const double* pc) {
    if constexpr (B == 18 || B == 30 || B == 24 || B == 40) {
        if (ctx->spmv_warp) {
            const int64_t etiles = NP > 0 ? (L.ne + 31) / 32 : 0;
            const int64_t g = std::max<int64_t>(1, std::min<int64_t>((L.nf + etiles + RT / 32 - 1) / (RT / 32), GMAX));
            k_jacobi_w<B, NP><<<(int)g, RT, 0, ctx->stream>>>(view<float>(L), etiles, w, den, v, z, Vp, ld, npend,
                                                              pc);
            return;
        }
    }
    Items it = items_v(L);
    if constexpr (NP == 0) it.etiles = 0;
    const int64_t g = std::max<int64_t>(1, std::min<int64_t>((it.total() + RT / 32 - 1) / (RT / 32), GMAX));
    k_jacobi_v<B, NP><<<(int)g, RT, 0, ctx->stream>>>(view<float>(L), it, w, den, v, z, Vp, ld, npend, pc);
}

#define HHO_BN_SWITCH(CALL)                                                                                        \
    switch (L.b * 64 + L.nP) {                                                                                     \
        case 2 * 64 + 1: CALL(2, 1); break;                                                                        \
        case 4 * 64 + 3: CALL(4, 3); break;                                                                        \
        case 4 * 64 + 1: CALL(4, 1); break;                                                                        \
        case 6 * 64 + 6: CALL(6, 6); break;                                                                        \
        case 6 * 64 + 1: CALL(6, 1); break;                                                                        \
        case 8 * 64 + 10: CALL(8, 10); break;                                                                      \
        case 8 * 64 + 1: CALL(8, 1); break;                                                                        \
        case 10 * 64 + 15: CALL(10, 15); break;                                                                    \
        case 10 * 64 + 1: CALL(10, 1); break;                                                                      \
        case 12 * 64 + 21: CALL(12, 21); break;                                                                    \
        case 12 * 64 + 1: CALL(12, 1); break;                                                                      \
        case 3 * 64 + 1: CALL(3, 1); break;                                                                        \
        case 9 * 64 + 4: CALL(9, 4); break;                                                                        \
        case 9 * 64 + 1: CALL(9, 1); break;                                                                        \
        case 18 * 64 + 10: CALL(18, 10); break;                                                                    \
        case 18 * 64 + 1: CALL(18, 1); break;                                                                      \
        case 30 * 64 + 20: CALL(30, 20); break;                                                                    \
        case 30 * 64 + 1: CALL(30, 1); break;                                                                      \
        case 3 * 64 + 0: CALL(3, 0); break;                                                                        \
        case 6 * 64 + 0: CALL(6, 0); break;                                                                        \
        case 9 * 64 + 0: CALL(9, 0); break;                                                                        \
        case 12 * 64 + 0: CALL(12, 0); break;                                                                      \
        case 24 * 64 + 0: CALL(24, 0); break;                                                                      \
        case 40 * 64 + 0: CALL(40, 0); break;                                                                      \
        default: return false;                                                                                     \
    }

static bool launch_spmv_v(hho_ctx* ctx, const LevelMat& L, const float* x, const float* bv, float* y, int mode,
                          const float* V, int64_t ld, int nv, int self, double* partial, unsigned* counter,
                          double* out, int hook, double* sc, GS gsl, int j, Restr rs) {
#define HHO_SPMV_V(BB, NN) \
    launch_spmv_v_BN<BB, NN>(ctx, L, x, bv, y, mode, V, ld, nv, self, partial, counter, out, hook, sc, gsl, j, rs)
    HHO_BN_SWITCH(HHO_SPMV_V)
#undef HHO_SPMV_V
    return true;
}

static bool launch_jacobi_v(hho_ctx* ctx, const LevelMat& L, const float* w, const double* den, float* v, float* z,
                            const float* Vp, int64_t ld, int npend, const double* pc) {
#define HHO_JAC_V(BB, NN) launch_jacobi_v_BN<BB, NN>(ctx, L, w, den, v, z, Vp, ld, npend, pc)
    HHO_BN_SWITCH(HHO_JAC_V)
#undef HHO_JAC_V
    return true;
}

template <typename T>
static bool launch_spmv_b(hho_ctx* ctx, const LevelMat& L, const T* x, const T* bv, T* y, int mode, const T* V,
                          int64_t ld, int nv, int self, double* partial, unsigned* counter, double* out, int hook,
                          double* sc, GS gsl, int j, Restr rs = Restr{0, 0, 0, 0, 1, 0}) {
    if constexpr (std::is_same<T, float>::value) {
        if (L.ilv) return launch_spmv_v(ctx, L, x, bv, y, mode, V, ld, nv, self, partial, counter, out, hook, sc, gsl,
                                        j, rs);
    }
    if (ctx->spmv_rows > 0) return false;  // explicit row grouping requested: generic kernel
#define HHO_B_CASE(BB)                                                                                             \
    case BB:                                                                                                       \
        return launch_spmv_b_B<BB, T>(ctx, L, x, bv, y, mode, V, ld, nv, self, partial, counter, out, hook, sc, gsl, j, \
                                      rs);
    switch (L.b) {
        HHO_B_CASE(2)
        HHO_B_CASE(3)
        HHO_B_CASE(4)
        HHO_B_CASE(6)
        HHO_B_CASE(8)
        HHO_B_CASE(9)
        HHO_B_CASE(10)
        HHO_B_CASE(12)
        HHO_B_CASE(18)
        HHO_B_CASE(24)
        HHO_B_CASE(30)
        HHO_B_CASE(40)
        default:
            return false;
    }
#undef HHO_B_CASE
}

template <typename T>
static void launch_spmv_dot(hho_ctx* ctx, int l, const T* x, const T* bv, T* y, int mode, const T* V, int64_t ld,
                            int nv, int self, double* out, int hook, double* sc, GS gsl, int j) {
    const LevelMat& L = ctx->levels[l];
    {
        double* partial = ctx->ws ? ctx->ws->partial : nullptr;
        unsigned* counter = ctx->ws ? ctx->ws->counter : nullptr;
        if (launch_spmv_b<T>(ctx, L, x, bv, y, mode, V, ld, nv, self, partial, counter, out, hook, sc, gsl, j)) {
            ++ctx->launches;
            return;
        }
    }
    const int R = op_rows(ctx, std::max(L.b, L.nP));
    Items it = items_for(L, R, L.b, L.nP);
    double* partial = ctx->ws ? ctx->ws->partial : nullptr;
    unsigned* counter = ctx->ws ? ctx->ws->counter : nullptr;
    const int g = op_grid(ctx, it);
    const LV<T> lv = view<T>(L);
    switch (R) {
        case 1:
            k_spmv_dot<1, T><<<g, RT, 0, ctx->stream>>>(lv, it, x, bv, y, mode, V, ld, nv, self, partial, counter, out,
                                                        hook, sc, gsl, j);
            break;
        case 2:
            k_spmv_dot<2, T><<<g, RT, 0, ctx->stream>>>(lv, it, x, bv, y, mode, V, ld, nv, self, partial, counter, out,
                                                        hook, sc, gsl, j);
            break;
        case 3:
            k_spmv_dot<3, T><<<g, RT, 0, ctx->stream>>>(lv, it, x, bv, y, mode, V, ld, nv, self, partial, counter, out,
                                                        hook, sc, gsl, j);
            break;
        default:
            k_spmv_dot<4, T><<<g, RT, 0, ctx->stream>>>(lv, it, x, bv, y, mode, V, ld, nv, self, partial, counter, out,
                                                        hook, sc, gsl, j);
    }
    ++ctx->launches;
}

hho_status spmv(hho_ctx* ctx, int l, const double* x, double* y) {
    launch_spmv_dot<double>(ctx, l, x, nullptr, y, 0, nullptr, 0, 0, 0, nullptr, HOOK_NONE, nullptr, gs_layout(1), 0);
    HHO_CUDA(cudaGetLastError());
    return HHO_OK;
}

hho_status jacobi_apply(hho_ctx* ctx, const double* r, const double* den, double* v, double* z) {
    launch_jacobi<double>(ctx, ctx->levels[0], r, den, v, z, nullptr, 0, 0, nullptr);
    HHO_CUDA(cudaGetLastError());
    return HHO_OK;
}

hho_status residual(hho_ctx* ctx, int l, const double* x, const double* b, double* r) {
    launch_spmv_dot<double>(ctx, l, x, b, r, 1, nullptr, 0, 0, 0, nullptr, HOOK_NONE, nullptr, gs_layout(1), 0);
    HHO_CUDA(cudaGetLastError());
    return HHO_OK;
}

hho_status spmv_f32(hho_ctx* ctx, int l, const float* x, float* y) {
    const LevelMat& L = ctx->levels[l];
    if (!L.ff32) {
        ctx->err = "hho_spmv_f32: no FP32 copy of this level (pmg_setup with HHO_FP32 keeps one below the coarse level)";
        return HHO_ERR_STATE;
    }
    launch_spmv_dot<float>(ctx, l, x, nullptr, y, 0, nullptr, 0, 0, 0, nullptr, HOOK_NONE, nullptr, gs_layout(1), 0);
    HHO_CUDA(cudaGetLastError());
    return HHO_OK;
}

template <typename T>
static void launch_update_dot(hho_ctx* ctx, int64_t n, T* w, const T* V, int64_t ld, int ncomb, const double* coef,
                              double sgn, const T* Vd, int nv, int self, double* out, int hook, double* sc, GS gsl,
                              int j) {
    Workspace* W = ctx->ws;
    // FP64: fewer, longer threads, since every warp's share of the block
    // reductions costs FP64 additions on this part's narrow FP64 pipe
    // (two blocks per SM)
    const int g = std::is_same<T, double>::value ? std::min(vgrid(n), 2 * sm_count()) : vgrid(n);
#define HHO_UPD(NVC)                                                                                               \
    k_update_dot<T, NVC><<<g, RT, 0, ctx->stream>>>(n, w, V, ld, ncomb, coef, sgn, Vd, self, W->partial, W->counter, \
                                                    out, hook, sc, gsl, j)
    switch (nv) {
        case 0: HHO_UPD(0); break;
        case 1: HHO_UPD(1); break;
        case 2: HHO_UPD(2); break;
        case 3: HHO_UPD(3); break;
        case 4: HHO_UPD(4); break;
        case 5: HHO_UPD(5); break;
        case 6: HHO_UPD(6); break;
        case 7: HHO_UPD(7); break;
        default: HHO_UPD(8); break;
    }
#undef HHO_UPD
    ++ctx->launches;
}

// dots of w with V_0..V_{nv-1} in chunks of NVMAX (no hook)
static void dots(hho_ctx* ctx, int64_t n, const double* V, int64_t ld, int nv, double* w, double* out, double* sc,
                 GS gsl, int j) {
    for (int v0 = 0; v0 < nv; v0 += NVMAX) {
        const int cnt = std::min(NVMAX, nv - v0);
        launch_update_dot<double>(ctx, n, w, nullptr, ld, 0, nullptr, 0.0, V + v0 * ld, cnt, 0, out + v0, HOOK_NONE, sc,
                                  gsl, j);
    }
}

// m iterations of right-preconditioned GMRES on level l: x <- x + Z y (x = Z y when x_zero).
// beta_ready: ||bv||^2 is already in sc[0] with the START hook run (by the restriction kernel).
template <typename T>
static hho_status smooth(hho_ctx* ctx, int l, const T* bv, T* x, bool x_zero, bool beta_ready, bool post) {
    const LevelMat& L = ctx->levels[l];
    LevelWork& lw = ctx->ws->lv[l];
    const int m = ctx->smooth_its;
    const int64_t n = L.n;
    if (m == 0) {
        if (x_zero) {
            k_zero<T><<<grid1d(n, 256), 256, 0, ctx->stream>>>(n, x);
            ++ctx->launches;
        }
        return HHO_OK;
    }
    GS G = gs_layout(m);
    double* sc = lw.sc;
    T* w = static_cast<T*>(lw.w);
    T* V = static_cast<T*>(lw.V);
    T* Z = static_cast<T*>(lw.Z);
    const T* w0;
    if (x_zero) {
        if (!beta_ready)
            launch_update_dot<T>(ctx, n, const_cast<T*>(bv), nullptr, n, 0, nullptr, 0.0, bv, 1, 0, sc + 0, HOOK_START,
                                 sc, G, 0);
        w0 = bv;
    } else {
        launch_spmv_dot<T>(ctx, l, x, bv, w, 1, nullptr, n, 0, 1, sc + 0, HOOK_START, sc, G, 0);
        w0 = w;
    }
    for (int j = 0; j < m; ++j) {
        T* vj = V + (int64_t)j * n;
        T* zj = Z + (int64_t)j * n;
        // the second pass of step j-1 (w'' = w' - V t2) is applied inside the Jacobi kernel
        if (ctx->smoother_kind == 1 && l < (int)ctx->ilu.size() && ctx->ilu[l]) {
            k_pend_scale<T><<<grid1d(n, 256), 256, 0, ctx->stream>>>(n, j == 0 ? w0 : w, sc + 5, vj, V, n, j,
                                                                     sc + G.t2);
            ++ctx->launches;
            HHO_TRY(ilu_apply<T>(ctx, l, vj, zj, static_cast<T*>(lw.ilu_tmp)));
        } else {
            launch_jacobi<T>(ctx, L, j == 0 ? w0 : w, sc + 5, vj, zj, V, n, j, sc + G.t2);
        }
        // learned correction in the finest-level post-smoother, whose error the coarse correction has
        // stripped of its low-frequency part (the distribution of the training pairs)
        if (l == 0 && post && ctx->use_learned && ctx->learned) HHO_TRY(mlp_apply<T>(ctx, vj, zj));
        if (std::is_same<T, float>::value) {
            // FP32 V-cycle: one reduction per step, w = S z_j, t2 = V^T w and ||w||^2 together; Hessenberg
            // column t2 with ||w - V t2||^2 = ||w||^2 - ||t2||^2, the projection left to the consumer
            launch_spmv_dot<T>(ctx, l, zj, nullptr, w, 0, V, n, j + 1, 1, sc + G.t2, HOOK_COLUMN_1R, sc, G, j);
        } else {
            launch_spmv_dot<T>(ctx, l, zj, nullptr, w, 0, V, n, j + 1, 0, sc + G.t1, HOOK_NONE, sc, G, j);
            // w' = w - V t1, t2 = V^T w', ||w'||^2; Hessenberg column with ||w''||^2 = ||w'||^2 - ||t2||^2
            launch_update_dot<T>(ctx, n, w, V, n, j + 1, sc + G.t1, -1.0, V, j + 1, 1, sc + G.t2, HOOK_COLUMN_PY, sc,
                                 G, j);
        }
    }
    k_update_x<T><<<vgrid(n), RT, xupd_smem(G.m), ctx->stream>>>(n, x, x_zero ? 0.0 : 1.0, Z, n, sc, G);
    ++ctx->launches;
    HHO_CUDA(cudaGetLastError());
    return HHO_OK;
}

static hho_status host_read(hho_ctx* ctx, const double* dsrc, double* hdst, int count) {
    HHO_CUDA(cudaMemcpyAsync(hdst, dsrc, count * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    HHO_CUDA(cudaStreamSynchronize(ctx->stream));
    return HHO_OK;
}

template <int R, typename T>
static void restrict_R(hho_ctx* ctx, const LevelMat& F, const LevelMat& C, Items it, const T* x, const T* bv, T* d,
                       int do_norm, double* sc, GS G) {
    Workspace* W = ctx->ws;
    const int ec = elem_comp(ctx->disc.cond, ctx->disc.d);
    k_residual_restrict<R, T><<<op_grid(ctx, it), RT, 0, ctx->stream>>>(view<T>(F), it, F.nF, C.b, C.nF, C.nP,
                                                                        F.nP / ec, C.nP / ec, x, bv, d, do_norm,
                                                                        W->partial, W->counter, sc, sc, G);
}

template <typename T>
static hho_status coarse_level(hho_ctx* ctx, int l, const T* d, T* c);

template <>
hho_status coarse_level<double>(hho_ctx* ctx, int, const double* d, double* c) {
    return coarse_apply(ctx, d, c);
}

template <>
hho_status coarse_level<float>(hho_ctx* ctx, int l, const float* d, float* c) {
    if (ctx->coarse_fp32 && coarse_has_f32(ctx)) return coarse_apply_f32(ctx, d, c);
    LevelWork& lw = ctx->ws->lv[l];
    const int64_t n = ctx->levels[l].n;
    k_convert<float, double><<<grid1d(n, 256), 256, 0, ctx->stream>>>(n, d, lw.cd);
    HHO_TRY(coarse_apply(ctx, lw.cd, lw.cc));
    k_convert<double, float><<<grid1d(n, 256), 256, 0, ctx->stream>>>(n, lw.cc, c);
    ctx->launches += 2;
    HHO_CUDA(cudaGetLastError());
    return HHO_OK;
}

// MG_V(l, b, w): iterate in x (zero initial guess when x_zero).
template <typename T>
static hho_status vcycle_level(hho_ctx* ctx, int l, const T* bv, T* x, bool x_zero, bool beta_ready) {
    const int Lc = (int)ctx->levels.size() - 1;
    const LevelMat& F = ctx->levels[l];
    const LevelMat& C = ctx->levels[l + 1];
    LevelWork& cw = ctx->ws->lv[l + 1];
    T* cbv = static_cast<T*>(cw.bv);
    T* cx = static_cast<T*>(cw.x);
    HHO_TRY(smooth<T>(ctx, l, bv, x, x_zero, beta_ready, false));
    const bool coarse_next = (l + 1 == Lc);
    const int Rc = op_rows(ctx, std::max(C.b, C.nP));
    Items it = items_for(F, Rc, C.b, C.nP);
    GS Gc = gs_layout(std::max(ctx->smooth_its, 1));
    const int do_norm = (!coarse_next && ctx->smooth_its > 0) ? 1 : 0;
    const int ec = elem_comp(ctx->disc.cond, ctx->disc.d);
    const Restr rs{F.nF, C.nF, C.b, C.nP, F.nP / ec, C.nP / ec};
    if (launch_spmv_b<T>(ctx, F, x, bv, cbv, 2, nullptr, 0, 0, do_norm, ctx->ws->partial, ctx->ws->counter, cw.sc,
                         do_norm ? HOOK_START : HOOK_NONE, cw.sc, Gc, 0, rs)) {
        // fused into the operator kernel specialised on the fine block size
    } else switch (Rc) {
        case 1: restrict_R<1, T>(ctx, F, C, it, x, bv, cbv, do_norm, cw.sc, Gc); break;
        case 2: restrict_R<2, T>(ctx, F, C, it, x, bv, cbv, do_norm, cw.sc, Gc); break;
        case 3: restrict_R<3, T>(ctx, F, C, it, x, bv, cbv, do_norm, cw.sc, Gc); break;
        default: restrict_R<4, T>(ctx, F, C, it, x, bv, cbv, do_norm, cw.sc, Gc);
    }
    ++ctx->launches;
    HHO_CUDA(cudaGetLastError());
    if (coarse_next) HHO_TRY(coarse_level<T>(ctx, l + 1, cbv, cx));
    else HHO_TRY(vcycle_level<T>(ctx, l + 1, cbv, cx, true, do_norm != 0));
    k_prolong_add<T><<<grid1d(C.n, 256), 256, 0, ctx->stream>>>(F.nf, F.ne, F.b, F.nF, F.nP, C.b, C.nF, C.nP,
                                                                F.nP / ec, C.nP / ec, cx, x);
    ++ctx->launches;
    HHO_CUDA(cudaGetLastError());
    // the iterate after the coarse correction, for the learned smoother's training pairs
    if (l == 0 && ctx->capture) {
        HHO_CUDA(cudaMemcpyAsync(ctx->capture, x, (size_t)F.n * sizeof(T), cudaMemcpyDeviceToDevice, ctx->stream));
    }
    HHO_TRY(smooth<T>(ctx, l, bv, x, false, false, true));
    return HHO_OK;
}

static hho_status vcycle_direct(hho_ctx* ctx, const double* r, double* z) {
    if (ctx->levels.size() == 1) return coarse_apply(ctx, r, z);
    if (ctx->prec == HHO_FP64) return vcycle_level<double>(ctx, 0, r, z, true, false);
    // mixed precision: FP32 copy of r in, FP32 iterate converted out
    LevelWork& lw = ctx->ws->lv[0];
    const int64_t n = ctx->levels[0].n;
    float* rb = static_cast<float*>(lw.bv);
    float* xz = static_cast<float*>(lw.x);
    k_convert<double, float><<<grid1d(n, 256), 256, 0, ctx->stream>>>(n, r, rb);
    ++ctx->launches;
    HHO_TRY(vcycle_level<float>(ctx, 0, rb, xz, true, false));
    k_convert<float, double><<<grid1d(n, 256), 256, 0, ctx->stream>>>(n, xz, z);
    ++ctx->launches;
    HHO_CUDA(cudaGetLastError());
    return HHO_OK;
}

// V-cycle through a CUDA graph captured once per (r, z) pair; direct launches on
// the legacy default stream, which cannot be captured.
hho_status vcycle(hho_ctx* ctx, const double* r, double* z) {
    Workspace* W = ctx->ws;
    if (ctx->stream == nullptr || !ctx->use_graphs) return vcycle_direct(ctx, r, z);
    auto key = std::make_pair(r, z);
    auto itg = W->graphs.find(key);
    if (itg == W->graphs.end()) {
        if (W->graphs.size() >= 128) free_graphs(W);
        const int64_t before = ctx->launches;
        const int64_t coarse_before = ctx->coarse_its_total;
        HHO_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        hho_status st = vcycle_direct(ctx, r, z);
        cudaGraph_t graph = nullptr;
        cudaError_t ee = cudaStreamEndCapture(ctx->stream, &graph);
        if (st != HHO_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        HHO_CUDA(ee);
        cudaGraphExec_t exec = nullptr;
        cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        HHO_CUDA(ie);
        W->graphs[key] = exec;
        W->graph_launches[key] = ctx->launches - before;
        ctx->launches = before;
        ctx->coarse_its_total = coarse_before;
        itg = W->graphs.find(key);
    }
    HHO_CUDA(cudaGraphLaunch(itg->second, ctx->stream));
    ctx->launches += W->graph_launches[key];
    ctx->coarse_its_total += 1;
    return HHO_OK;
}

template <typename T>
hho_status null_project(hho_ctx* ctx, const LevelMat& L, T* x) {
    if (!ctx->has_null) return HHO_OK;
    T* xp = x + null_slot(ctx, L, 0);
    const int stride = null_in_blocks(ctx->disc.cond) ? L.b : L.nP, nch = ctx->null_nch;
    const unsigned g = (unsigned)(ctx->probs.P * nch);
    k_null_dot<T><<<g, 512, 0, ctx->stream>>>(ctx->d_null_off, nch, ctx->null_w, xp, stride, ctx->null_part);
    k_null_sub<T><<<g, 512, 0, ctx->stream>>>(ctx->d_null_off, nch, ctx->null_w, xp, stride, ctx->null_part);
    ctx->launches += 2;
    HHO_CUDA(cudaGetLastError());
    return HHO_OK;
}
template hho_status null_project<double>(hho_ctx*, const LevelMat&, double*);
template hho_status null_project<float>(hho_ctx*, const LevelMat&, float*);

// Per-problem pressure kernels: a problem without Neumann face has the
// constant pressure in the kernel of its operator.  Scheme 1: its unit kernel
// vector has sqrt(|T|) / sqrt(|Omega_p|) on the first (constant) pressure
// unknown of each element T (orthonormal bases: the constant 1 has
// coefficient sqrt|T|).  HHO-hp: the constant hybrid pressure (p_T = p_F = 1)
// condensed to the skeleton is sqrt(|F|) on the constant face-pressure
// coefficient of every face F, normalised by sqrt(sum_F |F|).
hho_status null_build(hho_ctx* ctx) {
    Problems& pr = ctx->probs;
    const Disc& D = ctx->disc;
    pr.has_null.assign(pr.P, 1);
    for (int p = 0; p < pr.P; ++p)
        for (int64_t F = pr.face_off[p]; F < pr.face_off[p + 1]; ++F)
            if (D.h_fbc[F] == 2) {
                pr.has_null[p] = 0;
                break;
            }
    ctx->has_null = false;
    for (char h : pr.has_null) ctx->has_null |= (h != 0);
    dfree(ctx->null_w);
    ctx->null_w = nullptr;
    dfree(ctx->d_null_off);
    ctx->d_null_off = nullptr;
    dfree(ctx->null_part);
    ctx->null_part = nullptr;
    ctx->h_null_w.clear();
    if (!ctx->has_null) return HHO_OK;
    const bool hp = D.cond == HHO_HPCOND;
    const std::vector<int64_t>& off = hp ? pr.face_off : pr.elem_off;
    const int64_t ns = hp ? D.nf : D.ne;
    std::vector<double> meas(ns), w(ns, 0.0);
    if (hp) {
        std::vector<FaceGeo> g(D.nf);
        HHO_CUDA(cudaMemcpy(g.data(), D.fgeo, D.nf * sizeof(FaceGeo), cudaMemcpyDeviceToHost));
        for (int64_t F = 0; F < D.nf; ++F) meas[F] = g[F].meas;
    } else {
        HHO_CUDA(cudaMemcpy(meas.data(), D.emeas, D.ne * sizeof(double), cudaMemcpyDeviceToHost));
    }
    for (int p = 0; p < pr.P; ++p) {
        if (!pr.has_null[p]) continue;
        double tot = 0.0;
        for (int64_t E = off[p]; E < off[p + 1]; ++E) tot += meas[E];
        const double inv = 1.0 / std::sqrt(tot);
        for (int64_t E = off[p]; E < off[p + 1]; ++E) w[E] = std::sqrt(meas[E]) * inv;
    }
    ctx->h_null_w = w;
    HHO_TRY(dalloc(ctx, &ctx->null_w, w.size()));
    HHO_CUDA(cudaMemcpy(ctx->null_w, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice));
    HHO_TRY(dalloc(ctx, &ctx->d_null_off, off.size()));
    HHO_CUDA(cudaMemcpy(ctx->d_null_off, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    int64_t most = 1;
    for (int p = 0; p < pr.P; ++p) most = std::max<int64_t>(most, off[p + 1] - off[p]);
    ctx->null_nch = (int)((most + NP_CHUNK - 1) / NP_CHUNK);
    HHO_TRY(dalloc(ctx, &ctx->null_part, (size_t)pr.P * ctx->null_nch));
    return HHO_OK;
}

static hho_status make_fp32_copy(hho_ctx* ctx, const double* src, float** dst, size_t n) {
    dfree(*dst);
    *dst = nullptr;
    HHO_TRY(dalloc(ctx, dst, n));
    k_convert<double, float><<<grid1d((int64_t)n, 256), 256, 0, ctx->stream>>>((int64_t)n, src, *dst);
    HHO_CUDA(cudaGetLastError());
    return HHO_OK;
}

static hho_status make_fp32_interleaved(hho_ctx* ctx, const double* src, float** dst, int64_t planes, int R,
                                        int64_t N) {
    dfree(*dst);
    *dst = nullptr;
    HHO_TRY(dalloc(ctx, dst, (size_t)planes * R * N));
    k_interleave<<<grid1d(planes * R * N, 256), 256, 0, ctx->stream>>>(planes, R, N, src, *dst);
    HHO_CUDA(cudaGetLastError());
    return HHO_OK;
}

hho_status pmg_build(hho_ctx* ctx) {
    free_workspace(ctx);
    Workspace* W = new Workspace();
    ctx->ws = W;
    const int nl = (int)ctx->levels.size();
    W->lv.resize(nl);
    const int m = std::max(ctx->smooth_its, 1);
    GS G = gs_layout(m);
    const bool mixed = ctx->prec == HHO_FP32;
    const size_t es = mixed ? sizeof(float) : sizeof(double);
    for (int l = 0; l < nl; ++l) {
        LevelMat& L = ctx->levels[l];
        const int64_t n = L.n;
        LevelWork& w = W->lv[l];
        HHO_TRY(device_alloc(ctx, &w.bv, n * es));
        HHO_TRY(device_alloc(ctx, &w.x, n * es));
        HHO_TRY(device_alloc(ctx, &w.w, n * es));
        HHO_TRY(device_alloc(ctx, &w.V, (size_t)(m + 1) * n * es));
        HHO_TRY(device_alloc(ctx, &w.Z, (size_t)m * n * es));
        HHO_TRY(device_alloc(ctx, &w.ilu_tmp, (size_t)std::max<int64_t>(L.ne * L.nP, 1) * es));
        HHO_TRY(dalloc(ctx, &w.sc, G.total));
        HHO_CUDA(cudaMemset(w.sc, 0, G.total * sizeof(double)));
        if (mixed && l < nl - 1) {
            L.ilv = ilv_supported(L.b, L.nP);
            if (L.ilv) {
                HHO_TRY(make_fp32_interleaved(ctx, L.ff, &L.ff32, (int64_t)L.S_max * L.b, L.b, L.nf));
                HHO_TRY(make_fp32_interleaved(ctx, L.fp, &L.fp32, (int64_t)2 * L.nP, L.b, L.nf));
                HHO_TRY(make_fp32_interleaved(ctx, L.pf, &L.pf32, (int64_t)L.N_max * L.b, L.nP, L.ne));
                HHO_TRY(make_fp32_interleaved(ctx, L.pp, &L.pp32, L.nP, L.nP, L.ne));
                HHO_TRY(make_fp32_interleaved(ctx, L.dinv, &L.dinv32, L.b, L.b, L.nf));
                HHO_TRY(make_fp32_interleaved(ctx, L.minv, &L.minv32, L.nP, L.nP, L.ne));
            } else {
                HHO_TRY(make_fp32_copy(ctx, L.ff, &L.ff32, (size_t)L.S_max * L.b * L.b * L.nf));
                HHO_TRY(make_fp32_copy(ctx, L.fp, &L.fp32, (size_t)2 * L.nP * L.b * L.nf));
                HHO_TRY(make_fp32_copy(ctx, L.pf, &L.pf32, (size_t)L.N_max * L.b * L.nP * L.ne));
                HHO_TRY(make_fp32_copy(ctx, L.pp, &L.pp32, (size_t)L.nP * L.nP * L.ne));
                HHO_TRY(make_fp32_copy(ctx, L.dinv, &L.dinv32, (size_t)L.b * L.b * L.nf));
                HHO_TRY(make_fp32_copy(ctx, L.minv, &L.minv32, (size_t)L.nP * L.nP * L.ne));
            }
        }
        if (mixed && l == nl - 1 && nl > 1) {
            HHO_TRY(dalloc(ctx, &w.cd, n));
            HHO_TRY(dalloc(ctx, &w.cc, n));
        }
    }
    HHO_TRY(dalloc(ctx, &W->partial, (size_t)(NVMAX + 1) * GMAX));
    HHO_TRY(dalloc(ctx, &W->counter, 16));
    HHO_CUDA(cudaMemset(W->counter, 0, 16 * sizeof(unsigned)));
    HHO_CUDA(cudaMallocHost(&W->h_sc, 64 * sizeof(double)));
    HHO_TRY(null_build(ctx));
    ilu_free(ctx);
    if (ctx->smoother_kind == 1)
        for (int l = 0; l < nl - 1; ++l) HHO_TRY(ilu_setup(ctx, l, mixed));
    HHO_TRY(coarse_setup(ctx));
    return HHO_OK;
}

hho_status fgmres(hho_ctx* ctx, double rtol, int maxit, int restart, double* x, hho_solve_info* info) {
    Workspace* W = ctx->ws;
    const LevelMat& L0 = ctx->levels[0];
    const int64_t n = L0.n;
    if (restart < 1 || restart > 64 || maxit < 0 || !(rtol > 0.0)) {
        ctx->err = "hho_solve: invalid restart (1..64), maxit or rtol";
        return HHO_ERR_ARG;
    }
    if (W->restart != restart) {
        W->restart = 0;  // until every buffer below exists (a failed allocation must not leave stale ones)
        for (double** p : {&W->fV, &W->fZ, &W->fw, &W->fb, &W->fsc}) {
            dfree(*p);
            *p = nullptr;
        }
        HHO_TRY(dalloc(ctx, &W->fV, (size_t)(restart + 1) * n));
        HHO_TRY(dalloc(ctx, &W->fZ, (size_t)restart * n));
        HHO_TRY(dalloc(ctx, &W->fw, n));
        HHO_TRY(dalloc(ctx, &W->fb, n));
        HHO_TRY(dalloc(ctx, &W->fsc, gs_layout(restart).total + 8));
        HHO_CUDA(cudaMemset(W->fsc, 0, (gs_layout(restart).total + 8) * sizeof(double)));
        W->restart = restart;
    }
    GS G = gs_layout(restart);
    double* sc = W->fsc;
    double* hs = W->h_sc;
    double* bvec = W->fb;
    cudaEvent_t e0, e1;
    HHO_CUDA(cudaEventCreate(&e0));
    HHO_CUDA(cudaEventCreate(&e1));
    HHO_CUDA(cudaEventRecord(e0, ctx->stream));
    ctx->coarse_its_total = 0;
    k_convert<double, double><<<grid1d(n, 256), 256, 0, ctx->stream>>>(n, ctx->rhs, bvec);
    ++ctx->launches;
    HHO_TRY(null_project<double>(ctx, L0, bvec));
    k_zero<double><<<grid1d(n, 256), 256, 0, ctx->stream>>>(n, x);
    ++ctx->launches;
    // ||b||, which is also beta of the first restart cycle (r = b)
    launch_update_dot<double>(ctx, n, bvec, nullptr, n, 0, nullptr, 0.0, bvec, 1, 0, sc + 0, HOOK_START, sc, G, 0);
    HHO_TRY(host_read(ctx, sc + 1, hs, 1));
    const double bnorm = hs[0];
    int it = 0;
    double relres = 0.0;
    hho_status st = HHO_OK;
    if (bnorm > 0.0) {
        bool conv = false;
        const double* r = bvec;
        double beta = bnorm;
        while (it < maxit) {
            if (beta <= rtol * bnorm) {
                conv = true;
                break;
            }
            k_scale<<<grid1d(n, 256), 256, 0, ctx->stream>>>(n, r, sc + 5, W->fV);
            ++ctx->launches;
            for (int j = 0; j < restart; ++j) {
                double* vj = W->fV + (int64_t)j * n;
                double* zj = W->fZ + (int64_t)j * n;
                HHO_TRY(vcycle(ctx, vj, zj));
                const int nv = j + 1;
                const int c0 = std::min(nv, NVMAX);
                // w = S z_j, t1 = V^T w
                launch_spmv_dot<double>(ctx, 0, zj, nullptr, W->fw, 0, W->fV, n, c0, 0, sc + G.t1, HOOK_NONE, sc, G, j);
                if (nv > c0) dots(ctx, n, W->fV + (int64_t)c0 * n, n, nv - c0, W->fw, sc + G.t1 + c0, sc, G, j);
                // w -= V t1, t2 = V^T w
                launch_update_dot<double>(ctx, n, W->fw, W->fV, n, nv, sc + G.t1, -1.0, W->fV, c0, 0, sc + G.t2,
                                          HOOK_NONE, sc, G, j);
                if (nv > c0) dots(ctx, n, W->fV + (int64_t)c0 * n, n, nv - c0, W->fw, sc + G.t2 + c0, sc, G, j);
                // w -= V t2, ||w||^2, Hessenberg column and Givens rotation
                launch_update_dot<double>(ctx, n, W->fw, W->fV, n, nv, sc + G.t2, -1.0, nullptr, 0, 1, sc + G.nrm,
                                          HOOK_COLUMN, sc, G, j);
                ++it;
                HHO_TRY(host_read(ctx, sc + 3, hs, 2));
                const bool stop = hs[0] <= rtol * bnorm || hs[1] != 0.0 || it >= maxit;
                if (stop || j + 1 == restart) break;
                k_scale<<<grid1d(n, 256), 256, 0, ctx->stream>>>(n, W->fw, sc + 5, W->fV + (int64_t)(j + 1) * n);
                ++ctx->launches;
            }
            // x += Z y over the columns of this cycle
            k_update_x<double><<<vgrid(n), RT, xupd_smem(G.m), ctx->stream>>>(n, x, 1.0, W->fZ, n, sc, G);
            ++ctx->launches;
            // true residual, its norm and the START state of the next cycle
            launch_spmv_dot<double>(ctx, 0, x, bvec, W->fw, 1, nullptr, n, 0, 1, sc + 0, HOOK_START, sc, G, 0);
            HHO_TRY(host_read(ctx, sc + 1, hs, 1));
            beta = hs[0];
            r = W->fw;
            if (beta <= rtol * bnorm) {
                conv = true;
                break;
            }
        }
        if (ctx->has_null) {
            HHO_TRY(null_project<double>(ctx, L0, x));
            launch_spmv_dot<double>(ctx, 0, x, bvec, W->fw, 1, nullptr, n, 0, 1, sc + 0, HOOK_START, sc, G, 0);
            HHO_TRY(host_read(ctx, sc + 1, hs, 1));
            beta = hs[0];
        }
        relres = beta / bnorm;
        if (!conv && relres > rtol) st = HHO_ERR_NOT_CONVERGED;
    }
    HHO_CUDA(cudaEventRecord(e1, ctx->stream));
    HHO_CUDA(cudaEventSynchronize(e1));
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
