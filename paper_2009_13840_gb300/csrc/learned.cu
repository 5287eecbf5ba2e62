// Learned block smoother (an extension; the paper's smoother is ILU-GMRES,
// replaced here by block-Jacobi GMRES).  A two-layer MLP maps the residual of
// a face's neighbourhood to a correction of the block-Jacobi output on that
// face's rows, in the finest-level post-smoother's GMRES:
//   z = M_J^{-1} v + C(v),  C(v)_F = s_F (W2^T relu(W1^T x_F / s_F + b1) + b2)[:b]
// where x_F gathers the residual blocks of the faces in F's operator slots
// (F, the other faces of its first element, of its second) and the pressure
// blocks of its two elements, and s_F = ||x_F||.  The map is homogeneous of
// degree one; the smoother's GMRES stores its preconditioned vectors, so a
// nonlinear preconditioner is admissible (flexible form).
//
// Weights: FP32 masters, BF16 copies used by every forward pass; features in
// BF16; all accumulation in FP32.  Training data: pairs (r, e) generated by
// the FP64 V-cycle itself (see mlp_generate; by default the error and residual
// its finest-level post-smoother meets), with targets
// t_F = (e_F - (M_J^{-1} r)_F) / s_F; loss = mean ||y - t||^2.  The correction
// is applied in the finest-level post-smoother only, where the error matches
// that distribution.  Training runs on the GPU (forward, backward and Adam
// kernels below).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"
#include "tc.cuh"

namespace hho {

struct Learned {
    int din = 0, hid = 0, dout = 0, raw = 0;  // padded input, hidden, padded output, raw feature count
    int S_max = 0, b = 0, nP = 0;
    int64_t nf = 0;
    // parameters: FP32 masters, Adam moments, BF16 copies of the matrices
    float *W1 = nullptr, *b1 = nullptr, *W2 = nullptr, *b2 = nullptr;
    float *mW1 = nullptr, *mb1 = nullptr, *mW2 = nullptr, *mb2 = nullptr;
    float *vW1 = nullptr, *vb1 = nullptr, *vW2 = nullptr, *vb2 = nullptr;
    float *gW1 = nullptr, *gb1 = nullptr, *gW2 = nullptr, *gb2 = nullptr;
    __nv_bfloat16 *W1h = nullptr, *W2h = nullptr;
    int64_t adam_t = 0;
    // training set
    int64_t nsamp = 0;
    __nv_bfloat16* X = nullptr;  // nsamp x din
    float* T = nullptr;          // nsamp x dout
    // minibatch work
    int bcap = 0;
    __nv_bfloat16* Xb = nullptr;
    float *Tb = nullptr, *H = nullptr, *dY = nullptr, *dH = nullptr, *lossp = nullptr, *losses = nullptr;
    int loss_cap = 0;
    bool tc = false;              // first layer on the tensor cores (tc_ok)
    int* d_status = nullptr;      // device status word of the tensor-core kernels (bounded waits)
};

namespace {

constexpr int FB = 32;    // faces (samples) per block in the MLP kernels
constexpr int MT = 128;   // threads per block in the MLP kernels

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double u01(uint64_t h) { return ((h >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

// e[i] ~ N(0, 1) from a counter-based generator (SplitMix64 of seed and index,
// Box-Muller on the two halves of one draw pair)
__global__ void k_randn(int64_t n, uint64_t seed, double* __restrict__ e) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t h1 = mix64(seed ^ mix64(2 * (uint64_t)i)), h2 = mix64(seed ^ mix64(2 * (uint64_t)i + 1));
        const double u = u01(h1), v = u01(h2);
        e[i] = sqrt(-2.0 * log(u)) * cos(6.283185307179586 * v);
    }
}

__global__ void k_sub(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ c) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c[i] = a[i] - b[i];
}

__global__ void k_fill(int64_t n, double v, double* __restrict__ a) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = v;
}

struct Topo0 {
    int64_t nf;
    int b, nP, S_max, raw, din;
    const int32_t *ff_col, *ff_nsl, *fp_col;
};

// Raw feature j of face F from the vector r (level-0 layout), 0 when absent.
template <typename T>
__device__ __forceinline__ float feature(const Topo0& t, const T* __restrict__ r, int64_t F, int j) {
    if (j < t.S_max * t.b) {
        const int s = j / t.b, c = j - s * t.b;
        if (s >= t.ff_nsl[F]) return 0.f;
        const int64_t G = t.ff_col[(int64_t)s * t.nf + F];
        return (float)r[G * t.b + c];
    }
    if (j < t.raw) {
        const int q = j - t.S_max * t.b, p = q / t.nP, c = q - p * t.nP;
        const int E = t.fp_col[(int64_t)p * t.nf + F];
        if (E < 0) return 0.f;
        return (float)r[t.nf * t.b + (int64_t)E * t.nP + c];
    }
    return 0.f;
}

// s_F of face F: sequential FP32 sum of squares of its raw features in order
template <typename T>
__device__ __forceinline__ float feature_norm(const Topo0& t, const T* __restrict__ r, int64_t F) {
    float a = 0.f;
    for (int j = 0; j < t.raw; ++j) {
        const float f = feature(t, r, F, j);
        a += f * f;
    }
    return sqrtf(a);
}

// Stage FB faces' features in shared memory (sx[f][din], normalised) and their
// norms (ss[f]).  Faces past nf get zero features.
template <typename T>
__device__ void stage_features(const Topo0& t, const T* __restrict__ r, int64_t F0, float* sx, float* ss) {
    for (int idx = threadIdx.x; idx < FB * t.din; idx += blockDim.x) {
        const int f = idx / t.din, j = idx - f * t.din;
        const int64_t F = F0 + f;
        sx[idx] = (F < t.nf) ? feature(t, r, F, j) : 0.f;
    }
    __syncthreads();
    // s_F: sequential FP32 sum of squares in feature order (the same arithmetic
    // as feature_norm, so every kernel sees identical normalised features)
    for (int f = threadIdx.x; f < FB; f += blockDim.x) {
        float a = 0.f;
        for (int j = 0; j < t.din; ++j) a += sx[f * t.din + j] * sx[f * t.din + j];
        ss[f] = sqrtf(a);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < FB * t.din; idx += blockDim.x) {
        const float s = ss[idx / t.din];
        const float v = (s > 0.f) ? sx[idx] / s : 0.f;
        sx[idx] = __bfloat162float(__float2bfloat16_rn(v));  // the network sees BF16 inputs
    }
    __syncthreads();
}

// Hidden layer for FB samples held in shared memory: thread j < hid computes
// unit j for every sample: sh[f][j] = relu(sum_i sx[f][i] W1[i][j] + b1[j]).
__device__ void hidden_layer(int din, int hid, const float* sx, const __nv_bfloat16* __restrict__ W1,
                             const float* __restrict__ b1, float* sh) {
    for (int j = threadIdx.x; j < hid; j += blockDim.x) {
        float acc[FB];
#pragma unroll
        for (int f = 0; f < FB; ++f) acc[f] = b1[j];
        for (int i = 0; i < din; ++i) {
            const float w = __bfloat162float(W1[(int64_t)i * hid + j]);
#pragma unroll
            for (int f = 0; f < FB; ++f) acc[f] += sx[f * din + i] * w;
        }
#pragma unroll
        for (int f = 0; f < FB; ++f) sh[f * hid + j] = fmaxf(acc[f], 0.f);
    }
    __syncthreads();
}

// Output layer: y[f][k] = sum_j sh[f][j] W2[j][k] + b2[k] for f < FB, k < dout.
__device__ __forceinline__ float out_unit(int hid, int dout, const float* sh, const __nv_bfloat16* __restrict__ W2,
                                          const float* __restrict__ b2, int f, int k) {
    float a = b2[k];
    for (int j = 0; j < hid; ++j) a += sh[f * hid + j] * __bfloat162float(W2[(int64_t)j * dout + k]);
    return a;
}

// Smoother correction on the finest level: z_F += s_F y_F[:b] (face rows only).
template <typename T>
__global__ void __launch_bounds__(MT) k_mlp_apply(Topo0 t, int hid, int dout, const T* __restrict__ v,
                                                  T* __restrict__ z, const __nv_bfloat16* __restrict__ W1,
                                                  const float* __restrict__ b1, const __nv_bfloat16* __restrict__ W2,
                                                  const float* __restrict__ b2) {
    extern __shared__ float smem[];
    float* sx = smem;                 // FB x din
    float* sh = sx + FB * t.din;      // FB x hid
    float* ss = sh + FB * hid;        // FB
    const int64_t F0 = (int64_t)blockIdx.x * FB;
    stage_features<T>(t, v, F0, sx, ss);
    hidden_layer(t.din, hid, sx, W1, b1, sh);
    for (int idx = threadIdx.x; idx < FB * t.b; idx += blockDim.x) {
        const int f = idx / t.b, k = idx - f * t.b;
        const int64_t F = F0 + f;
        if (F >= t.nf || !(ss[f] > 0.f)) continue;
        const float y = out_unit(hid, dout, sh, W2, b2, f, k);
        z[F * t.b + k] += (T)(ss[f] * y);
    }
}

// ---------------------------------------------------------------------------
// Tensor-core first layer (tcgen05, BF16 x BF16 -> FP32 in TMEM).  A CTA of 128
// threads holds W1^T (hid x din, BF16) in shared memory for the whole launch
// and loops over tiles of 128 faces (samples): the tile's normalised BF16
// features are staged as the A operand, one thread issues the din/16 MMAs of
// the 128 x hid x din product, and every thread then reads its row of the
// accumulator from TMEM in chunks of 32 columns, applies b1 and the ReLU and
// runs the (small) second layer on the CUDA cores from W2 in shared memory.
// Products of BF16 values are exact in FP32, so the layer computes what the
// CUDA-core version computes up to the order of the FP32 additions.
// Requirements: hid a multiple of 32 in 32..256, din a multiple of 16,
// dout <= 32, and the shared-memory footprint of tc_smem.
// ---------------------------------------------------------------------------
constexpr int TC_ROWS = 128;
constexpr int TC_WAIT = 1 << 22;  // bounded polls of the MMA-completion barrier

__host__ __device__ inline uint32_t tc_cols(int hid) {
    uint32_t c = 32;
    while ((int)c < hid) c <<= 1;
    return c;
}

size_t tc_smem(int din, int hid, int dout) {
    return (size_t)(hid + TC_ROWS) * din * 2 + (size_t)(hid * dout + hid + dout + TC_ROWS) * 4;
}

bool tc_ok(int din, int hid, int dout) {
    return hid % 32 == 0 && hid >= 32 && hid <= 256 && din % 16 == 0 && dout <= 32 &&
           tc_smem(din, hid, dout) <= 227 * 1024;
}

struct TcSmem {
    __nv_bfloat16 *B, *A;
    float *W2, *b1, *b2, *ss;
};

__device__ TcSmem tc_carve(unsigned char* smem, int din, int hid, int dout) {
    TcSmem m;
    m.B = reinterpret_cast<__nv_bfloat16*>(smem);
    m.A = m.B + (size_t)hid * din;
    m.W2 = reinterpret_cast<float*>(m.A + (size_t)TC_ROWS * din);
    m.b1 = m.W2 + hid * dout;
    m.b2 = m.b1 + hid;
    m.ss = m.b2 + dout;
    return m;
}

// W1^T as the B operand (row n = hidden unit n over the din inputs), W2, biases
__device__ void tc_load_weights(const TcSmem& m, int din, int hid, int dout, const __nv_bfloat16* __restrict__ W1,
                                const float* __restrict__ b1, const __nv_bfloat16* __restrict__ W2,
                                const float* __restrict__ b2) {
    for (int idx = threadIdx.x; idx < din * hid; idx += blockDim.x) {
        const int i = idx / hid, j = idx - i * hid;
        m.B[tc::core_off(j, i, din)] = W1[idx];
    }
    for (int idx = threadIdx.x; idx < hid * dout; idx += blockDim.x) m.W2[idx] = __bfloat162float(W2[idx]);
    for (int idx = threadIdx.x; idx < hid; idx += blockDim.x) m.b1[idx] = b1[idx];
    for (int idx = threadIdx.x; idx < dout; idx += blockDim.x) m.b2[idx] = b2[idx];
}

// y[0..dout) = W2^T relu(acc + b1) + b2 for this thread's accumulator row
__device__ __forceinline__ void tc_second_layer(const TcSmem& m, uint32_t tmem, int hid, int dout, float (&y)[32],
                                                float* __restrict__ Hrow) {
    const int warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 32; ++k) y[k] = k < dout ? m.b2[k] : 0.f;
    for (int c0 = 0; c0 < hid; c0 += 32) {
        float h[32];
        tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, h);
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            const float hq = fmaxf(h[q] + m.b1[c0 + q], 0.f);
            if (Hrow) Hrow[c0 + q] = hq;
            const float* w = m.W2 + (c0 + q) * dout;
#pragma unroll
            for (int k = 0; k < 32; ++k)
                if (k < dout) y[k] += hq * w[k];
        }
    }
}

// Finest-level smoother correction z_F += s_F y_F[:b] with the first layer on
// the tensor cores (persistent: grid-stride over tiles of 128 faces).
template <typename T>
__global__ void __launch_bounds__(TC_ROWS, 1) k_mlp_apply_tc(Topo0 t, int hid, int dout, const T* __restrict__ v,
                                                            T* __restrict__ z, const __nv_bfloat16* __restrict__ W1,
                                                            const float* __restrict__ b1,
                                                            const __nv_bfloat16* __restrict__ W2,
                                                            const float* __restrict__ b2, int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_bar;
    const int din = t.din;
    const TcSmem m = tc_carve(tc_smem_raw, din, hid, dout);
    const uint32_t ncols = tc_cols(hid);
    tc_load_weights(m, din, hid, dout, W1, b1, W2, b2);
    if (threadIdx.x < 32) tc::tmem_alloc(&s_tmem, ncols);
    if (threadIdx.x == 0) tc::mbar_init(&s_bar);
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    uint32_t parity = 0;
    const int64_t ntiles = (t.nf + TC_ROWS - 1) / TC_ROWS;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t F = tile * TC_ROWS + threadIdx.x;
        const bool act = F < t.nf;
        const float sF = act ? feature_norm(t, v, F) : 0.f;
        m.ss[threadIdx.x] = sF;
        for (int j = 0; j < din; ++j) {
            const float x = (act && sF > 0.f) ? feature(t, v, F, j) / sF : 0.f;
            m.A[tc::core_off(threadIdx.x, j, din)] = __float2bfloat16_rn(x);
        }
        tc::fence_smem_to_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (threadIdx.x == 0) tc::mma_tile(tmem, m.A, m.B, din, hid, &s_bar);
        const bool ok = tc::mbar_wait(&s_bar, parity, TC_WAIT);
        parity ^= 1u;
        if (!ok) {
            if (threadIdx.x == 0) atomicExch(status, (int)HHO_ERR_TIMEOUT);
            break;  // uniform: every thread polls the same barrier
        }
        tc::fence_after_sync();
        float y[32];
        tc_second_layer(m, tmem, hid, dout, y, nullptr);
        if (act && sF > 0.f)
            for (int k = 0; k < t.b; ++k) z[F * t.b + k] += (T)(sF * y[k]);
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) tc::tmem_free(tmem, ncols);
}

// Training forward over a minibatch with the first layer on the tensor cores:
// H (B x hid, FP32 after relu), dY = 2 (Y - T) / B and one partial loss per
// tile of 128 samples.
template <typename XT>
__global__ void __launch_bounds__(TC_ROWS, 1) k_train_fwd_tc(int B, int din, int hid, int dout,
                                                            const XT* __restrict__ X, const float* __restrict__ Tt,
                                                            const __nv_bfloat16* __restrict__ W1,
                                                            const float* __restrict__ b1,
                                                            const __nv_bfloat16* __restrict__ W2,
                                                            const float* __restrict__ b2, float* __restrict__ H,
                                                            float* __restrict__ dY, float* __restrict__ lossp,
                                                            int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ float red[TC_ROWS];
    const TcSmem m = tc_carve(tc_smem_raw, din, hid, dout);
    const uint32_t ncols = tc_cols(hid);
    tc_load_weights(m, din, hid, dout, W1, b1, W2, b2);
    if (threadIdx.x < 32) tc::tmem_alloc(&s_tmem, ncols);
    if (threadIdx.x == 0) tc::mbar_init(&s_bar);
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    uint32_t parity = 0;
    const int ntiles = (B + TC_ROWS - 1) / TC_ROWS;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int i0 = tile * TC_ROWS;
        for (int idx = threadIdx.x; idx < TC_ROWS * din; idx += blockDim.x) {
            const int r = idx / din, j = idx - r * din;
            const float x = (i0 + r < B) ? (float)X[(int64_t)(i0 + r) * din + j] : 0.f;
            m.A[tc::core_off(r, j, din)] = __float2bfloat16_rn(x);
        }
        tc::fence_smem_to_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (threadIdx.x == 0) tc::mma_tile(tmem, m.A, m.B, din, hid, &s_bar);
        const bool ok = tc::mbar_wait(&s_bar, parity, TC_WAIT);
        parity ^= 1u;
        if (!ok) {
            if (threadIdx.x == 0) atomicExch(status, (int)HHO_ERR_TIMEOUT);
            break;
        }
        tc::fence_after_sync();
        const int i = i0 + threadIdx.x;
        float y[32];
        tc_second_layer(m, tmem, hid, dout, y, i < B ? H + (int64_t)i * hid : nullptr);
        float l = 0.f;
        if (i < B) {
            for (int k = 0; k < dout; ++k) {
                const float d = y[k] - Tt[(int64_t)i * dout + k];
                dY[(int64_t)i * dout + k] = 2.f * d / (float)B;
                l += d * d;
            }
        }
        red[threadIdx.x] = l;
        __syncthreads();
        for (int o = TC_ROWS / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) lossp[tile] = red[0] / (float)B;
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) tc::tmem_free(tmem, ncols);
}

// Training samples of one generated pair: X rows (BF16, normalised features),
// targets T = (e_F - (M_J^{-1} r)_F) / s_F (zero-padded to dout).
__global__ void __launch_bounds__(MT) k_samples(Topo0 t, int dout, const double* __restrict__ r,
                                                const double* __restrict__ e, const double* __restrict__ jr,
                                                __nv_bfloat16* __restrict__ X, float* __restrict__ Tt) {
    extern __shared__ float smem[];
    float* sx = smem;
    float* ss = sx + FB * t.din;
    const int64_t F0 = (int64_t)blockIdx.x * FB;
    stage_features<double>(t, r, F0, sx, ss);
    for (int idx = threadIdx.x; idx < FB * t.din; idx += blockDim.x) {
        const int64_t F = F0 + idx / t.din;
        if (F < t.nf) X[F * t.din + idx % t.din] = __float2bfloat16_rn(sx[idx]);
    }
    for (int idx = threadIdx.x; idx < FB * dout; idx += blockDim.x) {
        const int f = idx / dout, k = idx - f * dout;
        const int64_t F = F0 + f;
        if (F >= t.nf) continue;
        float v = 0.f;
        if (k < t.b && ss[f] > 0.f) v = (float)((e[F * t.b + k] - jr[F * t.b + k]) / (double)ss[f]);
        Tt[F * dout + k] = v;
    }
}

// Features of a vector (test hook): X (nf x din, FP32 values of the BF16 inputs) and norms
__global__ void __launch_bounds__(MT) k_features(Topo0 t, const double* __restrict__ r, float* __restrict__ X,
                                                 float* __restrict__ s) {
    extern __shared__ float smem[];
    float* sx = smem;
    float* ss = sx + FB * t.din;
    const int64_t F0 = (int64_t)blockIdx.x * FB;
    stage_features<double>(t, r, F0, sx, ss);
    for (int idx = threadIdx.x; idx < FB * t.din; idx += blockDim.x) {
        const int64_t F = F0 + idx / t.din;
        if (F < t.nf) X[F * t.din + idx % t.din] = sx[idx];
    }
    for (int f = threadIdx.x; f < FB; f += blockDim.x)
        if (F0 + f < t.nf) s[F0 + f] = ss[f];
}

// Minibatch: sample i takes training row hash(seed, i) mod nsamp.
__global__ void k_gather(int64_t nsamp, int din, int dout, int B, uint64_t seed,
                         const __nv_bfloat16* __restrict__ X, const float* __restrict__ T,
                         __nv_bfloat16* __restrict__ Xb, float* __restrict__ Tb) {
    for (int i = blockIdx.x; i < B; i += gridDim.x) {
        const int64_t row = (int64_t)(mix64(seed ^ mix64((uint64_t)i)) % (uint64_t)nsamp);
        for (int j = threadIdx.x; j < din; j += blockDim.x) Xb[(int64_t)i * din + j] = X[row * din + j];
        for (int j = threadIdx.x; j < dout; j += blockDim.x) Tb[(int64_t)i * dout + j] = T[row * dout + j];
    }
}

// Forward over a minibatch: H (B x hid, FP32 after relu), dY = 2 (Y - T) / B,
// per-block partial losses.  Inputs may be BF16 (training) or FP32 (grads hook).
template <typename XT>
__global__ void __launch_bounds__(MT) k_train_fwd(int B, int din, int hid, int dout, const XT* __restrict__ X,
                                                  const float* __restrict__ Tt, const __nv_bfloat16* __restrict__ W1,
                                                  const float* __restrict__ b1, const __nv_bfloat16* __restrict__ W2,
                                                  const float* __restrict__ b2, float* __restrict__ H,
                                                  float* __restrict__ dY, float* __restrict__ lossp) {
    extern __shared__ float smem[];
    float* sx = smem;
    float* sh = sx + FB * din;
    __shared__ float red[MT];
    const int i0 = blockIdx.x * FB;
    for (int idx = threadIdx.x; idx < FB * din; idx += blockDim.x) {
        const int i = i0 + idx / din;
        sx[idx] = (i < B) ? (float)X[(int64_t)i * din + idx % din] : 0.f;
    }
    __syncthreads();
    hidden_layer(din, hid, sx, W1, b1, sh);
    for (int idx = threadIdx.x; idx < FB * hid; idx += blockDim.x) {
        const int i = i0 + idx / hid;
        if (i < B) H[(int64_t)i * hid + idx % hid] = sh[idx];
    }
    float l = 0.f;
    for (int idx = threadIdx.x; idx < FB * dout; idx += blockDim.x) {
        const int f = idx / dout, k = idx - f * dout, i = i0 + f;
        if (i >= B) continue;
        const float d = out_unit(hid, dout, sh, W2, b2, f, k) - Tt[(int64_t)i * dout + k];
        dY[(int64_t)i * dout + k] = 2.f * d / (float)B;
        l += d * d;
    }
    red[threadIdx.x] = l;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) lossp[blockIdx.x] = red[0] / (float)B;
}

// dH = (dY W2^T) * [H > 0]
__global__ void k_train_dh(int B, int hid, int dout, const float* __restrict__ dY, const __nv_bfloat16* __restrict__ W2,
                           const float* __restrict__ H, float* __restrict__ dH) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)B * hid;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / hid;
        const int j = (int)(idx - i * hid);
        float a = 0.f;
        if (H[idx] > 0.f)
            for (int k = 0; k < dout; ++k) a += dY[i * dout + k] * __bfloat162float(W2[(int64_t)j * dout + k]);
        dH[idx] = a;
    }
}

// Weight gradients, one thread per parameter, samples in order (deterministic):
// dW1[i][j] = sum_s X[s][i] dH[s][j], db1[j] = sum_s dH[s][j],
// dW2[j][k] = sum_s H[s][j] dY[s][k], db2[k] = sum_s dY[s][k].
template <typename XT>
__global__ void k_train_gw(int B, int din, int hid, int dout, const XT* __restrict__ X, const float* __restrict__ dH,
                           const float* __restrict__ H, const float* __restrict__ dY, float* __restrict__ gW1,
                           float* __restrict__ gb1, float* __restrict__ gW2, float* __restrict__ gb2) {
    const int64_t n1 = (int64_t)din * hid, n2 = n1 + hid, n3 = n2 + (int64_t)hid * dout, n4 = n3 + dout;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n4; p += (int64_t)gridDim.x * blockDim.x) {
        float a = 0.f;
        if (p < n1) {
            const int i = (int)(p / hid), j = (int)(p % hid);
            for (int s = 0; s < B; ++s) a += (float)X[(int64_t)s * din + i] * dH[(int64_t)s * hid + j];
            gW1[p] = a;
        } else if (p < n2) {
            const int j = (int)(p - n1);
            for (int s = 0; s < B; ++s) a += dH[(int64_t)s * hid + j];
            gb1[j] = a;
        } else if (p < n3) {
            const int64_t q = p - n2;
            const int j = (int)(q / dout), k = (int)(q % dout);
            for (int s = 0; s < B; ++s) a += H[(int64_t)s * hid + j] * dY[(int64_t)s * dout + k];
            gW2[q] = a;
        } else {
            const int k = (int)(p - n3);
            for (int s = 0; s < B; ++s) a += dY[(int64_t)s * dout + k];
            gb2[k] = a;
        }
    }
}

// Adam (Kingma & Ba) on one parameter array; optional BF16 copy of the result
__global__ void k_adam(int64_t n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1c, float b2c, __nv_bfloat16* __restrict__ wh) {
    const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        m[i] = beta1 * m[i] + (1.f - beta1) * gi;
        v[i] = beta2 * v[i] + (1.f - beta2) * gi * gi;
        const float mh = m[i] / b1c, vh = v[i] / b2c;
        w[i] -= lr * mh / (sqrtf(vh) + eps);
        if (wh) wh[i] = __float2bfloat16_rn(w[i]);
    }
}

__global__ void k_to_bf16(int64_t n, const float* __restrict__ a, __nv_bfloat16* __restrict__ b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = __float2bfloat16_rn(a[i]);
}

__global__ void k_sum_losses(int nb, const float* __restrict__ lossp, float* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        float s = 0.f;
        for (int i = 0; i < nb; ++i) s += lossp[i];
        *out = s;
    }
}

int g1(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 32)); }

Topo0 topo0(const hho_ctx* ctx, const Learned* M) {
    const LevelMat& L = ctx->levels[0];
    return Topo0{L.nf, M->b, M->nP, M->S_max, M->raw, M->din, L.ff_col, L.ff_nsl, L.fp_col};
}

size_t feat_smem(int din, int hid) { return (size_t)(FB * din + FB * hid + FB) * sizeof(float); }

}  // namespace

void mlp_free(hho_ctx* ctx) {
    Learned* M = ctx->learned;
    if (!M) return;
    void* ps[] = {M->W1, M->b1, M->W2, M->b2, M->mW1, M->mb1, M->mW2, M->mb2, M->vW1, M->vb1, M->vW2, M->vb2,
                  M->gW1, M->gb1, M->gW2, M->gb2, M->W1h, M->W2h, M->X, M->T, M->Xb, M->Tb, M->H, M->dY, M->dH,
                  M->lossp, M->losses, M->d_status};
    for (void* p : ps) dfree(p);
    delete M;
    ctx->learned = nullptr;
}

hho_status mlp_init(hho_ctx* ctx, int hidden, uint64_t seed) {
    if (ctx->levels.empty() || !ctx->have_pmg) {
        ctx->err = "hho_mlp_init: call pmg_setup first";
        return HHO_ERR_STATE;
    }
    if (hidden < 8 || hidden > 256 || hidden % 8) {
        ctx->err = "hho_mlp_init: hidden width must be a multiple of 8 in 8..256";
        return HHO_ERR_ARG;
    }
    mlp_free(ctx);
    const LevelMat& L = ctx->levels[0];
    Learned* M = new Learned();
    ctx->learned = M;
    M->S_max = ctx->topo.S_max;
    M->b = L.b;
    M->nP = L.nP;
    M->nf = L.nf;
    M->raw = M->S_max * M->b + 2 * M->nP;
    M->din = (M->raw + 15) / 16 * 16;
    M->hid = hidden;
    M->dout = (M->b + 7) / 8 * 8;
    M->tc = tc_ok(M->din, M->hid, M->dout);
    if (M->din > (M->tc ? 512 : 256)) {
        ctx->err = "hho_mlp_init: neighbourhood features exceed the kernels' limit (256 values, 512 with the "
                   "tensor-core first layer: hidden width a multiple of 32)";
        mlp_free(ctx);
        return HHO_ERR_UNSUPPORTED;
    }
    HHO_TRY(dalloc(ctx, &M->d_status, 1));
    HHO_CUDA(cudaMemset(M->d_status, 0, sizeof(int)));
    {
        // dynamic shared memory above the default 48 KB where a kernel needs it
        const size_t fs = feat_smem(M->din, M->hid), ss = (size_t)(FB * M->din + FB) * 4;
        const size_t fw = (size_t)(FB * M->din + FB * M->hid) * 4;
        HHO_TRY(allow_smem(ctx, k_mlp_apply<double>, fs));
        HHO_TRY(allow_smem(ctx, k_mlp_apply<float>, fs));
        HHO_TRY(allow_smem(ctx, k_train_fwd<__nv_bfloat16>, fw));
        HHO_TRY(allow_smem(ctx, k_train_fwd<float>, fw));
        HHO_TRY(allow_smem(ctx, k_samples, ss));
        HHO_TRY(allow_smem(ctx, k_features, ss));
        if (M->tc) {
            const size_t ts = tc_smem(M->din, M->hid, M->dout);
            HHO_TRY(allow_smem(ctx, k_mlp_apply_tc<double>, ts));
            HHO_TRY(allow_smem(ctx, k_mlp_apply_tc<float>, ts));
            HHO_TRY(allow_smem(ctx, k_train_fwd_tc<__nv_bfloat16>, ts));
            HHO_TRY(allow_smem(ctx, k_train_fwd_tc<float>, ts));
        }
    }
    const int64_t n1 = (int64_t)M->din * M->hid, n2 = (int64_t)M->hid * M->dout;
    float** fp[] = {&M->W1, &M->mW1, &M->vW1, &M->gW1};
    for (float** p : fp) HHO_TRY(dalloc(ctx, p, (size_t)n1));
    float** fq[] = {&M->W2, &M->mW2, &M->vW2, &M->gW2};
    for (float** p : fq) HHO_TRY(dalloc(ctx, p, (size_t)n2));
    float** fr[] = {&M->b1, &M->mb1, &M->vb1, &M->gb1};
    for (float** p : fr) HHO_TRY(dalloc(ctx, p, (size_t)M->hid));
    float** fs[] = {&M->b2, &M->mb2, &M->vb2, &M->gb2};
    for (float** p : fs) HHO_TRY(dalloc(ctx, p, (size_t)M->dout));
    HHO_TRY(dalloc(ctx, &M->W1h, (size_t)n1));
    HHO_TRY(dalloc(ctx, &M->W2h, (size_t)n2));
    // He-uniform first layer, small second layer (the correction starts near zero)
    std::vector<float> w1(n1), w2(n2), z1(M->hid, 0.f), z2(M->dout, 0.f);
    uint64_t st = seed;
    auto next = [&]() {
        st += 0x9E3779B97F4A7C15ull;
        uint64_t z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return ((z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    };
    const double a1 = std::sqrt(6.0 / M->raw), a2 = 0.1 * std::sqrt(6.0 / M->hid);
    for (int64_t i = 0; i < n1; ++i) w1[i] = (float)((2.0 * next() - 1.0) * (i / M->hid < M->raw ? a1 : 0.0));
    for (int64_t i = 0; i < n2; ++i) w2[i] = (float)((2.0 * next() - 1.0) * ((i % M->dout) < M->b ? a2 : 0.0));
    HHO_CUDA(cudaMemcpy(M->W1, w1.data(), n1 * 4, cudaMemcpyHostToDevice));
    HHO_CUDA(cudaMemcpy(M->W2, w2.data(), n2 * 4, cudaMemcpyHostToDevice));
    HHO_CUDA(cudaMemcpy(M->b1, z1.data(), M->hid * 4, cudaMemcpyHostToDevice));
    HHO_CUDA(cudaMemcpy(M->b2, z2.data(), M->dout * 4, cudaMemcpyHostToDevice));
    float* zs[] = {M->mW1, M->vW1, M->mW2, M->vW2, M->mb1, M->vb1, M->mb2, M->vb2};
    const int64_t zn[] = {n1, n1, n2, n2, M->hid, M->hid, M->dout, M->dout};
    for (int i = 0; i < 8; ++i) HHO_CUDA(cudaMemset(zs[i], 0, zn[i] * 4));
    k_to_bf16<<<g1(n1), 256, 0, ctx->stream>>>(n1, M->W1, M->W1h);
    k_to_bf16<<<g1(n2), 256, 0, ctx->stream>>>(n2, M->W2, M->W2h);
    HHO_CUDA(cudaGetLastError());
    HHO_CUDA(cudaStreamSynchronize(ctx->stream));
    M->adam_t = 0;
    return HHO_OK;
}

hho_status mlp_dims(hho_ctx* ctx, int* dims) {
    const Learned* M = ctx->learned;
    if (!M) {
        ctx->err = "learned smoother: call hho_mlp_init first";
        return HHO_ERR_STATE;
    }
    dims[0] = M->din;
    dims[1] = M->hid;
    dims[2] = M->dout;
    dims[3] = M->raw;
    return HHO_OK;
}

hho_status mlp_weights(hho_ctx* ctx, int set, double* W1, double* b1, double* W2, double* b2) {
    Learned* M = ctx->learned;
    if (!M) {
        ctx->err = "learned smoother: call hho_mlp_init first";
        return HHO_ERR_STATE;
    }
    const int64_t n1 = (int64_t)M->din * M->hid, n2 = (int64_t)M->hid * M->dout;
    double* hp[] = {W1, b1, W2, b2};
    float* dp[] = {M->W1, M->b1, M->W2, M->b2};
    const int64_t nn[] = {n1, M->hid, n2, M->dout};
    for (int a = 0; a < 4; ++a) {
        std::vector<float> tmp(nn[a]);
        if (set) {
            for (int64_t i = 0; i < nn[a]; ++i) tmp[i] = (float)hp[a][i];
            HHO_CUDA(cudaMemcpy(dp[a], tmp.data(), nn[a] * 4, cudaMemcpyHostToDevice));
        } else {
            HHO_CUDA(cudaMemcpy(tmp.data(), dp[a], nn[a] * 4, cudaMemcpyDeviceToHost));
            for (int64_t i = 0; i < nn[a]; ++i) hp[a][i] = tmp[i];
        }
    }
    if (set) {
        k_to_bf16<<<g1(n1), 256, 0, ctx->stream>>>(n1, M->W1, M->W1h);
        k_to_bf16<<<g1(n2), 256, 0, ctx->stream>>>(n2, M->W2, M->W2h);
        HHO_CUDA(cudaGetLastError());
        HHO_CUDA(cudaStreamSynchronize(ctx->stream));
        invalidate_graphs(ctx);
    }
    return HHO_OK;
}

hho_status mlp_features(hho_ctx* ctx, const double* r, float* X, float* s) {
    Learned* M = ctx->learned;
    if (!M) {
        ctx->err = "learned smoother: call hho_mlp_init first";
        return HHO_ERR_STATE;
    }
    const Topo0 t = topo0(ctx, M);
    const int nb = (int)((M->nf + FB - 1) / FB);
    k_features<<<nb, MT, (size_t)(FB * M->din + FB) * 4, ctx->stream>>>(t, r, X, s);
    HHO_CUDA(cudaGetLastError());
    HHO_CUDA(cudaStreamSynchronize(ctx->stream));
    return HHO_OK;
}

template <typename T>
hho_status mlp_apply(hho_ctx* ctx, const T* v, T* z) {
    Learned* M = ctx->learned;
    const Topo0 t = topo0(ctx, M);
    if (M->tc) {
        const int64_t ntiles = (M->nf + TC_ROWS - 1) / TC_ROWS;
        const int g = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, sm_count()));
        k_mlp_apply_tc<T><<<g, TC_ROWS, tc_smem(M->din, M->hid, M->dout), ctx->stream>>>(
            t, M->hid, M->dout, v, z, M->W1h, M->b1, M->W2h, M->b2, M->d_status);
    } else {
        const int nb = (int)((M->nf + FB - 1) / FB);
        k_mlp_apply<T><<<nb, MT, feat_smem(M->din, M->hid), ctx->stream>>>(t, M->hid, M->dout, v, z, M->W1h, M->b1,
                                                                            M->W2h, M->b2);
    }
    ++ctx->launches;
    HHO_CUDA(cudaGetLastError());
    return HHO_OK;
}

// Status word of the tensor-core kernels (a bounded wait that expired), read
// after the synchronising entry points that ran them; cleared when read.
hho_status mlp_status(hho_ctx* ctx) {
    Learned* M = ctx->learned;
    if (!M || !M->tc) return HHO_OK;
    int st = 0;
    HHO_CUDA(cudaMemcpyAsync(&st, M->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    HHO_CUDA(cudaStreamSynchronize(ctx->stream));
    if (st != 0) {
        HHO_CUDA(cudaMemsetAsync(M->d_status, 0, sizeof(int), ctx->stream));
        ctx->err = "learned smoother: a tensor-core kernel gave up waiting for its MMAs";
        return (hho_status)st;
    }
    return HHO_OK;
}
template hho_status mlp_apply<double>(hho_ctx*, const double*, double*);
template hho_status mlp_apply<float>(hho_ctx*, const float*, float*);

// Forward pass of a minibatch (H, dY, partial losses): tensor-core first layer
// when available, else the CUDA-core kernel.
template <typename XT>
static void train_forward(hho_ctx* ctx, Learned* M, int B, const XT* X, const float* Tt, size_t sm) {
    if (M->tc) {
        const int ntiles = (B + TC_ROWS - 1) / TC_ROWS;
        const int g = std::max(1, std::min(ntiles, sm_count()));
        k_train_fwd_tc<XT><<<g, TC_ROWS, tc_smem(M->din, M->hid, M->dout), ctx->stream>>>(
            B, M->din, M->hid, M->dout, X, Tt, M->W1h, M->b1, M->W2h, M->b2, M->H, M->dY, M->lossp, M->d_status);
    } else {
        const int nbk = (B + FB - 1) / FB;
        k_train_fwd<XT><<<nbk, MT, sm, ctx->stream>>>(B, M->din, M->hid, M->dout, X, Tt, M->W1h, M->b1, M->W2h,
                                                      M->b2, M->H, M->dY, M->lossp);
    }
}

static hho_status ensure_batch(hho_ctx* ctx, Learned* M, int B) {
    if (B <= M->bcap) return HHO_OK;
    void* ps[] = {M->Xb, M->Tb, M->H, M->dY, M->dH, M->lossp};
    for (void* p : ps) dfree(p);
    HHO_TRY(dalloc(ctx, &M->Xb, (size_t)B * M->din));
    HHO_TRY(dalloc(ctx, &M->Tb, (size_t)B * M->dout));
    HHO_TRY(dalloc(ctx, &M->H, (size_t)B * M->hid));
    HHO_TRY(dalloc(ctx, &M->dY, (size_t)B * M->dout));
    HHO_TRY(dalloc(ctx, &M->dH, (size_t)B * M->hid));
    HHO_TRY(dalloc(ctx, &M->lossp, (size_t)(B + FB - 1) / FB));
    M->bcap = B;
    return HHO_OK;
}

// Training pairs from the FP64 V-cycle for n_vec white-noise errors e0 (the
// V-cycle applied to r0 = S e0):
//   kind 0  the pair it is applied to (e = e0, r = r0)
//   kind 1  the pair it leaves (e = e0 - MG(r0), r = S e)
//   kind 2  the pair its finest-level post-smoother meets: e = e0 - x_cc with
//           x_cc the iterate after the coarse correction, r = S e
hho_status mlp_generate(hho_ctx* ctx, int n_vec, uint64_t seed, int kind, int64_t* nsamp) {
    Learned* M = ctx->learned;
    if (!M) {
        ctx->err = "learned smoother: call hho_mlp_init first";
        return HHO_ERR_STATE;
    }
    if (ctx->prec != HHO_FP64) {
        ctx->err = "hho_mlp_generate: the training pairs come from the FP64 V-cycle (pmg_setup with HHO_FP64)";
        return HHO_ERR_STATE;
    }
    if (n_vec < 1 || n_vec > 4096 || kind < 0 || kind > 2) {
        ctx->err = "hho_mlp_generate: n_vec must be in 1..4096 and kind 0, 1 or 2";
        return HHO_ERR_ARG;
    }
    const LevelMat& L = ctx->levels[0];
    const int64_t n = L.n;
    dfree(M->X);
    dfree(M->T);
    M->X = nullptr;
    M->T = nullptr;
    M->nsamp = (int64_t)n_vec * M->nf;
    HHO_TRY(dalloc(ctx, &M->X, (size_t)M->nsamp * M->din));
    HHO_TRY(dalloc(ctx, &M->T, (size_t)M->nsamp * M->dout));
    double *e0 = nullptr, *r0 = nullptr, *z = nullptr, *e = nullptr, *r = nullptr, *jr = nullptr, *jv = nullptr,
           *one = nullptr;
    double** bufs[] = {&e0, &r0, &z, &e, &r, &jr, &jv};
    for (double** p : bufs) HHO_TRY(dalloc(ctx, p, (size_t)n));
    HHO_CUDA(cudaMemsetAsync(z, 0, (size_t)n * sizeof(double), ctx->stream));
    HHO_TRY(dalloc(ctx, &one, 1));
    k_fill<<<1, 32, 0, ctx->stream>>>(1, 1.0, one);
    const int saved = ctx->use_learned;
    const bool saved_graphs = ctx->use_graphs;
    ctx->use_learned = 0;
    ctx->use_graphs = false;  // the capture copy must see this call's buffers
    invalidate_graphs(ctx);
    const Topo0 t = topo0(ctx, M);
    const int nb = (int)((M->nf + FB - 1) / FB);
    hho_status st = HHO_OK;
    for (int v = 0; v < n_vec && st == HHO_OK; ++v) {
        k_randn<<<g1(n), 256, 0, ctx->stream>>>(n, seed * 0x100000001B3ull + (uint64_t)v, e0);
        st = spmv(ctx, 0, e0, r0);
        if (st != HHO_OK) break;
        if (kind == 0) {
            k_sub<<<g1(n), 256, 0, ctx->stream>>>(n, e0, z, e);  // z is still zero: e = e0
            st = spmv(ctx, 0, e, r);
        } else {
            double* xcc = jv;  // scratch: the iterate after the coarse correction
            ctx->capture = (kind == 2) ? xcc : nullptr;
            st = vcycle(ctx, r0, z);
            ctx->capture = nullptr;
            if (st != HHO_OK) break;
            k_sub<<<g1(n), 256, 0, ctx->stream>>>(n, e0, kind == 2 ? xcc : z, e);
            st = spmv(ctx, 0, e, r);
        }
        if (st == HHO_OK) st = jacobi_apply(ctx, r, one, jv, jr);
        if (st != HHO_OK) break;
        k_samples<<<nb, MT, (size_t)(FB * M->din + FB) * 4, ctx->stream>>>(
            t, M->dout, r, e, jr, M->X + (int64_t)v * M->nf * M->din, M->T + (int64_t)v * M->nf * M->dout);
    }
    cudaError_t le = cudaGetLastError();
    cudaError_t se = cudaStreamSynchronize(ctx->stream);
    ctx->use_learned = saved;
    ctx->use_graphs = saved_graphs;
    invalidate_graphs(ctx);
    for (double** p : bufs) dfree(*p);
    dfree(one);
    HHO_TRY(st);
    HHO_CUDA(le);
    HHO_CUDA(se);
    if (nsamp) *nsamp = M->nsamp;
    return HHO_OK;
}

hho_status mlp_train(hho_ctx* ctx, int steps, int B, double lr, uint64_t seed, double* h_loss) {
    Learned* M = ctx->learned;
    if (!M || !M->X) {
        ctx->err = "hho_mlp_train: call hho_mlp_init and hho_mlp_generate first";
        return HHO_ERR_STATE;
    }
    if (steps < 1 || steps > 1000000 || B < 1 || B > (1 << 20) || !(lr > 0.0)) {
        ctx->err = "hho_mlp_train: invalid steps, batch or learning rate";
        return HHO_ERR_ARG;
    }
    HHO_TRY(ensure_batch(ctx, M, B));
    if (M->loss_cap < steps) {
        dfree(M->losses);
        HHO_TRY(dalloc(ctx, &M->losses, (size_t)steps));
        M->loss_cap = steps;
    }
    const int64_t n1 = (int64_t)M->din * M->hid, n2 = (int64_t)M->hid * M->dout;
    const int nbk = M->tc ? (B + TC_ROWS - 1) / TC_ROWS : (B + FB - 1) / FB;
    const size_t sm = (size_t)(FB * M->din + FB * M->hid) * 4;
    for (int s = 0; s < steps; ++s) {
        k_gather<<<std::min(B, 4096), 64, 0, ctx->stream>>>(M->nsamp, M->din, M->dout, B,
                                                            seed * 0x9E3779B97F4A7C15ull + (uint64_t)s, M->X, M->T,
                                                            M->Xb, M->Tb);
        train_forward<__nv_bfloat16>(ctx, M, B, M->Xb, M->Tb, sm);
        k_sum_losses<<<1, 32, 0, ctx->stream>>>(nbk, M->lossp, M->losses + s);
        k_train_dh<<<g1((int64_t)B * M->hid), 256, 0, ctx->stream>>>(B, M->hid, M->dout, M->dY, M->W2h, M->H,
                                                                     M->dH);
        k_train_gw<__nv_bfloat16><<<g1(n1 + n2 + M->hid + M->dout), 256, 0, ctx->stream>>>(
            B, M->din, M->hid, M->dout, M->Xb, M->dH, M->H, M->dY, M->gW1, M->gb1, M->gW2, M->gb2);
        ++M->adam_t;
        const float b1c = 1.f - powf(0.9f, (float)M->adam_t), b2c = 1.f - powf(0.999f, (float)M->adam_t);
        k_adam<<<g1(n1), 256, 0, ctx->stream>>>(n1, M->W1, M->gW1, M->mW1, M->vW1, (float)lr, b1c, b2c, M->W1h);
        k_adam<<<g1(M->hid), 256, 0, ctx->stream>>>(M->hid, M->b1, M->gb1, M->mb1, M->vb1, (float)lr, b1c, b2c,
                                                    nullptr);
        k_adam<<<g1(n2), 256, 0, ctx->stream>>>(n2, M->W2, M->gW2, M->mW2, M->vW2, (float)lr, b1c, b2c, M->W2h);
        k_adam<<<g1(M->dout), 256, 0, ctx->stream>>>(M->dout, M->b2, M->gb2, M->mb2, M->vb2, (float)lr, b1c, b2c,
                                                     nullptr);
    }
    HHO_CUDA(cudaGetLastError());
    std::vector<float> l(steps);
    HHO_CUDA(cudaMemcpyAsync(l.data(), M->losses, steps * 4, cudaMemcpyDeviceToHost, ctx->stream));
    HHO_CUDA(cudaStreamSynchronize(ctx->stream));
    HHO_TRY(mlp_status(ctx));
    if (h_loss)
        for (int s = 0; s < steps; ++s) h_loss[s] = l[s];
    invalidate_graphs(ctx);
    return HHO_OK;
}

// Loss and gradients of a given minibatch (FP32 inputs X: B x din, targets T:
// B x dout) with the current BF16 weights: the training kernels' backward pass
// exposed for checking.
hho_status mlp_grads(hho_ctx* ctx, const float* X, const float* Tt, int B, double* loss, double* gW1, double* gb1,
                     double* gW2, double* gb2) {
    Learned* M = ctx->learned;
    if (!M) {
        ctx->err = "learned smoother: call hho_mlp_init first";
        return HHO_ERR_STATE;
    }
    if (B < 1 || B > (1 << 20)) return HHO_ERR_ARG;
    HHO_TRY(ensure_batch(ctx, M, B));
    const int nbk = M->tc ? (B + TC_ROWS - 1) / TC_ROWS : (B + FB - 1) / FB;
    const size_t sm = (size_t)(FB * M->din + FB * M->hid) * 4;
    const int64_t n1 = (int64_t)M->din * M->hid, n2 = (int64_t)M->hid * M->dout;
    if (M->loss_cap < 1) {
        HHO_TRY(dalloc(ctx, &M->losses, 1));
        M->loss_cap = 1;
    }
    train_forward<float>(ctx, M, B, X, Tt, sm);
    k_sum_losses<<<1, 32, 0, ctx->stream>>>(nbk, M->lossp, M->losses);
    k_train_dh<<<g1((int64_t)B * M->hid), 256, 0, ctx->stream>>>(B, M->hid, M->dout, M->dY, M->W2h, M->H, M->dH);
    k_train_gw<float><<<g1(n1 + n2 + M->hid + M->dout), 256, 0, ctx->stream>>>(
        B, M->din, M->hid, M->dout, X, M->dH, M->H, M->dY, M->gW1, M->gb1, M->gW2, M->gb2);
    HHO_CUDA(cudaGetLastError());
    float lf = 0.f;
    HHO_CUDA(cudaMemcpyAsync(&lf, M->losses, 4, cudaMemcpyDeviceToHost, ctx->stream));
    HHO_CUDA(cudaStreamSynchronize(ctx->stream));
    HHO_TRY(mlp_status(ctx));
    *loss = lf;
    double* hp[] = {gW1, gb1, gW2, gb2};
    float* dp[] = {M->gW1, M->gb1, M->gW2, M->gb2};
    const int64_t nn[] = {n1, M->hid, n2, M->dout};
    for (int a = 0; a < 4; ++a) {
        std::vector<float> tmp(nn[a]);
        HHO_CUDA(cudaMemcpy(tmp.data(), dp[a], nn[a] * 4, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < nn[a]; ++i) hp[a][i] = tmp[i];
    }
    return HHO_OK;
}

}  // namespace hho
