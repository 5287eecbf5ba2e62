// Element-batched setup on the GPU: geometry, hierarchical orthonormal bases,
// HHO-dp local operators (Scheme 1, k' = k) and static condensation.
//
//   Sec. 2.1      geometry, polynomial spaces, L2 projectors
//   Sec. 2.2      potential reconstruction p_T^{k+1}, face residual r_TF
//   Sec. 2.3.1    local residuals (Eq. HHOdiscr:residuals)
//   Sec. 4.1.1    local algebraic system (Eq. def:HHOAB)
//   Sec. 4.1.2    v-cond (Eq. ST.1) and v&p-cond (Eqs. zero-residual.T, ST.2)
//
// One CTA per element (grid-stride), global-memory scratch per CTA.  All
// arithmetic is FP64.  Quadrature: every element is split into simplices (fan
// from the vertex average; in 3D every face is first fanned from its own
// vertex average) and each simplex gets a collapsed-coordinate tensor
// Gauss-Legendre rule (segment n=ceil((p+1)/2), triangle n=ceil((p+2)/2),
// tetrahedron n=ceil((p+3)/2) points per direction).  Operator integrals use
// degree 2k+2, data integrals degree 2k+2 (exact for the polynomial data the
// scheme reproduces; the paper does not fix the data quadrature).
//
// Starting functions before orthonormalisation: collapsed-coordinate (Dubiner)
// polynomials on triangles, Legendre products on the bounding box otherwise;
// ordered by total degree, x-major; then modified Gram-Schmidt applied twice in
// the L2 Gram metric.  The degree-k basis is a prefix of the degree-(k+1) one.
//
// Readings taken where the paper is silent or garbled:
//   penalty eta_F = 4 (k+1)(k+d)/d |F| h_F / |T|;
//   the Dirichlet datum enters the momentum RHS as -int g_D.(n.grad P v)
//   + eta/h_F int g_D.v_F (the printed residual has the first sign flipped);
//   Neumann traction g_N = (grad u - p I) n;
//   the eliminated high-order pressure rows of v&p-cond carry their part of
//   the Dirichlet mass datum.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "internal.h"
#include "dense.cuh"

namespace hho {

namespace {

constexpr int TPB = 128;     // threads per element CTA
static_assert(TPB % 32 == 0, "element CTAs are whole warps (warp-shuffle reductions)");
constexpr int TQ = 32;       // quadrature points per tile
constexpr int RQ_E = TPB;    // element points per tile of the right-hand-side kernel (one per thread)
constexpr int RQ_F = 32;     // face points per tile of the right-hand-side kernel

__device__ __forceinline__ double glx(const double* gl, int n, int i) { return gl[n * MAX_GL + i]; }
__device__ __forceinline__ double glw(const double* gl, int n, int i) {
    return gl[(MAX_GL + 1) * MAX_GL + n * MAX_GL + i];
}

// Legendre P_0..P_K and derivatives at x (Bonnet recurrence).
__device__ void legendre(int K, double x, double* P, double* D) {
    P[0] = 1.0;
    D[0] = 0.0;
    if (K >= 1) {
        P[1] = x;
        D[1] = 1.0;
    }
    for (int n = 1; n < K; ++n) {
        P[n + 1] = ((2 * n + 1) * x * P[n] - n * P[n - 1]) / (n + 1);
        D[n + 1] = ((2 * n + 1) * (P[n] + x * D[n]) - n * D[n - 1]) / (n + 1);
    }
}

// Jacobi P_q^{(a,0)}(x) and its derivative.
__device__ void jacobi_q(int q, int a, double x, double* val, double* der) {
    double p0 = 1.0, d0 = 0.0;
    if (q == 0) {
        *val = p0;
        *der = d0;
        return;
    }
    double p1 = 0.5 * ((a + 2) * x + a), d1 = 0.5 * (a + 2);
    for (int n = 2; n <= q; ++n) {
        double c0 = 2.0 * n * (n + a) * (2 * n + a - 2);
        double c1 = (double)(2 * n + a - 1) * (2 * n + a) * (2 * n + a - 2);
        double c2 = (double)(2 * n + a - 1) * a * a;
        double c3 = 2.0 * (n + a - 1) * (n - 1) * (2 * n + a);
        double p2 = ((c1 * x + c2) * p1 - c3 * p0) / c0;
        double d2 = (c1 * p1 + (c1 * x + c2) * d1 - c3 * d0) / c0;
        p0 = p1;
        d0 = d1;
        p1 = p2;
        d1 = d2;
    }
    *val = p1;
    *der = d1;
}

struct ElemSh {
    int N;
    int fid[MAX_NFACE];
    int nvf[MAX_NFACE];
    int bcf[MAX_NFACE];
    double V[MAX_NFACE][MAX_FVERT][3];
    double xF[MAX_NFACE][3];
    double nTF[MAX_NFACE][3];
    double hF[MAX_NFACE], mF[MAX_NFACE];
    double xT[3], bc[3], br[3], meas;
    int simplex;
    double v0[2], Minv[2][2];
};

// Element starting functions (values, gradients [m*3+j]) at x; returns count.
__device__ int elem_start(const ElemSh& E, int d, int K, const double* x, double* val, double* grad) {
    if (E.simplex) {
        double dx = x[0] - E.v0[0], dy = x[1] - E.v0[1];
        double r = 2.0 * (E.Minv[0][0] * dx + E.Minv[0][1] * dy) - 1.0;
        double s = 2.0 * (E.Minv[1][0] * dx + E.Minv[1][1] * dy) - 1.0;
        double t = 0.5 * (1.0 - s), u = r + 0.5 * (1.0 + s);
        double Q[MAX_K2 + 2], Qr[MAX_K2 + 2], Qs[MAX_K2 + 2];
        Q[0] = 1.0;
        Qr[0] = 0.0;
        Qs[0] = 0.0;
        if (K >= 1) {
            Q[1] = u;
            Qr[1] = 1.0;
            Qs[1] = 0.5;
        }
        for (int p = 1; p < K; ++p) {
            Q[p + 1] = ((2 * p + 1) * u * Q[p] - p * t * t * Q[p - 1]) / (p + 1);
            Qr[p + 1] = ((2 * p + 1) * (Q[p] + u * Qr[p]) - p * t * t * Qr[p - 1]) / (p + 1);
            Qs[p + 1] = ((2 * p + 1) * (0.5 * Q[p] + u * Qs[p]) - p * (-t * Q[p - 1] + t * t * Qs[p - 1])) / (p + 1);
        }
        int m = 0;
        for (int l = 0; l <= K; ++l)
            for (int p = l; p >= 0; --p) {
                int q = l - p;
                double J, Jd;
                jacobi_q(q, 2 * p + 1, s, &J, &Jd);
                val[m] = Q[p] * J;
                double gr = Qr[p] * J, gs = Qs[p] * J + Q[p] * Jd;
                grad[m * 3 + 0] = 2.0 * (gr * E.Minv[0][0] + gs * E.Minv[1][0]);
                grad[m * 3 + 1] = 2.0 * (gr * E.Minv[0][1] + gs * E.Minv[1][1]);
                ++m;
            }
        return m;
    }
    double P[3][MAX_K2 + 2], D[3][MAX_K2 + 2];
    for (int i = 0; i < d; ++i) {
        double xi = (x[i] - E.bc[i]) / E.br[i];
        legendre(K, xi, P[i], D[i]);
        for (int n = 0; n <= K; ++n) D[i][n] /= E.br[i];
    }
    int m = 0;
    if (d == 2) {
        for (int l = 0; l <= K; ++l)
            for (int a = l; a >= 0; --a) {
                int b = l - a;
                val[m] = P[0][a] * P[1][b];
                grad[m * 3 + 0] = D[0][a] * P[1][b];
                grad[m * 3 + 1] = P[0][a] * D[1][b];
                ++m;
            }
    } else {
        for (int l = 0; l <= K; ++l)
            for (int a = l; a >= 0; --a)
                for (int b = l - a; b >= 0; --b) {
                    int c = l - a - b;
                    val[m] = P[0][a] * P[1][b] * P[2][c];
                    grad[m * 3 + 0] = D[0][a] * P[1][b] * P[2][c];
                    grad[m * 3 + 1] = P[0][a] * D[1][b] * P[2][c];
                    grad[m * 3 + 2] = P[0][a] * P[1][b] * D[2][c];
                    ++m;
                }
    }
    return m;
}

// Coefficients of the three-term recursions of elem_start divided through by
// their leading factor once per CTA, so that value-only evaluations need no
// FP64 division (a multi-instruction sequence on this part's narrow FP64 pipe):
//   Legendre / Dubiner radial part  P_{n+1} = qa[n] x P_n - qb[n] y P_{n-1}
//       qa[n] = (2n+1)/(n+1), qb[n] = n/(n+1)
//   Jacobi P^{(a,0)}, a = 2p+1      J_{n} = (ja x + jb) J_{n-1} - jc J_{n-2},
//       (ja, jb, jc)[p][n] = (c1, c2, c3)[n, a] / c0[n, a]   (n >= 2)
constexpr int REC_N = MAX_K2 + 2;  // degrees 0..MAX_K2+1 (HHO-hp element velocity)
struct RecTab {
    double qa[REC_N], qb[REC_N];
    double ja[REC_N][REC_N], jb[REC_N][REC_N], jc[REC_N][REC_N];
};

// Fill a RecTab (all threads of the CTA; ends with a barrier).
__device__ void rec_tab_fill(RecTab& T) {
    for (int i = threadIdx.x; i < REC_N; i += blockDim.x) {
        T.qa[i] = (2.0 * i + 1.0) / (i + 1.0);
        T.qb[i] = (double)i / (i + 1.0);
    }
    for (int i = threadIdx.x; i < REC_N * REC_N; i += blockDim.x) {
        const int p = i / REC_N, n = i % REC_N, a = 2 * p + 1;
        double A = 0.0, B = 0.0, C = 0.0;
        if (n >= 2) {
            const double c0 = 2.0 * n * (n + a) * (2 * n + a - 2);
            const double c1 = (double)(2 * n + a - 1) * (2 * n + a) * (2 * n + a - 2);
            const double c2 = (double)(2 * n + a - 1) * a * a;
            const double c3 = 2.0 * (n + a - 1) * (n - 1) * (2 * n + a);
            A = c1 / c0;
            B = c2 / c0;
            C = c3 / c0;
        }
        T.ja[p][n] = A;
        T.jb[p][n] = B;
        T.jc[p][n] = C;
    }
    __syncthreads();
}

// Values of the element starting functions of elem_start (same functions,
// same order; no gradients) at x, K <= MAX_K2 + 1, with the recursion
// coefficients of T; returns the count.
__device__ int elem_start_val(const ElemSh& E, int d, int K, const double* x, double* val, const RecTab& T) {
    if (E.simplex) {
        const double dx = x[0] - E.v0[0], dy = x[1] - E.v0[1];
        const double r = 2.0 * (E.Minv[0][0] * dx + E.Minv[0][1] * dy) - 1.0;
        const double s = 2.0 * (E.Minv[1][0] * dx + E.Minv[1][1] * dy) - 1.0;
        const double t = 0.5 * (1.0 - s), u = r + 0.5 * (1.0 + s), tt = t * t;
        double Q[REC_N + 1];
        Q[0] = 1.0;
        if (K >= 1) Q[1] = u;
        for (int p = 1; p < K; ++p) Q[p + 1] = T.qa[p] * u * Q[p] - T.qb[p] * tt * Q[p - 1];
        // function (l, p) with q = l - p sits at index l (l + 1) / 2 + q
        for (int p = 0; p <= K; ++p) {
            const int a = 2 * p + 1;
            double j0 = 1.0, j1 = 0.5 * ((a + 2) * s + a);
            for (int q = 0; q <= K - p; ++q) {
                double J;
                if (q == 0) {
                    J = 1.0;
                } else if (q == 1) {
                    J = j1;
                } else {
                    J = (T.ja[p][q] * s + T.jb[p][q]) * j1 - T.jc[p][q] * j0;
                    j0 = j1;
                    j1 = J;
                }
                const int l = p + q;
                val[l * (l + 1) / 2 + q] = Q[p] * J;
            }
        }
        return (K + 1) * (K + 2) / 2;
    }
    double P[3][REC_N + 1];
    for (int i = 0; i < d; ++i) {
        const double xi = (x[i] - E.bc[i]) / E.br[i];
        P[i][0] = 1.0;
        if (K >= 1) P[i][1] = xi;
        for (int n = 1; n < K; ++n) P[i][n + 1] = T.qa[n] * xi * P[i][n] - T.qb[n] * P[i][n - 1];
    }
    int m = 0;
    if (d == 2) {
        for (int l = 0; l <= K; ++l)
            for (int a = l; a >= 0; --a) val[m++] = P[0][a] * P[1][l - a];
    } else {
        for (int l = 0; l <= K; ++l)
            for (int a = l; a >= 0; --a)
                for (int b = l - a; b >= 0; --b) val[m++] = P[0][a] * P[1][b] * P[2][l - a - b];
    }
    return m;
}

// Face starting functions (values) at x.
__device__ int face_start(const FaceGeo& g, int d, int K, const double* x, double* val) {
    double y0 = 0.0, y1 = 0.0;
    for (int j = 0; j < d; ++j) {
        y0 += (x[j] - g.xF[j]) * g.t1[j];
        y1 += (x[j] - g.xF[j]) * g.t2[j];
    }
    double P0[MAX_K2 + 2], D0[MAX_K2 + 2];
    legendre(K, (y0 - g.bc[0]) / g.br[0], P0, D0);
    if (d == 2) {
        for (int j = 0; j <= K; ++j) val[j] = P0[j];
        return K + 1;
    }
    double P1[MAX_K2 + 2], D1[MAX_K2 + 2];
    legendre(K, (y1 - g.bc[1]) / g.br[1], P1, D1);
    int m = 0;
    for (int l = 0; l <= K; ++l)
        for (int a = l; a >= 0; --a) val[m++] = P0[a] * P1[l - a];
    return m;
}

// Quadrature point q of the element rule of degree p (fan of simplices).
__device__ void elem_point(const ElemSh& E, int d, const double* gl, int p, int q, double* x, double* w) {
    if (d == 2) {
        int n = (p + 3) / 2, nn = n * n;
        int f = q / nn, t = q % nn, iu = t / n, iv = t % n;
        const double* a = E.xT;
        const double* b = E.V[f][0];
        const double* c = E.V[f][1];
        double e1x = b[0] - a[0], e1y = b[1] - a[1], e2x = c[0] - a[0], e2y = c[1] - a[1];
        double area = 0.5 * fabs(e1x * e2y - e1y * e2x);
        double u = glx(gl, n, iu), v = glx(gl, n, iv);
        double xi = u, eta = v * (1.0 - u);
        x[0] = a[0] + xi * e1x + eta * e2x;
        x[1] = a[1] + xi * e1y + eta * e2y;
        *w = glw(gl, n, iu) * glw(gl, n, iv) * (1.0 - u) * 2.0 * area;
        return;
    }
    int n = (p + 4) / 2, n3 = n * n * n;
    int s = q / n3, t = q % n3;
    int f = 0;
    while (s >= E.nvf[f]) {
        s -= E.nvf[f];
        ++f;
    }
    int iu = t / (n * n), iv = (t / n) % n, iw = t % n;
    const double* a = E.xT;
    const double* b = E.xF[f];
    const double* c = E.V[f][s];
    const double* dd = E.V[f][(s + 1) % E.nvf[f]];
    double e1[3], e2[3], e3[3];
    for (int j = 0; j < 3; ++j) {
        e1[j] = b[j] - a[j];
        e2[j] = c[j] - a[j];
        e3[j] = dd[j] - a[j];
    }
    double det = e1[0] * (e2[1] * e3[2] - e2[2] * e3[1]) - e1[1] * (e2[0] * e3[2] - e2[2] * e3[0]) +
                 e1[2] * (e2[0] * e3[1] - e2[1] * e3[0]);
    double vol = fabs(det) / 6.0;
    double u = glx(gl, n, iu), v = glx(gl, n, iv), ww = glx(gl, n, iw);
    double xi = u, eta = v * (1.0 - u), zeta = ww * (1.0 - u) * (1.0 - v);
    for (int j = 0; j < 3; ++j) x[j] = a[j] + xi * e1[j] + eta * e2[j] + zeta * e3[j];
    *w = glw(gl, n, iu) * glw(gl, n, iv) * glw(gl, n, iw) * (1.0 - u) * (1.0 - u) * (1.0 - v) * 6.0 * vol;
}

__device__ int elem_npts(const ElemSh& E, int d, int p) {
    if (d == 2) {
        int n = (p + 3) / 2;
        return E.N * n * n;
    }
    int n = (p + 4) / 2, s = 0;
    for (int f = 0; f < E.N; ++f) s += E.nvf[f];
    return s * n * n * n;
}

// Quadrature point q of the face rule of degree p on a face with vertices V (nv of them) and centre xF.
__device__ void face_point(int d, const double (*V)[3], int nv, const double* xF, const double* gl, int p, int q,
                           double* x, double* w) {
    if (d == 2) {
        int n = (p + 2) / 2;
        double ex = V[1][0] - V[0][0], ey = V[1][1] - V[0][1];
        double len = sqrt(ex * ex + ey * ey);
        double u = glx(gl, n, q);
        x[0] = V[0][0] + u * ex;
        x[1] = V[0][1] + u * ey;
        *w = glw(gl, n, q) * len;
        return;
    }
    int n = (p + 3) / 2, nn = n * n;
    int s = q / nn, t = q % nn, iu = t / n, iv = t % n;
    const double* a = xF;
    const double* b = V[s];
    const double* c = V[(s + 1) % nv];
    double e1[3], e2[3];
    for (int j = 0; j < 3; ++j) {
        e1[j] = b[j] - a[j];
        e2[j] = c[j] - a[j];
    }
    double cx = e1[1] * e2[2] - e1[2] * e2[1], cy = e1[2] * e2[0] - e1[0] * e2[2], cz = e1[0] * e2[1] - e1[1] * e2[0];
    double area = 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
    double u = glx(gl, n, iu), v = glx(gl, n, iv);
    double xi = u, eta = v * (1.0 - u);
    for (int j = 0; j < 3; ++j) x[j] = a[j] + xi * e1[j] + eta * e2[j];
    *w = glw(gl, n, iu) * glw(gl, n, iv) * (1.0 - u) * 2.0 * area;
}

__device__ __host__ inline int face_npts(int d, int nv, int p) {
    if (d == 2) return (p + 2) / 2;
    int n = (p + 3) / 2;
    return nv * n * n;
}

// ---- CTA-level dense helpers (row-major) ----
__device__ void cta_mm(double* C, int ldc, const double* A, int lda, bool tA, const double* B, int ldb, bool tB,
                       int m, int n, int kk, double alpha, double beta) {
    for (int idx = threadIdx.x; idx < m * n; idx += blockDim.x) {
        int i = idx / n, j = idx % n;
        double s = 0.0;
        for (int l = 0; l < kk; ++l) s += (tA ? A[l * lda + i] : A[i * lda + l]) * (tB ? B[j * ldb + l] : B[l * ldb + j]);
        C[i * ldc + j] = alpha * s + (beta != 0.0 ? beta * C[i * ldc + j] : 0.0);
    }
    __syncthreads();
}

__device__ void cta_zero(double* A, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) A[i] = 0.0;
    __syncthreads();
}

// Modified Gram-Schmidt applied twice in the Gram metric G (n x n): rows of C.
// Executed by warp 0; tmp holds 2n doubles.
__device__ void warp_mgs2(const double* G, int n, double* C, double* tmp) {
    if (threadIdx.x >= 32) return;
    int lane = threadIdx.x;
    double* c = tmp;
    double* Gc = tmp + n;
    for (int i = 0; i < n; ++i) {
        for (int a = lane; a < n; a += 32) c[a] = (a == i) ? 1.0 : 0.0;
        __syncwarp();
        for (int pass = 0; pass < 2; ++pass)
            for (int j = 0; j < i; ++j) {
                for (int a = lane; a < n; a += 32) {
                    double s = 0.0;
                    for (int b = 0; b < n; ++b) s += G[a * n + b] * c[b];
                    Gc[a] = s;
                }
                __syncwarp();
                double part = 0.0;
                for (int a = lane; a < n; a += 32) part += C[j * n + a] * Gc[a];
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                for (int a = lane; a < n; a += 32) c[a] -= part * C[j * n + a];
                __syncwarp();
            }
        for (int a = lane; a < n; a += 32) {
            double s = 0.0;
            for (int b = 0; b < n; ++b) s += G[a * n + b] * c[b];
            Gc[a] = s;
        }
        __syncwarp();
        double part = 0.0;
        for (int a = lane; a < n; a += 32) part += c[a] * Gc[a];
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        double inv = 1.0 / sqrt(part);
        for (int a = lane; a < n; a += 32) C[i * n + a] = c[a] * inv;
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Face kernel: geometry and orthonormal face basis (one thread per face).
// ---------------------------------------------------------------------------
__global__ void k_faces(int d, int k, int64_t nf, const double* __restrict__ xyz, const int32_t* __restrict__ fv_ptr,
                        const int32_t* __restrict__ fv, const double* __restrict__ gl, FaceGeo* __restrict__ fgeo,
                        double* __restrict__ fC) {
    int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= nf) return;
    int nF = dimP(d - 1, k);
    int v0 = fv_ptr[f], nv = fv_ptr[f + 1] - v0;
    double V[MAX_FVERT][3] = {};
    for (int i = 0; i < nv; ++i)
        for (int j = 0; j < d; ++j) V[i][j] = xyz[(int64_t)fv[v0 + i] * d + j];
    FaceGeo g;
    for (int j = 0; j < 3; ++j) g.xF[j] = g.n[j] = g.t1[j] = g.t2[j] = 0.0;
    for (int i = 0; i < nv; ++i)
        for (int j = 0; j < d; ++j) g.xF[j] += V[i][j];
    for (int j = 0; j < d; ++j) g.xF[j] /= nv;
    double h = 0.0;
    for (int i = 0; i < nv; ++i)
        for (int l = i + 1; l < nv; ++l) {
            double s = 0.0;
            for (int j = 0; j < d; ++j) s += (V[i][j] - V[l][j]) * (V[i][j] - V[l][j]);
            h = fmax(h, sqrt(s));
        }
    g.hF = h;
    if (d == 2) {
        double tx = V[1][0] - V[0][0], ty = V[1][1] - V[0][1];
        double len = sqrt(tx * tx + ty * ty);
        g.meas = len;
        g.t1[0] = tx / len;
        g.t1[1] = ty / len;
        g.n[0] = g.t1[1];
        g.n[1] = -g.t1[0];
    } else {
        double nn[3] = {0, 0, 0}, area = 0.0;
        for (int i = 0; i < nv; ++i) {
            double a[3], b[3];
            for (int j = 0; j < 3; ++j) {
                a[j] = V[i][j] - g.xF[j];
                b[j] = V[(i + 1) % nv][j] - g.xF[j];
            }
            double c[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
            for (int j = 0; j < 3; ++j) nn[j] += c[j];
            area += 0.5 * sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        }
        g.meas = area;
        double ln = sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
        for (int j = 0; j < 3; ++j) g.n[j] = nn[j] / ln;
        double t[3], lt = 0.0;
        for (int j = 0; j < 3; ++j) {
            t[j] = V[1][j] - V[0][j];
            lt += t[j] * t[j];
        }
        lt = sqrt(lt);
        for (int j = 0; j < 3; ++j) g.t1[j] = t[j] / lt;
        g.t2[0] = g.n[1] * g.t1[2] - g.n[2] * g.t1[1];
        g.t2[1] = g.n[2] * g.t1[0] - g.n[0] * g.t1[2];
        g.t2[2] = g.n[0] * g.t1[1] - g.n[1] * g.t1[0];
    }
    double lo[2] = {1e300, 1e300}, hi[2] = {-1e300, -1e300};
    for (int i = 0; i < nv; ++i) {
        double y0 = 0.0, y1 = 0.0;
        for (int j = 0; j < d; ++j) {
            y0 += (V[i][j] - g.xF[j]) * g.t1[j];
            y1 += (V[i][j] - g.xF[j]) * g.t2[j];
        }
        lo[0] = fmin(lo[0], y0);
        hi[0] = fmax(hi[0], y0);
        lo[1] = fmin(lo[1], y1);
        hi[1] = fmax(hi[1], y1);
    }
    for (int j = 0; j < 2; ++j) {
        g.bc[j] = 0.5 * (lo[j] + hi[j]);
        g.br[j] = 0.5 * (hi[j] - lo[j]);
    }
    if (d == 2) {
        g.bc[1] = 0.0;
        g.br[1] = 1.0;
    }
    fgeo[f] = g;
    // Gram matrix of the starting functions (degree 2k rule), then MGS2.
    double G[10 * 10];
    for (int i = 0; i < nF * nF; ++i) G[i] = 0.0;
    int p = 2 * k, nq = face_npts(d, nv, p);
    for (int q = 0; q < nq; ++q) {
        double x[3] = {0, 0, 0}, w, val[10];
        face_point(d, V, nv, g.xF, gl, p, q, x, &w);
        face_start(g, d, k, x, val);
        for (int i = 0; i < nF; ++i)
            for (int j = 0; j < nF; ++j) G[i * nF + j] += w * val[i] * val[j];
    }
    double* C = fC + f * nF * nF;
    for (int i = 0; i < nF * nF; ++i) C[i] = 0.0;
    double c[10], Gc[10];
    for (int i = 0; i < nF; ++i) {
        for (int a = 0; a < nF; ++a) c[a] = (a == i) ? 1.0 : 0.0;
        for (int pass = 0; pass < 2; ++pass)
            for (int j = 0; j < i; ++j) {
                for (int a = 0; a < nF; ++a) {
                    double s = 0.0;
                    for (int b = 0; b < nF; ++b) s += G[a * nF + b] * c[b];
                    Gc[a] = s;
                }
                double t = 0.0;
                for (int a = 0; a < nF; ++a) t += C[j * nF + a] * Gc[a];
                for (int a = 0; a < nF; ++a) c[a] -= t * C[j * nF + a];
            }
        for (int a = 0; a < nF; ++a) {
            double s = 0.0;
            for (int b = 0; b < nF; ++b) s += G[a * nF + b] * c[b];
            Gc[a] = s;
        }
        double nrm = 0.0;
        for (int a = 0; a < nF; ++a) nrm += c[a] * Gc[a];
        nrm = 1.0 / sqrt(nrm);
        for (int a = 0; a < nF; ++a) C[i * nF + a] = c[a] * nrm;
    }
}

// Load the geometry of element t into shared memory (thread 0 writes).
__device__ void load_element(ElemSh& E, int d, int t, const int32_t* ef_ptr, const int32_t* ef, const int32_t* fv_ptr,
                             const int32_t* fv, const double* xyz, const FaceGeo* fgeo, const int8_t* fbc) {
    if (threadIdx.x == 0) {
        int f0 = ef_ptr[t];
        E.N = ef_ptr[t + 1] - f0;
        int vids[MAX_NFACE * MAX_FVERT];
        int nvid = 0;
        for (int f = 0; f < E.N; ++f) {
            int F = ef[f0 + f];
            E.fid[f] = F;
            E.bcf[f] = fbc[F];
            int a = fv_ptr[F];
            E.nvf[f] = fv_ptr[F + 1] - a;
            for (int i = 0; i < E.nvf[f]; ++i) {
                int v = fv[a + i];
                for (int j = 0; j < 3; ++j) E.V[f][i][j] = (j < d) ? xyz[(int64_t)v * d + j] : 0.0;
                bool seen = false;
                for (int s = 0; s < nvid; ++s) seen |= (vids[s] == v);
                if (!seen) vids[nvid++] = v;
            }
            const FaceGeo& g = fgeo[F];
            for (int j = 0; j < 3; ++j) E.xF[f][j] = g.xF[j];
            E.hF[f] = g.hF;
            E.mF[f] = g.meas;
        }
        // unique vertices in increasing id order (as a sorted unique list)
        for (int i = 1; i < nvid; ++i)
            for (int s = i; s > 0 && vids[s - 1] > vids[s]; --s) {
                int tmp = vids[s];
                vids[s] = vids[s - 1];
                vids[s - 1] = tmp;
            }
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int j = 0; j < 3; ++j) E.xT[j] = 0.0;
        for (int s = 0; s < nvid; ++s)
            for (int j = 0; j < d; ++j) {
                double x = xyz[(int64_t)vids[s] * d + j];
                E.xT[j] += x;
                lo[j] = fmin(lo[j], x);
                hi[j] = fmax(hi[j], x);
            }
        for (int j = 0; j < d; ++j) {
            E.xT[j] /= nvid;
            E.bc[j] = 0.5 * (lo[j] + hi[j]);
            E.br[j] = 0.5 * (hi[j] - lo[j]);
        }
        for (int f = 0; f < E.N; ++f) {
            const FaceGeo& g = fgeo[E.fid[f]];
            double s = 0.0;
            for (int j = 0; j < d; ++j) s += g.n[j] * (g.xF[j] - E.xT[j]);
            double sg = s > 0.0 ? 1.0 : -1.0;
            for (int j = 0; j < 3; ++j) E.nTF[f][j] = sg * g.n[j];
        }
        E.simplex = (d == 2 && E.N == 3);
        if (E.simplex) {
            const double* a = E.V[0][0];
            const double* b = E.V[0][1];
            int va = fv[fv_ptr[E.fid[0]]], vb = fv[fv_ptr[E.fid[0]] + 1];
            double c[2] = {0, 0};
            for (int f = 1; f < E.N; ++f)
                for (int i = 0; i < 2; ++i) {
                    int v = fv[fv_ptr[E.fid[f]] + i];
                    if (v != va && v != vb) {
                        c[0] = E.V[f][i][0];
                        c[1] = E.V[f][i][1];
                    }
                }
            double m00 = b[0] - a[0], m01 = c[0] - a[0], m10 = b[1] - a[1], m11 = c[1] - a[1];
            double det = m00 * m11 - m01 * m10;
            E.Minv[0][0] = m11 / det;
            E.Minv[0][1] = -m01 / det;
            E.Minv[1][0] = -m10 / det;
            E.Minv[1][1] = m00 / det;
            E.v0[0] = a[0];
            E.v0[1] = a[1];
        }
    }
    __syncthreads();
}

// Local sizes of one element.  Scheme 1 (v-cond, v&p-cond): element velocity
// in P^k (n_V = n_E), element pressure P^k, face blocks of d n_F velocity
// coefficients.  Scheme 2 (HHO-hp, Sec. 2.3.2): element velocity in P^{k+1}
// (n_V = n_R), element pressure P^k plus a face pressure P^k(F) per face, every
// element unknown eliminated, kept face blocks of (d+1) n_F (velocity, then
// the face pressure).
// Uncondensed Scheme 1 eliminates nothing and keeps the faces, then the
// element block [U_T | P_T].
// Local vector: [U_T (d n_V) | U_F (N d n_F) | P_T (n_E) | P_F (N n_F, HHO-hp)].
struct LocalDims {
    int d, k, nR, nE, nF, nV, bv, b, N, ns, nvec, npr, nloc, nel, nk, cond;
};

__host__ __device__ inline LocalDims local_dims(int d, int k, int N, int cond) {
    LocalDims D;
    D.d = d;
    D.k = k;
    D.nR = dimP(d, k + 1);
    D.nE = dimP(d, k);
    D.nF = dimP(d - 1, k);
    const bool hp = (cond == HHO_HPCOND);
    D.nV = hp ? D.nR : D.nE;
    D.bv = d * D.nF;
    D.b = hp ? (d + 1) * D.nF : D.bv;
    D.N = N;
    D.ns = D.nV + N * D.nF;
    D.nvec = d * D.nV + N * D.bv;
    D.npr = D.nE + (hp ? N * D.nF : 0);
    D.nloc = D.nvec + D.npr;
    D.cond = cond;
    if (hp) {
        D.nel = d * D.nV + D.nE;
        D.nk = N * D.b;
    } else if (cond == HHO_UNCOND) {
        D.nel = 0;
        D.nk = N * D.b + (d + 1) * D.nE;
    } else if (cond == HHO_DGCOND) {  // no local system: the element data of the DG couplings instead
        D.nel = 0;
        D.nk = 0;
    } else if (cond == HHO_VCOND) {
        D.nel = d * D.nE;
        D.nk = N * D.b + D.nE;
    } else {
        D.nel = d * D.nE + D.nE - 1;
        D.nk = N * D.b + 1;
    }
    return D;
}

// local index (in K) of the i-th eliminated / kept unknown
__device__ __forceinline__ int elim_idx(const LocalDims& D, int i) {
    const int nUT = D.d * D.nV;
    if (i < nUT) return i;
    return D.cond == HHO_HPCOND ? D.nvec + (i - nUT) : D.nvec + 1 + (i - nUT);
}
__device__ __forceinline__ int keep_idx(const LocalDims& D, int i) {
    if (D.cond == HHO_UNCOND) {  // faces, then the element block [U_T | P_T]
        if (i < D.N * D.b) return D.d * D.nE + i;
        const int e = i - D.N * D.b;
        return e < D.d * D.nE ? e : D.nvec + (e - D.d * D.nE);
    }
    if (D.cond != HHO_HPCOND) return D.d * D.nE + i;  // faces, then pressures (all for v-cond, the mean for v&p)
    const int f = i / D.b, r = i % D.b;                // HHO-hp: per face its velocity, then its pressure
    return r < D.bv ? D.d * D.nV + f * D.bv + r : D.nvec + D.nE + f * D.nF + (r - D.bv);
}
// vector index of scalar unknown a (0..ns) for component c
__device__ __forceinline__ int vmap(const LocalDims& D, int c, int a) {
    if (a < D.nV) return c * D.nV + a;
    int f = (a - D.nV) / D.nF, j = (a - D.nV) % D.nF;
    return D.d * D.nV + f * D.bv + c * D.nF + j;
}

struct ScratchLayout {
    int64_t Gt, Kt, Dt, T1, T2, T3, T4, T5, C, Kst, Rhs, P, A, B, Kl, W, R, Mr, tmp, total;
};

__host__ __device__ inline ScratchLayout scratch_layout(int d, int k, int maxN, int cond) {
    const LocalDims M = local_dims(d, k, maxN, cond);
    const int nR = M.nR, nE = M.nE, nF = M.nF, nV = M.nV;
    const int ns = M.ns, nloc = M.nloc;
    const int nel = d * nV + nE, nk = maxN * M.b + (d + 1) * nE;  // bounds over the condensation variants
    ScratchLayout L;
    int64_t o = 0;
    auto take = [&](int64_t n) {
        int64_t r = o;
        o += (n + 3) & ~int64_t(3);
        return r;
    };
    L.Gt = take(nR * nR);
    L.Kt = take(nR * nR);
    L.Dt = take(3 * nE * nV);
    L.T1 = take((int64_t)maxN * nR * nV);
    L.T2 = take((int64_t)maxN * nR * nF);
    L.T3 = take((int64_t)maxN * nR * nF);
    L.T4 = take((int64_t)maxN * nV * nV);
    L.T5 = take((int64_t)maxN * nF * nF);
    L.C = take(nR * nR);
    L.Kst = take(nR * nR);
    L.Rhs = take((int64_t)nR * ns);
    L.P = take((int64_t)nR * ns);
    L.A = take((int64_t)ns * ns);
    L.B = take((int64_t)M.npr * M.nvec);
    L.Kl = take((int64_t)nloc * nloc);
    L.W = take((int64_t)nel * (nel + nk + nel));
    L.R = take((int64_t)(nF + nV) * ns);
    L.Mr = take((int64_t)(nF + nV) * (nF + nV));
    L.tmp = take((int64_t)(nR + ns) * (nR + ns) + 4 * nR);
    L.total = o;
    return L;
}

// ---------------------------------------------------------------------------
// Element kernel: bases, local operators, condensation.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TPB) k_elements(int d, int k, int cond, int64_t ne, const double* __restrict__ xyz,
                                                  const int32_t* __restrict__ ef_ptr, const int32_t* __restrict__ ef,
                                                  const int32_t* __restrict__ fv_ptr, const int32_t* __restrict__ fv,
                                                  const int8_t* __restrict__ fbc, const FaceGeo* __restrict__ fgeo,
                                                  const double* __restrict__ fC, const double* __restrict__ gl,
                                                  int maxN, double* __restrict__ scratch, double* __restrict__ eC,
                                                  double* __restrict__ emeas, const int64_t* __restrict__ off_S,
                                                  const int64_t* __restrict__ off_X, const int64_t* __restrict__ off_Kei,
                                                  const int64_t* __restrict__ off_P, double* __restrict__ outS,
                                                  double* __restrict__ outX, double* __restrict__ outKei,
                                                  double* __restrict__ outP, int* __restrict__ status) {
    __shared__ ElemSh E;
    __shared__ double s_val[TQ][36];
    __shared__ double s_grad[TQ][36 * 3];
    __shared__ double s_fval[TQ][10];
    __shared__ double s_w[TQ];
    __shared__ int s_piv;
    const ScratchLayout SL = scratch_layout(d, k, maxN, cond);
    double* ws = scratch + (int64_t)blockIdx.x * SL.total;
    const int nR = dimP(d, k + 1), nE = dimP(d, k), nF = dimP(d - 1, k);
    const int nV = (cond == HHO_HPCOND) ? nR : nE;  // element velocity coefficients

    for (int64_t t = blockIdx.x; t < ne; t += gridDim.x) {
        load_element(E, d, (int)t, ef_ptr, ef, fv_ptr, fv, xyz, fgeo, fbc);
        const LocalDims D = local_dims(d, k, E.N, cond);
        const int N = E.N, ns = D.ns;
        double* Gt = ws + SL.Gt;
        double* Kt = ws + SL.Kt;
        double* Dt = ws + SL.Dt;
        cta_zero(Gt, nR * nR);
        cta_zero(Kt, nR * nR);
        cta_zero(Dt, 3 * nE * nV);
        // ---- element integrals in the starting basis (degree 2k+2) ----
        const int pop = 2 * k + 2;
        int nq = elem_npts(E, d, pop);
        double meas_part = 0.0;
        for (int q0 = 0; q0 < nq; q0 += TQ) {
            int nt = min(TQ, nq - q0);
            if (threadIdx.x < nt) {
                double x[3] = {0, 0, 0}, w;
                elem_point(E, d, gl, pop, q0 + threadIdx.x, x, &w);
                s_w[threadIdx.x] = w;
                elem_start(E, d, k + 1, x, s_val[threadIdx.x], s_grad[threadIdx.x]);
                meas_part += w;
            }
            __syncthreads();
            for (int idx = threadIdx.x; idx < nR * nR; idx += blockDim.x) {
                int i = idx / nR, j = idx % nR;
                double g = 0.0, kk = 0.0;
                for (int q = 0; q < nt; ++q) {
                    double w = s_w[q];
                    g += w * s_val[q][i] * s_val[q][j];
                    double s = 0.0;
                    for (int c = 0; c < d; ++c) s += s_grad[q][i * 3 + c] * s_grad[q][j * 3 + c];
                    kk += w * s;
                }
                Gt[idx] += g;
                Kt[idx] += kk;
            }
            for (int idx = threadIdx.x; idx < d * nE * nV; idx += blockDim.x) {
                int c = idx / (nE * nV), r = idx % (nE * nV), i = r / nV, j = r % nV;
                double s = 0.0;
                for (int q = 0; q < nt; ++q) s += s_w[q] * s_val[q][i] * s_grad[q][j * 3 + c];
                Dt[idx] += s;
            }
            __syncthreads();
        }
        // element measure = sum of weights (reduce over threads that evaluated points)
        {
            __shared__ double s_red[TPB];
            s_red[threadIdx.x] = meas_part;
            __syncthreads();
            if (threadIdx.x == 0) {
                double s = 0.0;
                for (int i = 0; i < TPB; ++i) s += s_red[i];
                E.meas = s;
                emeas[t] = s;
            }
            __syncthreads();
        }
        // ---- orthonormal element basis ----
        double* C = ws + SL.C;
        cta_zero(C, nR * nR);
        warp_mgs2(Gt, nR, C, ws + SL.tmp);
        __syncthreads();
        for (int i = threadIdx.x; i < nR * nR; i += blockDim.x) eC[t * nR * nR + i] = C[i];
        // ---- face integrals (degree 2k+2) ----
        double* T1 = ws + SL.T1;
        double* T2 = ws + SL.T2;
        double* T3 = ws + SL.T3;
        double* T4 = ws + SL.T4;
        double* T5 = ws + SL.T5;
        cta_zero(T1, N * nR * nV);
        cta_zero(T2, N * nR * nF);
        cta_zero(T3, N * nR * nF);
        cta_zero(T4, N * nV * nV);
        cta_zero(T5, N * nF * nF);
        for (int f = 0; f < N; ++f) {
            const FaceGeo& g = fgeo[E.fid[f]];
            int nqf = face_npts(d, E.nvf[f], pop);
            for (int q0 = 0; q0 < nqf; q0 += TQ) {
                int nt = min(TQ, nqf - q0);
                if (threadIdx.x < nt) {
                    double x[3] = {0, 0, 0}, w;
                    face_point(d, E.V[f], E.nvf[f], E.xF[f], gl, pop, q0 + threadIdx.x, x, &w);
                    s_w[threadIdx.x] = w;
                    elem_start(E, d, k + 1, x, s_val[threadIdx.x], s_grad[threadIdx.x]);
                    face_start(g, d, k, x, s_fval[threadIdx.x]);
                    // store the normal derivative in s_grad[.][m*3+0]
                    for (int m = 0; m < nR; ++m) {
                        double s = 0.0;
                        for (int c = 0; c < d; ++c) s += s_grad[threadIdx.x][m * 3 + c] * E.nTF[f][c];
                        s_grad[threadIdx.x][m * 3 + 0] = s;
                    }
                }
                __syncthreads();
                double* t1 = T1 + f * nR * nV;
                double* t2 = T2 + f * nR * nF;
                double* t3 = T3 + f * nR * nF;
                double* t4 = T4 + f * nV * nV;
                double* t5 = T5 + f * nF * nF;
                for (int idx = threadIdx.x; idx < nR * nV; idx += blockDim.x) {
                    int i = idx / nV, m = idx % nV;
                    double s = 0.0;
                    for (int q = 0; q < nt; ++q) s += s_w[q] * s_grad[q][i * 3] * s_val[q][m];
                    t1[idx] += s;
                }
                for (int idx = threadIdx.x; idx < nR * nF; idx += blockDim.x) {
                    int i = idx / nF, j = idx % nF;
                    double s2 = 0.0, s3 = 0.0;
                    for (int q = 0; q < nt; ++q) {
                        s2 += s_w[q] * s_grad[q][i * 3] * s_fval[q][j];
                        s3 += s_w[q] * s_val[q][i] * s_fval[q][j];
                    }
                    t2[idx] += s2;
                    t3[idx] += s3;
                }
                for (int idx = threadIdx.x; idx < nV * nV; idx += blockDim.x) {
                    int i = idx / nV, j = idx % nV;
                    double s = 0.0;
                    for (int q = 0; q < nt; ++q) s += s_w[q] * s_val[q][i] * s_val[q][j];
                    t4[idx] += s;
                }
                for (int idx = threadIdx.x; idx < nF * nF; idx += blockDim.x) {
                    int i = idx / nF, j = idx % nF;
                    double s = 0.0;
                    for (int q = 0; q < nt; ++q) s += s_w[q] * s_fval[q][i] * s_fval[q][j];
                    t5[idx] += s;
                }
                __syncthreads();
            }
        }
        // ---- transform to the orthonormal bases ----
        double* tmp = ws + SL.tmp;
        double* Kst = ws + SL.Kst;
        cta_mm(tmp, nR, C, nR, false, Kt, nR, false, nR, nR, nR, 1.0, 0.0);
        cta_mm(Kst, nR, tmp, nR, false, C, nR, true, nR, nR, nR, 1.0, 0.0);
        // D_c = C_E Dt_c C_V^T (in place via tmp; C is lower triangular, so its
        // leading n x n block maps the first n starting functions)
        for (int c = 0; c < d; ++c) {
            cta_mm(tmp, nV, C, nR, false, Dt + c * nE * nV, nV, false, nE, nV, nE, 1.0, 0.0);
            cta_mm(Dt + c * nE * nV, nV, tmp, nV, false, C, nR, true, nE, nV, nV, 1.0, 0.0);
        }
        for (int f = 0; f < N; ++f) {
            const double* CF = fC + (int64_t)E.fid[f] * nF * nF;
            double* t1 = T1 + f * nR * nV;
            double* t2 = T2 + f * nR * nF;
            double* t3 = T3 + f * nR * nF;
            double* t4 = T4 + f * nV * nV;
            double* t5 = T5 + f * nF * nF;
            // Dn_T = C t1 C_V^T  (nR x nV)
            cta_mm(tmp, nV, C, nR, false, t1, nV, false, nR, nV, nR, 1.0, 0.0);
            cta_mm(t1, nV, tmp, nV, false, C, nR, true, nR, nV, nV, 1.0, 0.0);
            // Dn_F = C t2 C_F^T  (nR x nF)
            cta_mm(tmp, nF, C, nR, false, t2, nF, false, nR, nF, nR, 1.0, 0.0);
            cta_mm(t2, nF, tmp, nF, false, CF, nF, true, nR, nF, nF, 1.0, 0.0);
            // M (element-face mass) = C t3 C_F^T  (nR x nF): M[m][j] = int phi_m psi_j
            cta_mm(tmp, nF, C, nR, false, t3, nF, false, nR, nF, nR, 1.0, 0.0);
            cta_mm(t3, nF, tmp, nF, false, CF, nF, true, nR, nF, nF, 1.0, 0.0);
            // Mtt = C_V t4 C_V^T
            cta_mm(tmp, nV, C, nR, false, t4, nV, false, nV, nV, nV, 1.0, 0.0);
            cta_mm(t4, nV, tmp, nV, false, C, nR, true, nV, nV, nV, 1.0, 0.0);
            // Mff = C_F t5 C_F^T
            cta_mm(tmp, nF, CF, nF, false, t5, nF, false, nF, nF, nF, 1.0, 0.0);
            cta_mm(t5, nF, tmp, nF, false, CF, nF, true, nF, nF, nF, 1.0, 0.0);
        }
        if (cond == HHO_DGCOND) {
            // DG scheme: the element's stiffness K, Dv[c][e][a] = int phi_e d_c phi_a, and per face the trace
            // matrices M[a][j] = int_F phi_a psi_j and DN[a][j] = int_F (grad phi_a . n_TF) psi_j (a < nE):
            // traces of P^k(T) on a planar face lie in P^k(F), so every face coupling is a product of these
            double* o = outS + off_S[t];
            for (int idx = threadIdx.x; idx < nE * nE; idx += blockDim.x)
                o[idx] = Kst[(idx / nE) * nR + idx % nE];
            o += nE * nE;
            for (int idx = threadIdx.x; idx < d * nE * nE; idx += blockDim.x) o[idx] = Dt[idx];
            o += d * nE * nE;
            for (int f = 0; f < N; ++f) {
                const double* t2 = T2 + f * nR * nF;
                const double* t3 = T3 + f * nR * nF;
                for (int idx = threadIdx.x; idx < nE * nF; idx += blockDim.x) {
                    o[idx] = t3[idx];
                    o[nE * nF + idx] = t2[idx];
                }
                o += 2 * nE * nF;
            }
            __syncthreads();
            continue;
        }
        // ---- reconstruction: Kst[1:,1:] P[1:,:] = Rhs[1:,:], P[0,:] = e_0 ----
        double* Rhs = ws + SL.Rhs;
        double* P = ws + SL.P;
        for (int idx = threadIdx.x; idx < nR * ns; idx += blockDim.x) {
            int i = idx / ns, a = idx % ns;
            double v;
            if (a < nV) {
                v = Kst[i * nR + a];
                for (int f = 0; f < N; ++f) v -= T1[f * nR * nV + i * nV + a];
            } else {
                int f = (a - nV) / nF, j = (a - nV) % nF;
                v = T2[f * nR * nF + i * nF + j];
            }
            Rhs[idx] = v;
        }
        __syncthreads();
        {
            int n1 = nR - 1, ldw = n1 + ns;
            double* W = ws + SL.Kl;  // reuse the local-matrix area as workspace
            for (int idx = threadIdx.x; idx < n1 * ldw; idx += blockDim.x) {
                int i = idx / ldw, c = idx % ldw;
                W[idx] = c < n1 ? Kst[(i + 1) * nR + (c + 1)] : Rhs[(i + 1) * ns + (c - n1)];
            }
            __syncthreads();
            if (!cta_gauss_jordan(W, ldw, n1, ns, &s_piv)) {
                if (threadIdx.x == 0) atomicExch(status, (int)HHO_ERR_SINGULAR);
            }
            for (int idx = threadIdx.x; idx < nR * ns; idx += blockDim.x) {
                int i = idx / ns, a = idx % ns;
                P[idx] = (i == 0) ? (a == 0 ? 1.0 : 0.0) : W[(i - 1) * ldw + n1 + a];
            }
            __syncthreads();
        }
        for (int i = threadIdx.x; i < nR * ns; i += blockDim.x) outP[off_P[t] + i] = P[i];
        // ---- scalar viscous form A (ns x ns) ----
        double* A = ws + SL.A;
        cta_mm(tmp, ns, Kst, nR, false, P, ns, false, nR, ns, nR, 1.0, 0.0);
        cta_mm(A, ns, P, ns, true, tmp, ns, false, ns, ns, nR, 1.0, 0.0);
        double* R = ws + SL.R;
        double* Mr = ws + SL.Mr;
        const int nr = nF + nV;
        for (int f = 0; f < N; ++f) {
            double* DnF = T2 + f * nR * nF;
            double* M = T3 + f * nR * nF;
            double* Mtt = T4 + f * nV * nV;
            double* Mff = T5 + f * nF * nF;
            // R = [E_F - M^T P ; E_T - P[:nV]]  ((nF+nV) x ns): the face residual's
            // element part is pi_T^{k'} (v_T - p v), the first nV coefficients
            for (int idx = threadIdx.x; idx < nr * ns; idx += blockDim.x) {
                int i = idx / ns, a = idx % ns;
                double v;
                if (i < nF) {
                    v = (a == nV + f * nF + i) ? 1.0 : 0.0;
                    for (int m = 0; m < nR; ++m) v -= M[m * nF + i] * P[m * ns + a];
                } else {
                    int ii = i - nF;
                    v = (a == ii ? 1.0 : 0.0) - P[ii * ns + a];
                }
                R[idx] = v;
            }
            // Mr = [[Mff, -Mft], [-Mft^T, Mtt]] / h_F with Mft[j][i] = M[i][j], i < nV
            double ih = 1.0 / E.hF[f];
            for (int idx = threadIdx.x; idx < nr * nr; idx += blockDim.x) {
                int i = idx / nr, j = idx % nr;
                double v;
                if (i < nF && j < nF) v = Mff[i * nF + j];
                else if (i < nF) v = -M[(j - nF) * nF + i];
                else if (j < nF) v = -M[(i - nF) * nF + j];
                else v = Mtt[(i - nF) * nV + (j - nF)];
                Mr[idx] = v * ih;
            }
            __syncthreads();
            cta_mm(tmp, ns, Mr, nr, false, R, ns, false, nr, ns, nr, 1.0, 0.0);
            cta_mm(A, ns, R, ns, true, tmp, ns, false, ns, ns, nr, 1.0, 1.0);
            if (E.bcf[f] == 1) {
                double eta = 4.0 * (k + 1) * (k + d) / (double)d * E.mF[f] * E.hF[f] / E.meas;
                // G = Dn_F^T P (nF x ns): int (n.grad p v) psi_j
                cta_mm(tmp, ns, DnF, nF, true, P, ns, false, nF, ns, nR, 1.0, 0.0);
                for (int idx = threadIdx.x; idx < ns * ns; idx += blockDim.x) {
                    int a = idx / ns, bb = idx % ns;
                    double v = 0.0;
                    int ja = a - nV - f * nF, jb = bb - nV - f * nF;
                    bool fa = (ja >= 0 && ja < nF), fb = (jb >= 0 && jb < nF);
                    if (fa) v -= tmp[ja * ns + bb];
                    if (fb) v -= tmp[jb * ns + a];
                    if (fa && fb) v += eta / E.hF[f] * Mff[ja * nF + jb];
                    A[idx] += v;
                }
                __syncthreads();
            }
        }
        // ---- local matrix K = [[A_vec, B^T], [B, 0]] ----
        double* Kl = ws + SL.Kl;
        const int nvec = D.nvec, nloc = D.nloc;
        cta_zero(Kl, nloc * nloc);
        for (int idx = threadIdx.x; idx < d * ns * ns; idx += blockDim.x) {
            int c = idx / (ns * ns), r = idx % (ns * ns), a = r / ns, bb = r % ns;
            Kl[vmap(D, c, a) * nloc + vmap(D, c, bb)] = A[r];
        }
        __syncthreads();
        // B rows: element pressure (i < nE), then the face pressures of HHO-hp
        for (int idx = threadIdx.x; idx < D.npr * nvec; idx += blockDim.x) {
            int i = idx / nvec, col = idx % nvec;
            double v = 0.0;
            if (i < nE) {
                if (col < d * nV) {
                    int c = col / nV, j = col % nV;
                    v = -Dt[c * nE * nV + i * nV + j];
                    if (cond != HHO_HPCOND)
                        for (int f = 0; f < N; ++f) v += E.nTF[f][c] * T4[f * nV * nV + i * nV + j];
                } else if (cond != HHO_HPCOND) {
                    int r = col - d * nV, f = r / D.bv, cc = (r % D.bv) / nF, j = r % nF;
                    if (E.bcf[f] != 1) v = -E.nTF[f][cc] * T3[f * nR * nF + i * nF + j];
                }
            } else {
                // int_F (v_T - v_F) . n q_F, v_F dropped on Dirichlet faces (Sec. 2.3.2)
                int f = (i - nE) / nF, ii = (i - nE) % nF;
                if (col < d * nV) {
                    int c = col / nV, j = col % nV;
                    v = E.nTF[f][c] * T3[f * nR * nF + j * nF + ii];
                } else {
                    int r = col - d * nV, g = r / D.bv, cc = (r % D.bv) / nF, j = r % nF;
                    if (g == f && E.bcf[f] != 1) v = -E.nTF[f][cc] * T5[f * nF * nF + ii * nF + j];
                }
            }
            Kl[(nvec + i) * nloc + col] = v;
            Kl[col * nloc + (nvec + i)] = v;
        }
        __syncthreads();
        // ---- static condensation: [Kee | Kek | I] -> [I | X | Kee^{-1}] ----
        const int nel = D.nel, nk = D.nk, ldw = nel + nk + nel;
        double* W = ws + SL.W;
        for (int idx = threadIdx.x; idx < nel * ldw; idx += blockDim.x) {
            int i = idx / ldw, c = idx % ldw;
            int gi = elim_idx(D, i);
            double v;
            if (c < nel) v = Kl[gi * nloc + elim_idx(D, c)];
            else if (c < nel + nk) v = Kl[gi * nloc + keep_idx(D, c - nel)];
            else v = (c - nel - nk == i) ? 1.0 : 0.0;
            W[idx] = v;
        }
        __syncthreads();
        if (!cta_gauss_jordan(W, ldw, nel, nk + nel, &s_piv)) {
            if (threadIdx.x == 0) atomicExch(status, (int)HHO_ERR_SINGULAR);
        }
        double* Xo = outX + off_X[t];
        double* Ko = outKei + off_Kei[t];
        double* So = outS + off_S[t];
        for (int idx = threadIdx.x; idx < nel * nk; idx += blockDim.x) {
            int i = idx / nk, c = idx % nk;
            Xo[idx] = W[i * ldw + nel + c];
        }
        for (int idx = threadIdx.x; idx < nel * nel; idx += blockDim.x) {
            int i = idx / nel, c = idx % nel;
            Ko[idx] = W[i * ldw + nel + nk + c];
        }
        // S = Kkk - Kke X
        for (int idx = threadIdx.x; idx < nk * nk; idx += blockDim.x) {
            int i = idx / nk, j = idx % nk;
            int gi = keep_idx(D, i);
            double s = Kl[gi * nloc + keep_idx(D, j)];
            double acc = 0.0;
            for (int l = 0; l < nel; ++l) acc += Kl[gi * nloc + elim_idx(D, l)] * W[l * ldw + nel + j];
            So[idx] = s - acc;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Right-hand side kernel (data integrals of degree 2k+2) and local condensation.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TPB) k_rhs(int d, int k, int cond, int64_t ne, const double* __restrict__ xyz,
                                             const int32_t* __restrict__ ef_ptr, const int32_t* __restrict__ ef,
                                             const int32_t* __restrict__ fv_ptr, const int32_t* __restrict__ fv,
                                             const int8_t* __restrict__ fbc, const FaceGeo* __restrict__ fgeo,
                                             const double* __restrict__ fC, const double* __restrict__ eC,
                                             const double* __restrict__ emeas, const double* __restrict__ gl,
                                             const int64_t* __restrict__ enode_off, const int64_t* __restrict__ fnode_off,
                                             const double* __restrict__ fdat, const double* __restrict__ gD,
                                             const double* __restrict__ gN, const int64_t* __restrict__ off_X,
                                             const int64_t* __restrict__ off_Kei, const int64_t* __restrict__ off_P,
                                             const int64_t* __restrict__ off_gT, const int64_t* __restrict__ off_yT,
                                             const double* __restrict__ X, const double* __restrict__ Kei,
                                             const double* __restrict__ Pm, double* __restrict__ gT,
                                             double* __restrict__ yT, double* __restrict__ scratch, int64_t scratch_per) {
    __shared__ ElemSh E;
    __shared__ double s_acc[3 * 36 + 3 * 10 + 36 + 10];
    __shared__ double s_tile[RQ_F * 86 > RQ_E * 39 ? RQ_F * 86 : RQ_E * 39];
    __shared__ RecTab tab;
    rec_tab_fill(tab);
    const int nR = dimP(d, k + 1), nE = dimP(d, k), nF = dimP(d - 1, k);
    const int nV = (cond == HHO_HPCOND) ? nR : nE;  // element velocity coefficients
    const int kv = (cond == HHO_HPCOND) ? k + 1 : k;
    const int pd = 2 * k + 2;
    double* ws = scratch + (int64_t)blockIdx.x * scratch_per;
    for (int64_t t = blockIdx.x; t < ne; t += gridDim.x) {
        load_element(E, d, (int)t, ef_ptr, ef, fv_ptr, fv, xyz, fgeo, fbc);
        if (threadIdx.x == 0) E.meas = emeas[t];
        __syncthreads();
        const LocalDims D = local_dims(d, k, E.N, cond);
        const int nloc = D.nloc, ns = D.ns;
        double* rhs = ws;  // nloc
        for (int i = threadIdx.x; i < nloc; i += blockDim.x) rhs[i] = 0.0;
        const double* C = eC + t * nR * nR;
        const double* P = Pm + off_P[t];
        __syncthreads();
        // body force: int f_c phi_j, j < nV (starting basis, then transform).
        // Tiles of RQ_E points: one thread per point evaluates the starting
        // functions into shared memory, then thread idx < d nV adds its
        // product over the tile's points in order (one register accumulator
        // per thread; every sum has a fixed order).
        {
            int nq = elem_npts(E, d, pd);
            int64_t o = enode_off[t];
            double* s_v = s_tile;                  // [RQ_E][nV]
            double* s_wf = s_tile + RQ_E * 36;     // [RQ_E][3] weight times f_c
            double acc = 0.0;
            const int cI = threadIdx.x / (nV > 0 ? nV : 1), aI = threadIdx.x - cI * nV;
            for (int q0 = 0; q0 < nq; q0 += RQ_E) {
                const int nt = min(RQ_E, nq - q0);
                if (threadIdx.x < nt) {
                    double x[3] = {0, 0, 0}, w;
                    elem_point(E, d, gl, pd, q0 + threadIdx.x, x, &w);
                    elem_start_val(E, d, kv, x, s_v + threadIdx.x * nV, tab);
                    for (int c = 0; c < d; ++c) s_wf[threadIdx.x * 3 + c] = w * fdat[(o + q0 + threadIdx.x) * d + c];
                }
                __syncthreads();
                if (threadIdx.x < d * nV)
                    for (int q = 0; q < nt; ++q) acc += s_wf[q * 3 + cI] * s_v[q * nV + aI];
                __syncthreads();
            }
            if (threadIdx.x < d * nV) s_acc[threadIdx.x] = acc;
            __syncthreads();
            for (int idx = threadIdx.x; idx < d * nV; idx += blockDim.x) {
                int c = idx / nV, j = idx % nV;
                double v = 0.0;
                for (int a = 0; a <= j; ++a) v += C[j * nR + a] * s_acc[c * nV + a];
                rhs[c * nV + j] += v;
            }
            __syncthreads();
        }
        // boundary faces
        for (int f = 0; f < E.N; ++f) {
            int bc = E.bcf[f];
            if (bc == 0) continue;
            int F = E.fid[f];
            const FaceGeo& g = fgeo[F];
            const double* CF = fC + (int64_t)F * nF * nF;
            int nqf = face_npts(d, E.nvf[f], pd);
            int64_t o = fnode_off[F];
            const double* gv = (bc == 1) ? gD : gN;
            // accumulators: for each c: sum w g_c dn phi~_m (nR), sum w g_c psi~_j (nF); sum w (g.n) phi~_i (nR);
            // sum w (g.n) psi~_j (nF).  Tiles of RQ_F points as for the body force; accumulator slot sl of
            // thread t is acc index t + sl TPB.
            {
                double* s_fv = s_tile;                 // [RQ_F][36] values
                double* s_dn = s_tile + RQ_F * 36;     // [RQ_F][36] normal derivatives
                double* s_ff = s_tile + RQ_F * 72;     // [RQ_F][10] face functions
                double* s_gw = s_tile + RQ_F * 82;     // [RQ_F][4] w g_c, w (g . n)
                const int n1 = d * nR, n2 = n1 + d * nF, n3 = n2 + nR, nacc = n3 + nF;
                double accf[2] = {0.0, 0.0};
                for (int q0 = 0; q0 < nqf; q0 += RQ_F) {
                    const int nt = min(RQ_F, nqf - q0);
                    if (threadIdx.x < nt) {
                        const int q = q0 + threadIdx.x;
                        double x[3] = {0, 0, 0}, w, grad[36 * 3];
                        face_point(d, E.V[f], E.nvf[f], E.xF[f], gl, pd, q, x, &w);
                        elem_start(E, d, k + 1, x, s_fv + threadIdx.x * 36, grad);
                        face_start(g, d, k, x, s_ff + threadIdx.x * 10);
                        for (int m = 0; m < nR; ++m) {
                            double dn = 0.0;
                            for (int c = 0; c < d; ++c) dn += grad[m * 3 + c] * E.nTF[f][c];
                            s_dn[threadIdx.x * 36 + m] = dn;
                        }
                        double gn = 0.0;
                        for (int c = 0; c < d; ++c) {
                            gn += gv[(o + q) * d + c] * E.nTF[f][c];
                            s_gw[threadIdx.x * 4 + c] = w * gv[(o + q) * d + c];
                        }
                        s_gw[threadIdx.x * 4 + 3] = w * gn;
                    }
                    __syncthreads();
                    for (int sl = 0; sl < 2; ++sl) {
                        const int i = threadIdx.x + sl * TPB;
                        if (i >= nacc) continue;
                        double sum = 0.0;
                        if (i < n1) {
                            const int c = i / nR, m = i % nR;
                            for (int qq = 0; qq < nt; ++qq) sum += s_gw[qq * 4 + c] * s_dn[qq * 36 + m];
                        } else if (i < n2) {
                            const int c = (i - n1) / nF, j = (i - n1) % nF;
                            for (int qq = 0; qq < nt; ++qq) sum += s_gw[qq * 4 + c] * s_ff[qq * 10 + j];
                        } else if (i < n3) {
                            const int m = i - n2;
                            for (int qq = 0; qq < nt; ++qq) sum += s_gw[qq * 4 + 3] * s_fv[qq * 36 + m];
                        } else {
                            const int j = i - n3;
                            for (int qq = 0; qq < nt; ++qq) sum += s_gw[qq * 4 + 3] * s_ff[qq * 10 + j];
                        }
                        accf[sl] += sum;
                    }
                    __syncthreads();
                }
                for (int sl = 0; sl < 2; ++sl) {
                    const int i = threadIdx.x + sl * TPB;
                    if (i >= nacc) continue;
                    int slot;
                    if (i < n1) slot = (i / nR) * 36 + i % nR;
                    else if (i < n2) slot = 3 * 36 + ((i - n1) / nF) * 10 + (i - n1) % nF;
                    else if (i < n3) slot = 3 * 36 + 3 * 10 + (i - n2);
                    else slot = 3 * 36 + 3 * 10 + 36 + (i - n3);
                    s_acc[slot] = accf[sl];
                }
            }
            __syncthreads();
            if (cond == HHO_DGCOND && threadIdx.x == 0) {
                // DG (Scheme 3): data through the face basis (traces of P^k(T) lie in P^k(F)):
                // Neumann: + int g_N . v_T; Dirichlet: the g_D part of the jump 2 (u_T - g_D) in the BR2 terms,
                // - (-int L_FT(-2 g_D) . grad v_T + eta int n . L_FT(-2 g_D) v_T), and + int (g_D . n) q_T
                const double* Dv = P + nE * nE;
                const double* Mf = P + (d + 1) * nE * nE + (int64_t)f * 2 * nE * nF;
                double G[3][10], Gn[10];
                for (int j = 0; j < nF; ++j) {
                    for (int c = 0; c < d; ++c) {
                        double v = 0.0;
                        for (int a = 0; a <= j; ++a) v += CF[j * nF + a] * s_acc[3 * 36 + c * 10 + a];
                        G[c][j] = v;
                    }
                    double v = 0.0;
                    for (int a = 0; a <= j; ++a) v += CF[j * nF + a] * s_acc[3 * 36 + 3 * 10 + 36 + a];
                    Gn[j] = v;
                }
                if (bc == 2) {
                    for (int c = 0; c < d; ++c)
                        for (int a = 0; a < nE; ++a) {
                            double v = 0.0;
                            for (int j = 0; j < nF; ++j) v += Mf[a * nF + j] * G[c][j];
                            rhs[c * nE + a] += v;
                        }
                } else {
                    const double eta = E.N + 1.0;
                    for (int c = 0; c < d; ++c) {
                        double MG[36], Wj[10];
                        for (int e = 0; e < nE; ++e) {
                            double v = 0.0;
                            for (int j = 0; j < nF; ++j) v += Mf[e * nF + j] * G[c][j];
                            MG[e] = v;
                        }
                        for (int j = 0; j < nF; ++j) {
                            double v = 0.0;
                            for (int e = 0; e < nE; ++e) v += Mf[e * nF + j] * MG[e];
                            Wj[j] = v;
                        }
                        for (int a = 0; a < nE; ++a) {
                            double a1 = 0.0, a3 = 0.0;
                            for (int cc = 0; cc < d; ++cc)
                                for (int e = 0; e < nE; ++e) a1 += E.nTF[f][cc] * Dv[(cc * nE + e) * nE + a] * MG[e];
                            for (int j = 0; j < nF; ++j) a3 -= eta * Mf[a * nF + j] * Wj[j];
                            rhs[c * nE + a] -= a1 + a3;
                        }
                    }
                    for (int a = 0; a < nE; ++a) {
                        double v = 0.0;
                        for (int j = 0; j < nF; ++j) v += Mf[a * nF + j] * Gn[j];
                        rhs[d * nE + a] += v;
                    }
                }
            } else if (threadIdx.x == 0) {
                double eta = 4.0 * (k + 1) * (k + d) / (double)d * E.mF[f] * E.hF[f] / E.meas;
                for (int c = 0; c < d; ++c) {
                    // face coefficients: int g_c psi_j
                    double gpsi[10];
                    for (int j = 0; j < nF; ++j) {
                        double v = 0.0;
                        for (int a = 0; a <= j; ++a) v += CF[j * nF + a] * s_acc[3 * 36 + c * 10 + a];
                        gpsi[j] = v;
                    }
                    int base = D.d * nV + f * D.bv + c * nF;
                    if (bc == 1) {
                        // tdn_m = int g_c dn phi_m (orthonormal)
                        double tdn[36];
                        for (int m = 0; m < nR; ++m) {
                            double v = 0.0;
                            for (int a = 0; a <= m; ++a) v += C[m * nR + a] * s_acc[c * 36 + a];
                            tdn[m] = v;
                        }
                        for (int a = 0; a < ns; ++a) {
                            double v = 0.0;
                            for (int m = 0; m < nR; ++m) v += P[m * ns + a] * tdn[m];
                            rhs[vmap(D, c, a)] -= v;
                        }
                        for (int j = 0; j < nF; ++j) rhs[base + j] += eta / E.hF[f] * gpsi[j];
                    } else {
                        for (int j = 0; j < nF; ++j) rhs[base + j] += gpsi[j];
                    }
                }
                if (bc == 1 && cond != HHO_HPCOND) {  // - int g_D . n q_T  (Eq. HHOdiscrCNT)
                    for (int i = 0; i < nE; ++i) {
                        double v = 0.0;
                        for (int a = 0; a <= i; ++a) v += C[i * nR + a] * s_acc[3 * 36 + 3 * 10 + a];
                        rhs[D.nvec + i] += v;
                    }
                } else if (bc == 1) {  // HHO-hp: - int g_D . n q_F on the Dirichlet face
                    for (int j = 0; j < nF; ++j) {
                        double v = 0.0;
                        for (int a = 0; a <= j; ++a) v += CF[j * nF + a] * s_acc[3 * 36 + 3 * 10 + 36 + a];
                        rhs[D.nvec + nE + f * nF + j] += v;
                    }
                }
            }
            __syncthreads();
        }
        if (cond == HHO_DGCOND) {  // DG: the element's block of the global right-hand side
            for (int i = threadIdx.x; i < (d + 1) * nE; i += blockDim.x) gT[off_gT[t] + i] = rhs[i];
            __syncthreads();
            continue;
        }
        // condensation of the RHS: g = rhs_k - X^T rhs_e, y = Kee^{-1} rhs_e
        const double* Xt = X + off_X[t];
        const double* Kt = Kei + off_Kei[t];
        for (int j = threadIdx.x; j < D.nk; j += blockDim.x) {
            double s = rhs[keep_idx(D, j)];
            for (int l = 0; l < D.nel; ++l) s -= Xt[l * D.nk + j] * rhs[elim_idx(D, l)];
            gT[off_gT[t] + j] = s;
        }
        for (int i = threadIdx.x; i < D.nel; i += blockDim.x) {
            double s = 0.0;
            for (int l = 0; l < D.nel; ++l) s += Kt[i * D.nel + l] * rhs[elim_idx(D, l)];
            yT[off_yT[t] + i] = s;
        }
        __syncthreads();
    }
}

__global__ void k_nodes(int d, int k, int which, int64_t n_items, const double* __restrict__ xyz,
                        const int32_t* __restrict__ ef_ptr, const int32_t* __restrict__ ef,
                        const int32_t* __restrict__ fv_ptr, const int32_t* __restrict__ fv, const int8_t* __restrict__ fbc,
                        const FaceGeo* __restrict__ fgeo, const int32_t* __restrict__ fe, const double* __restrict__ gl,
                        const int64_t* __restrict__ node_off, double* __restrict__ out, double* __restrict__ normals) {
    __shared__ ElemSh E;
    const int pd = 2 * k + 2;
    for (int64_t t = blockIdx.x; t < n_items; t += gridDim.x) {
        if (which == HHO_NODES_ELEM) {
            load_element(E, d, (int)t, ef_ptr, ef, fv_ptr, fv, xyz, fgeo, fbc);
            int nq = elem_npts(E, d, pd);
            for (int q = threadIdx.x; q < nq; q += blockDim.x) {
                double x[3] = {0, 0, 0}, w;
                elem_point(E, d, gl, pd, q, x, &w);
                for (int j = 0; j < d; ++j) out[(node_off[t] + q) * d + j] = x[j];
            }
        } else {
            const FaceGeo& g = fgeo[t];
            int a = fv_ptr[t], nv = fv_ptr[t + 1] - a;
            double V[MAX_FVERT][3] = {};
            for (int i = 0; i < nv; ++i)
                for (int j = 0; j < d; ++j) V[i][j] = xyz[(int64_t)fv[a + i] * d + j];
            // outward normal of the first element: sign from its vertex average
            int T = fe[2 * t];
            double xT[3] = {0, 0, 0};
            {
                // vertex average of element T over unique vertex ids
                int vids[MAX_NFACE * MAX_FVERT], nvid = 0;
                for (int ff = ef_ptr[T]; ff < ef_ptr[T + 1]; ++ff) {
                    int Fi = ef[ff];
                    for (int i = fv_ptr[Fi]; i < fv_ptr[Fi + 1]; ++i) {
                        bool seen = false;
                        for (int s = 0; s < nvid; ++s) seen |= (vids[s] == fv[i]);
                        if (!seen) vids[nvid++] = fv[i];
                    }
                }
                for (int s = 0; s < nvid; ++s)
                    for (int j = 0; j < d; ++j) xT[j] += xyz[(int64_t)vids[s] * d + j];
                for (int j = 0; j < d; ++j) xT[j] /= nvid;
            }
            double s = 0.0;
            for (int j = 0; j < d; ++j) s += g.n[j] * (g.xF[j] - xT[j]);
            double sg = s > 0.0 ? 1.0 : -1.0;
            int nq = face_npts(d, nv, pd);
            for (int q = threadIdx.x; q < nq; q += blockDim.x) {
                double x[3] = {0, 0, 0}, w;
                face_point(d, V, nv, g.xF, gl, pd, q, x, &w);
                for (int j = 0; j < d; ++j) {
                    out[(node_off[t] + q) * d + j] = x[j];
                    if (normals) normals[(node_off[t] + q) * d + j] = sg * g.n[j];
                }
            }
        }
        __syncthreads();
    }
}

// Recovery (back-substitution) of the eliminated unknowns.
__global__ void k_recover(int d, int k, int cond, int64_t ne, int64_t nf, int b, int nP, const int32_t* __restrict__ ef_ptr,
                          const int32_t* __restrict__ ef, const int64_t* __restrict__ off_X,
                          const int64_t* __restrict__ off_yT, const int64_t* __restrict__ off_loc,
                          const double* __restrict__ X, const double* __restrict__ yT, const double* __restrict__ x,
                          double* __restrict__ out) {
    const int nE = dimP(d, k);
    for (int64_t t = blockIdx.x; t < ne; t += gridDim.x) {
        int f0 = ef_ptr[t], N = ef_ptr[t + 1] - f0;
        LocalDims D = local_dims(d, k, N, cond);
        double* o = out + off_loc[t];
        // kept unknowns (face blocks, then the element's kept pressures; HHO-hp keeps face blocks only)
        for (int j = threadIdx.x; j < D.nk; j += blockDim.x) {
            double v;
            if (j < N * b) v = x[(int64_t)ef[f0 + j / b] * b + j % b];
            else v = x[nf * b + t * nP + (j - N * b)];
            o[keep_idx(D, j)] = v;
        }
        __syncthreads();
        const double* Xt = X + off_X[t];
        for (int i = threadIdx.x; i < D.nel; i += blockDim.x) {
            double s = yT[off_yT[t] + i];
            for (int j = 0; j < D.nk; ++j) s -= Xt[i * D.nk + j] * o[keep_idx(D, j)];
            o[elim_idx(D, i)] = s;
        }
        __syncthreads();
    }
}

// Error integrals per element: [ |Pu-u|^2, |grad(Pu-u)|^2, int (p_h-p)^2, int (p_h - p), |T|, |div u_T|^2 ].
__global__ void k_errors(int d, int k, int cond, int64_t ne, const double* __restrict__ xyz,
                         const int32_t* __restrict__ ef_ptr, const int32_t* __restrict__ ef,
                         const int32_t* __restrict__ fv_ptr, const int32_t* __restrict__ fv, const int8_t* __restrict__ fbc,
                         const FaceGeo* __restrict__ fgeo, const double* __restrict__ eC, const double* __restrict__ gl,
                         const int64_t* __restrict__ enode_off, const int64_t* __restrict__ off_P,
                         const int64_t* __restrict__ off_loc, const double* __restrict__ Pm,
                         const double* __restrict__ loc, const double* __restrict__ u, const double* __restrict__ gu,
                         const double* __restrict__ p, double* __restrict__ part) {
    __shared__ ElemSh E;
    __shared__ double s_coef[3][36];
    __shared__ double red[6][TPB];
    const int nR = dimP(d, k + 1), nE = dimP(d, k);
    const int nV = (cond == HHO_HPCOND) ? nR : nE;  // element velocity coefficients
    const int pd = 2 * k + 2;
    for (int64_t t = blockIdx.x; t < ne; t += gridDim.x) {
        load_element(E, d, (int)t, ef_ptr, ef, fv_ptr, fv, xyz, fgeo, fbc);
        LocalDims D = local_dims(d, k, E.N, cond);
        const double* C = eC + t * nR * nR;
        const double* P = Pm + off_P[t];
        const double* U = loc + off_loc[t];
        // reconstruction coefficients per component in the orthonormal basis, then starting basis
        for (int idx = threadIdx.x; idx < d * nR; idx += blockDim.x) {
            int c = idx / nR, m = idx % nR;
            double s = 0.0;
            if (cond == HHO_DGCOND) s = m < nE ? U[c * nE + m] : 0.0;  // DG: the element velocity itself
            else
                for (int a = 0; a < D.ns; ++a) s += P[m * D.ns + a] * U[vmap(D, c, a)];
            s_coef[c][m] = s;
        }
        __syncthreads();
        // convert to starting-basis coefficients: sum_m coef_m C[m][a]
        __shared__ double s_st[3][36], s_ut[3][36], s_pt[36];
        for (int idx = threadIdx.x; idx < d * nR; idx += blockDim.x) {
            int c = idx / nR, a = idx % nR;
            double s = 0.0, su = 0.0;
            for (int m = a; m < nR; ++m) s += s_coef[c][m] * C[m * nR + a];
            for (int m = a; m < nV; ++m) su += U[c * nV + m] * C[m * nR + a];
            s_st[c][a] = s;
            s_ut[c][a] = (a < nV) ? su : 0.0;
        }
        const double* Up = (cond == HHO_DGCOND) ? U + d * nE : U + D.nvec;  // element pressure coefficients
        for (int a = threadIdx.x; a < nR; a += blockDim.x) {
            double s = 0.0;
            for (int m = a; m < nE; ++m) s += Up[m] * C[m * nR + a];
            s_pt[a] = (a < nE) ? s : 0.0;
        }
        __syncthreads();
        double acc[6] = {0, 0, 0, 0, 0, 0};
        int nq = elem_npts(E, d, pd);
        int64_t o = enode_off[t];
        for (int q = threadIdx.x; q < nq; q += blockDim.x) {
            double x[3] = {0, 0, 0}, w, val[36], grad[36 * 3];
            elem_point(E, d, gl, pd, q, x, &w);
            elem_start(E, d, k + 1, x, val, grad);
            double div = 0.0;
            for (int c = 0; c < d; ++c) {
                double uh = 0.0, g[3] = {0, 0, 0};
                for (int a = 0; a < nR; ++a) {
                    uh += s_st[c][a] * val[a];
                    for (int j = 0; j < d; ++j) g[j] += s_st[c][a] * grad[a * 3 + j];
                    div += s_ut[c][a] * grad[a * 3 + c];
                }
                double e = uh - u[(o + q) * d + c];
                acc[0] += w * e * e;
                for (int j = 0; j < d; ++j) {
                    double ge = g[j] - gu[((o + q) * d + c) * d + j];
                    acc[1] += w * ge * ge;
                }
            }
            double ph = 0.0;
            for (int a = 0; a < nE; ++a) ph += s_pt[a] * val[a];
            double ep = ph - p[o + q];
            acc[2] += w * ep * ep;
            acc[3] += w * ep;
            acc[4] += w;
            acc[5] += w * div * div;
        }
        for (int i = 0; i < 6; ++i) red[i][threadIdx.x] = acc[i];
        __syncthreads();
        if (threadIdx.x < 6) {
            double s = 0.0;
            for (int i = 0; i < TPB; ++i) s += red[threadIdx.x][i];
            part[t * 6 + threadIdx.x] = s;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// DG scheme (Scheme 3, Sec. 2.4): the element-block operator.  Row block of
// element S: slot 0 = S itself, slot 1 + i = the neighbour across S's i-th
// interior face (local face order).  Every face coupling is formed from the
// element data of k_elements (K, Dv, and per face the trace matrices M, DN in
// the face basis): with M_X the traces of element X on face F,
//   int_F phi_a^S phi_b^X = (M_S M_X^T)[a][b],
//   int_F phi_a^S (grad phi_b^X . n_X) = (M_S DN_X^T)[a][b],
// and the BR2 lifting of a jump is 1/2 n (x) (M_S M_X^T) on S.  One CTA per
// element; each block entry is written by that CTA only (faces in order).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TPB) k_dg_assemble(int d, int k, int64_t ne, const double* __restrict__ xyz,
                                                     const int32_t* __restrict__ ef_ptr, const int32_t* __restrict__ ef,
                                                     const int32_t* __restrict__ fv_ptr, const int32_t* __restrict__ fv,
                                                     const int8_t* __restrict__ fbc, const FaceGeo* __restrict__ fgeo,
                                                     const int32_t* __restrict__ fe, const int32_t* __restrict__ flf,
                                                     const int64_t* __restrict__ off_S, const double* __restrict__ dgd,
                                                     int S_max, double* __restrict__ ff) {
    __shared__ ElemSh E;
    // nE, nF <= 10 and d nE^2 <= 300: hho_setup refuses DG degrees above 3 (2D) and 2 (3D)
    __shared__ double s_P[100], s_MDN[100], s_MQM[100], s_DP[300], s_Q[100];
    const int nE = dimP(d, k), nF = dimP(d - 1, k), b = (d + 1) * nE;
    for (int64_t S = blockIdx.x; S < ne; S += gridDim.x) {
        load_element(E, d, (int)S, ef_ptr, ef, fv_ptr, fv, xyz, fgeo, fbc);
        const double* dS = dgd + off_S[S];
        const double* K = dS;
        const double* Dv = dS + nE * nE;
        const int64_t bb = (int64_t)b * b;
        auto at = [&](int s, int r, int c) -> double& { return ff[((int64_t)s * bb + (int64_t)c * b + r) * ne + S]; };
        for (int64_t i = threadIdx.x; i < S_max * bb; i += blockDim.x) {
            const int s = (int)(i / bb), rc = (int)(i % bb);
            at(s, rc % b, rc / b) = 0.0;
        }
        __syncthreads();
        // volume: K per velocity component, -int p div v and its transpose
        for (int i = threadIdx.x; i < b * b; i += blockDim.x) {
            const int r = i / b, c = i % b;
            const int gr = r / nE, a = r % nE, gc = c / nE, q = c % nE;
            double v = 0.0;
            if (gr < d && gc == gr) v = K[a * nE + q];
            else if (gr < d && gc == d) v = -Dv[(gr * nE + q) * nE + a];
            else if (gr == d && gc < d) v = -Dv[(gc * nE + a) * nE + q];
            at(0, r, c) += v;
        }
        __syncthreads();
        int slot = 0;
        for (int f = 0; f < E.N; ++f) {
            const int F = E.fid[f];
            const bool interior = fe[2 * F] >= 0 && fe[2 * F + 1] >= 0;
            if (!interior && E.bcf[f] == 2) continue;  // Neumann faces carry no BR2 term and no coupling
            int Tn = -1, fn = -1;
            if (interior) {
                const int e0 = fe[2 * F];
                Tn = (e0 == (int)S) ? fe[2 * F + 1] : e0;
                fn = (e0 == (int)S) ? flf[2 * F + 1] : flf[2 * F];
                ++slot;
            }
            const double* MS = dS + (d + 1) * nE * nE + (int64_t)f * 2 * nE * nF;
            const double* MT = interior ? dgd + off_S[Tn] + (d + 1) * nE * nE + (int64_t)fn * 2 * nE * nF : nullptr;
            const int NS = E.N, NT = interior ? ef_ptr[Tn + 1] - ef_ptr[Tn] : 0;
            const double eta = (interior ? (double)max(NS, NT) : (double)NS) + 1.0;
            const double hF = E.hF[f];
            // Q = M_S^T M_S (+ M_T^T M_T on interior faces): nF x nF
            for (int i = threadIdx.x; i < nF * nF; i += blockDim.x) {
                const int j = i / nF, jj = i % nF;
                double v = 0.0;
                for (int e = 0; e < nE; ++e) v += MS[e * nF + j] * MS[e * nF + jj];
                if (interior)
                    for (int e = 0; e < nE; ++e) v += MT[e * nF + j] * MT[e * nF + jj];
                s_Q[i] = v;
            }
            __syncthreads();
            for (int side = 0; side < (interior ? 2 : 1); ++side) {
                const double* MX = side == 0 ? MS : MT;
                const double* DNX = MX + nE * nF;
                const double sig = interior ? (side == 0 ? 1.0 : -1.0) : 2.0;
                const int s = side == 0 ? 0 : slot;
                for (int i = threadIdx.x; i < nE * nE; i += blockDim.x) {
                    const int a = i / nE, q = i % nE;
                    double p = 0.0, m = 0.0, mq = 0.0;
                    for (int j = 0; j < nF; ++j) {
                        p += MS[a * nF + j] * MX[q * nF + j];
                        m += MS[a * nF + j] * DNX[q * nF + j];
                        double t = 0.0;
                        for (int jj = 0; jj < nF; ++jj) t += s_Q[j * nF + jj] * MX[q * nF + jj];
                        mq += MS[a * nF + j] * t;
                    }
                    s_P[i] = p;
                    s_MDN[i] = m;
                    s_MQM[i] = mq;
                }
                __syncthreads();
                for (int i = threadIdx.x; i < d * nE * nE; i += blockDim.x) {
                    const int c = i / (nE * nE), a = (i / nE) % nE, q = i % nE;
                    double v = 0.0;
                    for (int e = 0; e < nE; ++e) v += Dv[(c * nE + e) * nE + a] * s_P[e * nE + q];
                    s_DP[i] = v;
                }
                __syncthreads();
                for (int i = threadIdx.x; i < b * b; i += blockDim.x) {
                    const int r = i / b, c = i % b;
                    const int gr = r / nE, a = r % nE, gc = c / nE, q = c % nE;
                    const double P = s_P[a * nE + q];
                    double v = 0.0;
                    if (gr < d && gc == gr) {
                        double dp = 0.0;
                        for (int cc = 0; cc < d; ++cc) dp += E.nTF[f][cc] * s_DP[(cc * nE + a) * nE + q];
                        if (interior) v = -0.5 * sig * dp - 0.5 * sig * s_MDN[a * nE + q] + 0.25 * eta * sig * s_MQM[a * nE + q];
                        else v = -dp - s_MDN[a * nE + q] + eta * s_MQM[a * nE + q];
                    } else if (gr < d && gc == d) {
                        v = (interior ? 0.5 : 1.0) * E.nTF[f][gr] * P;
                    } else if (gr == d && gc < d) {
                        v = (interior ? 0.5 * sig : 1.0) * E.nTF[f][gc] * P;
                    } else if (gr == d && gc == d && interior) {
                        v = -hF * sig * P;
                    }
                    if (v != 0.0) at(s, r, c) += v;
                }
                __syncthreads();
            }
        }
    }
}

void gauss_legendre_tables(std::vector<double>& tab) {
    tab.assign(2 * (MAX_GL + 1) * MAX_GL, 0.0);
    for (int n = 1; n <= MAX_GL; ++n) {
        std::vector<double> xs(n), ws(n);
        for (int i = 0; i < n; ++i) {
            double x = std::cos(M_PI * (i + 0.75) / (n + 0.5));
            for (int it = 0; it < 100; ++it) {
                double p0 = 1.0, p1 = x;
                for (int m = 1; m < n; ++m) {
                    double p2 = ((2 * m + 1) * x * p1 - m * p0) / (m + 1);
                    p0 = p1;
                    p1 = p2;
                }
                double pn = (n == 0) ? 1.0 : p1, pnm1 = p0;
                if (n == 1) {
                    pn = x;
                    pnm1 = 1.0;
                }
                double dp = n * (x * pn - pnm1) / (x * x - 1.0);
                double dx = pn / dp;
                x -= dx;
                if (std::fabs(dx) < 1e-17) break;
            }
            double p0 = 1.0, p1 = x;
            for (int m = 1; m < n; ++m) {
                double p2 = ((2 * m + 1) * x * p1 - m * p0) / (m + 1);
                p0 = p1;
                p1 = p2;
            }
            double pn = (n == 1) ? x : p1, pnm1 = (n == 1) ? 1.0 : p0;
            double dp = n * (x * pn - pnm1) / (x * x - 1.0);
            xs[n - 1 - i] = x;  // ascending order
            ws[n - 1 - i] = 2.0 / ((1.0 - x * x) * dp * dp);
        }
        for (int i = 0; i < n; ++i) {
            tab[n * MAX_GL + i] = 0.5 * (xs[i] + 1.0);
            tab[(MAX_GL + 1) * MAX_GL + n * MAX_GL + i] = 0.5 * ws[i];
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host drivers
// ---------------------------------------------------------------------------
static int element_grid(int64_t ne) {
    int64_t g = (int64_t)sm_count() * 4;
    return (int)std::min<int64_t>(g, std::max<int64_t>(ne, 1));
}

// DG scheme: level-0 element-block operator from the element data of
// k_elements (one CTA per element, grid-stride).
hho_status dg_assemble_level0(hho_ctx* ctx, double* ff, int S_max) {
    const Disc& D = ctx->disc;
    k_dg_assemble<<<element_grid(D.ne), TPB, 0, ctx->stream>>>(D.d, D.k, D.ne, D.xyz, D.ef_ptr, D.ef, D.fv_ptr, D.fv,
                                                                D.fbc, D.fgeo, D.fe, D.flf, D.off_S, D.S, S_max, ff);
    HHO_CUDA(cudaGetLastError());
    return HHO_OK;
}

hho_status build_discretisation(hho_ctx* ctx, const hho_mesh* m, int k, int cond) {
    Disc& D = ctx->disc;
    const int d = m->dim;
    D.d = d;
    D.k = k;
    D.cond = cond;
    D.nv = m->n_vert;
    D.ne = m->n_elem;
    D.nf = m->n_face;
    D.nR = dimP(d, k + 1);
    D.nE = dimP(d, k);
    D.nF = dimP(d - 1, k);
    D.b = (cond == HHO_DGCOND) ? (d + 1) * D.nE : local_dims(d, k, 0, cond).b;
    D.nP = (cond == HHO_HPCOND || cond == HHO_DGCOND) ? 0
           : (cond == HHO_VPCOND)                      ? 1
           : (cond == HHO_UNCOND)                      ? (d + 1) * D.nE
                                                       : D.nE;
    // host topology (int32)
    D.h_ef_ptr.resize(D.ne + 1);
    D.h_ef.resize(m->elem_face_ptr[D.ne]);
    for (int64_t i = 0; i <= D.ne; ++i) D.h_ef_ptr[i] = (int32_t)m->elem_face_ptr[i];
    for (int64_t i = 0; i < (int64_t)D.h_ef.size(); ++i) D.h_ef[i] = (int32_t)m->elem_face[i];
    std::vector<int32_t> h_fv_ptr(D.nf + 1), h_fv(m->face_vert_ptr[D.nf]);
    for (int64_t i = 0; i <= D.nf; ++i) h_fv_ptr[i] = (int32_t)m->face_vert_ptr[i];
    for (int64_t i = 0; i < (int64_t)h_fv.size(); ++i) h_fv[i] = (int32_t)m->face_vert[i];
    D.h_fv_ptr = h_fv_ptr;
    D.h_fv = h_fv;
    D.h_xyz.assign(m->xyz, m->xyz + D.nv * d);
    D.h_fe.resize(2 * D.nf);
    for (int64_t i = 0; i < 2 * D.nf; ++i) D.h_fe[i] = (int32_t)m->face_elem[i];
    D.h_fbc.assign(m->face_bc, m->face_bc + D.nf);
    D.h_flf.assign(2 * D.nf, -1);
    D.maxN = 0;
    for (int64_t t = 0; t < D.ne; ++t) {
        int N = D.h_ef_ptr[t + 1] - D.h_ef_ptr[t];
        D.maxN = std::max(D.maxN, N);
        for (int f = 0; f < N; ++f) {
            int F = D.h_ef[D.h_ef_ptr[t] + f];
            if (D.h_fe[2 * F] == t) D.h_flf[2 * F] = f;
            else if (D.h_fe[2 * F + 1] == t) D.h_flf[2 * F + 1] = f;
        }
    }
    // per-element offsets of the local outputs
    std::vector<int64_t> oS(D.ne), oX(D.ne), oK(D.ne), oP(D.ne), oL(D.ne), oG(D.ne), oY(D.ne);
    int64_t tS = 0, tX = 0, tK = 0, tP = 0, tL = 0, tG = 0, tY = 0;
    for (int64_t t = 0; t < D.ne; ++t) {
        const LocalDims L = local_dims(d, k, D.h_ef_ptr[t + 1] - D.h_ef_ptr[t], cond);
        const int ns = L.ns, nloc = L.nloc, nel = L.nel, nk = L.nk;
        oS[t] = tS;
        tS += (cond == HHO_DGCOND) ? (int64_t)(d + 1) * D.nE * D.nE + 2LL * L.N * D.nE * D.nF : (int64_t)nk * nk;
        oX[t] = tX;
        tX += (int64_t)nel * nk;
        oK[t] = tK;
        tK += (int64_t)nel * nel;
        oP[t] = tP;
        tP += (int64_t)D.nR * ns;
        oL[t] = tL;
        tL += (cond == HHO_DGCOND) ? (int64_t)(d + 1) * D.nE : nloc;  // DG: the solution block itself
        oG[t] = tG;
        tG += (cond == HHO_DGCOND) ? (int64_t)(d + 1) * D.nE : nk;  // DG: the element's block of the global RHS
        oY[t] = tY;
        tY += nel;
    }
    D.h_off_S = oS;
    D.h_off_loc = oL;
    D.h_off_gT = oG;
    D.tot_S = tS;
    D.tot_X = tX;
    D.tot_Kei = tK;
    D.tot_P = tP;
    D.tot_loc = tL;
    D.tot_gT = tG;
    D.tot_yT = tY;
    // data-node offsets
    D.h_enode_off.resize(D.ne + 1);
    D.h_fnode_off.resize(D.nf + 1);
    const int pd = 2 * k + 2;
    int64_t on = 0;
    for (int64_t t = 0; t < D.ne; ++t) {
        D.h_enode_off[t] = on;
        int N = D.h_ef_ptr[t + 1] - D.h_ef_ptr[t];
        if (d == 2) {
            int n = (pd + 3) / 2;
            on += (int64_t)N * n * n;
        } else {
            int n = (pd + 4) / 2, s = 0;
            for (int f = 0; f < N; ++f) {
                int F = D.h_ef[D.h_ef_ptr[t] + f];
                s += h_fv_ptr[F + 1] - h_fv_ptr[F];
            }
            on += (int64_t)s * n * n * n;
        }
    }
    D.h_enode_off[D.ne] = on;
    D.n_enodes = on;
    on = 0;
    for (int64_t F = 0; F < D.nf; ++F) {
        D.h_fnode_off[F] = on;
        on += face_npts(d, h_fv_ptr[F + 1] - h_fv_ptr[F], pd);
    }
    D.h_fnode_off[D.nf] = on;
    D.n_fnodes = on;

    // ---- device allocations and uploads ----
    auto up = [&](auto** dst, const auto* src, size_t n) -> hho_status {
        HHO_TRY(dalloc(ctx, dst, n));
        HHO_CUDA(cudaMemcpyAsync(*dst, src, n * sizeof(**dst), cudaMemcpyHostToDevice, ctx->stream));
        return HHO_OK;
    };
    HHO_TRY(up(&D.xyz, m->xyz, (size_t)D.nv * d));
    HHO_TRY(up(&D.ef_ptr, D.h_ef_ptr.data(), D.h_ef_ptr.size()));
    HHO_TRY(up(&D.ef, D.h_ef.data(), D.h_ef.size()));
    HHO_TRY(up(&D.fv_ptr, h_fv_ptr.data(), h_fv_ptr.size()));
    HHO_TRY(up(&D.fv, h_fv.data(), h_fv.size()));
    HHO_TRY(up(&D.fe, D.h_fe.data(), D.h_fe.size()));
    HHO_TRY(up(&D.flf, D.h_flf.data(), D.h_flf.size()));
    HHO_TRY(up(&D.fbc, D.h_fbc.data(), D.h_fbc.size()));
    HHO_TRY(up(&D.off_S, oS.data(), oS.size()));
    HHO_TRY(up(&D.off_X, oX.data(), oX.size()));
    HHO_TRY(up(&D.off_Kei, oK.data(), oK.size()));
    HHO_TRY(up(&D.off_P, oP.data(), oP.size()));
    HHO_TRY(up(&D.off_loc, oL.data(), oL.size()));
    HHO_TRY(up(&D.off_gT, oG.data(), oG.size()));
    HHO_TRY(up(&D.off_yT, oY.data(), oY.size()));
    HHO_TRY(up(&D.enode_off, D.h_enode_off.data(), D.h_enode_off.size()));
    HHO_TRY(up(&D.fnode_off, D.h_fnode_off.data(), D.h_fnode_off.size()));
    std::vector<double> tab;
    gauss_legendre_tables(tab);
    HHO_TRY(up(&D.gl, tab.data(), tab.size()));
    HHO_TRY(dalloc(ctx, &D.fgeo, D.nf));
    HHO_TRY(dalloc(ctx, &D.fC, (size_t)D.nf * D.nF * D.nF));
    HHO_TRY(dalloc(ctx, &D.eC, (size_t)D.ne * D.nR * D.nR));
    HHO_TRY(dalloc(ctx, &D.emeas, D.ne));
    HHO_TRY(dalloc(ctx, &D.S, D.tot_S));
    HHO_TRY(dalloc(ctx, &D.X, D.tot_X));
    HHO_TRY(dalloc(ctx, &D.Kei, D.tot_Kei));
    HHO_TRY(dalloc(ctx, &D.P, D.tot_P));
    HHO_TRY(dalloc(ctx, &D.gT, D.tot_gT));
    HHO_TRY(dalloc(ctx, &D.yT, D.tot_yT));

    // ---- kernels ----
    k_faces<<<(unsigned)((D.nf + 127) / 128), 128, 0, ctx->stream>>>(d, k, D.nf, D.xyz, D.fv_ptr, D.fv, D.gl, D.fgeo,
                                                                      D.fC);
    HHO_CUDA(cudaGetLastError());
    int grid = element_grid(D.ne);
    ScratchLayout SL = scratch_layout(d, k, D.maxN, cond);
    double* scratch = nullptr;
    HHO_TRY(dalloc(ctx, &scratch, (size_t)grid * SL.total));
    HHO_CUDA(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream));
    k_elements<<<grid, TPB, 0, ctx->stream>>>(d, k, cond, D.ne, D.xyz, D.ef_ptr, D.ef, D.fv_ptr, D.fv, D.fbc, D.fgeo,
                                              D.fC, D.gl, D.maxN, scratch, D.eC, D.emeas, D.off_S, D.off_X, D.off_Kei,
                                              D.off_P, D.S, D.X, D.Kei, D.P, ctx->d_flag);
    cudaError_t le = cudaGetLastError();
    int flag = 0;
    cudaError_t ce = cudaMemcpyAsync(&flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    cudaError_t se = cudaStreamSynchronize(ctx->stream);
    dfree(scratch);
    HHO_CUDA(le);
    HHO_CUDA(ce);
    HHO_CUDA(se);
    if (flag != 0) {
        ctx->err = "hho_setup: zero pivot in a local factorisation";
        return HHO_ERR_SINGULAR;
    }
    return HHO_OK;
}

hho_status build_rhs(hho_ctx* ctx, const double* f, const double* gD, const double* gN) {
    Disc& D = ctx->disc;
    const bool dg = D.cond == HHO_DGCOND;  // the DG element data (D.S) take the place of the reconstruction
    int grid = element_grid(D.ne);
    const int64_t per = (local_dims(D.d, D.k, D.maxN, D.cond).nloc + 3) & ~3;
    double* scratch = nullptr;
    HHO_TRY(dalloc(ctx, &scratch, (size_t)grid * per));
    k_rhs<<<grid, TPB, 0, ctx->stream>>>(D.d, D.k, D.cond, D.ne, D.xyz, D.ef_ptr, D.ef, D.fv_ptr, D.fv, D.fbc, D.fgeo,
                                         D.fC, D.eC, D.emeas, D.gl, D.enode_off, D.fnode_off, f, gD, gN, D.off_X,
                                         D.off_Kei, dg ? D.off_S : D.off_P, D.off_gT, D.off_yT, D.X, D.Kei,
                                         dg ? D.S : D.P, D.gT, D.yT, scratch, per);
    cudaError_t le = cudaGetLastError();
    cudaError_t se = cudaStreamSynchronize(ctx->stream);
    dfree(scratch);
    HHO_CUDA(le);
    HHO_CUDA(se);
    return HHO_OK;
}

// Same element right-hand-side kernel as build_rhs, with caller-provided working
// memory of `capacity` doubles instead of a fresh allocation.  Enqueues only;
// the grid is shrunk so that every CTA gets one local vector of scratch.
hho_status build_rhs_scratch(hho_ctx* ctx, const double* f, const double* gD, const double* gN, double* scratch,
                             int64_t capacity) {
    Disc& D = ctx->disc;
    const bool dg = D.cond == HHO_DGCOND;
    const int64_t per = (local_dims(D.d, D.k, D.maxN, D.cond).nloc + 3) & ~3;
    const int64_t fit = capacity / per;
    if (fit < 1) {
        ctx->err = "hho_assemble_noalloc: one element's local system needs more working memory than the fixed array holds";
        return HHO_ERR_ARG;
    }
    const int grid = (int)std::min<int64_t>(element_grid(D.ne), fit);
    k_rhs<<<grid, TPB, 0, ctx->stream>>>(D.d, D.k, D.cond, D.ne, D.xyz, D.ef_ptr, D.ef, D.fv_ptr, D.fv, D.fbc, D.fgeo,
                                         D.fC, D.eC, D.emeas, D.gl, D.enode_off, D.fnode_off, f, gD, gN, D.off_X,
                                         D.off_Kei, dg ? D.off_S : D.off_P, D.off_gT, D.off_yT, D.X, D.Kei,
                                         dg ? D.S : D.P, D.gT, D.yT, scratch, per);
    HHO_CUDA(cudaGetLastError());
    return HHO_OK;
}

hho_status quad_nodes(hho_ctx* ctx, int which, int64_t* n, double* xyz, double* normals) {
    Disc& D = ctx->disc;
    if (which != HHO_NODES_ELEM && which != HHO_NODES_FACE) {
        ctx->err = "hho_quad_nodes: unknown node set";
        return HHO_ERR_ARG;
    }
    *n = (which == HHO_NODES_ELEM) ? D.n_enodes : D.n_fnodes;
    if (!xyz) return HHO_OK;
    int64_t items = (which == HHO_NODES_ELEM) ? D.ne : D.nf;
    int grid = element_grid(items);
    k_nodes<<<grid, 64, 0, ctx->stream>>>(D.d, D.k, which, items, D.xyz, D.ef_ptr, D.ef, D.fv_ptr, D.fv, D.fbc, D.fgeo,
                                          D.fe, D.gl, which == HHO_NODES_ELEM ? D.enode_off : D.fnode_off, xyz,
                                          which == HHO_NODES_FACE ? normals : nullptr);
    HHO_CUDA(cudaGetLastError());
    HHO_CUDA(cudaStreamSynchronize(ctx->stream));
    return HHO_OK;
}

hho_status recover_local(hho_ctx* ctx, const double* x, double* local) {
    Disc& D = ctx->disc;
    if (D.cond == HHO_DGCOND) {  // no eliminated unknowns: the local vectors are the solution's element blocks
        HHO_CUDA(cudaMemcpyAsync(local, x, (size_t)D.ne * D.b * sizeof(double), cudaMemcpyDeviceToDevice,
                                 ctx->stream));
        return HHO_OK;
    }
    int grid = element_grid(D.ne);
    k_recover<<<grid, 64, 0, ctx->stream>>>(D.d, D.k, D.cond, D.ne, D.nf, D.b, D.nP, D.ef_ptr, D.ef, D.off_X, D.off_yT,
                                            D.off_loc, D.X, D.yT, x, local);
    HHO_CUDA(cudaGetLastError());
    return HHO_OK;
}

hho_status compute_errors(hho_ctx* ctx, const double* local, const double* u, const double* gu, const double* p,
                          double out[4]) {
    Disc& D = ctx->disc;
    double* part = nullptr;
    HHO_TRY(dalloc(ctx, &part, (size_t)D.ne * 6));
    int grid = element_grid(D.ne);
    k_errors<<<grid, TPB, 0, ctx->stream>>>(D.d, D.k, D.cond, D.ne, D.xyz, D.ef_ptr, D.ef, D.fv_ptr, D.fv, D.fbc,
                                            D.fgeo, D.eC, D.gl, D.enode_off, D.off_P, D.off_loc, D.P, local, u, gu, p,
                                            part);
    cudaError_t le = cudaGetLastError();
    std::vector<double> h((size_t)D.ne * 6);
    cudaError_t ce = cudaMemcpyAsync(h.data(), part, h.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    cudaError_t se = cudaStreamSynchronize(ctx->stream);
    dfree(part);
    HHO_CUDA(le);
    HHO_CUDA(ce);
    HHO_CUDA(se);
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t t = 0; t < D.ne; ++t)
        for (int i = 0; i < 6; ++i) s[i] += h[t * 6 + i];
    bool neumann = false;
    for (auto b : D.h_fbc) neumann |= (b == 2);
    double ep2 = s[2];
    if (!neumann) {
        double delta = s[3] / s[4];
        ep2 = s[2] - 2.0 * delta * s[3] + delta * delta * s[4];
    }
    out[0] = std::sqrt(s[0]);
    out[1] = std::sqrt(s[1]);
    out[2] = std::sqrt(std::fmax(ep2, 0.0));
    out[3] = std::sqrt(s[5]);
    return HHO_OK;
}

}  // namespace hho
