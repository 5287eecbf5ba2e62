"""Hierarchical L2-orthonormal modal bases (oracle), Secs. 2.1 and 4.2.

The space P^K(X) on an element or face X is spanned by starting functions
chosen to be well conditioned on X:
* triangles: the collapsed-coordinate orthogonal polynomials of the reference
  triangle (Dubiner), pulled back by the affine map x = v0 + (r+1)/2 (v1-v0) +
  (s+1)/2 (v2-v0); psi_pq = Q_p(r,s) J_q^{(2p+1,0)}(s) with Q_p = P_p(a) t^p,
  t = (1-s)/2, a t = r + (1+s)/2, evaluated by the division-free recurrence
  (p+1) Q_{p+1} = (2p+1) (a t) Q_p - p t^2 Q_{p-1};
* every other element or face: products P_a1(xi_1) ... P_ad(xi_d) of Legendre
  polynomials of the bounding-box coordinates xi = (y - c)/r (y = x for
  elements, y = the coordinates in the face's tangent frame for faces).
They are ordered by total degree 0..K and, within a degree, by decreasing
first index (x-major), and orthonormalised in L2(X) by modified Gram-Schmidt applied twice per function
(MGS2), in that order, with inner products taken from the quadrature Gram
matrix.  Because the order is by degree, the first dim P^l functions span
P^l(X) for every l <= K: restriction to a lower degree is truncation of the
coefficient vector (Sec. 4.2, the unit-diagonal I^{l+1}_l), and the degree-k
basis is a prefix of the degree-(k+1) one.
"""
from __future__ import annotations

import numpy as np


def dim_P(n_var: int, deg: int) -> int:
    if deg < 0:
        return 0
    if n_var == 0:
        return 1
    if n_var == 1:
        return deg + 1
    if n_var == 2:
        return (deg + 1) * (deg + 2) // 2
    return (deg + 1) * (deg + 2) * (deg + 3) // 6


def multi_indices(n_var: int, K: int):
    out = []
    for l in range(K + 1):
        if n_var == 1:
            out.append((l,))
        elif n_var == 2:
            for a in range(l, -1, -1):
                out.append((a, l - a))
        else:
            for a in range(l, -1, -1):
                for b in range(l - a, -1, -1):
                    out.append((a, b, l - a - b))
    return out


def legendre(nmax, x):
    """Values and derivatives of P_0..P_nmax at x (Bonnet recurrence)."""
    x = np.asarray(x, float)
    P = np.zeros((nmax + 1,) + x.shape)
    D = np.zeros_like(P)
    P[0] = 1.0
    if nmax >= 1:
        P[1] = x
        D[1] = 1.0
    for n in range(1, nmax):
        P[n + 1] = ((2 * n + 1) * x * P[n] - n * P[n - 1]) / (n + 1)
        D[n + 1] = ((2 * n + 1) * (P[n] + x * D[n]) - n * D[n - 1]) / (n + 1)
    return P, D


def jacobi(nmax, alpha, x):
    """Values and derivatives of the Jacobi polynomials P_n^{(alpha,0)}, n <= nmax."""
    x = np.asarray(x, float)
    P = np.zeros((nmax + 1,) + x.shape)
    D = np.zeros_like(P)
    P[0] = 1.0
    if nmax >= 1:
        P[1] = 0.5 * ((alpha + 2) * x + alpha)
        D[1] = 0.5 * (alpha + 2)
    a = alpha
    for n in range(2, nmax + 1):
        c0 = 2.0 * n * (n + a) * (2 * n + a - 2)
        c1 = (2 * n + a - 1) * (2 * n + a) * (2 * n + a - 2)
        c2 = (2 * n + a - 1) * a * a
        c3 = 2.0 * (n + a - 1) * (n - 1) * (2 * n + a)
        P[n] = ((c1 * x + c2) * P[n - 1] - c3 * P[n - 2]) / c0
        D[n] = (c1 * P[n - 1] + (c1 * x + c2) * D[n - 1] - c3 * D[n - 2]) / c0
    return P, D


def dubiner(K, r, s):
    """Values and (r, s)-gradients of the Dubiner functions of degree <= K.

    Returned in the order of multi_indices(2, K) with (p, q) = (a1, a2).
    """
    t = 0.5 * (1.0 - s)
    u = r + 0.5 * (1.0 + s)
    Q = np.zeros((K + 1,) + r.shape)
    Qr = np.zeros_like(Q)
    Qs = np.zeros_like(Q)
    Q[0] = 1.0
    if K >= 1:
        Q[1] = u
        Qr[1] = 1.0
        Qs[1] = 0.5
    for p in range(1, K):
        Q[p + 1] = ((2 * p + 1) * u * Q[p] - p * t * t * Q[p - 1]) / (p + 1)
        Qr[p + 1] = ((2 * p + 1) * (Q[p] + u * Qr[p]) - p * t * t * Qr[p - 1]) / (p + 1)
        Qs[p + 1] = ((2 * p + 1) * (0.5 * Q[p] + u * Qs[p]) - p * (-t * Q[p - 1] + t * t * Qs[p - 1])) / (p + 1)
    idx = multi_indices(2, K)
    V = np.zeros(r.shape + (len(idx),))
    G = np.zeros(r.shape + (len(idx), 2))
    for m, (p, q) in enumerate(idx):
        J, Jd = jacobi(q, 2 * p + 1, s)
        V[..., m] = Q[p] * J[q]
        G[..., m, 0] = Qr[p] * J[q]
        G[..., m, 1] = Qs[p] * J[q] + Q[p] * Jd[q]
    return V, G


class Basis:
    """Orthonormal basis of P^K on an element (n_var = d) or face (n_var = d-1)."""

    def __init__(self, K, n_var, origin, frame, bb_c, bb_r, rule_pts, rule_wts, simplex=None):
        self.simplex = simplex      # (v0, v1, v2) for the Dubiner starting functions
        self.K = K
        self.n_var = n_var
        self.origin = origin
        self.frame = frame          # (n_var, d) rows = axes of the local coordinates
        self.c = bb_c
        self.r = bb_r
        self.alpha = multi_indices(n_var, K)
        self.n = len(self.alpha)
        Phi, _ = self._start(rule_pts)
        G = Phi.T @ (rule_wts[:, None] * Phi)
        self.C = mgs2(G)

    def _start(self, X):
        if self.simplex is not None:
            v0, v1, v2 = self.simplex
            M = np.stack([v1 - v0, v2 - v0], axis=1)
            Minv = np.linalg.inv(M)
            rs = (X - v0) @ Minv.T * 2.0 - 1.0
            V, G = dubiner(self.K, rs[:, 0], rs[:, 1])
            # grad_x = 2 M^{-T} grad_rs
            return V, 2.0 * G @ Minv
        Y = (X - self.origin) @ self.frame.T
        xi = (Y - self.c) / self.r
        vals = []
        ders = []
        for i in range(self.n_var):
            P, D = legendre(self.K, xi[:, i])
            vals.append(P)
            ders.append(D / self.r[i])
        nq = X.shape[0]
        Phi = np.ones((nq, self.n))
        dPhi = np.ones((nq, self.n, self.n_var))
        for m, a in enumerate(self.alpha):
            for i in range(self.n_var):
                Phi[:, m] *= vals[i][a[i]]
                for j in range(self.n_var):
                    dPhi[:, m, j] *= ders[i][a[i]] if i == j else vals[i][a[i]]
        return Phi, dPhi

    def eval(self, X, n=None):
        """Values (nq, n) of the first n basis functions at points X."""
        n = self.n if n is None else n
        Phi, _ = self._start(X)
        return Phi @ self.C[:n].T

    def eval_grad(self, X, n=None):
        """Values (nq, n) and gradients (nq, n, d) in ambient coordinates."""
        n = self.n if n is None else n
        Phi, dPhi = self._start(X)
        vals = Phi @ self.C[:n].T
        # d/dx_j = sum_i d/dy_i * frame[i, j]
        dloc = np.einsum("qmi,nm->qni", dPhi, self.C[:n])
        grads = dloc @ self.frame
        return vals, grads


def mgs2(G):
    """Coefficients C (row i = function i) orthonormal in the Gram metric G.

    Modified Gram-Schmidt, two passes per function, in index order.
    """
    n = G.shape[0]
    C = np.zeros((n, n))
    for i in range(n):
        c = np.zeros(n)
        c[i] = 1.0
        for _ in range(2):
            for j in range(i):
                c = c - (C[j] @ (G @ c)) * C[j]
        C[i] = c / np.sqrt(c @ (G @ c))
    return C


def element_basis(eg, K):
    d = eg.dim
    pts, wts = eg.rule(2 * K)
    simplex = None
    if d == 2 and len(eg.faces) == 3:
        F0 = eg.faces[0]
        v0, v1 = F0.V[0], F0.V[1]
        others = [F.V[j] for F in eg.faces[1:] for j in range(2)]
        v2 = next(v for v in others if not (np.array_equal(v, v0) or np.array_equal(v, v1)))
        simplex = (v0, v1, v2)
    return Basis(K, d, np.zeros(d), np.eye(d), eg.bb_c, eg.bb_r, pts, wts, simplex)


def face_basis(fg, K):
    pts, wts = fg.rule(2 * K)
    return Basis(K, fg.dim - 1, fg.xF, fg.frame, fg.bb_c, fg.bb_r, pts, wts)
