"""Analytic manufactured fields, evaluated at caller-chosen points.

Each field set gives, at points x of shape (n, d):
  u(x)      (n, d)      velocity
  grad_u(x) (n, d, d)   grad_u[:, i, j] = d u_i / d x_j
  p(x)      (n,)        pressure
  f(x)      (n, d)      body force  f = -Lap u + grad p       (Eq. stokesProb)
The boundary data are g_D = u on Dirichlet faces and, on Neumann faces,
g_N = (grad_u - p I) n, the traction that makes the momentum residual of
Scheme 1 consistent (the residual subtracts the integral of g_N . v_F).
"""
from __future__ import annotations

import numpy as np

PI = np.pi


class Field:
    name = "field"
    p_mean = 0.0  # mean of p over the unit box

    def g_neumann(self, x, n):
        gu = self.grad_u(x)
        p = self.p(x)
        return np.einsum("qij,qj->qi", gu, n) - p[:, None] * n


class TrigStokes2D(Field):
    """u = (sin(pi x) cos(pi y), -cos(pi x) sin(pi y)), p = sin(2 pi x) sin(2 pi y)."""
    name = "trig2d"

    def u(self, x):
        X, Y = x[:, 0], x[:, 1]
        return np.stack([np.sin(PI * X) * np.cos(PI * Y), -np.cos(PI * X) * np.sin(PI * Y)], axis=1)

    def grad_u(self, x):
        X, Y = x[:, 0], x[:, 1]
        g = np.empty((x.shape[0], 2, 2))
        g[:, 0, 0] = PI * np.cos(PI * X) * np.cos(PI * Y)
        g[:, 0, 1] = -PI * np.sin(PI * X) * np.sin(PI * Y)
        g[:, 1, 0] = PI * np.sin(PI * X) * np.sin(PI * Y)
        g[:, 1, 1] = -PI * np.cos(PI * X) * np.cos(PI * Y)
        return g

    def p(self, x):
        return np.sin(2 * PI * x[:, 0]) * np.sin(2 * PI * x[:, 1])

    def f(self, x):
        X, Y = x[:, 0], x[:, 1]
        f1 = 2 * PI ** 2 * np.sin(PI * X) * np.cos(PI * Y) + 2 * PI * np.cos(2 * PI * X) * np.sin(2 * PI * Y)
        f2 = -2 * PI ** 2 * np.cos(PI * X) * np.sin(PI * Y) + 2 * PI * np.sin(2 * PI * X) * np.cos(2 * PI * Y)
        return np.stack([f1, f2], axis=1)


class CurlStokes3D(Field):
    """u = curl(psi (1,1,1)) with psi = sin(pi x) sin(pi y) sin(pi z); p = cos(pi x) cos(pi y) cos(pi z)."""
    name = "curl3d"

    @staticmethod
    def _psi_derivs(x):
        s = np.sin(PI * x)
        c = np.cos(PI * x)
        sx, sy, sz = s[:, 0], s[:, 1], s[:, 2]
        cx, cy, cz = c[:, 0], c[:, 1], c[:, 2]
        d1 = np.stack([PI * cx * sy * sz, PI * sx * cy * sz, PI * sx * sy * cz], axis=1)
        d2 = np.empty((x.shape[0], 3, 3))
        d2[:, 0, 0] = -PI ** 2 * sx * sy * sz
        d2[:, 1, 1] = -PI ** 2 * sx * sy * sz
        d2[:, 2, 2] = -PI ** 2 * sx * sy * sz
        d2[:, 0, 1] = d2[:, 1, 0] = PI ** 2 * cx * cy * sz
        d2[:, 0, 2] = d2[:, 2, 0] = PI ** 2 * cx * sy * cz
        d2[:, 1, 2] = d2[:, 2, 1] = PI ** 2 * sx * cy * cz
        return d1, d2

    def u(self, x):
        d1, _ = self._psi_derivs(x)
        return np.stack([d1[:, 1] - d1[:, 2], d1[:, 2] - d1[:, 0], d1[:, 0] - d1[:, 1]], axis=1)

    def grad_u(self, x):
        _, d2 = self._psi_derivs(x)
        g = np.empty((x.shape[0], 3, 3))
        g[:, 0, :] = d2[:, 1, :] - d2[:, 2, :]
        g[:, 1, :] = d2[:, 2, :] - d2[:, 0, :]
        g[:, 2, :] = d2[:, 0, :] - d2[:, 1, :]
        return g

    def p(self, x):
        return np.cos(PI * x[:, 0]) * np.cos(PI * x[:, 1]) * np.cos(PI * x[:, 2])

    def f(self, x):
        # each first derivative of psi is an eigenfunction of the Laplacian with eigenvalue -3 pi^2
        s = np.sin(PI * x)
        c = np.cos(PI * x)
        gp = -PI * np.stack([s[:, 0] * c[:, 1] * c[:, 2], c[:, 0] * s[:, 1] * c[:, 2],
                             c[:, 0] * c[:, 1] * s[:, 2]], axis=1)
        return 3 * PI ** 2 * self.u(x) + gp


class PolyStokes(Field):
    """Divergence-free polynomial velocity and polynomial pressure.

    2D: u = (d psi/dy, -d psi/dx) for a stream function psi of degree deg_u+1.
    3D: u = curl(A) for a vector potential A of degree deg_u+1.
    Coefficients are monomial coefficient arrays (numpy.polynomial layout).
    """
    name = "poly"

    def __init__(self, dim, deg_u, deg_p, rng: np.random.Generator):
        from numpy.polynomial import polynomial as P
        self.P = P
        self.dim = dim
        n = deg_u + 2
        m = deg_p + 1

        def rand_coef(deg, nd):
            c = np.zeros((deg + 1,) * nd)
            for idx in np.ndindex(*c.shape):
                if sum(idx) <= deg:
                    c[idx] = rng.standard_normal()
            return c

        if dim == 2:
            psi = rand_coef(n - 1, 2)
            self.uc = [P.polyder(psi, axis=1), -P.polyder(psi, axis=0)]
        else:
            A = [rand_coef(n - 1, 3) for _ in range(3)]
            d = lambda c, ax: P.polyder(c, axis=ax)
            self.uc = [_sub(d(A[2], 1), d(A[1], 2)), _sub(d(A[0], 2), d(A[2], 0)), _sub(d(A[1], 0), d(A[0], 1))]
        self.pc = rand_coef(m - 1, dim)

    def _val(self, c, x):
        if self.dim == 2:
            return self.P.polyval2d(x[:, 0], x[:, 1], c)
        return self.P.polyval3d(x[:, 0], x[:, 1], x[:, 2], c)

    def u(self, x):
        return np.stack([self._val(c, x) for c in self.uc], axis=1)

    def grad_u(self, x):
        g = np.empty((x.shape[0], self.dim, self.dim))
        for i, c in enumerate(self.uc):
            for j in range(self.dim):
                g[:, i, j] = self._val(self.P.polyder(c, axis=j), x)
        return g

    def p(self, x):
        return self._val(self.pc, x)

    def f(self, x):
        out = np.zeros((x.shape[0], self.dim))
        for i, c in enumerate(self.uc):
            lap = sum(self._val(self.P.polyder(c, m=2, axis=j), x) for j in range(self.dim))
            out[:, i] = -lap + self._val(self.P.polyder(self.pc, axis=i), x)
        return out


def _sub(a, b):
    shape = tuple(max(sa, sb) for sa, sb in zip(a.shape, b.shape))
    out = np.zeros(shape)
    out[tuple(slice(0, s) for s in a.shape)] += a
    out[tuple(slice(0, s) for s in b.shape)] -= b
    return out
