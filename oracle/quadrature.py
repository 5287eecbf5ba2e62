"""Quadrature rules (oracle).

Polytopal elements and faces are integrated by splitting them into simplices
(fan from the vertex average, Sec. 2.1 allows general polytopes) and applying
collapsed-coordinate tensor Gauss-Legendre rules on each simplex.

Simplex rules (reading: the paper does not fix its quadrature):
  segment [a,b], degree p:   n = ceil((p+1)/2) points, x = a + u (b-a)
  triangle (a,b,c), degree p: n = ceil((p+2)/2) per direction,
      xi = u, eta = v (1-u), weight w_u w_v (1-u) * 2|T|
  tetrahedron (a,b,c,d), degree p: n = ceil((p+3)/2) per direction,
      xi = u, eta = v (1-u), zeta = w (1-u)(1-v), weight w_u w_v w_w (1-u)^2 (1-v) * 6|T|
  with (u,v,w) Gauss-Legendre nodes mapped to [0,1], u outermost.
"""
from __future__ import annotations

import numpy as np


def gauss01(n: int):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def segment_rule(a, b, p):
    n = (p + 2) // 2
    u, w = gauss01(n)
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    pts = a[None, :] + u[:, None] * (b - a)[None, :]
    return pts, w * np.linalg.norm(b - a)


def triangle_rule(a, b, c, p):
    n = (p + 3) // 2
    u, w = gauss01(n)
    a, b, c = (np.asarray(z, float) for z in (a, b, c))
    e1, e2 = b - a, c - a
    if a.shape[0] == 2:
        area = 0.5 * abs(e1[0] * e2[1] - e1[1] * e2[0])
    else:
        area = 0.5 * np.linalg.norm(np.cross(e1, e2))
    pts, wts = [], []
    for iu in range(n):
        for iv in range(n):
            xi = u[iu]
            eta = u[iv] * (1.0 - u[iu])
            pts.append(a + xi * e1 + eta * e2)
            wts.append(w[iu] * w[iv] * (1.0 - u[iu]) * 2.0 * area)
    return np.array(pts), np.array(wts)


def tet_rule(a, b, c, d, p):
    n = (p + 4) // 2
    u, w = gauss01(n)
    a, b, c, d = (np.asarray(z, float) for z in (a, b, c, d))
    e1, e2, e3 = b - a, c - a, d - a
    vol = abs(np.linalg.det(np.stack([e1, e2, e3]))) / 6.0
    pts, wts = [], []
    for iu in range(n):
        for iv in range(n):
            for iw in range(n):
                xi = u[iu]
                eta = u[iv] * (1.0 - u[iu])
                zeta = u[iw] * (1.0 - u[iu]) * (1.0 - u[iv])
                pts.append(a + xi * e1 + eta * e2 + zeta * e3)
                wts.append(w[iu] * w[iv] * w[iw] * (1.0 - u[iu]) ** 2 * (1.0 - u[iv]) * 6.0 * vol)
    return np.array(pts), np.array(wts)
