"""Pins of the oracle's quadrature and hierarchical orthonormal bases (Sec. 2.1, Sec. 4.2)."""
from math import factorial

import numpy as np
import pytest

from oracle.basis import dim_P, legendre, multi_indices, element_basis, face_basis
from oracle.geometry import mesh_geometry
from oracle.quadrature import segment_rule, triangle_rule, tet_rule
from synthetic import quad_mesh, tri_mesh, hex_mesh


@pytest.mark.parametrize("p", range(0, 13))
def test_simplex_rules_exact_on_monomials(p):
    # closed forms on reference simplices: int x^a y^b = a! b! / (a+b+2)!, etc.
    X, W = segment_rule([0.0], [1.0], p)
    assert abs(W @ X[:, 0] ** p - 1.0 / (p + 1)) < 1e-14
    X, W = triangle_rule([0.0, 0.0], [1.0, 0.0], [0.0, 1.0], p)
    for a in range(p + 1):
        b = p - a
        exact = factorial(a) * factorial(b) / factorial(a + b + 2)
        assert abs(W @ (X[:, 0] ** a * X[:, 1] ** b) - exact) < 1e-14
    if p <= 8:
        X, W = tet_rule([0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], p)
        for a in range(p + 1):
            for b in range(p + 1 - a):
                c = p - a - b
                exact = factorial(a) * factorial(b) * factorial(c) / factorial(a + b + c + 3)
                assert abs(W @ (X[:, 0] ** a * X[:, 1] ** b * X[:, 2] ** c) - exact) < 1e-14


def test_element_measures_match_shoelace():
    m = quad_mesh(4, jitter=0.25, seed=11)
    elems, _ = mesh_geometry(m)
    for e in elems:
        P = np.array([m.xyz[v] for v in _ccw_vertices(m, e.id)])
        shoelace = 0.5 * abs(np.dot(P[:, 0], np.roll(P[:, 1], -1)) - np.dot(P[:, 1], np.roll(P[:, 0], -1)))
        assert abs(e.meas - shoelace) < 1e-14


def _ccw_vertices(m, t):
    # quad faces are (bottom, right, top, left) with vertices (v00,v10),(v10,v11),(v01,v11),(v00,v01)
    b, r, tp, l = m.faces_of(t)
    v00, v10 = m.verts_of_face(b)
    v11 = m.verts_of_face(r)[1]
    v01 = m.verts_of_face(tp)[0]
    return [v00, v10, v11, v01]


def test_legendre_matches_library():
    x = np.linspace(-1, 1, 37)
    P, D = legendre(8, x)
    for n in range(9):
        c = np.zeros(n + 1)
        c[n] = 1.0
        assert np.allclose(P[n], np.polynomial.legendre.legval(x, c), atol=1e-14)
        assert np.allclose(D[n], np.polynomial.legendre.legval(x, np.polynomial.legendre.legder(c)), atol=1e-12)


def test_multi_index_counts():
    for nv in (1, 2, 3):
        for K in range(7):
            idx = multi_indices(nv, K)
            assert len(idx) == dim_P(nv, K)
            assert len(set(idx)) == len(idx)
            degs = [sum(a) for a in idx]
            assert degs == sorted(degs)


@pytest.mark.parametrize("mesh", [quad_mesh(3, jitter=0.3, seed=2), tri_mesh(3, jitter=0.3, seed=2),
                                  hex_mesh(2, jitter=0.3, seed=2)], ids=["quad", "tri", "hex"])
def test_bases_orthonormal_and_hierarchical(mesh):
    elems, faces = mesh_geometry(mesh)
    K = 4 if mesh.dim == 2 else 3
    rng = np.random.default_rng(0)
    for e in elems[:4]:
        B = element_basis(e, K)
        X, W = e.rule(2 * K + 2)
        V = B.eval(X)
        assert np.abs(V.T @ (W[:, None] * V) - np.eye(B.n)).max() < 1e-13
        # first basis function is the constant 1/sqrt|T|
        assert np.allclose(V[:, 0], 1.0 / np.sqrt(e.meas), rtol=1e-13)
        # hierarchy: the first dim P^l functions reproduce any polynomial of degree l
        for l in range(K + 1):
            n = dim_P(mesh.dim, l)
            coef = rng.standard_normal(len(multi_indices(mesh.dim, l)))
            vals = sum(c * np.prod(X ** np.array(a), axis=1) for c, a in zip(coef, multi_indices(mesh.dim, l)))
            proj = V[:, :n] @ (V[:, :n].T @ (W * vals))
            assert np.abs(proj - vals).max() < 1e-9 * max(1.0, np.abs(vals).max())
    for F in faces[:6]:
        B = face_basis(F, K)
        X, W = F.rule(2 * K + 2)
        V = B.eval(X)
        assert np.abs(V.T @ (W[:, None] * V) - np.eye(B.n)).max() < 1e-13


@pytest.mark.parametrize("mk", [lambda: tri_mesh(5, 4, jitter=0.25, seed=2),
                                lambda: quad_mesh(4, jitter=0.25, seed=3),
                                lambda: hex_mesh(3, jitter=0.15, seed=4)])
def test_closed_elements_and_outward_normals(mk):
    """Each element is closed (sum over its faces of |F| n_TF = 0, the
    divergence theorem for a constant field), n_TF is a unit vector pointing
    away from x_T, |T| = (1/d) sum_F |F| x_F . n_TF (the divergence theorem for
    the field x on planar faces), and the element measures tile the unit domain."""
    m = mk()
    elems, faces = mesh_geometry(m)
    d = m.dim
    total = 0.0
    for e in elems:
        s = sum(F.meas * n for F, n in zip(e.faces, e.nTF))
        assert np.abs(s).max() < 1e-13
        for F, n in zip(e.faces, e.nTF):
            assert float(n @ (F.xF - e.xT)) > 0.0
            assert abs(np.linalg.norm(n) - 1.0) < 1e-14
        # divergence theorem for the field x / d: |T| = (1/d) sum_F |F| (x_F . n_TF) on planar faces
        vol = sum(F.meas * float(F.xF @ n) for F, n in zip(e.faces, e.nTF)) / d
        assert abs(vol - e.meas) < 1e-13
        total += e.meas
    assert abs(total - 1.0) < 1e-13


def _monomials(dim, deg):
    if dim == 2:
        return [(a, m - a) for m in range(deg + 1) for a in range(m + 1)]
    return [(a, b, m - a - b) for m in range(deg + 1) for a in range(m + 1) for b in range(m - a + 1)]


def _segment_integral(P0, P1, g, deg):
    """int over the segment P0-P1 of g (a polynomial of degree deg), Gauss-Legendre from numpy."""
    t, w = np.polynomial.legendre.leggauss(deg // 2 + 2)
    t, w = 0.5 * (t + 1.0), 0.5 * w
    X = P0[None, :] + t[:, None] * (P1 - P0)[None, :]
    return float(np.linalg.norm(P1 - P0) * (w @ g(X)))


def _triangle_integral(P0, P1, P2, g, deg):
    """int over a 3D triangle of g (degree deg), collapsed square (Duffy) with numpy Gauss-Legendre."""
    t, w = np.polynomial.legendre.leggauss(deg // 2 + 3)
    t, w = 0.5 * (t + 1.0), 0.5 * w
    u, v = np.meshgrid(t, t, indexing="ij")
    wu = np.outer(w, w)
    X = P0 + u.ravel()[:, None] * (P1 - P0) + (u * v).ravel()[:, None] * (P2 - P1)
    jac = np.linalg.norm(np.cross(P1 - P0, P2 - P1))
    return float(jac * np.sum(wu.ravel() * u.ravel() * g(X)))


def _polygon_face_integral(V, g, deg):
    return sum(_triangle_integral(V[0], V[i], V[i + 1], g, deg) for i in range(1, len(V) - 1))


@pytest.mark.parametrize("mk", [lambda: tri_mesh(3, jitter=0.3, seed=2), lambda: quad_mesh(3, jitter=0.3, seed=2),
                                lambda: hex_mesh(2, jitter=0.3, seed=2)], ids=["tri", "quad", "hex"])
def test_element_and_face_rules_exact_to_their_order(mk):
    """ElemGeom.rule(p) and FaceGeom.rule(p) integrate every monomial of degree
    <= p exactly.  Reference values from the mesh's vertices alone: element
    integrals by the divergence theorem (int_T x^a y^b.. = int_dT x^(a+1) y^b.. /
    (a+1) n_x, outward normals from the vertex average), boundary and face
    integrals by numpy's Gauss-Legendre on segments and on collapsed triangles
    of a fan of every planar face."""
    mesh = mk()
    d = mesh.dim
    elems, faces = mesh_geometry(mesh)
    for p in ((1, 4, 7) if d == 2 else (1, 3, 5)):
        for t in range(min(mesh.n_elem, 5)):
            e = elems[t]
            fs = mesh.faces_of(t)
            c = mesh.xyz[np.unique(np.concatenate([mesh.verts_of_face(int(F)) for F in fs]))].mean(axis=0)
            h = e.hT
            X, W = e.rule(p)
            for mono in _monomials(d, p):
                f = lambda Y, m=mono: np.prod(((Y - c) / h) ** np.array(m), axis=1)
                G = lambda Y, m=mono: ((Y[:, 0] - c[0]) / h) ** (m[0] + 1) * h / (m[0] + 1) * np.prod(
                    ((Y[:, 1:] - c[1:]) / h) ** np.array(m[1:]), axis=1)
                exact = 0.0
                for F in fs:
                    V = mesh.xyz[mesh.verts_of_face(int(F))]
                    if d == 2:
                        tan = V[1] - V[0]
                        n = np.array([tan[1], -tan[0]]) / np.linalg.norm(tan)
                        n = n if n @ (V.mean(axis=0) - c) > 0 else -n
                        exact += n[0] * _segment_integral(V[0], V[1], G, sum(mono) + 1)
                    else:
                        n = np.cross(V[1] - V[0], V[2] - V[0])
                        n /= np.linalg.norm(n)
                        n = n if n @ (V.mean(axis=0) - c) > 0 else -n
                        exact += n[0] * _polygon_face_integral(V, G, sum(mono) + 1)
                assert abs(W @ f(X) - exact) <= 1e-12 * e.meas, (t, p, mono)
        for F in faces[:6]:
            V = F.V
            c = V.mean(axis=0)
            X, W = F.rule(p)
            for mono in _monomials(d, p):
                f = lambda Y, m=mono: np.prod(((Y - c) / F.hF) ** np.array(m), axis=1)
                exact = (_segment_integral(V[0], V[1], f, sum(mono)) if d == 2
                         else _polygon_face_integral(V, f, sum(mono)))
                assert abs(W @ f(X) - exact) <= 1e-12 * F.meas, (F.id, p, mono)
