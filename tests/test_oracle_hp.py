"""Pins of the HHO-hp oracle (Scheme 2, Sec. 2.3.2) against what the paper and
the mathematics fix, independent of the oracle's own formulas:

* exact reproduction of a polynomial Stokes solution (u in P^{k+1}
  divergence free, p in P^k): the scheme is consistent for it, so the discrete
  velocity reconstruction, its gradient and the element pressure equal the
  exact fields up to rounding (2D triangles with a Neumann side, quadrilaterals,
  hexahedra);
* the element velocity is divergence free pointwise for any data (the
  property the paper states for Scheme 2);
* the condensed operator is symmetric, has exactly the constant hybrid
  pressure as kernel for all-Dirichlet problems and none with a Neumann side;
* static condensation and back-substitution give the solution of the full
  (uncondensed) system;
* h-convergence orders on smooth data (velocity k+2, its gradient and the
  pressure k+1, up to the pre-asymptotic range of 4x4 -> 8x8 meshes);
* p-multilevel transfers: the restriction maps the fine kernel onto the
  coarse one, the Galerkin coarse operators keep it, and FGMRES with the
  V-cycle reaches the direct solution; the restriction equals the L2
  projections from independently built face bases (face pressure included)
  and the coarse operators the Galerkin products with them.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.hho_hp import HHOhp
from oracle.pmg import PMG, fgmres, restriction
from synthetic import tri_mesh, quad_mesh, hex_mesh, fields

MESHES = {
    "tri4-neumann": lambda: tri_mesh(4, jitter=0.2, seed=1, neumann_sides=(1,)),
    "tri4": lambda: tri_mesh(4, jitter=0.2, seed=1),
    "quad3": lambda: quad_mesh(3, 3, jitter=0.15, seed=2),
    "hex2": lambda: hex_mesh(2, jitter=0.1, seed=2),
}


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("k", [0, 1, 2])
def test_polynomial_solution_reproduced(name, k):
    mesh = MESHES[name]()
    if mesh.dim == 3 and k == 2:
        pytest.skip("kept small")
    h = HHOhp(mesh, k)
    fld = fields.PolyStokes(mesh.dim, k + 1, k, np.random.default_rng(3 + k))
    rhs = h.assemble_rhs(*h.data_values(fld))
    x = h.direct_solve(rhs)
    e = h.errors(fld, h.recover(x))
    # field sizes are O(1..10); rounding of the local solves gives ~1e-13..1e-12
    assert e["u"] < 1e-11 and e["gu"] < 1e-10 and e["p"] < 1e-10, e
    assert e["div"] < 1e-11, e


@pytest.mark.parametrize("name", ["tri4-neumann", "quad3", "hex2"])
def test_element_velocity_divergence_free(name):
    mesh = MESHES[name]()
    h = HHOhp(mesh, 2)
    fld = fields.TrigStokes2D() if mesh.dim == 2 else fields.CurlStokes3D()
    rhs = h.assemble_rhs(*h.data_values(fld))
    e = h.errors(fld, h.recover(h.direct_solve(rhs)))
    assert e["u"] > 1e-6  # not a polynomial solution: the velocity error is genuine
    assert e["div"] < 1e-12, e


@pytest.mark.parametrize("neumann", [False, True])
def test_symmetry_and_kernel(neumann):
    mesh = tri_mesh(3, jitter=0.2, seed=4, neumann_sides=(1,) if neumann else ())
    h = HHOhp(mesh, 1)
    S = h.S.toarray()
    assert np.abs(S - S.T).max() <= 1e-14 * np.abs(S).max()
    sv = np.linalg.svd(S, compute_uv=False)
    gap = sv[-1] / sv[0]
    if neumann:
        assert h.null_vector() is None and gap > 1e-8
    else:
        n = h.null_vector()
        assert np.abs(S @ n).max() <= 1e-14 * np.abs(S).max()
        assert gap < 1e-15 and sv[-2] / sv[0] > 1e-8  # a one-dimensional kernel


def test_condensation_matches_full_system():
    mesh = quad_mesh(3, 2, jitter=0.15, seed=6, neumann_sides=(1,))
    h = HHOhp(mesh, 2)
    fld = fields.TrigStokes2D()
    data = h.data_values(fld)
    rhs = h.assemble_rhs(*data)
    loc = h.recover(h.direct_solve(rhs))
    K, b, null = h.uncondensed(*data)
    assert null is None
    xf = np.linalg.solve(K.toarray(), b)
    for t, L in enumerate(h.local):
        elim, keep = L.split()
        xt = np.zeros(L.K.shape[0])
        xt[keep] = xf[h.global_kept(t)]
        base = mesh.n_face * h.b + t * (h.d * h.nV + h.nE)
        xt[elim] = xf[base:base + len(elim)]
        assert np.abs(loc[t] - xt).max() <= 1e-10 * np.abs(xf).max()


@pytest.mark.parametrize("k", [1, 2])
def test_convergence_orders(k):
    fld = fields.TrigStokes2D()
    errs = []
    for n in (4, 8):
        h = HHOhp(tri_mesh(n, jitter=0.2, seed=1), k)
        rhs = h.assemble_rhs(*h.data_values(fld))
        errs.append(h.errors(fld, h.recover(h.direct_solve(rhs))))
    rate = {key: np.log2(errs[0][key] / errs[1][key]) for key in ("u", "gu", "p")}
    assert rate["u"] > k + 1.5 and rate["gu"] > k + 0.7 and rate["p"] > k + 0.7, rate


def test_pmg_transfers_keep_the_kernel_and_fgmres_converges():
    mesh = tri_mesh(4, jitter=0.2, seed=1)
    k = 3
    h = HHOhp(mesh, k)
    degrees = [3, 2, 1, 0]
    pmg = PMG(h, degrees)
    n = h.null_vector()
    for l, R in enumerate(pmg.R):
        n = R @ n
        Sc = pmg.levels[l + 1].S
        assert np.abs(Sc @ n).max() <= 1e-13 * abs(Sc).max()
        assert pmg.levels[l + 1].b == 3 * (degrees[l + 1] + 1)
    nc = pmg.null
    assert abs(abs(n @ nc) / np.linalg.norm(n) - 1.0) < 1e-14  # the coarse kernel is the restricted one
    # R R^T = I (selection) and R S R^T is the leading sub-block of every face block pair
    R = restriction(mesh, 2, 3, 2, "hp")
    assert abs(R @ R.T - sp.identity(R.shape[0])).max() == 0.0
    fld = fields.TrigStokes2D()
    rhs = h.assemble_rhs(*h.data_values(fld))
    xd = h.direct_solve(rhs)
    x, its, rr = fgmres(h.S, pmg.apply, rhs, rtol=1e-10, null=h.null_vector())
    assert rr <= 1e-10 and its < 40
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-6


def test_restriction_is_the_l2_projection_and_galerkin():
    """The HHO-hp restriction (every face component, the face pressure
    included, truncated on its own) equals the L2 projections
    int psi_i^{l+1} psi_j^l from independently built face bases, and the
    coarse operators are R S R^T with those projections."""
    from oracle.basis import dim_P, face_basis
    mesh = tri_mesh(2, jitter=0.2, seed=3)
    h = HHOhp(mesh, 3)
    d = mesh.dim

    def explicit(k_f, k_c):
        nFf, nFc = dim_P(d - 1, k_f), dim_P(d - 1, k_c)
        R = np.zeros((mesh.n_face * (d + 1) * nFc, mesh.n_face * (d + 1) * nFf))
        for F in h.faces:
            Bf, Bc = face_basis(F, k_f), face_basis(F, k_c)
            X, W = F.rule(2 * k_f + 2)
            I = Bc.eval(X).T @ (W[:, None] * Bf.eval(X))
            for c in range(d + 1):
                r0, c0 = (F.id * (d + 1) + c) * nFc, (F.id * (d + 1) + c) * nFf
                R[r0:r0 + nFc, c0:c0 + nFf] = I
        return R

    for k_f, k_c in ((3, 2), (3, 0), (2, 1)):
        assert np.abs(restriction(mesh, d, k_f, k_c, "hp").toarray() - explicit(k_f, k_c)).max() < 1e-13
    pmg = PMG(h, [3, 2, 1, 0], coarse="lu")
    S = h.S.toarray()
    Sl = S
    for l in range(1, 4):
        Rx = explicit(pmg.degrees[l - 1], pmg.degrees[l])
        Sl = Rx @ Sl @ Rx.T
        assert np.abs(pmg.levels[l].S.toarray() - Sl).max() < 1e-13 * np.abs(S).max()
