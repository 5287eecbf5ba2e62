"""Pins of the DG oracle (Scheme 3, Sec. 2.4: BR2 vector Laplacian with a
stabilised equal-order pressure coupling) against what the mathematics fixes
independently of the oracle's element-by-element assembly:

* exact reproduction of a divergence-free polynomial velocity of degree k and
  a pressure of degree k (the scheme is consistent, and the exact solution
  lies in the discrete space);
* symmetry, the constant pressure as the only kernel of all-Dirichlet
  problems, no kernel with a Neumann side;
* saddle-point inertia: exactly as many negative eigenvalues as pressure
  unknowns (the sign reading of the pressure stabilisation);
* the velocity energy u^T A u equals the face-based BR2 form
  sum_T |grad u|^2 - 2 sum_F int {grad u} . n [u] + eta sum_F sum_T ||L_FT([u])||^2
  (Dirichlet faces with [u] = 2 u and -int (grad u . n) [u]) computed from the
  lifting coefficients directly;
* h-convergence orders on smooth data (velocity k+1, pressure about k);
* the restriction equals the L2 projections from independently built bases
  and the coarse operators are the Galerkin products with them.
"""
import numpy as np
import pytest

from oracle.basis import dim_P
from oracle.dg import DG
from synthetic import tri_mesh, quad_mesh, hex_mesh, fields

MESHES = {
    "tri3-neumann": lambda: tri_mesh(3, jitter=0.2, seed=1, neumann_sides=(1,)),
    "quad3": lambda: quad_mesh(3, 3, jitter=0.15, seed=2),
    "hex2": lambda: hex_mesh(2, jitter=0.1, seed=2),
}


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("k", [1, 2])
def test_dg_polynomial_solution_reproduced(name, k):
    mesh = MESHES[name]()
    if mesh.dim == 3 and k == 2:
        pytest.skip("kept small")
    h = DG(mesh, k)
    fld = fields.PolyStokes(mesh.dim, k, k, np.random.default_rng(3 + k))
    x = h.direct_solve(h.assemble_rhs(*h.data_values(fld)))
    e = h.errors(fld, x)
    assert e["u"] < 1e-10 and e["gu"] < 1e-9 and e["p"] < 1e-9, e


@pytest.mark.parametrize("neumann", [False, True])
def test_dg_symmetry_kernel_inertia(neumann):
    mesh = tri_mesh(3, jitter=0.2, seed=4, neumann_sides=(1,) if neumann else ())
    h = DG(mesh, 1)
    S = h.S.toarray()
    assert np.abs(S - S.T).max() <= 1e-14 * np.abs(S).max()
    ev = np.linalg.eigvalsh(S)
    tol = 1e-12 * np.abs(ev).max()
    n_p = mesh.n_elem * h.nE
    if neumann:
        assert h.null_vector() is None
        assert (np.abs(ev) > tol).all()
        assert (ev < -tol).sum() == n_p
    else:
        n = h.null_vector()
        assert np.abs(S @ n).max() <= 1e-14 * np.abs(S).max()
        assert (np.abs(ev) <= tol).sum() == 1
        assert (ev < -tol).sum() == n_p - 1


def test_dg_velocity_energy_equals_face_based_br2_form():
    mesh = tri_mesh(3, 2, jitter=0.2, seed=6, neumann_sides=(1,))
    k = 2
    h = DG(mesh, k)
    d, nE, nb = h.d, h.nE, h.nb
    rng = np.random.default_rng(5)
    x = np.zeros(h.ndof)
    for T in range(mesh.n_elem):  # velocity only (one component: the BR2 form acts componentwise)
        x[T * nb:T * nb + nE] = rng.standard_normal(nE)
    e1 = x @ (h.S @ x)
    e2 = 0.0
    for T in range(mesh.n_elem):
        X, W = h.elems[T].rule(h.q)
        _, g = h.ebases[T].eval_grad(X)
        gu = np.einsum("qad,a->qd", g, x[T * nb:T * nb + nE])
        e2 += W @ np.sum(gu ** 2, axis=1)
    for F in range(mesh.n_face):
        T1, T2 = (int(t) for t in mesh.face_elem[F])
        bc = mesh.face_bc[F]
        if bc == 2:
            continue
        n1, X, W = h._face_side(F, T1)
        v1, g1 = h.ebases[T1].eval_grad(X)
        u1 = v1 @ x[T1 * nb:T1 * nb + nE]
        du1 = np.einsum("qad,a,d->q", g1, x[T1 * nb:T1 * nb + nE], n1)
        eta = h._eta(F)
        if T2 < 0:  # Dirichlet, zero datum: [u] = 2 u
            jump = 2.0 * u1
            e2 -= W @ (du1 * jump)
            L = 0.5 * np.einsum("q,q,qa,c->ca", W, jump, v1, n1)
            e2 += eta * np.sum(L ** 2)
            continue
        v2, g2 = h.ebases[T2].eval_grad(X)
        u2 = v2 @ x[T2 * nb:T2 * nb + nE]
        du2 = np.einsum("qad,a,d->q", g2, x[T2 * nb:T2 * nb + nE], n1)
        jump = u1 - u2
        e2 -= 2.0 * (W @ (0.5 * (du1 + du2) * jump))
        for vS, nS, s in ((v1, n1, 1.0), (v2, -n1, -1.0)):
            L = 0.5 * np.einsum("q,q,qa,c->ca", W, s * jump, vS, nS)
            e2 += eta * np.sum(L ** 2)
    assert abs(e1 - e2) <= 1e-12 * abs(e2), (e1, e2)


@pytest.mark.parametrize("k", [1, 2])
def test_dg_convergence_orders(k):
    fld = fields.TrigStokes2D()
    errs = []
    for n in (4, 8):
        h = DG(tri_mesh(n, jitter=0.2, seed=1, neumann_sides=(1,)), k)
        errs.append(h.errors(fld, h.direct_solve(h.assemble_rhs(*h.data_values(fld)))))
    rate = {key: np.log2(errs[0][key] / errs[1][key]) for key in ("u", "gu", "p")}
    assert rate["u"] > k + 0.6 and rate["gu"] > k - 0.3 and rate["p"] > k - 0.4, rate


def test_dg_pmg_transfers_keep_the_kernel_and_fgmres_converges():
    """p-multilevel hierarchy of the DG operator (Sec. 4.2 with element blocks:
    every velocity component and the pressure truncated): the transfers keep
    the constant-pressure kernel, and FGMRES with the element block-Jacobi
    smoothed V-cycle reaches the direct solution."""
    from oracle.pmg import PMG, fgmres
    mesh = quad_mesh(6, 5, jitter=0.15, seed=2)
    h = DG(mesh, 2)
    pmg = PMG(h, [2, 1, 0])
    n = h.null_vector()
    for l, R in enumerate(pmg.R):
        n = R @ n
        Sc = pmg.levels[l + 1].S
        assert np.abs(Sc @ n).max() <= 1e-13 * abs(Sc).max()
    assert abs(abs(n @ pmg.null) / np.linalg.norm(n) - 1.0) < 1e-14
    rhs = h.assemble_rhs(*h.data_values(fields.TrigStokes2D()))
    xd = h.direct_solve(rhs)
    x, its, rr = fgmres(h.S, pmg.apply, rhs, rtol=1e-10, null=h.null_vector(), maxit=300)
    assert rr <= 1e-10
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-6  # kappa(S) rtol


def test_dg_restriction_is_the_l2_projection_and_galerkin():
    """The DG restriction (Sec. 4.2 patched element by element: every velocity
    component and the pressure) equals the L2 projections int phi_i^{l+1}
    phi_j^l computed from independently built bases of each degree, and the
    hierarchy's coarse operators are R S R^T with those projections."""
    from oracle.basis import element_basis
    from oracle.pmg import PMG, restriction
    mesh = tri_mesh(2, jitter=0.2, seed=3)
    h = DG(mesh, 3)
    d = mesh.dim

    def explicit(k_f, k_c):
        nEf, nEc = dim_P(d, k_f), dim_P(d, k_c)
        R = np.zeros((mesh.n_elem * (d + 1) * nEc, mesh.n_elem * (d + 1) * nEf))
        for e in h.elems:
            Bf, Bc = element_basis(e, k_f), element_basis(e, k_c)
            X, W = e.rule(2 * k_f + 2)
            I = Bc.eval(X).T @ (W[:, None] * Bf.eval(X))
            for c in range(d + 1):
                r0, c0 = (e.id * (d + 1) + c) * nEc, (e.id * (d + 1) + c) * nEf
                R[r0:r0 + nEc, c0:c0 + nEf] = I
        return R

    for k_f, k_c in ((3, 2), (3, 0), (2, 1)):
        R = restriction(mesh, d, k_f, k_c, "dg").toarray()
        assert np.abs(R - explicit(k_f, k_c)).max() < 1e-13
    pmg = PMG(h, [3, 2, 1, 0], coarse="lu")
    S = h.S.toarray()
    Sl = S
    for l in range(1, 4):
        Rx = explicit(pmg.degrees[l - 1], pmg.degrees[l])
        Sl = Rx @ Sl @ Rx.T
        assert np.abs(pmg.levels[l].S.toarray() - Sl).max() < 1e-13 * np.abs(S).max()
