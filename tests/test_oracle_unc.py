"""Pins of the oracle's uncondensed HHO-dp formulation (Sec. 5.4's reference
point: no element unknown eliminated) and of its p-multilevel hierarchy,
against what the mathematics fixes independently of the formulation's own
code:

* the uncondensed system (face blocks, then one [U_T | P_T] block per element)
  has the same solution as velocity-only condensation followed by
  back-substitution, element by element;
* it is symmetric and its kernel is exactly the constant pressure placed on
  every element's mean-pressure slot (all-Dirichlet);
* its restriction equals the L2 projections int psi_i^{l+1} psi_j^l computed
  from independently built bases on every face and every element (velocity
  components and pressure each truncated), and the Galerkin coarse operators
  equal R S R^T with those projections (Sec. 4.2);
* the transfers keep the kernel, and FGMRES with the V-cycle (block ILU(0)
  smoother, the paper's smoother) reaches the direct solution.
"""
import numpy as np
import pytest

from oracle.basis import dim_P, element_basis, face_basis
from oracle.hho import HHO
from oracle.pmg import PMG, fgmres, restriction
from synthetic import tri_mesh, quad_mesh, fields


def _explicit_restriction_unc(h, k_f, k_c):
    m, d = h.mesh, h.d
    nFf, nFc = dim_P(d - 1, k_f), dim_P(d - 1, k_c)
    nEf, nEc = dim_P(d, k_f), dim_P(d, k_c)
    nf, ne = m.n_face, m.n_elem
    R = np.zeros((nf * d * nFc + ne * (d + 1) * nEc, nf * d * nFf + ne * (d + 1) * nEf))
    for F in h.faces:
        Bf, Bc = face_basis(F, k_f), face_basis(F, k_c)
        X, W = F.rule(2 * k_f + 2)
        I = Bc.eval(X).T @ (W[:, None] * Bf.eval(X))
        for c in range(d):
            R[np.ix_(F.id * d * nFc + c * nFc + np.arange(nFc), F.id * d * nFf + c * nFf + np.arange(nFf))] = I
    for e in h.elems:
        Bf, Bc = element_basis(e, k_f), element_basis(e, k_c)
        X, W = e.rule(2 * k_f + 2)
        I = (Bc.eval(X).T @ (W[:, None] * Bf.eval(X)))[:nEc, :nEf]
        for c in range(d + 1):
            r0 = nf * d * nFc + e.id * (d + 1) * nEc + c * nEc
            c0 = nf * d * nFf + e.id * (d + 1) * nEf + c * nEf
            R[np.ix_(r0 + np.arange(nEc), c0 + np.arange(nEf))] = I
    return R


@pytest.mark.parametrize("neumann", [False, True])
def test_uncondensed_equals_vcond_solution(neumann):
    m = tri_mesh(4, 3, jitter=0.2, seed=9, neumann_sides=(1,) if neumann else ())
    k = 2
    fld = fields.TrigStokes2D()
    hu, hv = HHO(m, k, "unc"), HHO(m, k, "v")
    data = hu.data_values(fld)
    lu = hu.recover(hu.direct_solve(hu.assemble_rhs(*data)))
    lv = hv.recover(hv.direct_solve(hv.assemble_rhs(*data)))
    for a, b in zip(lu, lv):
        if not neumann:  # the pressures are fixed up to a constant: compare modulo the mean
            pa, pb = a[hu.local[0].nvec:], b[hv.local[0].nvec:]
            a, b = a.copy(), b.copy()
            a[hu.local[0].nvec] -= pa[0]
            b[hv.local[0].nvec] -= pb[0]
        assert np.abs(a - b).max() <= 1e-9 * np.abs(b).max()


def test_uncondensed_symmetric_with_constant_pressure_kernel():
    m = tri_mesh(3, jitter=0.2, seed=4)
    h = HHO(m, 1, "unc")
    S = h.S.toarray()
    assert np.abs(S - S.T).max() <= 1e-14 * np.abs(S).max()
    n = h.null_vector()
    assert np.abs(S @ n).max() <= 1e-14 * np.abs(S).max()
    sv = np.linalg.svd(S, compute_uv=False)
    assert sv[-1] / sv[0] < 1e-15 and sv[-2] / sv[0] > 1e-9


def test_uncondensed_restriction_and_galerkin():
    h = HHO(tri_mesh(2, jitter=0.2, seed=3), 3, "unc")
    S = h.S.toarray()
    for k_f, k_c in ((3, 2), (3, 1), (2, 0)):
        R = restriction(h.mesh, 2, k_f, k_c, "unc").toarray()
        assert np.abs(R - _explicit_restriction_unc(h, k_f, k_c)).max() < 1e-13
    pmg = PMG(h, [3, 2, 1, 0], coarse="lu")
    Sl = S
    for l in range(1, 4):
        Rx = _explicit_restriction_unc(h, pmg.degrees[l - 1], pmg.degrees[l])
        Sl = Rx @ Sl @ Rx.T
        assert np.abs(pmg.levels[l].S.toarray() - Sl).max() < 1e-13 * np.abs(S).max()


def test_uncondensed_pmg_keeps_kernel_and_converges():
    m = quad_mesh(5, 4, jitter=0.15, seed=2)
    k = 3
    h = HHO(m, k, "unc")
    pmg = PMG(h, [3, 2, 1, 0], smoother="ilu")
    n = h.null_vector()
    for l, R in enumerate(pmg.R):
        n = R @ n
        Sc = pmg.levels[l + 1].S
        assert np.abs(Sc @ n).max() <= 1e-13 * abs(Sc).max()
    assert abs(abs(n @ pmg.null) / np.linalg.norm(n) - 1.0) < 1e-14
    rhs = h.assemble_rhs(*h.data_values(fields.TrigStokes2D()))
    xd = h.direct_solve(rhs)
    x, its, rr = fgmres(h.S, pmg.apply, rhs, rtol=1e-10, null=h.null_vector())
    assert rr <= 1e-10 and its <= 30
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-7
