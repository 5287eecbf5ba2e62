"""Pins of the block ILU(0) oracle (oracle/ilu.py).

* the colouring is proper: faces sharing an element get different colours;
* on one element every block is coupled to every other, so ILU(0) drops
  nothing and its application is the exact solve;
* on any mesh the factors reproduce S on the block pattern, (L U)_ij = S_ij for
  every pattern block (the defining property of ILU(0));
* as the smoother preconditioner it beats block Jacobi on the velocity-pressure
  condensed system (FGMRES iterations of the V-cycle).
"""
import numpy as np
import pytest

from oracle.hho import HHO
from oracle.ilu import BlockILU, face_colors
from oracle.pmg import PMG, fgmres
from synthetic import Mesh, tri_mesh, quad_mesh, fields


def test_colouring_is_proper():
    for m in (tri_mesh(5, 4, jitter=0.2, seed=1), quad_mesh(4, 3, jitter=0.1, seed=2)):
        col = face_colors(m)
        for T in range(m.n_elem):
            fs = m.faces_of(T)
            assert len({int(col[F]) for F in fs}) == len(fs)


def _one_triangle():
    xyz = np.array([[0.0, 0.0], [1.0, 0.1], [0.2, 0.9]])
    return Mesh(dim=2, xyz=xyz, elem_face_ptr=np.array([0, 3]), elem_face=np.array([0, 1, 2]),
                face_vert_ptr=np.array([0, 2, 4, 6]), face_vert=np.array([0, 1, 1, 2, 2, 0]),
                face_elem=np.array([[0, -1], [0, -1], [0, -1]]), face_bc=np.array([2, 1, 1], dtype=np.int8),
                face_side=np.array([0, 1, 2], dtype=np.int8))


@pytest.mark.parametrize("cond", ["v", "vp"])
def test_single_element_is_exact(cond):
    """One element: every block couples to every other, ILU(0) drops nothing and equals LU."""
    m = _one_triangle()
    h = HHO(m, 2, cond)
    ilu = BlockILU(h.S, m, h.b, 1 if cond == "vp" else h.nE)
    v = np.random.default_rng(0).standard_normal(h.S.shape[0])
    z = ilu.apply(v)
    assert np.linalg.norm(h.S @ z - v) <= 1e-10 * np.linalg.norm(v)


@pytest.mark.parametrize("cond", ["v", "vp"])
def test_factors_reproduce_S_on_the_pattern(cond):
    m = tri_mesh(4, 3, jitter=0.2, seed=3, neumann_sides=(1,))
    h = HHO(m, 1, cond)
    ilu = BlockILU(h.S, m, h.b, 1 if cond == "vp" else h.nE)
    S = h.S.toarray()
    scale = np.abs(S).max()
    for i, row in ilu.pat.items():
        for j in row:
            assert np.abs(_lu_block(ilu, i, j) - S[ilu.sl(i), ilu.sl(j)]).max() <= 1e-10 * scale


def _lu_block(ilu, i, j):
    """(L U)_ij with L unit lower (strict part in blocks[(i,k)], k < i) and U upper."""
    rank = ilu.rank
    out = 0.0
    for k in ilu.pat[i]:
        if rank[k] <= rank[j] and (k, j) in ilu.blocks:
            if rank[k] < rank[i]:
                out = out + ilu.blocks[(i, k)] @ ilu.blocks[(k, j)]
            elif k == i:
                out = out + ilu.blocks[(i, j)]
    return out


def test_ilu_smoother_beats_block_jacobi_under_vp_condensation():
    m = tri_mesh(8, 8, jitter=0.2, seed=5, neumann_sides=(1,))
    h = HHO(m, 2, "vp")
    rhs = h.assemble_rhs(*h.data_values(fields.TrigStokes2D()))
    its = {}
    for sm in ("jacobi", "ilu"):
        pmg = PMG(h, [2, 1, 0], smoother=sm)
        _, it, rr = fgmres(h.S, pmg.apply, rhs, rtol=1e-8, null=h.null_vector())
        assert rr <= 1e-8
        its[sm] = it
    assert its["ilu"] < its["jacobi"], its
