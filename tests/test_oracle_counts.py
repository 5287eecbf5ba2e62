"""Sizes and non-zero counts of the HHO-hp, DG and uncondensed systems.

* Counted from the mesh topology alone (blocks each scheme couples: a face
  with the faces of its elements for HHO-hp; an element with itself and its
  neighbours across interior faces for DG, velocity components uncoupled), the
  DOFs and MNZs equal the values the paper prints for its 128x128 quadrilateral
  and 32768-triangle meshes (Sec. 5.3, Tables 2 and 3; stored in
  tests/golden/paper_counts_schemes.txt).
* On small meshes the oracle's assembled matrices have exactly that block
  structure: every counted block holds a non-zero and nothing else does.
"""
import os

import numpy as np
import pytest

from oracle.basis import dim_P
from oracle.dg import DG
from oracle.hho import HHO
from oracle.hho_hp import HHOhp
from synthetic import quad_mesh, tri_mesh

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _counts(mesh, k, scheme):
    d = mesh.dim
    nF, nE = dim_P(d - 1, k), dim_P(d, k)
    fe = mesh.face_elem
    nFT = np.diff(mesh.elem_face_ptr)
    TF = (fe >= 0).sum(1)
    if scheme == "dg":  # element blocks [u_T (d components) | p_T]: d + 2d + 1 non-zero nE x nE sub-blocks each
        inner = fe[(fe[:, 0] >= 0) & (fe[:, 1] >= 0)]
        nbr = 1 + np.bincount(inner.ravel(), minlength=mesh.n_elem)
        return mesh.n_elem * (d + 1) * nE, int((nbr * (3 * d + 1) * nE * nE).sum())
    if scheme == "hp":  # full face blocks of (d+1) nF: the face with every face of its elements
        nbr = np.array([sum(nFT[t] for t in fe[f] if t >= 0) - (TF[f] - 1) for f in range(mesh.n_face)])
        return mesh.n_face * (d + 1) * nF, int((nbr * ((d + 1) * nF) ** 2).sum())
    return mesh.n_face * d * nF + mesh.n_elem * (d + 1) * nE, None


def test_counts_match_paper_tables():
    meshes = {"quad128": quad_mesh(128), "tri128": tri_mesh(128)}
    for line in open(os.path.join(GOLDEN, "paper_counts_schemes.txt")):
        if line.startswith("#") or not line.strip():
            continue
        mesh, k, scheme, qty, val = line.split()
        dofs, mnz = _counts(meshes[mesh], int(k), scheme)
        got = dofs if qty == "dofs" else mnz
        assert float(f"{got:.3g}") == pytest.approx(float(val), rel=1e-12) or \
            abs(got - float(val)) <= 0.005 * float(val), (line, got)


def _pattern_size(S, sub):
    """Entries of the sub x sub tiles of S that hold a non-zero."""
    C = S.tocoo()
    nz = np.abs(C.data) > 0.0
    tiles = set(zip((C.row[nz] // sub).tolist(), (C.col[nz] // sub).tolist()))
    return len(tiles) * sub * sub


@pytest.mark.parametrize("k", [1, 2])
def test_dg_pattern_matches_counts(k):
    m = tri_mesh(4, 3, jitter=0.2, seed=1, neumann_sides=(1,))
    h = DG(m, k)
    dofs, mnz = _counts(m, k, "dg")
    assert h.ndof == dofs and _pattern_size(h.S, h.nE) == mnz


def test_hp_pattern_matches_counts():
    m = quad_mesh(3, 4, jitter=0.2, seed=2)
    h = HHOhp(m, 1)
    dofs, mnz = _counts(m, 1, "hp")
    assert h.ndof == dofs and _pattern_size(h.S, h.b) == mnz


def test_uncondensed_size_matches_counts():
    m = tri_mesh(3, jitter=0.2, seed=4)
    assert HHO(m, 2, "unc").ndof == _counts(m, 2, "unc")[0]
