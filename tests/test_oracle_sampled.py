"""Pin of the oracle's sampled residual rows (oracle/sampled.py): on meshes
small enough for the full oracle, the rows of b - S x at sampled faces and at
their elements' kept pressures, computed from the submesh around the faces,
equal the same rows of the fully assembled system (end of Sec. 4.1.2: the
condensed operator and right-hand side are sums of element contributions)."""
import numpy as np
import pytest

from oracle.hho import HHO
from oracle.sampled import residual_rows, sample_interior_faces
from synthetic import hex_mesh, tri_mesh, quad_mesh, fields


@pytest.mark.parametrize("mk,k,cond,fld", [
    (lambda: tri_mesh(6, 5, jitter=0.2, seed=3, neumann_sides=(1,)), 2, "v", fields.TrigStokes2D()),
    (lambda: quad_mesh(5, 4, jitter=0.15, seed=4), 3, "vp", fields.TrigStokes2D()),
    (lambda: hex_mesh(3, jitter=0.15, seed=2), 2, "vp", fields.CurlStokes3D()),
])
def test_sampled_rows_equal_full_system_rows(mk, k, cond, fld):
    mesh = mk()
    h = HHO(mesh, k, cond)
    b = h.assemble_rhs(*h.data_values(fld))
    x = np.random.default_rng(1).standard_normal(h.ndof)
    full = b - h.S @ x
    faces = sample_interior_faces(mesh, 7, seed=5)
    rows, r, bs = residual_rows(mesh, k, cond, fld, x, faces)
    assert len(rows) == len(set(rows.tolist()))
    scale = np.abs(full).max()
    assert np.abs(r - full[rows]).max() <= 1e-12 * scale
    assert np.abs(bs - b[rows]).max() <= 1e-12 * np.abs(b).max()
    # the rows include both elements of every sampled interior face
    nfb = mesh.n_face * h.b
    elem_rows = {int(q - nfb) // h.nP for q in rows if q >= nfb}
    for F in faces:
        for t in mesh.face_elem[F]:
            if t >= 0:
                assert int(t) in elem_rows
