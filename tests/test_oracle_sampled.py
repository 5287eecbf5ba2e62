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


@pytest.mark.parametrize("mk,k,fld", [
    (lambda: tri_mesh(6, 5, jitter=0.2, seed=3, neumann_sides=(1,)), 2, fields.TrigStokes2D()),
    (lambda: hex_mesh(3, jitter=0.15, seed=2), 1, fields.CurlStokes3D()),
])
def test_sampled_rows_hp(mk, k, fld):
    """The same pin for Scheme 2 (HHO-hp): face rows only, no element rows."""
    from oracle.hho_hp import HHOhp
    mesh = mk()
    h = HHOhp(mesh, k)
    b = h.assemble_rhs(*h.data_values(fld))
    x = np.random.default_rng(2).standard_normal(h.ndof)
    full = b - h.S @ x
    faces = sample_interior_faces(mesh, 7, seed=6)
    rows, r, bs = residual_rows(mesh, k, "hp", fld, x, faces)
    assert len(rows) == len(faces) * h.b and rows.max() < h.ndof
    assert np.abs(r - full[rows]).max() <= 1e-12 * np.abs(full).max()
    assert np.abs(bs - b[rows]).max() <= 1e-12 * np.abs(b).max()


def test_row_scale_bounds_element_perturbations():
    """The row scale of residual_rows bounds |b| + |S||x| and the change of the
    residual rows when every element Schur complement moves by eps times its
    largest entry (the tolerance of the full-size residual check)."""
    mesh = tri_mesh(6, 5, jitter=0.2, seed=3, neumann_sides=(1,))
    k, cond, fld = 2, "vp", fields.TrigStokes2D()
    h = HHO(mesh, k, cond)
    b = h.assemble_rhs(*h.data_values(fld))
    x = np.random.default_rng(1).standard_normal(h.ndof)
    faces = sample_interior_faces(mesh, 9, seed=2)
    rows, r, bs, sc = residual_rows(mesh, k, cond, fld, x, faces, with_scale=True)
    assert np.all(sc >= np.abs(bs) + (abs(h.S) @ np.abs(x))[rows] * (1 - 1e-12))
    eps = 1e-9
    rng = np.random.default_rng(7)
    rr, cc, vv = [], [], []
    for t, S in enumerate(h.S_T):
        g = h.global_kept(t)
        dS = eps * np.abs(S).max() * rng.uniform(-1, 1, S.shape)
        rr.append(np.repeat(g, len(g)))
        cc.append(np.tile(g, len(g)))
        vv.append(dS.ravel())
    import scipy.sparse as sp
    dS = sp.csr_matrix((np.concatenate(vv), (np.concatenate(rr), np.concatenate(cc))), shape=h.S.shape)
    assert np.all(np.abs((dS @ x)[rows]) <= eps * sc)


@pytest.mark.parametrize("mk,k,fld", [
    (lambda: tri_mesh(6, 5, jitter=0.2, seed=3, neumann_sides=(1,)), 2, fields.TrigStokes2D()),
    (lambda: quad_mesh(5, 4, jitter=0.15, seed=4), 3, fields.TrigStokes2D()),
    (lambda: hex_mesh(3, jitter=0.15, seed=2), 1, fields.CurlStokes3D()),
])
def test_sampled_rows_dg(mk, k, fld):
    """The DG scheme (Scheme 3): the element rows of sampled elements, from the
    submesh of those elements and their neighbours, equal the rows of the full
    oracle's b - S x, and the row scale bounds |b| + |S||x| on them."""
    from oracle.dg import DG
    from oracle.sampled import residual_rows_dg, sample_elements
    mesh = mk()
    h = DG(mesh, k)
    b = h.assemble_rhs(*h.data_values(fld))
    x = np.random.default_rng(3).standard_normal(h.ndof)
    full = b - h.S @ x
    sample = sample_elements(mesh, 5, seed=7)
    rows, r, bs, sc = residual_rows_dg(mesh, k, fld, x, sample, with_scale=True)
    assert len(rows) == len(sample) * h.nb and len(set(rows.tolist())) == len(rows)
    assert np.abs(r - full[rows]).max() <= 1e-12 * np.abs(full).max()
    assert np.abs(bs - b[rows]).max() <= 1e-12 * np.abs(b).max()
    bound = np.abs(b[rows]) + (abs(h.S) @ np.abs(x))[rows]
    assert (sc >= bound * (1 - 1e-12)).all()
