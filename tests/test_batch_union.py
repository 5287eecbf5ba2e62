"""Union meshes of independent problems (the batched workload's input).

The batched solver relies on the union of problems being a block-diagonal
system whose blocks are the problems' own systems: the HHO discretisation is
translation invariant and no face couples two problems.  Pinned here with the
oracle: the condensed operator and right-hand side of a union equal those of
its problems assembled alone, block by block.
"""
import numpy as np
import pytest

from oracle.hho import HHO
from synthetic import quad_mesh, tri_mesh
from synthetic.batch import BatchField, TrigForcing, batch_problems, group_by_degree, union_mesh, slot_shift


def _meshes():
    return [tri_mesh(3, 2, jitter=0.2, seed=1, neumann_sides=(1,)), quad_mesh(2, 3, jitter=0.15, seed=2),
            tri_mesh(2, 2, jitter=0.1, seed=3)]


def test_union_offsets_and_no_coupling():
    ms = _meshes()
    m, fo, eo, sh = union_mesh(ms, per_row=2)
    assert fo[-1] == m.n_face and eo[-1] == m.n_elem
    assert np.array_equal(np.diff(fo), [x.n_face for x in ms])
    assert np.array_equal(np.diff(eo), [x.n_elem for x in ms])
    for p, mp in enumerate(ms):
        F = np.arange(fo[p], fo[p + 1])
        T = m.face_elem[F]
        assert np.all((T < 0) | ((T >= eo[p]) & (T < eo[p + 1])))
        assert np.array_equal(m.face_bc[F], mp.face_bc)
        assert np.allclose(sh[p], slot_shift(p, 2))


def test_batch_field_routes_nodes_to_their_problem():
    rng = np.random.default_rng(0)
    fields = [TrigForcing(rng) for _ in range(3)]
    sh = np.array([slot_shift(p, 2) for p in range(3)])
    bf = BatchField(fields, sh, per_row=2)
    pts = rng.uniform(0.0, 1.0, size=(7, 2))
    for p in range(3):
        assert np.allclose(bf.f(pts + sh[p]), fields[p].f(pts))
        assert np.allclose(bf.u(pts + sh[p]), 0.0)


@pytest.mark.parametrize("cond", ["v", "vp"])
def test_union_operator_is_block_diagonal_of_the_problems(cond):
    ms = _meshes()
    k = 1
    m, fo, eo, sh = union_mesh(ms, per_row=2)
    rng = np.random.default_rng(5)
    fields = [TrigForcing(rng) for _ in ms]
    hu = HHO(m, k, cond)
    ru = hu.assemble_rhs(*hu.data_values(BatchField(fields, sh, per_row=2)))
    Su = hu.S.toarray()
    b, nP = hu.b, (1 if cond == "vp" else hu.nE)
    NF = m.n_face
    idx = []
    for p, mp in enumerate(ms):
        rows = np.concatenate([np.arange(fo[p] * b, fo[p + 1] * b), NF * b + np.arange(eo[p] * nP, eo[p + 1] * nP)])
        idx.append(rows)
        hp = HHO(mp, k, cond)
        rp = hp.assemble_rhs(*hp.data_values(fields[p]))
        Sp = hp.S.toarray()
        scale = np.abs(Sp).max()
        assert np.abs(Su[np.ix_(rows, rows)] - Sp).max() <= 1e-11 * scale
        assert np.abs(ru[rows] - rp).max() <= 1e-11 * max(np.abs(rp).max(), 1.0)
    # nothing outside the diagonal blocks
    mask = np.ones_like(Su, dtype=bool)
    for rows in idx:
        mask[np.ix_(rows, rows)] = False
    assert np.abs(Su[mask]).max() == 0.0


def test_batch_problem_family_is_seeded_and_in_range():
    a = batch_problems(12, seed=7)
    b = batch_problems(12, seed=7)
    assert [(p.shape, p.n, p.k) for p in a] == [(p.shape, p.n, p.k) for p in b]
    assert all(8 <= p.n <= 64 and 1 <= p.k <= 4 and p.shape in ("quad", "tri") for p in a)
    assert all(not p.mesh.has_neumann() for p in a)
    g = group_by_degree(a)
    assert sorted(i for v in g.values() for i in v) == list(range(12))
