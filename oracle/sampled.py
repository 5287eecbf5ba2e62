"""Condensed residual rows at sampled faces and elements (oracle), for
full-size checks of a solution the oracle cannot solve for itself.

Test infrastructure.  The condensed system (Eq. ST.1 / ST.2) is assembled from
element contributions (end of Sec. 4.1.2): the row block of face F is
sum over T in T_F of (S_T x_T - g_T) restricted to F, and the row block of an
element's kept pressure is (S_T x_T - g_T) restricted to it.  So the residual
b - S x on the rows of a set of sampled faces needs the local systems of their
elements only.  Every geometric and basis quantity of an element or a face is
intrinsic (its vertices in their stored order, its boundary tag), so the local
systems are computed on the submesh made of the sampled faces' elements and
all of their faces, with the element and face numbering of the full mesh kept
in increasing order; HHO of Sec. 2 on that submesh gives the same S_T and g_T
as on the full mesh.  The DG scheme's element rows (residual_rows_dg) are
taken the same way from the submesh of the sampled elements and their
neighbours.  Pinned in tests against the rows of b - S x of the full oracle
on small meshes.
"""
from __future__ import annotations

import numpy as np

from .dg import DG
from .hho import HHO
from .hho_hp import HHOhp


def _submesh(mesh, elems):
    """Submesh of the given elements (sorted) and all of their faces."""
    from synthetic.meshes import Mesh
    elems = np.unique(np.asarray(elems, dtype=np.int64))
    faces = np.unique(np.concatenate([mesh.faces_of(int(t)) for t in elems]))
    fmap = {int(F): i for i, F in enumerate(faces)}
    emap = {int(t): i for i, t in enumerate(elems)}
    efp = np.zeros(len(elems) + 1, dtype=np.int64)
    ef = []
    for i, t in enumerate(elems):
        fs = [fmap[int(F)] for F in mesh.faces_of(int(t))]
        ef.extend(fs)
        efp[i + 1] = efp[i] + len(fs)
    verts = np.unique(np.concatenate([mesh.verts_of_face(int(F)) for F in faces]))
    vmap = {int(v): i for i, v in enumerate(verts)}
    fvp = np.zeros(len(faces) + 1, dtype=np.int64)
    fv = []
    fe = np.full((len(faces), 2), -1, dtype=np.int64)
    for i, F in enumerate(faces):
        vs = [vmap[int(v)] for v in mesh.verts_of_face(int(F))]
        fv.extend(vs)
        fvp[i + 1] = fvp[i] + len(vs)
        es = [emap[int(t)] for t in mesh.face_elem[int(F)] if t >= 0 and int(t) in emap]
        fe[i, :len(es)] = sorted(es)
    sub = Mesh(mesh.dim, mesh.xyz[verts].copy(), efp, np.asarray(ef, dtype=np.int64), fvp,
               np.asarray(fv, dtype=np.int64), fe, mesh.face_bc[faces].copy(), mesh.face_side[faces].copy(),
               name=mesh.name + "-sub")
    return sub, elems, faces


def residual_rows(mesh, k, cond, field, x, sample_faces, with_scale=False):
    """(rows, r, b): global indices of the condensed rows of the sampled faces
    and of the kept pressures of their elements (none for HHO-hp, cond "hp"), the residual b - S x and the
    right-hand side b on those rows, from the oracle's local systems.  x is the
    condensed vector of the full mesh (faces then elements).  With with_scale,
    also the scale |b_i| + sum over the elements T of row i of
    max|S_T| ||x_T||_1 (x_T: the element's kept unknowns).  Row i of S x is the
    sum of the rows of S_T x_T (end of Sec. 4.1.2), so two element Schur
    complements that agree to eps of their largest entry give rows of S x
    that agree to eps times this scale; it bounds |b| + |S| |x| from above."""
    sample_faces = np.unique(np.asarray(sample_faces, dtype=np.int64))
    elems = np.unique([int(t) for F in sample_faces for t in mesh.face_elem[int(F)] if t >= 0])
    sub, elems, faces = _submesh(mesh, elems)
    h = HHOhp(sub, k) if cond == "hp" else HHO(sub, k, cond)
    b_loc = h.assemble_rhs(*h.data_values(field))
    nF_glob = mesh.n_face
    bb, nP = h.b, h.nP
    # condensed vector of the submesh from the full-mesh x
    xs = np.zeros(h.ndof)
    for i, F in enumerate(faces):
        xs[i * bb:(i + 1) * bb] = x[int(F) * bb:(int(F) + 1) * bb]
    for i, t in enumerate(elems):
        xs[h.n_face_dofs + i * nP:h.n_face_dofs + (i + 1) * nP] = x[nF_glob * bb + int(t) * nP:
                                                                   nF_glob * bb + (int(t) + 1) * nP]
    r_loc = b_loc - h.S @ xs
    sc_loc = np.abs(b_loc)
    for t in range(len(elems)):
        g = h.global_kept(t)
        sc_loc[g] += np.abs(h.S_T[t]).max() * np.abs(xs[g]).sum()
    rows, r, b, sc = [], [], [], []
    fpos = {int(F): i for i, F in enumerate(faces)}
    for F in sample_faces:
        i = fpos[int(F)]
        rows.extend(int(F) * bb + np.arange(bb))
        r.extend(r_loc[i * bb:(i + 1) * bb])
        b.extend(b_loc[i * bb:(i + 1) * bb])
        sc.extend(sc_loc[i * bb:(i + 1) * bb])
    for i, t in enumerate(elems):
        o = h.n_face_dofs + i * nP
        rows.extend(nF_glob * bb + int(t) * nP + np.arange(nP))
        r.extend(r_loc[o:o + nP])
        b.extend(b_loc[o:o + nP])
        sc.extend(sc_loc[o:o + nP])
    out = (np.asarray(rows), np.asarray(r), np.asarray(b))
    return out + (np.asarray(sc),) if with_scale else out


def residual_rows_dg(mesh, k, field, x, sample_elems, with_scale=False):
    """DG scheme (Scheme 3, Sec. 2.4): (rows, r, b), the residual b - S x and
    b on the element blocks of the sampled elements, x the DG vector of the
    full mesh (one block of (d+1) n_E per element).  The block row of an
    element S couples S with the neighbours across its interior faces only, and
    each coupling is intrinsic to S, that neighbour and their shared face (the
    BR2 penalty takes the face counts of both).  So the rows are
    computed on the submesh of the sampled elements and their neighbours with
    all of their faces: there the neighbours' own rows change (their outer
    faces lose a side), the sampled rows do not.  With with_scale, also the
    scale |b_i| + sum over the blocks (S, T) of row i of max|block| ||x_T||_1,
    the bound on rows of S x whose blocks agree to eps of their largest
    entry."""
    sample = np.unique(np.asarray(sample_elems, dtype=np.int64))
    nbrs = [int(t) for S in sample for F in mesh.faces_of(int(S)) for t in mesh.face_elem[int(F)] if t >= 0]
    sub, elems, _ = _submesh(mesh, np.concatenate([sample, np.asarray(nbrs, dtype=np.int64)]))
    h = DG(sub, k)
    b_loc = h.assemble_rhs(*h.data_values(field))
    nb = h.nb
    xs = np.concatenate([x[int(t) * nb:(int(t) + 1) * nb] for t in elems])
    r_loc = b_loc - h.S @ xs
    epos = {int(t): i for i, t in enumerate(elems)}
    rows, r, b, sc = [], [], [], []
    for S in sample:
        i = epos[int(S)]
        sl = slice(i * nb, (i + 1) * nb)
        s = np.abs(b_loc[sl])
        for (p, q), M in h.blocks.items():
            if p == i:
                s = s + np.abs(M).max() * np.abs(xs[q * nb:(q + 1) * nb]).sum()
        rows.extend(int(S) * nb + np.arange(nb))
        r.extend(r_loc[sl])
        b.extend(b_loc[sl])
        sc.extend(s)
    out = (np.asarray(rows), np.asarray(r), np.asarray(b))
    return out + (np.asarray(sc),) if with_scale else out


def sample_elements(mesh, count, seed):
    """`count` elements drawn without replacement (seeded) from the elements of the mesh."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(mesh.n_elem, size=min(count, mesh.n_elem), replace=False))


def sample_interior_faces(mesh, count, seed):
    """`count` faces drawn without replacement (seeded) from the faces of the mesh."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(mesh.n_face, size=min(count, mesh.n_face), replace=False))
