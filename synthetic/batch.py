"""Batches of independent 2D problems (synthetic inputs for the batched solver).

``union_mesh`` lays problems out on a grid of unit-square slots (slot p at
(2 (p mod per_row), 2 (p div per_row))) and concatenates them into one mesh
whose faces and elements stay contiguous per problem; ``BatchField`` evaluates
each problem's data at its own local coordinates, recognising a node's
problem by its slot.  ``batch_problems`` draws the family of the batched
workload: quadrilateral or triangular meshes of 8^2 .. 64^2 cells with
interior vertices jittered by +-0.2h, degree k in 1..4, homogeneous Dirichlet
data on the whole boundary and a forcing made of 8 random trigonometric modes
per component with N(0, 1) coefficients.  Nothing here computes any part of
the method.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .meshes import Mesh, quad_mesh, tri_mesh

SLOT = 2.0


def slot_shift(p: int, per_row: int) -> np.ndarray:
    return np.array([SLOT * (p % per_row), SLOT * (p // per_row)])


def union_mesh(meshes, per_row: int = 16):
    """Disjoint union of 2D meshes on unit-square slots.

    Returns (mesh, face_off, elem_off, shifts): problem p owns faces
    face_off[p]:face_off[p+1] and elements elem_off[p]:elem_off[p+1], and its
    vertices are those of meshes[p] moved by shifts[p]."""
    xyz, efp, ef, fvp, fv, fe, fbc, fside = [], [0], [], [0], [], [], [], []
    face_off, elem_off, shifts = [0], [0], []
    nv = nf = ne = 0
    for p, m in enumerate(meshes):
        if m.dim != 2:
            raise ValueError("union_mesh builds 2D batches")
        sh = slot_shift(p, per_row)
        shifts.append(sh)
        xyz.append(m.xyz + sh)
        ef.append(m.elem_face + nf)
        efp.extend((m.elem_face_ptr[1:] + efp[-1]).tolist())
        fv.append(m.face_vert + nv)
        fvp.extend((m.face_vert_ptr[1:] + fvp[-1]).tolist())
        fe.append(np.where(m.face_elem >= 0, m.face_elem + ne, -1))
        fbc.append(m.face_bc)
        fside.append(m.face_side)
        nv += m.n_vert
        nf += m.n_face
        ne += m.n_elem
        face_off.append(nf)
        elem_off.append(ne)
    mesh = Mesh(dim=2, xyz=np.concatenate(xyz), elem_face_ptr=np.asarray(efp, dtype=np.int64),
                elem_face=np.concatenate(ef).astype(np.int64), face_vert_ptr=np.asarray(fvp, dtype=np.int64),
                face_vert=np.concatenate(fv).astype(np.int64), face_elem=np.concatenate(fe).astype(np.int64),
                face_bc=np.concatenate(fbc).astype(np.int8), face_side=np.concatenate(fside).astype(np.int8),
                name=f"union of {len(meshes)}", meta={"per_row": per_row})
    return mesh, np.asarray(face_off, dtype=np.int64), np.asarray(elem_off, dtype=np.int64), np.asarray(shifts)


class TrigForcing:
    """f_i(x, y) = sum_m c_{m,i} sin(pi (a_m x + b_m y) + phi_m), a_m, b_m in 1..4,
    phi_m in [0, 2 pi), c ~ N(0, 1); homogeneous boundary data."""

    def __init__(self, rng: np.random.Generator, modes: int = 8):
        self.a = rng.integers(1, 5, size=modes)
        self.b = rng.integers(1, 5, size=modes)
        self.phi = rng.uniform(0.0, 2.0 * np.pi, size=modes)
        self.c = rng.standard_normal((modes, 2))

    def f(self, x):
        x = np.atleast_2d(x)
        arg = np.pi * (np.outer(x[:, 0], self.a) + np.outer(x[:, 1], self.b)) + self.phi
        return np.sin(arg) @ self.c

    def u(self, x):
        return np.zeros((np.atleast_2d(x).shape[0], 2))

    def g_neumann(self, x, n):
        return np.zeros((np.atleast_2d(x).shape[0], 2))


class BatchField:
    """Data of a batch: node -> problem by its slot, then that problem's field at
    local coordinates."""

    def __init__(self, fields, shifts, per_row: int = 16):
        self.fields = list(fields)
        self.shifts = np.asarray(shifts)
        self.per_row = per_row

    def _split(self, x):
        x = np.atleast_2d(x)
        ij = np.floor(x / SLOT).astype(np.int64)
        p = ij[:, 1] * self.per_row + ij[:, 0]
        return x - self.shifts[p], p

    def _eval(self, name, x, extra=None):
        xl, p = self._split(x)
        out = np.zeros((xl.shape[0], 2))
        for q in np.unique(p):
            sel = p == q
            fn = getattr(self.fields[q], name)
            out[sel] = fn(xl[sel]) if extra is None else fn(xl[sel], extra[sel])
        return out

    def f(self, x):
        return self._eval("f", x)

    def u(self, x):
        return self._eval("u", x)

    def g_neumann(self, x, n):
        return self._eval("g_neumann", x, np.atleast_2d(n))


@dataclass
class Problem:
    mesh: Mesh
    k: int
    field: object
    shape: str
    n: int


def batch_problems(n_prob: int = 256, seed: int = 12345, n_min: int = 8, n_max: int = 64, k_min: int = 1,
                   k_max: int = 4, jitter: float = 0.2):
    """The batched workload's problem family (see the module docstring)."""
    rng = np.random.default_rng(seed)
    out = []
    for p in range(n_prob):
        shape = "quad" if rng.integers(0, 2) == 0 else "tri"
        n = int(rng.integers(n_min, n_max + 1))
        k = int(rng.integers(k_min, k_max + 1))
        mseed = int(rng.integers(0, 2**31 - 1))
        mesh = (quad_mesh if shape == "quad" else tri_mesh)(n, jitter=jitter, seed=mseed)
        out.append(Problem(mesh=mesh, k=k, field=TrigForcing(rng), shape=shape, n=n))
    return out


def group_by_degree(problems):
    """{k: [indices]} in increasing k."""
    groups = {}
    for i, pr in enumerate(problems):
        groups.setdefault(pr.k, []).append(i)
    return dict(sorted(groups.items()))
