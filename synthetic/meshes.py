"""Seeded mesh generators (topology and vertex coordinates only).

A mesh is the couple (elements, faces) of Sec. 2.1: every element lists its
faces, every face lists its vertices (a segment in 2D, a planar polygon in 3D
with vertices in cyclic order) and the one or two elements that share it, and
every boundary face carries a boundary-condition tag (1 Dirichlet, 2 Neumann).

Conventions used by every generator:

* ``face_elem[f] = (T1, T2)`` with ``T1 < T2``; a boundary face has ``T2 = -1``.
* Element faces are listed counter-clockwise in 2D; in 3D in the order
  x-, x+, y-, y+, z-, z+.
* Jitter: interior vertices (2D) or interior grid planes (3D) are displaced by
  uniform random offsets drawn from SplitMix64(seed), one draw per coordinate in
  vertex-index (plane-index) order; boundary vertices stay on the boundary so
  the domain is exact.
* Boundary sides are numbered 0: x=x0, 1: x=x1, 2: y=y0, 3: y=y1, 4: z=z0,
  5: z=z1.  Sides listed in ``neumann_sides`` get tag 2, the others tag 1.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_MASK64 = (1 << 64) - 1


def splitmix64_doubles(seed: int, count: int) -> np.ndarray:
    """``count`` doubles in [0, 1) from SplitMix64 (Steele, Lea, Flood 2014).

    Each 64-bit output is reduced to its top 53 bits and scaled by 2**-53.
    """
    out = np.empty(count, dtype=np.float64)
    state = seed & _MASK64
    for i in range(count):
        state = (state + 0x9E3779B97F4A7C15) & _MASK64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        z = z ^ (z >> 31)
        out[i] = (z >> 11) * (1.0 / 9007199254740992.0)
    return out


@dataclass
class Mesh:
    dim: int
    xyz: np.ndarray            # (n_vert, dim) float64
    elem_face_ptr: np.ndarray  # (n_elem+1,) int64
    elem_face: np.ndarray      # (sum |F_T|,) int64
    face_vert_ptr: np.ndarray  # (n_face+1,) int64
    face_vert: np.ndarray      # (sum |V_F|,) int64
    face_elem: np.ndarray      # (n_face, 2) int64, -1 = none
    face_bc: np.ndarray        # (n_face,) int8: 0 interior, 1 Dirichlet, 2 Neumann
    face_side: np.ndarray      # (n_face,) int8: boundary side index, -1 interior
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_vert(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_elem(self) -> int:
        return int(self.elem_face_ptr.shape[0] - 1)

    @property
    def n_face(self) -> int:
        return int(self.face_vert_ptr.shape[0] - 1)

    def faces_of(self, t: int) -> np.ndarray:
        return self.elem_face[self.elem_face_ptr[t]:self.elem_face_ptr[t + 1]]

    def verts_of_face(self, f: int) -> np.ndarray:
        return self.face_vert[self.face_vert_ptr[f]:self.face_vert_ptr[f + 1]]

    def has_neumann(self) -> bool:
        return bool(np.any(self.face_bc == 2))


def _finish(dim, xyz, elem_faces, face_verts, face_side, neumann_sides, name, meta):
    n_elem = len(elem_faces)
    n_face = len(face_verts)
    efp = np.zeros(n_elem + 1, dtype=np.int64)
    efp[1:] = np.cumsum([len(f) for f in elem_faces])
    ef = np.fromiter((f for fs in elem_faces for f in fs), dtype=np.int64, count=int(efp[-1]))
    fvp = np.zeros(n_face + 1, dtype=np.int64)
    fvp[1:] = np.cumsum([len(v) for v in face_verts])
    fv = np.fromiter((v for vs in face_verts for v in vs), dtype=np.int64, count=int(fvp[-1]))
    fe = np.full((n_face, 2), -1, dtype=np.int64)
    cnt = np.zeros(n_face, dtype=np.int64)
    for t, fs in enumerate(elem_faces):
        for f in fs:
            if cnt[f] >= 2:
                raise ValueError("face shared by more than two elements")
            fe[f, cnt[f]] = t
            cnt[f] += 1
    side = np.asarray(face_side, dtype=np.int8)
    bc = np.zeros(n_face, dtype=np.int8)
    bnd = fe[:, 1] < 0
    if np.any(bnd != (side >= 0)):
        raise ValueError("boundary side tags disagree with the face-element map")
    bc[bnd] = 1
    for s in neumann_sides:
        bc[bnd & (side == s)] = 2
    return Mesh(dim, np.ascontiguousarray(xyz, dtype=np.float64), efp, ef, fvp, fv, fe, bc, side,
                name, meta)


def _jitter_2d(xyz, nx, ny, hx, hy, jitter, seed):
    if jitter == 0.0:
        return xyz
    interior = [i + (nx + 1) * j for j in range(1, ny) for i in range(1, nx)]
    u = splitmix64_doubles(seed, 2 * len(interior))
    for n, v in enumerate(interior):
        xyz[v, 0] += jitter * hx * (2.0 * u[2 * n] - 1.0)
        xyz[v, 1] += jitter * hy * (2.0 * u[2 * n + 1] - 1.0)
    return xyz


def _grid_2d(nx, ny, x0, x1, y0, y1):
    xs = np.linspace(x0, x1, nx + 1)
    ys = np.linspace(y0, y1, ny + 1)
    xyz = np.zeros(((nx + 1) * (ny + 1), 2))
    for j in range(ny + 1):
        for i in range(nx + 1):
            xyz[i + (nx + 1) * j] = (xs[i], ys[j])
    return xyz


def quad_mesh(nx: int, ny: int | None = None, jitter: float = 0.0, seed: int = 0,
              neumann_sides=(), box=(0.0, 1.0, 0.0, 1.0)) -> Mesh:
    """nx x ny quadrilaterals on a box; faces: horizontal edges then vertical edges."""
    ny = nx if ny is None else ny
    x0, x1, y0, y1 = box
    hx, hy = (x1 - x0) / nx, (y1 - y0) / ny
    xyz = _jitter_2d(_grid_2d(nx, ny, x0, x1, y0, y1), nx, ny, hx, hy, jitter, seed)

    def v(i, j):
        return i + (nx + 1) * j

    nH = nx * (ny + 1)

    def H(i, j):
        return j * nx + i

    def V(i, j):
        return nH + j * (nx + 1) + i

    face_verts = [None] * (nH + (nx + 1) * ny)
    face_side = [-1] * len(face_verts)
    for j in range(ny + 1):
        for i in range(nx):
            face_verts[H(i, j)] = (v(i, j), v(i + 1, j))
            if j == 0:
                face_side[H(i, j)] = 2
            elif j == ny:
                face_side[H(i, j)] = 3
    for j in range(ny):
        for i in range(nx + 1):
            face_verts[V(i, j)] = (v(i, j), v(i, j + 1))
            if i == 0:
                face_side[V(i, j)] = 0
            elif i == nx:
                face_side[V(i, j)] = 1
    elem_faces = [(H(i, j), V(i + 1, j), H(i, j + 1), V(i, j)) for j in range(ny) for i in range(nx)]
    return _finish(2, xyz, elem_faces, face_verts, face_side, neumann_sides,
                   f"quad{nx}x{ny}", dict(kind="quad", nx=nx, ny=ny, jitter=jitter, seed=seed))


def tri_mesh(nx: int, ny: int | None = None, jitter: float = 0.0, seed: int = 0,
             neumann_sides=(), box=(0.0, 1.0, 0.0, 1.0)) -> Mesh:
    """nx x ny squares, each split by its lower-left to upper-right diagonal.

    Square (i, j) gives triangle 2s = (v00, v10, v11) and 2s+1 = (v00, v11, v01)
    with s = i + nx*j.  Faces: horizontal, vertical, then diagonal edges.
    """
    ny = nx if ny is None else ny
    x0, x1, y0, y1 = box
    hx, hy = (x1 - x0) / nx, (y1 - y0) / ny
    xyz = _jitter_2d(_grid_2d(nx, ny, x0, x1, y0, y1), nx, ny, hx, hy, jitter, seed)

    def v(i, j):
        return i + (nx + 1) * j

    nH = nx * (ny + 1)
    nV = (nx + 1) * ny

    def H(i, j):
        return j * nx + i

    def V(i, j):
        return nH + j * (nx + 1) + i

    def D(i, j):
        return nH + nV + j * nx + i

    n_face = nH + nV + nx * ny
    face_verts = [None] * n_face
    face_side = [-1] * n_face
    for j in range(ny + 1):
        for i in range(nx):
            face_verts[H(i, j)] = (v(i, j), v(i + 1, j))
            if j == 0:
                face_side[H(i, j)] = 2
            elif j == ny:
                face_side[H(i, j)] = 3
    for j in range(ny):
        for i in range(nx + 1):
            face_verts[V(i, j)] = (v(i, j), v(i, j + 1))
            if i == 0:
                face_side[V(i, j)] = 0
            elif i == nx:
                face_side[V(i, j)] = 1
    for j in range(ny):
        for i in range(nx):
            face_verts[D(i, j)] = (v(i, j), v(i + 1, j + 1))
    elem_faces = []
    for j in range(ny):
        for i in range(nx):
            elem_faces.append((H(i, j), V(i + 1, j), D(i, j)))
            elem_faces.append((D(i, j), H(i, j + 1), V(i, j)))
    return _finish(2, xyz, elem_faces, face_verts, face_side, neumann_sides,
                   f"tri{nx}x{ny}", dict(kind="tri", nx=nx, ny=ny, jitter=jitter, seed=seed))


def hex_mesh(n: int, jitter: float = 0.0, seed: int = 0, neumann_sides=()) -> Mesh:
    """n^3 hexahedra on the unit cube with planar faces.

    Every interior grid plane of each family is moved by a random affine map
    x = x_i + o + t*(y - 1/2) + s*(z - 1/2) (and cyclically for y-, z-planes),
    with |o| + |t|/2 + |s|/2 <= jitter*h, so all faces stay planar while the
    vertices move by up to about jitter*h.  Three draws (o, t, s) per interior
    plane, x-planes first, then y-planes, then z-planes.
    """
    h = 1.0 / n
    nint = n - 1
    coef = np.zeros((3, n + 1, 3))  # family, plane index, (o, t, s)
    if jitter != 0.0 and nint > 0:
        u = splitmix64_doubles(seed, 3 * 3 * nint)
        c = 0
        for fam in range(3):
            for i in range(1, n):
                coef[fam, i, 0] = 0.5 * jitter * h * (2.0 * u[c] - 1.0)
                coef[fam, i, 1] = 0.5 * jitter * h * (2.0 * u[c + 1] - 1.0)
                coef[fam, i, 2] = 0.5 * jitter * h * (2.0 * u[c + 2] - 1.0)
                c += 3
    # plane of family a, index i: x_a - t*x_b - s*x_c = i*h + o - t/2 - s/2 with (b, c) the other axes
    others = ((1, 2), (0, 2), (0, 1))

    def vid(i, j, k):
        return i + (n + 1) * (j + (n + 1) * k)

    xyz = np.zeros(((n + 1) ** 3, 3))
    for k in range(n + 1):
        for j in range(n + 1):
            for i in range(n + 1):
                idx = (i, j, k)
                M = np.zeros((3, 3))
                rhs = np.zeros(3)
                for a in range(3):
                    o, t, s = coef[a, idx[a]]
                    b, c = others[a]
                    M[a, a] = 1.0
                    M[a, b] = -t
                    M[a, c] = -s
                    rhs[a] = idx[a] * h + o - 0.5 * t - 0.5 * s
                xyz[vid(i, j, k)] = np.linalg.solve(M, rhs)
    nXf = (n + 1) * n * n

    def X(i, j, k):
        return i + (n + 1) * (j + n * k)

    def Y(i, j, k):
        return nXf + j + (n + 1) * (i + n * k)

    def Z(i, j, k):
        return 2 * nXf + k + (n + 1) * (i + n * j)

    face_verts = [None] * (3 * nXf)
    face_side = [-1] * (3 * nXf)
    for k in range(n):
        for j in range(n):
            for i in range(n + 1):
                face_verts[X(i, j, k)] = (vid(i, j, k), vid(i, j + 1, k), vid(i, j + 1, k + 1), vid(i, j, k + 1))
                if i == 0 or i == n:
                    face_side[X(i, j, k)] = 0 if i == 0 else 1
    for k in range(n):
        for i in range(n):
            for j in range(n + 1):
                face_verts[Y(i, j, k)] = (vid(i, j, k), vid(i, j, k + 1), vid(i + 1, j, k + 1), vid(i + 1, j, k))
                if j == 0 or j == n:
                    face_side[Y(i, j, k)] = 2 if j == 0 else 3
    for j in range(n):
        for i in range(n):
            for k in range(n + 1):
                face_verts[Z(i, j, k)] = (vid(i, j, k), vid(i + 1, j, k), vid(i + 1, j + 1, k), vid(i, j + 1, k))
                if k == 0 or k == n:
                    face_side[Z(i, j, k)] = 4 if k == 0 else 5
    elem_faces = []
    for k in range(n):
        for j in range(n):
            for i in range(n):
                elem_faces.append((X(i, j, k), X(i + 1, j, k), Y(i, j, k), Y(i, j + 1, k),
                                   Z(i, j, k), Z(i, j, k + 1)))
    return _finish(3, xyz, elem_faces, face_verts, face_side, neumann_sides,
                   f"hex{n}", dict(kind="hex", n=n, jitter=jitter, seed=seed))
