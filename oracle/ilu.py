"""Block ILU(0) smoother preconditioner (oracle) for the condensed level operators.

Test infrastructure.  The paper smooths with "ILU preconditioned GMRES"
(Sec. 3.3, two iterations per Sec. 5.2.2) without fixing the ordering or the
fill.  Reading: block ILU(0) on the block sparsity of S (face blocks of b
unknowns, element pressure blocks of n_P), no fill, with
* the faces first, in a greedy multicolour order: faces are adjacent when they
  share an element; face F (in index order) takes the smallest colour not used
  by an already coloured adjacent face; faces sorted by (colour, index);
* the element pressure blocks last (index order), so that the mean-pressure
  rows, whose diagonal is zero, are pivoted on the Schur-like block
  S_TT - sum L_TF U_FT.
Factorisation (IKJ form, on the pattern only): for each block row i in order,
for each k < i in the row's pattern: A_ik <- A_ik A_kk^{-1}, then for every
j > k in the pattern of both rows i and k: A_ij <- A_ij - A_ik A_kj.
Application: z = U^{-1} L^{-1} v (L unit lower, U upper with the pivots).
"""
from __future__ import annotations

import numpy as np


def face_colors(mesh):
    """Greedy colouring of the faces by index (faces sharing an element differ)."""
    nf = mesh.n_face
    col = -np.ones(nf, dtype=np.int64)
    for F in range(nf):
        used = set()
        for T in mesh.face_elem[F]:
            if T < 0:
                continue
            for G in mesh.faces_of(T):
                if G != F and col[G] >= 0:
                    used.add(int(col[G]))
        c = 0
        while c in used:
            c += 1
        col[F] = c
    return col


class BlockILU:
    """Block ILU(0) of a level operator S (scipy sparse, faces then elements)."""

    def __init__(self, S, mesh, b, nP):
        self.mesh, self.b, self.nP = mesh, b, nP
        nf, ne = mesh.n_face, mesh.n_elem
        self.nf, self.ne = nf, ne
        col = face_colors(mesh)
        self.colors = col
        # block order: faces by (colour, index), then elements
        forder = sorted(range(nf), key=lambda F: (col[F], F))
        self.order = [("f", F) for F in forder] + [("e", T) for T in range(ne)]
        self.rank = {blk: i for i, blk in enumerate(self.order)}
        A = S.tocsr()

        def sl(blk):
            kind, i = blk
            return slice(i * b, (i + 1) * b) if kind == "f" else slice(nf * b + i * nP, nf * b + (i + 1) * nP)

        self.sl = sl
        # block pattern of every block row
        pat = {}
        for F in range(nf):
            nb = {("f", F)}
            for T in mesh.face_elem[F]:
                if T < 0:
                    continue
                nb.add(("e", int(T)))
                for G in mesh.faces_of(T):
                    nb.add(("f", int(G)))
            pat[("f", F)] = nb
        for T in range(ne):
            pat[("e", T)] = {("e", T)} | {("f", int(G)) for G in mesh.faces_of(T)}
        self.pat = pat
        blocks = {}
        for i, row in pat.items():
            for j in row:
                blocks[(i, j)] = A[sl(i), sl(j)].toarray()
        # IKJ elimination on the pattern
        for i in self.order:
            ri = self.rank[i]
            lower = sorted((k for k in pat[i] if self.rank[k] < ri), key=lambda k: self.rank[k])
            for k in lower:
                blocks[(i, k)] = blocks[(i, k)] @ np.linalg.inv(blocks[(k, k)])
                for j in pat[i]:
                    if self.rank[j] > self.rank[k] and j in pat[k]:
                        blocks[(i, j)] = blocks[(i, j)] - blocks[(i, k)] @ blocks[(k, j)]
        self.blocks = blocks

    def apply(self, v):
        z = np.array(v, dtype=float)
        sl, pat, rank, B = self.sl, self.pat, self.rank, self.blocks
        for i in self.order:  # L y = v (unit lower)
            for k in pat[i]:
                if rank[k] < rank[i]:
                    z[sl(i)] -= B[(i, k)] @ z[sl(k)]
        for i in reversed(self.order):  # U z = y
            s = z[sl(i)].copy()
            for j in pat[i]:
                if rank[j] > rank[i]:
                    s -= B[(i, j)] @ z[sl(j)]
            z[sl(i)] = np.linalg.solve(B[(i, i)], s)
        return z
