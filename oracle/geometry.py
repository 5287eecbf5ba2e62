"""Element and face geometry (oracle), Sec. 2.1.

For an element T: the vertex average x_T, the measure |T|, the diameter h_T,
the bounding box, the outward unit normals n_TF of its faces and its
sub-simplices (fan from x_T over every face; in 3D each face is first fanned
from its own vertex average).  For a face F: its vertex average x_F, measure
|F|, diameter h_F, a fixed unit normal n_F, a tangent frame and bounding box in
that frame.  n_TF = +-n_F with the sign making n_TF point from x_T to x_F.
"""
from __future__ import annotations

import numpy as np

from .quadrature import segment_rule, triangle_rule, tet_rule


def _diameter(P):
    d = 0.0
    for i in range(len(P)):
        for j in range(i + 1, len(P)):
            d = max(d, float(np.linalg.norm(P[i] - P[j])))
    return d


class FaceGeom:
    def __init__(self, mesh, f):
        self.id = f
        V = mesh.xyz[mesh.verts_of_face(f)]
        self.V = V
        self.dim = mesh.dim
        self.xF = V.mean(axis=0)
        self.hF = _diameter(V)
        if mesh.dim == 2:
            t = V[1] - V[0]
            self.meas = float(np.linalg.norm(t))
            t = t / self.meas
            self.n = np.array([t[1], -t[0]])
            self.frame = t[None, :]
        else:
            m = len(V)
            nn = np.zeros(3)
            area = 0.0
            for i in range(m):
                c = np.cross(V[i] - self.xF, V[(i + 1) % m] - self.xF)
                nn += c
                area += 0.5 * np.linalg.norm(c)
            self.meas = area
            self.n = nn / np.linalg.norm(nn)
            t1 = V[1] - V[0]
            t1 = t1 / np.linalg.norm(t1)
            t2 = np.cross(self.n, t1)
            self.frame = np.stack([t1, t2])
        Y = (V - self.xF) @ self.frame.T
        lo, hi = Y.min(axis=0), Y.max(axis=0)
        self.bb_c = 0.5 * (lo + hi)
        self.bb_r = 0.5 * (hi - lo)

    def local_coords(self, X):
        return (X - self.xF) @ self.frame.T

    def rule(self, p):
        if self.dim == 2:
            return segment_rule(self.V[0], self.V[1], p)
        pts, wts = [], []
        m = len(self.V)
        for i in range(m):
            P, W = triangle_rule(self.xF, self.V[i], self.V[(i + 1) % m], p)
            pts.append(P)
            wts.append(W)
        return np.concatenate(pts), np.concatenate(wts)


class ElemGeom:
    def __init__(self, mesh, t, faces):
        self.id = t
        self.dim = mesh.dim
        self.faces = [faces[f] for f in mesh.faces_of(t)]
        vids = np.unique(np.concatenate([mesh.verts_of_face(F.id) for F in self.faces]))
        V = mesh.xyz[vids]
        self.xT = V.mean(axis=0)
        self.hT = _diameter(V)
        lo, hi = V.min(axis=0), V.max(axis=0)
        self.bb_c = 0.5 * (lo + hi)
        self.bb_r = 0.5 * (hi - lo)
        self.nTF = []
        for F in self.faces:
            s = 1.0 if float(F.n @ (F.xF - self.xT)) > 0 else -1.0
            self.nTF.append(s * F.n)
        _, w = self.rule(0)
        self.meas = float(w.sum())

    def rule(self, p):
        pts, wts = [], []
        for F in self.faces:
            if self.dim == 2:
                P, W = triangle_rule(self.xT, F.V[0], F.V[1], p)
                pts.append(P)
                wts.append(W)
            else:
                m = len(F.V)
                for i in range(m):
                    P, W = tet_rule(self.xT, F.xF, F.V[i], F.V[(i + 1) % m], p)
                    pts.append(P)
                    wts.append(W)
        return np.concatenate(pts), np.concatenate(wts)


def mesh_geometry(mesh):
    faces = [FaceGeom(mesh, f) for f in range(mesh.n_face)]
    elems = [ElemGeom(mesh, t, faces) for t in range(mesh.n_elem)]
    return elems, faces
