"""HHO-hp (Scheme 2 of Sec. 2.3.2: the HHO viscous term with element velocity
of degree k+1 and face velocity of degree k, and a hybrid pressure made of an
element part in P^k(T) and a face part in P^k(F)): local operators, static
condensation of every element unknown, assembly, direct solve, recovery and
error norms (oracle).

Test infrastructure: only tests, the smoke check and the bench's CPU baseline
use this module.

Local unknown ordering: [U_T | U_F1 .. U_FN | P_T | P_F1 .. P_FN] with U_T the d
components of v_T in P^{k+1}(T) (n_V = dim P^{k+1}_d coefficients each), U_F
the d components of v_F (n_F each, component-major), P_T the n_E element
pressure coefficients and P_F the n_F coefficients of the face pressure.

Condensation (Sec. 4.1.2 applied to Scheme 2, the last paragraph of
Sec. 2.3.2): every element unknown (U_T and all of P_T) is eliminated; the
element block [A_TT B_TT^T; B_TT 0] is invertible because the divergence maps
P^{k+1}(T)^d onto P^k(T).  The kept unknowns are the face velocity and the
face pressure, so the global condensed system has one block of
b = (d+1) n_F per face (velocity component-major, then pressure) and no
element rows.

Readings of the paper:
* The local residuals are those of Scheme 1 with k' = k+1 except for the boxed
  terms of Sec. 2.3.2, and the reconstruction, face residual (Sec. 2.2 with
  k' = k+1: the element part of r_TF is the whole trace of v_T - p v, which
  has degree k+1), Nitsche terms and penalty eta_F are unchanged.
* The printed mass residual of Scheme 2 has no Dirichlet terms.  Its momentum
  residual adds int p_F (v_F . n) on Dirichlet faces, which removes the face
  velocity from the pressure coupling there; the mass residual is read the same
  way, int (u_T - g_D) . n q_F on Dirichlet faces (as Scheme 1 carries
  - int g_D . n q_T).  This keeps the system symmetric and consistent: a
  polynomial solution (u in P^{k+1}, p in P^k) is reproduced exactly.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .basis import dim_P
from .hho import HHO, penalty, schur

HPCOND = "hp"


class LocalSystemHP:
    """Local matrices of one element for Scheme 2 (the analogue of Eq. def:HHOAB)."""

    def __init__(self, hho, t):
        self.t = t
        k, d = hho.k, hho.d
        eg = hho.elems[t]
        eb = hho.ebases[t]
        nR, nE, nF = dim_P(d, k + 1), dim_P(d, k), dim_P(d - 1, k)
        nV = nR  # element velocity in P^{k+1}(T)
        N = len(eg.faces)
        ns = nV + N * nF
        self.nV, self.nE, self.nF, self.N, self.ns = nV, nE, nF, N, ns
        q_op = 2 * k + 2

        # --- p_T^{k+1} with k' = k+1 (Sec. 2.2.1) ---
        X, W = eg.rule(q_op)
        ev, eg_ = eb.eval_grad(X)
        Kst = np.einsum("q,qid,qjd->ij", W, eg_, eg_)
        Rhs = np.zeros((nR, ns))
        Rhs[:, :nV] = Kst[:, :nV]
        face_data = []
        for f, F in enumerate(eg.faces):
            n = eg.nTF[f]
            Xf, Wf = F.rule(q_op)
            fv, fg = eb.eval_grad(Xf)
            dn = fg @ n
            psi = hho.fbases[F.id].eval(Xf)
            sl = slice(nV + f * nF, nV + (f + 1) * nF)
            Rhs[:, sl] += np.einsum("q,qi,qj->ij", Wf, dn, psi)
            Rhs[:, :nV] -= np.einsum("q,qi,qj->ij", Wf, dn, fv[:, :nV])
            face_data.append((n, Wf, fv, dn, psi, sl))
        P = np.zeros((nR, ns))
        P[0, 0] = 1.0
        P[1:, :] = np.linalg.solve(Kst[1:, 1:], Rhs[1:, :])
        self.P = P

        # --- viscous form: the face residual's element part pi_T^{k+1}(v_T - p v) is v_T - p v itself ---
        A = P.T @ Kst @ P
        ET = np.zeros((nV, ns))
        ET[:, :nV] = np.eye(nV)
        for f, F in enumerate(eg.faces):
            n, Wf, fv, dn, psi, sl = face_data[f]
            EF = np.zeros((nF, ns))
            EF[:, sl] = np.eye(nF)
            MFT = np.einsum("q,qj,qm->jm", Wf, psi, fv)
            r = psi @ (EF - MFT @ P) - fv[:, :nV] @ (ET - P[:nV, :])
            A += (r.T * Wf) @ r / F.hF
            if hho.mesh.face_bc[F.id] == 1:
                eta = penalty(k, d, F.meas, F.hF, eg.meas)
                G = dn @ P
                V = psi @ EF
                A += -(V.T * Wf) @ G - (G.T * Wf) @ V + eta / F.hF * (V.T * Wf) @ V
        self.A_scalar = A

        nvec = d * nV + N * d * nF
        self.nvec = nvec
        vmap = np.zeros((d, ns), dtype=np.int64)
        for c in range(d):
            vmap[c, :nV] = c * nV + np.arange(nV)
            for f in range(N):
                vmap[c, nV + f * nF: nV + (f + 1) * nF] = d * nV + f * d * nF + c * nF + np.arange(nF)
        self.vmap = vmap
        Avec = np.zeros((nvec, nvec))
        for c in range(d):
            Avec[np.ix_(vmap[c], vmap[c])] = A

        # --- hybrid pressure coupling (boxed terms of Sec. 2.3.2) ---
        npr = nE + N * nF
        B = np.zeros((npr, nvec))
        for c in range(d):  # - int_T q_T div v_T
            B[:nE, c * nV:(c + 1) * nV] -= np.einsum("q,qi,qj->ij", W, ev[:, :nE], eg_[:, :nV, c])
        for f, F in enumerate(eg.faces):
            n, Wf, fv, dn, psi, sl = face_data[f]
            rows = nE + f * nF + np.arange(nF)
            for c in range(d):  # int_F (v_T - v_F) . n q_F, v_F dropped on Dirichlet faces
                B[rows, c * nV:(c + 1) * nV] += n[c] * np.einsum("q,qi,qj->ij", Wf, psi, fv[:, :nV])
                if hho.mesh.face_bc[F.id] != 1:
                    cols = d * nV + f * d * nF + c * nF + np.arange(nF)
                    B[np.ix_(rows, cols)] -= n[c] * np.einsum("q,qi,qj->ij", Wf, psi, psi)
        self.B = B
        self.npr = npr
        K = np.zeros((nvec + npr, nvec + npr))
        K[:nvec, :nvec] = Avec
        K[nvec:, :nvec] = B
        K[:nvec, nvec:] = B.T
        self.K = K

    def rhs(self, hho, f_vals, gD_vals, gN_vals):
        k, d = hho.k, hho.d
        eg, eb = hho.elems[self.t], hho.ebases[self.t]
        nV, nE, nF = self.nV, self.nE, self.nF
        q_dat = 2 * k + 2
        b = np.zeros(self.nvec + self.npr)
        X, W = eg.rule(q_dat)
        ev = eb.eval(X, nV)
        fv = f_vals[self.t]
        for c in range(d):
            b[c * nV:(c + 1) * nV] += ev.T @ (W * fv[:, c])
        for f, F in enumerate(eg.faces):
            bc = hho.mesh.face_bc[F.id]
            if bc == 0:
                continue
            Xf, Wf = F.rule(q_dat)
            psi = hho.fbases[F.id].eval(Xf)
            if bc == 1:
                g = gD_vals[F.id]
                n = eg.nTF[f]
                fvv, fg = eb.eval_grad(Xf)
                G = (fg @ n) @ self.P
                eta = penalty(k, d, F.meas, F.hF, eg.meas)
                for c in range(d):
                    b[self.vmap[c]] -= G.T @ (Wf * g[:, c])
                    cols = d * nV + f * d * nF + c * nF + np.arange(nF)
                    b[cols] += eta / F.hF * (psi.T @ (Wf * g[:, c]))
                b[self.nvec + nE + f * nF + np.arange(nF)] += psi.T @ (Wf * (g @ n))
            else:
                g = gN_vals[F.id]
                for c in range(d):
                    cols = d * nV + f * d * nF + c * nF + np.arange(nF)
                    b[cols] += psi.T @ (Wf * g[:, c])
        return b

    def split(self, cond=HPCOND):
        """Eliminated (U_T, P_T) and kept (per face: U_F then P_F) local indices."""
        d, nV, nE, nF = self.vmap.shape[0], self.nV, self.nE, self.nF
        elim = list(range(d * nV)) + [self.nvec + i for i in range(nE)]
        keep = []
        for f in range(self.N):
            keep.extend(d * nV + f * d * nF + np.arange(d * nF))
            keep.extend(self.nvec + nE + f * nF + np.arange(nF))
        return elim, [int(i) for i in keep]


class HHOhp(HHO):
    """Discretisation of the Stokes problem by Scheme 2 (HHO-hp), condensed to the skeleton."""

    def __init__(self, mesh, k):
        from .basis import element_basis, face_basis
        from .geometry import mesh_geometry
        self.mesh = mesh
        self.k = k
        self.d = mesh.dim
        self.cond = HPCOND
        self.elems, self.faces = mesh_geometry(mesh)
        self.ebases = [element_basis(e, k + 1) for e in self.elems]
        self.fbases = [face_basis(f, k) for f in self.faces]
        self.nE = dim_P(self.d, k)
        self.nV = dim_P(self.d, k + 1)
        self.nF = dim_P(self.d - 1, k)
        self.b = (self.d + 1) * self.nF
        self.nP = 0
        self.local = [LocalSystemHP(self, t) for t in range(mesh.n_elem)]
        self.n_face_dofs = mesh.n_face * self.b
        self.ndof = self.n_face_dofs
        self._condense()

    def global_kept(self, t):
        b = self.b
        return np.concatenate([int(F) * b + np.arange(b) for F in self.mesh.faces_of(t)]).astype(np.int64)

    def null_vector(self):
        """Constant hybrid pressure (p_T = p_F = 1) restricted to the kept face
        pressures: the constant face mode has coefficient sqrt(|F|) in the
        orthonormal face basis.  None when a Neumann face exists."""
        if self.mesh.has_neumann():
            return None
        n = np.zeros(self.ndof)
        for F in range(self.mesh.n_face):
            n[F * self.b + self.d * self.nF] = np.sqrt(self.faces[F].meas)
        return n / np.linalg.norm(n)

    def uncondensed(self, f_vals, gD, gN):
        """Full system over [U_T of all elements | P_T | face blocks (U_F, P_F)]."""
        d, nV, nE, b = self.d, self.nV, self.nE, self.b
        nf, ne = self.mesh.n_face, self.mesh.n_elem
        n_tot = nf * b + ne * (d * nV + nE)
        rows, cols, vals = [], [], []
        rhs = np.zeros(n_tot)
        for t, L in enumerate(self.local):
            elim, keep = L.split()
            g = np.zeros(L.K.shape[0], dtype=np.int64)
            g[elim] = nf * b + t * (d * nV + nE) + np.arange(len(elim))
            g[keep] = self.global_kept(t)
            rows.append(np.repeat(g, len(g)))
            cols.append(np.tile(g, len(g)))
            vals.append(L.K.ravel())
            rhs[g] += L.rhs(self, f_vals, gD, gN)
        K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n_tot, n_tot))
        null = None
        if not self.mesh.has_neumann():
            null = np.zeros(n_tot)
            for F in range(nf):
                null[F * b + d * self.nF] = np.sqrt(self.faces[F].meas)
            for t in range(ne):
                null[nf * b + t * (d * nV + nE) + d * nV] = np.sqrt(self.elems[t].meas)
            null /= np.linalg.norm(null)
        return K, rhs, null

    def errors(self, field, local_vecs):
        """L2 errors: P u_h, grad P u_h, element pressure p_T (means removed
        for all-Dirichlet problems) and the divergence of the element velocity
        u_T, which Scheme 2 makes zero pointwise."""
        k, d, nV, nE = self.k, self.d, self.nV, self.nE
        q = 2 * k + 2
        eu = egu = ep = ediv = 0.0
        pm_h = pm_x = vol = 0.0
        cache = []
        for t, L in enumerate(self.local):
            eg, eb = self.elems[t], self.ebases[t]
            X, W = eg.rule(q)
            ev, egr = eb.eval_grad(X)
            U = local_vecs[t]
            ph = ev[:, :nE] @ U[L.nvec:L.nvec + nE]
            px = field.p(X)
            pm_h += W @ ph
            pm_x += W @ px
            vol += W.sum()
            cache.append((W, ph, px))
            ux, gux = field.u(X), field.grad_u(X)
            div = np.zeros(X.shape[0])
            for c in range(d):
                coef = L.P @ U[L.vmap[c]]
                uh = ev @ coef
                guh = np.einsum("qnd,n->qd", egr, coef)
                eu += W @ (uh - ux[:, c]) ** 2
                egu += W @ np.sum((guh - gux[:, c, :]) ** 2, axis=1)
                div += egr[:, :nV, c] @ U[c * nV:(c + 1) * nV]
            ediv += W @ div ** 2
        shift = not self.mesh.has_neumann()
        for W, ph, px in cache:
            if shift:
                ph = ph - pm_h / vol
                px = px - pm_x / vol
            ep += W @ (ph - px) ** 2
        return dict(u=np.sqrt(eu), gu=np.sqrt(egu), p=np.sqrt(ep), div=np.sqrt(ediv))
