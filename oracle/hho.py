"""HHO-dp (Scheme 1, equal order k' = k) local operators, static condensation,
assembly, direct solves, recovery and error norms (oracle).

Follows Sec. 2.2 (reconstruction p_T^{k+1}, face residual r_TF), Sec. 2.3.1
(local residuals, Eq. HHOdiscr:residuals), Sec. 4.1.1 (local algebraic system,
Eq. def:HHOAB) and Sec. 4.1.2 (v-cond Eq. ST.1, v&p-cond Eqs. zero-residual.T
and ST.2).

Local unknown ordering (vector): [U_T | U_F1 .. U_FN | P_T] with U_T = the d
components of v_T one after the other (n_E coefficients each), U_F = the d
components of v_F one after the other (n_F each), P_T = n_E pressure
coefficients whose first is the mean mode (the constant basis function).

Global condensed ordering: one block of b = d*n_F per face (component-major),
then one block of n_P per element (n_P = 1 for v&p-cond, n_E for v-cond).
Uncondensed ("unc", Sec. 5.4's reference formulation): the same face blocks,
then one block of n_P = (d+1) n_E per element, [U_T (d components) | P_T].

Readings of the paper:
* Penalty (Eq. HHOdiscrMNT, "eta large enough"): eta_F = 4 (k+1)(k+d)/d |F| h_F / |T|.
* Neumann datum: the residual subtracts int g_N . v_F, which is consistent with
  g_N = (grad u - p I) n (the problem statement prints the opposite sign).
* Dirichlet datum: the momentum residual must contain + int g_D . (n . grad P v)
  - eta/h_F int g_D . v_F to cancel the symmetric consistency and penalty terms
  at u_F = g_D; the printed residual carries the first term with a minus sign.
* The Dirichlet-datum term int g_D . (n . grad P v) depends on every local
  velocity unknown through the reconstruction, so the momentum right-hand side
  has entries on U_T as well as on U_dT.
* Eq. ST.2 writes 0 for the right-hand side of the eliminated high-order
  pressure rows; we carry the high-order part of G-hat there, which vanishes
  only when g_D . n has no high-order content (needed for exact consistency).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from .basis import dim_P, element_basis, face_basis
from .geometry import mesh_geometry

VCOND = "v"
VPCOND = "vp"
UNCOND = "unc"  # uncondensed (the reference point of Sec. 5.4): nothing eliminated


def penalty(k, d, meas_F, h_F, meas_T):
    """Nitsche penalty eta_F (reading of Eq. HHOdiscrMNT)."""
    return 4.0 * (k + 1) * (k + d) / d * meas_F * h_F / meas_T


class LocalSystem:
    """Local matrices of one element (Eq. def:HHOAB) plus the reconstruction."""

    def __init__(self, hho, t):
        self.t = t
        k, d = hho.k, hho.d
        eg = hho.elems[t]
        eb = hho.ebases[t]
        nR, nE, nF = dim_P(d, k + 1), dim_P(d, k), dim_P(d - 1, k)
        N = len(eg.faces)
        ns = nE + N * nF
        self.nE, self.nF, self.N, self.ns = nE, nF, N, ns
        q_op = 2 * k + 2

        # --- scalar potential reconstruction p_T^{k+1} (Sec. 2.2.1) ---
        X, W = eg.rule(q_op)
        ev, eg_ = eb.eval_grad(X)
        Kst = np.einsum("q,qid,qjd->ij", W, eg_, eg_)
        Rhs = np.zeros((nR, ns))
        Rhs[:, :nE] = Kst[:, :nE]
        face_data = []
        for f, F in enumerate(eg.faces):
            n = eg.nTF[f]
            Xf, Wf = F.rule(q_op)
            fv, fg = eb.eval_grad(Xf)
            dn = fg @ n
            psi = hho.fbases[F.id].eval(Xf)
            sl = slice(nE + f * nF, nE + (f + 1) * nF)
            Rhs[:, sl] += np.einsum("q,qi,qj->ij", Wf, dn, psi)
            Rhs[:, :nE] -= np.einsum("q,qi,qj->ij", Wf, dn, fv[:, :nE])
            face_data.append((n, Wf, fv, dn, psi, sl))
        P = np.zeros((nR, ns))
        P[0, 0] = 1.0  # mean of p_T v equals mean of v_T; phi_0 is the constant
        P[1:, :] = np.linalg.solve(Kst[1:, 1:], Rhs[1:, :])
        self.P = P

        # --- viscous bilinear form of Eq. HHOdiscrMNT (scalar, one component) ---
        A = P.T @ Kst @ P
        ET = np.zeros((nE, ns))
        ET[:, :nE] = np.eye(nE)
        for f, F in enumerate(eg.faces):
            n, Wf, fv, dn, psi, sl = face_data[f]
            EF = np.zeros((nF, ns))
            EF[:, sl] = np.eye(nF)
            MFT = np.einsum("q,qj,qm->jm", Wf, psi, fv)
            # face residual r_TF = pi_F(v_F - p v) - pi_T^k(v_T - p v), at face nodes
            r = psi @ (EF - MFT @ P) - fv[:, :nE] @ (ET - P[:nE, :])
            A += (r.T * Wf) @ r / F.hF
            if hho.mesh.face_bc[F.id] == 1:
                eta = penalty(k, d, F.meas, F.hF, eg.meas)
                G = dn @ P
                V = psi @ EF
                A += -(V.T * Wf) @ G - (G.T * Wf) @ V + eta / F.hF * (V.T * Wf) @ V
        self.A_scalar = A

        # --- vector layout ---
        nvec = d * nE + N * d * nF
        self.nvec = nvec
        vmap = np.zeros((d, ns), dtype=np.int64)
        for c in range(d):
            vmap[c, :nE] = c * nE + np.arange(nE)
            for f in range(N):
                vmap[c, nE + f * nF: nE + (f + 1) * nF] = d * nE + f * d * nF + c * nF + np.arange(nF)
        self.vmap = vmap
        Avec = np.zeros((nvec, nvec))
        for c in range(d):
            Avec[np.ix_(vmap[c], vmap[c])] = A

        # --- pressure-velocity coupling (first line of Eq. HHOdiscrCNT) ---
        B = np.zeros((nE, nvec))
        for c in range(d):
            B[:, c * nE:(c + 1) * nE] -= np.einsum("q,qi,qj->ij", W, ev[:, :nE], eg_[:, :nE, c])
        for f, F in enumerate(eg.faces):
            n, Wf, fv, dn, psi, sl = face_data[f]
            for c in range(d):
                B[:, c * nE:(c + 1) * nE] += n[c] * np.einsum("q,qi,qj->ij", Wf, fv[:, :nE], fv[:, :nE])
                if hho.mesh.face_bc[F.id] != 1:
                    cols = d * nE + f * d * nF + c * nF + np.arange(nF)
                    B[:, cols] -= n[c] * np.einsum("q,qi,qj->ij", Wf, fv[:, :nE], psi)
        self.B = B
        K = np.zeros((nvec + nE, nvec + nE))
        K[:nvec, :nvec] = Avec
        K[nvec:, :nvec] = B
        K[:nvec, nvec:] = B.T
        self.K = K

    def rhs(self, hho, f_vals, gD_vals, gN_vals):
        """Right-hand side of Eq. def:HHOAB from data values at the data nodes."""
        k, d = hho.k, hho.d
        eg, eb = hho.elems[self.t], hho.ebases[self.t]
        nE, nF = self.nE, self.nF
        q_dat = 2 * k + 2
        b = np.zeros(self.nvec + nE)
        X, W = eg.rule(q_dat)
        ev = eb.eval(X, nE)
        fv = f_vals[self.t]
        for c in range(d):
            b[c * nE:(c + 1) * nE] += ev.T @ (W * fv[:, c])
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
                    cols = d * nE + f * d * nF + c * nF + np.arange(nF)
                    b[cols] += eta / F.hF * (psi.T @ (Wf * g[:, c]))
                b[self.nvec:] += fvv[:, :nE].T @ (Wf * (g @ n))
            else:
                g = gN_vals[F.id]
                for c in range(d):
                    cols = d * nE + f * d * nF + c * nF + np.arange(nF)
                    b[cols] += psi.T @ (Wf * g[:, c])
        return b

    def split(self, cond):
        """Eliminated and kept local index sets (Eq. ST.1 / Eq. zero-residual.T)."""
        nE = self.nE
        nUT = self.vmap.shape[0] * nE
        UT = list(range(nUT))
        UdT = list(range(nUT, self.nvec))
        Pidx = [self.nvec + i for i in range(nE)]
        if cond == UNCOND:
            return [], UdT + UT + Pidx
        if cond == VCOND:
            return UT, UdT + Pidx
        return UT + Pidx[1:], UdT + Pidx[:1]


def schur(K, rhs, elim, keep):
    """Schur complement of the eliminated block: S = K_kk - K_ke K_ee^{-1} K_ek."""
    if not elim:  # nothing eliminated (uncondensed)
        S = K[np.ix_(keep, keep)]
        return S, (None if rhs is None else rhs[keep]), np.zeros((0, len(keep))), (None if rhs is None else np.zeros(0))
    Kee = K[np.ix_(elim, elim)]
    Kek = K[np.ix_(elim, keep)]
    Kke = K[np.ix_(keep, elim)]
    X = np.linalg.solve(Kee, Kek)
    S = K[np.ix_(keep, keep)] - Kke @ X
    if rhs is None:
        return S, None, X, None
    y = np.linalg.solve(Kee, rhs[elim])
    g = rhs[keep] - Kke @ y
    return S, g, X, y


class HHO:
    """Discretisation of the Stokes problem (Eq. stokesProb) by Scheme 1."""

    def __init__(self, mesh, k, cond=VPCOND):
        self.mesh = mesh
        self.k = k
        self.d = mesh.dim
        self.cond = cond
        self.elems, self.faces = mesh_geometry(mesh)
        self.ebases = [element_basis(e, k + 1) for e in self.elems]
        self.fbases = [face_basis(f, k) for f in self.faces]
        self.nE = dim_P(self.d, k)
        self.nF = dim_P(self.d - 1, k)
        self.b = self.d * self.nF
        self.nP = 1 if cond == VPCOND else (self.d + 1) * self.nE if cond == UNCOND else self.nE
        self.local = [LocalSystem(self, t) for t in range(mesh.n_elem)]
        self.n_face_dofs = mesh.n_face * self.b
        self.ndof = self.n_face_dofs + mesh.n_elem * self.nP
        self._condense()

    # --- quadrature nodes where the data are evaluated (degree 2k+2: exact for the
    # polynomial data of the consistency pins; the paper does not fix it) ---
    def data_nodes(self):
        q = 2 * self.k + 2
        elem = [e.rule(q)[0] for e in self.elems]
        face = [f.rule(q)[0] for f in self.faces]
        return elem, face

    def data_values(self, field):
        elem, face = self.data_nodes()
        f_vals = [field.f(X) for X in elem]
        gD, gN = {}, {}
        for F in self.faces:
            bc = self.mesh.face_bc[F.id]
            if bc == 1:
                gD[F.id] = field.u(face[F.id])
            elif bc == 2:
                T = self.mesh.face_elem[F.id, 0]
                eg = self.elems[T]
                n = eg.nTF[list(self.mesh.faces_of(T)).index(F.id)]
                gN[F.id] = field.g_neumann(face[F.id], np.tile(n, (face[F.id].shape[0], 1)))
        return f_vals, gD, gN

    def global_kept(self, t):
        """Global indices of the kept local unknowns of element t."""
        d, nF, b = self.d, self.nF, self.b
        idx = []
        for F in self.mesh.faces_of(t):
            idx.extend(int(F) * b + np.arange(b))
        idx.extend(self.n_face_dofs + t * self.nP + np.arange(self.nP))
        return np.array(idx, dtype=np.int64)

    def _condense(self):
        rows, cols, vals = [], [], []
        self.S_T = []
        self.elim_ops = []
        for t, L in enumerate(self.local):
            elim, keep = L.split(self.cond)
            S, _, X, _ = schur(L.K, None, elim, keep)
            self.S_T.append(S)
            self.elim_ops.append((elim, keep, X))
            g = self.global_kept(t)
            rows.append(np.repeat(g, len(g)))
            cols.append(np.tile(g, len(g)))
            vals.append(S.ravel())
        self.S = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(self.ndof, self.ndof))

    def assemble_rhs(self, f_vals, gD, gN):
        """Condensed right-hand side (Eq. ST.1 / Eq. ST.2) and local RHS for recovery."""
        rhs = np.zeros(self.ndof)
        self.local_rhs = []
        for t, L in enumerate(self.local):
            r = L.rhs(self, f_vals, gD, gN)
            self.local_rhs.append(r)
            elim, keep, X = self.elim_ops[t]
            y = np.linalg.solve(L.K[np.ix_(elim, elim)], r[elim]) if elim else np.zeros(0)
            g = r[keep] - L.K[np.ix_(keep, elim)] @ y
            rhs[self.global_kept(t)] += g
        return rhs

    # --- pressure null space of the all-Dirichlet problem ---
    def null_vector(self):
        """Constant-pressure kernel vector (None when a Neumann face exists)."""
        if self.mesh.has_neumann():
            return None
        n = np.zeros(self.ndof)
        off = self.d * self.nE if self.cond == UNCOND else 0  # the mean pressure in the element block
        for t in range(self.mesh.n_elem):
            n[self.n_face_dofs + t * self.nP + off] = np.sqrt(self.elems[t].meas)
        return n / np.linalg.norm(n)

    def direct_solve(self, rhs):
        """Sparse direct solve of the condensed system (rank-one fix on the null space)."""
        n = self.null_vector()
        A = self.S
        if n is not None:
            alpha = float(np.mean(np.abs(A.diagonal())))
            A = (A + alpha * sp.csr_matrix(np.outer(n, n))).tocsc()
            rhs = rhs - (n @ rhs) * n
        return spla.spsolve(A.tocsc(), rhs)

    # --- uncondensed system (cross-check of the condensation) ---
    def uncondensed(self, f_vals, gD, gN):
        d, nE, b = self.d, self.nE, self.b
        nf, ne = self.mesh.n_face, self.mesh.n_elem
        n_tot = nf * b + ne * d * nE + ne * nE
        rows, cols, vals = [], [], []
        rhs = np.zeros(n_tot)
        for t, L in enumerate(self.local):
            g = np.concatenate([nf * b + t * d * nE + np.arange(d * nE),
                                np.concatenate([int(F) * b + np.arange(b) for F in self.mesh.faces_of(t)]),
                                nf * b + ne * d * nE + t * nE + np.arange(nE)])
            rows.append(np.repeat(g, len(g)))
            cols.append(np.tile(g, len(g)))
            vals.append(L.K.ravel())
            rhs[g] += L.rhs(self, f_vals, gD, gN)
        K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n_tot, n_tot))
        null = None
        if not self.mesh.has_neumann():
            null = np.zeros(n_tot)
            for t in range(ne):
                null[nf * b + ne * d * nE + t * nE] = np.sqrt(self.elems[t].meas)
            null /= np.linalg.norm(null)
        return K, rhs, null

    def solve_uncondensed(self, f_vals, gD, gN):
        K, rhs, null = self.uncondensed(f_vals, gD, gN)
        if null is not None:
            alpha = float(np.mean(np.abs(K.diagonal())))
            K = K + alpha * sp.csr_matrix(np.outer(null, null))
            rhs = rhs - (null @ rhs) * null
        return spla.spsolve(K.tocsc(), rhs)

    # --- recovery of the eliminated unknowns (back-substitution) ---
    def recover(self, x):
        """Full local vectors [U_T | U_dT | P_T] per element from the condensed solution."""
        out = []
        for t, L in enumerate(self.local):
            elim, keep, X = self.elim_ops[t]
            xk = x[self.global_kept(t)]
            r = self.local_rhs[t]
            y = np.linalg.solve(L.K[np.ix_(elim, elim)], r[elim]) if elim else np.zeros(0)
            full = np.zeros(L.K.shape[0])
            full[keep] = xk
            full[elim] = y - X @ xk
            out.append(full)
        return out

    def errors(self, field, local_vecs):
        """L2 errors (Sec. 5.2.2): P u_h, grad P u_h, p_h (mean removed), div u_T.

        Reading: the velocity error uses the reconstruction P_T^{k+1} u_T; the
        divergence error uses the element velocity u_T; the pressure of an
        all-Dirichlet problem is compared after removing both means.
        """
        k, d, nE = self.k, self.d, self.nE
        q = 2 * self.k + 2
        eu = egu = ep = ediv = 0.0
        pm_h = pm_x = vol = 0.0
        cache = []
        for t, L in enumerate(self.local):
            eg, eb = self.elems[t], self.ebases[t]
            X, W = eg.rule(q)
            ev, egr = eb.eval_grad(X)
            U = local_vecs[t]
            ph = ev[:, :nE] @ U[L.nvec:]
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
                div += egr[:, :nE, c] @ U[c * nE:(c + 1) * nE]
            ediv += W @ div ** 2
        shift = not self.mesh.has_neumann()
        for W, ph, px in cache:
            if shift:
                ph = ph - pm_h / vol
                px = px - pm_x / vol
            ep += W @ (ph - px) ** 2
        return dict(u=np.sqrt(eu), gu=np.sqrt(egu), p=np.sqrt(ep), div=np.sqrt(ediv))
