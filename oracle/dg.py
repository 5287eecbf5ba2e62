"""DG scheme (Scheme 3 of Sec. 2.4): BR2 discretisation of the vector
Laplacian with a stabilised equal-order pressure coupling; element unknowns
only (oracle).

Test infrastructure: only tests, the smoke check and the bench's CPU baseline
use this module.

Unknowns per element: u_T in P^k(T)^d and p_T in P^k(T), one block of
(d+1) n_E coefficients [U_T (d components, n_E each) | P_T] in the
orthonormal element basis; the global vector is these blocks in element
order.  The global operator couples an element with itself and with its face
neighbours.

Readings of the paper:
* The BR2 terms act on every velocity component separately (the vector
  Laplacian), with the lifting L_FT(phi) in P^k(T)^d defined by
  int_T L_FT(phi) . tau = 1/2 int_F phi (tau . n_TF); the jump is
  u_T - u_T' on interior faces and 2 (u_T - g_D) on Dirichlet faces, averages
  are traces on boundary faces, and Neumann faces carry no BR2 term.
* Penalty: eta_F = max(N_T, N_T') + 1 on interior faces and N_T + 1 on
  Dirichlet faces (N = number of faces), just above the paper's bounds.
* The printed mass residual sums the velocity-average term over interior and
  Dirichlet faces with the trace of u_T on Dirichlet faces and no boundary
  datum.  We read it as: interior faces {u} . n q_T; Neumann faces u_T . n q_T;
  Dirichlet faces g_D . n q_T (the datum, as Scheme 1 carries it), which makes
  the pressure-velocity coupling the transpose of the momentum's and the
  scheme consistent.
* The pressure stabilisation h_F int_F [p] q_T enters the mass equation with
  the sign that makes the pressure Schur complement definite (the momentum
  pressure term is -int p div v, so the stabilisation is subtracted); the
  printed sign gives an indefinite pressure block.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .basis import dim_P, element_basis
from .geometry import mesh_geometry

DGCOND = "dg"


class DG:
    """Scheme 3 on a mesh: assembled operator, right-hand side, solves, errors."""

    def __init__(self, mesh, k):
        assert k >= 1
        self.mesh, self.k, self.d = mesh, k, mesh.dim
        self.cond = DGCOND
        self.elems, self.faces = mesh_geometry(mesh)
        self.ebases = [element_basis(e, k) for e in self.elems]
        self.nE = dim_P(self.d, k)
        self.nb = (self.d + 1) * self.nE
        self.ndof = mesh.n_elem * self.nb
        self.q = 2 * k + 2
        self._build()

    # --- helpers ---
    def _eta(self, F):
        T1, T2 = self.mesh.face_elem[F]
        n1 = len(self.mesh.faces_of(int(T1)))
        if T2 < 0:
            return n1 + 1.0
        return max(n1, len(self.mesh.faces_of(int(T2)))) + 1.0

    def _face_side(self, F, T):
        """Outward normal of element T on face F and the quadrature of F."""
        eg = self.elems[T]
        loc = list(self.mesh.faces_of(T)).index(F)
        X, W = self.faces[F].rule(self.q)
        return eg.nTF[loc], X, W

    def _build(self):
        d, nE, nb, mesh = self.d, self.nE, self.nb, self.mesh
        ne = mesh.n_elem
        blocks = {}

        def add(i, j, M):
            if (i, j) in blocks:
                blocks[(i, j)] += M
            else:
                blocks[(i, j)] = M.copy()

        vel = lambda c: slice(c * nE, (c + 1) * nE)
        pre = slice(d * nE, (d + 1) * nE)
        # volume terms
        for T in range(ne):
            eg, eb = self.elems[T], self.ebases[T]
            X, W = eg.rule(self.q)
            v, g = eb.eval_grad(X)  # (nq, nE), (nq, nE, d)
            K = np.einsum("q,qad,qbd->ab", W, g, g)
            M = np.zeros((nb, nb))
            for c in range(d):
                M[vel(c), vel(c)] += K
                # -int p div v: row v_c (test a), column p (trial b)
                Bc = -np.einsum("q,qa,qb->ab", W, g[:, :, c], v)
                M[vel(c), pre] += Bc
                M[pre, vel(c)] += Bc.T  # mass: int u . grad q  ->  -int div u q + boundary terms below
            add(T, T, M)
        # the mass term int_T u . grad q equals -int_T q div u + int_dT u.n q; we assembled -int q div u
        # (symmetric with the momentum) and add the boundary parts face by face below
        for F in range(mesh.n_face):
            T1, T2 = (int(t) for t in mesh.face_elem[F])
            bc = mesh.face_bc[F]
            fg = self.faces[F]
            if bc == 2:  # Neumann: only the mass boundary part int u_T.n q_T - int u_T.n q_T = 0
                continue
            sides = [T1] if T2 < 0 else [T1, T2]
            n1, X, W = self._face_side(F, T1)
            tr = {}
            for T in sides:
                v, g = self.ebases[T].eval_grad(X)
                tr[T] = (v, g)
            eta = self._eta(F)
            hF = fg.hF
            # jump operator J_T: [u]_{T1 F} = sum_T s_T u_T (s = +1, -1 interior; 2 on Dirichlet)
            sgn = {T1: 2.0} if T2 < 0 else {T1: 1.0, T2: -1.0}
            # liftings of the jump on each side: L_{F,S}([u]_{S F}) coefficients, for a trial basis function
            # phi_b of element T (component c): jump value s_T phi_b (oriented from S's side: [u]_{S F} =
            # (+/-) [u]_{T1 F}); lift coefficient (c', a) on S = 1/2 int phi * phi^S_a n_{S,c'}
            nS = {T1: n1}
            if T2 >= 0:
                nS[T2] = -n1
            for S in sides:
                for T in sides:
                    # orientation: [u]_{S F} = o_S [u]_{T1 F}, o = +1 for T1, -1 for T2
                    o = 1.0 if S == T1 else -1.0
                    vS, gS = tr[S]
                    vT, gT = tr[T]
                    # Lift matrix Lm[c', a, b]: coefficient (c', a) of L_{F S}(o s_T phi_b^T) (scalar jump,
                    # one velocity component at a time)
                    Lm = 0.5 * o * sgn[T] * np.einsum("q,qa,qb,c->cab", W, vS, vT, nS[S])
                    # (a) -int_S L_{F S}([u]) . grad v_S  (test a of S):
                    # int_S L . grad phi_a^S = sum_c' sum_e L[c', e] int_S phi_e^S d_c' phi_a^S
                    Xe, We = self.elems[S].rule(self.q)
                    ve, ge = self.ebases[S].eval_grad(Xe)
                    Dv = np.einsum("q,qe,qac->cea", We, ve, ge)  # int phi_e d_c phi_a
                    A1 = -np.einsum("cea,ceb->ab", Dv, Lm)
                    # (c) + eta int_F n_{S F} . {L_F([u])} v_S: {L} = 1/2 (L_{F T1} + L_{F T2}) interior, trace
                    # on Dirichlet faces; contributions of side R's lifting evaluated on F
                    A3 = np.zeros((nE, nE))
                    for R in sides:
                        oR = 1.0 if R == T1 else -1.0
                        vR, _ = tr[R]
                        LmR = 0.5 * oR * sgn[T] * np.einsum("q,qa,qb,c->cab", W, vR, vT, nS[R])
                        wavg = 0.5 if len(sides) == 2 else 1.0
                        # value of L_{F R} on F: sum_e L[c, e] phi_e^R(x); dotted with n_{S F}
                        Lval = np.einsum("cab,qa,c->qb", LmR, vR, nS[S])  # (nq, nb_trial)
                        A3 += eta * wavg * np.einsum("q,qa,qb->ab", W, vS, Lval)
                    # (b) - int_F n_{S F} . {grad u} v_S: {grad u} = 1/2 (grad u_T1 + grad u_T2) interior, trace
                    wavg = 0.5 if len(sides) == 2 else 1.0
                    A2 = -wavg * np.einsum("q,qa,qbc,c->ab", W, vS, gT, nS[S])
                    Mv = A1 + A2 + A3
                    M = np.zeros((nb, nb))
                    for c in range(d):
                        M[vel(c), vel(c)] = Mv
                    # pressure: + int_F {p} v_S . n_{S F}  (test v_S comp c, trial p_T)
                    for c in range(d):
                        M[vel(c), pre] += wavg * nS[S][c] * np.einsum("q,qa,qb->ab", W, vS, vT)
                    # mass: int_S u . grad q = -int_S q div u + int_dS u_S . n q (the volume part is above);
                    # interior faces add int_F (u_S - {u}) . n_{S F} q_S, Dirichlet faces int_F u_S . n q_S (their
                    # - int g_D . n q_S goes to the right-hand side), Neumann faces nothing (the boundary part
                    # cancels the residual's - int u_S . n q_S)
                    for c in range(d):
                        Mq = nS[S][c] * np.einsum("q,qa,qb->ab", W, vS, vT)
                        if len(sides) == 2:
                            Mq = (0.5 if S == T else -0.5) * Mq
                        M[pre, vel(c)] += Mq
                    # stabilisation - h_F int_F [p]_{S F} q_S (interior faces)
                    if len(sides) == 2:
                        sT = 1.0 if T == S else -1.0
                        M[pre, pre] -= hF * sT * np.einsum("q,qa,qb->ab", W, vS, vT)
                    add(S, T, M)
        rows, cols, vals = [], [], []
        for (i, j), M in blocks.items():
            r = i * nb + np.arange(nb)
            c = j * nb + np.arange(nb)
            rows.append(np.repeat(r, nb))
            cols.append(np.tile(c, nb))
            vals.append(M.ravel())
        self.S = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(self.ndof, self.ndof))
        self.blocks = blocks

    def data_nodes(self):
        elem = [e.rule(self.q)[0] for e in self.elems]
        face = [f.rule(self.q)[0] for f in self.faces]
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
                n = self.elems[T].nTF[list(self.mesh.faces_of(T)).index(F.id)]
                gN[F.id] = field.g_neumann(face[F.id], np.tile(n, (face[F.id].shape[0], 1)))
        return f_vals, gD, gN

    def assemble_rhs(self, f_vals, gD, gN):
        d, nE, nb, mesh = self.d, self.nE, self.nb, self.mesh
        b = np.zeros(self.ndof)
        for T in range(mesh.n_elem):
            X, W = self.elems[T].rule(self.q)
            v = self.ebases[T].eval(X)
            for c in range(d):
                b[T * nb + c * nE + np.arange(nE)] += v.T @ (W * f_vals[T][:, c])
        for F in range(mesh.n_face):
            bc = mesh.face_bc[F]
            if bc == 0:
                continue
            T = int(mesh.face_elem[F, 0])
            n, X, W = self._face_side(F, T)
            v, g = self.ebases[T].eval_grad(X)
            if bc == 2:
                for c in range(d):
                    b[T * nb + c * nE + np.arange(nE)] += v.T @ (W * gN[F][:, c])
                continue
            gd = gD[F]
            eta = self._eta(F)
            # the Dirichlet jump 2 (u_T - g_D): the g_D part of the BR2 terms moves to the right-hand side
            Xe, We = self.elems[T].rule(self.q)
            ve, ge = self.ebases[T].eval_grad(Xe)
            Dv = np.einsum("q,qe,qac->cea", We, ve, ge)
            for c in range(d):
                # lifting of -2 g_D (component c): coefficients L[c', e] = 1/2 int_F (-2 g_c) phi_e n_c'
                L = 0.5 * np.einsum("q,q,qe,k->ke", W, -2.0 * gd[:, c], v, n)
                a1 = -np.einsum("kea,ke->a", Dv, L)
                Lval = np.einsum("ke,qe,k->q", L, v, n)
                a3 = eta * np.einsum("q,qa,q->a", W, v, Lval)
                b[T * nb + c * nE + np.arange(nE)] -= a1 + a3
            # mass: the residual's - int g_D . n q_T moves to the right-hand side
            b[T * nb + d * nE + np.arange(nE)] += v.T @ (W * (gd @ n))
        return b

    def null_vector(self):
        if self.mesh.has_neumann():
            return None
        n = np.zeros(self.ndof)
        for T in range(self.mesh.n_elem):
            n[T * self.nb + self.d * self.nE] = np.sqrt(self.elems[T].meas)
        return n / np.linalg.norm(n)

    def direct_solve(self, rhs):
        n = self.null_vector()
        A = self.S
        if n is not None:
            alpha = float(np.mean(np.abs(A.diagonal())))
            A = A + alpha * sp.csr_matrix(np.outer(n, n))
            rhs = rhs - (n @ rhs) * n
        return spla.spsolve(A.tocsc(), rhs)

    def errors(self, field, x):
        d, nE, nb = self.d, self.nE, self.nb
        eu = egu = ep = ediv = 0.0
        pm_h = pm_x = vol = 0.0
        cache = []
        for T in range(self.mesh.n_elem):
            X, W = self.elems[T].rule(self.q)
            v, g = self.ebases[T].eval_grad(X)
            U = x[T * nb:(T + 1) * nb]
            ux, gux = field.u(X), field.grad_u(X)
            div = np.zeros(X.shape[0])
            for c in range(d):
                coef = U[c * nE:(c + 1) * nE]
                eu += W @ (v @ coef - ux[:, c]) ** 2
                egu += W @ np.sum((np.einsum("qad,a->qd", g, coef) - gux[:, c, :]) ** 2, axis=1)
                div += g[:, :, c] @ coef
            ediv += W @ div ** 2
            ph, px = v @ U[d * nE:], field.p(X)
            pm_h += W @ ph
            pm_x += W @ px
            vol += W.sum()
            cache.append((W, ph, px))
        shift = not self.mesh.has_neumann()
        for W, ph, px in cache:
            if shift:
                ph, px = ph - pm_h / vol, px - pm_x / vol
            ep += W @ (ph - px) ** 2
        return dict(u=np.sqrt(eu), gu=np.sqrt(egu), p=np.sqrt(ep), div=np.sqrt(ediv))
