"""p-multilevel V-cycle preconditioner and FGMRES (oracle), Secs. 3 and 4.2.

* Transfers (Sec. 3.1, Eq. def:restOp; Sec. 4.2): with hierarchical
  orthonormal bases the restriction keeps, per face and per velocity component,
  the first dim P^{k_{l+1}}_{d-1} coefficients, and per element the first
  n_P(k_{l+1}) pressure coefficients (n_P = 1 for v&p-cond); prolongation is
  its transpose (zero padding).  Uncondensed, every element block is d+1
  components (velocity, pressure) truncated the same way.  For HHO-hp (Scheme 2) the face pressure is one
  more face component truncated the same way, and there are no element rows.
* Coarse operators (Sec. 4.2): S^{l+1} = I^{l+1}_l S^l I^l_{l+1}, formed here
  as a sparse triple product with the selection matrix.
* V-cycle (Sec. 3.3, Algorithm MG_V): pre-smooth, restrict the defect, solve
  (l+1 = L) or recurse with a zero guess, prolongate and correct, post-smooth.
* Smoother (Sec. 3.3 / Sec. 5.2.2, two GMRES iterations): reading - the ILU
  preconditioner is replaced by a block-Jacobi preconditioner: exact inverses of
  the face diagonal blocks and, for the element pressure rows (whose mean-mode
  diagonal entry is exactly zero), inverses of the pivot block that a block
  ILU(0) with faces ordered before pressures would produce when only the face
  diagonal blocks are kept: M_T = S_TT - sum_{F in F_T} S_TF S_FF^{-1} S_FT.
  Right preconditioning, initial guess = current iterate.
* Coarse solver (Sec. 5.2.2 uses LU in 2D): an exact solve of the coarse
  system, c = S_L^{-1} d.  Dense LU when n_L <= 10^4 (with a rank-one fix
  alpha n n^T on the constant-pressure kernel n of all-Dirichlet problems),
  otherwise a sparse LU of S_L (the kernel pinned by alpha on the diagonal of
  the first mean-pressure unknown, then the result projected on the complement
  of n).  Both give the unique solution orthogonal to n.  The block-Jacobi
  GMRES variant (to a 1e-3 relative residual) is kept as an option.
* FGMRES (Sec. 3.3): right-preconditioned flexible GMRES, one V-cycle per
  iteration, classical Gram-Schmidt applied twice (CGS2), x0 = 0, restart 50.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .basis import dim_P


def n_comp(d, cond):
    """Components of a face block: d velocity components, plus the face
    pressure for HHO-hp (Scheme 2)."""
    if cond == "dg":  # the DG scheme has element unknowns only
        return 0
    return d + 1 if cond == "hp" else d


def n_pres(d, k_l, cond):
    """Kept unknowns per element: the mean pressure for v&p-cond, all of
    P^k_l for v-cond, none for HHO-hp (its element pressure is eliminated),
    the d velocity components and the pressure (d+1 blocks of P^k_l) when
    nothing is condensed."""
    if cond == "hp":
        return 0
    if cond in ("unc", "dg"):
        return (d + 1) * dim_P(d, k_l)
    return 1 if cond == "vp" else dim_P(d, k_l)


def e_comp(d, cond):
    """Components of an element block, each truncated on its own: d + 1
    (velocity and pressure) when nothing is condensed, else 1 (the kept
    pressure coefficients form one prefix)."""
    return d + 1 if cond in ("unc", "dg") else 1


def mean_offset(d, k_l, cond):
    """Position of the constant pressure mode in an element block."""
    return d * dim_P(d, k_l) if cond in ("unc", "dg") else 0


class Level:
    """One level of the hierarchy: matrix, block layout and smoother data."""

    def __init__(self, S, mesh, d, k_l, cond, n_elem_faces):
        self.S = S.tocsr()
        self.k = k_l
        self.nF = dim_P(d - 1, k_l)
        self.b = n_comp(d, cond) * self.nF
        self.nP = n_pres(d, k_l, cond)
        self.nf = mesh.n_face
        self.ne = mesh.n_elem
        self.n = self.nf * self.b + self.ne * self.nP
        assert S.shape == (self.n, self.n)
        self.mesh = mesh
        self._jacobi()

    def face_slice(self, F):
        return slice(F * self.b, (F + 1) * self.b)

    def elem_slice(self, T):
        o = self.nf * self.b + T * self.nP
        return slice(o, o + self.nP)

    def _jacobi(self):
        """Block-Jacobi inverses (reading of the ILU smoother preconditioner)."""
        S = self.S
        self.Dinv = []
        for F in range(self.nf):
            sl = self.face_slice(F)
            self.Dinv.append(np.linalg.inv(S[sl, sl].toarray()))
        self.Minv = []
        for T in range(self.ne if self.nP > 0 else 0):
            st = self.elem_slice(T)
            M = S[st, st].toarray()
            for F in self.mesh.faces_of(T):
                sf = self.face_slice(int(F))
                M -= S[st, sf].toarray() @ self.Dinv[int(F)] @ S[sf, st].toarray()
            self.Minv.append(np.linalg.inv(M))

    def precond(self, r):
        z = np.empty_like(r)
        for F in range(self.nf):
            sl = self.face_slice(F)
            z[sl] = self.Dinv[F] @ r[sl]
        for T in range(len(self.Minv)):
            st = self.elem_slice(T)
            z[st] = self.Minv[T] @ r[st]
        return z


def restriction(mesh, d, k_fine, k_coarse, cond):
    """Selection matrix I^{l+1}_l (Sec. 4.2: unit-diagonal local restrictions)."""
    nFf, nFc = dim_P(d - 1, k_fine), dim_P(d - 1, k_coarse)
    nc_ = n_comp(d, cond)
    bf, bc = nc_ * nFf, nc_ * nFc
    nPf, nPc = n_pres(d, k_fine, cond), n_pres(d, k_coarse, cond)
    rows, cols = [], []
    for F in range(mesh.n_face):
        for c in range(nc_):
            for j in range(nFc):
                rows.append(F * bc + c * nFc + j)
                cols.append(F * bf + c * nFf + j)
    ec = e_comp(d, cond)
    nEc, nEf = nPc // ec if ec else 0, nPf // ec if ec else 0
    for T in range(mesh.n_elem):
        for c in range(ec):
            for i in range(nEc):
                rows.append(mesh.n_face * bc + T * nPc + c * nEc + i)
                cols.append(mesh.n_face * bf + T * nPf + c * nEf + i)
    nc = mesh.n_face * bc + mesh.n_elem * nPc
    nf_ = mesh.n_face * bf + mesh.n_elem * nPf
    return sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(nc, nf_))


def gmres_steps(A, precond, b, x0, m, x0_zero=False):
    """m iterations of right-preconditioned GMRES from x0 (the smoother).

    Arnoldi with classical Gram-Schmidt applied twice; the small least-squares
    problem is solved by a library least-squares routine.  Stops early on an
    exact (zero) subdiagonal.
    """
    r = b.copy() if x0_zero else b - A @ x0
    beta = np.linalg.norm(r)
    if beta == 0.0:
        return x0.copy()
    V = [r / beta]
    Z = []
    H = np.zeros((m + 1, m))
    j_end = m
    for j in range(m):
        Z.append(precond(V[j]))
        w = A @ Z[j]
        Vm = np.stack(V, axis=1)
        h1 = Vm.T @ w
        w = w - Vm @ h1
        h2 = Vm.T @ w
        w = w - Vm @ h2
        H[:j + 1, j] = h1 + h2
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] == 0.0:
            j_end = j + 1
            break
        V.append(w / H[j + 1, j])
    e1 = np.zeros(j_end + 1)
    e1[0] = beta
    y = np.linalg.lstsq(H[:j_end + 1, :j_end], e1, rcond=None)[0]
    x = x0.copy()
    for j in range(j_end):
        x = x + y[j] * Z[j]
    return x


def gmres_solve(A, precond, b, rtol, restart=50, maxit=1000):
    """Right-preconditioned GMRES(restart) from x0 = 0 to ||r|| <= rtol ||b||.

    Returns (x, iterations).  The residual estimate of the Arnoldi relation is
    used for the stopping test.
    """
    x = np.zeros_like(b)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0
    it = 0
    r = b.copy()
    while it < maxit:
        beta = np.linalg.norm(r)
        if beta <= rtol * bnorm:
            break
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart))
        y = None
        for j in range(restart):
            Z.append(precond(V[j]))
            w = A @ Z[j]
            Vm = np.stack(V, axis=1)
            h1 = Vm.T @ w
            w = w - Vm @ h1
            h2 = Vm.T @ w
            w = w - Vm @ h2
            H[:j + 1, j] = h1 + h2
            H[j + 1, j] = np.linalg.norm(w)
            it += 1
            e1 = np.zeros(j + 2)
            e1[0] = beta
            y, res = _lsq(H[:j + 2, :j + 1], e1)
            if res <= rtol * bnorm or H[j + 1, j] == 0.0 or it >= maxit:
                break
            V.append(w / H[j + 1, j])
        for i in range(len(y)):
            x = x + y[i] * Z[i]
        r = b - A @ x
        if res <= rtol * bnorm:
            break
    return x, it


def _lsq(H, e1):
    y = np.linalg.lstsq(H, e1, rcond=None)[0]
    return y, float(np.linalg.norm(e1 - H @ y))


class PMG:
    """Hierarchy of Galerkin-inherited levels and the V-cycle (Sec. 3.3)."""

    def __init__(self, hho, degrees, smooth_its=2, coarse="auto", coarse_rtol=1e-3,
                 lu_max=10000, smoother="jacobi"):
        assert degrees[0] == hho.k and all(a > b for a, b in zip(degrees, degrees[1:]))
        self.hho = hho
        self.degrees = list(degrees)
        self.m = smooth_its
        mesh, d, cond = hho.mesh, hho.d, hho.cond
        self.levels = []
        self.R = []
        S = hho.S
        for l, kl in enumerate(degrees):
            if l > 0:
                R = restriction(mesh, d, degrees[l - 1], kl, cond)
                self.R.append(R)
                S = (R @ S @ R.T).tocsr()
            self.levels.append(Level(S, mesh, d, kl, cond, None))
        if smoother == "ilu":  # block ILU(0), multicolour faces then pressures (oracle/ilu.py)
            from .ilu import BlockILU
            for lev in self.levels[:-1]:
                lev.ilu = BlockILU(lev.S, mesh, lev.b, lev.nP)
                lev.precond = lev.ilu.apply
        L = self.levels[-1]
        self.coarse_rtol = coarse_rtol
        if coarse == "auto":
            coarse = "lu" if L.n <= lu_max else "splu"
        self.coarse = coarse
        self.null = None
        if not mesh.has_neumann():
            n = np.zeros(L.n)
            if cond == "hp":  # constant hybrid pressure: the constant mode of every face pressure
                for F in range(L.nf):
                    n[F * L.b + d * L.nF] = np.sqrt(hho.faces[F].meas)
            else:
                off = mean_offset(d, L.k, cond)
                for T in range(L.ne):
                    n[L.elem_slice(T).start + off] = np.sqrt(hho.elems[T].meas)
            self.null = n / np.linalg.norm(n)
        if coarse == "lu":
            A = L.S.toarray()
            if self.null is not None:
                alpha = float(np.mean(np.abs(np.diag(A))))
                A = A + alpha * np.outer(self.null, self.null)
            self.lu = sla.lu_factor(A)
        elif coarse == "splu":
            A = L.S.tocsc().astype(np.float64)
            if self.null is not None:
                alpha = float(np.mean(np.abs(A.diagonal())))
                pin = d * L.nF if cond == "hp" else L.elem_slice(0).start + mean_offset(d, L.k, cond)
                A = (A + sp.csc_matrix(([alpha], ([pin], [pin])), shape=A.shape)).tocsc()
            self.splu = spla.splu(A)
        self.coarse_its = []

    def coarse_solve(self, d):
        L = self.levels[-1]
        if self.coarse == "lu":
            return sla.lu_solve(self.lu, d)
        if self.coarse == "splu":
            c = self.splu.solve(d)
            if self.null is not None:
                c = c - (self.null @ c) * self.null
            self.coarse_its.append(1)
            return c
        c, its = gmres_solve(L.S, L.precond, d, self.coarse_rtol)
        self.coarse_its.append(its)
        return c

    def vcycle(self, l, b, w=None):
        """MG_V(l, b, w) of the Algorithm in Sec. 3.3."""
        lev = self.levels[l]
        zero = w is None
        if zero:
            w = np.zeros(lev.n)
        w = gmres_steps(lev.S, lev.precond, b, w, self.m, x0_zero=zero)
        dvec = self.R[l] @ (b - lev.S @ w)
        if l + 1 == len(self.levels) - 1:
            c = self.coarse_solve(dvec)
        else:
            c = self.vcycle(l + 1, dvec)
        w = w + self.R[l].T @ c
        w = gmres_steps(lev.S, lev.precond, b, w, self.m)
        return w

    def apply(self, r):
        return self.vcycle(0, r)


def fgmres(A, apply_prec, b, rtol=1e-8, restart=50, maxit=1000, null=None):
    """Flexible GMRES with right preconditioning (Sec. 3.3), CGS2, x0 = 0.

    Stops when the Arnoldi residual estimate satisfies ||r|| <= rtol ||b||;
    then recomputes the true residual and restarts if it is above the
    tolerance.  With a null vector the right-hand side is projected first.
    Returns (x, iterations, true relative residual).
    """
    if null is not None:
        b = b - (null @ b) * null
    bnorm = np.linalg.norm(b)
    x = np.zeros_like(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    it = 0
    r = b.copy()
    while it < maxit:
        beta = np.linalg.norm(r)
        if beta <= rtol * bnorm:
            break
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart))
        for j in range(restart):
            Z.append(apply_prec(V[j]))
            w = A @ Z[j]
            Vm = np.stack(V, axis=1)
            h1 = Vm.T @ w
            w = w - Vm @ h1
            h2 = Vm.T @ w
            w = w - Vm @ h2
            H[:j + 1, j] = h1 + h2
            H[j + 1, j] = np.linalg.norm(w)
            it += 1
            e1 = np.zeros(j + 2)
            e1[0] = beta
            y, res = _lsq(H[:j + 2, :j + 1], e1)
            if res <= rtol * bnorm or H[j + 1, j] == 0.0 or it >= maxit:
                break
            V.append(w / H[j + 1, j])
        for i in range(len(y)):
            x = x + y[i] * Z[i]
        r = b - A @ x
    if null is not None:
        x = x - (null @ x) * null
    return x, it, float(np.linalg.norm(b - A @ x) / bnorm)
