"""Planted mistakes: each test plants one plausible mistake in the oracle (on
the CPU, by patching it for the duration of the test) and checks that one of
the oracle's pins fails.  The pins are the same functions the CPU suite runs
on the unmodified oracle; here they must raise.  Kinds of mistakes covered: a
dropped term (the Nitsche penalty, the BR2 penalty), a wrong sign (one of the
two pressure-coupling blocks, the smoother's pressure pivot, the printed sign
of the DG pressure stabilisation), a wrong orientation (an inward normal), a
wrong index (the restriction keeping the wrong coefficients), too low a
quadrature order, a dropped sweep (the ILU forward solve), a dropped factor in
a gradient, truncation in place of round-to-nearest-even."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle.dg as odg
import oracle.geometry as ogeo
import oracle.hho as ohho
import oracle.ilu as oilu
import oracle.pmg as opmg
import test_oracle_dg as pins_dg
import test_oracle_hho as pins_hho
import test_oracle_hp as pins_hp
import test_oracle_ilu as pins_ilu
import test_oracle_mlp as pins_mlp
import test_oracle_pmg as pins_pmg
import test_oracle_quadrature_basis as pins_quad


def _fails(pin, *args):
    with pytest.raises(AssertionError):
        pin(*args)


def _flip_first_normal(monkeypatch, module):
    """An inward normal on the first face of every element (an orientation slip)."""
    real = module.mesh_geometry

    def wrong(mesh):
        elems, faces = real(mesh)
        for e in elems:
            e.nTF[0] = -e.nTF[0]
        return elems, faces
    monkeypatch.setattr(module, "mesh_geometry", wrong)


# --- Scheme 1 (HHO-dp) ---

def test_dropped_nitsche_penalty_breaks_coercivity(monkeypatch):
    monkeypatch.setattr(ohho, "penalty", lambda *a: 0.0)
    _fails(pins_hho.test_velocity_block_coercive)


def test_sign_slip_in_one_coupling_block(monkeypatch):
    """-B^T in the momentum rows while the mass rows keep B."""
    real = ohho.LocalSystem.__init__

    def wrong(self, hho, t):
        real(self, hho, t)
        self.K[:self.nvec, self.nvec:] *= -1.0
    monkeypatch.setattr(ohho.LocalSystem, "__init__", wrong)
    _fails(pins_hho.test_condensed_operator_symmetric_and_zero_mean_diagonal, "v")
    _fails(pins_hho.test_polynomial_reproduction_2d, "tri-neu", pins_hho.MESHES_2D[2][1], "vp", 1)


def test_inward_normal(monkeypatch):
    _flip_first_normal(monkeypatch, ohho)
    _fails(pins_hho.test_polynomial_reproduction_2d, "quad-dir", pins_hho.MESHES_2D[0][1], "v", 2)


@pytest.mark.filterwarnings("ignore")  # the broken rules make singular Gram matrices and systems
@pytest.mark.parametrize("cls", [ogeo.ElemGeom, ogeo.FaceGeom], ids=["element", "face"])
def test_quadrature_order_halved(monkeypatch, cls):
    """A rule of half the requested order.  On elements the discrete scheme stays
    polynomially consistent (every volume term uses the same inexact rule), so
    only the rules' own exactness pin sees it; on faces reproduction fails too."""
    real = cls.rule
    monkeypatch.setattr(cls, "rule", lambda self, p: real(self, max(p // 2, 1)))
    tri = lambda: pins_quad.tri_mesh(3, jitter=0.3, seed=2)  # noqa: E731
    _fails(pins_quad.test_element_and_face_rules_exact_to_their_order, tri)
    if cls is ogeo.FaceGeom:
        _fails(pins_hho.test_polynomial_reproduction_2d, "tri-dir", pins_hho.MESHES_2D[1][1], "v", 2)


# --- Scheme 2 (HHO-hp) ---

def test_hp_inward_normal(monkeypatch):
    _flip_first_normal(monkeypatch, ogeo)
    _fails(pins_hp.test_polynomial_solution_reproduced, "quad3", 1)


# --- p-multilevel hierarchy and smoother ---

def test_restriction_keeps_the_wrong_coefficients(monkeypatch):
    """Each truncated component keeps coefficients 1..n_c instead of 0..n_c-1."""
    real = opmg.restriction

    def wrong(mesh, d, k_fine, k_coarse, cond):
        R = real(mesh, d, k_fine, k_coarse, cond).tocoo()
        return sp.csr_matrix((R.data, (R.row, R.col + 1)), shape=R.shape)
    monkeypatch.setattr(opmg, "restriction", wrong)
    monkeypatch.setattr(pins_pmg, "restriction", wrong)
    _fails(pins_pmg.test_restriction_is_unit_diagonal_and_galerkin_is_extraction, "v")


def test_pressure_pivot_sign_slip(monkeypatch):
    """M_T = S_TT + sum_F S_TF S_FF^-1 S_FT instead of the Schur complement."""
    def wrong(self):
        S = self.S
        self.Dinv = [np.linalg.inv(S[self.face_slice(F), self.face_slice(F)].toarray()) for F in range(self.nf)]
        self.Minv = []
        for T in range(self.ne if self.nP > 0 else 0):
            st = self.elem_slice(T)
            M = S[st, st].toarray()
            for F in self.mesh.faces_of(T):
                sf = self.face_slice(int(F))
                M += S[st, sf].toarray() @ self.Dinv[int(F)] @ S[sf, st].toarray()
            self.Minv.append(np.linalg.inv(M))
    monkeypatch.setattr(opmg.Level, "_jacobi", wrong)
    _fails(pins_pmg.test_jacobi_pivot_blocks_equal_ilu_pivots_without_face_coupling, "v",
           lambda: pins_pmg.quad_mesh(3, 3, jitter=0.15, seed=2))


def test_ilu_apply_without_the_forward_sweep(monkeypatch):
    """z = U^-1 v instead of U^-1 L^-1 v."""
    def wrong(self, v):
        z = np.array(v, dtype=float)
        sl, pat, rank, B = self.sl, self.pat, self.rank, self.blocks
        for i in reversed(self.order):
            s = z[sl(i)].copy()
            for j in pat[i]:
                if rank[j] > rank[i]:
                    s -= B[(i, j)] @ z[sl(j)]
            z[sl(i)] = np.linalg.solve(B[(i, i)], s)
        return z
    monkeypatch.setattr(oilu.BlockILU, "apply", wrong)
    _fails(pins_ilu.test_single_element_is_exact, "vp")


# --- DG scheme (Scheme 3) ---

def test_dg_inward_normal(monkeypatch):
    _flip_first_normal(monkeypatch, odg)
    _fails(pins_dg.test_dg_polynomial_solution_reproduced, "quad3", 1)


def test_dg_dropped_br2_penalty(monkeypatch):
    monkeypatch.setattr(odg.DG, "_eta", lambda self, F: 0.0)
    _fails(pins_dg.test_dg_symmetry_kernel_inertia, False)


def test_dg_printed_stabilisation_sign(monkeypatch):
    """The jump stabilisation with the printed sign (+h_F int [p] q_T): adds
    2 h_F int [p] q_T to the oracle's reading on every interior face."""
    real = odg.DG._build

    def wrong(self):
        real(self)
        d, nE, nb, mesh = self.d, self.nE, self.nb, self.mesh
        S = self.S.tolil()
        pre = d * nE + np.arange(nE)
        for F in range(mesh.n_face):
            T1, T2 = (int(t) for t in mesh.face_elem[F])
            if T2 < 0:
                continue
            _, X, W = self._face_side(F, T1)
            v = {T: self.ebases[T].eval(X)[:, :nE] for T in (T1, T2)}
            for Sx in (T1, T2):
                for Tx in (T1, T2):
                    sgn = 1.0 if Sx == Tx else -1.0
                    M = 2.0 * self.faces[F].hF * sgn * np.einsum("q,qa,qb->ab", W, v[Sx], v[Tx])
                    r, c = Sx * nb + pre, Tx * nb + pre
                    S[np.ix_(r, c)] = S[np.ix_(r, c)].toarray() + M
        self.S = S.tocsr()
    monkeypatch.setattr(odg.DG, "_build", wrong)
    _fails(pins_dg.test_dg_symmetry_kernel_inertia, True)


# --- learned-smoother oracle ---

def test_mlp_gradient_without_the_factor_two(monkeypatch):
    """d|D|^2 = 2 D dD: the gradients of the loss with the 2 dropped."""
    real = pins_mlp.loss_and_grads

    def wrong(*args):
        loss, g = real(*args)
        return loss, {k: 0.5 * v for k, v in g.items()}
    monkeypatch.setattr(pins_mlp, "loss_and_grads", wrong)
    _fails(pins_mlp.test_gradients_match_finite_differences)


def test_bf16_truncation_instead_of_rounding(monkeypatch):
    def truncate(a):
        u = np.asarray(a, dtype=np.float32).copy().view(np.uint32) & np.uint32(0xFFFF0000)
        return u.view(np.float32).astype(np.float64)
    monkeypatch.setattr(pins_mlp, "bf16_round", truncate)
    _fails(pins_mlp.test_bf16_rounding)
