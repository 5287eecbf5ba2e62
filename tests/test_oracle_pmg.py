"""Pins of the oracle's p-multilevel solver (Secs. 3 and 4.2): explicit
projection matrices, Galerkin coarse operators, the GMRES smoother's residual
minimisation, closed forms of the two-level correction, and FGMRES versus a
direct solve."""
import numpy as np
import pytest

from oracle.basis import dim_P, element_basis, face_basis
from oracle.hho import HHO
from oracle.pmg import PMG, fgmres, gmres_steps, restriction
from synthetic import quad_mesh, tri_mesh, fields


def _explicit_restriction(h, k_f, k_c):
    """I^{l+1}_l from the integrals int psi_i^{l+1} psi_j^l over every face and element."""
    m, d = h.mesh, h.d
    nFf, nFc = dim_P(d - 1, k_f), dim_P(d - 1, k_c)
    nPf = 1 if h.cond == "vp" else dim_P(d, k_f)
    nPc = 1 if h.cond == "vp" else dim_P(d, k_c)
    nf, ne = m.n_face, m.n_elem
    R = np.zeros((nf * d * nFc + ne * nPc, nf * d * nFf + ne * nPf))
    for F in h.faces:
        # independent bases of degree k_f and k_c built on this face
        Bf, Bc = face_basis(F, k_f), face_basis(F, k_c)
        X, W = F.rule(2 * k_f + 2)
        I = Bc.eval(X).T @ (W[:, None] * Bf.eval(X))
        for c in range(d):
            R[np.ix_(F.id * d * nFc + c * nFc + np.arange(nFc), F.id * d * nFf + c * nFf + np.arange(nFf))] = I
    for e in h.elems:
        Bf, Bc = element_basis(e, k_f), element_basis(e, k_c)
        X, W = e.rule(2 * k_f + 2)
        I = Bc.eval(X).T @ (W[:, None] * Bf.eval(X))
        R[np.ix_(nf * d * nFc + e.id * nPc + np.arange(nPc), nf * d * nFf + e.id * nPf + np.arange(nPf))] = I[:nPc, :nPf]
    return R


@pytest.mark.parametrize("cond", ["vp", "v"])
def test_restriction_is_unit_diagonal_and_galerkin_is_extraction(cond):
    h = HHO(tri_mesh(2, jitter=0.2, seed=3), 3, cond)
    S = h.S.toarray()
    for k_f, k_c in ((3, 2), (3, 1), (2, 0)):
        R = restriction(h.mesh, 2, k_f, k_c, cond).toarray()
        Rx = _explicit_restriction(h, k_f, k_c)
        assert np.abs(R - Rx).max() < 1e-13
    pmg = PMG(h, [3, 2, 1, 0], coarse="lu")
    Sl = S
    for l in range(1, 4):
        Rx = _explicit_restriction(h, pmg.degrees[l - 1], pmg.degrees[l])
        Sl = Rx @ Sl @ Rx.T
        got = pmg.levels[l].S.toarray()
        assert np.abs(got - Sl).max() < 1e-13 * np.abs(S).max()


def test_gmres_smoother_minimises_over_krylov_space():
    h = HHO(tri_mesh(3, jitter=0.2, seed=3, neumann_sides=(1,)), 2, "v")
    pmg = PMG(h, [2, 1, 0])
    lev = pmg.levels[0]
    rng = np.random.default_rng(1)
    b = rng.standard_normal(lev.n)
    x0 = rng.standard_normal(lev.n)
    x = gmres_steps(lev.S, lev.precond, b, x0, 2)
    # brute force: min over y of ||b - S (x0 + Z y)||, Z = [M^-1 r0, M^-1 S M^-1 r0]
    S = lev.S.toarray()
    r0 = b - S @ x0
    z1 = lev.precond(r0)
    z2 = lev.precond(S @ z1)
    Z = np.stack([z1, z2], axis=1)
    y = np.linalg.lstsq(S @ Z, r0, rcond=None)[0]
    ref = x0 + Z @ y
    assert np.linalg.norm(x - ref) < 1e-9 * np.linalg.norm(ref)


@pytest.mark.parametrize("cond", ["vp", "v"])
def test_two_level_correction_closed_forms(cond):
    """With no smoothing the V-cycle is I^T S_L^{-1} I b; on S I^T c it returns I^T c."""
    h = HHO(tri_mesh(3, jitter=0.2, seed=3, neumann_sides=(1,)), 2, cond)
    pmg = PMG(h, [2, 0], smooth_its=0, coarse="lu")
    R = pmg.R[0].toarray()
    SL = pmg.levels[1].S.toarray()
    rng = np.random.default_rng(2)
    b = rng.standard_normal(h.ndof)
    z = pmg.apply(b)
    ref = R.T @ np.linalg.solve(SL, R @ b)
    assert np.linalg.norm(z - ref) < 1e-10 * np.linalg.norm(ref)
    c = rng.standard_normal(SL.shape[0])
    z = pmg.apply(h.S @ (R.T @ c))
    assert np.linalg.norm(z - R.T @ c) < 1e-9 * np.linalg.norm(c)


def test_smoother_with_full_krylov_space_is_exact():
    h = HHO(quad_mesh(2), 1, "v")
    pmg = PMG(h, [1, 0])
    lev = pmg.levels[0]
    rng = np.random.default_rng(3)
    b = lev.S @ rng.standard_normal(lev.n)
    x = gmres_steps(lev.S, lev.precond, b, np.zeros(lev.n), lev.n, x0_zero=True)
    assert np.linalg.norm(lev.S @ x - b) < 1e-8 * np.linalg.norm(b)


@pytest.mark.parametrize("mk,cond", [(lambda: quad_mesh(4), "vp"),
                                     (lambda: tri_mesh(4, jitter=0.2, seed=1, neumann_sides=(1,)), "v")])
def test_fgmres_matches_direct_solve(mk, cond):
    h = HHO(mk(), 3, cond)
    rhs = h.assemble_rhs(*h.data_values(fields.TrigStokes2D()))
    pmg = PMG(h, [3, 2, 1, 0])
    x, it, rr = fgmres(h.S, pmg.apply, rhs, rtol=1e-12, null=h.null_vector())
    xd = h.direct_solve(rhs)
    assert rr <= 1e-12
    assert np.linalg.norm(x - xd) < 1e-8 * np.linalg.norm(xd)


def test_iteration_counts_mesh_independent_vcond():
    """Near h-independence of the FGMRES count on uniform meshes (Sec. 5.5)."""
    its = []
    for n in (4, 8, 16):
        h = HHO(quad_mesh(n), 2, "v")
        rhs = h.assemble_rhs(*h.data_values(fields.TrigStokes2D()))
        pmg = PMG(h, [2, 1, 0])
        _, it, _ = fgmres(h.S, pmg.apply, rhs, rtol=1e-8, null=h.null_vector())
        its.append(it)
    assert its[-1] <= its[0] + 6, its


def _dense_block_jacobi(S, mesh, b, nP):
    """The smoother preconditioner (face diagonal blocks, element pressure pivot
    blocks S_TT - sum_F S_TF S_FF^-1 S_FT) as one dense matrix, from index sets
    of its own."""
    nf = mesh.n_face
    Minv = np.zeros_like(S)
    fidx = [np.arange(F * b, (F + 1) * b) for F in range(nf)]
    for F in range(nf):
        Minv[np.ix_(fidx[F], fidx[F])] = np.linalg.inv(S[np.ix_(fidx[F], fidx[F])])
    for T in range(mesh.n_elem):
        t = nf * b + T * nP + np.arange(nP)
        M = S[np.ix_(t, t)].copy()
        for F in mesh.faces_of(T):
            f = fidx[int(F)]
            M -= S[np.ix_(t, f)] @ np.linalg.solve(S[np.ix_(f, f)], S[np.ix_(f, t)])
        Minv[np.ix_(t, t)] = np.linalg.inv(M)
    return Minv


def _dense_smooth(S, Minv, b, x0, m):
    """m GMRES iterations with right preconditioning as an explicit least-squares
    problem over the monomial Krylov basis of S Minv (no Arnoldi)."""
    r0 = b - S @ x0
    K = [r0]
    for _ in range(m - 1):
        K.append(S @ (Minv @ K[-1]))
    Z = Minv @ np.stack(K, axis=1)
    y = np.linalg.lstsq(S @ Z, r0, rcond=None)[0]
    return x0 + Z @ y


@pytest.mark.parametrize("cond", ["v", "vp"])
def test_vcycle_against_dense_brute_force(cond):
    """One V-cycle (Algorithm MG_V, Sec. 3.3) on three levels with two smoothing
    iterations, against a dense restatement: dense Galerkin operators, dense
    block-Jacobi preconditioners, smoothing by explicit Krylov least squares,
    dense coarse solve."""
    mesh = tri_mesh(3, 2, jitter=0.2, seed=11, neumann_sides=(1,))
    h = HHO(mesh, 2, cond)
    degrees = [2, 1, 0]
    pmg = PMG(h, degrees, smooth_its=2, coarse="lu")
    Rs = [restriction(mesh, 2, degrees[l], degrees[l + 1], cond).toarray() for l in range(2)]
    Ss = [h.S.toarray()]
    for R in Rs:
        Ss.append(R @ Ss[-1] @ R.T)
    Ms = [_dense_block_jacobi(Ss[l], mesh, pmg.levels[l].b, pmg.levels[l].nP) for l in range(2)]
    rng = np.random.default_rng(12)
    for l in range(2):  # the oracle's preconditioner is the dense one
        v = rng.standard_normal(Ss[l].shape[0])
        assert np.linalg.norm(pmg.levels[l].precond(v) - Ms[l] @ v) < 1e-11 * np.linalg.norm(Ms[l] @ v)

    def vcycle(l, b):
        w = _dense_smooth(Ss[l], Ms[l], b, np.zeros_like(b), 2)
        d = Rs[l] @ (b - Ss[l] @ w)
        c = np.linalg.solve(Ss[l + 1], d) if l + 1 == 2 else vcycle(l + 1, d)
        w = w + Rs[l].T @ c
        return _dense_smooth(Ss[l], Ms[l], b, w, 2)

    b = rng.standard_normal(h.ndof)
    ref = vcycle(0, b)
    z = pmg.apply(b)
    assert np.linalg.norm(z - ref) < 1e-9 * np.linalg.norm(ref)


@pytest.mark.parametrize("cond", ["vp", "v"])
@pytest.mark.parametrize("mk", [lambda: tri_mesh(4, 3, jitter=0.2, seed=6, neumann_sides=(1,)),
                                lambda: quad_mesh(3, 3, jitter=0.15, seed=2)])
def test_jacobi_pivot_blocks_equal_ilu_pivots_without_face_coupling(cond, mk):
    """The smoother's element pressure pivot M_T (reading of the ILU smoother of
    Sec. 5.2.2) checked by a different algorithm: block ILU(0) (faces before
    pressures, IKJ elimination) applied to S with every face-face block off the
    diagonal set to zero performs exactly the eliminations that define M_T, so
    its element pivot blocks must be M_T and its face pivots the face diagonal
    blocks.  A sign slip or a dropped face in Level._jacobi fails this."""
    import scipy.sparse as sps
    from oracle.ilu import BlockILU
    h = HHO(mk(), 2, cond)
    pmg = PMG(h, [2, 1], coarse="lu")
    for lev in pmg.levels:
        S = lev.S.tolil(copy=True)
        nfb = lev.nf * lev.b
        A = S.toarray()
        for F in range(lev.nf):
            for G in range(lev.nf):
                if F != G:
                    A[F * lev.b:(F + 1) * lev.b, G * lev.b:(G + 1) * lev.b] = 0.0
        ilu = BlockILU(sps.csr_matrix(A), h.mesh, lev.b, lev.nP)
        scale = np.abs(A).max()
        for F in range(lev.nf):
            piv = ilu.blocks[(("f", F), ("f", F))]
            assert np.abs(piv - A[F * lev.b:(F + 1) * lev.b, F * lev.b:(F + 1) * lev.b]).max() == 0.0
            assert np.abs(np.linalg.inv(piv) - lev.Dinv[F]).max() <= 1e-12 * np.abs(lev.Dinv[F]).max()
        for T in range(lev.ne):
            piv = ilu.blocks[(("e", T), ("e", T))]
            M = np.linalg.inv(lev.Minv[T])
            assert np.abs(piv - M).max() <= 1e-12 * scale, (T, piv, M)
        assert nfb + lev.ne * lev.nP == lev.n


@pytest.mark.parametrize("cond", ["vp", "v"])
def test_sparse_lu_coarse_branch_equals_dense_rank_one_lu(cond):
    """The sparse direct coarse solve (alpha pin on one mean pressure, then
    projection on the complement of the pressure kernel n) against the dense LU
    with the rank-one term alpha n n^T, on an all-Dirichlet level: after
    projecting both on the complement of n they agree, solve S c = d for every
    d orthogonal to n, and are orthogonal to n themselves."""
    h = HHO(quad_mesh(4, 3, jitter=0.15, seed=9), 2, cond)
    degrees = [2, 1, 0]
    dense = PMG(h, degrees, coarse="lu")
    sparse = PMG(h, degrees, coarse="splu")
    L = dense.levels[-1]
    n = dense.null
    assert n is not None and sparse.null is not None
    S = L.S.toarray()
    assert np.linalg.norm(S @ n) <= 1e-12 * np.abs(S).max()  # n spans the kernel
    rng = np.random.default_rng(4)
    for _ in range(3):
        d = rng.standard_normal(L.n)
        d -= (n @ d) * n
        c_dense = dense.coarse_solve(d)
        c_dense = c_dense - (n @ c_dense) * n
        c_sparse = sparse.coarse_solve(d)
        assert abs(n @ c_sparse) <= 1e-12 * np.linalg.norm(c_sparse)
        assert np.linalg.norm(c_sparse - c_dense) <= 1e-10 * np.linalg.norm(c_dense)
        assert np.linalg.norm(S @ c_sparse - d) <= 1e-11 * np.linalg.norm(d)
