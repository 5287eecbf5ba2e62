"""Degenerate cases of the method on the GPU, against the oracle.

* one element with every face on the boundary, one of them Neumann (a lone
  all-Dirichlet element is excluded: its smoother pivot block is singular);
* a single-level hierarchy (the V-cycle is the exact coarse solve, FGMRES
  converges in one iteration);
* a zero right-hand side (FGMRES returns x = 0 at once);
* zero smoothing iterations (the V-cycle is transfers and the coarse solve);
* an element with four faces next to triangles (mixed element shapes);
* the restart boundary of FGMRES (restart 1, several cycles);
* maxit reached above the tolerance (status HHO_ERR_NOT_CONVERGED).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.hho import HHO  # noqa: E402
from oracle.pmg import PMG  # noqa: E402
from synthetic import Mesh, tri_mesh, fields  # noqa: E402


@pytest.fixture(scope="module")
def hho_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_13840_gb300 import build, hho
    build.build()
    return hho


def _one_triangle(bc=(2, 1, 1)):
    xyz = np.array([[0.0, 0.0], [1.0, 0.1], [0.2, 0.9]])
    return Mesh(dim=2, xyz=xyz, elem_face_ptr=np.array([0, 3]), elem_face=np.array([0, 1, 2]),
                face_vert_ptr=np.array([0, 2, 4, 6]), face_vert=np.array([0, 1, 1, 2, 2, 0]),
                face_elem=np.array([[0, -1], [0, -1], [0, -1]]), face_bc=np.array(bc, dtype=np.int8),
                face_side=np.array([0, 1, 2], dtype=np.int8))


def _tri_and_quad():
    # a quadrilateral (0,1,2,3) and a triangle (1,4,2) sharing the edge 1-2, Neumann on the triangle's far edges
    xyz = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0], [1.8, 0.4]])
    fv = [(0, 1), (1, 2), (2, 3), (3, 0), (1, 4), (4, 2)]
    face_vert = np.array([v for f in fv for v in f])
    face_vert_ptr = np.arange(0, 2 * len(fv) + 1, 2)
    elem_face = np.array([0, 1, 2, 3, 4, 5, 1])
    elem_face_ptr = np.array([0, 4, 7])
    face_elem = np.array([[0, -1], [0, 1], [0, -1], [0, -1], [1, -1], [1, -1]])
    face_bc = np.array([1, 0, 1, 1, 2, 2], dtype=np.int8)
    return Mesh(dim=2, xyz=xyz, elem_face_ptr=elem_face_ptr, elem_face=elem_face, face_vert_ptr=face_vert_ptr,
                face_vert=face_vert, face_elem=face_elem, face_bc=face_bc,
                face_side=np.array([0, -1, 2, 3, 1, 1], dtype=np.int8))


def _solve_vs_oracle(hho_mod, mesh, k, cond, degrees, smooth_its=2, restart=50):
    fld = fields.TrigStokes2D()
    h = HHO(mesh, k, cond)
    rhs = h.assemble_rhs(*h.data_values(fld))
    xd = h.direct_solve(rhs)
    ctx = hho_mod.Context(mesh, k, cond)
    ctx.assemble(*hho_mod.data_arrays(ctx, fld))
    ctx.pmg_setup(degrees, smooth_its=smooth_its)
    x = torch.empty(ctx.ndof(0), dtype=torch.float64, device="cuda")
    info = ctx.solve(x, rtol=1e-10, restart=restart)
    xs = x.cpu().numpy()
    nv = h.null_vector()
    if nv is not None:
        xs, xd = xs - (nv @ xs) * nv, xd - (nv @ xd) * nv
    err = np.linalg.norm(xs - xd) / max(np.linalg.norm(xd), 1e-300)
    ctx.close()
    return info, err


@pytest.mark.parametrize("cond", ["v", "vp"])
def test_one_element(hho_mod, cond):
    """One element with a Neumann face: the whole hierarchy on 3 faces solves to 1e-10."""
    info, err = _solve_vs_oracle(hho_mod, _one_triangle(), 2, cond, [2, 1, 0])
    assert info["rel_residual"] <= 1e-10 and err < 1e-8, (info, err)


@pytest.mark.parametrize("cond", ["v", "vp"])
def test_single_level_hierarchy(hho_mod, cond):
    mesh = tri_mesh(5, 4, jitter=0.2, seed=1, neumann_sides=(1,))
    info, err = _solve_vs_oracle(hho_mod, mesh, 2, cond, [2])
    assert info["iterations"] == 1 and info["rel_residual"] <= 1e-10 and err < 1e-8, (info, err)


def test_zero_rhs(hho_mod):
    mesh = tri_mesh(4, jitter=0.1, seed=2, neumann_sides=(1,))
    ctx = hho_mod.Context(mesh, 1, "v")
    f, gD, gN = hho_mod.data_arrays(ctx, fields.TrigStokes2D())
    ctx.assemble(torch.zeros_like(f), torch.zeros_like(gD), torch.zeros_like(gN))
    ctx.pmg_setup([1, 0])
    x = torch.full((ctx.ndof(0),), 7.0, dtype=torch.float64, device="cuda")
    info = ctx.solve(x, rtol=1e-8)
    assert info["iterations"] == 0 and torch.all(x == 0.0)
    ctx.close()


@pytest.mark.parametrize("cond", ["v", "vp"])
def test_no_smoothing(hho_mod, cond):
    """m = 0: the V-cycle is restriction, the exact coarse solve and prolongation;
    it equals the oracle's V-cycle with zero smoothing iterations."""
    mesh = tri_mesh(5, 5, jitter=0.2, seed=3, neumann_sides=(1,))
    k = 2
    h = HHO(mesh, k, cond)
    ctx = hho_mod.Context(mesh, k, cond)
    ctx.set_element_schur(np.concatenate([s.ravel() for s in h.S_T]))
    ctx.pmg_setup([2, 1, 0], smooth_its=0)
    pmg = PMG(h, [2, 1, 0], smooth_its=0)
    b = np.random.default_rng(4).standard_normal(ctx.ndof(0))
    z = torch.empty(ctx.ndof(0), dtype=torch.float64, device="cuda")
    ctx.vcycle(torch.from_numpy(b).cuda(), z)
    ref = pmg.apply(b)
    assert np.linalg.norm(z.cpu().numpy() - ref) <= 1e-10 * np.linalg.norm(ref)
    ctx.close()


@pytest.mark.parametrize("cond", ["v", "vp"])
def test_mixed_element_shapes(hho_mod, cond):
    info, err = _solve_vs_oracle(hho_mod, _tri_and_quad(), 3, cond, [3, 2, 1, 0])
    assert info["rel_residual"] <= 1e-10 and err < 1e-8, (info, err)


def test_restart_one(hho_mod):
    """restart = 1: every FGMRES cycle is one V-cycle plus the true-residual restart."""
    mesh = tri_mesh(6, jitter=0.2, seed=5, neumann_sides=(1,))
    info, err = _solve_vs_oracle(hho_mod, mesh, 2, "v", [2, 1, 0], restart=1)
    assert info["rel_residual"] <= 1e-10 and err < 1e-8, (info, err)
    assert info["iterations"] > 1


def test_maxit_reached_reports_not_converged(hho_mod):
    """FGMRES stopped by maxit above the tolerance: HHO_ERR_NOT_CONVERGED (6)
    with the information filled in, and the context stays usable."""
    mesh = tri_mesh(8, jitter=0.2, seed=6, neumann_sides=(1,))
    ctx = hho_mod.Context(mesh, 2, "v")
    ctx.assemble(*hho_mod.data_arrays(ctx, fields.TrigStokes2D()))
    ctx.pmg_setup([2, 1, 0])
    x = torch.empty(ctx.ndof(0), dtype=torch.float64, device="cuda")
    info = ctx.solve(x, rtol=1e-14, maxit=2, raise_on_fail=False)
    assert info["status"] == 6 and info["iterations"] == 2 and info["rel_residual"] > 1e-14, info
    with pytest.raises(hho_mod.HHOError) as exc:
        ctx.solve(x, rtol=1e-14, maxit=2)
    assert exc.value.status == 6
    info = ctx.solve(x, rtol=1e-8)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-8, info
    ctx.close()
