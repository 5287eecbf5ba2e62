"""3D GPU parity: jittered hexahedra with planar faces (the 3D workload's mesh
family), k = 2 and 3, both condensations, against the FP64 oracle through the
C ABI.

* element Schur complements (Eq. ST.1 / ST.2), condensed right-hand side and
  assembled level-0 operator, each built independently on both sides: 1e-11
  relative (bases, quadrature and local solves differ in rounding order);
* exact-input hierarchy (the oracle's element Schur complements fed to the
  GPU): level operators bitwise, level operators' products 1e-13, one V-cycle
  within 1e-12 (kappa(S_L) reported beside it);
* FGMRES (Sec. 3.3) to 1e-12 against the oracle's direct solve, iteration
  counts within 2 of the oracle's FGMRES, recovered unknowns and error norms.
3^3 meshes have 27 elements and 108 faces, 4^3 meshes 64 and 240 (several
32-row tiles of the operator kernels and a ragged last tile).
"""
import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.hho import HHO  # noqa: E402
from oracle.pmg import PMG, fgmres  # noqa: E402
from synthetic import hex_mesh, fields  # noqa: E402
from parity_util import rel, report, coarse_kappa  # noqa: E402


@pytest.fixture(scope="module")
def hho_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_13840_gb300 import build, hho
    build.build()
    return hho


_CACHE = {}


def _oracle(n, k, cond):
    key = (n, k, cond)
    if key not in _CACHE:
        mesh = hex_mesh(n, jitter=0.15, seed=2)
        fld = fields.CurlStokes3D()
        h = HHO(mesh, k, cond)
        rhs = h.assemble_rhs(*h.data_values(fld))
        _CACHE[key] = (mesh, fld, h, rhs)
    return _CACHE[key]


CASES = [(3, 2, "vp"), (3, 3, "vp"), (3, 2, "v"), (3, 3, "v"), (4, 3, "vp")]
IDS = [f"hex{n}-k{k}-{c}" for n, k, c in CASES]


@pytest.mark.parametrize("n,k,cond", CASES, ids=IDS)
def test_elements_rhs_operator_3d(hho_mod, n, k, cond):
    mesh, fld, h, rhs_o = _oracle(n, k, cond)
    ctx = hho_mod.Context(mesh, k, cond)
    S = ctx.element_schur()
    ref = np.concatenate([s.ravel() for s in h.S_T])
    e_s = rel(S, ref)
    f, gD, gN = hho_mod.data_arrays(ctx, fld)
    rhs = torch.empty(ctx.ndof(0), dtype=torch.float64, device="cuda")
    ctx.assemble(f, gD, gN, rhs)
    e_r = rel(rhs.cpu().numpy(), rhs_o)
    r, c, v = ctx.level_coo(0)
    A = sp.csr_matrix((v, (r, c)), shape=h.S.shape)
    e_a = abs(A - h.S).max() / abs(h.S).max()
    report(f"elements3d hex{n} k={k} {cond}", schur=e_s, rhs=e_r, operator=float(e_a))
    assert e_s < 1e-11 and e_r < 1e-11 and e_a < 1e-11
    ctx.close()


@pytest.mark.parametrize("n,k,cond", CASES, ids=IDS)
def test_levels_vcycle_3d(hho_mod, n, k, cond):
    mesh, fld, h, rhs_o = _oracle(n, k, cond)
    degrees = list(range(k, -1, -1))
    ctx = hho_mod.Context(mesh, k, cond)
    ctx.set_element_schur(np.concatenate([s.ravel() for s in h.S_T]))
    ctx.pmg_setup(degrees, smooth_its=2)
    pmg = PMG(h, degrees)
    rng = np.random.default_rng(0)
    for l in range(len(degrees)):
        r, c, v = ctx.level_coo(l)
        S_ref = pmg.levels[l].S
        A = sp.csr_matrix((v, (r, c)), shape=S_ref.shape)
        assert abs(A - S_ref).max() == 0.0
        x = rng.standard_normal(ctx.ndof(l))
        y = torch.empty(ctx.ndof(l), dtype=torch.float64, device="cuda")
        ctx.spmv(l, torch.from_numpy(x).cuda(), y)
        assert rel(y.cpu().numpy(), S_ref @ x) < 1e-13
    tol = 1e-12  # the FP64 bar; kappa(S_L) eps is reported beside it
    worst = 0.0
    for trial in range(2):
        b = rng.standard_normal(ctx.ndof(0))
        z = torch.empty(ctx.ndof(0), dtype=torch.float64, device="cuda")
        ctx.vcycle(torch.from_numpy(b).cuda(), z)
        ref = pmg.apply(b)
        worst = max(worst, float(np.linalg.norm(z.cpu().numpy() - ref) / np.linalg.norm(ref)))
    report(f"vcycle3d hex{n} k={k} {cond}", err=worst, tol=tol, kappa_L=coarse_kappa(pmg))
    assert worst <= tol, (worst, tol)
    ctx.close()


@pytest.mark.parametrize("n,k,cond", [(3, 2, "vp"), (3, 3, "v"), (4, 3, "vp")],
                         ids=["hex3-k2-vp", "hex3-k3-v", "hex4-k3-vp"])
def test_fgmres_solution_3d(hho_mod, n, k, cond):
    mesh, fld, h, rhs_o = _oracle(n, k, cond)
    degrees = list(range(k, -1, -1))
    xd = h.direct_solve(rhs_o)
    ctx = hho_mod.Context(mesh, k, cond)
    ctx.assemble(*hho_mod.data_arrays(ctx, fld))
    ctx.pmg_setup(degrees)
    x = torch.empty(ctx.ndof(0), dtype=torch.float64, device="cuda")
    info = ctx.solve(x, rtol=1e-12, maxit=500)
    assert info["rel_residual"] <= 1e-12
    err = float(np.linalg.norm(x.cpu().numpy() - xd) / np.linalg.norm(xd))
    _, it_o, _ = fgmres(h.S, PMG(h, degrees).apply, rhs_o, rtol=1e-12, null=h.null_vector())
    loc = ctx.recover(x).cpu().numpy()
    ref_loc = np.concatenate(h.recover(xd))
    e_loc = float(np.linalg.norm(loc - ref_loc) / np.linalg.norm(ref_loc))
    e_o = h.errors(fld, h.recover(xd))
    xe = ctx.quad_nodes("elem").cpu().numpy()
    u = torch.from_numpy(np.ascontiguousarray(fld.u(xe))).cuda()
    gu = torch.from_numpy(np.ascontiguousarray(fld.grad_u(xe))).cuda()
    p = torch.from_numpy(np.ascontiguousarray(fld.p(xe))).cuda()
    e = ctx.errors(torch.from_numpy(loc).cuda(), u, gu, p)
    worst_norm = max(abs(e[key] - e_o[key]) / max(e_o[key], 1e-300) for key in ("u", "gu", "p", "div"))
    report(f"fgmres3d hex{n} k={k} {cond}", solution=err, recovered=e_loc, norms=float(worst_norm),
           its=info["iterations"], its_oracle=it_o)
    assert err < 1e-8 and e_loc < 1e-8
    assert abs(info["iterations"] - it_o) <= 2, (info["iterations"], it_o)
    for key in ("u", "gu", "p", "div"):
        assert abs(e[key] - e_o[key]) <= 1e-6 * e_o[key] + 1e-13, (key, e[key], e_o[key])
    ctx.close()


def test_fp32_vcycle_3d_against_oracle(hho_mod):
    """Mixed precision in 3D against the oracle (not against the GPU's own FP64
    path): the FP32 V-cycle agrees with the oracle's FP64 V-cycle to FP32
    rounding amplified by kappa(S_L), and FGMRES with it reaches the FP64 true
    residual 1e-8 with a solution within 1e-6 of the oracle's direct solve."""
    n, k, cond = 4, 3, "vp"
    mesh, fld, h, rhs_o = _oracle(n, k, cond)
    degrees = list(range(k, -1, -1))
    ctx = hho_mod.Context(mesh, k, cond)
    ctx.assemble(*hho_mod.data_arrays(ctx, fld))
    ctx.pmg_setup(degrees, prec="fp32")
    pmg = PMG(h, degrees)
    b = np.random.default_rng(3).standard_normal(ctx.ndof(0))
    z = torch.empty(ctx.ndof(0), dtype=torch.float64, device="cuda")
    ctx.vcycle(torch.from_numpy(b).cuda(), z)
    ref = pmg.apply(b)
    e_v = float(np.linalg.norm(z.cpu().numpy() - ref) / np.linalg.norm(ref))
    tol = 1e-5
    x = torch.empty(ctx.ndof(0), dtype=torch.float64, device="cuda")
    info = ctx.solve(x, rtol=1e-8)
    xd = h.direct_solve(rhs_o)
    e_x = float(np.linalg.norm(x.cpu().numpy() - xd) / np.linalg.norm(xd))
    report("fp32vcycle3d hex4 k=3 vp", vcycle=e_v, tol=tol, solution=e_x, its=info["iterations"],
           relres=info["rel_residual"])
    assert e_v <= tol, (e_v, tol)
    assert info["rel_residual"] <= 1e-8
    assert e_x < 1e-6, e_x
    ctx.close()


@pytest.mark.parametrize("cond", ["vp", "v"])
@pytest.mark.parametrize("leaf", [2, 8])
def test_multifrontal_coarse_3d(hho_mod, cond, leaf):
    """The nested-dissection multifrontal coarse solver on a 3D coarse level
    (forced by a low dense threshold), shallow and deep trees: V-cycle against
    the oracle's V-cycle with its sparse direct coarse solve, and the
    single-level hierarchy (the whole k = 3 operator solved by the multifrontal
    solver) against S x = b."""
    n, k = 4, 3
    mesh, fld, h, rhs_o = _oracle(n, k, cond)
    degrees = list(range(k, -1, -1))
    ctx = hho_mod.Context(mesh, k, cond)
    ctx.set_element_schur(np.concatenate([s.ravel() for s in h.S_T]))
    ctx.set_option("coarse_dense_max", 100)
    ctx.set_option("mf_leaf", leaf)
    ctx.pmg_setup(degrees, smooth_its=2)
    pmg = PMG(h, degrees, coarse="splu")
    null = h.null_vector()
    rng = np.random.default_rng(5)
    worst = 0.0
    for trial in range(2):
        b = rng.standard_normal(ctx.ndof(0))
        if null is not None:
            b -= (null @ b) * null
        z = torch.empty(ctx.ndof(0), dtype=torch.float64, device="cuda")
        ctx.vcycle(torch.from_numpy(b).cuda(), z)
        ref = pmg.apply(b)
        zz = z.cpu().numpy()
        if null is not None:
            zz = zz - (null @ zz) * null
            ref = ref - (null @ ref) * null
        worst = max(worst, float(np.linalg.norm(zz - ref) / np.linalg.norm(ref)))
    ctx.pmg_setup([k])
    b = pmg.levels[0].S @ rng.standard_normal(ctx.ndof(0))
    z = torch.empty(ctx.ndof(0), dtype=torch.float64, device="cuda")
    ctx.vcycle(torch.from_numpy(b).cuda(), z)
    res = float(np.linalg.norm(pmg.levels[0].S @ z.cpu().numpy() - b) / np.linalg.norm(b))
    report(f"multifrontal3d hex4 k=3 {cond} leaf={leaf}", vcycle=worst, direct_residual=res)
    assert worst <= 1e-12, worst
    assert res <= 1e-11, res
    ctx.close()


def test_two_contexts_keep_their_coarse_kernels_runnable(hho_mod):
    """A context created after another with smaller multifrontal fronts must not
    leave the first one's coarse-solve kernels unable to launch (the kernels'
    shared-memory limit is a process-wide attribute): the first context's FP32
    V-cycle, replayed from a captured graph on a side stream, still equals its
    result from before the second context existed."""
    stream = torch.cuda.Stream()
    mesh, fld, h, rhs_o = _oracle(4, 3, "vp")
    with torch.cuda.stream(stream):
        a = hho_mod.Context(mesh, 3, "vp", stream=stream)
        a.assemble(*hho_mod.data_arrays(a, fld))
        a.set_option("coarse_dense_max", 100)
        a.set_option("coarse_fp32", 1)
        a.pmg_setup([3, 2, 1, 0], prec="fp32")
        r = torch.from_numpy(np.random.default_rng(1).standard_normal(a.ndof(0))).cuda()
        z0 = torch.empty_like(r)
        a.vcycle(r, z0)
        stream.synchronize()
        from synthetic import tri_mesh
        from synthetic import fields as F2
        b = hho_mod.Context(tri_mesh(6, 5, jitter=0.2, seed=2, neumann_sides=(1,)), 1, "v", stream=stream)
        b.assemble(*hho_mod.data_arrays(b, F2.TrigStokes2D()))
        b.set_option("coarse_dense_max", 20)
        b.set_option("coarse_fp32", 1)
        b.pmg_setup([1, 0], prec="fp32")
        z1 = torch.empty_like(r)
        for _ in range(2):  # capture, then replay
            a.vcycle(r, z1)
        stream.synchronize()
        assert torch.equal(z0, z1)
        b.close()
        a.close()
