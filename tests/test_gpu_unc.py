"""GPU parity of the uncondensed HHO-dp formulation (Sec. 5.4's reference
point: face blocks, then one [U_T | P_T] block per element, nothing
eliminated) against the FP64 oracle through the C ABI.

* element blocks (the local matrices reordered, built independently on both
  sides), right-hand side and assembled level-0 operator: 1e-11 relative;
* exact-input hierarchy: level operators bitwise (every element component
  truncated on its own), their products 1e-13;
* the V-cycle with the block ILU(0) smoother (the smoother this formulation
  needs: block Jacobi does not converge here) against the oracle's: 1e-12,
  with the dense and with the multifrontal coarse solve (the latter modulo
  the pressure kernel, on kernel-free input, like the oracle's sparse-LU
  branch);
* FGMRES to 1e-12 against the oracle's direct solve and its iteration count,
  the recovered unknowns and the error norms (equal to velocity-only
  condensation's: the same discrete solution);
* the FP32 V-cycle inside FP64 FGMRES to a true residual of 1e-8.
"""
import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.hho import HHO  # noqa: E402
from oracle.pmg import PMG, fgmres  # noqa: E402
from synthetic import quad_mesh, tri_mesh, hex_mesh, fields  # noqa: E402
from parity_util import coarse_kappa, rel, report  # noqa: E402


@pytest.fixture(scope="module")
def hho_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_13840_gb300 import build, hho
    build.build()
    return hho


MESHES = {
    "tri9x8-neu": lambda: tri_mesh(9, 8, jitter=0.2, seed=3, neumann_sides=(1,)),
    "quad9x7-dir": lambda: quad_mesh(9, 7, jitter=0.15, seed=5),
    "hex3-dir": lambda: hex_mesh(3, jitter=0.15, seed=2),
}
_CACHE = {}


def _oracle(name, k):
    key = (name, k)
    if key not in _CACHE:
        mesh = MESHES[name]()
        fld = fields.TrigStokes2D() if mesh.dim == 2 else fields.CurlStokes3D()
        h = HHO(mesh, k, "unc")
        rhs = h.assemble_rhs(*h.data_values(fld))
        _CACHE[key] = (mesh, fld, h, rhs)
    return _CACHE[key]


ELEM = [("tri9x8-neu", 0), ("tri9x8-neu", 1), ("tri9x8-neu", 3), ("quad9x7-dir", 2), ("hex3-dir", 1)]


@pytest.mark.parametrize("name,k", ELEM, ids=[f"{n}-k{k}" for n, k in ELEM])
def test_unc_elements_rhs_operator(hho_mod, name, k):
    mesh, fld, h, rhs_o = _oracle(name, k)
    ctx = hho_mod.Context(mesh, k, "unc")
    assert ctx.ndof(0) == h.ndof
    S = ctx.element_schur()
    ref = np.concatenate([s.ravel() for s in h.S_T])
    assert S.shape == ref.shape
    e_s = rel(S, ref)
    f, gD, gN = hho_mod.data_arrays(ctx, fld)
    rhs = torch.empty(ctx.ndof(0), dtype=torch.float64, device="cuda")
    ctx.assemble(f, gD, gN, rhs)
    e_r = rel(rhs.cpu().numpy(), rhs_o)
    r, c, v = ctx.level_coo(0)
    A = sp.csr_matrix((v, (r, c)), shape=h.S.shape)
    e_a = abs(A - h.S).max() / abs(h.S).max()
    report(f"unc-elements {name} k={k}", schur=e_s, rhs=e_r, operator=float(e_a))
    assert e_s < 1e-11 and e_r < 1e-11 and e_a < 1e-11
    ctx.close()


VC = [("tri9x8-neu", 3, "dense"), ("quad9x7-dir", 3, "dense"), ("quad9x7-dir", 2, "mf"), ("tri9x8-neu", 2, "mf"),
      ("hex3-dir", 1, "dense")]


@pytest.mark.parametrize("name,k,coarse", VC, ids=[f"{n}-k{k}-{c}" for n, k, c in VC])
def test_unc_levels_and_ilu_vcycle(hho_mod, name, k, coarse):
    mesh, fld, h, rhs_o = _oracle(name, k)
    degrees = list(range(k, -1, -1))
    ctx = hho_mod.Context(mesh, k, "unc")
    ctx.set_element_schur(np.concatenate([s.ravel() for s in h.S_T]))
    ctx.set_option("smoother", 1)
    if coarse == "mf":
        ctx.set_option("coarse_dense_max", 1)
        ctx.set_option("mf_leaf", 4)
    ctx.pmg_setup(degrees, smooth_its=2)
    assert ctx.coarse_info()["kind"] == ("multifrontal" if coarse == "mf" else "dense")
    pmg = PMG(h, degrees, smoother="ilu", coarse="splu" if coarse == "mf" else "auto")
    null = h.null_vector() if coarse == "mf" else None
    rng = np.random.default_rng(1)
    for l in range(len(degrees)):
        r, c, v = ctx.level_coo(l)
        S_ref = pmg.levels[l].S
        A = sp.csr_matrix((v, (r, c)), shape=S_ref.shape)
        assert abs(A - S_ref).max() == 0.0, l
        x = rng.standard_normal(ctx.ndof(l))
        y = torch.empty(ctx.ndof(l), dtype=torch.float64, device="cuda")
        ctx.spmv(l, torch.from_numpy(x).cuda(), y)
        assert rel(y.cpu().numpy(), S_ref @ x) < 1e-13
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
    report(f"unc-vcycle-ilu {name} k={k} {coarse}", err=worst, tol=1e-12, kappa_L=coarse_kappa(pmg))
    assert worst <= 1e-12, worst
    ctx.close()


FG = [("tri9x8-neu", 3), ("quad9x7-dir", 2)]


@pytest.mark.parametrize("name,k", FG, ids=[f"{n}-k{k}" for n, k in FG])
def test_unc_fgmres_solution(hho_mod, name, k):
    mesh, fld, h, rhs_o = _oracle(name, k)
    degrees = list(range(k, -1, -1))
    xd = h.direct_solve(rhs_o)
    ctx = hho_mod.Context(mesh, k, "unc")
    ctx.assemble(*hho_mod.data_arrays(ctx, fld))
    ctx.set_option("smoother", 1)
    ctx.pmg_setup(degrees)
    x = torch.empty(ctx.ndof(0), dtype=torch.float64, device="cuda")
    info = ctx.solve(x, rtol=1e-12, maxit=500)
    assert info["rel_residual"] <= 1e-12
    err = float(np.linalg.norm(x.cpu().numpy() - xd) / np.linalg.norm(xd))
    _, it_o, _ = fgmres(h.S, PMG(h, degrees, smoother="ilu").apply, rhs_o, rtol=1e-12, null=h.null_vector())
    loc = ctx.recover(x).cpu().numpy()
    ref_loc = np.concatenate(h.recover(xd))
    e_loc = float(np.linalg.norm(loc - ref_loc) / np.linalg.norm(ref_loc))
    hv = HHO(mesh, k, "v")  # velocity-only condensation: the same discrete solution
    e_v = hv.errors(fld, hv.recover(hv.direct_solve(hv.assemble_rhs(*hv.data_values(fld)))))
    xe = ctx.quad_nodes("elem").cpu().numpy()
    u = torch.from_numpy(np.ascontiguousarray(fld.u(xe))).cuda()
    gu = torch.from_numpy(np.ascontiguousarray(fld.grad_u(xe))).cuda()
    p = torch.from_numpy(np.ascontiguousarray(fld.p(xe))).cuda()
    e = ctx.errors(torch.from_numpy(loc).cuda(), u, gu, p)
    report(f"unc-fgmres {name} k={k}", solution=err, recovered=e_loc, its=info["iterations"], its_oracle=it_o,
           u=e["u"], u_vcond=e_v["u"])
    assert err < 1e-8 and e_loc < 1e-8
    assert abs(info["iterations"] - it_o) <= 2, (info["iterations"], it_o)
    for key in ("u", "gu", "p", "div"):
        assert abs(e[key] - e_v[key]) <= 1e-6 * e_v[key] + 1e-12, (key, e[key], e_v[key])
    ctx.close()


def test_unc_mixed_precision(hho_mod):
    mesh, fld, h, rhs_o = _oracle("quad9x7-dir", 3)
    ctx = hho_mod.Context(mesh, 3, "unc")
    ctx.assemble(*hho_mod.data_arrays(ctx, fld))
    ctx.set_option("smoother", 1)
    ctx.pmg_setup([3, 2, 1, 0], prec="fp32")
    x = torch.empty(ctx.ndof(0), dtype=torch.float64, device="cuda")
    info = ctx.solve(x, rtol=1e-8)
    xd = h.direct_solve(rhs_o)
    e_x = float(np.linalg.norm(x.cpu().numpy() - xd) / np.linalg.norm(xd))
    report("unc-fp32 quad9x7-dir k=3", solution=e_x, its=info["iterations"], relres=info["rel_residual"])
    assert info["rel_residual"] <= 1e-8
    assert e_x < 1e-5, e_x
    ctx.close()
