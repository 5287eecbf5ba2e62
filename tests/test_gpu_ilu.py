"""Block ILU(0) smoother on the GPU against the oracle (oracle/ilu.py).

* the factorised preconditioner applied to a vector, on the two finest levels,
  equals the oracle's block ILU(0) with the same multicolour ordering;
* a V-cycle with the ILU smoother equals the oracle's V-cycle with it;
* FGMRES with the ILU smoother converges in about the oracle's iteration count,
  well below block Jacobi under velocity-pressure condensation, in FP64 and in
  the FP32 V-cycle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.hho import HHO  # noqa: E402
from oracle.ilu import BlockILU  # noqa: E402
from oracle.pmg import PMG, fgmres  # noqa: E402
from synthetic import tri_mesh, quad_mesh, fields  # noqa: E402
from parity_util import coarse_kappa, report  # noqa: E402


@pytest.fixture(scope="module")
def hho_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_13840_gb300 import build, hho
    build.build()
    return hho


CASES = [("tri", lambda: tri_mesh(7, 6, jitter=0.2, seed=3, neumann_sides=(1,)), 2),
         ("quad", lambda: quad_mesh(6, 5, jitter=0.15, seed=4), 1)]


def _ctx(hho_mod, mesh, k, cond, h, prec="fp64"):
    ctx = hho_mod.Context(mesh, k, cond)
    ctx.set_element_schur(np.concatenate([s.ravel() for s in h.S_T]))
    ctx.set_option("smoother", 1)
    ctx.pmg_setup(list(range(k, -1, -1)), prec=prec)
    return ctx


@pytest.mark.parametrize("cond", ["v", "vp"])
@pytest.mark.parametrize("name,mk,k", CASES, ids=[c[0] for c in CASES])
def test_ilu_apply_and_vcycle_match_oracle(hho_mod, name, mk, k, cond):
    mesh = mk()
    h = HHO(mesh, k, cond)
    ctx = _ctx(hho_mod, mesh, k, cond, h)
    pmg = PMG(h, list(range(k, -1, -1)), smoother="ilu")
    rng = np.random.default_rng(1)
    for l in range(len(pmg.levels) - 1):
        lev = pmg.levels[l]
        v = rng.standard_normal(lev.n)
        z = torch.empty(lev.n, dtype=torch.float64, device="cuda")
        ctx.ilu_apply(l, torch.from_numpy(v).cuda(), z)
        ref = lev.ilu.apply(v)
        err = float(np.linalg.norm(z.cpu().numpy() - ref) / np.linalg.norm(ref))
        report(f"ilu-apply {name} k={k} {cond} level={l}", err=err)
        assert err < 1e-12, (l, err)
    b = rng.standard_normal(ctx.ndof(0))
    z = torch.empty(ctx.ndof(0), dtype=torch.float64, device="cuda")
    ctx.vcycle(torch.from_numpy(b).cuda(), z)
    ref = pmg.apply(b)
    err = float(np.linalg.norm(z.cpu().numpy() - ref) / np.linalg.norm(ref))
    tol = 1e-12  # the FP64 bar; kappa(S_L) eps is reported beside it
    report(f"vcycle-ilu {name} k={k} {cond}", err=err, tol=tol, kappa_L=coarse_kappa(pmg))
    assert err <= tol, (err, tol)
    ctx.close()


@pytest.mark.parametrize("cond", ["v", "vp"])
def test_ilu_solve_iterations(hho_mod, cond):
    mesh = tri_mesh(12, jitter=0.2, seed=0, neumann_sides=(1,))
    k = 3
    h = HHO(mesh, k, cond)
    rhs_o = h.assemble_rhs(*h.data_values(fields.TrigStokes2D()))
    _, it_o, _ = fgmres(h.S, PMG(h, [3, 2, 1, 0], smoother="ilu").apply, rhs_o, rtol=1e-8, null=h.null_vector())
    ctx = hho_mod.Context(mesh, k, cond)
    ctx.assemble(*hho_mod.data_arrays(ctx, fields.TrigStokes2D()))
    res = {}
    for sm in (0, 1):
        for prec in ("fp64", "fp32"):
            ctx.set_option("smoother", sm)
            ctx.pmg_setup([3, 2, 1, 0], prec=prec)
            x = torch.empty(ctx.ndof(0), dtype=torch.float64, device="cuda")
            info = ctx.solve(x, rtol=1e-8)
            assert info["rel_residual"] <= 1e-8
            res[(sm, prec)] = info["iterations"]
    ctx.close()
    print(cond, "oracle ILU", it_o, res)
    assert abs(res[(1, "fp64")] - it_o) <= 2, (res, it_o)
    assert res[(1, "fp32")] <= it_o + 3, (res, it_o)
    assert res[(1, "fp64")] < res[(0, "fp64")]
