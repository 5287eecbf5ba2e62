"""Batched solves on the GPU against the FP64 oracle, problem by problem.

A batch is a disjoint union of problems; hho_solve_batch runs one FGMRES per
problem with segmented reductions.  Each problem's block of the batched
solution must match the oracle's direct solve of that problem alone (up to the
solver tolerance), each problem must reach its own relative residual, and a
problem without Neumann boundary keeps its own pressure kernel.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.hho import HHO  # noqa: E402
from synthetic import quad_mesh, tri_mesh  # noqa: E402
from synthetic.batch import BatchField, TrigForcing, union_mesh  # noqa: E402


@pytest.fixture(scope="module")
def hho_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_13840_gb300 import build, hho
    build.build()
    return hho


def _problems():
    # mixed element shapes and sizes; problems 1 and 3 all-Dirichlet (pressure kernel), the others with a Neumann side
    ms = [tri_mesh(7, 6, jitter=0.2, seed=11, neumann_sides=(1,)), quad_mesh(6, 5, jitter=0.15, seed=12),
          tri_mesh(9, 8, jitter=0.2, seed=13, neumann_sides=(1,)), tri_mesh(5, 5, jitter=0.2, seed=14),
          quad_mesh(8, 7, jitter=0.15, seed=15, neumann_sides=(1,))]
    rng = np.random.default_rng(21)
    return ms, [TrigForcing(rng) for _ in ms]


def _block(x, fo, eo, p, NF, b, nP):
    return np.concatenate([x[fo[p] * b:fo[p + 1] * b], x[NF * b + eo[p] * nP:NF * b + eo[p + 1] * nP]])


def _oracle_solutions(ms, flds, k, cond):
    out = []
    for m, f in zip(ms, flds):
        h = HHO(m, k, cond)
        rhs = h.assemble_rhs(*h.data_values(f))
        x = h.direct_solve(rhs)
        nv = h.null_vector()
        out.append((x, nv))
    return out


def _solve_batch(hho_mod, ms, flds, k, cond, prec="fp64", options=(), rtol=1e-10):
    m, fo, eo, sh = union_mesh(ms, per_row=4)
    ctx = hho_mod.Context(m, k, cond)
    ctx.set_batch(fo, eo)
    ctx.assemble(*hho_mod.data_arrays(ctx, BatchField(flds, sh, per_row=4)))
    for key, val in options:
        ctx.set_option(key, val)
    ctx.pmg_setup(list(range(k, -1, -1)), prec=prec)
    x = torch.empty(ctx.ndof(0), dtype=torch.float64, device="cuda")
    info, its, rr = ctx.solve_batch(x, rtol=rtol)
    return ctx, m, fo, eo, x.cpu().numpy(), info, its, rr


@pytest.mark.parametrize("cond", ["v", "vp"])
@pytest.mark.parametrize("coarse", ["dense", "multifrontal", "twolevel"])
def test_batch_matches_oracle_per_problem(hho_mod, cond, coarse):
    ms, flds = _problems()
    k = 2
    opts = {"dense": (), "multifrontal": (("coarse_dense_max", 50), ("mf_leaf", 4)),
            "twolevel": (("coarse_dense_max", 50), ("coarse_twolevel", 1), ("dd_elements", 16))}[coarse]
    ctx, m, fo, eo, x, info, its, rr = _solve_batch(hho_mod, ms, flds, k, cond, options=opts)
    ref = _oracle_solutions(ms, flds, k, cond)
    b = 2 * (k + 1)
    nP = 1 if cond == "vp" else (k + 1) * (k + 2) // 2
    assert np.all(rr <= 1e-10), rr
    assert np.all(its >= 1) and np.all(its <= info["iterations"])
    for p, (xr, nv) in enumerate(ref):
        xp = _block(x, fo, eo, p, m.n_face, b, nP)
        if nv is not None:  # pressure defined up to its kernel
            xp = xp - (nv @ xp) * nv
            xr = xr - (nv @ xr) * nv
        err = np.linalg.norm(xp - xr) / np.linalg.norm(xr)
        assert err < 1e-7, (p, err)
    ctx.close()


def test_batch_iterations_close_to_single_solves(hho_mod):
    """The shared smoother coefficients cost little: each problem's iteration
    count in the batch is close to its count when solved alone."""
    ms, flds = _problems()
    k, cond = 2, "v"
    ctx, m, fo, eo, x, info, its, rr = _solve_batch(hho_mod, ms, flds, k, cond, rtol=1e-8)
    ctx.close()
    for p, (mp, f) in enumerate(zip(ms, flds)):
        c1 = hho_mod.Context(mp, k, cond)
        c1.assemble(*hho_mod.data_arrays(c1, f))
        c1.pmg_setup(list(range(k, -1, -1)))
        x1 = torch.empty(c1.ndof(0), dtype=torch.float64, device="cuda")
        i1 = c1.solve(x1, rtol=1e-8)["iterations"]
        c1.close()
        assert its[p] <= 2 * i1 + 4, (p, its[p], i1)


def test_batch_mixed_precision(hho_mod):
    ms, flds = _problems()
    k, cond = 3, "v"
    ctx, m, fo, eo, x, info, its, rr = _solve_batch(hho_mod, ms, flds, k, cond, prec="fp32", rtol=1e-8)
    ctx.close()
    assert np.all(rr <= 1e-8), rr
    ref = _oracle_solutions(ms, flds, k, cond)
    b, nP = 2 * (k + 1), (k + 1) * (k + 2) // 2
    for p, (xr, nv) in enumerate(ref):
        xp = _block(x, fo, eo, p, m.n_face, b, nP)
        if nv is not None:
            xp, xr = xp - (nv @ xp) * nv, xr - (nv @ xr) * nv
        assert np.linalg.norm(xp - xr) / np.linalg.norm(xr) < 1e-5, p


def test_autotune_keeps_results(hho_mod):
    ms, flds = _problems()
    k, cond = 2, "v"
    m, fo, eo, sh = union_mesh(ms, per_row=4)
    ctx = hho_mod.Context(m, k, cond)
    ctx.set_batch(fo, eo)
    ctx.assemble(*hho_mod.data_arrays(ctx, BatchField(flds, sh, per_row=4)))
    ctx.pmg_setup([2, 1, 0])
    x0 = torch.empty(ctx.ndof(0), dtype=torch.float64, device="cuda")
    _, its0, rr0 = ctx.solve_batch(x0, rtol=1e-10)
    ch = ctx.autotune(reps=2)
    assert ch["spmv_rows"] in (0, 2, 4) and ch["spmv_grid"] in (0, 1216, 2432)
    assert ch["tile_rows"] in (1024, 2048, 4096, 8192)
    x1 = torch.empty_like(x0)
    _, its1, rr1 = ctx.solve_batch(x1, rtol=1e-10)
    assert np.all(rr1 <= 1e-10)
    assert (torch.linalg.norm(x1 - x0) / torch.linalg.norm(x0)).item() < 1e-8
    ctx.close()


def test_batch_declaration_errors(hho_mod):
    ms, flds = _problems()
    m, fo, eo, sh = union_mesh(ms[:2], per_row=4)
    ctx = hho_mod.Context(m, 1, "v")
    bad = fo.copy()
    bad[1] += 1  # a face of problem 1 declared in problem 0
    with pytest.raises(hho_mod.HHOError):
        ctx.set_batch(bad, eo)
    with pytest.raises(hho_mod.HHOError):
        ctx.set_batch(fo[:-1], eo[:-1])  # does not cover the mesh
    ctx.set_batch(fo, eo)
    ctx.assemble(*hho_mod.data_arrays(ctx, BatchField(flds[:2], sh, per_row=4)))
    ctx.pmg_setup([1, 0])
    with pytest.raises(hho_mod.HHOError):
        ctx.set_batch(fo, eo)  # after pmg_setup
    ctx.close()


@pytest.mark.parametrize("cond", ["v", "vp"])
def test_graph_captured_solve_equals_host_driven(hho_mod, cond):
    """hho_solve_batch as one captured CUDA graph (restart cycles in a WHILE
    node, Arnoldi steps in IF nodes, every convergence test on the device)
    takes the same decisions as the host-driven loop: identical iteration
    counts per problem and bitwise-identical solutions; replaying it gives the
    same result again, and a restart shorter than the iteration count (several
    cycles) still converges every problem."""
    ms, flds = _problems()
    k = 2
    m, fo, eo, sh = union_mesh(ms, per_row=4)
    ctx = hho_mod.Context(m, k, cond, stream=torch.cuda.Stream())
    ctx.set_batch(fo, eo)
    ctx.assemble(*hho_mod.data_arrays(ctx, BatchField(flds, sh, per_row=4)))
    ctx.pmg_setup(list(range(k, -1, -1)))
    n = ctx.ndof(0)
    res = {}
    for graph in (0, 1):
        ctx.set_option("solve_graph", graph)
        for restart in (50, 4):
            x = torch.empty(n, dtype=torch.float64, device="cuda")
            info, its, rr = ctx.solve_batch(x, rtol=1e-9, restart=restart)
            res[(graph, restart)] = (x.cpu().numpy(), its.copy(), rr.copy(), info["iterations"])
    for restart in (50, 4):
        xh, ith, rrh, ih = res[(0, restart)]
        xg, itg, rrg, ig = res[(1, restart)]
        assert np.all(rrg <= 1e-9) and ig == ih
        assert np.array_equal(ith, itg), (ith, itg)
        assert np.array_equal(xh, xg)
    ctx.set_option("solve_graph", 1)
    x2 = torch.empty(n, dtype=torch.float64, device="cuda")
    ctx.solve_batch(x2, rtol=1e-9, restart=4)
    assert np.array_equal(x2.cpu().numpy(), res[(1, 4)][0])
    ctx.close()


@pytest.mark.parametrize("cond", ["v", "vp"])
def test_single_solve_through_the_graph(hho_mod, cond):
    """hho_solve with option solve_graph_single runs the graph-captured FGMRES
    on one problem: same tolerance reached, solution within 1e-8 of the
    host-driven FGMRES's (both solve to 1e-10), and replays give the same
    iterate bitwise."""
    from synthetic import fields
    mesh = tri_mesh(13, 11, jitter=0.2, seed=3, neumann_sides=(1,)) if cond == "v" else quad_mesh(9, 8, jitter=0.15,
                                                                                                  seed=2)
    k = 2
    ctx = hho_mod.Context(mesh, k, cond, stream=torch.cuda.Stream())
    ctx.assemble(*hho_mod.data_arrays(ctx, fields.TrigStokes2D()))
    ctx.pmg_setup(list(range(k, -1, -1)), prec="fp32")
    n = ctx.ndof(0)
    x0 = torch.empty(n, dtype=torch.float64, device="cuda")
    i0 = ctx.solve(x0, rtol=1e-10)
    ctx.set_option("solve_graph_single", 1)
    x1 = torch.empty(n, dtype=torch.float64, device="cuda")
    i1 = ctx.solve(x1, rtol=1e-10)
    x2 = torch.empty_like(x1)
    x2.copy_(x1)
    ctx.solve(x1, rtol=1e-10)
    assert i1["rel_residual"] <= 1e-10 and i0["rel_residual"] <= 1e-10
    assert abs(i1["iterations"] - i0["iterations"]) <= 2, (i0, i1)
    assert (torch.linalg.norm(x1 - x0) / torch.linalg.norm(x0)).item() < 1e-8
    assert torch.equal(x1, x2)
    ctx.close()
