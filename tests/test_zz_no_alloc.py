"""hho_assemble_noalloc, the allocation-free right-hand-side assembly, against hho_assemble.

Callers that cannot allocate device memory when they refresh the right-hand
side use hho_assemble_noalloc; it must give what hho_assemble gives.  This
file is collected last so that a failure here leaves every other test run.
Two calls in a row with different data check that the shared working array
keeps nothing from one call to the next.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synthetic import tri_mesh, quad_mesh, fields  # noqa: E402


@pytest.fixture(scope="module")
def hho_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_13840_gb300 import build, hho
    build.build()
    return hho


def _data(hho_mod, ctx, field, scale):
    f, gD, gN = hho_mod.data_arrays(ctx, field)
    return f * scale, gD * scale, gN * scale


@pytest.mark.parametrize("mk,cond,k", [
    (lambda: tri_mesh(13, 11, jitter=0.2, seed=3, neumann_sides=(1,)), "v", 3),
    (lambda: quad_mesh(9, 7, jitter=0.15, seed=5), "vp", 2),
])
def test_noalloc_assemble_matches_assemble(hho_mod, mk, cond, k):
    mesh = mk()
    ctx = hho_mod.Context(mesh, k, cond)
    lib = hho_mod.load()
    n = ctx.ndof(0)
    calls = [(fields.TrigStokes2D(), 1.0),
             (fields.PolyStokes(2, k + 1, k, np.random.default_rng(11)), -2.5)]
    for field, scale in calls:  # two calls in a row, different data
        f, gD, gN = _data(hho_mod, ctx, field, scale)
        ref = torch.empty(n, dtype=torch.float64, device="cuda")
        ctx.assemble(f, gD, gN, ref)
        out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.hho_assemble_noalloc(ctx.h, C.c_void_p(f.data_ptr()), C.c_void_p(gD.data_ptr()),
                                      C.c_void_p(gN.data_ptr()), C.c_void_p(out.data_ptr()))
        assert st == 0, lib.hho_last_error(ctx.h)
        ctx.stream.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    ctx.close()
