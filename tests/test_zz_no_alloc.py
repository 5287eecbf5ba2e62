"""hho_assemble_noalloc, the allocation-free right-hand-side assembly, against hho_assemble.

Callers that cannot allocate device memory when they refresh the right-hand
side (all device memory handed to their own pool, or a loop where a
cudaMalloc, which may synchronise the device or fail, is not acceptable) use
hho_assemble_noalloc; it must give what hho_assemble gives.  This file is
collected last so that a failure here leaves every other test run.  Two calls
in a row with different data check that the shared working array keeps
nothing from one call to the next.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synthetic import tri_mesh, quad_mesh, hex_mesh, fields  # noqa: E402


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


def _poly(d, k, seed):
    return fields.PolyStokes(d, k + 1, k, np.random.default_rng(seed))


# the 3D case has 512 elements of k = 3: one local system needs about 260
# doubles of working memory, so at most 504 elements fit the 2^17-double array
# at once and the element kernel runs on a shrunk grid
CASES = [
    ("tri13x11-v-k3", lambda: tri_mesh(13, 11, jitter=0.2, seed=3, neumann_sides=(1,)), "v", 3),
    ("quad9x7-vp-k2", lambda: quad_mesh(9, 7, jitter=0.15, seed=5), "vp", 2),
    ("hex8-vp-k3", lambda: hex_mesh(8, jitter=0.15, seed=2), "vp", 3),
]


@pytest.mark.parametrize("name,mk,cond,k", CASES, ids=[c[0] for c in CASES])
def test_noalloc_assemble_matches_assemble(hho_mod, name, mk, cond, k):
    """Through the C ABI: two calls in a row against hho_assemble to 1e-12."""
    mesh = mk()
    ctx = hho_mod.Context(mesh, k, cond)
    lib = hho_mod.load()
    n = ctx.ndof(0)
    d = mesh.dim
    base = fields.TrigStokes2D() if d == 2 else fields.CurlStokes3D()
    calls = [(base, 1.0), (_poly(d, k, 11), -2.5)]
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


def test_noalloc_binding_frees_inputs_and_allocates_nothing(hho_mod):
    """Through the Python binding, with the context on its own stream: the
    inputs are dropped right after the call and their memory is handed out
    again at once, which must not disturb the queued kernels; two further calls
    leave the device's free memory and torch's allocated bytes unchanged."""
    mesh = tri_mesh(13, 11, jitter=0.2, seed=3, neumann_sides=(1,))
    k = 3
    side = torch.cuda.Stream()
    ctx = hho_mod.Context(mesh, k, "v", stream=side)
    n = ctx.ndof(0)
    field = _poly(2, k, 4)
    f, gD, gN = _data(hho_mod, ctx, field, 1.5)
    ref = torch.empty(n, dtype=torch.float64, device="cuda")
    ctx.assemble(f, gD, gN, ref)
    torch.cuda.synchronize()
    out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    ctx.assemble_noalloc(f.clone(), gD.clone(), gN.clone(), out)
    # the clones are gone now; new tensors of the same sizes overwrite any reused memory
    junk = [torch.full_like(t, 1e30) for t in (f, gD, gN)]
    torch.cuda.synchronize()
    assert np.abs(out.cpu().numpy() - ref.cpu().numpy()).max() <= 1e-12 * ref.abs().max().item()
    del junk
    # two further calls in a row (the first call above did the one-time set-up)
    fs, gDs, gNs = f * -0.5, gD * -0.5, gN * -0.5
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    ctx.assemble_noalloc(f, gD, gN, out)
    ctx.assemble_noalloc(fs, gDs, gNs, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == alloc0
    assert free1 == free0, (free0, free1)
    ref2 = torch.empty(n, dtype=torch.float64, device="cuda")
    ctx.assemble(fs, gDs, gNs, ref2)
    torch.cuda.synchronize()
    assert np.abs(out.cpu().numpy() - ref2.cpu().numpy()).max() <= 1e-12 * ref2.abs().max().item()
    ctx.close()
