"""FP32 level operators of the mixed-precision hierarchy against the FP64 ones.

The FP32 copies of the level operators use per-block-size kernels and, where
one exists, a row-interleaved layout read with vector loads.  Every level
above the coarse one is checked against the FP64 operator for the block sizes
of 2D triangles (k = 1..5: face blocks of 4..12 unknowns, pressure blocks of
3..21) and 3D hexahedra (k = 1, 2: face blocks of 9 and 18), under both
condensations, and one FP32 V-cycle is compared with the FP64 one.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synthetic import tri_mesh, hex_mesh, fields  # noqa: E402


@pytest.fixture(scope="module")
def hho_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_13840_gb300 import build, hho
    build.build()
    return hho


CASES = [("tri", k) for k in (1, 2, 3, 4, 5)] + [("hex", 1), ("hex", 2)]


@pytest.mark.parametrize("cond", ["v", "vp"])
@pytest.mark.parametrize("shape,k", CASES, ids=[f"{s}-k{k}" for s, k in CASES])
def test_fp32_levels_match_fp64(hho_mod, shape, k, cond):
    if shape == "tri":
        mesh, fld = tri_mesh(7, 5, jitter=0.2, seed=9, neumann_sides=(1,)), fields.TrigStokes2D()
    else:
        mesh, fld = hex_mesh(3, jitter=0.15, seed=4), fields.CurlStokes3D()
    ctx = hho_mod.Context(mesh, k, cond)
    ctx.assemble(*hho_mod.data_arrays(ctx, fld))
    degrees = list(range(k, -1, -1))
    ctx.pmg_setup(degrees, prec="fp32")
    rng = np.random.default_rng(k)
    for l in range(len(degrees) - 1):
        n = ctx.ndof(l)
        x = torch.from_numpy(rng.standard_normal(n)).cuda()
        y64 = torch.empty(n, dtype=torch.float64, device="cuda")
        y32 = torch.empty(n, dtype=torch.float32, device="cuda")
        ctx.spmv(l, x, y64)
        ctx.spmv_f32(l, x.float(), y32)
        err = (torch.linalg.norm(y32.double() - y64) / torch.linalg.norm(y64)).item()
        assert err < 1e-5, (l, err)
    b = torch.from_numpy(rng.standard_normal(ctx.ndof(0))).cuda()
    z32 = torch.empty_like(b)
    ctx.vcycle(b, z32)
    ctx.pmg_setup(degrees, prec="fp64")
    z64 = torch.empty_like(b)
    ctx.vcycle(b, z64)
    if cond == "v" or shape == "tri":
        assert (torch.linalg.norm(z32 - z64) / torch.linalg.norm(z64)).item() < 1e-3
    assert torch.isfinite(z32).all()
    ctx.close()
