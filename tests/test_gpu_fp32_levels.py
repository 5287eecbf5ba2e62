"""FP32 level operators and V-cycle of the mixed-precision hierarchy.

The FP32 copies of the level operators use per-block-size kernels and, where
one exists, a row-interleaved layout read with vector loads (large 3D face
blocks: one warp per face).  Every level above the coarse one is checked
against the FP64 operator (itself pinned to the oracle at 1e-13) for the block
sizes of 2D triangles (k = 1..5: face blocks of 4..12 unknowns, pressure
blocks of 3..21) and 3D hexahedra (k = 1..3: face blocks of 9, 18 and 30),
under both condensations and for HHO-hp (face blocks of 3 (k+1) in 2D, 12, 24
and 40 in 3D, no element rows); for the large 3D blocks the warp-per-face
kernel is also compared with the one-thread-per-face one.  One FP32 V-cycle is
compared with the oracle's FP64 V-cycle: FP32 rounding amplified by the coarse
conditioning, 1e-3 relative.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.hho import HHO  # noqa: E402
from oracle.hho_hp import HHOhp  # noqa: E402
from oracle.pmg import PMG  # noqa: E402
from synthetic import tri_mesh, hex_mesh, fields  # noqa: E402
from parity_util import report  # noqa: E402


@pytest.fixture(scope="module")
def hho_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_13840_gb300 import build, hho
    build.build()
    return hho


CASES = [("tri", k) for k in (1, 2, 3, 4, 5)] + [("hex", 1), ("hex", 2), ("hex", 3)]


@pytest.mark.parametrize("cond", ["v", "vp", "hp"])
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
    worst = 0.0
    for l in range(len(degrees) - 1):
        n = ctx.ndof(l)
        x = torch.from_numpy(rng.standard_normal(n)).cuda()
        y64 = torch.empty(n, dtype=torch.float64, device="cuda")
        y32 = torch.empty(n, dtype=torch.float32, device="cuda")
        ctx.spmv(l, x, y64)
        ctx.spmv_f32(l, x.float(), y32)
        err = (torch.linalg.norm(y32.double() - y64) / torch.linalg.norm(y64)).item()
        worst = max(worst, err)
        assert err < 1e-5, (l, err)
        if shape == "hex":
            ctx.set_option("spmv_warp", 0)
            y32b = torch.empty(n, dtype=torch.float32, device="cuda")
            ctx.spmv_f32(l, x.float(), y32b)
            ctx.set_option("spmv_warp", 1)
            e2 = (torch.linalg.norm(y32b.double() - y64) / torch.linalg.norm(y64)).item()
            assert e2 < 1e-5, (l, e2)
    b = rng.standard_normal(ctx.ndof(0))
    z32 = torch.empty(ctx.ndof(0), dtype=torch.float64, device="cuda")
    ctx.vcycle(torch.from_numpy(b).cuda(), z32)
    h = HHOhp(mesh, k) if cond == "hp" else HHO(mesh, k, cond)
    ref = PMG(h, degrees).apply(b)
    e_v = float(np.linalg.norm(z32.cpu().numpy() - ref) / np.linalg.norm(ref))
    report(f"fp32levels {shape} k={k} {cond}", operator=worst, vcycle_vs_oracle=e_v)
    assert torch.isfinite(z32).all()
    assert e_v < 1e-3, e_v
    ctx.close()
