"""Full-size checks against the oracle on sampled outputs (the benched
configurations, in the launch configuration the bench uses).

The oracle cannot assemble or solve these systems whole, but every element's
local system and every row of the condensed system are local (end of
Sec. 4.1.2), so it recomputes them on the submesh around sampled faces
(oracle/sampled.py):
* element Schur complements (Eq. ST.1 / ST.2) and condensed right-hand-side
  rows of sampled elements and faces against the GPU's, 1e-11 relative (the
  element kernels handle many elements per CTA at these sizes, which the
  small parity meshes never exercise);
* the residual b - S x of the GPU's FGMRES solution (FP32 V-cycle, 1e-8) on
  the sampled rows, recomputed by the oracle: equal to the GPU's own residual
  on those rows to the element tolerance (1e-11 of each row's |b_i| +
  sum_T max|S_T| ||x_T||_1: the rows are sums of element contributions whose
  Schur complements agree to 1e-11 of their largest entry), and,
  scaled to the global right-hand side (||r_S|| / ||b|| sqrt(n / |S|)),
  within 1e-6 (the global relative residual is 1e-8; the sampled rows are a
  random subset).  The rows of one face are not compared with the right-hand
  side on the same rows alone: boundary rows carry the Nitsche terms and
  dominate ||b||, so interior rows have a much smaller right-hand side.
The cases cover Scheme 1 (v-cond, v&p-cond), Scheme 2 (HHO-hp) and the
uncondensed formulation.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.hho import HHO  # noqa: E402
from oracle.hho_hp import HHOhp  # noqa: E402
from oracle.sampled import _submesh, residual_rows, sample_interior_faces  # noqa: E402
from synthetic import tri_mesh, hex_mesh, fields  # noqa: E402
from parity_util import report  # noqa: E402


@pytest.fixture(scope="module")
def hho_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_13840_gb300 import build, hho
    build.build()
    return hho


CASES = [
    ("tri128-mixed-k3-v", lambda: tri_mesh(128, jitter=0.2, seed=0, neumann_sides=(1,)), fields.TrigStokes2D(), 3, "v",
     True),
    ("tri128-mixed-k3-vp", lambda: tri_mesh(128, jitter=0.2, seed=0, neumann_sides=(1,)), fields.TrigStokes2D(), 3,
     "vp", True),
    ("hex16-dir-k3-vp", lambda: hex_mesh(16, jitter=0.15, seed=0), fields.CurlStokes3D(), 3, "vp", True),
    ("hex32-dir-k3-vp", lambda: hex_mesh(32, jitter=0.15, seed=0), fields.CurlStokes3D(), 3, "vp", False),
    # HHO-hp (Scheme 2) and the uncondensed formulation (block ILU(0) smoother) at the sizes of their workloads
    ("hex16-dir-k3-hp", lambda: hex_mesh(16, jitter=0.15, seed=0), fields.CurlStokes3D(), 3, "hp", True),
    ("tri128-mixed-k3-hp", lambda: tri_mesh(128, jitter=0.2, seed=0, neumann_sides=(1,)), fields.TrigStokes2D(), 3,
     "hp", False),
    ("tri128-mixed-k3-unc", lambda: tri_mesh(128, jitter=0.2, seed=0, neumann_sides=(1,)), fields.TrigStokes2D(), 3,
     "unc", True),
]


@pytest.mark.parametrize("name,mk,fld,k,cond,schur", CASES, ids=[c[0] for c in CASES])
def test_sampled_elements_rhs_and_residual(hho_mod, name, mk, fld, k, cond, schur):
    mesh = mk()
    ctx = hho_mod.Context(mesh, k, cond)
    f, gD, gN = hho_mod.data_arrays(ctx, fld)
    rhs = torch.empty(ctx.ndof(0), dtype=torch.float64, device="cuda")
    ctx.assemble(f, gD, gN, rhs)
    del f, gD, gN
    faces = sample_interior_faces(mesh, 16, seed=3)
    # both ends of the element range (the first and the last CTAs' elements)
    faces = np.unique(np.concatenate([faces, mesh.elem_face[mesh.elem_face_ptr[[0, mesh.n_elem - 1]]]]))
    if schur:
        S = ctx.element_schur()
        elems = np.unique([int(t) for F in faces for t in mesh.face_elem[F] if t >= 0])
        sub, el, _ = _submesh(mesh, elems)
        h = HHOhp(sub, k) if cond == "hp" else HHO(sub, k, cond)
        nk = np.array([len(mesh.faces_of(int(t))) * h.b + h.nP for t in range(mesh.n_elem)])
        off = np.concatenate([[0], np.cumsum(nk * nk)])
        worst, where = 0.0, None
        for i, t in enumerate(el):
            g = S[off[t]:off[t + 1]].reshape(nk[t], nk[t])
            e = np.abs(g - h.S_T[i]).max() / np.abs(h.S_T[i]).max()
            if e > worst:
                worst, where = e, int(t)
        report(f"fullsize-schur {name}", max_rel=worst, worst_elem=where, elems=len(el))
        assert worst < 1e-11, (worst, where)
    if cond == "unc":
        ctx.set_option("smoother", 1)  # block Jacobi does not smooth the uncondensed system
    ctx.pmg_setup(list(range(k, -1, -1)), prec="fp32")
    x = torch.empty(ctx.ndof(0), dtype=torch.float64, device="cuda")
    info = ctx.solve(x, rtol=1e-8, maxit=2000)
    xs = x.cpu().numpy()
    sx = torch.empty_like(x)
    ctx.spmv(0, x, sx)
    bg, sxg = rhs.cpu().numpy(), sx.cpu().numpy()
    rows, r, b, sc = residual_rows(mesh, k, cond, fld, xs, faces, with_scale=True)
    e_b = float(np.abs(bg[rows] - b).max() / np.abs(b).max())
    e_sys = float(np.max(np.abs(r - (bg[rows] - sxg[rows])) / sc))
    e_r = float(np.linalg.norm(r) / np.linalg.norm(bg) * np.sqrt(len(bg) / len(rows)))
    report(f"fullsize-residual {name}", rhs_rows=e_b, system_rows=e_sys, residual_rows_scaled=e_r,
           relres=info["rel_residual"], its=info["iterations"], rows=len(rows))
    assert info["rel_residual"] <= 1e-8
    assert e_b < 1e-11, e_b
    assert e_sys < 1e-11, e_sys
    assert e_r < 1e-6, e_r
    ctx.close()
