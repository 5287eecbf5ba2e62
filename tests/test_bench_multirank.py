"""The replicas path of bench.py on two gloo ranks (CPU): the reported time is
the slowest rank's, the whole-job rate counts every rank's units, and the
reference arm prints from rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    sys.path.insert(0, ROOT)
    import bench
    ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
    slow = bench.max_over_ranks(ms, ws, "cpu")
    out.put((rank, slow, bench.whole_job_rate(1000, ws, slow / 1e3)))
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]
    assert all(abs(r[2] - 2 * 1000 / 0.015) < 1e-6 for r in res)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.whole_job_rate(10, 1, 2.0) == 5.0


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                          "--warmup", "0", "--workload", "c2", "--sample-n", "4", "--k", "1"], cwd=ROOT, env=env,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    assert not [l for l in out.stdout.splitlines() if l.startswith("{")]
    env["RANK"], env["LOCAL_RANK"] = "0", "0"
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                          "--warmup", "0", "--workload", "c2", "--sample-n", "4", "--k", "1"], cwd=ROOT, env=env,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads([l for l in out.stdout.splitlines() if l.startswith("{")][0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2


def test_oracle_row_checks_on_cpu():
    """bench.py's full-size row checks on an oracle-made system (no GPU): with
    the oracle's own right-hand side and S x as the 'GPU' vectors, the rows
    agree to rounding, for Scheme 1 (faces) and the DG scheme (elements)."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    from oracle.dg import DG
    from oracle.hho import HHO
    from synthetic import tri_mesh, fields
    mesh = tri_mesh(6, 5, jitter=0.2, seed=3, neumann_sides=(1,))
    fld = fields.TrigStokes2D()
    for h, check in ((HHO(mesh, 2, "v"), lambda h, x, b, sx: bench.oracle_check(mesh, 2, "v", fld, x, b, sx, 5)),
                     (DG(mesh, 2), lambda h, x, b, sx: bench.oracle_check_dg(mesh, 2, fld, x, b, sx, 5))):
        b = h.assemble_rhs(*h.data_values(fld))
        x = np.random.default_rng(4).standard_normal(h.ndof)
        c = check(h, x, b, h.S @ x)
        assert c["rows"] > 0 and c["system_rows_max_diff_rel"] < 1e-13 and c["rhs_rows_max_diff_rel"] < 1e-13
