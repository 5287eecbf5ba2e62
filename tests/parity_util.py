"""Shared helpers of the GPU parity tests (no GPU code here).

The V-cycle ends with an exact coarse solve, and two exact solvers of the
same system in FP64 (the GPU's explicit inverses, the oracle's LU) differ by
up to about kappa(S_L) * eps relative.  The tests hold the FP64 V-cycle to
the 1e-12 bar and report kappa(S_L) beside the measured error."""
import numpy as np

EPS = np.finfo(np.float64).eps


def coarse_kappa(pmg):
    """2-norm condition number of the coarse level operator of an oracle
    hierarchy, on the complement of its pressure kernel when it has one."""
    A = pmg.levels[-1].S.toarray()
    sv = np.linalg.svd(A, compute_uv=False)
    sv = np.sort(sv)
    smin = sv[1] if pmg.null is not None else sv[0]
    return float(sv[-1] / smin)


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def report(tag, **vals):
    """One PARITY line per result (printed with `pytest -s`)."""
    print("PARITY " + tag + " " + " ".join(f"{k}={v:.3e}" if isinstance(v, float) else f"{k}={v}"
                                          for k, v in vals.items()), flush=True)
