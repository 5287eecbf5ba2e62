"""The bench's algorithmic byte model (bench.level_counts, the numerator of
every reported roofline fraction) against the oracle's level operators: for
every scheme and level, the model's unknowns equal the level dimension and its
stored values equal the entries of every block the operator couples (face and
element blocks, all diagonal blocks included), i.e. what a block layout that
stores each coupled block whole must read."""
import os
import sys

import numpy as np
import pytest

from oracle.dg import DG
from oracle.hho import HHO
from oracle.hho_hp import HHOhp
from oracle.pmg import PMG
from synthetic import quad_mesh, tri_mesh

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _block_entries(lev):
    """Entries of the coupled blocks of a level (faces of b, then elements of nP unknowns)."""
    S = lev.S.tocoo()
    nfb = lev.nf * lev.b
    nz = S.data != 0.0

    def blk(i):
        return np.where(i < nfb, i // max(lev.b, 1), lev.nf + (i - nfb) // max(lev.nP, 1))
    pairs = set(zip(blk(S.row[nz]).tolist(), blk(S.col[nz]).tolist()))
    pairs |= {(i, i) for i in range(lev.nf if lev.b else 0)}
    pairs |= {(lev.nf + t, lev.nf + t) for t in range(lev.ne if lev.nP else 0)}
    size = lambda i: lev.b if i < lev.nf else lev.nP  # noqa: E731
    return sum(size(i) * size(j) for i, j in pairs)


@pytest.mark.parametrize("cond", ["v", "vp", "hp", "unc", "dg"])
@pytest.mark.parametrize("mk", [lambda: tri_mesh(4, 3, jitter=0.2, seed=1, neumann_sides=(1,)),
                                lambda: quad_mesh(3, 3, jitter=0.15, seed=2)], ids=["tri", "quad"])
def test_level_counts_equal_the_oracle_block_structure(cond, mk):
    mesh = mk()
    k = 2
    h = {"hp": lambda: HHOhp(mesh, k), "dg": lambda: DG(mesh, k)}.get(cond, lambda: HHO(mesh, k, cond))()
    pmg = PMG(h, [2, 1, 0], coarse="lu")
    for lev in pmg.levels:
        n, z, _, _, b, nP = bench.level_counts(mesh, lev.k, cond)
        assert n == lev.n, (cond, lev.k)
        assert z == _block_entries(lev), (cond, lev.k, z, _block_entries(lev))
