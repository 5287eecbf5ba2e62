"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This package holds mesh generators (topology + seeded vertex jitter) and the
analytic manufactured fields evaluated at points the caller chooses.  It holds
none of the method's arithmetic: no basis, quadrature, local operator,
condensation or solver code lives here.
"""
from .meshes import Mesh, quad_mesh, tri_mesh, hex_mesh, splitmix64_doubles  # noqa: F401
from . import fields  # noqa: F401
