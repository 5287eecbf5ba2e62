"""GB300 (sm_103a) library for p-multilevel preconditioning of statically
condensed HHO Stokes systems (Botti & Di Pietro, arXiv 2009.13840).

The compute path is ``libhho.so`` (CUDA, C ABI in ``include/hho.h``); the
binding in :mod:`paper_2009_13840_gb300.hho` only marshals arguments.
"""
__all__ = ["hho", "build"]
