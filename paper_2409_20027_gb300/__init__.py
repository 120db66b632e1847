"""Parallel-in-time Newton solver for constrained nonlinear MPC on GB300 (sm_103a).

The compute path is the CUDA library ``libptn.so`` built from ``csrc/``; the
Python binding in :mod:`paper_2409_20027_gb300.ptn` only marshals arguments.
Importing this package does not load the library; :func:`ptn.load` does, and
raises when it is missing.
"""
__all__ = ["workloads"]
