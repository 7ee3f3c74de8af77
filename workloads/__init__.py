"""Seeded synthetic problem generator shared by the oracle, the tests and the bench.

It holds no arithmetic of the method itself: it only lays out the structured patch
grid, the knot vectors, the geometry control nets, the per-element material data
and the coil-source parameters.  Everything that involves B-splines, assembly,
gauging or solving lives separately in ``oracle/`` (the CPU checker) and in the
CUDA library.
"""
from .configs import Problem, make_problem, CONFIGS, small_problem, sub_problem  # noqa: F401
