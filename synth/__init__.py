"""Seeded synthetic inputs shared by the CPU oracle, the tests and the benchmark.

This package holds no arithmetic of the minimisation method: it only draws
initial magnetisations, applied fields, easy axes and request streams from a
counter-based generator, so that the oracle and the CUDA path start from the
same bytes.
"""
from .inputs import *  # noqa: F401,F403
from .meshes import ball_mesh, jittered_cube, l_shape  # noqa: F401
