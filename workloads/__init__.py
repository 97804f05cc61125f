"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This package holds only input generation (random unitaries, fixed gate matrices,
circuit layouts, random site tensors).  It contains none of the gate-application
arithmetic of the method itself.
"""
from .circuits import *  # noqa: F401,F403
