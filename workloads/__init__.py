"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This package holds input generation only (random operators, potentials and
starting points).  It contains none of the PLAM/PCAL arithmetic, so both the
FP64 oracle and the GPU path can draw identical bytes from it without sharing
any part of the method.
"""
from .generators import *  # noqa: F401,F403
