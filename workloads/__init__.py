"""Seeded synthetic wave-tank inputs shared by the oracle and the CUDA path.

This package holds only input generation: a counter-based random number generator,
closed-form fields (surface elevation, velocity, manufactured pressure and its
fluxes) and the workload descriptors.  It contains none of the solver's arithmetic:
each side computes its own node coordinates and evaluates these fields there.
"""
from .generators import *  # noqa: F401,F403
