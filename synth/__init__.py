"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package only draws the Hamiltonian, the trial wavefunction and the run
parameters. It holds none of the ph-AFQMC arithmetic, so both sides can
consume it without sharing any part of the method.
"""
from .systems import (  # noqa: F401
    System,
    sym,
    make_h1,
    make_system,
    small_system,
    config_c1,
    config_c2,
    config_c3,
    config_c4,
    serving_run,
    CONFIGS,
)
