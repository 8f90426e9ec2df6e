"""Seeded synthetic inputs for the MBT array solver.

This package only *generates* problem data: the offset blocks of a regular
Nx x Ny lattice of identical elements with b basis functions each, and the
port excitations.  It holds none of the solver's arithmetic (no matvec, no
preconditioner, no Krylov method, no FFT), so both the CPU oracle and the
CUDA library can consume what it produces without sharing any method code.
"""
from .rng import SplitMix64, splitmix64_stream
from .lattice import (
    LatticeSpec,
    element_geometry,
    offset_blocks,
    offset_blocks_torch,
    margin_geometry,
    margin_blocks,
    excitation,
    scan_phase,
    config_c1,
    config_c2,
    config_c3_angles,
)

__all__ = [
    "SplitMix64",
    "splitmix64_stream",
    "LatticeSpec",
    "element_geometry",
    "offset_blocks",
    "offset_blocks_torch",
    "margin_geometry",
    "margin_blocks",
    "excitation",
    "scan_phase",
    "config_c1",
    "config_c2",
    "config_c3_angles",
]
