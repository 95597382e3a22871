"""Plain FP64 CPU oracle for the fugacity-based multicomponent LBM.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the smoke check and by
the benchmark's CPU-baseline leg, never by the CUDA library or its binding.
The C part (``lbm_oracle.c``) holds the lattice Boltzmann step and the
Peng-Robinson thermodynamics; ``thermo.py`` holds the Maxwell construction,
the two-phase flash and the unit conversion used to pin it against the
paper's printed results.
"""
from .orc import OracleProblem, build_oracle, lattice_info, feq_forcing  # noqa: F401
