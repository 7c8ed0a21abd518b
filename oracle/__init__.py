"""CPU oracle for the FE-LBM contact-line step (TEST INFRASTRUCTURE ONLY).

A plain, slow, FP64 restatement of the paper's scheme (Matin, Misztal,
Hernandez-Garcia, Mathiesen, "Finite Element Lattice Boltzmann Simulations of
Contact Line Dynamics", arXiv:1708.04678).  Only the test-suite, the smoke
check and the CPU baseline of the benchmark may import it; the product path
(the CUDA library and its Python binding) never does, and shares no code with
it.
"""
from .felbm_oracle import (  # noqa: F401
    D2Q9_E,
    D2Q9_W,
    D2Q9_OPP,
    OracleMesh,
    OracleParams,
    OracleSim,
    params_from_physical,
)
