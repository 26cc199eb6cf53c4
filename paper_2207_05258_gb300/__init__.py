"""GB300-native L-HWENO (Zhang & Zhao, arXiv:2207.05258): the fifth-order
finite-difference HWENO right-hand side with limiter and the SSP-RK3 stage
update for 1D/2D Burgers and Euler, as hand-written sm_103a CUDA behind a C ABI.

Importing the package loads nothing; ``paper_2207_05258_gb300.hweno`` loads the
compiled library (and fails loudly if it is missing).
"""
__all__ = ["hweno", "workloads"]
