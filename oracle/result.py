"""Common result record of the oracle solvers (test infrastructure only)."""
from dataclasses import dataclass, field

import numpy as np


@dataclass
class EigResult:
    theta: np.ndarray                 # Ritz values, ascending (n_ev or n_b)
    X: np.ndarray                     # Ritz vectors (n x len(theta))
    relres: np.ndarray                # per-column relative residual (estimate or computed)
    converged: bool
    iterations: int
    spmm: int = 0                     # number of H-times-block products
    spmv: int = 0                     # SpMV count as the paper counts it (Sec. 2.6)
    HX: np.ndarray = None             # H X when the method has it without extra work
    history: list = field(default_factory=list)
    extra: dict = field(default_factory=dict)
