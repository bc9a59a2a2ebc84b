"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This package holds no arithmetic of the eigensolvers: it only draws matrices and
start vectors.  Both sides consume the same arrays, so neither re-derives them.
"""
from .synth import (CSRUpper, ci_matrix, ci_levels, laplacian_kron, laplacian_kron_eigs,
                    principal_submatrix, random_block, pad_rows, diagonal_matrix,
                    round_to_storage, bf16_bits_to_f32, f32_to_bf16_bits,
                    family_perturbation, family_member)

__all__ = ["CSRUpper", "ci_matrix", "ci_levels", "laplacian_kron", "laplacian_kron_eigs",
           "principal_submatrix", "random_block", "pad_rows", "diagonal_matrix",
           "round_to_storage", "bf16_bits_to_f32", "f32_to_bf16_bits",
           "family_perturbation", "family_member"]
