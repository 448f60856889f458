"""FLOP counts of the DPD schemes the paper compares (Sec. III-B, III-C, IV-B).

TEST INFRASTRUCTURE / analysis only: closed forms that reproduce the numbers
of Fig. 2.  Nothing on the GPU path uses them.
"""
from __future__ import annotations

import math


def td_gmp_per_sample(K: int, L3: int, G: int) -> int:
    """Eq. (10): FLOPs per input sample of one GMP DPD (order K, memory L3, cross length G)."""
    return (8 * ((L3 + 1) * (K + 2 * K * G) - G * (G + 1) // 2 * (K - 1))
            + 10 + 2 * K + 2 * (K - 1) * G + 2 * K * min(G, L3))


def td_gmp(K: int, L3: int, G: int, N: int, B: int, U: int, per_sample: int | None = None) -> float:
    """Eq. (11): per-UE FLOPs for one OFDM symbol with one GMP DPD per antenna."""
    c = td_gmp_per_sample(K, L3, G) if per_sample is None else per_sample
    return c * N * B / U


def fd_nn(N: int, N_d: int, U: int, B: int, L: int, D: int, K_nn: int) -> float:
    """Eq. (12): per-UE FLOPs of the FD-NN (NN part, U IDFT/DFT pairs at 5 N log2 N
    each, and precoding of the N_g guard bins the DFTs fill)."""
    N_g = N - N_d
    nn = N * (4 * U * (L + 1) * D + 2 * (K_nn - 1) * D * D + 4 * D * U)
    ffts = 10 * U * N * math.log2(N)
    extra = (6 + 2) * N_g * U * B
    return (nn + ffts + extra) / U


def fd_cnn(N_d: int, L_U: int, K_C: int, K_S: int, N_conv: int, grid_cells: float | None = None) -> float:
    """Sec. IV-B: C_conv + C_FC per UE per symbol.  `grid_cells` is the
    (ceil(sqrt(N_d))/K_S)^2 factor of both terms; Fig. 2 is reproduced only
    when it is replaced by N_d / K_S^2 (the unpadded grid)."""
    cells = (math.ceil(math.sqrt(N_d)) / K_S) ** 2 if grid_cells is None else grid_cells
    conv = 2 * N_conv * L_U * (2 * K_C * K_C - 1) * cells
    fc = 8 * N_d * L_U * cells
    return conv + fc
