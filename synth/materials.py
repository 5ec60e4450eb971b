"""Stiffness tables for synthetic microstructures.

Every stiffness is a 6x6 Voigt matrix in the order 11, 22, 33, 23, 13, 12
with the engineering-shear convention: ``sigma_V = C @ eps_V`` where
``eps_V = (e11, e22, e33, 2 e23, 2 e13, 2 e12)``.  With that convention the
4th-order tensor components equal the Voigt entries, ``C_ijkl = C[I, J]``.
"""
from __future__ import annotations

import numpy as np

# Voigt index of the tensor pair (i, j), order 11,22,33,23,13,12
_VOIGT = np.array([[0, 5, 4],
                   [5, 1, 3],
                   [4, 3, 2]])
_PAIRS = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def isotropic_voigt(E, nu):
    """Isotropic stiffness from Young's modulus and Poisson's ratio.

    ``E = 0`` gives the zero matrix (a void)."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    C[0, 0] = C[1, 1] = C[2, 2] = lam + 2.0 * mu
    C[3, 3] = C[4, 4] = C[5, 5] = mu
    return C


def cubic_voigt(C11, C12, C44):
    C = np.zeros((6, 6))
    C[:3, :3] = C12
    C[0, 0] = C[1, 1] = C[2, 2] = C11
    C[3, 3] = C[4, 4] = C[5, 5] = C44
    return C


def _to_tensor(C6):
    C4 = np.empty((3, 3, 3, 3))
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    C4[i, j, k, l] = C6[_VOIGT[i, j], _VOIGT[k, l]]
    return C4


def _to_voigt(C4):
    C6 = np.empty((6, 6))
    for I, (i, j) in enumerate(_PAIRS):
        for J, (k, l) in enumerate(_PAIRS):
            C6[I, J] = C4[i, j, k, l]
    return C6


def rotate_voigt(C6, R):
    """``C'_ijkl = R_ip R_jq R_kr R_ls C_pqrs`` for one rotation ``R``."""
    C4 = _to_tensor(np.asarray(C6, dtype=np.float64))
    C4r = np.einsum("ip,jq,kr,ls,pqrs->ijkl", R, R, R, R, C4, optimize=True)
    C6r = _to_voigt(C4r)
    return 0.5 * (C6r + C6r.T)


def two_phase_table(E_m, nu_m, E_i, nu_i):
    """Phase 0 = matrix, phase 1 = inclusion.  Shape ``(2, 6, 6)``."""
    return np.stack([isotropic_voigt(E_m, nu_m), isotropic_voigt(E_i, nu_i)])


def polycrystal_table(C11, C12, C44, rotations):
    """One rotated cubic stiffness per grain.  Shape ``(n, 6, 6)``."""
    Cc = cubic_voigt(C11, C12, C44)
    return np.stack([rotate_voigt(Cc, R) for R in rotations])
