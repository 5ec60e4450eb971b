"""Brute-force real-space solve of the tetrahedral-stencil equilibrium (test infrastructure).

Independent of the q-space formulation: no FFT, no symbol ``D(q)``, no Green
function.  The discrete problem is written in real space exactly as the paper
states it and solved with dense linear algebra, so it only suits tiny grids
(up to about 8^3 voxels).

* Unknowns: the displacement at every corner ``R = r + (+-1/2, +-1/2, +-1/2)``
  of the voxel grid (Section 2.1).  The corner at ``(l+1/2, m+1/2, n+1/2)`` is
  labelled ``(l, m, n)``; labels are periodic (Eq. PBC).
* Difference operators: ``D^(A1)`` term by term as printed in Eq. (DA1); the
  second tetrahedron's operator is ``-C_r{D^(A1)}`` (Eqs. DB1, DA2: the central
  symmetry about the voxel centre), and ``D^(B2) = D^(A1)`` (Eq. DB2).  Per the
  collapse of Section 2.4 the field T1 uses the first operator on every voxel
  and T2 the second (Eq. X_T1_T2_R).
* Strains ``deps_ij = 1/2 (D_i u_j + D_j u_i)`` (Eq. deps).
* Energy ``E = 1/2 (E^(1) + E^(2)) = 1/4 sum_r sum_T (eps^T - eps0):lambda:(eps^T - eps0)``
  (Eqs. Elast_energy_k, Elast_energy with d = 1).  ``E`` is quadratic in ``u``:
  ``E = 1/2 u.K.u + g.u + c``; its gradient is the nodal force.
* Equilibrium (Eq. Equilibrium_real): ``K u = -g``, solved with the
  pseudo-inverse (the minimum-norm solution; the null space is the uniform
  translations of the two FCC corner subgrids).
* Basic scheme in real space: ``u <- u - K0^+ (K u + g)`` where ``K0`` is the
  Hessian with the homogeneous reference stiffness ``lambda0``.  In q-space
  ``K0^+`` is the Green function times 2 with zeros on the translation modes,
  so these iterates are those of Algorithm 1.
* Error: ``L2 = sqrt(1/N sum_R |dE/du(R)|^2)`` (Eq. L2-norm, real-space form)
  divided by the Frobenius norm of ``<sigma>`` (Eq. tolerance).
"""
from __future__ import annotations

import numpy as np

from .tetra import stiffness_tensor

# Eq. (DA1): (coefficient, corner offset in units of 1/2) per term, for D_1, D_2, D_3
_DA1 = [
    [(+1, (1, 1, 1)), (+1, (1, -1, -1)), (-1, (-1, -1, 1)), (-1, (-1, 1, -1))],
    [(+1, (1, 1, 1)), (+1, (-1, 1, -1)), (-1, (-1, -1, 1)), (-1, (1, -1, -1))],
    [(+1, (1, 1, 1)), (+1, (-1, -1, 1)), (-1, (-1, 1, -1)), (-1, (1, -1, -1))],
]


def _operators():
    """Term lists for the T1 operator (Eq. DA1) and the T2 operator (Eq. DA2)."""
    T1 = _DA1
    # -C_r{...}: reflect every offset through the voxel centre and flip the sign
    T2 = [[(-c, (-o[0], -o[1], -o[2])) for (c, o) in terms] for terms in _DA1]
    return T1, T2


def _corner_label(r, o, grid):
    """Label of the corner at ``r + o/2`` (``o`` in {-1,1}^3)."""
    n1, n2, n3 = grid
    x = (r[0] + (o[0] - 1) // 2) % n1
    y = (r[1] + (o[1] - 1) // 2) % n2
    z = (r[2] + (o[2] - 1) // 2) % n3
    return (z * n2 + y) * n1 + x


def strain_matrix(grid, terms):
    """Dense ``B`` with ``deps[(ij), r] = B @ u`` for one tetrahedron type.

    Row index ``(i*3 + j) * N + r``; column index ``j * N + R``."""
    n1, n2, n3 = grid
    N = n1 * n2 * n3
    B = np.zeros((9 * N, 3 * N))
    for z in range(n3):
        for y in range(n2):
            for x in range(n1):
                r = (z * n2 + y) * n1 + x
                for i in range(3):
                    for (c, o) in terms[i]:
                        R = _corner_label((x, y, z), o, grid)
                        # D_i u_j contributes 1/2 * (1/2 c) to eps_ij and eps_ji
                        for j in range(3):
                            B[(i * 3 + j) * N + r, j * N + R] += 0.25 * c
                            B[(j * 3 + i) * N + r, j * N + R] += 0.25 * c
    return B


def _lambda_blocks(C4_per_voxel):
    """Block matrix acting on 9N strain vectors: (ij, r) x (kl, r)."""
    N = C4_per_voxel.shape[0]
    L = np.zeros((9 * N, 9 * N))
    idx = np.arange(N)
    for a in range(9):
        for b in range(9):
            L[a * N + idx, b * N + idx] = C4_per_voxel[:, a // 3, a % 3, b // 3, b % 3]
    return L


class DenseProblem:
    """The discrete equilibrium as a dense quadratic form."""

    def __init__(self, ids, table, lam0=None, eigen=None):
        ids = np.asarray(ids)
        n3, n2, n1 = ids.shape
        self.grid = (n1, n2, n3)
        self.N = N = n1 * n2 * n3
        C4 = np.stack([stiffness_tensor(c) for c in np.asarray(table)])
        self.C4v = C4[ids.reshape(-1)]
        T1, T2 = _operators()
        self.B = [strain_matrix(self.grid, T1), strain_matrix(self.grid, T2)]
        self.L = _lambda_blocks(self.C4v)
        self.K = 0.5 * sum(Bt.T @ self.L @ Bt for Bt in self.B)
        self.eigen = None
        if eigen is not None:
            self.eigen = np.asarray(eigen, dtype=np.float64)[ids.reshape(-1)]  # (N,3,3)
        if lam0 is not None:
            L0 = _lambda_blocks(np.broadcast_to(np.asarray(lam0), (N, 3, 3, 3, 3)))
            self.K0 = 0.5 * sum(Bt.T @ L0 @ Bt for Bt in self.B)
            self.K0p = np.linalg.pinv(self.K0, rcond=1e-12, hermitian=True)

    def _e(self, eps_bar):
        N = self.N
        e = np.repeat(np.asarray(eps_bar, dtype=np.float64).reshape(9), N)
        if self.eigen is not None:
            e = e - self.eigen.reshape(N, 9).T.reshape(-1)
        return e

    def gradient_offset(self, eps_bar):
        e = self._e(eps_bar)
        return 0.5 * sum(Bt.T @ (self.L @ e) for Bt in self.B)

    def force(self, u, eps_bar):
        """``dE/du`` at every corner, shape (3N,) (component-major)."""
        return self.K @ u + self.gradient_offset(eps_bar)

    def energy(self, u, eps_bar):
        e = self._e(eps_bar)
        return 0.25 * sum((e + Bt @ u) @ (self.L @ (e + Bt @ u)) for Bt in self.B)

    def fields(self, u, eps_bar):
        """``(deps1, deps2, sig1, sig2)`` each shaped (3, 3, N3, N2, N1)."""
        n1, n2, n3 = self.grid
        e = self._e(eps_bar)
        out = []
        for Bt in self.B:
            out.append((Bt @ u).reshape(3, 3, n3, n2, n1))
        for Bt in self.B:
            out.append((self.L @ (e + Bt @ u)).reshape(3, 3, n3, n2, n1))
        return tuple(out)

    def solve(self, eps_bar):
        """Minimum-norm equilibrium displacement."""
        g = self.gradient_offset(eps_bar)
        return -np.linalg.pinv(self.K, rcond=1e-12, hermitian=True) @ g

    def error(self, u, eps_bar):
        F = self.force(u, eps_bar)
        L2 = np.sqrt(np.sum(F ** 2) / self.N)
        _, _, s1, s2 = self.fields(u, eps_bar)
        sm = 0.5 * (s1.reshape(3, 3, -1).mean(axis=2) + s2.reshape(3, 3, -1).mean(axis=2))
        return L2 / np.sqrt(np.sum(sm ** 2)), sm

    def richardson(self, eps_bar, n_iter):
        """Basic-scheme iterates ``u_0 = 0, u_{n+1} = u_n - K0^+ (K u_n + g)``.

        Returns the list of ``u_n`` for ``n = 0..n_iter-1`` (state at evaluation n+1)."""
        g = self.gradient_offset(eps_bar)
        u = np.zeros(3 * self.N)
        us = []
        for _ in range(n_iter):
            us.append(u.copy())
            u = u - self.K0p @ (self.K @ u + g)
        return us
