"""Tetrahedral-stencil FFT homogenization: plain FP64 oracle (test infrastructure).

Follows the paper (Finel, "A fast and robust discrete FFT-based solver for
computational homogenization", arXiv 2405.11168) in its own notation and
Fourier convention:

* voxel centres ``r`` on the simple-cubic strain grid (Eq. r-vectors),
  displacements on the corner grid ``r + (+-1/2, +-1/2, +-1/2)``;
* q-vectors ``q_i = 2 pi h_i / N_i``, ``h_i = 0..N_i-1`` (Eq. q-vectors);
* forward transform with ``1/N``, inverse without (Eqs. FT, IFT_u);
* ``D_i(q)`` of Eq. (Dq), the T1/T2 strains of Eq. (deps_dep_Q),
  the Green function of Eq. (Green_tensor) with ``Omega = 0`` at ``q = 0`` and
  ``q = (pi, pi, pi)`` (Section 2.3, end);
* Algorithm 1 (displacement form, Eq. basic_scheme_dep_2), the stopping test
  of Eqs. (L2-norm, tolerance), the final fields of Eq. (final_fields) and the
  applied-stress update of Section 2.5;
* Algorithm 2 (strain form, Eq. Lippmann_Schwinger_strain_3) as an
  iterate-equivalent cross-check.

Everything is FP64.  A library FFT (``scipy.fft`` real transforms with
``norm="forward"``, i.e. 1/N on the forward transform exactly as Eq. FT) is the
only non-elementary step; the fields stored in q-space are kept on the half
spectrum ``h1 = 0..N1/2`` because every transformed field is the transform of a
real field on the integer strain grid.

Readings of the paper taken here (where it is ambiguous or garbled):

1. Eq. (Dq) drops closing parentheses; each term is read as
   ``exp(i/2 (+-q1 +-q2 +-q3))``, signs as printed.
2. In Eq. (Lippmann_Schwinger_strain_2) the second line's right-hand side
   starts with ``deps^(T2)_(n)`` (the printed ``deps^(T1)_(n)`` is a typo), as
   in Eq. (Lippmann_Schwinger_strain_3) and Algorithm 2.
3. The iteration count is the number of residual evaluations; a homogeneous
   medium stops after 1.  The test is ``err < tol`` (so ``tol = 0`` never
   stops early).
4. Index placement of ``conj(D) . lambda0 . D``: the matrix whose product with
   ``u`` gives ``sigma^(T1).conj(D) - sigma^(T2).D`` for ``sigma = lambda0 : eps``,
   i.e. ``Omega^-1_jl = sum_ik lambda0_jikl (conj(D_i) D_k + D_i conj(D_k))``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.fft as sfft

# --------------------------------------------------------------------------
# Voigt <-> tensor (order 11,22,33,23,13,12; engineering shear in stiffness)
# --------------------------------------------------------------------------
_V = np.array([[0, 5, 4], [5, 1, 3], [4, 3, 2]])
_PAIRS = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def stiffness_tensor(C6):
    """4th-order tensor ``lambda_ijkl`` from a 6x6 engineering-Voigt stiffness."""
    C6 = np.asarray(C6, dtype=np.float64)
    C4 = np.zeros((3, 3, 3, 3))
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    C4[i, j, k, l] = C6[_V[i, j], _V[k, l]]
    return C4


def strain_tensor_from_voigt(e6):
    """3x3 strain from 6 tensor components in Voigt order (e[3] = eps23)."""
    e = np.asarray(e6, dtype=np.float64)
    out = np.empty((3, 3))
    for I, (i, j) in enumerate(_PAIRS):
        out[i, j] = out[j, i] = e[I]
    return out


def voigt_from_tensor(t):
    """6 Voigt components (11,22,33,23,13,12) of a symmetric 3x3(...) array."""
    return np.stack([t[i, j] for (i, j) in _PAIRS])


def isotropic_lambda0(lam, mu):
    d = np.eye(3)
    return (lam * np.einsum("ij,kl->ijkl", d, d)
            + mu * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d)))


def c0_alpha_rule(table):
    """Reference medium of the paper's contrast study (Section 3.4).

    Two isotropic phases (0 = matrix, 1 = inclusion).  Same Poisson ratio as
    the phases (the matrix's when they differ) and bulk modulus
    ``k0 = alpha k_m + (1 - alpha) k_i``, ``alpha = 0.55`` if ``k_i/k_m < 1``
    else ``0.45``.  Returns the 4th-order ``lambda0``.
    """
    table = np.asarray(table, dtype=np.float64)
    lam_m, mu_m = table[0, 0, 1], table[0, 3, 3]
    lam_i, mu_i = table[1, 0, 1], table[1, 3, 3]
    k_m = lam_m + 2.0 * mu_m / 3.0
    k_i = lam_i + 2.0 * mu_i / 3.0
    alpha = 0.55 if k_i < k_m else 0.45
    k0 = alpha * k_m + (1.0 - alpha) * k_i
    nu0 = lam_m / (2.0 * (lam_m + mu_m))
    mu0 = 3.0 * k0 * (1.0 - 2.0 * nu0) / (2.0 * (1.0 + nu0))
    lam0 = k0 - 2.0 * mu0 / 3.0
    return isotropic_lambda0(lam0, mu0)


# --------------------------------------------------------------------------
# q-space symbols (Section 2.2) and Green function (Section 2.3)
# --------------------------------------------------------------------------
def q_vectors(grid, half=True):
    """``q_i = 2 pi h_i / N_i`` broadcast to ``(N3, N2, N1h)`` (Eq. q-vectors).

    With ``half=True`` the x axis keeps ``h1 = 0..N1/2`` only."""
    n1, n2, n3 = grid
    h1 = np.arange(n1 // 2 + 1) if half else np.arange(n1)
    q1 = (2.0 * np.pi * h1 / n1)[None, None, :]
    q2 = (2.0 * np.pi * np.arange(n2) / n2)[None, :, None]
    q3 = (2.0 * np.pi * np.arange(n3) / n3)[:, None, None]
    return q1, q2, q3


def D_of_q(grid, half=True):
    """The tetrahedral gradient symbols ``D_i(q)``, Eq. (Dq), on the q grid."""
    return D_at(*q_vectors(grid, half))


def D_at(q1, q2, q3):
    """``D_i(q)`` of Eq. (Dq) at arbitrary (broadcastable) ``q``.  Shape (3, ...)."""
    t_ppp = np.exp(0.5j * (q1 + q2 + q3))
    t_pmm = np.exp(0.5j * (q1 - q2 - q3))
    t_mpm = np.exp(0.5j * (-q1 + q2 - q3))
    t_mmp = np.exp(0.5j * (-q1 - q2 + q3))
    D1 = 0.5 * (t_ppp + t_pmm - t_mpm - t_mmp)
    D2 = 0.5 * (t_ppp - t_pmm + t_mpm - t_mmp)
    D3 = 0.5 * (t_ppp - t_pmm - t_mpm + t_mmp)
    return np.stack(np.broadcast_arrays(D1, D2, D3))


def translation_modes(grid, half=True):
    """Boolean mask of ``q = 0`` and ``q = (pi, pi, pi)`` (Eq. q_0 discussion)."""
    n1, n2, n3 = grid
    n1h = n1 // 2 + 1 if half else n1
    m = np.zeros((n3, n2, n1h), dtype=bool)
    m[0, 0, 0] = True
    m[n3 // 2, n2 // 2, n1 // 2] = True
    return m


def green_inverse(D, lam0):
    """``Omega^-1(q) = conj(D).lambda0.D + D.lambda0.conj(D)``, Eq. (Green_tensor).

    Returns the real part (the imaginary part vanishes identically)."""
    Dc = np.conj(D)
    A = (np.einsum("i...,jikl,k...->jl...", Dc, lam0, D)
         + np.einsum("i...,jikl,k...->jl...", D, lam0, Dc))
    return A.real


def green(D, lam0, grid, half=True):
    """``Omega(q)``, zero at ``q = 0`` and ``q = (pi,pi,pi)`` (Section 2.3)."""
    Ainv = green_inverse(D, lam0)
    mask = translation_modes(grid, half)
    A = np.moveaxis(Ainv, (0, 1), (-2, -1)).copy()
    A[mask] = np.eye(3)
    Om = np.linalg.inv(A)
    Om[mask] = 0.0
    return np.moveaxis(Om, (-2, -1), (0, 1))


def gamma3(D, Om):
    """``Gamma_ijk = 1/2 (D_i Omega_jk + D_j Omega_ik)`` (Algorithm 2)."""
    return 0.5 * (np.einsum("i...,jk...->ijk...", D, Om) + np.einsum("j...,ik...->ijk...", D, Om))


def strain_green_operators(D, Om):
    """``G^d`` and ``G^nd`` of Eq. (strain_based_Green_functions_tetrahedral_stencil)."""
    Dc = np.conj(D)
    Gd = 0.25 * (np.einsum("i...,jk...,l...->ijkl...", D, Om, Dc)
                 + np.einsum("j...,ik...,l...->ijkl...", D, Om, Dc)
                 + np.einsum("i...,jl...,k...->ijkl...", D, Om, Dc)
                 + np.einsum("j...,il...,k...->ijkl...", D, Om, Dc))
    Gnd = -0.25 * (np.einsum("i...,jk...,l...->ijkl...", D, Om, D)
                   + np.einsum("j...,ik...,l...->ijkl...", D, Om, D)
                   + np.einsum("i...,jl...,k...->ijkl...", D, Om, D)
                   + np.einsum("j...,il...,k...->ijkl...", D, Om, D))
    return Gd, Gnd


def sym_outer(a, b):
    """Symmetrised tensor product ``(a (x)_s b)_ij = 1/2 (a_i b_j + a_j b_i)``."""
    return 0.5 * (np.einsum("i...,j...->ij...", a, b) + np.einsum("j...,i...->ij...", a, b))


# --------------------------------------------------------------------------
# transforms (Eqs. FT and IFT_u: 1/N on the forward transform only)
# --------------------------------------------------------------------------
def _workers():
    import os
    return os.cpu_count() or 1


def ft(field_r, workers=None):
    """Forward transform of a real field ``(..., N3, N2, N1)`` -> half spectrum."""
    return sfft.rfftn(field_r, axes=(-3, -2, -1), norm="forward",
                      workers=workers or _workers())


def ift(field_q, grid, workers=None):
    """Inverse transform (no 1/N) of a half-spectrum field -> real field."""
    n1, n2, n3 = grid
    return sfft.irfftn(field_q, s=(n3, n2, n1), axes=(-3, -2, -1), norm="forward",
                       workers=workers or _workers())


def half_weights(grid):
    """Multiplicity of each half-spectrum point in the full q set."""
    n1 = grid[0]
    w = np.full(n1 // 2 + 1, 2.0)
    w[0] = 1.0
    w[n1 // 2] = 1.0
    return w[None, None, :]


# --------------------------------------------------------------------------
# material
# --------------------------------------------------------------------------
class Material:
    """Phase map + per-phase stiffness (and optional per-phase eigenstrain)."""

    def __init__(self, ids, table, eigen=None):
        self.ids = np.asarray(ids)
        self.shape = self.ids.shape
        self.C4 = np.stack([stiffness_tensor(c) for c in np.asarray(table)])
        flat = self.ids.reshape(-1)
        order = np.argsort(flat, kind="stable")
        counts = np.bincount(flat, minlength=len(self.C4))
        self.index = np.split(order, np.cumsum(counts)[:-1])
        self.eigen = None if eigen is None else np.asarray(eigen, dtype=np.float64)

    def stress(self, eps, with_eigen=True):
        """``sigma(r) = lambda(r) : (eps(r) - eps0(r))``, Eq. (linear_elasticity).

        ``with_eigen=False`` gives ``lambda(r) : eps(r)``."""
        e = eps.reshape(3, 3, -1)
        out = np.empty_like(e)
        for p, idx in enumerate(self.index):
            if idx.size == 0:
                continue
            ep = e[:, :, idx]
            if with_eigen and self.eigen is not None:
                ep = ep - self.eigen[p][:, :, None]
            out[:, :, idx] = np.einsum("ijkl,kln->ijn", self.C4[p], ep)
        return out.reshape(eps.shape)

    def mean_stiffness(self):
        n = float(self.ids.size)
        return sum(self.C4[p] * (idx.size / n) for p, idx in enumerate(self.index))

    def mean_stiffness_eigen(self):
        """``<lambda : eps0>``."""
        out = np.zeros((3, 3))
        if self.eigen is None:
            return out
        n = float(self.ids.size)
        for p, idx in enumerate(self.index):
            out += np.einsum("ijkl,kl->ij", self.C4[p], self.eigen[p]) * (idx.size / n)
        return out


# --------------------------------------------------------------------------
# Algorithm 1
# --------------------------------------------------------------------------
@dataclass
class Result:
    iters: int
    errs: list
    converged: bool
    u_q: np.ndarray            # displacement in q (paper convention), half spectrum
    eps: np.ndarray            # (3,3,N3,N2,N1), Eq. (final_strain)
    sig: np.ndarray            # (3,3,N3,N2,N1), Eq. (final_stress)
    sig_mean: np.ndarray       # (3,3)
    eps_bar: np.ndarray        # (3,3)
    deps1: np.ndarray = field(repr=False, default=None)
    deps2: np.ndarray = field(repr=False, default=None)
    sig1: np.ndarray = field(repr=False, default=None)
    sig2: np.ndarray = field(repr=False, default=None)


def evaluate(u_q, D, mat, eps_bar, grid, workers=None):
    """Steps 1-4 of Algorithm 1 and the equilibrium residual at state ``u_q``.

    Returns ``(deps1_r, deps2_r, sig1_r, sig2_r, f_q, L2, sig_mean)``."""
    deps1_q = sym_outer(D, u_q)                      # Eq. desp_T1_dep_Q
    deps2_q = sym_outer(-np.conj(D), u_q)            # Eq. desp_T2_dep_Q
    deps1 = ift(deps1_q, grid, workers)
    deps2 = ift(deps2_q, grid, workers)
    eb = eps_bar[:, :, None, None, None]
    sig1 = mat.stress(eb + deps1)
    sig2 = mat.stress(eb + deps2)
    s1q = ft(sig1, workers)
    s2q = ft(sig2, workers)
    # f = sigma^T1(q).conj(D) - sigma^T2(q).D   (Eq. basic_scheme_dep_2)
    f = np.einsum("ji...,i...->j...", s1q, np.conj(D)) - np.einsum("ji...,i...->j...", s2q, D)
    w = half_weights(grid)
    L2 = np.sqrt(np.sum(w * np.abs(0.5 * f) ** 2))  # Eq. (L2-norm), q-space form
    sig_mean = 0.5 * (s1q[:, :, 0, 0, 0].real + s2q[:, :, 0, 0, 0].real)
    return deps1, deps2, sig1, sig2, f, L2, sig_mean


def solve_alg1(ids, table, lam0, eps_bar=None, tol=1e-8, max_iter=1000, u0=None,
               eigen=None, applied_stress=None, callback=None, keep_T_fields=False,
               workers=None):
    """Algorithm 1 of the paper (displacement-based basic scheme).

    ``eps_bar``: applied macroscopic strain (3x3) for strain control.
    ``applied_stress``: 3x3 ``sigma^a`` for stress control (Section 2.5);
    then ``eps_bar`` starts at ``(lambda0)^-1 : sigma^a``.
    ``callback(n, err, deps1, deps2, sig_mean)`` is called after every
    evaluation.  Returns a :class:`Result`.
    """
    ids = np.asarray(ids)
    n3, n2, n1 = ids.shape
    grid = (n1, n2, n3)
    if any(n % 2 for n in grid):
        raise ValueError("N_i must be even (Section 2.1)")
    mat = Material(ids, table, eigen)
    lam0 = np.asarray(lam0, dtype=np.float64)
    D = D_of_q(grid)
    Om = green(D, lam0, grid)
    if applied_stress is not None:
        eps_bar = _solve_lam(lam0, np.asarray(applied_stress, dtype=np.float64))
    eps_bar = np.array(eps_bar, dtype=np.float64)
    u = np.zeros((3, n3, n2, n1 // 2 + 1), dtype=np.complex128) if u0 is None else np.array(u0)
    errs = []
    converged = False
    for n in range(1, max_iter + 1):
        deps1, deps2, sig1, sig2, f, L2, sig_mean = evaluate(u, D, mat, eps_bar, grid, workers)
        nrm = np.sqrt(np.sum(sig_mean ** 2))
        err = L2 / nrm if nrm > 0 else (0.0 if L2 == 0 else np.inf)  # Eq. (tolerance)
        errs.append(err)
        if callback is not None:
            callback(n, err, deps1, deps2, sig_mean)
        if err < tol:
            converged = True
            break
        if n == max_iter:
            break
        u = u - np.einsum("jk...,k...->j...", Om, f)   # Algorithm 1 step 5
        if applied_stress is not None:                  # Algorithm 1 step 6
            deps = 0.5 * (deps1 + deps2)
            lam_deps_mean = mat.stress(deps, with_eigen=False).reshape(3, 3, -1).mean(axis=2)
            rhs = (np.asarray(applied_stress)
                   + np.einsum("ijkl,kl->ij", lam0 - mat.mean_stiffness(), eps_bar)
                   - lam_deps_mean + mat.mean_stiffness_eigen())
            eps_bar = _solve_lam(lam0, rhs)
    eps = eps_bar[:, :, None, None, None] + 0.5 * (deps1 + deps2)   # Eq. (final_strain)
    sig = 0.5 * (sig1 + sig2)                                       # Eq. (final_stress)
    res = Result(iters=n, errs=errs, converged=converged, u_q=u, eps=eps, sig=sig,
                 sig_mean=sig_mean, eps_bar=eps_bar)
    if keep_T_fields:
        res.deps1, res.deps2, res.sig1, res.sig2 = deps1, deps2, sig1, sig2
    return res


def _solve_lam(lam, rhs):
    """Symmetric ``X`` with ``lam : X = rhs`` (through the 6x6 Voigt matrix)."""
    C6 = np.empty((6, 6))
    for I, (i, j) in enumerate(_PAIRS):
        for J, (k, l) in enumerate(_PAIRS):
            C6[I, J] = lam[i, j, k, l]
    r6 = np.array([rhs[i, j] for (i, j) in _PAIRS])
    x6 = np.linalg.solve(C6, r6)          # engineering shear strains
    X = np.empty((3, 3))
    for I, (i, j) in enumerate(_PAIRS):
        X[i, j] = X[j, i] = x6[I] if I < 3 else 0.5 * x6[I]
    return X


# --------------------------------------------------------------------------
# Algorithm 2 (strain form), iterate-equivalent to Algorithm 1
# --------------------------------------------------------------------------
def solve_alg2(ids, table, lam0, eps_bar, tol=1e-8, max_iter=1000, callback=None, workers=None):
    """Algorithm 2 (Eq. Lippmann_Schwinger_strain_3): iterate on the T1/T2 strains."""
    ids = np.asarray(ids)
    n3, n2, n1 = ids.shape
    grid = (n1, n2, n3)
    mat = Material(ids, table)
    D = D_of_q(grid)
    Om = green(D, np.asarray(lam0, dtype=np.float64), grid)
    G = gamma3(D, Om)
    eps_bar = np.asarray(eps_bar, dtype=np.float64)
    e1q = np.zeros((3, 3, n3, n2, n1 // 2 + 1), dtype=np.complex128)
    e2q = np.zeros_like(e1q)
    w = half_weights(grid)
    errs = []
    for n in range(1, max_iter + 1):
        deps1 = ift(e1q, grid, workers)
        deps2 = ift(e2q, grid, workers)
        eb = eps_bar[:, :, None, None, None]
        s1q = ft(mat.stress(eb + deps1), workers)
        s2q = ft(mat.stress(eb + deps2), workers)
        f = np.einsum("ji...,i...->j...", s1q, np.conj(D)) - np.einsum("ji...,i...->j...", s2q, D)
        L2 = np.sqrt(np.sum(w * np.abs(0.5 * f) ** 2))
        sig_mean = 0.5 * (s1q[:, :, 0, 0, 0].real + s2q[:, :, 0, 0, 0].real)
        err = L2 / np.sqrt(np.sum(sig_mean ** 2))
        errs.append(err)
        if callback is not None:
            callback(n, err, deps1, deps2, sig_mean)
        if err < tol or n == max_iter:
            break
        Gf = np.einsum("ijk...,k...->ij...", G, f)
        e1q = e1q - Gf
        e2q = e2q + np.einsum("ijk...,k...->ij...", np.conj(G), f)
    return errs, deps1, deps2, sig_mean


# --------------------------------------------------------------------------
# effective stiffness from 6 load cases
# --------------------------------------------------------------------------
def unit_load(J):
    """Unit tensor strain of Voigt column J (shear: eps_ij = eps_ji = 1/2)."""
    e = np.zeros(6)
    e[J] = 1.0 if J < 3 else 0.5
    return strain_tensor_from_voigt(e)


def effective_stiffness(ids, table, lam0, tol=1e-10, max_iter=2000, workers=None):
    """6x6 effective stiffness: column J = Voigt ``<sigma>`` under load ``unit_load(J)``."""
    C = np.zeros((6, 6))
    iters = []
    for J in range(6):
        r = solve_alg1(ids, table, lam0, unit_load(J), tol=tol, max_iter=max_iter, workers=workers)
        C[:, J] = voigt_from_tensor(r.sig_mean)
        iters.append(r.iters)
    return C, iters
