"""Pins of the oracle's q-space building blocks against what the paper fixes.

Each test checks a value or identity printed or stated in the paper, a closed
form, or a library routine; none re-types the oracle's own formula.
"""
import os

import numpy as np
import pytest

from oracle import tetra as T

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_D_special_points_golden():
    """Hand-evaluated D(q) at special points (Eq. Dq), tests/golden/dq_special_points.txt."""
    rows = np.loadtxt(os.path.join(GOLDEN, "dq_special_points.txt"))
    for row in rows:
        q = row[:3] * np.pi
        D = T.D_at(np.array(q[0]), np.array(q[1]), np.array(q[2]))
        want = row[3::2] + 1j * row[4::2]
        np.testing.assert_allclose(D, want, atol=1e-15)


def test_D_one_axis_is_staggered_difference():
    """For q = (t,0,0): D = (2i sin(t/2), 0, 0), the centred staggered difference."""
    t = np.linspace(0, 2 * np.pi, 37)
    D = T.D_at(t, 0 * t, 0 * t)
    np.testing.assert_allclose(D[0], 2j * np.sin(t / 2), atol=1e-15)
    np.testing.assert_allclose(D[1:], 0, atol=1e-15)


@pytest.mark.parametrize("grid", [(4, 4, 4), (6, 6, 6), (8, 6, 4), (12, 4, 10)])
def test_D_vanishes_only_on_translation_modes(grid):
    """Section 2.2: D(q) = 0 exactly at q = 0 and q = (pi,pi,pi), nonzero elsewhere."""
    D = T.D_of_q(grid, half=False)
    mag = np.sum(np.abs(D) ** 2, axis=0)
    mask = T.translation_modes(grid, half=False)
    assert np.all(mag[mask] < 1e-28)
    assert np.min(mag[~mask]) > 1e-6


def test_D_omega_shift_relation():
    """Eq. (Fourier_component_relations_3): D(q + Q) = D(q) conj(C1(Q)), Q in Omega,
    with C1(pi s) = exp(-i pi (s1+s2+s3)/2) (Eq. functions_C1)."""
    rng = np.random.default_rng(0)
    q = rng.uniform(0, 2 * np.pi, size=(3, 50))
    for s in np.array(np.meshgrid([-1, 1], [-1, 1], [-1, 1])).reshape(3, -1).T:
        Q = np.pi * s
        C1 = np.exp(-0.5j * np.pi * s.sum())
        lhs = T.D_at(q[0] + Q[0], q[1] + Q[1], q[2] + Q[2])
        rhs = T.D_at(q[0], q[1], q[2]) * np.conj(C1)
        np.testing.assert_allclose(lhs, rhs, atol=1e-13)


def _lam0_aniso():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((6, 6))
    C6 = A @ A.T + 6 * np.eye(6)
    return T.stiffness_tensor(C6)


@pytest.mark.parametrize("lam0", [T.isotropic_lambda0(1.3, 0.7), _lam0_aniso()])
def test_green_real_symmetric_and_periodic(lam0):
    """Eqs. (displacement_Green_function_symmetry) and (Fourier_component_relations_4)."""
    rng = np.random.default_rng(1)
    q = rng.uniform(0, 2 * np.pi, size=(3, 40))
    D = T.D_at(*q)
    Dc = np.conj(D)
    full = (np.einsum("i...,jikl,k...->jl...", Dc, lam0, D)
            + np.einsum("i...,jikl,k...->jl...", D, lam0, Dc))
    assert np.max(np.abs(full.imag)) < 1e-13
    A = T.green_inverse(D, lam0)
    np.testing.assert_allclose(A, np.swapaxes(A, 0, 1), atol=1e-13)
    for s in np.array(np.meshgrid([-1, 1], [-1, 1], [-1, 1])).reshape(3, -1).T:
        A2 = T.green_inverse(T.D_at(*(q + np.pi * s[:, None])), lam0)
        np.testing.assert_allclose(A2, A, atol=1e-12)


def test_green_isotropic_closed_form():
    """Isotropic lambda0: Omega^-1 = mu0 tr(M) I + (lam0+mu0) M, M_jk = 2 Re(D_j conj D_k)."""
    lam, mu = 2.1, 0.9
    rng = np.random.default_rng(2)
    q = rng.uniform(0, 2 * np.pi, size=(3, 30))
    D = T.D_at(*q)
    M = 2 * np.real(np.einsum("j...,k...->jk...", D, np.conj(D)))
    trM = np.trace(M)
    want = mu * trM * np.eye(3)[:, :, None] + (lam + mu) * M
    got = T.green_inverse(D, T.isotropic_lambda0(lam, mu))
    np.testing.assert_allclose(got, want, atol=1e-13)


def test_green_zero_on_translation_modes_and_inverse_elsewhere():
    grid = (6, 4, 8)
    lam0 = T.isotropic_lambda0(1.0, 1.0)
    D = T.D_of_q(grid)
    Om = T.green(D, lam0, grid)
    Ainv = T.green_inverse(D, lam0)
    mask = T.translation_modes(grid)
    assert np.all(Om[:, :, mask] == 0)
    prod = np.einsum("ij...,jk...->ik...", Om, Ainv)
    eye = np.broadcast_to(np.eye(3)[:, :, None, None, None], prod.shape)
    np.testing.assert_allclose(prod[:, :, ~mask], eye[:, :, ~mask], atol=1e-12)


@pytest.mark.parametrize("lam0", [T.isotropic_lambda0(1.3, 0.7), _lam0_aniso()])
def test_green_reproduces_displacement(lam0):
    """The identity stated before Eq. (basic_scheme_dep_2):
    Omega . lambda0 : {D (x)_s u . conj(D) + conj(D) (x)_s u . D} = u (u = 0 on translation modes)."""
    grid = (6, 6, 4)
    rng = np.random.default_rng(5)
    D = T.D_of_q(grid)
    mask = T.translation_modes(grid)
    u = rng.standard_normal((3,) + D.shape[1:]) + 1j * rng.standard_normal((3,) + D.shape[1:])
    u[:, mask] = 0
    Om = T.green(D, lam0, grid)
    e1 = T.sym_outer(D, u)
    e2 = T.sym_outer(np.conj(D), u)
    s1 = np.einsum("ijkl,kl...->ij...", lam0, e1)
    s2 = np.einsum("ijkl,kl...->ij...", lam0, e2)
    v = np.einsum("ij...,j...->i...", s1, np.conj(D)) + np.einsum("ij...,j...->i...", s2, D)
    np.testing.assert_allclose(np.einsum("ij...,j...->i...", Om, v), u, atol=1e-12)


def test_strain_green_operator_symmetries_and_projection():
    """Symmetries of G^d, G^nd and the strain identities of Section 2.6."""
    grid = (4, 6, 6)
    lam0 = T.isotropic_lambda0(0.8, 1.1)
    D = T.D_of_q(grid)
    Om = T.green(D, lam0, grid)
    Gd, Gnd = T.strain_green_operators(D, Om)
    np.testing.assert_allclose(Gd, np.swapaxes(Gd, 0, 1), atol=1e-13)
    np.testing.assert_allclose(Gd, np.swapaxes(Gd, 2, 3), atol=1e-13)
    np.testing.assert_allclose(Gd, np.conj(np.transpose(Gd, (2, 3, 0, 1, 4, 5, 6))), atol=1e-13)
    np.testing.assert_allclose(Gnd, np.swapaxes(Gnd, 0, 1), atol=1e-13)
    np.testing.assert_allclose(Gnd, np.swapaxes(Gnd, 2, 3), atol=1e-13)
    np.testing.assert_allclose(Gnd, np.transpose(Gnd, (2, 3, 0, 1, 4, 5, 6)), atol=1e-13)
    G3 = T.gamma3(D, Om)
    np.testing.assert_allclose(G3, np.swapaxes(G3, 0, 1), atol=1e-13)
    # projection identities for compatible strain pairs
    rng = np.random.default_rng(7)
    mask = T.translation_modes(grid)
    u = rng.standard_normal((3,) + D.shape[1:]) + 1j * rng.standard_normal((3,) + D.shape[1:])
    u[:, mask] = 0
    e1 = T.sym_outer(D, u)
    e2 = T.sym_outer(-np.conj(D), u)
    l1 = np.einsum("ijkl,kl...->ij...", lam0, e1)
    l2 = np.einsum("ijkl,kl...->ij...", lam0, e2)
    lhs1 = np.einsum("ijkl...,kl...->ij...", Gd, l1) + np.einsum("ijkl...,kl...->ij...", Gnd, l2)
    lhs2 = (np.einsum("ijkl...,kl...->ij...", np.conj(Gnd), l1)
            + np.einsum("ijkl...,kl...->ij...", np.conj(Gd), l2))
    np.testing.assert_allclose(lhs1, e1, atol=1e-12)
    np.testing.assert_allclose(lhs2, e2, atol=1e-12)


def test_transforms_match_numpy_fft_convention():
    """Eqs. (FT), (IFT): 1/N forward, none inverse; half-spectrum weights give Parseval."""
    grid = (6, 4, 10)
    rng = np.random.default_rng(11)
    x = rng.standard_normal((2, grid[2], grid[1], grid[0]))
    X = T.ft(x)
    N = np.prod(grid)
    ref = np.fft.fftn(x, axes=(-3, -2, -1))[..., : grid[0] // 2 + 1] / N
    np.testing.assert_allclose(X, ref, atol=1e-14)
    np.testing.assert_allclose(T.ift(X, grid), x, atol=1e-13)
    w = T.half_weights(grid)
    np.testing.assert_allclose(np.sum(w * np.abs(X) ** 2), np.sum(x ** 2) / N, rtol=1e-13)
