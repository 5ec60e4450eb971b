"""Pins of the oracle's solver (Algorithm 1) against closed forms, invariants and
an independent brute-force real-space solve of the same discrete equilibrium."""
import numpy as np
import pytest

import synth
from oracle import dense as Dn
from oracle import tetra as T


def _three_phase(grid, seed):
    ids = synth.random_phase_map(grid, 3, seed=seed)
    table = np.stack([synth.isotropic_voigt(1.0, 0.3),
                      synth.isotropic_voigt(10.0, 0.25),
                      synth.isotropic_voigt(0.0, 0.3)])      # phase 2: void (C = 0)
    return ids, table


def _aniso_table(n, seed):
    R = synth.random_rotations(n, seed)
    return synth.polycrystal_table(168.4, 121.4, 75.4, R)


E_MIXED = T.strain_tensor_from_voigt([1e-3, -2e-4, 5e-4, 3e-4, -1e-4, 2e-3])


def test_homogeneous_medium_converges_in_one_evaluation():
    """Homogeneous medium: f(q) = 0 at the first evaluation, eps = E, sigma = lambda:E."""
    grid = (8, 6, 4)
    ids = np.zeros((grid[2], grid[1], grid[0]), dtype=np.uint8)
    table = synth.isotropic_voigt(3.0, 0.2)[None]
    lam0 = T.isotropic_lambda0(0.4, 2.5)          # deliberately not the medium
    r = T.solve_alg1(ids, table, lam0, E_MIXED, tol=1e-12, max_iter=50)
    assert r.iters == 1 and r.converged and r.errs[0] == 0.0
    np.testing.assert_allclose(r.eps, np.broadcast_to(E_MIXED[:, :, None, None, None], r.eps.shape), atol=1e-18)
    s = np.einsum("ijkl,kl->ij", T.stiffness_tensor(table[0]), E_MIXED)
    np.testing.assert_allclose(r.sig_mean, s, rtol=1e-14)


def _laminate_closed_form(table, fractions):
    """Backus averages for layers normal to x (isotropic phases)."""
    lam = np.array([t[0, 1] for t in table])
    mu = np.array([t[3, 3] for t in table])
    M = lam + 2 * mu
    f = np.asarray(fractions)
    a = lambda x: np.sum(f * x)
    C = np.zeros((6, 6))
    C[0, 0] = 1 / a(1 / M)
    C[0, 1] = C[1, 0] = C[0, 2] = C[2, 0] = a(lam / M) / a(1 / M)
    C[1, 1] = C[2, 2] = a(lam + 2 * mu - lam ** 2 / M) + a(lam / M) ** 2 / a(1 / M)
    C[1, 2] = C[2, 1] = a(lam - lam ** 2 / M) + a(lam / M) ** 2 / a(1 / M)
    C[3, 3] = a(mu)
    C[4, 4] = C[5, 5] = 1 / a(1 / mu)
    return C


def test_laminate_matches_backus_closed_form():
    """Fields depending on x only: the stencil reduces to the exact staggered 1D
    difference, so C_eff equals the Backus/Reuss/Voigt closed forms."""
    grid = (8, 4, 4)
    layers = [0, 0, 1, 1, 1, 0, 1, 0]
    ids = synth.laminate_x(grid, layers)
    table = synth.two_phase_table(1.0, 0.3, 7.0, 0.2)
    lam0 = T.isotropic_lambda0(2.0, 2.0)          # 2 lambda0 >= both phases
    C, _ = T.effective_stiffness(ids, table, lam0, tol=1e-12)
    f1 = np.mean(layers)
    want = _laminate_closed_form(table, [1 - f1, f1])
    np.testing.assert_allclose(C, want, rtol=1e-9, atol=1e-9 * np.abs(want).max())


@pytest.mark.parametrize("grid,seed", [((4, 4, 4), 1), ((6, 6, 6), 2), ((6, 4, 8), 3)])
def test_iterates_match_dense_richardson(grid, seed):
    """Algorithm 1 (q-space) iterate by iterate == real-space basic scheme
    u <- u - K0^+ (K u + g) built from the printed difference operators; the
    error values agree too (pins the L2 norm, the f/2 force and Parseval)."""
    ids, table = _three_phase(grid, seed)
    lam0 = T.isotropic_lambda0(3.0, 2.0)
    seen = []
    T.solve_alg1(ids, table, lam0, E_MIXED, tol=0, max_iter=5,
                 callback=lambda n, e, d1, d2, sm: seen.append((e, d1.copy(), d2.copy(), sm.copy())))
    P = Dn.DenseProblem(ids, table, lam0)
    for n, u in enumerate(P.richardson(E_MIXED, 5)):
        d1, d2, _, _ = P.fields(u, E_MIXED)
        err, sm = P.error(u, E_MIXED)
        scale = np.abs(E_MIXED).max()
        np.testing.assert_allclose(seen[n][1], d1, atol=1e-12 * scale)
        np.testing.assert_allclose(seen[n][2], d2, atol=1e-12 * scale)
        np.testing.assert_allclose(seen[n][3], sm, atol=1e-12 * np.abs(sm).max())
        assert abs(seen[n][0] - err) <= 1e-10 * err


def test_fixed_point_matches_dense_pseudoinverse_solve():
    grid = (6, 6, 4)
    ids = synth.random_phase_map(grid, 4, seed=9)
    table = _aniso_table(4, seed=4)
    lam0 = T.isotropic_lambda0(137.07 - 2 * 49.45 / 3, 49.45)
    r = T.solve_alg1(ids, table, lam0, E_MIXED, tol=1e-13, max_iter=5000, keep_T_fields=True)
    assert r.converged
    P = Dn.DenseProblem(ids, table)
    u = P.solve(E_MIXED)
    d1, d2, s1, s2 = P.fields(u, E_MIXED)
    np.testing.assert_allclose(r.deps1, d1, atol=1e-11 * np.abs(E_MIXED).max())
    np.testing.assert_allclose(r.deps2, d2, atol=1e-11 * np.abs(E_MIXED).max())
    np.testing.assert_allclose(r.sig, 0.5 * (s1 + s2), atol=1e-10 * np.abs(s1).max())


def test_dense_force_is_energy_gradient():
    """Central finite differences of the printed energy == the assembled force."""
    grid = (4, 4, 4)
    ids, table = _three_phase(grid, 4)
    P = Dn.DenseProblem(ids, table)
    rng = np.random.default_rng(0)
    u = 1e-3 * rng.standard_normal(3 * P.N)
    F = P.force(u, E_MIXED)
    h = 1e-6
    for k in rng.choice(3 * P.N, 12, replace=False):
        e = np.zeros_like(u)
        e[k] = h
        fd = (P.energy(u + e, E_MIXED) - P.energy(u - e, E_MIXED)) / (2 * h)
        assert abs(fd - F[k]) <= 1e-7 * max(1.0, np.abs(F).max())


def test_strain_form_is_iterate_equivalent():
    """Algorithm 2 (strain form) gives the same iterates as Algorithm 1 (Section 2.6)."""
    grid = (6, 6, 6)
    ids, table = _three_phase(grid, 5)
    lam0 = T.isotropic_lambda0(3.0, 2.0)
    a1, a2 = [], []
    T.solve_alg1(ids, table, lam0, E_MIXED, tol=0, max_iter=6,
                 callback=lambda n, e, d1, d2, sm: a1.append((e, d1.copy(), d2.copy())))
    T.solve_alg2(ids, table, lam0, E_MIXED, tol=0, max_iter=6,
                 callback=lambda n, e, d1, d2, sm: a2.append((e, d1.copy(), d2.copy())))
    for x, y in zip(a1, a2):
        assert abs(x[0] - y[0]) <= 1e-12 * x[0]
        np.testing.assert_allclose(x[1], y[1], atol=1e-15)
        np.testing.assert_allclose(x[2], y[2], atol=1e-15)


def _sphere_case(grid=(10, 10, 10), contrast=10.0):
    ids = synth.centred_sphere(grid, volume_fraction=0.2)
    table = synth.two_phase_table(1.0, 0.3, contrast, 0.3)
    return ids, table


def test_effective_stiffness_bounds_symmetry_and_cubic_symmetry():
    ids, table = _sphere_case()
    lam0 = T.c0_alpha_rule(table)
    C, _ = T.effective_stiffness(ids, table, lam0, tol=1e-11)
    np.testing.assert_allclose(C, C.T, atol=1e-8 * np.abs(C).max())
    f = ids.mean()
    voigt = (1 - f) * table[0] + f * table[1]
    reuss = np.linalg.inv((1 - f) * np.linalg.inv(table[0]) + f * np.linalg.inv(table[1]))
    assert np.min(np.linalg.eigvalsh(voigt - C)) > -1e-9
    assert np.min(np.linalg.eigvalsh(C - reuss)) > -1e-9
    # cubic symmetry of the centred sphere
    np.testing.assert_allclose(np.diag(C)[:3], C[0, 0], rtol=1e-8)
    np.testing.assert_allclose(np.diag(C)[3:], C[3, 3], rtol=1e-8)
    np.testing.assert_allclose([C[0, 1], C[0, 2], C[1, 2]], C[0, 1], rtol=1e-8)
    assert np.abs(C[:3, 3:]).max() < 1e-8 * C[0, 0]
    assert np.abs(C[3:, 3:] - np.diag(np.diag(C[3:, 3:]))).max() < 1e-8 * C[0, 0]


def test_fixed_point_independent_of_reference_medium():
    ids, table = _three_phase((6, 6, 6), 6)
    ra = T.solve_alg1(ids, table, T.isotropic_lambda0(3.0, 2.0), E_MIXED, tol=1e-12, max_iter=5000)
    rb = T.solve_alg1(ids, table, T.isotropic_lambda0(6.0, 3.5), E_MIXED, tol=1e-12, max_iter=5000)
    assert ra.converged and rb.converged
    np.testing.assert_allclose(ra.sig, rb.sig, atol=1e-9 * np.abs(ra.sig).max())
    np.testing.assert_allclose(ra.eps, rb.eps, atol=1e-9 * np.abs(ra.eps).max())


def test_hill_mandel_at_convergence():
    """1/2 <sigma^T1 : eps^T1 + sigma^T2 : eps^T2> = <sigma> : E at equilibrium."""
    ids, table = _sphere_case((8, 8, 8), 20.0)
    r = T.solve_alg1(ids, table, T.c0_alpha_rule(table), E_MIXED, tol=1e-12,
                     max_iter=2000, keep_T_fields=True)
    e1 = E_MIXED[:, :, None, None, None] + r.deps1
    e2 = E_MIXED[:, :, None, None, None] + r.deps2
    lhs = 0.5 * (np.einsum("ij...,ij...->...", r.sig1, e1).mean()
                 + np.einsum("ij...,ij...->...", r.sig2, e2).mean())
    rhs = np.einsum("ij,ij->", r.sig_mean, E_MIXED)
    assert abs(lhs - rhs) <= 1e-10 * abs(rhs)


def test_applied_stress_loop():
    """Section 2.5: under applied stress, <sigma> -> sigma^a, and the solution is the
    strain-controlled solution at the converged average strain."""
    ids, table = _sphere_case((8, 8, 8), 5.0)
    lam0 = T.c0_alpha_rule(table)
    sa = T.strain_tensor_from_voigt([0.3, -0.1, 0.05, 0.02, 0.0, 0.1])
    r = T.solve_alg1(ids, table, lam0, applied_stress=sa, tol=1e-12, max_iter=3000)
    assert r.converged
    np.testing.assert_allclose(r.sig_mean, sa, atol=1e-9 * np.abs(sa).max())
    r2 = T.solve_alg1(ids, table, lam0, r.eps_bar, tol=1e-12, max_iter=3000)
    np.testing.assert_allclose(r2.sig, r.sig, atol=1e-9 * np.abs(r.sig).max())


def test_applied_stress_on_a_laminate_gives_the_closed_form_compliance():
    """Section 2.5 under stress control on a laminate: the converged average strain is
    the closed-form compliance (inverse of the Backus stiffness) applied to sigma^a,
    and the layers carry the stress components that continuity fixes (sigma_11,
    sigma_12, sigma_13 uniform through the layers)."""
    grid = (8, 4, 4)
    layers = [0, 1, 1, 0, 0, 0, 1, 0]
    ids = synth.laminate_x(grid, layers)
    table = synth.two_phase_table(1.0, 0.3, 4.0, 0.25)
    lam0 = T.isotropic_lambda0(1.5, 1.2)
    sa_v = np.array([0.2, -0.05, 0.1, 0.03, -0.02, 0.04])
    r = T.solve_alg1(ids, table, lam0, applied_stress=T.strain_tensor_from_voigt(sa_v), tol=1e-12,
                     max_iter=5000)
    assert r.converged
    C = _laminate_closed_form(table, [1 - np.mean(layers), np.mean(layers)])
    e_eng = np.linalg.solve(C, sa_v)
    want = np.concatenate([e_eng[:3], 0.5 * e_eng[3:]])  # tensor components
    np.testing.assert_allclose(T.voigt_from_tensor(r.eps_bar), want, rtol=0, atol=1e-9 * np.abs(want).max())
    sig = T.voigt_from_tensor(r.sig)                      # [6][N3][N2][N1]
    for i in (0, 4, 5):                                   # sigma_11, sigma_13, sigma_12: traction continuity
        np.testing.assert_allclose(sig[i], sa_v[i], rtol=0, atol=1e-8 * np.abs(sa_v).max())


def test_eigenstrain_matches_dense_solve():
    """Eq. (linear_elasticity) with an eigenstrain in phase 1, zero applied strain."""
    grid = (6, 6, 6)
    ids = synth.cubic_inclusion(grid, 2)
    table = np.stack([synth.isotropic_voigt(2.0, 0.26)] * 2)
    eig = np.zeros((2, 3, 3))
    eig[1, 2, 2] = 1e-2
    lam0 = T.isotropic_lambda0(*(lambda t: (t[0, 1], t[3, 3]))(table[0]))
    r = T.solve_alg1(ids, table, lam0, np.zeros((3, 3)), tol=1e-13, max_iter=2000,
                     eigen=eig, keep_T_fields=True)
    assert r.converged
    P = Dn.DenseProblem(ids, table, eigen=eig)
    u = P.solve(np.zeros((3, 3)))
    _, _, s1, s2 = P.fields(u, np.zeros((3, 3)))
    np.testing.assert_allclose(r.sig, 0.5 * (s1 + s2), atol=1e-10 * np.abs(s1).max())


def test_homogeneous_with_lam0_equal_medium_solves_inclusion_eigenstrain_in_one_update():
    """lambda0 = lambda (homogeneous elasticity): the basic scheme is exact after one update."""
    grid = (6, 6, 6)
    ids = synth.cubic_inclusion(grid, 2)
    table = np.stack([synth.isotropic_voigt(2.0, 0.26)] * 2)
    eig = np.zeros((2, 3, 3))
    eig[1, 0, 0] = 1e-2
    lam0 = T.stiffness_tensor(table[0])
    r = T.solve_alg1(ids, table, lam0, np.zeros((3, 3)), tol=1e-12, max_iter=10, eigen=eig)
    assert r.converged and r.iters == 2
