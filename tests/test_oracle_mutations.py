"""Plant plausible mistakes in the oracle (on the CPU) and check that its pins
catch every one: a dropped term, a wrong sign, a wrong conjugation, a wrong
normalisation, a transposed operand."""
import os

import numpy as np
import pytest

import synth
from oracle import dense as Dn
from oracle import tetra as T

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
E = T.strain_tensor_from_voigt([1e-3, -2e-4, 5e-4, 3e-4, -1e-4, 2e-3])


def _pins_hold():
    rows = np.loadtxt(os.path.join(GOLDEN, "dq_special_points.txt"))
    for row in rows:
        D = T.D_at(*(np.array(v) for v in row[:3] * np.pi))
        if not np.allclose(D, row[3::2] + 1j * row[4::2], atol=1e-12):
            return False
    grid = (4, 4, 4)
    ids = synth.random_phase_map(grid, 3, seed=1)
    table = np.stack([synth.isotropic_voigt(1.0, 0.3), synth.isotropic_voigt(10.0, 0.25),
                      synth.isotropic_voigt(0.0, 0.3)])
    rng = np.random.default_rng(0)
    A = rng.standard_normal((6, 6))
    lam0 = T.stiffness_tensor(A @ A.T + 30 * np.eye(6))
    seen = []
    try:
        T.solve_alg1(ids, table, lam0, E, tol=0, max_iter=3,
                     callback=lambda n, e, d1, d2, sm: seen.append((e, d1.copy(), d2.copy())))
    except Exception:
        return False
    P = Dn.DenseProblem(ids, table, lam0)
    for n, u in enumerate(P.richardson(E, 3)):
        d1, d2, _, _ = P.fields(u, E)
        err, _ = P.error(u, E)
        if not (np.allclose(seen[n][1], d1, atol=1e-14) and np.allclose(seen[n][2], d2, atol=1e-14)
                and abs(seen[n][0] - err) <= 1e-9 * err):
            return False
    return True


def test_pins_hold_unmutated():
    assert _pins_hold()


def _mut_D_sign(orig):
    def D_at(q1, q2, q3):
        D = orig(q1, q2, q3).copy()
        D[1] = 0.5 * (np.exp(0.5j * (q1 + q2 + q3)) - np.exp(0.5j * (q1 - q2 - q3))
                      + np.exp(0.5j * (-q1 + q2 - q3)) + np.exp(0.5j * (-q1 - q2 + q3)))
        return D
    return D_at


def _mut_drop_T2(orig):
    def evaluate(u_q, D, mat, eps_bar, grid, workers=None):
        d1, d2, s1, s2, f, L2, sm = orig(u_q, D, mat, eps_bar, grid, workers)
        s1q = T.ft(s1)
        f = np.einsum("ji...,i...->j...", s1q, np.conj(D))
        return d1, d2, s1, s2, f, L2, sm
    return evaluate


def _mut_conj_T1(orig):
    def sym_outer(a, b):
        return orig(np.conj(a), b)
    return sym_outer


def _mut_ift_norm(orig):
    def ift(field_q, grid, workers=None):
        return orig(field_q, grid, workers) / np.prod(grid)
    return ift


def _mut_L2_factor(orig):
    def evaluate(u_q, D, mat, eps_bar, grid, workers=None):
        out = list(orig(u_q, D, mat, eps_bar, grid, workers))
        out[5] = 2 * out[5]
        return tuple(out)
    return evaluate


def _mut_green_transpose(orig):
    def green(D, lam0, grid, half=True):
        Om = orig(D, lam0, grid, half)
        # transposed operand in the contraction with lambda0 (j <-> i) is invisible
        # for symmetric tensors, so plant the non-symmetric analogue: drop the
        # second term of Eq. (Green_tensor)
        A = np.einsum("i...,jikl,k...->jl...", np.conj(D), lam0, D).real
        mask = T.translation_modes(grid, half)
        A = np.moveaxis(A, (0, 1), (-2, -1)).copy()
        A[mask] = np.eye(3)
        Om2 = np.linalg.inv(A)
        Om2[mask] = 0
        return np.moveaxis(Om2, (-2, -1), (0, 1))
    return green


@pytest.mark.parametrize("name,factory", [
    ("D_at", _mut_D_sign),
    ("evaluate", _mut_drop_T2),
    ("sym_outer", _mut_conj_T1),
    ("ift", _mut_ift_norm),
    ("evaluate", _mut_L2_factor),
    ("green", _mut_green_transpose),
])
def test_planted_mistake_is_caught(monkeypatch, name, factory):
    monkeypatch.setattr(T, name, factory(getattr(T, name)))
    assert not _pins_hold()


# ---- the applied-stress loop (Section 2.5, Algorithm 1 step 6) --------------------------
def _laminate_compliance_pin_holds():
    """Stress control on a laminate reaches the closed-form compliance (inverse Backus
    stiffness) applied to sigma^a."""
    grid = (8, 4, 4)
    layers = [0, 1, 1, 0, 0, 0, 1, 0]
    ids = synth.laminate_x(grid, layers)
    table = synth.two_phase_table(1.0, 0.3, 4.0, 0.25)
    lam = np.array([t[0, 1] for t in table])
    mu = np.array([t[3, 3] for t in table])
    f = np.array([1 - np.mean(layers), np.mean(layers)])
    a = lambda x: np.sum(f * x)  # noqa: E731
    M = lam + 2 * mu
    C = np.zeros((6, 6))
    C[0, 0] = 1 / a(1 / M)
    C[0, 1] = C[1, 0] = C[0, 2] = C[2, 0] = a(lam / M) / a(1 / M)
    C[1, 1] = C[2, 2] = a(lam + 2 * mu - lam ** 2 / M) + a(lam / M) ** 2 / a(1 / M)
    C[1, 2] = C[2, 1] = a(lam - lam ** 2 / M) + a(lam / M) ** 2 / a(1 / M)
    C[3, 3] = a(mu)
    C[4, 4] = C[5, 5] = 1 / a(1 / mu)
    sa_v = np.array([0.2, -0.05, 0.1, 0.03, -0.02, 0.04])
    try:
        r = T.solve_alg1(ids, table, T.isotropic_lambda0(1.5, 1.2),
                         applied_stress=T.strain_tensor_from_voigt(sa_v), tol=1e-11, max_iter=2000)
    except Exception:
        return False
    e_eng = np.linalg.solve(C, sa_v)
    want = np.concatenate([e_eng[:3], 0.5 * e_eng[3:]])
    return bool(r.converged and np.allclose(T.voigt_from_tensor(r.eps_bar), want, rtol=0,
                                            atol=1e-8 * np.abs(want).max()))


def test_stress_loop_pin_holds_unmutated():
    assert _laminate_compliance_pin_holds()


def _mut_solve_lam_shear(orig):
    def solve_lam(lam, rhs):
        X = orig(lam, rhs)
        off = ~np.eye(3, dtype=bool)
        X[off] *= 2.0                    # engineering shear strains taken as tensor components
        return X
    return solve_lam


@pytest.mark.parametrize("mutate", ["shear_convention", "dropped_mean_stiffness"])
def test_planted_stress_loop_mistake_is_caught(monkeypatch, mutate):
    if mutate == "shear_convention":
        monkeypatch.setattr(T, "_solve_lam", _mut_solve_lam_shear(T._solve_lam))
    else:
        monkeypatch.setattr(T.Material, "mean_stiffness", lambda self: np.zeros((3, 3, 3, 3)))
    assert not _laminate_compliance_pin_holds()


# ---- the reference-medium rule (Section 3.4) ----------------------------------------------
def _mut_alpha_swapped(orig):
    def c0_alpha_rule(table):
        table = np.asarray(table, dtype=np.float64)
        lam_m, mu_m = table[0, 0, 1], table[0, 3, 3]
        lam_i, mu_i = table[1, 0, 1], table[1, 3, 3]
        k_m, k_i = lam_m + 2 * mu_m / 3, lam_i + 2 * mu_i / 3
        alpha = 0.45 if k_i < k_m else 0.55            # the two weights exchanged
        k0 = alpha * k_m + (1 - alpha) * k_i
        nu0 = lam_m / (2 * (lam_m + mu_m))
        mu0 = 3 * k0 * (1 - 2 * nu0) / (2 * (1 + nu0))
        return T.isotropic_lambda0(k0 - 2 * mu0 / 3, mu0)
    return c0_alpha_rule


def _mut_nu_from_inclusion(orig):
    def c0_alpha_rule(table):
        table = np.asarray(table, dtype=np.float64)
        lam0 = orig(table)
        # Poisson ratio taken from phase 1 instead of the matrix: same k0, other split
        lam_i, mu_i = table[1, 0, 1], table[1, 3, 3]
        nu_i = lam_i / (2 * (lam_i + mu_i)) if (lam_i + mu_i) > 0 else 0.0
        k0 = (lam0[0, 0, 0, 0] + 2 * lam0[0, 0, 1, 1]) / 3
        mu0 = 3 * k0 * (1 - 2 * nu_i) / (2 * (1 + nu_i))
        return T.isotropic_lambda0(k0 - 2 * mu0 / 3, mu0)
    return c0_alpha_rule


@pytest.mark.parametrize("factory", [_mut_alpha_swapped, _mut_nu_from_inclusion])
def test_planted_reference_medium_mistake_is_caught(monkeypatch, factory):
    from tests.test_oracle_c0_rule import alpha_rule_matches_golden

    assert alpha_rule_matches_golden()
    monkeypatch.setattr(T, "c0_alpha_rule", factory(T.c0_alpha_rule))
    assert not alpha_rule_matches_golden()
