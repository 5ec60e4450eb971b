"""Batched solves (hs_batch_*): many RVEs of uneven size and their load cases in shared,
graph-captured launches.

Every item of a batch must give exactly what a single hs_solve of that item gives (the batched
kernels are the single-solve kernels run over a grid.z of items, with the same reductions), and
the FP64 items the oracle's iterates: the same number of evaluations, the same error history
(1e-9) and the same effective stress (1e-10).  FP32 items are held to the oracle at 1e-5, refined
items at their equilibrium tolerance."""
import numpy as np
import pytest

import synth
from oracle import tetra as T

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_11168_gb300 import build, hs as _hs

    build.build()
    _hs.load()
    return _hs


def unit(J):
    e = np.zeros(6)
    e[J] = 1.0 if J < 3 else 0.5
    return e


def mixed_batch():
    """Five RVEs in four size classes (two share 16^3), isotropic two-phase spheres of several
    contrasts (voids included) and one anisotropic 3-grain polycrystal; 1-6 loads each."""
    rves = [
        (synth.centred_sphere((16, 16, 16), volume_fraction=0.2), synth.two_phase_table(1.0, 0.3, 10.0, 0.3)),
        (synth.centred_sphere((24, 24, 24), volume_fraction=0.15), synth.two_phase_table(1.0, 0.3, 0.0, 0.3)),
        (synth.random_phase_map((16, 24, 12), 2, seed=4), synth.two_phase_table(2.0, 0.25, 30.0, 0.3)),
        (synth.centred_sphere((16, 16, 16), volume_fraction=0.3), synth.two_phase_table(1.0, 0.3, 1.5, 0.3)),
        (synth.voronoi_grains((12, 12, 12), 3, seed=2)[0],
         synth.polycrystal_table(168.4, 121.4, 75.4, synth.random_rotations(3, seed=3))),
    ]
    loads = [[0, 3, 5], [0, 1], [2, 4, 5, 1], [0, 1, 2, 3, 4, 5], [5, 0]]
    item_rve, E = [], []
    for r, js in enumerate(loads):
        for J in js:
            item_rve.append(r)
            E.append(1e-3 * unit(J))
    return rves, item_rve, np.array(E)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_batch_items_equal_single_solves(hs, prec):
    rves, item_rve, E = mixed_batch()
    tol = {0: 1e-9, 1: 1e-5, 2: 1e-8}[prec]
    stream = torch.cuda.Stream()
    b = hs.Batch(rves, item_rve, precision=prec, stream=stream, check_every=4)
    nclass, cls = b.classes()
    assert nclass == 4 and cls[0] == cls[len([0, 3, 5]) + 2 + 4]  # the two 16^3 isotropic RVEs share a class
    out = b.solve(E, tol=tol, max_iter=3000)
    out2 = b.solve(E, tol=tol, max_iter=3000)          # a second solve replays the captured graphs
    assert b.launches() > 0
    for i, r in enumerate(item_rve):
        ids, table = rves[r]
        s = hs.Solver(ids, table, precision=prec, stream=stream, check_every=4)
        ref = s.solve(E[i], tol=tol, max_iter=3000, fields=False)
        hist = s.err_history()
        s.close()
        for o in (out, out2):
            assert o["item_status"][i] == ref["status"] == hs.HS_OK, (i, o["item_status"][i], ref["status"])
            assert o["iters"][i] == ref["iters"]
            assert o["err"][i] == ref["err"]
            np.testing.assert_array_equal(o["sig_eff"][i], ref["sig_eff"])
        if prec != 2:
            np.testing.assert_array_equal(b.err_history(i), hist)
        else:  # refined: the history holds the FP64 sweeps, the last of which stopped the solve
            assert b.err_history(i)[-1] == ref["err"] == hist[-1]
    assert out["status"] == hs.HS_OK
    b.close()


def test_batch_fp64_items_follow_the_oracle(hs):
    """Every FP64 item against Algorithm 1 of the oracle: same evaluations, error history, <sigma>."""
    rves, item_rve, E = mixed_batch()
    b = hs.Batch(rves, item_rve, precision=hs.HS_FP64, stream=torch.cuda.Stream())
    out = b.solve(E, tol=1e-8, max_iter=2000)
    for i, r in enumerate(item_rve):
        ids, table = rves[r]
        if len(table) == 2:
            lam0 = T.c0_alpha_rule(table)
        else:  # cubic polycrystal: K0 and mu0 at the midpoints of the grains' ranges
            K0 = (168.4 + 2 * 121.4) / 3
            mu0 = 0.5 * (75.4 + 0.5 * (168.4 - 121.4))
            lam0 = T.isotropic_lambda0(K0 - 2 * mu0 / 3, mu0)
        ref = T.solve_alg1(ids, table, lam0, T.strain_tensor_from_voigt(E[i]), tol=1e-8, max_iter=2000)
        assert out["item_status"][i] == hs.HS_OK and out["iters"][i] == ref.iters, (i, out["iters"][i], ref.iters)
        np.testing.assert_allclose(b.err_history(i), ref.errs, rtol=1e-9, atol=1e-14)
        se = T.voigt_from_tensor(ref.sig_mean)
        np.testing.assert_allclose(out["sig_eff"][i], se, rtol=0, atol=1e-10 * np.abs(se).max())
    b.close()


def test_batch_fp32_and_refined_effective_stiffness_against_the_oracle(hs):
    """The 6x6 effective stiffness of a 16^3 sphere and a 24^3 void RVE from one batch of 12
    items, in FP32 (err < 1e-5) and FP32 + FP64 refinement (err < 1e-9), against the oracle's
    converged C_eff (1e-12): FP32 columns within 1e-4 (relative to the largest entry), refined
    within 1e-8."""
    rves = [(synth.centred_sphere((16, 16, 16), volume_fraction=0.2), synth.two_phase_table(1.0, 0.3, 10.0, 0.3)),
            (synth.centred_sphere((24, 24, 24), volume_fraction=0.15), synth.two_phase_table(1.0, 0.3, 0.0, 0.3))]
    item_rve = [r for r in range(2) for _ in range(6)]
    E = np.array([unit(J) for _ in range(2) for J in range(6)])
    refC = [T.effective_stiffness(ids, table, T.c0_alpha_rule(table), tol=1e-12, max_iter=3000)[0]
            for ids, table in rves]
    for prec, tol, bound in ((hs.HS_FP32, 1e-5, 1e-4), (hs.HS_FP32_REFINED, 1e-9, 1e-8)):
        b = hs.Batch(rves, item_rve, precision=prec, stream=torch.cuda.Stream())
        out = b.solve(E, tol=tol, max_iter=5000)
        assert out["status"] == hs.HS_OK, out["item_status"]
        for r in range(2):
            C = out["sig_eff"][6 * r:6 * r + 6].T
            np.testing.assert_allclose(C, refC[r], rtol=0, atol=bound * np.abs(refC[r]).max())
        b.close()


def test_batch_graph_replay_matches_plain_launches(hs):
    rves, item_rve, E = mixed_batch()
    res = []
    for graphs in (0, 1):
        b = hs.Batch(rves, item_rve, precision=hs.HS_FP32_REFINED, stream=torch.cuda.Stream(), use_graphs=graphs,
                     check_every=2)
        res.append(b.solve(E, tol=1e-7, max_iter=3000))
        b.close()
    for k in ("item_status", "iters", "err", "sig_eff"):
        np.testing.assert_array_equal(res[0][k], res[1][k])


def test_batch_rejects_bad_descriptions(hs):
    rves, item_rve, E = mixed_batch()
    with pytest.raises(hs.HSError):
        hs.Batch(rves, [0, 7], precision=hs.HS_FP64)
    b = hs.Batch(rves[:1], [0], precision=hs.HS_FP64)
    with pytest.raises(hs.HSError):
        b.solve(np.zeros((1, 6)))
    b.close()
