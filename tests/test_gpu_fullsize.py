"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

* 256^3 random spheres (R = 8, f = 0.30, seed 1): the first evaluations of the
  FP64 and FP32 kernels against the oracle's Algorithm 1 (error history and a
  random sample of 20000 voxels of eps and sigma); the refined path's first
  FP64 sweep and its first (FP32) solve against the oracle's first errors, then
  convergence to 1e-6.
* 512^3 periodic Voronoi polycrystal (500 grains, cubic C11/C12/C44 =
  168.4/121.4/75.4 rotated per grain, shear E12 = 1e-3, refined, tol 1e-6):
  too large for the oracle, so checked through properties that hold at any
  size: the FP64 equilibrium error reached, <eps> = E, sigma = C(r):eps voxel
  by voxel, and the reported <sigma> equals the mean of the stress field.
"""
import numpy as np
import pytest

import synth
from oracle import tetra as T

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N256 = (256, 256, 256)
E11 = np.array([1.0, 0, 0, 0, 0, 0])


@pytest.fixture(scope="module")
def hs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_11168_gb300 import build, hs as _hs

    build.build()
    _hs.load()
    return _hs


@pytest.fixture(scope="module")
def spheres256():
    ids, _ = synth.random_spheres(N256, 8.0, 0.30, 1)
    return ids


@pytest.fixture(scope="module")
def oracle256(spheres256):
    table = synth.two_phase_table(1.0, 0.3, 1e3, 0.3)
    r = T.solve_alg1(spheres256, table, T.c0_alpha_rule(table), T.strain_tensor_from_voigt(E11), tol=0.0,
                     max_iter=2)
    rng = np.random.default_rng(123)
    sample = rng.choice(spheres256.size, 20000, replace=False)
    eps = T.voigt_from_tensor(r.eps).reshape(6, -1)[:, sample]
    sig = T.voigt_from_tensor(r.sig).reshape(6, -1)[:, sample]
    return dict(table=table, errs=np.array(r.errs), sample=sample, eps=eps, sig=sig)


def _sampled(t, sample):
    idx = torch.from_numpy(sample).to(t.device)
    return t.reshape(6, -1)[:, idx].double().cpu().numpy()


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 2e-5)])
def test_256_bench_microstructure_first_iterations(hs, spheres256, oracle256, prec, tol):
    s = hs.Solver(torch.from_numpy(spheres256).cuda(), oracle256["table"], precision=prec)
    out = s.solve(E11, tol=0.0, max_iter=2)
    np.testing.assert_allclose(s.err_history(), oracle256["errs"], rtol=tol)
    for key in ("eps", "sig"):
        got = _sampled(out[key], oracle256["sample"])
        want = oracle256[key]
        assert np.abs(got - want).max() <= tol * np.abs(want).max()
    s.close()


def test_256_refined_first_sweep_and_convergence(hs, spheres256, oracle256):
    s = hs.Solver(torch.from_numpy(spheres256).cuda(), oracle256["table"], precision=hs.HS_FP32_REFINED)
    out = s.solve(E11, tol=0.0, max_iter=1)
    # one evaluation: the FP64 sweep of u = 0
    assert abs(s.err_history()[0] - oracle256["errs"][0]) <= 1e-12 * oracle256["errs"][0]
    # longer solves start with the plain FP32 basic scheme (the correction equation at u = 0)
    out = s.solve(E11, tol=0.0, max_iter=4)
    np.testing.assert_allclose(s.err_history()[:2], oracle256["errs"], rtol=2e-5)
    s.close()
    table = synth.two_phase_table(1.0, 0.3, 1e-3, 0.3)
    s = hs.Solver(torch.from_numpy(spheres256).cuda(), table, precision=hs.HS_FP32_REFINED)
    out = s.solve(E11, tol=1e-6, max_iter=5000)
    assert out["status"] == hs.HS_OK and out["err"] < 1e-6
    eps = out["eps"].reshape(6, -1)
    np.testing.assert_allclose(eps.mean(dim=1).cpu().numpy(), E11, atol=1e-12)
    s.close()


def test_512_polycrystal_refined_properties(hs):
    grid = (512, 512, 512)
    ids, _ = synth.voronoi_grains(grid, 500, seed=2)
    table = synth.polycrystal_table(168.4, 121.4, 75.4, synth.random_rotations(500, seed=3))
    E = np.array([0, 0, 0, 0, 0, 1e-3])
    s = hs.Solver(torch.from_numpy(ids.astype(np.int16)).cuda(), table, precision=hs.HS_FP32_REFINED)
    out = s.solve(E, tol=1e-6, max_iter=5000)
    assert out["status"] == hs.HS_OK and out["err"] < 1e-6
    eps = out["eps"].reshape(6, -1)
    sig = out["sig"].reshape(6, -1)
    np.testing.assert_allclose(eps.mean(dim=1).cpu().numpy(), E, atol=1e-13)
    np.testing.assert_allclose(sig.mean(dim=1).cpu().numpy(), out["sig_eff"], rtol=0,
                               atol=1e-9 * np.abs(out["sig_eff"]).max())
    rng = np.random.default_rng(7)
    sample = rng.choice(ids.size, 20000, replace=False)
    e_s = _sampled(out["eps"], sample)
    s_s = _sampled(out["sig"], sample)
    C = table[ids.reshape(-1)[sample]]                           # (n, 6, 6)
    eng = e_s.T * np.array([1, 1, 1, 2, 2, 2])
    want = np.einsum("nij,nj->in", C, eng)
    assert np.abs(s_s - want).max() <= 1e-12 * np.abs(want).max()
    s.close()
