"""The torch.fft comparison pipeline that bench.py times beside the CUDA path
computes the same iteration as the oracle (Algorithm 1): same error history
and mean stress, iterate by iterate, in FP64 on the CPU; FP32 within rounding.
"""
import numpy as np
import pytest

import synth
from oracle import tetra as T

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("case", ["stiff_sphere", "voids", "ragged"])
def test_torch_pipeline_matches_oracle(case):
    import bench

    if case == "stiff_sphere":
        grid = (12, 12, 12)
        ids = synth.centred_sphere(grid, volume_fraction=0.2)
        table = synth.two_phase_table(1.0, 0.3, 10.0, 0.3)
        E = np.array([1e-3, 0, 0, 0, 0, 0])
    elif case == "voids":
        grid = (10, 8, 12)
        ids = synth.random_phase_map(grid, 2, seed=5)
        table = synth.two_phase_table(1.0, 0.3, 0.0, 0.3)
        E = np.array([0, 0, 0, 0.5, 0, 0])
    else:
        grid = (6, 14, 10)
        ids = synth.random_phase_map(grid, 2, seed=9)
        table = synth.two_phase_table(2.0, 0.25, 0.5, 0.25)
        E = np.array([1e-3, -2e-4, 5e-4, 3e-4, -1e-4, 2e-3])
    k = 8
    ref = T.solve_alg1(ids, table, T.c0_alpha_rule(table), T.strain_tensor_from_voigt(E), tol=0.0, max_iter=k)
    p = bench.TorchFFTPipeline(ids, table, torch.device("cpu"), dtype=torch.float64)
    errs, sms = [], []
    for _ in range(k):
        err, sm = p.step(E)
        errs.append(float(err))
        sms.append(sm.numpy())
    np.testing.assert_allclose(errs, ref.errs[:k], rtol=1e-10)
    np.testing.assert_allclose(sms[-1], T.voigt_from_tensor(ref.sig_mean), rtol=0,
                               atol=1e-12 * np.abs(sms[-1]).max())
    p32 = bench.TorchFFTPipeline(ids, table, torch.device("cpu"))
    errs32 = [float(p32.step(E)[0]) for _ in range(k)]
    np.testing.assert_allclose(errs32, ref.errs[:k], rtol=1e-4)
