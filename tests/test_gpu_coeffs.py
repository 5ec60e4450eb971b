"""A full per-voxel stiffness field (hs_material kind HS_COEFFS_F32, 21 coefficients
per voxel, as a device tensor or a host array) runs the same solve as the grain-id
form of the same field: bit-identical error history, effective stress and fields
(the grain-id form of the field being its FP32 coefficients widened to FP64)."""
import numpy as np
import pytest

import synth

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


@pytest.mark.parametrize("prec", [0, 2])
def test_per_voxel_stiffness_matches_grain_ids(hs, prec):
    grid = (24, 18, 12)
    gids, _ = synth.voronoi_grains(grid, 7, seed=4)
    table = synth.polycrystal_table(168.4, 121.4, 75.4, synth.random_rotations(7, seed=5))
    t32 = table.astype(np.float32).astype(np.float64)
    coeffs = np.moveaxis(hs.upper_triangle(t32)[gids.astype(np.int64)], -1, 0).astype(np.float32)
    C0 = synth.isotropic_voigt(120.0, 0.3)
    E = np.array([0, 0, 0, 0, 0, 1e-3])
    ref = hs.Solver(gids.astype(np.uint16), t32, C0=C0, precision=prec)
    want = ref.solve(E, tol=0.0, max_iter=6)
    want_hist = ref.err_history()
    ref.close()
    for src in (torch.from_numpy(coeffs).cuda(), coeffs):
        s = hs.Solver(None, None, C0=C0, precision=prec, coeffs=src)
        got = s.solve(E, tol=0.0, max_iter=6)
        np.testing.assert_array_equal(s.err_history(), want_hist)
        np.testing.assert_array_equal(got["sig_eff"], want["sig_eff"])
        assert torch.equal(got["eps"], want["eps"]) and torch.equal(got["sig"], want["sig"])
        s.close()
