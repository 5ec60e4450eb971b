"""The seeded input generators produce the structures their recipes state: the
centred sphere's radius and cubic symmetry, non-overlapping periodic spheres that
reach the target fraction, minimum-image Voronoi cells, uniform rotations, and
rotated cubic stiffnesses with the crystal's invariants."""
import itertools

import numpy as np

import synth


def _min_image(d, n):
    return d - n * np.round(d / n)


def test_centred_sphere_radius_fraction_and_cubic_symmetry():
    grid = (32, 32, 32)
    ids = synth.centred_sphere(grid, volume_fraction=0.2)
    R = 32 * (3 * 0.2 / (4 * np.pi)) ** (1 / 3)
    assert abs(R - 11.61) < 0.01
    assert abs(ids.mean() - 0.2) < 0.005
    for perm in itertools.permutations(range(3)):
        assert np.array_equal(ids, ids.transpose(perm))
    for ax in range(3):
        assert np.array_equal(ids, np.flip(ids, axis=ax))


def test_random_spheres_are_periodic_non_overlapping_balls():
    grid, R, f = (40, 32, 24), 4.0, 0.3
    ids, c = synth.random_spheres(grid, R, f, seed=3)
    n = np.array(grid, dtype=float)
    assert ids.mean() >= f
    d = c[:, None, :] - c[None, :, :]
    d = _min_image(d, n)
    dist = np.sqrt((d ** 2).sum(-1)) + np.eye(len(c)) * 1e9
    assert dist.min() >= 2 * R
    # the phase-1 voxels are exactly the voxels whose centre lies in some ball
    z, y, x = np.meshgrid(*(np.arange(k) + 0.5 for k in grid[::-1]), indexing="ij")
    inside = np.zeros(ids.shape, dtype=bool)
    for cc in c:
        r2 = (_min_image(x - cc[0], n[0]) ** 2 + _min_image(y - cc[1], n[1]) ** 2
              + _min_image(z - cc[2], n[2]) ** 2)
        inside |= r2 <= R * R
    assert np.array_equal(ids.astype(bool), inside)
    ids2, c2 = synth.random_spheres(grid, R, f, seed=3)
    assert np.array_equal(ids, ids2) and np.array_equal(c, c2)


def test_voronoi_cells_are_minimum_image_nearest_seed():
    grid = (10, 8, 6)
    ids, seeds = synth.voronoi_grains(grid, 9, seed=7)
    n = np.array(grid, dtype=float)
    z, y, x = np.meshgrid(*(np.arange(k) + 0.5 for k in grid[::-1]), indexing="ij")
    p = np.stack([x, y, z], axis=-1)[..., None, :]
    d = _min_image(p - seeds, n)
    want = np.argmin((d ** 2).sum(-1), axis=-1)
    assert np.array_equal(ids, want)


def test_rotations_are_proper_and_uniform():
    R = synth.random_rotations(20000, seed=3)
    np.testing.assert_allclose(np.einsum("nij,nkj->nik", R, R), np.broadcast_to(np.eye(3), R.shape), atol=1e-12)
    np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-12)
    # uniform on SO(3): E[R] = 0 and E[R_ij^2] = 1/3
    assert np.abs(R.mean(axis=0)).max() < 0.02
    assert np.abs((R ** 2).mean(axis=0) - 1 / 3).max() < 0.02


def test_rotated_cubic_stiffness_keeps_the_crystal_invariants():
    C11, C12, C44 = 168.4, 121.4, 75.4
    tab = synth.polycrystal_table(C11, C12, C44, synth.random_rotations(50, seed=5))
    np.testing.assert_allclose(tab, np.swapaxes(tab, 1, 2), atol=1e-9)
    # Voigt bulk modulus and the eigenvalues of the Mandel matrix are rotation invariants
    K = (tab[:, :3, :3].sum(axis=(1, 2))) / 9
    np.testing.assert_allclose(K, (C11 + 2 * C12) / 3, rtol=1e-12)
    mandel = tab.copy()
    mandel[:, :3, 3:] *= np.sqrt(2)
    mandel[:, 3:, :3] *= np.sqrt(2)
    mandel[:, 3:, 3:] *= 2
    ev = np.sort(np.linalg.eigvalsh(mandel), axis=1)
    want = np.sort([C11 + 2 * C12, C11 - C12, C11 - C12, 2 * C44, 2 * C44, 2 * C44])
    np.testing.assert_allclose(ev, np.broadcast_to(want, ev.shape), rtol=1e-10)


def test_laminate_and_void_tables():
    ids = synth.laminate_x((6, 4, 2), [0, 1, 1, 0, 1, 0])
    assert np.array_equal(ids, np.broadcast_to(ids[:1, :1, :], ids.shape))
    assert not synth.two_phase_table(1.0, 0.3, 0.0, 0.3)[1].any()
