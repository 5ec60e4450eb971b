"""Seeded periodic voxel microstructures.

Conventions (used by every generator here):

* ``grid = (N1, N2, N3)``; arrays are returned with shape ``(N3, N2, N1)``
  (row-major ``[z][y][x]``, x fastest), the layout the solver library reads.
* Voxel ``l`` occupies ``[l, l+1)`` along each axis, so its centre is at
  ``l + 1/2``; the box is periodic with period ``N_i``.  Inside tests use the
  minimum-image distance.
* Phase ids are small integers: ``uint8`` for few phases, ``uint16`` for grains.
"""
from __future__ import annotations

import numpy as np


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _centres_1d(n):
    return np.arange(n, dtype=np.float64) + 0.5


def _min_image(d, n):
    return d - n * np.round(d / n)


def centred_sphere(grid, volume_fraction=None, radius=None, centre=None):
    """One sphere of phase 1 in a matrix of phase 0.

    ``radius`` defaults to the radius whose continuous volume is
    ``volume_fraction`` of the box (for a cube ``R = N (3 f / 4 pi)^(1/3)``).
    ``centre`` defaults to the box centre ``(N1/2, N2/2, N3/2)``, which makes
    the voxel set invariant under the cube's symmetry group on a cubic grid.
    """
    n1, n2, n3 = grid
    if radius is None:
        if volume_fraction is None:
            raise ValueError("give volume_fraction or radius")
        radius = (3.0 * volume_fraction * n1 * n2 * n3 / (4.0 * np.pi)) ** (1.0 / 3.0)
    if centre is None:
        centre = (n1 / 2.0, n2 / 2.0, n3 / 2.0)
    dx = _min_image(_centres_1d(n1) - centre[0], n1)
    dy = _min_image(_centres_1d(n2) - centre[1], n2)
    dz = _min_image(_centres_1d(n3) - centre[2], n3)
    r2 = dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2
    return (r2 <= radius * radius).astype(np.uint8)


def cubic_inclusion(grid, size, centre_voxel=None):
    """A cube of ``size^3`` voxels of phase 1 (e.g. a void) in phase 0."""
    n1, n2, n3 = grid
    ids = np.zeros((n3, n2, n1), dtype=np.uint8)
    if centre_voxel is None:
        centre_voxel = (n1 // 2, n2 // 2, n3 // 2)
    lo = [c - size // 2 for c in centre_voxel]
    ix = np.arange(lo[0], lo[0] + size) % n1
    iy = np.arange(lo[1], lo[1] + size) % n2
    iz = np.arange(lo[2], lo[2] + size) % n3
    ids[np.ix_(iz, iy, ix)] = 1
    return ids


def laminate_x(grid, layer_phases):
    """Layers normal to x: voxel column ``x`` gets ``layer_phases[x]``.

    ``layer_phases`` has length ``N1``; fields of a laminate depend on x only.
    """
    n1, n2, n3 = grid
    layer_phases = np.asarray(layer_phases, dtype=np.uint8)
    if layer_phases.shape != (n1,):
        raise ValueError("layer_phases must have length N1")
    return np.broadcast_to(layer_phases[None, None, :], (n3, n2, n1)).copy()


def random_phase_map(grid, nphase, seed):
    """Independent uniform phase per voxel (a rough test medium)."""
    n1, n2, n3 = grid
    dtype = np.uint8 if nphase <= 256 else np.uint16
    return _rng(seed).integers(0, nphase, size=(n3, n2, n1)).astype(dtype)


def random_spheres(grid, radius, target_fraction, seed, max_tries=10_000_000):
    """Random sequential addition of non-overlapping periodic spheres.

    Centres are uniform in the box; a candidate is kept when its minimum-image
    distance to every kept centre is at least ``2 * radius``.  Spheres are
    added until the voxel fraction of phase 1 reaches ``target_fraction``.
    Returns ``(ids, centres)``.
    """
    n = np.array(grid, dtype=np.float64)
    rng = _rng(seed)
    ids = np.zeros((grid[2], grid[1], grid[0]), dtype=np.uint8)
    total = ids.size
    filled = 0
    centres = np.zeros((0, 3))
    r = float(radius)
    span = int(np.ceil(r)) + 1
    offs = np.arange(-span, span + 1)
    tries = 0
    while filled < target_fraction * total:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("random_spheres: target fraction not reached")
        c = rng.random(3) * n
        if centres.shape[0]:
            d = centres - c
            d -= n * np.round(d / n)
            if np.min(np.einsum("ij,ij->i", d, d)) < (2.0 * r) ** 2:
                continue
        centres = np.vstack([centres, c])
        # stamp: voxels whose centre lies within r of c (minimum image)
        base = np.floor(c).astype(np.int64)
        ix = (base[0] + offs) % grid[0]
        iy = (base[1] + offs) % grid[1]
        iz = (base[2] + offs) % grid[2]
        dx = _min_image(ix + 0.5 - c[0], n[0])
        dy = _min_image(iy + 0.5 - c[1], n[1])
        dz = _min_image(iz + 0.5 - c[2], n[2])
        inside = (dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2) <= r * r
        block = ids[np.ix_(iz, iy, ix)]
        new = inside & (block == 0)
        filled += int(new.sum())
        block[inside] = 1
        ids[np.ix_(iz, iy, ix)] = block
    return ids, centres


def voronoi_grains(grid, n_grains, seed, chunk=1 << 22):
    """Periodic Voronoi tessellation from uniform random seeds.

    Each voxel takes the id of the seed nearest to its centre under the
    minimum-image distance (``scipy.spatial.cKDTree`` with a periodic box).
    Returns ``(ids uint16, seeds)``.
    """
    from scipy.spatial import cKDTree

    n1, n2, n3 = grid
    rng = _rng(seed)
    seeds = rng.random((n_grains, 3)) * np.array([n1, n2, n3], dtype=np.float64)
    tree = cKDTree(seeds, boxsize=[n1, n2, n3])
    ids = np.empty(n1 * n2 * n3, dtype=np.uint16)
    xs = _centres_1d(n1)
    flat = np.arange(n1 * n2 * n3, dtype=np.int64)
    for start in range(0, flat.size, chunk):
        f = flat[start:start + chunk]
        x = xs[f % n1]
        y = _centres_1d(n2)[(f // n1) % n2]
        z = _centres_1d(n3)[f // (n1 * n2)]
        pts = np.stack([x, y, z], axis=1)
        _, idx = tree.query(pts, k=1, workers=-1)
        ids[start:start + chunk] = idx.astype(np.uint16)
    return ids.reshape(n3, n2, n1), seeds


def random_rotations(n, seed):
    """``n`` rotation matrices, uniform on SO(3).

    Draws a 4D standard Gaussian vector per rotation, normalises it to a unit
    quaternion ``(w, x, y, z)`` and converts it to a 3x3 matrix.
    """
    q = _rng(seed).standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R
