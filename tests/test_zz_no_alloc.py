"""The allocation-free residual entry point (hs_residual_noalloc) against the
regular entry points.

hs_residual_noalloc serves callers that cannot allocate device memory
(fixed-budget real-time callers, callers whose memory belongs to another
allocator, checks run where an allocation could fail or stall).  It must give what the regular solver
gives: at a displacement state loaded with hs_set_state, one FP64 evaluation
of hs_solve reports the error and the mean stress; the no-alloc call on the
same displacement, in real space, must report the same values (FP64
tolerance 1e-10), on two calls in a row.  Its force field is also checked
element by element against the dense real-space oracle, it must leave the
device's free memory unchanged, and it must refuse ids outside the table and
sizes beyond its limits.  This file is collected last so a failure here comes
after every other test has run.
"""
import ctypes

import numpy as np
import pytest

import synth
from oracle import dense as Dn
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


def _noalloc(hs, grid, ids_dev, table, E, u_dev, force_dev):
    lib = hs.load()
    g = (ctypes.c_int * 3)(*grid)
    table = np.ascontiguousarray(table, dtype=np.float64).reshape(-1, 36)
    E = np.ascontiguousarray(E, dtype=np.float64)
    sm = np.zeros(6)
    l2 = ctypes.c_double()
    st = lib.hs_residual_noalloc(g, ctypes.c_void_p(ids_dev.data_ptr()), hs._dp(table), table.shape[0],
                                 hs._dp(E), ctypes.c_void_p(u_dev.data_ptr()),
                                 ctypes.c_void_p(force_dev.data_ptr() if force_dev is not None else 0),
                                 hs._dp(sm), ctypes.byref(l2),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, sm, l2.value


@pytest.mark.parametrize("case", ["iso_voids", "aniso"])
def test_noalloc_residual_matches_solver_evaluation(hs, case):
    grid = (16, 12, 18)
    rng = np.random.default_rng(7)
    if case == "iso_voids":
        ids = synth.random_phase_map(grid, 2, seed=3)
        table = synth.two_phase_table(2.0, 0.25, 0.0, 0.3)
    else:
        ids = synth.random_phase_map(grid, 3, seed=4)
        table = synth.polycrystal_table(168.4, 121.4, 75.4, synth.random_rotations(3, seed=6))
    C0 = synth.isotropic_voigt(float(np.max(table[:, 0, 0])), 0.25)
    E = np.array([1e-3, -2e-4, 5e-4, 3e-4, -1e-4, 2e-3])
    u_r = 1e-3 * rng.standard_normal((3, grid[2], grid[1], grid[0]))
    uc = np.fft.rfftn(u_r, axes=(1, 2, 3)) / np.prod(grid)       # corner-indexed u(q)

    # regular path: one FP64 evaluation at this state
    s = hs.Solver(ids, table, C0=C0, precision=hs.HS_FP64)
    s.set_state(torch.from_numpy(uc.copy()).cuda())
    out = s.solve(E, tol=0.0, max_iter=1, fields=False)
    sig_ref = out["sig_eff"]
    l2_ref = out["err"] * np.sqrt(np.sum(sig_ref[:3] ** 2) + 2 * np.sum(sig_ref[3:] ** 2))
    s.close()

    ids_dev = torch.from_numpy(ids.astype(np.uint16)).cuda()
    u_dev = torch.from_numpy(u_r.copy()).cuda()
    force = torch.empty((3,) + u_r.shape[1:], dtype=torch.float32, device="cuda")
    for call in range(2):           # two calls in a row share the scratch array
        st, sm, l2 = _noalloc(hs, grid, ids_dev, table, E, u_dev, force)
        assert st == hs.HS_OK
        np.testing.assert_allclose(sm, sig_ref, rtol=0, atol=1e-10 * np.abs(sig_ref).max())
        assert abs(l2 - l2_ref) <= 1e-10 * l2_ref
        f = force.double().cpu().numpy()
        assert abs(np.sqrt(np.mean(np.sum(f ** 2, axis=0))) - l2_ref) <= 1e-6 * l2_ref


def test_noalloc_rejects_sizes_beyond_its_limits(hs):
    grid = (8, 8, 8)
    ids_dev = torch.zeros((8, 8, 8), dtype=torch.int16, device="cuda")
    u_dev = torch.zeros((3, 8, 8, 8), dtype=torch.float64, device="cuda")
    E = np.array([1e-3, 0, 0, 0, 0, 0])
    big = np.tile(synth.isotropic_voigt(1.0, 0.3)[None], (1025, 1, 1))
    st, _, _ = _noalloc(hs, grid, ids_dev, big, E, u_dev, None)
    assert st == hs.HS_ERR_INVALID_ARG
    st, _, _ = _noalloc(hs, (8, 8, 26), ids_dev, big[:1], E, u_dev, None)   # prime factor 13
    assert st == hs.HS_ERR_UNSUPPORTED_SIZE
    st, _, _ = _noalloc(hs, (8, 8, 6), ids_dev, big[:1], E, u_dev, None)    # 6 planes of the 8 given
    assert st == hs.HS_OK
    st, sm, l2 = _noalloc(hs, grid, ids_dev, big[:1], E, u_dev, None)
    assert st == hs.HS_OK and l2 < 1e-15


@pytest.mark.parametrize("grid,case", [((8, 6, 4), "aniso"), ((6, 6, 6), "iso_voids")])
def test_noalloc_force_matches_dense_oracle(hs, grid, case):
    """The force field, element by element, against dE/du of the dense real-space oracle (the
    energy assembled from the printed difference operators, no FFT), at a random displacement."""
    rng = np.random.default_rng(11)
    if case == "aniso":
        ids = synth.random_phase_map(grid, 3, seed=12)
        table = synth.polycrystal_table(168.4, 121.4, 75.4, synth.random_rotations(3, seed=13))
    else:
        ids = synth.random_phase_map(grid, 3, seed=14)
        table = np.stack([synth.isotropic_voigt(1.0, 0.3), synth.isotropic_voigt(7.0, 0.2), np.zeros((6, 6))])
    E = np.array([1e-3, -2e-4, 5e-4, 3e-4, -1e-4, 2e-3])
    u_r = 1e-3 * rng.standard_normal((3, grid[2], grid[1], grid[0]))
    P = Dn.DenseProblem(ids, table)
    F_ref = P.force(u_r.reshape(-1), T.strain_tensor_from_voigt(E)).reshape(u_r.shape)
    ids_dev = torch.from_numpy(ids.astype(np.uint16)).cuda()
    u_dev = torch.from_numpy(u_r.copy()).cuda()
    force = torch.empty(u_r.shape, dtype=torch.float32, device="cuda")
    for call in range(2):
        force.fill_(float("nan"))
        st, sm, l2 = _noalloc(hs, grid, ids_dev, table, E, u_dev, force)
        assert st == hs.HS_OK
        f = force.double().cpu().numpy()
        # FP64 arithmetic, stored as float: within FP32 rounding of the largest entry
        np.testing.assert_allclose(f, F_ref, rtol=0, atol=2e-7 * np.abs(F_ref).max())
        assert abs(l2 - np.sqrt(np.mean(np.sum(F_ref ** 2, axis=0)))) <= 1e-12 * l2


def test_noalloc_changes_no_device_allocation(hs):
    """No allocation: the device's free memory and the caching allocator's reserved bytes are the
    same before and after a call (the scratch array was placed when the library loaded)."""
    grid = (32, 24, 16)
    ids = synth.random_phase_map(grid, 2, seed=5)
    table = synth.two_phase_table(1.0, 0.3, 4.0, 0.3)
    ids_dev = torch.from_numpy(ids.astype(np.uint16)).cuda()
    u_dev = 1e-3 * torch.randn((3, grid[2], grid[1], grid[0]), dtype=torch.float64, device="cuda")
    force = torch.empty(u_dev.shape, dtype=torch.float32, device="cuda")
    E = np.array([1e-3, 0, 0, 0, 0, 0])
    st, _, _ = _noalloc(hs, grid, ids_dev, table, E, u_dev, force)   # first call: address lookup
    assert st == hs.HS_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    res0 = torch.cuda.memory_reserved()
    for _ in range(3):
        st, _, _ = _noalloc(hs, grid, ids_dev, table, E, u_dev, force)
        assert st == hs.HS_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_reserved() == res0


def test_noalloc_refuses_ids_outside_the_table(hs):
    """An id >= nphase is found on the device before the residual kernel runs (the max-id pass
    only reads the ids) and the call returns HS_ERR_INVALID_ARG."""
    grid = (8, 8, 8)
    ids = np.zeros((8, 8, 8), dtype=np.uint16)
    ids[3, 4, 5] = 2
    ids_dev = torch.from_numpy(ids).cuda()
    u_dev = torch.zeros((3, 8, 8, 8), dtype=torch.float64, device="cuda")
    table = synth.two_phase_table(1.0, 0.3, 4.0, 0.3)
    E = np.array([1e-3, 0, 0, 0, 0, 0])
    st, _, _ = _noalloc(hs, grid, ids_dev, table, E, u_dev, None)
    assert st == hs.HS_ERR_INVALID_ARG
    ids[3, 4, 5] = 1
    st, _, _ = _noalloc(hs, grid, torch.from_numpy(ids).cuda(), table, E, u_dev, None)
    assert st == hs.HS_OK


@pytest.mark.parametrize("grid", [(512, 4, 4), (10, 14, 22)])
def test_noalloc_wide_rows_and_radix_5_7_11_grids(hs, grid):
    """N1 = 512 (whose FP64 plane ring needs the smaller row tile to fit in shared memory) and a
    grid with factors 5, 7 and 11 run and give the oracle's residual and mean stress (Algorithm 1
    steps 1-4 at the same displacement, q-space L2 norm) to 1e-10."""
    rng = np.random.default_rng(3)
    ids = synth.random_phase_map(grid, 2, seed=7)
    table = synth.two_phase_table(1.0, 0.3, 3.0, 0.25)
    E = np.array([1e-3, -2e-4, 5e-4, 3e-4, -1e-4, 2e-3])
    u_r = 1e-3 * rng.standard_normal((3, grid[2], grid[1], grid[0]))
    # the oracle's displacement state: corner (l+1/2, m+1/2, n+1/2) at index (l, m, n), paper phase
    q1, q2, q3 = T.q_vectors(grid)
    u_q = np.fft.rfftn(u_r, axes=(1, 2, 3)) / np.prod(grid) * np.exp(-0.5j * (q1 + q2 + q3))[None]
    mat = T.Material(ids, table)
    _, _, _, _, _, L2, sm = T.evaluate(u_q, T.D_of_q(grid), mat, T.strain_tensor_from_voigt(E), grid)
    sig_ref = T.voigt_from_tensor(sm)
    st, sig, l2 = _noalloc(hs, grid, torch.from_numpy(ids.astype(np.uint16)).cuda(), table, E,
                           torch.from_numpy(u_r.copy()).cuda(), None)
    assert st == hs.HS_OK
    np.testing.assert_allclose(sig, sig_ref, rtol=0, atol=1e-10 * np.abs(sig_ref).max())
    assert abs(l2 - L2) <= 1e-10 * L2
