"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads,
exports every function that include/hs.h declares, and rejects bad input
before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2405_11168_gb300 import build, hs

    build.build()
    return hs.load()


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "hs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hs_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_binding_exports():
    from paper_2405_11168_gb300 import hs

    assert _declared_functions() == sorted(hs.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_default_options_and_status_strings(lib):
    from paper_2405_11168_gb300 import hs

    o = hs.default_options()
    assert (o.precision, o.check_every, o.out_f32, o.inner_max) == (hs.HS_FP64, 8, 0, 200)
    assert o.inner_ratio == pytest.approx(1e-3)
    for s in range(-6, 2):
        assert lib.hs_error_string(s)


@pytest.mark.parametrize("grid,ok", [((32, 32, 32), True), ((48, 24, 12), True), ((6, 4, 8), True),
                                     ((31, 32, 32), False), ((2, 4, 4), False), ((40, 32, 32), True),
                                     ((1024, 32, 32), False), ((44, 44, 44), True), ((26, 32, 32), False),
                                     ((40, 28, 22), True)])
def test_workspace_size_validates_grid(lib, grid, ok):
    from paper_2405_11168_gb300 import hs

    if ok:
        n = hs.workspace_size(grid, 2, hs.default_options())
        nh = grid[0] // 2 + 1
        assert n >= 3 * 3 * grid[1] * grid[2] * nh * 16   # three complex128 state-sized buffers
    else:
        with pytest.raises(hs.HSError) as e:
            hs.workspace_size(grid, 2, hs.default_options())
        assert e.value.status == hs.HS_ERR_UNSUPPORTED_SIZE


def test_create_rejects_bad_arguments_before_any_device_work(lib):
    from paper_2405_11168_gb300 import hs

    ids = np.zeros((8, 8, 8), dtype=np.uint8)
    table = np.eye(6).reshape(1, 36).copy()
    ctx = ctypes.c_void_p()
    opt = hs.default_options()
    grid = (ctypes.c_int * 3)(8, 8, 7)
    m = hs.hs_material(hs.HS_IDS_U8, ctypes.c_void_p(ids.ctypes.data),
                       table.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1)
    fake_ws = ctypes.c_void_p(1 << 20)   # never dereferenced: validation fails first
    s = lib.hs_create(ctypes.byref(ctx), grid, ctypes.byref(m), None, ctypes.byref(opt), fake_ws, 1 << 30, None)
    assert s == hs.HS_ERR_UNSUPPORTED_SIZE
    grid = (ctypes.c_int * 3)(8, 8, 8)
    bad = table.reshape(6, 6).copy()
    bad[0, 1] = 1.0                      # not symmetric
    mb = hs.hs_material(hs.HS_IDS_U8, ctypes.c_void_p(ids.ctypes.data),
                        bad.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1)
    s = lib.hs_create(ctypes.byref(ctx), grid, ctypes.byref(mb), None, ctypes.byref(opt), fake_ws, 1 << 30, None)
    assert s == hs.HS_ERR_INVALID_ARG
    o2 = hs.default_options(precision=7)
    s = lib.hs_create(ctypes.byref(ctx), grid, ctypes.byref(m), None, ctypes.byref(o2), fake_ws, 1 << 30, None)
    assert s == hs.HS_ERR_INVALID_ARG
    unaligned = ctypes.c_void_p((1 << 20) + 8)
    s = lib.hs_create(ctypes.byref(ctx), grid, ctypes.byref(m), None, ctypes.byref(opt), unaligned, 1 << 30, None)
    assert s == hs.HS_ERR_INVALID_ARG
    C0 = -np.eye(6)                      # not positive definite
    s = lib.hs_create(ctypes.byref(ctx), grid, ctypes.byref(m), C0.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                      ctypes.byref(opt), fake_ws, 1 << 30, None)
    assert s == hs.HS_ERR_INVALID_ARG
    assert ctx.value is None


def test_binding_normalises_phase_ids_for_the_c_abi():
    """The binding hands the C ABI only uint8 or 16-bit contiguous ids, and
    refuses ids it would otherwise misread (floats, negatives, > 65535)."""
    torch = pytest.importorskip("torch")
    from paper_2405_11168_gb300 import hs

    cpu = torch.device("cpu")
    for dt, kind in ((torch.uint8, hs.HS_IDS_U8), (torch.int16, hs.HS_IDS_U16), (torch.int32, hs.HS_IDS_U16),
                     (torch.int64, hs.HS_IDS_U16)):
        t = torch.arange(60, dtype=torch.int64).reshape(3, 4, 5).to(dt).transpose(1, 2)
        out, k = hs._ids_tensor(t, cpu)
        assert k == kind and out.is_contiguous()
        assert torch.equal(out.to(torch.int64), t.to(torch.int64))
    out, k = hs._ids_tensor(torch.tensor([0, 40000, 65535]).reshape(1, 1, 3), cpu)
    assert k == hs.HS_IDS_U16
    assert (out.to(torch.int32) & 0xFFFF).tolist() == [[[0, 40000, 65535]]]
    with pytest.raises(ValueError):
        hs._ids_tensor(torch.tensor([-1, 0]).reshape(1, 1, 2), cpu)
    with pytest.raises(ValueError):
        hs._ids_tensor(torch.tensor([65536]).reshape(1, 1, 1), cpu)
    with pytest.raises(TypeError):
        hs._ids_tensor(torch.zeros(2, 2, 2), cpu)
    with pytest.raises(ValueError):
        hs._ids_tensor(torch.zeros(4, 4, dtype=torch.uint8), cpu)


def test_compress_coefficients_is_exact_and_ordered(lib):
    """hs_compress_coefficients (host only) turns a per-voxel stiffness field into
    phase ids and a table that reproduce every voxel's coefficients exactly, with
    phases numbered by first appearance (x fastest), -0 read as +0, and refuses
    non-finite fields or more stiffnesses than its capacity."""
    from paper_2405_11168_gb300 import hs
    import synth

    grid = (12, 10, 8)
    gids, _ = synth.voronoi_grains(grid, 7, seed=4)
    rot = synth.polycrystal_table(168.4, 121.4, 75.4, synth.random_rotations(7, seed=5)).astype(np.float32)
    coeffs = np.moveaxis(hs.upper_triangle(rot)[gids.astype(np.int64)], -1, 0).copy()  # [21][N3][N2][N1]
    ids, table = hs.compress_coefficients(coeffs)
    assert ids.dtype == np.uint16 and ids.shape == gids.shape
    assert table.shape == (len(np.unique(gids)), 6, 6)
    np.testing.assert_array_equal(np.moveaxis(hs.upper_triangle(table)[ids.astype(np.int64)], -1, 0),
                                  coeffs.astype(np.float64))
    np.testing.assert_array_equal(table, np.swapaxes(table, 1, 2))
    first = [int(v) for v in dict.fromkeys(gids.reshape(-1).tolist())]  # grains in order of appearance
    assert [int(ids.reshape(-1)[np.argmax(gids.reshape(-1) == g)]) for g in first] == list(range(len(first)))
    # -0 and +0 are one stiffness
    two = np.zeros((21, 1, 1, 2), dtype=np.float32)
    two[0] = 1.0
    two[1, 0, 0, 1] = -0.0
    ids2, table2 = hs.compress_coefficients(two)
    assert ids2.tolist() == [[[0, 0]]] and table2.shape == (1, 6, 6)
    # capacity and finiteness
    with pytest.raises(hs.HSError) as ei:
        hs.compress_coefficients(coeffs, capacity=len(first) - 1)
    assert ei.value.status == hs.HS_ERR_UNSUPPORTED_SIZE
    bad = coeffs.copy()
    bad[5, 1, 2, 3] = np.nan
    with pytest.raises(hs.HSError) as ei:
        hs.compress_coefficients(bad)
    assert ei.value.status == hs.HS_ERR_INVALID_ARG


def test_create_rejects_null_coefficient_field(lib):
    from paper_2405_11168_gb300 import hs

    g = (ctypes.c_int * 3)(8, 8, 8)
    m = hs.hs_material(hs.HS_COEFFS_F32, None, None, 0, None)
    ctx = ctypes.c_void_p()
    o = hs.default_options()
    ws = ctypes.create_string_buffer(512)
    addr = (ctypes.addressof(ws) + 255) & ~255
    st = lib.hs_create(ctypes.byref(ctx), g, ctypes.byref(m), None, ctypes.byref(o), ctypes.c_void_p(addr),
                       ctypes.c_size_t(256), None)
    assert st == hs.HS_ERR_INVALID_ARG


@pytest.mark.parametrize("field,value", [
    ("check_every", 0), ("inner_max", 0), ("inner_ratio", 0.0), ("inner_ratio", 1.0), ("zchunk", -1),
    ("ytile", 3), ("ytile", 16), ("xfuse", 2), ("col_tile", -1), ("col_tile", 12), ("col_threads", 48),
    ("col_threads", 4096), ("use_graphs", 2), ("col_copy", -1), ("col_copy", 3), ("col_pipe", 3),
])
def test_create_rejects_bad_options_before_any_device_work(lib, field, value):
    from paper_2405_11168_gb300 import hs

    ids = np.zeros((8, 8, 8), dtype=np.uint8)
    table = np.eye(6).reshape(1, 36).copy()
    m = hs.hs_material(hs.HS_IDS_U8, ctypes.c_void_p(ids.ctypes.data),
                       table.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1)
    opt = hs.default_options(**{field: value})
    ctx = ctypes.c_void_p()
    grid = (ctypes.c_int * 3)(8, 8, 8)
    s = lib.hs_create(ctypes.byref(ctx), grid, ctypes.byref(m), None, ctypes.byref(opt), ctypes.c_void_p(1 << 20),
                      1 << 30, None)
    assert s == hs.HS_ERR_INVALID_ARG, (field, value, s)
    assert ctx.value is None


def test_create_rejects_non_finite_per_voxel_stiffness(lib):
    from paper_2405_11168_gb300 import hs

    coeffs = np.zeros((21, 8, 8, 8), dtype=np.float32)
    coeffs[0] = 1.0
    coeffs[2, 3, 4, 5] = np.inf
    m = hs.hs_material(hs.HS_COEFFS_F32, None, None, 0, ctypes.c_void_p(coeffs.ctypes.data))
    ctx = ctypes.c_void_p()
    grid = (ctypes.c_int * 3)(8, 8, 8)
    opt = hs.default_options()
    s = lib.hs_create(ctypes.byref(ctx), grid, ctypes.byref(m), None, ctypes.byref(opt), ctypes.c_void_p(1 << 20),
                      1 << 30, None)
    assert s == hs.HS_ERR_INVALID_ARG
    assert ctx.value is None
