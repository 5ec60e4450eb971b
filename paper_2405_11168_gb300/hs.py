"""Thin ctypes binding of the C ABI in ``include/hs.h`` (argument marshalling only).

Every function here forwards to the function of the same name in
``libhs.so``; all arithmetic runs in the library's CUDA kernels.  Loading
fails loudly when the library has not been built.

``Solver`` is a convenience wrapper that allocates the workspace as a PyTorch
tensor (PyTorch provides device memory and the stream) and calls
``hs_create`` / ``hs_solve`` / ``hs_destroy``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhs.so")

HS_OK = 0
HS_NOT_CONVERGED = 1
HS_ERR_INVALID_ARG = -1
HS_ERR_UNSUPPORTED_SIZE = -2
HS_ERR_OOM = -3
HS_ERR_CUDA = -4
HS_DIVERGED = -5
HS_ERR_TIMEOUT = -6

HS_FP64, HS_FP32, HS_FP32_REFINED = 0, 1, 2
KERNEL_CLASSES = ["xpass", "y_fwd", "z_green", "y_inv", "resid64", "fields", "other", "x_inv", "x_fwd", "xpass_src"]
HS_IDS_U8, HS_IDS_U16, HS_COEFFS_F32 = 0, 1, 2
HS_MAX_PHASES = 65536

# every exported function of include/hs.h
EXPORTS = [
    "hs_default_options",
    "hs_autotune",
    "hs_workspace_size",
    "hs_create",
    "hs_solve",
    "hs_solve_stress",
    "hs_set_eigenstrain",
    "hs_err_history",
    "hs_get_state",
    "hs_set_state",
    "hs_get_reference_medium",
    "hs_profile_enable",
    "hs_profile_read",
    "hs_residual_noalloc",
    "hs_compress_coefficients",
    "hs_create_sized",
    "hs_set_material",
    "hs_get_displacement",
    "hs_batch_workspace_size",
    "hs_batch_create",
    "hs_batch_solve",
    "hs_batch_err_history",
    "hs_batch_launches",
    "hs_batch_classes",
    "hs_batch_last_error",
    "hs_batch_destroy",
    "hs_destroy",
    "hs_error_string",
    "hs_last_error",
]


class hs_material(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("ids", ctypes.c_void_p),
                ("table", ctypes.POINTER(ctypes.c_double)), ("nphase", ctypes.c_int),
                ("coeffs", ctypes.c_void_p)]


class hs_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("check_every", ctypes.c_int), ("out_f32", ctypes.c_int),
                ("inner_max", ctypes.c_int), ("inner_ratio", ctypes.c_double), ("zchunk", ctypes.c_int),
                ("ytile", ctypes.c_int), ("xfuse", ctypes.c_int), ("col_tile", ctypes.c_int),
                ("col_threads", ctypes.c_int), ("use_graphs", ctypes.c_int), ("col_state", ctypes.c_int),
                ("col_pipe", ctypes.c_int), ("col_copy", ctypes.c_int)]


class HSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load ``libhs.so`` (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} not built; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I = ctypes.c_int
    D = ctypes.c_double
    dptr = ctypes.POINTER(ctypes.c_double)
    iptr = ctypes.POINTER(ctypes.c_int)
    lib.hs_default_options.argtypes = [ctypes.POINTER(hs_options)]
    lib.hs_workspace_size.argtypes = [ctypes.POINTER(ctypes.c_int), I, ctypes.POINTER(hs_options),
                                      ctypes.POINTER(ctypes.c_size_t)]
    lib.hs_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(hs_material),
                              dptr, ctypes.POINTER(hs_options), P, ctypes.c_size_t, P]
    lib.hs_solve.argtypes = [P, dptr, D, I, P, P, dptr, iptr, dptr]
    lib.hs_create_sized.argtypes = [ctypes.POINTER(P), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(hs_material),
                                    dptr, ctypes.POINTER(hs_options), I, P, ctypes.c_size_t, P]
    lib.hs_set_material.argtypes = [P, ctypes.POINTER(hs_material), dptr]
    lib.hs_get_displacement.argtypes = [P, P]
    lib.hs_autotune.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(hs_material),
                                ctypes.POINTER(hs_options), P, ctypes.c_size_t, P, I,
                                ctypes.POINTER(hs_options), dptr]
    lib.hs_solve_stress.argtypes = [P, dptr, D, I, P, P, dptr, dptr, iptr, dptr]
    lib.hs_set_eigenstrain.argtypes = [P, dptr]
    lib.hs_err_history.argtypes = [P, dptr, I, iptr]
    lib.hs_get_state.argtypes = [P, P]
    lib.hs_set_state.argtypes = [P, P]
    lib.hs_get_reference_medium.argtypes = [P, dptr]
    lib.hs_profile_enable.argtypes = [P, I]
    lib.hs_profile_read.argtypes = [P, dptr, ctypes.POINTER(ctypes.c_longlong)]
    lib.hs_residual_noalloc.argtypes = [ctypes.POINTER(ctypes.c_int), P, dptr, I, dptr, P, P, dptr, dptr, P]
    lib.hs_compress_coefficients.argtypes = [ctypes.POINTER(ctypes.c_int), P, P, dptr, I, iptr]
    lib.hs_batch_workspace_size.argtypes = [I, iptr, iptr, I, iptr, ctypes.POINTER(hs_options),
                                            ctypes.POINTER(ctypes.c_size_t)]
    lib.hs_batch_create.argtypes = [ctypes.POINTER(P), I, iptr, ctypes.POINTER(hs_material), I, iptr,
                                    ctypes.POINTER(hs_options), I, P, ctypes.c_size_t, P]
    lib.hs_batch_solve.argtypes = [P, dptr, D, I, dptr, iptr, dptr, iptr]
    lib.hs_batch_err_history.argtypes = [P, I, dptr, I, iptr]
    lib.hs_batch_launches.argtypes = [P, ctypes.POINTER(ctypes.c_longlong)]
    lib.hs_batch_classes.argtypes = [P, iptr, iptr]
    lib.hs_batch_last_error.argtypes = [P]
    lib.hs_batch_last_error.restype = ctypes.c_char_p
    lib.hs_batch_destroy.argtypes = [P]
    lib.hs_batch_destroy.restype = None
    lib.hs_destroy.argtypes = [P]
    lib.hs_destroy.restype = None
    lib.hs_error_string.argtypes = [I]
    lib.hs_error_string.restype = ctypes.c_char_p
    lib.hs_last_error.argtypes = [P]
    lib.hs_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("hs_destroy", "hs_error_string", "hs_last_error", "hs_batch_destroy", "hs_batch_last_error"):
            getattr(lib, name).restype = I
    _lib = lib
    return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ids_tensor(ids, device):
    """Phase ids as a contiguous device tensor the C ABI can read: uint8 stays
    uint8 (HS_IDS_U8); every other integer type becomes 16-bit (HS_IDS_U16,
    int16 carrying the uint16 bit pattern)."""
    import torch

    t = ids if isinstance(ids, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(ids))
    if t.dtype.is_floating_point or t.dtype.is_complex or t.dtype == torch.bool:
        raise TypeError(f"phase ids must be an integer array, got {t.dtype}")
    if t.dim() != 3:
        raise ValueError(f"phase ids must be [N3][N2][N1], got shape {tuple(t.shape)}")
    if t.dtype != torch.uint8 and t.dtype != torch.int16:
        if t.numel() and (int(t.min()) < 0 or int(t.max()) > 65535):
            raise ValueError("phase ids must lie in 0..65535")
        t = t.to(torch.int32).to(torch.int16)  # wraps 32768..65535 to the same 16-bit pattern
    t = t.to(device).contiguous()
    kind = HS_IDS_U8 if t.dtype == torch.uint8 else HS_IDS_U16
    return t, kind


def _check(lib, s, ctx=None):
    if s < 0:
        msg = lib.hs_last_error(ctx).decode() if ctx is not None else lib.hs_last_error(None).decode()
        raise HSError(s, f"{lib.hs_error_string(s).decode()}: {msg}")
    return s


def default_options(**kw):
    lib = load()
    o = hs_options()
    lib.hs_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def workspace_size(grid, nphase, opt):
    lib = load()
    g = (ctypes.c_int * 3)(*grid)
    n = ctypes.c_size_t()
    _check(lib, lib.hs_workspace_size(g, int(nphase), ctypes.byref(opt), ctypes.byref(n)))
    return n.value


OPTION_FIELDS = [f for f, _ in hs_options._fields_]


def upper_triangle(C):
    """The 21 upper-triangle entries of 6x6 stiffness matrices (..., 6, 6), in the row order of
    hs_material.coeffs (C11 C12 .. C16 C22 .. C66)."""
    C = np.asarray(C)
    iu = np.triu_indices(6)
    return C[..., iu[0], iu[1]]


def compress_coefficients(coeffs, capacity=HS_MAX_PHASES):
    """hs_compress_coefficients on a host array [21][N3][N2][N1]: (ids uint16 [N3][N2][N1],
    table [nphase, 6, 6]), exact (voxels with identical coefficients share a phase)."""
    lib = load()
    c = np.ascontiguousarray(coeffs, dtype=np.float32)
    if c.ndim != 4 or c.shape[0] != 21:
        raise ValueError(f"coefficients must be [21][N3][N2][N1], got {c.shape}")
    n3, n2, n1 = c.shape[1:]
    ids = np.empty((n3, n2, n1), dtype=np.uint16)
    table = np.empty((capacity, 36))
    n = ctypes.c_int()
    g = (ctypes.c_int * 3)(n1, n2, n3)
    _check(lib, lib.hs_compress_coefficients(g, c.ctypes.data, ids.ctypes.data, _dp(table), int(capacity),
                                             ctypes.byref(n)))
    return ids, table[: n.value].reshape(-1, 6, 6).copy()


def autotune(ids, table, precision=HS_FP32, iters=8, device="cuda", stream=None, **optkw):
    """hs_autotune on a device copy of ``ids``; returns (options dict, ms per evaluation or -1 if cached)."""
    import torch

    lib = load()
    dev = ids.device if isinstance(ids, torch.Tensor) and ids.is_cuda else torch.device(device)
    ids_t, kind = _ids_tensor(ids, dev)
    table = np.ascontiguousarray(np.asarray(table, dtype=np.float64).reshape(-1, 6, 6))
    shape = tuple(ids_t.shape)
    grid = (shape[2], shape[1], shape[0])
    base = default_options(precision=precision, **optkw)
    nbytes = workspace_size(grid, table.shape[0], base)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=ids_t.device)
    ptr = (ws.data_ptr() + 255) & ~255
    m = hs_material(kind, ctypes.c_void_p(ids_t.data_ptr()), _dp(table), table.shape[0], None)
    st = stream if stream is not None else torch.cuda.current_stream(ids_t.device)
    st.wait_stream(torch.cuda.current_stream(ids_t.device))
    best = hs_options()
    ms = ctypes.c_double()
    g = (ctypes.c_int * 3)(*grid)
    _check(lib, lib.hs_autotune(g, ctypes.byref(m), ctypes.byref(base), ctypes.c_void_p(ptr), ctypes.c_size_t(nbytes),
                                ctypes.c_void_p(st.cuda_stream), int(iters), ctypes.byref(best), ctypes.byref(ms)))
    torch.cuda.synchronize(ids_t.device)
    return {f: getattr(best, f) for f in OPTION_FIELDS}, ms.value


class Solver:
    """One microstructure on one device (thin wrapper over hs_create / hs_solve)."""

    def __init__(self, ids, table, C0=None, precision=HS_FP64, device="cuda", stream=None, coeffs=None,
                 layout_nphase=None, **optkw):
        """ids [N3][N2][N1] and table [nphase][6][6]; or ids = table = None and ``coeffs``, the full
        stiffness of every voxel as [21][N3][N2][N1] float32 (upper triangles, host array or
        device tensor), which the library stores exactly as phases.  ``layout_nphase``: size the
        workspace for this many phases (hs_create_sized), so that set_material can bind any
        material of up to that many phases later."""
        import torch

        self.lib = load()
        self.torch = torch
        if coeffs is not None:
            shape = tuple(coeffs.shape[1:])
        else:
            shape = tuple(ids.shape)
        ids_t = ids if isinstance(ids, torch.Tensor) else None
        self.grid = (shape[2], shape[1], shape[0])
        self.N = int(np.prod(shape))
        self.opt = default_options(precision=precision, **optkw)
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        if coeffs is not None:
            table = np.zeros((1, 6, 6))
            self.nphase = HS_MAX_PHASES  # workspace for the largest phase count the field may hold
        else:
            table = np.ascontiguousarray(np.asarray(table, dtype=np.float64).reshape(-1, 6, 6))
            self.nphase = table.shape[0]
        self.layout_nphase = max(self.nphase, int(layout_nphase or 0))
        nbytes = workspace_size(self.grid, self.layout_nphase, self.opt)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) & ~255
        if coeffs is not None:
            if isinstance(coeffs, torch.Tensor):
                ct = coeffs.to(dtype=torch.float32).contiguous()
                self.stream.wait_stream(torch.cuda.current_stream(ct.device) if ct.is_cuda
                                        else torch.cuda.current_stream(device))
                cptr = ct.data_ptr()
            else:
                ct = np.ascontiguousarray(coeffs, dtype=np.float32)
                cptr = ct.ctypes.data
            if tuple(ct.shape)[0] != 21 or len(ct.shape) != 4:
                raise ValueError(f"coefficients must be [21][N3][N2][N1], got {tuple(ct.shape)}")
            self._ids_keep = ct
            kind, ids_ptr = HS_COEFFS_F32, None
        elif ids_t is None:
            # host ids: hs_create copies them to the device
            ids_np = np.ascontiguousarray(ids)
            if ids_np.ndim != 3 or ids_np.dtype.kind not in "iu":
                raise TypeError(f"phase ids must be an integer [N3][N2][N1] array, got {ids_np.dtype} "
                                f"{ids_np.shape}")
            kind = HS_IDS_U8 if ids_np.dtype == np.uint8 else HS_IDS_U16
            if kind == HS_IDS_U16 and ids_np.size and (ids_np.min() < 0 or ids_np.max() > 65535):
                raise ValueError("phase ids must lie in 0..65535")
            ids_np = ids_np.astype(np.uint8 if kind == HS_IDS_U8 else np.uint16, copy=False)
            ids_ptr = ids_np.ctypes.data
            self._ids_keep = ids_np
        else:
            dev = ids_t.device if ids_t.is_cuda else torch.device(device)
            ids_t, kind = _ids_tensor(ids_t, dev)
            # hs_create reads the ids on the solver's stream: order it after the work
            # that produced them (and any conversion above) on the current stream
            self.stream.wait_stream(torch.cuda.current_stream(ids_t.device))
            ids_ptr = ids_t.data_ptr()
            self._ids_keep = ids_t
        self._table = table
        if kind == HS_COEFFS_F32:
            m = hs_material(kind, None, None, 0, ctypes.c_void_p(cptr))
        else:
            m = hs_material(kind, ctypes.c_void_p(ids_ptr), _dp(table), self.nphase, None)
        c0 = None if C0 is None else np.ascontiguousarray(np.asarray(C0, dtype=np.float64).reshape(36))
        self._c0 = c0
        ctx = ctypes.c_void_p()
        g = (ctypes.c_int * 3)(*self.grid)
        self.workspace_bytes = nbytes
        s = self.lib.hs_create_sized(ctypes.byref(ctx), g, ctypes.byref(m), None if c0 is None else _dp(c0),
                                     ctypes.byref(self.opt), self.layout_nphase, ctypes.c_void_p(self._ws_ptr),
                                     ctypes.c_size_t(nbytes), ctypes.c_void_p(self.stream.cuda_stream))
        _check(self.lib, s)
        self.ctx = ctx

    def set_material(self, ids, table, C0=None):
        """Bind another microstructure of the same grid (hs_set_material): ids [N3][N2][N1] host
        array, table [nphase][6][6] with nphase <= layout_nphase.  Workspace, launch shapes and
        captured graphs stay resident."""
        ids_np = np.ascontiguousarray(ids)
        if tuple(ids_np.shape) != (self.grid[2], self.grid[1], self.grid[0]) or ids_np.dtype.kind not in "iu":
            raise ValueError(f"phase ids must be an integer array of shape {(self.grid[2], self.grid[1], self.grid[0])}")
        kind = HS_IDS_U8 if ids_np.dtype == np.uint8 else HS_IDS_U16
        if kind == HS_IDS_U16 and ids_np.size and (ids_np.min() < 0 or ids_np.max() > 65535):
            raise ValueError("phase ids must lie in 0..65535")
        ids_np = ids_np.astype(np.uint8 if kind == HS_IDS_U8 else np.uint16, copy=False)
        table = np.ascontiguousarray(np.asarray(table, dtype=np.float64).reshape(-1, 6, 6))
        m = hs_material(kind, ctypes.c_void_p(ids_np.ctypes.data), _dp(table), table.shape[0], None)
        c0 = None if C0 is None else np.ascontiguousarray(np.asarray(C0, dtype=np.float64).reshape(36))
        _check(self.lib, self.lib.hs_set_material(self.ctx, ctypes.byref(m), None if c0 is None else _dp(c0)),
               self.ctx)
        self._ids_keep, self._table, self._c0, self.nphase = ids_np, table, c0, table.shape[0]

    def get_displacement(self):
        """hs_get_displacement: the FP64 real-space corner displacement [3][N3][N2][N1] (torch tensor)."""
        torch = self.torch
        n1, n2, n3 = self.grid
        out = torch.empty((3, n3, n2, n1), dtype=torch.float64, device=self.workspace.device)
        _check(self.lib, self.lib.hs_get_displacement(self.ctx, ctypes.c_void_p(out.data_ptr())), self.ctx)
        return out

    def solve(self, E, tol=1e-8, max_iter=1000, fields=True, out=None):
        """Returns dict(status, iters, err, sig_eff, eps, sig); eps/sig are torch tensors [6,N3,N2,N1]
        (``out``: a pair of such tensors to write into instead of new ones)."""
        torch = self.torch
        E = np.ascontiguousarray(np.asarray(E, dtype=np.float64).reshape(6))
        eps = sig = None
        if fields and out is not None:
            eps, sig = out
        elif fields:
            dt = torch.float32 if self.opt.out_f32 else torch.float64
            shp = (6, self.grid[2], self.grid[1], self.grid[0])
            eps = torch.empty(shp, dtype=dt, device=self.workspace.device)
            sig = torch.empty(shp, dtype=dt, device=self.workspace.device)
        sig_eff = np.zeros(6)
        iters = ctypes.c_int()
        err = ctypes.c_double()
        s = self.lib.hs_solve(self.ctx, _dp(E), float(tol), int(max_iter),
                              ctypes.c_void_p(eps.data_ptr() if fields else 0),
                              ctypes.c_void_p(sig.data_ptr() if fields else 0),
                              _dp(sig_eff), ctypes.byref(iters), ctypes.byref(err))
        _check(self.lib, s, self.ctx)
        return dict(status=s, iters=iters.value, err=err.value, sig_eff=sig_eff, eps=eps, sig=sig)

    def _fields(self, fields):
        torch = self.torch
        if not fields:
            return None, None
        dt = torch.float32 if self.opt.out_f32 else torch.float64
        shp = (6, self.grid[2], self.grid[1], self.grid[0])
        return (torch.empty(shp, dtype=dt, device=self.workspace.device),
                torch.empty(shp, dtype=dt, device=self.workspace.device))

    def solve_stress(self, S, tol=1e-8, max_iter=1000, fields=True):
        """Applied-stress solve; returns dict(status, iters, err, sig_eff, E, eps, sig)."""
        S = np.ascontiguousarray(np.asarray(S, dtype=np.float64).reshape(6))
        eps, sig = self._fields(fields)
        sig_eff = np.zeros(6)
        E = np.zeros(6)
        iters = ctypes.c_int()
        err = ctypes.c_double()
        s = self.lib.hs_solve_stress(self.ctx, _dp(S), float(tol), int(max_iter),
                                     ctypes.c_void_p(eps.data_ptr() if fields else 0),
                                     ctypes.c_void_p(sig.data_ptr() if fields else 0),
                                     _dp(sig_eff), _dp(E), ctypes.byref(iters), ctypes.byref(err))
        _check(self.lib, s, self.ctx)
        return dict(status=s, iters=iters.value, err=err.value, sig_eff=sig_eff, E=E, eps=eps, sig=sig)

    def set_eigenstrain(self, eps0):
        """Per-phase eigenstrain, (nphase, 6) tensor components in Voigt order; None removes it."""
        if eps0 is None:
            _check(self.lib, self.lib.hs_set_eigenstrain(self.ctx, None), self.ctx)
            return
        e = np.ascontiguousarray(np.asarray(eps0, dtype=np.float64).reshape(-1, 6))
        _check(self.lib, self.lib.hs_set_eigenstrain(self.ctx, _dp(e)), self.ctx)

    def err_history(self, n=1 << 16):
        out = np.zeros(n)
        k = ctypes.c_int()
        _check(self.lib, self.lib.hs_err_history(self.ctx, _dp(out), n, ctypes.byref(k)), self.ctx)
        return out[: k.value]

    def get_state(self):
        torch = self.torch
        n1, n2, n3 = self.grid
        out = torch.empty((3, n3, n2, n1 // 2 + 1), dtype=torch.complex128, device=self.workspace.device)
        _check(self.lib, self.lib.hs_get_state(self.ctx, ctypes.c_void_p(out.data_ptr())), self.ctx)
        return out

    def set_state(self, uhat):
        n1, n2, n3 = self.grid
        if tuple(uhat.shape) != (3, n3, n2, n1 // 2 + 1):
            raise ValueError(f"state must be [3][N3][N2][N1/2+1], got {tuple(uhat.shape)}")
        uhat = uhat.to(device=self.workspace.device, dtype=self.torch.complex128).contiguous()
        self.stream.wait_stream(self.torch.cuda.current_stream(uhat.device))
        self._state_keep = uhat
        _check(self.lib, self.lib.hs_set_state(self.ctx, ctypes.c_void_p(uhat.data_ptr())), self.ctx)

    def reference_medium(self):
        out = np.zeros(36)
        _check(self.lib, self.lib.hs_get_reference_medium(self.ctx, _dp(out)), self.ctx)
        return out.reshape(6, 6)

    def profile(self, on=True):
        """Start timing (True, or n: one iteration chunk in n) or stop it (False / 0)."""
        _check(self.lib, self.lib.hs_profile_enable(self.ctx, int(on)), self.ctx)

    def profile_read(self):
        """{class: (ms, launches)} since the last read."""
        ms = np.zeros(len(KERNEL_CLASSES))
        n = (ctypes.c_longlong * len(KERNEL_CLASSES))()
        _check(self.lib, self.lib.hs_profile_read(self.ctx, _dp(ms), n), self.ctx)
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_CLASSES)}

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.hs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many RVEs and load cases solved in shared launches (thin wrapper over hs_batch_*).

    ``rves``: list of (ids [N3][N2][N1], table [nphase][6][6]) pairs (host arrays); ``item_rve``:
    the RVE of every item.  The workspace is one PyTorch tensor."""

    def __init__(self, rves, item_rve, precision=HS_FP32_REFINED, device="cuda", stream=None, autotune=False,
                 **optkw):
        import torch

        self.lib = load()
        self.torch = torch
        self.opt = default_options(precision=precision, **optkw)
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        nrve = len(rves)
        self._ids, self._tables = [], []
        grids = []
        for ids, table in rves:
            ids_np = np.ascontiguousarray(ids)
            if ids_np.ndim != 3 or ids_np.dtype.kind not in "iu":
                raise TypeError("phase ids must be an integer [N3][N2][N1] array")
            if ids_np.dtype != np.uint8:
                if ids_np.size and (ids_np.min() < 0 or ids_np.max() > 65535):
                    raise ValueError("phase ids must lie in 0..65535")
                ids_np = ids_np.astype(np.uint16)
            self._ids.append(ids_np)
            self._tables.append(np.ascontiguousarray(np.asarray(table, dtype=np.float64).reshape(-1, 6, 6)))
            n3, n2, n1 = ids_np.shape
            grids += [n1, n2, n3]
        self.nitem = len(item_rve)
        g = (ctypes.c_int * (3 * nrve))(*grids)
        npn = (ctypes.c_int * nrve)(*[t.shape[0] for t in self._tables])
        ir = (ctypes.c_int * self.nitem)(*[int(r) for r in item_rve])
        nbytes = ctypes.c_size_t()
        _check(self.lib, self.lib.hs_batch_workspace_size(nrve, g, npn, self.nitem, ir, ctypes.byref(self.opt),
                                                          ctypes.byref(nbytes)))
        self.workspace_bytes = nbytes.value
        self.workspace = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=device)
        ptr = (self.workspace.data_ptr() + 255) & ~255
        mats = (hs_material * nrve)()
        for r in range(nrve):
            kind = HS_IDS_U8 if self._ids[r].dtype == np.uint8 else HS_IDS_U16
            mats[r] = hs_material(kind, ctypes.c_void_p(self._ids[r].ctypes.data), _dp(self._tables[r]),
                                  self._tables[r].shape[0], None)
        self.stream.wait_stream(torch.cuda.current_stream(device))
        b = ctypes.c_void_p()
        s = self.lib.hs_batch_create(ctypes.byref(b), nrve, g, mats, self.nitem, ir, ctypes.byref(self.opt),
                                     1 if autotune else 0, ctypes.c_void_p(ptr), ctypes.c_size_t(nbytes.value),
                                     ctypes.c_void_p(self.stream.cuda_stream))
        if s < 0:
            raise HSError(s, f"{self.lib.hs_error_string(s).decode()}: {self.lib.hs_batch_last_error(None).decode()}")
        self.b = b

    def solve(self, E, tol=1e-6, max_iter=1000):
        """E: (nitem, 6) tensor strains.  Returns dict(status (overall), item_status, iters, err, sig_eff)."""
        E = np.ascontiguousarray(np.asarray(E, dtype=np.float64).reshape(self.nitem, 6))
        sig = np.zeros((self.nitem, 6))
        it = np.zeros(self.nitem, dtype=np.int32)
        err = np.zeros(self.nitem)
        st = np.zeros(self.nitem, dtype=np.int32)
        iptr = ctypes.POINTER(ctypes.c_int)
        s = self.lib.hs_batch_solve(self.b, _dp(E), float(tol), int(max_iter), _dp(sig), it.ctypes.data_as(iptr),
                                    _dp(err), st.ctypes.data_as(iptr))
        if s < 0:
            raise HSError(s, f"{self.lib.hs_error_string(s).decode()}: {self.lib.hs_batch_last_error(self.b).decode()}")
        return dict(status=s, item_status=st, iters=it, err=err, sig_eff=sig)

    def err_history(self, item, n=1 << 16):
        out = np.zeros(n)
        k = ctypes.c_int()
        _check(self.lib, self.lib.hs_batch_err_history(self.b, int(item), _dp(out), n, ctypes.byref(k)))
        return out[: k.value]

    def launches(self):
        n = ctypes.c_longlong()
        _check(self.lib, self.lib.hs_batch_launches(self.b, ctypes.byref(n)))
        return n.value

    def classes(self):
        nc = ctypes.c_int()
        out = np.zeros(self.nitem, dtype=np.int32)
        _check(self.lib, self.lib.hs_batch_classes(self.b, ctypes.byref(nc),
                                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
        return nc.value, out

    def close(self):
        if getattr(self, "b", None):
            self.lib.hs_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
