"""Python binding of libpcg (AINV-preconditioned CG for the ocean free-surface
system on one B300). Argument marshalling only: every step of the solve runs
in the library's CUDA kernels. The functions carry the names of the C ABI in
``include/pcg.h``; vectors may be torch tensors (CUDA or CPU) or NumPy arrays,
binary64, shaped [ny][nx] (or flat with ny*nx entries), C-contiguous.

The library must have been built (``__graft_entry__.build()`` or
``python paper_1210_1878_b300/build.py``); importing this module raises if
``libpcg.so`` is missing or fails to load: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpcg.so")

PCG_OK, PCG_EINVAL, PCG_ENOMEM, PCG_EBUDGET, PCG_ENOTCONV, PCG_EBREAKDOWN, PCG_ETIMEOUT, PCG_ECUDA, \
    PCG_ECANCELLED = range(9)
PCG_PAT_TRIL_A, PCG_PAT_TRIL_A2, PCG_PAT_FULL, PCG_PAT_BAND_T, PCG_PAT_DIAG = range(5)
PCG_FP64, PCG_MIXED = 0, 1

EXPORTED = [
    "ainv_setup", "ainv_factor_host", "pcg_clone", "pcg_solve", "pcg_solve_batched", "pcg_sync", "pcg_spmv", "pcg_spmv_noalloc", "pcg_precond_apply",
    "pcg_apply_f32", "pcg_autotune", "pcg_tiles",
    "pcg_ainv_export", "pcg_resident_bytes", "pcg_n_wet", "pcg_free", "pcg_status_string",
    "pcg_last_error_message", "pcg_debug_wait_timeout", "pcg_profile_kernels", "pcg_kernel_launches",
    "pcg_fp64_fma_rate", "pcg_band_plan", "pcg_shard_create", "pcg_shard_bands", "pcg_shard_solve",
    "pcg_shard_free", "solver_server_create", "solver_server_register", "solver_server_submit",
    "solver_server_wait", "solver_server_cancel", "solver_server_stats", "solver_server_destroy",
]


class pcg_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("wet", C.c_void_p), ("c_e", C.c_void_p),
                ("c_n", C.c_void_p), ("shift", C.c_void_p)]


class ainv_opts(C.Structure):
    _fields_ = [("pattern", C.c_int32), ("drop_tol", C.c_double), ("band_q", C.c_int32),
                ("tile_x", C.c_int32), ("tile_y", C.c_int32)]


class pcg_opts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("max_iter", C.c_int32), ("prec", C.c_int32),
                ("inner_rtol", C.c_double), ("max_outer", C.c_int32), ("use_x0", C.c_int32),
                ("max_replace", C.c_int32)]


class pcg_stats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("outer_iters", C.c_int32), ("status", C.c_int32),
                ("replacements", C.c_int32), ("relres", C.c_double), ("true_relres", C.c_double),
                ("seconds", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class pcg_server_opts(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("max_slots", C.c_int32), ("chunk_iters", C.c_int32),
                ("solve", pcg_opts)]


class pcg_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64),
                ("rejected", C.c_uint64), ("p50_latency_ms", C.c_double), ("p99_latency_ms", C.c_double),
                ("mean_latency_ms", C.c_double), ("solves_per_s", C.c_double), ("in_flight", C.c_int32),
                ("queued", C.c_int32), ("hbm_used_bytes", C.c_size_t)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


DONE_CB = C.CFUNCTYPE(None, C.c_void_p, C.POINTER(pcg_stats))


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libpcg.so not built at {LIB_PATH}; run paper_1210_1878_b300/build.py")
    lib = C.CDLL(LIB_PATH)
    vp, i32, dbl = C.c_void_p, C.c_int32, C.c_double
    sig = {
        "ainv_setup": (C.c_int, [C.POINTER(pcg_grid), C.POINTER(ainv_opts), vp, C.POINTER(vp)]),
        "ainv_factor_host": (C.c_int, [C.POINTER(pcg_grid), C.POINTER(ainv_opts), C.POINTER(i32), vp, vp, vp]),
        "pcg_solve": (C.c_int, [vp, vp, vp, C.POINTER(pcg_opts), C.POINTER(pcg_stats), vp]),
        "pcg_solve_batched": (C.c_int, [C.POINTER(vp), i32, C.POINTER(vp), C.POINTER(vp), C.POINTER(pcg_opts),
                                        C.POINTER(pcg_stats), vp]),
        "pcg_sync": (C.c_int, [vp]),
        "pcg_spmv": (C.c_int, [vp, vp, vp, vp]),
        "pcg_spmv_noalloc": (C.c_int, [vp, vp, vp, vp]),
        "pcg_precond_apply": (C.c_int, [vp, vp, vp, vp]),
        "pcg_apply_f32": (C.c_int, [vp, i32, vp, vp, vp]),
        "pcg_autotune": (C.c_int, [vp, i32, i32, C.POINTER(i32), C.POINTER(i32), vp]),
        "pcg_tiles": (C.c_int, [vp, i32, C.POINTER(i32), C.POINTER(i32)]),
        "pcg_ainv_export": (C.c_int, [vp, C.POINTER(i32), vp, vp, vp]),
        "pcg_resident_bytes": (C.c_size_t, [vp]),
        "pcg_n_wet": (i32, [vp]),
        "pcg_free": (None, [vp]),
        "pcg_clone": (C.c_int, [vp, vp, C.POINTER(vp)]),
        "pcg_status_string": (C.c_char_p, [C.c_int]),
        "pcg_last_error_message": (C.c_char_p, []),
        "pcg_debug_wait_timeout": (C.c_int, [vp, i32, dbl, vp]),
        "pcg_profile_kernels": (C.c_int, [vp, vp, i32, i32, C.POINTER(dbl), C.POINTER(dbl), vp]),
        "pcg_kernel_launches": (C.c_uint64, []),
        "pcg_fp64_fma_rate": (C.c_int, [i32, C.POINTER(dbl), C.POINTER(dbl), vp]),
        "pcg_band_plan": (C.c_int, [i32, i32, vp, i32, i32, vp, C.POINTER(i32)]),
        "pcg_shard_create": (C.c_int, [vp, i32, vp, C.POINTER(vp)]),
        "pcg_shard_bands": (C.c_int, [vp, C.POINTER(i32), vp, C.POINTER(i32)]),
        "pcg_shard_solve": (C.c_int, [vp, vp, vp, C.POINTER(pcg_opts), C.POINTER(pcg_stats), vp]),
        "pcg_shard_free": (None, [vp]),
        "solver_server_create": (C.c_int, [C.POINTER(pcg_server_opts), C.POINTER(vp)]),
        "solver_server_register": (C.c_int, [vp, vp, C.POINTER(i32)]),
        "solver_server_submit": (C.c_int, [vp, i32, vp, vp, i32, DONE_CB, vp, C.POINTER(C.c_uint64)]),
        "solver_server_wait": (C.c_int, [vp, C.c_uint64, i32, C.POINTER(pcg_stats)]),
        "solver_server_cancel": (C.c_int, [vp, C.c_uint64]),
        "solver_server_stats": (C.c_int, [vp, C.POINTER(pcg_server_stats)]),
        "solver_server_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        if not hasattr(lib, name):
            continue
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


class PCGError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        msg = lib.pcg_last_error_message().decode(errors="replace")
        super().__init__(f"{where}: {lib.pcg_status_string(status).decode()} ({status}): {msg}")


def _ptr(a):
    """Device or host address of a contiguous binary64 buffer (torch or numpy)."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return C.c_void_p(a.ctypes.data)
    raise TypeError("expected a torch tensor or a numpy array")


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return C.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _grid_struct(nx, ny, wet, c_e, c_n, shift):
    keep = [np.ascontiguousarray(wet, dtype=np.uint8), np.ascontiguousarray(c_e, dtype=np.float64),
            np.ascontiguousarray(c_n, dtype=np.float64), np.ascontiguousarray(shift, dtype=np.float64)]
    g = pcg_grid(int(nx), int(ny), keep[0].ctypes.data, keep[1].ctypes.data, keep[2].ctypes.data,
                 keep[3].ctypes.data)
    return g, keep


class Handle:
    """Owns one pcg_handle (one grid's A, Z, D^-1 and work vectors on the device)."""

    def __init__(self, ptr, nx, ny):
        self._p = C.c_void_p(ptr)
        self.nx, self.ny = nx, ny
        self._inflight = None      # arguments of an enqueued solve, kept alive until pcg_sync

    @property
    def ptr(self):
        return self._p

    def close(self):
        if self._p and self._p.value:
            lib.pcg_free(self._p)
            self._p = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_wet(self):
        return int(lib.pcg_n_wet(self._p))

    @property
    def resident_bytes(self):
        return int(lib.pcg_resident_bytes(self._p))


def ainv_setup(nx, ny, wet, c_e, c_n, shift, pattern=PCG_PAT_TRIL_A2, drop_tol=0.0, band_q=0, tile_x=0, tile_y=0,
               stream=None) -> Handle:
    g, keep = _grid_struct(nx, ny, wet, c_e, c_n, shift)
    o = ainv_opts(int(pattern), float(drop_tol), int(band_q), int(tile_x), int(tile_y))
    out = C.c_void_p()
    st = lib.ainv_setup(C.byref(g), C.byref(o), _stream(stream), C.byref(out))
    if st != PCG_OK:
        raise PCGError(st, "ainv_setup")
    return Handle(out.value, nx, ny)


def ainv_setup_grid(grid, **kw) -> Handle:
    return ainv_setup(grid.nx, grid.ny, grid.wet, grid.c_e, grid.c_n, grid.shift, **kw)


def pcg_clone(h: Handle, stream=None) -> Handle:
    """A second handle of h's grid and factor (pcg_clone): its own device
    planes, so that two solves of the grid can be in flight."""
    out = C.c_void_p()
    st = lib.pcg_clone(h.ptr, _stream(stream), C.byref(out))
    if st != PCG_OK:
        raise PCGError(st, "pcg_clone")
    return Handle(out.value, h.nx, h.ny)


def ainv_factor_host(nx, ny, wet, c_e, c_n, shift, pattern=PCG_PAT_TRIL_A2, drop_tol=0.0, band_q=0):
    """The library's own factor, built on the host: (D [n], rows [n][8], vals [n][8])."""
    g, keep = _grid_struct(nx, ny, wet, c_e, c_n, shift)
    o = ainv_opts(int(pattern), float(drop_tol), int(band_q), 0, 0)
    cap = int(nx) * int(ny)
    D = np.zeros(cap)
    rows = np.full((cap, 8), -1, np.int32)
    vals = np.zeros((cap, 8))
    n = C.c_int32()
    st = lib.ainv_factor_host(C.byref(g), C.byref(o), C.byref(n), D.ctypes.data, rows.ctypes.data, vals.ctypes.data)
    if st != PCG_OK:
        raise PCGError(st, "ainv_factor_host")
    k = n.value
    return D[:k].copy(), rows[:k].copy(), vals[:k].copy()


def make_opts(rtol=1e-10, max_iter=0, prec=PCG_FP64, inner_rtol=0.0, max_outer=0, use_x0=False, max_replace=3):
    return pcg_opts(float(rtol), int(max_iter), int(prec), float(inner_rtol), int(max_outer), int(bool(use_x0)),
                    int(max_replace))


def pcg_solve(h: Handle, b, x, opts: pcg_opts | None = None, stream=None, check=True, sync=True) -> pcg_stats:
    """Enqueue one solve; with sync (default) wait for it (pcg_sync) and return
    its statistics (.rc holds the status). With sync=False the statistics are
    filled by a later ``pcg_sync(h)``; keep b, x and the returned object alive
    until then."""
    st = pcg_stats()
    o = opts if opts is not None else make_opts()
    rc = lib.pcg_solve(h.ptr, _ptr(b), _ptr(x), C.byref(o), C.byref(st), _stream(stream))
    if rc != PCG_OK:
        if check:
            raise PCGError(rc, "pcg_solve")
        st.rc = rc
        return st
    h._inflight = (st, o, b, x)
    if sync:
        rc = pcg_sync(h)
        if check and rc != PCG_OK:
            raise PCGError(rc, "pcg_solve")
    st.rc = rc
    return st


def pcg_sync(h: Handle) -> int:
    """Wait for the solve enqueued on h and return its status (pcg_sync)."""
    rc = int(lib.pcg_sync(h.ptr))
    h._inflight = None
    return rc


def pcg_solve_batched(hs, bs, xs, opts: pcg_opts | None = None, stream=None, check=True, sync=True):
    n = len(hs)
    H = (C.c_void_p * n)(*[h.ptr for h in hs])
    B = (C.c_void_p * n)(*[_ptr(b) for b in bs])
    X = (C.c_void_p * n)(*[_ptr(x) for x in xs])
    stats = (pcg_stats * n)()
    o = opts if opts is not None else make_opts()
    rc = lib.pcg_solve_batched(H, n, B, X, C.byref(o), stats, _stream(stream))
    if rc == PCG_OK:
        for h in hs:
            h._inflight = (stats, o, bs, xs)
        if sync:
            rc = pcg_sync(hs[0])
            for h in hs:
                h._inflight = None
    if check and rc != PCG_OK:
        raise PCGError(rc, "pcg_solve_batched")
    return rc, list(stats)


def pcg_spmv(h: Handle, v, q, stream=None):
    rc = lib.pcg_spmv(h.ptr, _ptr(v), _ptr(q), _stream(stream))
    if rc != PCG_OK:
        raise PCGError(rc, "pcg_spmv")


def pcg_spmv_noalloc(h: Handle, v, q, stream=None) -> int:
    """q = A v through the allocation-free entry point; returns the status."""
    return int(lib.pcg_spmv_noalloc(h.ptr, _ptr(v), _ptr(q), _stream(stream)))


def pcg_precond_apply(h: Handle, r, s, stream=None):
    rc = lib.pcg_precond_apply(h.ptr, _ptr(r), _ptr(s), _stream(stream))
    if rc != PCG_OK:
        raise PCGError(rc, "pcg_precond_apply")


def pcg_apply_f32(h: Handle, op: int, v, out, stream=None):
    """The binary32 kernels on one operand: op 0 out = A v, op 1 out = M^-1 v."""
    rc = lib.pcg_apply_f32(h.ptr, int(op), _ptr(v), _ptr(out), _stream(stream))
    if rc != PCG_OK:
        raise PCGError(rc, "pcg_apply_f32")


def pcg_autotune(h: Handle, prec: int = 1, objective: int = 0, stream=None):
    """Time the strip shapes for precision prec on h, apply and remember the
    best (objective 0: alone, 1: as a batch member); returns (tile_x, tile_y)."""
    tx, ty = C.c_int32(), C.c_int32()
    rc = lib.pcg_autotune(h.ptr, int(prec), int(objective), C.byref(tx), C.byref(ty), _stream(stream))
    if rc != PCG_OK:
        raise PCGError(rc, "pcg_autotune")
    return tx.value, ty.value


def pcg_tiles(h: Handle, prec: int = 0):
    tx, ty = C.c_int32(), C.c_int32()
    rc = lib.pcg_tiles(h.ptr, int(prec), C.byref(tx), C.byref(ty))
    if rc != PCG_OK:
        raise PCGError(rc, "pcg_tiles")
    return tx.value, ty.value


def pcg_ainv_export(h: Handle):
    n = h.n_wet
    D = np.zeros(n)
    rows = np.full((n, 8), -1, np.int32)
    vals = np.zeros((n, 8))
    cn = C.c_int32()
    rc = lib.pcg_ainv_export(h.ptr, C.byref(cn), D.ctypes.data, rows.ctypes.data, vals.ctypes.data)
    if rc != PCG_OK:
        raise PCGError(rc, "pcg_ainv_export")
    return D, rows, vals


def pcg_debug_wait_timeout(h: Handle, unit=0, timeout_ms=50.0, stream=None) -> int:
    return int(lib.pcg_debug_wait_timeout(h.ptr, int(unit), float(timeout_ms), _stream(stream)))


def pcg_profile_kernels(h: Handle, b, iters=20, prec=PCG_FP64, stream=None):
    """Mean duration (ms) of one stencil launch and one preconditioner launch."""
    a, c = C.c_double(), C.c_double()
    rc = lib.pcg_profile_kernels(h.ptr, _ptr(b), int(iters), int(prec), C.byref(a), C.byref(c), _stream(stream))
    if rc != PCG_OK:
        raise PCGError(rc, "pcg_profile_kernels")
    return a.value, c.value


def pcg_fp64_fma_rate(launches=10, stream=None):
    """Measured binary64 FMA rate of the current GPU: (TFLOP/s, ms per launch)."""
    t, ms = C.c_double(), C.c_double()
    rc = lib.pcg_fp64_fma_rate(int(launches), C.byref(t), C.byref(ms), _stream(stream))
    if rc != PCG_OK:
        raise PCGError(rc, "pcg_fp64_fma_rate")
    return t.value, ms.value


def pcg_kernel_launches() -> int:
    return int(lib.pcg_kernel_launches())


# ------------------------------------------------------------ row-band sharding
def pcg_band_plan(wet, pattern=PCG_PAT_TRIL_A2, nbands=2):
    """Row bands of about equal wet count: (row0 [nbands + 1], halo rows)."""
    w = np.ascontiguousarray(wet, dtype=np.uint8)
    ny, nx = w.shape
    row0 = np.zeros(int(nbands) + 1, np.int32)
    halo = C.c_int32()
    rc = lib.pcg_band_plan(int(nx), int(ny), w.ctypes.data, int(pattern), int(nbands), row0.ctypes.data, C.byref(halo))
    if rc != PCG_OK:
        raise PCGError(rc, "pcg_band_plan")
    return row0, halo.value


class Shard:
    """A grid split into row bands on the current GPU (pcg_shard_*)."""

    def __init__(self, h: Handle, nbands=2, stream=None):
        out = C.c_void_p()
        rc = lib.pcg_shard_create(h.ptr, int(nbands), _stream(stream), C.byref(out))
        if rc != PCG_OK:
            raise PCGError(rc, "pcg_shard_create")
        self._s = out
        self._h = h                 # the whole grid must outlive the shard

    def bands(self):
        n = C.c_int32()
        lib.pcg_shard_bands(self._s, C.byref(n), None, None)
        row0 = np.zeros(n.value + 1, np.int32)
        halo = C.c_int32()
        lib.pcg_shard_bands(self._s, None, row0.ctypes.data, C.byref(halo))
        return row0, halo.value

    def solve(self, b, x, opts: pcg_opts | None = None, stream=None, check=True) -> pcg_stats:
        st = pcg_stats()
        o = opts if opts is not None else make_opts()
        rc = lib.pcg_shard_solve(self._s, _ptr(b), _ptr(x), C.byref(o), C.byref(st), _stream(stream))
        if check and rc != PCG_OK:
            raise PCGError(rc, "pcg_shard_solve")
        st.rc = rc
        return st

    def close(self):
        if self._s and self._s.value:
            lib.pcg_shard_free(self._s)
            self._s = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# -------------------------------------------------------------------- serving
class Server:
    """Continuous-batching solver server (solver_server_* of the C ABI)."""

    def __init__(self, hbm_budget_bytes, max_slots=16, chunk_iters=16, opts: pcg_opts | None = None):
        so = pcg_server_opts(int(hbm_budget_bytes), int(max_slots), int(chunk_iters), opts or make_opts())
        out = C.c_void_p()
        rc = lib.solver_server_create(C.byref(so), C.byref(out))
        if rc != PCG_OK:
            raise PCGError(rc, "solver_server_create")
        self._s = out
        self._keep = {}

    def register(self, h: Handle) -> int:
        gid = C.c_int32()
        rc = lib.solver_server_register(self._s, h.ptr, C.byref(gid))
        if rc != PCG_OK:
            raise PCGError(rc, "solver_server_register")
        return gid.value

    def submit(self, grid_id, b, x_out, warm_start=False) -> int:
        rid = C.c_uint64()
        rc = lib.solver_server_submit(self._s, int(grid_id), _ptr(b), _ptr(x_out), int(bool(warm_start)),
                                      DONE_CB(), None, C.byref(rid))
        if rc != PCG_OK:
            raise PCGError(rc, "solver_server_submit")
        self._keep[rid.value] = x_out
        return rid.value

    def wait(self, req_id, timeout_ms=-1):
        st = pcg_stats()
        rc = lib.solver_server_wait(self._s, C.c_uint64(req_id), int(timeout_ms), C.byref(st))
        self._keep.pop(req_id, None)
        return rc, st

    def cancel(self, req_id) -> int:
        return int(lib.solver_server_cancel(self._s, C.c_uint64(req_id)))

    def stats(self) -> dict:
        st = pcg_server_stats()
        lib.solver_server_stats(self._s, C.byref(st))
        return st.as_dict()

    def close(self):
        if self._s and self._s.value:
            lib.solver_server_destroy(self._s)
            self._s = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
