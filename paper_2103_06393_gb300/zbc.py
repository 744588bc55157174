"""Thin ctypes binding of libzbc (argument marshalling only: every step runs in the library).

Function names follow the C ABI in include/zbc.h.  Tensors are torch tensors on the GPU
(complex64 / complex128 / int32 / float64, column-major where the ABI says so: pass
Fortran-ordered data as the transpose of a contiguous tensor, or use the helpers here that
allocate column-major buffers).  The library must be built (paper_2103_06393_gb300.build);
importing this module without it raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libzbc.so")

ZBC_OK, ZBC_EINVAL, ZBC_ENOMEM, ZBC_ECUDA, ZBC_ETOL, ZBC_ETIMEOUT, ZBC_ENAN, ZBC_EIO = 0, -1, -2, -3, -4, -5, -6, -7
C64, C128 = 0, 1
FP32_SIMT, TF32X3, BF16X3, AUTO, TC2, TC_MODE1, TC_DC = 0, 1, 2, 3, 4, 5, 6
HOSVD, RANDOMIZED_LEARNED, RANDOMIZED_FIXED = 0, 1, 2
ACA_DENSE_U, ACA_ALG3 = 0, 1
PRECISIONS = {"fp32_simt": FP32_SIMT, "tf32x3": TF32X3, "bf16x3": BF16X3}


class ZbcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"zbc status {status}: {msg}")
        self.status = status


class zbc_grid(C.Structure):
    _fields_ = [("n1", C.c_int32), ("n2", C.c_int32), ("n3", C.c_int32), ("h", C.c_double),
                ("mask_radius", C.c_double), ("mask_box", C.c_double)]


class zbc_segments(C.Structure):
    _fields_ = [("m", C.c_int32), ("centre", C.c_void_p), ("tangent", C.c_void_p), ("length", C.c_void_p)]


class zbc_info(C.Structure):
    _fields_ = [("n1", C.c_int32), ("n2", C.c_int32), ("n3", C.c_int32), ("q", C.c_int32), ("M", C.c_int32),
                ("m", C.c_int32), ("has_v", C.c_int32), ("max_rank", C.c_int32), ("pool_bytes", C.c_int64),
                ("v_bytes", C.c_int64)]


class zbc_compress_stats(C.Structure):
    _fields_ = [("n_tensors", C.c_int32), ("n_fallback", C.c_int32), ("max_rank", C.c_int32),
                ("max_rel_err", C.c_double)]


class zbc_rank_model(C.Structure):
    _fields_ = [("mlp", C.c_void_p), ("features", C.c_void_p), ("oversample", C.c_int32),
                ("fixed_width", C.c_int32), ("sketch1", C.c_void_p), ("sketch2", C.c_void_p),
                ("sketch3", C.c_void_p), ("lmax", C.c_int32)]


class zbc_cross_params(C.Structure):
    _fields_ = [("sweeps", C.c_int32), ("s0", C.c_int32), ("over", C.c_int32), ("rmax", C.c_int32)]


class zbc_cross_stats(C.Structure):
    _fields_ = [("entries", C.c_int64), ("max_check_err", C.c_double)]


class zbc_aca_stats(C.Structure):
    _fields_ = [("rank", C.c_int32), ("converged", C.c_int32), ("row_restarts", C.c_int32),
                ("max_tucker_rank", C.c_int32), ("tucker_fallbacks", C.c_int32), ("reserved", C.c_int32),
                ("s2", C.c_double), ("last_term", C.c_double), ("max_tucker_err", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libzbc.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, dbl = C.c_void_p, C.c_int, C.c_int64, C.c_double
        sig = {
            "zbc_last_error": ([], C.c_char_p),
            "zbc_version": ([], C.c_char_p),
            "zbc_kernel_launches": ([], C.c_int64),
            "vsie_assemble_columns": ([C.POINTER(zbc_grid), C.POINTER(zbc_segments), dbl, vp, i32, i32, vp, i64, i32, vp], i32),
            "vsie_assemble_columns_op": ([C.POINTER(zbc_grid), C.POINTER(zbc_segments), dbl, vp, i32, i32, i32, i32, vp, i64,
                                          i32, vp], i32),
            "tucker_compress": ([vp, i64, i32, C.POINTER(zbc_grid), i32, i32, dbl, i32, C.POINTER(zbc_rank_model),
                                 i32, C.POINTER(vp), C.POINTER(zbc_compress_stats), vp], i32),
            "zbc_matvec": ([vp, vp, i64, i32, vp, i64, i32, vp], i32),
            "zbc_rmatvec": ([vp, vp, i64, i32, vp, i64, i32, vp], i32),
            "zbc_free": ([vp], i32),
            "zbc_get_info": ([vp, C.POINTER(zbc_info)], i32),
            "zbc_memory_bytes": ([vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)], i32),
            "zbc_device_bytes": ([vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)], i32),
            "zbc_create_from_host": ([C.POINTER(zbc_grid), i32, i32, i32, vp, vp, i64, vp, C.POINTER(vp)], i32),
            "zbc_export_host": ([vp, vp, vp, vp], i32),
            "zbc_save": ([vp, C.c_char_p], i32),
            "zbc_load": ([C.c_char_p, C.POINTER(vp)], i32),
            "zbc_tc_selftest": ([vp, vp, vp, i32, i32, i32], i32),
            "aca_compress": ([C.POINTER(zbc_grid), C.POINTER(zbc_segments), dbl, i32, dbl, i32, i32, dbl, i32,
                              C.POINTER(zbc_rank_model), C.POINTER(vp), C.POINTER(zbc_aca_stats), vp, vp], i32),
            "tucker_compress_randomized": ([vp, i64, i32, C.POINTER(zbc_grid), i32, i32, dbl, vp, vp, vp, vp, i32,
                                            C.POINTER(vp), C.POINTER(zbc_compress_stats), vp], i32),
            "zbc_mlp_num_params": ([], i32),
            "zbc_mlp_create": ([vp, i32, C.POINTER(vp)], i32),
            "zbc_mlp_free": ([vp], i32),
            "zbc_mlp_get_params": ([vp, vp, vp], i32),
            "zbc_mlp_forward": ([vp, vp, i32, vp, vp], i32),
            "zbc_mlp_backward": ([vp, vp, vp, i32, vp, vp, vp], i32),
            "zbc_mlp_adam_step": ([vp, vp, C.c_float, vp], i32),
            "zbc_mlp_train": ([vp, vp, vp, i32, i32, C.c_float, vp, vp], i32),
            "zbc_rank_widths": ([vp, vp, i32, C.POINTER(zbc_grid), i32, vp, vp], i32),
            "zbc_rmatvec_noalloc": ([vp, vp, i64, i32, vp, i64, vp], i32),
            "zbc_product_status": ([vp, vp], i32),
            "zbc_test_wait_limit": ([vp, C.c_uint32], i32),
            "zbc_tune": ([vp, i32, vp, vp], i32),
            "cross_tucker_compress": ([vp, i64, i32, C.POINTER(zbc_grid), i32, i32, dbl, C.POINTER(zbc_cross_params),
                                       vp, i32, C.POINTER(vp), C.POINTER(zbc_compress_stats),
                                       C.POINTER(zbc_cross_stats), vp], i32),
            "cross_tucker_assemble": ([C.POINTER(zbc_grid), C.POINTER(zbc_segments), dbl, vp, i32, i32, i32, i32, dbl,
                                       C.POINTER(zbc_cross_params), vp, i32, C.POINTER(vp),
                                       C.POINTER(zbc_compress_stats), C.POINTER(zbc_cross_stats), vp], i32),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def kernel_launches() -> int:
    return int(lib().zbc_kernel_launches())


def _check(status):
    if status != ZBC_OK:
        raise ZbcError(status, lib().zbc_last_error().decode())


def _stream(stream):
    import torch
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(getattr(stream, "cuda_stream", stream))


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _ld(t) -> int:
    """Leading dimension of a column-major matrix held as a (cols, rows) tensor.  A single
    column may carry any stride for its size-1 dimension, so its ld is its row count."""
    if t.shape[0] == 1:
        return int(t.shape[1])
    if t.shape[1] == 1:  # one row: the within-column stride is irrelevant
        return max(1, int(t.stride(0)))
    assert t.stride(1) == 1, "column-major buffers need unit stride within a column"
    return int(t.stride(0))


def colmajor(rows: int, cols: int, dtype, device="cuda"):
    """A rows x cols column-major buffer: returned as a (cols, rows) contiguous tensor whose
    row c is column c of the matrix."""
    import torch
    return torch.empty((cols, rows), dtype=dtype, device=device)


def to_colmajor(a: np.ndarray, dtype=None, device="cuda"):
    """numpy matrix -> torch tensor holding it column-major (shape (cols, rows))."""
    import torch
    a = np.asarray(a)
    if dtype is not None:
        a = a.astype(dtype)
    return torch.from_numpy(np.ascontiguousarray(a.T)).to(device)


def from_colmajor(t) -> np.ndarray:
    return t.detach().cpu().numpy().T


def from_colmajor_rows(t, rows) -> np.ndarray:
    """Rows `rows` (an int64 CUDA tensor) of a column-major buffer, as a host (len(rows), cols) array."""
    return t.index_select(1, rows).cpu().numpy().T


def grid_struct(grid) -> zbc_grid:
    return zbc_grid(grid.n1, grid.n2, grid.n3, grid.h, getattr(grid, "mask_radius", 0.0),
                    getattr(grid, "mask_box", 0.0))


class Handle:
    """Owns a zbc_handle*."""

    def __init__(self, ptr: C.c_void_p):
        self.ptr = ptr

    def __del__(self):
        if getattr(self, "ptr", None) and lib is not None:
            try:
                lib().zbc_free(self.ptr)
            except Exception:
                pass
            self.ptr = None

    def info(self) -> zbc_info:
        inf = zbc_info()
        _check(lib().zbc_get_info(self.ptr, C.byref(inf)))
        return inf

    def memory_bytes(self):
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        _check(lib().zbc_memory_bytes(self.ptr, C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value

    def device_bytes(self):
        """{"pool", "caches", "work"}: device bytes this handle holds now (zbc_device_bytes)."""
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        _check(lib().zbc_device_bytes(self.ptr, C.byref(a), C.byref(b), C.byref(c)))
        return {"pool": a.value, "caches": b.value, "work": c.value}

    def export(self):
        """(ranks (M, q, 3) int32, pool complex64, V (m x M) or None)."""
        inf = self.info()
        ranks = np.zeros(3 * inf.M * inf.q, dtype=np.int32)
        pool = np.zeros(inf.pool_bytes // 8, dtype=np.complex64)
        V = np.zeros((inf.M, inf.m), dtype=np.complex64) if inf.has_v else None
        _check(lib().zbc_export_host(self.ptr, ranks.ctypes.data_as(C.c_void_p), pool.ctypes.data_as(C.c_void_p),
                                     V.ctypes.data_as(C.c_void_p) if V is not None else None))
        return ranks.reshape(inf.M, inf.q, 3), pool, (V.T.copy() if V is not None else None)

    def tensors(self):
        """Unpack to the oracle's format: list over j of list over k of (G, [U1,U2,U3]) (complex128)."""
        inf = self.info()
        ranks, pool, V = self.export()
        n = (inf.n1, inf.n2, inf.n3)
        out, off = [], 0
        for j in range(inf.M):
            comps = []
            for k in range(inf.q):
                r1, r2, r3 = (int(x) for x in ranks[j, k])
                G = pool[off:off + r1 * r2 * r3].reshape((r1, r2, r3), order="F").astype(np.complex128)
                off += r1 * r2 * r3
                Us = []
                for g, r in enumerate((r1, r2, r3)):
                    Us.append(pool[off:off + n[g] * r].reshape((n[g], r), order="F").astype(np.complex128))
                    off += n[g] * r
                comps.append((G, Us))
            out.append(comps)
        return out, V

    def save(self, path: str):
        _check(lib().zbc_save(self.ptr, path.encode()))


def pack_tensors(tensors, n) -> tuple:
    """Oracle format -> (ranks int32[3*M*q], pool complex64) in the ABI's host layout."""
    ranks, parts = [], []
    for tj in tensors:
        for t in tj:
            G, Us = t[0], t[1]
            ranks.extend(G.shape)
            parts.append(np.asarray(G).reshape(-1, order="F"))
            for U in Us:
                parts.append(np.asarray(U).reshape(-1, order="F"))
    return np.array(ranks, dtype=np.int32), np.concatenate(parts).astype(np.complex64)


def zbc_create_from_host(grid, q, tensors, V=None) -> Handle:
    ranks, pool = pack_tensors(tensors, grid.shape if hasattr(grid, "shape") else None)
    M = len(tensors)
    m = M if V is None else V.shape[0]
    vcol = None
    if V is not None:
        vcol = np.asfortranarray(np.asarray(V, dtype=np.complex64))
    h = C.c_void_p()
    g = grid_struct(grid)
    _check(lib().zbc_create_from_host(C.byref(g), q, M, m, ranks.ctypes.data_as(C.c_void_p),
                                      pool.ctypes.data_as(C.c_void_p), pool.size,
                                      vcol.ctypes.data_as(C.c_void_p) if vcol is not None else None, C.byref(h)))
    return Handle(h)


def zbc_tc_selftest(A: np.ndarray, B: np.ndarray, fmt: int) -> np.ndarray:
    """D = A B^T through one tcgen05 MMA chain (A 128 x K, B N x K float32)."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    D = np.zeros((128, B.shape[0]), dtype=np.float32)
    _check(lib().zbc_tc_selftest(A.ctypes.data_as(C.c_void_p), B.ctypes.data_as(C.c_void_p),
                                 D.ctypes.data_as(C.c_void_p), B.shape[0], A.shape[1], fmt))
    return D


def zbc_load(path: str) -> Handle:
    h = C.c_void_p()
    _check(lib().zbc_load(path.encode(), C.byref(h)))
    return Handle(h)


class DeviceSegments:
    """Segments uploaded to the device (float64)."""

    def __init__(self, segs, device="cuda"):
        import torch
        self.centre = torch.from_numpy(np.ascontiguousarray(segs.centre, dtype=np.float64)).to(device)
        self.tangent = torch.from_numpy(np.ascontiguousarray(segs.tangent, dtype=np.float64)).to(device)
        self.length = torch.from_numpy(np.ascontiguousarray(segs.length, dtype=np.float64)).to(device)
        self.m = int(segs.length.shape[0])

    def struct(self) -> zbc_segments:
        return zbc_segments(self.m, self.centre.data_ptr(), self.tangent.data_ptr(), self.length.data_ptr())


OP_N, OP_K = 0, 1


def vsie_assemble_columns(grid, dsegs: DeviceSegments, freq_hz: float, cols, out, q=3, stream=None):
    """cols: int32 CUDA tensor; out: column-major buffer (ncols, ld) complex64/complex128."""
    import torch
    g = grid_struct(grid)
    s = dsegs.struct()
    dt = C128 if out.dtype == torch.complex128 else C64
    _check(lib().vsie_assemble_columns(C.byref(g), C.byref(s), freq_hz, _ptr(cols), int(cols.numel()), q, _ptr(out),
                                       _ld(out), dt, _stream(stream)))
    return out


def vsie_assemble_columns_op(grid, dsegs: DeviceSegments, freq_hz: float, cols, out, op=OP_N, nq=1, q=3,
                             stream=None):
    """vsie_assemble_columns with the operator (OP_N: Eq. nNt, OP_K: Eq. nKt) and nq Gauss-Legendre
    points along each segment."""
    import torch
    g = grid_struct(grid)
    s = dsegs.struct()
    dt = C128 if out.dtype == torch.complex128 else C64
    _check(lib().vsie_assemble_columns_op(C.byref(g), C.byref(s), freq_hz, _ptr(cols), int(cols.numel()), q, int(op),
                                          int(nq), _ptr(out), _ld(out), dt, _stream(stream)))
    return out


def rank_model(sketches, lmax: int, mlp=None, features=None, oversample=4, fixed_width=0) -> zbc_rank_model:
    """Inputs of the randomized methods of tucker_compress.  sketches: three complex64 CUDA tensors
    holding Omega_g column-major (shape (lmax, N_g)); mlp / features (CUDA float32, ncols x 7) for
    RANDOMIZED_LEARNED, fixed_width for RANDOMIZED_FIXED.  The structure refers to the tensors'
    memory: keep them alive while it is used."""
    return zbc_rank_model(mlp.ptr if mlp is not None else None,
                          features.data_ptr() if features is not None else None, int(oversample),
                          int(fixed_width), _ptr(sketches[0]), _ptr(sketches[1]), _ptr(sketches[2]), int(lmax))


def tucker_compress(cols, grid, tol: float, q=3, method=HOSVD, model: zbc_rank_model | None = None,
                    append_to: Handle | None = None, stream=None):
    """cols: column-major buffer (ncols, ld).  method: HOSVD, RANDOMIZED_LEARNED or
    RANDOMIZED_FIXED (the latter two need `model`, see rank_model).  Returns (Handle, stats)."""
    import torch
    g = grid_struct(grid)
    dt = C128 if cols.dtype == torch.complex128 else C64
    h = C.c_void_p(append_to.ptr.value if append_to is not None else None)
    st = zbc_compress_stats()
    _check(lib().tucker_compress(_ptr(cols), _ld(cols), cols.shape[0], C.byref(g), q, dt, tol, method,
                                 C.byref(model) if model is not None else None, C64, C.byref(h), C.byref(st),
                                 _stream(stream)))
    if append_to is not None:
        return append_to, st
    return Handle(h), st


def _cross_args(params, checks):
    prm = None
    if params is not None:
        prm = zbc_cross_params(**{k: int(v) for k, v in dict(params).items()})
    chk = np.ascontiguousarray(np.zeros((0, 3)) if checks is None else checks, dtype=np.int32).reshape(-1, 3)
    return prm, chk


def cross_tucker_compress(cols, grid, tol: float, q=3, params=None, checks=None, append_to: Handle | None = None,
                          stream=None):
    """Tucker compression from fibres of columns held on the device (cols: column-major (ncols, ld)).
    params: dict with sweeps / s0 / over / rmax (None: the defaults); checks: int array (n, 3) of
    check fibres (g, i_a, i_b).  Returns (Handle, stats, cross stats)."""
    import torch
    g = grid_struct(grid)
    dt = C128 if cols.dtype == torch.complex128 else C64
    prm, chk = _cross_args(params, checks)
    h = C.c_void_p(append_to.ptr.value if append_to is not None else None)
    st, xs = zbc_compress_stats(), zbc_cross_stats()
    _check(lib().cross_tucker_compress(_ptr(cols), _ld(cols), cols.shape[0], C.byref(g), q, dt, tol,
                                       C.byref(prm) if prm is not None else None,
                                       chk.ctypes.data_as(C.c_void_p), chk.shape[0], C.byref(h), C.byref(st),
                                       C.byref(xs), _stream(stream)))
    return (append_to if append_to is not None else Handle(h)), st, xs


def cross_tucker_assemble(grid, dsegs: DeviceSegments, freq_hz: float, cols, tol: float, q=3, op=OP_N, nq=1,
                          params=None, checks=None, append_to: Handle | None = None, stream=None):
    """Tucker compression from fibres whose entries are evaluated from the Green's function (no
    column is assembled).  cols: host segment indices.  Returns (Handle, stats, cross stats)."""
    g = grid_struct(grid)
    s = dsegs.struct()
    cidx = np.ascontiguousarray(np.atleast_1d(cols), dtype=np.int32)
    prm, chk = _cross_args(params, checks)
    h = C.c_void_p(append_to.ptr.value if append_to is not None else None)
    st, xs = zbc_compress_stats(), zbc_cross_stats()
    _check(lib().cross_tucker_assemble(C.byref(g), C.byref(s), freq_hz, cidx.ctypes.data_as(C.c_void_p), cidx.size,
                                       q, op, nq, tol, C.byref(prm) if prm is not None else None,
                                       chk.ctypes.data_as(C.c_void_p), chk.shape[0], C.byref(h), C.byref(st),
                                       C.byref(xs), _stream(stream)))
    return (append_to if append_to is not None else Handle(h)), st, xs


def aca_compress(grid, dsegs: DeviceSegments, freq_hz: float, tol: float, max_rank: int, mode=ACA_DENSE_U,
                 tucker_tol: float = 0.0, q=3, method=HOSVD, model: zbc_rank_model | None = None, stream=None):
    """method: how U's tensors are compressed (HOSVD, or RANDOMIZED_FIXED with `model`, see
    rank_model).  Returns (Handle with U (Tucker) and V, stats, pivots array (r_c, 2))."""
    g = grid_struct(grid)
    s = dsegs.struct()
    h = C.c_void_p()
    st = zbc_aca_stats()
    piv = np.zeros(2 * max_rank, dtype=np.int32)
    _check(lib().aca_compress(C.byref(g), C.byref(s), freq_hz, q, tol, max_rank, mode, tucker_tol, method,
                              C.byref(model) if model is not None else None, C.byref(h), C.byref(st),
                              piv.ctypes.data_as(C.c_void_p), _stream(stream)))
    return Handle(h), st, piv[:2 * st.rank].reshape(-1, 2)


def tucker_compress_randomized(cols, grid, tol: float, widths: np.ndarray, sketches, lmax: int, q=3,
                               append_to: Handle | None = None, stream=None):
    """widths: int32[3*ncols*q]; sketches: three complex64 CUDA tensors holding Omega_g
    column-major (shape (lmax, N_g)).  Returns (Handle, stats)."""
    import torch
    g = grid_struct(grid)
    dt = C128 if cols.dtype == torch.complex128 else C64
    wdt = np.ascontiguousarray(widths, dtype=np.int32)
    h = C.c_void_p(append_to.ptr.value if append_to is not None else None)
    st = zbc_compress_stats()
    _check(lib().tucker_compress_randomized(_ptr(cols), _ld(cols), cols.shape[0], C.byref(g), q, dt, tol,
                                            wdt.ctypes.data_as(C.c_void_p), _ptr(sketches[0]), _ptr(sketches[1]),
                                            _ptr(sketches[2]), lmax, C.byref(h), C.byref(st), _stream(stream)))
    return (append_to if append_to is not None else Handle(h)), st


class Mlp:
    """Owns a zbc_mlp* (rank predictor)."""

    def __init__(self, params: np.ndarray):
        n = int(lib().zbc_mlp_num_params())
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == n, (p.size, n)
        self.ptr = C.c_void_p()
        _check(lib().zbc_mlp_create(p.ctypes.data_as(C.c_void_p), n, C.byref(self.ptr)))
        self.n = n

    def __del__(self):
        if getattr(self, "ptr", None):
            try:
                lib().zbc_mlp_free(self.ptr)
            except Exception:
                pass
            self.ptr = None

    def params(self):
        a = np.zeros(self.n, dtype=np.float32)
        b = np.zeros(self.n, dtype=np.float32)
        _check(lib().zbc_mlp_get_params(self.ptr, a.ctypes.data_as(C.c_void_p), b.ctypes.data_as(C.c_void_p)))
        return a, b

    def forward(self, X, stream=None):
        import torch
        out = torch.empty((X.shape[0], 9), dtype=torch.float32, device=X.device)
        _check(lib().zbc_mlp_forward(self.ptr, _ptr(X), X.shape[0], _ptr(out), _stream(stream)))
        return out

    def backward(self, X, T, stream=None):
        import torch
        g = torch.empty(self.n, dtype=torch.float32, device=X.device)
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        _check(lib().zbc_mlp_backward(self.ptr, _ptr(X), _ptr(T), X.shape[0], _ptr(g), _ptr(loss), _stream(stream)))
        return g, loss

    def adam_step(self, grads, lr, stream=None):
        _check(lib().zbc_mlp_adam_step(self.ptr, _ptr(grads), lr, _stream(stream)))

    def train(self, X, T, steps, lr, stream=None):
        import torch
        hist = torch.empty(steps, dtype=torch.float32, device=X.device)
        _check(lib().zbc_mlp_train(self.ptr, _ptr(X), _ptr(T), X.shape[0], steps, lr, _ptr(hist), _stream(stream)))
        return hist

    def widths(self, features, grid, oversample=4, stream=None):
        g = grid_struct(grid)
        w = np.zeros(9 * features.shape[0], dtype=np.int32)
        _check(lib().zbc_rank_widths(self.ptr, _ptr(features), features.shape[0], C.byref(g), oversample,
                                     w.ctypes.data_as(C.c_void_p), _stream(stream)))
        return w


def zbc_matvec(h: Handle, X, Y, prec=FP32_SIMT, stream=None):
    """Y = Z X.  X: (p, ldx) complex64 (column-major m x p); Y: (p, ldy) complex64.  prec:
    FP32_SIMT, TF32X3, BF16X3, TC2, TC_MODE1 or AUTO."""
    p = X.shape[0]
    _check(lib().zbc_matvec(h.ptr, _ptr(X), _ld(X), p, _ptr(Y), _ld(Y), prec, _stream(stream)))
    return Y


def zbc_rmatvec_noalloc(h: Handle, Phi, Psi, stream=None):
    """Psi = Z^H Phi (FP32) using the library's fixed scratch array instead of allocating: for
    callers that cannot allocate at call time (e.g. during CUDA graph capture).  The handle
    needs one earlier zbc_matvec / zbc_rmatvec call."""
    p = Phi.shape[0]
    _check(lib().zbc_rmatvec_noalloc(h.ptr, _ptr(Phi), _ld(Phi), p, _ptr(Psi), _ld(Psi), _stream(stream)))
    return Psi


TUNE_VARIANTS = (
    "fwd_simt6", "fwd_simt9", "fwd_tf32x3", "fwd_bf16x3", "fwd_tc2", "fwd_mode1", "fwd_dc",
    "adj_simt6", "adj_simt9", "adj_mode1",
)


def zbc_tune(h: Handle, p: int, stream=None) -> dict:
    """Time the product variants for p right-hand sides and record the fastest for AUTO; returns
    {variant: ms per call} (inf for a variant that does not fit)."""
    t = (C.c_float * len(TUNE_VARIANTS))()
    _check(lib().zbc_tune(h.ptr, int(p), _stream(stream), t))
    return dict(zip(TUNE_VARIANTS, [float(x) for x in t]))


def zbc_test_wait_limit(h: Handle, polls: int):
    """Test hook: the next FP32 SIMT adjoint launch on h allows its consumers' first stage wait
    `polls` polls (0: give up at once, so zbc_product_status reports ZBC_ETIMEOUT)."""
    _check(lib().zbc_test_wait_limit(h.ptr, int(polls)))


def zbc_product_status(h: Handle, stream=None):
    """Synchronise the stream; raise ZbcError(ZBC_ETIMEOUT) if a product kernel of h gave up a
    bounded device wait since the last check, else ZbcError(ZBC_ENAN) if one read a NaN or Inf
    from X or Phi.  Clears the handle's error word."""
    _check(lib().zbc_product_status(h.ptr, _stream(stream)))


def zbc_rmatvec(h: Handle, Phi, Psi, prec=FP32_SIMT, stream=None):
    """Psi = Z^H Phi.  Phi: (p, ldphi) complex64 (column-major q n_v x p); Psi: (p, ldpsi)
    complex64.  prec: FP32_SIMT, TC_MODE1 or AUTO."""
    p = Phi.shape[0]
    _check(lib().zbc_rmatvec(h.ptr, _ptr(Phi), _ld(Phi), p, _ptr(Psi), _ld(Psi), prec, _stream(stream)))
    return Psi
