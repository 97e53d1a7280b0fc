"""GB300 sparse symbolic LU factorisation (gSoFa, arXiv 2007.00840).

Thin Python binding over ``libgsofa.so`` (C ABI: ``include/gsofa.h``).  Every
step of the computation runs in the library's CUDA kernels; this module only
marshals arguments.  PyTorch is used for device memory and streams.

    import paper_2007_00840_gb300 as gs
    r = gs.symbolic_device(rowptr_cuda, colidx_cuda)      # torch int32 CUDA tensors
    r.L_rowptr, r.L_colidx, r.U_rowptr, r.U_colidx, r.fill_count, r.super_start
    h = gs.symbolic_host(rowptr_np, colidx_np)            # numpy in, numpy out
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import GsofaError, gsofa_options, gsofa_result

__all__ = ["options", "symbolic_device", "symbolic_host", "batch_device", "row_counts_noalloc", "Server",
           "DeviceResult", "HostResult", "results_to_host", "GsofaError", "load", "version"]

load = _lib.load


def version() -> int:
    return load().gsofa_version()


def options(**kw) -> gsofa_options:
    """gsofa_options with defaults, overridden by keyword (field names of the C struct)."""
    lib = load()
    o = gsofa_options()
    lib.gsofa_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


class _CAI:
    """__cuda_array_interface__ holder that keeps the owning result alive."""

    def __init__(self, ptr: int, count: int, typestr: str, owner, stream: int):
        self.__cuda_array_interface__ = {
            "shape": (int(count),), "typestr": typestr, "data": (int(ptr) if count else 0, False),
            "version": 3, "strides": None, "stream": stream if stream else None,
        }
        self._owner = owner


class _Owner:
    def __init__(self, res: gsofa_result):
        self.res = res

    def __del__(self):
        try:
            _lib.load().gsofa_free(ctypes.byref(self.res))
        except Exception:
            pass


def _stats(res: gsofa_result) -> dict:
    s = res.stats
    return {f: getattr(s, f) for f, _ in s._fields_}


_FIELDS = ("L_rowptr", "L_colidx", "U_rowptr", "U_colidx", "fill_count", "super_start")


class DeviceResult:
    """Device-resident result; the arrays alias library memory (freed when the
    result and every tensor taken from it are gone).  Tensors are created on
    first access."""

    def __init__(self, res: gsofa_result, stream: int, group=None):
        self._owner = _Owner(res)
        self._stream = stream
        self._group = group  # results of one gsofa_batch call share one device block
        self._t = {}
        self.n = res.n
        self.nnz_L = int(res.nnz_L)
        self.nnz_U = int(res.nnz_U)
        self.n_super = int(res.n_super)
        self.stats = _stats(res)

    def _raw(self, name: str):
        """(device pointer, element count, typestr, torch dtype) of one output array."""
        import torch
        r, n = self._owner.res, self.n
        return {"L_rowptr": (r.L_rowptr, n + 1, "<i8", torch.int64),
                "L_colidx": (r.L_colidx, self.nnz_L, "<i4", torch.int32),
                "U_rowptr": (r.U_rowptr, n + 1, "<i8", torch.int64),
                "U_colidx": (r.U_colidx, self.nnz_U, "<i4", torch.int32),
                "fill_count": (r.fill_count, n, "<i4", torch.int32),
                "super_start": (r.super_start, self.n_super + 1, "<i4", torch.int32)}[name]

    def _tensor(self, name: str):
        import torch
        t = self._t.get(name)
        if t is None:
            ptr, count, typestr, dtype = self._raw(name)
            if count == 0:
                t = torch.empty(0, dtype=dtype, device="cuda")
            else:
                t = torch.as_tensor(_CAI(ptr, count, typestr, self._owner, self._stream), device="cuda")
            self._t[name] = t
        return t

    L_rowptr = property(lambda self: self._tensor("L_rowptr"))
    L_colidx = property(lambda self: self._tensor("L_colidx"))
    U_rowptr = property(lambda self: self._tensor("U_rowptr"))
    U_colidx = property(lambda self: self._tensor("U_colidx"))
    fill_count = property(lambda self: self._tensor("fill_count"))
    super_start = property(lambda self: self._tensor("super_start"))

    def to_host(self) -> "HostResult":
        return results_to_host([self])[0]


def results_to_host(results) -> list:
    """Copy device results to host arrays through pinned memory on the current
    stream, with one synchronisation for all.  Arrays of one batch call that are
    adjacent in device memory (its results share one block per field) are copied
    as one span, so a batch costs a few large copies instead of six per matrix;
    arrays of different calls are separate allocations and are copied apart."""
    import torch
    out = [[None] * len(_FIELDS) for _ in results]
    pending = []
    for f, nm in enumerate(_FIELDS):
        arrs = []
        for k, r in enumerate(results):
            ptr, count, typestr, dtype = r._raw(nm)
            if count == 0:
                out[k][f] = (torch.empty(0, dtype=dtype), 0, 0)
            else:
                # members of one batch call share a block (matrices above the on-chip
                # limit, and empty ones, run alone and report their own traversal launches)
                member = r._group is not None and r.n > 0 and r.stats.get("traverse_launches", 1) == 0
                arrs.append((int(ptr), int(count), typestr, dtype, k, ("batch", r._group) if member else ("one", k)))
        arrs.sort(key=lambda x: x[0])
        i = 0
        while i < len(arrs):
            ptr0, _, typestr, dtype, _, _ = arrs[i]
            esz = 8 if typestr == "<i8" else 4
            end = ptr0 + arrs[i][1] * esz
            j = i + 1
            while (j < len(arrs) and arrs[j][2] == typestr and arrs[j][0] == end and arrs[j][5] == arrs[i][5]
                   and arrs[i][5][0] == "batch"):
                end += arrs[j][1] * esz
                j += 1
            group = arrs[i:j]
            total = sum(g[1] for g in group)
            owners = [results[g[4]]._owner for g in group]
            span = torch.as_tensor(_CAI(ptr0, total, typestr, owners, results[group[0][4]]._stream),
                                   device="cuda")
            h = torch.empty(total, dtype=dtype, pin_memory=True)
            h.copy_(span, non_blocking=True)
            pending.append((span, h))
            off = 0
            for g in group:
                out[g[4]][f] = (h, off, g[1])
                off += g[1]
            i = j
    torch.cuda.current_stream().synchronize()
    return [HostResult(r.n, *[h[o:o + c].numpy() for h, o, c in out[k]], r.stats) for k, r in enumerate(results)]


class HostResult:
    def __init__(self, n, L_rowptr, L_colidx, U_rowptr, U_colidx, fill_count, super_start, stats=None):
        self.n = n
        self.L_rowptr, self.L_colidx = L_rowptr, L_colidx
        self.U_rowptr, self.U_colidx = U_rowptr, U_colidx
        self.fill_count, self.super_start = fill_count, super_start
        self.nnz_L, self.nnz_U = int(L_rowptr[-1]), int(U_rowptr[-1])
        self.n_super = int(super_start.size - 1)
        self.stats = stats or {}


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def symbolic_device(rowptr, colidx, n: int | None = None, opts: gsofa_options | None = None,
                    stream=None) -> DeviceResult:
    """Symbolic LU of a device CSR (int32 CUDA tensors) -> DeviceResult (gsofa_symbolic_device)."""
    import torch
    lib = load()
    if not (rowptr.is_cuda and colidx.is_cuda):
        raise ValueError("symbolic_device needs CUDA tensors; use symbolic_host for host arrays")
    if rowptr.dtype != torch.int32 or colidx.dtype != torch.int32:
        raise TypeError("rowptr and colidx must be int32")
    rowptr = rowptr.contiguous()
    colidx = colidx.contiguous()
    n = int(rowptr.numel() - 1) if n is None else int(n)
    res = gsofa_result()
    sh = _stream_handle(stream)
    rc = lib.gsofa_symbolic_device(n, ctypes.c_void_p(rowptr.data_ptr()),
                                   ctypes.c_void_p(colidx.data_ptr() if colidx.numel() else rowptr.data_ptr()),
                                   ctypes.byref(opts) if opts is not None else None, ctypes.c_void_p(sh),
                                   ctypes.byref(res))
    if rc != 0:
        raise GsofaError(rc, res.err_detail, "gsofa_symbolic_device")
    return DeviceResult(res, sh)


def symbolic_host_raw(rowptr: np.ndarray, colidx: np.ndarray, opts: gsofa_options | None = None) -> gsofa_result:
    """gsofa_symbolic on host arrays; returns the raw result (caller frees with free_raw)."""
    lib = load()
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    colidx = np.ascontiguousarray(colidx, dtype=np.int32)
    n = int(rowptr.size - 1)
    res = gsofa_result()
    ci = colidx if colidx.size else np.zeros(1, np.int32)
    rc = lib.gsofa_symbolic(n, rowptr.ctypes.data_as(ctypes.c_void_p), ci.ctypes.data_as(ctypes.c_void_p),
                            ctypes.byref(opts) if opts is not None else None, ctypes.byref(res))
    if rc != 0:
        raise GsofaError(rc, res.err_detail, "gsofa_symbolic")
    return res


def free_raw(res: gsofa_result) -> None:
    load().gsofa_free(ctypes.byref(res))


def _host_array(ptr, count, ctype, dtype):
    if count == 0:
        return np.zeros(0, dtype=dtype)
    buf = (ctype * int(count)).from_address(int(ptr))
    return np.frombuffer(buf, dtype=dtype).copy()


def symbolic_host(rowptr: np.ndarray, colidx: np.ndarray, opts: gsofa_options | None = None) -> HostResult:
    """Symbolic LU of a host CSR (numpy int32) -> HostResult with numpy arrays (gsofa_symbolic)."""
    res = symbolic_host_raw(rowptr, colidx, opts)
    try:
        n = res.n
        out = HostResult(
            n,
            _host_array(res.L_rowptr, n + 1, ctypes.c_int64, np.int64),
            _host_array(res.L_colidx, res.nnz_L, ctypes.c_int32, np.int32),
            _host_array(res.U_rowptr, n + 1, ctypes.c_int64, np.int64),
            _host_array(res.U_colidx, res.nnz_U, ctypes.c_int32, np.int32),
            _host_array(res.fill_count, n, ctypes.c_int32, np.int32),
            _host_array(res.super_start, res.n_super + 1, ctypes.c_int32, np.int32),
            _stats(res),
        )
    finally:
        free_raw(res)
    return out


def batch_device(mats, opts: gsofa_options | None = None, stream=None) -> list:
    """Many device CSRs [(rowptr, colidx), ...] in one gsofa_batch call -> list of DeviceResult."""
    lib = load()
    k = len(mats)
    ns = (ctypes.c_int32 * max(k, 1))()
    rps = (ctypes.c_void_p * max(k, 1))()
    cis = (ctypes.c_void_p * max(k, 1))()
    keep = []
    for i, (rp, ci) in enumerate(mats):
        rp = rp.contiguous()
        ci = ci.contiguous()
        keep.append((rp, ci))
        ns[i] = rp.numel() - 1
        rps[i] = rp.data_ptr()
        cis[i] = ci.data_ptr() if ci.numel() else rp.data_ptr()
    outs = (gsofa_result * max(k, 1))()
    sh = _stream_handle(stream)
    rc = lib.gsofa_batch(k, ctypes.cast(ns, ctypes.c_void_p), ctypes.cast(rps, ctypes.c_void_p),
                         ctypes.cast(cis, ctypes.c_void_p), ctypes.byref(opts) if opts is not None else None,
                         ctypes.c_void_p(sh), ctypes.cast(outs, ctypes.c_void_p))
    if rc != 0:
        raise GsofaError(rc, -1, "gsofa_batch")
    res = []
    group = object()
    for i in range(k):
        r = gsofa_result()
        ctypes.pointer(r)[0] = outs[i]
        res.append(DeviceResult(r, sh, group))
    return res


def row_counts_noalloc(rowptr, colidx, nnzL, nnzU, fill_count, stream=None) -> None:
    """gsofa_row_counts_noalloc into caller-provided int32 CUDA tensors (no device allocation)."""
    lib = load()
    n = int(rowptr.numel() - 1)
    rc = lib.gsofa_row_counts_noalloc(n, ctypes.c_void_p(rowptr.data_ptr()), ctypes.c_void_p(colidx.data_ptr()),
                                      ctypes.c_void_p(nnzL.data_ptr()), ctypes.c_void_p(nnzU.data_ptr()),
                                      ctypes.c_void_p(fill_count.data_ptr()), ctypes.c_void_p(_stream_handle(stream)))
    if rc != 0:
        raise GsofaError(rc, -1, "gsofa_row_counts_noalloc")


class Server:
    """Continuous-batching server (gsofa_server_*).  Inputs must stay alive until collected."""

    def __init__(self, mem_cap_bytes: int = 0, streams: int = 0, max_batch: int = 0, max_inflight: int = 0,
                 queue_capacity: int = 0, opts: gsofa_options | None = None):
        lib = load()
        cfg = _lib.gsofa_server_config()
        lib.gsofa_server_default_config(ctypes.byref(cfg))
        if mem_cap_bytes:
            cfg.mem_cap_bytes = mem_cap_bytes
        if streams:
            cfg.streams = streams
        if max_batch:
            cfg.max_batch = max_batch
        if max_inflight:
            cfg.max_inflight = max_inflight
        if queue_capacity:
            cfg.queue_capacity = queue_capacity
        if opts is not None:
            cfg.opts = opts
        h = ctypes.c_void_p()
        rc = lib.gsofa_server_create(ctypes.byref(cfg), ctypes.byref(h))
        if rc != 0:
            raise GsofaError(rc, -1, "gsofa_server_create")
        self._h = h
        self._keep = {}

    def submit(self, rowptr, colidx) -> int:
        """Queue a pattern: int32 CUDA tensors (device-resident) or numpy arrays (host)."""
        lib = load()
        t = ctypes.c_uint64()
        if hasattr(rowptr, "is_cuda") and rowptr.is_cuda:
            n = int(rowptr.numel() - 1)
            rc = lib.gsofa_server_submit(self._h, n, ctypes.c_void_p(rowptr.data_ptr()),
                                         ctypes.c_void_p(colidx.data_ptr() if colidx.numel() else rowptr.data_ptr()),
                                         1, ctypes.byref(t))
        else:
            rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
            colidx = np.ascontiguousarray(colidx, dtype=np.int32)
            if colidx.size == 0:
                colidx = np.zeros(1, np.int32)
            rc = lib.gsofa_server_submit(self._h, int(rowptr.size - 1), rowptr.ctypes.data_as(ctypes.c_void_p),
                                         colidx.ctypes.data_as(ctypes.c_void_p), 0, ctypes.byref(t))
        if rc != 0:
            raise GsofaError(rc, -1, "gsofa_server_submit")
        self._keep[t.value] = (rowptr, colidx)
        return t.value

    def poll(self, ticket: int):
        """(DeviceResult, latency_ms) if finished, else None."""
        lib = load()
        r = gsofa_result()
        lat = ctypes.c_double()
        rc = lib.gsofa_server_poll(self._h, ctypes.c_uint64(ticket), ctypes.byref(r), ctypes.byref(lat))
        if rc == _lib.GSOFA_E_PENDING:
            return None
        self._keep.pop(ticket, None)
        if rc != 0:
            raise GsofaError(rc, -1, "gsofa_server_poll")
        return DeviceResult(r, 0), lat.value

    def wait(self, ticket: int, timeout: float = 600.0, keep_result: bool = True):
        lib = load()
        r = gsofa_result()
        lat = ctypes.c_double()
        rc = lib.gsofa_server_wait(self._h, ctypes.c_uint64(ticket), timeout,
                                   ctypes.byref(r) if keep_result else None, ctypes.byref(lat))
        self._keep.pop(ticket, None)
        if rc != 0:
            raise GsofaError(rc, -1, "gsofa_server_wait")
        return (DeviceResult(r, 0) if keep_result else None), lat.value

    def stats(self) -> dict:
        st = _lib.gsofa_server_stats()
        load().gsofa_server_get_stats(self._h, ctypes.byref(st))
        return {f: getattr(st, f) for f, _ in st._fields_ if not f.startswith("pad")}

    def close(self):
        if getattr(self, "_h", None):
            load().gsofa_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
