"""Binding of the serving loop (C ABI: include/nufft_serve.h).

``nufft_server_*`` carry the C names and only marshal arguments.  ``Server``
adds torch tensors: inputs are moved to the server's device on the caller's
current stream, an event recorded after them is handed to the request (the
slot stream waits on it), and every tensor a request touches is kept alive
until its completion has been polled.  All transform work runs in the
library's kernels on the server's slot streams.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

from . import NufftError, NUFFT_C64, NUFFT_C128, _L as _base_lib  # noqa: F401 (re-exported)

NUFFT_REQ_TYPE1 = 1
NUFFT_REQ_TYPE2 = 2
NUFFT_REQ_LSQ_GRAD = 3
NUFFT_FLAG_XGRAD_KERNEL = 1
NUFFT_ERR_TIMEOUT = -8
NUFFT_ERR_REJECTED = -9
NUFFT_ERR_SHUTDOWN = -10


class nufft_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("flags", ctypes.c_int), ("dim", ctypes.c_int), ("nmodes", ctypes.c_int64 * 3),
                ("isign", ctypes.c_int), ("prec", ctypes.c_int), ("eps", ctypes.c_double),
                ("upsampfac", ctypes.c_double), ("M", ctypes.c_int64),
                ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("in_", ctypes.c_void_p), ("in2", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("out2", ctypes.c_void_p), ("out3", ctypes.c_void_p), ("points_key", ctypes.c_uint64),
                ("ready_event", ctypes.c_void_p), ("tag", ctypes.c_uint64)]


class nufft_completion(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_int64), ("tag", ctypes.c_uint64), ("status", ctypes.c_int),
                ("reused", ctypes.c_int), ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double), ("pending", ctypes.c_int)]


class nufft_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "submitted", "completed", "timeouts", "rejected", "entries_created", "entries_evicted", "entries_reused",
        "binning_skipped", "queued", "inflight", "peak_inflight", "bytes_in_use", "peak_bytes", "budget_bytes")]


ESTIMATE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(nufft_request), ctypes.c_int64,
                               ctypes.POINTER(ctypes.c_size_t))
CREATE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(nufft_request), ctypes.c_int64,
                             ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_size_t))
LAUNCH_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(nufft_request),
                             ctypes.c_int, ctypes.c_int, ctypes.c_int64)
DESTROY_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class nufft_executor(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("estimate", ESTIMATE_FN), ("create", CREATE_FN), ("launch", LAUNCH_FN),
                ("destroy", DESTROY_FN)]


_ready = False


def _L():
    global _ready
    lib = _base_lib()
    if not _ready:
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        lib.nufft_server_create.argtypes = [ctypes.c_size_t, i32, dbl, ctypes.POINTER(vp)]
        lib.nufft_server_create_with_executor.argtypes = [ctypes.POINTER(nufft_executor), ctypes.c_size_t, i32, dbl,
                                                          ctypes.POINTER(vp)]
        lib.nufft_server_submit.argtypes = [vp, ctypes.POINTER(nufft_request), ctypes.POINTER(i64)]
        lib.nufft_server_poll.argtypes = [vp, ctypes.POINTER(nufft_completion), i32, ctypes.POINTER(i32), dbl]
        lib.nufft_server_drain.argtypes = [vp, dbl]
        lib.nufft_server_set_shutdown_wait.argtypes = [vp, dbl]
        lib.nufft_server_stats_get.argtypes = [vp, ctypes.POINTER(nufft_server_stats)]
        lib.nufft_server_destroy.argtypes = [vp]
        lib.nufft_server_clock.argtypes = []
        lib.nufft_server_clock.restype = dbl
        lib.nufft_server_complete.argtypes = [vp, i64, i32]
        lib.nufft_server_complete.restype = None
        lib.nufft_request_bytes.argtypes = [ctypes.POINTER(nufft_request), i64, ctypes.POINTER(ctypes.c_size_t)]
        lib.nufft_request_upsampfac.argtypes = [ctypes.POINTER(nufft_request)]
        lib.nufft_request_upsampfac.restype = dbl
        _ready = True
    return lib


# ------------------------------------------------------------ C-name wrappers
def nufft_server_create(budget_bytes: int, max_inflight: int, timeout_s: float):
    h = ctypes.c_void_p()
    st = _L().nufft_server_create(int(budget_bytes), int(max_inflight), float(timeout_s), ctypes.byref(h))
    return st, h


def nufft_server_create_with_executor(ex: nufft_executor, budget_bytes: int, max_inflight: int, timeout_s: float):
    h = ctypes.c_void_p()
    st = _L().nufft_server_create_with_executor(ctypes.byref(ex), int(budget_bytes), int(max_inflight),
                                                float(timeout_s), ctypes.byref(h))
    return st, h


def nufft_server_submit(server, req: nufft_request):
    t = ctypes.c_int64()
    st = _L().nufft_server_submit(server, ctypes.byref(req), ctypes.byref(t))
    return st, t.value


def nufft_server_poll(server, max_n: int = 256, wait_s: float = 0.0):
    buf = (nufft_completion * max(1, max_n))()
    n = ctypes.c_int()
    st = _L().nufft_server_poll(server, buf, int(max_n), ctypes.byref(n), float(wait_s))
    return st, [buf[i] for i in range(n.value)]


def nufft_server_set_shutdown_wait(server, seconds: float) -> int:
    return _L().nufft_server_set_shutdown_wait(server, float(seconds))


def nufft_server_drain(server, timeout_s: float = 0.0) -> int:
    return _L().nufft_server_drain(server, float(timeout_s))


def nufft_server_stats_get(server) -> dict:
    s = nufft_server_stats()
    _L().nufft_server_stats_get(server, ctypes.byref(s))
    return {n: getattr(s, n) for n, _ in nufft_server_stats._fields_}


def nufft_server_destroy(server) -> int:
    return _L().nufft_server_destroy(server)


def nufft_server_clock() -> float:
    return float(_L().nufft_server_clock())


def nufft_server_complete(server, ticket: int, status: int) -> None:
    _L().nufft_server_complete(server, int(ticket), int(status))


def nufft_request_bytes(req: nufft_request, mcap: int):
    b = ctypes.c_size_t()
    st = _L().nufft_request_bytes(ctypes.byref(req), int(mcap), ctypes.byref(b))
    return st, b.value


def nufft_request_upsampfac(req: nufft_request) -> float:
    return float(_L().nufft_request_upsampfac(ctypes.byref(req)))


def upsampfac_for(kind: int, n_modes, eps: float, M: int, prec: int = NUFFT_C64, upsampfac: float = 0.0) -> float:
    """The upsampling factor the server would use for such a request."""
    return nufft_request_upsampfac(make_request(kind, len(n_modes), n_modes, -1, prec, eps, M, upsampfac=upsampfac))


def make_request(kind: int, dim: int, n_modes, isign: int, prec: int, eps: float, M: int, tag: int = 0,
                 points_key: int = 0, flags: int = 0, upsampfac: float = 0.0) -> nufft_request:
    r = nufft_request()
    r.flags = int(flags)
    r.upsampfac = float(upsampfac)
    r.kind, r.dim, r.isign, r.prec, r.eps, r.M = int(kind), int(dim), int(isign), int(prec), float(eps), int(M)
    for i, v in enumerate(n_modes):
        r.nmodes[i] = int(v)
    for i in range(len(n_modes), 3):
        r.nmodes[i] = 1
    r.points_key, r.tag = int(points_key), int(tag)
    return r


# --------------------------------------------------------------- torch layer
@dataclass
class Completion:
    ticket: int
    tag: int
    status: int
    reused: int
    t_submit: float
    t_admit: float
    t_done: float
    outputs: dict = field(default_factory=dict)
    pending: int = 0  # 1: an early time-limit report; the final completion of the ticket follows


class Server:
    """A request loop on one CUDA device (see include/nufft_serve.h).

    ``type1(x, c, n_modes, ...)``, ``type2(x, f, ...)`` and
    ``lsq_grad(x, f, y, ...)`` queue a request and return its ticket at once;
    ``poll`` returns finished requests with their output tensors
    (type 1: ``f``, type 2: ``c``, gradient: ``loss``, ``grad_f``, ``grad_x``).
    ``x`` is a (d, M) real tensor or a list of d coordinate tensors.
    """

    def __init__(self, budget_bytes: int | None = None, max_inflight: int = 8, timeout_s: float = 0.0, device=None):
        import torch
        self._torch = torch
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self._h = None
        with torch.cuda.device(self.device):
            if budget_bytes is None:
                free, _ = torch.cuda.mem_get_info(self.device)
                budget_bytes = int(free * 0.5)
            st, h = nufft_server_create(budget_bytes, max_inflight, timeout_s)
        if st < 0:
            raise NufftError(st, "nufft_server_create")
        self._h = h
        self.budget_bytes = int(budget_bytes)
        self._live = {}
        self._late = {}  # ticket -> tensors of a request reported early (time limit), held until its final completion

    def _coords(self, x, rdt):
        torch = self._torch
        if isinstance(x, torch.Tensor) and x.dim() == 2:
            xs = list(x.unbind(0))
        else:
            xs = list(x)
        return [torch.as_tensor(v).to(device=self.device, dtype=rdt).contiguous() for v in xs]

    def _submit(self, kind, xs, data, n_modes, eps, isign, dtype, y=None, points_key=0, tag=0, flags=0,
                upsampfac=0.0):
        torch = self._torch
        cdt = dtype
        rdt = torch.float32 if cdt == torch.complex64 else torch.float64
        prec = NUFFT_C64 if cdt == torch.complex64 else NUFFT_C128
        with torch.cuda.device(self.device):
            xs = self._coords(xs, rdt)
            d = len(xs)
            M = xs[0].numel()
            data = torch.as_tensor(data).to(device=self.device, dtype=cdt).contiguous()
            r = make_request(kind, d, n_modes, isign, prec, eps, M, tag=tag, points_key=points_key, flags=flags,
                             upsampfac=upsampfac)
            ptr = [v.data_ptr() for v in xs] + [0] * (3 - d)
            r.x, r.y, r.z = ptr
            r.in_ = data.data_ptr()
            outs = {}
            keep = [xs, data]
            shape_f = tuple(reversed([int(v) for v in n_modes]))
            if kind == NUFFT_REQ_TYPE1:
                outs["f"] = torch.empty(shape_f, dtype=cdt, device=self.device)
                r.out = outs["f"].data_ptr()
            elif kind == NUFFT_REQ_TYPE2:
                outs["c"] = torch.empty(M, dtype=cdt, device=self.device)
                r.out = outs["c"].data_ptr()
            else:
                yv = torch.as_tensor(y).to(device=self.device, dtype=cdt).contiguous()
                keep.append(yv)
                r.in2 = yv.data_ptr()
                outs["grad_f"] = torch.empty(shape_f, dtype=cdt, device=self.device)
                outs["grad_x"] = torch.empty((d, M), dtype=rdt, device=self.device)
                outs["loss"] = torch.empty(1, dtype=torch.float64, device=self.device)
                r.out, r.out2, r.out3 = (outs["grad_f"].data_ptr(), outs["grad_x"].data_ptr(),
                                         outs["loss"].data_ptr())
            ev = torch.cuda.Event()
            ev.record(torch.cuda.current_stream(self.device))
            r.ready_event = ev.cuda_event
            st, ticket = nufft_server_submit(self._h, r)
        if st < 0:
            raise NufftError(st, "nufft_server_submit")
        self._live[ticket] = (keep, outs, ev)
        return ticket

    # upsampfac: 2 or 1.25, or 0 (the server picks per request, see nufft_request_upsampfac)
    def type1(self, x, c, n_modes, eps=1e-6, isign=1, dtype=None, points_key=0, tag=0, upsampfac=0.0):
        dtype = dtype or self._torch.complex64
        return self._submit(NUFFT_REQ_TYPE1, x, c, n_modes, eps, isign, dtype, points_key=points_key, tag=tag,
                            upsampfac=upsampfac)

    def type2(self, x, f, eps=1e-6, isign=-1, dtype=None, points_key=0, tag=0, upsampfac=0.0):
        dtype = dtype or self._torch.complex64
        n_modes = tuple(reversed(f.shape))
        return self._submit(NUFFT_REQ_TYPE2, x, f, n_modes, eps, isign, dtype, points_key=points_key, tag=tag,
                            upsampfac=upsampfac)

    def lsq_grad(self, x, f, y, eps=1e-6, isign=-1, dtype=None, points_key=0, tag=0, xgrad="exact", upsampfac=0.0):
        """loss = ||F2_isign(f; x) - y||^2 with its gradients in f and in the points
        (``xgrad``: "exact" or "kernel", as in the autograd functions)."""
        if xgrad not in ("exact", "kernel"):
            raise ValueError("xgrad must be 'exact' or 'kernel'")
        dtype = dtype or self._torch.complex64
        n_modes = tuple(reversed(f.shape))
        return self._submit(NUFFT_REQ_LSQ_GRAD, x, f, n_modes, eps, isign, dtype, y=y, points_key=points_key,
                            tag=tag, flags=NUFFT_FLAG_XGRAD_KERNEL if xgrad == "kernel" else 0, upsampfac=upsampfac)

    def poll(self, max_n: int = 256, wait_s: float = 0.0):
        st, cs = nufft_server_poll(self._h, max_n, wait_s)
        out = []
        for c in cs:
            if c.pending:  # its kernels may still write: hold its tensors until the final completion
                self._late[c.ticket] = self._live.pop(c.ticket, (None, {}, None))
                out.append(Completion(c.ticket, c.tag, c.status, c.reused, c.t_submit, c.t_admit, c.t_done, {}, 1))
                continue
            keep = self._live.pop(c.ticket, None)
            if keep is None:
                keep = self._late.pop(c.ticket, (None, {}, None))
            out.append(Completion(c.ticket, c.tag, c.status, c.reused, c.t_submit, c.t_admit, c.t_done,
                                  keep[1] if c.status == 0 else {}))
        return out

    def drain(self, timeout_s: float = 0.0) -> int:
        st = nufft_server_drain(self._h, timeout_s)
        if st == 0:
            self._late = {}
        return st

    def stats(self) -> dict:
        return nufft_server_stats_get(self._h)

    @staticmethod
    def clock() -> float:
        return nufft_server_clock()

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            nufft_server_destroy(self._h)
        self._h = None
        self._live = {}
        self._late = {}  # ticket -> tensors of a request reported early (time limit), held until its final completion

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
