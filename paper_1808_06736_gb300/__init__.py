"""GB300 (sm_103a) type-1 / type-2 NUFFT with the "exponential of semicircle" kernel
(Barnett, Magland & af Klinteberg, arXiv:1808.06736).

Python binding of ``libnufft_gb300.so`` (C ABI: include/nufft_gb300.h).  The
module-level ``nufft_*`` functions carry the C names and only marshal
arguments; ``Plan`` adds torch-tensor handling (device memory, the current
CUDA stream, host <-> device copies for CPU tensors).  Every step of a
transform runs in the library's CUDA kernels and cuFFT; there is no CPU
fallback: without the built library every call raises.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

__all__ = [
    "Plan", "NufftError", "nufft_opts", "nufft_default_opts", "nufft_makeplan", "nufft_setpts",
    "nufft_execute", "nufft_execute_grad", "nufft_destroy", "nufft_get_status", "nufft_get_timings", "nufft_plan_info",
    "nufft_strerror", "nufft_choose_params", "nufft_choose_params_sigma", "nufft_correction_factors", "nufft_next235",
    "nufft_horner_coeffs", "nufft_measure_peaks",
    "nufft_spread_noalloc", "library_path", "BatchPlan", "nufft_batch_makeplan", "nufft_batch_setpts",
    "nufft_batch_execute", "nufft_batch_get_status", "nufft_batch_destroy", "nufft_tune", "nufft_batch_tune",
    "nufft_tune_candidates", "opts_dict", "tune_plan", "tune_batch", "Plan3", "nufft3_makeplan", "nufft3_setpts",
    "nufft3_execute", "nufft3_plan_info", "nufft3_get_status", "nufft3_destroy",
    "NUFFT_C64", "NUFFT_C128",
]

NUFFT_C64 = 1
NUFFT_C128 = 2
STATUS = {
    0: "NUFFT_OK", 1: "NUFFT_WARN_EPS_TOO_SMALL", -1: "NUFFT_ERR_BAD_ARG", -2: "NUFFT_ERR_OUT_OF_RANGE",
    -3: "NUFFT_ERR_ALLOC", -4: "NUFFT_ERR_CUDA", -5: "NUFFT_ERR_CUFFT", -6: "NUFFT_ERR_NOT_SET",
    -7: "NUFFT_ERR_TOO_BIG",
}


class NufftError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__("%s: %s (%d)" % (where, STATUS.get(code, "unknown"), code))


class nufft_opts(ctypes.Structure):
    _fields_ = [("debug", ctypes.c_int), ("chkbnds", ctypes.c_int), ("modeord", ctypes.c_int),
                ("bin_size", ctypes.c_int * 3), ("max_subprob", ctypes.c_int), ("threads", ctypes.c_int),
                ("sparse_max", ctypes.c_int), ("kerevalmeth", ctypes.c_int), ("kernel", ctypes.c_int),
                ("reserved", ctypes.c_int * 5),
                ("upsampfac", ctypes.c_double)]


_lib = None


def library_path() -> str:
    return _build.LIB_PATH


def _L():
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB_PATH
    if not os.path.exists(path):
        raise ImportError("libnufft_gb300.so is not built (expected at %s); run "
                          "paper_1808_06736_gb300.build.build() or __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    pi64 = ctypes.POINTER(ctypes.c_int64)
    lib.nufft_default_opts.argtypes = [ctypes.POINTER(nufft_opts)]
    lib.nufft_makeplan.argtypes = [i32, i32, pi64, i32, i32, dbl, i32, vp, ctypes.POINTER(nufft_opts),
                                   ctypes.POINTER(vp)]
    lib.nufft_setpts.argtypes = [vp, i64, vp, vp, vp]
    lib.nufft_setpts_from.argtypes = [vp, vp]
    lib.nufft_execute.argtypes = [vp, vp, vp]
    lib.nufft_execute_grad.argtypes = [vp, vp, vp, vp]
    lib.nufft_destroy.argtypes = [vp]
    lib.nufft_get_status.argtypes = [vp]
    lib.nufft_get_timings.argtypes = [vp, ctypes.POINTER(ctypes.c_double), i32]
    lib.nufft_plan_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(dbl), pi64, ctypes.POINTER(i32), pi64]
    lib.nufft_strerror.argtypes = [i32]
    lib.nufft_strerror.restype = ctypes.c_char_p
    lib.nufft_choose_params.argtypes = [i32, pi64, dbl, i32, ctypes.POINTER(i32), ctypes.POINTER(dbl), pi64]
    lib.nufft_choose_params_sigma.argtypes = [i32, pi64, dbl, i32, dbl, ctypes.POINTER(i32), ctypes.POINTER(dbl),
                                              pi64]
    lib.nufft_correction_factors.argtypes = [i64, i64, i32, dbl, ctypes.POINTER(ctypes.c_double)]
    lib.nufft_next235.argtypes = [i64]
    lib.nufft_horner_coeffs.argtypes = [i32, dbl, ctypes.POINTER(ctypes.c_double)]
    lib.nufft_next235.restype = i64
    lib.nufft_spread_noalloc.argtypes = [i32, pi64, i32, dbl, i64, vp, vp, vp, vp, vp, vp]
    lib.nufft_batch_makeplan.argtypes = [i32, i32, i32, pi64, i32, dbl, i32, vp, ctypes.POINTER(nufft_opts),
                                         ctypes.POINTER(vp)]
    lib.nufft_batch_setpts.argtypes = [vp, pi64, vp, vp, vp]
    lib.nufft_batch_execute.argtypes = [vp, vp, vp]
    lib.nufft_batch_get_status.argtypes = [vp]
    lib.nufft_batch_destroy.argtypes = [vp]
    pd = ctypes.POINTER(ctypes.c_double)
    lib.nufft_tune.argtypes = [i32, i32, pi64, i32, dbl, i32, i64, vp, vp, vp, vp, vp, vp, i32,
                               ctypes.POINTER(nufft_opts), pd, pd]
    lib.nufft_batch_tune.argtypes = [i32, i32, i32, pi64, i32, dbl, i32, pi64, vp, vp, vp, vp, vp, vp, i32,
                                     ctypes.POINTER(nufft_opts), pd, pd]
    lib.nufft_tune_candidates.argtypes = [i32, i32, i32, ctypes.POINTER(i32), i32]
    lib.nufft_measure_peaks.argtypes = [vp, pd, i32]
    lib.nufft3_makeplan.argtypes = [i32, i32, dbl, i32, vp, ctypes.POINTER(nufft_opts), ctypes.POINTER(vp)]
    lib.nufft3_setpts.argtypes = [vp, i64, vp, vp, vp, i64, vp, vp, vp]
    lib.nufft3_execute.argtypes = [vp, vp, vp]
    lib.nufft3_plan_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(dbl), pi64, pd]
    lib.nufft3_get_status.argtypes = [vp]
    lib.nufft3_destroy.argtypes = [vp]
    _lib = lib
    return lib


# ------------------------------------------------------------ C-name wrappers
def nufft_default_opts() -> nufft_opts:
    o = nufft_opts()
    _L().nufft_default_opts(ctypes.byref(o))
    return o


def nufft_makeplan(type_: int, dim: int, nmodes, isign: int, ntransf: int, eps: float, prec: int,
                   stream: int | None, opts: nufft_opts | None):
    """Returns (status, plan handle)."""
    arr = (ctypes.c_int64 * 3)(*([int(v) for v in nmodes] + [1] * (3 - len(nmodes))))
    h = ctypes.c_void_p()
    st = _L().nufft_makeplan(int(type_), int(dim), arr, int(isign), int(ntransf), float(eps), int(prec),
                             ctypes.c_void_p(stream or 0), ctypes.byref(opts) if opts is not None else None,
                             ctypes.byref(h))
    return st, h


def nufft_setpts(plan, M: int, x: int, y: int, z: int) -> int:
    return _L().nufft_setpts(plan, int(M), ctypes.c_void_p(x or 0), ctypes.c_void_p(y or 0), ctypes.c_void_p(z or 0))


def nufft_setpts_from(dst, src) -> int:
    return _L().nufft_setpts_from(dst, src)


def nufft_execute(plan, c: int, f: int) -> int:
    return _L().nufft_execute(plan, ctypes.c_void_p(c or 0), ctypes.c_void_p(f or 0))


def nufft_execute_grad(plan, c: int, dc: int, f: int) -> int:
    return _L().nufft_execute_grad(plan, ctypes.c_void_p(c or 0), ctypes.c_void_p(dc or 0), ctypes.c_void_p(f or 0))


def nufft_destroy(plan) -> int:
    return _L().nufft_destroy(plan)


def nufft_get_status(plan) -> int:
    return _L().nufft_get_status(plan)


def nufft_get_timings(plan, n: int = 6):
    buf = (ctypes.c_double * n)()
    k = _L().nufft_get_timings(plan, buf, n)
    return k, list(buf)[: max(k, 0)]


def nufft_plan_info(plan, dim: int):
    w, beta = ctypes.c_int(), ctypes.c_double()
    n = (ctypes.c_int64 * 3)()
    bins = (ctypes.c_int * 3)()
    nsub = ctypes.c_int64()
    st = _L().nufft_plan_info(plan, ctypes.byref(w), ctypes.byref(beta), n, bins, ctypes.byref(nsub))
    return st, dict(w=w.value, beta=beta.value, n=list(n)[:dim], bins=list(bins)[:dim], nsub=nsub.value)


def nufft_strerror(code: int) -> str:
    return _L().nufft_strerror(int(code)).decode()


def nufft_choose_params(dim: int, nmodes, eps: float, prec: int = NUFFT_C128):
    arr = (ctypes.c_int64 * 3)(*([int(v) for v in nmodes] + [1] * (3 - len(nmodes))))
    w, beta = ctypes.c_int(), ctypes.c_double()
    n = (ctypes.c_int64 * 3)()
    st = _L().nufft_choose_params(int(dim), arr, float(eps), int(prec), ctypes.byref(w), ctypes.byref(beta), n)
    return st, w.value, beta.value, list(n)[:dim]


def nufft_choose_params_sigma(dim: int, nmodes, eps: float, prec: int, sigma: float):
    arr = (ctypes.c_int64 * 3)(*([int(v) for v in nmodes] + [1] * (3 - len(nmodes))))
    w, beta = ctypes.c_int(), ctypes.c_double()
    n = (ctypes.c_int64 * 3)()
    st = _L().nufft_choose_params_sigma(int(dim), arr, float(eps), int(prec), float(sigma), ctypes.byref(w),
                                        ctypes.byref(beta), n)
    return st, w.value, beta.value, list(n)[:dim]


def nufft_correction_factors(N: int, n: int, w: int, beta: float):
    out = (ctypes.c_double * int(N))()
    st = _L().nufft_correction_factors(int(N), int(n), int(w), float(beta), out)
    return st, list(out)


def nufft_horner_coeffs(w: int, beta: float):
    """(status, w x (w + 4) nested list of the Sec. 5.3 polynomial coefficients)."""
    buf = (ctypes.c_double * (w * (w + 4)))() if 2 <= w <= 16 else None
    st = _L().nufft_horner_coeffs(int(w), float(beta), buf)
    if st != 0:
        return st, None
    v = list(buf)
    return st, [v[t * (w + 4):(t + 1) * (w + 4)] for t in range(w)]


def nufft_next235(m: int) -> int:
    return int(_L().nufft_next235(int(m)))


def nufft_spread_noalloc(dim: int, n, w: int, beta: float, M: int, x: int, y: int, z: int, c: int,
                         grid: int, stream: int | None) -> int:
    """Spreading onto a caller-provided complex64 fine grid with no device allocation
    (pointers are device addresses)."""
    arr = (ctypes.c_int64 * 3)(*([int(v) for v in n] + [1] * (3 - len(n))))
    vp = ctypes.c_void_p
    return _L().nufft_spread_noalloc(int(dim), arr, int(w), float(beta), int(M), vp(x or 0), vp(y or 0),
                                     vp(z or 0), vp(c or 0), vp(grid or 0), vp(stream or 0))


def nufft_batch_makeplan(type_: int, dim: int, nmodes, isign: int, eps: float, prec: int, stream: int | None,
                         opts: nufft_opts | None):
    """nmodes: list of B mode-count tuples.  Returns (status, handle)."""
    B = len(nmodes)
    flat = [int(v) for m in nmodes for v in m]
    arr = (ctypes.c_int64 * len(flat))(*flat)
    h = ctypes.c_void_p()
    st = _L().nufft_batch_makeplan(int(type_), int(dim), B, arr, int(isign), float(eps), int(prec),
                                   ctypes.c_void_p(stream or 0), ctypes.byref(opts) if opts is not None else None,
                                   ctypes.byref(h))
    return st, h


def nufft_batch_setpts(plan, offsets, x: int, y: int, z: int) -> int:
    arr = (ctypes.c_int64 * len(offsets))(*[int(v) for v in offsets])
    return _L().nufft_batch_setpts(plan, arr, ctypes.c_void_p(x or 0), ctypes.c_void_p(y or 0), ctypes.c_void_p(z or 0))


def nufft_batch_execute(plan, c: int, f: int) -> int:
    return _L().nufft_batch_execute(plan, ctypes.c_void_p(c or 0), ctypes.c_void_p(f or 0))


def nufft_batch_get_status(plan) -> int:
    return _L().nufft_batch_get_status(plan)


def nufft_batch_destroy(plan) -> int:
    return _L().nufft_batch_destroy(plan)


def nufft_tune_candidates(dim: int, prec: int, w: int):
    n = _L().nufft_tune_candidates(int(dim), int(prec), int(w), None, 0)
    if n < 0:
        return n, []
    buf = (ctypes.c_int * (3 * max(n, 1)))()
    _L().nufft_tune_candidates(int(dim), int(prec), int(w), buf, n)
    return n, [tuple(buf[3 * k:3 * k + 3]) for k in range(n)]


def nufft_tune(type_: int, dim: int, nmodes, isign: int, eps: float, prec: int, M: int, x: int, y: int, z: int,
               inp: int, out: int, stream: int | None, reps: int = 3):
    """Returns (status, best nufft_opts, best ms, default ms)."""
    arr = (ctypes.c_int64 * 3)(*([int(v) for v in nmodes] + [1] * (3 - len(nmodes))))
    o = nufft_opts()
    b, d = ctypes.c_double(), ctypes.c_double()
    vp = ctypes.c_void_p
    st = _L().nufft_tune(int(type_), int(dim), arr, int(isign), float(eps), int(prec), int(M), vp(x or 0), vp(y or 0),
                         vp(z or 0), vp(inp or 0), vp(out or 0), vp(stream or 0), int(reps), ctypes.byref(o),
                         ctypes.byref(b), ctypes.byref(d))
    return st, o, b.value, d.value


def nufft_batch_tune(type_: int, dim: int, nmodes, isign: int, eps: float, prec: int, offsets, x: int, y: int,
                     z: int, inp: int, out: int, stream: int | None, reps: int = 3):
    """nmodes: list of B mode-count tuples.  Returns (status, best nufft_opts, best ms, default ms)."""
    flat = [int(v) for m in nmodes for v in m]
    arr = (ctypes.c_int64 * len(flat))(*flat)
    offs = (ctypes.c_int64 * len(offsets))(*[int(v) for v in offsets])
    o = nufft_opts()
    b, d = ctypes.c_double(), ctypes.c_double()
    vp = ctypes.c_void_p
    st = _L().nufft_batch_tune(int(type_), int(dim), len(nmodes), arr, int(isign), float(eps), int(prec), offs,
                               vp(x or 0), vp(y or 0), vp(z or 0), vp(inp or 0), vp(out or 0), vp(stream or 0),
                               int(reps), ctypes.byref(o), ctypes.byref(b), ctypes.byref(d))
    return st, o, b.value, d.value


def nufft_measure_peaks(stream: int | None = None):
    """(status, {fp32_tflops, fp64_tflops, sfu_gops, smem_atomics_per_s}) on the current device."""
    buf = (ctypes.c_double * 4)()
    st = _L().nufft_measure_peaks(ctypes.c_void_p(stream or 0), buf, 4)
    keys = ("fp32_tflops", "fp64_tflops", "sfu_gops", "smem_atomics_per_s")
    return st, (dict(zip(keys, list(buf))) if st == 0 else None)


def nufft3_makeplan(dim: int, isign: int, eps: float, prec: int, stream: int | None, opts: nufft_opts | None):
    """Returns (status, type-3 plan handle)."""
    h = ctypes.c_void_p()
    st = _L().nufft3_makeplan(int(dim), int(isign), float(eps), int(prec), ctypes.c_void_p(stream or 0),
                              ctypes.byref(opts) if opts is not None else None, ctypes.byref(h))
    return st, h


def nufft3_setpts(plan, M: int, x: int, y: int, z: int, N: int, s: int, t: int, u: int) -> int:
    v = lambda a: ctypes.c_void_p(a or 0)  # noqa: E731
    return _L().nufft3_setpts(plan, int(M), v(x), v(y), v(z), int(N), v(s), v(t), v(u))


def nufft3_execute(plan, c: int, f: int) -> int:
    return _L().nufft3_execute(plan, ctypes.c_void_p(c or 0), ctypes.c_void_p(f or 0))


def nufft3_plan_info(plan, dim: int):
    w, beta = ctypes.c_int(), ctypes.c_double()
    n = (ctypes.c_int64 * 3)()
    g = (ctypes.c_double * 3)()
    st = _L().nufft3_plan_info(plan, ctypes.byref(w), ctypes.byref(beta), n, g)
    return st, dict(w=w.value, beta=beta.value, n=list(n)[:dim], gamma=list(g)[:dim])


def nufft3_get_status(plan) -> int:
    return _L().nufft3_get_status(plan)


def nufft3_destroy(plan) -> int:
    return _L().nufft3_destroy(plan)


def _make_opts(opts: dict) -> nufft_opts:
    o = nufft_default_opts()
    for k, v in opts.items():
        if k == "bin_size":
            for i, b in enumerate(v):
                o.bin_size[i] = int(b)
        elif k == "upsampfac":
            o.upsampfac = float(v)
        else:
            setattr(o, k, int(v))
    return o


def opts_dict(o: nufft_opts) -> dict:
    """The tunable fields of an options struct, as keyword arguments for Plan / BatchPlan."""
    return {"bin_size": tuple(o.bin_size), "max_subprob": o.max_subprob, "threads": o.threads,
            "sparse_max": o.sparse_max, "kerevalmeth": o.kerevalmeth, "kernel": o.kernel, "upsampfac": o.upsampfac}


# --------------------------------------------------------------- torch layer
class Plan:
    """A type-1 or type-2 plan on one CUDA device, driven with torch tensors.

    type 1: ``execute(c)`` with c of shape (M,) or (ntransf, M) returns f of
    shape (ntransf, N_d, ..., N_1) (dimension 1 fastest).  type 2:
    ``execute(f)`` returns c of shape (ntransf, M).  CPU tensors are copied to
    the device and the result copied back (the end-to-end path).
    """

    def __init__(self, nufft_type: int, n_modes, eps: float = 1e-6, isign: int | None = None,
                 n_trans: int = 1, dtype=None, device=None, stream=None, **opts):
        import torch
        self._torch = torch
        self.type = int(nufft_type)
        self.n_modes = tuple(int(v) for v in n_modes)
        self.dim = len(self.n_modes)
        self.isign = int(isign) if isign is not None else (1 if self.type == 1 else -1)
        self.n_trans = int(n_trans)
        self.dtype = dtype if dtype is not None else torch.complex64
        if self.dtype not in (torch.complex64, torch.complex128):
            raise ValueError("dtype must be complex64 or complex128")
        self.real_dtype = torch.float32 if self.dtype == torch.complex64 else torch.float64
        self.prec = NUFFT_C64 if self.dtype == torch.complex64 else NUFFT_C128
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.type != "cuda":
            raise ValueError("Plan needs a CUDA device")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            o = nufft_default_opts()
            for k, v in opts.items():
                if k == "bin_size":
                    for i, b in enumerate(v):
                        o.bin_size[i] = int(b)
                elif k == "upsampfac":
                    o.upsampfac = float(v)
                else:
                    setattr(o, k, int(v))
            self._h = None
            st, h = nufft_makeplan(self.type, self.dim, self.n_modes, self.isign, self.n_trans, eps, self.prec,
                                   self.stream.cuda_stream, o)
            if st < 0:
                raise NufftError(st, "nufft_makeplan")
            self.warning = st
            self._h = h
        self.M = None
        self._keep = ()
        st, self.info = nufft_plan_info(self._h, self.dim)

    # -- points
    def setpts(self, x, y=None, z=None):
        torch = self._torch
        coords = [x, y, z][: self.dim]
        if any(v is None for v in coords):
            raise ValueError("need %d coordinate arrays" % self.dim)
        dev = []
        for v in coords:
            v = torch.as_tensor(v)
            v = v.to(device=self.device, dtype=self.real_dtype, non_blocking=True).contiguous()
            dev.append(v)
        M = dev[0].numel()
        if any(v.numel() != M for v in dev):
            raise ValueError("coordinate arrays differ in length")
        ptrs = [v.data_ptr() for v in dev] + [0] * (3 - self.dim)
        with torch.cuda.device(self.device), torch.cuda.stream(self.stream):
            st = nufft_setpts(self._h, M, *ptrs)
        if st < 0:
            raise NufftError(st, "nufft_setpts")
        self.M = M
        self._keep = tuple(dev)
        return self

    def setpts_from(self, other: "Plan"):
        """Use the points ``other`` has binned (nufft_setpts_from): no second binning.  This
        plan's stream waits for ``other``'s, where the binning was enqueued."""
        torch = self._torch
        if self.stream != other.stream:
            self.stream.wait_stream(other.stream)
        st = nufft_setpts_from(self._h, other._h)
        if st < 0:
            raise NufftError(st, "nufft_setpts_from")
        self.M = other.M
        self._keep = other._keep
        return self

    # -- transform
    def execute(self, data, out=None):
        torch = self._torch
        if self.M is None:
            raise NufftError(-6, "Plan.execute")
        host = isinstance(data, torch.Tensor) and data.device.type == "cpu"
        d = torch.as_tensor(data).to(device=self.device, dtype=self.dtype, non_blocking=True).contiguous()
        nt = self.n_trans
        Nt = 1
        for v in self.n_modes:
            Nt *= v
        if self.type == 1:
            if d.numel() != nt * self.M:
                raise ValueError("expected %d strengths" % (nt * self.M))
            shape = (nt,) + tuple(reversed(self.n_modes))
            res = out if out is not None else torch.empty(shape, dtype=self.dtype, device=self.device)
            c_ptr, f_ptr = d.data_ptr(), res.data_ptr()
        else:
            if d.numel() != nt * Nt:
                raise ValueError("expected %d coefficients" % (nt * Nt))
            res = out if out is not None else torch.empty((nt, self.M), dtype=self.dtype, device=self.device)
            c_ptr, f_ptr = res.data_ptr(), d.data_ptr()
        if not res.is_contiguous() or res.device != self.device or res.dtype != self.dtype:
            raise ValueError("out must be a contiguous %s tensor on %s" % (self.dtype, self.device))
        with torch.cuda.device(self.device), torch.cuda.stream(self.stream):
            st = nufft_execute(self._h, c_ptr, f_ptr)
        if st < 0:
            raise NufftError(st, "nufft_execute")
        self._keep_exec = (d,)
        if host:
            return res.to("cpu")
        return res

    def execute_grad(self, f, out=None, dout=None):
        """Type-2 plans: (c, dc) with c of shape (ntransf, M) and dc of shape
        (ntransf, dim, M), dc[t, d, j] = d c[t, j] / d x_{j,d} through the
        derivative of the ES kernel."""
        torch = self._torch
        if self.type != 2:
            raise ValueError("execute_grad needs a type-2 plan")
        if self.M is None:
            raise NufftError(-6, "Plan.execute_grad")
        d = torch.as_tensor(f).to(device=self.device, dtype=self.dtype, non_blocking=True).contiguous()
        Nt = 1
        for v in self.n_modes:
            Nt *= v
        if d.numel() != self.n_trans * Nt:
            raise ValueError("expected %d coefficients" % (self.n_trans * Nt))
        res = out if out is not None else torch.empty((self.n_trans, self.M), dtype=self.dtype, device=self.device)
        dres = dout if dout is not None else torch.empty((self.n_trans, self.dim, self.M), dtype=self.dtype,
                                                         device=self.device)
        for t in (res, dres):
            if not t.is_contiguous() or t.device != self.device or t.dtype != self.dtype:
                raise ValueError("outputs must be contiguous %s tensors on %s" % (self.dtype, self.device))
        with torch.cuda.device(self.device), torch.cuda.stream(self.stream):
            st = nufft_execute_grad(self._h, res.data_ptr(), dres.data_ptr(), d.data_ptr())
        if st < 0:
            raise NufftError(st, "nufft_execute_grad")
        self._keep_exec = (d,)
        return res, dres

    def status(self) -> int:
        return nufft_get_status(self._h)

    def timings(self):
        return nufft_get_timings(self._h)[1]

    def nsub(self) -> int:
        return nufft_plan_info(self._h, self.dim)[1]["nsub"]

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            nufft_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan3:
    """A type-3 plan (Eq. (3)) on one CUDA device, driven with torch tensors.

    ``setpts(x, s)`` takes the sources x and target frequencies s as sequences
    of dim coordinate arrays (M and N reals each); ``execute(c)`` with c of
    shape (M,) returns f of shape (N,), f_k = sum_j c_j exp(i isign s_k.x_j).
    CPU tensors are copied to the device and the result copied back.
    """

    def __init__(self, dim: int, eps: float = 1e-6, isign: int = 1, dtype=None, device=None, stream=None, **opts):
        import torch
        self._torch = torch
        self.dim = int(dim)
        self.isign = int(isign)
        self.dtype = dtype if dtype is not None else torch.complex64
        if self.dtype not in (torch.complex64, torch.complex128):
            raise ValueError("dtype must be complex64 or complex128")
        self.real_dtype = torch.float32 if self.dtype == torch.complex64 else torch.float64
        self.prec = NUFFT_C64 if self.dtype == torch.complex64 else NUFFT_C128
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.type != "cuda":
            raise ValueError("Plan3 needs a CUDA device")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self._h = None
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            st, h = nufft3_makeplan(self.dim, self.isign, eps, self.prec, self.stream.cuda_stream, _make_opts(opts))
            if st < 0:
                raise NufftError(st, "nufft3_makeplan")
            self.warning = st
            self._h = h
        self.M = self.N = None
        self._keep = ()
        self.info = None

    def _dev(self, coords, what):
        torch = self._torch
        coords = list(coords)
        if len(coords) != self.dim:
            raise ValueError("need %d %s coordinate arrays" % (self.dim, what))
        dev = [torch.as_tensor(v).to(device=self.device, dtype=self.real_dtype, non_blocking=True).contiguous()
               for v in coords]
        n = dev[0].numel()
        if any(v.numel() != n for v in dev):
            raise ValueError("%s coordinate arrays differ in length" % what)
        return dev, n

    def setpts(self, x, s):
        torch = self._torch
        xd, M = self._dev(x, "source")
        sd, N = self._dev(s, "target")
        px = [v.data_ptr() for v in xd] + [0] * (3 - self.dim)
        ps = [v.data_ptr() for v in sd] + [0] * (3 - self.dim)
        with torch.cuda.device(self.device), torch.cuda.stream(self.stream):
            st = nufft3_setpts(self._h, M, *px, N, *ps)
        if st < 0:
            raise NufftError(st, "nufft3_setpts")
        self.M, self.N = M, N
        self._keep = tuple(xd + sd)
        self.info = nufft3_plan_info(self._h, self.dim)[1]
        return self

    def execute(self, c, out=None):
        torch = self._torch
        if self.M is None:
            raise NufftError(-6, "Plan3.execute")
        host = isinstance(c, torch.Tensor) and c.device.type == "cpu"
        d = torch.as_tensor(c).to(device=self.device, dtype=self.dtype, non_blocking=True).contiguous()
        if d.numel() != self.M:
            raise ValueError("expected %d strengths" % self.M)
        res = out if out is not None else torch.empty((self.N,), dtype=self.dtype, device=self.device)
        if not res.is_contiguous() or res.device != self.device or res.dtype != self.dtype or res.numel() != self.N:
            raise ValueError("out must be a contiguous %s tensor of %d values on %s" % (self.dtype, self.N,
                                                                                        self.device))
        with torch.cuda.device(self.device), torch.cuda.stream(self.stream):
            st = nufft3_execute(self._h, d.data_ptr(), res.data_ptr())
        if st < 0:
            raise NufftError(st, "nufft3_execute")
        self._keep_exec = (d,)
        return res.to("cpu") if host else res

    def status(self) -> int:
        return nufft3_get_status(self._h)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            nufft3_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchPlan:
    """B independent transforms of one type / dimension / precision / eps with their own
    mode counts, run as one launch per step (replayed from a CUDA graph).

    ``setpts(x, y, z, offsets)``: concatenated coordinates, transform t owning
    points offsets[t]..offsets[t+1]-1.  type 1: ``execute(c)`` returns all mode
    arrays concatenated (``mode_offsets`` gives each start); type 2:
    ``execute(f)`` with the concatenated mode arrays returns the concatenated
    values at the points.
    """

    def __init__(self, nufft_type: int, modes, eps: float = 1e-6, isign: int | None = None, dtype=None,
                 device=None, stream=None, **opts):
        import torch
        self._torch = torch
        self.type = int(nufft_type)
        self.modes = [tuple(int(v) for v in m) for m in modes]
        self.B = len(self.modes)
        self.dim = len(self.modes[0])
        if any(len(m) != self.dim for m in self.modes):
            raise ValueError("all transforms need the same dimension")
        self.isign = int(isign) if isign is not None else (1 if self.type == 1 else -1)
        self.dtype = dtype if dtype is not None else torch.complex64
        self.real_dtype = torch.float32 if self.dtype == torch.complex64 else torch.float64
        prec = NUFFT_C64 if self.dtype == torch.complex64 else NUFFT_C128
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.mode_offsets = [0]
        for m in self.modes:
            n = 1
            for v in m:
                n *= v
            self.mode_offsets.append(self.mode_offsets[-1] + n)
        self._h = None
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            o = nufft_default_opts()
            for k, v in opts.items():
                if k == "bin_size":
                    for i, b in enumerate(v):
                        o.bin_size[i] = int(b)
                elif k == "upsampfac":
                    o.upsampfac = float(v)
                else:
                    setattr(o, k, int(v))
            st, h = nufft_batch_makeplan(self.type, self.dim, self.modes, self.isign, eps, prec,
                                         self.stream.cuda_stream, o)
            if st < 0:
                raise NufftError(st, "nufft_batch_makeplan")
            self._h = h
        self.M = None

    def setpts(self, x, y=None, z=None, offsets=None):
        torch = self._torch
        coords = [x, y, z][: self.dim]
        dev = [torch.as_tensor(v).to(device=self.device, dtype=self.real_dtype, non_blocking=True).contiguous()
               for v in coords]
        M = dev[0].numel()
        if offsets is None or len(offsets) != self.B + 1 or int(offsets[-1]) != M:
            raise ValueError("offsets must have B + 1 entries ending at the number of points")
        ptrs = [v.data_ptr() for v in dev] + [0] * (3 - self.dim)
        with torch.cuda.device(self.device), torch.cuda.stream(self.stream):
            st = nufft_batch_setpts(self._h, [int(v) for v in offsets], *ptrs)
        if st < 0:
            raise NufftError(st, "nufft_batch_setpts")
        self.M = M
        self._keep = tuple(dev)
        return self

    def execute(self, data, out=None):
        torch = self._torch
        if self.M is None:
            raise NufftError(-6, "BatchPlan.execute")
        d = torch.as_tensor(data).to(device=self.device, dtype=self.dtype, non_blocking=True).contiguous()
        if self.type == 1:
            if d.numel() != self.M:
                raise ValueError("expected %d strengths" % self.M)
            res = out if out is not None else torch.empty(self.mode_offsets[-1], dtype=self.dtype, device=self.device)
            c_ptr, f_ptr = d.data_ptr(), res.data_ptr()
        else:
            if d.numel() != self.mode_offsets[-1]:
                raise ValueError("expected %d coefficients" % self.mode_offsets[-1])
            res = out if out is not None else torch.empty(self.M, dtype=self.dtype, device=self.device)
            c_ptr, f_ptr = res.data_ptr(), d.data_ptr()
        with torch.cuda.device(self.device), torch.cuda.stream(self.stream):
            st = nufft_batch_execute(self._h, c_ptr, f_ptr)
        if st < 0:
            raise NufftError(st, "nufft_batch_execute")
        self._keep_exec = (d, res)
        return res

    def status(self) -> int:
        return nufft_batch_get_status(self._h)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            nufft_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tune_plan(nufft_type: int, n_modes, x, data, eps: float = 1e-6, isign: int | None = None, dtype=None,
              device=None, reps: int = 3):
    """Autotune a plan on these points and this input (nufft_tune).  x: list of d
    coordinate tensors; data: c (type 1) or f (type 2).  Returns (options for
    Plan(**opts), best ms, default ms) for one setpts + execute."""
    import torch
    dtype = dtype if dtype is not None else torch.complex64
    dev = torch.device(device if device is not None else "cuda")
    if dev.index is None:
        dev = torch.device("cuda", torch.cuda.current_device())
    rdt = torch.float32 if dtype == torch.complex64 else torch.float64
    prec = NUFFT_C64 if dtype == torch.complex64 else NUFFT_C128
    isign = int(isign) if isign is not None else (1 if nufft_type == 1 else -1)
    xs = [torch.as_tensor(v).to(device=dev, dtype=rdt).contiguous() for v in x]
    d = torch.as_tensor(data).to(device=dev, dtype=dtype).contiguous()
    M = xs[0].numel()
    Nt = 1
    for v in n_modes:
        Nt *= int(v)
    out = torch.empty(Nt if nufft_type == 1 else M, dtype=dtype, device=dev)
    ptrs = [v.data_ptr() for v in xs] + [0] * (3 - len(xs))
    with torch.cuda.device(dev):
        st, o, best, default = nufft_tune(nufft_type, len(xs), n_modes, isign, eps, prec, M, *ptrs, d.data_ptr(),
                                          out.data_ptr(), torch.cuda.current_stream(dev).cuda_stream, reps)
    if st < 0:
        raise NufftError(st, "nufft_tune")
    return opts_dict(o), best, default


def tune_batch(nufft_type: int, modes, x, data, offsets, eps: float = 1e-6, isign: int | None = None, dtype=None,
               device=None, reps: int = 3):
    """Autotune a BatchPlan (nufft_batch_tune); arguments as BatchPlan.setpts / execute.
    Returns (options for BatchPlan(**opts), best ms, default ms)."""
    import torch
    dtype = dtype if dtype is not None else torch.complex64
    dev = torch.device(device if device is not None else "cuda")
    if dev.index is None:
        dev = torch.device("cuda", torch.cuda.current_device())
    rdt = torch.float32 if dtype == torch.complex64 else torch.float64
    prec = NUFFT_C64 if dtype == torch.complex64 else NUFFT_C128
    isign = int(isign) if isign is not None else (1 if nufft_type == 1 else -1)
    xs = [torch.as_tensor(v).to(device=dev, dtype=rdt).contiguous() for v in x]
    d = torch.as_tensor(data).to(device=dev, dtype=dtype).contiguous()
    M = xs[0].numel()
    total_modes = 0
    for m in modes:
        t = 1
        for v in m:
            t *= int(v)
        total_modes += t
    out = torch.empty(total_modes if nufft_type == 1 else M, dtype=dtype, device=dev)
    ptrs = [v.data_ptr() for v in xs] + [0] * (3 - len(xs))
    with torch.cuda.device(dev):
        st, o, best, default = nufft_batch_tune(nufft_type, len(xs), modes, isign, eps, prec, offsets, *ptrs,
                                                d.data_ptr(), out.data_ptr(),
                                                torch.cuda.current_stream(dev).cuda_stream, reps)
    if st < 0:
        raise NufftError(st, "nufft_batch_tune")
    return opts_dict(o), best, default
