"""CPU oracle for the type-1 / type-2 ES-kernel NUFFT (arXiv:1808.06736).

TEST INFRASTRUCTURE ONLY.  The product path (the CUDA library and its Python
binding) never imports, loads or calls this package.  Only the tests, the
smoke check and the CPU-baseline leg of the benchmark use it.  It shares no
code with the CUDA path; the two meet only through the seeded input
generators in ``nufft_inputs.py``, which hold none of the method's arithmetic.

Two levels, both in IEEE double precision:

* O1 -- direct evaluation of the exponential sums Eq. (1) (type 1) and
  Eq. (2) (type 2), in ``nufft_oracle.c``.
* O2 -- the paper's three-step algorithm written plainly: parameters by
  Eq. (params) and Sec. 3.1 (fine grid size), spreading Eq. (bl) /
  interpolation Eq. (interp) as direct loops (C), the n-point DFT Eq. (dft1) /
  Eq. (dft) with scipy's FFT, and the correction Eq. (pk) with the kernel
  transform from the Gauss-Legendre rule Eq. (quad).

Also: the piecewise polynomial kernel of Sec. 5.3 (``piecewise_poly``,
``piecewise_eval``) by the paper's own fitting method, and the type-3 sum and
algorithm (``direct_type3``, ``type3``, Sec. 3.3).

Readings of the paper that these functions fix (where it is silent or
inconsistent):

* mode arrays run over increasing k in every dimension, dimension 1 fastest;
* both types compute sums with exp(+i isign k.x); the type-2 DFT uses the
  same sign as the transform (Eq. (dft) prints "+", which only holds for
  isign = +1);
* w = ceil(log10(1/eps) - 1e-9) + 1, clamped to [2, 16] (the guard keeps
  eps = 1e-5 at w = 6 against rounding in log10; the clamp is beta <= 36,
  Sec. 3.3);
* the w nodes of a coordinate start at ceil(u - w/2), u = x / h;
* p = ceil(1.5 w + 2) positive Gauss-Legendre nodes (Sec. 3.1.1).

Parity pins for every function live in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nufft_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``nufft_oracle.c`` into ``liboracle.so`` with gcc (IEEE math, OpenMP)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int64)
        i64 = ctypes.c_int64
        lib.oracle_type1_direct.argtypes = [ctypes.c_int, i64, dp, dp, dp, dp, ctypes.c_int, i64, ip, dp]
        lib.oracle_type2_direct.argtypes = [ctypes.c_int, i64, dp, dp, dp, ip, dp, ctypes.c_int, dp]
        lib.oracle_type3_direct.argtypes = [ctypes.c_int, i64, dp, dp, dp, dp, ctypes.c_int, i64, dp, dp, dp, dp]
        lib.oracle_spread.argtypes = [ctypes.c_int, i64, dp, dp, dp, dp, ip, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_int, dp]
        lib.oracle_interp.argtypes = [ctypes.c_int, i64, dp, dp, dp, dp, ip, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_int, dp]
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
        lib.oracle_set_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def num_threads() -> int:
    """OpenMP threads the direct sums, spreading and interpolation use."""
    return int(_L().oracle_num_threads())


def set_num_threads(n: int) -> int:
    """Use n OpenMP threads from now on; returns the number in effect."""
    return int(_L().oracle_set_num_threads(int(n)))


# ----------------------------------------------------------------- helpers
def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _coords(xs):
    """List of d float64 contiguous coordinate arrays (+ padding for the C ABI)."""
    xs = [np.ascontiguousarray(np.asarray(v, dtype=np.float64)) for v in xs]
    d = len(xs)
    assert 1 <= d <= 3
    dummy = np.zeros(1)
    full = xs + [dummy] * (3 - d)
    return d, xs, full


def _cplx(a) -> np.ndarray:
    """complex128 contiguous copy viewed as interleaved float64."""
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def mode_range(N: int) -> np.ndarray:
    """The index set I_N of Sec. 1: -N/2..N/2-1 (N even), -(N-1)/2..(N-1)/2 (N odd)."""
    return np.arange(N, dtype=np.int64) - (N // 2)


def mode_list(Ns) -> np.ndarray:
    """All k in I_{N_1} x ... x I_{N_d} as an (N, d) int64 array, dimension 1 fastest."""
    grids = np.meshgrid(*[mode_range(n) for n in reversed(Ns)], indexing="ij")
    return np.stack([g.ravel() for g in reversed(grids)], axis=1).astype(np.int64)


def mode_index(k: np.ndarray, Ns) -> np.ndarray:
    """Flat position of mode vectors k (m x d) in a mode array (dimension 1 fastest)."""
    idx = np.zeros(k.shape[0], dtype=np.int64)
    stride = 1
    for i, n in enumerate(Ns):
        idx += (k[:, i] + n // 2) * stride
        stride *= n
    return idx


def rel_l2(a, b) -> float:
    """Relative l2 error ||a - b|| / ||b|| (Sec. 4.2's epsilon)."""
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a - b))


# --------------------------------------------------------------- O1 (truth)
def direct_type1(xs, c, isign: int, Ns, modes: np.ndarray | None = None) -> np.ndarray:
    """Eq. (1): f_k = sum_j c_j exp(i isign k.x_j), for all k in I_N or the given (m, d) modes."""
    d, xs, full = _coords(xs)
    c = _cplx(c)
    M = c.shape[0]
    k = mode_list(Ns) if modes is None else np.ascontiguousarray(modes, dtype=np.int64)
    assert k.shape[1] == d
    f = np.zeros(k.shape[0], dtype=np.complex128)
    _L().oracle_type1_direct(d, M, _dptr(full[0]), _dptr(full[1]), _dptr(full[2]),
                             _dptr(c.view(np.float64)), int(isign), k.shape[0], _iptr(k),
                             _dptr(f.view(np.float64)))
    return f


def direct_type2(xs, f, isign: int, Ns) -> np.ndarray:
    """Eq. (2) with the interface sign: c_j = sum_{k in I_N} f_k exp(i isign k.x_j)."""
    d, xs, full = _coords(xs)
    f = _cplx(f).ravel()
    N = np.ascontiguousarray(Ns, dtype=np.int64)
    assert f.shape[0] == int(np.prod(N))
    nt = xs[0].shape[0]
    c = np.zeros(nt, dtype=np.complex128)
    _L().oracle_type2_direct(d, nt, _dptr(full[0]), _dptr(full[1]), _dptr(full[2]), _iptr(N),
                             _dptr(f.view(np.float64)), int(isign), _dptr(c.view(np.float64)))
    return c


def direct_type3(xs, c, isign: int, ss) -> np.ndarray:
    """Eq. (3): f_k = sum_j c_j exp(i isign s_k . x_j) for real frequencies ss (one array per dimension)."""
    d, xs, full = _coords(xs)
    _, ss, sfull = _coords(ss)
    c = _cplx(c)
    nt = ss[0].shape[0]
    f = np.zeros(nt, dtype=np.complex128)
    _L().oracle_type3_direct(d, c.shape[0], _dptr(full[0]), _dptr(full[1]), _dptr(full[2]),
                             _dptr(c.view(np.float64)), int(isign), nt, _dptr(sfull[0]), _dptr(sfull[1]),
                             _dptr(sfull[2]), _dptr(f.view(np.float64)))
    return f


# ---------------------------------------------------------- parameters (a0)
def next235(m: int) -> int:
    """Smallest integer of the form 2^q 3^p 5^r that is >= m (Sec. 3.1.1)."""
    m = max(int(m), 1)
    n = m
    while True:
        r = n
        for p in (2, 3, 5):
            while r % p == 0:
                r //= p
        if r == 1:
            return n
        n += 1


GAMMA = 0.976            # Eq. (gam)'s safety factor that gives beta = 2.30 w at sigma = 2 (Sec. 4.3)
SIGMA_54_OFFSET = 0.43   # reading: the paper gives no w rule for sigma = 5/4; offset calibrated on O2


def eserr_slope(sigma: float, gamma: float = GAMMA) -> float:
    """w per decade of 1/eps from Eq. (ESerr) with its algebraic prefactor dropped (Sec. 4.3):
    ln(10) / (pi gamma sqrt(1 - 1/sigma - (gamma^-2 - 1) / (4 sigma^2)))."""
    return math.log(10.0) / (math.pi * gamma * math.sqrt(1.0 - 1.0 / sigma - (gamma ** -2 - 1.0) / (4.0 * sigma ** 2)))


def kernel_width(eps: float, sigma: float = 2.0) -> int:
    """sigma = 2, Eq. (params): w = ceil(log10(1/eps)) + 1, with the guard and clamp read in the
    module docstring.  sigma = 5/4: w = ceil(slope log10(1/eps) + offset), slope from Eq. (ESerr)."""
    if sigma == 2.0:
        w = int(math.ceil(math.log10(1.0 / eps) - 1e-9)) + 1
    else:
        w = int(math.ceil(eserr_slope(sigma) * math.log10(1.0 / eps) + SIGMA_54_OFFSET - 1e-9))
    return min(max(w, 2), 16)


def es_beta(w: int, sigma: float = 2.0) -> float:
    """Eq. (params): beta = 2.30 w at sigma = 2; otherwise Eq. (gam): gamma pi w (1 - 1/(2 sigma))."""
    if sigma == 2.0:
        return 2.30 * w
    return GAMMA * math.pi * w * (1.0 - 1.0 / (2.0 * sigma))


def fine_grid_size(N: int, w: int, sigma: float = 2.0) -> int:
    """Sec. 3.1.1: smallest 2^q 3^p 5^r not less than sigma N nor 2w."""
    return next235(max(int(math.ceil(sigma * N)), 2 * w))


def choose_params(eps: float, Ns, sigma: float = 2.0):
    """(w, beta, [n_1..n_d]) for tolerance eps and mode counts Ns (Sec. 3, Eq. (params))."""
    w = kernel_width(eps, sigma)
    return w, es_beta(w, sigma), [fine_grid_size(n, w, sigma) for n in Ns]


# --------------------------------------------------- kernel and its transform
KERNELS = {"es": 0, "cosh": 1}


def es_cosh_kernel(z, beta: float):
    """The smooth variant of the Remark in Sec. 7: 2 exp(-beta) cosh(beta sqrt(1 - z^2)) on
    |z| <= 1, zero outside (within exp(-beta) of Eq. (ES), with bounded derivatives)."""
    z = np.asarray(z, dtype=np.float64)
    out = np.zeros_like(z)
    m = np.abs(z) <= 1.0
    out[m] = 2.0 * np.exp(-beta) * np.cosh(beta * np.sqrt(1.0 - z[m] ** 2))
    return out


def kernel_fn(kernel: str, beta: float):
    """phi as a function of z for kernel 'es' (Eq. (ES)) or 'cosh' (Remark in Sec. 7)."""
    if kernel == "es":
        return lambda z: es_kernel(z, beta)
    if kernel == "cosh":
        return lambda z: es_cosh_kernel(z, beta)
    raise ValueError(kernel)


def es_kernel(z, beta: float):
    """Eq. (ES): exp(beta (sqrt(1 - z^2) - 1)) on |z| <= 1, zero outside."""
    z = np.asarray(z, dtype=np.float64)
    out = np.zeros_like(z)
    m = np.abs(z) <= 1.0
    out[m] = np.exp(beta * (np.sqrt(1.0 - z[m] ** 2) - 1.0))
    return out


def piecewise_poly(w: int, beta: float, p: int | None = None, kernel=None) -> np.ndarray:
    """Sec. 5.3: the kernel psi on its support of w fine-grid cells is split into w unit
    intervals, and on interval t (cell offsets tau in [t - w/2, t - w/2 + 1]) approximated by a
    polynomial of degree p = w + 3 in the centred variable s = 2 (tau - (t - w/2)) - 1 in [-1, 1].
    Monomial coefficients by a least-squares Vandermonde solve at collocation points on the
    boundary of the square with corners +-1 +- i in the complex s-plane (the square tightly
    enclosing the interval), with the kernel continued to complex arguments (principal square
    root).  Returns a (w, p + 1) array, row t holding the coefficients of s^0 .. s^p.

    ``kernel`` (a function of complex z = 2 tau / w) replaces the ES kernel, so the tests can
    fit a function with a known polynomial form."""
    p = w + 3 if p is None else int(p)
    K = 2 * (p + 1)                                   # points per side
    u = (np.arange(K) + 0.5) / K * 2.0 - 1.0
    pts = np.concatenate([u - 1j, 1.0 + 1j * u, -u + 1j, -1.0 - 1j * u])
    V = pts[:, None] ** np.arange(p + 1)
    if kernel is None:
        kernel = lambda z: np.exp(beta * (np.sqrt(1.0 - z * z + 0j) - 1.0))  # noqa: E731
    C = np.empty((w, p + 1))
    for t in range(w):
        z = (t - w / 2.0 + 0.5 + 0.5 * pts) * (2.0 / w)
        a = np.linalg.lstsq(V, kernel(z), rcond=None)[0]
        C[t] = a.real
    return C


def piecewise_eval(C: np.ndarray, w: int, z) -> np.ndarray:
    """The piecewise polynomial of ``piecewise_poly`` at real z in [-1, 1] (z = 2 tau / w), zero
    outside: interval t = floor(tau + w/2), s = 2 (tau + w/2 - t) - 1, Horner's scheme."""
    z = np.asarray(z, dtype=np.float64)
    tau = z * (w / 2.0)
    t = np.clip(np.floor(tau + w / 2.0).astype(np.int64), 0, w - 1)
    s = 2.0 * (tau + w / 2.0 - t) - 1.0
    y = np.zeros_like(z)
    for m in range(C.shape[1] - 1, -1, -1):
        y = y * s + C[t, m]
    return np.where(np.abs(z) <= 1.0, y, 0.0)


def gl_quadrature_nodes(w: int):
    """Positive nodes and weights of the 2p-point Gauss-Legendre rule, p = ceil(1.5 w + 2) (Sec. 3.1.1)."""
    p = int(math.ceil(1.5 * w + 2))
    q, wq = np.polynomial.legendre.leggauss(2 * p)
    keep = q > 0
    return q[keep], wq[keep]


def kernel_ft(xi, w: int, beta: float, kernel=None):
    """phi^(xi) = int_{-1}^{1} phi(z) e^{i xi z} dz by Eq. (quad)'s rule: 2 sum_j w_j phi(q_j) cos(xi q_j).

    ``kernel`` (a function of z) replaces the ES kernel, which lets the tests
    push a kernel with a known transform through the same rule.
    """
    q, wq = gl_quadrature_nodes(w)
    phi = es_kernel(q, beta) if kernel is None else kernel(q)
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    return 2.0 * (np.cos(np.outer(xi, q)) @ (wq * phi))


def correction_factors(N: int, n: int, w: int, beta: float, kernel: str = "es") -> np.ndarray:
    """Eq. (pk1): p_k = h / psi^(k) = 2 / (w phi^(alpha k)), alpha = pi w / n (Eq. (al)), k in I_N."""
    alpha = math.pi * w / n
    return 2.0 / (w * kernel_ft(alpha * mode_range(N), w, beta, kernel=kernel_fn(kernel, beta)))


# ------------------------------------------------------------- O2 pieces
def spread(xs, c, ns, w: int, beta: float, kernel: str = "es") -> np.ndarray:
    """Eq. (bl): fine-grid values b_l (complex, shape (n_d, ..., n_1))."""
    d, xs, full = _coords(xs)
    c = _cplx(c)
    n = np.ascontiguousarray(ns, dtype=np.int64)
    b = np.zeros(int(np.prod(n)), dtype=np.complex128)
    _L().oracle_spread(d, c.shape[0], _dptr(full[0]), _dptr(full[1]), _dptr(full[2]),
                       _dptr(c.view(np.float64)), _iptr(n), int(w), float(beta), KERNELS[kernel],
                       _dptr(b.view(np.float64)))
    return b.reshape(tuple(reversed([int(v) for v in ns])))


def interp(xs, b, ns, w: int, beta: float, kernel: str = "es") -> np.ndarray:
    """Eq. (interp): c_j = sum_l b_l psi~(l h - x_j)."""
    d, xs, full = _coords(xs)
    b = _cplx(b).ravel()
    n = np.ascontiguousarray(ns, dtype=np.int64)
    M = xs[0].shape[0]
    c = np.zeros(M, dtype=np.complex128)
    _L().oracle_interp(d, M, _dptr(full[0]), _dptr(full[1]), _dptr(full[2]),
                       _dptr(b.view(np.float64)), _iptr(n), int(w), float(beta), KERNELS[kernel],
                       _dptr(c.view(np.float64)))
    return c


def _workers() -> int:
    return max(1, len(os.sched_getaffinity(0)))


def dft(b: np.ndarray, isign: int) -> np.ndarray:
    """Eq. (dft1) / Eq. (dft): sum_l exp(isign 2 pi i l.k / n) b_l over all axes (unnormalised)."""
    import scipy.fft as sfft
    if isign > 0:
        return sfft.ifftn(b, norm="forward", workers=_workers())
    return sfft.fftn(b, workers=_workers())


def _truncation_index(Ns, ns):
    """Fine-grid positions k mod n of the modes k in I_N, per axis in array order (slowest first)."""
    return np.ix_(*[np.mod(mode_range(N), n) for N, n in zip(reversed(Ns), reversed(ns))])


def _outer_correction(Ns, ns, w, beta, kernel="es"):
    """Eq. (pk): the separable p_k as an array of shape (N_d, ..., N_1)."""
    p = None
    for N, n in zip(reversed(Ns), reversed(ns)):
        pk = correction_factors(N, n, w, beta, kernel)
        p = pk if p is None else np.multiply.outer(p, pk)
    return p


def deconvolve(bh: np.ndarray, Ns, ns, w: int, beta: float, kernel: str = "es") -> np.ndarray:
    """Type-1 step 3, Eq. (pb1) with Eq. (pk): f_k = p_k b^_{k mod n} for k in I_N (mode order)."""
    return (bh[_truncation_index(Ns, ns)] * _outer_correction(Ns, ns, w, beta, kernel)).ravel()


def precorrect(f, Ns, ns, w: int, beta: float, kernel: str = "es") -> np.ndarray:
    """Type-2 step 1 (Sec. 3.2): b^_{k mod n} = p_k f_k on I_N, zero elsewhere on the fine grid."""
    f = _cplx(f).reshape(tuple(reversed([int(v) for v in Ns])))
    bh = np.zeros(tuple(reversed([int(v) for v in ns])), dtype=np.complex128)
    bh[_truncation_index(Ns, ns)] = f * _outer_correction(Ns, ns, w, beta, kernel)
    return bh


def type1(xs, c, isign: int, Ns, eps: float | None = None, w: int | None = None,
          beta: float | None = None, ns=None, kernel: str = "es") -> np.ndarray:
    """O2 type 1 (Sec. 3.1): spread Eq. (bl), DFT Eq. (dft1) with sign isign, truncate and
    correct Eq. (pb1)/(pk).  Parameters from eps unless (w, beta, ns) are given; kernel 'es'
    (Eq. (ES)) or 'cosh' (Remark in Sec. 7, same w and beta)."""
    Ns = [int(v) for v in Ns]
    if w is None:
        w, beta, ns = choose_params(eps, Ns)
    b = spread(xs, c, ns, w, beta, kernel)
    return deconvolve(dft(b, isign), Ns, ns, w, beta, kernel)


def type2(xs, f, isign: int, Ns, eps: float | None = None, w: int | None = None,
          beta: float | None = None, ns=None, kernel: str = "es") -> np.ndarray:
    """O2 type 2 (Sec. 3.2): pre-correct and zero-pad, DFT Eq. (dft) with sign isign,
    interpolate Eq. (interp)."""
    Ns = [int(v) for v in Ns]
    if w is None:
        w, beta, ns = choose_params(eps, Ns)
    b = dft(precorrect(f, Ns, ns, w, beta, kernel), isign)
    return interp(xs, b, ns, w, beta, kernel)


# ------------------------------------------------------------- O2 type 3
def type3_params(eps: float, xs, ss, sigma: float = 2.0):
    """Sec. 3.3, step 0: centres x0, s0 (midpoints of the bounding boxes; the translation of
    Eq. (trans) is always applied), half-widths X_i, S_i (Eq. (XS) after centring), fine grid
    n_i = next235(max(2 sigma X_i S_i / pi + w, 2 w)) and dilation gamma_i = n_i / (2 sigma S_i)
    (Eq. (ng)); a dimension with S_i = 0 takes the smallest gamma_i that keeps
    X_i / gamma_i <= pi (1 - w / n_i) (Eq. (cond1)), or 1."""
    w = kernel_width(eps, sigma)
    beta = es_beta(w, sigma)
    x0, s0, X, S, ns, gam = [], [], [], [], [], []
    for xv, sv in zip(xs, ss):
        xv = np.asarray(xv, dtype=np.float64)
        sv = np.asarray(sv, dtype=np.float64)
        xa, xb = float(xv.min()), float(xv.max())
        sa, sb = float(sv.min()), float(sv.max())
        x0.append(0.5 * (xa + xb))
        s0.append(0.5 * (sa + sb))
        Xi, Si = 0.5 * (xb - xa), 0.5 * (sb - sa)
        n = next235(max(int(math.ceil(2.0 * sigma / math.pi * Xi * Si + w)), 2 * w))
        if Si > 0:
            g = n / (2.0 * sigma * Si)
        else:
            g = Xi / (math.pi * (1.0 - w / n)) if Xi > 0 else 1.0
        X.append(Xi)
        S.append(Si)
        ns.append(n)
        gam.append(g)
    return dict(w=w, beta=beta, x0=x0, s0=s0, X=X, S=S, ns=ns, gamma=gam)


def type3(xs, c, isign: int, ss, eps: float) -> np.ndarray:
    """O2 type 3 (Sec. 3.3): translate (Eq. (trans)), dilate and spread onto the n_i grid
    (step 1, Eq. (blt3)), evaluate that grid as a Fourier series at the rescaled targets
    with the O2 type 2 (step 2, Eq. (bkt3)), correct by p_k = prod_i 2 / (w phi^(alpha_i s'_k))
    (step 3), undo the translation."""
    P = type3_params(eps, xs, ss)
    w, beta, ns = P["w"], P["beta"], P["ns"]
    d = len(xs)
    xt = [np.asarray(xs[i], dtype=np.float64) - P["x0"][i] for i in range(d)]
    st = [np.asarray(ss[i], dtype=np.float64) - P["s0"][i] for i in range(d)]
    pre = np.exp(1j * isign * sum(P["s0"][i] * xt[i] for i in range(d)))
    xp = [xt[i] / P["gamma"][i] for i in range(d)]
    b = spread(xp, _cplx(c) * pre, ns, w, beta)          # grid index l <-> Fourier index l mod n
    for ax, n in enumerate(reversed(ns)):                  # to increasing Fourier index
        b = np.roll(b, n // 2, axis=ax)
    spp = [2 * math.pi / ns[i] * P["gamma"][i] * st[i] for i in range(d)]
    bk = type2(spp, b.ravel(), isign, ns, eps=eps)
    p = np.ones(st[0].shape[0])
    for i in range(d):
        alpha = math.pi * w / ns[i]
        p = p * 2.0 / (w * kernel_ft(alpha * P["gamma"][i] * st[i], w, beta))
    post = np.exp(1j * isign * sum(np.asarray(ss[i], dtype=np.float64) * P["x0"][i] for i in range(d)))
    return p * bk * post
