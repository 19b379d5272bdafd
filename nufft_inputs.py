"""Seeded synthetic inputs for the NUFFT tests and benchmark.

This module only draws random numbers and lays out points; it holds none of
the transform's arithmetic, so the CUDA path and the CPU oracle can both be
fed from it without sharing any of the method.

Recipe (the paper uses no dataset; Sec. 6 draws its own synthetic points):
  * "uniform" points: x_i iid U[-pi, pi) per coordinate;
  * "clustered" points: x_i iid N(0, sigma^2) per coordinate (sigma = 0.3),
    wrapped into [-pi, pi);
  * strengths / coefficients: real and imaginary parts iid N(0, 1);
  * type-3 sources and frequencies: uniform (or clipped Gaussian) in an
    off-centre box centre +- half per coordinate (box_points).
Seeds are plain integers; every generator is numpy PCG64 (host) or torch's
Philox generator (device, for the 1e7..1e8-point workloads).
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def wrap(x: np.ndarray) -> np.ndarray:
    """Map values into [-pi, pi) by a period shift."""
    y = np.mod(x + math.pi, TWO_PI) - math.pi
    return np.where(y >= math.pi, y - TWO_PI, y)


def points(seed: int, M: int, d: int, kind: str = "uniform", dtype=np.float64, sigma: float = 0.3):
    """d coordinate arrays of M points ('uniform' or 'clustered')."""
    g = rng(seed)
    out = []
    for _ in range(d):
        if kind == "uniform":
            v = g.uniform(-math.pi, math.pi, size=M)
        elif kind == "clustered":
            v = wrap(g.normal(0.0, sigma, size=M))
        else:
            raise ValueError(kind)
        v = v.astype(dtype)
        # float32 rounding can land on +pi; keep the half-open range
        v[v >= np.asarray(math.pi, dtype=dtype)] = np.asarray(-math.pi, dtype=dtype)
        out.append(v)
    return out


def box_points(seed: int, n: int, centre, half, kind: str = "uniform", dtype=np.float64):
    """Type-3 sources or targets: len(centre) coordinate arrays of n reals in the box
    centre_i +- half_i, iid uniform ('uniform') or Gaussian about the centre with
    standard deviation half_i / 4 clipped to the box ('clustered')."""
    g = rng(seed)
    out = []
    for c, h in zip(centre, half):
        if kind == "uniform":
            v = g.uniform(c - h, c + h, size=n)
        elif kind == "clustered":
            v = np.clip(g.normal(c, h / 4.0, size=n), c - h, c + h)
        else:
            raise ValueError(kind)
        out.append(v.astype(dtype))
    return out


def complex_normal(seed: int, n: int, dtype=np.complex128) -> np.ndarray:
    """n complex values with re, im iid N(0, 1)."""
    g = rng(seed)
    v = g.standard_normal(n) + 1j * g.standard_normal(n)
    return v.astype(dtype)


def edge_points(d: int, ns, dtype=np.float64):
    """Hand-placed points at awkward places of the fine grid of sizes ns:
    x = -pi, x = 0, the largest value below pi, exact fine-grid nodes, bin
    edges (multiples of 8 cells), half-cell offsets, and values in
    [-3 pi, 3 pi] outside the base period.  Returns d coordinate arrays."""
    cols = []
    for i in range(d):
        n = int(ns[i])
        h = TWO_PI / n
        base = [-math.pi, 0.0, np.nextafter(np.asarray(math.pi, dtype=dtype), np.asarray(0, dtype=dtype)),
                h, 8 * h, 16 * h - math.pi, 0.5 * h, -0.5 * h, (n // 2 - 1) * h, 2.5 * math.pi,
                -2.9 * math.pi, 3 * h + 1e-9]
        cols.append(np.asarray(base, dtype=np.float64))
    M = len(cols[0])
    # decorrelate the columns so the points are not all on the diagonal
    out = []
    for i in range(d):
        out.append(np.roll(cols[i], i * 5).astype(dtype))
    return out, M


def torch_points(seed: int, M: int, d: int, kind: str, device, dtype):
    """Large point sets drawn on the device with torch's generator."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    out = []
    for _ in range(d):
        if kind == "uniform":
            v = torch.rand(M, generator=g, device=device, dtype=torch.float64) * TWO_PI - math.pi
        elif kind == "clustered":
            v = torch.randn(M, generator=g, device=device, dtype=torch.float64) * 0.3
            v = torch.remainder(v + math.pi, TWO_PI) - math.pi
        else:
            raise ValueError(kind)
        v = v.to(dtype)
        v = torch.where(v >= math.pi, torch.full_like(v, -math.pi), v)
        out.append(v.contiguous())
    return out


def torch_complex_normal(seed: int, n: int, device, dtype):
    """n complex values with re, im iid N(0, 1), drawn on the device."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    real = torch.float32 if dtype == torch.complex64 else torch.float64
    v = torch.randn(n, 2, generator=g, device=device, dtype=real)
    return torch.view_as_complex(v).contiguous()


# --------------------------------------------------------------- serving trace
SERVING_2D_N = (64, 128, 256, 512, 1024)
SERVING_3D_N = (64, 128, 256)


def serving_trace(seed: int, n: int, rate: float, pool: int = 10_000_000):
    """A mixed request stream: Poisson arrivals (mean ``rate`` per second) of
    complex64 requests.  20 % are least-squares gradient requests (3D, N = 64^3,
    M = 1e5); the rest are type 1 or type 2 (equally likely), 2D or 3D (equally
    likely) with N_i drawn from SERVING_2D_N / SERVING_3D_N, M log-uniform in
    [1e4, 1e7].  eps is 1e-3 or 1e-5 and the sign +1 or -1, each equally
    likely.  ``off`` is where the request's points and strengths start in a
    shared input pool of ``pool`` values."""
    r = rng(seed)
    t = np.cumsum(r.exponential(1.0 / rate, size=n))
    out = []
    for i in range(n):
        eps = float(r.choice([1e-3, 1e-5]))
        isign = int(r.choice([-1, 1]))
        if r.random() < 0.2:
            kind, d, modes, M = 3, 3, (64, 64, 64), 100_000
        else:
            kind = int(r.choice([1, 2]))
            d = int(r.choice([2, 3]))
            Nd = int(r.choice(SERVING_2D_N if d == 2 else SERVING_3D_N))
            modes = (Nd,) * d
            M = int(math.exp(r.uniform(math.log(1e4), math.log(1e7))))
        off = int(r.integers(0, pool - M + 1))
        out.append(dict(t=float(t[i]), kind=kind, d=d, modes=modes, M=M, eps=eps, isign=isign, off=off))
    return out
