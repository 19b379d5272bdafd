"""Differentiable type-1 / type-2 transforms (torch.autograd.Function).

For the type-1 transform f = F1_s(x) c, f_k = sum_j c_j exp(i s k.x_j), and the
type-2 transform c = F2_s(x) f, c_j = sum_k f_k exp(i s k.x_j) (Eq. (1),
Eq. (2)), with G the incoming gradient (torch's convention for complex
tensors):

  type 1:  grad_c = F2_{-s}(x) G                     (the adjoint, Sec. 1)
           grad_x_d = Re( c * conj( F2_{-s}(x) [(-s i k_d) G] ) )
  type 2:  grad_f = F1_{-s}(x) G
           grad_x_d = Re( conj(G) * F2_s(x) [(s i k_d) f] )

so every gradient is again a type-1 or type-2 transform on the GPU.  The point
gradient has two routes (``xgrad``):

  "exact"   d extra type-2 transforms of the mode data multiplied by (+-i k_d):
            the derivative of the exponential sum, to the transforms' own eps;
  "kernel"  one interpolation pass that also differentiates the ES kernel
            (nufft_execute_grad, phi'(z) = -beta z / sqrt(1 - z^2) phi(z)): the
            derivative of the type-2 approximation, whose relative error is a
            few times eps (aliased frequencies are weighted by their own size),
            for one FFT instead of d + 1.

Plans are cached per (type, modes, eps, sign, dtype, device); points are set
on every call.
"""
from __future__ import annotations

import torch

from . import Plan


class PlanCache:
    """Keeps one plan per (type, modes, eps, isign, dtype, device, options)."""

    def __init__(self):
        self._plans = {}

    def get(self, type_, n_modes, eps, isign, dtype, device, **opts):
        key = (type_, tuple(n_modes), float(eps), int(isign), dtype, str(device), tuple(sorted(opts.items())))
        p = self._plans.get(key)
        if p is None:
            p = Plan(type_, n_modes, eps=eps, isign=isign, dtype=dtype, device=device, **opts)
            self._plans[key] = p
        return p

    def clear(self):
        for p in self._plans.values():
            p.close()
        self._plans.clear()


_default_cache = PlanCache()


def _complex_of(real_dtype):
    return torch.complex64 if real_dtype == torch.float32 else torch.complex128


def _ik(n_modes, d, sign, dtype, device):
    """sign * i * k_d on the mode array (increasing k, dimension 1 fastest), broadcastable."""
    D = len(n_modes)
    N = n_modes[d]
    k = torch.arange(N, device=device, dtype=torch.float64) - (N // 2)
    shape = [1] * D
    shape[D - 1 - d] = N
    return (1j * sign * k).to(dtype).reshape(shape)


class _Type1(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, c, n_modes, eps, isign, cache, xgrad, opts):
        cdt = _complex_of(x.dtype)
        p = cache.get(1, n_modes, eps, isign, cdt, x.device, **opts)
        p.setpts(*x.unbind(0))
        f = p.execute(c).reshape(tuple(reversed(n_modes)))
        ctx.save_for_backward(x, c)
        ctx.cfg = (n_modes, eps, isign, cache, xgrad, opts)
        return f

    @staticmethod
    def backward(ctx, G):
        x, c = ctx.saved_tensors
        n_modes, eps, isign, cache, xgrad, opts = ctx.cfg
        cdt = _complex_of(x.dtype)
        p2 = cache.get(2, n_modes, eps, -isign, cdt, x.device, **opts)
        p2.setpts(*x.unbind(0))
        G = G.contiguous()
        grad_x = grad_c = None
        if ctx.needs_input_grad[0] and xgrad == "kernel":
            gc, dg = p2.execute_grad(G)
            if ctx.needs_input_grad[1]:
                grad_c = gc.reshape(c.shape)
            grad_x = (c.unsqueeze(0) * dg[0].conj()).real
            return grad_x, grad_c, None, None, None, None, None, None
        if ctx.needs_input_grad[1]:
            grad_c = p2.execute(G).reshape(c.shape)
        if ctx.needs_input_grad[0]:
            rows = []
            for d in range(x.shape[0]):
                gd = p2.execute(G * _ik(n_modes, d, -isign, cdt, x.device)).reshape(c.shape)
                rows.append((c * gd.conj()).real)
            grad_x = torch.stack(rows)
        return grad_x, grad_c, None, None, None, None, None, None


class _Type2(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, f, eps, isign, cache, xgrad, opts):
        cdt = _complex_of(x.dtype)
        n_modes = tuple(reversed(f.shape))
        p = cache.get(2, n_modes, eps, isign, cdt, x.device, **opts)
        p.setpts(*x.unbind(0))
        dc = None
        if xgrad == "kernel" and ctx.needs_input_grad[0]:
            c, dc = p.execute_grad(f)
            c, dc = c.reshape(x.shape[1]), dc[0]
        else:
            c = p.execute(f).reshape(x.shape[1])
        ctx.save_for_backward(x, f, dc)
        ctx.cfg = (n_modes, eps, isign, cache, xgrad, opts)
        return c

    @staticmethod
    def backward(ctx, G):
        x, f, dc = ctx.saved_tensors
        n_modes, eps, isign, cache, xgrad, opts = ctx.cfg
        cdt = _complex_of(x.dtype)
        G = G.contiguous()
        grad_x = grad_f = None
        if ctx.needs_input_grad[1]:
            p1 = cache.get(1, n_modes, eps, -isign, cdt, x.device, **opts)
            p1.setpts(*x.unbind(0))
            grad_f = p1.execute(G).reshape(f.shape)
        if ctx.needs_input_grad[0] and dc is not None:
            grad_x = (G.conj().unsqueeze(0) * dc).real
        elif ctx.needs_input_grad[0]:
            p2 = cache.get(2, n_modes, eps, isign, cdt, x.device, **opts)
            p2.setpts(*x.unbind(0))
            rows = []
            for d in range(x.shape[0]):
                cd = p2.execute(f * _ik(n_modes, d, isign, cdt, x.device)).reshape(G.shape)
                rows.append((G.conj() * cd).real)
            grad_x = torch.stack(rows)
        return grad_x, grad_f, None, None, None, None, None


def _check_xgrad(xgrad):
    if xgrad not in ("exact", "kernel"):
        raise ValueError("xgrad must be 'exact' or 'kernel'")


def nufft_type1(x: torch.Tensor, c: torch.Tensor, n_modes, eps: float = 1e-6, isign: int = 1,
                cache: PlanCache | None = None, xgrad: str = "exact", **opts) -> torch.Tensor:
    """f = F1_s(x) c: x real (d, M) on the GPU, c complex (M,); returns f of shape (N_d, ..., N_1).
    Differentiable in x and c; ``xgrad`` picks the point-gradient route; ``opts`` are plan
    options (e.g. upsampfac)."""
    if x.dim() != 2 or x.shape[0] != len(n_modes):
        raise ValueError("x must have shape (d, M) with d = len(n_modes)")
    _check_xgrad(xgrad)
    return _Type1.apply(x, c, tuple(int(v) for v in n_modes), eps, isign, cache or _default_cache, xgrad, opts)


def nufft_type2(x: torch.Tensor, f: torch.Tensor, eps: float = 1e-6, isign: int = -1,
                cache: PlanCache | None = None, xgrad: str = "exact", **opts) -> torch.Tensor:
    """c = F2_s(x) f: x real (d, M), f complex of shape (N_d, ..., N_1); returns c (M,).
    Differentiable in x and f; ``xgrad`` picks the point-gradient route; ``opts`` are plan
    options (e.g. upsampfac)."""
    if x.dim() != 2 or x.shape[0] != f.dim():
        raise ValueError("x must have shape (d, M) with d = f.dim()")
    _check_xgrad(xgrad)
    return _Type2.apply(x, f, eps, isign, cache or _default_cache, xgrad, opts)
