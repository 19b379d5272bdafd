"""The gradient formulas the autograd layer implements, pinned on the CPU:
torch's own autograd through a plain direct evaluation of Eq. (1) / Eq. (2)
against the formulas evaluated with the oracle's direct sums."""
import numpy as np
import pytest
import torch

import nufft_inputs as I


def _k(Ns):
    grids = torch.meshgrid(*[torch.arange(n, dtype=torch.float64) - n // 2 for n in reversed(Ns)], indexing="ij")
    return [g.reshape(-1) for g in reversed(grids)]  # k_1 fastest


def _phase(x, Ns, s):
    ks = _k(Ns)
    return torch.exp(1j * s * sum(k[:, None] * x[d][None, :] for d, k in enumerate(ks)))  # (N, M)


@pytest.mark.parametrize("s", [1, -1])
def test_type1_gradient_formulas(oracle_mod, s):
    Ns = [5, 4, 3]
    M = 11
    x = torch.tensor(np.stack(I.points(1, M, 3)), requires_grad=True)
    c = torch.tensor(I.complex_normal(2, M), requires_grad=True)
    y = torch.tensor(I.complex_normal(3, 60))
    f = _phase(x, Ns, s) @ c
    L = ((f - y).abs() ** 2).sum()
    L.backward()
    G = 2 * (f - y).detach().numpy()  # torch's incoming gradient for |f - y|^2
    xs = [v for v in x.detach().numpy()]
    cn = c.detach().numpy()
    grad_c = oracle_mod.direct_type2(xs, G, -s, Ns)
    np.testing.assert_allclose(c.grad.numpy(), grad_c, rtol=1e-10, atol=1e-10)
    ks = [k.numpy() for k in _k(Ns)]
    for d in range(3):
        gd = oracle_mod.direct_type2(xs, G * (-s * 1j * ks[d]), -s, Ns)
        np.testing.assert_allclose(x.grad[d].numpy(), np.real(cn * np.conj(gd)), rtol=1e-10, atol=1e-9)


@pytest.mark.parametrize("s", [1, -1])
def test_type2_gradient_formulas(oracle_mod, s):
    Ns = [6, 5]
    M = 13
    x = torch.tensor(np.stack(I.points(4, M, 2)), requires_grad=True)
    f = torch.tensor(I.complex_normal(5, 30), requires_grad=True)
    y = torch.tensor(I.complex_normal(6, M))
    c = _phase(x, Ns, s).T @ f
    L = ((c - y).abs() ** 2).sum()
    L.backward()
    G = 2 * (c - y).detach().numpy()
    xs = [v for v in x.detach().numpy()]
    fn = f.detach().numpy()
    np.testing.assert_allclose(f.grad.numpy(), oracle_mod.direct_type1(xs, G, -s, Ns), rtol=1e-10, atol=1e-10)
    ks = [k.numpy() for k in _k(Ns)]
    for d in range(2):
        cd = oracle_mod.direct_type2(xs, fn * (s * 1j * ks[d]), s, Ns)
        np.testing.assert_allclose(x.grad[d].numpy(), np.real(np.conj(G) * cd), rtol=1e-10, atol=1e-9)
