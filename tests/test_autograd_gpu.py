"""Differentiable transforms on the GPU (paper_1808_06736_gb300.autograd).

loss = ||F2(f; x) - y||^2 (and the type-1 analogue); gradients with respect to
the coefficients / strengths and the points, checked against the FP64
direct-sum gradient (sampled at the larger size) and central finite
differences of the GPU loss."""
import numpy as np
import pytest

import nufft_inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ag():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_06736_gb300 import build
    build.build()
    from paper_1808_06736_gb300 import autograd
    return autograd


def _k(Ns):
    grids = np.meshgrid(*[np.arange(n) - n // 2 for n in reversed(Ns)], indexing="ij")
    return [g.ravel() for g in reversed(grids)]


# "exact": the point gradient through d extra transforms of (i k_d) f, bar 10 eps;
# "kernel": through the derivative of the ES kernel, whose error is ~2 sqrt(12) times the
# values' (aliased frequencies weighted by their own size), bar 20 eps with an fp32 floor.
@pytest.mark.parametrize("cdt,eps,tol,xgrad", [("c128", 1e-11, 1e-9, "exact"), ("c64", 1e-5, 1e-4, "exact"),
                                               ("c128", 1e-11, 2e-10, "kernel"), ("c64", 1e-5, 2e-4, "kernel")])
def test_type2_loss_gradients_3d(ag, oracle_mod, cdt, eps, tol, xgrad):
    """3D, N = 64^3, M = 1e5: grad wrt f on sampled modes, wrt x on sampled points."""
    import torch
    dev = torch.device("cuda:0")
    Ns = [64, 64, 64]
    M = 100_000
    rdt = torch.float64 if cdt == "c128" else torch.float32
    cdtype = torch.complex128 if cdt == "c128" else torch.complex64
    x = torch.tensor(np.stack(I.points(61, M, 3)), dtype=rdt, device=dev, requires_grad=True)
    f = torch.tensor(I.complex_normal(62, 64 ** 3).reshape(64, 64, 64), dtype=cdtype, device=dev,
                     requires_grad=True)
    y = torch.tensor(I.complex_normal(63, M), dtype=cdtype, device=dev)
    c = ag.nufft_type2(x, f, eps=eps, isign=-1, xgrad=xgrad)
    loss = ((c - y).abs() ** 2).sum()
    loss.backward()
    xs = [v.astype(np.float64) for v in x.detach().cpu().numpy()]
    fn = f.detach().cpu().numpy().astype(np.complex128).ravel()
    yn = y.cpu().numpy().astype(np.complex128)
    rng = np.random.default_rng(64)
    tj = rng.choice(M, size=48, replace=False)
    ct = oracle_mod.direct_type2([v[tj] for v in xs], fn, -1, Ns)
    G = 2 * (ct - yn[tj])
    ks = _k(Ns)
    for d in range(3):
        cd = oracle_mod.direct_type2([v[tj] for v in xs], fn * (-1j * ks[d]), -1, Ns)
        ref = np.real(np.conj(G) * cd)
        got = x.grad[d].detach().cpu().numpy()[tj]
        assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)
    # grad_f = F1_{+1}(x) G over all points; sample modes, G from the GPU forward values
    Gall = 2 * (c.detach().cpu().numpy().astype(np.complex128) - yn)
    modes = rng.integers(-32, 32, size=(24, 3))
    ref_f = oracle_mod.direct_type1(xs, Gall, 1, Ns, modes=modes)
    got_f = f.grad.detach().cpu().numpy().ravel()[oracle_mod.mode_index(modes, Ns)]
    assert np.linalg.norm(got_f - ref_f) <= tol * np.linalg.norm(ref_f)


@pytest.mark.parametrize("xgrad", ["exact", "kernel"])
@pytest.mark.parametrize("typ", [1, 2])
def test_point_gradient_matches_finite_differences(ag, typ, xgrad):
    """Central differences of the GPU loss (complex128, eps = 1e-13) in a few coordinates."""
    import torch
    dev = torch.device("cuda:0")
    Ns = [12, 10, 8]
    M = 400
    x0 = np.stack(I.points(71, M, 3))
    c = torch.tensor(I.complex_normal(72, M), device=dev)
    f = torch.tensor(I.complex_normal(73, 960).reshape(8, 10, 12), device=dev)
    y1 = torch.tensor(I.complex_normal(74, 960).reshape(8, 10, 12), device=dev)
    y2 = torch.tensor(I.complex_normal(75, M), device=dev)
    eps = 1e-13

    def loss(xt):
        if typ == 1:
            out = ag.nufft_type1(xt, c, Ns, eps=eps, isign=1, xgrad=xgrad)
            return ((out - y1).abs() ** 2).sum()
        out = ag.nufft_type2(xt, f, eps=eps, isign=-1, xgrad=xgrad)
        return ((out - y2).abs() ** 2).sum()

    x = torch.tensor(x0, device=dev, requires_grad=True)
    loss(x).backward()
    h = 1e-5
    for d, j in [(0, 3), (1, 17), (2, 123), (0, 399)]:
        xp, xm = x0.copy(), x0.copy()
        xp[d, j] += h
        xm[d, j] -= h
        fd = (loss(torch.tensor(xp, device=dev)).item() - loss(torch.tensor(xm, device=dev)).item()) / (2 * h)
        g = x.grad[d, j].item()
        assert abs(fd - g) <= 1e-6 * max(1.0, abs(g)), (d, j, fd, g)


def test_strength_gradient_is_adjoint(ag):
    """d<F1 c, w>/dc = F2_{-s} w: the strength gradient of a linear loss equals the adjoint transform."""
    import torch
    dev = torch.device("cuda:0")
    Ns = [16, 12]
    M = 3000
    x = torch.tensor(np.stack(I.points(81, M, 2)), device=dev)
    c = torch.tensor(I.complex_normal(82, M), device=dev, requires_grad=True)
    wv = torch.tensor(I.complex_normal(83, 192).reshape(12, 16), device=dev)
    out = ag.nufft_type1(x, c, Ns, eps=1e-12, isign=1)
    (out * wv.conj()).real.sum().backward()
    ref = ag.nufft_type2(x, wv, eps=1e-12, isign=-1)
    assert torch.linalg.vector_norm(c.grad - ref) <= 1e-10 * torch.linalg.vector_norm(ref)
