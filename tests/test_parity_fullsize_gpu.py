"""Parity at the full workload sizes, in the launch configuration the benchmark times
(default plan options, one plan per transform type), on outputs the oracle's direct sums
compute one by one: a random sample of modes for type 1, of points for type 2.

Configurations:
  * 3D, N = 256^3 (fine grid 512^3), M = 1e8 points, complex64, eps = 1e-5 (w = 6),
    uniform and clustered points -- the benchmark workload;
  * 3D, N = 256^3, M = 3e7, complex128, eps = 1e-9 (w = 10);
  * 2D, N = 1024^2 (fine grid 2048^2), M = 1e7, complex64 eps = 1e-5 and complex128 eps = 1e-9,
    uniform and clustered.
Bar: relative l2 error over the sample <= 10 eps against the exact sums Eq. (1) / Eq. (2).
"""
import numpy as np
import pytest

import nufft_inputs as I

pytestmark = pytest.mark.gpu

N_MODES = 200     # sampled modes for type 1 (each an O(M) exact sum)
N_TARGETS = 2000  # sampled points for type 2 (each an O(N^d) exact sum)


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_06736_gb300 import build
    build.build()
    import paper_1808_06736_gb300 as p
    return p


CONFIGS = [
    # (d, N, M, complex dtype, eps, kind)
    (3, 256, 100_000_000, "c64", 1e-5, "uniform"),
    (3, 256, 100_000_000, "c64", 1e-5, "clustered"),
    (3, 256, 30_000_000, "c128", 1e-9, "uniform"),
    (2, 1024, 10_000_000, "c64", 1e-5, "uniform"),
    (2, 1024, 10_000_000, "c64", 1e-5, "clustered"),
    (2, 1024, 10_000_000, "c128", 1e-9, "uniform"),
    (2, 1024, 10_000_000, "c128", 1e-9, "clustered"),
]


@pytest.mark.parametrize("d,N,M,prec,eps,kind", CONFIGS)
def test_fullsize_sampled(pkg, oracle_mod, d, N, M, prec, eps, kind):
    import torch
    dev = torch.device("cuda:0")
    cdt = torch.complex64 if prec == "c64" else torch.complex128
    rdt = torch.float32 if prec == "c64" else torch.float64
    Ns = [N] * d
    seed = 5000 + 10 * d + (1 if kind == "clustered" else 0) + (2 if prec == "c128" else 0)
    xs = I.torch_points(seed, M, d, kind, dev, rdt)
    c = I.torch_complex_normal(seed + 1, M, dev, cdt)
    f = I.torch_complex_normal(seed + 2, N ** d, dev, cdt)

    p1 = pkg.Plan(1, Ns, eps=eps, isign=1, dtype=cdt, device=dev)
    p1.setpts(*xs)
    fk = p1.execute(c).reshape(-1)
    assert p1.status() == 0
    p1.close()
    p2 = pkg.Plan(2, Ns, eps=eps, isign=-1, dtype=cdt, device=dev)
    p2.setpts(*xs)
    cj = p2.execute(f).reshape(-1)
    assert p2.status() == 0
    p2.close()

    rng = np.random.default_rng(seed)
    modes = rng.integers(-(N // 2), N - N // 2, size=(N_MODES, d))
    targets = rng.choice(M, size=N_TARGETS, replace=False)
    pos = oracle_mod.mode_index(modes, Ns)

    x64 = [v.double().cpu().numpy() for v in xs]
    c64 = c.to(torch.complex128).cpu().numpy()
    ref1 = oracle_mod.direct_type1(x64, c64, 1, Ns, modes=modes)
    got1 = fk[torch.as_tensor(pos, device=dev)].to(torch.complex128).cpu().numpy()
    del c64
    ref2 = oracle_mod.direct_type2([v[targets] for v in x64], f.to(torch.complex128).cpu().numpy(), -1, Ns)
    got2 = cj[torch.as_tensor(targets, device=dev)].to(torch.complex128).cpu().numpy()
    e1 = oracle_mod.rel_l2(got1, ref1)
    e2 = oracle_mod.rel_l2(got2, ref2)
    assert e1 <= 10 * eps, e1
    assert e2 <= 10 * eps, e2
