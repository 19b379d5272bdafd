"""The autotuner (nufft_tune / nufft_batch_tune) on the GPU: it returns options no
slower than the default as measured, and plans made with them give the same
results as the default plan (rounding budget) and the exact sums (10 eps)."""
import numpy as np
import pytest

import nufft_inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_06736_gb300 import build
    build.build()
    import paper_1808_06736_gb300 as p
    return p


@pytest.mark.parametrize("typ", [1, 2])
@pytest.mark.parametrize("d,Ns,M", [(3, [32, 28, 24], 200_000), (2, [96, 80], 100_000), (1, [3000], 50_000)])
def test_tuned_plan_is_correct_and_not_slower(pkg, oracle_mod, typ, d, Ns, M):
    import torch
    dev = torch.device("cuda:0")
    xs = I.torch_points(900 + d, M, d, "clustered", dev, torch.float32)
    ntot = int(np.prod(Ns))
    data = I.torch_complex_normal(910 + d, M if typ == 1 else ntot, dev, torch.complex64)
    opts, best, default = pkg.tune_plan(typ, Ns, xs, data, eps=1e-5, reps=2)
    assert 0 < best <= default
    # the reference plan uses the grid the tuner picked (upsampling 2 or 5/4); only launch shapes differ
    ref = pkg.Plan(typ, Ns, eps=1e-5, device=dev, upsampfac=opts["upsampfac"])
    ref.setpts(*xs)
    r = ref.execute(data).reshape(-1)
    ref.close()
    p = pkg.Plan(typ, Ns, eps=1e-5, device=dev, **opts)
    p.setpts(*xs)
    out = p.execute(data).reshape(-1)
    assert p.status() == 0
    p.close()
    rel = float(torch.linalg.vector_norm((out - r).to(torch.complex128)) / torch.linalg.vector_norm(r.to(torch.complex128)))
    assert rel <= 3e-5, (opts, rel)
    x64 = [v.double().cpu().numpy() for v in xs]
    rng = np.random.default_rng(3)
    if typ == 1:
        modes = np.stack([rng.integers(-(n // 2), n - n // 2, size=16) for n in Ns], axis=1)
        exact = oracle_mod.direct_type1(x64, data.to(torch.complex128).cpu().numpy(), 1, Ns, modes=modes)
        got = out[torch.as_tensor(oracle_mod.mode_index(modes, Ns), device=dev)]
    else:
        tj = rng.choice(M, size=32, replace=False)
        exact = oracle_mod.direct_type2([v[tj] for v in x64], data.to(torch.complex128).cpu().numpy(), -1, Ns)
        got = out[torch.as_tensor(tj, device=dev)]
    assert oracle_mod.rel_l2(got.to(torch.complex128).cpu().numpy(), exact) <= 1e-4


def test_tuned_batch_is_correct_and_not_slower(pkg):
    import torch
    dev = torch.device("cuda:0")
    rng = I.rng(920)
    B = 24
    modes = [(int(v), int(v)) for v in rng.choice([32, 64, 128], size=B)]
    Ms = np.exp(rng.uniform(np.log(1e3), np.log(1e5), size=B)).astype(np.int64)
    offs = np.concatenate([[0], np.cumsum(Ms)]).astype(np.int64)
    xs = I.torch_points(921, int(offs[-1]), 2, "uniform", dev, torch.float32)
    nf = sum(a * b for a, b in modes)
    f = I.torch_complex_normal(922, nf, dev, torch.complex64)
    opts, best, default = pkg.tune_batch(2, modes, xs, f, offs, eps=1e-5, reps=2)
    assert 0 < best <= default
    bp = pkg.BatchPlan(2, modes, eps=1e-5, device=dev, **opts)
    bp.setpts(*xs, offsets=offs)
    out = bp.execute(f)
    assert bp.status() == 0
    moffs = bp.mode_offsets
    bp.close()
    for t in range(B):
        p = pkg.Plan(2, modes[t], eps=1e-5, device=dev, upsampfac=opts["upsampfac"])
        p.setpts(*[v[int(offs[t]):int(offs[t + 1])] for v in xs])
        r = p.execute(f[moffs[t]:moffs[t + 1]]).reshape(-1)
        p.close()
        o = out[int(offs[t]):int(offs[t + 1])]
        rel = float(torch.linalg.vector_norm((o - r).to(torch.complex128)) / torch.linalg.vector_norm(r.to(torch.complex128)))
        assert rel <= 3e-5, (t, opts, rel)
