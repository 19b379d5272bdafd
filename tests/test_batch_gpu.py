"""Batched transforms (one launch per step over many transforms of different
sizes, replayed from a CUDA graph) against the single-transform path and the
exact sums."""
import numpy as np
import pytest

import nufft_inputs as I

pytestmark = pytest.mark.gpu

TOL_SAME = {"c64": 3e-5, "c128": 1e-12}


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_06736_gb300 import build
    build.build()
    import paper_1808_06736_gb300 as p
    return p


def _case(d, seed):
    rng = np.random.default_rng(seed)
    shapes = {1: [(40,), (101,), (256,), (7,)], 2: [(16, 16), (24, 20), (64, 48), (9, 33), (32, 32)],
              3: [(12, 10, 8), (16, 16, 16), (20, 14, 9)]}[d]
    modes = [shapes[i % len(shapes)] for i in range(11)]
    Ms = [int(v) for v in rng.integers(0, 3000, size=len(modes))]
    Ms[3] = 0  # a transform without points
    return modes, Ms


@pytest.mark.parametrize("prec,eps", [("c64", 1e-5), ("c128", 1e-10)])
@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("typ", [1, 2])
def test_batch_matches_single_path(pkg, oracle_mod, prec, eps, d, typ):
    import torch
    dev = torch.device("cuda:0")
    cdt = torch.complex64 if prec == "c64" else torch.complex128
    rdt = np.float32 if prec == "c64" else np.float64
    modes, Ms = _case(d, 100 * d + typ)
    offs = np.concatenate([[0], np.cumsum(Ms)]).astype(np.int64)
    xs = [np.concatenate([I.points(1000 + 7 * t + i, Ms[t], 1, kind="clustered" if t % 2 else "uniform", dtype=rdt)[0]
                          for t in range(len(modes))]) for i in range(d)]
    bp = pkg.BatchPlan(typ, modes, eps=eps, isign=1 if typ == 1 else -1, dtype=cdt, device=dev)
    bp.setpts(*[torch.from_numpy(v).to(dev) for v in xs], offsets=offs)
    if typ == 1:
        data = I.complex_normal(5, int(offs[-1]))
    else:
        data = I.complex_normal(6, bp.mode_offsets[-1])
    td = torch.from_numpy(data).to(dev).to(cdt)
    out1 = bp.execute(td).cpu().numpy()
    out2 = bp.execute(td).cpu().numpy()  # graph replay
    assert bp.status() == 0
    np.testing.assert_array_equal(out1, out2) if typ == 2 else None
    for t, m in enumerate(modes):
        sl = slice(int(offs[t]), int(offs[t + 1]))
        ml = slice(bp.mode_offsets[t], bp.mode_offsets[t + 1])
        xt = [v[sl] for v in xs]
        p = pkg.Plan(typ, m, eps=eps, isign=1 if typ == 1 else -1, dtype=cdt, device=dev)
        p.setpts(*[torch.from_numpy(np.ascontiguousarray(v)).to(dev) for v in xt])
        got = out1[ml] if typ == 1 else out1[sl]
        ref_in = data[sl] if typ == 1 else data[ml]
        single = p.execute(torch.from_numpy(ref_in).to(dev).to(cdt)).cpu().numpy().ravel()
        p.close()
        if Ms[t] == 0:
            assert np.all(got == 0) if typ == 1 else got.size == 0
            continue
        assert oracle_mod.rel_l2(got, single) <= TOL_SAME[prec], t
        if t < 3:
            x64 = [v.astype(np.float64) for v in xt]
            ref = (oracle_mod.direct_type1(x64, ref_in, 1, list(m)) if typ == 1
                   else oracle_mod.direct_type2(x64, ref_in, -1, list(m)))
            assert oracle_mod.rel_l2(got, ref) <= max(10 * eps, 2e-5), t
    bp.close()


def test_batch_new_points_and_pointers(pkg):
    """setpts with other points, and a new output buffer: the graph is rebuilt or reused correctly."""
    import torch
    dev = torch.device("cuda:0")
    modes = [(32, 32), (16, 24), (64, 64)]
    bp = pkg.BatchPlan(2, modes, eps=1e-6, isign=-1, dtype=torch.complex128, device=dev)
    f = torch.from_numpy(I.complex_normal(9, bp.mode_offsets[-1])).to(dev)
    res = []
    for k, Ms in enumerate([[100, 200, 300], [500, 0, 50]]):
        offs = np.concatenate([[0], np.cumsum(Ms)])
        xs = [torch.from_numpy(I.points(20 + k + i, int(offs[-1]), 1)[0]).to(dev) for i in range(2)]
        bp.setpts(*xs, offsets=offs)
        out = bp.execute(f)
        out_b = torch.empty_like(out)
        bp.execute(f, out=out_b)
        assert torch.equal(out, out_b)
        p = pkg.Plan(2, modes[0], eps=1e-6, isign=-1, dtype=torch.complex128, device=dev)
        p.setpts(*[v[: Ms[0]] for v in xs])
        ref = p.execute(f[: 1024]).reshape(-1)
        p.close()
        assert torch.linalg.vector_norm(out[: Ms[0]] - ref) <= 1e-12 * torch.linalg.vector_norm(ref)
        res.append(out)
    bp.close()
