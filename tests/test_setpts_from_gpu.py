"""nufft_setpts_from: a type-2 plan takes the points a type-1 plan has binned (Sec. 5.1's bin
sort depends only on the points, the fine grid and the bins), so one binning serves both.

Checked through the C ABI (the Plan binding): both transforms against the exact sums Eq. (1) /
Eq. (2) (10 eps) and the plain algorithm at the same parameters (the rounding budget); the
type-2 values equal those of a plan that bins the points itself -- bit for bit in complex64,
where each value's sum does not depend on where the point sits in the bin order, and to
1e-14 in complex128; the shared set outlives the
plan that made it, and a later setpts on that plan leaves the sharing plan's points alone;
incompatible plans and a source without points are refused.
"""
import numpy as np
import pytest

import nufft_inputs as I

pytestmark = pytest.mark.gpu

TOL_SAME = {np.complex64: 3e-5, np.complex128: 1e-12}
SIZES = {1: ([800], 5000), 2: ([60, 44], 20000), 3: ([20, 18, 14], 30000)}


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_06736_gb300 import build
    build.build()
    import paper_1808_06736_gb300 as p
    return p


def _dev(v, dt):
    import torch
    return torch.from_numpy(np.ascontiguousarray(v, dtype=dt)).to("cuda:0")


@pytest.mark.parametrize("cdtype,eps", [(np.complex64, 1e-5), (np.complex128, 1e-10)])
@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("kind", ["uniform", "clustered"])
def test_type2_on_type1_points(pkg, oracle_mod, cdtype, eps, d, kind):
    import torch
    Ns, M = SIZES[d]
    rdt = np.float32 if cdtype == np.complex64 else np.float64
    tdt = torch.complex64 if cdtype == np.complex64 else torch.complex128
    xs = I.points(8100 + d, M, d, kind=kind, dtype=rdt)
    c = I.complex_normal(8110 + d, M, dtype=cdtype)
    f = I.complex_normal(8120 + d, int(np.prod(Ns)), dtype=cdtype)
    p1 = pkg.Plan(1, Ns, eps=eps, isign=1, dtype=tdt, device="cuda:0")
    p2 = pkg.Plan(2, Ns, eps=eps, isign=-1, dtype=tdt, device="cuda:0")
    p1.setpts(*[_dev(v, rdt) for v in xs])
    p2.setpts_from(p1)
    g1 = p1.execute(_dev(c, cdtype)).cpu().numpy().ravel()
    g2 = p2.execute(_dev(f, cdtype)).cpu().numpy().ravel()
    assert p1.status() == 0 and p2.status() == 0
    # the same type 2 with its own binning
    p3 = pkg.Plan(2, Ns, eps=eps, isign=-1, dtype=tdt, device="cuda:0")
    p3.setpts(*[_dev(v, rdt) for v in xs])
    g3 = p3.execute(_dev(f, cdtype)).cpu().numpy().ravel()
    assert p3.status() == 0
    for p in (p1, p2, p3):
        p.close()
    if cdtype == np.complex64:
        assert np.array_equal(g2, g3)
    else:  # the double-float interpolation may round differently with another order of the points in a bin
        assert oracle_mod.rel_l2(g2, g3) <= 1e-14
    x64 = [v.astype(np.float64) for v in xs]
    w, beta, ns = oracle_mod.choose_params(eps, Ns)
    assert oracle_mod.rel_l2(g1, oracle_mod.type1(x64, c, 1, Ns, w=w, beta=beta, ns=ns)) <= TOL_SAME[cdtype]
    assert oracle_mod.rel_l2(g2, oracle_mod.type2(x64, f, -1, Ns, w=w, beta=beta, ns=ns)) <= TOL_SAME[cdtype]
    assert oracle_mod.rel_l2(g1, oracle_mod.direct_type1(x64, c, 1, Ns)) <= 10 * eps
    assert oracle_mod.rel_l2(g2, oracle_mod.direct_type2(x64, f, -1, Ns)) <= 10 * eps


def test_shared_points_outlive_and_survive_new_points(pkg, oracle_mod):
    import torch
    Ns, M, eps = [24, 20, 16], 20000, 1e-5
    xa = I.points(8200, M, 3, dtype=np.float32)
    xb = I.points(8201, M, 3, kind="clustered", dtype=np.float32)
    f = I.complex_normal(8202, int(np.prod(Ns)), dtype=np.complex64)
    p1 = pkg.Plan(1, Ns, eps=eps, dtype=torch.complex64, device="cuda:0")
    p2 = pkg.Plan(2, Ns, eps=eps, dtype=torch.complex64, device="cuda:0")
    p1.setpts(*[_dev(v, np.float32) for v in xa])
    p2.setpts_from(p1)
    p1.setpts(*[_dev(v, np.float32) for v in xb])   # p1 moves to new points; p2 keeps xa
    ga = p2.execute(_dev(f, np.complex64)).cpu().numpy().ravel()
    p1.close()                                       # p2's points stay alive
    gb = p2.execute(_dev(f, np.complex64)).cpu().numpy().ravel()
    assert p2.status() == 0
    p2.close()
    ref = oracle_mod.direct_type2([v.astype(np.float64) for v in xa], f, -1, Ns)
    assert oracle_mod.rel_l2(ga, ref) <= 10 * eps
    assert np.array_equal(ga, gb)


def test_incompatible_or_unset_source_is_refused(pkg):
    import torch
    p1 = pkg.Plan(1, [16, 16], eps=1e-5, dtype=torch.complex64, device="cuda:0")
    p2 = pkg.Plan(2, [16, 16], eps=1e-5, dtype=torch.complex64, device="cuda:0")
    assert pkg.nufft_setpts_from(p2._h, p1._h) == -6          # p1 has no points yet
    p1.setpts(_dev(np.zeros(10), np.float32), _dev(np.zeros(10), np.float32))
    for other in (pkg.Plan(2, [32, 16], eps=1e-5, dtype=torch.complex64, device="cuda:0"),   # another grid
                  pkg.Plan(2, [16, 16], eps=1e-5, dtype=torch.complex128, device="cuda:0"),  # another precision
                  pkg.Plan(2, [16, 16], eps=1e-5, dtype=torch.complex64, device="cuda:0", max_subprob=256)):
        assert pkg.nufft_setpts_from(other._h, p1._h) == -1
        other.close()
    assert pkg.nufft_setpts_from(p2._h, p1._h) == 0
    assert pkg.nufft_setpts_from(None, p1._h) == -1
    for p in (p1, p2):
        p.close()
