"""GPU parity of the type-3 transform (Eq. (3), Sec. 3.3) against the CPU oracle.

Bars, over the whole output vector:
  * against O1 (the exact sum Eq. (3)): relative l2 error <= 10 eps (the
    Remark after step 3: eps in steps 1 and 2 gives an overall error near eps);
  * against O2 (the oracle's Sec. 3.3 algorithm at the same w, beta, n_i,
    gamma_i): they differ only by rounding.  fp64: 1e-12.  fp32: the dilated
    sources x' and rescaled targets s'' are rounded to float (|x'|, |s''| <= pi,
    so by up to 2^-24 pi), which moves the phase of grid frequency l by up to
    |l| 2^-24 pi with |l| <= n_i / 2; the budget is 3e-5 (the type-1/2 chain)
    plus that phase error at the largest n_i.
The plan's step-0 choices (n_i, gamma_i, w, beta) must equal the oracle's.
"""
import math

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


def same_budget(cdtype, ns):
    if cdtype == np.complex128:
        return 1e-12
    return 3e-5 + 2.0 * (max(ns) / 2) * math.pi * 2.0 ** -24


def run3(pkg, xs, ss, c, eps, isign, cdtype, plan=None, **opts):
    import torch
    dev = torch.device("cuda:0")
    tdt = torch.complex64 if cdtype == np.complex64 else torch.complex128
    rdt = np.float32 if cdtype == np.complex64 else np.float64
    own = plan is None
    p = plan if plan is not None else pkg.Plan3(len(xs), eps=eps, isign=isign, dtype=tdt, device=dev, **opts)
    p.setpts([torch.from_numpy(np.ascontiguousarray(v, dtype=rdt)).to(dev) for v in xs],
             [torch.from_numpy(np.ascontiguousarray(v, dtype=rdt)).to(dev) for v in ss])
    out = p.execute(torch.from_numpy(np.ascontiguousarray(c, dtype=cdtype)).to(dev)).cpu().numpy()
    info = dict(p.info)
    st = p.status()
    if own:
        p.close()
    assert st == 0, st
    return out, info


def inputs(d, M, N, X, S, cdtype, seed, kind="uniform"):
    rdt = np.float32 if cdtype == np.complex64 else np.float64
    xs = I.box_points(seed, M, [1.5 + 0.7 * i for i in range(d)], [X] * d, kind=kind, dtype=rdt)
    ss = I.box_points(seed + 1, N, [-4.0 + 3.0 * i for i in range(d)], [S] * d, kind=kind, dtype=rdt)
    c = I.complex_normal(seed + 2, M, dtype=cdtype)
    return xs, ss, c


# (d, M, N, X, S): grids of about 300, 90^2 and 36^3 cells at sigma = 2
CASES = [(1, 3000, 2500, 6.0, 40.0), (2, 6000, 5000, 5.0, 14.0), (3, 9000, 7000, 4.0, 6.5)]
PRECS = [(np.complex64, 1e-3), (np.complex64, 1e-5), (np.complex128, 1e-8), (np.complex128, 1e-11)]


@pytest.mark.parametrize("d,M,N,X,S", CASES)
@pytest.mark.parametrize("cdtype,eps", PRECS)
def test_type3_vs_exact_and_o2(pkg, oracle_mod, d, M, N, X, S, cdtype, eps):
    xs, ss, c = inputs(d, M, N, X, S, cdtype, 900 + d)
    for isign in (1, -1):
        f, info = run3(pkg, xs, ss, c, eps, isign, cdtype)
        P = oracle_mod.type3_params(eps, xs, ss)
        assert info["n"] == P["ns"] and info["w"] == P["w"]
        assert info["beta"] == pytest.approx(P["beta"], rel=1e-15)
        np.testing.assert_allclose(info["gamma"], P["gamma"], rtol=1e-14)
        e1 = oracle_mod.rel_l2(f, oracle_mod.direct_type3(xs, c, isign, ss))
        assert e1 <= 10 * eps, (isign, e1)
        e2 = oracle_mod.rel_l2(f, oracle_mod.type3(xs, c, isign, ss, eps))
        assert e2 <= same_budget(cdtype, P["ns"]), (isign, e2)


@pytest.mark.parametrize("cdtype,eps", [(np.complex64, 1e-5), (np.complex128, 1e-10)])
def test_type3_clustered(pkg, oracle_mod, cdtype, eps):
    xs, ss, c = inputs(3, 20000, 4000, 4.0, 6.5, cdtype, 950, kind="clustered")
    f, _ = run3(pkg, xs, ss, c, eps, 1, cdtype)
    assert oracle_mod.rel_l2(f, oracle_mod.direct_type3(xs, c, 1, ss)) <= 10 * eps


def test_type3_degenerate_boxes(pkg, oracle_mod):
    """X = 0 (all sources at one point), S = 0 (one target frequency), both, and one
    dimension degenerate while the others are not (gamma from Eq. (cond1))."""
    cd, eps = np.complex128, 1e-10
    rng = np.random.default_rng(960)
    c = I.complex_normal(961, 500, dtype=cd)
    spread_x = [rng.uniform(-3, 5, 500), rng.uniform(0, 2, 500)]
    spread_s = [rng.uniform(-9, 2, 300), rng.uniform(4, 6, 300)]
    point_x = [np.full(500, 1.25), np.full(500, -0.5)]
    point_s = [np.full(300, 3.5), np.full(300, -2.0)]
    mixed_x = [spread_x[0], np.full(500, 0.75)]
    mixed_s = [np.full(300, 7.0), spread_s[1]]
    for xs, ss in [(point_x, spread_s), (spread_x, point_s), (point_x, point_s), (mixed_x, mixed_s)]:
        f, _ = run3(pkg, xs, ss, c, eps, -1, cd)
        ref = oracle_mod.direct_type3(xs, c, -1, ss)
        assert oracle_mod.rel_l2(f, ref) <= 10 * eps


def test_type3_far_from_origin(pkg, oracle_mod):
    """Boxes centred far from 0: the translation (Eq. (trans)) keeps the grid small."""
    cd, eps = np.complex128, 1e-9
    rng = np.random.default_rng(970)
    xs = [rng.uniform(1000.0, 1003.0, 2000), rng.uniform(-500.0, -499.0, 2000)]
    ss = [rng.uniform(-2000.0, -1990.0, 1500), rng.uniform(300.0, 320.0, 1500)]
    c = I.complex_normal(971, 2000, dtype=cd)
    f, info = run3(pkg, xs, ss, c, eps, 1, cd)
    assert max(info["n"]) < 128
    assert oracle_mod.rel_l2(f, oracle_mod.direct_type3(xs, c, 1, ss)) <= 10 * eps


def test_type3_empty_and_reuse(pkg, oracle_mod):
    """M = 0 gives zeros; N = 0 runs; one plan re-used across point sets whose grids
    grow and shrink gives the results of fresh plans.  Not bit for bit: the order
    of points inside a bin (scatter cursors) differs between runs, hence the
    subproblems' fixed-point scales and the order of the grid's float reductions;
    the runs agree to the fp32 rounding budget."""
    import torch
    cd, eps = np.complex64, 1e-5
    dev = torch.device("cuda:0")
    p = pkg.Plan3(2, eps=eps, isign=1, dtype=torch.complex64, device=dev)
    xs, ss, c = inputs(2, 0, 100, 2.0, 5.0, cd, 980)
    f, _ = run3(pkg, xs, ss, c, eps, 1, cd, plan=p)
    assert f.shape == (100,) and np.all(f == 0)
    xs, ss, c = inputs(2, 100, 0, 2.0, 5.0, cd, 981)
    f, _ = run3(pkg, xs, ss, c, eps, 1, cd, plan=p)
    assert f.shape == (0,)
    for seed, X, S in [(982, 2.0, 5.0), (983, 6.0, 20.0), (984, 1.0, 3.0)]:
        xs, ss, c = inputs(2, 3000, 2000, X, S, cd, seed)
        f, info = run3(pkg, xs, ss, c, eps, 1, cd, plan=p)
        g, info2 = run3(pkg, xs, ss, c, eps, 1, cd)
        assert info["n"] == info2["n"]
        assert oracle_mod.rel_l2(f, g) <= 3e-5
        assert oracle_mod.rel_l2(f, oracle_mod.direct_type3(xs, c, 1, ss)) <= 10 * eps
    p.close()


def test_type3_large_sampled(pkg, oracle_mod):
    """4e6 sources and 4e6 frequencies in 3D (a 128^3 grid); 64 sampled outputs
    against the exact sum over all sources."""
    import torch
    cd, eps = np.complex64, 1e-5
    xs, ss, c = inputs(3, 4_000_000, 4_000_000, 3.0 * math.pi, 10.0, cd, 990)
    f, info = run3(pkg, xs, ss, c, eps, 1, cd)
    assert min(info["n"]) >= 120
    idx = np.random.default_rng(991).choice(len(f), 64, replace=False)
    ref = oracle_mod.direct_type3(xs, c, 1, [v[idx] for v in ss])
    assert oracle_mod.rel_l2(f[idx], ref) <= 10 * eps
    del torch


@pytest.mark.parametrize("opts", [{"kerevalmeth": 1}, {"kernel": 1}, {"kernel": 1, "kerevalmeth": 1},
                                  {"upsampfac": 1.25}])
def test_type3_plan_options(pkg, oracle_mod, opts):
    """The plan options reach both steps of type 3 (the spreading grid and the inner type 2):
    the piecewise polynomial kernel, the smooth cosh kernel, and sigma = 5/4 (n_i then follows
    Eq. (ng) with sigma = 5/4).  complex128, 2D, against the exact sum."""
    cd, eps = np.complex128, 1e-9
    xs, ss, c = inputs(2, 4000, 3000, 5.0, 14.0, cd, 995)
    f, info = run3(pkg, xs, ss, c, eps, 1, cd, **opts)
    sigma = opts.get("upsampfac", 2.0)
    P = oracle_mod.type3_params(eps, xs, ss, sigma=sigma)
    assert info["n"] == P["ns"] and info["w"] == P["w"]
    assert oracle_mod.rel_l2(f, oracle_mod.direct_type3(xs, c, 1, ss)) <= 10 * eps
