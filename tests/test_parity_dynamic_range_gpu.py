"""Type-1 parity when the strengths span many decades.

The spreading kernels accumulate each subproblem's tile in fixed point, scaled by the
subproblem's largest |c_j| (2^22 steps in complex64, 2^51 in complex128).  The regime that
choice changes is strengths of very different sizes in one subproblem, so these cases put
them there:
  * |c_j| log-uniform over 8 decades (10^-8 .. 1) with uniform phases, every subproblem
    holding points of all sizes;
  * one strength 1e6 times the others (re, im iid N(0, 1)) inside a cluster of points, so one
    bin holds the outlier among small strengths.
Checked element by element over the whole mode vector: against the exact sums Eq. (1)
(relative l2 <= 10 eps), against the plain algorithm at the same (w, beta, n) (relative l2
within the rounding budget of tests/test_parity_gpu.py), and mode by mode against that
algorithm: max_k |f~_k - f2_k| within the same budget times max_k |f_k|, so no single mode
loses the small strengths' share to the fixed-point rounding.
"""
import numpy as np
import pytest

import nufft_inputs as I

pytestmark = pytest.mark.gpu

TOL_SAME = {np.complex64: 3e-5, np.complex128: 1e-12}
SIZES = {1: ([600], 8000), 2: ([48, 40], 20000), 3: ([18, 16, 14], 30000)}
CASES = [(np.complex64, 1e-5), (np.complex128, 1e-11)]


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_06736_gb300 import build
    build.build()
    import paper_1808_06736_gb300 as p
    return p


def type1_gpu(pkg, Ns, xs, c, eps, cdtype):
    import torch
    dev = torch.device("cuda:0")
    tdt = torch.complex64 if cdtype == np.complex64 else torch.complex128
    rdt = np.float32 if cdtype == np.complex64 else np.float64
    p = pkg.Plan(1, Ns, eps=eps, isign=1, dtype=tdt, device=dev)
    p.setpts(*[torch.from_numpy(np.ascontiguousarray(v, dtype=rdt)).to(dev) for v in xs])
    out = p.execute(torch.from_numpy(np.ascontiguousarray(c, dtype=cdtype)).to(dev)).cpu().numpy().ravel()
    st = p.status()
    p.close()
    assert st == 0, st
    return out


def check(pkg, oracle_mod, d, xs, c, eps, cdtype):
    Ns, _ = SIZES[d]
    x64 = [np.asarray(v, dtype=np.float64) for v in xs]
    c64 = np.asarray(c, dtype=cdtype).astype(np.complex128)  # the strengths the GPU sees
    got = type1_gpu(pkg, Ns, xs, c, eps, cdtype).astype(np.complex128)
    w, beta, ns = oracle_mod.choose_params(eps, Ns)
    o2 = oracle_mod.type1(x64, c64, 1, Ns, w=w, beta=beta, ns=ns)
    o1 = oracle_mod.direct_type1(x64, c64, 1, Ns)
    e_o2 = oracle_mod.rel_l2(got, o2)
    e_o1 = oracle_mod.rel_l2(got, o1)
    e_max = np.max(np.abs(got - o2)) / np.max(np.abs(o1))
    assert e_o2 <= TOL_SAME[cdtype], ("O2", e_o2)
    assert e_o1 <= 10 * eps, ("O1", e_o1)
    assert e_max <= TOL_SAME[cdtype], ("O2 mode by mode", e_max)


@pytest.mark.parametrize("cdtype,eps", CASES)
@pytest.mark.parametrize("d", [1, 2, 3])
def test_strengths_over_eight_decades(pkg, oracle_mod, cdtype, eps, d):
    Ns, M = SIZES[d]
    rdt = np.float32 if cdtype == np.complex64 else np.float64
    xs = I.points(6100 + d, M, d, dtype=rdt)
    rng = I.rng(6110 + d)
    mag = 10.0 ** rng.uniform(-8.0, 0.0, size=M)
    c = (mag * np.exp(1j * rng.uniform(-np.pi, np.pi, size=M))).astype(cdtype)
    check(pkg, oracle_mod, d, xs, c, eps, cdtype)


@pytest.mark.parametrize("cdtype,eps", CASES)
@pytest.mark.parametrize("d", [1, 2, 3])
def test_one_large_outlier_among_small_strengths(pkg, oracle_mod, cdtype, eps, d):
    Ns, M = SIZES[d]
    rdt = np.float32 if cdtype == np.complex64 else np.float64
    xs = I.points(6200 + d, M, d, kind="clustered", dtype=rdt)
    c = I.complex_normal(6210 + d, M, dtype=np.complex128)
    # the point nearest the cluster centre: its bin is crowded with small strengths
    j = int(np.argmin(sum(np.asarray(v, dtype=np.float64) ** 2 for v in xs)))
    c[j] = 1e6 * (0.6 - 0.8j)
    check(pkg, oracle_mod, d, xs, c.astype(cdtype), eps, cdtype)
