"""GPU parity of the complex128 spread that accumulates in 32-bit fixed-point words.

The complex128 spread of kernel widths w <= 12 forms each contribution c_j psi in double-float
arithmetic and adds it to the shared tile as three 32-bit integer words; a subproblem of more
than 512 points runs in chunks of 512, each flushed on its own, so that no word's sum can leave
int32.  Widths w >= 13 keep 64-bit words.  These cases exercise what the other parity tests
leave out:
  * subproblems of 2048 and 700 points (clustered points, max_subprob raised), i.e. four full
    chunks, and one full chunk plus a ragged one;
  * w = 12 (the widest width on 32-bit words, eps = 1e-11) and w = 13 (eps = 1e-12, 64-bit words);
  * blocks of 512 threads (3D, one block per SM) and of 256 threads (2D, two blocks per SM).
Bars: relative l2 <= 10 eps against the exact sums Eq. (1), and within the fp64 rounding
budget (1e-12) against the plain algorithm at the same (w, beta, n), element by element over
the whole mode vector.
"""
import numpy as np
import pytest

import nufft_inputs as I

pytestmark = pytest.mark.gpu

TOL_SAME = 1e-12


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_06736_gb300 import build
    build.build()
    import paper_1808_06736_gb300 as p
    return p


def type1(pkg, Ns, xs, c, eps, **opts):
    import torch
    dev = torch.device("cuda:0")
    p = pkg.Plan(1, Ns, eps=eps, isign=1, dtype=torch.complex128, device=dev, **opts)
    p.setpts(*[torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).to(dev) for v in xs])
    out = p.execute(torch.from_numpy(np.ascontiguousarray(c, dtype=np.complex128)).to(dev)).cpu().numpy().ravel()
    st, info = p.status(), p.info
    p.close()
    assert st == 0, st
    return out, info


def check(pkg, oracle_mod, Ns, xs, c, eps, **opts):
    got, info = type1(pkg, Ns, xs, c, eps, **opts)
    w, beta, ns = oracle_mod.choose_params(eps, Ns)
    assert info["w"] == w and list(info["n"]) == list(ns)
    o2 = oracle_mod.type1(xs, c, 1, Ns, w=w, beta=beta, ns=ns)
    o1 = oracle_mod.direct_type1(xs, c, 1, Ns)
    assert oracle_mod.rel_l2(got, o2) <= TOL_SAME, ("O2", oracle_mod.rel_l2(got, o2))
    assert oracle_mod.rel_l2(got, o1) <= 10 * eps, ("O1", oracle_mod.rel_l2(got, o1))
    return info


@pytest.mark.parametrize("maxsub", [2048, 700])
@pytest.mark.parametrize("d,Ns,M", [(1, [400], 20000), (2, [40, 36], 30000), (3, [18, 16, 14], 40000)])
def test_chunked_subproblems(pkg, oracle_mod, maxsub, d, Ns, M):
    """Clustered points fill bins beyond 512 points, so subproblems of up to maxsub points run
    in several chunks."""
    xs = I.points(7100 + d, M, d, kind="clustered", dtype=np.float64)
    c = I.complex_normal(7110 + d, M, dtype=np.complex128)
    check(pkg, oracle_mod, Ns, xs, c, 1e-9, max_subprob=maxsub)


@pytest.mark.parametrize("eps", [1e-11, 1e-12])
@pytest.mark.parametrize("d,Ns,M", [(2, [48, 40], 20000), (3, [20, 18, 14], 30000)])
def test_widest_words_and_int64_words(pkg, oracle_mod, eps, d, Ns, M):
    """eps = 1e-11 gives w = 12, the widest kernel on 32-bit words; eps = 1e-12 gives w = 13, on
    64-bit words."""
    xs = I.points(7200 + d, M, d, dtype=np.float64)
    c = I.complex_normal(7210 + d, M, dtype=np.complex128)
    check(pkg, oracle_mod, Ns, xs, c, eps)


def test_one_and_two_blocks_per_sm(pkg, oracle_mod):
    """3D at w = 10 takes 16x8x8 bins, whose six-word tile (213 KB) fits one 512-thread block
    per SM; forced 8x8x4 bins take two 256-thread blocks.  Same points, both against the
    oracle and against each other."""
    Ns, M = [24, 20, 18], 60000
    xs = I.points(7300, M, 3, dtype=np.float64)
    c = I.complex_normal(7301, M, dtype=np.complex128)
    info = check(pkg, oracle_mod, Ns, xs, c, 1e-9)
    assert info["bins"] == [16, 8, 8]
    info2 = check(pkg, oracle_mod, Ns, xs, c, 1e-9, bin_size=(8, 8, 4))
    assert info2["bins"] == [8, 8, 4]
    a, _ = type1(pkg, Ns, xs, c, 1e-9)
    b, _ = type1(pkg, Ns, xs, c, 1e-9, bin_size=(8, 8, 4))
    assert oracle_mod.rel_l2(a, b) <= TOL_SAME
