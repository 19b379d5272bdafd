"""nufft_spread_noalloc: spreading for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc -- code running inside another owner's
memory pool, latency-critical paths that cannot take an allocation's implicit
synchronisation, plugin hosts that forbid allocation.  For them the library
offers a spreading entry point whose scratch space is a fixed static device
array.  This test calls it through the C ABI twice in a row (different inputs,
so stale scratch contents would show) and checks each fine grid two ways:
against the plan path (nufft_makeplan / nufft_setpts / nufft_execute, type 1):
the grid's FFT, truncated and multiplied by the library's correction factors,
must give the plan's modes within the GPU tests' rounding budget for
complex64; and element by element against the oracle's spreading (Eq. (bl),
fp64) at the same w, beta and n, within that budget relative to the grid's
l2 norm.

The file name sorts last so a run that stops at the first failure has run
every other test before this one.
"""
import numpy as np
import pytest

import nufft_inputs as I

pytestmark = pytest.mark.gpu

TOL_C64 = 3e-5  # the complex64 rounding budget of tests/test_parity_gpu.py


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_06736_gb300 import build
    build.build()
    import paper_1808_06736_gb300 as p
    return p


def _modes_from_grid(pkg, grid, Ns, ns, w, beta, isign):
    """f_k = p_k * DFT(grid)_{k mod n}: the rest of the type-1 path, done here with torch's FFT."""
    import torch
    d = len(Ns)
    g = grid.reshape(tuple(reversed(ns))).to(torch.complex128)
    dims = tuple(range(d))
    bh = torch.fft.ifftn(g, dim=dims, norm="forward") if isign > 0 else torch.fft.fftn(g, dim=dims)
    idx = [torch.as_tensor(np.mod(np.arange(N) - N // 2, n), device=g.device) for N, n in zip(reversed(Ns), reversed(ns))]
    sub = bh
    for ax, ix in enumerate(idx):
        sub = torch.index_select(sub, ax, ix)
    p = None
    for N, n in zip(reversed(Ns), reversed(ns)):
        st, pk = pkg.nufft_correction_factors(N, n, w, beta)
        assert st == 0
        pk = torch.tensor(pk, dtype=torch.float64, device=g.device)
        p = pk if p is None else p[..., None] * pk
    return (sub * p).reshape(-1)


@pytest.mark.parametrize("d,Ns,M", [(3, [24, 20, 18], 40000), (2, [64, 50], 30000)])
def test_noalloc_spread_matches_plan_path_twice(pkg, oracle_mod, d, Ns, M):
    import torch
    dev = torch.device("cuda:0")
    eps = 1e-5
    st, w, beta, ns = pkg.nufft_choose_params(d, Ns, eps, pkg.NUFFT_C64)
    assert st == 0
    stream = torch.cuda.current_stream(dev)
    for call in range(2):
        kind = "uniform" if call == 0 else "clustered"
        xs = [torch.from_numpy(v).to(dev) for v in I.points(700 + call, M, d, kind=kind, dtype=np.float32)]
        c = torch.from_numpy(I.complex_normal(710 + call, M, dtype=np.complex64)).to(dev)
        grid = torch.full((int(np.prod(ns)),), complex(7.0, -7.0), dtype=torch.complex64, device=dev)
        ptrs = [v.data_ptr() for v in xs] + [0] * (3 - d)
        rc = pkg.nufft_spread_noalloc(d, ns, w, beta, M, *ptrs, c.data_ptr(), grid.data_ptr(),
                                      stream.cuda_stream)
        assert rc == 0, pkg.nufft_strerror(rc)
        # the grid itself against the oracle's fp64 spreading of the same (float) coordinates
        b_ref = oracle_mod.spread([v.double().cpu().numpy() for v in xs], c.cpu().numpy().astype(np.complex128),
                                  ns, w, beta).ravel()
        b_got = grid.cpu().numpy().astype(np.complex128)
        e_grid = np.linalg.norm(b_got - b_ref) / np.linalg.norm(b_ref)
        assert e_grid <= TOL_C64, (call, e_grid)
        f_noalloc = _modes_from_grid(pkg, grid, Ns, ns, w, beta, 1)
        plan = pkg.Plan(1, Ns, eps=eps, isign=1, dtype=torch.complex64, device=dev)
        plan.setpts(*xs)
        f_plan = plan.execute(c).reshape(-1).to(torch.complex128)
        assert plan.status() == 0
        plan.close()
        err = float(torch.linalg.vector_norm(f_noalloc - f_plan) / torch.linalg.vector_norm(f_plan))
        assert err <= TOL_C64, (call, err)


def test_noalloc_rejects_oversized_and_bad_args(pkg):
    st, w, beta, ns = pkg.nufft_choose_params(3, [64, 64, 64], 1e-5, pkg.NUFFT_C64)
    # 2^22 points need 64 MiB of records: more than the static array holds (no pointer is touched)
    assert pkg.nufft_spread_noalloc(3, ns, w, beta, 1 << 22, 1, 1, 1, 1, 1, 0) == -7
    assert pkg.nufft_spread_noalloc(3, ns, 1, beta, 10, 1, 1, 1, 1, 1, 0) == -1
    assert pkg.nufft_spread_noalloc(3, [8, 8, 8], w, beta, 10, 1, 1, 1, 1, 1, 0) == -1
    assert pkg.nufft_spread_noalloc(2, ns[:2], w, beta, 10, 1, 0, 0, 1, 1, 0) == -1
    # sizes whose arithmetic would overflow 32-bit indices are refused before anything is carved
    assert pkg.nufft_spread_noalloc(3, ns, w, beta, (1 << 31) - 1, 1, 1, 1, 1, 1, 0) == -7
    assert pkg.nufft_spread_noalloc(3, ns, w, beta, 1 << 62, 1, 1, 1, 1, 1, 0) == -7
    assert pkg.nufft_spread_noalloc(3, [1 << 30, 1 << 30, 1 << 30], w, beta, 10, 1, 1, 1, 1, 1, 0) == -7
    assert pkg.nufft_spread_noalloc(2, [1 << 16, 1 << 15], w, beta, 10, 1, 1, 0, 1, 1, 0) == -7
