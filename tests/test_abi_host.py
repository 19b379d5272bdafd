"""The C-ABI library loads, exports every symbol the header declares, and its
host-only parameter logic agrees with the oracle's (independent code).  No
device call is made."""
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in ("nufft_gb300.h", "nufft_serve.h")]


@pytest.fixture(scope="module")
def lib():
    from paper_1808_06736_gb300 import build
    build.build()
    import paper_1808_06736_gb300 as pkg
    return pkg


def _declared():
    text = "".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nufft[0-9]*_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    import ctypes
    names = _declared()
    assert len(names) >= 28
    so = ctypes.CDLL(lib.library_path())
    for n in names:
        assert hasattr(so, n), n


def test_strerror_and_defaults(lib):
    assert lib.nufft_strerror(0) == "success"
    assert "argument" in lib.nufft_strerror(-1)
    o = lib.nufft_default_opts()
    assert o.debug == 0 and o.modeord == 0 and o.bin_size[0] == 0


def test_choose_params_matches_oracle(lib, oracle_mod):
    for eps in [0.5, 1e-2, 1e-3, 1e-5, 1e-6, 1e-9, 1e-12, 1e-15, 1e-18]:
        for Ns in ([1000], [24, 17], [256, 256, 256], [1, 3, 7]):
            st, w, beta, n = lib.nufft_choose_params(len(Ns), Ns, eps, lib.NUFFT_C128)
            wo, bo, no = oracle_mod.choose_params(eps, Ns)
            assert (w, n) == (wo, no), (eps, Ns)
            assert beta == pytest.approx(bo, rel=1e-15)
            assert st == (1 if eps < 1e-15 else 0)
    st, *_ = lib.nufft_choose_params(3, [8, 8, 8], 1e-7, lib.NUFFT_C64)
    assert st == 1  # fp32 cannot deliver 1e-7


def test_choose_params_rejects_bad_args(lib):
    assert lib.nufft_choose_params(4, [8] * 3, 1e-6)[0] == -1
    assert lib.nufft_choose_params(2, [8, 0], 1e-6)[0] == -1
    assert lib.nufft_choose_params(1, [8], 0.0)[0] == -1
    assert lib.nufft_choose_params(1, [8], float("nan"))[0] == -1


def test_next235_matches_oracle(lib, oracle_mod):
    for m in list(range(1, 400)) + [1000, 1023, 2047, 5001, 123457]:
        assert lib.nufft_next235(m) == oracle_mod.next235(m)
    assert lib.nufft_next235(0) == -1


@pytest.mark.parametrize("w", [2, 4, 6, 7, 10, 13, 16])
@pytest.mark.parametrize("N,n", [(1000, 2000), (255, 512), (7, 20), (3000, 6000)])
def test_correction_factors_match_oracle(lib, oracle_mod, w, N, n):
    """Library: Newton GL nodes + phase winding.  Oracle: numpy leggauss + direct cosines."""
    beta = 2.30 * w
    st, p = lib.nufft_correction_factors(N, n, w, beta)
    assert st == 0
    ref = oracle_mod.correction_factors(N, n, w, beta)
    np.testing.assert_allclose(np.array(p), ref, rtol=1e-12, atol=0)


def test_make_plan_validates_before_device_use(lib):
    # argument errors are reported without touching a device
    assert lib.nufft_makeplan(3, 1, [8], 1, 1, 1e-6, 1, None, None)[0] == -1
    assert lib.nufft_makeplan(1, 1, [8], 0, 1, 1e-6, 1, None, None)[0] == -1
    assert lib.nufft_makeplan(1, 1, [8], 1, 0, 1e-6, 1, None, None)[0] == -1
    assert lib.nufft_makeplan(1, 1, [8], 1, 1, -1.0, 1, None, None)[0] == -1
    assert lib.nufft_makeplan(1, 1, [8], 1, 1, 1e-6, 3, None, None)[0] == -1
    assert lib.nufft_setpts(None, 10, 0, 0, 0) == -1
    assert lib.nufft_execute(None, 0, 0) == -1
    assert lib.nufft_destroy(None) == 0


def test_type3_and_peaks_validate_before_device_use(lib):
    # type 3: dimension, sign, tolerance and precision are checked before any device call
    assert lib.nufft3_makeplan(0, 1, 1e-6, 1, None, None)[0] == -1
    assert lib.nufft3_makeplan(4, 1, 1e-6, 1, None, None)[0] == -1
    assert lib.nufft3_makeplan(2, 0, 1e-6, 1, None, None)[0] == -1
    assert lib.nufft3_makeplan(2, 1, -1.0, 1, None, None)[0] == -1
    assert lib.nufft3_makeplan(2, 1, 1e-6, 7, None, None)[0] == -1
    assert lib.nufft3_setpts(None, 10, 0, 0, 0, 10, 0, 0, 0) == -1
    assert lib.nufft3_execute(None, 0, 0) == -1
    assert lib.nufft3_plan_info(None, 2)[0] == -1
    assert lib.nufft3_get_status(None) == -1
    assert lib.nufft3_destroy(None) == 0
    # the peak microbenchmarks need room for four figures
    import ctypes
    assert lib._L().nufft_measure_peaks(None, None, 4) == -1
    buf = (ctypes.c_double * 2)()
    assert lib._L().nufft_measure_peaks(None, buf, 2) == -1


def test_tune_candidates_host_only(lib):
    for d, default in ((1, (1024, 1, 1)), (2, (32, 32, 1)), (3, (16, 8, 8))):
        for prec in (lib.NUFFT_C64, lib.NUFFT_C128):
            n, shapes = lib.nufft_tune_candidates(d, prec, 6)
            assert n == len(shapes) and n >= 5
            assert default in shapes
            for b in shapes:
                assert all(v == 1 for v in b[d:])
                if d == 1:
                    assert 256 <= b[0] <= 4096
                elif d == 2:
                    assert all(8 <= v <= 64 for v in b[:2])
                else:
                    assert all(4 <= v <= 32 for v in b) and b[0] >= b[1] >= b[2]
    # wider kernels leave fewer tiles that fit in shared memory
    assert lib.nufft_tune_candidates(3, lib.NUFFT_C128, 16)[0] < lib.nufft_tune_candidates(3, lib.NUFFT_C64, 2)[0]
    assert lib.nufft_tune_candidates(4, lib.NUFFT_C64, 6)[0] == -1
    assert lib.nufft_tune_candidates(2, lib.NUFFT_C64, 17)[0] == -1


def test_choose_params_sigma54_matches_oracle(lib, oracle_mod):
    for eps in [0.1, 1e-2, 3e-3, 1e-3, 1e-4, 1e-5, 2e-6, 1e-6, 1e-7, 1e-8, 1e-9]:
        for Ns in ([1], [7], [100], [256], [1000, 3], [64, 64, 64], [33, 17, 250]):
            st, w, beta, ns = lib.nufft_choose_params_sigma(len(Ns), Ns, eps, lib.NUFFT_C128, 1.25)
            ow, obeta, ons = oracle_mod.choose_params(eps, Ns, 1.25)
            assert st >= 0 and w == ow and abs(beta - obeta) < 1e-12 * obeta and ns == ons, (eps, Ns)
    # sigma = 2 through the same entry point is the paper's rule
    assert lib.nufft_choose_params_sigma(3, [64] * 3, 1e-5, lib.NUFFT_C64, 2.0)[1:] == \
        lib.nufft_choose_params(3, [64] * 3, 1e-5, lib.NUFFT_C64)[1:]
    # rounding amplified by rmax^dim (Eq. (rmax)) beyond eps: warning (complex64 3D at 1e-4, not at 1e-3;
    # complex128 3D at 1e-9, not at 1e-6)
    assert lib.nufft_choose_params_sigma(3, [64] * 3, 1e-3, lib.NUFFT_C64, 1.25)[0] == 0
    assert lib.nufft_choose_params_sigma(3, [64] * 3, 1e-4, lib.NUFFT_C64, 1.25)[0] == 1
    assert lib.nufft_choose_params_sigma(1, [64], 1e-5, lib.NUFFT_C64, 1.25)[0] == 0
    assert lib.nufft_choose_params_sigma(3, [64] * 3, 1e-6, lib.NUFFT_C128, 1.25)[0] == 0
    assert lib.nufft_choose_params_sigma(3, [64] * 3, 1e-9, lib.NUFFT_C128, 1.25)[0] == 1
    # w > 16 needed: warning, w clamped; any other sigma: bad argument
    st, w, _, _ = lib.nufft_choose_params_sigma(1, [100], 1e-11, lib.NUFFT_C128, 1.25)
    assert st == 1 and w == 16
    assert lib.nufft_choose_params_sigma(1, [100], 1e-5, lib.NUFFT_C64, 1.5)[0] == -1


def _eps_of_width(oracle_mod, w, sigma):
    if sigma == 2.0:
        return 10.0 ** (1 - w)
    return 10.0 ** (-(w - oracle_mod.SIGMA_54_OFFSET) / oracle_mod.eserr_slope(sigma))


@pytest.mark.parametrize("sigma", [2.0, 1.25])
def test_horner_coeffs_against_kernel_and_oracle(lib, oracle_mod, sigma):
    """The library's Sec. 5.3 table (Chebyshev interpolation) against the ES kernel: max error
    <= eps / 10 for the tolerance that selects w (floor 1e-14); and against the oracle's own fit
    (complex-square Vandermonde, a different method) to within the sum of their bounds."""
    z = np.linspace(-1, 1, 3001)
    for w in range(2, 17):
        beta = oracle_mod.es_beta(w, sigma)
        st, C = lib.nufft_horner_coeffs(w, beta)
        assert st == 0
        C = np.asarray(C)
        assert C.shape == (w, w + 4)
        mine = oracle_mod.piecewise_eval(C, w, z)
        err = np.abs(mine - oracle_mod.es_kernel(z, beta)).max()
        eps_w = _eps_of_width(oracle_mod, w, sigma)
        assert err <= max(0.1 * eps_w, 1e-14), (w, err)
        theirs = oracle_mod.piecewise_eval(oracle_mod.piecewise_poly(w, beta), w, z)
        assert np.abs(mine - theirs).max() <= max(0.6 * eps_w, 2e-14)


def test_horner_coeffs_rejects_bad_args(lib):
    assert lib.nufft_horner_coeffs(1, 5.0)[0] == -1
    assert lib.nufft_horner_coeffs(17, 5.0)[0] == -1
    assert lib.nufft_horner_coeffs(6, 0.0)[0] == -1


def test_setpts_from_rejects_null_plans(lib):
    """nufft_setpts_from checks its plan arguments before any device work."""
    import ctypes
    assert lib.nufft_setpts_from(ctypes.c_void_p(0), ctypes.c_void_p(0)) == -1
