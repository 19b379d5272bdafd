"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every check compares the oracle with something other than itself: numpy's
FFT (the uniform-point special case of Eq. (1)), scipy's adaptive quadrature
and the Kaiser-Bessel closed form Eq. (KBhat) (for the Gauss-Legendre rule of
Eq. (quad)), the asymptotic form Eq. (EShat1), values the paper prints
(tests/golden/paper_parameters.txt), the exact adjoint relation of Sec. 4.1,
the heuristic error level of Remark r:heur, and brute force on tiny inputs.
The last tests plant mistakes in the oracle and check the pins catch them.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, special

import nufft_inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.txt")


def _golden():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(line.split())
    return rows


def _es_ft_adaptive(beta, xi):
    """phi^(xi) by scipy's adaptive quadrature (independent of the GL rule)."""
    f = lambda z: math.exp(beta * (math.sqrt(max(1.0 - z * z, 0.0)) - 1.0)) * math.cos(xi * z)
    return 2.0 * integrate.quad(f, 0.0, 1.0, epsabs=0.0, epsrel=1e-12, limit=800)[0]


# ------------------------------------------------------------ parameters
def test_width_golden(oracle_mod):
    rows = [r for r in _golden() if r[0] == "width"]
    assert len(rows) == 3
    for _, eps, w, *_ in rows:
        assert oracle_mod.kernel_width(float(eps)) == int(w), (eps, w)


def test_beta_golden(oracle_mod):
    (row,) = [r for r in _golden() if r[0] == "beta_w"]
    w, beta = int(row[1]), float(row[2])
    assert abs(oracle_mod.es_beta(w) - beta) < 0.5


def test_gamma_golden(oracle_mod):
    # Eq. (gam): beta = gamma pi w (1 - 1/(2 sigma)), sigma = 2
    for row in [r for r in _golden() if r[0] == "gamma"]:
        factor, gamma = float(row[1]), float(row[2])
        assert abs(factor / (math.pi * (1 - 1 / 4.0)) - gamma) < 1e-3
    # the oracle's beta/w is the 2.30 factor
    assert oracle_mod.es_beta(10) / 10 == pytest.approx(2.30)


def test_grid_golden(oracle_mod):
    (row,) = [r for r in _golden() if r[0] == "grid"]
    N, w, n = int(row[1]), int(row[2]), int(row[3])
    assert oracle_mod.fine_grid_size(N, w) == n


def test_next235_against_enumeration(oracle_mod):
    # all 2^a 3^b 5^c up to 5000, built by products (not by factoring)
    vals = sorted({2 ** a * 3 ** b * 5 ** c for a in range(13) for b in range(9) for c in range(7)
                   if 2 ** a * 3 ** b * 5 ** c <= 5000})
    for m in list(range(1, 700)) + [999, 1000, 1001, 2047, 2049, 4000]:
        expect = min(v for v in vals if v >= m)
        assert oracle_mod.next235(m) == expect, m


def test_eps_guard(oracle_mod):
    # A4 reading: rounding in log10 must not push eps = 1e-k to the next width
    for k in range(1, 15):
        assert oracle_mod.kernel_width(10.0 ** (-k)) == min(k + 1, 16)
    assert oracle_mod.kernel_width(0.99e-5) == 7
    assert oracle_mod.kernel_width(1e-20) == 16
    assert oracle_mod.kernel_width(0.5) == 2


# --------------------------------------------------- kernel transform
@pytest.mark.parametrize("w", [2, 3, 4, 5, 6, 7, 8, 10, 13, 16])
def test_kernel_ft_vs_adaptive_quadrature(oracle_mod, w):
    """Sec. 3.1.1: p >= 1.5 w + 2 nodes give errors below eps = 10^-(w-1) for |k| <= N/2."""
    beta = oracle_mod.es_beta(w)
    xi = np.linspace(0.0, math.pi * w / 4.0, 7)  # alpha k for |k| <= N/2 with n = 2N
    gl = oracle_mod.kernel_ft(xi, w, beta)
    ref = np.array([_es_ft_adaptive(beta, v) for v in xi])
    err = np.max(np.abs(gl - ref) / np.abs(ref))
    assert err < max(10.0 ** (-(w - 1)), 1e-14), err  # 1e-14: double rounding floor


@pytest.mark.parametrize("w", [4, 6, 10, 16])
def test_kernel_ft_rule_on_kaiser_bessel(oracle_mod, w):
    """The same rule applied to the KB kernel Eq. (KB) reproduces its closed form Eq. (KBhat)."""
    beta = oracle_mod.es_beta(w)
    kb = lambda z: special.i0(beta * np.sqrt(np.maximum(1.0 - z * z, 0.0))) / special.i0(beta)
    xi = np.linspace(0.0, math.pi * w / 4.0, 9)  # the range |k| <= N/2 needs
    s = np.sqrt(beta ** 2 - xi ** 2)
    closed = 2.0 / special.i0(beta) * np.sinh(s) / s
    got = oracle_mod.kernel_ft(xi, w, beta, kernel=kb)
    assert np.max(np.abs(got - closed) / closed) < 1e-10


@pytest.mark.parametrize("w", [4, 8, 12, 16])
def test_kernel_ft_asymptotic(oracle_mod, w):
    """Eq. (EShat1): phi^(rho beta) ~ sqrt(2 pi / beta) (1 - rho^2)^(-3/4) e^{beta (sqrt(1-rho^2) - 1)} [1 + O(1/beta)]."""
    beta = oracle_mod.es_beta(w)
    for rho in (0.0, 0.3, 0.6):
        got = oracle_mod.kernel_ft([rho * beta], w, beta)[0]
        asy = math.sqrt(2 * math.pi / beta) * (1 - rho ** 2) ** -0.75 * math.exp(beta * (math.sqrt(1 - rho ** 2) - 1))
        rel = abs(got - asy) / got
        assert rel * beta < 1.0, (rho, rel)
        assert rel * beta > 0.1  # the O(1/beta) term is really there (not an accidental match)


def test_correction_factor_definition(oracle_mod):
    """Eq. (pk1): p_k = h / psi^(k), with psi^(k) = alpha phi^(alpha k) and phi^ from adaptive quadrature."""
    N, n, w = 40, 80, 6
    beta = oracle_mod.es_beta(w)
    p = oracle_mod.correction_factors(N, n, w, beta)
    h, alpha = 2 * math.pi / n, math.pi * w / n
    for m in (0, 7, 20, 39):
        k = m - N // 2
        ref = h / (alpha * _es_ft_adaptive(beta, alpha * k))
        assert p[m] == pytest.approx(ref, rel=1e-8)


# -------------------------------------------------------- O1 direct sums
@pytest.mark.parametrize("N", [16, 15])
@pytest.mark.parametrize("isign", [1, -1])
def test_direct_type1_is_dft_on_uniform_points(oracle_mod, N, isign):
    """Sec. 1: with x_j = 2 pi j / M and M = N, Eq. (1) is a DFT."""
    x = 2 * math.pi * np.arange(N) / N
    c = I.complex_normal(11, N)
    f = oracle_mod.direct_type1([x], c, isign, [N])
    ref = np.fft.ifft(c) * N if isign > 0 else np.fft.fft(c)
    k = oracle_mod.mode_range(N)
    np.testing.assert_allclose(f, ref[np.mod(k, N)], rtol=0, atol=1e-11 * np.abs(ref).max())


@pytest.mark.parametrize("isign", [1, -1])
def test_direct_type2_is_dft_on_uniform_points_2d(oracle_mod, isign):
    """Eq. (2) on a tensor grid of points equals a 2D DFT; N1 != N2 catches transposed axes."""
    N1, N2 = 8, 5
    j1, j2 = np.meshgrid(np.arange(N1), np.arange(N2), indexing="xy")
    x = (2 * math.pi * j1 / N1).ravel()
    y = (2 * math.pi * j2 / N2).ravel()
    f = I.complex_normal(12, N1 * N2)
    c = oracle_mod.direct_type2([x, y], f, isign, [N1, N2])
    # place f (k1 fastest, increasing k) into FFT order, axes (k2, k1)
    F = np.zeros((N2, N1), dtype=complex)
    K1, K2 = np.meshgrid(oracle_mod.mode_range(N1), oracle_mod.mode_range(N2), indexing="xy")
    F[np.mod(K2, N2), np.mod(K1, N1)] = f.reshape(N2, N1)
    ref = np.fft.ifft2(F) * (N1 * N2) if isign > 0 else np.fft.fft2(F)
    np.testing.assert_allclose(c, ref.ravel(), rtol=0, atol=1e-11 * np.abs(ref).max())


def test_direct_type1_3d_matches_fftn(oracle_mod):
    N = (4, 6, 5)
    g = np.meshgrid(*[np.arange(n) for n in reversed(N)], indexing="ij")
    xs = [(2 * math.pi * g[2 - i] / N[i]).ravel() for i in range(3)]
    c = I.complex_normal(13, int(np.prod(N)))
    f = oracle_mod.direct_type1(xs, c, -1, list(N))
    C = c.reshape(tuple(reversed(N)))
    ref = np.fft.fftn(C)
    idx = np.ix_(*[np.mod(oracle_mod.mode_range(n), n) for n in reversed(N)])
    np.testing.assert_allclose(f, ref[idx].ravel(), rtol=0, atol=1e-11 * np.abs(ref).max())


def test_direct_adjoint(oracle_mod):
    """Sec. 1: type 2 with sign -s is the adjoint of type 1 with sign s."""
    N = [5, 4, 3]
    xs = I.points(21, 17, 3)
    c = I.complex_normal(22, 17)
    f = I.complex_normal(23, 60)
    a = np.vdot(f, oracle_mod.direct_type1(xs, c, 1, N))
    b = np.vdot(oracle_mod.direct_type2(xs, f, -1, N), c)
    assert abs(a - b) < 1e-12 * abs(a)


def test_direct_type1_mode_subset(oracle_mod):
    N = [6, 5]
    xs = I.points(24, 30, 2)
    c = I.complex_normal(25, 30)
    full = oracle_mod.direct_type1(xs, c, 1, N)
    k = np.array([[-3, -2], [2, 2], [0, 0], [1, -1]])
    sub = oracle_mod.direct_type1(xs, c, 1, N, modes=k)
    np.testing.assert_allclose(sub, full[oracle_mod.mode_index(k, N)], rtol=1e-13, atol=1e-13)


def test_direct_large_point_split_path(oracle_mod):
    """The few-modes / many-points branch of the type-1 sum agrees with the per-mode branch."""
    xs = I.points(26, 20000, 3)
    c = I.complex_normal(27, 20000)
    k = np.array([[1, 2, 3], [-4, 0, 5]])
    a = oracle_mod.direct_type1(xs, c, 1, [8, 8, 12], modes=k)
    ph = np.outer(k[:, 0], xs[0]) + np.outer(k[:, 1], xs[1]) + np.outer(k[:, 2], xs[2])
    b = np.exp(1j * ph) @ c
    np.testing.assert_allclose(a, b, rtol=1e-11)


# ----------------------------------------------------------- O2 algorithm
CASES = [(1, [100], 300), (2, [24, 17], 400), (3, [12, 10, 9], 500)]


def _heuristic_eps_inf(oracle_mod, eps, Ns):
    """Remark r:heur: eps_inf ~ |psi^(n - N/2) / psi^(N/2)|, worst dimension (adaptive quadrature)."""
    w, beta, ns = oracle_mod.choose_params(eps, Ns)
    out = 0.0
    for N, n in zip(Ns, ns):
        a = math.pi * w / n
        out = max(out, abs(_es_ft_adaptive(beta, a * (n - N / 2)) / _es_ft_adaptive(beta, a * N / 2)))
    return out


@pytest.mark.parametrize("d,Ns,M", CASES)
@pytest.mark.parametrize("eps", [1e-3, 1e-5, 1e-9, 1e-12])
def test_o2_error_vs_truth(oracle_mod, d, Ns, M, eps):
    """Sec. 4.2: relative l2 error of the ES NUFFT tracks eps; within 10 eps and within the
    heuristic level eps_inf of Remark r:heur (between eps_inf/20 and 1.5 eps_inf)."""
    xs = I.points(1, M, d)
    c = I.complex_normal(2, M)
    f = I.complex_normal(3, int(np.prod(Ns)))
    heur = _heuristic_eps_inf(oracle_mod, eps, Ns)
    e1 = oracle_mod.rel_l2(oracle_mod.type1(xs, c, 1, Ns, eps=eps), oracle_mod.direct_type1(xs, c, 1, Ns))
    e2 = oracle_mod.rel_l2(oracle_mod.type2(xs, f, -1, Ns, eps=eps), oracle_mod.direct_type2(xs, f, -1, Ns))
    for e in (e1, e2):
        assert e <= 10 * eps
        assert heur / 20 < e < 1.5 * heur, (e, heur)


@pytest.mark.parametrize("d,Ns,M", CASES)
@pytest.mark.parametrize("isign", [1, -1])
def test_o2_adjoint_to_rounding(oracle_mod, d, Ns, M, isign):
    """Sec. 4.1: the discrete type-2 algorithm is the exact adjoint of the type-1 algorithm."""
    xs = I.points(4, M, d)
    c = I.complex_normal(5, M)
    f = I.complex_normal(6, int(np.prod(Ns)))
    w, beta, ns = oracle_mod.choose_params(1e-6, Ns)
    F1c = oracle_mod.type1(xs, c, isign, Ns, w=w, beta=beta, ns=ns)
    F2f = oracle_mod.type2(xs, f, -isign, Ns, w=w, beta=beta, ns=ns)
    a, b = np.vdot(f, F1c), np.vdot(F2f, c)
    assert abs(a - b) < 1e-12 * np.linalg.norm(f) * np.linalg.norm(F1c)


def test_o2_single_point(oracle_mod):
    """M = 1, c = 1: Eq. (1) gives f_k = exp(i k.x0); x0 = 0 gives f = 1."""
    Ns = [9, 8]
    for x0 in ([0.0, 0.0], [1.1, -2.7]):
        f = oracle_mod.type1([[x0[0]], [x0[1]]], [1.0 + 0j], 1, Ns, eps=1e-9)
        k = oracle_mod.mode_list(Ns)
        ref = np.exp(1j * (k[:, 0] * x0[0] + k[:, 1] * x0[1]))
        assert np.max(np.abs(f - ref)) < 1e-8


def test_o2_single_mode(oracle_mod):
    """f = delta_{k,k0}: Eq. (2) gives c_j = exp(i isign k0.x_j) at every point (O1 exactly, O2 to eps),
    for a mode at the Nyquist edge -N/2 and an interior one, both signs."""
    Ns = [10, 7]
    xs = I.points(60, 200, 2)
    modes = oracle_mod.mode_list(Ns)
    for k0 in ([-5, 3], [2, -1]):
        f = np.zeros(int(np.prod(Ns)), dtype=np.complex128)
        f[oracle_mod.mode_index(np.array([k0]), Ns)[0]] = 1.0
        assert np.array_equal(modes[oracle_mod.mode_index(np.array([k0]), Ns)[0]], k0)
        for isign in (1, -1):
            ref = np.exp(1j * isign * (k0[0] * xs[0] + k0[1] * xs[1]))
            np.testing.assert_allclose(oracle_mod.direct_type2(xs, f, isign, Ns), ref, rtol=0, atol=1e-13)
            assert np.max(np.abs(oracle_mod.type2(xs, f, isign, Ns, eps=1e-9) - ref)) < 1e-8


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("eps", [1e-4, 1e-10])
def test_o2_brute_force_tiny_with_edge_points(oracle_mod, d, eps):
    """N_i <= 8, M <= 12 with points on grid nodes, at -pi, just below pi and outside [-pi, pi)."""
    Ns = [8, 7, 6][:d]
    w, beta, ns = oracle_mod.choose_params(eps, Ns)
    xs, M = I.edge_points(d, ns)
    c = I.complex_normal(7, M)
    f = I.complex_normal(8, int(np.prod(Ns)))
    e1 = oracle_mod.rel_l2(oracle_mod.type1(xs, c, 1, Ns, eps=eps), oracle_mod.direct_type1(xs, c, 1, Ns))
    e2 = oracle_mod.rel_l2(oracle_mod.type2(xs, f, -1, Ns, eps=eps), oracle_mod.direct_type2(xs, f, -1, Ns))
    assert e1 <= 10 * eps and e2 <= 10 * eps, (e1, e2)


def test_o2_periodicity(oracle_mod):
    """Eq. (ppsi1): shifting every point by 2 pi leaves the transforms unchanged."""
    xs = I.points(9, 50, 2)
    c = I.complex_normal(10, 50)
    a = oracle_mod.type1(xs, c, 1, [10, 12], eps=1e-8)
    b = oracle_mod.type1([xs[0] + 2 * math.pi, xs[1] - 2 * math.pi], c, 1, [10, 12], eps=1e-8)
    assert oracle_mod.rel_l2(a, b) < 1e-12


# -------------------------------------------------- planted mistakes
def _err_t1(oracle_mod, Ns=(12, 10, 9), eps=1e-6):
    xs = I.points(31, 200, len(Ns))
    c = I.complex_normal(32, 200)
    return oracle_mod.rel_l2(oracle_mod.type1(xs, c, 1, list(Ns), eps=eps),
                             oracle_mod.direct_type1(xs, c, 1, list(Ns)))


def test_planted_mistakes_are_caught(oracle_mod, monkeypatch):
    base = _err_t1(oracle_mod)
    assert base < 1e-5
    # (a) a dropped factor 2/w in Eq. (pk1)
    orig_cf = oracle_mod.correction_factors
    monkeypatch.setattr(oracle_mod, "correction_factors", lambda N, n, w, b, k="es": orig_cf(N, n, w, b, k) * w / 2)
    assert _err_t1(oracle_mod) > 1e-1
    monkeypatch.setattr(oracle_mod, "correction_factors", orig_cf)
    # (b) the wrong DFT sign
    orig_dft = oracle_mod.dft
    monkeypatch.setattr(oracle_mod, "dft", lambda b, s: orig_dft(b, -s))
    assert _err_t1(oracle_mod) > 1e-1
    monkeypatch.setattr(oracle_mod, "dft", orig_dft)
    # (c) beta off by 10 percent (a mis-typed 2.30)
    orig_beta = oracle_mod.es_beta
    monkeypatch.setattr(oracle_mod, "es_beta", lambda w, sigma=2.0: 2.07 * w)
    assert _err_t1(oracle_mod) > 2 * base  # and test_beta_golden fails too
    monkeypatch.setattr(oracle_mod, "es_beta", orig_beta)
    # (d) each dimension's correction computed with another dimension's fine-grid size
    orig_outer = oracle_mod._outer_correction
    monkeypatch.setattr(oracle_mod, "_outer_correction",
                        lambda Ns, ns, w, b, k="es": orig_outer(Ns, list(ns)[::-1], w, b, k))
    assert _err_t1(oracle_mod) > 1e-3
    monkeypatch.setattr(oracle_mod, "_outer_correction", orig_outer)
    # (e) the nodes of a coordinate starting one cell late (ceil(u - w/2) + 1)
    orig_spread = oracle_mod.spread
    monkeypatch.setattr(oracle_mod, "spread",
                        lambda xs, c, ns, w, b, k="es": orig_spread(
                            [np.asarray(v) - 2 * math.pi / n for v, n in zip(xs, ns)], c, ns, w, b, k))
    assert _err_t1(oracle_mod) > 1e-1
    monkeypatch.setattr(oracle_mod, "spread", orig_spread)
    assert _err_t1(oracle_mod) == pytest.approx(base)


# ------------------------------------------------ upsampling factor sigma = 5/4
def test_eserr_slope_golden(oracle_mod):
    """The slope of Eq. (ESerr) that the sigma = 5/4 width rule uses, checked at sigma = 2
    against the value the paper prints."""
    (row,) = [r for r in _golden() if r[0] == "slope"]
    sigma, slope = float(row[1]), float(row[2])
    assert abs(oracle_mod.eserr_slope(sigma) - slope) < 1e-3
    # and Eq. (gam) with the same gamma gives the paper's 2.30
    assert abs(oracle_mod.GAMMA * math.pi * (1 - 1 / (2 * 2.0)) - 2.30) < 1e-3


@pytest.mark.parametrize("w", [4, 6, 9, 11, 13, 16])
def test_kernel_ft_at_sigma54_frequencies(oracle_mod, w):
    """The GL rule stays accurate up to the largest correction frequency at sigma = 5/4,
    alpha N/2 = pi w / (2 sigma) = 0.4 pi w, far below the tolerance that w serves."""
    beta = oracle_mod.es_beta(w, 1.25)
    xi = np.linspace(0.0, 0.4 * math.pi * w, 9)
    gl = oracle_mod.kernel_ft(xi, w, beta)
    ref = np.array([_es_ft_adaptive(beta, v) for v in xi])
    err = np.max(np.abs(gl - ref) / np.abs(ref))
    assert err < 1e-2 * 10.0 ** (-w / oracle_mod.eserr_slope(1.25)), err


def _heuristic_eps_inf_sigma(oracle_mod, eps, Ns, sigma):
    w, beta, ns = oracle_mod.choose_params(eps, Ns, sigma)
    out = 0.0
    for N, n in zip(Ns, ns):
        a = math.pi * w / n
        out = max(out, abs(_es_ft_adaptive(beta, a * (n - N / 2)) / _es_ft_adaptive(beta, a * N / 2)))
    return out


CASES54 = [(1, [200], 400), (2, [40, 33], 500), (3, [32, 28, 24], 600)]


@pytest.mark.parametrize("d,Ns,M", CASES54)
@pytest.mark.parametrize("eps", [1e-3, 1e-5, 1e-7, 1e-9])
def test_o2_sigma54_error_vs_truth(oracle_mod, d, Ns, M, eps):
    """sigma = 5/4 (reading R15: w from the slope of Eq. (ESerr) plus a calibrated offset, beta
    from Eq. (gam)): the error against the exact sums is within 10 eps, not far below eps
    (a grid or width mistake would overshoot), and within the heuristic level of Remark
    r:heur evaluated at this sigma."""
    xs = I.points(11, M, d)
    c = I.complex_normal(12, M)
    f = I.complex_normal(13, int(np.prod(Ns)))
    w, beta, ns = oracle_mod.choose_params(eps, Ns, 1.25)
    low = all(n < 2 * N for n, N in zip(ns, Ns))  # else 2w sets some n_i and the error drops further
    heur = _heuristic_eps_inf_sigma(oracle_mod, eps, Ns, 1.25)
    e1 = oracle_mod.rel_l2(oracle_mod.type1(xs, c, 1, Ns, w=w, beta=beta, ns=ns), oracle_mod.direct_type1(xs, c, 1, Ns))
    e2 = oracle_mod.rel_l2(oracle_mod.type2(xs, f, -1, Ns, w=w, beta=beta, ns=ns), oracle_mod.direct_type2(xs, f, -1, Ns))
    for e in (e1, e2):
        assert e <= 10 * eps, (e, eps)
        assert not low or e > eps / 100, (e, eps)
        assert heur / 20 < e < 1.5 * heur, (e, heur)


# ------------------------------------------------------------------ type 3
def test_direct_type3_integer_frequencies_equal_type1(oracle_mod):
    """Eq. (3) at integer frequencies is Eq. (1) at those modes (two independent code paths)."""
    rng = np.random.default_rng(31)
    xs = [rng.uniform(-math.pi, math.pi, 300) for _ in range(2)]
    c = I.complex_normal(32, 300)
    modes = rng.integers(-20, 20, size=(50, 2))
    for isign in (1, -1):
        f1 = oracle_mod.direct_type1(xs, c, isign, [40, 40], modes=modes)
        f3 = oracle_mod.direct_type3(xs, c, isign, [modes[:, 0].astype(float), modes[:, 1].astype(float)])
        np.testing.assert_allclose(f3, f1, rtol=0, atol=1e-11 * np.abs(f1).max())


def test_direct_type3_brute_force_and_translation(oracle_mod):
    """Tiny inputs against a dense exponential matrix, and the translation identity Eq. (trans)."""
    rng = np.random.default_rng(33)
    x = [rng.uniform(-3, 7, 9), rng.uniform(0, 2, 9), rng.uniform(-1, 1, 9)]
    s = [rng.uniform(-30, 5, 7), rng.uniform(-1, 1, 7), rng.uniform(10, 12, 7)]
    c = I.complex_normal(34, 9)
    ph = sum(np.outer(s[i], x[i]) for i in range(3))
    for isign in (1, -1):
        np.testing.assert_allclose(oracle_mod.direct_type3(x, c, isign, s), np.exp(1j * isign * ph) @ c,
                                   rtol=1e-12, atol=1e-12)
    x0, s0 = [0.3, -1.2, 2.0], [4.0, 0.5, -7.0]
    lhs = oracle_mod.direct_type3([x[i] + x0[i] for i in range(3)], c, 1, [s[i] + s0[i] for i in range(3)])
    pre = np.exp(1j * sum(s0[i] * x[i] for i in range(3)))
    post = np.exp(1j * sum((s[i] + s0[i]) * x0[i] for i in range(3)))
    np.testing.assert_allclose(lhs, post * oracle_mod.direct_type3(x, c * pre, 1, s), rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-9])
def test_type3_params_satisfy_the_paper_conditions(oracle_mod, eps):
    """Eq. (cond1): rescaled sources stay w/2 cells from +-pi; Eq. (cond2): gamma S <= n / (2 sigma)."""
    rng = np.random.default_rng(35)
    xs = [rng.uniform(-50, 10, 100), rng.uniform(3, 4, 100)]
    ss = [rng.uniform(-2, 9, 80), np.full(80, 5.0)]   # second dimension: all targets equal
    P = oracle_mod.type3_params(eps, xs, ss)
    for i in range(2):
        n, g, X, S, w = P["ns"][i], P["gamma"][i], P["X"][i], P["S"][i], P["w"]
        assert X / g <= math.pi * (1 - w / n) * (1 + 1e-12)
        assert g * S <= n / 4.0 * (1 + 1e-12)
        assert n >= 2 * w


T3_CASES = [(1, 600, 500), (2, 700, 600), (3, 800, 700)]


@pytest.mark.parametrize("d,M,N", T3_CASES)
@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-9])
def test_o2_type3_error_vs_truth(oracle_mod, d, M, N, eps):
    """Sec. 3.3's algorithm (O2) against the exact sum (O1): within 10 eps (the Remark after step 3:
    using eps in steps 1 and 2 gives an overall error close to eps) and not far below eps.
    Sources and targets are off-centre, so the translation of Eq. (trans) matters."""
    rng = np.random.default_rng(40 + d)
    xs = [rng.uniform(-2, 11, M) for _ in range(d)]
    ss = [rng.uniform(-25, 8, N) for _ in range(d)]
    c = I.complex_normal(41 + d, M)
    for isign in (1, -1):
        e = oracle_mod.rel_l2(oracle_mod.type3(xs, c, isign, ss, eps), oracle_mod.direct_type3(xs, c, isign, ss))
        assert eps / 100 < e <= 10 * eps, (isign, e)


# ------------------------------------------------ piecewise polynomial kernel
def _eps_of_width(oracle_mod, w, sigma):
    """Smallest tolerance that the width rule maps to w (10^(1 - w) at sigma = 2)."""
    if sigma == 2.0:
        return 10.0 ** (1 - w)
    return 10.0 ** (-(w - oracle_mod.SIGMA_54_OFFSET) / oracle_mod.eserr_slope(sigma))


def test_piecewise_poly_reproduces_polynomials(oracle_mod):
    """A kernel that is itself a polynomial of degree <= p is reproduced exactly (checks the
    interval centres, the local variable and the Vandermonde solve); degree p + 2 is not."""
    w = 7
    p = w + 3
    z = np.linspace(-1, 1, 1001)
    for deg, exact in ((p, True), (p - 4, True), (p + 2, False)):
        coef = np.random.default_rng(deg).standard_normal(deg + 1)
        poly = lambda v, c=coef: np.polynomial.polynomial.polyval(v, c)  # noqa: E731
        C = oracle_mod.piecewise_poly(w, 0.0, kernel=poly)
        err = np.abs(oracle_mod.piecewise_eval(C, w, z) - poly(z)).max()
        if exact:
            assert err < 1e-11, (deg, err)
        else:
            assert err > 1e-8, (deg, err)


@pytest.mark.parametrize("sigma", [2.0, 1.25])
def test_piecewise_poly_error_small_against_eps(oracle_mod, sigma):
    """Sec. 5.3: with p = w + 3 the approximation error is small relative to the tolerance that
    selects w: max |poly - ES| <= eps / 2 (floor 1e-14, double rounding), every w = 2..16."""
    z = np.linspace(-1, 1, 4001)
    for w in range(2, 17):
        beta = oracle_mod.es_beta(w, sigma)
        C = oracle_mod.piecewise_poly(w, beta)
        err = np.abs(oracle_mod.piecewise_eval(C, w, z) - oracle_mod.es_kernel(z, beta)).max()
        assert err <= max(0.5 * _eps_of_width(oracle_mod, w, sigma), 1e-14), (w, err)


def test_piecewise_poly_planted_mistakes(oracle_mod):
    """The error pin catches a reversed local variable and coefficients of the wrong interval."""
    w, sigma = 6, 2.0
    beta = oracle_mod.es_beta(w, sigma)
    z = np.linspace(-1, 1, 2001)
    C = oracle_mod.piecewise_poly(w, beta)
    ref = oracle_mod.es_kernel(z, beta)
    bound = 0.5 * _eps_of_width(oracle_mod, w, sigma)
    flipped = C * ((-1.0) ** np.arange(C.shape[1]))      # s -> -s
    rolled = np.roll(C, 1, axis=0)                         # interval t uses t - 1's polynomial
    for bad in (flipped, rolled):
        assert np.abs(oracle_mod.piecewise_eval(bad, w, z) - ref).max() > 100 * bound


# ------------------------------------------------ smooth (cosh) kernel variant
def test_cosh_kernel_closed_forms(oracle_mod):
    """Remark in Sec. 7: 2 e^-beta cosh(beta sqrt(1 - z^2)) = ES + e^{-beta (sqrt(1 - z^2) + 1)},
    so it lies within e^-beta of ES (the gap is largest at z = +-1), equals 1 + e^{-2 beta} at 0,
    and its derivative tends to the finite -2 beta^2 e^-beta z at the support's ends, where
    ES's derivative is unbounded."""
    beta = oracle_mod.es_beta(7)
    z = np.linspace(-1, 1, 2001)
    gap = oracle_mod.es_cosh_kernel(z, beta) - oracle_mod.es_kernel(z, beta)
    np.testing.assert_allclose(gap, np.exp(-beta * (np.sqrt(1 - z * z) + 1)), rtol=1e-9, atol=4e-15)  # the difference of two O(1) values
    assert gap.max() <= math.exp(-beta) * (1 + 1e-12)
    assert oracle_mod.es_cosh_kernel(np.array([0.0]), beta)[0] == pytest.approx(1 + math.exp(-2 * beta), rel=1e-15)
    h = 1e-7
    for z0 in (1 - 1e-6, 1 - 1e-9):
        fd = (oracle_mod.es_cosh_kernel(np.array([z0]), beta)[0]
              - oracle_mod.es_cosh_kernel(np.array([z0 - h]), beta)[0]) / h
        assert fd == pytest.approx(-2 * beta ** 2 * math.exp(-beta), rel=1e-3)
        fd_es = (oracle_mod.es_kernel(np.array([z0]), beta)[0]
                 - oracle_mod.es_kernel(np.array([z0 - h]), beta)[0]) / h
        assert abs(fd_es) > 10 * abs(fd)


@pytest.mark.parametrize("w", [2, 4, 6, 10, 16])
def test_cosh_kernel_ft_vs_adaptive_quadrature(oracle_mod, w):
    """The Gauss-Legendre rule of Eq. (quad) on the cosh kernel against scipy's adaptive quadrature."""
    beta = oracle_mod.es_beta(w)
    xi = np.linspace(0.0, math.pi * w / 4.0, 7)
    gl = oracle_mod.kernel_ft(xi, w, beta, kernel=oracle_mod.kernel_fn("cosh", beta))
    f = lambda z, x: 2 * math.exp(-beta) * math.cosh(beta * math.sqrt(max(1 - z * z, 0.0))) * math.cos(x * z)  # noqa: E731
    ref = np.array([2.0 * integrate.quad(f, 0.0, 1.0, args=(v,), epsabs=0.0, epsrel=1e-12, limit=800)[0]
                    for v in xi])
    assert np.max(np.abs(gl - ref) / np.abs(ref)) < max(10.0 ** (-(w - 1)), 1e-14)


@pytest.mark.parametrize("d,Ns,M", CASES)
@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-10])
def test_o2_cosh_error_vs_truth(oracle_mod, d, Ns, M, eps):
    """O2 with the cosh kernel (same w, beta) against the exact sums: within 10 eps, and within
    a few eps of O2 with ES (the kernels differ by at most e^-beta)."""
    xs = I.points(11, M, d)
    c = I.complex_normal(12, M)
    f = I.complex_normal(13, int(np.prod(Ns)))
    t1 = oracle_mod.type1(xs, c, 1, Ns, eps=eps, kernel="cosh")
    t2 = oracle_mod.type2(xs, f, -1, Ns, eps=eps, kernel="cosh")
    assert oracle_mod.rel_l2(t1, oracle_mod.direct_type1(xs, c, 1, Ns)) <= 10 * eps
    assert oracle_mod.rel_l2(t2, oracle_mod.direct_type2(xs, f, -1, Ns)) <= 10 * eps
    assert oracle_mod.rel_l2(t1, oracle_mod.type1(xs, c, 1, Ns, eps=eps)) <= 3 * eps


# ------------------------------------------------ aliasing error (Eq. (gkx), (epsest), (1nrm))
def _single_point_error(oracle_mod, N, n, w, beta, x):
    """g_k(x) of Eq. (gkx) for k in I_N, written as the finite sum it equals by Poisson summation:
    (h / psi^(k)) sum_l psi(l h - x) e^{i k l h} - e^{i k x}, psi(t) = phi(t / alpha), alpha = w h / 2,
    over the grid nodes l h within the kernel's support (numpy; independent of O2's C spreader)."""
    h = 2 * np.pi / n
    alpha = w * h / 2
    k = oracle_mod.mode_range(N)
    lo, hi = int(np.floor((x - alpha) / h)) - 1, int(np.ceil((x + alpha) / h)) + 1
    ls = np.arange(lo, hi + 1)
    psi = oracle_mod.es_kernel((ls * h - x) / alpha, beta)
    psihat = alpha * oracle_mod.kernel_ft(alpha * k, w, beta)
    s = (np.exp(1j * np.outer(k, ls * h)) * psi).sum(axis=1)
    return h / psihat * s - np.exp(1j * k * x)


def test_single_point_error_is_the_aliasing_sum(oracle_mod):
    """Sec. 4.1: for one point (c = 1) the type-1 error is g_k(x), Eq. (gkx); O2 (C spreading,
    scipy DFT, Eq. (pk1) correction) matches the finite-sum form of g_k to rounding, at points
    off, on and between grid nodes."""
    N, eps = 48, 1e-6
    w, beta, ns = oracle_mod.choose_params(eps, [N])
    n = ns[0]
    for x in (0.3, -2.1, 2 * np.pi / n * 5, 2 * np.pi / n * 5.5, np.pi - 1e-3):
        f2 = oracle_mod.type1([np.array([x])], np.array([1.0 + 0j]), 1, [N], w=w, beta=beta, ns=ns)
        g = _single_point_error(oracle_mod, N, n, w, beta, x)
        np.testing.assert_allclose(f2 - np.exp(1j * oracle_mod.mode_range(N) * x), g, rtol=0, atol=1e-13)
        assert np.abs(g).max() < 10 * eps


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-9])
def test_l1_linf_bound(oracle_mod, eps):
    """Eq. (1nrm): max_k |f~_k - f_k| <= eps_inf ||c||_1 and max_j |c~_j - c_j| <= eps_inf ||f||_1, with
    eps_inf of Eq. (epsest) = max over k and x of |g_k(x)| (g_k is h-periodic in x up to a phase, so
    x is sampled over one grid cell, 400 points, and the bound is taken 5 % above the sampled max);
    also eps_inf is within a factor 4 of the heuristic of Remark r:heur."""
    N = 64
    w, beta, ns = oracle_mod.choose_params(eps, [N])
    n = ns[0]
    h = 2 * np.pi / n
    eps_inf = max(np.abs(_single_point_error(oracle_mod, N, n, w, beta, x)).max()
                  for x in np.linspace(0, h, 400, endpoint=False))
    bound = 1.05 * eps_inf
    xs = I.points(50, 3000, 1)
    c = I.complex_normal(51, 3000)
    f = I.complex_normal(52, N)
    e1 = np.abs(oracle_mod.type1(xs, c, 1, [N], w=w, beta=beta, ns=ns) - oracle_mod.direct_type1(xs, c, 1, [N])).max()
    e2 = np.abs(oracle_mod.type2(xs, f, -1, [N], w=w, beta=beta, ns=ns) - oracle_mod.direct_type2(xs, f, -1, [N])).max()
    assert e1 <= bound * np.abs(c).sum()
    assert e2 <= bound * np.abs(f).sum()
    a = math.pi * w / n
    heur = abs(oracle_mod.kernel_ft([a * (n - N / 2)], w, beta)[0] / oracle_mod.kernel_ft([a * N / 2], w, beta)[0])
    assert heur / 4 < eps_inf < 4 * heur, (eps_inf, heur)


@pytest.mark.parametrize("d,ns", [(1, [40]), (2, [24, 12]), (3, [12, 16, 14])])
def test_threads_do_not_change_spread_or_interp(oracle_mod, d, ns):
    # the threaded spreading owns slabs of the last grid index and the threaded interpolation
    # splits the points; both must give the single-thread results bit for bit, also with more
    # threads than slabs (empty slabs) and with points whose stencil wraps around the grid
    rng = np.random.default_rng(77 + d)
    M = 3000
    xs = [rng.uniform(-np.pi, np.pi, M) for _ in range(d)]
    xs[0][:4] = [-np.pi, np.pi - 1e-12, 0.0, 3 * np.pi - 1e-9]
    c = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    w, beta = 6, 13.8
    b = (rng.standard_normal(int(np.prod(ns))) + 1j * rng.standard_normal(int(np.prod(ns)))).reshape(
        tuple(reversed(ns)))
    n0 = oracle_mod.num_threads()
    try:
        res = {}
        for t in (1, 3, 64):
            assert oracle_mod.set_num_threads(t) == t
            res[t] = (oracle_mod.spread(xs, c, ns, w, beta), oracle_mod.interp(xs, b, ns, w, beta))
    finally:
        oracle_mod.set_num_threads(n0)
    for t in (3, 64):
        assert np.array_equal(res[t][0], res[1][0])
        assert np.array_equal(res[t][1], res[1][1])
