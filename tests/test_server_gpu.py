"""The serving loop on the GPU (paper_1808_06736_gb300.serve, include/nufft_serve.h).

* Every request of a mixed batch (type 1, type 2 and least-squares gradient
  requests; d = 1, 2, 3; complex64 and complex128; several eps) gives the same
  result in the mix -- eight slots, all submitted at once, overlapping on the
  device -- as alone (a one-slot server, one request at a time): relative l2
  difference <= 1e-5 (complex64) / 1e-12 (complex128), far below eps; the
  only difference is the order of the fine grid's atomic tile additions.
* The served results are right: type 1 / type 2 against the plan path and
  against the oracle's direct sums (sampled) within 10 eps.
* Gradient requests at 3D, N = 64^3, M = 1e5: loss against the plan path's
  values, grad_x against the FP64 direct-sum gradient on sampled points,
  grad_f on sampled modes; central finite differences at a small size.
* Resident points (binning skipped), eviction under a small budget,
  rejection of an oversized request, and the time limit.
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
    from paper_1808_06736_gb300 import serve
    return p, serve


def _rel(a, b):
    import torch
    return float(torch.linalg.vector_norm((a - b).to(torch.complex128)) /
                 max(float(torch.linalg.vector_norm(b.to(torch.complex128))), 1e-300))


def _mix(seed, n):
    """n requests: kind, d, modes, M, eps, dtype, inputs (device tensors)."""
    import torch
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(seed)
    shapes = {1: [(200,), (1000,), (4096,)], 2: [(64, 64), (128, 96), (256, 256)], 3: [(16, 16, 16), (32, 24, 20), (64, 64, 64)]}
    reqs = []
    for i in range(n):
        kind = int(rng.choice([1, 2, 3], p=[0.4, 0.4, 0.2]))
        d = 3 if kind == 3 else int(rng.integers(1, 4))
        modes = shapes[d][int(rng.integers(0, 3))]
        M = int(math.exp(rng.uniform(math.log(1e3), math.log(2e5))))
        c128 = rng.random() < 0.25
        cdt = torch.complex128 if c128 else torch.complex64
        rdt = torch.float64 if c128 else torch.float32
        eps = 1e-9 if c128 else float(rng.choice([1e-3, 1e-5]))
        kindp = "clustered" if rng.random() < 0.3 else "uniform"
        xs = I.torch_points(seed * 100 + i, M, d, kindp, dev, rdt)
        ntot = int(np.prod(modes))
        if kind == 1:
            data = I.torch_complex_normal(seed * 100 + i + 50, M, dev, cdt)
            y = None
        else:
            data = I.torch_complex_normal(seed * 100 + i + 50, ntot, dev, cdt).reshape(tuple(reversed(modes)))
            y = I.torch_complex_normal(seed * 100 + i + 70, M, dev, cdt) if kind == 3 else None
        isign = int(rng.choice([-1, 1]))
        reqs.append(dict(kind=kind, d=d, modes=modes, M=M, eps=eps, dtype=cdt, x=xs, data=data, y=y, isign=isign))
    return reqs


def _submit(srv, q, tag):
    if q["kind"] == 1:
        return srv.type1(q["x"], q["data"], q["modes"], eps=q["eps"], isign=q["isign"], dtype=q["dtype"], tag=tag)
    if q["kind"] == 2:
        return srv.type2(q["x"], q["data"], eps=q["eps"], isign=q["isign"], dtype=q["dtype"], tag=tag)
    return srv.lsq_grad(q["x"], q["data"], q["y"], eps=q["eps"], isign=q["isign"], dtype=q["dtype"], tag=tag)


def _collect(srv, n, timeout=120.0):
    import time
    got = {}
    t0 = time.time()
    while len(got) < n and time.time() - t0 < timeout:
        for c in srv.poll(256, 0.2):
            got[c.tag] = c
    return got


def test_mix_equals_alone_and_is_right(pkg, oracle_mod):
    import torch
    p, S = pkg
    reqs = _mix(11, 36)
    alone = {}
    srv1 = S.Server(budget_bytes=8 << 30, max_inflight=1)
    for i, q in enumerate(reqs):
        _submit(srv1, q, i)
        got = _collect(srv1, 1)
        assert got[i].status == 0, (i, got[i].status)
        alone[i] = got[i].outputs
    srv1.close()
    srv = S.Server(budget_bytes=8 << 30, max_inflight=8)
    for i, q in enumerate(reqs):
        _submit(srv, q, i)
    mix = _collect(srv, len(reqs))
    st = srv.stats()
    srv.close()
    assert len(mix) == len(reqs)
    assert st["peak_inflight"] > 1  # the mix did overlap
    for i, q in enumerate(reqs):
        c = mix[i]
        assert c.status == 0, (i, c.status)
        tol = 1e-12 if q["dtype"] == torch.complex128 else 1e-5
        for k, v in alone[i].items():
            assert _rel(c.outputs[k], v) <= tol, (i, k, _rel(c.outputs[k], v))
    # correctness of the served values: plan path (all) and direct sums (sampled)
    rng = np.random.default_rng(5)
    for i, q in enumerate(reqs):
        if q["kind"] == 3:
            continue
        prec = S.NUFFT_C128 if q["dtype"] == torch.complex128 else S.NUFFT_C64
        sigma = S.upsampfac_for(q["kind"], q["modes"], q["eps"], q["M"], prec)  # the server's per-request choice
        plan = p.Plan(q["kind"], q["modes"], eps=q["eps"], isign=q["isign"], dtype=q["dtype"], device="cuda:0",
                      upsampfac=sigma)
        plan.setpts(*q["x"])
        ref = plan.execute(q["data"]).reshape(-1)
        plan.close()
        out = (mix[i].outputs["f"] if q["kind"] == 1 else mix[i].outputs["c"]).reshape(-1)
        tol = 1e-12 if q["dtype"] == torch.complex128 else 1e-5
        assert _rel(out, ref) <= tol
        xs = [v.double().cpu().numpy() for v in q["x"]]
        if q["kind"] == 1:
            N = q["modes"]
            modes = np.stack([rng.integers(-(n // 2), n - n // 2, size=16) for n in N], axis=1)
            exact = oracle_mod.direct_type1(xs, q["data"].to(torch.complex128).cpu().numpy(), q["isign"], N, modes=modes)
            got = out[torch.as_tensor(oracle_mod.mode_index(modes, N), device=out.device)]
        else:
            tj = rng.choice(q["M"], size=min(q["M"], 32), replace=False)
            exact = oracle_mod.direct_type2([v[tj] for v in xs], q["data"].to(torch.complex128).cpu().numpy().ravel(),
                                            q["isign"], q["modes"])
            got = out[torch.as_tensor(tj, device=out.device)]
        err = oracle_mod.rel_l2(got.to(torch.complex128).cpu().numpy(), exact)
        assert err <= 10 * max(q["eps"], 2e-6 if q["dtype"] == torch.complex64 else 0), (i, err)


def _k(Ns):
    grids = np.meshgrid(*[np.arange(n) - n // 2 for n in reversed(Ns)], indexing="ij")
    return [g.ravel() for g in reversed(grids)]


@pytest.mark.parametrize("cdt,eps,xgrad", [("c64", 1e-5, "exact"), ("c64", 1e-3, "exact"), ("c128", 1e-11, "exact"),
                                           ("c64", 1e-5, "kernel"), ("c128", 1e-11, "kernel")])
def test_lsq_gradient_request_3d_against_direct_sums(pkg, oracle_mod, cdt, eps, xgrad):
    import torch
    p, S = pkg
    dev = torch.device("cuda:0")
    Ns = [64, 64, 64]
    M = 100_000
    cdtype = torch.complex128 if cdt == "c128" else torch.complex64
    rdt = torch.float64 if cdt == "c128" else torch.float32
    xs = I.torch_points(81, M, 3, "uniform", dev, rdt)
    f = I.torch_complex_normal(82, 64 ** 3, dev, cdtype).reshape(64, 64, 64)
    y = I.torch_complex_normal(83, M, dev, cdtype)
    srv = S.Server(budget_bytes=4 << 30, max_inflight=2)
    srv.lsq_grad(xs, f, y, eps=eps, isign=-1, dtype=cdtype, tag=1, xgrad=xgrad)
    c = _collect(srv, 1)[1]
    srv.close()
    assert c.status == 0
    gx, gf, loss = c.outputs["grad_x"], c.outputs["grad_f"], float(c.outputs["loss"].item())
    tol = 10 * max(eps, 2e-6 if cdt == "c64" else 0)
    # the kernel route's point gradient: ~2 sqrt(12) times the values' error (aliased
    # frequencies weighted by their own size), bar 20 eps with an fp32 floor
    tol_x = tol if xgrad == "exact" else 20 * max(eps, 1e-5 if cdt == "c64" else 0)
    # loss against the plan path's forward values, on the fine grid the server chose
    sigma = S.upsampfac_for(S.NUFFT_REQ_LSQ_GRAD, Ns, eps, M, S.NUFFT_C128 if cdt == "c128" else S.NUFFT_C64)
    plan = p.Plan(2, Ns, eps=eps, isign=-1, dtype=cdtype, device=dev, upsampfac=sigma)
    plan.setpts(*xs)
    cv = plan.execute(f).reshape(-1)
    plan.close()
    ref_loss = float(((cv - y).abs().double() ** 2).sum())
    assert abs(loss - ref_loss) <= 1e-5 * ref_loss
    # grad_x on sampled points against the FP64 direct-sum gradient
    x64 = [v.double().cpu().numpy() for v in xs]
    fn = f.to(torch.complex128).cpu().numpy().ravel()
    yn = y.to(torch.complex128).cpu().numpy()
    rng = np.random.default_rng(84)
    tj = rng.choice(M, size=48, replace=False)
    ct = oracle_mod.direct_type2([v[tj] for v in x64], fn, -1, Ns)
    G = 2 * (ct - yn[tj])
    ks = _k(Ns)
    for d in range(3):
        cd = oracle_mod.direct_type2([v[tj] for v in x64], fn * (-1j * ks[d]), -1, Ns)
        ref = np.real(np.conj(G) * cd)
        got = gx[d].double().cpu().numpy()[tj]
        assert np.linalg.norm(got - ref) <= tol_x * np.linalg.norm(ref)
    # grad_f = 2 F1_{+1}(x) (c - y) on sampled modes, with c from the plan path
    Gall = 2 * (cv.to(torch.complex128).cpu().numpy() - yn)
    modes = rng.integers(-32, 32, size=(24, 3))
    ref_f = oracle_mod.direct_type1(x64, Gall, 1, Ns, modes=modes)
    got_f = gf.reshape(-1)[torch.as_tensor(oracle_mod.mode_index(modes, Ns), device=dev)]
    assert oracle_mod.rel_l2(got_f.to(torch.complex128).cpu().numpy(), ref_f) <= tol


def test_lsq_gradient_request_finite_differences(pkg):
    """Central differences of the served loss (complex128, eps = 1e-13) in a few coordinates of x and f."""
    import torch
    p, S = pkg
    dev = torch.device("cuda:0")
    Ns = [10, 9, 8]
    M = 300
    x0 = torch.tensor(np.stack(I.points(91, M, 3)), dtype=torch.float64, device=dev)
    f0 = torch.tensor(I.complex_normal(92, 720).reshape(8, 9, 10), device=dev)
    y = torch.tensor(I.complex_normal(93, M), device=dev)
    srv = S.Server(budget_bytes=1 << 30, max_inflight=4)

    def run(x, f):
        t = srv.lsq_grad(x, f, y, eps=1e-13, isign=1, dtype=torch.complex128, tag=0)
        got = _collect(srv, 1)[0]
        assert got.status == 0 and got.ticket == t
        return got.outputs

    base = run(x0, f0)
    h = 1e-6
    rng = np.random.default_rng(94)
    for _ in range(6):
        d, j = int(rng.integers(0, 3)), int(rng.integers(0, M))
        xp, xm = x0.clone(), x0.clone()
        xp[d, j] += h
        xm[d, j] -= h
        fd = (float(run(xp, f0)["loss"].item()) - float(run(xm, f0)["loss"].item())) / (2 * h)
        g = float(base["grad_x"][d, j].item())
        assert abs(fd - g) <= 1e-6 * max(1.0, abs(g)), (d, j, fd, g)
    for _ in range(4):
        k = tuple(int(rng.integers(0, n)) for n in (8, 9, 10))
        for part in (1.0, 1j):
            fp, fm = f0.clone(), f0.clone()
            fp[k] += h * part
            fm[k] -= h * part
            fd = (float(run(x0, fp)["loss"].item()) - float(run(x0, fm)["loss"].item())) / (2 * h)
            g = base["grad_f"][k]
            gv = float(g.real) if part == 1.0 else float(g.imag)
            assert abs(fd - gv) <= 1e-6 * max(1.0, abs(gv)), (k, part, fd, gv)
    srv.close()


def test_resident_points_skip_binning(pkg):
    import torch
    p, S = pkg
    dev = torch.device("cuda:0")
    xs = I.torch_points(101, 50_000, 2, "clustered", dev, torch.float32)
    f1 = I.torch_complex_normal(102, 128 * 128, dev, torch.complex64).reshape(128, 128)
    f2 = I.torch_complex_normal(103, 128 * 128, dev, torch.complex64).reshape(128, 128)
    srv = S.Server(budget_bytes=1 << 30, max_inflight=2)
    srv.type2(xs, f1, eps=1e-5, points_key=42, tag=1)
    a = _collect(srv, 1)[1]
    srv.type2(xs, f2, eps=1e-5, points_key=42, tag=2)
    b = _collect(srv, 1)[2]
    st = srv.stats()
    srv.close()
    assert a.status == 0 and b.status == 0
    assert a.reused == 0 and b.reused == 2 and st["binning_skipped"] == 1
    plan = p.Plan(2, (128, 128), eps=1e-5, dtype=torch.complex64, device=dev)
    plan.setpts(*xs)
    assert _rel(b.outputs["c"], plan.execute(f2).reshape(-1)) <= 1e-6
    plan.close()


def test_budget_eviction_and_rejection(pkg):
    import torch
    p, S = pkg
    dev = torch.device("cuda:0")
    # admission estimates two fine grids per new entry (grid + a bound on cuFFT's work
    # area, 220..268 MB here) and counts at least one grid (110..134 MB) per resident
    # entry, so no more than two entries fit and the five shapes force evictions
    budget = 400 << 20
    srv = S.Server(budget_bytes=budget, max_inflight=4)
    xs = I.torch_points(111, 20_000, 3, "uniform", dev, torch.float32)
    c = I.torch_complex_normal(112, 20_000, dev, torch.complex64)
    shapes = [(128, 128, 128), (128, 128, 120), (120, 120, 120), (128, 120, 120), (128, 128, 128)]
    for i, n in enumerate(shapes):
        srv.type1(xs, c, n, eps=1e-5, tag=i)
    got = _collect(srv, len(shapes))
    assert all(got[i].status == 0 for i in range(len(shapes)))
    srv.type1(xs, c, (256, 256, 256), eps=1e-5, tag=99)  # fine grid alone is 1 GB
    big = _collect(srv, 1)[99]
    st = srv.stats()
    srv.close()
    assert big.status == S.NUFFT_ERR_REJECTED
    assert st["entries_evicted"] >= 1 and st["peak_bytes"] <= budget and st["rejected"] == 1


def test_time_limit_reports_timeout_and_server_recovers(pkg):
    import torch
    p, S = pkg
    dev = torch.device("cuda:0")
    xs = I.torch_points(121, 2_000_000, 3, "uniform", dev, torch.float32)
    c = I.torch_complex_normal(122, 2_000_000, dev, torch.complex64)
    srv = S.Server(budget_bytes=4 << 30, max_inflight=2, timeout_s=1e-4)
    srv.type1(xs, c, (128, 128, 128), eps=1e-5, tag=1)
    got = _collect(srv, 1)[1]
    assert got.status == S.NUFFT_ERR_TIMEOUT
    assert srv.drain(60.0) == 0  # the work itself finishes
    assert srv.stats()["timeouts"] == 1
    srv.close()
    srv = S.Server(budget_bytes=4 << 30, max_inflight=2)
    srv.type1(xs, c, (128, 128, 128), eps=1e-5, tag=2)
    assert _collect(srv, 1)[2].status == 0
    srv.close()
