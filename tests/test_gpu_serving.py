"""Serving loop (continuous batching) through the C ABI: every result is the same alone and in the
mix, for requests served as plans and by the grouped step engine; grouped results agree with the plans'
and with the oracle; admission respects the HBM budget; oversized requests are rejected; a grouped
step whose descriptor table never comes gives up within its bound and reports TRALS_E_TIMEOUT."""
import numpy as np
import pytest

import trals_inputs as TI

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2210_11362_gb300")

pytestmark = pytest.mark.gpu

# a mix of orders, sizes and ranks in the range of the serving workload (orders 3-5, sizes
# 16-64, ranks 2-8), kept small enough for a quick test
SHAPES = [((40, 24, 33), (4, 6, 3)), ((16, 20, 18, 22), (2, 5, 3, 4)), ((24, 16, 20, 16, 18), (3, 2, 4, 2, 3)),
          ((64, 48, 32), (8, 7, 6)), ((30, 30, 30, 30), (6, 6, 6, 6)), ((17, 23, 19, 21), (5, 3, 2, 4)),
          ((20, 24, 22, 18), (8, 8, 8, 8))]   # r = 64 in every mode: the widest S_n, L and solve rows


def _request(k, I, R, ctx):
    truth = TI.gaussian_cores(100 + k, I, R)
    cd = [P.core_to_device(G) for G in truth]
    Xt = torch.empty(int(np.prod(I)), dtype=torch.float64, device="cuda")
    P.trals_reconstruct(ctx, I, R, cd, Xt)
    noise = torch.from_numpy(TI.flat_f(TI.gaussian_noise(100 + k, I))).cuda()
    X = Xt + 1e-2 * (torch.linalg.vector_norm(Xt) / torch.linalg.vector_norm(noise)) * noise
    return X.to(torch.float32).contiguous(), TI.init_cores(100 + k, I, R)


@pytest.fixture(scope="module")
def ctx():
    c = P.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def problems(ctx):
    return [_request(k, I, R, ctx) for k, (I, R) in enumerate(SHAPES)]


@pytest.mark.parametrize("mode", ["bf16", "fp32"])
def test_plan_results_same_alone_and_in_the_mix(ctx, problems, mode):
    """Requests served as plans (the grouped engine switched off) equal trals_decompose bit for bit."""
    sweeps = 5
    opts = P.make_opts(mode)
    alone = []
    for (I, R), (X, init) in zip(SHAPES, problems):
        cores = [G.copy() for G in init]
        res = P.trals_decompose(ctx, I, R, X, cores, sweeps, opts)
        alone.append((cores, res))
    srv = P.Server(0, hbm_budget_bytes=8 << 30, max_slots=4)
    try:
        srv.set_group_limit(0)
        tickets = [srv.submit(I, R, X, init, sweeps, opts) for (I, R), (X, init) in zip(SHAPES, problems)]
        out = [srv.wait(t, timeout=120.0) for t in tickets]
        stats = srv.stats()
    finally:
        srv.close()
    assert stats["peak_active"] >= 2, stats        # requests really overlapped
    assert stats["grouped_completed"] == 0, stats
    for (cores_a, res_a), got in zip(alone, out):
        assert got is not None
        info, cores_m, res_m = got
        assert info["status"] == P.OK, info
        for a, b in zip(cores_a, cores_m):
            np.testing.assert_array_equal(a, b)   # deterministic kernels, no shared device state
        np.testing.assert_array_equal(res_a[-1], res_m[-1])
        assert info["submit_s"] <= info["admit_s"] <= info["done_s"]


GROUP_ALL = 1 << 22   # a group limit above every test shape: all of them join the grouped engine


def _serve(problems, sweeps, opts, picks, budget=8 << 30, limit=GROUP_ALL, one_at_a_time=False, slots=4):
    srv = P.Server(0, hbm_budget_bytes=budget, max_slots=slots)
    try:
        if limit is not None:
            srv.set_group_limit(limit)
        out = []
        if one_at_a_time:
            for k in picks:
                t = srv.submit(SHAPES[k][0], SHAPES[k][1], problems[k][0], problems[k][1], sweeps, opts)
                out.append(srv.wait(t, timeout=120.0))
        else:
            tickets = [srv.submit(SHAPES[k][0], SHAPES[k][1], problems[k][0], problems[k][1], sweeps, opts)
                       for k in picks]
            out = [srv.wait(t, timeout=120.0) for t in tickets]
        stats = srv.stats()
    finally:
        srv.close()
    return out, stats


@pytest.mark.parametrize("mode", ["bf16", "fp32"])
def test_grouped_results_same_alone_and_in_the_mix(problems, mode):
    """The grouped step engine: each request served alone and served in the mix (all active together,
    in different modes n at every step) gives the same cores and residual bit for bit."""
    opts = P.make_opts(mode)
    picks = list(range(len(SHAPES)))
    alone, st_a = _serve(problems, 5, opts, picks, one_at_a_time=True)
    mixed, st_m = _serve(problems, 5, opts, picks)
    assert st_a["grouped_completed"] == st_m["grouped_completed"] == len(SHAPES), (st_a, st_m)
    assert st_m["peak_active"] >= 2, st_m
    for k, (a, m) in enumerate(zip(alone, mixed)):
        assert a[0]["status"] == P.OK and m[0]["status"] == P.OK, (k, a[0], m[0])
        for ga, gm in zip(a[1], m[1]):
            np.testing.assert_array_equal(ga, gm)
        np.testing.assert_array_equal(a[2], m[2])
        assert np.isnan(a[2][:-1]).all() and 0.0 < a[2][-1] < 1.0


@pytest.mark.parametrize("mode", ["bf16", "fp32"])
def test_grouped_results_agree_with_the_plans(ctx, problems, mode):
    """Grouped and plan results of the same requests, started near the generating cores.  In the FP32
    mode both compute the same method in the same precisions, summed in different orders: the cores
    agree to FP32 rounding (amplified by the conditioning of the solves) and the final residuals to
    1e-6.  In the BF16 mode the tensor-core plans also round the subchain table to BF16 where the
    grouped MTTSP keeps it in FP32, so the two differ by BF16 rounding: 2e-5 on the residual, 2e-2 on
    the cores (both far inside the 1e-4 residual gap the reduced precision is held to)."""
    rng = np.random.default_rng(3)
    opts = P.make_opts(mode)
    tol, rtol = (2e-2, 2e-5) if mode == "bf16" else (1e-4, 1e-6)
    for k, (I, R) in enumerate(SHAPES):
        init = [G + 1e-2 * rng.standard_normal(G.shape) for G in TI.gaussian_cores(100 + k, I, R)]
        cores = [G.copy() for G in init]
        res = P.trals_decompose(ctx, I, R, problems[k][0], cores, 5, opts)
        srv = P.Server(0, hbm_budget_bytes=8 << 30, max_slots=2)
        try:
            srv.set_group_limit(GROUP_ALL)
            got = srv.wait(srv.submit(I, R, problems[k][0], init, 5, opts), timeout=120.0)
            assert srv.stats()["grouped_completed"] == 1
        finally:
            srv.close()
        assert got[0]["status"] == P.OK, got[0]
        assert abs(got[2][-1] - res[-1]) <= rtol, (k, got[2][-1], res[-1])
        for a, b in zip(cores, got[1]):
            assert np.linalg.norm(a - b) <= tol * np.linalg.norm(a), (k, np.linalg.norm(a - b) / np.linalg.norm(a))


def test_grouped_and_plan_requests_together(problems):
    """With the group limit between the sizes, the small requests go to the grouped engine and the rest
    to plans in the same run; all complete."""
    sizes = [int(np.prod(I)) for I, _ in SHAPES]
    limit = int(np.median(sizes))
    out, stats = _serve(problems, 3, P.make_opts("bf16"), list(range(len(SHAPES))), limit=limit)
    assert all(o is not None and o[0]["status"] == P.OK for o in out)
    assert stats["grouped_completed"] == sum(n <= limit for n in sizes), (stats, sizes, limit)


def test_grouped_step_timeout_reports_status(problems):
    """A step launched without its descriptor table: the doorbell wait gives up after its bound (2e6
    cycles, about a millisecond), the step does no work, the requests it carried complete with
    TRALS_E_TIMEOUT, and the next requests are served normally."""
    opts = P.make_opts("fp32")
    srv = P.Server(0, hbm_budget_bytes=8 << 30, max_slots=2)
    try:
        srv.set_group_limit(GROUP_ALL)
        srv.testing_withhold_steps(1, 2_000_000)
        t = [srv.submit(SHAPES[k][0], SHAPES[k][1], problems[k][0], problems[k][1], 2, opts) for k in (0, 1)]
        first = [srv.wait(x, timeout=60.0) for x in t]
        again = srv.wait(srv.submit(SHAPES[0][0], SHAPES[0][1], problems[0][0], problems[0][1], 2, opts),
                         timeout=60.0)
    finally:
        srv.close()
    assert any(f[0]["status"] == P.E_TIMEOUT for f in first), [f[0] for f in first]
    assert all(f[0]["status"] in (P.OK, P.E_TIMEOUT) for f in first)
    assert again[0]["status"] == P.OK, again[0]


def test_admission_respects_the_budget(ctx, problems):
    opts = P.make_opts("bf16")
    fps = [P.trals_plan_footprint(ctx, I, R, X, opts) for (I, R), (X, _) in zip(SHAPES, problems)]
    budget = sorted(fps)[-1] + sorted(fps)[-2]     # room for the two largest at most
    srv = P.Server(0, hbm_budget_bytes=budget, max_slots=8)
    try:
        srv.set_group_limit(0)
        tickets = [srv.submit(I, R, X, init, 3, opts) for (I, R), (X, init) in zip(SHAPES, problems)]
        out = [srv.wait(t, timeout=120.0) for t in tickets]
        stats = srv.stats()
    finally:
        srv.close()
    assert all(o is not None and o[0]["status"] == P.OK for o in out)
    assert stats["peak_used_bytes"] <= budget, (stats, budget)
    assert stats["completed"] == len(SHAPES)
    for o, fp in zip(out, fps):
        assert o[0]["footprint_bytes"] == fp


def test_grouped_admission_respects_the_budget(problems):
    opts = P.make_opts("bf16")
    picks = list(range(len(SHAPES)))
    alone, _ = _serve(problems, 2, opts, picks, one_at_a_time=True)
    fps = sorted(a[0]["footprint_bytes"] for a in alone)
    budget = fps[-1] + fps[-2]
    out, stats = _serve(problems, 2, opts, picks, budget=budget)
    assert all(o is not None and o[0]["status"] == P.OK for o in out)
    assert stats["peak_used_bytes"] <= budget, (stats, budget)
    assert stats["grouped_completed"] == len(SHAPES)


def test_footprint_equals_plan_bytes(ctx, problems):
    for mode in ("fp64", "bf16", "fp32"):
        for (I, R), (X, _) in zip(SHAPES, problems):
            Xm = X.to(torch.float64) if mode == "fp64" else X
            opts = P.make_opts(mode)
            plan = P.Plan(ctx, I, R, Xm, opts)
            try:
                paths = [plan.mttsp_path(n) for n in range(len(I))]
                assert plan.nbytes() == P.trals_plan_footprint(ctx, I, R, Xm, opts), (mode, I, R, paths)
            finally:
                plan.close()


def test_oversized_request_rejected_and_host_X_matches_device_X(ctx, problems):
    (I, R), (X, init) = SHAPES[0], problems[0]
    opts = P.make_opts("bf16")
    srv = P.Server(0, hbm_budget_bytes=1 << 16, max_slots=2)
    try:
        with pytest.raises(P.TralsError) as e:
            srv.submit(I, R, X, init, 2, opts)
        assert e.value.status == P.E_REJECTED
    finally:
        srv.close()
    srv = P.Server(0, hbm_budget_bytes=4 << 30, max_slots=2)
    try:
        t_dev = srv.submit(I, R, X, init, 3, opts)
        t_host = srv.submit(I, R, X.cpu().numpy(), init, 3, opts)
        a = srv.wait(t_dev, timeout=60.0)
        b = srv.wait(t_host, timeout=60.0)
        with pytest.raises(P.TralsError):         # the ticket was released by wait
            srv.poll(t_dev)
    finally:
        srv.close()
    for ga, gb in zip(a[1], b[1]):
        np.testing.assert_array_equal(ga, gb)


@pytest.mark.parametrize("mode", ["fp32", "bf16"])
def test_served_results_match_the_oracle_on_a_subsample(ctx, problems, mode):
    """A subsample of served requests (orders 3 and 4) against the FP64 oracle run alone from the same
    init for the serving workload's 15 sweeps: the final relative residual, measured against the
    request's own X, is within 1e-4 of the oracle's.  The runs start near the generating cores (plus a
    1e-2 perturbation), so both precisions are compared at convergence: trajectories of different
    precisions from a random start part ways before they converge."""
    import oracle as O
    rng = np.random.default_rng(7)
    picks = [0, 1, 3, 6]
    inits = {k: [G + 1e-2 * rng.standard_normal(G.shape) for G in TI.gaussian_cores(100 + k, *SHAPES[k])]
             for k in picks}
    srv = P.Server(0, hbm_budget_bytes=8 << 30, max_slots=4)
    try:
        tickets = [srv.submit(SHAPES[k][0], SHAPES[k][1], problems[k][0], inits[k], 15, P.make_opts(mode))
                   for k in picks]
        out = [srv.wait(t, timeout=300.0) for t in tickets]
    finally:
        srv.close()
    for k, got in zip(picks, out):
        I, R = SHAPES[k]
        X = TI.unflat_f(problems[k][0].double().cpu().numpy(), I)
        assert got is not None and got[0]["status"] == P.OK
        _, ref_res = O.tr_als(X, inits[k], 15, "chol")
        assert abs(O.rel_residual(X, got[1]) - ref_res[-1]) <= 1e-4, (k, O.rel_residual(X, got[1]), ref_res[-1])
