"""Serving loop (continuous batching) through the C ABI: every result is the same alone and in the
mix, admission respects the HBM budget, and oversized requests are rejected."""
import numpy as np
import pytest

import trals_inputs as TI

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2210_11362_gb300")

pytestmark = pytest.mark.gpu

# a mix of orders, sizes and ranks in the range of the serving workload (orders 3-5, sizes
# 16-64, ranks 2-8), kept small enough for a quick test
SHAPES = [((40, 24, 33), (4, 6, 3)), ((16, 20, 18, 22), (2, 5, 3, 4)), ((24, 16, 20, 16, 18), (3, 2, 4, 2, 3)),
          ((64, 48, 32), (8, 7, 6)), ((30, 30, 30, 30), (6, 6, 6, 6)), ((17, 23, 19, 21), (5, 3, 2, 4))]


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
def test_results_same_alone_and_in_the_mix(ctx, problems, mode):
    sweeps = 5
    opts = P.make_opts(mode)
    alone = []
    for (I, R), (X, init) in zip(SHAPES, problems):
        cores = [G.copy() for G in init]
        res = P.trals_decompose(ctx, I, R, X, cores, sweeps, opts)
        alone.append((cores, res))
    srv = P.Server(0, hbm_budget_bytes=8 << 30, max_slots=4)
    try:
        tickets = [srv.submit(I, R, X, init, sweeps, opts) for (I, R), (X, init) in zip(SHAPES, problems)]
        out = [srv.wait(t, timeout=120.0) for t in tickets]
        stats = srv.stats()
    finally:
        srv.close()
    assert stats["peak_active"] >= 2, stats        # requests really overlapped
    for (cores_a, res_a), got in zip(alone, out):
        assert got is not None
        info, cores_m, res_m = got
        assert info["status"] == P.OK, info
        for a, b in zip(cores_a, cores_m):
            np.testing.assert_array_equal(a, b)   # deterministic kernels, no shared device state
        np.testing.assert_array_equal(res_a[-1], res_m[-1])
        assert info["submit_s"] <= info["admit_s"] <= info["done_s"]


def test_admission_respects_the_budget(ctx, problems):
    opts = P.make_opts("bf16")
    fps = [P.trals_plan_footprint(ctx, I, R, X, opts) for (I, R), (X, _) in zip(SHAPES, problems)]
    budget = sorted(fps)[-1] + sorted(fps)[-2]     # room for the two largest at most
    srv = P.Server(0, hbm_budget_bytes=budget, max_slots=8)
    try:
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
    picks = [0, 1, 3]
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
