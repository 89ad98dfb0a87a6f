"""Parity of the CUDA path (through the C ABI) with the CPU oracle, step by step and end to end.

Tolerances: the FP64 path must match the oracle's cores after one sweep within 1e-9
relative; single steps in FP64 within 1e-12 relative (FP64 rounding of sums of a few
thousand terms); integer/byte work (BF16 quantisation) bit-exact.
"""
import numpy as np
import pytest

import oracle as O
import trals_inputs as TI

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU hosts
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2210_11362_gb300 as P  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    return P.trals_create(0)


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


SHAPES = [
    ((7, 5, 9, 4), (2, 3, 4, 2)),           # ragged sizes, mixed ranks
    ((20, 20, 20), (3, 3, 3)),              # the 20^3 rank-3 workload shape
    ((3, 11, 6), (2, 2, 3)),                # I_1 < R_1 R_2
    ((13, 3, 5, 2, 4), (2, 3, 2, 2, 3)),    # order 5, tiny modes
    ((33, 17, 40), (5, 4, 6)),              # several tiles per block, ragged tail
]


def _problem(I, R, seed=3, eta=1e-2):
    truth = TI.gaussian_cores(seed, I, R)
    X = TI.add_relative_noise(O.tr_full(truth), TI.gaussian_noise(seed, I), eta)
    return X, TI.init_cores(seed, I, R)


def test_gamma_matches_definition(ctx):
    for (Rn, In, Rn1) in [(3, 20, 3), (2, 7, 5), (10, 60, 10), (16, 3, 16), (1, 4, 1)]:
        G = np.random.default_rng(Rn * 100 + In).standard_normal((Rn, In, Rn1))
        Gd = P.core_to_device(G)
        out = torch.zeros(Rn * Rn * Rn1 * Rn1, dtype=torch.float64, device="cuda")
        P.trals_gamma(ctx, Gd, Rn, In, Rn1, out)
        ref = O.gamma(G)
        got = out.cpu().numpy().reshape(Rn * Rn, Rn1 * Rn1, order="F")
        assert rel(got, ref) < 1e-13


@pytest.mark.parametrize("I,R", SHAPES)
def test_coef_matrix_equals_explicit_gram(ctx, I, R):
    cores = TI.gaussian_cores(5, I, R)
    gams = []
    for G in cores:
        g = O.gamma(G)
        gams.append(torch.from_numpy(g.reshape(-1, order="F").copy()).cuda())
    N = len(I)
    for n in range(N):
        r = R[n] * R[(n + 1) % N]
        S = torch.zeros(r * r, dtype=torch.float64, device="cuda")
        P.trals_coef_matrix(ctx, R, gams, n, S)
        A = O.subchain_unfolded(cores, n)
        ref = A.T @ A
        assert rel(S.cpu().numpy().reshape(r, r, order="F"), ref) < 1e-12


@pytest.mark.parametrize("I,R", SHAPES + [((60, 60, 60, 60), (10, 10, 10, 10))])
def test_coef_matrix_explicit_subchain_gram(ctx, I, R):
    """Explicit-subchain variant (regular TR-ALS): S_n = A^T A with A formed on the device, FP64
    within 1e-12 of the oracle's explicit A^T A; FP32 rows within FP32 rounding (1e-5)."""
    cores = TI.gaussian_cores(5, I, R)
    cd = [P.core_to_device(G) for G in cores]
    N = len(I)
    for n in range(N):
        r = R[n] * R[(n + 1) % N]
        if np.prod(I) > 1e6 and n > 0:
            continue                       # full-size shape: one mode (the oracle's A is 216000 x 100)
        A = O.subchain_unfolded(cores, n)
        ref = A.T @ A
        for fp64, tol in ((True, 1e-12), (False, 1e-5)):
            S = torch.zeros(r * r, dtype=torch.float64, device="cuda")
            P.trals_coef_matrix_explicit(ctx, I, R, cd, n, S, fp64)
            got = S.cpu().numpy().reshape(r, r, order="F")
            assert np.array_equal(got, got.T)
            assert rel(got, ref) < tol, (n, fp64, rel(got, ref))


@pytest.mark.parametrize("I,R", SHAPES[:3])
def test_decompose_explicit_gram_one_sweep_matches_oracle(ctx, I, R):
    """gram = explicit (regular TR-ALS normal equations) in FP64: cores after one sweep within 1e-9
    of the oracle's Cholesky normal equations on the explicit subchain matrix."""
    X, init = _problem(I, R)
    cores = [G.copy() for G in init]
    P.trals_decompose(ctx, I, R, X, cores, 1, P.make_opts("fp64", gram=P.GRAM_EXPLICIT))
    ref, _ = O.tr_als(X, init, 1, "chol")
    for a, b in zip(cores, ref):
        assert rel(a, b) < 1e-9


@pytest.mark.parametrize("I,R", SHAPES + [((40, 40, 40, 40), (8, 10, 12, 10)), ((300, 30, 400), (3, 4, 2))])
def test_qr_r_factor_matches_householder_qr(ctx, I, R):
    """R factor of G^{!=n}_[2] by the structured recursive QR (never forming S_n) equals the R of a
    Householder QR of the explicit subchain matrix (LAPACK), rows scaled to a positive diagonal."""
    cores = TI.gaussian_cores(6, I, R)
    cd = [P.core_to_device(G) for G in cores]
    N = len(I)
    for n in range(N):
        r = R[n] * R[(n + 1) % N]
        A = O.subchain_unfolded(cores, n)
        Rref = np.linalg.qr(A, mode="r")
        Rref = Rref * np.sign(np.diag(Rref))[:, None]
        Rd = torch.zeros(r * r, dtype=torch.float64, device="cuda")
        P.trals_qr_r_factor(ctx, I, R, cd, n, Rd)
        got = Rd.cpu().numpy().reshape(r, r, order="F")
        assert np.allclose(np.tril(got, -1), 0.0)
        assert rel(got, Rref) < 1e-11, (n, rel(got, Rref))


def test_qr_r_factor_structurally_rank_deficient_subchain(ctx):
    """Core n+1 zero for one value of its left rank index makes the columns of G^{!=n}_[2] with that
    index vanish.  The TSQR leaves and merges take their skip paths for those columns (no reflector:
    the column is already zero), the call reports the rank deficiency as TRALS_E_NOT_SPD (a zero
    diagonal of R), and the factor it leaves still satisfies R^T R = A^T A: R is not unique for a
    rank-deficient A, its Gram matrix is."""
    I, R = (40, 24, 33, 20), (4, 6, 3, 5)
    cores = TI.gaussian_cores(6, I, R)
    n = 0
    cores[1][2, :, :] = 0.0   # G_1(i) row r_1 = 2 is zero for every i
    A = O.subchain_unfolded(cores, n)
    zero_cols = np.where(~A.any(axis=0))[0]
    assert list(zero_cols) == [8, 9, 10, 11]   # columns a + R_0 r_1 with r_1 = 2
    r = R[0] * R[1]
    Rd = torch.zeros(r * r, dtype=torch.float64, device="cuda")
    with pytest.raises(P.TralsError) as err:
        P.trals_qr_r_factor(ctx, I, R, [P.core_to_device(G) for G in cores], n, Rd)
    assert err.value.status == P.E_NOT_SPD
    got = Rd.cpu().numpy().reshape(r, r, order="F")
    assert np.allclose(np.tril(got, -1), 0.0)
    assert np.all(np.diag(got)[zero_cols] == 0.0)
    assert np.all(got[:, zero_cols] == 0.0)
    assert rel(got.T @ got, A.T @ A) < 1e-12


@pytest.mark.parametrize("I,R", SHAPES[:3] + [((40, 24, 33, 20), (4, 6, 3, 5))])
def test_decompose_qr_one_sweep_matches_oracle(ctx, I, R):
    """solver = QR in FP64: cores after one sweep within 1e-9 of the oracle's Householder QR least
    squares (regular TR-ALS, which TR-ALS-QR equals in exact arithmetic)."""
    X, init = _problem(I, R)
    cores = [G.copy() for G in init]
    res = P.trals_decompose(ctx, I, R, X, cores, 2, P.make_opts("fp64", solver=P.SOLVE_QR))
    ref, ref_res = O.tr_als(X, init, 2, "qr")
    for a, b in zip(cores, ref):
        assert rel(a, b) < 1e-9
    np.testing.assert_allclose(res, ref_res, rtol=1e-8)


@pytest.mark.parametrize("eta", [1e-9, 1e-3])
def test_qr_solver_stays_accurate_where_normal_equations_do_not(ctx, eta):
    """Collinear cores (unit-norm unfolding columns with pairwise inner product 1 - 1e-6, the
    construction of the paper's ill-conditioned experiments): the first core update of a sweep is a
    least-squares problem with cond(G^{!=1}_[2]) ~ 3.5e6, whose solution LAPACK's QR and SVD solvers
    agree on to ~1e-14.  The QR-stabilised solve matches it to 1e-8; the Cholesky normal equations
    (cond^2 ~ 1.2e13) break down or land far off.  Only core 1 is compared: the later updates of
    the sweep become far worse conditioned (~1e10), where no solver is reproducible."""
    I, R = (60, 50, 40), (2, 3, 2)
    truth = TI.collinear_cores(31, I, R, 1.0 - 1e-6)
    X = TI.add_relative_noise(O.tr_full(truth), TI.gaussian_noise(31, I), eta)
    init = TI.collinear_cores(32, I, R, 1.0 - 1e-6)
    ref = O.als_update(X, [G.copy() for G in init], 0, "qr")
    errs = {}
    for name, solver in (("qr", P.SOLVE_QR), ("chol", P.SOLVE_CHOL)):
        cores = [G.copy() for G in init]
        try:
            P.trals_decompose(ctx, I, R, X, cores, 1, P.make_opts("fp64", solver=solver))
            errs[name] = rel(cores[0], ref)
        except P.TralsError as e:      # the normal equations may not even be numerically SPD
            assert name == "chol" and e.status == P.E_NOT_SPD
            errs[name] = np.inf
    assert errs["qr"] < 1e-8, errs
    assert errs["chol"] > 100 * errs["qr"], errs


@pytest.mark.parametrize("I,R", SHAPES)
def test_mttsp_fp64_matches_oracle(ctx, I, R):
    X, _ = _problem(I, R)
    cores = TI.gaussian_cores(9, I, R)
    Xd = P.tensor_to_device(X)
    cd = [P.core_to_device(G) for G in cores]
    N = len(I)
    for n in range(N):
        r = R[n] * R[(n + 1) % N]
        M = torch.zeros(I[n] * r, dtype=torch.float64, device="cuda")
        P.trals_mttsp(ctx, I, R, Xd, "fp64", cd, n, M)
        ref = O.unfold_mode(X, n) @ O.subchain_unfolded(cores, n)
        assert rel(M.cpu().numpy().reshape(I[n], r, order="F"), ref) < 1e-12


@pytest.mark.parametrize("I,R", SHAPES + [((40, 24, 33, 20), (4, 6, 3, 5)), ((64, 17, 50), (8, 7, 6))])
def test_mttsp_fp32_cuda_cores_match_oracle(ctx, I, R):
    """FP32 X on the FP32-arithmetic CUDA-core kernel (memory-order tiles): the result matches
    X_fp32 G^{!=n} in FP64 to FP32 rounding of the factors and the per-CTA sums (1e-5)."""
    X, _ = _problem(I, R)
    cores = TI.gaussian_cores(9, I, R)
    Xf = P.tensor_to_device(X, torch.float32)
    Xq = TI.unflat_f(Xf.cpu().numpy().astype(np.float64), I)
    cd = [P.core_to_device(G) for G in cores]
    N = len(I)
    for n in range(N):
        r = R[n] * R[(n + 1) % N]
        M = torch.zeros(I[n] * r, dtype=torch.float64, device="cuda")
        P.trals_mttsp(ctx, I, R, Xf, "fp32", cd, n, M)
        ref = O.unfold_mode(Xq, n) @ O.subchain_unfolded(cores, n)
        got = M.cpu().numpy().reshape(I[n], r, order="F")
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < 1e-5, (n, err)


TC_SHAPES = [
    ((16, 24, 32, 20), (3, 4, 2, 5)),        # every tensor-core geometry, small ranks
    ((40, 40, 40, 40), (8, 10, 12, 10)),     # 40^4 with the ranks of the 40^5 workload
    ((40, 40, 40, 32, 4), (4, 5, 6, 5, 4)),    # order 5: K-major tiles with a large table and with mid modes
    ((24, 20, 18, 29, 40), (3, 7, 4, 8, 5)),   # short middle modes: K-major tiles of 6, 7 and 4 repetitions
]

# Componentwise error bound of the reduced-precision MTTSP against M_ref = X_q G^{!=n}_[2] in FP64
# (X_q: the BF16, or hi + lo, values the kernel reads):
#   |M - M_ref| <= (c u + (N - 2)(R_max + 1) 2^-24 + lambda sqrt(J_n) 2^-24) (|X_q,[n]| |G|^{!=n}_[2])
# where |G|^{!=n} is the subchain of the elementwise absolute cores, an upper bound of |F| |Tab| for any
# split of the chain into the stage-1 table Tab and the stage-2 factor F.
#  - c u: the storage rounding of the stage-1 table: RNE to BF16 (2^-9 relative) with u = 2^-8 and
#    c = 1; for the split-BF16 mode the dropped lo x lo product and the rounding of the lo planes
#    (2 x 2^-18) with u = 2^-16 and c = 1;
#  - (N - 2)(R_max + 1) 2^-24: the FP32 chain products that build the table and the factor;
#  - lambda sqrt(J_n) 2^-24: the FP32 accumulation over the J_n terms, by the probabilistic bound of
#    Higham & Mary (SIAM J. Sci. Comput. 2019) with lambda = 10 (failure probability below 1e-15).
U_BF16, U_BF16X3, LAMBDA_FP32 = 2.0 ** -8, 2.0 ** -16, 10.0


def componentwise_tol(Xq, cores, n, u, c=1.0):
    N = len(cores)
    J = Xq.size // Xq.shape[n]
    Rmax = max(G.shape[0] for G in cores)
    B = O.mttsp(np.abs(Xq), [np.abs(G) for G in cores], n)
    return (c * u + (N - 2) * (Rmax + 1) * 2.0 ** -24 + LAMBDA_FP32 * np.sqrt(J) * 2.0 ** -24) * B


def _integer_problem(I, R, seed=5):
    """Small-integer X and signed-selection cores: every product and sum of the reduced-precision
    MTTSP is an exact integer in BF16/FP32, so the result must equal the FP64 oracle exactly."""
    return TI.small_integer_tensor(seed, I), TI.signed_selection_cores(seed, I, R)


def _mode_input(ctx, X, mode):
    """The device X a mode reads: BF16, or the hi and lo BF16 halves of split-BF16 (2 prod(I) values),
    with the FP64 values they hold."""
    I = X.shape
    numel = int(np.prod(I))
    if mode in ("bf16", "bf16x2"):
        Xb = P.tensor_to_device(X, torch.bfloat16)
        return Xb, TI.unflat_f(Xb.double().cpu().numpy(), I)
    Xd = P.tensor_to_device(X)
    hl = torch.zeros(2 * numel, dtype=torch.bfloat16, device="cuda")
    P.trals_quantize_bf16(ctx, Xd, hl[:numel], hl[numel:])
    return hl, TI.unflat_f(hl[:numel].double().cpu().numpy() + hl[numel:].double().cpu().numpy(), I)


def _run_mttsp(ctx, I, R, Xdev, mode, cores, n):
    r = R[n] * R[(n + 1) % len(I)]
    M = torch.full((I[n] * r,), float("nan"), dtype=torch.float64, device="cuda")
    P.trals_mttsp(ctx, I, R, Xdev, mode, [P.core_to_device(G) for G in cores], n, M)
    return M.cpu().numpy().reshape(I[n], r, order="F"), P.trals_last_mttsp_path(ctx)


@pytest.mark.parametrize("mode", ["bf16", "bf16x2", "bf16x3"])
@pytest.mark.parametrize("I,R", TC_SHAPES)
def test_mttsp_tensor_cores_exact_on_integer_data(ctx, I, R, mode):
    """On data where every intermediate is exact (small-integer X, subchain entries in {-1, 0, 1})
    the tensor-core MTTSP must give the FP64 oracle's M_n bit for bit: any wrong row, column,
    factor or K step shows as an integer difference.  The kernel that ran is the tensor-core one."""
    X, cores = _integer_problem(I, R)
    Xdev, Xq = _mode_input(ctx, X, mode)
    assert np.array_equal(Xq, X)
    for n in range(len(I)):
        got, path = _run_mttsp(ctx, I, R, Xdev, mode, cores, n)
        assert path == P.trals_mttsp_path(I, R, n, mode) > 0, (n, path)
        ref = O.mttsp(X, cores, n)
        assert np.array_equal(got, ref), (n, P.MTTSP_PATHS[path], np.abs(got - ref).max())


def test_mttsp_bf16_pair_input(ctx):
    """X given as a BF16 hi/lo pair (X_BF16PAIR): bf16x3 reads both planes, bit for bit what the same
    buffer gives when typed as plain BF16 (the layout bf16x3 has always taken); BF16 and bf16x2 read the
    hi plane only, bit for bit what the hi plane alone gives."""
    I, R = TC_SHAPES[1]
    X, _ = _problem(I, R)
    cores = TI.gaussian_cores(9, I, R)
    pair, _ = _mode_input(ctx, X, "bf16x3")
    numel = int(np.prod(I))
    hi = pair[:numel].clone()
    cd = [P.core_to_device(G) for G in cores]
    r = R[1] * R[2]
    outs = {}
    for tag, buf, mode, xt in [("x3pair", pair, "bf16x3", P.X_BF16PAIR), ("x3bf16", pair, "bf16x3", None),
                               ("bfpair", pair, "bf16", P.X_BF16PAIR), ("bfhi", hi, "bf16", None),
                               ("x2pair", pair, "bf16x2", P.X_BF16PAIR), ("x2hi", hi, "bf16x2", None)]:
        M = torch.full((I[1] * r,), float("nan"), dtype=torch.float64, device="cuda")
        P.trals_mttsp(ctx, I, R, buf, mode, cd, 1, M, xt=xt)
        assert P.trals_last_mttsp_path(ctx) > 0, tag
        outs[tag] = M.cpu().numpy()
    assert np.array_equal(outs["x3pair"], outs["x3bf16"])
    assert np.array_equal(outs["bfpair"], outs["bfhi"])
    assert np.array_equal(outs["x2pair"], outs["x2hi"])
    assert not np.array_equal(outs["x3pair"], outs["bfhi"])


@pytest.mark.parametrize("mode", ["bf16", "bf16x2", "bf16x3"])
@pytest.mark.parametrize("I,R", TC_SHAPES)
def test_mttsp_tensor_cores_componentwise_bound(ctx, I, R, mode):
    """Gaussian data: every element of M_n within the componentwise bound above (and normwise
    within 4e-3 for BF16, 5e-5 for split-BF16), on the tensor-core kernel."""
    X, _ = _problem(I, R)
    cores = TI.gaussian_cores(9, I, R)
    Xdev, Xq = _mode_input(ctx, X, mode)
    # bf16x2 rounds X (the reference is taken on the rounded X) but splits the table: only the table's
    # hi/lo residue and the FP32 accumulation remain, as in bf16x3
    u, normwise = (U_BF16, 4e-3) if mode == "bf16" else (U_BF16X3, 5e-5)
    for n in range(len(I)):
        got, path = _run_mttsp(ctx, I, R, Xdev, mode, cores, n)
        assert path == P.trals_mttsp_path(I, R, n, mode) > 0, (n, path)
        ref = O.mttsp(Xq, cores, n)
        tol = componentwise_tol(Xq, cores, n, u)
        ratio = float((np.abs(got - ref) / tol).max())
        assert ratio <= 1.0, (n, P.MTTSP_PATHS[path], ratio)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < normwise, (n, P.MTTSP_PATHS[path], err)


PADDED_SHAPES = [((41, 39, 47, 33), (3, 4, 2, 5)), ((60, 60, 60, 60), (10, 10, 10, 10)),
                 ((45, 53, 64, 55, 36), (7, 2, 3, 5, 4))]


@pytest.mark.parametrize("I,R", PADDED_SHAPES)
def test_plan_mttsp_bf16_with_padded_leading_mode(ctx, I, R):
    """A plan stores the BF16 copy of X with mode 0 zero-padded to a multiple of 8 so that the
    tensor-core geometries apply; M_n of every mode (including mode 0, whose padded rows are
    dropped) is within the componentwise bound of X_bf16 G^{!=n} element by element, and exactly
    equal to it on integer data."""
    N = len(I)
    for exact in (False, True):
        if exact:
            X, cores = _integer_problem(I, R)
        else:
            X, _ = _problem(I, R)
            cores = TI.gaussian_cores(9, I, R)
        Xf = P.tensor_to_device(X, torch.float32)
        Xq = TI.unflat_f(Xf.to(torch.bfloat16).double().cpu().numpy(), I)
        plan = P.Plan(ctx, I, R, Xf, P.make_opts("bf16"))
        try:
            plan.set_cores(cores)
            paths = [plan.mttsp_path(n) for n in range(N)]
            assert paths == [P.trals_mttsp_path(I, R, n, "bf16") for n in range(N)]
            assert sum(p_ > 0 for p_ in paths) >= N - 2, paths
            for n in range(N):
                r = R[n] * R[(n + 1) % N]
                M = torch.full((I[n] * r,), float("nan"), dtype=torch.float64, device="cuda")
                plan.mttsp(n, M)
                torch.cuda.synchronize()
                got = M.cpu().numpy().reshape(I[n], r, order="F")
                ref = O.mttsp(Xq, cores, n)
                if exact:
                    assert np.array_equal(got, ref), (n, paths[n], np.abs(got - ref).max())
                else:
                    ratio = float((np.abs(got - ref) / componentwise_tol(Xq, cores, n, U_BF16)).max())
                    assert ratio <= 1.0, (n, paths[n], ratio)
        finally:
            plan.close()


def test_plan_mttsp_full_size_40x5(ctx):
    """The 40^5 workload shape, R = (8,10,12,10,8), through the plan exactly as a sweep runs it,
    every mode on its tensor-core geometry (mode 0 MN-major with the factor on the left, mode 1
    MN-major with the factor on the right and whole-tile work shares): integer data must match the
    FP64 oracle exactly; Gaussian data must stay within the componentwise bound in the MN-major
    modes (0, 1) and the K-major-right mode (4)."""
    I, R = (40,) * 5, (8, 10, 12, 10, 8)
    for exact, modes in ((True, range(5)), (False, (0, 1, 4))):
        if exact:
            X, cores = _integer_problem(I, R, seed=6)
        else:
            X = TI.gaussian_noise(6, I)
            cores = TI.gaussian_cores(6, I, R)
        Xf = P.tensor_to_device(X, torch.float32)
        Xq = TI.unflat_f(Xf.to(torch.bfloat16).double().cpu().numpy(), I)
        plan = P.Plan(ctx, I, R, Xf, P.make_opts("bf16"))
        try:
            plan.set_cores(cores)
            assert [plan.mttsp_path(n) for n in range(5)] == [4, 3, 1, 1, 2]
            for n in modes:
                r = R[n] * R[(n + 1) % 5]
                M = torch.full((I[n] * r,), float("nan"), dtype=torch.float64, device="cuda")
                plan.mttsp(n, M)
                torch.cuda.synchronize()
                got = M.cpu().numpy().reshape(I[n], r, order="F")
                ref = O.mttsp(Xq, cores, n)
                if exact:
                    assert np.array_equal(got, ref), (n, np.abs(got - ref).max())
                else:
                    ratio = float((np.abs(got - ref) / componentwise_tol(Xq, cores, n, U_BF16)).max())
                    assert ratio <= 1.0, (n, ratio)
        finally:
            plan.close()


# Wide subchain tables (R = 16: 256 columns) have no tensor-core geometry; with at least 2^21 entries the
# reduced modes take the two-stage GEMM MTTSP (path 5).  I_0 = 60 makes the BF16 modes pad mode 0 to 64,
# which the GEMM's table (modes 1-3) and T's rows (mode 0) must follow.
GEMM_SHAPE = ((60, 64, 3, 200), (16, 16, 16, 16))
_GEMM_REF = {}


def _gemm_plan_M(ctx, I, R, X, cores, mode, n):
    plan = P.Plan(ctx, I, R, P.tensor_to_device(X, torch.float32), P.make_opts(mode))
    try:
        plan.set_cores(cores)
        assert [plan.mttsp_path(k) for k in range(len(I))] == [5] * len(I)
        r = R[n] * R[(n + 1) % len(I)]
        M = torch.full((I[n] * r,), float("nan"), dtype=torch.float64, device="cuda")
        plan.mttsp(n, M)
        torch.cuda.synchronize()
        return M.cpu().numpy().reshape(I[n], r, order="F")
    finally:
        plan.close()


@pytest.mark.parametrize("mode", ["fp32", "bf16", "bf16x2"])
def test_plan_two_stage_gemm_mttsp_exact_on_integer_data(ctx, mode):
    """Integer X and signed-selection cores: every product and sum of both stages is an exact integer
    in FP32 and BF16, so M_n must equal the FP64 oracle bit for bit in every mode n (forms 1 and 2, the
    padded leading mode included)."""
    I, R = GEMM_SHAPE
    X, cores = _integer_problem(I, R, seed=8)
    for n in range(len(I)):
        if ("int", n) not in _GEMM_REF:
            _GEMM_REF[("int", n)] = O.mttsp(X, cores, n)
        got = _gemm_plan_M(ctx, I, R, X, cores, mode, n)
        ref = _GEMM_REF[("int", n)]
        assert np.array_equal(got, ref), (mode, n, np.abs(got - ref).max())


@pytest.mark.parametrize("mode,n", [("fp32", 2), ("fp32", 3), ("bf16", 0), ("bf16x2", 1)])
def test_plan_two_stage_gemm_mttsp_componentwise_bound(ctx, mode, n):
    """Gaussian data: every element of M_n within the componentwise bound of the X the mode reads
    (FP32, or BF16 with the table in BF16 or split)."""
    I, R = GEMM_SHAPE
    X = TI.gaussian_noise(8, I)
    cores = TI.gaussian_cores(8, I, R)
    Xt = torch.from_numpy(TI.flat_f(X)).to(torch.float32)
    xq_t = Xt if mode == "fp32" else Xt.to(torch.bfloat16)
    Xq = TI.unflat_f(xq_t.double().numpy(), I)
    u = {"fp32": 2.0 ** -24, "bf16": U_BF16, "bf16x2": U_BF16X3}[mode]
    got = _gemm_plan_M(ctx, I, R, X, cores, mode, n)
    ref = O.mttsp(Xq, cores, n)
    ratio = float((np.abs(got - ref) / componentwise_tol(Xq, cores, n, u)).max())
    assert ratio <= 1.0, (mode, n, ratio)


def test_qr_solver_two_stage_refinement_matches_fp64(ctx):
    """QR-stabilised solve in the FP32 mode on a shape whose MTTSPs take the two-stage GEMM route: its
    refinement steps form the residual tensor E = X - X_hat and the MTTSP of E by GEMMs as well.  Started
    near the generating cores, two sweeps must land on the FP64 QR run's residual to 1e-7 (the
    refinement lifts the FP32 right-hand side to the accuracy of the source X)."""
    I, R = (60, 64, 3, 200), (8, 8, 8, 8)
    truth = TI.gaussian_cores(11, I, R)
    cd = [P.core_to_device(G) for G in truth]
    Xt = torch.empty(int(np.prod(I)), dtype=torch.float64, device="cuda")
    P.trals_reconstruct(ctx, I, R, cd, Xt)
    noise = torch.from_numpy(TI.flat_f(TI.gaussian_noise(11, I))).cuda()
    X64 = (Xt + 1e-2 * (torch.linalg.vector_norm(Xt) / torch.linalg.vector_norm(noise)) * noise).contiguous()
    X32 = X64.to(torch.float32)
    rng = np.random.default_rng(11)
    init = [G + 1e-2 * rng.standard_normal(G.shape) for G in truth]
    res = {}
    for mode, X in (("fp64", X64), ("fp32", X32)):
        plan = P.Plan(ctx, I, R, X, P.make_opts(mode, solver=P.SOLVE_QR))
        try:
            if mode == "fp32":
                assert [plan.mttsp_path(n) for n in range(4)] == [5] * 4
            plan.set_cores(init)
            plan.run(2)
            torch.cuda.synchronize()
            r2, x2 = P.trals_residual_explicit(ctx, I, R, X64, [plan.core_dev(n) for n in range(4)])
            res[mode] = float(np.sqrt(max(r2, 0.0) / x2))
        finally:
            plan.close()
    assert 1e-3 < res["fp64"] < 1e-1
    assert abs(res["fp32"] - res["fp64"]) <= 1e-7, res


def test_solve_chol_matches_oracle(ctx):
    I, R = (9, 8, 7), (3, 4, 2)
    X, init = _problem(I, R)
    for n in range(3):
        S, M = O.normal_equation_terms(X, init, n)
        Rn, Rn1 = R[n], R[(n + 1) % 3]
        G = torch.zeros(Rn * I[n] * Rn1, dtype=torch.float64, device="cuda")
        P.trals_solve_chol(ctx, Rn, I[n], Rn1, torch.from_numpy(S.reshape(-1, order="F").copy()).cuda(),
                           torch.from_numpy(M.reshape(-1, order="F").copy()).cuda(), G)
        ref = O.core_fold2(O.ls_solve_normal(S, M), Rn, Rn1)
        assert rel(P.core_from_device(G, Rn, I[n], Rn1), ref) < 1e-10


@pytest.mark.parametrize("r", [1, 7, 64, 97, 120, 128, 200])
@pytest.mark.parametrize("scale", [1.0, 2.0 ** 700, 2.0 ** -700, 3.0e150, 7.0e-160])
def test_solve_chol_across_sizes_and_scales(ctx, r, scale):
    """Cholesky + triangular solves on random SPD systems (cond ~ 1e3) from r = 1 through the blocked
    many-SM factorization (r = 97: a one-column last panel; 200: the solve reading L from global
    memory), with S and M scaled together far outside FP32 range (the pivot's reciprocal square root
    is rescaled by exact powers of two): the solution is scale-free."""
    rng = np.random.default_rng(r)
    A = rng.standard_normal((3 * r + 5, r))
    S = A.T @ A + 1e-3 * np.eye(r)
    In = 13
    M = rng.standard_normal((In, r))
    ref = np.linalg.solve(S, M.T).T
    G = torch.zeros(In * r, dtype=torch.float64, device="cuda")
    P.trals_solve_chol(ctx, r, In, 1, torch.from_numpy((S * scale).reshape(-1, order="F").copy()).cuda(),
                       torch.from_numpy((M * scale).reshape(-1, order="F").copy()).cuda(), G)
    got = G.cpu().numpy().reshape(r, In, order="F").T        # core layout with R_n = r, R_{n+1} = 1
    assert rel(got, ref) < 1e-11, rel(got, ref)


def test_pivot_rsqrt_against_cuda_rsqrt(ctx):
    """The Cholesky pivots' reciprocal square root (FP32 estimate + one third-order Householder step,
    rescaled path outside the FP32 exponent range) against CUDA's double rsqrt, which is documented
    within 1 ulp: over the whole normal exponent range, exact powers of four, and both sides of the
    fast path's exponent limits."""
    rng = np.random.default_rng(11)
    frac = 1.0 + rng.random(200000)
    exps = rng.integers(-1020, 1020, size=frac.size)
    d = np.ldexp(frac, exps)
    edges = [np.ldexp(f, e) for e in (-122, -121, -120, -119, 119, 120, 121, 122)
             for f in (1.0, 1.5, np.nextafter(2.0, 0.0))]
    quads = [4.0 ** k for k in range(-200, 201)]
    d = np.concatenate([d, edges, quads, [np.finfo(np.float64).tiny, np.finfo(np.float64).max]])
    dd = torch.from_numpy(d).cuda()
    out = torch.empty_like(dd)
    ref = torch.empty_like(dd)
    P.trals_check_pivot_rsqrt(ctx, dd, out, ref)
    o, f = out.cpu().numpy(), ref.cpu().numpy()
    ulp = np.spacing(np.abs(f))
    assert np.all(np.isfinite(o))
    assert np.max(np.abs(o - f) / ulp) <= 3.0
    # powers of four: the exact result is a power of two
    q = np.array(quads)
    oq = o[-len(quads) - 2:-2]
    exact = np.ldexp(1.0, -np.arange(-200, 201))
    assert np.max(np.abs(oq - exact) / np.spacing(exact)) <= 1.0
    assert np.array_equal(exact, 1.0 / np.sqrt(q))


@pytest.mark.parametrize("r,k", [(40, 1), (40, 2), (40, 37), (40, 39), (120, 64), (120, 119), (5, 0), (97, 96),
                                 (200, 150), (200, 0)])
def test_solve_chol_reports_not_spd_mid_factorization(ctx, r, k):
    """A non-positive pivot at column k (of either step parity, including the first and the last)
    stops the factorization with NOT_SPD; a later call on the same context still works."""
    S = np.eye(r)
    S[k, k] = -1.0
    M = np.ones((3, r))
    G = torch.zeros(r * 3, dtype=torch.float64, device="cuda")
    with pytest.raises(P.TralsError) as e:
        P.trals_solve_chol(ctx, r, 3, 1, torch.from_numpy(S.reshape(-1, order="F").copy()).cuda(),
                           torch.from_numpy(M.reshape(-1, order="F").copy()).cuda(), G)
    assert e.value.status == P.E_NOT_SPD
    S[k, k] = np.nan
    with pytest.raises(P.TralsError) as e:
        P.trals_solve_chol(ctx, r, 3, 1, torch.from_numpy(S.reshape(-1, order="F").copy()).cuda(),
                           torch.from_numpy(M.reshape(-1, order="F").copy()).cuda(), G)
    assert e.value.status == P.E_NONFINITE
    S[k, k] = 2.0
    P.trals_solve_chol(ctx, r, 3, 1, torch.from_numpy(S.reshape(-1, order="F").copy()).cuda(),
                       torch.from_numpy(M.reshape(-1, order="F").copy()).cuda(), G)
    want = np.ones((3, r))
    want[:, k] = 0.5
    assert rel(G.cpu().numpy().reshape(r, 3, order="F").T, want) < 1e-14


def test_solve_chol_reports_not_spd(ctx):
    r = 6
    S = -np.eye(r)
    M = np.ones((4, r))
    G = torch.zeros(2 * 4 * 3, dtype=torch.float64, device="cuda")
    with pytest.raises(P.TralsError) as e:
        P.trals_solve_chol(ctx, 2, 4, 3, torch.from_numpy(S.reshape(-1, order="F").copy()).cuda(),
                           torch.from_numpy(M.reshape(-1, order="F").copy()).cuda(), G)
    assert e.value.status == P.E_NOT_SPD
    # the context stays usable afterwards
    test_gamma_matches_definition(ctx)


@pytest.mark.parametrize("I,R", SHAPES)
def test_decompose_fp64_one_sweep_matches_oracle(ctx, I, R):
    X, init = _problem(I, R)
    cores = [G.copy() for G in init]
    res = P.trals_decompose(ctx, I, R, X, cores, 1)
    ref, ref_res = O.tr_als(X, init, 1, "qr")
    for a, b in zip(cores, ref):
        assert rel(a, b) < 1e-9
    assert abs(res[0] - ref_res[0]) <= 1e-9 * ref_res[0]


def test_tr20_rank3_ten_sweeps(ctx):
    """The 20x20x20 rank-3 workload: 1e-3 noise, seeded N(0,1) init, 10 sweeps, Cholesky."""
    w = TI.WORKLOADS["tr20x3_r3"]
    X = TI.make_tensor_host(w, 0, O.tr_full)
    init = TI.init_cores(0, w.I, w.R_fit)
    cores = [G.copy() for G in init]
    res = P.trals_decompose(ctx, w.I, w.R_fit, X, cores, w.sweeps)
    c1 = [G.copy() for G in init]
    P.trals_decompose(ctx, w.I, w.R_fit, X, c1, 1)
    ref1, _ = O.tr_als(X, init, 1, "chol", residual=False)
    for a, b in zip(c1, ref1):
        assert rel(a, b) < 1e-9
    ref, ref_res = O.tr_als(X, init, w.sweeps, "chol")
    np.testing.assert_allclose(res, ref_res, rtol=1e-7)
    for r0, r1 in zip(res, res[1:]):
        assert r1 <= r0 * (1 + 1e-9)


def test_plan_graph_replay_is_bitwise_equal_to_eager(ctx):
    I, R = (17, 12, 9, 10), (3, 4, 2, 3)
    X, init = _problem(I, R)
    Xd = P.tensor_to_device(X)
    outs = []
    for use_graph in (False, True, True):
        plan = P.Plan(ctx, I, R, Xd)
        plan.set_cores(init)
        plan.run(3, use_graph=use_graph)
        outs.append((plan.get_cores(), plan.residuals()))
        plan.close()
    for cores, res in outs[1:]:
        for a, b in zip(cores, outs[0][0]):
            np.testing.assert_array_equal(a, b)
        np.testing.assert_array_equal(res, outs[0][1])


def test_plan_bf16_split_runs_match_one_run(ctx):
    """A reduced-precision sweep prepares the next sweep's mode 0 (its tensor-core table pre-phase and
    Gamma-chain prefix); a run after set_cores prepares it in a prologue.  Three sweeps in one run, in
    three runs, and again after set_cores, all give the same cores bit for bit."""
    I, R = (40, 40, 40, 40), (8, 10, 12, 10)
    X, init = _problem(I, R)
    Xd = P.tensor_to_device(X, torch.float32)
    outs = []
    for split in (False, True):
        plan = P.Plan(ctx, I, R, Xd, P.make_opts("bf16"))
        plan.set_cores(init)
        if split:
            for _ in range(3):
                plan.run(1, use_graph=True)
        else:
            plan.run(3, use_graph=True)
        outs.append(plan.get_cores())
        if split:
            plan.set_cores(init)
            plan.run(3, use_graph=True)
            outs.append(plan.get_cores())
        plan.close()
    for other in outs[1:]:
        for a, b in zip(other, outs[0]):
            np.testing.assert_array_equal(a, b)


def test_reconstruct_and_explicit_residual(ctx):
    for I, R in SHAPES:
        cores = TI.gaussian_cores(4, I, R)
        cd = [P.core_to_device(G) for G in cores]
        out = torch.zeros(int(np.prod(I)), dtype=torch.float64, device="cuda")
        P.trals_reconstruct(ctx, I, R, cd, out)
        ref = O.tr_full(cores)
        assert rel(TI.unflat_f(out.cpu().numpy(), I), ref) < 1e-12
        X = ref + 0.1 * TI.gaussian_noise(4, I)
        r2, x2 = P.trals_residual_explicit(ctx, I, R, P.tensor_to_device(X), cd)
        assert abs(r2 - np.sum((X - ref) ** 2)) <= 1e-10 * np.sum(X ** 2)
        assert abs(x2 - np.sum(X ** 2)) <= 1e-12 * np.sum(X ** 2)


def test_explicit_residual_option_matches_identity(ctx):
    I, R = (11, 10, 9), (2, 3, 2)
    X, init = _problem(I, R, eta=0.05)
    a = [G.copy() for G in init]
    b = [G.copy() for G in init]
    ra = P.trals_decompose(ctx, I, R, X, a, 4)
    rb = P.trals_decompose(ctx, I, R, X, b, 4, P.make_opts("fp64", explicit_residual=True))
    np.testing.assert_allclose(ra, rb, rtol=1e-8)
    _, ref_res = O.tr_als(X, init, 4, "qr")
    np.testing.assert_allclose(rb, ref_res, rtol=1e-9)


def test_quantize_bitexact(ctx):
    x = np.random.default_rng(8).standard_normal(100003) * 10.0 ** np.random.default_rng(9).integers(-6, 6, 100003)
    xd = torch.from_numpy(x).cuda()
    hi = torch.zeros(x.size, dtype=torch.bfloat16, device="cuda")
    lo = torch.zeros(x.size, dtype=torch.bfloat16, device="cuda")
    P.trals_quantize_bf16(ctx, xd, hi, lo)
    rh, rl = O.bf16_split(x)
    np.testing.assert_array_equal(hi.view(torch.int16).cpu().numpy().view(np.uint16), rh)
    np.testing.assert_array_equal(lo.view(torch.int16).cpu().numpy().view(np.uint16), rl)


def test_argument_errors(ctx):
    X = torch.zeros(2 * 2 * 2, dtype=torch.float64, device="cuda")
    with pytest.raises(P.TralsError) as e:   # J_n = 4 < R_n R_{n+1} = 9
        P.Plan(ctx, (2, 2, 2), (3, 3, 3), X)
    assert e.value.status == P.E_ARG
    with pytest.raises(P.TralsError):        # order 2
        P.Plan(ctx, (4, 4), (2, 2), torch.zeros(16, dtype=torch.float64, device="cuda"))
    with pytest.raises(P.TralsError):        # FP64 mode with an FP32 X
        P.Plan(ctx, (4, 4, 4), (2, 2, 2), torch.zeros(64, dtype=torch.float32, device="cuda"))


def _near_truth_problem(I, R, eta, seed):
    truth = TI.gaussian_cores(seed, I, R)
    X = TI.add_relative_noise(O.tr_full(truth), TI.gaussian_noise(seed, I), eta)
    rng = np.random.default_rng(seed + 1)
    init = [G + 1e-2 * rng.standard_normal(G.shape) for G in truth]
    return X, init


@pytest.mark.parametrize("solver", ["chol", "qr"])
@pytest.mark.parametrize("mode", ["fp32", "bf16", "bf16x2", "bf16x3"])
@pytest.mark.parametrize("I,R,eta", [((30, 30, 30, 30), (6, 6, 6, 6), 1e-3), ((40, 24, 32), (4, 5, 3), 1e-2)])
def test_reduced_precision_residual_gap(ctx, mode, I, R, eta, solver):
    """Reduced-precision modes reach the FP64 oracle's residual within 1e-4 (absolute), compared at
    convergence (runs start near the truth, so both precisions sit at the noise floor)."""
    X, init = _near_truth_problem(I, R, eta, 11)
    cores = [G.copy() for G in init]
    Xd = P.tensor_to_device(X, torch.float32)
    res = P.trals_decompose(ctx, I, R, Xd, cores, 6,
                            P.make_opts(mode, solver=P.SOLVE_QR if solver == "qr" else P.SOLVE_CHOL))
    _, ref_res = O.tr_als(X, init, 6, "chol")
    gap = abs(O.rel_residual(X, cores) - ref_res[-1])
    assert gap <= 1e-4, gap
    # no per-sweep residual in the reduced modes by default; the last one is the explicit pass
    # (FP32 regeneration against the FP32 X): equal to the oracle's residual of the same cores
    assert np.isnan(res[:-1]).all()
    assert abs(res[-1] - O.rel_residual(X, cores)) < 1e-6
    for n in range(len(I)):
        assert O.subchain_principal_angle(cores, O.tr_als(X, init, 6, "chol", residual=False)[0], n) < 1e-2


def test_tr60x4_rank10_full_size_one_sweep(ctx):
    """60^4 (12.96M entries), ranks 10: GPU FP64 cores after one sweep vs the oracle (blockwise NE)."""
    w = TI.WORKLOADS["tr60x4_r10"]
    X = TI.make_tensor_host(w, 0, O.tr_full)
    init = TI.init_cores(0, w.I, w.R_fit)
    cores = [G.copy() for G in init]
    P.trals_decompose(ctx, w.I, w.R_fit, X, cores, 1)
    ref = [G.copy() for G in init]
    for n in range(4):
        S, M = O.normal_equation_terms(X, ref, n)
        ref[n] = O.core_fold2(O.ls_solve_normal(S, M), ref[n].shape[0], ref[n].shape[2])
    for a, b in zip(cores, ref):
        assert rel(a, b) < 1e-9


@pytest.mark.parametrize("mode", ["bf16", "bf16x2", "bf16x3"])
def test_explicit_per_sweep_residual_in_reduced_modes(ctx, mode):
    """explicit_residual=1 in a reduced-precision mode: every sweep's residual comes from the FP32
    regeneration pass and matches the oracle's residual of the cores after that sweep."""
    I, R = (30, 26, 28, 24), (5, 4, 6, 3)
    X, init = _near_truth_problem(I, R, 1e-2, 21)
    Xd = P.tensor_to_device(X, torch.float32)
    plan = P.Plan(ctx, I, R, Xd, P.make_opts(mode, explicit_residual=True))
    try:
        plan.set_cores(init)
        per = []
        for _ in range(3):
            plan.run(1, use_graph=False)
            per.append(O.rel_residual(X, plan.get_cores()))
        got = plan.residuals()
        direct = plan.explicit_residual()
    finally:
        plan.close()
    np.testing.assert_allclose(got, per, rtol=0, atol=1e-6)
    assert abs(direct - per[-1]) < 1e-6


@pytest.mark.parametrize("I,R,n", [((40, 40, 40, 40), (8, 10, 12, 10), 1), ((40, 40, 40, 40), (8, 10, 12, 10), 0)])
def test_tensor_core_wait_timeout_returns_status(ctx, I, R, n):
    """A copy the TMA producer never issues (fault injection on the host side of the launch): the MMA
    issuer's bounded wait gives up after ~1 ms, the kernel drains what it did issue, frees its tensor
    memory and reports TRALS_E_TIMEOUT; the same context then computes the MTTSP correctly."""
    X, cores = _integer_problem(I, R)
    Xb = P.tensor_to_device(X, torch.bfloat16)
    cd = [P.core_to_device(G) for G in cores]
    r = R[n] * R[(n + 1) % len(I)]
    M = torch.zeros(I[n] * r, dtype=torch.float64, device="cuda")
    with pytest.raises(P.TralsError) as e:
        P.trals_testing_mttsp_withheld_copy(ctx, I, R, Xb, "bf16", cd, n, M, 2_000_000)
    assert e.value.status == P.E_TIMEOUT
    assert "bounded wait" in str(e.value)
    got, path = _run_mttsp(ctx, I, R, Xb, "bf16", cores, n)
    assert path > 0
    assert np.array_equal(got, O.mttsp(X, cores, n))


def test_plan_uses_the_tensor_core_geometry_it_reports(ctx):
    """The plan of the 40^5 workload runs every mode on the tensor cores, in the geometry the host
    query reports (no silent fallback to the CUDA cores)."""
    I, R = (40,) * 5, (8, 10, 12, 10, 8)
    X = torch.zeros(int(np.prod(I)), dtype=torch.bfloat16, device="cuda")
    plan = P.Plan(ctx, I, R, X, P.make_opts("bf16"))
    try:
        got = [plan.mttsp_path(n) for n in range(5)]
    finally:
        plan.close()
    assert got == [P.trals_mttsp_path(I, R, n, "bf16") for n in range(5)] == [4, 3, 1, 1, 2]


@pytest.mark.parametrize("I,R", [((300, 30, 400), (3, 4, 2)), ((40, 3, 50, 36), (2, 3, 2, 2)),
                                 ((20, 20, 20), (3, 3, 3)), ((13, 3, 5, 2, 4), (2, 3, 2, 2, 3))])
def test_decompose_qrne_matches_oracle(ctx, I, R):
    """TR-ALS-QRNE (Alg. 4) on the GPU: CholeskyQR2 of every compressible core, the Multi-TTM of X with
    the Q factors, the FP64 MTTSP of the compressed tensor with the R cores, the structured Gram chain of
    the R cores and the Cholesky solve.  Two sweeps from the same init give the cores of the oracle's
    literal Alg. 4 (which equals regular TR-ALS) within 1e-9 relative, and the same residuals.  The
    shapes mix compressible modes (I_j > R_j R_{j+1}) with modes kept whole (I_j <= R_j R_{j+1})."""
    X, init = _problem(I, R)
    cores = [G.copy() for G in init]
    res = P.trals_decompose(ctx, I, R, X, cores, 2, P.make_opts("fp64", solver=P.SOLVE_QRNE))
    ref, ref_res = O.tr_als_qrne(X, init, 2)
    for a, b in zip(cores, ref):
        assert rel(a, b) < 1e-9, rel(a, b)
    np.testing.assert_allclose(res, ref_res, rtol=1e-9)


def test_qrne_rejects_reduced_precision(ctx):
    X, init = _problem((20, 20, 20), (3, 3, 3))
    with pytest.raises(P.TralsError) as e:
        P.trals_decompose(ctx, (20, 20, 20), (3, 3, 3), P.tensor_to_device(X, torch.float32), [G.copy() for G in init],
                          1, P.make_opts("fp32", solver=P.SOLVE_QRNE))
    assert e.value.status == P.E_ARG


@pytest.mark.parametrize("I,R", [((300, 30, 400), (3, 4, 2)), ((40, 3, 50, 36), (2, 3, 2, 2)),
                                 ((20, 20, 20), (3, 3, 3)), ((60, 3, 50, 30), (2, 2, 2, 3))])
def test_decompose_literal_qr_compressed_matches_oracle(ctx, I, R):
    """The literal TR-ALS-QR (Alg. 3) in the compressible regime on the GPU: Householder mode-2 QRs of
    the cores, the Multi-TTM, the explicit subchain V_n of the R factors and its Householder QR with Q_0
    formed, W_n = Y_[n] Q_0 and the triangular solve.  Two sweeps agree with the oracle's Alg. 3 and
    with Householder least squares on the explicit subchain matrix (regular TR-ALS) within 1e-9."""
    X, init = _problem(I, R)
    cores = [G.copy() for G in init]
    res = P.trals_decompose(ctx, I, R, X, cores, 2, P.make_opts("fp64", solver=P.SOLVE_QR_COMPRESSED))
    ref, ref_res = O.tr_als_qr(X, init, 2)
    ls, ls_res = O.tr_als(X, init, 2, "qr")
    for a, b, c in zip(cores, ref, ls):
        assert rel(a, b) < 1e-9, rel(a, b)
        assert rel(a, c) < 1e-9, rel(a, c)
    np.testing.assert_allclose(res, ref_res, rtol=1e-9)


def test_literal_qr_rank_deficient_subproblem_takes_the_svd_of_r(ctx):
    """The SVD option of the remark after Alg. 3: core 3 with two equal rank channels (its last index,
    so the columns a = 0 and a = 1 of every G^{!=1}(k) coincide) makes the first core update rank
    deficient.  The Householder QRs keep the dependent columns (R_kk = 0), and the solve of
    G_{n(2)} R^T = W_n goes through the SVD of R (one-sided Jacobi) with the negligible singular values
    dropped: the minimum-norm least-squares core, as the oracle's SVD least squares on the explicit
    subchain matrix gives it.  One sweep agrees within 1e-8 relative."""
    I, R = (30, 20, 25), (2, 2, 3)
    X, init = _problem(I, R)
    init[2][:, :, 1] = init[2][:, :, 0]
    A = O.subchain_unfolded(init, 0)
    s = np.linalg.svd(A, compute_uv=False)
    assert s[-1] < 1e-12 * s[0]                   # the first subproblem is rank deficient
    cores = [G.copy() for G in init]
    res = P.trals_decompose(ctx, I, R, X, cores, 1, P.make_opts("fp64", solver=P.SOLVE_QR_COMPRESSED))
    ref, ref_res = O.tr_als(X, init, 1, "svd")
    for a, b in zip(cores, ref):
        assert rel(a, b) < 1e-8, rel(a, b)
    np.testing.assert_allclose(res, ref_res, rtol=1e-9)
