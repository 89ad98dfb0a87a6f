"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks it against a
hand-worked example, a brute-force loop over the definitions, a closed form,
a library special case, or a property the exact LS solution must have.  Some
tests plant a plausible mistake in a copy of an oracle step and check that the
pins catch it.
"""
import itertools
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
import trals_inputs as TI

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_example():
    G1 = np.zeros((2, 2, 1)); G1[:, 0, 0] = [1, 2]; G1[:, 1, 0] = [0, -1]
    G2 = np.zeros((1, 2, 1)); G2[0, 0, 0] = 3; G2[0, 1, 0] = -2
    G3 = np.zeros((1, 2, 2)); G3[0, 0, :] = [1, 1]; G3[0, 1, :] = [2, -1]
    rows = {}
    with open(os.path.join(GOLDEN, "tr_worked_example.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            rows[key] = np.array([float(v) for v in vals])
    return [G1, G2, G3], rows


def _brute_unfold(X, n, classical):
    """Entrywise unfolding from the index definitions of Sec. 2 (loops only)."""
    N = X.ndim
    I = X.shape
    others = [j for j in range(N) if j != n] if classical else [(n + t) % N for t in range(1, N)]
    out = np.zeros((I[n], int(np.prod([I[j] for j in others]))))
    for idx in itertools.product(*[range(i) for i in I]):
        col = O.linear_index([idx[j] for j in others], [I[j] for j in others])
        out[idx[n], col] = X[idx]
    return out


# --------------------------------------------------------------------------- Sec. 1 / Sec. 2
def test_worked_example_element_and_unfolding():
    cores, g = _golden_example()
    X = O.tr_full(cores)
    np.testing.assert_array_equal(TI.flat_f(X), g["X"])
    np.testing.assert_array_equal(O.unfold_mode(X, 1)[0], g["X_[2]row0"])
    np.testing.assert_array_equal(O.unfold_mode(X, 1)[1], g["X_[2]row1"])
    assert float(np.sum(X * X)) == g["normsq"][0]
    for idx in itertools.product(range(2), range(2), range(2)):
        assert O.tr_element(cores, idx) == X[idx]


def test_rank_one_cores_give_outer_product():
    # R = 1: X(i) = prod_n g_n(i_n), the outer product (closed form)
    I = (3, 4, 2, 5)
    cores = TI.gaussian_cores(5, I, (1, 1, 1, 1))
    expect = cores[0][0, :, 0]
    for G in cores[1:]:
        expect = np.multiply.outer(expect, G[0, :, 0])
    np.testing.assert_allclose(O.tr_full(cores), expect, rtol=1e-13, atol=1e-13)


def test_diagonal_cores_give_cp_model():
    # Diagonal lateral slices: X(i) = sum_r prod_n U_n[i_n, r], the CP model (closed form)
    I = (4, 3, 5); Rk = 3
    rng = np.random.default_rng(7)
    U = [rng.standard_normal((i, Rk)) for i in I]
    cores = []
    for n, i in enumerate(I):
        G = np.zeros((Rk, i, Rk))
        for r in range(Rk):
            G[r, :, r] = U[n][:, r]
        cores.append(G)
    expect = np.einsum("ar,br,cr->abc", *U)
    np.testing.assert_allclose(O.tr_full(cores), expect, rtol=1e-12, atol=1e-12)


def test_tr_full_matches_element_brute_force_mixed_ranks():
    I = (3, 2, 4, 2); R = (2, 3, 1, 2)
    cores = TI.gaussian_cores(11, I, R)
    X = O.tr_full(cores)
    for idx in itertools.product(*[range(i) for i in I]):
        assert abs(X[idx] - O.tr_element(cores, idx)) < 1e-12


@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_unfoldings_match_index_definitions(n):
    X = np.random.default_rng(3).standard_normal((3, 2, 4, 5))
    np.testing.assert_array_equal(O.unfold_mode(X, n), _brute_unfold(X, n, classical=False))
    np.testing.assert_array_equal(O.unfold_classical(X, n), _brute_unfold(X, n, classical=True))


def test_unfolding_library_special_cases():
    X = np.random.default_rng(4).standard_normal((3, 2, 4))
    # mode 1: both unfoldings are the column-major reshape (numpy library routine)
    np.testing.assert_array_equal(O.unfold_mode(X, 0), X.reshape(3, -1, order="F"))
    np.testing.assert_array_equal(O.unfold_classical(X, 0), X.reshape(3, -1, order="F"))
    # last mode classical unfolding is the row-major-transposed reshape
    np.testing.assert_array_equal(O.unfold_classical(X, 2), X.reshape(-1, 4, order="F").T)
    # n-unfolding: library reshape
    np.testing.assert_array_equal(O.n_unfolding(X, 2), X.reshape(6, 4, order="F"))


def test_core_fold_roundtrip_and_layout():
    G = np.random.default_rng(5).standard_normal((2, 3, 4))
    Z = O.core_unfold2(G)
    for a, i, b in itertools.product(range(2), range(3), range(4)):
        assert Z[i, a + 2 * b] == G[a, i, b]
    np.testing.assert_array_equal(O.core_fold2(Z, 2, 4), G)


@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_subchain_rows_brute_force(n):
    I = (3, 2, 4, 2); R = (2, 3, 1, 2)
    cores = TI.gaussian_cores(12, I, R)
    A = O.subchain_unfolded(cores, n)
    N = 4
    modes = [(n + t) % N for t in range(1, N)]
    for idx in itertools.product(*[range(I[m]) for m in modes]):
        k = O.linear_index(idx, [I[m] for m in modes])
        P = np.eye(cores[modes[0]].shape[0])
        for m, i in zip(modes, idx):
            P = P @ cores[m][:, i, :]
        Rn = cores[n].shape[0]
        for a, b in itertools.product(range(Rn), range(cores[n].shape[2])):
            assert abs(A[k, a + Rn * b] - P[b, a]) < 1e-13
    np.testing.assert_allclose(O.subchain_rows(cores, n, 0, A.shape[0]), A, rtol=0, atol=1e-13)
    np.testing.assert_allclose(O.subchain_rows(cores, n, 5, 11), A[5:11], rtol=0, atol=1e-13)


@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_als_model_identity(n):
    # X_[n] = G_{n(2)} (G^{!=n}_[2])^T for X = TR(cores) (the model behind eq. tr_als),
    # with X from the element formula evaluated by brute force.
    I = (3, 2, 4, 2); R = (2, 3, 1, 2)
    cores = TI.gaussian_cores(13, I, R)
    X = np.zeros(I)
    for idx in itertools.product(*[range(i) for i in I]):
        X[idx] = O.tr_element(cores, idx)
    lhs = O.unfold_mode(X, n)
    rhs = O.core_unfold2(cores[n]) @ O.subchain_unfolded(cores, n).T
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


def test_subchain_product_definition():
    A = np.random.default_rng(6).standard_normal((2, 3, 4))
    B = np.random.default_rng(7).standard_normal((4, 5, 3))
    C = O.subchain_product(A, B)
    for j1, j2 in itertools.product(range(3), range(5)):
        np.testing.assert_allclose(C[:, j1 + 3 * j2, :], A[:, j1, :] @ B[:, j2, :], rtol=1e-14, atol=1e-14)


def test_slice_kron_proposition():
    # Prop. slice_kron: (A x_2 Ma) [x] (B x_2 Mb) = (A [x] B) x_2 (Mb (x) Ma)
    rng = np.random.default_rng(8)
    A = rng.standard_normal((2, 3, 4)); B = rng.standard_normal((4, 5, 2))
    Ma = rng.standard_normal((6, 3)); Mb = rng.standard_normal((7, 5))
    ttm2 = lambda T, M: np.einsum("ajb,kj->akb", T, M)
    lhs = O.subchain_product(ttm2(A, Ma), ttm2(B, Mb))
    rhs = ttm2(O.subchain_product(A, B), np.kron(Mb, Ma))
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------------------- Sec. 3.1 structure
@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_structured_coefficient_matrix_equals_explicit_gram(n):
    I = (4, 3, 5, 3); R = (2, 3, 2, 4)
    cores = TI.gaussian_cores(14, I, R)
    A = O.subchain_unfolded(cores, n)
    S = A.T @ A
    Sp = O.paper_coefficient_matrix(cores, n)
    assert np.abs(S - Sp).max() <= 1e-12 * np.abs(S).max()
    # Gamma-chain form: Pi_n = Gamma_{n+1} ... Gamma_{n-1};  S[(a,b),(a',b')] = Pi[(b,b'),(a,a')]
    N = 4
    modes = [(n + t) % N for t in range(1, N)]
    Pi = O.gamma(cores[modes[0]])
    for m in modes[1:]:
        Pi = Pi @ O.gamma(cores[m])
    Rn, Rn1 = cores[n].shape[0], cores[n].shape[2]
    S2 = Pi.reshape(Rn1, Rn1, Rn, Rn).transpose(3, 1, 2, 0).reshape(Rn * Rn1, Rn * Rn1, order="F")
    assert np.abs(S - S2).max() <= 1e-12 * np.abs(S).max()


def test_gamma_is_regrouped_core_gram():
    G = np.random.default_rng(9).standard_normal((3, 7, 2))
    Gm = O.gamma(G)
    C = O.core_unfold2(G).T @ O.core_unfold2(G)      # (a + 3b, a' + 3b')
    for p, q, s, t in itertools.product(range(3), range(3), range(2), range(2)):
        assert abs(Gm[p * 3 + q, s * 2 + t] - C[p + 3 * s, q + 3 * t]) < 1e-12


def test_trace_identity_and_inner_product_reading():
    I = (3, 4, 2, 3)
    ca = TI.gaussian_cores(15, I, (2, 3, 2, 2))
    cb = TI.gaussian_cores(16, I, (3, 1, 2, 2))
    Xa, Xb = O.tr_full(ca), O.tr_full(cb)
    # |TR|^2 = Trace(Gamma_1 ... Gamma_N)
    P = O.gamma(ca[0])
    for G in ca[1:]:
        P = P @ O.gamma(G)
    assert abs(np.trace(P) - np.sum(Xa * Xa)) <= 1e-12 * np.sum(Xa * Xa)
    # corrected reading of the by-product proposition
    assert abs(O.tr_inner(ca, cb) - np.sum(Xa * Xb)) <= 1e-12 * np.sqrt(np.sum(Xa**2) * np.sum(Xb**2))
    assert abs(O.tr_inner(ca, ca) - np.sum(Xa * Xa)) <= 1e-12 * np.sum(Xa * Xa)
    # the printed Trace(T_<2>) is not the inner product
    assert abs(O.tr_inner_as_printed(ca, ca) - np.sum(Xa * Xa)) > 1e-3 * np.sum(Xa * Xa)


# --------------------------------------------------------------------------- least squares
def _small_problem(seed=20, I=(5, 4, 6, 3), R=(2, 3, 2, 2), eta=0.05):
    cores = TI.gaussian_cores(seed, I, R)
    X = TI.add_relative_noise(O.tr_full(cores), TI.gaussian_noise(seed, I), eta)
    return X, TI.init_cores(seed, I, R)


@pytest.mark.parametrize("n", [0, 2])
def test_ls_solution_optimality(n):
    X, init = _small_problem()
    A = O.subchain_unfolded(init, n)
    Xn = O.unfold_mode(X, n)
    Z = O.ls_solve_qr(A, Xn)
    # first-order optimality: A^T (A Z^T - Xn^T) = 0
    g = A.T @ (A @ Z.T - Xn.T)
    assert np.abs(g).max() <= 1e-10 * np.abs(A).max() ** 2 * np.abs(Z).max()
    # agrees with LAPACK's SVD-based least squares (library special case)
    Zs = sla.lstsq(A, Xn.T, lapack_driver="gelsd")[0].T
    np.testing.assert_allclose(Z, Zs, rtol=1e-10, atol=1e-12)
    # no random perturbation does better
    base = np.linalg.norm(A @ Z.T - Xn.T)
    rng = np.random.default_rng(1)
    for _ in range(5):
        Zp = Z + 1e-3 * rng.standard_normal(Z.shape)
        assert np.linalg.norm(A @ Zp.T - Xn.T) > base


def test_normal_equations_blockwise_match_explicit():
    X, init = _small_problem()
    for n in range(4):
        A = O.subchain_unfolded(init, n)
        S, M = O.normal_equation_terms(X, init, n, block=7)
        np.testing.assert_allclose(S, A.T @ A, rtol=1e-12, atol=1e-10)
        np.testing.assert_allclose(M, O.unfold_mode(X, n) @ A, rtol=1e-12, atol=1e-10)


def test_mttsp_blockwise_matches_model_identity():
    """O.mttsp (blockwise over subchain rows) against two independent facts: the explicit product
    X_[n] G^{!=n}_[2] for any X, and, for an exact TR tensor X = TR(cores), the ALS model identity
    X_[n] = G_{n(2)} (G^{!=n}_[2])^T, which gives M_n = G_{n(2)} S_n with S_n the structured
    coefficient matrix of Prop. subchain_gram (chained Gram tensors, no subchain matrix)."""
    X, init = _small_problem()
    for n in range(4):
        A = O.subchain_unfolded(init, n)
        np.testing.assert_allclose(O.mttsp(X, init, n, block=7), O.unfold_mode(X, n) @ A, rtol=1e-12, atol=1e-10)
        Xt = O.tr_full(init)
        S = O.paper_coefficient_matrix(init, n)
        want = O.core_unfold2(init[n]) @ S
        np.testing.assert_allclose(O.mttsp(Xt, init, n, block=5), want, rtol=1e-10, atol=1e-9 * np.abs(want).max())


def test_mttsp_column_matches_brute_force():
    """O.mttsp_column (one column of M_n from the subchain entries carried through the chain, for
    sampled checks of large tensors) against a brute-force sum over every multi-index of the other
    modes: M_n[i, a + R_n b] = sum X(.., i_n = i, ..) (G_{n+1}(i_{n+1}) ... G_{n-1}(i_{n-1}))[b, a]
    (the mode-n unfolding and eq. subchain_new), with the other modes indexed through the tensor's
    axes, not through a linear index."""
    I, R = (3, 4, 2, 3), (2, 3, 2, 2)
    N = len(I)
    cores = TI.gaussian_cores(11, I, R)
    X = np.random.default_rng(11).standard_normal(I)
    for n in range(N):
        others = [(n + t) % N for t in range(1, N)]
        for a in range(R[n]):
            for b in range(R[(n + 1) % N]):
                want = np.zeros(I[n])
                for i in range(I[n]):
                    for idx in itertools.product(*[range(I[m]) for m in others]):
                        P = np.eye(R[(n + 1) % N])
                        full = [0] * N
                        full[n] = i
                        for m, im in zip(others, idx):
                            P = P @ cores[m][:, im, :]
                            full[m] = im
                        want[i] += X[tuple(full)] * P[b, a]
                got = O.mttsp_column(X, cores, n, a, b)
                np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


def test_signed_selection_cores_keep_subchain_entries_ternary():
    """The exact-arithmetic GPU tests rely on every subchain entry of these cores being -1, 0 or +1
    with at most one nonzero per row of each G^{!=n}(k) (brute force through the oracle)."""
    I, R = (5, 4, 6, 3), (3, 4, 2, 5)
    cores = TI.signed_selection_cores(3, I, R)
    for G in cores:
        assert set(np.unique(G)) <= {-1.0, 0.0, 1.0}
        assert (np.abs(G).sum(axis=2) <= 1).all()
    for n in range(4):
        T = O.subchain_tensor(cores, n)          # (R_{n+1}, J, R_n)
        assert set(np.unique(T)) <= {-1.0, 0.0, 1.0}
        assert (np.abs(T).sum(axis=2) <= 1).all()
        assert np.count_nonzero(T) > 0
    X = TI.small_integer_tensor(3, I, amp=8)
    assert np.array_equal(X, np.round(X)) and np.abs(X).max() <= 8


def test_svd_solve_is_the_minimum_norm_least_squares_solution():
    """ls_solve_svd: equal to the QR solution for full-rank A; for a rank-deficient A (two equal columns)
    it satisfies the normal equations and has no component in the null space of A (the minimum-norm
    solution), and it is unique where QR least squares is not defined."""
    rng = np.random.default_rng(30)
    A = rng.standard_normal((40, 6))
    Xn = rng.standard_normal((5, 40))
    np.testing.assert_allclose(O.ls_solve_svd(A, Xn), O.ls_solve_qr(A, Xn), rtol=1e-10, atol=1e-12)
    A[:, 4] = A[:, 1]
    Z = O.ls_solve_svd(A, Xn)
    np.testing.assert_allclose(A.T @ (A @ Z.T - Xn.T), 0.0, atol=1e-10)
    null = np.zeros(6); null[1], null[4] = 1.0, -1.0
    assert np.abs(Z @ null).max() < 1e-12
    # any other least-squares solution (adding a null-space component) is longer
    Z2 = Z + 0.3 * np.outer(np.ones(5), null)
    np.testing.assert_allclose(A.T @ (A @ Z2.T - Xn.T), 0.0, atol=1e-10)
    assert np.linalg.norm(Z2) > np.linalg.norm(Z)


def test_ne_and_qr_agree_after_one_sweep():
    X, init = _small_problem()
    c_qr, _ = O.tr_als(X, init, 1, "qr", residual=False)
    c_ne, _ = O.tr_als(X, init, 1, "chol", residual=False)
    for a, b in zip(c_qr, c_ne):
        assert np.abs(a - b).max() <= 1e-11 * np.abs(a).max()


def test_residual_monotone_non_increasing():
    X, init = _small_problem(eta=0.2)
    _, res = O.tr_als(X, init, 8, "qr")
    for r0, r1 in zip(res, res[1:]):
        assert r1 <= r0 * (1 + 1e-12)


def test_exact_recovery_from_perturbed_truth():
    I = (10, 9, 11); R = (2, 3, 2)
    truth = TI.gaussian_cores(21, I, R)
    X = O.tr_full(truth)
    rng = np.random.default_rng(2)
    init = [G + 1e-2 * rng.standard_normal(G.shape) for G in truth]
    _, res = O.tr_als(X, init, 40, "qr")
    assert res[-1] < 1e-10


def test_noise_floor_true_rank_fit():
    # fit rank = true rank: the converged relative residual sits near eta (observation model of Sec. 4)
    I = (20, 20, 20); R = (3, 3, 3); eta = 1e-3
    truth = TI.gaussian_cores(22, I, R)
    X = TI.add_relative_noise(O.tr_full(truth), TI.gaussian_noise(22, I), eta)
    rng = np.random.default_rng(3)
    init = [G + 1e-2 * rng.standard_normal(G.shape) for G in truth]
    _, res = O.tr_als(X, init, 10, "chol")
    assert 0.9 * eta < res[-1] < 1.0 * eta


def test_relative_noise_level():
    Xt = np.random.default_rng(1).standard_normal((4, 5, 6))
    Nz = TI.gaussian_noise(3, (4, 5, 6))
    X = TI.add_relative_noise(Xt, Nz, 0.3)
    assert abs(np.linalg.norm(X - Xt) / np.linalg.norm(Xt) - 0.3) < 1e-14


def test_residual_identity_matches_explicit():
    X, init = _small_problem(eta=0.1)
    cores, res = O.tr_als(X, init, 2, "chol")
    n = 3
    S, M = O.normal_equation_terms(X, cores, n)
    # re-solve the last mode from the converged others: the identity then holds at the update
    Z = O.ls_solve_normal(S, M)
    c2 = list(cores); c2[n] = O.core_fold2(Z, cores[n].shape[0], cores[n].shape[2])
    r2 = O.residual_identity(float(np.sum(X * X)), M, Z, S)
    explicit = np.sum((X - O.tr_full(c2)) ** 2)
    assert abs(r2 - explicit) <= 1e-9 * np.sum(X * X)


# --------------------------------------------------------------------------- Sec. 3.2 QR
def test_mode2_qr_definition_both_cases():
    rng = np.random.default_rng(30)
    for shape in [(2, 9, 3), (4, 3, 4)]:          # I_2 >= I_1 I_3 and I_2 <= I_1 I_3
        T = rng.standard_normal(shape)
        Rt, Q = O.mode2_qr(T)
        np.testing.assert_allclose(Q.T @ Q, np.eye(Q.shape[1]), atol=1e-13)
        recon = np.einsum("ajb,kj->akb", Rt, Q)
        np.testing.assert_allclose(recon, T, rtol=1e-12, atol=1e-12)
        R2 = O.unfold3_mode2(Rt)
        assert np.allclose(np.tril(R2, -1), 0.0)


@pytest.mark.parametrize("I,R", [((5, 4, 6, 3), (2, 3, 2, 2)), ((4, 6, 3, 5), (2, 2, 2, 2))])
def test_tr_als_qr_matches_regular_als(I, R):
    # remark after Alg. 3: TR-ALS-QR equals TR-ALS in exact arithmetic (incl. I_j < R_j R_{j+1})
    X, init = _small_problem(I=I, R=R)
    c_ref, r_ref = O.tr_als(X, init, 3, "qr")
    c_qr, r_qr = O.tr_als_qr(X, init, 3)
    for a, b in zip(c_ref, c_qr):
        assert np.abs(a - b).max() <= 1e-9 * np.abs(a).max()
    np.testing.assert_allclose(r_qr, r_ref, rtol=1e-10)


@pytest.mark.parametrize("I,R", [((9, 8, 10), (2, 2, 2)), ((12, 3, 11, 10), (2, 3, 2, 2))])
def test_tr_als_qrne_matches_regular_als(I, R):
    """TR-ALS-QRNE solves the same least-squares problems as TR-ALS (Sec. 3.3): the cores after a
    sweep agree with Householder least squares on the explicit subchain matrix.  Modes 1 and 3 of
    the second shape compress (I_j > R_j R_{j+1}); mode 2 (I = 3 < 6) keeps its square Q."""
    X, init = _small_problem(seed=23, I=I, R=R, eta=0.05)
    a, ra = O.tr_als_qrne(X, init, 2)
    b, rb = O.tr_als(X, init, 2, "qr")
    for Ga, Gb in zip(a, b):
        np.testing.assert_allclose(Ga, Gb, rtol=1e-9, atol=1e-10 * np.abs(Gb).max())
    np.testing.assert_allclose(ra, rb, rtol=1e-10)


def test_qrne_compressed_terms_equal_the_uncompressed_ones():
    """M_n = Y_[n] V_n[2] with Y = X x_{j!=n} Q_j^T equals X_[n] G^{!=n}_[2] (Prop. slice_kron and
    Prop. ttm), and the coefficient matrix from the Gram tensors of the R factors equals the explicit
    (G^{!=n}_[2])^T G^{!=n}_[2]."""
    I, R = (7, 3, 9, 8), (2, 2, 3, 2)
    X, cores = _small_problem(seed=24, I=I, R=R, eta=0.1)
    QR = [O.mode2_qr(G) for G in cores]
    for n in range(4):
        Yn = O.multi_ttm_mode_unfolded(X, [q[1] for q in QR], n)
        V2 = O.subchain_unfolded([q[0] for q in QR], n)
        A = O.subchain_unfolded(cores, n)          # pinned to brute force in test_subchain_rows_brute_force
        np.testing.assert_allclose(Yn @ V2, O.unfold_mode(X, n) @ A, rtol=1e-11, atol=1e-11 * np.abs(X).max())
        S = O.paper_coefficient_matrix([q[0] for q in QR], n)
        np.testing.assert_allclose(S, A.T @ A, rtol=1e-11, atol=1e-11 * np.abs(A.T @ A).max())


def test_subspace_angle_gauge_invariance():
    X, init = _small_problem()
    cores, _ = O.tr_als(X, init, 2, "qr", residual=False)
    rng = np.random.default_rng(31)
    N = len(cores)
    gauges = [rng.standard_normal((G.shape[0], G.shape[0])) + 3 * np.eye(G.shape[0]) for G in cores]
    # G_n(i) -> A_n^{-1} G_n(i) A_{n+1}
    gauged = [np.einsum("ab,bic,cd->aid", np.linalg.inv(gauges[n]), cores[n], gauges[(n + 1) % N]) for n in range(N)]
    np.testing.assert_allclose(O.tr_full(gauged), O.tr_full(cores), rtol=1e-9, atol=1e-9)
    for n in range(N):
        assert O.subchain_principal_angle(cores, gauged, n) < 1e-6
    other = TI.gaussian_cores(99, X.shape, [G.shape[0] for G in cores])
    assert O.subchain_principal_angle(cores, other, 0) > 1e-3


# --------------------------------------------------------------------------- planted mistakes
def test_pins_catch_planted_mistakes(monkeypatch):
    """Plant a plausible error in a copy of an oracle step; the pins above must reject it."""
    I = (3, 2, 4); R = (2, 3, 2)
    cores = TI.gaussian_cores(40, I, R)
    X = O.tr_full(cores)

    # (1) reversed chain order in the subchain (G_{n-1} ... G_{n+1}) breaks the model identity
    Ieq = (3, 2, 4, 3); Req = (2, 2, 2, 2)
    ceq = TI.gaussian_cores(41, Ieq, Req)
    Xeq = O.tr_full(ceq)

    def wrong_chain(N, n):
        return [(n - t) % N for t in range(1, N)]
    monkeypatch.setattr(O.trals_oracle, "chain_modes", wrong_chain)
    bad = O.core_unfold2(ceq[0]) @ O.subchain_unfolded(ceq, 0).T
    monkeypatch.undo()
    assert np.abs(bad - O.unfold_mode(Xeq, 0)).max() > 1e-3
    good = O.core_unfold2(ceq[0]) @ O.subchain_unfolded(ceq, 0).T
    assert np.abs(good - O.unfold_mode(Xeq, 0)).max() < 1e-12

    # (2) a dropped term in Gamma (first slice omitted) breaks the trace identity
    good = O.gamma(cores[0]) @ O.gamma(cores[1]) @ O.gamma(cores[2])
    assert abs(np.trace(good) - np.sum(X * X)) < 1e-10 * np.sum(X * X)
    dropped = [sum(np.kron(G[:, i, :], G[:, i, :]) for i in range(1, G.shape[1])) for G in cores]
    assert abs(np.trace(dropped[0] @ dropped[1] @ dropped[2]) - np.sum(X * X)) > 1e-6 * np.sum(X * X)
    # ... and so does a transposed Kronecker factor order in the regrouping of S_n
    A = O.subchain_unfolded(ceq, 1)
    Pi = O.gamma(ceq[2]) @ O.gamma(ceq[3]) @ O.gamma(ceq[0])
    S_wrong = Pi.reshape(2, 2, 2, 2).transpose(1, 3, 0, 2).reshape(4, 4, order="F")
    assert np.abs(S_wrong - A.T @ A).max() > 1e-6 * np.abs(A.T @ A).max()

    # (3) a sign flip in the residual identity's cross term breaks its agreement with the explicit residual
    Xn = TI.add_relative_noise(X, TI.gaussian_noise(1, I), 0.1)
    S, M = O.normal_equation_terms(Xn, cores, 2)
    Z = O.ls_solve_normal(S, M)
    c2 = list(cores); c2[2] = O.core_fold2(Z, 2, 2)
    explicit = np.sum((Xn - O.tr_full(c2)) ** 2)
    flipped = float(np.sum(Xn * Xn) + 2.0 * np.sum(M * Z) + np.sum(S * (Z.T @ Z)))
    assert abs(flipped - explicit) > 1e-3 * explicit
    assert abs(O.residual_identity(float(np.sum(Xn * Xn)), M, Z, S) - explicit) < 1e-9 * np.sum(Xn * Xn)


# --------------------------------------------------------------------------- BF16 storage
def test_bf16_rne_matches_torch_and_ties():
    import torch
    rng = np.random.default_rng(50)
    x = np.concatenate([rng.standard_normal(10000) * 10.0 ** rng.integers(-8, 8, 10000),
                        [0.0, -0.0, 1.0, -2.5, 3.0e38, 1e-40]])
    bits = O.bf16_rne_bits(x)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(bits, ref)
    # exact ties: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7 -> even (1.0); 1 + 3*2^-8 -> 1 + 2^-6
    assert O.bf16_bits_to_f64(O.bf16_rne_bits(1.0 + 2.0 ** -8))[()] == 1.0
    assert O.bf16_bits_to_f64(O.bf16_rne_bits(1.0 + 3 * 2.0 ** -8))[()] == 1.0 + 2.0 ** -6
    hi, lo = O.bf16_split(x[:10000])
    rel = np.abs(O.bf16_bits_to_f64(hi) + O.bf16_bits_to_f64(lo) - x[:10000]) / np.abs(x[:10000])
    assert rel.max() < 2.0 ** -16
