"""Plain, slow, FP64 CPU oracle for tensor-ring ALS.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
link this module: only the tests, the smoke check and the benchmark's CPU
baseline leg use it.  It shares no code with the CUDA path.

It follows Yu & Li, "Practical Alternating Least Squares for Tensor Ring
Decomposition" (arXiv 2210.11362).  Every function states the passage it
implements.  Mode indices are 0-based in code (the paper's mode n is code
mode n-1); every other index convention is the paper's:

* linear index overline{i_1 ... i_N} = sum_n i_n prod_{j<n} I_j, first index
  fastest (Sec. 2), so dense tensors flatten in column-major order;
* core G_n has shape (R_n, I_n, R_{n+1}), R_{N+1} = R_1, lateral slice
  G_n(i_n) = G_n[:, i_n, :] (Sec. 1);
* the classical mode-2 unfolding G_{n(2)} of a core is I_n x R_n R_{n+1} with
  column r_n + R_n r_{n+1} (Def. classical mode-n unfolding);
* the subchain unfolding G^{!=n}_[2] is J_n x R_n R_{n+1} with row
  overline{i_{n+1} ... i_N i_1 ... i_{n-1}} and column r_n + R_n r_{n+1}
  (Def. subchain tensor, Def. mode-n unfolding).

What it computes is regular TR-ALS (Alg. 1): the subchain matrix is formed
explicitly and each subproblem (eq. tr_als) is solved by Householder QR
least squares, or by Cholesky on the explicit normal equations (the
Golub & Van Loan Sec. 5.3.2 method the paper cites for Alg. 2), plus
TR-ALS-QR (Alg. 3, derived from the least-squares problem of Sec. 3.2) for
small shapes.  The paper proves TR-ALS-NE and TR-ALS-QR equal TR-ALS in exact
arithmetic (remarks after Alg. 2 and Alg. 3), so this oracle is the reference
for every GPU solver.

Parity pins: every function here is pinned by tests/test_oracle_pins.py to
brute force, closed forms or library special cases; nothing is "parity
unpinned" except where stated in a function's docstring.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np
import scipy.linalg as sla


# ---------------------------------------------------------------------------
# Sec. 1 / Sec. 2: the TR format, linear index and unfoldings
# ---------------------------------------------------------------------------
def linear_index(idx: Sequence[int], dims: Sequence[int]) -> int:
    """overline{i_1 ... i_N} (Sec. 2), 0-based: sum_n i_n prod_{j<n} I_j."""
    lin, stride = 0, 1
    for i, d in zip(idx, dims):
        lin += int(i) * stride
        stride *= int(d)
    return lin


def tr_element(cores: Sequence[np.ndarray], idx: Sequence[int]) -> float:
    """X(i_1..i_N) = Trace(G_1(i_1) G_2(i_2) ... G_N(i_N)) (Sec. 1), by the definition."""
    P = cores[0][:, idx[0], :]
    for n in range(1, len(cores)):
        P = P @ cores[n][:, idx[n], :]
    return float(np.trace(P))


def tr_full(cores: Sequence[np.ndarray]) -> np.ndarray:
    """The dense tensor TR({G_n}) of shape (I_1..I_N) (Sec. 1).

    Forms the running products Z(i_1..i_m) = G_1(i_1)...G_m(i_m) for every
    prefix index m < N (a library batched matmul per step), then evaluates
    Trace(Z(i_1..i_{N-1}) G_N(i_N)) = sum_{a,c} Z[a, k, c] G_N[c, i_N, a] for all
    indices at once: the element formula, without an R x J x I x R intermediate.
    """
    N = len(cores)
    I = [G.shape[1] for G in cores]
    # Z: (R_1, K, R_{m+1}) with K = overline{i_1..i_m} (i_1 fastest)
    Z = cores[0]
    for m in range(1, N - 1):
        G = cores[m]
        # new[r, k + K*i_m, s] = sum_c Z[r, k, c] G[c, i_m, s]
        new = np.einsum("akc,cis->akis", Z, G, optimize=True)
        Z = new.reshape(Z.shape[0], Z.shape[1] * G.shape[1], G.shape[2], order="F")
    GN = cores[N - 1]
    # vals[k, i_N] = sum_{a,c} Z[a, k, c] GN[c, i_N, a]
    Zm = np.transpose(Z, (1, 0, 2)).reshape(Z.shape[1], -1)            # (K, a*R_N + c)
    Gm = np.transpose(GN, (2, 0, 1)).reshape(-1, GN.shape[1])          # (a*R_N + c, I_N)
    vals = Zm @ Gm
    return vals.reshape(tuple(I), order="F")


def unfold_classical(X: np.ndarray, n: int) -> np.ndarray:
    """Classical mode-n unfolding X_(n) (Def. classical mode-n unfolding).

    I_n x prod_{j!=n} I_j; column overline{i_1 .. i_{n-1} i_{n+1} .. i_N}.
    """
    N = X.ndim
    order = [n] + [j for j in range(N) if j != n]
    return np.transpose(X, order).reshape(X.shape[n], -1, order="F")


def unfold_mode(X: np.ndarray, n: int) -> np.ndarray:
    """Mode-n unfolding X_[n] (Def. mode-n unfolding).

    I_n x prod_{j!=n} I_j; column overline{i_{n+1} .. i_N i_1 .. i_{n-1}}.
    """
    N = X.ndim
    order = [n] + [(n + t) % N for t in range(1, N)]
    return np.transpose(X, order).reshape(X.shape[n], -1, order="F")


def core_unfold2(G: np.ndarray) -> np.ndarray:
    """Classical mode-2 unfolding G_{n(2)} of a core: I_n x R_n R_{n+1}, column r_n + R_n r_{n+1}."""
    return unfold_classical(G, 1)


def core_fold2(Z: np.ndarray, Rn: int, Rn1: int) -> np.ndarray:
    """Inverse of ``core_unfold2``: G[a, i, b] = Z[i, a + Rn b]."""
    In = Z.shape[0]
    return np.transpose(Z.reshape(In, Rn, Rn1, order="F"), (1, 0, 2)).copy()


# ---------------------------------------------------------------------------
# Sec. 2: subchain product and subchain tensor
# ---------------------------------------------------------------------------
def subchain_product(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Mode-2 subchain product (Def. subchain product): (A [x]_2 B)(overline{j1 j2}) = A(j1) B(j2).

    A: I1 x J1 x K, B: K x J2 x I2  ->  I1 x J1 J2 x I2, lateral index j1 + J1 j2.
    """
    assert A.shape[2] == B.shape[0]
    out = np.einsum("ajk,kbc->ajbc", A, B)  # out[:, j1, j2, :] = A(j1) @ B(j2)
    return out.reshape(A.shape[0], A.shape[1] * B.shape[1], B.shape[2], order="F")


def chain_modes(N: int, n: int) -> List[int]:
    """The order of the other modes in the subchain: n+1, ..., N, 1, ..., n-1 (eq. subchain_new)."""
    return [(n + t) % N for t in range(1, N)]


def subchain_tensor(cores: Sequence[np.ndarray], n: int) -> np.ndarray:
    """G^{!=n} = G_{n+1} [x]_2 ... [x]_2 G_N [x]_2 G_1 [x]_2 ... [x]_2 G_{n-1} (eq. subchain_new).

    Shape R_{n+1} x J_n x R_n with lateral slice overline{i_{n+1}..i_{n-1}} equal
    to G_{n+1}(i_{n+1}) ... G_{n-1}(i_{n-1}) (Def. subchain tensor).
    """
    modes = chain_modes(len(cores), n)
    T = cores[modes[0]]
    for m in modes[1:]:
        T = subchain_product(T, cores[m])
    return T


def subchain_unfolded(cores: Sequence[np.ndarray], n: int) -> np.ndarray:
    """G^{!=n}_[2]: J_n x R_n R_{n+1}, row k, column a + R_n b, entry G^{!=n}(k)[b, a]."""
    T = subchain_tensor(cores, n)          # (R_{n+1}, J, R_n)
    J = T.shape[1]
    return np.transpose(T, (1, 2, 0)).reshape(J, -1, order="F")


def subchain_rows(cores: Sequence[np.ndarray], n: int, k0: int, k1: int) -> np.ndarray:
    """Rows k0..k1-1 of G^{!=n}_[2], formed row by row from the definition (for blockwise use)."""
    N = len(cores)
    modes = chain_modes(N, n)
    dims = [cores[m].shape[1] for m in modes]
    ks = np.arange(k0, k1)
    # decode k = overline{i_{n+1} .. i_{n-1}} (first fastest)
    idx = []
    rem = ks.copy()
    for d in dims:
        idx.append(rem % d)
        rem //= d
    P = cores[modes[0]][:, idx[0], :].transpose(1, 0, 2)        # (B, R_{n+1}, R)
    for t in range(1, len(modes)):
        P = P @ cores[modes[t]][:, idx[t], :].transpose(1, 0, 2)
    # P[k] = G^{!=n}(k) : (B, R_{n+1}, R_n); row of G_[2]: column a + R_n b -> P[k][b, a]
    return np.transpose(P, (0, 2, 1)).reshape(len(ks), -1, order="F")


# ---------------------------------------------------------------------------
# Alg. 1 (TR-ALS): subproblem eq. tr_als solved explicitly
# ---------------------------------------------------------------------------
def ls_solve_qr(A: np.ndarray, Xn: np.ndarray) -> np.ndarray:
    """argmin_Z |A Z^T - Xn^T|_F by Householder QR of A (regular least squares); returns Z."""
    Q, Rf = np.linalg.qr(A, mode="reduced")
    return sla.solve_triangular(Rf, Q.T @ Xn.T, lower=False).T


def ls_solve_svd(A: np.ndarray, Xn: np.ndarray, rcond: float = 1e-12) -> np.ndarray:
    """Minimum-norm argmin_Z |A Z^T - Xn^T|_F through the SVD of A, singular values below
    rcond * sigma_max dropped (the SVD option of the remark after Alg. 3, for rank-deficient A)."""
    return np.linalg.lstsq(A, Xn.T, rcond=rcond)[0].T


def ls_solve_normal(S: np.ndarray, M: np.ndarray) -> np.ndarray:
    """Solve Z S = M with S = A^T A symmetric positive definite, by Cholesky S = L L^T
    and two triangular solves (Golub & Van Loan Sec. 5.3.2, cited for Alg. 2 line 9)."""
    L = np.linalg.cholesky(S)
    Y = sla.solve_triangular(L, M.T, lower=True)
    return sla.solve_triangular(L.T, Y, lower=False).T


def normal_equation_terms(X: np.ndarray, cores: Sequence[np.ndarray], n: int,
                          block: int = 1 << 18) -> Tuple[np.ndarray, np.ndarray]:
    """(S_n, M_n) = ((G^{!=n}_[2])^T G^{!=n}_[2],  X_[n] G^{!=n}_[2]) from the explicit
    subchain matrix (Sec. 3.1 normal equation; Alg. 2 lines 7-9 by definition),
    accumulated over row blocks of G^{!=n}_[2] so it never sits in memory whole."""
    Xn = unfold_mode(X, n)
    J = Xn.shape[1]
    r = cores[n].shape[0] * cores[n].shape[2]
    S = np.zeros((r, r))
    M = np.zeros((Xn.shape[0], r))
    for k0 in range(0, J, block):
        k1 = min(J, k0 + block)
        A = subchain_rows(cores, n, k0, k1)
        S += A.T @ A
        M += Xn[:, k0:k1] @ A
    return S, M


def mttsp(X: np.ndarray, cores: Sequence[np.ndarray], n: int, block: int = 1 << 17) -> np.ndarray:
    """M_n = X_[n] G^{!=n}_[2] (Alg. 2 lines 7-8, the tensor-times-subchain product, by its
    definition), accumulated over row blocks of the explicit subchain matrix so that it never sits
    in memory whole."""
    Xn = unfold_mode(X, n)
    J = Xn.shape[1]
    r = cores[n].shape[0] * cores[n].shape[2]
    M = np.zeros((Xn.shape[0], r))
    for k0 in range(0, J, block):
        k1 = min(J, k0 + block)
        M += Xn[:, k0:k1] @ subchain_rows(cores, n, k0, k1)
    return M


def mttsp_column(X: np.ndarray, cores: Sequence[np.ndarray], n: int, a: int, b: int) -> np.ndarray:
    """Column a + R_n b of M_n = X_[n] G^{!=n}_[2] (Alg. 2 lines 7-8) without the subchain matrix:
    the column's subchain entries g(k) = G^{!=n}(k)[b, a] = e_b^T G_{n+1}(i_{n+1}) ... G_{n-1}(i_{n-1}) e_a
    (eq. subchain_new) are formed for all k by carrying the row vector e_b^T G_{n+1}(i_{n+1}) ... through
    the chain, one mode at a time (k = overline{i_{n+1} .. i_{n-1}}, first index fastest), then
    M_n[:, a + R_n b] = X_[n] g.  Memory is J_n / I_{n-1} x R plus J_n, so sampled columns of a large
    tensor's M_n stay cheap."""
    N = len(cores)
    modes = chain_modes(N, n)
    V = cores[modes[0]][b, :, :]                      # (I_{c1}, R): row vectors over k so far
    for m in modes[1:-1]:
        G = cores[m]                                  # (R_c, I_c, R_{c+1})
        Rc, Ic, Rd = G.shape
        # V'[k + K i, :] = V[k, :] @ G(i)
        W = (V @ G.reshape(Rc, Ic * Rd)).reshape(V.shape[0], Ic, Rd)   # W[k, i, d]
        V = W.transpose(1, 0, 2).reshape(Ic * V.shape[0], Rd)           # row i K + k
    last = cores[modes[-1]]                           # (R_c, I_c, R_n): the column a of each slice
    g = (V @ last[:, :, a]).reshape(-1, order="F")    # g[k + K i] = V[k] . G_last(i)[:, a]
    return unfold_mode(X, n) @ g


def als_update(X: np.ndarray, cores: List[np.ndarray], n: int, solver: str = "qr") -> np.ndarray:
    """One TR-ALS core update (Alg. 1 lines 4-5): G_n = argmin |G^{!=n}_[2] Z^T - X_[n]^T|_F."""
    Rn, Rn1 = cores[n].shape[0], cores[n].shape[2]
    if solver == "qr":
        A = subchain_unfolded(cores, n)
        Z = ls_solve_qr(A, unfold_mode(X, n))
    elif solver == "chol":
        S, M = normal_equation_terms(X, cores, n)
        Z = ls_solve_normal(S, M)
    elif solver == "svd":
        Z = ls_solve_svd(subchain_unfolded(cores, n), unfold_mode(X, n))
    else:
        raise ValueError(solver)
    return core_fold2(Z, Rn, Rn1)


def rel_residual(X: np.ndarray, cores: Sequence[np.ndarray]) -> float:
    """|X - TR(cores)|_F / |X|_F with an explicit reconstruction (Sec. 4 error formula)."""
    return float(np.linalg.norm((X - tr_full(cores)).ravel()) / np.linalg.norm(X.ravel()))


def tr_als(X: np.ndarray, init: Sequence[np.ndarray], sweeps: int, solver: str = "qr",
           residual: bool = True) -> Tuple[List[np.ndarray], List[float]]:
    """Regular TR-ALS (Alg. 1) for a fixed number of sweeps over n = 1..N (Sec. 4 protocol).

    Returns the final cores and the explicit relative residual after each sweep.
    """
    cores = [np.array(G, dtype=np.float64, copy=True) for G in init]
    res = []
    for _ in range(sweeps):
        for n in range(len(cores)):
            cores[n] = als_update(X, cores, n, solver)
        if residual:
            res.append(rel_residual(X, cores))
    return cores, res


# ---------------------------------------------------------------------------
# Sec. 3.1: Gram tensors, general contracted product, structured coefficient matrix
# ---------------------------------------------------------------------------
def paper_gram_tensor(G: np.ndarray, Z: np.ndarray | None = None) -> np.ndarray:
    """P = sum_i G(i)^T o Z(i)^T (Alg. 2 line 2; by-product proposition with Z).

    P(p, q, s, t) = sum_i G(i)^T[p, q] Z(i)^T[s, t]; shape R_{n+1} x R_n x S_{n+1} x S_n.
    """
    if Z is None:
        Z = G
    return np.einsum("qip,tis->pqst", G, Z)


def general_contracted(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """(A x_{2,4}^{1,3} B)(i1, i2, r1, r2) = sum_{j,k} A(i1, j, r1, k) B(j, i2, k, r2) (Remark after Prop. subchain_gram)."""
    return np.einsum("ajrk,jbks->abrs", A, B)


def n_unfolding(T: np.ndarray, m: int) -> np.ndarray:
    """n-unfolding X_<m> (Def. n-unfolding): rows overline{i_1..i_m}, columns overline{i_{m+1}..i_N}."""
    rows = int(np.prod(T.shape[:m]))
    return T.reshape(rows, -1, order="F")


def paper_coefficient_tensor(cores: Sequence[np.ndarray], n: int) -> np.ndarray:
    """S_n = P_{n-1} x ... x P_1 x P_N x ... x P_{n+1} (Alg. 2 line 6), contracted with
    the general contracted product, as written in the paper."""
    N = len(cores)
    order = [(n - t) % N for t in range(1, N)]   # n-1, n-2, ..., n+1 (cyclic, descending)
    S = paper_gram_tensor(cores[order[0]])
    for m in order[1:]:
        S = general_contracted(S, paper_gram_tensor(cores[m]))
    return S


def paper_coefficient_matrix(cores: Sequence[np.ndarray], n: int) -> np.ndarray:
    """S_{n<2>}, the normal-equation matrix of Alg. 2 line 9 (Prop. subchain_gram)."""
    return n_unfolding(paper_coefficient_tensor(cores, n), 2)


def gamma(G: np.ndarray) -> np.ndarray:
    """Gamma = sum_i G(i) (x) G(i): R_n^2 x R_{n+1}^2, Kronecker row index p R_n + q.

    A regrouping of the paper's Gram tensor P (Alg. 2 line 2): as a matrix over
    (dim1, dim3) x (dim2, dim4), P equals Gamma^T.
    """
    return sum(np.kron(G[:, i, :], G[:, i, :]) for i in range(G.shape[1]))


# ---------------------------------------------------------------------------
# Sec. 3.4 by-product: inner product of two TR tensors, and the error identity of Sec. 4
# ---------------------------------------------------------------------------
def tr_inner(cores_a: Sequence[np.ndarray], cores_b: Sequence[np.ndarray]) -> float:
    """<TR(G), TR(Z)> from the mixed Gram tensors (by-product proposition, Sec. 3.4).

    Reading adopted: with T = P_N x ... x P_1 (general contracted product) and
    P_n = sum_i G_n(i)^T o Z_n(i)^T, the inner product is sum_{x,y} T(x, x, y, y),
    i.e. the trace that pairs dims (1,2) and (3,4).  The formula as printed,
    Trace(T_<2>), pairs (1,3) with (2,4); it disagrees with brute force (the
    tests show both).
    """
    N = len(cores_a)
    T = paper_gram_tensor(cores_a[N - 1], cores_b[N - 1])
    for m in range(N - 2, -1, -1):
        T = general_contracted(T, paper_gram_tensor(cores_a[m], cores_b[m]))
    return float(np.einsum("xxyy->", T))


def tr_inner_as_printed(cores_a: Sequence[np.ndarray], cores_b: Sequence[np.ndarray]) -> float:
    """Trace((P_N x ... x P_1)_<2>) exactly as the by-product proposition prints it (for the reading test)."""
    N = len(cores_a)
    T = paper_gram_tensor(cores_a[N - 1], cores_b[N - 1])
    for m in range(N - 2, -1, -1):
        T = general_contracted(T, paper_gram_tensor(cores_a[m], cores_b[m]))
    return float(np.trace(n_unfolding(T, 2)))


def residual_identity(normX2: float, M_last: np.ndarray, G_last: np.ndarray, S_last: np.ndarray) -> float:
    """|X - X_hat|_F^2 = |X|^2 - 2 <M_N, G_N(2)> + <S_N, G_N(2)^T G_N(2)> (Sec. 4, TR-ALS-NE case).

    M_last, S_last are the MTTSP result and coefficient matrix of the last mode
    of a sweep, G_last its updated core unfolding G_{N(2)}.
    """
    Z = G_last
    return float(normX2 - 2.0 * np.sum(M_last * Z) + np.sum(S_last * (Z.T @ Z)))


# ---------------------------------------------------------------------------
# Sec. 3.2: mode-2 QR of a 3rd-order tensor and TR-ALS-QR (Alg. 3), small shapes only
# ---------------------------------------------------------------------------
def unfold3_mode2(T: np.ndarray) -> np.ndarray:
    """Mode-2 unfolding T_[2] of a 3rd-order tensor: column overline{i_3 i_1}."""
    return unfold_mode(T, 1)


def fold3_mode2(Z: np.ndarray, I1: int, I3: int) -> np.ndarray:
    """Inverse of ``unfold3_mode2`` for a tensor of shape I1 x Z.shape[0] x I3."""
    I2 = Z.shape[0]
    # Z[i2, i3 + I3 i1] = T[i1, i2, i3]
    return np.transpose(Z.reshape(I2, I3, I1, order="F"), (2, 0, 1)).copy()


def mode2_qr(T: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Mode-2 QR T = R x_2 Q (Def. mode-n QR factorization, both size cases).

    Returns (Rtensor, Q); Rtensor_[2] is upper triangular/trapezoidal of size
    min(I_2, I_1 I_3) x I_1 I_3 and Q has orthonormal columns.
    """
    I1, I2, I3 = T.shape
    Q, Rm = np.linalg.qr(unfold3_mode2(T), mode="reduced")
    return fold3_mode2(Rm, I1, I3), Q


def kron_chain(mats: Sequence[np.ndarray]) -> np.ndarray:
    out = mats[0]
    for m in mats[1:]:
        out = np.kron(out, m)
    return out


def multi_ttm_mode_unfolded(X: np.ndarray, Qs: Sequence[np.ndarray], n: int) -> np.ndarray:
    """Y_[n] for Y = X x_{j!=n} Q_j^T (Alg. 3 line 7) via Prop. ttm:
    Y_[n] = X_[n] (Q_{n-1} (x) ... (x) Q_1 (x) Q_N (x) ... (x) Q_{n+1})."""
    N = X.ndim
    order = [(n - t) % N for t in range(1, N)]   # n-1, ..., 1, N, ..., n+1
    return unfold_mode(X, n) @ kron_chain([Qs[m] for m in order])


def tr_als_qr(X: np.ndarray, init: Sequence[np.ndarray], sweeps: int,
              residual: bool = True) -> Tuple[List[np.ndarray], List[float]]:
    """TR-ALS-QR (Alg. 3) for small shapes only (the QR of V_n costs O(R^{2N+2})).

    Derivation from the least-squares problem of Sec. 3.2, min |G^{!=n}_[2] Z^T - X_[n]^T|_F:
    with each core factored as G_j = R_j x_2 Q_j (mode-2 QR), Prop. slice_kron moves every Q_j out
    of the subchain, G^{!=n}_[2] = (Q_{n-1} (x) ... (x) Q_{n+1}) V_n[2] with V_n the subchain of the
    R_j; a QR V_n[2] = Q_0 R makes G^{!=n}_[2] = Q R with Q = (Q_{n-1} (x) ... (x) Q_{n+1}) Q_0
    orthonormal.  The least-squares solution then solves R Z^T = Q^T X_[n]^T = W_n^T, where
    W_n = (X_[n] (Q_{n-1} (x) ... (x) Q_{n+1})) Q_0 = Y_[n] Q_0 and Y = X x_{j!=n} Q_j^T (Prop. ttm).
    Columns follow G^{!=n}_[2] (r_n + R_n r_{n+1}).  tests/test_oracle_pins.py checks the result
    against the Householder least-squares solution on the explicit subchain matrix.
    """
    cores = [np.array(G, dtype=np.float64, copy=True) for G in init]
    N = len(cores)
    QR = [mode2_qr(G) for G in cores]
    res = []
    for _ in range(sweeps):
        for n in range(N):
            modes = chain_modes(N, n)
            V = QR[modes[0]][0]
            for m in modes[1:]:
                V = subchain_product(V, QR[m][0])
            Rv, Q0 = mode2_qr(V)                       # V (R_{n+1}, prod m, R_n)
            R2 = unfold3_mode2(Rv)                     # columns a + R_n b (dim3 + R_n dim1)
            Yn = multi_ttm_mode_unfolded(X, [q for (_, q) in QR], n)
            W = Yn @ Q0
            # G_{n(2)} R2^T = W  <=>  R2 G_{n(2)}^T = W^T, back substitution (Alg. 3 line 9).
            # R2 is wide only when G^{!=n}_[2] has fewer rows than columns; then take the
            # minimum-norm solution (the SVD option of the remark after Alg. 3).
            if R2.shape[0] == R2.shape[1]:
                Zt = sla.solve_triangular(R2, W.T, lower=False)
            else:
                Zt = np.linalg.lstsq(R2, W.T, rcond=None)[0]
            Rn, Rn1 = cores[n].shape[0], cores[n].shape[2]
            cores[n] = core_fold2(Zt.T, Rn, Rn1)
            QR[n] = mode2_qr(cores[n])
        if residual:
            res.append(rel_residual(X, cores))
    return cores, res


def tr_als_qrne(X: np.ndarray, init: Sequence[np.ndarray], sweeps: int,
                residual: bool = True) -> Tuple[List[np.ndarray], List[float]]:
    """TR-ALS-QRNE (Alg. 4, Sec. 3.3): the normal equations of the QR-compressed problem.

    The mode-2 QR G_j = R_j x_2 Q_j of every core compresses the least-squares problem: with
    Y = X x_{j!=n} Q_j^T (Multi-TTM) and V_n the subchain of the R_j, the compressed problem
    min |Y_[n] - G_{n(2)} V_n[2]^T|_F (eq. qrhalf_ls) is solved through its normal equations:
    M_n = Y_[n] V_n[2], S_n = the structured coefficient matrix chained from the Gram tensors of
    the R_j (Prop. subchain_gram applied to V_n), then G_{n(2)} S_n = M_n by Cholesky.  After each
    update the new core's QR and Gram tensor are recomputed.  Small shapes only (the Multi-TTM is
    formed through an explicit Kronecker product).
    """
    cores = [np.array(G, dtype=np.float64, copy=True) for G in init]
    N = len(cores)
    QR = [mode2_qr(G) for G in cores]
    res = []
    for _ in range(sweeps):
        for n in range(N):
            Rs = [q[0] for q in QR]
            S = paper_coefficient_matrix(Rs, n)                     # from the Gram tensors of the R_j
            V2 = subchain_unfolded(Rs, n)                           # V_n[2]
            Yn = multi_ttm_mode_unfolded(X, [q[1] for q in QR], n)  # Y_[n]
            M = Yn @ V2
            Rn, Rn1 = cores[n].shape[0], cores[n].shape[2]
            cores[n] = core_fold2(ls_solve_normal(S, M), Rn, Rn1)
            QR[n] = mode2_qr(cores[n])
        if residual:
            res.append(rel_residual(X, cores))
    return cores, res


# ---------------------------------------------------------------------------
# Gauge-invariant comparison of two solutions (subspace angle) and Gamma-chain helpers
# ---------------------------------------------------------------------------
def subchain_principal_angle(cores_a: Sequence[np.ndarray], cores_b: Sequence[np.ndarray], n: int) -> float:
    """Largest principal angle (radians) between range(G^{!=n}_[2]) of two TR solutions.

    Gauge changes of the cores other than n multiply G^{!=n}_[2] on the right by an
    invertible matrix, so this angle is gauge invariant.  Formed explicitly (small shapes).
    """
    A = subchain_unfolded(cores_a, n)
    B = subchain_unfolded(cores_b, n)
    Qa, _ = np.linalg.qr(A)
    Qb, _ = np.linalg.qr(B)
    s = np.linalg.svd(Qa.T @ Qb, compute_uv=False)
    return float(np.arccos(np.clip(s.min(), -1.0, 1.0)))


# ---------------------------------------------------------------------------
# BF16 storage of X for the mixed-precision mode: round to nearest even
# ---------------------------------------------------------------------------
def bf16_rne_bits(x) -> np.ndarray:
    """BF16 bit pattern of x: x is first rounded to FP32 (nearest even), then the FP32 bit
    pattern is rounded to its top 16 bits, ties to even (finite inputs)."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    return (((b + 0x7FFF + ((b >> 16) & 1)) >> 16) & 0xFFFF).astype(np.uint16)


def bf16_bits_to_f64(u) -> np.ndarray:
    return (np.asarray(u, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def bf16_split(x) -> Tuple[np.ndarray, np.ndarray]:
    """hi = bf16(x), lo = bf16(x - hi) (both as bit patterns): the split-BF16 pair of x."""
    x = np.asarray(x, dtype=np.float64)
    hi = bf16_rne_bits(x)
    lo = bf16_rne_bits(x - bf16_bits_to_f64(hi))
    return hi, lo
