"""Seeded synthetic inputs for tensor-ring ALS workloads.

This module is shared by the CPU oracle, the tests and the benchmark.  It
draws random numbers and lays out the synthetic workloads described in the
experiments section of Yu & Li (arXiv 2210.11362, Sec. 4): Gaussian TR-cores,
a Gaussian noise tensor scaled to a relative level, Gaussian initial cores,
and (for the smooth, not-exactly-low-rank workload) a sum of separable
sinusoid products.  It deliberately holds none of the ALS arithmetic: it never
evaluates the tensor-ring format, an unfolding, a Gram matrix or a solve.

Conventions
-----------
* Core n has shape (R_n, I_n, R_{n+1}) with R_{N+1} = R_1 (Sec. 1).
* Dense tensors are numpy arrays of shape (I_1, ..., I_N).  Their flat memory
  order everywhere in this project is column-major (i_1 fastest), which is the
  paper's linear index (Sec. 2).  ``flat_f`` / ``unflat_f`` convert.
* Every stream is ``numpy.random.default_rng([seed, stream_id])`` so that the
  true cores, the noise and the initial cores are independent and
  reproducible on any machine.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

STREAM_TRUE_CORES = 0
STREAM_NOISE = 1
STREAM_INIT = 2
STREAM_SINUSOID = 3
STREAM_REQUESTS = 4


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(stream)])


def gaussian_cores(seed: int, I: Sequence[int], R: Sequence[int], stream: int = STREAM_TRUE_CORES,
                   scale: float = 1.0) -> List[np.ndarray]:
    """iid N(0, scale^2) cores G_n of shape (R_n, I_n, R_{n+1}), float64."""
    N = len(I)
    assert len(R) == N
    g = _rng(seed, stream)
    cores = []
    for n in range(N):
        shape = (int(R[n]), int(I[n]), int(R[(n + 1) % N]))
        cores.append(scale * g.standard_normal(shape))
    return cores


def init_cores(seed: int, I: Sequence[int], R: Sequence[int]) -> List[np.ndarray]:
    """Seeded N(0,1) initial cores for the ALS (Sec. 4: Gaussian initialisation)."""
    return gaussian_cores(seed, I, R, stream=STREAM_INIT)


def gaussian_noise(seed: int, I: Sequence[int]) -> np.ndarray:
    """A standard-normal tensor N of shape I (float64)."""
    return _rng(seed, STREAM_NOISE).standard_normal(tuple(int(i) for i in I))


def add_relative_noise(X_true: np.ndarray, noise: np.ndarray, eta: float) -> np.ndarray:
    """The observation model of Sec. 4: X = X_true + eta * (|X_true|_F / |N|_F) * N."""
    if eta == 0.0:
        return X_true.copy()
    return X_true + eta * (np.linalg.norm(X_true.ravel()) / np.linalg.norm(noise.ravel())) * noise


def sinusoid_params(seed: int, terms: int, order: int) -> Tuple[np.ndarray, np.ndarray]:
    """Frequencies f ~ U(0, 8) and phases phi ~ U(0, 2 pi), each of shape (terms, order)."""
    g = _rng(seed, STREAM_SINUSOID)
    f = g.uniform(0.0, 8.0, size=(terms, order))
    phi = g.uniform(0.0, 2.0 * math.pi, size=(terms, order))
    return f, phi


def sinusoid_tensor(I: Sequence[int], f: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """X[i] = sum_t prod_n sin(2 pi f[t,n] i_n / I_n + phi[t,n]), i_n 0-based (float64).

    A smooth tensor that is not exactly of low TR rank; it stands in for the
    paper's real video / hyperspectral tensors (Sec. 4.3), which are not used.
    """
    I = [int(i) for i in I]
    T, order = f.shape
    assert order == len(I)
    X = np.zeros(tuple(I))
    for t in range(T):
        term = None
        for n in range(order):
            v = np.sin(2.0 * math.pi * f[t, n] * np.arange(I[n]) / I[n] + phi[t, n])
            term = v if term is None else np.multiply.outer(term, v)
        X += term
    return X


def flat_f(X: np.ndarray) -> np.ndarray:
    """Column-major (i_1 fastest) flat copy."""
    return np.asarray(X).reshape(-1, order="F")


def unflat_f(x: np.ndarray, I: Sequence[int]) -> np.ndarray:
    return np.asarray(x).reshape(tuple(int(i) for i in I), order="F")


def core_flat_f(G: np.ndarray) -> np.ndarray:
    """Column-major flat copy of a core (r_n fastest, then i_n, then r_{n+1})."""
    return np.asarray(G).reshape(-1, order="F")


def core_unflat_f(g: np.ndarray, Rn: int, In: int, Rn1: int) -> np.ndarray:
    return np.asarray(g).reshape((Rn, In, Rn1), order="F")


# ---------------------------------------------------------------------------
# Workload descriptions
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    I: Tuple[int, ...]
    R_true: Tuple[int, ...] | None      # None: not generated from a TR (sinusoid workload)
    R_fit: Tuple[int, ...]
    eta: float                          # relative noise level (Sec. 4); for the sinusoid workload: absolute std
    sweeps: int
    kind: str = "tr"                    # "tr" or "sinusoid"
    terms: int = 64                     # sinusoid workload only

    @property
    def numel(self) -> int:
        return int(np.prod(self.I))


WORKLOADS = {
    # 20x20x20, TR ranks (3,3,3), 1e-3 relative noise, 10 sweeps (plain FP64).
    "tr20x3_r3": Workload("tr20x3_r3", (20, 20, 20), (3, 3, 3), (3, 3, 3), 1e-3, 10),
    # 60^4 (12.96M entries), TR ranks 10, 1e-2 relative noise, 20 sweeps.
    "tr60x4_r10": Workload("tr60x4_r10", (60, 60, 60, 60), (10,) * 4, (10,) * 4, 1e-2, 20),
    # 40^5 (102.4M entries), TR ranks (8,10,12,10,8), 1e-3 relative noise, 30 sweeps.
    "tr40x5_r8-12": Workload("tr40x5_r8-12", (40,) * 5, (8, 10, 12, 10, 8), (8, 10, 12, 10, 8), 1e-3, 30),
    # 256x256x3x256 sum of 64 separable sinusoid products + N(0, 0.05^2); fit ranks 16; 25 sweeps.
    "sin256x256x3x256_r16": Workload("sin256x256x3x256_r16", (256, 256, 3, 256), None, (16,) * 4, 0.05, 25,
                                     kind="sinusoid"),
}


def make_tensor_host(w: Workload, seed: int, tr_full) -> np.ndarray:
    """Build the observed tensor X (float64) for workload ``w``.

    ``tr_full`` is the caller's tensor-ring evaluator (cores -> dense tensor);
    this module does not evaluate the TR format itself.
    """
    if w.kind == "sinusoid":
        f, phi = sinusoid_params(seed, w.terms, len(w.I))
        X = sinusoid_tensor(w.I, f, phi)
        return X + w.eta * gaussian_noise(seed, w.I)
    cores = gaussian_cores(seed, w.I, w.R_true)
    X_true = tr_full(cores)
    return add_relative_noise(X_true, gaussian_noise(seed, w.I), w.eta)


# ---------------------------------------------------------------------------
# Serving workload: a seeded stream of requests (Poisson arrivals)
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Request:
    rid: int
    arrival_s: float
    I: Tuple[int, ...]
    R: Tuple[int, ...]
    seed: int
    sweeps: int
    eta: float


def collinear_cores(seed: int, I: Sequence[int], R: Sequence[int], gamma: float,
                    stream: int = STREAM_TRUE_CORES) -> List[np.ndarray]:
    """Cores whose mode-2 unfoldings (I_n x R_n R_{n+1}) have unit-norm columns with pairwise inner
    product ``gamma`` (the collinearity-controlled construction of the paper's ill-conditioned
    experiments, Sec. 4): column k = sqrt(gamma) u_0 + sqrt(1 - gamma) u_k with u_0, u_1, ... orthonormal.
    Needs I_n > R_n R_{n+1}.  Pure sampling: no tensor-ring arithmetic."""
    g = _rng(seed, stream)
    N = len(I)
    out = []
    for n in range(N):
        Rn, Rn1 = int(R[n]), int(R[(n + 1) % N])
        r = Rn * Rn1
        if I[n] <= r:
            raise ValueError("collinear_cores needs I_n > R_n R_{n+1}")
        U, _ = np.linalg.qr(g.standard_normal((int(I[n]), r + 1)))
        cols = np.sqrt(gamma) * U[:, :1] + np.sqrt(1.0 - gamma) * U[:, 1:]
        # column c = a + R_n b of the unfolding is the lateral fibre G[a, :, b]
        G = np.empty((Rn, int(I[n]), Rn1))
        for b in range(Rn1):
            for a in range(Rn):
                G[a, :, b] = cols[:, a + Rn * b]
        out.append(G)
    return out


def multivariate_t_cores(seed: int, I: Sequence[int], R: Sequence[int], theta: float, dof: float = 1.0,
                         stream: int = STREAM_TRUE_CORES) -> List[np.ndarray]:
    """Cores whose mode-2 unfoldings (I_n x R_n R_{n+1}) have rows drawn from the multivariate t
    distribution with ``dof`` degrees of freedom and correlation matrix C_ij = theta^|i-j| (the
    correlated-core construction of the paper's second ill-conditioned experiment, Sec. 4).  Each row
    is z / sqrt(w / dof) with z ~ N(0, C) and w ~ chi^2_dof.  z is sampled as the stationary AR(1)
    sequence z_0 = g_0, z_k = theta z_{k-1} + sqrt(1 - theta^2) g_k (g iid N(0,1)), whose covariance is
    exactly theta^|i-j|, so no factorization of the nearly singular C is needed.  Column
    c = a + R_n b of the unfolding is the lateral fibre G[a, :, b].  Pure sampling: no tensor-ring
    arithmetic."""
    g = _rng(seed, stream)
    N = len(I)
    c = math.sqrt(max(0.0, 1.0 - theta * theta))
    out = []
    for n in range(N):
        Rn, In, Rn1 = int(R[n]), int(I[n]), int(R[(n + 1) % N])
        r = Rn * Rn1
        gau = g.standard_normal((In, r))
        z = np.empty((In, r))
        z[:, 0] = gau[:, 0]
        for k in range(1, r):
            z[:, k] = theta * z[:, k - 1] + c * gau[:, k]
        w = g.chisquare(dof, size=In)
        rows = z / np.sqrt(w / dof)[:, None]
        G = np.empty((Rn, In, Rn1))
        for b in range(Rn1):
            for a in range(Rn):
                G[a, :, b] = rows[:, a + Rn * b]
        out.append(G)
    return out


def signed_selection_cores(seed: int, I: Sequence[int], R: Sequence[int], dead: float = 0.15,
                           stream: int = STREAM_TRUE_CORES) -> List[np.ndarray]:
    """Cores whose lateral slices G_n(i) (R_n x R_{n+1}) hold at most one nonzero per row, +1 or -1
    at a uniformly drawn column; a row is all zero with probability ``dead``.  Every product of such
    slices has the same form, so all subchain entries are -1, 0 or +1: exact in BF16 and FP32.  With
    small-integer data every sum of the RHS contraction is then an exact integer in FP32, which makes
    reduced-precision kernels comparable element by element, without tolerance, to an FP64
    reference.  Pure sampling: no tensor-ring arithmetic."""
    g = _rng(seed, stream)
    N = len(I)
    out = []
    for n in range(N):
        Rn, In, Rn1 = int(R[n]), int(I[n]), int(R[(n + 1) % N])
        G = np.zeros((Rn, In, Rn1))
        col = g.integers(0, Rn1, size=(Rn, In))
        sign = np.where(g.random((Rn, In)) < 0.5, -1.0, 1.0)
        live = g.random((Rn, In)) >= dead
        a, i = np.nonzero(live)
        G[a, i, col[a, i]] = sign[a, i]
        out.append(G)
    return out


def small_integer_tensor(seed: int, I: Sequence[int], amp: int = 8) -> np.ndarray:
    """iid integers uniform in [-amp, amp] (float64, shape I): exactly representable in BF16 for
    amp <= 256."""
    return _rng(seed, STREAM_NOISE).integers(-amp, amp + 1, size=tuple(int(i) for i in I)).astype(np.float64)


def request_stream(seed: int, count: int = 512, rate_hz: float = 200.0, order_range=(3, 5),
                   size_range=(16, 64), rank_range=(2, 8), sweeps: int = 15, eta: float = 1e-2) -> List[Request]:
    """Poisson arrivals at ``rate_hz``; order, mode sizes and ranks drawn uniformly per request."""
    g = _rng(seed, STREAM_REQUESTS)
    t = 0.0
    out = []
    for rid in range(count):
        t += g.exponential(1.0 / rate_hz)
        N = int(g.integers(order_range[0], order_range[1] + 1))
        I = tuple(int(v) for v in g.integers(size_range[0], size_range[1] + 1, size=N))
        R = tuple(int(v) for v in g.integers(rank_range[0], rank_range[1] + 1, size=N))
        out.append(Request(rid, t, I, R, int(g.integers(0, 2**31 - 1)), sweeps, eta))
    return out
