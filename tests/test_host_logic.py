"""Host-side logic that needs no GPU: the MTTSP kernel choice per mode and argument checks."""
import pytest

import paper_2210_11362_gb300 as P


def test_mttsp_path_choice_40x5():
    I, R = (40,) * 5, (8, 10, 12, 10, 8)
    paths = [P.trals_mttsp_path(I, R, n, "bf16") for n in range(5)]
    # every mode of the 40^5 workload runs on tensor cores; modes 0-1 need MN-major tiles (mode 0 with
    # the factor on the left, so that its rows are consecutive elements of X)
    assert paths == [4, 3, 1, 1, 2]


def test_mttsp_path_choice_fp64_is_cuda_cores():
    I, R = (40,) * 5, (8, 10, 12, 10, 8)
    assert all(P.trals_mttsp_path(I, R, n, "fp64") == 0 for n in range(5))


def test_mttsp_path_pads_the_leading_mode_and_falls_back_when_too_large():
    # 60^4: plans store the BF16 copy with mode 0 padded to 64, so every mode meets TMA's 16-byte
    # stride rule and runs on tensor cores
    assert all(P.trals_mttsp_path((60,) * 4, (10,) * 4, n, "bf16") > 0 for n in range(4))
    # a middle mode longer than the 128-row tile and a long MN-major block: no tensor-core geometry
    assert P.trals_mttsp_path((41, 39, 200, 41, 39), (2, 2, 7, 8, 3), 2, "bf16") == 0
    # a short middle mode (I_n = 20) takes K-major tiles of six repetitions of its rows
    assert P.trals_mttsp_path((41, 39, 20, 41, 39), (2, 2, 7, 8, 3), 2, "bf16") == 1
    # rank-16 cores: stage-1 table wider than the 128-column accumulator -> no tensor-core geometry
    # (trals_mttsp runs the CUDA cores; a plan takes the two-stage GEMM MTTSP there)
    assert all(P.trals_mttsp_path((256, 256, 3, 256), (16,) * 4, n, "bf16") == 0 for n in range(4))
    # tiny tensors: contraction too short for a tensor-core tile
    assert all(P.trals_mttsp_path((20, 20, 20), (3, 3, 3), n, "bf16") == 0 for n in range(3))


def test_split_bf16_modes_take_the_bf16_geometries():
    """bf16x2 and bf16x3 run the same tensor-core geometries as BF16 on the bench workloads: their
    stages (two BF16 planes of the table, and of X for bf16x3) still fit the shared-memory plan."""
    for I, R in (((40,) * 5, (8, 10, 12, 10, 8)), ((60,) * 4, (10,) * 4)):
        ref = [P.trals_mttsp_path(I, R, n, "bf16") for n in range(len(I))]
        assert all(p > 0 for p in ref)
        for mode in ("bf16x2", "bf16x3"):
            assert [P.trals_mttsp_path(I, R, n, mode) for n in range(len(I))] == ref, mode


def test_mttsp_path_rejects_bad_arguments():
    assert P.trals_mttsp_path((4, 4), (2, 2), 0, "bf16") < 0
    assert P.trals_mttsp_path((4, 4, 4), (2, 2, 2), 3, "bf16") < 0


def test_bench_subspace_angle_matches_the_oracle():
    """The bench's gauge-invariant angle (mixed Gram chains, no subchain matrix) against the oracle's
    explicit QR-based principal angle, and its mixed Gram against the explicit A^T B."""
    import numpy as np

    import bench
    import oracle as O
    import trals_inputs as TI

    I, R = (6, 5, 7, 4), (2, 3, 2, 3)
    a = TI.gaussian_cores(1, I, R)
    rng = np.random.default_rng(2)
    b = [G + 0.05 * rng.standard_normal(G.shape) for G in a]
    for n in range(4):
        C = bench.mixed_subchain_gram(a, b, n)
        np.testing.assert_allclose(C, O.subchain_unfolded(a, n).T @ O.subchain_unfolded(b, n), rtol=1e-12,
                                   atol=1e-12 * np.abs(C).max())
        ang = bench.subspace_angle(a, b, n)
        assert ang > 1e-4
        assert abs(ang - O.subchain_principal_angle(a, b, n)) < 1e-9
        assert bench.subspace_angle(a, a, n) < 1e-6


def test_multivariate_t_cores_correlation_and_layout():
    """Rows of the mode-2 unfolding follow the correlation theta^|i-j| (checked by sampling with a
    large degree of freedom, where the t distribution approaches the Gaussian), and the unfolding's
    column a + R_n b is the lateral fibre G[a, :, b]."""
    import numpy as np

    import oracle as O
    import trals_inputs as TI

    G = TI.multivariate_t_cores(1, (40000, 6, 6), (5, 5, 5), 0.8, dof=1e12)[0]
    Z = O.core_unfold2(G)                                       # I x R_n R_{n+1}, column a + R_n b
    assert np.array_equal(Z[:, 2 + 5 * 3], G[2, :, 3])
    want = 0.8 ** np.abs(np.subtract.outer(np.arange(25), np.arange(25)))
    assert np.abs(np.corrcoef(Z.T) - want).max() < 0.03
    # d = 1: heavy tails (Cauchy-like marginals), still finite
    H = TI.multivariate_t_cores(2, (100, 100, 100), (5, 5, 5), 1 - 1e-7, dof=1.0)
    assert all(np.isfinite(h).all() for h in H)
    # near-perfect correlation: neighbouring unfolding columns nearly parallel
    Z = O.core_unfold2(H[0])
    cos = abs(Z[:, 0] @ Z[:, 1]) / (np.linalg.norm(Z[:, 0]) * np.linalg.norm(Z[:, 1]))
    assert cos > 1 - 1e-5


def test_sinusoid_tensor_matches_its_definition():
    """The smooth workload's generator against its elementwise definition (a sum of separable sinusoid
    products, 0-based indices), and the column-major flattening the library reads."""
    import itertools
    import math

    import numpy as np

    import trals_inputs as TI
    I = (4, 5, 3)
    f, phi = TI.sinusoid_params(3, 5, len(I))
    X = TI.sinusoid_tensor(I, f, phi)
    for idx in itertools.product(*[range(d) for d in I]):
        want = sum(math.prod(math.sin(2.0 * math.pi * f[t, m] * idx[m] / I[m] + phi[t, m]) for m in range(len(I)))
                   for t in range(f.shape[0]))
        assert abs(X[idx] - want) < 1e-12
    flat = TI.flat_f(X)
    assert flat[1] == X[1, 0, 0] and flat[I[0]] == X[0, 1, 0] and flat[I[0] * I[1]] == X[0, 0, 1]
