"""trals_mttsp_noalloc: the FP64 MTTSP for callers that cannot allocate device memory.

It must give the same M_n as trals_mttsp (FP64, within the 1e-12 relative tolerance of the FP64
step tests) on consecutive calls, which also exercises reuse of its static scratch array.  This file
is collected last so a run that stops at the first failure has already run every other test.
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


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("I,R", [((20, 20, 20), (3, 3, 3)), ((33, 17, 40), (5, 4, 6)), ((13, 3, 5, 2, 4), (2, 3, 2, 2, 3))])
def test_noalloc_matches_allocating_entry_point_twice(I, R):
    ctx = P.trals_create(0)
    X = TI.add_relative_noise(O.tr_full(TI.gaussian_cores(2, I, R)), TI.gaussian_noise(2, I), 1e-2)
    Xd = P.tensor_to_device(X)
    N = len(I)
    for call in range(2):
        cores = TI.gaussian_cores(10 + call, I, R)   # different cores on each call: stale scratch would show
        cd = [P.core_to_device(G) for G in cores]
        for n in range(N):
            r = R[n] * R[(n + 1) % N]
            ref = torch.zeros(I[n] * r, dtype=torch.float64, device="cuda")
            got = torch.full((I[n] * r,), float("nan"), dtype=torch.float64, device="cuda")
            P.trals_mttsp(ctx, I, R, Xd, "fp64", cd, n, ref)
            P.trals_mttsp_noalloc(ctx, I, R, Xd, cd, n, got)
            assert _rel(got.cpu().numpy(), ref.cpu().numpy()) < 1e-12
            # and both agree with the oracle's X_[n] G^{!=n}_[2]
            want = O.unfold_mode(X, n) @ O.subchain_unfolded(cores, n)
            assert _rel(got.cpu().numpy().reshape(I[n], r, order="F"), want) < 1e-12
    ctx.close()


def test_noalloc_rejects_shapes_beyond_the_scratch():
    ctx = P.trals_create(0)
    # n = 0: the subchain tables over modes 1 and 2 need 3 x 131072 x 16 x 16 doubles (~800 MB) > 32 MiB,
    # so the call is rejected on the host before any CUDA call; the tiny buffers below are never read
    I, R = (8, 1 << 17, 1 << 17), (16, 16, 16)
    Xd = torch.zeros(1, dtype=torch.float64, device="cuda")
    cd = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in range(3)]
    M = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(P.TralsError) as e:
        P.trals_mttsp_noalloc(ctx, I, R, Xd, cd, 0, M)
    assert e.value.status == P.E_ARG and "static scratch" in str(e.value)
    ctx.close()


def test_noalloc_rejects_what_the_allocating_entry_point_rejects():
    """R_n R_{n+1} = 400 > 256 (and other invalid shapes): trals_mttsp refuses them, and so does the
    no-allocation variant, with the same status, before any CUDA call."""
    ctx = P.trals_create(0)
    Xd = torch.zeros(1, dtype=torch.float64, device="cuda")
    cd = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in range(3)]
    M = torch.zeros(1, dtype=torch.float64, device="cuda")
    for I, R, n in (((30, 30, 30), (20, 20, 20), 0), ((2, 2, 2), (3, 3, 3), 1), ((4, 4), (2, 2), 0),
                    ((1 << 20, 1 << 20, 1 << 20), (2, 2, 2), 0), ((8, 8, 8), (2, 2, 2), 3)):
        for call in (lambda: P.trals_mttsp(ctx, I, R, Xd, "fp64", cd[:len(I)], n, M),
                     lambda: P.trals_mttsp_noalloc(ctx, I, R, Xd, cd[:len(I)], n, M)):
            with pytest.raises(P.TralsError) as e:
                call()
            assert e.value.status == P.E_ARG, (I, R, n)
    ctx.close()
