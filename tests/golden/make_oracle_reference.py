"""Write the FP64 oracle's reference run of a workload: per-sweep relative residuals and final cores.

The stored values come from ``oracle/`` alone (regular TR-ALS, Alg. 1, with Cholesky on the
explicit normal equations, blockwise over rows of the subchain matrix) on the seeded input of
``trals_inputs`` (the experiment protocol of Sec. 4: Gaussian TR cores plus relative Gaussian noise,
Gaussian initial cores, a fixed sweep count).  Nothing here touches the CUDA path.

The accuracy statement of the mixed-precision modes compares against these files: the final
relative residual gap and the largest principal angle between the subchain ranges of the GPU and
the oracle solutions (both gauge invariant).

Usage:  python tests/golden/make_oracle_reference.py tr40x5_r8-12 [seed] [sweeps]
writes  tests/golden/oracle_<workload>_seed<seed>.npz  with arrays
        residuals (sweeps,), core0 .. core{N-1}, I, R, and the scalar sweeps.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import trals_inputs as TI  # noqa: E402


def reference_path(workload: str, seed: int) -> str:
    return os.path.join(HERE, f"oracle_{workload}_seed{seed}.npz")


def main():
    name = sys.argv[1]
    seed = int(sys.argv[2]) if len(sys.argv) > 2 else 0
    w = TI.WORKLOADS[name]
    sweeps = int(sys.argv[3]) if len(sys.argv) > 3 else w.sweeps
    X = TI.make_tensor_host(w, seed, O.tr_full)
    cores = TI.init_cores(seed, w.I, w.R_fit)
    res = []
    t0 = time.time()
    for s in range(sweeps):
        for n in range(len(w.I)):
            cores[n] = O.als_update(X, cores, n, "chol")
        res.append(O.rel_residual(X, cores))
        print(f"sweep {s + 1}: residual {res[-1]:.12e} ({time.time() - t0:.0f} s)", flush=True)
    out = {"residuals": np.array(res), "I": np.array(w.I), "R": np.array(w.R_fit), "sweeps": np.array(sweeps)}
    for n, G in enumerate(cores):
        out[f"core{n}"] = G
    np.savez(reference_path(name, seed), **out)
    print("wrote", reference_path(name, seed))


if __name__ == "__main__":
    main()
