"""Writes oracle_iters_shifted3d_<N>.txt: the FP64 oracle's Alg. 2 iteration
counts for the four right-hand sides of system 1 of the N^3 shifted
convection-diffusion sequence, with the fixed k = 20 right-only space
(random_recycle_basis seed 11) that the CPU-baseline sample of bench.py
times.  The baseline extrapolates its per-iteration time by their mean.
Calls only oracle/ and the seeded input generators.

    python tests/golden/make_oracle_iters.py [N]
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import scipy.sparse as sp  # noqa: E402

from oracle import rbicgstab as orb  # noqa: E402
from paper_1406_2831_gb300 import inputs  # noqa: E402


def main(N=128, k=20):
    spec = inputs.config_shifted_3d(N=N, n_shifts=20, n_rhs=4, k=k)
    P = spec.pattern
    S = sp.csr_matrix((spec.values[0](), P.col, P.row_ptr), shape=(P.n, P.n))
    rec = orb.recycle_setup(S, inputs.random_recycle_basis(P.n, k, 11))
    its = []
    for g in spec.rhs[0]:
        _, info = orb.rbicgstab(S, g(), rec, tol=1e-8, true_residual=False)
        its.append(info.iters)
        print(info.iters, flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"oracle_iters_shifted3d_{N}.txt")
    with open(path, "w") as f:
        f.write(f"# FP64 oracle Alg. 2 iterations, system 1 of the {N}^3 shifted sequence, 4 right-hand sides,\n")
        f.write(f"# fixed k = {k} right-only random space (seed 11), tol 1e-8; written by make_oracle_iters.py\n")
        for it in its:
            f.write(f"{it}\n")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 128)
