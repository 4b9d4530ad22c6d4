"""Write ``splat_eigenvalues.txt``: the 66 lowest generalized eigenvalues of
H_w c = lambda M c (Sec. 3.2, Eq. 15) for the splat-like cloud of the
benchmark (1,000,000 points from 64 anisotropic Gaussians, seed 3) through the
paper's two-set construction (Supp. Sec. B): the points as quadrature points,
K = 1,000 farthest-point centres from point 0, Gaussian kernels of radius the
second-nearest-centre distance cut at 3 r_k, per-point E, nu = 0.45.  Computed
by the FP64 oracle alone (farthest-point sampling, Gaussian shape functions,
sparse H_w and M, dense LAPACK eigensolve); the two eigenvalues past k = 64
give the gap at the cut-off.  Runs several minutes on CPU cores:

    python tests/golden/make_splat_eigenvalues.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import eigen, twoset  # noqa: E402
from paper_2605_29318_gb300 import synth  # noqa: E402

K, K_OUT = 1000, 66


def main():
    c = synth.gaussian_mixture(1_000_000)
    centres, r, H, M = twoset.build(c.X, c.v, K, np.asarray(c.E, np.float64), float(c.nu),
                                    trunc=3.0, start=0, dense=True)
    lam, C = eigen.eigh_dense(H, M, K_OUT)
    res = eigen.residuals(H, M, lam, C)
    out = os.path.join(HERE, "splat_eigenvalues.txt")
    with open(out, "w") as f:
        f.write("# The 66 lowest eigenvalues of H_w c = lambda M c (Sec. 3.2, Eq. 15) for the\n"
                "# 1,000,000-point splat-like cloud (seed 3) through the two-set construction\n"
                "# (K = 1,000 farthest-point centres from point 0, Gaussian kernels cut at\n"
                "# 3 r_k, per-point E, nu = 0.45): FP64 oracle, dense LAPACK eigensolve.\n"
                "# Written by make_splat_eigenvalues.py.\n"
                f"# largest relative residual of indices 1..{K_OUT - 1}: "
                f"{res[1:].max():.3e}\n")
        for j, x in enumerate(lam):
            f.write(f"{j} {float(x)!r}\n")
    print(out)


if __name__ == "__main__":
    main()
