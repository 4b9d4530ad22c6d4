"""Write ``torus50k_eigenvalues.txt``: the 34 lowest generalized eigenvalues of
H_w c = lambda M c (Sec. 3.2, Eq. 15) for the 50,000-particle solid torus
(R = 0.5, r = 0.2, seed 2, cubic B-spline support 2.0x spacing, E = 1e6,
nu = 0.4), computed by the FP64 oracle alone: brute-force neighbours, shape
functions, sparse H_w and M, shift-invert Lanczos.  The two eigenvalues past
k = 32 give the gap at the cut-off that the full-size subspace test needs.
Runs a few minutes on CPU cores:

    python tests/golden/make_torus50k_eigenvalues.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import assembly, eigen, rkpm  # noqa: E402
from paper_2605_29318_gb300 import synth  # noqa: E402

K_OUT = 34


def main():
    c = synth.torus(50000, seed=2)
    ptr, idx = rkpm.neighbours(c.X, c.a, chunk=64)
    phi, dphi, _ = rkpm.shape_functions(c.X, c.a, ptr, idx)
    H, M = assembly.assemble(c.n, ptr, idx, phi, dphi, c.v, c.E, c.nu)
    lam, C = eigen.eigsh_sparse(H, M, K_OUT)
    res = eigen.residuals(H, M, lam, C)
    out = os.path.join(HERE, "torus50k_eigenvalues.txt")
    with open(out, "w") as f:
        f.write("# The 34 lowest eigenvalues of H_w c = lambda M c (Sec. 3.2, Eq. 15) for the\n"
                "# 50,000-particle solid torus R=0.5 r=0.2 (seed 2), cubic B-spline support\n"
                "# 2.0x spacing, E=1e6, nu=0.4: FP64 oracle, sparse H_w and M, shift-invert\n"
                "# Lanczos (eigsh, tol 1e-12).  Written by make_torus50k_eigenvalues.py.\n"
                f"# largest relative residual of indices 1..{K_OUT - 1}: "
                f"{res[1:].max():.3e}\n")
        for j, x in enumerate(lam):
            f.write(f"{j} {float(x)!r}\n")
    print(out)


if __name__ == "__main__":
    main()
