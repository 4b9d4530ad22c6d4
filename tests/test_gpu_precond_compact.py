"""GPU check of the packed preconditioner (precond_compact = 1), which runs
the Chebyshev steps on the columns still above tol only, packed to a
multiple of 8.  On tensor cores every column is computed alone (the k-steps
are split over warps independently of the width, and an MMA keeps its B
columns apart), so the eigenpairs and iteration counts must be bit-identical
to the full-width steps.  The CUDA-core step splits a row's nonzeros over
32 / (width / 8) lane groups, so there the summation order, and W, change at
FP32 rounding: the eigenvalues must agree to 1e-10 and the iteration counts
within three."""
import numpy as np
import pytest

from paper_2605_29318_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tc", [("fp64", 1), ("fp64", 0), ("fp32", 1)])
def test_packed_preconditioner_gives_the_same_modes(prec, tc):
    import torch
    from paper_2605_29318_gb300 import binding
    c = synth.torus(8000, seed=2)
    out = []
    for compact in (0, 1):
        ctx = binding.Context(0, prec)
        ctx.rkpm_build(*(torch.from_numpy(x).cuda() for x in (c.X, c.v, c.a)))
        ctx.assemble_hessian(None, None, c.E, c.nu)
        o = binding.default_opts(tol=1e-6 if prec == "fp64" else 1e-4, precond_tc=tc,
                                 precond_compact=compact)
        ev, modes, rep, st = ctx.eigenmodes(16, o)
        assert st == 0
        out.append((ev, modes.cpu().numpy(), rep))
        ctx.close()
    (e0, m0, r0), (e1, m1, r1) = out
    if tc:
        assert np.array_equal(e0, e1) and np.array_equal(m0, m1)
        assert r0["iterations"] == r1["iterations"]
        assert r0["precond_spmv_calls"] == r1["precond_spmv_calls"]
    else:
        np.testing.assert_allclose(e1[1:], e0[1:], rtol=1e-10)
        assert abs(r0["iterations"] - r1["iterations"]) <= 3
