"""GPU parity of the matrix-free operator ff_apply_operators_matfree (Prop. 1
and Eq. 14 applied from the shape-function tables, through the C ABI): H_w X
and M X against the oracle's assembled FP64 matrices, for a nodal cloud with
per-particle material and a two-set cloud, in both precisions; and against
the library's own assembled product.  Tolerances as for the assembled
products: 1e-5 (FP32) / 1e-11 (FP64) of the result's largest entry."""
import numpy as np
import pytest

from oracle import assembly, rkpm, twoset
from paper_2605_29318_gb300 import synth

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_matfree_nodal_heterogeneous(prec):
    import torch
    from paper_2605_29318_gb300 import binding
    c = synth.layered_sphere(3000, seed=6)
    ptr, idx = rkpm.neighbours(c.X, c.a)
    phi, dphi, _ = rkpm.shape_functions(c.X, c.a, ptr, idx)
    H, M = assembly.assemble(c.n, ptr, idx, phi, dphi, c.v, c.E, c.nu)
    ctx = binding.Context(0, prec)
    ctx.rkpm_build(_dev(c.X), _dev(c.v), _dev(c.a))
    E = _dev(np.asarray(c.E, np.float32))
    X = np.random.default_rng(3).standard_normal((c.n, 37))
    dt = torch.float64 if prec == "fp64" else torch.float32
    YH, YM = ctx.apply_operators_matfree(_dev(X).to(dt), E, None, 1.0, float(c.nu))
    tol = 1e-5 if prec == "fp32" else 1e-11
    for got, ref in ((YH, H @ X), (YM, M @ X)):
        got = got.double().cpu().numpy()
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    # the assembled product of the same context agrees
    ctx.assemble_hessian(E, None, 1.0, float(c.nu))
    AH, AM = ctx.apply_operators(_dev(X).to(dt))
    assert (torch.abs(AH - YH).max() <= 2 * tol * torch.abs(AH).max()).item()
    assert (torch.abs(AM - YM).max() <= 2 * tol * torch.abs(AM).max()).item()
    ctx.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_matfree_twoset(prec):
    import torch
    from paper_2605_29318_gb300 import binding
    Xq, v = synth.torus_grid(0.05)
    K, E, nu = 120, 1e6, 0.4
    ctx = binding.Context(0, prec)
    ctx.rkpm_build_twoset(_dev(Xq), _dev(v), K, 3.0, 0)
    _, cen, rad = ctx.twoset()
    P = Xq[cen]
    optr, oidx, ophi, odphi, _ = twoset.shape_functions(Xq, P, rad, 3.0,
                                                        scale=float(np.float32(rad.max())))
    H, M = twoset.assemble(Xq.shape[0], K, optr, oidx, ophi, odphi, v, E, nu)
    X = np.random.default_rng(4).standard_normal((K, 20))
    dt = torch.float64 if prec == "fp64" else torch.float32
    YH, YM = ctx.apply_operators_matfree(_dev(X).to(dt), None, None, E, nu)
    tol = 1e-5 if prec == "fp32" else 1e-11
    for got, ref in ((YH, H @ X), (YM, M @ X)):
        got = got.double().cpu().numpy()
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    ctx.close()
