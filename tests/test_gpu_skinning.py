"""GPU parity of the skinning weight fields and linear blend skinning (Sec. 3.2,
Eq. 1; through the C ABI) against the FP64 oracle of ``oracle/skinning.py``.

Tolerances: weights 1e-10 of max |W| in FP64 contexts (double-float shape
functions), 2e-5 in FP32 ones; the constant and linear reproduction 1e-12 /
2e-5 absolute (unit-scale fields); LBS 1e-12 / 1e-5 of max |x|.
"""
import numpy as np
import pytest

from oracle import skinning
from paper_2605_29318_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 2e-5}


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def _queries(c, count, seed):
    rng = np.random.default_rng(seed)
    pick = rng.choice(c.n, count, replace=False)
    Q = c.X[pick].astype(np.float64) + 0.1 * c.a[pick, None] * rng.uniform(-1, 1, (count, 3))
    return np.concatenate([c.X[:50], Q.astype(np.float32)]).astype(np.float32)


def _ctx(c, prec):
    from paper_2605_29318_gb300 import binding
    ctx = binding.Context(0, prec)
    ctx.rkpm_build(_dev(c.X), _dev(c.v), _dev(c.a))
    return ctx


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_weights_of_the_modes_match_the_oracle(prec):
    """The weight fields of the computed modes at the particles and at points
    between them, and their linear blend skinning."""
    import torch
    from paper_2605_29318_gb300 import binding
    c = synth.torus(4000, seed=2)
    ctx = _ctx(c, prec)
    ctx.assemble_hessian(None, None, c.E, c.nu)
    ev, modes, rep, st = ctx.eigenmodes(8, binding.default_opts(tol=1e-6 if prec == "fp64"
                                                                 else 1e-4))
    Q = _queries(c, 300, 1)
    Wg = ctx.skinning_weights(_dev(Q), modes).double().cpu().numpy()
    C = modes.double().cpu().numpy()
    Wo = skinning.weights(Q, c.X, c.a, C)
    assert np.abs(Wg - Wo).max() <= TOL[prec] * np.abs(Wo).max()
    # LBS with random affine transforms on these weights
    rng = np.random.default_rng(2)
    Z = 0.1 * rng.standard_normal((8, 3, 4))
    xg = ctx.lbs(_dev(Q), torch.from_numpy(Wg).to("cuda:0", ctx.dtype),
                 _dev(Z).to(ctx.dtype)).double().cpu().numpy()
    Zr = Z.astype(np.float32).astype(np.float64) if prec == "fp32" else Z
    Wr = Wg.astype(np.float32).astype(np.float64) if prec == "fp32" else Wg
    xo = skinning.lbs(Q, Wr, Zr)
    assert np.abs(xg - xo).max() <= (1e-12 if prec == "fp64" else 1e-5) * np.abs(xo).max()
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_weights_reproduce_constant_and_linear_fields(prec):
    """Consistency at any point the supports cover: constant nodal values give
    the constant, the nodes' coordinates give the point (Eq. 8)."""
    c = synth.unit_cube(2000, seed=1)
    ctx = _ctx(c, prec)
    Q = _queries(c, 500, 7)
    dt = np.float64 if prec == "fp64" else np.float32
    W1 = ctx.skinning_weights(_dev(Q), _dev(np.ones((c.n, 1), dt))).double().cpu().numpy()
    tol = 1e-12 if prec == "fp64" else 2e-5
    assert np.abs(W1 - 1.0).max() < tol
    WX = ctx.skinning_weights(_dev(Q), _dev(c.X.astype(dt))).double().cpu().numpy()
    assert np.abs(WX - Q.astype(np.float64)).max() < tol * max(1.0, np.abs(Q).max())
    ctx.close()


def test_uncovered_point_is_reported_and_the_context_stays_usable():
    """A query point no support reaches is refused with the point's index; the
    next call on the same context works."""
    from paper_2605_29318_gb300 import binding
    c = synth.unit_cube(2000, seed=1)
    ctx = _ctx(c, "fp64")
    Q = _queries(c, 20, 3)
    Q[7] = np.array([5.0, 5.0, 5.0], np.float32)
    with pytest.raises(binding.FreeformError) as e:
        ctx.skinning_weights(_dev(Q), _dev(np.ones((c.n, 2))))
    assert e.value.status == 4 and "query point 7" in str(e.value)
    Q[7] = Q[6]
    W = ctx.skinning_weights(_dev(Q), _dev(np.ones((c.n, 2)))).cpu().numpy()
    assert np.abs(W - 1.0).max() < 1e-12
    ctx.close()
