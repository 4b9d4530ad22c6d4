"""GPU checks of eigenmodes_batched (through the C ABI): every object's
results are bit-identical to the single-object calls (same kernels, same
arithmetic, only the streams differ), failures are reported per object, and
the 256-object batch (cube / torus / ellipsoid unions, 2,000-200,000
particles, k from 16 to 48) reaches the residual bar on every object (the
solver's residuals are FP64 against the FP64 matrices)."""
import numpy as np
import pytest

from paper_2605_29318_gb300 import synth

pytestmark = pytest.mark.gpu


def _objects(clouds):
    import torch
    out = []
    for c in clouds:
        out.append({"X": torch.from_numpy(c.X).cuda(), "v": torch.from_numpy(c.v).cuda(),
                    "a": torch.from_numpy(c.a).cuda(), "E0": c.E, "nu0": c.nu, "k": c.k})
    return out


def test_batch_equals_single_calls():
    from paper_2605_29318_gb300 import binding
    clouds = synth.batch(10, seed=4, nmin=2000, nmax=20000, kmin=8, kmax=16)
    objs = _objects(clouds)
    opts = binding.default_opts(tol=1e-6)
    st, res = binding.eigenmodes_batched(objs, "fp64", opts, workers=4)
    assert st == 0, [r[4] for r in res]
    for o, (ev, modes, rep, s, err) in zip(objs, res):
        ctx = binding.Context(0, "fp64")
        ctx.rkpm_build(o["X"], o["v"], o["a"])
        ctx.assemble_hessian(None, None, o["E0"], o["nu0"])
        ev1, modes1, rep1, s1 = ctx.eigenmodes(o["k"], opts)
        assert s == s1 == 0 and err == ""
        assert np.array_equal(ev, ev1)
        assert bool((modes == modes1).all())
        assert rep["iterations"] == rep1["iterations"]
        ctx.close()


def test_failures_are_reported_per_object():
    import torch
    from paper_2605_29318_gb300 import binding
    clouds = synth.batch(4, seed=9, nmin=2000, nmax=5000, kmin=8, kmax=8)
    objs = _objects(clouds)
    bad = objs[2]["v"].clone()
    bad[17] = -1.0
    objs[2]["v"] = bad
    st, res = binding.eigenmodes_batched(objs, "fp64", None, workers=2)
    assert st == 1
    assert res[2][3] == 1 and "invalid particle 17" in res[2][4]
    for j in (0, 1, 3):
        assert res[j][3] == 0 and res[j][4] == ""
    torch.cuda.synchronize()


def test_batch_of_256_objects():
    from paper_2605_29318_gb300 import binding
    clouds = synth.batch(256, seed=4)
    objs = _objects(clouds)
    st, res = binding.eigenmodes_batched(objs, "fp64", binding.default_opts(tol=1e-6))
    assert st == 0, [(j, r[4]) for j, r in enumerate(res) if r[3] != 0][:5]
    worst = max(r[2]["max_residual"] for r in res)
    assert worst <= 1e-6
    assert all(r[2]["converged"] == o["k"] for r, o in zip(res, objs))
