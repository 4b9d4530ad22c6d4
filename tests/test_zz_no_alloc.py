"""The allocation-free entry point ff_apply_operators_noalloc.

It serves callers that cannot allocate device memory when they call the
library (real-time loops that forbid driver allocations, processes whose
device memory is held by another allocator, plug-ins given a fixed memory
budget): its staging panels live in a fixed array of the library's device
image.  Checked through the C ABI against the
allocating entry point ff_apply_operators on two calls in a row (the array
keeps the previous call's contents), in both precisions, and on an oversize
block, which must be refused.  Collected last so that a failure here cannot
hide the other tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_noalloc_matches_allocating_entry_point(prec):
    import torch
    from paper_2605_29318_gb300 import binding, synth
    c = synth.torus(4000, seed=2)
    ctx = binding.Context(0, prec)
    dev = "cuda:0"
    ctx.rkpm_build(*(torch.from_numpy(x).to(dev) for x in (c.X, c.v, c.a)))
    ctx.assemble_hessian(None, None, c.E, c.nu)
    tol = 1e-5 if prec == "fp32" else 1e-12
    rng = np.random.default_rng(7)
    for call in range(2):
        X = torch.from_numpy(rng.standard_normal((c.n, 24 + 8 * call))).to(ctx.dtype).to(dev)
        ref_h, ref_m = ctx.apply_operators(X)
        got_h, got_m = ctx.apply_operators_noalloc(X)
        for ref, got in ((ref_h, got_h), (ref_m, got_m)):
            ref = ref.double().cpu().numpy()
            got = got.double().cpu().numpy()
            assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    if prec == "fp64":
        # 3 panels of 4000 x 512 doubles (49 MB) exceed the 32 MiB static scratch:
        # refused with a clear error, nothing launched
        big = torch.zeros((c.n, 512), dtype=ctx.dtype, device=dev)
        with pytest.raises(binding.FreeformError) as e:
            ctx.apply_operators_noalloc(big)
        assert e.value.status == 1 and "static scratch" in str(e.value)
    ctx.close()
