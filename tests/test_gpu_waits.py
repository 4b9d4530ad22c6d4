"""Failure detection without a GPU fault: the library's device-side waits (the
grid barrier of the whole-GPU farthest-point sampling, the mbarriers of the
tensor-core Gram) give up after a bounded number of clock cycles.  The
self-check runs the grid barrier with one arrival missing, so its wait can
only end by running out: the kernel must return FF_ERR_TIMEOUT within its
limit, and the device must stay usable afterwards."""
import time

import numpy as np
import pytest

from paper_2605_29318_gb300 import synth

pytestmark = pytest.mark.gpu


def test_grid_wait_runs_out_and_the_device_stays_usable():
    import torch
    from paper_2605_29318_gb300 import binding
    t0 = time.time()
    st = binding.selftest_device_wait(0, 200_000_000)   # ~0.1 s of SM clock cycles
    assert st == 7                                       # FF_ERR_TIMEOUT
    assert time.time() - t0 < 60
    assert binding.selftest_device_wait(0, 10) == 1      # below the smallest limit
    # the device and the library still work
    c = synth.unit_cube(400, seed=2)
    ctx = binding.Context(0, "fp64")
    ctx.rkpm_build(*(torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (c.X, c.v, c.a)))
    ctx.assemble_hessian(None, None, c.E, c.nu)
    ev, modes, rep, status = ctx.eigenmodes(4, binding.default_opts(tol=1e-6))
    assert status == 0 and np.all(np.diff(ev) > 0)
    ctx.close()
