"""CPU checks of the C ABI: the library builds, loads, and exports every
function that include/freeform.h declares; the ctypes structures match the
header's field lists.  No CUDA call is made."""
import argparse
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "freeform.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2605_29318_gb300 import binding, build
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    return binding.load_library()


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                       text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "defined")))


def test_header_declares_the_paper_calls():
    names = _declared_functions()
    for n in ("rkpm_build", "assemble_hessian", "eigenmodes"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2605_29318_gb300 import binding
    names = _declared_functions()
    assert sorted(binding.EXPORTS) == names
    for n in names:
        assert hasattr(lib, n), n


def test_version_string(lib):
    assert lib.ff_version().decode().startswith("freeform-gb300")


def _struct_fields(name):
    text = open(HEADER).read()
    m = re.search(r"typedef struct \{([^}]*)\}\s*" + name + ";", text)
    body = re.sub(r"/\*.*?\*/", "", m.group(1), flags=re.S)
    return [re.findall(r"([A-Za-z_][A-Za-z0-9_]*)\s*(?:\[[^\]]*\])?\s*;", l)[0]
            for l in body.split("\n") if ";" in l]


def test_ctypes_structs_match_header():
    from paper_2605_29318_gb300 import binding
    assert [f for f, _ in binding.EigOpts._fields_] == _struct_fields("ff_eig_opts")
    assert [f for f, _ in binding.EigReport._fields_] == _struct_fields("ff_eig_report")
    assert [f for f, _ in binding.BatchItem._fields_] == _struct_fields("ff_batch_item")


def test_default_options_without_gpu(lib):
    from paper_2605_29318_gb300 import binding
    o = binding.default_opts()
    assert o.tol == 1e-6 and o.max_iter == 500 and o.cheb_degree == 16 and o.guard == 8
    assert o.fp32_phase == 1 and o.fp32_tol == 1e-4 and o.cheb_degree_fp64 == 48
    assert o.precond_tc == 1 and o.precond_compact == 0


def test_create_without_device_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = lib.ff_create(ctypes.byref(h), 0, None, 0)
    assert st != 0 and not h.value
    assert lib.ff_create(None, 0, None, 0) == 1
    assert lib.ff_create(ctypes.byref(h), 0, None, 7) == 1


def test_null_context_calls_are_rejected(lib):
    assert lib.rkpm_build(None, None, None, None, 10) == 1
    assert lib.assemble_hessian(None, None, None, 1.0, 0.3) == 1
    assert lib.eigenmodes(None, 3, None, None, None, None, None) == 1
    assert lib.ff_get_sizes(None, None, None, None) == 1
    assert lib.ff_get_precond_layout(None, None, None) == 1
    assert lib.ff_skinning_weights(None, None, 1, None, 1, None) == 1
    assert lib.ff_lbs_deform(None, None, 1, None, 1, None, None) == 1
    assert lib.rkpm_build_twoset(None, None, None, 100, 10, 3.0, 0) == 1
    assert lib.ff_get_twoset(None, None, None, None, None) == 1
    # batched call: argument checks come before any device use
    assert lib.eigenmodes_batched(0, 1, None, 3, None, 0) == 1
    assert lib.eigenmodes_batched(0, 1, None, -1, None, 0) == 1
    assert lib.eigenmodes_batched(0, 7, None, 0, None, 0) == 1
    assert lib.eigenmodes_batched(0, 1, None, 0, None, -2) == 1
    assert lib.eigenmodes_batched(0, 1, None, 0, None, 0) == 0


def test_no_fallback_without_library(tmp_path):
    from paper_2605_29318_gb300 import binding
    saved = binding._lib
    binding._lib = None
    try:
        with pytest.raises(RuntimeError):
            binding.load_library(str(tmp_path / "missing.so"))
    finally:
        binding._lib = saved


@pytest.mark.parametrize("workload", ["splat", "torus", "twoset-torus"])
def test_reference_arm_prints_the_contract_line(workload):
    """bench.py --impl reference times the FP64 oracle on the host cores and
    prints one JSON line with the contract's keys (no GPU needed), with the
    same config object as our arm prints for the workload."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import bench
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--workload", workload], cwd=root,
                         capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "dtype", "data", "config"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and not line["higher_is_better"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    args = argparse.Namespace(prec="fp64", tol=1e-6)
    ours = {"splat": bench.splat_config, "torus": bench.torus_config,
            "twoset-torus": bench.twoset_torus_config}[workload](args)
    assert line["config"] == ours


def _replica_worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        q.put((rank, bench.max_over_ranks([1.0 + rank, 10.0 - rank], "cpu")))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replica_timing_takes_the_slowest_rank():
    """The N > 1 path (replicas, one object per rank, no data-path collective):
    the step time every rank reports is the slowest rank's (world size 2, gloo)."""
    import multiprocessing as mp
    import socket
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_replica_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert got[0] == got[1] == [2.0, 10.0]


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun only rank 0 times the oracle; the other ranks exit at once."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], cwd=root, env=env, capture_output=True, text=True,
                         timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == ""
