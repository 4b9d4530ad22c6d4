"""Thin ctypes binding of ``libfreeform.so`` (argument marshalling only).

The names follow the C ABI in ``include/freeform.h``: ``rkpm_build``,
``assemble_hessian``, ``eigenmodes`` (plus the inspection exports).  Every step
of the computation runs in the CUDA library; this module only turns torch
tensors into device pointers and host arrays into ctypes buffers.  It raises
if the library has not been built -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfreeform.so")

FF_OK = 0
STATUS = {0: "FF_OK", 1: "FF_ERR_INVALID_ARG", 2: "FF_ERR_CUDA", 3: "FF_ERR_OOM",
          4: "FF_ERR_SINGULAR_MOMENT", 5: "FF_ERR_NOT_CONVERGED", 6: "FF_ERR_NUMERIC",
          7: "FF_ERR_TIMEOUT", 8: "FF_ERR_STATE"}
PREC = {"fp32": 0, "fp64": 1}

# every symbol the header declares (checked by the CPU tests)
EXPORTS = ["ff_create", "ff_destroy", "ff_last_error", "ff_version", "rkpm_build",
           "assemble_hessian", "ff_eig_opts_default", "eigenmodes", "ff_get_sizes", "ff_get_precond_layout",
           "ff_export_rkpm", "ff_export_matrices", "ff_apply_operators",
           "ff_apply_operators_noalloc", "ff_profile_enable", "ff_profile_read", "ff_launch_count",
           "ff_net_num_params", "ff_net_create", "ff_net_destroy", "ff_net_last_error",
           "ff_net_init", "ff_net_set_params", "ff_net_get_params", "ff_warmstart_features",
           "ff_net_forward", "ff_net_loss_grad", "ff_net_train_step", "ff_warmstart_block",
           "ff_skinning_weights", "ff_lbs_deform", "rkpm_build_twoset", "ff_get_twoset",
           "eigenmodes_batched", "ff_profile_classes", "ff_subspace_host",
           "ff_subspace_twoset_host", "ff_export_row_ptr", "ff_apply_operators_matfree",
           "ff_selftest_device_wait", "ff_set_build_precision"]
PROF = {"precond": 0, "spmm": 1, "gram": 2, "rayleigh_ritz": 3, "update": 4, "build": 5,
        "assemble": 6, "setup": 7, "fps": 8, "cover": 9, "shape": 10, "pattern": 11,
        "asm_values": 12}


class EigOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("guard", ctypes.c_int),
                ("cheb_degree", ctypes.c_int), ("cheb_ratio", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("time_budget_s", ctypes.c_double),
                ("exclude_constant", ctypes.c_int), ("verbose", ctypes.c_int),
                ("fp32_phase", ctypes.c_int), ("fp32_tol", ctypes.c_double),
                ("cheb_degree_fp64", ctypes.c_int), ("precond_tc", ctypes.c_int),
                ("precond_compact", ctypes.c_int)]


class EigReport(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int),
                ("spmm_calls", ctypes.c_int), ("precond_spmv_calls", ctypes.c_int),
                ("max_residual", ctypes.c_double), ("seconds", ctypes.c_double),
                ("warm_start_used", ctypes.c_int), ("fp32_iterations", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class BatchItem(ctypes.Structure):
    _fields_ = [("particles", ctypes.c_void_p), ("volumes", ctypes.c_void_p),
                ("support", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("E", ctypes.c_void_p), ("nu", ctypes.c_void_p),
                ("E0", ctypes.c_double), ("nu0", ctypes.c_double), ("k", ctypes.c_int),
                ("eigvals", ctypes.c_void_p), ("modes", ctypes.c_void_p),
                ("report", ctypes.c_void_p), ("status", ctypes.c_int),
                ("error", ctypes.c_char * 192)]


class FreeformError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libfreeform.so and declare its signatures (no CUDA call is made)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built; run `python -m paper_2605_29318_gb300.build`")
    L = ctypes.CDLL(path)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    L.ff_create.argtypes = [ctypes.POINTER(vp), i32, vp, i32]
    L.ff_destroy.argtypes = [vp]
    L.ff_destroy.restype = None
    L.ff_last_error.argtypes = [vp]
    L.ff_last_error.restype = ctypes.c_char_p
    L.ff_version.restype = ctypes.c_char_p
    L.rkpm_build.argtypes = [vp, vp, vp, vp, i64]
    L.assemble_hessian.argtypes = [vp, vp, vp, dbl, dbl]
    L.ff_eig_opts_default.argtypes = [ctypes.POINTER(EigOpts)]
    L.ff_eig_opts_default.restype = None
    L.eigenmodes.argtypes = [vp, i32, ctypes.POINTER(EigOpts), vp, vp, vp,
                             ctypes.POINTER(EigReport)]
    L.ff_get_sizes.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.ff_get_precond_layout.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.ff_export_rkpm.argtypes = [vp, vp, vp, vp, vp]
    L.ff_export_matrices.argtypes = [vp, vp, vp, vp, vp]
    L.ff_apply_operators.argtypes = [vp, vp, i32, vp, vp]
    L.ff_apply_operators_noalloc.argtypes = [vp, vp, i32, vp, vp]
    L.ff_profile_enable.argtypes = [vp, i32]
    L.ff_profile_read.argtypes = [vp, i32, ctypes.POINTER(i64), ctypes.POINTER(dbl)]
    L.ff_launch_count.argtypes = []
    u64, fp = ctypes.c_uint64, ctypes.POINTER(ctypes.c_float)
    L.ff_net_num_params.argtypes = []
    L.ff_net_create.argtypes = [ctypes.POINTER(vp), i32, vp]
    L.ff_net_destroy.argtypes = [vp]
    L.ff_net_init.argtypes = [vp, u64]
    L.ff_net_set_params.argtypes = [vp, vp, i64]
    L.ff_net_get_params.argtypes = [vp, vp, i64]
    L.ff_warmstart_features.argtypes = [vp, vp]
    L.ff_net_forward.argtypes = [vp, vp, i64, vp]
    L.ff_net_loss_grad.argtypes = [vp, vp, vp, i64, vp, i32, ctypes.POINTER(dbl), vp]
    L.ff_net_train_step.argtypes = [vp, vp, vp, i64, vp, i32, ctypes.c_float, ctypes.POINTER(dbl)]
    L.ff_warmstart_block.argtypes = [vp, vp, i32, ctypes.POINTER(EigOpts), vp]
    L.ff_skinning_weights.argtypes = [vp, vp, i64, vp, i32, vp]
    L.ff_lbs_deform.argtypes = [vp, vp, i64, vp, i32, vp, vp]
    L.rkpm_build_twoset.argtypes = [vp, vp, vp, i64, i32, dbl, i64]
    L.ff_get_twoset.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i32), vp, vp]
    L.eigenmodes_batched.argtypes = [i32, i32, ctypes.POINTER(BatchItem), i32,
                                     ctypes.POINTER(EigOpts), i32]
    L.ff_profile_classes.argtypes = [vp, ctypes.c_uint32]
    L.ff_export_row_ptr.argtypes = [vp, vp]
    L.ff_selftest_device_wait.argtypes = [i32, i64]
    L.ff_set_build_precision.argtypes = [vp, i32]
    L.ff_apply_operators_matfree.argtypes = [vp, vp, vp, dbl, dbl, vp, i32, vp, vp]
    L.ff_subspace_host.argtypes = [vp, vp, vp, vp, vp, vp, i64, dbl, dbl, i32,
                                   ctypes.POINTER(EigOpts), vp, vp, ctypes.POINTER(EigReport)]
    L.ff_subspace_twoset_host.argtypes = [vp, vp, vp, vp, vp, i64, i32, dbl, i64, dbl, dbl, i32,
                                          ctypes.POINTER(EigOpts), vp, vp,
                                          ctypes.POINTER(EigReport)]
    del fp
    for name in EXPORTS:
        if name not in ("ff_destroy", "ff_last_error", "ff_version", "ff_eig_opts_default",
                        "ff_launch_count", "ff_net_num_params", "ff_net_destroy",
                        "ff_net_last_error"):
            getattr(L, name).restype = ctypes.c_int
    L.ff_launch_count.restype = ctypes.c_int64
    L.ff_net_num_params.restype = ctypes.c_int64
    L.ff_net_destroy.restype = None
    L.ff_net_last_error.restype = ctypes.c_char_p
    L.ff_net_last_error.argtypes = [ctypes.c_void_p]
    _lib = L
    return L


def selftest_device_wait(device: int = 0, wait_cycles: int = 200_000_000) -> int:
    """Run the library's grid barrier with one arrival missing: its bounded
    wait runs out; returns the status (FF_ERR_TIMEOUT = 7 expected)."""
    return int(load_library().ff_selftest_device_wait(int(device), int(wait_cycles)))


def launch_count() -> int:
    """Kernel launches issued by the library in this process."""
    return int(load_library().ff_launch_count())


def default_opts(**kw) -> EigOpts:
    o = EigOpts()
    load_library().ff_eig_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return int(t.data_ptr())


class Context:
    """One ff_ctx: a particle cloud, its matrices and eigen-solver workspace."""

    def __init__(self, device: int = 0, precision: str = "fp32", stream=None):
        import torch
        self.L = load_library()
        self.device = device
        self.precision = precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = ctypes.c_void_p()
        st = self.L.ff_create(ctypes.byref(h), device, ctypes.c_void_p(stream.cuda_stream),
                              PREC[precision])
        if st != FF_OK:
            raise FreeformError(st, "ff_create failed")
        self.h = h
        self.n = 0

    def close(self):
        if getattr(self, "h", None):
            self.L.ff_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != FF_OK:
            raise FreeformError(st, self.L.ff_last_error(self.h).decode())

    # ---- the three calls of the paper's pipeline
    def rkpm_build(self, particles, volumes, support):
        """particles (n, 3), volumes (n,), support radii (n,): float32 CUDA tensors."""
        for t in (particles, volumes, support):
            assert t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.float32"
        self.n = int(particles.shape[0])
        self._keep = (particles, volumes, support)
        self._check(self.L.rkpm_build(self.h, _ptr(particles), _ptr(volumes), _ptr(support),
                                      self.n))

    def rkpm_build_twoset(self, points, volumes, K: int, trunc: float = 3.0, start: int = 0):
        """The two-set construction: quadrature points (n, 3) and volumes (n,), float32
        CUDA tensors; K farthest-point centres from point ``start``; Gaussian kernels
        cut at ``trunc`` r_k (0: untruncated).  The unknowns are then the K centres."""
        for t in (points, volumes):
            assert t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.float32"
        self._keep = (points, volumes)
        self._check(self.L.rkpm_build_twoset(self.h, _ptr(points), _ptr(volumes),
                                             int(points.shape[0]), int(K), float(trunc),
                                             int(start)))
        self.n = int(K)

    def set_build_precision(self, precision: str):
        """"fp32" or "fp64": the precision of the following two-set builds
        (shape functions and assembly sums) in an FP64 context."""
        self._check(self.L.ff_set_build_precision(self.h, PREC[precision]))

    def twoset(self):
        """(n_points, centres int64 (K,), radii float64 (K,)) of a two-set cloud."""
        npt, K = ctypes.c_int64(), ctypes.c_int32()
        self._check(self.L.ff_get_twoset(self.h, ctypes.byref(npt), ctypes.byref(K), None, None))
        cen = np.zeros(K.value, np.int64)
        rad = np.zeros(K.value, np.float64)
        self._check(self.L.ff_get_twoset(self.h, None, None, cen.ctypes.data, rad.ctypes.data))
        return npt.value, cen, rad

    def assemble_hessian(self, E=None, nu=None, E0: float = 1e5, nu0: float = 0.45):
        """E, nu: per-particle float32 CUDA tensors or None (uniform E0, nu0)."""
        self._check(self.L.assemble_hessian(self.h, _ptr(E), _ptr(nu), float(E0), float(nu0)))

    def eigenmodes(self, k: int, opts: Optional[EigOpts] = None, X0=None, want_modes=True,
                   modes_out=None, check=True):
        """Returns (eigvals numpy (k,), modes torch (n, k) column-major view, report, status)."""
        import torch
        if X0 is not None:
            guard = opts.guard if opts is not None else 8
            kw = k if (opts is not None and opts.exclude_constant) else k - 1
            if (X0.dtype != self.dtype or not X0.is_contiguous()
                    or X0.numel() != self.n * (kw + max(0, guard))):
                raise ValueError(f"X0 must be a contiguous {self.dtype} block of "
                                 f"(k - 1 + guard) x n = {kw + max(0, guard)} x {self.n} values")
        ev = np.zeros(k, dtype=np.float64)
        modes = modes_out
        if want_modes and modes is None:
            modes = torch.empty((k, self.n), dtype=self.dtype, device=f"cuda:{self.device}")
        rep = EigReport()
        st = self.L.eigenmodes(self.h, int(k), ctypes.byref(opts) if opts is not None else None,
                               _ptr(X0), ev.ctypes.data_as(ctypes.c_void_p), _ptr(modes),
                               ctypes.byref(rep))
        if check and st not in (FF_OK,):
            raise FreeformError(st, self.L.ff_last_error(self.h).decode())
        return ev, (modes.t() if modes is not None else None), rep.as_dict(), st

    # ---- learned warm start
    def warmstart_features(self):
        """Features of the cloud: float32 CUDA tensor (n, 16), caller order."""
        import torch
        f = torch.empty((self.n, 16), dtype=torch.float32, device=f"cuda:{self.device}")
        self._check(self.L.ff_warmstart_features(self.h, _ptr(f)))
        return f

    def warmstart_block(self, net: "Net", k: int, opts: Optional[EigOpts] = None):
        """Start block for eigenmodes(k, opts, X0=...): (m + guard, n) tensor of
        the context's precision (column-major n x (m + guard))."""
        import torch
        guard = opts.guard if opts is not None else 8
        kw = k if (opts is not None and opts.exclude_constant) else k - 1
        X0 = torch.empty((kw + max(0, guard), self.n), dtype=self.dtype,
                         device=f"cuda:{self.device}")
        self._check(self.L.ff_warmstart_block(self.h, net.h, int(k),
                                              ctypes.byref(opts) if opts is not None else None,
                                              _ptr(X0)))
        return X0

    # ---- profiling
    def profile(self, on: bool, classes=None):
        """Start (reset) or stop the event profiler; `classes` restricts the
        recording to those profile classes (names of PROF)."""
        if classes is None:
            self._check(self.L.ff_profile_enable(self.h, 1 if on else 0))
        else:
            mask = 0
            for name in classes:
                mask |= 1 << PROF[name]
            self._check(self.L.ff_profile_classes(self.h, mask if on else 0))

    def profile_read(self):
        """{class: (scopes, total_ms)} for every profile class."""
        out = {}
        for name, cls in PROF.items():
            cnt, ms = ctypes.c_int64(), ctypes.c_double()
            self._check(self.L.ff_profile_read(self.h, cls, ctypes.byref(cnt), ctypes.byref(ms)))
            out[name] = (cnt.value, ms.value)
        return out

    # ---- inspection
    def sizes(self):
        n, n1, n2 = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self._check(self.L.ff_get_sizes(self.h, ctypes.byref(n), ctypes.byref(n1),
                                        ctypes.byref(n2)))
        return n.value, n1.value, n2.value

    def row_ptr(self):
        """Row offsets (int64, rows + 1) of the neighbour / covering lists."""
        npt = ctypes.c_int64()
        st = self.L.ff_get_twoset(self.h, ctypes.byref(npt), None, None, None)
        rows = npt.value if st == FF_OK else self.sizes()[0]
        out = np.zeros(rows + 1, np.int64)
        self._check(self.L.ff_export_row_ptr(self.h, out.ctypes.data))
        return out

    def pair_products(self):
        """sum over rows of (row length)^2: the pair products of the assembly."""
        c = np.diff(self.row_ptr()).astype(np.float64)
        return int(np.dot(c, c))

    def precond_layout(self):
        """(row_blocks, ksteps) of the preconditioner's tensor-core tiles; (0, 0)
        when they were not built."""
        rb, ks = ctypes.c_int64(), ctypes.c_int64()
        self._check(self.L.ff_get_precond_layout(self.h, ctypes.byref(rb), ctypes.byref(ks)))
        return rb.value, ks.value

    def export_rkpm(self):
        n, n1, _ = self.sizes()
        npt = ctypes.c_int64()
        if self.L.ff_get_twoset(self.h, ctypes.byref(npt), None, None, None) == FF_OK:
            n = npt.value                # rows: the quadrature points
        ptr = np.zeros(n + 1, np.int64)
        idx = np.zeros(n1, np.int32)
        phi = np.zeros(n1, np.float64)
        dphi = np.zeros(3 * n1, np.float64)
        self._check(self.L.ff_export_rkpm(self.h, ptr.ctypes.data, idx.ctypes.data,
                                          phi.ctypes.data, dphi.ctypes.data))
        return ptr, idx, phi, dphi.reshape(3, n1)

    def export_matrices(self):
        n, _, n2 = self.sizes()
        ptr = np.zeros(n + 1, np.int64)
        col = np.zeros(n2, np.int32)
        H = np.zeros(n2, np.float64)
        M = np.zeros(n2, np.float64)
        self._check(self.L.ff_export_matrices(self.h, ptr.ctypes.data, col.ctypes.data,
                                              H.ctypes.data, M.ctypes.data))
        return ptr, col, H, M

    def apply_operators(self, X):
        """X: (n, m) CUDA tensor of the context dtype -> (H X, M X)."""
        import torch
        m = int(X.shape[1])
        Xc = X.t().contiguous()          # column-major n x m
        YH = torch.empty_like(Xc)
        YM = torch.empty_like(Xc)
        self._check(self.L.ff_apply_operators(self.h, _ptr(Xc), m, _ptr(YH), _ptr(YM)))
        return YH.t(), YM.t()

    def apply_operators_matfree(self, X, E=None, nu=None, E0=1e5, nu0=0.45):
        """(H X, M X) from the shape-function tables without assembled matrices;
        the material as for assemble_hessian (E, nu per-particle float32 CUDA
        tensors or None for the uniform E0, nu0)."""
        import torch
        m = int(X.shape[1])
        Xc = X.t().contiguous()
        YH = torch.empty_like(Xc)
        YM = torch.empty_like(Xc)
        self._check(self.L.ff_apply_operators_matfree(self.h, _ptr(E), _ptr(nu), float(E0),
                                                      float(nu0), _ptr(Xc), m, _ptr(YH),
                                                      _ptr(YM)))
        return YH.t(), YM.t()

    def apply_operators_noalloc(self, X, YH=None, YM=None):
        """Same as apply_operators, through the allocation-free entry point; the
        caller may pass preallocated column-major outputs (m, n) tensors."""
        import torch
        m = int(X.shape[1])
        Xc = X.t().contiguous()
        YH = torch.empty_like(Xc) if YH is None else YH
        YM = torch.empty_like(Xc) if YM is None else YM
        self._check(self.L.ff_apply_operators_noalloc(self.h, _ptr(Xc), m, _ptr(YH), _ptr(YM)))
        return YH.t(), YM.t()

    # ---- skinning weights and linear blend skinning (Sec. 3.2, Eq. 1)
    def skinning_weights(self, Q, C):
        """W (nq, m) with W[q, j] = sum_k phi_k(Q_q) C[k, j]: Q a (nq, 3) float32 CUDA
        tensor, C the (n, m) nodal values in the context dtype and the caller's
        particle order (e.g. the modes eigenmodes returns)."""
        import torch
        Q = Q.contiguous()
        Ct = C.t().contiguous()          # column-major n x m
        nq, m = int(Q.shape[0]), int(Ct.shape[0])
        W = torch.empty((nq, m), dtype=self.dtype, device=Q.device)
        self._check(self.L.ff_skinning_weights(self.h, _ptr(Q), nq, _ptr(Ct), m, _ptr(W)))
        return W

    def lbs(self, Q, W, Z):
        """x = X + sum_j W[:, j] Z_j [X; 1] (Eq. 1) for rest positions Q (nq, 3) float32,
        weights W (nq, m) and affine transforms Z (m, 3, 4), both in the context dtype."""
        import torch
        Q, W, Z = Q.contiguous(), W.contiguous(), Z.contiguous()
        nq, m = int(Q.shape[0]), int(W.shape[1])
        x = torch.empty((nq, 3), dtype=self.dtype, device=Q.device)
        self._check(self.L.ff_lbs_deform(self.h, _ptr(Q), nq, _ptr(W), m, _ptr(Z), _ptr(x)))
        return x


# module-level names matching the C ABI
def rkpm_build(ctx: Context, particles, volumes, support):
    return ctx.rkpm_build(particles, volumes, support)


def eigenmodes_batched(objects, precision="fp64", opts: Optional[EigOpts] = None,
                       workers: int = 0, device: int = 0):
    """The three calls for many objects in one call, overlapped on one GPU.

    objects: list of dicts with float32 CUDA tensors X (n, 3), v (n,), a (n,),
    optional per-particle E and nu tensors (else the scalars E0, nu0) and k.
    Returns (status, results) with one (eigvals numpy (k,), modes torch (n, k)
    column-major view, report dict, status, error message) per object."""
    import torch
    L = load_library()
    dtype = torch.float64 if precision == "fp64" else torch.float32
    items = (BatchItem * max(len(objects), 1))()
    keep, outs = [], []
    for it, o in zip(items, objects):
        for t in (o["X"], o["v"], o["a"]):
            assert t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.float32"
        n, k = int(o["X"].shape[0]), int(o["k"])
        ev = np.zeros(k, np.float64)
        modes = torch.empty((k, n), dtype=dtype, device=f"cuda:{device}")
        rep = EigReport()
        it.particles, it.volumes, it.support = _ptr(o["X"]), _ptr(o["v"]), _ptr(o["a"])
        it.n, it.k = n, k
        it.E, it.nu = _ptr(o.get("E")), _ptr(o.get("nu"))
        it.E0, it.nu0 = float(o.get("E0", 1e5)), float(o.get("nu0", 0.45))
        it.eigvals = ev.ctypes.data
        it.modes = _ptr(modes)
        it.report = ctypes.addressof(rep)
        keep.append(o)
        outs.append((ev, modes, rep))
    st = L.eigenmodes_batched(device, PREC[precision], items, len(objects),
                              ctypes.byref(opts) if opts is not None else None, int(workers))
    res = [(ev, modes.t(), rep.as_dict(), it.status, it.error.decode())
           for (ev, modes, rep), it in zip(outs, items)]
    return st, res


def rkpm_build_twoset(ctx: Context, points, volumes, K, trunc=3.0, start=0):
    return ctx.rkpm_build_twoset(points, volumes, K, trunc, start)


def assemble_hessian(ctx: Context, E=None, nu=None, E0=1e5, nu0=0.45):
    return ctx.assemble_hessian(E, nu, E0, nu0)


def eigenmodes(ctx: Context, k, opts=None, X0=None):
    return ctx.eigenmodes(k, opts, X0)


def _host(x, dtype=np.float32):
    """(host pointer, bytes, keep-alive) of a host array: a numpy array or a CPU
    (optionally pinned) torch tensor; None passes through as NULL."""
    if x is None:
        return None, 0, None
    if hasattr(x, "data_ptr"):
        assert not x.is_cuda and x.is_contiguous()
        return int(x.data_ptr()), x.numel() * x.element_size(), x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, a.nbytes, a


def subspace_from_host(X, v, a, E, nu, k, precision="fp32", opts=None, device=0, ctx=None):
    """End-to-end public call on HOST arrays (ff_subspace_host): the library
    copies the cloud to the device, builds, assembles, solves, and copies
    eigenvalues and modes back.  X, v, a (and E, nu when they are arrays) are
    numpy arrays or CPU torch tensors (pinned ones copy asynchronously); E, nu
    may be scalars.  Returns (eigvals, modes (n, k) numpy, report, bytes_h2d,
    bytes_d2h, status)."""
    own = ctx is None
    if own:
        ctx = Context(device, precision)
    n = int(X.shape[0])
    ptrs = [_host(t) for t in (X, v, a)]
    Ep = _host(E) if np.ndim(E) > 0 else (None, 0, None)
    nup = _host(nu) if np.ndim(nu) > 0 else (None, 0, None)
    E0 = 1.0 if Ep[0] else float(E)
    nu0 = 0.3 if nup[0] else float(nu)
    ev = np.zeros(k, np.float64)
    modes = np.zeros((k, n), np.float64 if precision == "fp64" else np.float32)
    rep = EigReport()
    st = ctx.L.ff_subspace_host(ctx.h, ptrs[0][0], ptrs[1][0], ptrs[2][0], Ep[0], nup[0], n,
                                E0, nu0, int(k), ctypes.byref(opts) if opts is not None else None,
                                ev.ctypes.data, modes.ctypes.data, ctypes.byref(rep))
    if st not in (FF_OK, 5, 7):
        raise FreeformError(st, ctx.L.ff_last_error(ctx.h).decode())
    h2d_bytes = sum(p[1] for p in ptrs) + Ep[1] + nup[1]
    d2h_bytes = modes.nbytes + ev.nbytes
    if own:
        ctx.close()
    return ev, modes.T, rep.as_dict(), h2d_bytes, d2h_bytes, st


def subspace_twoset_from_host(points, volumes, E, nu, K, k, trunc=3.0, start=0,
                              precision="fp64", opts=None, device=0, ctx=None, modes_out=None):
    """The two-set construction end to end from HOST arrays
    (ff_subspace_twoset_host).  points (n, 3), volumes (n,) and E / nu (arrays
    of n, or scalars) are numpy arrays or CPU torch tensors; modes_out, if
    given, is a host array (k, K) of the context precision to write into.
    Returns (eigvals, modes (k, K): row j = mode j, report, bytes_h2d,
    bytes_d2h, status)."""
    own = ctx is None
    if own:
        ctx = Context(device, precision)
    n = int(points.shape[0])
    Xp, vp_ = _host(points), _host(volumes)
    Ep = _host(E) if np.ndim(E) > 0 else (None, 0, None)
    nup = _host(nu) if np.ndim(nu) > 0 else (None, 0, None)
    E0 = 1.0 if Ep[0] else float(E)
    nu0 = 0.3 if nup[0] else float(nu)
    ev = np.zeros(k, np.float64)
    if modes_out is None:
        modes_out = np.zeros((k, K), np.float64 if precision == "fp64" else np.float32)
    Mp = _host(modes_out, modes_out.dtype if isinstance(modes_out, np.ndarray) else None)
    rep = EigReport()
    st = ctx.L.ff_subspace_twoset_host(ctx.h, Xp[0], vp_[0], Ep[0], nup[0], n, int(K),
                                       float(trunc), int(start), E0, nu0, int(k),
                                       ctypes.byref(opts) if opts is not None else None,
                                       ev.ctypes.data, Mp[0], ctypes.byref(rep))
    if st not in (FF_OK, 5, 7):
        raise FreeformError(st, ctx.L.ff_last_error(ctx.h).decode())
    h2d_bytes = Xp[1] + vp_[1] + Ep[1] + nup[1]
    d2h_bytes = Mp[1] + ev.nbytes
    if own:
        ctx.close()
    return ev, modes_out, rep.as_dict(), h2d_bytes, d2h_bytes, st


class Net:
    """The warm-start point network (ff_net): parameters, Adam state, kernels."""

    def __init__(self, device: int = 0, stream=None, seed: Optional[int] = None):
        import torch
        self.L = load_library()
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = ctypes.c_void_p()
        st = self.L.ff_net_create(ctypes.byref(h), device, ctypes.c_void_p(stream.cuda_stream))
        if st != FF_OK:
            raise FreeformError(st, "ff_net_create failed")
        self.h = h
        self.P = int(self.L.ff_net_num_params())
        if seed is not None:
            self._check(self.L.ff_net_init(self.h, int(seed)))

    def _check(self, st):
        if st != FF_OK:
            raise FreeformError(st, self.L.ff_net_last_error(self.h).decode())

    def close(self):
        if self.h:
            self.L.ff_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        out = np.empty(self.P, dtype=np.float32)
        self._check(self.L.ff_net_get_params(self.h, out.ctypes.data_as(ctypes.c_void_p), self.P))
        return out

    def set_params(self, theta) -> None:
        theta = np.ascontiguousarray(theta, dtype=np.float32)
        if theta.size != self.P:
            raise ValueError(f"expected {self.P} parameters")
        self._check(self.L.ff_net_set_params(self.h, theta.ctypes.data_as(ctypes.c_void_p), self.P))

    def forward(self, feat):
        import torch
        n = int(feat.shape[0])
        out = torch.empty((n, 32), dtype=torch.float32, device=feat.device)
        self._check(self.L.ff_net_forward(self.h, _ptr(feat), n, _ptr(out)))
        return out

    @staticmethod
    def _cloud_args(feat, vol, modes):
        n = int(feat.shape[0])
        if modes.dim() != 2 or modes.shape[1] != n or not modes.is_contiguous():
            raise ValueError("modes must be a contiguous (m, n) tensor (column-major n x m)")
        return n, int(modes.shape[0])

    def loss_grad(self, feat, vol, modes):
        """(loss, grad numpy float32) for one cloud; modes is (m, n)."""
        n, m = self._cloud_args(feat, vol, modes)
        loss = ctypes.c_double()
        grad = np.empty(self.P, dtype=np.float32)
        self._check(self.L.ff_net_loss_grad(self.h, _ptr(feat), _ptr(vol), n, _ptr(modes), m,
                                            ctypes.byref(loss), grad.ctypes.data_as(ctypes.c_void_p)))
        return loss.value, grad

    def train_step(self, feat, vol, modes, lr: float) -> float:
        n, m = self._cloud_args(feat, vol, modes)
        loss = ctypes.c_double()
        self._check(self.L.ff_net_train_step(self.h, _ptr(feat), _ptr(vol), n, _ptr(modes), m,
                                             ctypes.c_float(lr), ctypes.byref(loss)))
        return loss.value
