"""GB300 expectation propagation for image restoration with an l1-TV prior.

Python front end of libeptv (include/ep_tv.h): a thin ctypes binding with the
same names as the C ABI.  PyTorch supplies device memory and streams; every step
of the method runs in the library's CUDA kernels.

Method: Yao, McLaughlin and Altmann, "Fast Scalable Image Restoration using
Total Variation Priors and Expectation Propagation", arXiv:2110.01585.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np

from . import _lib
from ._lib import (OP_CONV_PERIODIC, OP_DENSE, OP_HADAMARD, OP_IDENTITY, PRIOR_BG, PRIOR_L1, PRIOR_MOG2,
                   EPTVError)

__all__ = ["EPTV", "Batch", "solve_host", "EPTVError", "OP_IDENTITY", "OP_CONV_PERIODIC", "OP_DENSE",
           "OP_HADAMARD",
           "PRIOR_L1", "PRIOR_MOG2", "PRIOR_BG",
           "default_params"]


def _torch():
    import torch
    return torch


def default_params(**kw) -> _lib.Params:
    lib = _lib.load()
    p = _lib.Params()
    _lib.check(lib.ep_tv_default_params(ctypes.byref(p)), "ep_tv_default_params")
    for k, v in kw.items():
        if v is None:
            continue
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


def _operator(op: int, height: int, width: int, m: int, kernel=None, dense=None, patterns=None):
    o = _lib.Operator()
    o.op, o.height, o.width, o.m = op, height, width, m
    keep = []
    if kernel is not None:
        k = np.ascontiguousarray(kernel, dtype=np.float32)
        o.kernel = k.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        o.kh, o.kw = k.shape
        keep.append(k)
    if dense is not None:
        o.dense = ctypes.c_void_p(dense.data_ptr())
    if patterns is not None:
        pt = np.ascontiguousarray(patterns, dtype=np.int32)
        o.patterns = pt.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        keep.append(pt)
    return o, keep


class EPTV:
    """One restoration problem on the GPU (wraps an ``ep_tv_ctx``).

    y: CUDA float32 tensor, (H, W) for identity/convolution, (M,) for dense and
        Hadamard sensing.
    kernel: host array (kh, kw) for the periodic convolution.
    dense: CUDA float32 tensor (M, N) for compressive sensing; kept alive here.
    patterns: host integer array of M Paley-ordered pattern indices p = kr * W + kc
        for the subsampled Hadamard operator (op=OP_HADAMARD).
    xi_plane: CUDA float32 tensor of M noise variances (a diagonal noise
        covariance, ep_tv_init_noise); xi is then ignored.
    stream: torch.cuda.Stream (default: the current stream).
    Remaining keyword arguments set fields of ``ep_tv_params``.
    """

    def __init__(self, y, xi: float, beta: float, op: int = OP_IDENTITY, height: int = None,
                 width: int = None, kernel=None, dense=None, stream=None, xi_plane=None,
                 patterns=None, **params):
        torch = _torch()
        self._lib = _lib.load()
        if not (isinstance(y, torch.Tensor) and y.is_cuda and y.dtype == torch.float32):
            raise TypeError("y must be a CUDA float32 tensor")
        y = y.contiguous()
        if height is None or width is None:
            if y.dim() != 2:
                raise ValueError("height and width are needed when y is not an image")
            height, width = y.shape
        self.height, self.width = int(height), int(width)
        self.n = self.height * self.width
        self.device = y.device
        self.stream = stream if stream is not None else torch.cuda.current_stream(y.device)
        self._dense = dense.contiguous() if dense is not None else None
        o, self._kernel_keep = _operator(op, self.height, self.width, y.numel(), kernel, self._dense,
                                         patterns)
        self.params = default_params(xi=float(xi), beta=float(beta), **params)
        ctx = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            if xi_plane is None:
                code = self._lib.ep_tv_init(ctypes.byref(o), ctypes.c_void_p(y.data_ptr()),
                                            ctypes.byref(self.params),
                                            ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(ctx))
            else:
                self._xi_keep = xi_plane.contiguous()
                code = self._lib.ep_tv_init_noise(ctypes.byref(o), ctypes.c_void_p(y.data_ptr()),
                                                  ctypes.c_void_p(self._xi_keep.data_ptr()),
                                                  ctypes.byref(self.params),
                                                  ctypes.c_void_p(self.stream.cuda_stream),
                                                  ctypes.byref(ctx))
        _lib.check(code, "ep_tv_init" if xi_plane is None else "ep_tv_init_noise")
        self._ctx = ctx

    # -- lifecycle
    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.ep_tv_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- method
    def set_probes(self, eps1, eps2):
        """Caller-drawn RBMC probes: CUDA float32 (S, M) and (S, N)."""
        eps1 = eps1.contiguous()
        eps2 = eps2.contiguous()
        _lib.check(self._lib.ep_tv_set_probes(self._ctx, ctypes.c_void_p(eps1.data_ptr()),
                                              ctypes.c_void_p(eps2.data_ptr()), int(eps1.shape[0])),
                   "ep_tv_set_probes")
        self._probes_keep = (eps1, eps2)

    def sweep(self, n: int = 1, k_order: Optional[Sequence[Sequence[int]]] = None, em_every: int = 0):
        ko = None
        if k_order is not None:
            flat = np.asarray(k_order, dtype=np.int8).reshape(-1)
            if flat.size != 4 * n:
                raise ValueError("k_order needs 4 entries per sweep")
            ko = (ctypes.c_int8 * flat.size)(*flat.tolist())
        _lib.check(self._lib.ep_tv_sweep(self._ctx, int(n), ko, int(em_every)), "ep_tv_sweep")

    def em_beta(self, sync: bool = True):
        """EM step beta = N / a_u; returns (beta, a_u) when sync is set."""
        if not sync:
            _lib.check(self._lib.ep_tv_em_beta(self._ctx, None, None), "ep_tv_em_beta")
            return None
        b, a = ctypes.c_double(), ctypes.c_double()
        _lib.check(self._lib.ep_tv_em_beta(self._ctx, ctypes.byref(b), ctypes.byref(a)), "ep_tv_em_beta")
        return b.value, a.value

    def ep_em(self, n_em: int, max_sweeps: int = 200, tol: float = 1e-5):
        """Algorithm 2 with EP run to convergence inside every EM iteration;
        returns (beta after each iteration, sweeps of each inner run)."""
        betas = (ctypes.c_double * n_em)()
        sweeps = (ctypes.c_int32 * n_em)()
        _lib.check(self._lib.ep_tv_ep_em(self._ctx, int(n_em), int(max_sweeps), float(tol), betas,
                                         sweeps), "ep_tv_ep_em")
        return list(betas), list(sweeps)

    def set_beta(self, beta: float):
        _lib.check(self._lib.ep_tv_set_beta(self._ctx, float(beta)), "ep_tv_set_beta")

    def posterior(self, mean=None, var=None):
        """Posterior mean and marginal variance as CUDA float32 (H, W) tensors."""
        torch = _torch()
        if mean is None:
            mean = torch.empty((self.height, self.width), device=self.device, dtype=torch.float32)
        if var is None:
            var = torch.empty((self.height, self.width), device=self.device, dtype=torch.float32)
        _lib.check(self._lib.ep_tv_posterior(self._ctx, ctypes.c_void_p(mean.data_ptr()),
                                             ctypes.c_void_p(var.data_ptr())), "ep_tv_posterior")
        return mean, var

    def sites(self):
        """(tau, nu) as CUDA float32 (5, H, W) tensors."""
        torch = _torch()
        tau = torch.empty((5, self.height, self.width), device=self.device, dtype=torch.float32)
        nu = torch.empty_like(tau)
        _lib.check(self._lib.ep_tv_get_sites(self._ctx, ctypes.c_void_p(tau.data_ptr()),
                                             ctypes.c_void_p(nu.data_ptr())), "ep_tv_get_sites")
        return tau, nu

    def status(self) -> int:
        return int(self._lib.ep_tv_status_check(self._ctx))

    def stats(self):
        it = ctypes.c_int32()
        f64 = ctypes.c_uint64()
        cap = ctypes.c_uint64()
        _lib.check(self._lib.ep_tv_stats(self._ctx, ctypes.byref(it), ctypes.byref(f64), ctypes.byref(cap)),
                   "ep_tv_stats")
        return {"cg_iters": it.value, "n_fp64": f64.value, "n_capped": cap.value}

    def solver_report(self):
        """Last likelihood-site update: refinement passes, CG iterations, final
        relative residual of the mean solve and worst probe solve."""
        a, b = ctypes.c_int32(), ctypes.c_int32()
        rm, rp = ctypes.c_double(), ctypes.c_double()
        _lib.check(self._lib.ep_tv_solver_report(self._ctx, ctypes.byref(a), ctypes.byref(b),
                                                 ctypes.byref(rm), ctypes.byref(rp)), "ep_tv_solver_report")
        return {"passes": a.value, "iterations": b.value, "relres_mean": rm.value,
                "relres_probe_max": rp.value}

    def graph_sweeps(self) -> int:
        """Sweeps of this context that ran from captured-graph replays."""
        return int(self._lib.ep_tv_graph_sweeps(self._ctx))

    def trace(self, on: bool = True):
        """Enable (and reset) or disable per-kernel CUDA-event tracing."""
        _lib.check(self._lib.ep_tv_trace_enable(self._ctx, int(bool(on))), "ep_tv_trace_enable")

    def trace_read(self):
        """{kernel name: (ms, launches, units, bytes_per_unit)} since tracing was enabled."""
        out = {}
        for kid, name in _lib.KERNELS.items():
            ms, n, u, b = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
            _lib.check(self._lib.ep_tv_trace_read(self._ctx, kid, ctypes.byref(ms), ctypes.byref(n),
                                                  ctypes.byref(u), ctypes.byref(b)), "ep_tv_trace_read")
            out[name] = (ms.value, n.value, u.value, b.value)
        return out

    def state_export(self) -> bytes:
        size = ctypes.c_size_t()
        _lib.check(self._lib.ep_tv_state_export(self._ctx, None, ctypes.byref(size)), "ep_tv_state_export")
        buf = ctypes.create_string_buffer(size.value)
        _lib.check(self._lib.ep_tv_state_export(self._ctx, buf, ctypes.byref(size)), "ep_tv_state_export")
        return buf.raw

    def state_import(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _lib.check(self._lib.ep_tv_state_import(self._ctx, buf, len(blob)), "ep_tv_state_import")

    def reset(self):
        _lib.check(self._lib.ep_tv_reset(self._ctx), "ep_tv_reset")


class Batch:
    """Many EPTV problems advanced together (``ep_tv_batch_*``).

    The problems must share one device and one stream and use order_mode 0.
    The batch keeps references to them; close the batch before the problems.
    """

    def __init__(self, problems):
        self._lib = _lib.load()
        self.problems = list(problems)
        arr = (ctypes.c_void_p * len(self.problems))(*[p._ctx.value for p in self.problems])
        out = ctypes.c_void_p()
        _lib.check(self._lib.ep_tv_batch_create(len(self.problems), arr, ctypes.byref(out)),
                   "ep_tv_batch_create")
        self._b = out

    def sweep(self, n: int = 1, em_every: int = 0):
        _lib.check(self._lib.ep_tv_batch_sweep(self._b, int(n), int(em_every)), "ep_tv_batch_sweep")

    def close(self):
        if getattr(self, "_b", None):
            self._lib.ep_tv_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def solve_host(y: np.ndarray, xi: float, beta: float, n_sweeps: int, em_every: int = 0,
               op: int = OP_IDENTITY, kernel=None, dense=None, height=None, width=None,
               patterns=None, **params):
    """One complete restoration from host memory (``ep_tv_solve_host``).

    Returns (mean, var, beta) as numpy arrays / float.
    """
    lib = _lib.load()
    y = np.ascontiguousarray(y, dtype=np.float32)
    if height is None or width is None:
        height, width = y.shape
    o, keep = _operator(op, int(height), int(width), y.size, kernel, dense, patterns)
    p = default_params(xi=float(xi), beta=float(beta), **params)
    mean = np.empty((height, width), np.float32)
    var = np.empty((height, width), np.float32)
    b = ctypes.c_double()
    code = lib.ep_tv_solve_host(ctypes.byref(o), y.ctypes.data_as(ctypes.c_void_p), ctypes.byref(p),
                                int(n_sweeps), int(em_every), mean.ctypes.data_as(ctypes.c_void_p),
                                var.ctypes.data_as(ctypes.c_void_p), ctypes.byref(b))
    _lib.check(code, "ep_tv_solve_host")
    return mean, var, b.value


WARM_ALL_SITES, WARM_SITE0, WARM_PRIOR = 0, 1, 2


def warm_start(ep: "EPTV", out, mode: int = WARM_ALL_SITES):
    """``ep_tv_warm_start``: set sites of ``ep`` from the warm-start network's
    output for its observation (CUDA float32 tensor, (6, H, W)); mode
    WARM_ALL_SITES, WARM_SITE0 (likelihood site only) or WARM_PRIOR (prior sites
    only)."""
    out = out.contiguous()
    _lib.check(ep._lib.ep_tv_warm_start(ep._ctx, ctypes.c_void_p(out.data_ptr()), int(mode)),
               "ep_tv_warm_start")
    ep._warm_keep = out
