"""Python face of the C ABI: one plan per point cloud, evaluations on it.

Only argument marshalling happens here; every step of an evaluation runs in
libkifmm.so's CUDA kernels.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _native as N


def _ptr(a):
    """Raw address of a numpy array or a torch tensor."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _points(a, what="points"):
    """(n, 3) float64 numpy array or torch tensor, contiguous."""
    if isinstance(a, np.ndarray):
        pts = np.ascontiguousarray(a, dtype=np.float64)
        if pts.ndim != 2 or pts.shape[1] != 3:
            raise ValueError(f"{what} must be (n, 3)")
        return pts
    pts = a.contiguous()
    if str(pts.dtype) != "torch.float64" or pts.dim() != 2 or pts.shape[1] != 3:
        raise ValueError(f"{what} must be a (n, 3) float64 tensor")
    return pts


def _options(options):
    L = N.lib()
    opts = N.Options()
    L.fmm_options_init(ctypes.byref(opts))
    for k, v in options.items():
        if not hasattr(opts, k):
            raise TypeError(f"unknown option {k}")
        setattr(opts, k, v)
    return opts


def set_operator_cache(directory):
    """Keep the FP64 operator precomputation in files under ``directory``
    (an existing directory; None turns the cache off, the default).  Plans
    created afterwards in this process read their operators from there, or
    compute and write them; see fmm_set_operator_cache in kifmm.h."""
    d = None if directory is None else os.fsencode(directory)
    N.check(N.lib().fmm_set_operator_cache(d))


class FMMPlan:
    """A KIFMM plan over n points.

    points: (n, 3) float64, numpy (host) or torch tensor (host or CUDA); the
    sources, which are also the targets (Eq. (1)) unless ``targets`` gives n
    distinct target points (the tree is then built on the union).
    p: expansion order; ncrit: largest leaf before a split.
    Options (see include/kifmm.h): alpha_inner, alpha_outer, rcond, eps_svd,
    max_level, balance, m2l_mode, host_only, device, tree_build, direct_wx.
    """

    def __init__(self, points, p: int, ncrit: int, targets=None, **options):
        L = N.lib()
        opts = _options(options)
        pts = _points(points)
        tgt = None if targets is None else _points(targets, "targets")
        if tgt is not None and tgt.shape[0] != pts.shape[0]:
            raise ValueError("targets must have as many rows as points")
        self._keep = (pts, tgt)
        self.n = int(pts.shape[0])
        self.p, self.ncrit = p, ncrit
        self.host_only = bool(options.get("host_only", 0))
        self.sizes = [self.n]
        h = ctypes.c_void_p()
        N.check(L.fmm_plan_create_ex(_ptr(pts), None if tgt is None else _ptr(tgt), self.n, p,
                                     ncrit, ctypes.byref(opts), ctypes.byref(h)))
        self._h = h

    @classmethod
    def batch(cls, point_sets, p: int, ncrit: int, target_sets=None, **options):
        """One plan for independent problems (fmm_plan_create_batch).

        point_sets: list of (n_i, 3) float64 arrays or tensors; target_sets:
        None or a list with None (targets = sources) or (n_i, 3) per problem.
        Evaluations take charges of sum(n_i) rows, problem 0 first; use
        ``split`` to cut the result per problem.
        """
        L = N.lib()
        opts = _options(options)
        pts = [_points(x) for x in point_sets]
        if not pts:
            raise ValueError("no problems")
        tgts = [None] * len(pts) if target_sets is None else \
            [None if t is None else _points(t, "targets") for t in target_sets]
        if len(tgts) != len(pts):
            raise ValueError("one target set per problem")
        sizes = [int(x.shape[0]) for x in pts]
        for t, n in zip(tgts, sizes):
            if t is not None and int(t.shape[0]) != n:
                raise ValueError("targets must have as many rows as the problem's points")
        self = cls.__new__(cls)
        self._keep = (pts, tgts)
        self.sizes = sizes
        self.n = sum(sizes)
        self.p, self.ncrit = p, ncrit
        self.host_only = bool(options.get("host_only", 0))
        src_arr = (ctypes.c_void_p * len(pts))(*[_ptr(x) for x in pts])
        tgt_arr = (ctypes.c_void_p * len(pts))(*[None if t is None else _ptr(t) for t in tgts])
        n_arr = (ctypes.c_int64 * len(pts))(*sizes)
        h = ctypes.c_void_p()
        N.check(L.fmm_plan_create_batch_ex(src_arr, tgt_arr, n_arr, len(pts), p, ncrit,
                                           ctypes.byref(opts), ctypes.byref(h)))
        self._h = h
        return self

    def split(self, result):
        """Cut an evaluation result (rows of all problems) per problem."""
        out, r = [], 0
        for n in self.sizes:
            out.append(result[r:r + n])
            r += n
        return out

    # ---------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            N.lib().fmm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---------------------------------------------------------------
    def set_m2l_mode(self, mode: int):
        N.check(N.lib().fmm_plan_set_option(self._h, N.OPT_M2L_MODE, float(mode)))

    def set_autotune(self, on: bool):
        """Time the level products' tile shapes on the first evaluation of
        each nrhs (default on; results are bit-identical either way)."""
        N.check(N.lib().fmm_plan_set_option(self._h, N.OPT_AUTOTUNE, 1.0 if on else 0.0))

    def set_gemm_shape(self, shape: int):
        """Force one level-product tile shape (0, 1, 2) or -1 for automatic."""
        N.check(N.lib().fmm_plan_set_option(self._h, N.OPT_GEMM_SHAPE, float(shape)))

    def set_knobs(self, knobs: int):
        """-1: the autotuner's choice of the M2L block schedule and the leaf
        launch order; 0..3 forces them (FMM_OPT_FORCE_KNOBS)."""
        N.check(N.lib().fmm_plan_set_option(self._h, N.OPT_FORCE_KNOBS, float(knobs)))

    def set_m2l_kernel(self, kernel: int):
        """Tensor-core M2L kernel: 0 pair columns (operand width <= 128),
        1 target tiles (the default) (FMM_OPT_M2L_KERNEL)."""
        N.check(N.lib().fmm_plan_set_option(self._h, N.OPT_M2L_KERNEL, float(kernel)))

    def set_graph(self, on: bool):
        """Capture/replay evaluations as a CUDA graph (default on; never on
        the legacy default stream)."""
        N.check(N.lib().fmm_plan_set_option(self._h, N.OPT_GRAPH, 1.0 if on else 0.0))

    def evaluate(self, charges, out=None, stream=None):
        """Potentials (n, nrhs) float64 for charges (n,) or (n, nrhs) float32.

        Torch CUDA tensors: the work is enqueued on ``stream`` (default: the
        current torch stream) and the call returns at once.  Numpy arrays:
        the library stages them through device memory and returns when done.
        """
        if isinstance(charges, np.ndarray):
            q = np.ascontiguousarray(charges, dtype=np.float32)
            vec = q.ndim == 1
            q = q.reshape(self.n, -1)
            nrhs = q.shape[1]
            if out is None:
                out = np.empty((self.n, nrhs), dtype=np.float64)
            st = 0 if stream is None else int(stream)
            N.check(N.lib().fmm_evaluate(self._h, q.ctypes.data, nrhs, out.ctypes.data,
                                         ctypes.c_void_p(st)))
            return out[:, 0] if vec else out
        import torch
        q = charges
        if q.dtype != torch.float32:
            raise TypeError("charges must be float32")
        vec = q.dim() == 1
        q = q.reshape(self.n, -1).contiguous()
        nrhs = q.shape[1]
        if out is None:
            out = torch.empty((self.n, nrhs), dtype=torch.float64, device=q.device)
        if stream is None:
            stream = torch.cuda.current_stream(q.device) if q.is_cuda else None
        st = 0 if stream is None else stream.cuda_stream
        N.check(N.lib().fmm_evaluate(self._h, q.data_ptr(), nrhs, out.data_ptr(),
                                     ctypes.c_void_p(st)))
        return out[:, 0] if vec else out

    def evaluate_gradient(self, charges, grad_out=None, out=None, potentials=True, stream=None):
        """(potentials, gradients) for charges (n,) or (n, nrhs) float32: the
        gradient of each target's potential with respect to its position,
        (n, 3) or (n, nrhs, 3) float64 (the field is minus this).  With
        potentials=False only the gradients are written (the first item is
        None).  Streams and host/device handling as in evaluate()."""
        if isinstance(charges, np.ndarray):
            q = np.ascontiguousarray(charges, dtype=np.float32)
            vec = q.ndim == 1
            q = q.reshape(self.n, -1)
            nrhs = q.shape[1]
            if grad_out is None:
                grad_out = np.empty((self.n, nrhs, 3), dtype=np.float64)
            if potentials and out is None:
                out = np.empty((self.n, nrhs), dtype=np.float64)
            st = 0 if stream is None else int(stream)
            N.check(N.lib().fmm_evaluate_gradient(
                self._h, q.ctypes.data, nrhs, out.ctypes.data if potentials else None,
                grad_out.ctypes.data, ctypes.c_void_p(st)))
        else:
            import torch
            q = charges
            if q.dtype != torch.float32:
                raise TypeError("charges must be float32")
            vec = q.dim() == 1
            q = q.reshape(self.n, -1).contiguous()
            nrhs = q.shape[1]
            if grad_out is None:
                grad_out = torch.empty((self.n, nrhs, 3), dtype=torch.float64, device=q.device)
            if potentials and out is None:
                out = torch.empty((self.n, nrhs), dtype=torch.float64, device=q.device)
            if stream is None:
                stream = torch.cuda.current_stream(q.device) if q.is_cuda else None
            st = 0 if stream is None else stream.cuda_stream
            N.check(N.lib().fmm_evaluate_gradient(
                self._h, q.data_ptr(), nrhs, out.data_ptr() if potentials else None,
                grad_out.data_ptr(), ctypes.c_void_p(st)))
        phi = (out[:, 0] if vec else out) if potentials else None
        return phi, (grad_out[:, 0, :] if vec else grad_out)

    # ---------------------------------------------------------------
    def info(self, key: str) -> int:
        v = ctypes.c_int64()
        N.check(N.lib().fmm_plan_info(self._h, N.INFO[key], ctypes.byref(v)))
        return v.value

    def array(self, name: str) -> np.ndarray:
        which, dt = N.ARRAYS[name]
        need = ctypes.c_int64()
        N.check(N.lib().fmm_plan_get_array(self._h, which, None, 0, ctypes.byref(need)))
        out = np.empty(need.value // np.dtype(dt).itemsize, dtype=dt)
        N.check(N.lib().fmm_plan_get_array(self._h, which, out.ctypes.data, need.value,
                                           ctypes.byref(need)))
        return out

    def workspace(self, name: str) -> np.ndarray:
        """Per-box results of the last evaluation's passes, float32
        (nodes, nrhs, ld): "up", "down", "qhat" or "chat" (conventions in
        fmm_plan_get_workspace, kifmm.h)."""
        which = {"up": 0, "down": 1, "qhat": 2, "chat": 3}[name]
        need = ctypes.c_int64()
        N.check(N.lib().fmm_plan_get_workspace(self._h, which, None, 0, ctypes.byref(need)))
        out = np.empty(need.value // 4, dtype=np.float32)
        N.check(N.lib().fmm_plan_get_workspace(self._h, which, out.ctypes.data, need.value,
                                               ctypes.byref(need)))
        return out.reshape(self.info("nodes"), -1, self._ws_ld(name))

    def _ws_ld(self, name):
        if name in ("up", "down"):
            return (self.info("nsurf") + 3) // 4 * 4
        return (self.info("rank_m2l") + 15) // 16 * 16

    def phase_ms(self):
        """Per-phase milliseconds of the last evaluation (needs FMM_TIMING=1)."""
        out = []
        for ph in range(4):
            v = ctypes.c_double()
            N.check(N.lib().fmm_plan_phase_ms(self._h, ph, ctypes.byref(v)))
            out.append(v.value)
        return dict(zip(("upward", "m2l", "downward", "leaf"), out))
