"""GB300-native HyperNetVec V-cycle: the Python binding of ``libhnv.so``.

Argument marshalling only: every step of coarsening, projection and
refinement runs in the library's CUDA kernels. PyTorch supplies device
memory (tensors) and streams. Importing this package does not load the
library; the first call does, and raises ``HNVLibraryMissing`` when the
in-tree ``libhnv.so`` has not been built -- there is no CPU fallback.

The functions named like the C entry points (``hnv_build_incidence``,
``hnv_coarsen``, ``hnv_project``, ``hnv_refine``, ``hnv_vcycle``) take the
same arguments as in ``include/hnv.h`` with tensors/arrays in place of raw
pointers; ``Graph`` wraps them for convenience.
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

import numpy as np

__all__ = [
    "HNVError", "HNVLibraryMissing", "lib", "library_path",
    "ASSIGN_HASH", "ASSIGN_LOW_DEGREE", "ASSIGN_HIGH_WEIGHT", "ASSIGN_EXPLICIT",
    "SWEEP_TWO_PHASE", "SWEEP_JACOBI", "F32", "BF16", "BATCH_KERNEL_PER_CLASS",
    "BATCH_KERNEL_PERSISTENT",
    "ARR_E_PTR", "ARR_E_NODES", "ARR_V_PTR", "ARR_V_EDGES", "ARR_W", "ARR_REP_V",
    "ARR_REP_E", "ARR_DEG_V",
    "PHASE_BUILD", "PHASE_COARSEN", "PHASE_PROJECT", "PHASE_REFINE_E", "PHASE_REFINE_V",
    "PHASE_ADJOINT_REPLAY", "PHASE_ADJOINT_REVERSE", "PHASE_ADJOINT_PROJECT",
    "Graph", "hnv_build_incidence", "hnv_coarsen", "hnv_project", "hnv_refine",
    "hnv_vcycle", "hnv_refine_noalloc", "hnv_set_weights", "hnv_checkpoint_floats",
    "hnv_vcycle_save", "hnv_vcycle_backward", "vcycle_autograd", "Batch", "kernel_launch_count",
    "hnv_set_node_features", "hnv_copy_level_features", "hnv_refine_until", "timing_enable", "timing_reset", "timing_read",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "libhnv.so")

# enums of include/hnv.h
ASSIGN_HASH, ASSIGN_LOW_DEGREE, ASSIGN_HIGH_WEIGHT, ASSIGN_EXPLICIT, ASSIGN_COSINE = 0, 1, 2, 3, 4
SWEEP_TWO_PHASE, SWEEP_JACOBI = 0, 1
F32, BF16 = 0, 1
BATCH_KERNEL_PER_CLASS, BATCH_KERNEL_PERSISTENT = 0, 1
(ARR_E_PTR, ARR_E_NODES, ARR_V_PTR, ARR_V_EDGES, ARR_W, ARR_REP_V, ARR_REP_E,
 ARR_DEG_V) = range(8)
(PHASE_BUILD, PHASE_COARSEN, PHASE_PROJECT, PHASE_REFINE_E, PHASE_REFINE_V,
 PHASE_ADJOINT_REPLAY, PHASE_ADJOINT_REVERSE, PHASE_ADJOINT_PROJECT) = range(8)

ERR_NAMES = {0: "HNV_OK", -1: "HNV_ERR_INVALID_ARG", -2: "HNV_ERR_OUT_OF_RANGE",
             -3: "HNV_ERR_TOO_LARGE", -4: "HNV_ERR_OOM", -5: "HNV_ERR_CUDA",
             -6: "HNV_ERR_TIMEOUT", -7: "HNV_ERR_UNSUPPORTED_D", -8: "HNV_ERR_STATE"}


class HNVError(RuntimeError):
    """A non-zero status returned by libhnv.so."""

    def __init__(self, code: int, where: str, detail: str):
        self.code = code
        super().__init__("%s returned %s (%d): %s" % (where, ERR_NAMES.get(code, "?"), code, detail))


class HNVLibraryMissing(ImportError):
    pass


class CoarsenParams(ctypes.Structure):
    _fields_ = [("policy", ctypes.c_int32), ("min_nodes", ctypes.c_int32),
                ("max_levels", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("explicit_prio", ctypes.c_void_p)]


class BatchTuning(ctypes.Structure):
    _fields_ = [("a_max", ctypes.c_int32), ("b_max", ctypes.c_int32), ("c_max", ctypes.c_int32),
                ("lanes_a", ctypes.c_int32), ("lanes_b", ctypes.c_int32),
                ("lanes_rest", ctypes.c_int32), ("best_ms", ctypes.c_float),
                ("from_cache", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("persistent_ms", ctypes.c_float)]


_lib = None
_P = ctypes.c_void_p


def _declare(L):
    i32, i64, f32, sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_size_t
    sig = {
        "hnv_build_incidence": (ctypes.c_int, [i32, i32, _P, _P, _P, ctypes.c_int, _P, ctypes.POINTER(_P)]),
        "hnv_coarsen": (ctypes.c_int, [_P, ctypes.POINTER(CoarsenParams), ctypes.POINTER(i32)]),
        "hnv_num_levels": (ctypes.c_int, [_P, ctypes.POINTER(i32)]),
        "hnv_level_info": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i64)]),
        "hnv_get_level_arrays": (ctypes.c_int, [_P, ctypes.c_int] + [ctypes.POINTER(_P)] * 7),
        "hnv_copy_level_array": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, sz, ctypes.c_int, _P]),
        "hnv_project": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P, ctypes.c_int, ctypes.c_int, _P]),
        "hnv_refine": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_int, ctypes.c_int, f32, ctypes.c_int, ctypes.c_int, _P]),
        "hnv_vcycle": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, ctypes.c_int, f32, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]),
        "hnv_refine_noalloc": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_int, ctypes.c_int, f32, ctypes.c_int, _P]),
        "hnv_graph_free": (None, [_P]),
        "hnv_sync_status": (ctypes.c_int, [_P, _P]),
        "hnv_set_node_features": (ctypes.c_int, [_P, _P, i32, ctypes.c_int, _P]),
        "hnv_refine_until": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_int, ctypes.c_int,
                                            f32, ctypes.c_int, f32, ctypes.c_int,
                                            ctypes.POINTER(i32), ctypes.POINTER(f32), _P]),
        "hnv_copy_level_features": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_size_t,
                                                   ctypes.c_int, _P]),
        "hnv_level_feature_dim": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(i32)]),
        "hnv_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), i32, ctypes.POINTER(_P)]),
        "hnv_batch_offsets": (ctypes.c_int, [_P, _P, _P, _P]),
        "hnv_batch_autotune": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, f32, ctypes.POINTER(BatchTuning)]),
        "hnv_batch_vcycle": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, ctypes.c_int, f32, ctypes.c_int, ctypes.c_int, _P]),
        "hnv_batch_free": (None, [_P]),
        "hnv_batch_set_kernel": (ctypes.c_int, [_P, ctypes.c_int]),
        "hnv_release_cached_memory": (ctypes.c_int, []),
        "hnv_selftest_wait_timeout": (ctypes.c_int, [_P, ctypes.c_uint32, _P]),
        "hnv_batch_get_kernel": (ctypes.c_int, [_P]),
        "hnv_set_weights": (ctypes.c_int, [_P, _P, ctypes.c_int, _P]),
        "hnv_checkpoint_floats": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(i64)]),
        "hnv_vcycle_save": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, f32, ctypes.c_int, _P, _P]),
        "hnv_vcycle_backward": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, ctypes.c_int, f32, ctypes.c_int, _P]),
        "hnv_error_string": (ctypes.c_char_p, [ctypes.c_int]),
        "hnv_last_error_detail": (ctypes.c_char_p, []),
        "hnv_set_allocator": (ctypes.c_int, [_P, _P, _P]),
        "hnv_kernel_launch_count": (i64, []),
        "hnv_timing_enable": (ctypes.c_int, [ctypes.c_int]),
        "hnv_timing_reset": (ctypes.c_int, []),
        "hnv_timing_read": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_double)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def lib():
    """The loaded library (loads it on first use; raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(library_path):
            raise HNVLibraryMissing(
                "libhnv.so is not built (run paper_2103_09660_gb300/build.py); "
                "there is no CPU fallback")
        _lib = _declare(ctypes.CDLL(library_path))
    return _lib


def _check(rc: int, where: str):
    if rc != 0:
        raise HNVError(rc, where, lib().hnv_last_error_detail().decode(errors="replace"))


def _stream_handle(stream) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _dev_ptr(t, dtype, name: str, rows: Optional[int] = None, d: Optional[int] = None) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError("%s must be a contiguous %s tensor" % (name, dtype))
    if rows is not None and d is not None and tuple(t.shape) != (rows, d):
        raise ValueError("%s must have shape (%d, %d), got %s" % (name, rows, d, tuple(t.shape)))
    return t.data_ptr()


def _emb_dtype(t):
    """(hnv dtype code, torch dtype) of an embedding tensor: float32 -> F32,
    bfloat16 -> BF16 (stored as bfloat16, summed in float32)."""
    import torch
    if t.dtype == torch.float32:
        return F32, torch.float32
    if t.dtype == torch.bfloat16:
        return BF16, torch.bfloat16
    raise TypeError("embeddings must be float32 or bfloat16, got %s" % t.dtype)


# ---------------------------------------------------------------------------
# Entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

def hnv_build_incidence(n: int, m: int, edge_ptr, edge_nodes, edge_w=None, stream=None) -> int:
    """Returns the opaque graph handle. Arrays are numpy (host) or CUDA
    tensors (device): int64 edge_ptr[m+1], int32 edge_nodes[nnz], float32
    edge_w[m] or None."""
    import torch
    on_dev = isinstance(edge_ptr, torch.Tensor)
    keep = []
    if on_dev:
        p = _dev_ptr(edge_ptr, torch.int64, "edge_ptr")
        q = _dev_ptr(edge_nodes, torch.int32, "edge_nodes")
        w = _dev_ptr(edge_w, torch.float32, "edge_w") if edge_w is not None else None
    else:
        a = np.ascontiguousarray(edge_ptr, dtype=np.int64)
        b = np.ascontiguousarray(edge_nodes, dtype=np.int32)
        c = np.ascontiguousarray(edge_w, dtype=np.float32) if edge_w is not None else None
        keep = [a, b, c]
        p, q = a.ctypes.data, (b.ctypes.data if b.size else None)
        w = c.ctypes.data if c is not None else None
    g = _P()
    rc = lib().hnv_build_incidence(int(n), int(m), p, q, w, 1 if on_dev else 0,
                                   _stream_handle(stream), ctypes.byref(g))
    del keep
    _check(rc, "hnv_build_incidence")
    return g.value


def hnv_coarsen(g: int, policy: int = ASSIGN_HASH, seed: int = 0, min_nodes: int = 200,
                max_levels: int = 32, explicit_prio=None) -> int:
    tab = None
    if explicit_prio is not None:
        tab = np.ascontiguousarray(explicit_prio, dtype=np.uint64)
    prm = CoarsenParams(policy, min_nodes, max_levels, 0, seed & ((1 << 64) - 1),
                        tab.ctypes.data if tab is not None else None)
    out = ctypes.c_int32()
    _check(lib().hnv_coarsen(g, ctypes.byref(prm), ctypes.byref(out)), "hnv_coarsen")
    return out.value


def hnv_set_node_features(g: int, x, stream=None):
    """Level-0 node features (float32 [n0, k]): a numpy array (host) or a
    CUDA tensor (device)."""
    import torch
    if isinstance(x, torch.Tensor) and x.is_cuda:
        if x.dtype != torch.float32 or x.dim() != 2 or not x.is_contiguous():
            raise TypeError("features must be a contiguous float32 [n, k] tensor")
        _check(lib().hnv_set_node_features(g, x.data_ptr(), int(x.shape[1]), 1,
                                           _stream_handle(stream)), "hnv_set_node_features")
        return
    a = np.ascontiguousarray(x, dtype=np.float32)
    if a.ndim != 2:
        raise TypeError("features must be [n, k]")
    _check(lib().hnv_set_node_features(g, a.ctypes.data, int(a.shape[1]), 0,
                                       _stream_handle(stream)), "hnv_set_node_features")


def hnv_copy_level_features(g: int, level: int, stream=None) -> np.ndarray:
    """Host copy of a level's node features (float32 [n_l, k])."""
    k = ctypes.c_int32()
    _check(lib().hnv_level_feature_dim(g, level, ctypes.byref(k)), "hnv_level_feature_dim")
    n, m, nnz = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check(lib().hnv_level_info(g, level, ctypes.byref(n), ctypes.byref(m), ctypes.byref(nnz)),
           "hnv_level_info")
    out = np.empty((n.value, max(k.value, 1)), dtype=np.float32)
    _check(lib().hnv_copy_level_features(g, level, out.ctypes.data, out.nbytes, 0,
                                         _stream_handle(stream)), "hnv_copy_level_features")
    return out


def hnv_project(g: int, fine_level: int, zc_v, zc_e, zf_v, zf_e, stream=None):
    dt, tdt = _emb_dtype(zf_v)
    d = zf_v.shape[1]
    _check(lib().hnv_project(g, fine_level, _dev_ptr(zc_v, tdt, "zc_v"),
                             _dev_ptr(zc_e, tdt, "zc_e"), _dev_ptr(zf_v, tdt, "zf_v"),
                             _dev_ptr(zf_e, tdt, "zf_e"), dt, int(d),
                             _stream_handle(stream)), "hnv_project")


def hnv_refine(g: int, level: int, z_v, z_e, omega: float = 0.5, sweeps: int = 10,
               mode: int = SWEEP_TWO_PHASE, stream=None):
    dt, tdt = _emb_dtype(z_v)
    d = z_v.shape[1]
    _check(lib().hnv_refine(g, level, _dev_ptr(z_v, tdt, "z_v"), _dev_ptr(z_e, tdt, "z_e"), dt,
                            int(d), float(omega), int(sweeps), int(mode),
                            _stream_handle(stream)), "hnv_refine")


def hnv_refine_noalloc(g: int, level: int, z_v, z_e, omega: float = 0.5, sweeps: int = 10,
                       stream=None):
    """Two-phase refinement that allocates no device memory (fixed scratch
    inside the library; see include/hnv.h)."""
    import torch
    d = z_v.shape[1]
    _check(lib().hnv_refine_noalloc(g, level, _dev_ptr(z_v, torch.float32, "z_v"),
                                    _dev_ptr(z_e, torch.float32, "z_e"), F32, int(d),
                                    float(omega), int(sweeps), _stream_handle(stream)),
           "hnv_refine_noalloc")


def hnv_refine_until(g: int, level: int, z_v, z_e, omega: float = 0.5, max_sweeps: int = 80,
                     eps: float = 1e-4, mode: int = SWEEP_TWO_PHASE, stream=None):
    """Sweeps until one changes no coordinate by more than eps (or
    max_sweeps). Returns (sweeps_done, last_difference)."""
    dt, tdt = _emb_dtype(z_v)
    d = z_v.shape[1]
    done, delta = ctypes.c_int32(), ctypes.c_float()
    _check(lib().hnv_refine_until(g, level, _dev_ptr(z_v, tdt, "z_v"), _dev_ptr(z_e, tdt, "z_e"),
                                  dt, int(d), float(omega), int(max_sweeps), float(eps), int(mode),
                                  ctypes.byref(done), ctypes.byref(delta),
                                  _stream_handle(stream)), "hnv_refine_until")
    return done.value, delta.value


def hnv_vcycle(g: int, z_coarsest, z_v_out, z_e_out, omega: float = 0.5, sweeps: int = 10,
               mode: int = SWEEP_TWO_PHASE, stream=None):
    """Buffers are CUDA tensors (asynchronous), or host buffers: numpy
    float32 arrays or CPU tensors (float32 or bfloat16; the call copies in and
    out and synchronises)."""
    import torch
    if isinstance(z_coarsest, torch.Tensor):
        dt, tdt = _emb_dtype(z_coarsest)
        d = z_coarsest.shape[1]
        if z_coarsest.is_cuda:
            args = (_dev_ptr(z_coarsest, tdt, "z_coarsest"), _dev_ptr(z_v_out, tdt, "z_v_out"),
                    _dev_ptr(z_e_out, tdt, "z_e_out"))
            on_dev = 1
        else:
            for a, nm in ((z_coarsest, "z_coarsest"), (z_v_out, "z_v_out"), (z_e_out, "z_e_out")):
                if a.is_cuda or a.dtype != tdt or not a.is_contiguous():
                    raise TypeError("%s must be a contiguous CPU %s tensor" % (nm, tdt))
            args = (z_coarsest.data_ptr(), z_v_out.data_ptr(), z_e_out.data_ptr())
            on_dev = 0
    else:
        for a, nm in ((z_coarsest, "z_coarsest"), (z_v_out, "z_v_out"), (z_e_out, "z_e_out")):
            if a.dtype != np.float32 or not a.flags.c_contiguous:
                raise TypeError("%s must be a C-contiguous float32 array" % nm)
        dt = F32
        d = z_coarsest.shape[1]
        args = (z_coarsest.ctypes.data, z_v_out.ctypes.data, z_e_out.ctypes.data)
        on_dev = 0
    _check(lib().hnv_vcycle(g, *args, dt, int(d), float(omega), int(sweeps), int(mode), on_dev,
                            _stream_handle(stream)), "hnv_vcycle")


def hnv_set_weights(g: int, w0, stream=None):
    """Level-0 hyperedge weights (numpy float32 or a float32 tensor, host or
    device) for every level of the hierarchy."""
    import torch
    if isinstance(w0, torch.Tensor):
        t = w0.detach().contiguous().float()
        on_dev = 1 if t.is_cuda else 0
        _check(lib().hnv_set_weights(g, t.data_ptr(), on_dev, _stream_handle(stream)),
               "hnv_set_weights")
    else:
        a = np.ascontiguousarray(w0, dtype=np.float32)
        _check(lib().hnv_set_weights(g, a.ctypes.data, 0, _stream_handle(stream)),
               "hnv_set_weights")


def hnv_checkpoint_floats(g: int, d: int) -> int:
    out = ctypes.c_int64()
    _check(lib().hnv_checkpoint_floats(g, int(d), ctypes.byref(out)), "hnv_checkpoint_floats")
    return out.value


def hnv_vcycle_save(g: int, z_coarsest, z_v_out, z_e_out, checkpoints, omega: float = 0.5,
                    sweeps: int = 10, stream=None):
    import torch
    d = z_coarsest.shape[1]
    _check(lib().hnv_vcycle_save(g, _dev_ptr(z_coarsest, torch.float32, "z_coarsest"),
                                 _dev_ptr(z_v_out, torch.float32, "z_v_out"),
                                 _dev_ptr(z_e_out, torch.float32, "z_e_out"), int(d),
                                 float(omega), int(sweeps),
                                 _dev_ptr(checkpoints, torch.float32, "checkpoints"),
                                 _stream_handle(stream)), "hnv_vcycle_save")


def hnv_vcycle_backward(g: int, checkpoints, g_v0, g_e0, grad_w0, grad_z_coarsest,
                        omega: float = 0.5, sweeps: int = 10, stream=None):
    import torch
    d = grad_z_coarsest.shape[1]
    gv = _dev_ptr(g_v0, torch.float32, "g_v0") if g_v0 is not None else None
    ge = _dev_ptr(g_e0, torch.float32, "g_e0") if g_e0 is not None else None
    _check(lib().hnv_vcycle_backward(g, _dev_ptr(checkpoints, torch.float32, "checkpoints"), gv,
                                     ge, _dev_ptr(grad_w0, torch.float32, "grad_w0"),
                                     _dev_ptr(grad_z_coarsest, torch.float32, "grad_z_coarsest"),
                                     int(d), float(omega), int(sweeps), _stream_handle(stream)),
           "hnv_vcycle_backward")


def _autograd_function():
    import torch

    class VCycleFunction(torch.autograd.Function):
        """(w0, Z^L) -> (Z_V^0, Z_E^0) through the two-phase float32 V-cycle;
        backward runs the library's adjoint (per-level checkpoints, sweeps
        recomputed)."""

        @staticmethod
        def forward(ctx, w0, z_coarsest, graph, omega, sweeps):
            w = w0.detach().contiguous().float()
            zc = z_coarsest.detach().contiguous().float()
            graph.set_weights(w)
            n0, m0, _ = graph.level_info(0)
            d = zc.shape[1]
            ckpt = torch.empty(hnv_checkpoint_floats(graph.handle, d), device=zc.device)
            zv = torch.empty((n0, d), device=zc.device)
            ze = torch.empty((m0, d), device=zc.device)
            hnv_vcycle_save(graph.handle, zc, zv, ze, ckpt, omega, sweeps, graph.stream)
            ctx.graph, ctx.ckpt, ctx.w = graph, ckpt, w
            ctx.omega, ctx.sweeps, ctx.zc_shape = omega, sweeps, tuple(zc.shape)
            return zv, ze

        @staticmethod
        def backward(ctx, g_v, g_e):
            graph = ctx.graph
            graph.set_weights(ctx.w)      # the weights of the forward call
            dev = ctx.ckpt.device
            m0 = ctx.w.shape[0]
            gw = torch.empty(m0, device=dev)
            gz = torch.empty(ctx.zc_shape, device=dev)
            hnv_vcycle_backward(graph.handle, ctx.ckpt,
                                g_v.contiguous().float() if g_v is not None else None,
                                g_e.contiguous().float() if g_e is not None else None,
                                gw, gz, ctx.omega, ctx.sweeps, graph.stream)
            return gw, gz, None, None, None

    return VCycleFunction


_VCYCLE_FN = None


def vcycle_autograd(graph, w0, z_coarsest, omega: float = 0.5, sweeps: int = 10):
    """Differentiable V-cycle: returns (Z_V^0, Z_E^0); gradients flow to the
    level-0 hyperedge weights w0 and the coarsest rows z_coarsest."""
    global _VCYCLE_FN
    if _VCYCLE_FN is None:
        _VCYCLE_FN = _autograd_function()
    return _VCYCLE_FN.apply(w0, z_coarsest, graph, float(omega), int(sweeps))


def kernel_launch_count() -> int:
    return int(lib().hnv_kernel_launch_count())


def timing_enable(on: bool = True):
    _check(lib().hnv_timing_enable(1 if on else 0), "hnv_timing_enable")


def timing_reset():
    _check(lib().hnv_timing_reset(), "hnv_timing_reset")


def timing_read(phase: int) -> Tuple[float, int, float]:
    """(total ms, launches, algorithmic bytes) recorded for one phase."""
    ms = ctypes.c_double()
    cnt = ctypes.c_int64()
    by = ctypes.c_double()
    _check(lib().hnv_timing_read(phase, ctypes.byref(ms), ctypes.byref(cnt), ctypes.byref(by)),
           "hnv_timing_read")
    return ms.value, cnt.value, by.value


# ---------------------------------------------------------------------------
# Convenience wrapper
# ---------------------------------------------------------------------------

class Graph:
    """An owned hierarchy (``hnv_graph``) built from a hypergraph."""

    def __init__(self, n: int, m: int, edge_ptr, edge_nodes, edge_w=None, stream=None):
        import torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.handle = hnv_build_incidence(n, m, edge_ptr, edge_nodes, edge_w, self.stream)

    @classmethod
    def from_hypergraph(cls, hg, on_device: bool = False, stream=None) -> "Graph":
        if on_device:
            import torch
            return cls(hg.n, hg.m, torch.from_numpy(hg.edge_ptr).cuda(),
                       torch.from_numpy(hg.edge_nodes).cuda(),
                       torch.from_numpy(hg.weights).cuda(), stream)
        return cls(hg.n, hg.m, hg.edge_ptr, hg.edge_nodes, hg.weights, stream)

    def close(self):
        if getattr(self, "handle", None):
            lib().hnv_graph_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def sync_status(self):
        """Synchronise the graph's stream and raise if a device-side wait of
        an asynchronous call gave up (HNV_ERR_TIMEOUT)."""
        _check(lib().hnv_sync_status(self.handle, _stream_handle(self.stream)), "hnv_sync_status")

    def set_weights(self, w0):
        hnv_set_weights(self.handle, w0, self.stream)

    def set_node_features(self, x):
        hnv_set_node_features(self.handle, x, self.stream)

    def level_features(self, level: int) -> np.ndarray:
        return hnv_copy_level_features(self.handle, level, self.stream)

    def coarsen(self, **kw) -> int:
        return hnv_coarsen(self.handle, **kw)

    @property
    def num_levels(self) -> int:
        out = ctypes.c_int32()
        _check(lib().hnv_num_levels(self.handle, ctypes.byref(out)), "hnv_num_levels")
        return out.value

    def level_info(self, level: int) -> Tuple[int, int, int]:
        n, m, nnz = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        _check(lib().hnv_level_info(self.handle, level, ctypes.byref(n), ctypes.byref(m),
                                    ctypes.byref(nnz)), "hnv_level_info")
        return n.value, m.value, nnz.value

    def level_array(self, level: int, which: int) -> np.ndarray:
        """Host copy of one array of a level."""
        n, m, nnz = self.level_info(level)
        count = {ARR_E_PTR: m + 1, ARR_E_NODES: nnz, ARR_V_PTR: n + 1, ARR_V_EDGES: nnz,
                 ARR_W: m, ARR_REP_V: n, ARR_REP_E: m, ARR_DEG_V: n}[which]
        dt = np.float32 if which in (ARR_W, ARR_DEG_V) else np.int32
        out = np.empty(count, dtype=dt)
        _check(lib().hnv_copy_level_array(self.handle, level, which,
                                          out.ctypes.data if count else None, out.nbytes, 0,
                                          _stream_handle(self.stream)),
               "hnv_copy_level_array")
        return out

    def refine(self, level: int, z_v, z_e, omega=0.5, sweeps=10, mode=SWEEP_TWO_PHASE):
        hnv_refine(self.handle, level, z_v, z_e, omega, sweeps, mode, self.stream)

    def refine_until(self, level: int, z_v, z_e, omega=0.5, max_sweeps=80, eps=1e-4,
                     mode=SWEEP_TWO_PHASE):
        return hnv_refine_until(self.handle, level, z_v, z_e, omega, max_sweeps, eps, mode,
                                self.stream)

    def project(self, fine_level: int, zc_v, zc_e, zf_v, zf_e):
        hnv_project(self.handle, fine_level, zc_v, zc_e, zf_v, zf_e, self.stream)

    def vcycle(self, z_coarsest, z_v_out, z_e_out, omega=0.5, sweeps=10, mode=SWEEP_TWO_PHASE):
        hnv_vcycle(self.handle, z_coarsest, z_v_out, z_e_out, omega, sweeps, mode, self.stream)


class Batch:
    """Many hypergraphs refined together (hnv_batch_*): one launch per row
    class (or one persistent launch) per half-sweep covers every graph, the
    V-cycle is captured into a CUDA graph. The graphs must stay alive while
    the batch is used."""

    def __init__(self, graphs):
        self.graphs = list(graphs)
        arr = (_P * len(self.graphs))(*[g.handle for g in self.graphs])
        out = _P()
        _check(lib().hnv_batch_create(arr, len(self.graphs), ctypes.byref(out)), "hnv_batch_create")
        self.handle = out.value
        self.stream = self.graphs[0].stream
        self._rows = tuple(int(a[-1]) for a in self.offsets())

    def offsets(self):
        """(coarsest, node, hyperedge) row offsets, each count + 1 int64."""
        k = len(self.graphs) + 1
        a, b, c = (np.empty(k, np.int64) for _ in range(3))
        _check(lib().hnv_batch_offsets(self.handle, a.ctypes.data, b.ctypes.data, c.ctypes.data),
               "hnv_batch_offsets")
        return a, b, c

    def autotune(self, dtype: int, d: int, omega: float = 0.5) -> dict:
        t = BatchTuning()
        _check(lib().hnv_batch_autotune(self.handle, dtype, int(d), float(omega), ctypes.byref(t)),
               "hnv_batch_autotune")
        return {f: getattr(t, f) for f, _ in BatchTuning._fields_}

    @property
    def kernel(self) -> int:
        """The half-sweep kernel (BATCH_KERNEL_PER_CLASS or BATCH_KERNEL_PERSISTENT)."""
        k = lib().hnv_batch_get_kernel(self.handle)
        _check(min(k, 0), "hnv_batch_get_kernel")
        return k

    @kernel.setter
    def kernel(self, k: int):
        _check(lib().hnv_batch_set_kernel(self.handle, int(k)), "hnv_batch_set_kernel")

    def vcycle(self, z_coarsest, z_v_out, z_e_out, omega=0.5, sweeps=10, use_cuda_graph=True):
        dt, tdt = _emb_dtype(z_coarsest)
        d = z_coarsest.shape[1]
        rc, rv, re = self._rows
        _check(lib().hnv_batch_vcycle(self.handle, _dev_ptr(z_coarsest, tdt, "z_coarsest", rc, d),
                                      _dev_ptr(z_v_out, tdt, "z_v_out", rv, d),
                                      _dev_ptr(z_e_out, tdt, "z_e_out", re, d), dt, int(d), float(omega),
                                      int(sweeps), 1 if use_cuda_graph else 0,
                                      _stream_handle(self.stream)), "hnv_batch_vcycle")

    def close(self):
        if getattr(self, "handle", None):
            lib().hnv_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
