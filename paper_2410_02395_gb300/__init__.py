"""GB300-native modified Born series (MBS) solver with block domain decomposition.

Thin ctypes binding over the C ABI in ``include/mbs.h`` (argument marshalling
only: every step of the method runs in the library's CUDA kernels). Arrays are
complex64 in C order, shape (n0, n1, n2), axis 0 slowest. Inputs may be torch
tensors (CUDA or CPU) or numpy arrays; host data is copied by the library.

There is no CPU fallback: if the compiled library is missing the import of
``Plan`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

__all__ = ["Plan", "Batch", "MBSError", "load_library", "OP", "STATUS", "build"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_lib", "libmbs_gb300.so")

STATUS = {0: "MBS_OK", 1: "MBS_EINVAL", 2: "MBS_ENOMEM", 3: "MBS_ECUDA", 4: "MBS_ENOCONV", 5: "MBS_ENAN",
          6: "MBS_EDIVERGE", 7: "MBS_ETIMEOUT", 8: "MBS_EUNSUPPORTED"}
OP = {"A": 0, "PRECOND": 1, "V": 2, "L": 3, "PROPAGATE": 4, "E": 5, "FFT": 6, "IFFT": 7}
MAX_SPLIT = 16
KERNEL_KINDS = 8


class MBSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class _Options(C.Structure):
    _fields_ = [("truncation", C.c_int32), ("alpha", C.c_double), ("periodic_mask", C.c_uint32),
                ("absorb_kappa", C.c_double), ("split_sizes", C.POINTER(C.c_int64)), ("flags", C.c_uint32),
                ("graph_iters", C.c_int32), ("stream", C.c_void_p), ("workspace", C.c_void_p),
                ("workspace_bytes", C.c_size_t), ("tma_wait_cycles", C.c_int64),
                ("activation_threshold", C.c_double)]


class _Info(C.Structure):
    _fields_ = [("c_re", C.c_double), ("c_im", C.c_double), ("k0sq_re", C.c_double), ("k0sq_im", C.c_double),
                ("contrast", C.c_double), ("block_norm", C.c_double), ("a", C.c_int32 * 3), ("t", C.c_int32),
                ("alpha", C.c_double), ("shape", C.c_int64 * 3), ("split", C.c_int32 * 3),
                ("sizes", (C.c_int64 * MAX_SPLIT) * 3), ("device_bytes", C.c_size_t), ("graph_iters", C.c_int32),
                ("tma_groups", C.c_int32), ("tune_source", C.c_int32), ("tuning", C.c_char * 256)]


_lib = None


def build(verbose=False, bounds_check=False):
    """Compile the CUDA library in-tree (nvcc, sm_103a); bounds_check=True builds the
    index-checking variant (``mbs_build_checks_bounds``) beside it."""
    from . import _build

    return _build.build(verbose=verbose, bounds_check=bounds_check)


CHECKED_LIB_PATH = os.path.join(_HERE, "_lib", "libmbs_gb300_checked.so")


def load_library(path=None):
    """Load the compiled library (no fallback when it is missing)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _LIB_PATH
    if not os.path.exists(p):
        raise ImportError("libmbs_gb300.so not built (run paper_2410_02395_gb300.build()): %s" % p)
    lib = C.CDLL(p)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    lib.mbs_default_options.argtypes = [C.POINTER(_Options)]
    lib.mbs_default_options.restype = None
    lib.mbs_plan_create.argtypes = [C.POINTER(vp), C.POINTER(i64), dbl, dbl, vp, C.POINTER(i32), C.POINTER(i32),
                                    C.POINTER(_Options)]
    lib.mbs_workspace_bytes.argtypes = [C.POINTER(i64), C.POINTER(i32), C.POINTER(_Options), C.POINTER(C.c_size_t)]
    lib.mbs_plan_get_info.argtypes = [vp, C.POINTER(_Info)]
    lib.mbs_apply_operator.argtypes = [vp, i32, vp, vp]
    lib.mbs_set_source.argtypes = [vp, vp]
    lib.mbs_set_initial_field.argtypes = [vp, vp]
    lib.mbs_iterate.argtypes = [vp, i32, dbl, i32, C.POINTER(i32), C.POINTER(dbl)]
    lib.mbs_get_field.argtypes = [vp, vp]
    lib.mbs_get_active_subdomains.argtypes = [vp, C.POINTER(i32), i32, C.POINTER(i32)]
    lib.mbs_get_history.argtypes = [vp, C.POINTER(dbl), i32, C.POINTER(i32)]
    lib.mbs_solve.argtypes = [vp, vp, vp, dbl, i32, C.POINTER(i32), C.POINTER(dbl), C.POINTER(dbl)]
    lib.mbs_profile_iterations.argtypes = [vp, i32, C.POINTER(i32), C.POINTER(dbl)]
    lib.mbs_kernel_kind_name.argtypes = [i32]
    lib.mbs_kernel_kind_name.restype = C.c_char_p
    lib.mbs_batch_create.argtypes = [C.POINTER(vp), i32, C.POINTER(vp), vp, i32]
    lib.mbs_batch_iterate.argtypes = [vp, i32, dbl, i32, C.POINTER(i32), C.POINTER(dbl), C.POINTER(i32)]
    lib.mbs_batch_launches_per_iteration.argtypes = [vp, C.POINTER(i32)]
    lib.mbs_batch_set_fused.argtypes = [vp, i32]
    lib.mbs_batch_set_fused.restype = C.c_int
    lib.mbs_batch_launches_per_iteration.restype = C.c_int32
    lib.mbs_batch_destroy.argtypes = [vp]
    lib.mbs_batch_destroy.restype = None
    lib.mbs_plan_destroy.argtypes = [vp]
    lib.mbs_plan_destroy.restype = None
    lib.mbs_last_error.argtypes = []
    lib.mbs_last_error.restype = C.c_char_p
    lib.mbs_build_checks_bounds.argtypes = []
    lib.mbs_build_checks_bounds.restype = C.c_int32
    for name in ("mbs_plan_create", "mbs_workspace_bytes", "mbs_plan_get_info", "mbs_apply_operator",
                 "mbs_set_source", "mbs_set_initial_field", "mbs_get_active_subdomains", "mbs_iterate", "mbs_get_field", "mbs_get_history", "mbs_solve",
                 "mbs_profile_iterations", "mbs_batch_create", "mbs_batch_iterate"):
        getattr(lib, name).restype = C.c_int
    if path is None:
        _lib = lib
    return lib


def _check(lib, status, ok=(0,)):
    if status not in ok:
        raise MBSError(status, lib.mbs_last_error().decode())
    return status


class _Buf:
    """A pointer to complex64 C-ordered data, keeping its owner alive.

    The library reads and writes device data on the plan's own stream. For a CUDA
    tensor, torch's current stream on its device is synchronised first, so that
    work torch has queued on that tensor (its initialisation, say) is complete
    before the library's stream reads it."""

    def __init__(self, arr, shape, writable=False):
        self.owner = None
        self.torch_out = None
        try:
            import torch
        except ImportError:  # pragma: no cover - torch is part of the environment
            torch = None
        if torch is not None and isinstance(arr, torch.Tensor):
            if arr.dtype != torch.complex64:
                if writable:
                    raise TypeError("output tensor must be complex64")
                arr = arr.to(torch.complex64)
            if tuple(arr.shape) != tuple(shape):
                raise ValueError("array shape %s != grid %s" % (tuple(arr.shape), tuple(shape)))
            if not arr.is_contiguous():
                if writable:
                    raise ValueError("output tensor must be contiguous")
                arr = arr.contiguous()
            if arr.is_cuda:
                torch.cuda.current_stream(arr.device).synchronize()
            self.owner = arr
            self.ptr = arr.data_ptr()
            return
        a = np.asarray(arr)
        if tuple(a.shape) != tuple(shape):
            raise ValueError("array shape %s != grid %s" % (a.shape, tuple(shape)))
        if writable:
            if a.dtype != np.complex64 or not a.flags.c_contiguous or not a.flags.writeable:
                raise TypeError("output array must be a writable C-contiguous complex64 array")
        else:
            a = np.ascontiguousarray(a, dtype=np.complex64)
        self.owner = a
        self.ptr = a.ctypes.data


class Plan:
    """An MBS problem on one GPU (see ``mbs_plan_create`` in include/mbs.h).

    Parameters follow the paper's statement of the problem: grid shape, pixel
    size, wavelength, refractive index n(r), absorbing boundary widths and the
    subdomain split.
    """

    def __init__(self, shape, pixel_size, wavelength, refractive_index, boundary_widths=((0, 0),) * 3,
                 split=(1, 1, 1), truncation=8, alpha=0.75, periodic=(False, False, False), kappa=0.5,
                 split_sizes=None, graph_iters=0, no_graph=False, corr_tf32=False, residual_form=False,
                 no_tma=False, force_tma=False, plain_steps=False, activation=False, activation_threshold=0.0,
                 no_tune=False,
                 tma_wait_cycles=0, stream=None, workspace=None, library=None):
        self.lib = library if library is not None else load_library()
        self.shape = tuple(int(s) for s in shape)
        opts = _Options()
        self.lib.mbs_default_options(C.byref(opts))
        opts.truncation = -1 if int(truncation) == 0 else int(truncation)  # t = 0: MBS_T_NONE
        opts.alpha = float(alpha)
        opts.periodic_mask = sum((1 << d) for d in range(3) if periodic[d])
        opts.absorb_kappa = float(kappa)
        opts.graph_iters = int(graph_iters)
        opts.flags = (1 if no_graph else 0) | (2 if corr_tf32 else 0) | (4 if residual_form else 0) | \
            (8 if no_tma else 0) | (16 if force_tma else 0) | (32 if plain_steps else 0) | (64 if activation else 0) | \
            (128 if no_tune else 0)
        opts.tma_wait_cycles = int(tma_wait_cycles)
        opts.activation_threshold = float(activation_threshold)
        self._split_sizes = None
        if split_sizes is not None:
            flat = [int(v) for d in range(3) for v in split_sizes[d]]
            self._split_sizes = (C.c_int64 * len(flat))(*flat)
            opts.split_sizes = C.cast(self._split_sizes, C.POINTER(C.c_int64))
        if stream is not None:
            opts.stream = C.c_void_p(int(stream))
        self._workspace = workspace
        if workspace is not None:
            opts.workspace = C.c_void_p(workspace.data_ptr())
            opts.workspace_bytes = workspace.numel() * workspace.element_size()
        self._opts = opts
        w = [int(v) for pair in boundary_widths for v in pair]
        n = _Buf(refractive_index, self.shape)
        handle = C.c_void_p()
        st = self.lib.mbs_plan_create(C.byref(handle), (C.c_int64 * 3)(*self.shape), float(pixel_size),
                                      float(wavelength), C.c_void_p(n.ptr), (C.c_int32 * 6)(*w),
                                      (C.c_int32 * 3)(*[int(s) for s in split]), C.byref(opts))
        _check(self.lib, st)
        self.handle = handle

    # -- information ---------------------------------------------------------
    def info(self):
        inf = _Info()
        _check(self.lib, self.lib.mbs_plan_get_info(self.handle, C.byref(inf)))
        return dict(c=complex(inf.c_re, inf.c_im), k0sq=complex(inf.k0sq_re, inf.k0sq_im), contrast=inf.contrast,
                    block_norm=inf.block_norm, a=list(inf.a), t=inf.t, alpha=inf.alpha, shape=tuple(inf.shape),
                    split=tuple(inf.split),
                    sizes=[list(inf.sizes[d][:inf.split[d]]) for d in range(3)], device_bytes=inf.device_bytes,
                    graph_iters=inf.graph_iters, tma_groups=inf.tma_groups, tune_source=inf.tune_source,
                    tuning=inf.tuning.decode())

    @staticmethod
    def workspace_bytes(shape, split, truncation=8, split_sizes=None, residual_form=False):
        lib = load_library()
        opts = _Options()
        lib.mbs_default_options(C.byref(opts))
        opts.truncation = -1 if int(truncation) == 0 else int(truncation)  # t = 0: MBS_T_NONE
        opts.flags = 4 if residual_form else 0
        keep = None
        if split_sizes is not None:
            flat = [int(v) for d in range(3) for v in split_sizes[d]]
            keep = (C.c_int64 * len(flat))(*flat)
            opts.split_sizes = C.cast(keep, C.POINTER(C.c_int64))
        out = C.c_size_t()
        _check(lib, lib.mbs_workspace_bytes((C.c_int64 * 3)(*shape), (C.c_int32 * 3)(*split), C.byref(opts),
                                            C.byref(out)))
        return out.value

    # -- operators ---------------------------------------------------------------
    def _out(self, out, like):
        if out is not None:
            return out
        try:
            import torch

            if isinstance(like, torch.Tensor):
                return torch.empty(self.shape, dtype=torch.complex64, device=like.device)
        except ImportError:  # pragma: no cover
            pass
        return np.empty(self.shape, dtype=np.complex64)

    def apply(self, which, x, out=None):
        """out = op(x) for op in 'A', 'PRECOND', 'V', 'L', 'PROPAGATE', 'E', 'FFT', 'IFFT'."""
        xb = _Buf(x, self.shape)
        out = self._out(out, x)
        ob = _Buf(out, self.shape, writable=True)
        _check(self.lib, self.lib.mbs_apply_operator(self.handle, OP[which] if isinstance(which, str) else int(which),
                                                     C.c_void_p(xb.ptr), C.c_void_p(ob.ptr)))
        return out

    # -- solving -----------------------------------------------------------------
    def set_source(self, source):
        sb = _Buf(source, self.shape)
        _check(self.lib, self.lib.mbs_set_source(self.handle, C.c_void_p(sb.ptr)))

    def set_initial_field(self, x0):
        """Warm start from x0 after set_source (eps stays normalised by the residual of x = 0)."""
        xb = _Buf(x0, self.shape)
        _check(self.lib, self.lib.mbs_set_initial_field(self.handle, C.c_void_p(xb.ptr)))

    def iterate(self, n_iter, tol=0.0, no_poll=False):
        """Run up to n_iter iterations; returns (status_name, iterations, residual)."""
        it = C.c_int32()
        res = C.c_double()
        st = self.lib.mbs_iterate(self.handle, int(n_iter), float(tol), 1 if no_poll else 0, C.byref(it),
                                  C.byref(res))
        _check(self.lib, st, ok=(0, 4))
        return STATUS[st], it.value, res.value

    def active_subdomains(self):
        """Activation flags of the subdomains, shape split (all 1 without activation)."""
        sp = self.info()["split"]
        nsub = sp[0] * sp[1] * sp[2]
        flags = (C.c_int32 * nsub)()
        na = C.c_int32()
        _check(self.lib, self.lib.mbs_get_active_subdomains(self.handle, flags, nsub, C.byref(na)))
        return np.array(flags[:], dtype=np.int32).reshape(sp)

    def field(self, out=None, like=None):
        out = self._out(out, like)
        ob = _Buf(out, self.shape, writable=True)
        _check(self.lib, self.lib.mbs_get_field(self.handle, C.c_void_p(ob.ptr)))
        return out

    def history(self, cap=1 << 16):
        h = (C.c_double * cap)()
        n = C.c_int32()
        _check(self.lib, self.lib.mbs_get_history(self.handle, h, cap, C.byref(n)))
        return np.array(h[:n.value])

    def solve(self, source, tol=1e-6, max_iter=10000, out=None, with_history=False):
        """Full solve from x = 0 (Eq. wavesim_iter); returns (field, iterations, residual[, history])."""
        sb = _Buf(source, self.shape)
        out = self._out(out, source)
        ob = _Buf(out, self.shape, writable=True)
        it = C.c_int32()
        res = C.c_double()
        hist = (C.c_double * max(1, max_iter))() if with_history else None
        st = self.lib.mbs_solve(self.handle, C.c_void_p(sb.ptr), C.c_void_p(ob.ptr), float(tol), int(max_iter),
                                C.byref(it), C.byref(res), hist)
        _check(self.lib, st, ok=(0, 4))
        if with_history:
            return out, it.value, res.value, np.array(hist[:it.value])
        return out, it.value, res.value

    def profile(self, n_iter):
        """Per-kernel-kind launches and device milliseconds over n_iter iterations."""
        launches = (C.c_int32 * KERNEL_KINDS)()
        ms = (C.c_double * KERNEL_KINDS)()
        _check(self.lib, self.lib.mbs_profile_iterations(self.handle, int(n_iter), launches, ms))
        return {self.lib.mbs_kernel_kind_name(k).decode(): (launches[k], ms[k]) for k in range(KERNEL_KINDS)}

    def close(self):
        if getattr(self, "handle", None):
            self.lib.mbs_plan_destroy(self.handle)
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


class Batch:
    """Several plans advanced together (``mbs_batch_*`` in include/mbs.h)."""

    def __init__(self, plans, stream=None, graph_iters=0, fused=None):
        self.lib = load_library()
        self.plans = list(plans)
        arr = (C.c_void_p * len(self.plans))(*[p.handle for p in self.plans])
        h = C.c_void_p()
        _check(self.lib, self.lib.mbs_batch_create(C.byref(h), len(self.plans), arr,
                                                   C.c_void_p(int(stream)) if stream is not None else None,
                                                   int(graph_iters)))
        self.handle = h
        if fused is not None:
            _check(self.lib, self.lib.mbs_batch_set_fused(self.handle, 1 if fused else 0))

    def iterate(self, n_iter, tol=0.0, no_poll=False):
        """Returns a list of (status_name, iterations, residual), one per plan."""
        n = len(self.plans)
        it = (C.c_int32 * n)()
        res = (C.c_double * n)()
        sts = (C.c_int32 * n)()
        _check(self.lib, self.lib.mbs_batch_iterate(self.handle, int(n_iter), float(tol), 1 if no_poll else 0,
                                                    it, res, sts), ok=(0, 4))
        return [(STATUS[sts[i]], it[i], res[i]) for i in range(n)]

    def set_fused(self, on):
        """Run as one launch per pass and edge over all plans (on) or as a graph of every plan's own launches."""
        _check(self.lib, self.lib.mbs_batch_set_fused(self.handle, 1 if on else 0))

    def launches_per_iteration(self):
        """(kernel launches per iteration of the whole batch, fused form or not)."""
        fused = C.c_int32()
        n = self.lib.mbs_batch_launches_per_iteration(self.handle, C.byref(fused))
        if n < 0:
            raise MBSError(3, self.lib.mbs_last_error().decode())
        return n, bool(fused.value)

    def close(self):
        if getattr(self, "handle", None):
            self.lib.mbs_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

