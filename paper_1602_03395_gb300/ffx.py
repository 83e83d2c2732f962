"""Thin Python binding of libffx (include/ffx.h): argument marshalling only.

Every step of the expansion runs in the library's CUDA kernels; this module
passes device pointers of PyTorch tensors and the current CUDA stream through
ctypes.  It fails loudly if the library is missing: there is no fallback.

The names follow the C ABI (``ffx_plan``, ``ffx_expand``, ``ffx_expand_field``,
``ffx_expand_backward``, ``ffx_expand_adjoint``, ``ffx_plan_destroy``).
``Plan`` wraps a plan handle; ``expand_density`` is a differentiable
``torch.autograd.Function`` front end whose backward is the library's
hand-written adjoint.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libffx.so")

FFX_OK, FFX_EINVAL, FFX_ENOMEM, FFX_ECUDA, FFX_EUNSUPPORTED, FFX_ETIMEOUT = 0, 1, 2, 3, 4, 5
FFX_FORM_AUTO, FFX_FORM_PAPER, FFX_FORM_FOLD, FFX_FORM_DENSE, FFX_FORM_TC = 0x0, 0x1, 0x2, 0x3, 0x4
FFX_ACCUMULATE = 0x10
FFX_TUNE = 0x20
FFX_UNFUSED = 0x40
FFX_TC_UNSPLIT = 0x80
FFX_TC_BF16 = 0x100
FFX_TC_TF32 = 0x200

_FORMS = {"auto": FFX_FORM_AUTO, "paper": FFX_FORM_PAPER, "fold": FFX_FORM_FOLD, "dense": FFX_FORM_DENSE,
          "tc": FFX_FORM_TC}
_FORM_NAMES = {FFX_FORM_AUTO: "mixed", FFX_FORM_PAPER: "paper", FFX_FORM_FOLD: "fold", FFX_FORM_DENSE: "dense",
               FFX_FORM_TC: "tc"}

_lib = None


class InstanceDesc(ctypes.Structure):
    """ffx_instance_desc of include/ffx.h."""
    _fields_ = [("ndim", ctypes.c_int32), ("dims", ctypes.c_int64 * 3), ("spacing", ctypes.c_double * 3),
                ("t", ctypes.c_double), ("magnification", ctypes.c_int32 * 3),
                ("has_offsets", ctypes.c_int32), ("a", ctypes.c_double * 3), ("abar", ctypes.c_double * 3)]


class FfxError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {msg} (code {code})")
        self.code = code


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libffx.so (built by ``paper_1602_03395_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing; build it with "
                           "`python -m paper_1602_03395_gb300.build`")
    lib = ctypes.CDLL(path)
    vp, i64, i32, u32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint32, ctypes.c_double
    lib.ffx_plan.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(i64), ctypes.POINTER(dbl), dbl,
                             ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(dbl), ctypes.POINTER(dbl), u32]
    lib.ffx_plan.restype = i32
    lib.ffx_plan_dispersion.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(i64), ctypes.POINTER(dbl), dbl,
                                        ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(dbl), ctypes.POINTER(dbl),
                                        ctypes.POINTER(ctypes.POINTER(dbl)), u32]
    lib.ffx_plan_dispersion.restype = i32
    lib.ffx_plan_destroy.argtypes = [vp]
    lib.ffx_plan_destroy.restype = i32
    lib.ffx_expand.argtypes = [vp, vp, i64, vp, vp]
    lib.ffx_expand.restype = i32
    lib.ffx_expand_host.argtypes = [vp, vp, i64, vp, vp]
    lib.ffx_expand_host.restype = i32
    lib.ffx_expand_field.argtypes = [vp, vp, i64, vp, vp]
    lib.ffx_expand_field.restype = i32
    lib.ffx_expand_backward.argtypes = [vp, vp, vp, i64, vp, vp]
    lib.ffx_expand_backward.restype = i32
    lib.ffx_expand_adjoint.argtypes = [vp, vp, i64, vp, vp]
    lib.ffx_expand_adjoint.restype = i32
    lib.ffx_supported_length.argtypes = [i64]
    lib.ffx_supported_length.restype = i32
    lib.ffx_workspace_bytes.argtypes = [vp, i64]
    lib.ffx_workspace_bytes.restype = i64
    lib.ffx_plan_form.argtypes = [vp]
    lib.ffx_plan_form.restype = i32
    lib.ffx_plan_axis_form.argtypes = [vp, i32]
    lib.ffx_plan_axis_form.restype = i32
    lib.ffx_launches_per_call.argtypes = [vp, i32]
    lib.ffx_launches_per_call.restype = i32
    lib.ffx_plan_fused.argtypes = [vp]
    lib.ffx_plan_fused.restype = i64
    lib.ffx_plan_call_form.argtypes = [vp, i32, i64]
    lib.ffx_plan_call_form.restype = i32
    lib.ffx_plan_bf16_chain.argtypes = [vp, i64]
    lib.ffx_plan_bf16_chain.restype = i32
    lib.ffx_plan_launch_count.argtypes = [vp]
    lib.ffx_plan_launch_count.restype = i64
    lib.ffx_expand_positive_p.argtypes = [vp, vp, vp, i64, vp, vp]
    lib.ffx_expand_positive_p.restype = i32
    lib.ffx_expand_column.argtypes = [vp, vp, i64, i32, vp, vp]
    lib.ffx_expand_column.restype = i32
    lib.ffx_plan_output_axis.argtypes = [vp, i32, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
    lib.ffx_plan_output_axis.restype = i32
    lib.ffx_fringe_phase.argtypes = [vp, i64, i64, i64, i64, dbl, dbl, dbl, dbl, vp, vp]
    lib.ffx_fringe_phase.restype = i32
    lib.ffx_plan_pass_order.argtypes = [vp, ctypes.POINTER(ctypes.c_int32)]
    lib.ffx_plan_pass_order.restype = i32
    lib.ffx_plan_trace.argtypes = [vp, ctypes.POINTER(vp), i64]
    lib.ffx_plan_trace.restype = i32
    lib.ffx_plan_trace_count.argtypes = [vp]
    lib.ffx_plan_trace_count.restype = i64
    lib.ffx_plan_device_errors.argtypes = [vp]
    lib.ffx_plan_device_errors.restype = i32
    lib.ffx_plan_set_wait_limit.argtypes = [vp, i64]
    lib.ffx_plan_set_wait_limit.restype = i32
    lib.ffx_plan_tc_bf16.argtypes = [vp]
    lib.ffx_plan_tc_bf16.restype = i32
    lib.ffx_expand_noalloc.argtypes = [i32, ctypes.POINTER(i64), ctypes.POINTER(dbl), dbl,
                                       ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(dbl),
                                       ctypes.POINTER(dbl), vp, i64, vp, vp]
    lib.ffx_expand_noalloc.restype = i32
    lib.ffx_plan_many.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(InstanceDesc), u32]
    lib.ffx_plan_many.restype = i32
    lib.ffx_plan_many_offset.argtypes = [vp, i32]
    lib.ffx_plan_many_offset.restype = i64
    lib.ffx_plan_points.argtypes = [vp]
    lib.ffx_plan_points.restype = i64
    lib.ffx_error_string.argtypes = [i32]
    lib.ffx_error_string.restype = ctypes.c_char_p
    lib.ffx_last_error.argtypes = []
    lib.ffx_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(code: int, where: str):
    if code != FFX_OK:
        lib = load_library()
        raise FfxError(code, where, lib.ffx_last_error().decode() or lib.ffx_error_string(code).decode())


def _ptr(x: torch.Tensor | None):
    return None if x is None else ctypes.c_void_p(x.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _need(x: torch.Tensor, dtype, name: str):
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if x.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {x.dtype}")
    if not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def ffx_supported_length(n: int) -> bool:
    return bool(load_library().ffx_supported_length(int(n)))


def fine_wavevectors(N: int, dx: float, lam: int) -> np.ndarray:
    """The lam N huge-lattice wavevectors k_u = 2 pi u~ / (lam N dx), u~ the
    symmetric index of u (the sample points of a dispersion for ``omega=``)."""
    M = lam * N
    u = np.arange(M)
    return 2.0 * np.pi * np.where(2 * u < M, u, u - M) / (lam * N * dx)


class Plan:
    """A plan for one geometry (dims, spacing, t, magnification, offsets).

    ``unsplit=True`` (with ``form="tc"``) runs one TF32 product per K-step
    on rounded operands instead of the split products: faster, with a
    density error of order 1e-3 (FFX_TC_UNSPLIT).  ``bf16=True`` (automatic
    or tc form) gives the streaming tensor-core passes BF16 operands
    (FFX_TC_BF16): split into heads and tails, or unsplit with
    ``unsplit=True``; the automatic form takes split BF16 by default, and
    ``tf32=True`` keeps split TF32 operands there (FFX_TC_TF32)."""

    def __init__(self, dims, spacing, t, magnification, a=None, abar=None,
                 form: str = "auto", accumulate: bool = False, tune: bool = False, fused: bool = True,
                 omega=None, unsplit: bool = False, bf16: bool = False, tf32: bool = False):
        lib = load_library()
        d = len(dims)
        self.dims = tuple(int(v) for v in dims)
        self.spacing = tuple(float(v) for v in spacing)
        self.t = float(t)
        self.magnification = tuple(int(v) for v in magnification)
        self.accumulate = bool(accumulate)
        flags = (_FORMS[form] | (FFX_ACCUMULATE if accumulate else 0) | (FFX_TUNE if tune else 0)
                 | (0 if fused else FFX_UNFUSED) | (FFX_TC_UNSPLIT if unsplit else 0)
                 | (FFX_TC_BF16 if bf16 else 0) | (FFX_TC_TF32 if tf32 else 0))
        self.unsplit = bool(unsplit)
        arr = lambda ct, v: (ct * d)(*v) if v is not None else None  # noqa: E731
        h = ctypes.c_void_p()
        if omega is None:
            _check(lib.ffx_plan(ctypes.byref(h), d, arr(ctypes.c_int64, self.dims),
                                arr(ctypes.c_double, self.spacing), self.t,
                                arr(ctypes.c_int32, self.magnification),
                                arr(ctypes.c_double, a), arr(ctypes.c_double, abar), flags), "ffx_plan")
        else:
            # per axis None (free) or lam_j N_j values of omega_j at fine_wavevectors(...)
            if len(omega) != d:
                raise ValueError(f"omega needs {d} entries")
            keep = [None if w is None else np.ascontiguousarray(w, dtype=np.float64) for w in omega]
            ptrs = (ctypes.POINTER(ctypes.c_double) * d)()
            for j, w in enumerate(keep):
                if w is not None:
                    if w.shape != (self.magnification[j] * self.dims[j],):
                        raise ValueError(f"omega[{j}] must hold lam*N = {self.magnification[j] * self.dims[j]} values")
                    ptrs[j] = w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            _check(lib.ffx_plan_dispersion(ctypes.byref(h), d, arr(ctypes.c_int64, self.dims),
                                           arr(ctypes.c_double, self.spacing), self.t,
                                           arr(ctypes.c_int32, self.magnification),
                                           arr(ctypes.c_double, a), arr(ctypes.c_double, abar), ptrs, flags),
                   "ffx_plan_dispersion")
        self._h = h
        self.form = _FORM_NAMES[lib.ffx_plan_form(h)]
        self.axis_forms = tuple(_FORM_NAMES[lib.ffx_plan_axis_form(h, j)] for j in range(d))
        # largest batch whose forward calls run as one launch (0: never)
        self.fused_max_batch = int(lib.ffx_plan_fused(h))
        # BF16 operands on the streaming tensor-core passes (asked for, or the automatic default)
        self.bf16 = lib.ffx_plan_tc_bf16(h) == 1
        self.fused = self.fused_max_batch >= 1
        self.M = 1
        for v in self.dims:
            self.M *= v

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("plan destroyed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            load_library().ffx_plan_destroy(self._h)
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

    def _batch(self, x: torch.Tensor) -> int:
        if tuple(x.shape[x.dim() - len(self.dims):]) != self.dims:
            raise ValueError(f"trailing shape {tuple(x.shape)} does not match dims {self.dims}")
        return int(x.numel() // self.M)

    def workspace_bytes(self, batch: int) -> int:
        return int(load_library().ffx_workspace_bytes(self.handle, batch))

    def launches_per_call(self, backward: bool = False, batch: int = 1) -> int:
        """Passes a call makes (one launch for a fused call), plus the input
        split of a BF16 chain.  A per-axis BF16 pass over contiguous FP32
        lines adds its own split launch; launch_count() counts exactly."""
        n = len(self.dims)
        # a BF16 chain adds the split of its input (the forward half of a
        # backward call takes a chain except on 2-D plans, its adjoint half
        # always, with the split of its gradient factors)
        bf = self.bf16_chain(batch)
        chain = (1 if bf and (not backward or n != 2) else 0) + (1 if bf and backward else 0)
        if not backward and self.fused and batch > self.fused_max_batch:
            return n + chain
        return int(load_library().ffx_launches_per_call(self.handle, int(backward))) + chain

    def call_forms(self, batch: int = 1):
        """Per lattice axis, the form whose kernel a forward call with this batch runs."""
        return tuple(_FORM_NAMES[load_library().ffx_plan_call_form(self.handle, j, batch)]
                     for j in range(len(self.dims)))

    def launch_count(self) -> int:
        """Kernels this plan's calls have launched so far (captured calls
        count once; graph replays do not)."""
        return int(load_library().ffx_plan_launch_count(self.handle))

    def bf16_chain(self, batch: int = 1) -> bool:
        """Whether forward calls with this batch run as a BF16 chain (the
        passes from the last axis to the first, BF16 planes between them)."""
        return load_library().ffx_plan_bf16_chain(self.handle, batch) == 1

    def pass_order(self):
        order = (ctypes.c_int32 * len(self.dims))()
        _check(load_library().ffx_plan_pass_order(self.handle, order), "ffx_plan_pass_order")
        return tuple(order)

    def trace(self, events):
        """Record each kernel launch between a pair of the given
        torch.cuda.Event objects (enable_timing=True); None switches off."""
        lib = load_library()
        if not events:
            self._trace_arr = None
            _check(lib.ffx_plan_trace(self.handle, None, 0), "ffx_plan_trace")
            return
        for ev in events:  # make sure the CUDA events exist
            if ev.cuda_event == 0:
                ev.record()
        arr = (ctypes.c_void_p * len(events))(*[ev.cuda_event for ev in events])
        self._trace_arr = arr  # the library keeps the pointer
        _check(lib.ffx_plan_trace(self.handle, arr, len(events)), "ffx_plan_trace")

    def trace_count(self) -> int:
        return int(load_library().ffx_plan_trace_count(self.handle))

    def device_errors(self) -> int:
        """Bounded waits that ran out in this plan's kernels (0 when all is well)."""
        return int(load_library().ffx_plan_device_errors(self.handle))

    def set_wait_limit(self, polls: int):
        """Poll budget of the fused launch's waits on other blocks (0: default)."""
        _check(load_library().ffx_plan_set_wait_limit(self.handle, int(polls)), "ffx_plan_set_wait_limit")


class PlanMany(Plan):
    """A plan over many instances of (possibly) different lattices.

    ``instances``: sequence of (dims, spacing, t, magnification) or
    (dims, spacing, t, magnification, a, abar).  Inputs and outputs are packed
    1-D tensors of ``points`` elements; instance i starts at ``offsets[i]``.
    ``tf32=True`` keeps split TF32 operands on every tensor-core phase
    (FFX_TC_TF32); by default they take split BF16 operands (but the first
    adjoint pass of a backward call)."""

    def __init__(self, instances, form: str = "auto", tf32: bool = False):
        lib = load_library()
        n = len(instances)
        descs = (InstanceDesc * n)()
        for i, spec in enumerate(instances):
            dims, spacing, t, lam = spec[:4]
            d = descs[i]
            d.ndim = len(dims)
            for j in range(len(dims)):
                d.dims[j] = int(dims[j])
                d.spacing[j] = float(spacing[j])
                d.magnification[j] = int(lam[j])
            d.t = float(t)
            if len(spec) > 4 and spec[4] is not None:
                d.has_offsets = 1
                for j in range(len(dims)):
                    d.a[j] = float(spec[4][j])
                    d.abar[j] = float(spec[5][j])
        h = ctypes.c_void_p()
        flags = _FORMS[form] | (FFX_TC_TF32 if tf32 else 0)
        _check(lib.ffx_plan_many(ctypes.byref(h), n, descs, flags), "ffx_plan_many")
        self._h = h
        self.accumulate = False
        self.form = _FORM_NAMES[lib.ffx_plan_form(h)]
        self.instances = [tuple(tuple(x) if hasattr(x, "__len__") else x for x in spec[:4]) for spec in instances]
        self.points = int(lib.ffx_plan_points(h))
        self.offsets = [int(lib.ffx_plan_many_offset(h, i)) for i in range(n)]
        self.bf16 = lib.ffx_plan_tc_bf16(h) == 1
        self.fused, self.fused_max_batch = False, 0
        self.dims = (self.points,)
        self.M = self.points

    def _batch(self, x: torch.Tensor) -> int:
        if x.numel() != self.points:
            raise ValueError(f"packed tensor must have {self.points} elements, got {x.numel()}")
        return 1

    def unpack(self, x: torch.Tensor):
        """Views of a packed tensor, one per instance, shaped like its lattice."""
        out = []
        for i, spec in enumerate(self.instances):
            dims = spec[0]
            m = 1
            for v in dims:
                m *= int(v)
            out.append(x.reshape(-1)[self.offsets[i]:self.offsets[i] + m].view(*dims))
        return out


def ffx_plan(dims, spacing, t, magnification, a=None, abar=None, form="auto", accumulate=False,
             tune=False) -> Plan:
    return Plan(dims, spacing, t, magnification, a, abar, form, accumulate, tune)


def ffx_plan_destroy(plan: Plan):
    plan.close()


def ffx_expand(plan: Plan, psi0: torch.Tensor, out_density: torch.Tensor | None = None,
               stream=None) -> torch.Tensor:
    """Densities |Psibar|^2 ([B, *dims] float32), or their batch sum added to
    ``out_density`` ([*dims]) for an accumulating plan."""
    _need(psi0, torch.complex64, "psi0")
    B = plan._batch(psi0)
    if out_density is None:
        shape = plan.dims if plan.accumulate else psi0.shape
        out_density = torch.zeros(shape, dtype=torch.float32, device=psi0.device)
    _need(out_density, torch.float32, "out_density")
    _check(load_library().ffx_expand(plan.handle, _ptr(psi0), B, _ptr(out_density), _stream(stream)),
           "ffx_expand")
    return out_density


def ffx_expand_host(plan: Plan, psi0: torch.Tensor, out_density: torch.Tensor, stream=None) -> torch.Tensor:
    """ffx_expand on host tensors in one C call: psi0 (complex64, CPU,
    contiguous; pinned for overlap) is copied to the device, expanded, and the
    densities are copied into out_density (float32, CPU; [B, *dims], or
    [*dims] accumulated for an accumulating plan).  Asynchronous on `stream`:
    synchronize it before reading out_density."""
    for x, dt, name in ((psi0, torch.complex64, "psi0"), (out_density, torch.float32, "out_density")):
        if x.device.type != "cpu" or x.dtype != dt or not x.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {dt} tensor in host memory")
    B = plan._batch(psi0)
    need = (plan.M if plan.accumulate else B * plan.M)
    if out_density.numel() != need:
        raise ValueError(f"out_density must have {need} elements")
    _check(load_library().ffx_expand_host(plan.handle, ctypes.c_void_p(psi0.data_ptr()), B,
                                          ctypes.c_void_p(out_density.data_ptr()), _stream(stream)),
           "ffx_expand_host")
    return out_density


def ffx_expand_field(plan: Plan, psi0: torch.Tensor, out_field: torch.Tensor | None = None,
                     stream=None) -> torch.Tensor:
    _need(psi0, torch.complex64, "psi0")
    B = plan._batch(psi0)
    if out_field is None:
        out_field = torch.empty_like(psi0)
    _need(out_field, torch.complex64, "out_field")
    _check(load_library().ffx_expand_field(plan.handle, _ptr(psi0), B, _ptr(out_field), _stream(stream)),
           "ffx_expand_field")
    return out_field


def ffx_expand_adjoint(plan: Plan, g: torch.Tensor, out: torch.Tensor | None = None,
                       stream=None) -> torch.Tensor:
    _need(g, torch.complex64, "g")
    B = plan._batch(g)
    if out is None:
        out = torch.empty_like(g)
    _need(out, torch.complex64, "out")
    _check(load_library().ffx_expand_adjoint(plan.handle, _ptr(g), B, _ptr(out), _stream(stream)),
           "ffx_expand_adjoint")
    return out


def ffx_expand_backward(plan: Plan, psi0: torch.Tensor, grad_density: torch.Tensor,
                        grad_psi0: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    _need(psi0, torch.complex64, "psi0")
    _need(grad_density, torch.float32, "grad_density")
    B = plan._batch(psi0)
    if grad_psi0 is None:
        grad_psi0 = torch.empty_like(psi0)
    _need(grad_psi0, torch.complex64, "grad_psi0")
    _check(load_library().ffx_expand_backward(plan.handle, _ptr(psi0), _ptr(grad_density), B,
                                              _ptr(grad_psi0), _stream(stream)), "ffx_expand_backward")
    return grad_psi0


def ffx_expand_column(plan: Plan, psi0: torch.Tensor, axis: int, out_column: torch.Tensor | None = None,
                      stream=None) -> torch.Tensor:
    """Detector image: |Psibar|^2 integrated along lattice axis ``axis`` (Sec. 6)."""
    _need(psi0, torch.complex64, "psi0")
    B = plan._batch(psi0)
    d = len(plan.dims)
    if not 0 <= axis < d:
        raise ValueError(f"axis {axis} out of range for {d} lattice axes")
    rest = tuple(n for j, n in enumerate(plan.dims) if j != axis)
    if out_column is None:
        shape = rest if plan.accumulate else tuple(psi0.shape[:psi0.dim() - d]) + rest
        out_column = torch.zeros(shape, dtype=torch.float32, device=psi0.device)
    _need(out_column, torch.float32, "out_column")
    _check(load_library().ffx_expand_column(plan.handle, _ptr(psi0), B, axis, _ptr(out_column), _stream(stream)),
           "ffx_expand_column")
    return out_column


def ffx_expand_positive_p(plan: Plan, psi0: torch.Tensor, psi0_plus: torch.Tensor,
                          out_density: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Re(Psibar+ Psibar) of positive-P pairs: psi0 by the map, psi0_plus by its conjugate."""
    _need(psi0, torch.complex64, "psi0")
    _need(psi0_plus, torch.complex64, "psi0_plus")
    if psi0_plus.shape != psi0.shape:
        raise ValueError("psi0 and psi0_plus must have the same shape")
    B = plan._batch(psi0)
    if out_density is None:
        shape = plan.dims if plan.accumulate else psi0.shape
        out_density = torch.zeros(shape, dtype=torch.float32, device=psi0.device)
    _need(out_density, torch.float32, "out_density")
    _check(load_library().ffx_expand_positive_p(plan.handle, _ptr(psi0), _ptr(psi0_plus), B, _ptr(out_density),
                                                _stream(stream)), "ffx_expand_positive_p")
    return out_density


def output_axis(plan: Plan, axis: int):
    """(x0, step) of the magnified output lattice along ``axis`` (eq. wbx)."""
    x0, step = ctypes.c_double(), ctypes.c_double()
    _check(load_library().ffx_plan_output_axis(plan.handle, axis, ctypes.byref(x0), ctypes.byref(step)),
           "ffx_plan_output_axis")
    return x0.value, step.value


def ffx_fringe_phase(image: torch.Tensor, y0: float, dy: float, D: float, t: float, y_dim: int = -1,
                     stream=None) -> torch.Tensor:
    """Eq. dphase2 per row of a 2-D float32 image whose dimension ``y_dim`` is y."""
    if not isinstance(image, torch.Tensor) or not image.is_cuda or image.dtype != torch.float32:
        raise TypeError("image must be a float32 CUDA tensor")
    if image.dim() != 2:
        raise ValueError("image must be 2-D (rows, y) or (y, rows)")
    yd = y_dim % 2
    rows, ny = image.shape[1 - yd], image.shape[yd]
    out = torch.empty(rows, dtype=torch.float64, device=image.device)
    _check(load_library().ffx_fringe_phase(_ptr(image), rows, ny, image.stride(1 - yd), image.stride(yd),
                                           y0, dy, D, t, _ptr(out), _stream(stream)), "ffx_fringe_phase")
    return out


class _ExpandDensity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, psi0, plan):
        psi0 = psi0.contiguous()
        ctx.plan = plan
        ctx.save_for_backward(psi0)
        return ffx_expand(plan, psi0)

    @staticmethod
    def backward(ctx, grad):
        (psi0,) = ctx.saved_tensors
        g = ffx_expand_backward(ctx.plan, psi0, grad.contiguous().to(torch.float32))
        return g, None


def expand_density(psi0: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Differentiable densities after free flight (gradient via the adjoint kernels)."""
    return _ExpandDensity.apply(psi0, plan)


def ffx_expand_noalloc(dims, spacing, t, magnification, psi0: torch.Tensor,
                       out_density: torch.Tensor, a=None, abar=None, stream=None) -> torch.Tensor:
    """Densities through the entry point that allocates no device memory.

    For callers that cannot allocate while they run (a framework owning the
    device memory pool, a real-time loop): the library uses fixed static
    device scratch instead of a plan's tables and workspace.  ``out_density``
    must be given (this function creates no tensors).  Calls sharing a GPU
    must not overlap (they share the scratch); see include/ffx.h."""
    _need(psi0, torch.complex64, "psi0")
    _need(out_density, torch.float32, "out_density")
    d = len(dims)
    M = 1
    for v in dims:
        M *= int(v)
    arr = lambda ct, v: (ct * d)(*v) if v is not None else None  # noqa: E731
    _check(load_library().ffx_expand_noalloc(
        d, arr(ctypes.c_int64, [int(v) for v in dims]), arr(ctypes.c_double, [float(v) for v in spacing]),
        float(t), arr(ctypes.c_int32, [int(v) for v in magnification]), arr(ctypes.c_double, a),
        arr(ctypes.c_double, abar), _ptr(psi0), int(psi0.numel() // M), _ptr(out_density),
        _stream(stream)), "ffx_expand_noalloc")
    return out_density
