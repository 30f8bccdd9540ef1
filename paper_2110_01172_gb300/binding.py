"""Thin ctypes binding of the C ABI in include/gbdct.h (argument marshalling only).

Every transform step runs in the CUDA kernels of ``libgbdct.so``; this module
only checks tensors, allocates outputs with PyTorch and passes raw device
pointers and the current CUDA stream.  There is no CPU fallback: if the
library is missing or fails to load, every entry point raises.
"""

from __future__ import annotations

import ctypes
import os
import re
import threading

from . import build as _build

OK = 0
ERR_INVALID_ARG = 1
ERR_UNSUPPORTED = 2
ERR_OOM = 3
ERR_CUDA = 4
ERR_TIMEOUT = 5

KINDS = {"dct2": 0, "dst2": 1, "idct_idxst": 2, "idxst_idct": 3}
F32 = 0
GRAPH = 1   # GBDCT_MULTI_GRAPH
TUNE = 2    # GBDCT_MULTI_TUNE

HEADER = os.path.join(_build.ROOT, "include", "gbdct.h")

_lib = None
_lock = threading.Lock()


class GbdctError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_name(status)}")


def declared_functions(header: str = HEADER):
    """Names of the functions declared in the C header (used by the ABI tests)."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gbdct_[a-z0-9_]+)\s*\(", text)))


def load(path: str | None = None, build_if_missing: bool = True) -> ctypes.CDLL:
    """Load (building first if needed) the in-tree CUDA library."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if path is None:
            path = _build.library_path()
            if build_if_missing and _build.is_stale():
                _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libgbdct not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        c_i64p = ctypes.POINTER(ctypes.c_int64)
        plan_p = ctypes.c_void_p
        sigs = {
            "gbdct_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "gbdct_version": (ctypes.c_char_p, []),
            "gbdct_plan_create": (ctypes.c_int, [ctypes.POINTER(plan_p), ctypes.c_int, c_i64p,
                                                 ctypes.c_int, ctypes.c_int]),
            "gbdct_plan_create_batched": (ctypes.c_int, [ctypes.POINTER(plan_p), ctypes.c_int, c_i64p,
                                                         ctypes.c_int64, ctypes.c_int, ctypes.c_int]),
            "gbdct_exec_forward": (ctypes.c_int, [plan_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
            "gbdct_exec_inverse": (ctypes.c_int, [plan_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
            "gbdct_plan_workspace_bytes": (ctypes.c_size_t, [plan_p]),
            "gbdct_plan_launches_per_exec": (ctypes.c_int, [plan_p]),
            "gbdct_plan_kernel_family": (ctypes.c_char_p, [plan_p]),
            "gbdct_plan_check_device_error": (ctypes.c_int, [plan_p]),
            "gbdct_plan_set_wait_limit": (ctypes.c_int, [plan_p, ctypes.c_uint32]),
            "gbdct_plan_set_threshold": (ctypes.c_int, [plan_p, ctypes.c_float]),
            "gbdct_exec_step": (ctypes.c_int, [plan_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_void_p]),
            "gbdct_plan_step_name": (ctypes.c_char_p, [plan_p, ctypes.c_int, ctypes.c_int]),
            "gbdct_plan_destroy": (ctypes.c_int, [plan_p]),
            "gbdct_poisson_create": (ctypes.c_int, [ctypes.POINTER(plan_p), ctypes.c_int64, ctypes.c_int64]),
            "gbdct_poisson_solve": (ctypes.c_int, [plan_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                   ctypes.c_void_p, ctypes.c_void_p]),
            "gbdct_poisson_workspace_bytes": (ctypes.c_size_t, [plan_p]),
            "gbdct_poisson_destroy": (ctypes.c_int, [plan_p]),
            "gbdct_dct2d_forward_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                                           ctypes.c_int64, ctypes.c_void_p]),
            "gbdct_plan_set_precision": (ctypes.c_int, [plan_p, ctypes.c_int]),
            "gbdct_plan_create_family": (ctypes.c_int, [ctypes.POINTER(plan_p), ctypes.c_int, c_i64p,
                                                        ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                                        ctypes.c_char_p]),
            "gbdct_plan_create_tuned": (ctypes.c_int, [ctypes.POINTER(plan_p), ctypes.c_int, c_i64p,
                                                       ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                                       ctypes.c_char_p, ctypes.c_size_t]),
            "gbdct_multi_create": (ctypes.c_int, [ctypes.POINTER(plan_p), ctypes.c_int, c_i64p, ctypes.c_int,
                                                  ctypes.c_int]),
            "gbdct_multi_layout": (ctypes.c_int64, [ctypes.c_int, c_i64p, c_i64p, ctypes.POINTER(ctypes.c_int)]),
            "gbdct_multi_offset": (ctypes.c_int64, [plan_p, ctypes.c_int]),
            "gbdct_multi_total_elems": (ctypes.c_int64, [plan_p]),
            "gbdct_multi_group_count": (ctypes.c_int, [plan_p]),
            "gbdct_multi_group_family": (ctypes.c_char_p, [plan_p, ctypes.c_int]),
            "gbdct_multi_exec": (ctypes.c_int, [plan_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p]),
            "gbdct_multi_destroy": (ctypes.c_int, [plan_p]),
        }
        for name, (res, args) in sigs.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def status_name(status: int) -> str:
    try:
        return load().gbdct_status_string(int(status)).decode()
    except Exception:  # library unavailable: still give a readable message
        return f"status {status}"


def _check(status: int, what: str):
    if status != OK:
        raise GbdctError(status, what)


def _torch():
    import torch
    return torch


def _stream_handle(stream, device):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """A transform plan: twiddle tables and workspace resident on one GPU.

    shape: (N1, N2) of one transform; batch: number of transforms stored back
    to back; kind: "dct2" (forward DCT-II, inverse = exact inverse).
    """

    def __init__(self, shape, kind: str = "dct2", batch: int = 1, device=None, family: str | None = None,
                 tuned: bool = False):
        """family: force a kernel family ("seq", "pair", "fs2", "tp", "fs2/<A>" for a
        four-step split, or "tp/<NP>" for a two-pass strip width);
        tuned: pick the fastest family by timing (gbdct_plan_create_tuned)."""
        torch = _torch()
        lib = load()
        if kind not in KINDS:
            raise ValueError(f"unknown kind {kind!r}")
        self.shape = tuple(int(s) for s in shape)
        self.kind = kind
        self.batch = int(batch)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        dims = (ctypes.c_int64 * len(self.shape))(*self.shape)
        handle = ctypes.c_void_p()
        args = (ctypes.byref(handle), len(self.shape), dims, self.batch, KINDS[kind], F32)
        self.choice = family   # the forced or tuned family / tile choice, e.g. "fs2/32", "tp/2"
        with torch.cuda.device(self.device):
            if family is not None:
                _check(lib.gbdct_plan_create_family(*args, family.encode()), "gbdct_plan_create_family")
            elif tuned:
                buf = ctypes.create_string_buffer(32)
                _check(lib.gbdct_plan_create_tuned(*args, buf, 32), "gbdct_plan_create_tuned")
                self.choice = buf.value.decode()
            else:
                _check(lib.gbdct_plan_create_batched(*args), "gbdct_plan_create")
        self._h = handle
        self._lib = lib

    @property
    def workspace_bytes(self) -> int:
        return int(self._lib.gbdct_plan_workspace_bytes(self._h))

    def set_precision(self, precision: str):
        """"fp32" (the FFT kernels) or "split_bf16" (tcgen05 tensor-core DFT-GEMMs, ~5e-6 error)."""
        modes = {"fp32": 0, "split_bf16": 1}
        if precision not in modes:
            raise ValueError(f"unknown precision {precision!r}")
        with _torch().cuda.device(self.device):
            _check(self._lib.gbdct_plan_set_precision(self._h, modes[precision]), "gbdct_plan_set_precision")
        return self

    @property
    def family(self) -> str:
        return self._lib.gbdct_plan_kernel_family(self._h).decode()

    @property
    def launches_per_exec(self) -> int:
        return int(self._lib.gbdct_plan_launches_per_exec(self._h))

    def _prep(self, x, out):
        """x and out: CUDA float32 tensors, or page-locked CPU float32 tensors
        (read/written by the kernels over the host link, no staging copy)."""
        torch = _torch()
        want = ((self.batch,) if self.batch > 1 else ()) + self.shape

        def usable(t):
            return t.dtype == torch.float32 and (t.is_cuda or (t.device.type == "cpu" and t.is_pinned()))

        if not usable(x):
            raise TypeError("expected a CUDA or page-locked CPU float32 tensor")
        if tuple(x.shape) != want:
            raise ValueError(f"expected shape {want}, got {tuple(x.shape)}")
        if not x.is_contiguous():
            x = x.contiguous()
        if out is None:
            out = torch.empty_like(x) if x.is_cuda else torch.empty(want, dtype=torch.float32, pin_memory=True)
        elif tuple(out.shape) != want or not usable(out) or not out.is_contiguous():
            raise ValueError("out must be a contiguous CUDA or page-locked float32 tensor of the input's shape")
        return x, out

    def forward(self, x, out=None, stream=None):
        x, out = self._prep(x, out)
        _check(self._lib.gbdct_exec_forward(self._h, ctypes.c_void_p(x.data_ptr()),
                                            ctypes.c_void_p(out.data_ptr()),
                                            _stream_handle(stream, self.device)), "gbdct_exec_forward")
        return out

    def inverse(self, x, out=None, stream=None):
        x, out = self._prep(x, out)
        _check(self._lib.gbdct_exec_inverse(self._h, ctypes.c_void_p(x.data_ptr()),
                                            ctypes.c_void_p(out.data_ptr()),
                                            _stream_handle(stream, self.device)), "gbdct_exec_inverse")
        return out

    def step(self, inverse: bool, step: int, x, out, stream=None):
        """Run launch `step` of the forward/inverse sequence alone (per-kernel timing)."""
        _check(self._lib.gbdct_exec_step(self._h, int(bool(inverse)), int(step), ctypes.c_void_p(x.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), _stream_handle(stream, self.device)),
               "gbdct_exec_step")
        return out

    def step_name(self, inverse: bool, step: int) -> str:
        return self._lib.gbdct_plan_step_name(self._h, int(bool(inverse)), int(step)).decode()

    def check_device_error(self) -> int:
        """Status of the device error word (OK, or ERR_TIMEOUT after a bounded wait gave up)."""
        return int(self._lib.gbdct_plan_check_device_error(self._h))

    def set_threshold(self, eps: float):
        """Forward outputs with |X| < eps stored as zero (Section V-A compression; 0: off)."""
        _check(self._lib.gbdct_plan_set_threshold(self._h, float(eps)), "gbdct_plan_set_threshold")
        return self

    def set_wait_limit(self, polls: int):
        """Bound of the plan's device-side waits in polls (0: the default)."""
        _check(self._lib.gbdct_plan_set_wait_limit(self._h, int(polls)), "gbdct_plan_set_wait_limit")
        return self

    def forward_ptr(self, in_ptr: int, out_ptr: int, stream_ptr: int = 0) -> int:
        """Raw-pointer forward call (returns the status code, never raises)."""
        return int(self._lib.gbdct_exec_forward(self._h, ctypes.c_void_p(in_ptr),
                                                ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream_ptr)))

    def inverse_ptr(self, in_ptr: int, out_ptr: int, stream_ptr: int = 0) -> int:
        return int(self._lib.gbdct_exec_inverse(self._h, ctypes.c_void_p(in_ptr),
                                                ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream_ptr)))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.gbdct_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def multi_layout(shapes):
    """(offsets, total floats, groups) of the packed layout of an uneven batch;
    host-only (no CUDA call)."""
    lib = load()
    n = len(shapes)
    flat = (ctypes.c_int64 * (2 * n))(*[int(v) for sh in shapes for v in sh])
    offs = (ctypes.c_int64 * n)()
    groups = ctypes.c_int()
    total = int(lib.gbdct_multi_layout(n, flat, offs, ctypes.byref(groups)))
    if total < 0:
        raise ValueError("invalid shapes for an uneven batch")
    return list(offs), total, groups.value


class MultiPlan:
    """Uneven-size batch of 2D transforms (gbdct_multi_*): groups by shape into
    batched plans over one packed buffer; optionally replayed as a CUDA graph."""

    def __init__(self, shapes, kind: str = "dct2", graph: bool = True, tuned: bool = False, device=None):
        torch = _torch()
        lib = load()
        if kind not in KINDS:
            raise ValueError(f"unknown kind {kind!r}")
        self.shapes = [tuple(int(v) for v in sh) for sh in shapes]
        if not self.shapes or any(len(sh) != 2 for sh in self.shapes):
            raise ValueError("expected a non-empty list of (N1, N2) shapes")
        self.kind = kind
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        flat = (ctypes.c_int64 * (2 * len(self.shapes)))(*[v for sh in self.shapes for v in sh])
        flags = (GRAPH if graph else 0) | (TUNE if tuned else 0)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib.gbdct_multi_create(ctypes.byref(h), len(self.shapes), flat, KINDS[kind], flags),
                   "gbdct_multi_create")
        self._h = h
        self._lib = lib
        self.offsets = [int(lib.gbdct_multi_offset(h, i)) for i in range(len(self.shapes))]
        self.total = int(lib.gbdct_multi_total_elems(h))

    @property
    def groups(self) -> int:
        return int(self._lib.gbdct_multi_group_count(self._h))

    def group_families(self):
        return [self._lib.gbdct_multi_group_family(self._h, g).decode() for g in range(self.groups)]

    def pack(self, tensors, out=None):
        """Copy a list of (N1, N2) tensors into one packed CUDA float32 buffer."""
        torch = _torch()
        buf = torch.empty(self.total, dtype=torch.float32, device=self.device) if out is None else out
        for t, off, sh in zip(tensors, self.offsets, self.shapes):
            buf[off:off + sh[0] * sh[1]].view(sh).copy_(t)
        return buf

    def unpack(self, buf):
        """Views of the transforms inside a packed buffer."""
        return [buf[off:off + sh[0] * sh[1]].view(sh) for off, sh in zip(self.offsets, self.shapes)]

    def _exec(self, inverse, x, out, stream):
        torch = _torch()
        if x.dtype != torch.float32 or not x.is_cuda or x.numel() != self.total or not x.is_contiguous():
            raise ValueError(f"expected a contiguous CUDA float32 buffer of {self.total} values")
        out = torch.empty_like(x) if out is None else out
        _check(self._lib.gbdct_multi_exec(self._h, int(inverse), ctypes.c_void_p(x.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()), _stream_handle(stream, self.device)),
               "gbdct_multi_exec")
        return out

    def forward(self, x, out=None, stream=None):
        return self._exec(False, x, out, stream)

    def inverse(self, x, out=None, stream=None):
        return self._exec(True, x, out, stream)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.gbdct_multi_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PoissonSolver:
    """Spectral Neumann Poisson solver (Algorithm 4): rho -> (psi, xi0, xi1) on one GPU."""

    def __init__(self, shape, device=None):
        torch = _torch()
        lib = load()
        self.shape = tuple(int(s) for s in shape)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib.gbdct_poisson_create(ctypes.byref(h), *self.shape), "gbdct_poisson_create")
        self._h = h
        self._lib = lib

    @property
    def workspace_bytes(self) -> int:
        return int(self._lib.gbdct_poisson_workspace_bytes(self._h))

    def solve(self, rho, psi=None, xi0=None, xi1=None, stream=None):
        torch = _torch()
        if rho.dtype != torch.float32 or not rho.is_cuda or tuple(rho.shape) != self.shape:
            raise ValueError(f"expected a CUDA float32 tensor of shape {self.shape}")
        rho = rho.contiguous()
        psi = torch.empty_like(rho) if psi is None else psi
        xi0 = torch.empty_like(rho) if xi0 is None else xi0
        xi1 = torch.empty_like(rho) if xi1 is None else xi1
        _check(self._lib.gbdct_poisson_solve(self._h, ctypes.c_void_p(rho.data_ptr()),
                                             ctypes.c_void_p(psi.data_ptr()), ctypes.c_void_p(xi0.data_ptr()),
                                             ctypes.c_void_p(xi1.data_ptr()), _stream_handle(stream, rho.device)),
               "gbdct_poisson_solve")
        return psi, xi0, xi1

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.gbdct_poisson_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_plans: dict = {}


def _cached_plan(shape, kind, batch, device):
    key = (tuple(shape), kind, batch, device)
    p = _plans.get(key)
    if p is None:
        p = Plan(shape, kind, batch, device)
        _plans[key] = p
    return p


def _split(x):
    if x.dim() == 2:
        return tuple(x.shape), 1
    if x.dim() == 3:
        return tuple(x.shape[1:]), int(x.shape[0])
    raise ValueError("expected a 2D tensor or a batch of 2D tensors")


def dct2(x, out=None):
    """2D DCT-II (unnormalised) of a CUDA float32 (N1, N2) or (B, N1, N2) tensor."""
    shape, batch = _split(x)
    return _cached_plan(shape, "dct2", batch, x.device).forward(x, out)


def idct2(x, out=None):
    """Exact inverse of ``dct2`` (2/N-scaled DCT-III per axis)."""
    shape, batch = _split(x)
    return _cached_plan(shape, "dct2", batch, x.device).inverse(x, out)


def dct3(x, out=None):
    """3D DCT-II (unnormalised, the 1D DCT-II along every axis) of a CUDA float32
    (N0, N1, N2) tensor."""
    if x.dim() != 3:
        raise ValueError("expected a 3D tensor")
    return _cached_plan(tuple(x.shape), "dct2", 1, x.device).forward(x, out)


def idct3(x, out=None):
    """Exact inverse of ``dct3``."""
    if x.dim() != 3:
        raise ValueError("expected a 3D tensor")
    return _cached_plan(tuple(x.shape), "dct2", 1, x.device).inverse(x, out)


def dst2(x, out=None):
    """2D DST-II (unnormalised sine analogue of ``dct2``)."""
    shape, batch = _split(x)
    return _cached_plan(shape, "dst2", batch, x.device).forward(x, out)


def idst2(x, out=None):
    """Exact inverse of ``dst2``."""
    shape, batch = _split(x)
    return _cached_plan(shape, "dst2", batch, x.device).inverse(x, out)


def idct_idxst(x, out=None):
    """IDCT along axis 0 and IDXST along axis 1 (2/N-scaled, like ``idct2``)."""
    shape, batch = _split(x)
    return _cached_plan(shape, "idct_idxst", batch, x.device).inverse(x, out)


def idxst_idct(x, out=None):
    """IDXST along axis 0 and IDCT along axis 1."""
    shape, batch = _split(x)
    return _cached_plan(shape, "idxst_idct", batch, x.device).inverse(x, out)


def dct2_noalloc(x, out=None, stream=None):
    """2D DCT-II through the entry point that allocates no device memory.

    For callers that cannot allocate on the call path (a host framework that
    owns all device memory, or loops where a cudaMalloc would stall other
    streams); the transform's scratch is a static device array shared by all
    calls, so calls must not overlap on the GPU.  N1 * N2 <= 2**20.
    """
    torch = _torch()
    lib = load()
    if x.dim() != 2 or x.dtype != torch.float32 or not x.is_cuda or not x.is_contiguous():
        raise TypeError("expected a contiguous 2D CUDA float32 tensor")
    if out is None:
        out = torch.empty_like(x)
    n1, n2 = x.shape
    _check(lib.gbdct_dct2d_forward_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                           n1, n2, _stream_handle(stream, x.device)),
           "gbdct_dct2d_forward_noalloc")
    return out
