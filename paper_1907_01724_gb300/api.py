"""Thin Python binding of the HSMA C ABI (include/hsma.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  Arrays are numpy float64
(host) or torch CUDA tensors (device); PyTorch provides the device workspace and streams.
All arithmetic of the method runs in the CUDA library; nothing here computes any of it.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import numpy as np

from . import _native

HSMA_OK = 0
HSMA_FP32 = 0
HSMA_FP64 = 1
HSMA_TOTAL = 0
HSMA_REACTION = 1
HSMA_COULOMB = 2
ERRORS = {
    -1: "HSMA_E_INVALID_ARG", -2: "HSMA_E_OUTSIDE", -3: "HSMA_E_STATE", -4: "HSMA_E_OOM", -5: "HSMA_E_CUDA",
    -6: "HSMA_E_TIMEOUT", -7: "HSMA_E_BUSY", -8: "HSMA_E_NONFINITE",
}


class HsmaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def _check(rc: int, handle=None, what: str = ""):
    if rc != HSMA_OK:
        lib = _native.load()
        msg = lib.hsma_last_error(handle).decode() if handle else what
        raise HsmaError(rc, msg or what)


def hsma_version() -> str:
    return _native.load().hsma_version().decode()


def hsma_default_params(**overrides) -> _native.HsmaParams:
    p = _native.HsmaParams()
    _check(_native.load().hsma_default_params(ctypes.byref(p)), what="default params")
    for k, v in overrides.items():
        if k == "stream" and v is not None and not isinstance(v, int):
            v = int(v.cuda_stream)
        setattr(p, k, v)
    return p


def _host_f64(x, shape=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


_dptr = _native.host_ptr


def _is_torch_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and bool(getattr(x, "is_cuda"))


class Handle:
    """Owns an hsma_t and the PyTorch tensor used as its device workspace."""

    def __init__(self, ptr: ctypes.c_void_p, device: int, use_torch_workspace: bool):
        self.ptr = ptr
        self.device = device
        self.use_torch_workspace = use_torch_workspace
        self.workspace = None
        self.n = -1
        self.ptrs = {}  # host addresses per call slot (_native.cached_ptr)

    def __del__(self):
        try:
            if self.ptr:
                _native.load().hsma_destroy(self.ptr)
                self.ptr = None
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        return self.ptr


def hsma_create(a: float, eps1: float, eps2: float, kappa: float, params: _native.HsmaParams | None = None,
                use_torch_workspace: bool = True) -> Handle:
    lib = _native.load()
    params = params if params is not None else hsma_default_params()
    out = ctypes.c_void_p()
    rc = lib.hsma_create(float(a), float(eps1), float(eps2), float(kappa), ctypes.byref(params), ctypes.byref(out))
    _check(rc, what="hsma_create")
    return Handle(out, params.device, use_torch_workspace)


def hsma_destroy(h: Handle) -> None:
    if h.ptr:
        _native.load().hsma_destroy(h.ptr)
        h.ptr = None


def hsma_workspace_size(h: Handle, n: int) -> int:
    b = ctypes.c_size_t()
    _check(_native.load().hsma_workspace_size(h.ptr, int(n), ctypes.byref(b)), h.ptr)
    return int(b.value)


def hsma_attach_workspace(h: Handle, tensor) -> None:
    """Attach a torch uint8 CUDA tensor (kept alive by the handle) as the device workspace."""
    h.workspace = tensor
    ptr = tensor.data_ptr() if tensor is not None else None
    size = tensor.numel() if tensor is not None else 0
    _check(_native.load().hsma_attach_workspace(h.ptr, ctypes.c_void_p(ptr), ctypes.c_size_t(size)), h.ptr)


def _ensure_workspace(h: Handle, n: int) -> None:
    if not h.use_torch_workspace:
        return
    if getattr(h, "_ws_n", None) == n:
        return
    need = hsma_workspace_size(h, n)
    h._ws_n = n
    if h.workspace is None or h.workspace.numel() < need:
        import torch
        t = torch.empty(need + need // 4 + 256, dtype=torch.uint8, device=f"cuda:{h.device}")
        off = (-t.data_ptr()) % 256
        hsma_attach_workspace(h, t[off:])


def hsma_build_sources(h: Handle, xyz, q) -> None:
    """Build Kelvin and surface images (Sec. 2.4) from host numpy or device torch arrays."""
    lib = _native.load()
    if _is_torch_cuda(xyz):
        import torch
        xyz_t = xyz.to(torch.float64).contiguous()
        q_t = q.to(torch.float64).contiguous()
        n = int(q_t.numel())
        _ensure_workspace(h, n)
        _check(lib.hsma_build_sources_device(h.ptr, n, ctypes.c_void_p(xyz_t.data_ptr()),
                                             ctypes.c_void_p(q_t.data_ptr())), h.ptr)
        h._keep = (xyz_t, q_t)
    else:
        xyz_a = _host_f64(xyz, (-1, 3))
        q_a = _host_f64(q)
        n = int(q_a.shape[0])
        if xyz_a.shape[0] != n:
            raise ValueError("xyz and q sizes differ")
        _ensure_workspace(h, n)
        _check(lib.hsma_build_sources(h.ptr, n, _native.cached_ptr(h.ptrs, "xyz", xyz_a),
                                      _native.cached_ptr(h.ptrs, "q", q_a)), h.ptr)
        h._keep = (xyz_a, q_a)  # page-locked arrays are read by the next evaluation
    h.n = n


def hsma_potential(h: Handle, what: int = HSMA_TOTAL, out=None):
    """Potentials at the charges: into out (a torch CUDA tensor, or a float64 numpy array of n
    entries, written by the device itself when it is page-locked), else a new numpy array."""
    lib = _native.load()
    if out is not None and _is_torch_cuda(out):
        _check(lib.hsma_potential_device(h.ptr, ctypes.c_void_p(out.data_ptr()), int(what)), h.ptr)
        return out
    if out is not None:
        if not (isinstance(out, np.ndarray) and out.dtype == np.float64 and out.flags.c_contiguous
                and out.flags.writeable and out.size == max(h.n, 0)):
            raise ValueError(f"out must be a writable C-contiguous float64 array of {max(h.n, 0)} entries")
        phi = out
    else:
        phi = np.empty(max(h.n, 0), dtype=np.float64)
    _check(lib.hsma_potential(h.ptr, _native.cached_ptr(h.ptrs, "phi", phi), int(what)), h.ptr)
    return phi


def hsma_field(h: Handle, what: int = HSMA_TOTAL, out=None):
    """Fields E = -grad phi at the charges, (n, 3): numpy array, or into a torch CUDA tensor given as out."""
    lib = _native.load()
    if out is not None and _is_torch_cuda(out):
        _check(lib.hsma_field_device(h.ptr, ctypes.c_void_p(out.data_ptr()), int(what)), h.ptr)
        return out
    E = np.empty((max(h.n, 0), 3), dtype=np.float64)
    _check(lib.hsma_field(h.ptr, _dptr(E), int(what)), h.ptr)
    return E


def hsma_energy(h: Handle) -> tuple[float, float]:
    et, er = ctypes.c_double(), ctypes.c_double()
    _check(_native.load().hsma_energy(h.ptr, ctypes.byref(et), ctypes.byref(er)), h.ptr)
    return et.value, er.value


def hsma_delta_energy(h: Handle, k: int, x_new) -> float:
    x = _host_f64(x_new, (3,))
    de = ctypes.c_double()
    _check(_native.load().hsma_delta_energy(h.ptr, int(k), _dptr(x), ctypes.byref(de)), h.ptr)
    return de.value


def hsma_apply_move(h: Handle, k: int, x_new) -> None:
    x = _host_f64(x_new, (3,))
    _check(_native.load().hsma_apply_move(h.ptr, int(k), _dptr(x)), h.ptr)


def hsma_set_overlap(h: Handle, on: bool) -> None:
    _check(_native.load().hsma_set_overlap(h.ptr, 1 if on else 0), h.ptr)


def hsma_kernel_launches(h: Handle) -> int:
    return int(_native.load().hsma_kernel_launches(h.ptr))


def hsma_coefficients(h: Handle, p: int) -> np.ndarray:
    """Correction coefficients (eq. phim) in the real normalised solid-harmonic basis, (p+1)^2 values."""
    out = np.empty((p + 1) ** 2, dtype=np.float64)
    _check(_native.load().hsma_coefficients(h.ptr, _dptr(out), out.size), h.ptr)
    return out


def hsma_last_pair_time(h: Handle) -> float:
    """Milliseconds of the most recent pair-sum kernel launch (CUDA events on the handle's stream)."""
    ms = ctypes.c_float()
    _check(_native.load().hsma_last_pair_time(h.ptr, ctypes.byref(ms)), h.ptr)
    return float(ms.value)


def hsma_set_far_field(h: Handle, theta: float, order: int = 12) -> None:
    """Real/Kelvin pair sums by the treecode (opening criterion theta, multipole order 8/12/16);
    theta = 0 restores the direct sum.  Takes effect at the next hsma_build_sources."""
    _check(_native.load().hsma_set_far_field(h.ptr, float(theta), int(order)), h.ptr)
    h._ws_n = None  # the layout (and its workspace size) changes


def hsma_last_far_time(h: Handle) -> float:
    """Milliseconds of the most recent treecode evaluation kernel (CUDA events)."""
    ms = ctypes.c_float()
    _check(_native.load().hsma_last_far_time(h.ptr, ctypes.byref(ms)), h.ptr)
    return float(ms.value)


@dataclass
class Result:
    phi: np.ndarray
    phi_rf: np.ndarray
    E_total: float
    E_rf: float


def solve(system, precision: int = HSMA_FP32, device: int = 0, **params) -> Result:
    """Convenience: one cavity system (inputs.System-like) -> potentials and energies."""
    prm = hsma_default_params(p=system.p, M=system.M, tau=getattr(system, "tau", 0.1), precision=precision,
                              device=device, **params)
    h = hsma_create(system.a, system.eps1, system.eps2, system.kappa, prm)
    hsma_build_sources(h, system.xyz, system.q)
    phi = hsma_potential(h, HSMA_TOTAL)
    phi_rf = hsma_potential(h, HSMA_REACTION)
    et, er = hsma_energy(h)
    hsma_destroy(h)
    return Result(phi, phi_rf, et, er)


PAPER_COULOMB_K = 1.0 / (4.0 * math.pi)
