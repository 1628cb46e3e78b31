"""Python binding of the batched C ABI (hsma_batch_* in include/hsma.h): argument marshalling only.

A Batch evaluates many independent cavities (uneven N) with the same kernels in single
launches; each system's results equal those of evaluating it alone.
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np

from . import _native
from .api import HSMA_FP32, HSMA_TOTAL, HsmaError, hsma_default_params


def _arr(x, dtype):
    return np.ascontiguousarray(np.asarray(x, dtype=dtype))


_p = _native.host_ptr


def _host_out(out, count: int) -> np.ndarray:
    """A writable C-contiguous float64 host array of count entries: out itself, or a new one."""
    if out is None:
        return np.empty(count, dtype=np.float64)
    if not (isinstance(out, np.ndarray) and out.dtype == np.float64 and out.flags.c_contiguous
            and out.flags.writeable and out.size == count):
        raise ValueError(f"out must be a writable C-contiguous float64 array of {count} entries")
    return out


def _is_torch_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and bool(getattr(x, "is_cuda"))


class Batch:
    """hsma_batch_t with a PyTorch-allocated workspace."""

    def __init__(self, a, eps1, eps2, kappa, params=None, max_requests: int = 1, use_torch_workspace: bool = True):
        self.lib = _native.load()
        self.params = params if params is not None else hsma_default_params()
        self.nsys = len(a)
        # keep every array alive across the call (ctypes holds only the addresses)
        self._a = _arr(a, np.float64)
        self._eps1 = _arr(eps1, np.float64)
        self._eps2 = _arr(eps2, np.float64)
        self._kappa = _arr(kappa, np.float64)
        out = ctypes.c_void_p()
        rc = self.lib.hsma_batch_create(self.nsys, _p(self._a), _p(self._eps1), _p(self._eps2), _p(self._kappa),
                                        ctypes.byref(self.params), ctypes.byref(out))
        if rc:
            raise HsmaError(rc, "hsma_batch_create")
        self.ptr = out
        self.use_torch_workspace = use_torch_workspace
        self.workspace = None
        self.n = None
        self._ntot = 0
        if max_requests != 1:
            self.hsma_batch_set_max_requests(max_requests)

    def __del__(self):
        try:
            if self.ptr:
                self.lib.hsma_batch_destroy(self.ptr)
                self.ptr = None
        except Exception:
            pass

    def _check(self, rc):
        if rc:
            raise HsmaError(rc, self.lib.hsma_batch_last_error(self.ptr).decode())

    # --- C entry points ---------------------------------------------------------------
    def hsma_batch_destroy(self):
        if self.ptr:
            self.lib.hsma_batch_destroy(self.ptr)
            self.ptr = None

    def hsma_batch_set_max_requests(self, m: int):
        self._check(self.lib.hsma_batch_set_max_requests(self.ptr, int(m)))

    def hsma_batch_workspace_size(self, n) -> int:
        n = _arr(n, np.int64)
        b = ctypes.c_size_t()
        self._check(self.lib.hsma_batch_workspace_size(self.ptr, _p(n), ctypes.byref(b)))
        return int(b.value)

    def _ensure_workspace(self, n):
        if not self.use_torch_workspace:
            return
        key = tuple(n.tolist())
        if getattr(self, "_ws_key", None) == key:
            return
        need = self.hsma_batch_workspace_size(n)
        self._ws_key = key
        if self.workspace is None or self.workspace.numel() < need:
            import torch
            t = torch.empty(need + need // 4 + 256, dtype=torch.uint8, device=f"cuda:{self.params.device}")
            off = (-t.data_ptr()) % 256
            self.workspace = t[off:]
            self._check(self.lib.hsma_batch_attach_workspace(self.ptr, ctypes.c_void_p(self.workspace.data_ptr()),
                                                             ctypes.c_size_t(self.workspace.numel())))

    def _ptr(self, slot, a):
        cache = self.__dict__.setdefault("_ptrs", {})
        return _native.cached_ptr(cache, slot, a)

    def hsma_batch_build_sources(self, n, xyz, q):
        n = _arr(n, np.int64)
        self._ensure_workspace(n)
        if _is_torch_cuda(xyz):
            import torch
            x = xyz.to(torch.float64).contiguous()
            qq = q.to(torch.float64).contiguous()
            self._keep = (x, qq)
            self._check(self.lib.hsma_batch_build_sources_device(self.ptr, _p(n), ctypes.c_void_p(x.data_ptr()),
                                                                 ctypes.c_void_p(qq.data_ptr())))
        else:
            x = _arr(xyz, np.float64)
            if x.ndim != 2:
                x = x.reshape(-1, 3)
            qq = _arr(q, np.float64)
            self._keep = (x, qq)  # page-locked arrays are read by the next evaluation
            self._check(self.lib.hsma_batch_build_sources(self.ptr, self._ptr("n", n), self._ptr("xyz", x),
                                                          self._ptr("q", qq)))
        self.n = n
        self._ntot = int(n.sum())

    def hsma_batch_potential(self, what: int = HSMA_TOTAL, out=None):
        """Potentials of all charges: into out (a torch CUDA tensor, or a float64 numpy array of
        sum n entries, written by the device itself when it is page-locked), else a new array."""
        if out is not None and _is_torch_cuda(out):
            self._check(self.lib.hsma_batch_potential_device(self.ptr, ctypes.c_void_p(out.data_ptr()), int(what)))
            return out
        phi = _host_out(out, self._ntot)
        self._check(self.lib.hsma_batch_potential(self.ptr, self._ptr("phi", phi), int(what)))
        return phi

    def hsma_batch_set_overlap(self, on: bool):
        self._check(self.lib.hsma_batch_set_overlap(self.ptr, 1 if on else 0))

    def hsma_batch_field(self, what: int = HSMA_TOTAL, out=None):
        if out is not None and _is_torch_cuda(out):
            self._check(self.lib.hsma_batch_field_device(self.ptr, ctypes.c_void_p(out.data_ptr()), int(what)))
            return out
        E = np.empty((self._ntot, 3), dtype=np.float64)
        self._check(self.lib.hsma_batch_field(self.ptr, _p(E), int(what)))
        return E

    def hsma_batch_energy(self):
        # (E_total, E_rf) rows of one reused buffer (its two addresses computed once); the caller
        # gets copies
        buf = self.__dict__.get("_ebuf")
        if buf is None or buf[0].shape[1] != self.nsys:
            e = np.empty((2, self.nsys))
            p = _p(e).value
            buf = (e, ctypes.c_void_p(p), ctypes.c_void_p(p + 8 * self.nsys))
            self._ebuf = buf
        e, p0, p1 = buf
        self._check(self.lib.hsma_batch_energy(self.ptr, p0, p1))
        return e[0].copy(), e[1].copy()

    def hsma_batch_delta_energy(self, sys, k, x_new):
        sys = _arr(sys, np.int32)
        k = _arr(k, np.int64)
        x = _arr(x_new, np.float64).reshape(-1, 3)
        de = np.empty(len(sys))
        self._check(self.lib.hsma_batch_delta_energy(self.ptr, len(sys), _p(sys), _p(k), _p(x), _p(de)))
        return de

    def hsma_batch_apply_moves(self, sys, k, x_new):
        sys = _arr(sys, np.int32)
        k = _arr(k, np.int64)
        x = _arr(x_new, np.float64).reshape(-1, 3)
        self._check(self.lib.hsma_batch_apply_moves(self.ptr, len(sys), _p(sys), _p(k), _p(x)))

    def hsma_batch_kernel_launches(self) -> int:
        return int(self.lib.hsma_batch_kernel_launches(self.ptr))

    def hsma_batch_last_pair_time(self) -> float:
        ms = ctypes.c_float()
        self._check(self.lib.hsma_batch_last_pair_time(self.ptr, ctypes.byref(ms)))
        return float(ms.value)

    def hsma_batch_set_pair_config(self, cfg: int):
        self._check(self.lib.hsma_batch_set_pair_config(self.ptr, int(cfg)))

    def hsma_batch_set_pair_schedule(self, mode: int):
        self._check(self.lib.hsma_batch_set_pair_schedule(self.ptr, int(mode)))

    def hsma_batch_pair_schedule(self) -> int:
        mode = ctypes.c_int()
        self._check(self.lib.hsma_batch_pair_schedule(self.ptr, ctypes.byref(mode)))
        return int(mode.value)

    def hsma_batch_autotune(self, reps: int = 5):
        best = ctypes.c_int()
        ms = ctypes.c_float()
        self._check(self.lib.hsma_batch_autotune(self.ptr, int(reps), ctypes.byref(best), ctypes.byref(ms)))
        return int(best.value), float(ms.value)


def pair_configs() -> list[tuple[int, int, int]]:
    """(CTA threads, targets per thread, pair items per CTA slot) of every configuration."""
    lib = _native.load()
    out = []
    for i in range(lib.hsma_pair_config_count()):
        t, k, m = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        lib.hsma_pair_config_info(i, ctypes.byref(t), ctypes.byref(k), ctypes.byref(m))
        out.append((t.value, k.value, m.value))
    return out


def from_systems(systems, precision: int = HSMA_FP32, device: int = 0, stream=None, max_requests: int = 1,
                 **params) -> Batch:
    """A Batch for a list of inputs.System-like objects sharing p, M and tau."""
    s0 = systems[0]
    prm = hsma_default_params(p=s0.p, M=s0.M, tau=s0.tau, precision=precision, device=device,
                              stream=stream, **params)
    return Batch([s.a for s in systems], [s.eps1 for s in systems], [s.eps2 for s in systems],
                 [s.kappa for s in systems], prm, max_requests=max_requests)


def concat(systems):
    n = np.array([s.n for s in systems], dtype=np.int64)
    xyz = np.concatenate([s.xyz for s in systems]) if len(systems) else np.zeros((0, 3))
    q = np.concatenate([s.q for s in systems]) if len(systems) else np.zeros(0)
    return n, xyz, q


class TuneCache:
    """Autotuned pair configuration per (size class, GPU name), kept in a JSON file."""

    def __init__(self, path: str | None = None):
        self.path = path or os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")
        try:
            self.data = json.load(open(self.path))
        except Exception:
            self.data = {}

    @staticmethod
    def key(n, gpu: str, params=None) -> str:
        """Size class (number of systems, log2 of the total charge count) and everything else that
        changes the pair work of a step: the truncation order, the quadrature (M, F1, F2), the
        precision, and the library's set of tile configurations."""
        tot = int(np.sum(n))
        ncfg = _native.load().hsma_pair_config_count()
        k = f"{gpu}|ncfg={ncfg}|step|nsys={len(n)}|log2N={max(tot, 1).bit_length()}"
        if params is not None:
            k += f"|p={params.p}|M={params.M}|F={params.F1},{params.F2}|prec={params.precision}"
        return k

    def get(self, n, gpu: str, params=None):
        return self.data.get(self.key(n, gpu, params))

    def put(self, n, gpu: str, cfg: int, ms: float, params=None, schedule: int = -1):
        self.data[self.key(n, gpu, params)] = {"cfg": int(cfg), "ms": float(ms), "schedule": int(schedule)}
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        tmp = self.path + f".{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(self.data, f, indent=1)
        os.replace(tmp, self.path)


def autotuned(batch: Batch, n, xyz, q, gpu: str = "", reps: int = 5, cache: TuneCache | None = None) -> int:
    """Build, then use the cached tile configuration and pair schedule for this size class or
    autotune and cache them."""
    cache = cache or TuneCache()
    hit = cache.get(n, gpu, batch.params)
    if hit is not None:
        batch.hsma_batch_set_pair_config(hit["cfg"])
        batch.hsma_batch_set_pair_schedule(hit.get("schedule", -1))
        batch.hsma_batch_build_sources(n, xyz, q)
        return hit["cfg"]
    batch.hsma_batch_build_sources(n, xyz, q)
    cfg, ms = batch.hsma_batch_autotune(reps)
    batch.hsma_batch_set_pair_config(cfg)
    batch.hsma_batch_build_sources(n, xyz, q)
    cache.put(n, gpu, cfg, ms, batch.params, schedule=batch.hsma_batch_pair_schedule())
    return cfg
