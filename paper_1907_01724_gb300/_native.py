"""Build and load the CUDA library (libhsma.so) in-tree.

The library is compiled with nvcc for sm_103a only (``-gencode arch=compute_103a,code=sm_103a``)
into ``paper_1907_01724_gb300/_build/`` and loaded with ctypes.  There is no CPU fallback:
if the library cannot be built or loaded, every entry point raises.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import shutil
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
CSRC = os.path.join(_HERE, "csrc")
INCLUDE = os.path.join(_ROOT, "include")
BUILD = os.path.join(_HERE, "_build")
LIB = os.path.join(BUILD, "libhsma.so")
SOURCES = ["k_order.cu", "k_sources.cu", "k_pairs.cu", "k_reduce.cu", "k_field.cu", "k_delta.cu", "engine.cu", "batch.cu", "server.cu", "noalloc.cu", "k_tree.cu"]
HEADERS = ["hsma_internal.cuh", "engine.h", "df64.cuh", "k_pairs_f32.cuh", "pair_work.cuh", "fp32_pair.cuh", "tree.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden"]
LINK_FLAGS = ["-Xlinker", "--exclude-libs,ALL", "-Xcompiler", "-fPIC"]

_lock = threading.Lock()
_lib = None



def host_ptr(a) -> ctypes.c_void_p:
    """Address of a host array's data as a ctypes argument.  A writable buffer's address comes
    from a ctypes view of it (a fraction of the cost of ndarray.ctypes, which matters on the
    per-call path); read-only and empty arrays take ndarray.ctypes."""
    try:
        return ctypes.c_void_p(ctypes.addressof(ctypes.c_char.from_buffer(a)))
    except (TypeError, ValueError, BufferError):
        return ctypes.c_void_p(a.ctypes.data)

def cached_ptr(cache: dict, slot: str, a) -> ctypes.c_void_p:
    """host_ptr(a), remembered per call slot while the caller passes the same array object again
    (a per-step loop's inputs and outputs): the cache keeps a reference to the array, which also
    keeps numpy from resizing it in place under the remembered address."""
    ent = cache.get(slot)
    if ent is not None and ent[0] is a:
        return ent[1]
    ptr = host_ptr(a)
    cache[slot] = (a, ptr)
    return ptr


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the HSMA CUDA library cannot be built")


def _sources():
    return [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]


def _digest() -> str:
    h = hashlib.sha256()
    for name in _sources() + HEADERS:
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode() + f.read())
    with open(os.path.join(INCLUDE, "hsma.h"), "rb") as f:
        h.update(f.read())
    h.update(" ".join(ARCH + NVCC_FLAGS + LINK_FLAGS).encode())
    return h.hexdigest()[:16]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit in parallel and link libhsma.so (idempotent)."""
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "stamp")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == dig:
        return LIB
    nvcc = _nvcc()
    procs = []
    objs = []
    for src in _sources():
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, "-I", INCLUDE, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errs = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errs.append(f"{src}:\n{out.decode(errors='replace')}")
    if errs:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errs))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, *LINK_FLAGS]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(dig)
    return LIB


class HsmaParams(ctypes.Structure):
    _fields_ = [
        ("p", ctypes.c_int),
        ("M", ctypes.c_int),
        ("F1", ctypes.c_int),
        ("F2", ctypes.c_int),
        ("tau", ctypes.c_double),
        ("dy_rel", ctypes.c_double),
        ("coulomb_k", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("device", ctypes.c_int),
        ("stream", ctypes.c_void_p),
    ]


def _declare(lib):
    vp, dp, i64, sz = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.c_size_t
    pp = ctypes.POINTER(HsmaParams)
    sigs = {
        "hsma_version": (ctypes.c_char_p, []),
        "hsma_default_params": (ctypes.c_int, [pp]),
        "hsma_create": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, pp,
                                       ctypes.POINTER(vp)]),
        "hsma_destroy": (None, [vp]),
        "hsma_last_error": (ctypes.c_char_p, [vp]),
        "hsma_workspace_size": (ctypes.c_int, [vp, i64, ctypes.POINTER(sz)]),
        "hsma_attach_workspace": (ctypes.c_int, [vp, vp, sz]),
        "hsma_build_sources": (ctypes.c_int, [vp, i64, vp, vp]),
        "hsma_build_sources_device": (ctypes.c_int, [vp, i64, vp, vp]),
        "hsma_potential": (ctypes.c_int, [vp, vp, ctypes.c_int]),
        "hsma_potential_device": (ctypes.c_int, [vp, vp, ctypes.c_int]),
        "hsma_field": (ctypes.c_int, [vp, vp, ctypes.c_int]),
        "hsma_field_device": (ctypes.c_int, [vp, vp, ctypes.c_int]),
        "hsma_energy": (ctypes.c_int, [vp, dp, dp]),
        "hsma_delta_energy": (ctypes.c_int, [vp, i64, vp, dp]),
        "hsma_apply_move": (ctypes.c_int, [vp, i64, vp]),
        "hsma_kernel_launches": (ctypes.c_int64, [vp]),
        "hsma_set_overlap": (ctypes.c_int, [vp, ctypes.c_int]),
        "hsma_last_pair_time": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_float)]),
        "hsma_set_far_field": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_int]),
        "hsma_last_far_time": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_float)]),
        "hsma_coefficients": (ctypes.c_int, [vp, vp, i64]),
        "hsma_batch_create": (ctypes.c_int, [ctypes.c_int, vp, vp, vp, vp, pp, ctypes.POINTER(vp)]),
        "hsma_batch_destroy": (None, [vp]),
        "hsma_batch_last_error": (ctypes.c_char_p, [vp]),
        "hsma_batch_workspace_size": (ctypes.c_int, [vp, vp, ctypes.POINTER(sz)]),
        "hsma_batch_attach_workspace": (ctypes.c_int, [vp, vp, sz]),
        "hsma_batch_set_max_requests": (ctypes.c_int, [vp, ctypes.c_int]),
        "hsma_batch_build_sources": (ctypes.c_int, [vp, vp, vp, vp]),
        "hsma_batch_build_sources_device": (ctypes.c_int, [vp, vp, vp, vp]),
        "hsma_batch_potential": (ctypes.c_int, [vp, vp, ctypes.c_int]),
        "hsma_batch_potential_device": (ctypes.c_int, [vp, vp, ctypes.c_int]),
        "hsma_batch_field": (ctypes.c_int, [vp, vp, ctypes.c_int]),
        "hsma_batch_field_device": (ctypes.c_int, [vp, vp, ctypes.c_int]),
        "hsma_batch_energy": (ctypes.c_int, [vp, vp, vp]),
        "hsma_batch_delta_energy": (ctypes.c_int, [vp, ctypes.c_int, vp, vp, vp, vp]),
        "hsma_batch_apply_moves": (ctypes.c_int, [vp, ctypes.c_int, vp, vp, vp]),
        "hsma_batch_kernel_launches": (ctypes.c_int64, [vp]),
        "hsma_batch_set_overlap": (ctypes.c_int, [vp, ctypes.c_int]),
        "hsma_batch_set_pair_schedule": (ctypes.c_int, [vp, ctypes.c_int]),
        "hsma_batch_pair_schedule": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int)]),
        "hsma_batch_last_pair_time": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_float)]),
        "hsma_pair_config_count": (ctypes.c_int, []),
        "hsma_pair_config_info": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                                  ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
        "hsma_batch_set_pair_config": (ctypes.c_int, [vp, ctypes.c_int]),
        "hsma_batch_autotune": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                               ctypes.POINTER(ctypes.c_float)]),
        "hsma_coulomb_potential_noalloc": (ctypes.c_int, [i64, vp, vp, ctypes.c_double, vp, vp]),
        "hsma_server_create": (ctypes.c_int, [ctypes.c_int, vp, vp, vp, vp, pp, sz, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_double, ctypes.POINTER(vp)]),
        "hsma_server_destroy": (None, [vp]),
        "hsma_server_last_error": (ctypes.c_char_p, [vp]),
        "hsma_server_load": (ctypes.c_int, [vp, vp, vp, vp, ctypes.POINTER(ctypes.c_int)]),
        "hsma_server_close_chain": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
        "hsma_server_run": (ctypes.c_int, [vp, ctypes.c_int, vp, vp]),
        "hsma_server_start": (ctypes.c_int, [vp]),
        "hsma_server_submit": (ctypes.c_int, [vp, vp, ctypes.POINTER(i64)]),
        "hsma_server_poll": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_int)]),
        "hsma_server_stop": (ctypes.c_int, [vp, ctypes.c_int]),
        "hsma_server_positions": (ctypes.c_int, [vp, ctypes.c_int, vp, i64]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    extra = getattr(_declare, "extra", None)
    if extra:
        extra(lib)
    return lib


def load():
    """Build (if needed) and load libhsma.so; raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            _lib = _declare(ctypes.CDLL(path))
    return _lib


def exported_symbols(path: str | None = None) -> set[str]:
    """Dynamic symbols defined by the built library (via nm -D)."""
    path = path or build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], stdout=subprocess.PIPE, check=True).stdout.decode()
    return {line.split()[-1] for line in out.splitlines() if line.strip()}
