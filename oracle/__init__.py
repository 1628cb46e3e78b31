"""FP64 CPU oracle of the harmonic surface mapping algorithm (arXiv:1907.01724).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` leg are the only users.  The product path (the CUDA
library and its binding) never imports this package, and this package imports
nothing from the product path.

The arithmetic lives in ``hsma_oracle.c`` (plain C, FP64, no SIMD intrinsics,
OpenMP over independent targets only); this module compiles it with gcc on first
use and wraps it with ctypes and numpy.  Each wrapper names the section of the
paper it follows.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hsma_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


class OracleParams(ctypes.Structure):
    _fields_ = [
        ("a", ctypes.c_double),
        ("eps1", ctypes.c_double),
        ("eps2", ctypes.c_double),
        ("kappa", ctypes.c_double),
        ("p", ctypes.c_int),
        ("F1", ctypes.c_int),
        ("F2", ctypes.c_int),
        ("tau", ctypes.c_double),
        ("dy_rel", ctypes.c_double),
        ("coulomb_k", ctypes.c_double),
        ("dipole_form", ctypes.c_int),
        ("nthreads", ctypes.c_int),
        ("image_rel", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            dp = ctypes.POINTER(ctypes.c_double)
            i64p = ctypes.POINTER(ctypes.c_int64)
            pp = ctypes.POINTER(OracleParams)
            lib.oracle_Sn.restype = ctypes.c_double
            lib.oracle_Sn.argtypes = [ctypes.c_int, ctypes.c_double]
            lib.oracle_Mn.restype = ctypes.c_double
            lib.oracle_Mn.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
            lib.oracle_decomposition.restype = None
            lib.oracle_decomposition.argtypes = [ctypes.c_double, ctypes.c_double, dp, dp, dp]
            lib.oracle_fibonacci.restype = ctypes.c_int
            lib.oracle_fibonacci.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp]
            lib.oracle_build.restype = ctypes.c_int
            lib.oracle_build.argtypes = [pp, ctypes.c_int64, dp, dp, dp, dp, dp, dp, dp, dp, dp]
            lib.oracle_eval.restype = ctypes.c_int
            lib.oracle_eval.argtypes = [pp, ctypes.c_int64, dp, dp, dp, dp, ctypes.c_int64, dp, dp, dp, dp,
                                        ctypes.c_double, ctypes.c_int64, dp, i64p, dp, dp]
            lib.oracle_field.restype = ctypes.c_int
            lib.oracle_field.argtypes = [pp, ctypes.c_int64, dp, dp, dp, dp, ctypes.c_int64, dp, dp, dp, dp,
                                         ctypes.c_int64, dp, i64p, dp, dp]
            lib.oracle_energy.restype = ctypes.c_int
            lib.oracle_energy.argtypes = [ctypes.c_int64, dp, dp, dp, dp, dp]
            lib.oracle_hsma.restype = ctypes.c_int
            lib.oracle_hsma.argtypes = [pp, ctypes.c_int64, dp, dp, dp, dp, dp, dp]
            lib.oracle_threads.restype = ctypes.c_int
            lib.oracle_threads.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


class using_library:
    """Context manager that points this module at another build of the oracle source
    (used by the mutation test, which compiles copies with planted mistakes)."""

    def __init__(self, path):
        self.path = path
        self.saved = None

    def __enter__(self):
        global _lib
        _load()
        self.saved = _lib
        lib = ctypes.CDLL(self.path)
        for name in ("oracle_Sn", "oracle_Mn", "oracle_decomposition", "oracle_fibonacci", "oracle_build",
                     "oracle_eval", "oracle_field", "oracle_energy", "oracle_hsma", "oracle_threads"):
            f, g = getattr(lib, name), getattr(self.saved, name)
            f.restype, f.argtypes = g.restype, g.argtypes
        _lib = lib
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def compile_variant(src_text: str, out_path: str) -> str:
    """Compile oracle C source text (e.g. a planted-mistake copy) to a shared library."""
    c_path = out_path + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", out_path, c_path,
                    "-lm"], check=True)
    return out_path


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _dptr(arr):
    if arr is None:
        return None
    return arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(x, shape=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def fibonacci_pair(M: int) -> tuple[int, int]:
    """(F1, F2) for M points per shell: M = 2(F2+1), F1 = round(F2 (sqrt5-1)/2).

    This reproduces the paper's pairs 987/1597 and 4181/6765 (Sec. 4)."""
    if M < 4 or M % 2:
        raise ValueError("M must be even and >= 4")
    F2 = M // 2 - 1
    F1 = int(round(F2 * (math.sqrt(5.0) - 1.0) / 2.0))
    return F1, F2


def make_params(a=1.0, eps1=1.0, eps2=80.0, kappa=1.0, p=20, M=None, F1=None, F2=None, tau=0.1,
                dy_rel=1e-5, coulomb_k=1.0 / (4.0 * math.pi), dipole_form=1, nthreads=0,
                image_rel=0.0) -> OracleParams:
    if F2 is None:
        if M is None:
            M = 400
        F1, F2 = fibonacci_pair(M)
    elif F1 is None:
        F1 = int(round(F2 * (math.sqrt(5.0) - 1.0) / 2.0))
    return OracleParams(float(a), float(eps1), float(eps2), float(kappa), int(p), int(F1), int(F2),
                        float(tau), float(dy_rel), float(coulomb_k), int(dipole_form), int(nthreads),
                        float(image_rel))


def S_n(n: int, mu: float) -> float:
    """S_n(mu) = k_n/(mu k_n') from the finite sum for k_n (Sec. 2.2)."""
    return _load().oracle_Sn(int(n), float(mu))


def M_n(n: int, eps: float, mu: float) -> float:
    """Kirkwood coefficient M_n (eq. Anuapp1), eps = eps1/eps2, mu = kappa R."""
    return _load().oracle_Mn(int(n), float(eps), float(mu))


def decomposition(eps: float, mu: float) -> tuple[float, float, float]:
    """(gamma, sigma, dbar) of Sec. 2.3."""
    g, s, d = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _load().oracle_decomposition(float(eps), float(mu), ctypes.byref(g), ctypes.byref(s), ctypes.byref(d))
    return g.value, s.value, d.value


def fibonacci(F1: int, F2: int, R: float):
    """Fibonacci points (2(F2+1), 3) on the sphere of radius R and weights (Sec. 2.4)."""
    m = 2 * (F2 + 1)
    pts = np.zeros((m, 3))
    w = np.zeros(m)
    rc = _load().oracle_fibonacci(int(F1), int(F2), float(R), _dptr(pts), _dptr(w))
    if rc:
        raise ValueError("bad Fibonacci pair")
    return pts, w


def build_sources(P: OracleParams, xyz, q):
    """Kelvin images, surface points/weights and Phi_corr, dPhi_corr/dr there (Sec. 2.4)."""
    xyz = _f64(xyz, (-1, 3))
    q = _f64(q)
    n = len(q)
    M = 2 * (P.F2 + 1)
    out = dict(
        kel_xyz=np.zeros((n, 3)), kel_q=np.zeros(n), surf_xyz=np.zeros((M, 3)), surf_w=np.zeros(M),
        surf_phi=np.zeros(M), surf_dphi=np.zeros(M),
    )
    c0 = ctypes.c_double()
    _load().oracle_build(ctypes.byref(P), n, _dptr(xyz), _dptr(q), _dptr(out["kel_xyz"]), _dptr(out["kel_q"]),
                         _dptr(out["surf_xyz"]), _dptr(out["surf_w"]), _dptr(out["surf_phi"]),
                         _dptr(out["surf_dphi"]), ctypes.byref(c0))
    out["r0_const"] = c0.value
    return out


def evaluate(P: OracleParams, xyz, q, src, targets, self_index=None, parts=("coul", "kelvin", "surface")):
    """Coulomb and reaction potentials at target points from a source set (eq. phirffinall)."""
    xyz = _f64(xyz, (-1, 3)) if xyz is not None else None
    q = _f64(q) if q is not None else None
    targets = _f64(targets, (-1, 3))
    nt = len(targets)
    n = len(q) if q is not None else 0
    pc = np.zeros(nt)
    pr = np.zeros(nt)
    si = None
    if self_index is not None:
        si = np.ascontiguousarray(np.asarray(self_index, dtype=np.int64))
    use_c = "coul" in parts
    use_k = "kelvin" in parts
    use_s = "surface" in parts
    M = len(src["surf_w"]) if (use_s and src is not None) else 0
    _load().oracle_eval(
        ctypes.byref(P), n,
        _dptr(xyz) if use_c else None, _dptr(q) if use_c else None,
        _dptr(src["kel_xyz"]) if use_k else None, _dptr(src["kel_q"]) if use_k else None,
        M,
        _dptr(src["surf_xyz"]) if use_s else None, _dptr(src["surf_w"]) if use_s else None,
        _dptr(src["surf_phi"]) if use_s else None, _dptr(src["surf_dphi"]) if use_s else None,
        float(src["r0_const"]) if use_k else 0.0,
        nt, _dptr(targets), si.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)) if si is not None else None,
        _dptr(pc), _dptr(pr))
    return pc, pr


def field_at(P: OracleParams, xyz, q, src, targets, self_index=None, parts=("coul", "kelvin", "surface")):
    """Coulomb and reaction fields E = -grad phi at target points from a source set (the
    gradient of every term of `evaluate`, sources fixed).  Returns two (nt, 3) arrays."""
    xyz = _f64(xyz, (-1, 3)) if xyz is not None else None
    q = _f64(q) if q is not None else None
    targets = _f64(targets, (-1, 3))
    nt = len(targets)
    n = len(q) if q is not None else 0
    ec = np.zeros((nt, 3))
    er = np.zeros((nt, 3))
    si = None
    if self_index is not None:
        si = np.ascontiguousarray(np.asarray(self_index, dtype=np.int64))
    use_c = "coul" in parts
    use_k = "kelvin" in parts
    use_s = "surface" in parts
    M = len(src["surf_w"]) if (use_s and src is not None) else 0
    _load().oracle_field(
        ctypes.byref(P), n,
        _dptr(xyz) if use_c else None, _dptr(q) if use_c else None,
        _dptr(src["kel_xyz"]) if use_k else None, _dptr(src["kel_q"]) if use_k else None,
        M,
        _dptr(src["surf_xyz"]) if use_s else None, _dptr(src["surf_w"]) if use_s else None,
        _dptr(src["surf_phi"]) if use_s else None, _dptr(src["surf_dphi"]) if use_s else None,
        nt, _dptr(targets), si.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)) if si is not None else None,
        _dptr(ec), _dptr(er))
    return ec, er


def field(P: OracleParams, xyz, q):
    """Whole method, fields at the charges (own Coulomb term excluded): dict(E_coul, E_rf, E)."""
    xyz = _f64(xyz, (-1, 3))
    q = _f64(q)
    src = build_sources(P, xyz, q)
    ec, er = field_at(P, xyz, q, src, xyz, self_index=np.arange(len(q)))
    return dict(E_coul=ec, E_rf=er, E=ec + er)


def energy(q, phi_coul, phi_rf):
    """(E_total, E_RF) = 1/2 sum q (phi_coul + phi_rf), 1/2 sum q phi_rf (Neumaier sums)."""
    q = _f64(q)
    pc = _f64(phi_coul)
    pr = _f64(phi_rf)
    et, er = ctypes.c_double(), ctypes.c_double()
    _load().oracle_energy(len(q), _dptr(q), _dptr(pc), _dptr(pr), ctypes.byref(et), ctypes.byref(er))
    return et.value, er.value


def hsma(P: OracleParams, xyz, q):
    """Whole method at the charges: dict(phi_coul, phi_rf, phi, E_total, E_rf)."""
    xyz = _f64(xyz, (-1, 3))
    q = _f64(q)
    n = len(q)
    pc = np.zeros(n)
    pr = np.zeros(n)
    et, er = ctypes.c_double(), ctypes.c_double()
    _load().oracle_hsma(ctypes.byref(P), n, _dptr(xyz), _dptr(q), _dptr(pc), _dptr(pr), ctypes.byref(et),
                        ctypes.byref(er))
    return dict(phi_coul=pc, phi_rf=pr, phi=pc + pr, E_total=et.value, E_rf=er.value)


def self_energy(P: OracleParams, x_s, q=1.0) -> float:
    """E_self = Phi_RF(x_s, x_s)/2 for a single charge (Sec. 4.1)."""
    r = hsma(P, np.asarray(x_s, dtype=np.float64).reshape(1, 3), np.array([q]))
    return r["E_rf"] / q if q != 1.0 else r["E_rf"]


def delta_energy(P: OracleParams, xyz, q, k: int, x_new):
    """E(after moving charge k to x_new) - E(before), both by the whole method."""
    xyz = _f64(xyz, (-1, 3)).copy()
    e0 = hsma(P, xyz, q)["E_total"]
    xyz[k] = np.asarray(x_new, dtype=np.float64)
    e1 = hsma(P, xyz, q)["E_total"]
    return e1 - e0


def threads(requested: int = 0) -> int:
    return _load().oracle_threads(int(requested))
