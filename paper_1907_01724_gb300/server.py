"""Python binding of the serving C ABI (hsma_server_* in include/hsma.h): marshalling only,
plus a seeded trace generator for Monte Carlo request streams."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native
from .api import HSMA_FP32, HsmaError, hsma_default_params
from .inputs import ServingWorkload, uniform_ball

REQ_DELTA = 0
REQ_ENERGY = 1

REQUEST = np.dtype([("t_arrival", "f8"), ("chain", "i4"), ("kind", "i4"), ("accept", "i4"), ("pad", "i4"),
                    ("k", "i8"), ("x", "f8", 3), ("id", "i8")], align=True)
RESULT = np.dtype([("id", "i8"), ("status", "i4"), ("chain", "i4"), ("value", "f8"), ("t_arrival", "f8"),
                   ("t_done", "f8"), ("ticket", "i8")], align=True)
assert REQUEST.itemsize == 64 and RESULT.itemsize == 48

HSMA_E_TIMEOUT = -6
HSMA_E_BUSY = -7


_p = _native.host_ptr


class Server:
    def __init__(self, chains, precision: int = HSMA_FP32, hbm_budget: int = 0, max_batch: int = 64,
                 energy_slots: int = 4, energy_sm_frac: float = 0.75, device: int = 0):
        self.lib = _native.load()
        s0 = chains[0]
        self.params = hsma_default_params(p=s0.p, M=s0.M, tau=s0.tau, precision=precision, device=device)
        self.chains = chains
        self._a = np.array([c.a for c in chains], dtype=np.float64)
        self._e1 = np.array([c.eps1 for c in chains], dtype=np.float64)
        self._e2 = np.array([c.eps2 for c in chains], dtype=np.float64)
        self._k = np.array([c.kappa for c in chains], dtype=np.float64)
        out = ctypes.c_void_p()
        rc = self.lib.hsma_server_create(len(chains), _p(self._a), _p(self._e1), _p(self._e2), _p(self._k),
                                         ctypes.byref(self.params), ctypes.c_size_t(int(hbm_budget)), int(max_batch),
                                         int(energy_slots), float(energy_sm_frac), ctypes.byref(out))
        if rc:
            raise HsmaError(rc, "hsma_server_create")
        self.ptr = out

    def _check(self, rc):
        if rc:
            raise HsmaError(rc, self.lib.hsma_server_last_error(self.ptr).decode())

    def __del__(self):
        try:
            if self.ptr:
                self.lib.hsma_server_destroy(self.ptr)
                self.ptr = None
        except Exception:
            pass

    def hsma_server_load(self) -> int:
        n = np.array([c.n for c in self.chains], dtype=np.int64)
        xyz = np.ascontiguousarray(np.concatenate([c.xyz for c in self.chains]), dtype=np.float64)
        q = np.ascontiguousarray(np.concatenate([c.q for c in self.chains]), dtype=np.float64)
        adm = ctypes.c_int()
        self._check(self.lib.hsma_server_load(self.ptr, _p(n), _p(xyz), _p(q), ctypes.byref(adm)))
        return adm.value

    def hsma_server_close_chain(self, c: int) -> int:
        adm = ctypes.c_int()
        self._check(self.lib.hsma_server_close_chain(self.ptr, int(c), ctypes.byref(adm)))
        return adm.value

    def hsma_server_run(self, reqs: np.ndarray) -> np.ndarray:
        reqs = np.ascontiguousarray(reqs, dtype=REQUEST)
        res = np.zeros(len(reqs), dtype=RESULT)
        self._check(self.lib.hsma_server_run(self.ptr, len(reqs), _p(reqs), _p(res)))
        return res

    def hsma_server_start(self):
        self._check(self.lib.hsma_server_start(self.ptr))

    def hsma_server_submit(self, req) -> int:
        """Submit one request (a REQUEST record); returns its ticket.  Raises HsmaError on a
        full queue (HSMA_E_BUSY) or a stopped loop (HSMA_E_STATE)."""
        r = np.ascontiguousarray(np.asarray(req, dtype=REQUEST).reshape(1))
        t = ctypes.c_int64()
        rc = self.lib.hsma_server_submit(self.ptr, _p(r), ctypes.byref(t))
        if rc:
            raise HsmaError(rc, "hsma_server_submit")
        return int(t.value)

    def hsma_server_poll(self, max_results: int = 256, timeout: float = 0.0) -> np.ndarray:
        """Answers available now (timeout 0) or within timeout seconds (an empty array when none
        came)."""
        out = np.zeros(max_results, dtype=RESULT)
        cnt = ctypes.c_int()
        rc = self.lib.hsma_server_poll(self.ptr, _p(out), int(max_results), float(timeout), ctypes.byref(cnt))
        if rc and rc != HSMA_E_TIMEOUT:
            raise HsmaError(rc, "hsma_server_poll")
        return out[:cnt.value]

    def hsma_server_stop(self, drain: bool = True):
        self._check(self.lib.hsma_server_stop(self.ptr, 1 if drain else 0))

    def hsma_server_positions(self, c: int) -> np.ndarray:
        n = self.chains[c].n
        out = np.empty((n, 3))
        self._check(self.lib.hsma_server_positions(self.ptr, int(c), _p(out), n))
        return out


def make_trace(workload: ServingWorkload, nreq: int, rate: float | None, positions=None):
    """Seeded request stream: Poisson arrivals at `rate` per second (None: all at t = 0), 90% moves
    (displacement uniform in a ball of radius 0.05a, redrawn until inside; accept with p = 0.5,
    independent of Delta E) and 10% full energies.  `positions` (default: the chains' initial
    ones) is where each chain stands when the trace starts.  Returns the requests and the
    positions each chain must end with."""
    pos = [p.copy() for p in positions] if positions is not None else [c.xyz.copy() for c in workload.chains]
    reqs = np.zeros(nreq, dtype=REQUEST)
    t = 0.0
    for i in range(nreq):
        if rate is not None:
            t += workload.interarrival(rate)
        r = workload.next_request(pos)
        reqs[i]["t_arrival"] = t
        reqs[i]["chain"] = r["chain"]
        reqs[i]["id"] = i
        if r["kind"] == "delta":
            reqs[i]["kind"] = REQ_DELTA
            reqs[i]["k"] = r["k"]
            reqs[i]["x"] = r["x_new"]
            reqs[i]["accept"] = int(r["accept"])
            if r["accept"]:
                pos[r["chain"]][r["k"]] = r["x_new"]
        else:
            reqs[i]["kind"] = REQ_ENERGY
    return reqs, pos


def latency_stats(res: np.ndarray, reqs: np.ndarray | None = None) -> dict:
    """p50/p99 latency and throughput of the answered requests; with the requests, also the
    latencies of the move and the full-energy requests apart."""
    ok = res["status"] == 0
    lat = (res["t_done"] - res["t_arrival"])[ok]
    span = float(res["t_done"][ok].max() - res["t_arrival"][ok].min()) if ok.any() else 0.0
    out = {"p50_ms": float(np.percentile(lat, 50) * 1e3) if lat.size else None,
           "p99_ms": float(np.percentile(lat, 99) * 1e3) if lat.size else None,
           "req_per_s": float(ok.sum() / span) if span > 0 else None, "answered": int(ok.sum())}
    if reqs is not None:
        for name, kind in (("delta", REQ_DELTA), ("energy", REQ_ENERGY)):
            m = ok & (reqs["kind"] == kind)
            lk = (res["t_done"] - res["t_arrival"])[m]
            out[name] = {"p50_ms": float(np.percentile(lk, 50) * 1e3) if lk.size else None,
                         "p99_ms": float(np.percentile(lk, 99) * 1e3) if lk.size else None, "answered": int(m.sum())}
    return out
