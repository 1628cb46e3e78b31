"""Pointwise error records of the GPU parity tests.

The parity bar is norm-wise (||phi - phi_ref||_2 / ||phi_ref||_2); the pointwise errors are
reported beside it: max_i |phi_i - phi_ref,i| / |phi_ref,i| (ill-conditioned where a potential
nearly cancels) and max_i |phi_i - phi_ref,i| / max_j |phi_ref,j|.  conftest.py prints the
records at the end of the session.
"""
import numpy as np

RECORDS = []


def record_pointwise(label, prec, phi, phi_ref, normwise):
    phi = np.asarray(phi, dtype=np.float64)
    phi_ref = np.asarray(phi_ref, dtype=np.float64)
    if phi_ref.size == 0:
        return
    d = np.abs(phi - phi_ref)
    den = np.abs(phi_ref)
    with np.errstate(divide="ignore", invalid="ignore"):
        pt = np.where(den > 0, d / den, np.where(d > 0, np.inf, 0.0))
    RECORDS.append({"case": label, "prec": prec, "n": int(phi.size), "normwise": float(normwise),
                    "pointwise_rel_max": float(np.max(pt)),
                    "pointwise_abs_over_max": float(np.max(d) / max(float(np.max(den)), 1e-300))})
