"""Measurement script (calls only the FP64 oracle; test infrastructure, not part of the product):
would a per-system truncation order p below the configured one keep the 1e-6 error bound?

For systems drawn like the batched and the serving workloads (charges uniform in the cavity,
N log-uniform), it computes the potentials of the method at p = 4, 6, ..., p_cfg - 2 with the
system's own quadrature (M points) and compares each with the method at the configured p_cfg
(the result the FP32 path is held to within 1e-6).  It prints, per system, max r_i / a and the
smallest p whose norm-wise differences from the p_cfg result are within 1e-6 for the total
potential alone and for both the total and the reaction potential (the two the parity tests
bound), next to p_cfg; and, for context, the error of the p_cfg result itself against a converged
reference (p_cfg + 10 on 4 M quadrature points).  The truncated expansion converges like
(r_i r_j / R_tau^2)^n over the charge pairs (Sec. 2.3 and Sec. 3): a cavity whose charges reach
close to the interface needs the full order whatever its N.

    python oracle/study_adaptive_p.py [--systems 24] [--n-max 3000]
"""
import argparse
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
from paper_1907_01724_gb300 import inputs  # noqa: E402


def study(systems, p_cfg: int, tol: float = 1e-6):
    def rel(x, y):
        return np.linalg.norm(x - y) / np.linalg.norm(y)

    rows = []
    for s in systems:
        base = dict(a=s.a, eps1=s.eps1, eps2=s.eps2, kappa=s.kappa, tau=s.tau)
        cfg = oracle.hsma(oracle.make_params(p=p_cfg, M=s.M, **base), s.xyz, s.q)
        conv = oracle.hsma(oracle.make_params(p=p_cfg + 10, M=4 * s.M, **base), s.xyz, s.q)
        p_tot = p_both = p_cfg
        tot_ok = both_ok = True
        for p in range(p_cfg - 2, 2, -2):
            r = oracle.hsma(oracle.make_params(p=p, M=s.M, **base), s.xyz, s.q)
            tot_ok = tot_ok and rel(r["phi"], cfg["phi"]) <= tol
            both_ok = both_ok and tot_ok and rel(r["phi_rf"], cfg["phi_rf"]) <= tol
            if tot_ok:
                p_tot = p
            if both_ok:
                p_both = p
            if not tot_ok:
                break
        rmax = float(np.max(np.linalg.norm(s.xyz, axis=1)) / s.a)
        rows.append((s.name, s.n, s.eps1, s.kappa * s.a, rmax, p_tot, p_both, rel(cfg["phi"], conv["phi"])))
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--systems", type=int, default=24)
    ap.add_argument("--n-max", type=int, default=3000)
    args = ap.parse_args()
    batched = [s for s in inputs.batched_systems() if s.n <= args.n_max][: args.systems]
    serving = [s for s in inputs.serving_workload().chains if s.n <= args.n_max][: max(1, args.systems // 3)]
    for title, systems in (("batched", batched), ("serving", serving)):
        p_cfg = systems[0].p
        print(f"{title}: {len(systems)} systems with N <= {args.n_max}, configured p = {p_cfg}")
        print(f"{'system':>10} {'N':>6} {'eps1':>5} {'ka':>5} {'max r/a':>8} {'min p: phi':>11} "
              f"{'min p: phi, phi_rf':>19} {'p_cfg vs converged':>19}")
        for name, n, e1, ka, rmax, p_tot, p_both, e_conv in study(systems, p_cfg):
            print(f"{name:>10} {n:6d} {e1:5.1f} {ka:5.2f} {rmax:8.4f} {p_tot:11d} {p_both:19d} {e_conv:19.2e}")


if __name__ == "__main__":
    main()
