"""Plant plausible mistakes in a copy of the oracle (CPU only) and check that the pins catch each.

Every mutant is a one-token change of the kind a transcription of the paper could make:
a dropped term, a wrong sign, an index off by one, a transposed operand, a missing
normalisation.  The original oracle passes all checks; each mutant must fail at least one.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1907_01724_gb300 import inputs

from test_oracle_pins import K4PI, kirkwood_rf, _mn_ratio_recurrence  # noqa: E402
from test_oracle_field_pins import fd_field_system, fd_gradient  # noqa: E402

MUTANTS = {
    "dbar_sign": ("*dbar = g * (1.0 - s) - mu / (1.0 + eps);", "*dbar = g * (1.0 - s) + mu / (1.0 + eps);"),
    "trapezoid_dropped": ("gamma * rK + dbar * (Rtau - rK) / 2.0", "gamma * rK"),
    "legendre_index": ("(2.0 * n + 1.0) * t * Pn", "(2.0 * n + 3.0) * t * Pn"),
    "fibonacci_weight": ("2.0 * ORACLE_PI * R * R / (double)F2", "ORACLE_PI * R * R / (double)F2"),
    "fibonacci_theta": ("double c = z + sin(ORACLE_PI * z) / ORACLE_PI;", "double c = z;"),
    "dipole_sign": ("pr += surf_w[l] * surf_phi[l] * inv4pi * 2.0 * (Rtau - xy)",
                    "pr += surf_w[l] * surf_phi[l] * inv4pi * 2.0 * (xy - Rtau)"),
    "Mn_transposed": ("(eps * (double)(n + 1) * S + 1.0) / (eps * (double)n * S - 1.0)",
                      "(eps * (double)n * S + 1.0) / (eps * (double)(n + 1) * S - 1.0)"),
    "corr_missing_rK": ("dbar * (Rtau - rK) / (2.0 * rK)", "dbar * (Rtau - rK) / 2.0"),
    "Sn_sign": ("(mu + 1.0) * sigma0 + sigma1", "(mu + 1.0) * sigma0 - sigma1"),
    "monopole_4pi": ("surf_w[l] * surf_dphi[l] * inv4pi / d", "surf_w[l] * surf_dphi[l] / d"),
    "kelvin_point": ("double s = (a / r) * (a / r);", "double s = (a / r);"),
    "self_not_excluded": ("if (j == self) continue;", "if (j == self + 1) continue;"),
    "radial_derivative": ("(double)k * un / rho * Pn", "(double)(k + 1) * un / rho * Pn"),
    "centre_limit": ("q[i] / a * (gamma - 0.5 * dbar)", "q[i] / a * (gamma + 0.5 * dbar)"),
    "truncation_off_by_one": ("for (int k = 0; k <= p; ++k) {\n                    double Mhat",
                              "for (int k = 0; k < p; ++k) {\n                    double Mhat"),
    "tau_radius": ("const double Rtau = (1.0 + P->tau) * a;\n    const int p", "const double Rtau = (1.0 + P->tau);\n    const int p"),
    # fields
    "field_kelvin_sign": ("double c = kc * kel_q[j] / (d * d * d);", "double c = -kc * kel_q[j] / (d * d * d);"),
    "field_coul_index": ("double u[3] = {x[0] - xyz[3 * j], x[1] - xyz[3 * j + 1], x[2] - xyz[3 * j + 2]};",
                         "double u[3] = {x[0] - xyz[3 * j], x[1] - xyz[3 * j + 2], x[2] - xyz[3 * j + 1]};"),
    "field_monopole_power": ("double c = surf_w[l] * surf_dphi[l] * inv4pi / (d * d * d);",
                             "double c = surf_w[l] * surf_dphi[l] * inv4pi / (d * d);"),
    "field_dipole_literal_sign": ("er[k] += strength * (um[k] / (dm * dm * dm) - up[k] / (dp * dp * dp));",
                                  "er[k] += strength * (up[k] / (dp * dp * dp) - um[k] / (dm * dm * dm));"),
    "field_dipole_fused_shell": ("er[k] += D * (yh[k] / dm3 + up[k] * f);", "er[k] += D * (yh[k] / dp3 + up[k] * f);"),
    "field_dipole_fused_factor": ("double f = 2.0 * (Rtau - xy)", "double f = (Rtau - xy)"),
    # near-interface-only image variant
    "variant_corr_sign": ("double corr_i = no_image ? -gamma :", "double corr_i = no_image ? gamma :"),
    "variant_centre": ("phi += pref * (no_image ? Mn[0] : Mn[0] - gamma + 0.5 * dbar);",
                       "phi += pref * (no_image ? Mn[0] - gamma : Mn[0] - gamma + 0.5 * dbar);"),
}


def _checks():
    """A compact subset of the pins; returns the names of the failed checks."""
    failed = []
    # Born / Debye-Hueckel at the centre
    P = oracle.make_params(a=1.3, eps1=1.0, eps2=80.0, kappa=0.8, p=10, M=400)
    e = oracle.hsma(P, np.zeros((1, 3)), np.array([1.0]))["E_rf"]
    ref = 0.5 * K4PI / 1.3 * (1.0 / (80.0 * (1.0 + 0.8 * 1.3)) - 1.0)
    if not abs(e - ref) < 1e-9 * abs(ref):
        failed.append("born")
    # Kirkwood pair response, off axis, a != 1
    rng = np.random.default_rng(7)
    a, eps1, eps2, kappa = 1.2, 1.0, 78.5, 1.5
    P = oracle.make_params(a=a, eps1=eps1, eps2=eps2, kappa=kappa, p=24, M=1600, tau=0.1)
    xyz = inputs.uniform_ball(rng, 2, 0.6 * a)
    q = np.array([1.0, -1.0])
    r = oracle.hsma(P, xyz, q)
    for i in range(2):
        refi = sum(q[j] * kirkwood_rf(xyz[i], xyz[j], a, eps1, eps2, kappa) for j in range(2))
        if not abs(r["phi_rf"][i] - refi) < 1e-9 * abs(refi):
            failed.append("kirkwood_pair")
            break
        d = np.linalg.norm(xyz[0] - xyz[1])
        if not abs(r["phi_coul"][i] - K4PI * q[1 - i] / d) < 1e-13:
            failed.append("coulomb_pair")
            break
    # a charge near the interface against Kirkwood within the paper's printed level
    P = oracle.make_params(a=1, eps1=2, eps2=80, kappa=5, p=20, F1=987, F2=1597, tau=0.1)
    e = oracle.self_energy(P, [0, 0, 0.9])
    if not abs(e - 0.5 * kirkwood_rf([0, 0, 0.9], [0, 0, 0.9], 1.0, 2.0, 80.0, 5.0)) < 1e-5:
        failed.append("paper_A1")
    # the coefficient against the independent ratio recurrence
    Mr = _mn_ratio_recurrence(10, 1 / 80, 1.0)
    if not all(abs(oracle.M_n(n, 1 / 80, 1.0) - Mr[n]) < 1e-13 for n in range(11)):
        failed.append("Mn")
    # truncated series evaluated directly at the target (no surface), low order p = 4
    a, eps1, eps2, kappa, p = 1.0, 1.0, 80.0, 2.0, 4
    xs = np.array([0.2, -0.3, 0.35])
    P = oracle.make_params(a=a, eps1=eps1, eps2=eps2, kappa=kappa, p=p, M=4000, tau=0.1)
    phi = oracle.hsma(P, xs[None, :], np.array([1.0]))["phi_rf"][0]
    gam, sig, dbar = oracle.decomposition(eps1 / eps2, kappa * a)
    Mn = _mn_ratio_recurrence(p, eps1 / eps2, kappa * a)
    rs = np.linalg.norm(xs)
    rK = a * a / rs
    ref = K4PI / eps1 * (gam * rK + dbar * (1.1 - rK) / 2) / a / (rK - rs)
    ref += K4PI / (eps1 * a) * sum((Mn[m] - gam - dbar * (1.1 - rK) / (2 * rK)) * (rs / rK) ** m for m in range(p + 1))
    if not abs(phi - ref) < 1e-9 * abs(ref):
        failed.append("direct_series")
    # Fibonacci weights and second moment
    pts, w = oracle.fibonacci(123, 199, 1.1)
    if not (abs(w.sum() - 4 * math.pi * 1.21) < 1e-12 and
            abs((w * (pts[:, 2] / 1.1) ** 2).sum() - 4 * math.pi * 1.21 / 3) < 1e-6):
        failed.append("fibonacci")
    # fields: minus the numerical gradient of the (pinned) potential, both dipole forms, with
    # charges next to the interface; and the Kirkwood reaction field of a pair
    rng = np.random.default_rng(11)
    xyz, q = fd_field_system(rng, n=6, near=2)
    for form in (0, 1):
        P = oracle.make_params(a=1.0, eps1=1.0, eps2=80.0, kappa=2.0, p=12, M=400, dipole_form=form)
        src = oracle.build_sources(P, xyz, q)
        ec, er = oracle.field_at(P, xyz, q, src, xyz, self_index=np.arange(len(q)))
        ok = True
        for i in range(len(q)):
            def phi(x):
                pc, pr = oracle.evaluate(P, xyz, q, src, x[None, :], self_index=[i])
                return pc[0] + pr[0]
            ref = -fd_gradient(phi, xyz[i], 1e-4)
            ok = ok and np.linalg.norm(ec[i] + er[i] - ref) <= 1e-7 * np.linalg.norm(ref)
        if not ok:
            failed.append(f"field_fd_form{form}")
    a, eps1, eps2, kappa = 1.2, 1.0, 78.5, 1.5
    P = oracle.make_params(a=a, eps1=eps1, eps2=eps2, kappa=kappa, p=24, M=1600, tau=0.1)
    xyz = inputs.uniform_ball(np.random.default_rng(7), 2, 0.6 * a)
    q = np.array([1.0, -1.0])
    E = oracle.field(P, xyz, q)["E_rf"]
    ref = -fd_gradient(lambda x: sum(q[j] * kirkwood_rf(x, xyz[j], a, eps1, eps2, kappa) for j in range(2)),
                       xyz[0], 1e-4)
    if not np.linalg.norm(E[0] - ref) <= 1e-9 * np.linalg.norm(ref):
        failed.append("kirkwood_field")
    # near-interface-only images: a charge without image is the truncated Kirkwood series, and a
    # centre charge without image is Born / Debye-Hueckel
    P = oracle.make_params(a=1.1, eps1=2.0, eps2=80.0, kappa=1.5, p=10, M=4000, tau=0.1, image_rel=0.7)
    xyz = np.array([[0.1, -0.2, 0.3], [-0.25, 0.05, 0.2]])
    q = np.array([1.0, -0.5])
    r = oracle.hsma(P, xyz, q)
    ref = [sum(q[j] * kirkwood_rf(xyz[i], xyz[j], 1.1, 2.0, 80.0, 1.5, nmax=10) for j in range(2)) for i in range(2)]
    if not np.allclose(r["phi_rf"], ref, rtol=1e-9, atol=1e-13):
        failed.append("variant_series")
    P = oracle.make_params(a=1.3, eps1=2.0, eps2=80.0, kappa=5.0, p=6, M=400, image_rel=0.5)
    e = oracle.hsma(P, np.zeros((1, 3)), np.array([1.0]))["E_rf"]
    if not abs(e - 0.5 * K4PI / 1.3 * (1.0 / (80.0 * (1.0 + 6.5)) - 0.5)) < 1e-9 * abs(e):
        failed.append("variant_born")
    return failed


def test_original_oracle_passes_checks():
    assert _checks() == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = oracle.source_text()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    lib = oracle.compile_variant(src.replace(old, new), str(tmp_path / f"mut_{name}.so"))
    with oracle.using_library(lib):
        failed = _checks()
    assert failed, f"planted mistake {name} was not caught by any pin"
