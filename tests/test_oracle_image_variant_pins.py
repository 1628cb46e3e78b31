"""Pins of the near-interface-only image variant (CPU only).

A charge with r_i < image_rel a gets no Kelvin (or line) image; its whole reaction potential is
the truncated harmonic series with the full Kirkwood coefficients M_n (Sec. 2.2-2.3: the image
terms capture the slowly converging part of the series, needed only for charges close to the
interface).  Pinned to the Kirkwood series (truncated at p, and converged), the Born / Debye-Hueckel
closed form at the centre, and to the paper's method where the variant does not apply.
"""
import numpy as np
import pytest

import oracle
from paper_1907_01724_gb300 import inputs

from test_oracle_pins import K4PI, _mn_ratio_recurrence, kirkwood_rf  # noqa: E402


def test_zero_threshold_is_the_papers_method():
    rng = np.random.default_rng(1)
    xyz = inputs.uniform_ball(rng, 40, 1.0)
    q = inputs.neutral_charges(rng, 40)
    r0 = oracle.hsma(oracle.make_params(p=12, M=400), xyz, q)
    r1 = oracle.hsma(oracle.make_params(p=12, M=400, image_rel=0.0), xyz, q)
    assert np.array_equal(r0["phi"], r1["phi"])


def test_no_images_reproduces_the_truncated_kirkwood_series():
    """Every charge below the threshold: phi_RF is the Kirkwood series truncated at n = p,
    evaluated through the surface images (quadrature error only)."""
    rng = np.random.default_rng(23)
    a, eps1, eps2, kappa, p = 1.1, 2.0, 80.0, 1.5, 10
    P = oracle.make_params(a=a, eps1=eps1, eps2=eps2, kappa=kappa, p=p, M=4000, tau=0.1, image_rel=0.7)
    xyz = inputs.uniform_ball(rng, 4, 0.55 * a)
    q = rng.standard_normal(4)
    r = oracle.hsma(P, xyz, q)
    src = oracle.build_sources(P, xyz, q)
    assert np.all(src["kel_q"] == 0.0) and src["r0_const"] == 0.0
    for i in range(4):
        ref = sum(q[j] * kirkwood_rf(xyz[i], xyz[j], a, eps1, eps2, kappa, nmax=p) for j in range(4))
        assert r["phi_rf"][i] == pytest.approx(ref, rel=1e-9, abs=1e-13)


@pytest.mark.parametrize("rs", [0.1, 0.25, 0.35])
def test_self_energy_without_image_within_the_truncation_bound(rs):
    """Against the converged Kirkwood series: the error is the dropped tail
    sum_{n > p} |M_n| (r_s^2/a^2)^n <= max|M_n| u^{p+1}/(1 - u), u = r_s^2/a^2."""
    p = 20
    P = oracle.make_params(a=1, eps1=2, eps2=80, kappa=5, p=p, F1=987, F2=1597, tau=0.1, image_rel=0.4)
    e = oracle.self_energy(P, [0.0, 0.0, rs])
    ref = 0.5 * kirkwood_rf([0, 0, rs], [0, 0, rs], 1.0, 2.0, 80.0, 5.0)
    Mn = _mn_ratio_recurrence(200, 2 / 80, 5.0)
    u = rs * rs
    bound = 0.5 * K4PI / 2.0 * max(abs(m) for m in Mn) * u ** (p + 1) / (1 - u)
    assert abs(e - ref) <= bound + 1e-12, (e, ref, bound)


@pytest.mark.parametrize("eps1,eps2,kappa", [(1.0, 80.0, 1.0), (2.0, 80.0, 5.0), (4.0, 4.0, 0.0)])
def test_centre_charge_without_image_is_born_debye_hueckel(eps1, eps2, kappa):
    P = oracle.make_params(a=1.3, eps1=eps1, eps2=eps2, kappa=kappa, p=6, M=400, image_rel=0.5)
    r = oracle.hsma(P, np.zeros((1, 3)), np.array([-1.5]))
    ref = 0.5 * 2.25 * K4PI / 1.3 * (1.0 / (eps2 * (1.0 + kappa * 1.3)) - 1.0 / eps1)
    assert r["E_rf"] == pytest.approx(ref, rel=1e-9, abs=1e-15)


def test_mixed_system_matches_the_papers_method_only_with_a_fine_quadrature():
    """Charges below 0.3a lose their images; their series tail at the other charges is below
    0.3^21.  What remains is the auxiliary-sphere quadrature of their larger series (M_n instead
    of the small hat M'_n): it decays with M (~2e-3 absolute at M = 1000, 4e-5 at 4000, 1e-8 at
    13532 for targets 0.02a from the interface), so the variant needs a much finer quadrature
    than the paper's method for the same accuracy near the interface."""
    rng = np.random.default_rng(5)
    xyz = inputs.uniform_ball(rng, 60, 1.0)
    q = inputs.neutral_charges(rng, 60)
    assert int(np.sum(np.linalg.norm(xyz, axis=1) < 0.3)) >= 1
    diffs = []
    for M in (1000, 13532):
        r_full = oracle.hsma(oracle.make_params(p=20, M=M), xyz, q)
        r_var = oracle.hsma(oracle.make_params(p=20, M=M, image_rel=0.3), xyz, q)
        diffs.append(np.max(np.abs(r_var["phi_rf"] - r_full["phi_rf"])))
    assert diffs[1] <= 1e-7
    assert diffs[0] > 1e3 * diffs[1]
