"""Pins of the oracle's fields E = -grad phi (CPU only).

The field is the gradient, with the sources held fixed, of the potential the paper defines
(Sec. 2.4 source set: real charges, Kelvin images, monopole and dipole layers of the auxiliary
sphere).  It is pinned to things other than its own code:
  * the Kirkwood series (the exact reaction potential of Sec. 2.2), differentiated numerically,
    for charges well inside the cavity where the method reproduces it to ~1e-11;
  * the oracle's potential (itself pinned in test_oracle_pins), differentiated numerically term
    by term, for both dipole forms and for charges next to the interface;
  * Newton's third law for the Coulomb part, and the Coulomb field of two charges.
"""
import numpy as np
import pytest

import oracle
from paper_1907_01724_gb300 import inputs

from test_oracle_pins import K4PI, kirkwood_rf  # noqa: E402


def fd_gradient(f, x, h):
    """Fourth-order central difference of a scalar function of a 3-vector."""
    g = np.zeros(3)
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        g[k] = (-f(x + 2 * e) + 8 * f(x + e) - 8 * f(x - e) + f(x - 2 * e)) / (12 * h)
    return g


def fd_field_system(rng, n=10, a=1.0, near=3):
    """Charges for the numerical-gradient pins: some within 0.03a of the interface (but at least
    0.015a inside, so the stencil stays far from each charge's own image), the rest anywhere."""
    xyz = inputs.uniform_ball(rng, n, 0.95 * a)
    for i in range(near):
        v = rng.normal(size=3)
        xyz[i] = v / np.linalg.norm(v) * a * rng.uniform(0.97, 0.985)
    q = inputs.neutral_charges(rng, n) if n % 2 == 0 else rng.choice([-1.0, 1.0], size=n)
    return xyz, q


@pytest.mark.parametrize("kappa", [0.0, 1.5])
def test_reaction_field_is_minus_gradient_of_kirkwood(kappa):
    rng = np.random.default_rng(7)
    a, eps1, eps2 = 1.2, 1.0, 78.5
    P = oracle.make_params(a=a, eps1=eps1, eps2=eps2, kappa=kappa, p=24, M=1600, tau=0.1)
    xyz = inputs.uniform_ball(rng, 2, 0.6 * a)
    q = np.array([1.0, -1.0])
    E = oracle.field(P, xyz, q)["E_rf"]
    for i in range(2):
        def phi(x):
            return sum(q[j] * kirkwood_rf(x, xyz[j], a, eps1, eps2, kappa) for j in range(2))
        ref = -fd_gradient(phi, xyz[i], 1e-4)
        assert np.linalg.norm(E[i] - ref) <= 1e-9 * np.linalg.norm(ref), i


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("part", ["coul", "kelvin", "surface"])
def test_field_is_minus_gradient_of_potential(form, part):
    rng = np.random.default_rng(11)
    P = oracle.make_params(a=1.0, eps1=1.0, eps2=80.0, kappa=2.0, p=16, M=400, dipole_form=form)
    xyz, q = fd_field_system(rng)
    src = oracle.build_sources(P, xyz, q)
    ec, er = oracle.field_at(P, xyz, q, src, xyz, self_index=np.arange(len(q)), parts=(part,))
    E = ec + er
    h = 1e-4
    for i in range(len(q)):
        def phi(x):
            pc, pr = oracle.evaluate(P, xyz, q, src, x[None, :], self_index=[i], parts=(part,))
            return pc[0] + pr[0]
        ref = -fd_gradient(phi, xyz[i], h)
        assert np.linalg.norm(E[i] - ref) <= 1e-7 * np.linalg.norm(ref) + 1e-12, (i, part, form)


def test_dipole_forms_agree_for_the_field():
    rng = np.random.default_rng(5)
    xyz, q = fd_field_system(rng, n=16, near=6)
    f0 = oracle.field(oracle.make_params(p=16, M=400, dipole_form=0), xyz, q)["E_rf"]
    f1 = oracle.field(oracle.make_params(p=16, M=400, dipole_form=1), xyz, q)["E_rf"]
    assert np.linalg.norm(f0 - f1) <= 1e-9 * np.linalg.norm(f1)


def test_coulomb_field_newton_third_law_and_pair():
    rng = np.random.default_rng(2)
    P = oracle.make_params(p=8, M=400)
    xyz = inputs.uniform_ball(rng, 30, 1.0)
    q = rng.normal(size=30)
    Ec = oracle.field(P, xyz, q)["E_coul"]
    total = (q[:, None] * Ec).sum(axis=0)
    assert np.linalg.norm(total) <= 1e-13 * np.abs(q[:, None] * Ec).sum()
    # two charges: E at 0 is k q1 (x0 - x1)/|x0 - x1|^3 / eps1
    P2 = oracle.make_params(eps1=2.0, p=4, M=400)
    x2 = np.array([[0.1, -0.2, 0.3], [-0.4, 0.25, 0.05]])
    E2 = oracle.field(P2, x2, np.array([1.0, -3.0]))["E_coul"]
    d = x2[0] - x2[1]
    ref = K4PI / 2.0 * (-3.0) * d / np.linalg.norm(d) ** 3
    assert np.allclose(E2[0], ref, rtol=1e-14, atol=0)


def test_field_is_linear_in_the_charges():
    rng = np.random.default_rng(4)
    P = oracle.make_params(p=10, M=400)
    xyz = inputs.uniform_ball(rng, 12, 1.0)
    q1, q2 = rng.normal(size=12), rng.normal(size=12)
    E1 = oracle.field(P, xyz, q1)["E"]
    E2 = oracle.field(P, xyz, q2)["E"]
    E12 = oracle.field(P, xyz, 2.0 * q1 - 0.5 * q2)["E"]
    assert np.linalg.norm(E12 - (2.0 * E1 - 0.5 * E2)) <= 1e-12 * np.linalg.norm(E12)


def test_force_is_minus_energy_gradient_within_the_method():
    """q_k E(x_k) against -dE_total/dx_k by central differences of the whole method: they agree
    to the method's own accuracy (its discrete Green's function is symmetric only to truncation
    and quadrature, and the sources move with the charge), ~1e-4 here."""
    s = inputs.small_system()
    P = oracle.make_params(a=s.a, eps1=s.eps1, eps2=s.eps2, kappa=s.kappa, p=s.p, M=s.M, tau=s.tau)
    E = oracle.field(P, s.xyz, s.q)["E"]
    rng = np.random.default_rng(0)
    h = 1e-5
    for k in rng.choice(len(s.q), 3, replace=False):
        g = np.zeros(3)
        for d in range(3):
            xp = s.xyz.copy()
            xp[k, d] += h
            xm = s.xyz.copy()
            xm[k, d] -= h
            g[d] = -(oracle.hsma(P, xp, s.q)["E_total"] - oracle.hsma(P, xm, s.q)["E_total"]) / (2 * h)
        F = s.q[k] * E[k]
        assert np.linalg.norm(F - g) <= 2e-3 * np.linalg.norm(g), k
