"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: exact rational
constants, special functions from an independent library (mpmath), the interface
conditions of the boundary-value problem, textbook closed forms (Born/Debye-Hueckel,
the Poisson image solution), the Kirkwood series, the accuracy levels the paper
prints, exact symmetries of the discrete scheme, Green's identity on harmonic
polynomials, and a direct (surface-free) evaluation of the same truncated series.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1907_01724_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")
K4PI = 1.0 / (4.0 * math.pi)


def _frac(pair):
    return Fraction(pair[0], pair[1])


# ----------------------------------------------------------------------------------------
# Sec. 2.2 / 2.3 coefficients
# ----------------------------------------------------------------------------------------

def test_rational_constants():
    g = json.load(open(os.path.join(GOLD, "rational_constants.json")))
    for c in g["cases"]:
        eps, mu = float(_frac(c["eps"])), float(_frac(c["mu"]))
        gam, sig, dbar = oracle.decomposition(eps, mu)
        assert gam == pytest.approx(float(_frac(c["gamma"])), abs=1e-15)
        assert sig == pytest.approx(float(_frac(c["sigma"])), rel=1e-15)
        assert dbar == pytest.approx(float(_frac(c["dbar"])), abs=1e-15)
    for mu in [0.0, 0.25, 1.0, 3.0, 17.0]:
        assert oracle.S_n(0, mu) == pytest.approx(-1.0 / (1.0 + mu), rel=1e-15)
        assert oracle.S_n(1, mu) == pytest.approx(-(1.0 + mu) / (2.0 + 2.0 * mu + mu * mu), rel=1e-15)


def _mp_S(n, mu):
    """S_n = k_n/(mu k_n') with k_n(x) = sqrt(pi/(2x)) K_{n+1/2}(x) from mpmath's Bessel K."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    nu = mp.mpf(n) + mp.mpf(1) / 2
    x = mp.mpf(mu)
    K = mp.besselk(nu, x)
    dK = -(mp.besselk(nu - 1, x) + mp.besselk(nu + 1, x)) / 2
    # mu k_n'/k_n = -1/2 + mu K'/K
    return float(1 / (-mp.mpf(1) / 2 + x * dK / K))


@pytest.mark.parametrize("mu", [0.1, 0.5, 1.0, 3.0, 5.0, 20.0])
def test_Sn_against_bessel_K(mu):
    for n in range(0, 41, 3):
        assert oracle.S_n(n, mu) == pytest.approx(_mp_S(n, mu), rel=1e-13)


@pytest.mark.parametrize("eps1,eps2,mu", [(1.0, 80.0, 1.0), (2.0, 80.0, 5.0), (78.5, 78.5, 3.0), (1.0, 78.5, 0.5)])
def test_Mn_satisfies_interface_conditions(eps1, eps2, mu):
    """Eq. Anm solves eq. boundarycondition: with Phi1_n = r_s^n/r^{n+1} + M_n r_s^n r^n/a^{2n+1}
    inside and Phi2_n = C k_n(kappa r) outside, continuity of Phi fixes C and continuity of
    eps dPhi/dr demands eps1(-(n+1) + n M_n) = eps2 (1 + M_n) mu k_n'(mu)/k_n(mu) (a = 1)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    eps = eps1 / eps2
    for n in range(0, 31, 2):
        Mn = oracle.M_n(n, eps, mu)
        nu = mp.mpf(n) + mp.mpf(1) / 2
        x = mp.mpf(mu)
        K = mp.besselk(nu, x)
        dK = -(mp.besselk(nu - 1, x) + mp.besselk(nu + 1, x)) / 2
        log_deriv = float(-mp.mpf(1) / 2 + x * dK / K)  # mu k_n'/k_n
        lhs = eps1 * (-(n + 1) + n * Mn)
        rhs = eps2 * (1.0 + Mn) * log_deriv
        assert lhs == pytest.approx(rhs, rel=1e-12, abs=1e-12 * eps2)


def test_Mn_poisson_dielectric_sphere():
    """kappa = 0: the textbook reaction-field coefficient of a dielectric sphere,
    (n+1)(eps1-eps2)/(eps1 n + eps2 (n+1)); and hat M_n vanishes identically."""
    for eps1, eps2 in [(1.0, 80.0), (2.0, 80.0), (78.5, 1.0)]:
        eps = eps1 / eps2
        gam, sig, dbar = oracle.decomposition(eps, 0.0)
        for n in range(0, 60):
            ref = (n + 1) * (eps1 - eps2) / (eps1 * n + eps2 * (n + 1))
            Mn = oracle.M_n(n, eps, 0.0)
            assert Mn == pytest.approx(ref, rel=1e-14, abs=1e-15)
            assert Mn - gam - dbar / (n + sig) == pytest.approx(0.0, abs=1e-14)


def test_Mn_large_n_limit_and_no_jump():
    """M_n -> gamma as n grows (the Kelvin image); eps1 = eps2 with kappa = 0 gives M_n = 0."""
    gam, _, _ = oracle.decomposition(1 / 80, 2.0)
    assert oracle.M_n(400, 1 / 80, 2.0) == pytest.approx(gam, abs=5e-3)
    for n in range(0, 40):
        assert oracle.M_n(n, 1.0, 0.0) == 0.0


# ----------------------------------------------------------------------------------------
# Quadrature (Sec. 2.4)
# ----------------------------------------------------------------------------------------

@pytest.mark.parametrize("F1,F2,R", [(123, 199, 1.1), (987, 1597, 1.1), (308, 499, 2.0)])
def test_fibonacci_rule(F1, F2, R):
    pts, w = oracle.fibonacci(F1, F2, R)
    assert pts.shape == (2 * (F2 + 1), 3)
    assert np.allclose(np.linalg.norm(pts, axis=1), R, rtol=1e-14)
    assert w.sum() == pytest.approx(4 * math.pi * R * R, rel=1e-13)
    z = pts[:, 2] / R
    assert (w * z * z).sum() == pytest.approx(4 * math.pi * R * R / 3, rel=1e-6)
    assert (w * pts[:, 0] * pts[:, 1]).sum() == pytest.approx(0.0, abs=1e-8)
    # the lattice is invariant under rotations by pi about the coordinate axes
    key = lambda P: np.round(P, 9)
    s = {tuple(v) for v in key(pts)}
    for flip in ([1, -1, -1], [-1, 1, -1], [-1, -1, 1]):
        t = {tuple(v) for v in key(pts * np.array(flip))}
        assert s == t


# ----------------------------------------------------------------------------------------
# Whole method, single charges
# ----------------------------------------------------------------------------------------

@pytest.mark.parametrize("eps1,eps2,kappa,a", [(1.0, 80.0, 1.0, 1.0), (2.0, 80.0, 5.0, 1.0), (78.5, 78.5, 3.0, 1.3),
                                               (1.0, 78.5, 0.0, 0.8)])
@pytest.mark.parametrize("form", [0, 1])
def test_born_debye_huckel_centre(eps1, eps2, kappa, a, form):
    """A charge at the centre: E_RF = q^2 k/(2a) (1/(eps2(1+kappa a)) - 1/eps1)."""
    P = oracle.make_params(a=a, eps1=eps1, eps2=eps2, kappa=kappa, p=10, M=400, dipole_form=form)
    for q in (1.0, -2.5):
        r = oracle.hsma(P, np.zeros((1, 3)), np.array([q]))
        mu = kappa * a
        ref = 0.5 * q * q * K4PI / a * (1.0 / (eps2 * (1.0 + mu)) - 1.0 / eps1)
        assert r["E_rf"] == pytest.approx(ref, rel=1e-9, abs=1e-15)
        assert r["phi_coul"][0] == 0.0


def _mn_ratio_recurrence(nmax, eps, mu):
    """M_n for n = 0..nmax from the upward ratio recurrence of K_{nu}: with
    t_n = mu k_{n-1}(mu)/k_n(mu), t_0 = mu, t_{n+1} = mu^2/(t_n + 2n + 1), mu k_n'/k_n = -(n+1) - t_n.
    (A route independent of the paper's finite sum; checked against mpmath below.)"""
    out = np.empty(nmax + 1)
    t = mu
    for n in range(nmax + 1):
        S = -1.0 / (n + 1 + t)
        out[n] = (eps * (n + 1) * S + 1.0) / (eps * n * S - 1.0)
        t = mu * mu / (t + 2 * n + 1)
    return out


def test_ratio_recurrence_matches_mpmath():
    eps, mu = 2 / 80, 5.0
    Mr = _mn_ratio_recurrence(40, eps, mu)
    for n in (0, 1, 7, 20, 40):
        S = _mp_S(n, mu)
        ref = (eps * (n + 1) * S + 1.0) / (eps * n * S - 1.0)
        assert Mr[n] == pytest.approx(ref, rel=1e-13)


def kirkwood_rf(x, xs, a, eps1, eps2, kappa, nmax=None, k=K4PI):
    """Kirkwood series for the reaction potential at x of a unit charge at xs (Sec. 2.2, eq. Anm
    with the addition theorem): k/(eps1 a) sum_n M_n (r r_s/a^2)^n P_n(cos angle)."""
    x, xs = np.asarray(x, float), np.asarray(xs, float)
    r, rs = np.linalg.norm(x), np.linalg.norm(xs)
    u = r * rs / (a * a)
    c = 1.0 if (r == 0 or rs == 0) else float(np.dot(x, xs) / (r * rs))
    if nmax is None:
        nmax = 5 if u == 0 else int(math.log(1e-19) / math.log(u)) + 10
    M = _mn_ratio_recurrence(nmax, eps1 / eps2, kappa * a)
    tot, P0, P1 = 0.0, 1.0, c
    un = 1.0
    for n in range(nmax + 1):
        Pn = P0 if n == 0 else P1
        tot += M[n] * un * Pn
        if n >= 1:
            P0, P1 = P1, ((2 * n + 1) * c * P1 - n * P0) / (n + 1)
        un *= u
    return k / (eps1 * a) * tot


@pytest.mark.parametrize("rs", [0.0, 0.2, 0.5, 0.7])
def test_self_energy_matches_kirkwood_deep_inside(rs):
    P = oracle.make_params(a=1, eps1=2, eps2=80, kappa=5, p=20, F1=987, F2=1597, tau=0.1)
    e = oracle.self_energy(P, [0.0, 0.0, rs])
    ref = 0.5 * kirkwood_rf([0, 0, rs], [0, 0, rs], 1.0, 2.0, 80.0, 5.0)
    # truncation bound of Sec. 3 (a): the dropped tail of the correction series,
    # |hat M'_n| <= |gamma| + |dbar| + |M_n|, times u^{p+1}/(1-u), u = r_s^2
    u = rs * rs
    gam, _, dbar = oracle.decomposition(2 / 80, 5.0)
    bound = 0.5 * K4PI / 2.0 * 2 * (abs(gam) + abs(dbar) + 1.0) * u ** 21 / (1 - u)
    assert abs(e - ref) < bound + 1e-13


def test_pair_green_function_matches_kirkwood():
    """Two charges: phi_rf at each is the Kirkwood response to both (off-axis, general angles)."""
    rng = np.random.default_rng(7)
    a, eps1, eps2, kappa = 1.2, 1.0, 78.5, 1.5
    P = oracle.make_params(a=a, eps1=eps1, eps2=eps2, kappa=kappa, p=24, M=1600, tau=0.1)
    xyz = inputs.uniform_ball(rng, 2, 0.6 * a)
    q = np.array([1.0, -1.0])
    r = oracle.hsma(P, xyz, q)
    for i in range(2):
        ref = sum(q[j] * kirkwood_rf(xyz[i], xyz[j], a, eps1, eps2, kappa) for j in range(2))
        assert r["phi_rf"][i] == pytest.approx(ref, rel=1e-9)
        d = np.linalg.norm(xyz[0] - xyz[1])
        assert r["phi_coul"][i] == pytest.approx(K4PI / eps1 * q[1 - i] / d, rel=1e-14)


# ----------------------------------------------------------------------------------------
# The paper's printed accuracy levels (Sec. 4.1, 4.2)
# ----------------------------------------------------------------------------------------

def _gold():
    return json.load(open(os.path.join(GOLD, "paper_accuracy.json")))


def _paper_P(p, F2, tau, F1=None):
    return oracle.make_params(a=1, eps1=2, eps2=80, kappa=5, p=p, F2=F2, F1=F1, tau=tau)


def _kirk_self(rs, nmax=None):
    return 0.5 * kirkwood_rf([0, 0, rs], [0, 0, rs], 1.0, 2.0, 80.0, 5.0, nmax=nmax)


def test_paper_A1_error_below_1e5_inside_093():
    g = _gold()["A1"]
    P = _paper_P(g["p"], g["F2"], g["tau"], g["F1"])
    for rs in g["r_s"]:
        err = abs(oracle.self_energy(P, [0, 0, rs]) - _kirk_self(rs))
        assert err < g["abs_err_below"], (rs, err)


def test_paper_A2_error_near_interface_order_1e4():
    g = _gold()["A2"]
    for tau in g["taus"]:
        P = _paper_P(g["p"], g["F2"], tau)
        err = abs(oracle.self_energy(P, [0, 0, g["r_s"]]) - _kirk_self(g["r_s"]))
        assert err < 2 * g["abs_err_order"], (tau, err)
        assert err > g["abs_err_order"] / 100, (tau, err)


def test_paper_A3_five_digits_at_p55():
    g = _gold()["A3"]
    P = _paper_P(g["p"], g["F2"], g["tau"])
    ref = _kirk_self(g["r_s"])
    rel = abs(oracle.self_energy(P, [0, 0, g["r_s"]]) - ref) / abs(ref)
    assert rel < 10.0 ** (-g["rel_err_digits"] + 0.5), rel
    # and a lower order does not reach five digits
    P40 = _paper_P(40, g["F2"], g["tau"])
    assert abs(oracle.self_energy(P40, [0, 0, g["r_s"]]) - ref) / abs(ref) > 1e-5


def test_paper_A5_A6_hsma_beats_kirkwood():
    g5, g6 = _gold()["A5"], _gold()["A6"]
    P = _paper_P(g5["p_hsma"], g5["F2"], g5["tau"])
    for rs in g5["r_s"]:
        ref = _kirk_self(rs)
        e_h = abs(oracle.self_energy(P, [0, 0, rs]) - ref)
        e_k40 = abs(_kirk_self(rs, nmax=g5["p_kirkwood"]) - ref)
        e_k60 = abs(_kirk_self(rs, nmax=g6["p_kirkwood"]) - ref)
        assert e_h < e_k40, (rs, e_h, e_k40)
        assert e_h < g6["abs_err_below"], (rs, e_h)
    # Kirkwood at p = 60 fails the 1e-2 bound somewhere in the range
    assert max(abs(_kirk_self(rs, nmax=60) - _kirk_self(rs)) for rs in g6["r_s"]) > g6["abs_err_below"]


# ----------------------------------------------------------------------------------------
# Closed forms of special cases
# ----------------------------------------------------------------------------------------

def test_poisson_case_is_kelvin_plus_line_image():
    """kappa = 0: hat M_n = 0 and Phi_RF is the Kelvin image plus the line image of eq. Phihybrid,
    a one-dimensional integral evaluated here with scipy's adaptive quadrature."""
    from scipy.integrate import quad
    a, eps1, eps2 = 1.0, 1.0, 80.0
    eps = eps1 / eps2
    gam, sig, dbar = oracle.decomposition(eps, 0.0)
    xs = np.array([0.1, -0.2, 0.4])
    x = np.array([-0.3, 0.25, 0.1])
    rs = np.linalg.norm(xs)
    rK = a * a / rs
    e = xs / rs
    kel = gam * rK / np.linalg.norm(x - rK * e)
    line, _ = quad(lambda t: dbar * (t / rK) ** (-sig) / np.linalg.norm(x - t * e), rK, np.inf,
                   epsabs=1e-15, epsrel=1e-13, limit=400)
    ref = K4PI / (eps1 * a) * (kel + line)
    P = oracle.make_params(a=a, eps1=eps1, eps2=eps2, kappa=0.0, p=30, M=2000)
    src = oracle.build_sources(P, xs[None, :], np.array([1.0]))
    _, pr = oracle.evaluate(P, xs[None, :], np.array([1.0]), src, x[None, :])
    assert pr[0] == pytest.approx(ref, rel=1e-9)


def test_no_dielectric_jump_no_screening_gives_zero_reaction():
    rng = np.random.default_rng(3)
    xyz = inputs.uniform_ball(rng, 40, 1.0)
    q = inputs.neutral_charges(rng, 40)
    P = oracle.make_params(a=1.0, eps1=5.0, eps2=5.0, kappa=0.0, p=12, M=200)
    r = oracle.hsma(P, xyz, q)
    assert np.all(r["phi_rf"] == 0.0)
    d = np.linalg.norm(xyz[:, None, :] - xyz[None, :, :], axis=2)
    np.fill_diagonal(d, np.inf)
    e_ref = 0.5 * np.sum(q[:, None] * q[None, :] / d) * K4PI / 5.0
    assert r["E_total"] == pytest.approx(e_ref, rel=1e-13)


# ----------------------------------------------------------------------------------------
# Structure of the discrete scheme
# ----------------------------------------------------------------------------------------

def _sys(n=24, seed=11, a=1.0, rmax=0.97):
    rng = np.random.default_rng(seed)
    return inputs.uniform_ball(rng, n, rmax * a), inputs.neutral_charges(rng, n)


def test_linearity_in_charges():
    xyz, q = _sys()
    P = oracle.make_params(a=1.0, eps1=1.0, eps2=80.0, kappa=1.0, p=16, M=400)
    rng = np.random.default_rng(5)
    q1 = rng.standard_normal(len(q))
    q2 = rng.standard_normal(len(q))
    r1 = oracle.hsma(P, xyz, q1)
    r2 = oracle.hsma(P, xyz, q2)
    r12 = oracle.hsma(P, xyz, 2.0 * q1 - 0.5 * q2)
    scale = np.abs(r1["phi"]).max() + np.abs(r2["phi"]).max()
    assert np.allclose(r12["phi_rf"], 2.0 * r1["phi_rf"] - 0.5 * r2["phi_rf"], atol=1e-13 * scale)
    assert np.allclose(r12["phi_coul"], 2.0 * r1["phi_coul"] - 0.5 * r2["phi_coul"], atol=1e-13 * scale)


def test_c2_axis_rotations_are_exact_symmetries():
    xyz, q = _sys(30, seed=13)
    P = oracle.make_params(a=1.0, eps1=1.0, eps2=80.0, kappa=1.0, p=20, M=400)
    e0 = oracle.hsma(P, xyz, q)["E_total"]
    for flip in ([1, -1, -1], [-1, 1, -1], [-1, -1, 1]):
        e1 = oracle.hsma(P, xyz * np.array(flip), q)["E_total"]
        assert e1 == pytest.approx(e0, rel=1e-12)


def test_general_rotation_and_reciprocity_within_truncation():
    xyz, q = _sys(20, seed=17, rmax=0.8)
    P = oracle.make_params(a=1.0, eps1=1.0, eps2=80.0, kappa=1.0, p=30, M=2000)
    th = 0.7
    Rz = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, math.cos(1.1), -math.sin(1.1)], [0, math.sin(1.1), math.cos(1.1)]])
    R = Rz @ Rx
    r0 = oracle.hsma(P, xyz, q)
    r1 = oracle.hsma(P, xyz @ R.T, q)
    assert r1["E_rf"] == pytest.approx(r0["E_rf"], rel=1e-8)
    # G_RF(x, y) = G_RF(y, x)
    x, y = xyz[0], xyz[1]
    src_y = oracle.build_sources(P, y[None, :], np.array([1.0]))
    src_x = oracle.build_sources(P, x[None, :], np.array([1.0]))
    _, gxy = oracle.evaluate(P, y[None, :], np.array([1.0]), src_y, x[None, :])
    _, gyx = oracle.evaluate(P, x[None, :], np.array([1.0]), src_x, y[None, :])
    assert gxy[0] == pytest.approx(gyx[0], rel=1e-8)


@pytest.mark.parametrize("M,rmax,tol", [(400, 0.5, 1e-7), (2000, 0.7, 1e-9), (8000, 0.9, 1e-9)])
def test_green_identity_reproduces_harmonic_polynomials(M, rmax, tol):
    """Feed the surface step a known harmonic function h (values and radial derivative on the
    auxiliary sphere); the monopole + dipole layers must reproduce h inside (eq. GreenSecond)."""
    P = oracle.make_params(a=1.0, eps1=1.0, eps2=80.0, kappa=1.0, p=4, M=M, tau=0.1)
    Rt = 1.1
    F1, F2 = oracle.fibonacci_pair(M)
    pts, w = oracle.fibonacci(F1, F2, Rt)

    def h(X):  # degree-3 harmonic polynomial plus lower terms
        x, y, z = X[..., 0], X[..., 1], X[..., 2]
        return x * y * z + 0.3 * (x * x - y * y) + 0.7 * z - 0.2

    def dh_dr(X):
        x, y, z = X[..., 0], X[..., 1], X[..., 2]
        r = np.linalg.norm(X, axis=-1)
        return (3 * x * y * z + 0.3 * 2 * (x * x - y * y) + 0.7 * z) / r

    src = dict(kel_xyz=np.zeros((0, 3)), kel_q=np.zeros(0), surf_xyz=pts, surf_w=w, surf_phi=h(pts),
               surf_dphi=dh_dr(pts), r0_const=0.0)
    rng = np.random.default_rng(19)
    tg = inputs.uniform_ball(rng, 50, rmax)
    _, pr = oracle.evaluate(P, None, None, src, tg, parts=("surface",))
    # quadrature error grows toward the auxiliary sphere and falls fast with M (Sec. 3 (c));
    # the floor ~1e-11 is the central difference with dy = 1e-5 R_tau (Sec. 3 (b))
    assert np.max(np.abs(pr - h(tg))) < tol


def test_surface_route_equals_direct_series():
    """The discrete surface images must reproduce the truncated correction series evaluated
    directly at the targets (Sec. 2.4), up to quadrature and central-difference error."""
    rng = np.random.default_rng(23)
    for n in (1, 2, 3, 5):
        a, eps1, eps2, kappa, p = 1.0, 1.0, 80.0, 2.0, 12
        xyz = inputs.uniform_ball(rng, n, 0.6)
        q = rng.standard_normal(n)
        P = oracle.make_params(a=a, eps1=eps1, eps2=eps2, kappa=kappa, p=p, M=4000, tau=0.1)
        r = oracle.hsma(P, xyz, q)
        eps, mu = eps1 / eps2, kappa * a
        gam, sig, dbar = oracle.decomposition(eps, mu)
        Rt = 1.1 * a
        Mn = _mn_ratio_recurrence(p, eps, mu)
        ref = np.zeros(n)
        for i in range(n):
            for j in range(n):
                rj = np.linalg.norm(xyz[j])
                rK = a * a / rj
                e = xyz[j] / rj
                qK = q[j] / a * (gam * rK + dbar * (Rt - rK) / 2)
                ref[i] += K4PI / eps1 * qK / np.linalg.norm(xyz[i] - rK * e)
                ri = np.linalg.norm(xyz[i])
                c = float(np.dot(xyz[i], e) / ri)
                u = ri / rK
                P0, P1, s = 1.0, c, 0.0
                for m in range(p + 1):
                    Pm = P0 if m == 0 else P1
                    s += (Mn[m] - gam - dbar * (Rt - rK) / (2 * rK)) * u ** m * Pm
                    if m >= 1:
                        P0, P1 = P1, ((2 * m + 1) * c * P1 - m * P0) / (m + 1)
                ref[i] += K4PI * q[j] / (eps1 * a) * s
        assert np.allclose(r["phi_rf"], ref, rtol=1e-9, atol=1e-12)


def test_dipole_forms_agree():
    xyz, q = _sys(16, seed=29)
    r0 = oracle.hsma(oracle.make_params(p=16, M=400, dipole_form=0), xyz, q)
    r1 = oracle.hsma(oracle.make_params(p=16, M=400, dipole_form=1), xyz, q)
    scale = np.linalg.norm(r1["phi_rf"])
    assert np.linalg.norm(r0["phi_rf"] - r1["phi_rf"]) / scale < 1e-9


def test_delta_energy_is_energy_difference():
    xyz, q = _sys(12, seed=31)
    P = oracle.make_params(p=12, M=400)
    x_new = xyz[3] * 0.5 + np.array([0.01, 0.02, -0.03])
    de = oracle.delta_energy(P, xyz, q, 3, x_new)
    xyz2 = xyz.copy()
    xyz2[3] = x_new
    assert de == pytest.approx(oracle.hsma(P, xyz2, q)["E_total"] - oracle.hsma(P, xyz, q)["E_total"], rel=1e-14)
