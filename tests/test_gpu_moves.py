"""Single-charge moves through the C ABI: hsma_delta_energy against the oracle's E(after) - E(before),
and hsma_apply_move against a full oracle evaluation of the moved configuration.

Delta E tolerance: |dE - dE_ref| <= tol (|dE_ref| + S) + 4e-16 (|E0| + |E1|), where
S = |q_k| (|phi_before(x_k)| + |phi_after(x')|) is the scale of the energy terms that change
and the last term is the rounding of the reference's own difference of two energies;
tol = 1e-6 (FP32 path), 1e-12 (FP64 path).
"""
import numpy as np
import pytest

import oracle
from paper_1907_01724_gb300 import api, inputs

pytestmark = pytest.mark.gpu

TOL = {api.HSMA_FP32: 1e-6, api.HSMA_FP64: 1e-12}


def P_of(s):
    return oracle.make_params(a=s.a, eps1=s.eps1, eps2=s.eps2, kappa=s.kappa, p=s.p, M=s.M, tau=s.tau)


def handle(s, prec):
    prm = api.hsma_default_params(p=s.p, M=s.M, tau=s.tau, precision=prec)
    h = api.hsma_create(s.a, s.eps1, s.eps2, s.kappa, prm)
    api.hsma_build_sources(h, s.xyz, s.q)
    return h


def check_delta(s, h, prec, k, x_new):
    P = P_of(s)
    r0 = oracle.hsma(P, s.xyz, s.q)
    xyz1 = s.xyz.copy()
    xyz1[k] = x_new
    r1 = oracle.hsma(P, xyz1, s.q)
    ref = r1["E_total"] - r0["E_total"]
    S = abs(s.q[k]) * (abs(r0["phi"][k]) + abs(r1["phi"][k]))
    de = api.hsma_delta_energy(h, k, x_new)
    bound = TOL[prec] * (abs(ref) + S) + 4e-16 * (abs(r0["E_total"]) + abs(r1["E_total"]))
    assert abs(de - ref) <= bound, (k, de, ref, abs(de - ref), bound)
    return de


@pytest.mark.parametrize("prec", [api.HSMA_FP32, api.HSMA_FP64])
def test_delta_energy_small_system(prec):
    s = inputs.small_system()
    h = handle(s, prec)
    rng = np.random.default_rng(5)
    for _ in range(6):
        k = int(rng.integers(s.n))
        x_new = s.xyz[k] + inputs.uniform_ball(rng, 1, 0.05 * s.a)[0]
        if np.linalg.norm(x_new) >= s.a:
            continue
        check_delta(s, h, prec, k, x_new)


@pytest.mark.parametrize("prec", [api.HSMA_FP32, api.HSMA_FP64])
def test_delta_energy_near_interface_and_centre(prec):
    s = inputs.near_interface_system(kappa_a=2.0, n=400)
    h = handle(s, prec)
    k_shell = int(np.argmax(np.linalg.norm(s.xyz, axis=1)))
    x = s.xyz[k_shell]
    check_delta(s, h, prec, k_shell, x / np.linalg.norm(x) * 0.99999)   # toward the interface
    check_delta(s, h, prec, k_shell, np.zeros(3))                        # to the centre
    check_delta(s, h, prec, 3, s.xyz[3] * 0.5)


@pytest.mark.parametrize("prec", [api.HSMA_FP32, api.HSMA_FP64])
def test_monte_carlo_chain_of_moves(prec):
    """Accepted moves are committed; the resident state must equal a fresh oracle evaluation."""
    s = inputs.near_interface_system(kappa_a=0.5, n=300)
    h = handle(s, prec)
    rng = np.random.default_rng(11)
    xyz = s.xyz.copy()
    e0, _ = api.hsma_energy(h)
    total = 0.0
    for step in range(25):
        k = int(rng.integers(s.n))
        while True:
            x_new = xyz[k] + inputs.uniform_ball(rng, 1, 0.05 * s.a)[0]
            if np.linalg.norm(x_new) < s.a:
                break
        de = api.hsma_delta_energy(h, k, x_new)
        if rng.random() < 0.5:
            api.hsma_apply_move(h, k, x_new)
            xyz[k] = x_new
            total += de
    ref = oracle.hsma(P_of(s), xyz, s.q)
    e1, er1 = api.hsma_energy(h)
    phi = api.hsma_potential(h)
    scale = max(abs(ref["E_total"]), 0.5 * np.sum(np.abs(s.q * ref["phi"])))
    assert abs(e1 - ref["E_total"]) <= TOL[prec] * scale * 4
    assert np.linalg.norm(phi - ref["phi"]) / np.linalg.norm(ref["phi"]) <= TOL[prec] * 4
    # the accepted Delta E add up to the change of the resident energy
    assert abs((e1 - e0) - total) <= TOL[prec] * scale * 4


def test_move_errors():
    s = inputs.small_system()
    h = handle(s, api.HSMA_FP32)
    with pytest.raises(api.HsmaError) as e:
        api.hsma_delta_energy(h, 0, [0.0, 0.0, 1.5])
    assert e.value.code == -2
    with pytest.raises(api.HsmaError) as e:
        api.hsma_delta_energy(h, s.n, [0.0, 0.0, 0.1])
    assert e.value.code == -1
    with pytest.raises(api.HsmaError) as e:
        api.hsma_apply_move(h, -1, [0.0, 0.0, 0.1])
    assert e.value.code == -1
