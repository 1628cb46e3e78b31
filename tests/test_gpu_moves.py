"""Single-charge moves through the C ABI: hsma_delta_energy against the oracle's E(after) - E(before),
and hsma_apply_move against a full oracle evaluation of the moved configuration.

Delta E tolerance: |dE - dE_ref| <= tol (|dE_ref| + S) + 4e-16 (|E0| + |E1|), where S is the sum
of the absolute values of the energy terms that the move changes (S = |q_k| (A(x') + A(x_k)) +
sum_{j != k} |q_j| (|K'_k(x_j)| + |K_k(x_j)|), A(x) the potential at x of the other charges, all
Kelvin images and the surface images with every strength replaced by its absolute value, K_k the
potential of k's Kelvin image before and K'_k after the move): dE is a difference of sums whose
terms cancel, and each term carries its own rounding, so their absolute sum is the scale the
error is relative to.  The last term is the rounding of the reference's own difference of two
energies.  tol = 1e-6 (FP32 path), 1e-12 (FP64 path).
"""
import numpy as np
import pytest

import oracle
from paper_1907_01724_gb300 import api, inputs

pytestmark = pytest.mark.gpu

TOL = {api.HSMA_FP32: 1e-6, api.HSMA_FP64: 1e-12}


def P_of(s):
    return oracle.make_params(a=s.a, eps1=s.eps1, eps2=s.eps2, kappa=s.kappa, p=s.p, M=s.M, tau=s.tau)


def handle(s, prec, xyz=None):
    prm = api.hsma_default_params(p=s.p, M=s.M, tau=s.tau, precision=prec)
    h = api.hsma_create(s.a, s.eps1, s.eps2, s.kappa, prm)
    api.hsma_build_sources(h, s.xyz if xyz is None else xyz, s.q)
    return h


def changed_terms_scale(P, s, xyz, k, x_new):
    """Sum of the absolute values of the energy terms that moving charge k to x_new changes."""
    src = oracle.build_sources(P, xyz, s.q)
    absrc = dict(src, kel_q=np.abs(src["kel_q"]), surf_phi=np.abs(src["surf_phi"]),
                 surf_dphi=np.abs(src["surf_dphi"]), r0_const=abs(src["r0_const"]))
    pc, pr = oracle.evaluate(P, xyz, np.abs(s.q), absrc, np.array([x_new, xyz[k]]), self_index=np.array([k, k]))
    xyz1 = xyz.copy()
    xyz1[k] = x_new
    src1 = oracle.build_sources(P, xyz1, s.q)
    kc = P.coulomb_k / s.eps1
    others = np.delete(np.arange(s.n), k)

    def own_image(sr):
        d = np.linalg.norm(xyz[others] - sr["kel_xyz"][k], axis=1)
        return np.abs(kc * sr["kel_q"][k] / d)

    return abs(s.q[k]) * float(pc.sum() + pr.sum()) + float(np.sum(np.abs(s.q[others]) *
                                                                   (own_image(src1) + own_image(src))))


def delta_bound(P, s, xyz, k, x_new, prec, r0, r1):
    ref = r1["E_total"] - r0["E_total"]
    S = changed_terms_scale(P, s, xyz, k, x_new)
    return TOL[prec] * (abs(ref) + S) + 4e-16 * (abs(r0["E_total"]) + abs(r1["E_total"])), S


def check_delta(s, h, prec, k, x_new):
    P = P_of(s)
    r0 = oracle.hsma(P, s.xyz, s.q)
    xyz1 = s.xyz.copy()
    xyz1[k] = x_new
    r1 = oracle.hsma(P, xyz1, s.q)
    ref = r1["E_total"] - r0["E_total"]
    de = api.hsma_delta_energy(h, k, x_new)
    bound, _ = delta_bound(P, s, s.xyz, k, x_new, prec, r0, r1)
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
    """Accepted moves are committed in place (records rewritten at the sorted slot, boxes grown,
    coefficients, surface strengths and surface potentials updated).  The resident state must
    equal a fresh oracle evaluation at the same tolerance as a fresh build, and must not drift
    from a fresh build of the same positions: a trial move on the committed state and on a fresh
    handle gives the same Delta E up to the order of the FP64 sums.  The accepted Delta E add up
    to the change of the resident energy within the sum of their own bounds."""
    s = inputs.near_interface_system(kappa_a=0.5, n=300)
    h = handle(s, prec)
    P = P_of(s)
    rng = np.random.default_rng(11)
    xyz = s.xyz.copy()
    e0, _ = api.hsma_energy(h)
    ref0 = oracle.hsma(P, xyz, s.q)
    scale0 = max(abs(ref0["E_total"]), 0.5 * np.sum(np.abs(s.q * ref0["phi"])))
    total = 0.0
    bound_sum = 0.0   # sum over the accepted moves of their Delta E bounds (module docstring)
    for step in range(25):
        k = int(rng.integers(s.n))
        while True:
            x_new = xyz[k] + inputs.uniform_ball(rng, 1, 0.05 * s.a)[0]
            if np.linalg.norm(x_new) < s.a:
                break
        de = api.hsma_delta_energy(h, k, x_new)
        if rng.random() < 0.5:
            xyz1 = xyz.copy()
            xyz1[k] = x_new
            ref1 = oracle.hsma(P, xyz1, s.q)
            b, S = delta_bound(P, s, xyz, k, x_new, prec, ref0, ref1)
            d_ref = ref1["E_total"] - ref0["E_total"]
            assert abs(de - d_ref) <= b, (step, de, d_ref, b)
            # no drift: the committed state answers as a fresh build of the same positions
            de_fresh = api.hsma_delta_energy(handle(s, prec, xyz), k, x_new)
            assert abs(de - de_fresh) <= 1e-12 * (abs(de) + S), (step, de, de_fresh)
            bound_sum += b
            api.hsma_apply_move(h, k, x_new)
            xyz, ref0 = xyz1, ref1
            total += de
    ref = ref0
    e1, er1 = api.hsma_energy(h)
    phi = api.hsma_potential(h)
    scale = max(abs(ref["E_total"]), 0.5 * np.sum(np.abs(s.q * ref["phi"])))
    assert abs(e1 - ref["E_total"]) <= TOL[prec] * scale
    assert np.linalg.norm(phi - ref["phi"]) / np.linalg.norm(ref["phi"]) <= TOL[prec]
    # (e1 - e0) - sum dE: each energy is within TOL * its scale of the oracle and each accepted dE
    # within its own bound, so their difference is within the sum of those bounds
    assert abs((e1 - e0) - total) <= TOL[prec] * (scale + scale0) + bound_sum


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
