"""Far-field treecode (hsma_set_far_field) against the FP64 oracle's direct sums.

The treecode approximates the real-charge and Kelvin-image pair sums of eq. phirffinall (the
paper uses the FMM at this point, Sec. 4.2); the oracle is the plain direct sum.  The FP32
tolerance of the direct path (1e-6 norm-wise for potentials, energies relative to their term
scale) is held here too: at theta = 0.5 and order 12 the truncation of the multipole series
stays near 1e-7.  Full-size parity where the oracle is quick, sampled targets at N = 200000.
"""
import numpy as np
import pytest

import oracle
from paper_1907_01724_gb300 import api, inputs
from pointwise import record_pointwise

pytestmark = pytest.mark.gpu

TOL = 1e-6


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def params_of(s):
    return oracle.make_params(a=s.a, eps1=s.eps1, eps2=s.eps2, kappa=s.kappa, p=s.p, M=s.M, tau=s.tau)


def run_tree(s, theta=0.5, order=12, what=(api.HSMA_TOTAL, api.HSMA_REACTION)):
    prm = api.hsma_default_params(p=s.p, M=s.M, tau=s.tau, precision=api.HSMA_FP32)
    h = api.hsma_create(s.a, s.eps1, s.eps2, s.kappa, prm)
    api.hsma_set_far_field(h, theta, order)
    api.hsma_build_sources(h, s.xyz, s.q)
    out = [api.hsma_potential(h, w) for w in what]
    e = api.hsma_energy(h)
    return h, out, e


def check_full(s, theta=0.5, order=12):
    ref = oracle.hsma(params_of(s), s.xyz, s.q)
    h, (phi, phi_rf), (et, er) = run_tree(s, theta, order)
    api.hsma_destroy(h)
    e_phi, e_rf = rel(phi, ref["phi"]), rel(phi_rf, ref["phi_rf"])
    record_pointwise(f"{s.name} tree theta={theta} P={order}", api.HSMA_FP32, phi, ref["phi"], e_phi)
    scale_t = max(abs(ref["E_total"]), 0.5 * np.sum(np.abs(s.q * ref["phi"])))
    scale_r = max(abs(ref["E_rf"]), 0.5 * np.sum(np.abs(s.q * ref["phi_rf"])))
    assert e_phi <= TOL, ("phi", e_phi)
    assert e_rf <= TOL, ("phi_rf", e_rf)
    assert abs(et - ref["E_total"]) / scale_t <= TOL
    assert abs(er - ref["E_rf"]) / scale_r <= TOL


def uniform(n, seed, eps1=1.0, eps2=80.0, ka=1.0, M=1000, p=20):
    rng = np.random.default_rng(inputs.SEED_BASE + 70 + seed)
    n = inputs.even(n)
    return inputs.System(1.0, eps1, eps2, ka, p, M, inputs.uniform_ball(rng, n, 1.0), inputs.neutral_charges(rng, n),
                         name=f"N{n}_uniform_eps{eps1:g}_{eps2:g}_ka{ka:g}")


@pytest.mark.parametrize("order", [8, 12, 16])
def test_tree_uniform_30000(order):
    """N = 30000 uniform (three node levels): every target's potential and both energies."""
    check_full(uniform(30000, 0), theta=0.5 if order >= 12 else 0.35, order=order)


def test_tree_near_interface():
    """25 % of the charges within 0.05 a of the interface (their Kelvin images within 0.1 a of
    them): the near field of the Kelvin tree, at the smallest tree (N = 2000)."""
    check_full(inputs.near_interface_system(kappa_a=2.0))


def test_tree_primitive_workload():
    """N = 20000, eps1 = eps2 = 78.5, kappa a = 3, M = 2000, p = 30 with the tree."""
    check_full(inputs.primitive_system())


def test_tree_edge_charges():
    """A charge at the centre (its image at infinity: a constant), one at 0.999999 a next to its
    own image, and a clustered group, among uniform charges."""
    rng = np.random.default_rng(inputs.SEED_BASE + 77)
    n = 12000
    xyz = inputs.uniform_ball(rng, n, 1.0)
    xyz[0] = 0.0
    xyz[1] = np.array([0.999999, 0.0, 0.0])
    xyz[2:400] = np.array([0.3, -0.2, 0.1]) + 0.02 * inputs.uniform_ball(rng, 398, 1.0)
    s = inputs.System(1.0, 2.0, 80.0, 5.0, 20, 1000, xyz, inputs.neutral_charges(rng, n), name="N12000_edge")
    check_full(s)


def test_tree_clustered_60000():
    """Three dense clusters (radius 0.04a, 15000 charges each: leaf cells of hundreds of charges,
    sorted in the scratch buffer) among 15000 uniform charges: every potential and both energies."""
    rng = np.random.default_rng(inputs.SEED_BASE + 78)
    parts = [inputs.uniform_ball(rng, 15000, 1.0)]
    for c in ([0.5, 0.1, -0.2], [-0.3, -0.6, 0.2], [0.0, 0.2, 0.9]):
        parts.append(np.array(c) + 0.04 * inputs.uniform_ball(rng, 15000, 1.0))
    xyz = np.concatenate(parts)
    xyz = xyz[rng.permutation(len(xyz))]
    s = inputs.System(1.0, 1.0, 80.0, 2.0, 20, 1000, xyz, inputs.neutral_charges(rng, len(xyz)),
                      name="N60000_clusters")
    check_full(s)


def test_tree_sampled_200000():
    """N = 200000 uniform (four node levels, far images): potentials at 2000 sampled charges
    against the oracle's direct sums at those charges."""
    s = uniform(200000, 1, eps1=2.0, eps2=80.0, ka=5.0)
    P = params_of(s)
    src = oracle.build_sources(P, s.xyz, s.q)
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(s.n, 2000, replace=False))
    pc, pr = oracle.evaluate(P, s.xyz, s.q, src, s.xyz[idx], self_index=idx)
    h, (phi, phi_rf), _ = run_tree(s)
    api.hsma_destroy(h)
    e_phi, e_rf = rel(phi[idx], pc + pr), rel(phi_rf[idx], pr)
    record_pointwise("N200000 tree sampled", api.HSMA_FP32, phi[idx], pc + pr, e_phi)
    assert e_phi <= TOL, ("phi", e_phi)
    assert e_rf <= TOL, ("phi_rf", e_rf)


@pytest.mark.parametrize("n", [1, 3, 33, 1001])
def test_tree_tiny_and_ragged(n):
    """A handful of charges (one partial group of 32, empty cells everywhere) and ragged tails."""
    rng = np.random.default_rng(inputs.SEED_BASE + 79 + n)
    q = inputs.neutral_charges(rng, n) if n > 1 else np.array([1.0])
    s = inputs.System(1.0, 1.0, 80.0, 1.0, 20, 400, inputs.uniform_ball(rng, n, 1.0), q, name=f"N{n}_tiny")
    check_full(s)


def test_tree_deterministic_and_switch_back():
    """Two tree builds give bitwise equal results; theta = 0 restores the direct path bitwise."""
    s = uniform(20000, 2)
    h, (a1, _), e1 = run_tree(s)
    api.hsma_build_sources(h, s.xyz, s.q)
    a2 = api.hsma_potential(h, api.HSMA_TOTAL)
    assert np.array_equal(a1, a2)
    assert api.hsma_last_far_time(h) > 0.0
    api.hsma_set_far_field(h, 0.0)
    api.hsma_build_sources(h, s.xyz, s.q)
    d1 = api.hsma_potential(h, api.HSMA_TOTAL)
    api.hsma_destroy(h)
    prm = api.hsma_default_params(p=s.p, M=s.M, tau=s.tau, precision=api.HSMA_FP32)
    h2 = api.hsma_create(s.a, s.eps1, s.eps2, s.kappa, prm)
    api.hsma_build_sources(h2, s.xyz, s.q)
    d2 = api.hsma_potential(h2, api.HSMA_TOTAL)
    api.hsma_destroy(h2)
    assert np.array_equal(d1, d2)
    assert rel(a1, d2) <= TOL


def test_tree_rejects():
    s = uniform(4000, 3)
    prm = api.hsma_default_params(p=s.p, M=s.M, tau=s.tau, precision=api.HSMA_FP32)
    h = api.hsma_create(s.a, s.eps1, s.eps2, s.kappa, prm)
    for theta, order in [(1.0, 12), (-0.1, 12), (0.5, 10)]:
        with pytest.raises(api.HsmaError) as ei:
            api.hsma_set_far_field(h, theta, order)
        assert ei.value.code == -1
    api.hsma_set_far_field(h, 0.5, 12)
    api.hsma_build_sources(h, s.xyz, s.q)
    api.hsma_potential(h, api.HSMA_TOTAL)
    with pytest.raises(api.HsmaError) as ei:
        api.hsma_field(h, api.HSMA_TOTAL)
    assert ei.value.code == -3
    with pytest.raises(api.HsmaError) as ei:
        api.hsma_delta_energy(h, 0, np.array([0.1, 0.0, 0.0]))
    assert ei.value.code == -3
    api.hsma_destroy(h)
    prm64 = api.hsma_default_params(p=s.p, M=s.M, tau=s.tau, precision=api.HSMA_FP64)
    h64 = api.hsma_create(s.a, s.eps1, s.eps2, s.kappa, prm64)
    with pytest.raises(api.HsmaError) as ei:
        api.hsma_set_far_field(h64, 0.5, 12)
    assert ei.value.code == -1
    api.hsma_destroy(h64)
