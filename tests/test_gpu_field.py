"""Fields E = -grad phi through the C ABI (hsma_field, hsma_batch_field) against the FP64 oracle.

Tolerance norm-wise over all components, ||E - E_ref||_2 / ||E_ref||_2: 1e-6 (FP32 path),
1e-12 (FP64 path), as for the potentials.
"""
import numpy as np
import pytest

import oracle
from paper_1907_01724_gb300 import api, batch, inputs

pytestmark = pytest.mark.gpu

TOL = {api.HSMA_FP32: 1e-6, api.HSMA_FP64: 1e-12}


def P_of(s):
    return oracle.make_params(a=s.a, eps1=s.eps1, eps2=s.eps2, kappa=s.kappa, p=s.p, M=s.M, tau=s.tau)


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a - b)


def handle(s, prec):
    prm = api.hsma_default_params(p=s.p, M=s.M, tau=s.tau, precision=prec)
    h = api.hsma_create(s.a, s.eps1, s.eps2, s.kappa, prm)
    api.hsma_build_sources(h, s.xyz, s.q)
    return h


def check_field(s, prec, tol=None):
    tol = tol if tol is not None else TOL[prec]
    ref = oracle.field(P_of(s), s.xyz, s.q)
    h = handle(s, prec)
    E = api.hsma_field(h, api.HSMA_TOTAL)
    Er = api.hsma_field(h, api.HSMA_REACTION)
    Ec = api.hsma_field(h, api.HSMA_COULOMB)
    api.hsma_destroy(h)
    assert rel(E, ref["E"]) <= tol, ("E", rel(E, ref["E"]))
    assert rel(Er, ref["E_rf"]) <= tol, ("E_rf", rel(Er, ref["E_rf"]))
    assert rel(Ec, ref["E_coul"]) <= tol, ("E_coul", rel(Ec, ref["E_coul"]))
    return E, ref


@pytest.mark.parametrize("prec", [api.HSMA_FP32, api.HSMA_FP64])
def test_field_small_uniform_system(prec):
    check_field(inputs.small_system(), prec)


@pytest.mark.parametrize("prec", [api.HSMA_FP32, api.HSMA_FP64])
@pytest.mark.parametrize("ka", [0.5, 2.0])
def test_field_near_interface_system(prec, ka):
    check_field(inputs.near_interface_system(kappa_a=ka), prec)


def test_field_near_interface_p30_fp32():
    check_field(inputs.near_interface_system(kappa_a=2.0, p=30), api.HSMA_FP32)


@pytest.mark.parametrize("prec", [api.HSMA_FP32, api.HSMA_FP64])
@pytest.mark.parametrize("n", [1, 2, 31, 33, 257, 1001])
def test_field_ragged_sizes(prec, n):
    rng = np.random.default_rng(1000 + n)
    s = inputs.System(xyz=inputs.uniform_ball(rng, n, 1.0), q=rng.choice([-1.0, 1.0], size=n), a=1.0, eps1=1.0,
                      eps2=80.0, kappa=1.0, p=12, M=400, tau=0.1)
    check_field(s, prec)


@pytest.mark.parametrize("prec", [api.HSMA_FP32, api.HSMA_FP64])
def test_field_primitive_full_size_sampled(prec):
    """N = 20000, M = 2000, p = 30 at full size; the oracle evaluates a sample of 400 targets."""
    s = inputs.primitive_system()
    P = P_of(s)
    h = handle(s, prec)
    E = api.hsma_field(h, api.HSMA_TOTAL)
    api.hsma_destroy(h)
    rng = np.random.default_rng(3)
    idx = np.sort(rng.choice(s.n, 400, replace=False))
    src = oracle.build_sources(P, s.xyz, s.q)
    ec, er = oracle.field_at(P, s.xyz, s.q, src, s.xyz[idx], self_index=idx)
    assert rel(E[idx], ec + er) <= TOL[prec]


@pytest.mark.parametrize("prec", [api.HSMA_FP32, api.HSMA_FP64])
def test_field_pass_refreshes_potentials_and_energies(prec):
    s = inputs.near_interface_system(kappa_a=2.0)
    ref = oracle.hsma(P_of(s), s.xyz, s.q)
    h = handle(s, prec)
    api.hsma_field(h)
    n0 = api.hsma_kernel_launches(h)
    phi = api.hsma_potential(h)
    et, er = api.hsma_energy(h)
    assert api.hsma_kernel_launches(h) == n0  # no second pair sum
    assert rel(phi, ref["phi"]) <= TOL[prec]
    scale = max(abs(ref["E_total"]), 0.5 * np.sum(np.abs(s.q * ref["phi"])))
    assert abs(et - ref["E_total"]) <= TOL[prec] * scale
    api.hsma_destroy(h)


@pytest.mark.parametrize("prec", [api.HSMA_FP32, api.HSMA_FP64])
def test_field_after_committed_moves(prec):
    s = inputs.near_interface_system(kappa_a=0.5)
    h = handle(s, prec)
    api.hsma_field(h)
    xyz = s.xyz.copy()
    rng = np.random.default_rng(8)
    for k in rng.choice(s.n, 5, replace=False):
        while True:
            x = xyz[k] + rng.uniform(-0.05, 0.05, 3) * s.a
            if np.linalg.norm(x) < 0.999 * s.a:
                break
        api.hsma_apply_move(h, int(k), x)
        xyz[k] = x
    E = api.hsma_field(h)
    api.hsma_destroy(h)
    ref = oracle.field(P_of(s), xyz, s.q)["E"]
    assert rel(E, ref) <= TOL[prec]


@pytest.mark.parametrize("prec", [api.HSMA_FP32, api.HSMA_FP64])
def test_batch_field_matches_oracle_per_system(prec):
    rng = np.random.default_rng(21)
    systems = []
    for i, n in enumerate((5, 640, 1500, 77)):
        systems.append(inputs.System(xyz=inputs.uniform_ball(rng, n, 1.0 + 0.1 * i), q=rng.choice([-1.0, 1.0], size=n),
                                     a=1.0 + 0.1 * i, eps1=1.0 if i % 2 else 78.5, eps2=78.5, kappa=0.5 + i,
                                     p=20, M=1000, tau=0.1))
    b = batch.from_systems(systems, precision=prec)
    n, xyz, q = batch.concat(systems)
    b.hsma_batch_build_sources(n, xyz, q)
    E = b.hsma_batch_field()
    again = b.hsma_batch_field()
    assert np.array_equal(E, again)
    off = 0
    for s in systems:
        ref = oracle.field(P_of(s), s.xyz, s.q)["E"]
        assert rel(E[off:off + s.n], ref) <= TOL[prec]
        off += s.n


def test_field_is_deterministic_and_device_output():
    torch = pytest.importorskip("torch")
    s = inputs.near_interface_system(kappa_a=2.0)
    h = handle(s, api.HSMA_FP32)
    E1 = api.hsma_field(h)
    api.hsma_build_sources(h, s.xyz, s.q)
    E2 = api.hsma_field(h)
    assert np.array_equal(E1, E2)
    out = torch.empty((s.n, 3), dtype=torch.float64, device="cuda")
    api.hsma_field(h, api.HSMA_TOTAL, out=out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), E1)
    api.hsma_destroy(h)


def test_field_forces_match_energy_gradient_within_the_method():
    """q_k E_k against -dE/dx_k from hsma_delta_energy central differences (~1e-4, see the oracle pin)."""
    s = inputs.small_system()
    h = handle(s, api.HSMA_FP64)
    E = api.hsma_field(h)
    rng = np.random.default_rng(0)
    hh = 1e-5
    for k in rng.choice(s.n, 3, replace=False):
        g = np.zeros(3)
        for d in range(3):
            xp = s.xyz[k].copy()
            xp[d] += hh
            xm = s.xyz[k].copy()
            xm[d] -= hh
            g[d] = -(api.hsma_delta_energy(h, int(k), xp) - api.hsma_delta_energy(h, int(k), xm)) / (2 * hh)
        F = s.q[k] * E[k]
        assert np.linalg.norm(F - g) <= 2e-3 * np.linalg.norm(g)
    api.hsma_destroy(h)


def test_field_errors():
    s = inputs.small_system()
    prm = api.hsma_default_params(p=s.p, M=s.M)
    h = api.hsma_create(s.a, s.eps1, s.eps2, s.kappa, prm)
    with pytest.raises(api.HsmaError):
        api.hsma_field(h)  # before build
    api.hsma_build_sources(h, s.xyz, s.q)
    with pytest.raises(api.HsmaError):
        api.hsma_field(h, what=7)
    api.hsma_destroy(h)


@pytest.mark.parametrize("prec", [api.HSMA_FP32, api.HSMA_FP64])
def test_batch_field_overlapped_build_matches_separate_passes(prec):
    """Build + field in one overlapped graph against the build and field graphs run one after the
    other: the same items and slots, so bitwise the same fields, potentials and energies."""
    rng = np.random.default_rng(22)
    systems = [inputs.System(xyz=inputs.uniform_ball(rng, n, 1.0), q=rng.choice([-1.0, 1.0], size=n), a=1.0,
                             eps1=1.0, eps2=78.5, kappa=1.0, p=20, M=1000, tau=0.1) for n in (1200, 333, 2048)]
    n, xyz, q = batch.concat(systems)
    out = {}
    for on in (True, False):
        b = batch.from_systems(systems, precision=prec)
        b.hsma_batch_set_overlap(on)
        b.hsma_batch_build_sources(n, xyz, q)
        E = b.hsma_batch_field()
        phi = b.hsma_batch_potential()
        out[on] = (E, phi, b.hsma_batch_energy())
    assert np.array_equal(out[True][0], out[False][0])
    assert np.array_equal(out[True][1], out[False][1])
    assert np.array_equal(np.asarray(out[True][2]), np.asarray(out[False][2]))
    off = 0
    for s in systems:
        ref = oracle.field(P_of(s), s.xyz, s.q)["E"]
        assert rel(out[True][0][off:off + s.n], ref) <= TOL[prec]
        off += s.n
